// Batched 1-D FFT passes in shared memory (mixed radix 8/4/2/3/5, Stockham
// autosort), the building block of every convolution of the hot path:
// the blur Phi (Eq. 3), its transpose (Eq. 5) and the certificate
// correlation against the kernel-family table (Section 2: "convolutions are
// made in Fourier domain").
//
// A CTA owns a tile of W lines.  Shared memory holds the tile point-major,
// row j of the tile at [j * (W + 1)], so that the W lines of a row are
// contiguous (coalesced loads of strided axes) and rows are padded by one
// element against bank conflicts.  Radix-R stages read R points L/R apart and
// write them Ns apart (Stockham), so no bit reversal is needed and the result
// is in natural order after the last stage.
#include <math.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <utility>

#include "sfw_internal.cuh"

namespace sfw {

// ------------------------------------------------------------------ host helpers

bool factorize(int L, Factors* f) {
    f->n = 0;
    if (L < 1 || L > kMaxLen) return false;
    const int radices[5] = {8, 4, 2, 3, 5};
    for (int q = 0; q < 5; ++q) {
        int r = radices[q];
        while (L % r == 0 && L > 1) {
            if (f->n >= kMaxFactors) return false;
            f->r[f->n++] = r;
            L /= r;
        }
    }
    return L == 1;
}

int next_smooth_even(int x) {
    if (x < 2) x = 2;
    for (int v = x + (x & 1);; v += 2) {
        int t = v;
        while (t % 2 == 0) t /= 2;
        while (t % 3 == 0) t /= 3;
        while (t % 5 == 0) t /= 5;
        if (t == 1) return v;
    }
}

sfw_status TwiddleCache::get(int L, const float2** out) {
    auto it = tables.find(L);
    if (it != tables.end()) {
        *out = it->second;
        return SFW_OK;
    }
    std::vector<float2> h(L);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < L; ++j) {
        double a = -two_pi * (double)j / (double)L;
        h[j] = make_float2((float)cos(a), (float)sin(a));
    }
    float2* d = nullptr;
    if (cudaMalloc(&d, sizeof(float2) * L) != cudaSuccess) return fail(SFW_ERR_ALLOC, "twiddle table");
    cudaError_t e = cudaMemcpy(d, h.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "twiddle upload");
    }
    tables[L] = d;
    *out = d;
    return SFW_OK;
}

void TwiddleCache::release() {
    for (auto& kv : tables) cudaFree(kv.second);
    tables.clear();
}

// ------------------------------------------------------------------ device arithmetic

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (DIR * i)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs: X[q] = sum_r v[r] exp(DIR 2 pi i r q / R).
template <int DIR>
__device__ __forceinline__ void dft2(float2* v) {
    float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <int DIR>
__device__ __forceinline__ void dft4v(float2& v0, float2& v1, float2& v2, float2& v3) {
    float2 t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = mul_i<DIR>(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* v) { dft4v<DIR>(v[0], v[1], v[2], v[3]); }

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4v<DIR>(e0, e1, e2, e3);
    dft4v<DIR>(o0, o1, o2, o3);
    const float c = 0.70710678118654752440f;
    // w = exp(DIR 2 pi i / 8): w^1 = c (1, DIR), w^2 = DIR i, w^3 = c (-1, DIR)
    float2 p1 = make_float2(c * (o1.x - DIR * o1.y), c * (o1.y + DIR * o1.x));
    float2 p2 = mul_i<DIR>(o2);
    float2 p3 = make_float2(c * (-o3.x - DIR * o3.y), c * (DIR * o3.x - o3.y));
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, p1);
    v[5] = csub(e1, p1);
    v[2] = cadd(e2, p2);
    v[6] = csub(e2, p2);
    v[3] = cadd(e3, p3);
    v[7] = csub(e3, p3);
}

template <int DIR>
__device__ __forceinline__ void dft3(float2* v) {
    const float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 t = cadd(v[1], v[2]);
    float2 u = csub(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 s = mul_i<DIR>(cscale(u, s3));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, s);
    v[2] = csub(m, s);
}

template <int DIR>
__device__ __forceinline__ void dft5(float2* v) {
    const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    float2 b1 = mul_i<DIR>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    float2 b2 = mul_i<DIR>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) dft2<DIR>(v);
    else if constexpr (R == 3) dft3<DIR>(v);
    else if constexpr (R == 4) dft4<DIR>(v);
    else if constexpr (R == 5) dft5<DIR>(v);
    else dft8<DIR>(v);
}

// One Stockham radix-R stage over the W lines of the tile.
template <int R, int DIR, int W>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                          int L, int Ns, const float2* __restrict__ tw) {
    constexpr int WS = W + 1;
    const int LR = L / R;
    const int tstep = L / (Ns * R);
    const int total = LR * W;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int i = t % W;
        const int jj = t / W;
        const int k = jj % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(jj + r * LR) * WS + i];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[k * r * tstep];
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<R, DIR>(v);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * WS + i] = v[r];
    }
}

// Full transform of the tile held in `a`; returns the buffer holding the result.
template <int DIR, int W>
__device__ float2* fft_tile(float2* a, float2* b, int L, const Factors& fac, const float2* tw) {
    int Ns = 1;
    for (int s = 0; s < fac.n; ++s) {
        const int R = fac.r[s];
        switch (R) {
            case 8: fft_stage<8, DIR, W>(a, b, L, Ns, tw); break;
            case 4: fft_stage<4, DIR, W>(a, b, L, Ns, tw); break;
            case 2: fft_stage<2, DIR, W>(a, b, L, Ns, tw); break;
            case 3: fft_stage<3, DIR, W>(a, b, L, Ns, tw); break;
            default: fft_stage<5, DIR, W>(a, b, L, Ns, tw); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* tw, int L) {
    for (int j = threadIdx.x; j < L; j += blockDim.x) s_tw[j] = tw[j];
}

// ------------------------------------------------------------------ kernels

constexpr int kThreads = 256;

template <int W, int DIR>
__global__ void __launch_bounds__(kThreads) k_c2c(C2CPass p) {
    constexpr int WS = W + 1;
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + p.L;
    float2* B = A + p.L * WS;
    __shared__ long long off_in[W], off_out[W];
    const long long l0 = (long long)blockIdx.x * W;
    if (threadIdx.x < W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, p.L);
    __syncthreads();
    for (int e = threadIdx.x; e < p.L * W; e += blockDim.x) {
        const int i = e % W, j = e / W;
        const int jj = j - p.in_off;
        float2 v = make_float2(0.f, 0.f);
        if (l0 + i < p.nlines && jj >= 0 && jj < p.in_len) v = p.in[off_in[i] + jj * p.lin.Sj];
        A[j * WS + i] = v;
    }
    __syncthreads();
    float2* res = fft_tile<DIR, W>(A, B, p.L, p.fac, s_tw);
    for (int e = threadIdx.x; e < p.out_len * W; e += blockDim.x) {
        const int i = e % W, j = e / W;
        if (l0 + i < p.nlines)
            p.out[off_out[i] + j * p.lout.Sj] = cscale(res[(j + p.out_off) * WS + i], p.scale);
    }
}

template <int KIND>
__device__ __forceinline__ float2 load_spec(const void* base, long long idx) {
    if constexpr (KIND == SPEC_C64) {
        return reinterpret_cast<const float2*>(base)[idx];
    } else if constexpr (KIND == SPEC_R32) {
        return make_float2(reinterpret_cast<const float*>(base)[idx], 0.f);
    } else if constexpr (KIND == SPEC_CBF16) {
        __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162*>(base)[idx];
        return __bfloat1622float2(h);
    } else {
        return make_float2(__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[idx]), 0.f);
    }
}

template <int W, int KIND>
__global__ void __launch_bounds__(kThreads) k_mul(MulPass p) {
    constexpr int WS = W + 1;
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + p.L;
    float2* B = A + p.L * WS;
    float2* C = B + p.L * WS;
    __shared__ long long off_in[W], off_out[W], off_spec[W];
    const long long l0 = (long long)blockIdx.x * W;
    if (threadIdx.x < W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
            off_spec[threadIdx.x] = line_offset(p.lspec, l);
        }
    }
    load_twiddles(s_tw, p.tw, p.L);
    __syncthreads();
    for (int e = threadIdx.x; e < p.L * W; e += blockDim.x) {
        const int i = e % W, j = e / W;
        const int jj = j - p.in_off;
        float2 v = make_float2(0.f, 0.f);
        if (l0 + i < p.nlines && jj >= 0 && jj < p.in_len) v = p.in[off_in[i] + jj * p.lin.Sj];
        A[j * WS + i] = v;
    }
    __syncthreads();
    float2* X = fft_tile<-1, W>(A, B, p.L, p.fac, s_tw);
    float2* S0 = (X == A) ? B : A;
    for (int s = 0; s < p.nspec; ++s) {
        const long long sbase = (long long)s * p.spec_stride;
        for (int e = threadIdx.x; e < p.L * W; e += blockDim.x) {
            const int i = e % W, j = e / W;
            float2 h = make_float2(0.f, 0.f);
            if (l0 + i < p.nlines) h = load_spec<KIND>(p.spec, sbase + off_spec[i] + j * p.lspec.Sj);
            if (p.conj_spec) h.y = -h.y;
            S0[j * WS + i] = cmul(X[j * WS + i], h);
        }
        __syncthreads();
        float2* res = fft_tile<1, W>(S0, C, p.L, p.fac, s_tw);
        float2* outp = p.out + (long long)s * p.out_stride;
        for (int e = threadIdx.x; e < p.out_len * W; e += blockDim.x) {
            const int i = e % W, j = e / W;
            if (l0 + i < p.nlines) outp[off_out[i] + j * p.lout.Sj] = res[(j + p.out_off) * WS + i];
        }
        __syncthreads();
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_r2c(R2CPass p) {
    constexpr int WS = W + 1;
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + p.L;
    float2* B = A + p.L * WS;
    __shared__ long long off_in[2 * W], off_out[2 * W];
    const long long l0 = (long long)blockIdx.x * (2 * W);
    if (threadIdx.x < 2 * W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, p.L);
    __syncthreads();
    float* Af = reinterpret_cast<float*>(A);
    for (int e = threadIdx.x; e < 2 * W * p.L; e += blockDim.x) {
        const int q = e / p.L, j = e - (e / p.L) * p.L;
        const int jj = j - p.in_off;
        float v = 0.f;
        if (l0 + q < p.nlines && jj >= 0 && jj < p.in_len) v = p.in[off_in[q] + jj];
        Af[(j * WS + (q >> 1)) * 2 + (q & 1)] = v;
    }
    __syncthreads();
    float2* Z = fft_tile<-1, W>(A, B, p.L, p.fac, s_tw);
    const int H = p.L / 2 + 1;
    for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
        const int i = e / H, k = e - (e / H) * H;
        const float2 z = Z[k * WS + i];
        const float2 zm = Z[((p.L - k) % p.L) * WS + i];
        // a = FFT of line 2i, b = FFT of line 2i+1 (two real lines in one complex FFT)
        const float2 a = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        const float2 b = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
        if (l0 + 2 * i < p.nlines) p.out[off_out[2 * i] + k] = a;
        if (l0 + 2 * i + 1 < p.nlines) p.out[off_out[2 * i + 1] + k] = b;
    }
}

constexpr int kC2RMaxSlots = 16;  // output values per thread in the certificate epilogue

template <int W, int MODE>
__global__ void __launch_bounds__(kThreads) k_c2r(C2RPass p) {
    constexpr int WS = W + 1;
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + p.L;
    float2* B = A + p.L * WS;
    __shared__ long long off_in[2 * W], off_out[2 * W];
    __shared__ double s_red[kThreads / 32];
    const long long l0 = (long long)blockIdx.x * (2 * W);
    if (threadIdx.x < 2 * W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, p.L);
    const int H = p.L / 2 + 1;
    const int nout = 2 * W * p.out_len;

    float mx[kC2RMaxSlots];
    int ak[kC2RMaxSlots];
    bool saw_nan = false;
    double acc = 0.0;
    if constexpr (MODE == C2R_CERTMAX) {
#pragma unroll
        for (int it = 0; it < kC2RMaxSlots; ++it) {
            mx[it] = -INFINITY;
            ak[it] = 0;
        }
    }
    const int nspec = (MODE == C2R_CERTMAX) ? p.nspec : 1;
    for (int s = 0; s < nspec; ++s) {
        __syncthreads();
        const float2* in = p.in + (long long)s * p.in_spec_stride;
        for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
            const int i = e / H, k = e - (e / H) * H;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (l0 + 2 * i < p.nlines) a = in[off_in[2 * i] + k];
            if (l0 + 2 * i + 1 < p.nlines) b = in[off_in[2 * i + 1] + k];
            // Z = A + i B on [0, L/2], Hermitian extension on (L/2, L)
            A[k * WS + i] = make_float2(a.x - b.y, a.y + b.x);
            if (k > 0 && k < p.L - k) A[(p.L - k) * WS + i] = make_float2(a.x + b.y, b.x - a.y);
        }
        __syncthreads();
        float2* z = fft_tile<1, W>(A, B, p.L, p.fac, s_tw);
        if constexpr (MODE != C2R_CERTMAX) {
            for (int e = threadIdx.x; e < nout; e += blockDim.x) {
                const int q = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                if (l0 + q >= p.nlines) continue;
                const float2 zz = z[(j + p.out_off) * WS + (q >> 1)];
                const float v = ((q & 1) ? zz.y : zz.x) * p.scale;
                const long long o = off_out[q] + j;
                if constexpr (MODE == C2R_STORE) {
                    p.out[o] = v;
                } else {
                    const float r = p.y[o] - v;
                    if (p.out) p.out[o] = r;
                    acc += (double)r * (double)r;
                }
            }
        } else {
#pragma unroll
            for (int it = 0; it < kC2RMaxSlots; ++it) {
                const int e = threadIdx.x + it * kThreads;
                if (e < nout) {
                    const int q = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                    if (l0 + q < p.nlines) {
                        const float2 zz = z[(j + p.out_off) * WS + (q >> 1)];
                        const float v = ((q & 1) ? zz.y : zz.x) * p.scale;
                        const long long o = off_out[q] + j;
                        if (p.eta_out) p.eta_out[(long long)s * p.V + o] = v;
                        if (v != v) saw_nan = true;
                        if (v > mx[it]) {
                            mx[it] = v;
                            ak[it] = s;
                        }
                    }
                }
            }
        }
    }
    if constexpr (MODE == C2R_RESIDUAL) {
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
            p.partials[blockIdx.x] = t;
        }
    }
    if constexpr (MODE == C2R_CERTMAX) {
        unsigned long long best = 0ull;
#pragma unroll
        for (int it = 0; it < kC2RMaxSlots; ++it) {
            const int e = threadIdx.x + it * kThreads;
            if (e < nout) {
                const int q = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                if (l0 + q < p.nlines) {
                    const long long o = off_out[q] + j;
                    if (p.max_out) p.max_out[o] = mx[it];
                    if (p.argk_out) p.argk_out[o] = ak[it];
                    unsigned long long key =
                        candidate_key(mx[it], (unsigned long long)ak[it] * p.V + o);
                    if (key > best) best = key;
                }
            }
        }
        if (saw_nan) best = ~0ull;
        if (p.best_key) {
            for (int off = 16; off > 0; off >>= 1) {
                unsigned long long o2 = __shfl_down_sync(0xffffffffu, best, off);
                if (o2 > best) best = o2;
            }
            if ((threadIdx.x & 31) == 0 && best) atomicMax(p.best_key, best);
        }
    }
}

// ------------------------------------------------------------------ launchers

static int tile_width(int L) { return L <= 256 ? 16 : 8; }

// Raise a kernel's dynamic shared-memory limit once per (device, kernel, size):
// the attribute call is kept out of stream captures after the first use.
template <typename KernelT>
static sfw_status prepare(KernelT kernel, size_t smem) {
    if (smem <= 48 * 1024) return SFW_OK;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    SFW_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, reinterpret_cast<const void*>(kernel));
    auto it = done.find(key);
    if (it != done.end() && it->second >= smem) return SFW_OK;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(smem)");
    done[key] = smem;
    return SFW_OK;
}

static size_t smem_bytes(int L, int W, int nbuf) {
    return sizeof(float2) * ((size_t)L + (size_t)nbuf * L * (W + 1));
}

sfw_status launch_c2c(const C2CPass& p, cudaStream_t st) {
    if (p.nlines <= 0) return SFW_OK;
    const int W = tile_width(p.L);
    const size_t smem = smem_bytes(p.L, W, 2);
    const unsigned blocks = (unsigned)((p.nlines + W - 1) / W);
#define SFW_C2C(WW, DD)                                              \
    do {                                                             \
        SFW_TRY(prepare(k_c2c<WW, DD>, smem));                       \
        SFW_LAUNCH(st, "k_c2c", k_c2c<WW, DD><<<blocks, kThreads, smem, st>>>(p)); \
    } while (0)
    if (W == 16) {
        if (p.dir < 0) SFW_C2C(16, -1); else SFW_C2C(16, 1);
    } else {
        if (p.dir < 0) SFW_C2C(8, -1); else SFW_C2C(8, 1);
    }
#undef SFW_C2C
    return launch_check("k_c2c");
}

sfw_status launch_mul(const MulPass& p, cudaStream_t st) {
    if (p.nlines <= 0) return SFW_OK;
    const int W = tile_width(p.L);
    const size_t smem = smem_bytes(p.L, W, 3);
    const unsigned blocks = (unsigned)((p.nlines + W - 1) / W);
#define SFW_MUL(WW, KK)                                              \
    do {                                                             \
        SFW_TRY(prepare(k_mul<WW, KK>, smem));                       \
        SFW_LAUNCH(st, "k_mul", k_mul<WW, KK><<<blocks, kThreads, smem, st>>>(p)); \
    } while (0)
    switch (p.spec_kind) {
        case SPEC_C64: if (W == 16) SFW_MUL(16, SPEC_C64); else SFW_MUL(8, SPEC_C64); break;
        case SPEC_R32: if (W == 16) SFW_MUL(16, SPEC_R32); else SFW_MUL(8, SPEC_R32); break;
        case SPEC_CBF16: if (W == 16) SFW_MUL(16, SPEC_CBF16); else SFW_MUL(8, SPEC_CBF16); break;
        default: if (W == 16) SFW_MUL(16, SPEC_RBF16); else SFW_MUL(8, SPEC_RBF16); break;
    }
#undef SFW_MUL
    return launch_check("k_mul");
}

sfw_status launch_r2c(const R2CPass& p, cudaStream_t st) {
    if (p.nlines <= 0) return SFW_OK;
    const int W = tile_width(p.L);
    const size_t smem = smem_bytes(p.L, W, 2);
    const unsigned blocks = (unsigned)((p.nlines + 2 * W - 1) / (2 * W));
    if (W == 16) {
        SFW_TRY(prepare(k_r2c<16>, smem));
        SFW_LAUNCH(st, "k_r2c", k_r2c<16><<<blocks, kThreads, smem, st>>>(p));
    } else {
        SFW_TRY(prepare(k_r2c<8>, smem));
        SFW_LAUNCH(st, "k_r2c", k_r2c<8><<<blocks, kThreads, smem, st>>>(p));
    }
    return launch_check("k_r2c");
}

// The certificate epilogue keeps 2W * out_len running maxima in registers.
static int c2r_width(const C2RPass& p) {
    int W = tile_width(p.L);
    if (p.mode == C2R_CERTMAX && 2 * W * p.out_len > kC2RMaxSlots * kThreads) W = 8;
    return W;
}

int c2r_blocks(const C2RPass& p) {
    const int W = c2r_width(p);
    return (int)((p.nlines + 2 * W - 1) / (2 * W));
}

sfw_status launch_c2r(const C2RPass& p, cudaStream_t st, int* blocks_out) {
    const int W = c2r_width(p);
    const int blocks = c2r_blocks(p);
    if (blocks_out) *blocks_out = blocks;
    if (p.nlines <= 0) return SFW_OK;
    if (p.mode == C2R_CERTMAX && 2 * W * p.out_len > kC2RMaxSlots * kThreads)
        return fail(SFW_ERR_SHAPE, "c2r: %d outputs per line exceed the epilogue tile", p.out_len);
    const size_t smem = smem_bytes(p.L, W, 2);
#define SFW_C2R(WW, MM)                                              \
    do {                                                             \
        SFW_TRY(prepare(k_c2r<WW, MM>, smem));                       \
        SFW_LAUNCH(st, "k_c2r", k_c2r<WW, MM><<<blocks, kThreads, smem, st>>>(p)); \
    } while (0)
    switch (p.mode) {
        case C2R_STORE: if (W == 16) SFW_C2R(16, C2R_STORE); else SFW_C2R(8, C2R_STORE); break;
        case C2R_RESIDUAL: if (W == 16) SFW_C2R(16, C2R_RESIDUAL); else SFW_C2R(8, C2R_RESIDUAL); break;
        default: if (W == 16) SFW_C2R(16, C2R_CERTMAX); else SFW_C2R(8, C2R_CERTMAX); break;
    }
#undef SFW_C2R
    return launch_check("k_c2r");
}

}  // namespace sfw
