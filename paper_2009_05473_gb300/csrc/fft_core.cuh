// Templated FFT pass kernels (see fft_kernels.cu for the design notes).  LL is a
// compile-time line length (0 = runtime length from the pass descriptor); the
// run_* launchers are explicitly instantiated per length in fft_len_*.cu.
#pragma once

#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "sfw_internal.cuh"

namespace sfw {

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

// a * (c + DIR i s)
template <int DIR>
__device__ __forceinline__ float2 cmulc(float2 a, float c, float s) {
    return make_float2(a.x * c - DIR * a.y * s, a.y * c + DIR * a.x * s);
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2.
template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        float2 x0 = v[n2], x1 = v[4 + n2], x2 = v[8 + n2], x3 = v[12 + n2];
        dft4v<DIR>(x0, x1, x2, x3);
        a[n2][0] = x0;
        a[n2][1] = x1;
        a[n2][2] = x2;
        a[n2][3] = x3;
    }
    const float c1 = 0.92387953251128675613f;  // cos(pi / 8)
    const float s1 = 0.38268343236508977173f;  // sin(pi / 8)
    const float h = 0.70710678118654752440f;
    a[1][1] = cmulc<DIR>(a[1][1], c1, s1);    // W16^1
    a[1][2] = cmulc<DIR>(a[1][2], h, h);      // W16^2
    a[1][3] = cmulc<DIR>(a[1][3], s1, c1);    // W16^3
    a[2][1] = cmulc<DIR>(a[2][1], h, h);      // W16^2
    a[2][2] = mul_i<DIR>(a[2][2]);            // W16^4
    a[2][3] = cmulc<DIR>(a[2][3], -h, h);     // W16^6
    a[3][1] = cmulc<DIR>(a[3][1], s1, c1);    // W16^3
    a[3][2] = cmulc<DIR>(a[3][2], -h, h);     // W16^6
    a[3][3] = cmulc<DIR>(a[3][3], -c1, -s1);  // W16^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 y0 = a[0][k1], y1 = a[1][k1], y2 = a[2][k1], y3 = a[3][k1];
        dft4v<DIR>(y0, y1, y2, y3);
        v[k1] = y0;
        v[k1 + 4] = y1;
        v[k1 + 8] = y2;
        v[k1 + 12] = y3;
    }
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) dft2<DIR>(v);
    else if constexpr (R == 3) dft3<DIR>(v);
    else if constexpr (R == 4) dft4<DIR>(v);
    else if constexpr (R == 5) dft5<DIR>(v);
    else if constexpr (R == 8) dft8<DIR>(v);
    else dft16<DIR>(v);
}

// ------------------------------------------------------------------ tile layout

// Point j of a line sits at phy(j) = j + j / 16: one padding slot every 16 points
// makes the strided writes of early Stockham stages (stride R up to 16)
// bank-conflict free.  Lines are pitch(L) apart (odd, so rows of a tile are too).
__host__ __device__ __forceinline__ constexpr int phy(int j) { return j + (j >> 4); }
__host__ __device__ __forceinline__ constexpr int pitch(int L) { return (L + (L >> 4) + 1) | 1; }

// Compile-time factorisation (radices 16, 8, 4, 2, 3, 5) of a specialised length:
// r[s] is the radix of stage s and ns[s] the product of the earlier radices.
struct CFac {
    int n;
    int r[kMaxFactors];
    int ns[kMaxFactors];
};

__host__ __device__ constexpr int max_radix_c(int L, int nl) {
    int r = 16;
    while (r > 2 && (L / r) * nl < 32) r >>= 1;
    return r;
}

// Same order as the host's factorize(L, maxr) (the twiddle layout depends on it).
__host__ __device__ constexpr CFac cfactor(int L, int maxr) {
    CFac f{};
    const int rad[6] = {16, 8, 4, 2, 3, 5};
    int ns = 1;
    for (int q = 0; q < 6; ++q) {
        if (rad[q] <= 16 && (rad[q] & (rad[q] - 1)) == 0 && rad[q] > maxr) continue;
        while (L % rad[q] == 0 && L > 1) {
            f.r[f.n] = rad[q];
            f.ns[f.n] = ns;
            ns *= rad[q];
            L /= rad[q];
            ++f.n;
        }
    }
    return f;
}

// ------------------------------------------------------------------ warp-level stages

// Radix-R Stockham stage over lines [li0, li0 + nl) of a line-major tile (pitch LS).
template <int R, int DIR, bool FIRST, class Load>
__device__ __forceinline__ void wstage(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int L, int LS, int li0, int nl, int Ns,
                                       const float2* __restrict__ tw, const Load& load) {
    const int LR = L / R;
    const int total = LR * nl;
    for (int t = (int)(threadIdx.x & 31); t < total; t += 32) {
        const int lq = t / LR;
        const int jj = t - lq * LR;
        const int li = li0 + lq;
        const int k = jj % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (FIRST) v[r] = load(li, jj + r * LR);
            else v[r] = src[li * LS + phy(jj + r * LR)];
        }
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[(Ns - 1) + (r - 1) * Ns + k];
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft<R, DIR>(v);
        const int base = (jj - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[li * LS + phy(base + r * Ns)] = v[r];
    }
    __syncwarp();
}

template <int DIR, bool FIRST, class Load>
__device__ __forceinline__ void wstage_any(int R, const float2* src, float2* dst, int L, int LS,
                                           int li0, int nl, int Ns, const float2* tw, const Load& load) {
    switch (R) {
        case 16: wstage<16, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
        case 8: wstage<8, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
        case 4: wstage<4, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
        case 2: wstage<2, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
        case 3: wstage<3, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
        default: wstage<5, DIR, FIRST>(src, dst, L, LS, li0, nl, Ns, tw, load); break;
    }
}

// Transform of this warp's lines.  Stage 0 reads through `load` and writes b;
// later stages alternate a <- b <- a ...  Returns the buffer with the result.
template <int DIR, class Load>
__device__ float2* warp_fft(float2* a, float2* b, int L, int LS, int li0, int nl,
                            const Factors& fac, const float2* tw, const Load& load) {
    int Ns = 1;
    wstage_any<DIR, true>(fac.r[0], nullptr, b, L, LS, li0, nl, Ns, tw, load);
    Ns *= fac.r[0];
    float2* src = b;
    float2* dst = a;
    for (int s = 1; s < fac.n; ++s) {
        wstage_any<DIR, false>(fac.r[s], src, dst, L, LS, li0, nl, Ns, tw, load);
        Ns *= fac.r[s];
        float2* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Compile-time version of wstage for a specialised length L (all index
// arithmetic folds to constants, the item loop unrolls).
template <int R, int DIR, bool FIRST, int L, int NS, int NL, class Load>
__device__ __forceinline__ void cstage(const float2* __restrict__ src, float2* __restrict__ dst,
                                       int li0, const float2* __restrict__ tw, const Load& load) {
    constexpr int LR = L / R;
    constexpr int TOTAL = LR * NL;
    constexpr int LS = pitch(L);
    const int lane = (int)(threadIdx.x & 31);
#pragma unroll
    for (int t0 = 0; t0 < TOTAL; t0 += 32) {
        const int t = t0 + lane;
        if ((TOTAL % 32) == 0 || t < TOTAL) {
            const int lq = t / LR;
            const int jj = t - lq * LR;
            const int li = li0 + lq;
            const int k = (NS == 1) ? 0 : jj % NS;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (FIRST) v[r] = load(li, jj + r * LR);
                else v[r] = src[li * LS + phy(jj + r * LR)];
            }
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw[(NS - 1) + (r - 1) * NS + k];
                    if (DIR > 0) w.y = -w.y;
                    v[r] = cmul(v[r], w);
                }
            }
            dft<R, DIR>(v);
            const int base = (jj - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[li * LS + phy(base + r * NS)] = v[r];
        }
    }
    __syncwarp();
}

template <int DIR, int L, int NL, int S, class Load>
__device__ __forceinline__ float2* cstages(float2* src, float2* dst, int li0, const float2* tw,
                                           const Load& load) {
    constexpr CFac F = cfactor(L, max_radix_c(L, NL));
    if constexpr (S >= F.n) {
        return src;
    } else {
        cstage<F.r[S], DIR, S == 0, L, F.ns[S], NL>(src, dst, li0, tw, load);
        return cstages<DIR, L, NL, S + 1>(dst, src, li0, tw, load);
    }
}

// Transform of this warp's lines, compile-time length LL (> 0) or runtime
// (LL == 0, factors from fac).  Stage 0 reads through `load` and writes b.
template <int DIR, int LL, int NL, class Load>
__device__ __forceinline__ float2* line_fft(float2* a, float2* b, int L, int LS, int li0,
                                            const Factors& fac, const float2* tw, const Load& load) {
    if constexpr (LL > 0) return cstages<DIR, LL, NL, 0>(a, b, li0, tw, load);
    else return warp_fft<DIR>(a, b, L, LS, li0, NL, fac, tw, load);
}

struct SmemLoad {
    const float2* a;
    int LS;
    __device__ __forceinline__ float2 operator()(int li, int j) const { return a[li * LS + phy(j)]; }
};

constexpr int kThreads = 256;

__device__ __forceinline__ void load_twiddles(float2* s_tw, const float2* tw, int L) {
    for (int j = threadIdx.x; j < L; j += kThreads) s_tw[j] = tw[j];
}

// ------------------------------------------------------------------ cp.async helpers

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// ------------------------------------------------------------------ last-tile reductions

// Fixed-order block sum of one double per thread (result in thread 0).
__device__ __forceinline__ double block_sum_d(double v, double* s_red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kThreads / 32; ++q) t += s_red[q];
    return t;
}

// ------------------------------------------------------------------ kernels

// Rows [in_off, in_off + in_len) of W strided lines -> tile (padded layout), by
// cp.async (no register round trip); other rows and missing lines are zeroed.
template <int W>
__device__ __forceinline__ void load_tile(const float2* in, long long Sj, const long long* off_in,
                                          long long l0, long long nlines, int in_off, int in_len,
                                          int L, float2* A, int LS) {
    for (int e = threadIdx.x; e < L * W; e += kThreads) {
        const int i = e % W, j = e / W;
        const int jj = j - in_off;
        float2* dst = A + i * LS + phy(j);
        if (l0 + i < nlines && jj >= 0 && jj < in_len) cp_async(dst, in + off_in[i] + jj * Sj, 8);
        else *dst = make_float2(0.f, 0.f);
    }
}

template <int W, int DIR, int LL>
__device__ __forceinline__ void c2c_body(const C2CPass& p, int bx, int by) {
    constexpr int NL = W / 8;
    const int L = LL > 0 ? LL : p.L;
    const int LS = pitch(L);
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + L;
    float2* B = A + W * LS;
    __shared__ long long off_in[W], off_out[W];
    const long long l0 = (long long)bx * W;
    if (threadIdx.x < W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, L);
    __syncthreads();
    load_tile<W>(p.in, p.lin.Sj, off_in, l0, p.nlines, p.in_off, p.in_len, L, A, LS);
    cp_async_commit();
    cp_async_wait0();
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    float2* res = line_fft<DIR, LL, NL>(A, B, L, LS, warp * NL, p.fac, s_tw, SmemLoad{A, LS});
    __syncthreads();
    for (int e = threadIdx.x; e < p.out_len * W; e += kThreads) {
        const int i = e % W, j = e / W;
        if (l0 + i < p.nlines)
            p.out[off_out[i] + j * p.lout.Sj] = cscale(res[i * LS + phy(j + p.out_off)], p.scale);
    }
}

template <int W, int DIR, int LL>
__global__ void __launch_bounds__(kThreads) k_c2c(C2CPass p) {
    c2c_body<W, DIR, LL>(p, blockIdx.x, blockIdx.y);
}

// Persistent variant: the CTAs stride over the tiles of n passes (device array).
template <int W, int DIR, int LL>
__global__ void __launch_bounds__(kThreads) k_c2c_g(const C2CPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        c2c_body<W, DIR, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}


template <int KIND>
struct SpecInfo;
template <> struct SpecInfo<SPEC_C64> { static constexpr int bytes = 8; };
template <> struct SpecInfo<SPEC_R32> { static constexpr int bytes = 4; };
template <> struct SpecInfo<SPEC_CBF16> { static constexpr int bytes = 4; };
template <> struct SpecInfo<SPEC_RBF16> { static constexpr int bytes = 2; };

template <int KIND>
__device__ __forceinline__ float2 spec_value(const unsigned char* base, int idx) {
    if constexpr (KIND == SPEC_C64) {
        return reinterpret_cast<const float2*>(base)[idx];
    } else if constexpr (KIND == SPEC_R32) {
        return make_float2(reinterpret_cast<const float*>(base)[idx], 0.f);
    } else if constexpr (KIND == SPEC_CBF16) {
        return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(base)[idx]);
    } else {
        return make_float2(__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[idx]), 0.f);
    }
}

// X[li][j] times the staged spectrum tile S[j][li] (row pitch SW), optionally conjugated.
template <int KIND>
struct MulLoad {
    const float2* X;
    int LS;
    const unsigned char* S;
    int SW;
    int conj;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        float2 h = spec_value<KIND>(S, j * SW + li);
        if (conj) h.y = -h.y;
        return cmul(X[li * LS + phy(j)], h);
    }
};

// Row pitch (elements) of a staged spectrum tile: W lines padded to a multiple of 16 bytes
// plus 16 bytes, so rows can be filled with 16-byte copies and read without bank conflicts.
template <int W, int ES>
struct SpecPitch {
    static constexpr int value = W + 16 / ES;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// Stage spectrum s of the tile (rows j < L of W lines) into shared memory S[j][i].
// A row whose W values are all present and 16-byte aligned travels as 16-byte
// cp.async chunks; other rows are copied element by element.
template <int W, int KIND, int NT = kThreads>
__device__ __forceinline__ void stage_spec(const MulPass& p, int L, int s, const long long* off_spec,
                                           long long l0, unsigned char* S) {
    constexpr int ES = SpecInfo<KIND>::bytes;
    constexpr int SW = SpecPitch<W, ES>::value;
    constexpr int CH = W * ES / 16;   // 16-byte chunks per full row
    const unsigned char* base = reinterpret_cast<const unsigned char*>(p.spec);
    const long long sbase = (long long)s * p.spec_stride;
    const bool full = l0 + W <= p.nlines && off_spec[W - 1] == off_spec[0] + (W - 1);
    for (int e = threadIdx.x; e < L * CH; e += NT) {
        const int j = e / CH, c = e - (e / CH) * CH;
        unsigned char* drow = S + (size_t)j * SW * ES;
        const unsigned char* srow = base + (size_t)(sbase + off_spec[0] + j * p.lspec.Sj) * ES;
        if (full && ((reinterpret_cast<uintptr_t>(srow) & 15) == 0)) {
            cp_async16(drow + 16 * c, srow + 16 * c);
        } else {
            // element-wise: chunk c covers lines [c * 16 / ES, (c + 1) * 16 / ES)
            for (int i = c * (16 / ES); i < (c + 1) * (16 / ES); ++i) {
                unsigned char* dst = drow + (size_t)i * ES;
                if (l0 + i < p.nlines) {
                    const unsigned char* src = base + (size_t)(sbase + off_spec[i] + j * p.lspec.Sj) * ES;
                    if constexpr (ES == 8) *reinterpret_cast<float2*>(dst) = *reinterpret_cast<const float2*>(src);
                    else if constexpr (ES == 4) *reinterpret_cast<float*>(dst) = *reinterpret_cast<const float*>(src);
                    else *reinterpret_cast<unsigned short*>(dst) = *reinterpret_cast<const unsigned short*>(src);
                } else {
                    if constexpr (ES == 8) *reinterpret_cast<float2*>(dst) = make_float2(0.f, 0.f);
                    else if constexpr (ES == 4) *reinterpret_cast<float*>(dst) = 0.f;
                    else *reinterpret_cast<unsigned short*>(dst) = 0;
                }
            }
        }
    }
}

template <int W, int KIND, int LL>
__device__ __forceinline__ void mul_body(const MulPass& p, int bx, int by) {
    constexpr int NL = W / 8;
    constexpr int ES = SpecInfo<KIND>::bytes;
    constexpr int SW = SpecPitch<W, ES>::value;
    const int L = LL > 0 ? LL : p.L;
    const int LS = pitch(L);
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + L;
    float2* B = A + W * LS;
    float2* C = B + W * LS;
    const size_t sp_bytes = (((size_t)L * SW * ES) + 15) & ~(size_t)15;
    unsigned char* SP0 = reinterpret_cast<unsigned char*>(C + W * LS);
    unsigned char* SP1 = SP0 + sp_bytes;
    __shared__ long long off_in[W], off_out[W], off_spec[W];
    const long long l0 = (long long)bx * W;
    if (threadIdx.x < W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
            off_spec[threadIdx.x] = line_offset(p.lspec, l);
        }
    }
    load_twiddles(s_tw, p.tw, L);
    __syncthreads();
    // grid.y splits the spectra into groups of p.nspec
    const int k0 = (int)by * p.nspec;
    const int nspec = min(p.nspec, p.ktotal - k0);
    // the first spectrum travels while the forward transform runs
    stage_spec<W, KIND>(p, L, k0, off_spec, l0, SP0);
    cp_async_commit();
    load_tile<W>(p.in, p.lin.Sj, off_in, l0, p.nlines, p.in_off, p.in_len, L, A, LS);
    cp_async_commit();
    cp_async_wait0();
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    float2* X = line_fft<-1, LL, NL>(A, B, L, LS, warp * NL, p.fac, s_tw, SmemLoad{A, LS});
    float2* U = (X == A) ? B : A;
    float2* V = C;
    for (int s = 0; s < nspec; ++s) {
        if (s + 1 < nspec) stage_spec<W, KIND>(p, L, k0 + s + 1, off_spec, l0, (s & 1) ? SP0 : SP1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const unsigned char* S = (s & 1) ? SP1 : SP0;
        float2* res = line_fft<1, LL, NL>(V, U, L, LS, warp * NL, p.fac, s_tw,
                                            MulLoad<KIND>{X, LS, S, SW, p.conj_spec});
        __syncthreads();
        float2* outp = p.out + (long long)(k0 + s) * p.out_stride;
        for (int e = threadIdx.x; e < p.out_len * W; e += kThreads) {
            const int i = e % W, j = e / W;
            if (l0 + i < p.nlines) outp[off_out[i] + j * p.lout.Sj] = res[i * LS + phy(j + p.out_off)];
        }
    }
}

template <int W, int KIND, int LL>
__global__ void __launch_bounds__(kThreads) k_mul(MulPass p) {
    mul_body<W, KIND, LL>(p, blockIdx.x, blockIdx.y);
}

// Persistent variant: the CTAs stride over the tiles of n passes (device array).
template <int W, int KIND, int LL>
__global__ void __launch_bounds__(kThreads) k_mul_g(const MulPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        mul_body<W, KIND, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}


// ------------------------------------------------------------------ register-resident transforms
//
// Lengths L = R1 * T with R1, T in {8, 16} (64, 128, 256) run as two Stockham
// stages held in registers.  T lanes own a line; lane t keeps points t + T m
// (m < R1).  Stage 1 is one radix-R1 DFT per lane (the points L / R1 = T apart),
// giving y[t R1 + q]; the lane multiplies them by the stage-2 twiddles
// w_L^(t q) and writes them to a warp-private exchange row; stage 2 reads
// y[c + R1 r] (r < T) for its R1 / T butterflies c = t + T h and leaves
// X[c + R1 r'] = X[t + T (h + (R1 / T) r')].  So a lane ends up holding the
// points t + T m of the result: the layout its stage 1 reads, which lets a
// forward spectrum stay in registers across the inverse transforms of a
// convolution.  The exchange row pads one slot per R1 points and its pitch is
// 8 (mod 16) float2, so the writes (17 t + q) and the reads (c + 17 r) of the two
// lines in a half-warp fall in distinct banks.

template <int L>
struct RegGeom;
template <> struct RegGeom<64> { static constexpr int R1 = 8, T = 8; };
template <> struct RegGeom<128> { static constexpr int R1 = 16, T = 8; };
template <> struct RegGeom<256> { static constexpr int R1 = 16, T = 16; };

template <int L>
struct RegFFT {
    static constexpr int R1 = RegGeom<L>::R1;
    static constexpr int T = RegGeom<L>::T;
    static constexpr int LPW = 32 / T;                                // lines per warp
    static constexpr int W = 16;                                      // lines per CTA
    static constexpr int NW = W / LPW;                                // warps per CTA
    static constexpr int NT = 32 * NW;                                // threads per CTA
    static constexpr int XS = ((L + L / R1 + 7) / 16) * 16 + 8;       // exchange pitch
    static constexpr int TWN = ((T - 1) * R1 + 1) & ~1;               // stage-2 twiddles (even)
    static constexpr int DEPTH = 3;                                   // spectra in flight per warp
};
template <int L>
__host__ __device__ constexpr bool reg_fft_length() { return L == 64 || L == 128 || L == 256; }

// Stage-2 twiddles w_L^(t q) (t = 1..T-1, q < R1) of the factorisation R1 x T: the
// last stage of the per-stage table (see twiddle_table), stored transposed at
// q (T - 1) + t - 1 so that the lanes of a warp read consecutive entries.
template <int L, int NT>
__device__ __forceinline__ void reg_twiddles(const float2* __restrict__ tw, float2* TW) {
    constexpr int R1 = RegGeom<L>::R1, T = RegGeom<L>::T;
    for (int i = threadIdx.x; i < (T - 1) * R1; i += NT) {
        const int q = i / (T - 1), tm = i - q * (T - 1);
        TW[i] = __ldg(tw + (R1 - 1) + tm * R1 + q);
    }
}

// In: v[m] = x[t + T m].  Out: v[m] = X[t + T m], X[k] = sum_j x[j] exp(DIR 2 pi i j k / L).
// TW: stage-2 twiddles (reg_twiddles); xl: this line's exchange row (XS float2), private
// to the warp.
template <int L, int DIR>
__device__ __forceinline__ void reg_fft(float2 (&v)[RegGeom<L>::R1], const float2* __restrict__ TW,
                                        float2* xl, int t) {
    constexpr int R1 = RegGeom<L>::R1, T = RegGeom<L>::T;
    dft<R1, DIR>(v);
    if (t > 0) {
        const float2* wt = TW + (t - 1);
#pragma unroll
        for (int q = 1; q < R1; ++q) {
            float2 c = wt[q * (T - 1)];
            if (DIR > 0) c.y = -c.y;
            v[q] = cmul(v[q], c);
        }
    }
#pragma unroll
    for (int q = 0; q < R1; ++q) xl[t * (R1 + 1) + q] = v[q];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < R1 / T; ++h) {
        float2 u[T];
#pragma unroll
        for (int r = 0; r < T; ++r) u[r] = xl[(t + T * h) + (R1 + 1) * r];
        dft<T, DIR>(u);
#pragma unroll
        for (int r = 0; r < T; ++r) v[h + (R1 / T) * r] = u[r];
    }
    __syncwarp();
}

// Copy rows [0, L) of spectrum s for the warp's LPW lines into S[j][li] (row pitch
// LPW * ES bytes).  When the lines are consecutive in the spectrum and every row
// starts 16-byte aligned (packed), rows travel as 16- or 8-byte cp.async chunks;
// otherwise element by element (lines >= nvalid read as 0).
template <int KIND, int L, int LPW>
__device__ __forceinline__ void stage_spec_warp(const MulPass& p, int s, const long long* offs, int nvalid,
                                                bool packed, unsigned char* S, int lane) {
    constexpr int ES = SpecInfo<KIND>::bytes;
    constexpr int RB = LPW * ES;                    // bytes per row
    const unsigned char* base = reinterpret_cast<const unsigned char*>(p.spec) + (long long)s * p.spec_stride * ES;
    const long long rs = p.lspec.Sj * ES;           // bytes between rows
    if (packed) {
        constexpr int CB = RB >= 16 ? 16 : RB;      // chunk bytes (RB is 4..32)
        constexpr int CPR = RB / CB;                // chunks per row
        const unsigned char* b0 = base + offs[0] * ES;
        for (int e = lane; e < L * CPR; e += 32) {
            const int j = e / CPR, c = e - (e / CPR) * CPR;
            const unsigned char* src = b0 + j * rs + c * CB;
            const unsigned sd = (unsigned)__cvta_generic_to_shared(S + j * RB + c * CB);
            if constexpr (CB == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sd), "l"(src));
            else if constexpr (CB == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sd), "l"(src));
            else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sd), "l"(src));
        }
    } else {
        for (int e = lane; e < L * LPW; e += 32) {
            const int j = e / LPW, i = e - (e / LPW) * LPW;
            unsigned char* dst = S + j * RB + i * ES;
            const unsigned char* src = base + (offs[i] + (long long)j * p.lspec.Sj) * ES;
            if constexpr (ES == 8) {
                if (i < nvalid) cp_async(dst, src, 8);
                else *reinterpret_cast<float2*>(dst) = make_float2(0.f, 0.f);
            } else if constexpr (ES == 4) {
                if (i < nvalid) cp_async(dst, src, 4);
                else *reinterpret_cast<float*>(dst) = 0.f;
            } else {
                *reinterpret_cast<unsigned short*>(dst) =
                    i < nvalid ? *reinterpret_cast<const unsigned short*>(src) : (unsigned short)0;
            }
        }
    }
}

// Spectrum multiply on a tile of 16 lines with the forward transform in registers.
// Each warp runs alone on its LPW lines: one forward transform, then for every
// spectrum s of the CTA's group, X * S_s, the inverse, and rows
// [out_off, out_off + out_len) stored straight from registers.  The warp keeps
// DEPTH spectra in flight in its own shared-memory ring (cp.async, __syncwarp).
template <int KIND, int LL>
__device__ __forceinline__ void mul_reg_items(const MulPass& p, int bx, int k0, int nspec) {
    using G = RegFFT<LL>;
    constexpr int L = LL, R1 = G::R1, T = G::T, LPW = G::LPW, D = G::DEPTH;
    constexpr int ES = SpecInfo<KIND>::bytes;
    constexpr int SB = L * LPW * ES;                 // bytes of one staged spectrum (per warp)
    extern __shared__ float4 smem_raw[];
    float2* TW = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* XW = TW + G::TWN + warp * (LPW * G::XS);                       // exchange rows
    unsigned char* SW0 = reinterpret_cast<unsigned char*>(TW + G::TWN + G::NW * LPW * G::XS) + warp * (D * SB);
    __shared__ long long offs[G::NW][3][LPW];        // in, out, spec offsets of the warp's lines
    const long long lw = (long long)bx * G::W + warp * LPW;     // first line of the warp
    const int nvalid = (int)max(0LL, min((long long)LPW, p.nlines - lw));
    if (lane < LPW && lane < nvalid) {
        offs[warp][0][lane] = line_offset(p.lin, lw + lane);
        offs[warp][1][lane] = line_offset(p.lout, lw + lane);
        offs[warp][2][lane] = line_offset(p.lspec, lw + lane);
    }
    reg_twiddles<L, G::NT>(p.tw, TW);
    __syncthreads();
    const int t = lane % T, li = lane / T;
    float2* xl = XW + li * G::XS;
    const bool valid = li < nvalid;
    bool packed = nvalid == LPW;
    if (packed) {
        const long long o0 = offs[warp][2][0];
#pragma unroll
        for (int i = 1; i < LPW; ++i) packed = packed && offs[warp][2][i] == o0 + i;
        constexpr int CB = LPW * ES >= 16 ? 16 : LPW * ES;   // chunk size of stage_spec_warp
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(p.spec) + (uintptr_t)(o0 * ES);
        const long long rs = p.lspec.Sj * ES;
        const long long ss = p.spec_stride * ES;
        packed = packed && a0 % CB == 0 && rs % CB == 0 && ss % CB == 0;
    }
    // prime the ring: spectra k0 .. k0 + D - 2 (one commit group each)
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
        if (q < nspec) stage_spec_warp<KIND, L, LPW>(p, k0 + q, offs[warp][2], nvalid, packed, SW0 + q * SB, lane);
        cp_async_commit();
    }
    float2 X[R1];
    {
        const float2* src = p.in + (valid ? offs[warp][0][li] : 0);
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int jj = t + T * m - p.in_off;
            X[m] = (valid && jj >= 0 && jj < p.in_len) ? __ldg(src + (long long)jj * p.lin.Sj)
                                                        : make_float2(0.f, 0.f);
        }
    }
    reg_fft<L, -1>(X, TW, xl, t);
    float2* dst = p.out + (valid ? offs[warp][1][li] : 0);
    for (int s = 0; s < nspec; ++s) {
        // refill the slot freed at s - 1 with spectrum s + D - 1
        if (s + D - 1 < nspec)
            stage_spec_warp<KIND, L, LPW>(p, k0 + s + D - 1, offs[warp][2], nvalid, packed,
                                          SW0 + ((s + D - 1) % D) * SB, lane);
        cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(D - 1));
        __syncwarp();
        const unsigned char* S = SW0 + (s % D) * SB;
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int e = (t + T * m) * LPW + li;
            if constexpr (KIND == SPEC_R32 || KIND == SPEC_RBF16) {
                const float h = spec_value<KIND>(S, e).x;
                v[m] = make_float2(X[m].x * h, X[m].y * h);
            } else {
                float2 h = spec_value<KIND>(S, e);
                if (p.conj_spec) h.y = -h.y;
                v[m] = cmul(X[m], h);
            }
        }
        reg_fft<L, 1>(v, TW, xl, t);
        if (valid) {
            float2* o = dst + (long long)(k0 + s) * p.out_stride;
#pragma unroll
            for (int m = 0; m < R1; ++m) {
                const int j = t + T * m - p.out_off;
                if (j >= 0 && j < p.out_len) o[(long long)j * p.lout.Sj] = v[m];
            }
        }
        __syncwarp();   // every lane is done with slot s % D before it is refilled
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// Batched complex transform of lines of a register-resident length: each warp
// loads its LPW lines straight into registers (rows [in_off, in_off + in_len)),
// transforms them and stores rows [out_off, out_off + out_len) scaled.
template <int DIR, int LL>
__device__ __forceinline__ void c2c_reg_body(const C2CPass& p, int bx, int by) {
    using G = RegFFT<LL>;
    constexpr int L = LL, R1 = G::R1, T = G::T, LPW = G::LPW;
    extern __shared__ float4 smem_raw[];
    float2* TW = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* XW = TW + G::TWN + warp * (LPW * G::XS);
    __shared__ long long offs[G::NW][2][LPW];
    const long long lw = (long long)bx * G::W + warp * LPW;
    const int nvalid = (int)max(0LL, min((long long)LPW, p.nlines - lw));
    if (lane < nvalid) {
        offs[warp][0][lane] = line_offset(p.lin, lw + lane);
        offs[warp][1][lane] = line_offset(p.lout, lw + lane);
    }
    reg_twiddles<L, G::NT>(p.tw, TW);
    __syncthreads();
    const int t = lane % T, li = lane / T;
    const bool valid = li < nvalid;
    float2 v[R1];
    {
        const float2* src = p.in + (valid ? offs[warp][0][li] : 0);
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int jj = t + T * m - p.in_off;
            v[m] = (valid && jj >= 0 && jj < p.in_len) ? __ldg(src + (long long)jj * p.lin.Sj)
                                                        : make_float2(0.f, 0.f);
        }
    }
    reg_fft<L, DIR>(v, TW, XW + li * G::XS, t);
    if (valid) {
        float2* o = p.out + offs[warp][1][li];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int j = t + T * m - p.out_off;
            if (j >= 0 && j < p.out_len) o[(long long)j * p.lout.Sj] = cscale(v[m], p.scale);
        }
    }
}

template <int DIR, int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_c2c_reg(C2CPass p) {
    c2c_reg_body<DIR, LL>(p, blockIdx.x, blockIdx.y);
}

template <int DIR, int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_c2c_reg_g(const C2CPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        c2c_reg_body<DIR, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}

// Tile bx of the lines, spectra [by nspec, (by + 1) nspec) of the pass.
template <int KIND, int LL>
__device__ __forceinline__ void mul_reg_body(const MulPass& p, int bx, int by) {
    const int k0 = by * p.nspec;
    mul_reg_items<KIND, LL>(p, bx, k0, min(p.nspec, p.ktotal - k0));
}

template <int KIND, int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_mul_reg(MulPass p) {
    mul_reg_body<KIND, LL>(p, blockIdx.x, blockIdx.y);
}

// Persistent form for many spectra: the (tile, spectrum) items, tile-major, are split
// into gridDim.x equal contiguous ranges (one per resident CTA), so the work is spread
// evenly instead of in whole waves of (tile, group) CTAs; a range runs as one piece per
// tile it touches (one forward transform per piece).
template <int KIND, int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_mul_reg_p(MulPass p, int ntiles) {
    const long long total = (long long)ntiles * p.ktotal;
    const long long lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
    for (long long it = lo; it < hi;) {
        const int tile = (int)(it / p.ktotal), k0 = (int)(it - (long long)tile * p.ktotal);
        const int nk = (int)min((long long)(p.ktotal - k0), hi - it);
        mul_reg_items<KIND, LL>(p, tile, k0, nk);
        __syncthreads();   // the twiddles and line offsets are reloaded by the next piece
        it += nk;
    }
}

template <int KIND, int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_mul_reg_g(const MulPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        mul_reg_body<KIND, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}

template <int W, int LL>
__device__ __forceinline__ void r2c_body(const R2CPass& p, int bx, int by) {
    constexpr int NL = W / 8;
    const int L = LL > 0 ? LL : p.L;
    const int LS = pitch(L);
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + L;
    float2* B = A + W * LS;
    __shared__ long long off_in[2 * W], off_out[2 * W];
    const long long l0 = (long long)bx * (2 * W);
    if (threadIdx.x < 2 * W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, L);
    __syncthreads();
    float* Af = reinterpret_cast<float*>(A);
    for (int e = threadIdx.x; e < 2 * W * L; e += kThreads) {
        const int q = e / L, j = e - (e / L) * L;
        const int jj = j - p.in_off;
        float* dst = Af + ((q >> 1) * LS + phy(j)) * 2 + (q & 1);
        if (l0 + q < p.nlines && jj >= 0 && jj < p.in_len) cp_async(dst, p.in + off_in[q] + jj, 4);
        else *dst = 0.f;
    }
    cp_async_commit();
    cp_async_wait0();
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    float2* Z = line_fft<-1, LL, NL>(A, B, L, LS, warp * NL, p.fac, s_tw, SmemLoad{A, LS});
    __syncthreads();
    const int H = L / 2 + 1;
    for (int e = threadIdx.x; e < W * H; e += kThreads) {
        const int i = e / H, k = e - (e / H) * H;
        const float2 z = Z[i * LS + phy(k)];
        const float2 zm = Z[i * LS + phy((L - k) % L)];
        // a = FFT of line 2i, b = FFT of line 2i+1 (two real lines in one complex FFT)
        const float2 a = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        const float2 b = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
        if (l0 + 2 * i < p.nlines) p.out[off_out[2 * i] + k] = a;
        if (l0 + 2 * i + 1 < p.nlines) p.out[off_out[2 * i + 1] + k] = b;
    }
}

template <int W, int LL>
__global__ void __launch_bounds__(kThreads) k_r2c(R2CPass p) {
    r2c_body<W, LL>(p, blockIdx.x, blockIdx.y);
}

// Persistent variant: the CTAs stride over the tiles of n passes (device array).
template <int W, int LL>
__global__ void __launch_bounds__(kThreads) k_r2c_g(const R2CPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        r2c_body<W, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}


// Z = A + i B for complex line li from the staged half spectra of real lines
// 2 li (A) and 2 li + 1 (B), with the Hermitian extension on (L/2, L).
struct HermLoad {
    const float2* R;   // raw half spectra, real line q at q * HS
    int HS, L;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        const bool lo = 2 * j <= L;
        const int k = lo ? j : L - j;
        const float2 a = R[(2 * li) * HS + k];
        const float2 b = R[(2 * li + 1) * HS + k];
        return lo ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, b.x - a.y);
    }
};

constexpr int kC2RMaxSlots = 16;  // max outputs per lane in the certificate epilogue

template <int W>
__device__ __forceinline__ void stage_half(const C2RPass& p, int L, int s, const long long* off_in,
                                           long long l0, float2* R, int HS) {
    const int H = L / 2 + 1;
    const float2* in = p.in + (long long)s * p.in_spec_stride;
    for (int e = threadIdx.x; e < 2 * W * H; e += kThreads) {
        const int q = e / H, k = e - (e / H) * H;
        if (l0 + q < p.nlines) cp_async(R + q * HS + k, in + off_in[q] + k, 8);
        else R[q * HS + k] = make_float2(0.f, 0.f);
    }
}

template <int W, int MODE, int SLOTS, int LL>
__device__ __forceinline__ void c2r_body(const C2RPass& p, int bx, int by) {
    constexpr int NL = W / 8;
    const int L = LL > 0 ? LL : p.L;
    const int LS = pitch(L);
    const int H = L / 2 + 1;
    const int HS = H + 1;
    extern __shared__ float4 smem_raw[];
    float2* s_tw = reinterpret_cast<float2*>(smem_raw);
    float2* A = s_tw + L;
    float2* B = A + W * LS;
    float2* R0 = B + W * LS;
    float2* R1 = R0 + 2 * W * HS;
    __shared__ long long off_in[2 * W], off_out[2 * W];
    __shared__ double s_red[kThreads / 32];
    const long long l0 = (long long)bx * (2 * W);
    if (threadIdx.x < 2 * W) {
        long long l = l0 + threadIdx.x;
        if (l < p.nlines) {
            off_in[threadIdx.x] = line_offset(p.lin, l);
            off_out[threadIdx.x] = line_offset(p.lout, l);
        }
    }
    load_twiddles(s_tw, p.tw, L);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q0 = 2 * NL * warp;                // first real output line of this warp
    const int nout = 2 * NL * p.out_len;         // outputs of this warp

    float mx[SLOTS];
    int ak[SLOTS];
    bool saw_nan = false;
    double acc = 0.0;
#pragma unroll
    for (int it = 0; it < SLOTS; ++it) {
        mx[it] = -INFINITY;
        ak[it] = 0;
    }
    // certificate: grid.y splits the kernels into groups of p.nspec
    const int k0 = (MODE == C2R_CERTMAX) ? (int)by * p.nspec : 0;
    const int nspec = (MODE == C2R_CERTMAX) ? min(p.nspec, p.ktotal - k0) : 1;
    stage_half<W>(p, L, k0, off_in, l0, R0, HS);
    // residual: the tile's observation rows travel with the spectrum, into the second
    // staging buffer (one spectrum per CTA in this mode; 2W out_len floats fit in it)
    float* Ys = reinterpret_cast<float*>(R1);
    if constexpr (MODE == C2R_RESIDUAL) {
        for (int e = threadIdx.x; e < 2 * W * p.out_len; e += kThreads) {
            const int q = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
            if (l0 + q < p.nlines) cp_async(Ys + e, p.y + off_out[q] + j, 4);
        }
    }
    cp_async_commit();
    for (int s = 0; s < nspec; ++s) {
        if (s + 1 < nspec) stage_half<W>(p, L, k0 + s + 1, off_in, l0, (s & 1) ? R0 : R1, HS);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const float2* Rs = (s & 1) ? R1 : R0;
        float2* z = line_fft<1, LL, NL>(B, A, L, LS, warp * NL, p.fac, s_tw, HermLoad{Rs, HS, L});
        if constexpr (MODE != C2R_CERTMAX) {
            for (int e = lane; e < nout; e += 32) {
                const int qq = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                const int q = q0 + qq;
                if (l0 + q >= p.nlines) continue;
                const float2 zz = z[(q >> 1) * LS + phy(j + p.out_off)];
                const float v = ((q & 1) ? zz.y : zz.x) * p.scale;
                const long long o = off_out[q] + j;
                if constexpr (MODE == C2R_STORE) {
                    p.out[o] = v;
                } else {
                    const float r = Ys[q * p.out_len + j] - v;
                    if (p.out) p.out[o] = r;
                    acc += (double)r * (double)r;
                }
            }
        } else {
            const int kk = k0 + s;
#pragma unroll
            for (int it = 0; it < SLOTS; ++it) {
                const int e = lane + 32 * it;
                if (e < nout) {
                    const int qq = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                    const int q = q0 + qq;
                    if (l0 + q < p.nlines) {
                        const float2 zz = z[(q >> 1) * LS + phy(j + p.out_off)];
                        const float v = ((q & 1) ? zz.y : zz.x) * p.scale;
                        if (p.eta_out) p.eta_out[(long long)kk * p.V + off_out[q] + j] = v;
                        if (v != v) saw_nan = true;
                        if (v > mx[it]) {
                            mx[it] = v;
                            ak[it] = kk;
                        }
                    }
                }
            }
        }
        __syncthreads();   // the staged buffer of spectrum s is refilled at s + 2
    }
    if constexpr (MODE == C2R_RESIDUAL) {
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) s_red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += s_red[w];
            p.partials[bx] = t;
        }
        // the last tile to finish forms C = 1/2 sum r^2 + lambda sum w (fixed order)
        if (p.loss_out && last_block(p.counter, p.ntiles)) {
            double a = 0.0;
            for (int i = threadIdx.x; i < p.ntiles; i += kThreads) a += __ldcg(p.partials + i);
            double wsum = 0.0;
            for (int i = threadIdx.x; i < p.nw; i += kThreads) wsum += (double)__ldg(p.w + (long long)i * p.w_stride);
            const double t = block_sum_d(0.5 * a + p.lambda * wsum, s_red);
            if (threadIdx.x == 0) {
                *p.loss_out = t;
                *p.counter = 0u;
            }
        }
    }
    if constexpr (MODE == C2R_CERTMAX) {
        unsigned long long best = 0ull;
#pragma unroll
        for (int it = 0; it < SLOTS; ++it) {
            const int e = lane + 32 * it;
            if (e < nout) {
                const int qq = e / p.out_len, j = e - (e / p.out_len) * p.out_len;
                const int q = q0 + qq;
                if (l0 + q < p.nlines) {
                    const long long o = off_out[q] + j;
                    const unsigned long long key =
                        candidate_key(mx[it], (unsigned long long)ak[it] * p.V + o);
                    if (p.vox_key) atomicMax(p.vox_key + o, key);
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
            if (lane == 0 && best) atomicMax(p.best_key, best);
            // the last tile decodes the key and re-arms it (0) for the next call
            __syncthreads();
            if (last_block(p.counter, p.ntiles) && threadIdx.x == 0) {
                const unsigned long long k = atomicExch(p.best_key, 0ull);
                if (k == ~0ull || k == 0ull) {
                    if (p.best_val) *p.best_val = __int_as_float(0x7fc00000);
                    if (p.best_idx) *p.best_idx = -1;
                } else {
                    if (p.best_val) *p.best_val = float_from_order_key((unsigned int)(k >> 32));
                    if (p.best_idx) *p.best_idx = (int64_t)(0xffffffffu - (unsigned int)(k & 0xffffffffu));
                }
                *p.counter = 0u;
            }
        }
    }
}

// Certificate epilogue on the register-resident transform (lengths 64/128/256, rows
// [0, out_len) kept with out_len <= L / 2).  Each complex line carries the real
// lines 2 li (real part) and 2 li + 1 (imaginary part); a warp owns LPW complex
// lines and stages the half spectra of its 2 LPW real lines (pitch HS, 4 mod 8
// float2 so the two lines a half-warp reads fall in distinct banks), two spectra
// deep.  Lane t keeps the running max over the CTA's kernels of its outputs
// t + T m (m < R1 / 2) of both real lines, then publishes them as candidate keys.
template <int LL>
struct RegC2R {
    using G = RegFFT<LL>;
    static constexpr int H = LL / 2 + 1;
    static constexpr int HS = ((H + 3) / 8) * 8 + 4;
    static constexpr int RL = 2 * G::LPW;          // real lines per warp
    static constexpr int D = 2;                    // staged spectra per warp
    static constexpr int SB = RL * HS;             // float2 per staged spectrum
    static size_t smem() {
        return sizeof(float2) * ((size_t)G::TWN + (size_t)G::NW * G::LPW * G::XS + (size_t)G::NW * D * SB);
    }
};

template <int LL>
__device__ __forceinline__ void c2r_reg_max_body(const C2RPass& p, int bx, int by) {
    using G = RegFFT<LL>;
    using C = RegC2R<LL>;
    constexpr int L = LL, R1 = G::R1, T = G::T, LPW = G::LPW, H = C::H, HS = C::HS, RL = C::RL;
    constexpr int MH = R1 / 2;                     // kept outputs per lane and real line
    extern __shared__ float4 smem_raw[];
    float2* TW = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* XW = TW + G::TWN + warp * (LPW * G::XS);
    float2* STG = TW + G::TWN + G::NW * LPW * G::XS + warp * (C::D * C::SB);
    __shared__ long long offs[G::NW][2][RL];
    const long long lw = ((long long)bx * G::W + warp * LPW) * 2;   // first real line of the warp
    const int nvalid = (int)max(0LL, min((long long)RL, p.nlines - lw));
    if (lane < nvalid) {
        offs[warp][0][lane] = line_offset(p.lin, lw + lane);
        offs[warp][1][lane] = line_offset(p.lout, lw + lane);
    }
    reg_twiddles<L, G::NT>(p.tw, TW);
    __syncthreads();
    const int t = lane % T, li = lane / T;
    float2* xl = XW + li * G::XS;
    const int k0 = (int)by * p.nspec;
    const int nspec = min(p.nspec, p.ktotal - k0);
    auto stage = [&](int s, float2* dst) {
        const float2* in = p.in + (long long)s * p.in_spec_stride;
        for (int e = lane; e < RL * H; e += 32) {
            const int r = e / H, k = e - (e / H) * H;
            if (r < nvalid) cp_async(dst + r * HS + k, in + offs[warp][0][r] + k, 8);
            else dst[r * HS + k] = make_float2(0.f, 0.f);
        }
    };
    stage(k0, STG);
    cp_async_commit();
    float mx[2][MH];
    int ak[2][MH];
#pragma unroll
    for (int m = 0; m < MH; ++m) {
        mx[0][m] = mx[1][m] = -INFINITY;
        ak[0][m] = ak[1][m] = 0;
    }
    bool saw_nan = false;
    const bool v0 = 2 * li < nvalid, v1 = 2 * li + 1 < nvalid;
    for (int s = 0; s < nspec; ++s) {
        if (s + 1 < nspec) stage(k0 + s + 1, STG + ((s + 1) & 1) * C::SB);
        cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        const float2* Rs = STG + (s & 1) * C::SB;
        const float2* ra = Rs + (2 * li) * HS;
        const float2* rb = ra + HS;
        float2 v[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) {
            const int j = t + T * m;
            const bool lo = 2 * j <= L;
            const int k = lo ? j : L - j;
            const float2 a = ra[k], b = rb[k];
            v[m] = lo ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, b.x - a.y);
        }
        reg_fft<L, 1>(v, TW, xl, t);
        const int kk = k0 + s;
#pragma unroll
        for (int m = 0; m < MH; ++m) {
            const int j = t + T * m;
            if (j < p.out_len) {
                const float a = v[m].x * p.scale, b = v[m].y * p.scale;
                if (p.eta_out) {
                    float* e = p.eta_out + (long long)kk * p.V + j;
                    if (v0) e[offs[warp][1][2 * li]] = a;
                    if (v1) e[offs[warp][1][2 * li + 1]] = b;
                }
                saw_nan = saw_nan || (v0 && a != a) || (v1 && b != b);
                if (a > mx[0][m]) {
                    mx[0][m] = a;
                    ak[0][m] = kk;
                }
                if (b > mx[1][m]) {
                    mx[1][m] = b;
                    ak[1][m] = kk;
                }
            }
        }
        __syncwarp();   // every lane is done with this slot before it is refilled
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!(h ? v1 : v0)) continue;
        const long long ob = offs[warp][1][2 * li + h];
#pragma unroll
        for (int m = 0; m < MH; ++m) {
            const int j = t + T * m;
            if (j < p.out_len && nspec > 0) {
                const long long o = ob + j;
                const unsigned long long key = candidate_key(mx[h][m], (unsigned long long)ak[h][m] * p.V + o);
                if (p.vox_key) atomicMax(p.vox_key + o, key);
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
        if (lane == 0 && best) atomicMax(p.best_key, best);
        __syncthreads();
        if (last_block(p.counter, p.ntiles) && threadIdx.x == 0) {
            const unsigned long long k = atomicExch(p.best_key, 0ull);
            if (k == ~0ull || k == 0ull) {
                if (p.best_val) *p.best_val = __int_as_float(0x7fc00000);
                if (p.best_idx) *p.best_idx = -1;
            } else {
                if (p.best_val) *p.best_val = float_from_order_key((unsigned int)(k >> 32));
                if (p.best_idx) *p.best_idx = (int64_t)(0xffffffffu - (unsigned int)(k & 0xffffffffu));
            }
            *p.counter = 0u;
        }
    }
}

template <int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_c2r_reg_max(C2RPass p) {
    c2r_reg_max_body<LL>(p, blockIdx.x, blockIdx.y);
}

template <int LL>
__global__ void __launch_bounds__(RegFFT<LL>::NT) k_c2r_reg_max_g(const C2RPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        c2r_reg_max_body<LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}

template <int W, int MODE, int SLOTS, int LL>
__global__ void __launch_bounds__(kThreads) k_c2r(C2RPass p) {
    c2r_body<W, MODE, SLOTS, LL>(p, blockIdx.x, blockIdx.y);
}

// Persistent variant: the CTAs stride over the tiles of n passes (device array).
template <int W, int MODE, int SLOTS, int LL>
__global__ void __launch_bounds__(kThreads) k_c2r_g(const C2RPass* __restrict__ ps,
        const int* __restrict__ start, const int* __restrict__ nbx, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const int local = t - start[q];
        c2r_body<W, MODE, SLOTS, LL>(ps[q], local % nbx[q], local / nbx[q]);
        __syncthreads();
    }
}


// ------------------------------------------------------------------ launchers

// The certificate epilogue runs on the register-resident transform when the length
// has one and the kept rows are [0, out_len) with out_len <= L / 2.
inline bool c2r_on_reg(const C2RPass& p) {
    return (p.L == 64 || p.L == 128 || p.L == 256) && p.mode == C2R_CERTMAX && p.out_off == 0 &&
           2 * p.out_len <= p.L;
}

// Raise a kernel's dynamic shared-memory limit once per (device, kernel, size):
// the attribute call is kept out of stream captures after the first use.
template <typename KernelT>
inline sfw_status prepare(KernelT kernel, size_t smem) {
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

inline size_t tile_bytes(int L, int W, int nbuf) {
    return sizeof(float2) * ((size_t)L + (size_t)nbuf * W * pitch(L));
}

inline int spec_bytes(int kind) {
    return kind == SPEC_C64 ? 8 : kind == SPEC_RBF16 ? 2 : 4;
}

// Single launch (g == NULL: one pass, kernel parameter by value) or persistent
// grouped launch (g: n passes of the same template variant in device memory).
template <class Single, class Grouped, class PassT>
inline sfw_status run_either(Single ks, Grouped kg, const char* name, const PassT& p, dim3 grid1,
                             size_t smem, cudaStream_t st, GroupArgs* g, int nt = kThreads) {
    if (!g) {
        SFW_TRY(prepare(ks, smem));
        SFW_LAUNCH(st, name, ks<<<grid1, nt, smem, st>>>(p));
    } else {
        SFW_TRY(prepare(kg, smem));
        if (g->grid <= 0) {  // resident CTAs, computed once (before any capture)
            int dev = 0, sms = 1, per = 1;
            SFW_CUDA(cudaGetDevice(&dev));
            SFW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            SFW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kg, nt, smem));
            if (per < 1) per = 1;
            g->grid = g->total < per * sms ? g->total : per * sms;
        }
        if (g->total <= 0) return SFW_OK;
        SFW_LAUNCH(st, name, kg<<<g->grid, nt, smem, st>>>(
            reinterpret_cast<const PassT*>(g->passes), g->start, g->nbx, g->n));
    }
    return launch_check(name);
}

template <int LL>
sfw_status run_c2c(const C2CPass& p, cudaStream_t st, GroupArgs* g) {
    if (!g && p.nlines <= 0) return SFW_OK;
    int W, nbx, nby;
    pass_tiles(p, &W, &nbx, &nby);
    const dim3 grid1((unsigned)nbx);
    if constexpr (reg_fft_length<LL>()) {
        using G = RegFFT<LL>;
        const size_t rs = sizeof(float2) * ((size_t)G::TWN + (size_t)G::NW * G::LPW * G::XS);
        if (p.dir < 0) return run_either(k_c2c_reg<-1, LL>, k_c2c_reg_g<-1, LL>, "k_c2c_reg", p, grid1, rs, st, g, G::NT);
        return run_either(k_c2c_reg<1, LL>, k_c2c_reg_g<1, LL>, "k_c2c_reg", p, grid1, rs, st, g, G::NT);
    }
    const size_t smem = tile_bytes(p.L, W, 2);
    if (W == 16) {
        if (p.dir < 0) return run_either(k_c2c<16, -1, LL>, k_c2c_g<16, -1, LL>, "k_c2c", p, grid1, smem, st, g);
        return run_either(k_c2c<16, 1, LL>, k_c2c_g<16, 1, LL>, "k_c2c", p, grid1, smem, st, g);
    }
    if (p.dir < 0) return run_either(k_c2c<8, -1, LL>, k_c2c_g<8, -1, LL>, "k_c2c", p, grid1, smem, st, g);
    return run_either(k_c2c<8, 1, LL>, k_c2c_g<8, 1, LL>, "k_c2c", p, grid1, smem, st, g);
}

// Launch of k_mul_reg_p with one CTA per resident slot (occupancy computed once per
// device, kernel and shared-memory size, outside any stream capture's first use).
template <typename KernelT>
inline sfw_status run_mul_persistent(KernelT kernel, const MulPass& p, int ntiles, size_t smem, int nt,
                                     cudaStream_t st) {
    SFW_TRY(prepare(kernel, smem));
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, int> slots;
    int dev = 0;
    SFW_CUDA(cudaGetDevice(&dev));
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto key = std::make_tuple(dev, reinterpret_cast<const void*>(kernel), smem);
        auto it = slots.find(key);
        if (it != slots.end()) {
            grid = it->second;
        } else {
            int sms = 1, per = 1;
            SFW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            SFW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, smem));
            grid = (per < 1 ? 1 : per) * sms;
            slots[key] = grid;
        }
    }
    const long long items = (long long)ntiles * p.ktotal;
    if (items < grid) grid = (int)items;
    if (grid <= 0) return SFW_OK;
    SFW_LAUNCH(st, "k_mul_reg", kernel<<<grid, nt, smem, st>>>(p, ntiles));
    return launch_check("k_mul_reg");
}

template <int LL>
sfw_status run_mul(const MulPass& p, cudaStream_t st, GroupArgs* g) {
    if (!g && p.nlines <= 0) return SFW_OK;
    int W, nbx, nby;
    pass_tiles(p, &W, &nbx, &nby);
    const int es = spec_bytes(p.spec_kind);
    const size_t sp = ((size_t)p.L * (W + 16 / es) * es + 15) & ~(size_t)15;
    const dim3 grid1((unsigned)nbx, (unsigned)nby);
    if constexpr (reg_fft_length<LL>()) {
        using G = RegFFT<LL>;
        const size_t smem = sizeof(float2) * ((size_t)G::TWN + (size_t)G::NW * G::LPW * G::XS) +
                            (size_t)G::NW * G::DEPTH * LL * G::LPW * es;
        if (!g && p.ktotal > 1) {   // many spectra: persistent, evenly split items
            switch (p.spec_kind) {
                case SPEC_C64: return run_mul_persistent(k_mul_reg_p<SPEC_C64, LL>, p, nbx, smem, G::NT, st);
                case SPEC_R32: return run_mul_persistent(k_mul_reg_p<SPEC_R32, LL>, p, nbx, smem, G::NT, st);
                case SPEC_CBF16: return run_mul_persistent(k_mul_reg_p<SPEC_CBF16, LL>, p, nbx, smem, G::NT, st);
                default: return run_mul_persistent(k_mul_reg_p<SPEC_RBF16, LL>, p, nbx, smem, G::NT, st);
            }
        }
#define SFW_MULR(KK) return run_either(k_mul_reg<KK, LL>, k_mul_reg_g<KK, LL>, "k_mul_reg", p, grid1, smem, st, g, G::NT)
        switch (p.spec_kind) {
            case SPEC_C64: SFW_MULR(SPEC_C64);
            case SPEC_R32: SFW_MULR(SPEC_R32);
            case SPEC_CBF16: SFW_MULR(SPEC_CBF16);
            default: SFW_MULR(SPEC_RBF16);
        }
#undef SFW_MULR
    }
    const size_t smem = tile_bytes(p.L, W, 3) + 2 * sp;
#define SFW_MUL(WW, KK) return run_either(k_mul<WW, KK, LL>, k_mul_g<WW, KK, LL>, "k_mul", p, grid1, smem, st, g)
    switch (p.spec_kind) {
        case SPEC_C64: if (W == 16) SFW_MUL(16, SPEC_C64); else SFW_MUL(8, SPEC_C64);
        case SPEC_R32: if (W == 16) SFW_MUL(16, SPEC_R32); else SFW_MUL(8, SPEC_R32);
        case SPEC_CBF16: if (W == 16) SFW_MUL(16, SPEC_CBF16); else SFW_MUL(8, SPEC_CBF16);
        default: if (W == 16) SFW_MUL(16, SPEC_RBF16); else SFW_MUL(8, SPEC_RBF16);
    }
#undef SFW_MUL
}

template <int LL>
sfw_status run_r2c(const R2CPass& p, cudaStream_t st, GroupArgs* g) {
    if (!g && p.nlines <= 0) return SFW_OK;
    int W, nbx, nby;
    pass_tiles(p, &W, &nbx, &nby);
    const size_t smem = tile_bytes(p.L, W, 2);
    const dim3 grid1((unsigned)nbx);
    if (W == 16) return run_either(k_r2c<16, LL>, k_r2c_g<16, LL>, "k_r2c", p, grid1, smem, st, g);
    return run_either(k_r2c<8, LL>, k_r2c_g<8, LL>, "k_r2c", p, grid1, smem, st, g);
}

template <int LL>
sfw_status run_c2r(const C2RPass& p, cudaStream_t st, int* blocks_out, GroupArgs* g) {
    int W, nbx, nby;
    pass_tiles(p, &W, &nbx, &nby);
    if (blocks_out) *blocks_out = nbx;
    if (!g && p.nlines <= 0) return SFW_OK;
    if constexpr (reg_fft_length<LL>()) {
        if (c2r_on_reg(p)) {
            const dim3 grid1((unsigned)nbx, (unsigned)nby);
            return run_either(k_c2r_reg_max<LL>, k_c2r_reg_max_g<LL>, "k_c2r_reg_max", p, grid1,
                              RegC2R<LL>::smem(), st, g, RegFFT<LL>::NT);
        }
    }
    const int need = (2 * (W / 8) * p.out_len + 31) / 32;
    if (p.mode == C2R_CERTMAX && need > kC2RMaxSlots)
        return fail(SFW_ERR_SHAPE, "c2r: %d outputs per line exceed the epilogue tile", p.out_len);
    const int H = p.L / 2 + 1;
    const size_t smem = tile_bytes(p.L, W, 2) + sizeof(float2) * 2 * 2 * (size_t)W * (H + 1);
    const dim3 grid1((unsigned)nbx, (unsigned)nby);
#define SFW_C2R(WW, MM, SS) return run_either(k_c2r<WW, MM, SS, LL>, k_c2r_g<WW, MM, SS, LL>, "k_c2r", p, grid1, smem, st, g)
    switch (p.mode) {
        case C2R_STORE: if (W == 16) SFW_C2R(16, C2R_STORE, 1); else SFW_C2R(8, C2R_STORE, 1);
        case C2R_RESIDUAL: if (W == 16) SFW_C2R(16, C2R_RESIDUAL, 1); else SFW_C2R(8, C2R_RESIDUAL, 1);
        default:
            if (need <= 4) SFW_C2R(8, C2R_CERTMAX, 4);
            else if (need <= 8) SFW_C2R(8, C2R_CERTMAX, 8);
            else SFW_C2R(8, C2R_CERTMAX, 16);
    }
#undef SFW_C2R
}

// explicit instantiations live in fft_len_*.cu
#define SFW_FFT_INSTANTIATE(LL)                                                       \
    template sfw_status run_c2c<LL>(const C2CPass&, cudaStream_t, GroupArgs*);        \
    template sfw_status run_mul<LL>(const MulPass&, cudaStream_t, GroupArgs*);        \
    template sfw_status run_r2c<LL>(const R2CPass&, cudaStream_t, GroupArgs*);        \
    template sfw_status run_c2r<LL>(const C2RPass&, cudaStream_t, int*, GroupArgs*);

#define SFW_FFT_DECLARE(LL)                                                           \
    extern template sfw_status run_c2c<LL>(const C2CPass&, cudaStream_t, GroupArgs*); \
    extern template sfw_status run_mul<LL>(const MulPass&, cudaStream_t, GroupArgs*); \
    extern template sfw_status run_r2c<LL>(const R2CPass&, cudaStream_t, GroupArgs*); \
    extern template sfw_status run_c2r<LL>(const C2RPass&, cudaStream_t, int*, GroupArgs*);

}  // namespace sfw
