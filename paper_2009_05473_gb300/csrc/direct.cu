// The plain FP32 route: the forward operator, its transpose and the grid
// certificate by direct sums, without any transform.
//
//   blur (Eq. 3)       y(s) = sum_j H[j] f_E[s + 2R - j],        s in the grid
//   transpose (Eq. 5)  b_E(t) = sum_j H[j] r[t - 2R + j],        t in E, s = t - 2R + j in the grid
//   certificate (Eq. 5, step 1 of Algorithms 1 and 2)
//                      eta_k(m) = (1/lambda) sum_delta g_k(delta) b_E[m + R + delta]
//
// with E index t <-> grid coordinate t - R (the extended grid of the rendered
// atoms) and g_k the unit atom (sigma_k, d_k) tabulated on the box of its cut-off
// radius (the same truncation g >= eps as the rendering; zero outside it).  Each
// thread owns one output voxel and walks the taps in order with FP32 accumulation:
// the straightforward form the transform route is measured against.  The
// criterion and the grid maximum use the same FP64 partial sums and 64-bit
// candidate keys as the transform route (ties -> lowest flat index k V + lin(m),
// NaN -> index -1).
#include "sfw_internal.cuh"

namespace sfw {

constexpr int kDirThreads = 256;

// One voxel of H * f_E on the grid.
__device__ __forceinline__ float direct_blur_at(const float* __restrict__ fE, const float* __restrict__ H,
                                                int s0, int s1, int s2, int R0, int R1, int R2, int E1,
                                                int E2) {
    const int w1 = 2 * R1 + 1, w2 = 2 * R2 + 1;
    float acc = 0.f;
    for (int j0 = 0; j0 <= 2 * R0; ++j0) {
        const float* frow0 = fE + (long long)(s0 + 2 * R0 - j0) * E1 * E2;
        float plane = 0.f;
        for (int j1 = 0; j1 <= 2 * R1; ++j1) {
            const float* frow = frow0 + (long long)(s1 + 2 * R1 - j1) * E2 + s2 + 2 * R2;
            const float* hrow = H + ((long long)j0 * w1 + j1) * w2;
            float row = 0.f;
            for (int j2 = 0; j2 < w2; ++j2) row = fmaf(__ldg(hrow + j2), __ldg(frow - j2), row);
            plane += row;
        }
        acc += plane;
    }
    return acc;
}

// Blur f_E onto the grid.  Store mode (y == NULL): out = H * f_E.  Residual mode:
// out = y - H * f_E (out may be NULL) and the criterion C = 1/2 sum r^2 + lambda sum w
// (FP64 partials per block; the last block sums them in block order and re-arms the
// counter).
__global__ void __launch_bounds__(kDirThreads)
k_direct_blur(const float* __restrict__ fE, const float* __restrict__ H, int n0, int n1, int n2, int R0,
              int R1, int R2, float* out, const float* __restrict__ y, double* partials,
              unsigned int* counter, double* loss_out, const float* w, int nw, double lambda) {
    const long long V = (long long)n0 * n1 * n2;
    const int E1 = n1 + 2 * R1, E2 = n2 + 2 * R2;
    double acc2 = 0.0;
    for (long long i = blockIdx.x * (long long)kDirThreads + threadIdx.x; i < V;
         i += (long long)gridDim.x * kDirThreads) {
        const int s2 = (int)(i % n2);
        const long long q = i / n2;
        const int s1 = (int)(q % n1);
        const int s0 = (int)(q / n1);
        const float v = direct_blur_at(fE, H, s0, s1, s2, R0, R1, R2, E1, E2);
        if (y) {
            const float r = y[i] - v;
            if (out) out[i] = r;
            acc2 += (double)r * (double)r;
        } else {
            out[i] = v;
        }
    }
    if (!y) return;
    __shared__ double s_red[kDirThreads / 32];
    for (int off = 16; off > 0; off >>= 1) acc2 += __shfl_down_sync(0xffffffffu, acc2, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kDirThreads / 32; ++q) t += s_red[q];
        partials[blockIdx.x] = t;
    }
    if (last_block(counter, gridDim.x) && threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) t += partials[b];
        double sw = 0.0;
        for (int q = 0; q < nw; ++q) sw += (double)w[q];
        if (loss_out) *loss_out = 0.5 * t + lambda * sw;
        *counter = 0u;
    }
}

// b_E = H^T r: every point of the extended grid, taps whose grid point lies inside.
__global__ void __launch_bounds__(kDirThreads)
k_direct_transpose(const float* __restrict__ r, const float* __restrict__ H, int n0, int n1, int n2,
                   int R0, int R1, int R2, float* __restrict__ bE) {
    const int E0 = n0 + 2 * R0, E1 = n1 + 2 * R1, E2 = n2 + 2 * R2;
    const long long VE = (long long)E0 * E1 * E2;
    const int w1 = 2 * R1 + 1, w2 = 2 * R2 + 1;
    for (long long i = blockIdx.x * (long long)kDirThreads + threadIdx.x; i < VE;
         i += (long long)gridDim.x * kDirThreads) {
        const int t2 = (int)(i % E2);
        const long long q = i / E2;
        const int t1 = (int)(q % E1);
        const int t0 = (int)(q / E1);
        // s_a = t_a - 2 R_a + j_a in [0, n_a)
        const int j0lo = max(0, 2 * R0 - t0), j0hi = min(2 * R0, n0 - 1 - t0 + 2 * R0);
        const int j1lo = max(0, 2 * R1 - t1), j1hi = min(2 * R1, n1 - 1 - t1 + 2 * R1);
        const int j2lo = max(0, 2 * R2 - t2), j2hi = min(2 * R2, n2 - 1 - t2 + 2 * R2);
        float acc = 0.f;
        for (int j0 = j0lo; j0 <= j0hi; ++j0) {
            float plane = 0.f;
            for (int j1 = j1lo; j1 <= j1hi; ++j1) {
                const float* rrow = r + ((long long)(t0 - 2 * R0 + j0) * n1 + (t1 - 2 * R1 + j1)) * n2 +
                                    (t2 - 2 * R2);
                const float* hrow = H + ((long long)j0 * w1 + j1) * w2;
                float row = 0.f;
                for (int j2 = j2lo; j2 <= j2hi; ++j2) row = fmaf(__ldg(hrow + j2), __ldg(rrow + j2), row);
                plane += row;
            }
            acc += plane;
        }
        bE[i] = acc;
    }
}

// Grid certificate by direct sums.  kern[k] = (offset of g_k in gtab, half-width h_k):
// g_k is stored on (2h_k + 1)^3, C order, centre at (h_k, h_k, h_k).  One thread per
// voxel runs every kernel; eta_out (K x V) optional; per-voxel max / argk (ties ->
// lowest k) optional; the grid maximum as a candidate key (last block decodes it).
__global__ void __launch_bounds__(kDirThreads)
k_direct_cert(const float* __restrict__ bE, const float* __restrict__ gtab, const int2* __restrict__ kern,
              int K, int n0, int n1, int n2, int R0, int R1, int R2, float scale, float* eta_out,
              float* max_out, int* argk_out, unsigned long long* best_key, unsigned int* counter,
              float* best_val, int64_t* best_idx) {
    const long long V = (long long)n0 * n1 * n2;
    const int E0 = n0 + 2 * R0, E1 = n1 + 2 * R1, E2 = n2 + 2 * R2;
    unsigned long long best = 0ull;
    for (long long i = blockIdx.x * (long long)kDirThreads + threadIdx.x; i < V;
         i += (long long)gridDim.x * kDirThreads) {
        const int m2 = (int)(i % n2);
        const long long q = i / n2;
        const int m1 = (int)(q % n1);
        const int m0 = (int)(q / n1);
        // E point of delta = 0
        const int c0 = m0 + R0, c1 = m1 + R1, c2 = m2 + R2;
        unsigned long long vkey = 0ull;
        for (int k = 0; k < K; ++k) {
            const int2 kh = kern[k];
            const int h = kh.y, wd = 2 * h + 1;
            const float* g = gtab + kh.x;
            const int d0lo = max(-h, -c0), d0hi = min(h, E0 - 1 - c0);
            const int d1lo = max(-h, -c1), d1hi = min(h, E1 - 1 - c1);
            const int d2lo = max(-h, -c2), d2hi = min(h, E2 - 1 - c2);
            float acc = 0.f;
            for (int d0 = d0lo; d0 <= d0hi; ++d0) {
                float plane = 0.f;
                for (int d1 = d1lo; d1 <= d1hi; ++d1) {
                    const float* grow = g + ((long long)(d0 + h) * wd + (d1 + h)) * wd + h;
                    const float* brow = bE + ((long long)(c0 + d0) * E1 + (c1 + d1)) * E2 + c2;
                    float row = 0.f;
                    for (int d2 = d2lo; d2 <= d2hi; ++d2) row = fmaf(__ldg(grow + d2), __ldg(brow + d2), row);
                    plane += row;
                }
                acc += plane;
            }
            const float eta = acc * scale;
            if (eta_out) eta_out[(long long)k * V + i] = eta;
            const unsigned long long key = candidate_key(eta, (unsigned long long)k * V + i);
            if (key > vkey) vkey = key;
        }
        if (max_out || argk_out) {
            float v;
            int a;
            if (vkey == ~0ull) {
                v = __int_as_float(0x7fc00000);
                a = 0;
            } else {
                v = float_from_order_key((unsigned int)(vkey >> 32));
                a = (int)((0xffffffffu - (unsigned int)(vkey & 0xffffffffu)) / V);
            }
            if (max_out) max_out[i] = v;
            if (argk_out) argk_out[i] = a;
        }
        if (vkey > best) best = vkey;
    }
    if (!best_key) return;
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, best, off);
        if (o > best) best = o;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(best_key, best);
    if (last_block(counter, gridDim.x) && threadIdx.x == 0) {
        const unsigned long long k = atomicExch(best_key, 0ull);
        if (k == ~0ull || k == 0ull) {
            if (best_val) *best_val = __int_as_float(0x7fc00000);
            if (best_idx) *best_idx = -1;
        } else {
            if (best_val) *best_val = float_from_order_key((unsigned int)(k >> 32));
            if (best_idx) *best_idx = (int64_t)(0xffffffffu - (unsigned int)(k & 0xffffffffu));
        }
        *counter = 0u;
    }
}

static int direct_blocks(long long items, int num_sms) {
    long long b = (items + kDirThreads - 1) / kDirThreads;
    const long long cap = 8LL * num_sms;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

sfw_status launch_direct_blur(const DirectBlur& p, cudaStream_t st) {
    const long long V = (long long)p.n[0] * p.n[1] * p.n[2];
    const int nb = direct_blocks(V, p.num_sms);
    if (p.y && nb > p.partials_len) return fail(SFW_ERR_SHAPE, "direct blur: partial buffer too small");
    SFW_LAUNCH(st, "k_direct_blur",
               k_direct_blur<<<nb, kDirThreads, 0, st>>>(p.fE, p.H, p.n[0], p.n[1], p.n[2], p.R[0], p.R[1],
                                                          p.R[2], p.out, p.y, p.partials, p.counter,
                                                          p.loss_out, p.w, p.nw, p.lambda));
    return launch_check("k_direct_blur");
}

sfw_status launch_direct_transpose(const float* r, const float* H, const int n[3], const int R[3],
                                   float* bE, int num_sms, cudaStream_t st) {
    const long long VE = (long long)(n[0] + 2 * R[0]) * (n[1] + 2 * R[1]) * (n[2] + 2 * R[2]);
    const int nb = direct_blocks(VE, num_sms);
    SFW_LAUNCH(st, "k_direct_transpose",
               k_direct_transpose<<<nb, kDirThreads, 0, st>>>(r, H, n[0], n[1], n[2], R[0], R[1], R[2], bE));
    return launch_check("k_direct_transpose");
}

sfw_status launch_direct_cert(const DirectCert& p, cudaStream_t st) {
    const long long V = (long long)p.n[0] * p.n[1] * p.n[2];
    const int nb = direct_blocks(V, p.num_sms);
    SFW_LAUNCH(st, "k_direct_cert",
               k_direct_cert<<<nb, kDirThreads, 0, st>>>(p.bE, p.gtab, p.kern, p.K, p.n[0], p.n[1], p.n[2],
                                                          p.R[0], p.R[1], p.R[2], p.scale, p.eta_out,
                                                          p.max_out, p.argk_out, p.best_key, p.counter,
                                                          p.best_val, p.best_idx));
    return launch_check("k_direct_cert");
}

}  // namespace sfw
