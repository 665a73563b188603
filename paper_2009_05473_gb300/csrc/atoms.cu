// Atom kernels: rendering of the measure's atoms on the extended grid (Eq. 2,
// summed as inside Eq. 3) and the per-atom adjoint sums of the analytic
// gradient of the criterion (Eq. 4; Section 2: "grad C is computed
// analytically", "parallelized across atoms").
//
// Both evaluate g(rho) = exp(-(rho/sigma)^d / 2) as
//     g = exp2(-log2(e)/2 * exp2((d/2) * log2(rho^2 / sigma^2))),
// which needs no special case at rho = 0 (log2(0) = -inf gives g = 1).  An
// atom is evaluated only inside its cut-off radius
//     rho_max = sigma * (2 ln(1/eps))^(1/d),   g(rho_max) = eps.
#include <math.h>

#include "sfw_internal.cuh"

namespace sfw {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ float atom_cut2(float sigma, float d, float log_inv_eps2) {
    // rho_max^2 = sigma^2 (2 ln(1/eps))^(2/d)
    return sigma * sigma * exp2f((2.0f / d) * log_inv_eps2);
}

// ------------------------------------------------------------------ render

constexpr int kRX = 32, kRY = 4, kRZ = 2;  // tile: axis 2 x axis 1 x axis 0
constexpr int kRenderThreads = kRX * kRY * kRZ;

__device__ __forceinline__ void render_body(const AtomsDev& a, int E0, int E1, int E2, int R0, int R1,
                                            int R2, float log_inv_eps2, float* f, int bx, int by,
                                            int bz) {
    __shared__ float s_m0[kRenderThreads], s_m1[kRenderThreads], s_m2[kRenderThreads];
    __shared__ float s_is2[kRenderThreads], s_hd[kRenderThreads], s_w[kRenderThreads];
    __shared__ float s_c2[kRenderThreads];
    __shared__ int s_wcount[kRenderThreads / 32];
    __shared__ int s_total;

    const int tx = threadIdx.x % kRX;
    const int ty = (threadIdx.x / kRX) % kRY;
    const int tz = threadIdx.x / (kRX * kRY);
    const int t2 = bx * kRX + tx;
    const int t1 = by * kRY + ty;
    const int t0 = bz * kRZ + tz;
    // grid coordinates of this voxel and of the tile's bounding box
    const float x0 = (float)(t0 - R0), x1 = (float)(t1 - R1), x2 = (float)(t2 - R2);
    const float b0lo = (float)(bz * kRZ - R0), b0hi = b0lo + (kRZ - 1);
    const float b1lo = (float)(by * kRY - R1), b1hi = b1lo + (kRY - 1);
    const float b2lo = (float)(bx * kRX - R2), b2hi = b2lo + (kRX - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float acc = 0.f;
    for (int base = 0; base < a.N; base += kRenderThreads) {
        const int ai = base + threadIdx.x;
        bool keep = false;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, sg = 1.f, dd = 2.f, w = 0.f, c2 = 0.f;
        if (ai < a.N) {
            m0 = a.m[a.ms * ai + 0];
            m1 = a.m[a.ms * ai + 1];
            m2 = a.m[a.ms * ai + 2];
            sg = a.sigma[a.ps * ai];
            dd = a.d[a.ps * ai];
            w = a.w[a.ps * ai];
            c2 = atom_cut2(sg, dd, log_inv_eps2);
            const float e0 = m0 - fminf(fmaxf(m0, b0lo), b0hi);
            const float e1 = m1 - fminf(fmaxf(m1, b1lo), b1hi);
            const float e2 = m2 - fminf(fmaxf(m2, b2lo), b2hi);
            keep = (e0 * e0 + e1 * e1 + e2 * e2) <= c2 && w != 0.f;
        }
        // order-preserving compaction of the kept atoms (deterministic sums)
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wcount[warp] = __popc(ball);
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int q = 0; q < kRenderThreads / 32; ++q) {
                const int c = s_wcount[q];
                s_wcount[q] = run;
                run += c;
            }
            s_total = run;
        }
        __syncthreads();
        if (keep) {
            const int pos = s_wcount[warp] + __popc(ball & ((1u << lane) - 1u));
            s_m0[pos] = m0;
            s_m1[pos] = m1;
            s_m2[pos] = m2;
            s_is2[pos] = 1.0f / (sg * sg);
            s_hd[pos] = 0.5f * dd;
            s_w[pos] = w;
            s_c2[pos] = c2;
        }
        __syncthreads();
        const int cnt = s_total;
        for (int q = 0; q < cnt; ++q) {
            const float e0 = x0 - s_m0[q], e1 = x1 - s_m1[q], e2 = x2 - s_m2[q];
            const float r2 = e0 * e0 + e1 * e1 + e2 * e2;
            if (r2 <= s_c2[q]) {
                const float u = exp2f(s_hd[q] * __log2f(r2 * s_is2[q]));
                acc += s_w[q] * exp2f(-0.5f * kLog2e * u);
            }
        }
        __syncthreads();
    }
    if (t0 < E0 && t1 < E1 && t2 < E2) f[((long long)t0 * E1 + t1) * E2 + t2] = acc;
}

__global__ void __launch_bounds__(kRenderThreads)
k_render(AtomsDev a, int E0, int E1, int E2, int R0, int R1, int R2, float log_inv_eps2, float* f) {
    render_body(a, E0, E1, E2, R0, R1, R2, log_inv_eps2, f, blockIdx.x, blockIdx.y, blockIdx.z);
}

int render_tiles(const RenderOp& op, int* nbx) {
    *nbx = (op.E[2] + kRX - 1) / kRX;
    return *nbx * ((op.E[1] + kRY - 1) / kRY) * ((op.E[0] + kRZ - 1) / kRZ);
}

// Persistent render over the tiles of n volumes.
__global__ void __launch_bounds__(kRenderThreads)
k_render_g(const RenderOp* __restrict__ ops, const int* __restrict__ start, const int* __restrict__ nbx,
           int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const RenderOp& o = ops[q];
        const int local = t - start[q];
        const int ny = (o.E[1] + kRY - 1) / kRY;
        const int bx = local % nbx[q], r = local / nbx[q];
        const float lie2 = log2f(2.0f * logf(1.0f / o.eps));
        render_body(o.a, o.E[0], o.E[1], o.E[2], o.R[0], o.R[1], o.R[2], lie2, o.f, bx, r % ny, r / ny);
        __syncthreads();
    }
}

sfw_status launch_render_group(const RenderOp* ops, const int* start, const int* nbx, int n,
                               int total, int grid, cudaStream_t st) {
    if (total <= 0) return SFW_OK;
    SFW_LAUNCH(st, "k_render", k_render_g<<<grid, kRenderThreads, 0, st>>>(ops, start, nbx, n));
    return launch_check("k_render_g");
}

sfw_status launch_render(const AtomsDev& a, const int E[3], const int R[3], float eps, float* f,
                         cudaStream_t st) {
    if (g_recorder) {
        RenderOp op;
        op.a = a;
        for (int q = 0; q < 3; ++q) {
            op.E[q] = E[q];
            op.R[q] = R[q];
        }
        op.eps = eps;
        op.f = f;
        return g_recorder->add(op);
    }
    dim3 grid((E[2] + kRX - 1) / kRX, (E[1] + kRY - 1) / kRY, (E[0] + kRZ - 1) / kRZ);
    const float log_inv_eps2 = log2f(2.0f * logf(1.0f / eps));
    SFW_LAUNCH(st, "k_render", k_render<<<grid, kRenderThreads, 0, st>>>(a, E[0], E[1], E[2], R[0], R[1], R[2], log_inv_eps2, f));
    return launch_check("k_render");
}

// ------------------------------------------------------------------ adjoint gradient

constexpr int kGradThreads = 256;

// Warp 0 sums the chunk partials of atom n in a fixed order (lane c takes chunks
// c, c + 32, ...); the six loads of a chunk are issued together.
__device__ __forceinline__ void warp_chunk_sums(int n, int chunks, const double* partials, double s[6]) {
    const int lane = threadIdx.x & 31;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = lane; c < chunks; c += 32) {
        const double* p = partials + ((long long)n * chunks + c) * 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] += __ldcg(p + q);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
        s[q] = v[q];
    }
}

// Chunk c (of nchunks) of atom n strides over the atom's box and writes six
// partial sums; the last chunk-block of the atom to finish turns the atom's
// partials into its gradient entries (mode 0) or its certificate and
// certificate gradient (mode 1), then re-arms the atom's counter.
template <bool ETA_ONLY>
__device__ __forceinline__ void atom_grad_body(const AtomsDev& a, int E0, int E1, int E2, int R0,
                                               int R1, int R2, float log_inv_eps2,
                                               const float* __restrict__ b, double* partials, int n,
                                               int c, int nchunks, const AdjFin& fin) {
    const float m0 = a.m[a.ms * n + 0], m1 = a.m[a.ms * n + 1], m2 = a.m[a.ms * n + 2];
    const float sg = a.sigma[a.ps * n], dd = a.d[a.ps * n];
    const float c2 = atom_cut2(sg, dd, log_inv_eps2);
    const float rmax = sqrtf(c2);
    const float is2 = 1.0f / (sg * sg);
    const float hd = 0.5f * dd;
    // box in E index coordinates (E index = grid coordinate + R)
    const int lo0 = max(0, (int)ceilf(m0 + R0 - rmax)), hi0 = min(E0 - 1, (int)floorf(m0 + R0 + rmax));
    const int lo1 = max(0, (int)ceilf(m1 + R1 - rmax)), hi1 = min(E1 - 1, (int)floorf(m1 + R1 + rmax));
    const int lo2 = max(0, (int)ceilf(m2 + R2 - rmax)), hi2 = min(E2 - 1, (int)floorf(m2 + R2 + rmax));
    const int n0 = max(0, hi0 - lo0 + 1), n1 = max(0, hi1 - lo1 + 1);
    const int nrows = n0 * n1;

    // warps of the atom's chunk-blocks take whole (t0, t1) rows of the box; the lanes
    // walk the part of a row inside the cut-off sphere along the contiguous axis.  A
    // warp loads RB rows (up to 64 points each) before evaluating any of them: the
    // loads of b, not the arithmetic, set the time of a row.
    constexpr int RB = 4;
    const int lane = threadIdx.x & 31;
    const int wpb = kGradThreads / 32;
    const int wstride = nchunks * wpb;
    float sg_b = 0.f, sm0 = 0.f, sm1 = 0.f, sm2 = 0.f, ss = 0.f, sd = 0.f;
    auto point = [&](float e0, float e1, float r01, int t2, float bt) {
        const float e2 = m2 - (float)(t2 - R2);
        const float r2 = r01 + e2 * e2;
        if (r2 > c2) return;
        const float lq = __log2f(r2 * is2);
        const float u = 0.5f * exp2f(hd * lq);
        const float g = exp2f(-kLog2e * u);
        const float gb = g * bt;
        sg_b += gb;
        if constexpr (ETA_ONLY) return;   // eta alone: no derivative sums
        if (r2 > 0.f) {
            // dg/dm_a = -g d u (m_a - x_a) / rho^2
            const float cm = -gb * dd * u / r2;
            sm0 += cm * e0;
            sm1 += cm * e1;
            sm2 += cm * e2;
            ss += gb * (dd / sg) * u;              // dg/dsigma = g (d/sigma) u
            sd += -gb * u * (0.5f * kLn2 * lq);    // dg/dd = -g u ln(rho/sigma)
        }
    };
    for (int row0 = c * wpb + (threadIdx.x >> 5); row0 < nrows; row0 += RB * wstride) {
        float e0s[RB], e1s[RB], r01s[RB], bv[RB][2];
        int a2s[RB], b2s[RB];
        const float* brows[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            const int row = row0 + q * wstride;
            a2s[q] = 0;
            b2s[q] = -1;
            e0s[q] = e1s[q] = r01s[q] = 0.f;
            brows[q] = b;
            if (row < nrows) {
                const int i0 = row / n1, i1 = row - (row / n1) * n1;
                const int t0 = lo0 + i0, t1 = lo1 + i1;
                e0s[q] = m0 - (float)(t0 - R0);
                e1s[q] = m1 - (float)(t1 - R1);
                r01s[q] = e0s[q] * e0s[q] + e1s[q] * e1s[q];
                if (r01s[q] <= c2) {
                    const float h = sqrtf(c2 - r01s[q]);
                    a2s[q] = max(lo2, (int)ceilf(m2 + R2 - h));
                    b2s[q] = min(hi2, (int)floorf(m2 + R2 + h));
                    brows[q] = b + ((long long)t0 * E1 + t1) * E2;
                }
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int t2 = a2s[q] + 32 * hh + lane;
                bv[q][hh] = t2 <= b2s[q] ? brows[q][t2] : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < RB; ++q) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int t2 = a2s[q] + 32 * hh + lane;
                if (t2 <= b2s[q]) point(e0s[q], e1s[q], r01s[q], t2, bv[q][hh]);
            }
            // rows longer than 64 points (broad atoms)
            for (int t2 = a2s[q] + 64 + lane; t2 <= b2s[q]; t2 += 32) point(e0s[q], e1s[q], r01s[q], t2, brows[q][t2]);
        }
    }
    // warp sums in FP32 (a pairwise tree of 32), the block's warp sums in FP64, one
    // quantity per thread (the FP64 pipe is narrow on this part)
    __shared__ double s_part[6][kGradThreads / 32];
    const float out[6] = {sm0, sm1, sm2, ss, sd, sg_b};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float v = out[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) s_part[q][threadIdx.x >> 5] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int w = 0; w < kGradThreads / 32; ++w) t += s_part[threadIdx.x][w];
        partials[((long long)n * nchunks + c) * 6 + threadIdx.x] = t;
    }
    if (!fin.counters || !last_block(fin.counters + n, nchunks)) return;
    if (threadIdx.x < 32) {
        double su[6];
        warp_chunk_sums(n, nchunks, partials, su);
        if (threadIdx.x == 0) {
            if (fin.mode == 0) {
                const double w = a.w[a.ps * n];
                const int N = a.N;
                fin.grad[3 * n + 0] = -w * su[0];
                fin.grad[3 * n + 1] = -w * su[1];
                fin.grad[3 * n + 2] = -w * su[2];
                fin.grad[3 * N + n] = -w * su[3];
                fin.grad[4 * N + n] = -w * su[4];
                fin.grad[5 * N + n] = fin.lambda - su[5];
            } else {
                fin.eta[n] = su[5] / fin.lambda;
                if (fin.grad)
                    for (int q = 0; q < 5; ++q) fin.grad[5 * n + q] = su[q] / fin.lambda;
            }
            fin.counters[n] = 0u;
        }
    }
}

template <bool ETA_ONLY>
__global__ void __launch_bounds__(kGradThreads, 3)
k_atom_grad(AtomsDev a, int E0, int E1, int E2, int R0, int R1, int R2, float log_inv_eps2,
            const float* __restrict__ b, double* partials, AdjFin fin) {
    atom_grad_body<ETA_ONLY>(a, E0, E1, E2, R0, R1, R2, log_inv_eps2, b, partials, blockIdx.x, blockIdx.y,
                             gridDim.y, fin);
}

int grad_tiles(const GradOp& op, int* nbx) {
    *nbx = kGradChunks;
    return op.a.N * kGradChunks;
}

__global__ void __launch_bounds__(kGradThreads, 3)
k_atom_grad_g(const GradOp* __restrict__ ops, const int* __restrict__ start, const int* __restrict__ nbx,
              int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        const GradOp& o = ops[q];
        const int local = t - start[q];
        const float lie2 = log2f(2.0f * logf(1.0f / o.eps));
        atom_grad_body<false>(o.a, o.E[0], o.E[1], o.E[2], o.R[0], o.R[1], o.R[2], lie2, o.b, o.partials,
                              local / kGradChunks, local % kGradChunks, kGradChunks, o.fin);
        __syncthreads();
    }
}

sfw_status launch_grad_group(const GradOp* ops, const int* start, const int* nbx, int n, int total,
                             int grid, cudaStream_t st) {
    if (total <= 0) return SFW_OK;
    SFW_LAUNCH(st, "k_atom_grad", k_atom_grad_g<<<grid, kGradThreads, 0, st>>>(ops, start, nbx, n));
    return launch_check("k_atom_grad_g");
}

static sfw_status adjoint(const AtomsDev& a, const int E[3], const int R[3], float eps,
                          const float* b, double* partials, const AdjFin& fin, cudaStream_t st) {
    if (a.N <= 0) return SFW_OK;
    if (g_recorder) {
        GradOp op;
        op.a = a;
        for (int q = 0; q < 3; ++q) {
            op.E[q] = E[q];
            op.R[q] = R[q];
        }
        op.eps = eps;
        op.b = b;
        op.partials = partials;
        op.fin = fin;
        return g_recorder->add(op);
    }
    const float log_inv_eps2 = log2f(2.0f * logf(1.0f / eps));
    dim3 grid(a.N, kGradChunks);
    // eta without its gradient (the FP32 re-score of grid candidates): the value sums alone
    if (fin.mode == 1 && !fin.grad)
        SFW_LAUNCH(st, "k_atom_grad", k_atom_grad<true><<<grid, kGradThreads, 0, st>>>(a, E[0], E[1], E[2], R[0], R[1], R[2], log_inv_eps2, b, partials, fin));
    else
        SFW_LAUNCH(st, "k_atom_grad", k_atom_grad<false><<<grid, kGradThreads, 0, st>>>(a, E[0], E[1], E[2], R[0], R[1], R[2], log_inv_eps2, b, partials, fin));
    return launch_check("k_atom_grad");
}

sfw_status launch_atom_grad(const AtomsDev& a, const int E[3], const int R[3], float eps,
                            const float* b, double lambda, double* partials, double* grad,
                            unsigned int* counters, cudaStream_t st) {
    AdjFin fin;
    fin.mode = 0;
    fin.lambda = lambda;
    fin.grad = grad;
    fin.eta = nullptr;
    fin.counters = counters;
    return adjoint(a, E, R, eps, b, partials, fin, st);
}

sfw_status launch_eta_points(const AtomsDev& pts, const int E[3], const int R[3], float eps,
                             const float* b, double lambda, double* partials, double* eta,
                             double* grad, unsigned int* counters, cudaStream_t st) {
    AdjFin fin;
    fin.mode = 1;
    fin.lambda = lambda;
    fin.grad = grad;
    fin.eta = eta;
    fin.counters = counters;
    return adjoint(pts, E, R, eps, b, partials, fin, st);
}

// ------------------------------------------------------------------ top-k re-scoring

__global__ void k_candidate_theta(const int64_t* vox, const int* argk, const float* grid_sd,
                                  int topk, int n0, int n1, int n2, float* theta) {
    const int i = threadIdx.x;
    if (i >= topk) return;
    const int64_t v = vox[i];
    if (v < 0) {  // NaN in the certificate: no candidate
        for (int q = 0; q < 5; ++q) theta[5 * i + q] = __int_as_float(0x7fc00000);
        return;
    }
    const int k = argk[v];
    theta[5 * i + 0] = (float)(v / ((int64_t)n1 * n2));
    theta[5 * i + 1] = (float)((v / n2) % n1);
    theta[5 * i + 2] = (float)(v % n2);
    theta[5 * i + 3] = grid_sd[2 * k];
    theta[5 * i + 4] = grid_sd[2 * k + 1];
}

sfw_status launch_candidate_theta(const int64_t* vox, const int* argk, const float* grid_sd,
                                  int topk, const int n[3], float* theta, cudaStream_t st) {
    SFW_LAUNCH(st, "k_candidate_theta", k_candidate_theta<<<1, 64, 0, st>>>(vox, argk, grid_sd, topk, n[0], n[1], n[2], theta));
    return launch_check("k_candidate_theta");
}

__global__ void k_candidate_select(const float* theta, const float* grid_val, const double* eta,
                                   int topk, float* theta_out, float* grid_out, double* eta_out,
                                   float* best_theta, double* best_eta) {
    const int i = threadIdx.x;
    if (i < topk) {
        if (theta_out)
            for (int q = 0; q < 5; ++q) theta_out[5 * i + q] = theta[5 * i + q];
        if (grid_out) grid_out[i] = grid_val[i];
        if (eta_out) eta_out[i] = eta[i];
    }
    if (i == 0) {
        int b = 0;
        for (int j = 1; j < topk; ++j)
            if (eta[j] > eta[b]) b = j;
        if (best_theta)
            for (int q = 0; q < 5; ++q) best_theta[q] = theta[5 * b + q];
        if (best_eta) *best_eta = eta[b];
    }
}

sfw_status launch_candidate_select(const float* theta, const float* grid_val, const double* eta,
                                   int topk, float* theta_out, float* grid_out, double* eta_out,
                                   float* best_theta, double* best_eta, cudaStream_t st) {
    SFW_LAUNCH(st, "k_candidate_select", k_candidate_select<<<1, 64, 0, st>>>(theta, grid_val, eta, topk, theta_out, grid_out, eta_out, best_theta, best_eta));
    return launch_check("k_candidate_select");
}

// ------------------------------------------------------------------ Gram matrix (LASSO of step 3)

// Copy atom i of a set into a one-atom slot with unit weight: (m0, m1, m2, sigma, d, 1).
__global__ void k_unit_atom(AtomsDev a, int i, float* slot) {
    if (threadIdx.x == 0) {
        slot[0] = a.m[a.ms * i + 0];
        slot[1] = a.m[a.ms * i + 1];
        slot[2] = a.m[a.ms * i + 2];
        slot[3] = a.sigma[a.ps * i];
        slot[4] = a.d[a.ps * i];
        slot[5] = 1.0f;
    }
}

sfw_status launch_unit_atom(const AtomsDev& a, int i, float* slot, cudaStream_t st) {
    SFW_LAUNCH(st, "k_unit_atom", k_unit_atom<<<1, 32, 0, st>>>(a, i, slot));
    return launch_check("k_unit_atom");
}

// One block per pair (i, j >= i) and per row (i, N) for <a_i, y>: FP64 sums over V.
__global__ void __launch_bounds__(256) k_gram(const float* __restrict__ A, const float* __restrict__ y,
                                              int N, long long V, double* G, double* c) {
    __shared__ double s_red[8];
    // block b -> pair index in the upper triangle (with the y column as j = N)
    int b = blockIdx.x, i = 0;
    while (b >= N + 1 - i) {
        b -= N + 1 - i;
        ++i;
    }
    const int j = i + b;
    const float* ai = A + (long long)i * V;
    const float* aj = j < N ? A + (long long)j * V : y;
    double acc = 0.0;
    for (long long v = threadIdx.x; v < V; v += 256) acc += (double)ai[v] * (double)aj[v];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += s_red[q];
        if (j < N) {
            G[(long long)i * N + j] = t;
            G[(long long)j * N + i] = t;
        } else {
            c[i] = t;
        }
    }
}

sfw_status launch_gram(const float* A, const float* y, int N, long long V, double* G, double* c,
                       cudaStream_t st) {
    const int pairs = N * (N + 1) / 2 + N;
    SFW_LAUNCH(st, "k_gram", k_gram<<<pairs, 256, 0, st>>>(A, y, N, V, G, c));
    return launch_check("k_gram");
}

}  // namespace sfw
