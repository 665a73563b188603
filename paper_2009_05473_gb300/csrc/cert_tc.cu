// The certificate's axis-0 inverse on the tensor cores (bf16 operands, FP32
// accumulation in tensor memory), for plans whose kernel-family table is real
// and stored in bfloat16 (the precision mode).
//
// For one line l = (p1, h2) of the half spectrum, the axis-0 stage of Eq. 5's
// correlation with the table (Section 2's lookup table) is
//     U_k[i0, l] = sum_{p0 < P0} W[i0, p0] X[p0, l] T_k[p0, l],   W[i0, p0] = e^{2 pi i i0 p0 / P0}
// with X the forward axis-0 spectrum of the residual ((P0, nl), row p0 holding every
// line) and T_k real.  In real arithmetic, with Z = X (.) T_k,
//     [Re U_k; Im U_k] = [Re W  -Im W; Im W  Re W] [Re Z; Im Z],
// a GEMM whose left factor (the inverse DFT rows, K = 2 P0) is the same for every line
// and kernel: it is built once per plan and held in shared memory, 64 output rows i0
// (128 real rows: the M = 128 of one tcgen05.mma) per CTA.  Each line contributes the
// right factor B' = [T_l (.) Re X_l | T_l (.) Im X_l] over its K kernels (N), built by the
// CTA's worker warps from a bulk-copied table block and the staged X line; LG lines
// accumulate side by side in tensor memory before they are written back as FP32 complex
// for the following passes (axes 1 and 2).  Operands use the 128-byte swizzled K-major
// layout.
#include <math.h>

#include "sfw_internal.cuh"
#include "tc_sm100.cuh"

namespace sfw {

constexpr int kTcThreads = 128;   // one thread per real output row
constexpr int kTcCols = 256;      // tensor-memory columns: two buffers of LG * Np <= 128

// ------------------------------------------------------------------ table in the MMA layout

// Tb[l] = T_l as the K-major B operand of Np rows (kernels) x Kp (p0), zero-padded.
__global__ void k_tc_table(const float2* __restrict__ full, long long spec_elems, int K, int P0, long long nl,
                           int Np, int Kp, __nv_bfloat16* __restrict__ Tb) {
    const long long per = (long long)Np * Kp;
    const long long total = nl * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long l = i / per;
        const int e = (int)(i - l * per);
        const int n = e / Kp, p0 = e - n * Kp;
        float v = 0.f;
        if (n < K && p0 < P0) v = full[(long long)n * spec_elems + (long long)p0 * nl + l].x;
        unsigned char* blk = reinterpret_cast<unsigned char*>(Tb + l * per);
        *reinterpret_cast<__nv_bfloat16*>(blk + tc::kmajor_offset(n, p0, Np)) = __float2bfloat16_rn(v);
    }
}

sfw_status launch_tc_table(const float2* full, long long spec_elems, int K, int P0, long long nl, int Np,
                           int Kp, __nv_bfloat16* Tb, cudaStream_t st) {
    SFW_LAUNCH(st, "k_tc_table", k_tc_table<<<2048, 256, 0, st>>>(full, spec_elems, K, P0, nl, Np, Kp, Tb));
    return launch_check("k_tc_table");
}

// A for every half h of the output rows: rows 2j, 2j+1 (i0 = 64 h + j) of the real form of
// W[i0, p0] = e^{2 pi i i0 p0 / P0} over K = 2 Kp columns, in the MMA layout:
//     row 2j   (Re U[i0]):  [ cos | -sin ],   row 2j+1 (Im U[i0]):  [ sin | cos ]
// (zero for i0 >= n0 or p0 >= P0), 128-byte swizzled; the argument i0 p0 is reduced mod P0
// exactly.
__global__ void k_tc_dft(int n0, int P0, int Kp, int halves, __nv_bfloat16* __restrict__ A) {
    const int K2 = 2 * Kp;
    const long long per = 128LL * K2;
    const long long total = per * halves;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(i / per);
        const int e = (int)(i - (long long)h * per);
        const int m = e / K2, k = e - m * K2;
        const int i0 = 64 * h + (m >> 1), im = m & 1;
        const int p0 = k < Kp ? k : k - Kp;
        float val = 0.f;
        if (i0 < n0 && p0 < P0) {
            const long long r = ((long long)i0 * p0) % P0;
            double sn, cs;
            sincospi(2.0 * (double)r / (double)P0, &sn, &cs);
            val = (float)(k < Kp ? (im ? sn : cs) : (im ? cs : -sn));
        }
        unsigned char* blk = reinterpret_cast<unsigned char*>(A + (long long)h * per);
        *reinterpret_cast<__nv_bfloat16*>(blk + tc::sw128_offset(m, k, 128)) = __float2bfloat16_rn(val);
    }
}

sfw_status launch_tc_dft(int n0, int P0, int Kp, __nv_bfloat16* A, cudaStream_t st) {
    const int halves = (n0 + 63) / 64;
    SFW_LAUNCH(st, "k_tc_dft", k_tc_dft<<<256, 256, 0, st>>>(n0, P0, Kp, halves, A));
    return launch_check("k_tc_dft");
}

// ------------------------------------------------------------------ the axis-0 GEMM pass

// Dynamic shared memory of the pass (byte offsets from a 1024-aligned base; every region a
// multiple of 1024 bytes, as the 128-byte swizzle wants).
struct TcSmem {
    uint32_t a, b[2], t[3], xs[2], total;
};

__host__ __device__ inline TcSmem tc_smem_layout(int Kp, int Np, int LG) {
    TcSmem s;
    const uint32_t K2 = 2u * (uint32_t)Kp;
    const uint32_t abytes = 128u * K2 * 2u, bbytes = (uint32_t)Np * K2 * 2u;
    const uint32_t tbytes = (uint32_t)Np * (uint32_t)Kp * 2u, xbytes = (uint32_t)Kp * (uint32_t)LG * 8u;
    s.a = 0;
    s.b[0] = abytes;
    s.b[1] = abytes + bbytes;
    for (int i = 0; i < 3; ++i) s.t[i] = abytes + 2 * bbytes + (uint32_t)i * tbytes;
    s.xs[0] = abytes + 2 * bbytes + 3 * tbytes;
    s.xs[1] = s.xs[0] + xbytes;
    s.total = s.xs[1] + xbytes + 1024u;   // + alignment slack of the base
    return s;
}

constexpr int kTcWorkers = 128;                 // warps 0-3: B' and the epilogue (one TMEM lane quadrant each)
constexpr int kTcThreadsWs = kTcWorkers + 32;   // + warp 4: table copies and the MMAs

__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

// One CTA per (half of the output rows, share of the line groups).  A = the real form of W's
// 64 rows of the half (prepared at plan creation, one bulk copy):
//     row 2j   (Re U[i0]):  [ Re W[i0, :] | -Im W[i0, :] ]
//     row 2j+1 (Im U[i0]):  [ Im W[i0, :] |  Re W[i0, :] ]      (K = 2 Kp)
// and per line B' = [ T_l (.) Re X_l | T_l (.) Im X_l ] (Np kernels x 2 Kp).  D = A B'^T =
// [Re U_k; Im U_k] for the line in tensor memory, LG lines side by side per buffer.
// Warp roles: warps 0-3 build B' from the table block (three bulk-copy stages, refilled as
// soon as a line's B' is built) and the staged X lines (copied one line group ahead), and
// write each line group's results; one lane of warp 4 issues the table copies and the MMAs.
// Hand-offs go through mbarriers: b_full (B' built, 4 warp arrivals), done (MMAs of a line
// finished, tcgen05.commit), t_full (table block landed), acc_full / acc_empty (a group's
// results ready / read).  Every wait is bounded; a wait that runs out sets p.err.
template <int LG>
__global__ void __launch_bounds__(kTcThreadsWs, 1) k_axis0_tc(Axis0TcPass p) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int Kp = p.Kp, Np = p.Np, P0 = p.P0, K2 = 2 * p.Kp;
    const TcSmem L = tc_smem_layout(Kp, Np, LG);
    __shared__ __align__(8) unsigned long long s_tfull[3], s_bfull[2], s_done[2], s_accf[2], s_acce[2], s_abar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tbytes = (uint32_t)Np * (uint32_t)Kp * 2u;
    const uint32_t idesc = tc::idesc_bf16_f32(128, Np);
    const int halves = (p.n0 + 63) / 64;
    const int h = blockIdx.x % halves;
    const long long G = gridDim.x / halves;          // CTAs per half (the grid is a multiple)
    const long long gi = blockIdx.x / halves;
    const long long ngroups = (p.nl + LG - 1) / LG;
    const long long my_groups = gi < ngroups ? (ngroups - 1 - gi) / G + 1 : 0;
    const long long my_lines = my_groups * LG;
    auto line_of = [&](long long t) -> long long { return (gi + (t / LG) * G) * LG + (t % LG); };
    auto tbar = [&](long long t) { return tc::smem_addr(&s_tfull[t % 3]); };

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(tc::smem_addr(&s_tfull[i]), 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(tc::smem_addr(&s_bfull[i]), 4);
            tc::mbar_init(tc::smem_addr(&s_done[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_accf[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_acce[i]), 4);
        }
        tc::mbar_init(tc::smem_addr(&s_abar), 1);
        tc::mbar_init_fence();
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, kTcCols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;

    if (warp == 4) {
        // ---------------- producer / MMA lane
        if (lane == 0) {
            auto issue_table = [&](long long t) {
                const long long l = min(line_of(t), p.nl - 1);   // padding lines reuse a real block
                tc::mbar_expect_tx(tbar(t), tbytes);
                tc::bulk_g2s(tc::smem_addr(base + L.t[t % 3]), p.Tb + (size_t)l * (size_t)Np * (size_t)Kp, tbytes,
                             tbar(t));
            };
            const uint32_t abytes = 128u * (uint32_t)K2 * 2u;
            tc::mbar_expect_tx(tc::smem_addr(&s_abar), abytes);
            tc::bulk_g2s(tc::smem_addr(base + L.a), p.A + (size_t)h * 128u * (size_t)K2, abytes,
                         tc::smem_addr(&s_abar));
            for (long long t = 0; t < 3 && t < my_lines; ++t) issue_table(t);
            if (!tc::mbar_wait(tc::smem_addr(&s_abar), 0)) s_abort = 1;
            const uint32_t a0 = tc::smem_addr(base + L.a);
            for (long long t = 0; t < my_lines && !s_abort; ++t) {
                const long long u = t / LG;
                const int j = (int)(t % LG), s = (int)(t & 1), b = (int)(u & 1);
                if (j == 0 && u >= 2 && !tc::mbar_wait(tc::smem_addr(&s_acce[b]), (uint32_t)((u - 2) >> 1) & 1u)) {
                    s_abort = 1;
                    break;
                }
                if (!tc::mbar_wait(tc::smem_addr(&s_bfull[s]), (uint32_t)(t >> 1) & 1u)) {
                    s_abort = 1;
                    break;
                }
                // the workers have read the table block of line t: refill its stage
                if (t + 3 < my_lines) issue_table(t + 3);
                tc::fence_after_sync();
                const uint32_t b0 = tc::smem_addr(base + L.b[s]);
                const uint32_t d = tmem + (uint32_t)(b * 128 + j * Np);
                for (int ks = 0; ks < K2 / 16; ++ks)
                    tc::mma_bf16(d, tc::desc_kmajor_sw128(a0 + tc::sw128_slice(ks, 128)),
                                 tc::desc_kmajor_sw128(b0 + tc::sw128_slice(ks, Np)), idesc, ks > 0 ? 1u : 0u);
                tc::mma_commit(tc::smem_addr(&s_done[s]));
                if (j == LG - 1) tc::mma_commit(tc::smem_addr(&s_accf[b]));
            }
        }
        __syncwarp();
    } else {
        // ---------------- workers: B' of every line, then each group's results
        auto stage_x = [&](long long u) {   // X lines of group u, per line contiguous (zero past the end)
            float2* xs = reinterpret_cast<float2*>(base + L.xs[u & 1]);
            const long long l0 = (gi + u * G) * LG;
            for (int e = tid; e < Kp * LG; e += kTcWorkers) {
                const int jl = e % LG, p0 = e / LG;
                float2* dst = xs + jl * Kp + p0;
                if (p0 < P0 && l0 + jl < p.nl) tc::cp_async8(dst, p.X + (long long)p0 * p.nl + l0 + jl);
                else *dst = make_float2(0.f, 0.f);
            }
            tc::cp_async_commit();
        };
        if (my_groups > 0) stage_x(0);
        const int m = tid, i0 = h * 64 + (m >> 1), im = m & 1;
        const bool live = i0 < p.n0;
        constexpr int HALF = LG >= 2 ? LG / 2 : 1;
        const int jw = (LG >= 2 && im) ? HALF : 0;
        const bool writer = live && (LG >= 2 || !im);
        float2* dst0 = p.out + (long long)i0 * p.lout.Sj;
        for (long long u = 0; u < my_groups && !s_abort; ++u) {
            const long long l0 = (gi + u * G) * LG;
            const int nlg = (int)min((long long)LG, p.nl - l0);
            const int b = (int)(u & 1);
            tc::cp_async_wait_all();
            workers_sync();
            if (u + 1 < my_groups) stage_x(u + 1);
            const float2* xs = reinterpret_cast<const float2*>(base + L.xs[u & 1]);
            for (int j = 0; j < LG; ++j) {
                const long long t = u * LG + j;
                const int s = (int)(t & 1);
                // B'[s] is free once the MMAs of line t - 2 are done; the table block of line t landed
                if (t >= 2 && !tc::mbar_wait(tc::smem_addr(&s_done[s]), (uint32_t)((t - 2) >> 1) & 1u)) s_abort = 1;
                if (!tc::mbar_wait(tbar(t), (uint32_t)(t / 3) & 1u)) s_abort = 1;
                if (s_abort) break;
                const unsigned char* Ts = base + L.t[t % 3];
                unsigned char* Bs = base + L.b[s];
                const float2* x = xs + j * Kp;
                for (int e = tid; e < Np * (Kp / 8); e += kTcWorkers) {
                    const int n = e % Np, c = e / Np;
                    const uint4 tv = *reinterpret_cast<const uint4*>(Ts + tc::kmajor_offset(n, 8 * c, Np));
                    const uint32_t tw[4] = {tv.x, tv.y, tv.z, tv.w};
                    const float4* x4 = reinterpret_cast<const float4*>(x + 8 * c);
                    uint32_t re[4], imv[4];
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2) {
                        const float t0 = __uint_as_float(tw[q2] << 16), t1 = __uint_as_float(tw[q2] & 0xFFFF0000u);
                        const float4 xx = x4[q2];   // (Re, Im) of points 2 q2 and 2 q2 + 1
                        re[q2] = tc::pack_bf16x2(t0 * xx.x, t1 * xx.z);
                        imv[q2] = tc::pack_bf16x2(t0 * xx.y, t1 * xx.w);
                    }
                    *reinterpret_cast<uint4*>(Bs + tc::sw128_offset(n, 8 * c, Np)) = make_uint4(re[0], re[1], re[2], re[3]);
                    *reinterpret_cast<uint4*>(Bs + tc::sw128_offset(n, 8 * c + Kp, Np)) =
                        make_uint4(imv[0], imv[1], imv[2], imv[3]);
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_addr(&s_bfull[s]));
            }
            if (s_abort) break;
            // the group's results
            if (!tc::mbar_wait(tc::smem_addr(&s_accf[b]), (uint32_t)(u >> 1) & 1u)) {
                s_abort = 1;
                break;
            }
            tc::fence_after_sync();
            long long off_line[HALF];
#pragma unroll
            for (int q2 = 0; q2 < HALF; ++q2) off_line[q2] = line_offset(p.lout, min(l0 + jw + q2, p.nl - 1));
            const uint32_t row_base = tmem + (uint32_t)(b * 128) + ((uint32_t)(warp * 32) << 16);
            for (int cb = 0; cb < Np; cb += 16) {
                float v[LG][16];
#pragma unroll
                for (int jj = 0; jj < LG; ++jj) tc::tmem_ld16(row_base + (uint32_t)(jj * Np + cb), v[jj]);
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    const int k = cb + kk;
                    float mine[HALF], other[HALF];
#pragma unroll
                    for (int q2 = 0; q2 < HALF; ++q2) {
                        // even sends its values of lines HALF + q2, odd its values of lines q2
                        const float send = (LG >= 2) ? (im ? v[q2][kk] : v[HALF + q2][kk]) : v[0][kk];
                        other[q2] = __shfl_xor_sync(0xffffffffu, send, 1);
                        mine[q2] = (LG >= 2) ? (im ? v[HALF + q2][kk] : v[q2][kk]) : v[0][kk];
                    }
                    if (k >= p.K || !writer) continue;
                    float2* dst = dst0 + (long long)k * p.out_stride;
#pragma unroll
                    for (int q2 = 0; q2 < HALF; ++q2) {
                        if (jw + q2 < nlg) {
                            const float2 z = im ? make_float2(other[q2], mine[q2]) : make_float2(mine[q2], other[q2]);
                            dst[off_line[q2]] = z;
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_addr(&s_acce[b]));
        }
        tc::cp_async_wait_all();
    }
    __syncthreads();
    if (s_abort) {
        // a bounded wait ran out: report it and give the copies and MMAs in flight time to
        // finish (bounded) before the tensor memory is released
        if (tid == 0) {
            atomicExch(p.err, 1);
            for (int i = 0; i < 3; ++i) tc::mbar_wait(tc::smem_addr(&s_tfull[i]), 0, 1 << 16);
            for (int i = 0; i < 2; ++i) tc::mbar_wait(tc::smem_addr(&s_done[i]), 0, 1 << 16);
            tc::mbar_wait(tc::smem_addr(&s_abar), 0, 1 << 16);
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

// Lines accumulated side by side in one tensor-memory buffer (LG * Np <= 128 columns).
int tc_lines_per_group(int Np) { return Np <= 16 ? 8 : Np <= 32 ? 4 : Np <= 64 ? 2 : 1; }

size_t tc_smem_bytes(int Kp, int Np, int P0) {
    (void)P0;
    return tc_smem_layout(Kp, Np, tc_lines_per_group(Np)).total;
}

template <int LG>
static sfw_status run_axis0_tc(const Axis0TcPass& p, int num_sms, cudaStream_t st) {
    const size_t smem = tc_smem_layout(p.Kp, p.Np, LG).total;
    static int configured = 0;   // largest dynamic shared memory set so far
    if ((int)smem > configured) {
        SFW_CUDA(cudaFuncSetAttribute(k_axis0_tc<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = (int)smem;
    }
    // CTAs per half: the SMs shared evenly, at most one per line group
    const int halves = (p.n0 + 63) / 64;
    const long long ngroups = (p.nl + LG - 1) / LG;
    long long per = num_sms / halves;
    if (per < 1) per = 1;
    if (per > ngroups) per = ngroups;
    const int grid = (int)(per * halves);
    SFW_LAUNCH(st, "k_axis0_tc", k_axis0_tc<LG><<<grid, kTcThreadsWs, smem, st>>>(p));
    return launch_check("k_axis0_tc");
}

sfw_status launch_axis0_tc(const Axis0TcPass& p, int num_sms, cudaStream_t st) {
    if (p.Np < 16 || p.Np > 128 || p.Np % 16 || p.Kp % 32 || p.Kp < p.P0 || p.n0 < 1)
        return fail(SFW_ERR_SHAPE, "axis-0 tensor-core pass: Np=%d Kp=%d P0=%d", p.Np, p.Kp, p.P0);
    if (tc_smem_bytes(p.Kp, p.Np, p.P0) > 227u * 1024u)
        return fail(SFW_ERR_SHAPE, "axis-0 tensor-core pass: shared memory for P0=%d", p.P0);
    switch (tc_lines_per_group(p.Np)) {
        case 8: return run_axis0_tc<8>(p, num_sms, st);
        case 4: return run_axis0_tc<4>(p, num_sms, st);
        case 2: return run_axis0_tc<2>(p, num_sms, st);
        default: return run_axis0_tc<1>(p, num_sms, st);
    }
}

// ------------------------------------------------------------------ a single-tile check

// D (128 x N, row-major FP32) = A (128 x K) . B^T (N x K), operands given in the MMA layout.
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm_check(const unsigned char* __restrict__ Ag, const unsigned char* __restrict__ Bg, int K, int N,
                int swz, float* __restrict__ D, int* err) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long s_done;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t abytes = 128u * (uint32_t)K * 2u, bbytes = (uint32_t)N * (uint32_t)K * 2u;
    for (uint32_t e = tid * 16u; e < abytes; e += kTcThreads * 16u)
        *reinterpret_cast<uint4*>(base + e) = *reinterpret_cast<const uint4*>(Ag + e);
    for (uint32_t e = tid * 16u; e < bbytes; e += kTcThreads * 16u)
        *reinterpret_cast<uint4*>(base + abytes + e) = *reinterpret_cast<const uint4*>(Bg + e);
    const uint32_t bar = tc::smem_addr(&s_done);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init_fence();
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, 256);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (tid == 0) {
        const uint32_t a0 = tc::smem_addr(base), b0 = a0 + abytes;
        const uint32_t lbo_a = 128u * 16u, lbo_b = (uint32_t)N * 16u;
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = swz ? tc::desc_kmajor_sw128(a0 + tc::sw128_slice(ks, 128))
                                    : tc::desc_kmajor(a0 + ks * 2u * lbo_a, lbo_a, 128u);
            const uint64_t bd = swz ? tc::desc_kmajor_sw128(b0 + tc::sw128_slice(ks, N))
                                    : tc::desc_kmajor(b0 + ks * 2u * lbo_b, lbo_b, 128u);
            tc::mma_bf16(tmem, ad, bd, tc::idesc_bf16_f32(128, N), ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    __syncthreads();
    const bool ok = tc::mbar_wait(bar, 0);
    if (!ok && tid == 0) atomicExch(err, 1);
    __syncthreads();
    tc::fence_after_sync();
    if (ok) {
        for (int cb = 0; cb < N; cb += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
            for (int i = 0; i < 16; ++i) D[(size_t)tid * N + cb + i] = v[i];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace sfw

// Test hook (not part of the public header): one tensor-core tile on host data.  A is 128 x K
// and B is N x K, row-major bf16 bit patterns; D receives A B^T (128 x N, FP32).  K a multiple
// of 16 in [16, 256] (of 64 in [64, 384] with swizzle), N a multiple of 16 in [16, 128]; swizzle 0: the
// operands in the interleaved layout, 1: in the 128-byte swizzled layout.  Synchronous.
extern "C" sfw_status sfw_test_tc_gemm(const uint16_t* A, const uint16_t* B, int K, int N, float* D, int swizzle) {
    using namespace sfw;
    clear_error();
    if (!A || !B || !D || K < 16 || K > (swizzle ? 384 : 256) || K % 16 || N < 16 || N > 128 || N % 16 ||
        (swizzle && K % 64))
        return fail(SFW_ERR_ARG, "sfw_test_tc_gemm: bad arguments");
    std::vector<uint16_t> a_l((size_t)128 * K), b_l((size_t)N * K);
    for (int r = 0; r < 128; ++r)
        for (int k = 0; k < K; ++k)
            a_l[(swizzle ? tc::sw128_offset(r, k, 128) : tc::kmajor_offset(r, k, 128)) / 2] = A[(size_t)r * K + k];
    for (int r = 0; r < N; ++r)
        for (int k = 0; k < K; ++k)
            b_l[(swizzle ? tc::sw128_offset(r, k, N) : tc::kmajor_offset(r, k, N)) / 2] = B[(size_t)r * K + k];
    unsigned char *da = nullptr, *db = nullptr;
    float* dd = nullptr;
    int* derr = nullptr;
    sfw_status s = SFW_OK;
    do {
        if (cudaMalloc(&da, a_l.size() * 2) != cudaSuccess || cudaMalloc(&db, b_l.size() * 2) != cudaSuccess ||
            cudaMalloc(&dd, sizeof(float) * 128 * N) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess) {
            s = cuda_fail(cudaGetLastError(), "sfw_test_tc_gemm alloc");
            break;
        }
        cudaMemcpy(da, a_l.data(), a_l.size() * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(db, b_l.data(), b_l.size() * 2, cudaMemcpyHostToDevice);
        cudaMemset(derr, 0, sizeof(int));
        // operands plus room for the MMAs' reads under either order of the descriptor strides
        const int smem = 200 * 1024;
        if (cudaFuncSetAttribute(k_tc_gemm_check, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            s = cuda_fail(cudaGetLastError(), "sfw_test_tc_gemm attribute");
            break;
        }
        SFW_LAUNCH(nullptr, "k_tc_gemm_check", k_tc_gemm_check<<<1, kTcThreads, smem>>>(da, db, K, N, swizzle, dd, derr));
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            s = cuda_fail(e, "sfw_test_tc_gemm");
            break;
        }
        int herr = 0;
        cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
        if (herr) {
            s = fail(SFW_ERR_TIMEOUT, "sfw_test_tc_gemm: the MMA completion did not arrive");
            break;
        }
        cudaMemcpy(D, dd, sizeof(float) * 128 * N, cudaMemcpyDeviceToHost);
    } while (0);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dd);
    cudaFree(derr);
    return s;
}
