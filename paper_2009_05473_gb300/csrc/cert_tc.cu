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

// A tile is LT = 128 / Np lines x Np kernels = 128 columns (the N of every MMA); K runs over
// blocks of 64 points p0, each block contributing a Re and an Im 64-column slice of K.
__host__ __device__ inline int tc_tile_lines(int Np) { return 128 / Np; }

// Dynamic shared memory (byte offsets from a 1024-aligned base; every region a multiple of
// 1024 bytes, as the 128-byte swizzle wants):
//   a      A, 128 rows x 2 Kp                       (resident)
//   t[3]   the table pieces of a block: LT lines x Np kernels x 64 points (16 KB, bulk copies)
//   b[2]   B' of a block: Re and Im slices, 128 rows x 64 each (32 KB)
//   xs[2]  X of a tile: LT lines x Kp points, FP32 complex (one tile ahead)
struct TcSmem {
    uint32_t a, t[3], b[2], xs[2], total;
};

__host__ __device__ inline TcSmem tc_smem_layout(int Kp, int Np) {
    TcSmem s;
    const uint32_t abytes = 128u * 2u * (uint32_t)Kp * 2u;
    const uint32_t tbytes = 128u * 64u * 2u;
    const uint32_t bbytes = 2u * 128u * 64u * 2u;
    const uint32_t xbytes = ((uint32_t)tc_tile_lines(Np) * (uint32_t)Kp * 8u + 1023u) & ~1023u;
    s.a = 0;
    for (int i = 0; i < 3; ++i) s.t[i] = abytes + (uint32_t)i * tbytes;
    for (int i = 0; i < 2; ++i) s.b[i] = abytes + 3u * tbytes + (uint32_t)i * bbytes;
    s.xs[0] = abytes + 3u * tbytes + 2u * bbytes;
    s.xs[1] = s.xs[0] + xbytes;
    s.total = s.xs[1] + xbytes + 1024u;   // + alignment slack of the base
    return s;
}

constexpr int kTcFormWarps = 8;                   // warps 0-7: B' of every block
constexpr int kTcEpiWarps = 4;                    // warps 8-11: results (TMEM lane quadrant = warp % 4)
constexpr int kTcMmaWarp = kTcFormWarps + kTcEpiWarps;                 // warp 12: the MMAs
constexpr int kTcProdWarp = kTcMmaWarp + 1;                            // warp 13: the table copies
constexpr int kTcThreadsWs = 32 * (kTcFormWarps + kTcEpiWarps + 2);
constexpr int kTcFormThreads = 32 * kTcFormWarps;

// One CTA per (half of the output rows, share of the tiles).  A = the real form of W's 64
// rows of the half (prepared at plan creation, one bulk copy):
//     row 2j   (Re U[i0]):  [ Re W[i0, :] | -Im W[i0, :] ]
//     row 2j+1 (Im U[i0]):  [ Im W[i0, :] |  Re W[i0, :] ]      (K = 2 Kp)
// For every tile and block of 64 points, B'_re = T (.) Re X and B'_im = T (.) Im X (128
// columns = LT lines x Np kernels); D (+)= A_re-block B'_re^T + A_im-block B'_im^T, so that
// after the last block D = [Re U_k; Im U_k] for the tile's lines, in tensor memory.
// Warp roles: one lane of warp 13 bulk-copies the table pieces of every block into a ring of
// three stages (a line's piece of a 64-point block is 4 KB contiguous at Np = 32); warps 0-7
// build B' from them (two stages; X staged a tile ahead); warps 8-11 write the results of a
// tile while the next one accumulates (two tensor-memory buffers); one lane of warp 12 issues
// the MMAs.  Hand-offs go through mbarriers: t_full / t_empty (table stage landed / read, 8
// arrivals), b_full (B' built, 8 arrivals), done (MMAs of a block finished, tcgen05.commit),
// acc_full / acc_empty (a tile's results ready / read, 4 arrivals).  Every wait is bounded; a
// wait that runs out sets p.err.
template <int LT>
__global__ void __launch_bounds__(kTcThreadsWs, 1) k_axis0_tc(Axis0TcPass p) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int Kp = p.Kp, Np = p.Np, P0 = p.P0;
    const int nb = Kp / 64;
    const TcSmem L = tc_smem_layout(Kp, Np);
    __shared__ __align__(8) unsigned long long s_tfull[3], s_tempty[3], s_bfull[2], s_done[2], s_accf[2],
        s_acce[2], s_abar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t idesc = tc::idesc_bf16_f32(128, 128);
    const int halves = (p.n0 + 63) / 64;
    const int h = blockIdx.x % halves;
    const long long G = gridDim.x / halves;          // CTAs per half (the grid is a multiple)
    const long long gi = blockIdx.x / halves;
    const long long ntiles = (p.nl + LT - 1) / LT;
    const long long my_tiles = gi < ntiles ? (ntiles - 1 - gi) / G + 1 : 0;
    auto tile_l0 = [&](long long u) -> long long { return (gi + u * G) * LT; };

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) {
            tc::mbar_init(tc::smem_addr(&s_tfull[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_tempty[i]), kTcFormWarps);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(tc::smem_addr(&s_bfull[i]), kTcFormWarps);
            tc::mbar_init(tc::smem_addr(&s_done[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_accf[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_acce[i]), kTcEpiWarps);
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

    if (warp == kTcProdWarp) {
        // ---------------- table pieces of every block: LT bulk copies (one per line)
        if (lane == 0) {
            const uint32_t piece = (uint32_t)Np * 64u * 2u;
            int ts = 0;
            uint32_t tph = 0;
            bool wrapped = false;
            for (long long u = 0; u < my_tiles && !s_abort; ++u) {
                const long long l0 = tile_l0(u);
                for (int b = 0; b < nb; ++b) {
                    // the stage is free once the formation warps have read its previous block
                    if (wrapped && !tc::mbar_wait(tc::smem_addr(&s_tempty[ts]), tph ^ 1u)) {
                        s_abort = 1;
                        break;
                    }
                    const uint32_t bar = tc::smem_addr(&s_tfull[ts]);
                    tc::mbar_expect_tx(bar, piece * (uint32_t)LT);
                    for (int j = 0; j < LT; ++j) {
                        const long long l = min(l0 + j, p.nl - 1);   // padding lines copy a real block
                        const __nv_bfloat16* src = p.Tb + (size_t)l * (size_t)Np * (size_t)Kp + (size_t)b * 64u * Np;
                        tc::bulk_g2s(tc::smem_addr(base + L.t[ts] + (uint32_t)j * piece), src, piece, bar);
                    }
                    if (++ts == 3) {
                        ts = 0;
                        tph ^= 1u;
                        wrapped = true;
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == kTcMmaWarp) {
        // ---------------- MMA lane
        if (lane == 0) {
            const uint32_t abytes = 128u * 2u * (uint32_t)Kp * 2u;
            tc::mbar_expect_tx(tc::smem_addr(&s_abar), abytes);
            tc::bulk_g2s(tc::smem_addr(base + L.a), p.A + (size_t)h * 128u * 2u * (size_t)Kp, abytes,
                         tc::smem_addr(&s_abar));
            if (!tc::mbar_wait(tc::smem_addr(&s_abar), 0)) s_abort = 1;
            // This one thread's instruction latency paces the MMAs: descriptors are built once
            // and advanced by adding to their address field (16-byte units), the B' stage ring
            // (2 stages) is tracked without divisions, a block's 8 MMAs are unrolled.
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_addr(base + L.a));
            // the B' stages lie 2 x 16 KB apart (Re and Im slices)
            const uint64_t dB0 = tc::desc_kmajor_sw128(tc::smem_addr(base + L.b[0]));
            constexpr uint64_t kAtom = (16u * 1024u) >> 4, kKStep = 32u >> 4, kImOff = (128u * 64u * 2u) >> 4;
            constexpr uint64_t kStage = 2 * kImOff;
            int s = 0;
            uint32_t ph = 0;
            for (long long u = 0; u < my_tiles && !s_abort; ++u) {
                const int ub = (int)(u & 1);
                // the tile's accumulator is free once the epilogue has read tile u - 2
                if (u >= 2 && !tc::mbar_wait(tc::smem_addr(&s_acce[ub]), (uint32_t)((u - 2) >> 1) & 1u)) {
                    s_abort = 1;
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(ub * 128);
                for (int b = 0; b < nb; ++b) {
                    if (!tc::mbar_wait(tc::smem_addr(&s_bfull[s]), ph)) {
                        s_abort = 1;
                        break;
                    }
                    tc::fence_after_sync();
                    // A's 64-column atoms: Re block b at column atom b, Im block b at atom nb + b
                    const uint64_t are = dA0 + (uint64_t)b * kAtom, aim = dA0 + (uint64_t)(nb + b) * kAtom;
                    const uint64_t bre = dB0 + (uint64_t)s * kStage, bim = bre + kImOff;
                    tc::mma_bf16(d, are, bre, idesc, b > 0 ? 1u : 0u);
                    tc::mma_bf16(d, are + kKStep, bre + kKStep, idesc, 1u);
                    tc::mma_bf16(d, are + 2 * kKStep, bre + 2 * kKStep, idesc, 1u);
                    tc::mma_bf16(d, are + 3 * kKStep, bre + 3 * kKStep, idesc, 1u);
                    tc::mma_bf16(d, aim, bim, idesc, 1u);
                    tc::mma_bf16(d, aim + kKStep, bim + kKStep, idesc, 1u);
                    tc::mma_bf16(d, aim + 2 * kKStep, bim + 2 * kKStep, idesc, 1u);
                    tc::mma_bf16(d, aim + 3 * kKStep, bim + 3 * kKStep, idesc, 1u);
                    tc::mma_commit(tc::smem_addr(&s_done[s]));
                    if (++s == 2) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (s_abort) break;
                tc::mma_commit(tc::smem_addr(&s_accf[ub]));
            }
        }
        __syncwarp();
    } else if (warp < kTcFormWarps) {
        // ---------------- B' of every block: column c' = j Np + n (line j of the tile, kernel n)
        auto stage_x = [&](long long u) {   // X lines of tile u, per line contiguous (zero past the end)
            float2* xs = reinterpret_cast<float2*>(base + L.xs[u & 1]);
            const long long l0 = tile_l0(u);
            for (int e = tid; e < Kp * LT; e += kTcFormThreads) {
                const int jl = e % LT, p0 = e / LT;
                float2* dst = xs + jl * Kp + p0;
                if (p0 < P0 && l0 + jl < p.nl) tc::cp_async8(dst, p.X + (long long)p0 * p.nl + l0 + jl);
                else *dst = make_float2(0.f, 0.f);
            }
            tc::cp_async_commit();
        };
        if (my_tiles > 0) stage_x(0);
        constexpr int PER = 128 * 8 / kTcFormThreads;     // items (16-byte chunks) per thread and block
        const uint32_t piece = (uint32_t)Np * 64u * 2u;
        const int lnp = __ffs(Np) - 1;                    // Np is a power of two
        int s = 0, ts = 0;  // B' stage (ring of 2) and table stage (ring of 3) of the next block
        uint32_t uses = 0, tph = 0;
        for (long long u = 0; u < my_tiles; ++u) {
            tc::cp_async_wait_all();
            // all formation threads stop together (a barrier with a missing thread never ends)
            if (tc::bar_sync_or<1, kTcFormThreads>(s_abort != 0)) break;
            if (u + 1 < my_tiles) stage_x(u + 1);
            const float2* xs = reinterpret_cast<const float2*>(base + L.xs[u & 1]);
            for (int b = 0; b < nb; ++b) {
                // the block's table pieces have landed; B'[s] is free once the MMAs of its
                // previous use (block q - 2) are done
                if (!tc::mbar_wait(tc::smem_addr(&s_tfull[ts]), tph)) s_abort = 1;
                if (uses > 0 && !tc::mbar_wait(tc::smem_addr(&s_done[s]), (uses - 1u) & 1u)) s_abort = 1;
                if (s_abort) break;
                const unsigned char* Ts = base + L.t[ts];
                unsigned char* Bre = base + L.b[s];
                unsigned char* Bim = Bre + 128u * 64u * 2u;
#pragma unroll
                for (int r = 0; r < PER; ++r) {
                    const int e = tid + r * kTcFormThreads;
                    const int col = e & 127, c = e >> 7;          // column of B', 8-point chunk of the block
                    const int j = col >> lnp, n = col - (j << lnp);
                    const uint4 tvr = *reinterpret_cast<const uint4*>(Ts + (uint32_t)j * piece +
                                                                      tc::kmajor_offset(n, 8 * c, Np));
                    const uint32_t tw[4] = {tvr.x, tvr.y, tvr.z, tvr.w};
                    const float4* x4 = reinterpret_cast<const float4*>(xs + j * Kp + 64 * b + 8 * c);
                    uint32_t re[4], imv[4];
#pragma unroll
                    for (int q2 = 0; q2 < 4; ++q2) {
                        const float t0 = __uint_as_float(tw[q2] << 16), t1 = __uint_as_float(tw[q2] & 0xFFFF0000u);
                        const float4 xx = x4[q2];   // (Re, Im) of points 2 q2 and 2 q2 + 1
                        re[q2] = tc::pack_bf16x2(t0 * xx.x, t1 * xx.z);
                        imv[q2] = tc::pack_bf16x2(t0 * xx.y, t1 * xx.w);
                    }
                    const uint32_t off = tc::sw128_offset(col, 8 * c, 128);
                    *reinterpret_cast<uint4*>(Bre + off) = make_uint4(re[0], re[1], re[2], re[3]);
                    *reinterpret_cast<uint4*>(Bim + off) = make_uint4(imv[0], imv[1], imv[2], imv[3]);
                }
                tc::fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(tc::smem_addr(&s_bfull[s]));
                    tc::mbar_arrive(tc::smem_addr(&s_tempty[ts]));
                }
                if (++s == 2) {
                    s = 0;
                    ++uses;
                }
                if (++ts == 3) {
                    ts = 0;
                    tph ^= 1u;
                }
            }
        }
        tc::cp_async_wait_all();
    } else {
        // ---------------- results: thread = TMEM lane = output row (i0, Re or Im)
        const int m = tid - kTcFormThreads;               // 0..127, lane quadrant = warp % 4
        const int i0 = h * 64 + (m >> 1), im = m & 1;
        const bool writer = i0 < p.n0 && (LT >= 2 || !im);
        float2* dst0 = p.out + (long long)i0 * p.lout.Sj;
        // lines per step: 4 (the even row writes the first two, the odd row the last two, as
        // one 16-byte store each), 2 (one line each) or 1 (the even row only)
        constexpr int STEP = LT >= 4 ? 4 : LT;
        constexpr int MINE = STEP >= 2 ? STEP / 2 : 1;
        for (long long u = 0; u < my_tiles && !s_abort; ++u) {
            const int ub = (int)(u & 1);
            if (!tc::mbar_wait(tc::smem_addr(&s_accf[ub]), (uint32_t)(u >> 1) & 1u)) {
                s_abort = 1;
                break;
            }
            tc::fence_after_sync();
            const long long l0 = tile_l0(u);
            const int nlt = (int)min((long long)LT, p.nl - l0);
            const uint32_t row_base = tmem + (uint32_t)(ub * 128) + ((uint32_t)((warp & 3) * 32) << 16);
            for (int j0 = 0; j0 < LT; j0 += STEP) {
                const int jm = j0 + ((STEP >= 2 && im) ? MINE : 0);   // first line this thread writes
                const long long off = line_offset(p.lout, min(l0 + jm, p.nl - 1));
                for (int cb = 0; cb < Np; cb += 16) {
                    float v[STEP][16];
#pragma unroll
                    for (int jj = 0; jj < STEP; ++jj) tc::tmem_ld16_nowait(row_base + (uint32_t)((j0 + jj) * Np + cb), v[jj]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) {
                        float mine[MINE], other[MINE];
#pragma unroll
                        for (int q2 = 0; q2 < MINE; ++q2) {
                            // even sends its values of lines MINE + q2, odd its values of lines q2
                            const float send = STEP >= 2 ? (im ? v[q2][kk] : v[MINE + q2][kk]) : v[0][kk];
                            other[q2] = __shfl_xor_sync(0xffffffffu, send, 1);
                            mine[q2] = STEP >= 2 ? (im ? v[MINE + q2][kk] : v[q2][kk]) : v[0][kk];
                        }
                        const int k = cb + kk;
                        if (k >= p.K || !writer) continue;
                        float2* dst = dst0 + (long long)k * p.out_stride + off;
                        const float2 z0 = im ? make_float2(other[0], mine[0]) : make_float2(mine[0], other[0]);
                        if constexpr (MINE == 2) {
                            const float2 z1 = im ? make_float2(other[1], mine[1]) : make_float2(mine[1], other[1]);
                            if (jm + 1 < nlt) *reinterpret_cast<float4*>(dst) = make_float4(z0.x, z0.y, z1.x, z1.y);
                            else if (jm < nlt) *dst = z0;
                        } else {
                            if (jm < nlt) *dst = z0;
                        }
                    }
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::smem_addr(&s_acce[ub]));
        }
    }
    __syncthreads();
    if (s_abort) {
        // a bounded wait ran out: report it and give the copies and MMAs in flight time to
        // finish (bounded) before the tensor memory is released
        if (tid == 0) {
            atomicExch(p.err, 1);
            for (int i = 0; i < 2; ++i) tc::mbar_wait(tc::smem_addr(&s_done[i]), 0, 1 << 16);
            for (int i = 0; i < 3; ++i) tc::mbar_wait(tc::smem_addr(&s_tfull[i]), 0, 1 << 16);
            tc::mbar_wait(tc::smem_addr(&s_abar), 0, 1 << 16);
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

size_t tc_smem_bytes(int Kp, int Np, int P0) {
    (void)P0;
    return tc_smem_layout(Kp, Np).total;
}

template <int LT>
static sfw_status run_axis0_tc(const Axis0TcPass& p, int num_sms, cudaStream_t st) {
    const size_t smem = tc_smem_layout(p.Kp, p.Np).total;
    static int configured = 0;   // largest dynamic shared memory set so far
    if ((int)smem > configured) {
        SFW_CUDA(cudaFuncSetAttribute(k_axis0_tc<LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = (int)smem;
    }
    // CTAs per half: the SMs shared evenly, at most one per tile
    const int halves = (p.n0 + 63) / 64;
    const long long ntiles = (p.nl + LT - 1) / LT;
    long long per = num_sms / halves;
    if (per < 1) per = 1;
    if (per > ntiles) per = ntiles;
    const int grid = (int)(per * halves);
    SFW_LAUNCH(st, "k_axis0_tc", k_axis0_tc<LT><<<grid, kTcThreadsWs, smem, st>>>(p));
    return launch_check("k_axis0_tc");
}

sfw_status launch_axis0_tc(const Axis0TcPass& p, int num_sms, cudaStream_t st) {
    if ((p.Np != 16 && p.Np != 32 && p.Np != 64 && p.Np != 128) || p.K > p.Np || p.Kp % 64 || p.Kp < p.P0 ||
        p.n0 < 1)
        return fail(SFW_ERR_SHAPE, "axis-0 tensor-core pass: Np=%d K=%d Kp=%d P0=%d", p.Np, p.K, p.Kp, p.P0);
    // results go out as 16-byte pairs of consecutive lines: even offsets, consecutive lines adjacent
    if (p.lout.Sb != 1 || p.lout.Sa % 2 || p.lout.Sj % 2 || p.lout.B % 2 || p.out_stride % 2)
        return fail(SFW_ERR_SHAPE, "axis-0 tensor-core pass: output layout");
    if (tc_smem_bytes(p.Kp, p.Np, p.P0) > 227u * 1024u)
        return fail(SFW_ERR_SHAPE, "axis-0 tensor-core pass: shared memory for P0=%d", p.P0);
    switch (tc_tile_lines(p.Np)) {
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
