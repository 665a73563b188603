// The certificate's last stage on the tensor cores (bf16 operands, FP32 accumulation in
// tensor memory): the real inverse along axis 2 with the maximum over the kernels.
//
// After the axes 0 and 1 every line L = (i0, i1) of kernel k holds the half spectrum
// V_k[L, h2], h2 < H2 = P2 / 2 + 1, of a real line, and Eq. 5's certificate is
//     eta_k(i0, i1, i2) = (1 / lambda) sum_h2 c_h2 (Re V cos(2 pi h2 i2 / P2) - Im V sin(...))
// (c_h2 = 1 at h2 = 0 and P2 / 2, else 2; the 1 / |P| of the inverse is in the table).  The
// sine vanishes at h2 = 0 and h2 = P2 / 2, so a line needs P2 real numbers: column 0 = Re V[0],
// column 1 = Re V[P2 / 2] (even P2), columns (2 h2, 2 h2 + 1) = (Re, Im) V[h2] otherwise.  Over
// 128 lines and all n2 outputs this is one GEMM per kernel,
//     D (128 lines x n2) = A (lines x Kc) . C^T (n2 x Kc),   Kc = P2 (+ 1 if odd) rounded to 16,
// with C fixed per plan (built once, resident in shared memory) and A converted from the FP32
// spectra.  A CTA takes a tile of 128 lines and a group of kernels; its epilogue warps keep
// each output's running maximum and its kernel in registers, then fold them into the
// per-voxel and grid-maximum candidate keys (value, then lowest flat index k V + lin(m)).
#include <math.h>

#include "sfw_internal.cuh"
#include "tc_sm100.cuh"

namespace sfw {

constexpr int kC2rRows = 128;      // lines per tile (M)
constexpr int kC2rN = 128;         // outputs per line (N), n2 <= 128
constexpr int kC2rSub = 32;        // lines per staged quarter of a tile
constexpr int kC2rFormWarps = 4;   // warps 0-3: A of every step; thread 0 also issues copies and MMAs
constexpr int kC2rEpiWarps = 16;   // warps 4-19: four per tensor-memory lane quadrant
constexpr int kC2rCols = kC2rN / (kC2rEpiWarps / 4);              // columns (outputs) per epilogue thread
constexpr int kC2rThreads = 32 * (kC2rFormWarps + kC2rEpiWarps);
constexpr int kC2rFormThreads = 32 * kC2rFormWarps;

// Column c of a line's A row: the bin h2 and the part (0 = Re, 1 = Im) it holds, or -1.
__host__ __device__ inline int c2r_col_bin(int c, int P2, int H2, int* part) {
    *part = 0;
    if (c == 0) return 0;
    if (c == 1) return (P2 & 1) ? -1 : P2 / 2;
    const int h2 = c >> 1;
    *part = c & 1;
    return (h2 < H2 && 2 * h2 != P2) ? h2 : -1;
}

// C for the real inverse of length P2 keeping outputs i2 < n2: row i2, column of (h2, part) =
// c_h2 (cos, -sin)(2 pi h2 i2 / P2), zero elsewhere; 128-byte swizzled, 128 rows.
__global__ void k_tc_c2r_matrix(int P2, int H2, int n2, int Kc, __nv_bfloat16* __restrict__ C) {
    const int total = kC2rN * Kc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int i2 = i / Kc, c = i - i2 * Kc;
        int part;
        const int h2 = c2r_col_bin(c, P2, H2, &part);
        float v = 0.f;
        if (i2 < n2 && h2 >= 0) {
            const long long r = ((long long)h2 * i2) % P2;
            double sn, cs;
            sincospi(2.0 * (double)r / (double)P2, &sn, &cs);
            const double w = (h2 == 0 || 2 * h2 == P2) ? 1.0 : 2.0;
            v = (float)(part ? -w * sn : w * cs);
        }
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(C) + tc::sw128_offset(i2, c, kC2rN)) =
            __float2bfloat16_rn(v);
    }
}

sfw_status launch_tc_c2r_matrix(int P2, int H2, int n2, int Kc, __nv_bfloat16* C, cudaStream_t st) {
    SFW_LAUNCH(st, "k_tc_c2r_matrix", k_tc_c2r_matrix<<<64, 256, 0, st>>>(P2, H2, n2, Kc, C));
    return launch_check("k_tc_c2r_matrix");
}

// Dynamic shared memory: C (128 rows x Kca), two A stages (128 rows x Kca), two staging
// buffers for the FP32 spectra of a quarter tile (32 lines); Kca = Kc rounded up to whole
// 64-column atoms.  Since H2 <= Kc / 2 + 1, a quarter holds at most 32 (Kc / 2 + 1) complex
// values (+ one of misalignment and one of rounding), 16-byte rounded.
__host__ __device__ inline uint32_t c2r_region(int Kc) { return (uint32_t)kC2rRows * (uint32_t)((Kc + 63) / 64 * 64) * 2u; }
__host__ __device__ inline uint32_t c2r_stage(int Kc) {
    return ((uint32_t)kC2rSub * (uint32_t)(Kc / 2 + 1) * 8u + 16u + 1023u) & ~1023u;
}
size_t tc_c2r_smem_bytes(int Kc) { return 3u * c2r_region(Kc) + 2u * c2r_stage(Kc) + 1024u; }

__device__ __forceinline__ void c2r_form_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

// Where quarter q of step (item it, kernel k) lies: the complex values f0 .. f0 + nf of the
// spectra; the bulk copy takes the 16-byte units [s, e) that hold them (lead = values before f0
// in the copy).  e may pass the end of the spectra by 8 bytes: their buffer has that slack.
struct C2rQuarter {
    long long f0;
    int rows, nf, lead, row0;
    uint32_t bytes;
};

__device__ __forceinline__ C2rQuarter c2r_quarter(const C2rTcPass& p, long long it, int ngroups, int k, int q) {
    C2rQuarter h;
    const int L0 = (int)(it / ngroups) * kC2rRows + kC2rSub * q;
    const int rows = max(0, min(kC2rSub, p.nlines - L0));
    h.row0 = kC2rSub * q;
    h.rows = rows;
    h.f0 = (long long)k * p.spec_stride + (long long)L0 * p.H2;
    h.nf = rows * p.H2;
    const unsigned long long a0 = (unsigned long long)h.f0 * 8ull, a1 = a0 + (unsigned long long)h.nf * 8ull;
    const unsigned long long s0 = a0 & ~15ull, e0 = (a1 + 15ull) & ~15ull;
    h.lead = (int)((a0 - s0) >> 3);
    h.bytes = h.nf > 0 ? (uint32_t)(e0 - s0) : 0u;
    return h;
}

// One CTA per (tile of 128 lines, group of kernels), persistent over such items; a step is one
// (item, kernel).  Warps 0-3 turn the spectra of a step (bulk-copied in quarters of 32 lines,
// two staging buffers) into A (two stages); their thread 0 issues the copies and, once A is
// built, the 128 x 128 MMAs over Kc (two tensor-memory buffers).  Warps 4-19 fold each kernel's
// D into the running maxima and, after the group's last kernel, into the candidate keys.
// mbarriers: v_full (a quarter's spectra landed), done (MMAs of a step finished), acc_empty
// (D read, 16 arrivals).  Every wait is bounded; a wait that runs out sets p.err.
__global__ void __launch_bounds__(kC2rThreads, 1) k_c2r_tc(C2rTcPass p) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t region = c2r_region(p.Kc), stage = c2r_stage(p.Kc);
    unsigned char* Cs = base;   // C, resident
    // A stage i at base + (1 + i) region, staging buffer i at base + 3 region + i stage
    auto A_stage = [&](int i) { return base + (uint32_t)(1 + i) * region; };
    auto V_stage = [&](int i) { return base + 3u * region + (uint32_t)i * stage; };
    __shared__ __align__(8) unsigned long long s_vfull[2], s_done[2], s_acce[2], s_cbar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (p.nlines + kC2rRows - 1) / kC2rRows;
    const int ngroups = (p.K + p.kgroup - 1) / p.kgroup;
    const long long items = (long long)ntiles * ngroups;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(tc::smem_addr(&s_vfull[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_done[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_acce[i]), kC2rEpiWarps);
        }
        tc::mbar_init(tc::smem_addr(&s_cbar), 1);
        tc::mbar_init_fence();
        s_abort = 0;
    }
    // A's padding columns (past Kc) stay zero in both stages
    for (uint32_t e = (uint32_t)tid * 16u; e < 2u * region; e += kC2rThreads * 16u)
        *reinterpret_cast<uint4*>(A_stage(0) + e) = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) tc::tmem_alloc(&s_tmem, 256);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    // the kernels of item `it`: [k0, k1)
    auto item_k = [&](long long it, int* k0, int* k1) {
        const int g = (int)(it % ngroups);
        *k0 = g * p.kgroup;
        *k1 = min(p.K, *k0 + p.kgroup);
    };
    unsigned long long best = 0ull;

    if (warp < kC2rFormWarps) {
        // ---------------- A of every step: row = line, the line's P2 real numbers (c2r_col_bin)
        const unsigned char* spec_b = reinterpret_cast<const unsigned char*>(p.spec);
        const int nyq = (p.P2 & 1) ? -1 : p.P2 / 2;
        const int nyq_sl = nyq >= 0 ? nyq >> 5 : 0;
        const uint32_t lane_chunk = (uint32_t)lane >> 2, lane_byte = 4u * (uint32_t)(lane & 3);
        // quarter q of a step is staged in buffer q & 1, whose uses alternate phase parity
        auto issue_quarter = [&](long long it, int k, int q) {
            const C2rQuarter h = c2r_quarter(p, it, ngroups, k, q);
            const uint32_t bar = tc::smem_addr(&s_vfull[q & 1]);
            tc::mbar_expect_tx(bar, h.bytes);
            if (h.bytes)
                tc::bulk_g2s(tc::smem_addr(V_stage(q & 1)), spec_b + (((unsigned long long)h.f0 * 8ull) & ~15ull),
                             h.bytes, bar);
        };
        // thread 0's cursor: the quarter whose copy goes out next, two ahead of the one read
        long long nit = blockIdx.x;
        int nk = 0, nk1 = 0, nq = 0;
        auto advance = [&]() {
            if (++nq == 4) {
                nq = 0;
                if (++nk >= nk1) {
                    nit += gridDim.x;
                    if (nit < items) item_k(nit, &nk, &nk1);
                }
            }
        };
        if (tid == 0) {
            tc::mbar_expect_tx(tc::smem_addr(&s_cbar), region);
            tc::bulk_g2s(tc::smem_addr(Cs), p.C, region, tc::smem_addr(&s_cbar));
            if (nit < items) {
                item_k(nit, &nk, &nk1);
                issue_quarter(nit, nk, 0);
                issue_quarter(nit, nk, 1);
                advance();
                advance();
            }
        }
        const uint32_t idesc = tc::idesc_bf16_f32(kC2rRows, kC2rN);
        const uint32_t c0 = tc::smem_addr(Cs);
        // an abort is only acted on through a barrier of the formation warps that tells all of
        // them at once, so that they leave the loops together
        bool stop = false;
        uint32_t t = 0;
        for (long long it = blockIdx.x; it < items && !stop; it += gridDim.x) {
            int k0, k1;
            item_k(it, &k0, &k1);
            for (int k = k0; k < k1 && !stop; ++k, ++t) {
                const int s = (int)(t & 1);
                unsigned char* As = A_stage(s);
                // A[s] is free once the MMAs of step t - 2 are done
                bool ok = t < 2 || tc::mbar_wait(tc::smem_addr(&s_done[s]), ((t - 2) >> 1) & 1u);
                for (int q = 0; q < 4; ++q) {
                    ok = ok && tc::mbar_wait(tc::smem_addr(&s_vfull[q & 1]), (uint32_t)(q >> 1) & 1u);
                    stop = tc::bar_sync_or<1, kC2rFormThreads>(!ok || s_abort != 0);
                    if (stop) break;
                    const C2rQuarter h = c2r_quarter(p, it, ngroups, k, q);
                    const float2* vs = reinterpret_cast<const float2*>(V_stage(q & 1)) + h.lead;
                    // warp w takes lines w, w + 4, ... (two per pass); lane l the bins l, l + 32,
                    // l + 64, l + 96 (H2 <= Kc / 2 + 1 <= 97: the shared-memory bound keeps
                    // Kc <= 192).  Lane 0 stores Re V[0] with Re V[P2 / 2] (columns 0, 1).
#pragma unroll 1
                    for (int r0 = warp; r0 < h.rows; r0 += 2 * kC2rFormWarps) {
                        float2 z[2][4];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int r = r0 + u * kC2rFormWarps;
                            const float2* src = vs + r * p.H2 + lane;
#pragma unroll
                            for (int sl = 0; sl < 4; ++sl)
                                z[u][sl] = (r < h.rows && lane + 32 * sl < p.H2) ? src[32 * sl] : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int r = r0 + u * kC2rFormWarps;
                            if (r >= h.rows) break;
                            const float zs = nyq_sl == 0 ? z[u][0].x : nyq_sl == 1 ? z[u][1].x
                                           : nyq_sl == 2 ? z[u][2].x : z[u][3].x;
                            const float zn = nyq >= 0 ? __shfl_sync(0xffffffffu, zs, nyq & 31) : 0.f;
                            const int row = h.row0 + r;
                            // 64-column atoms 16 KB apart (128 rows); the lane's swizzled chunk
                            unsigned char* dst = As + (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
                                                 ((lane_chunk ^ (uint32_t)(row & 7)) << 4) + lane_byte;
#pragma unroll
                            for (int sl = 0; sl < 4; ++sl) {
                                const int h2 = lane + 32 * sl;
                                const uint32_t w = tc::pack_bf16x2(z[u][sl].x, (sl == 0 && lane == 0) ? zn : z[u][sl].y);
                                if (h2 < p.H2 && h2 != nyq)
                                    *reinterpret_cast<uint32_t*>(dst + (uint32_t)sl * (uint32_t)(kC2rRows / 8) * 1024u) = w;
                            }
                        }
                    }
                    tc::fence_async_smem();
                    c2r_form_sync();
                    // staging buffer q & 1 is read: the quarter two ahead goes out
                    if (tid == 0 && nit < items) {
                        issue_quarter(nit, nk, nq);
                        advance();
                    }
                }
                if (stop) break;
                if (tid == 0) {
                    // D[s] is free once the epilogue has read step t - 2; C has landed
                    bool ok2 = t > 0 || tc::mbar_wait(tc::smem_addr(&s_cbar), 0);
                    ok2 = ok2 && (t < 2 || tc::mbar_wait(tc::smem_addr(&s_acce[s]), ((t - 2) >> 1) & 1u));
                    if (ok2) {
                        tc::fence_after_sync();
                        const uint32_t a0 = tc::smem_addr(As);
                        const uint32_t d = tmem + (uint32_t)(s * kC2rN);
                        for (int ks = 0; ks < p.Kc / 16; ++ks) {
                            const uint32_t off = (uint32_t)(ks >> 2) * 16u * 1024u + (uint32_t)(ks & 3) * 32u;
                            tc::mma_bf16(d, tc::desc_kmajor_sw128(a0 + off), tc::desc_kmajor_sw128(c0 + off), idesc,
                                         ks > 0 ? 1u : 0u);
                        }
                        tc::mma_commit(tc::smem_addr(&s_done[s]));
                    } else {
                        s_abort = 1;   // the formation warps see it at their next barrier
                    }
                }
            }
        }
        if (stop) s_abort = 1;
    } else {
        // ---------------- running maxima: TMEM lane = line, kC2rCols columns (outputs i2) per thread
        const int ew = warp - kC2rFormWarps;            // 0..15
        const int quad = warp & 3, part = ew >> 2;
        const int cbase = kC2rCols * part;
        float mx[kC2rCols];
        uint32_t akp[kC2rCols / 4];   // the kernel of each maximum, one byte per column (K <= 256)
        bool saw_nan = false;
        uint32_t t = 0;
        for (long long it = blockIdx.x; it < items && !s_abort; it += gridDim.x) {
            int k0, k1;
            item_k(it, &k0, &k1);
            const int L = (int)(it / ngroups) * kC2rRows + 32 * quad + lane;
#pragma unroll
            for (int c = 0; c < kC2rCols; ++c) mx[c] = -INFINITY;
#pragma unroll
            for (int c = 0; c < kC2rCols / 4; ++c) akp[c] = 0u;
            for (int k = k0; k < k1 && !s_abort; ++k, ++t) {
                const int s = (int)(t & 1);
                if (!tc::mbar_wait(tc::smem_addr(&s_done[s]), (t >> 1) & 1u)) {
                    s_abort = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t row = tmem + (uint32_t)(s * kC2rN + cbase) + ((uint32_t)(quad * 32) << 16);
#pragma unroll
                for (int cb = 0; cb < kC2rCols; cb += 32) {
                    float v0[16], v1[16];
                    tc::tmem_ld16_nowait(row + (uint32_t)cb, v0);
                    tc::tmem_ld16_nowait(row + (uint32_t)(cb + 16), v1);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        const float v = (c < 16 ? v0[c] : v1[c - 16]) * p.scale;
                        const int i2 = cbase + cb + c;
                        if (v != v) saw_nan = true;
                        if (v > mx[cb + c]) {
                            mx[cb + c] = v;
                            const int sh = 8 * ((cb + c) & 3);
                            akp[(cb + c) >> 2] = (akp[(cb + c) >> 2] & ~(0xFFu << sh)) | ((uint32_t)k << sh);
                        }
                        if (p.eta_out && L < p.nlines && i2 < p.n2)
                            p.eta_out[(long long)k * p.V + (long long)L * p.n2 + i2] = v;
                    }
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::smem_addr(&s_acce[s]));
            }
            // the group's maxima into the candidate keys
#pragma unroll
            for (int c = 0; c < kC2rCols; ++c) {
                const int i2 = cbase + c;
                if (L < p.nlines && i2 < p.n2) {
                    const long long o = (long long)L * p.n2 + i2;
                    const unsigned int kc = (akp[c >> 2] >> (8 * (c & 3))) & 0xFFu;
                    const unsigned long long key = candidate_key(mx[c], (unsigned long long)kc * p.V + o);
                    if (p.vox_key) {
                        // one group holds every kernel (the launcher's choice when per-voxel
                        // keys are wanted): the key is final
                        if (ngroups == 1) p.vox_key[o] = key;
                        else atomicMax(p.vox_key + o, key);
                    }
                    if (key > best) best = key;
                }
            }
        }
        if (saw_nan) best = ~0ull;
    }
    __syncthreads();
    if (s_abort) {
        // a bounded wait ran out: report it and give the MMAs and copies in flight time to
        // finish (bounded; a copy still in flight after that is not waited for)
        if (tid == 0) {
            atomicExch(p.err, 1);
            for (int i = 0; i < 2; ++i) tc::mbar_wait(tc::smem_addr(&s_done[i]), 0, 1 << 16);
            for (int i = 0; i < 2; ++i) tc::mbar_wait(tc::smem_addr(&s_vfull[i]), 0, 1 << 16);
            tc::mbar_wait(tc::smem_addr(&s_cbar), 0, 1 << 16);
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
    // the grid maximum: a key per warp, decoded by the CTA that finishes last
    if (p.best_key) {
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_down_sync(0xffffffffu, best, off);
            if (o > best) best = o;
        }
        if (lane == 0 && best) atomicMax(p.best_key, best);
        if (last_block(p.counter, gridDim.x) && tid == 0) {
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

sfw_status launch_c2r_tc(const C2rTcPass& p0, int num_sms, cudaStream_t st) {
    C2rTcPass p = p0;
    if (p.n2 < 1 || p.n2 > kC2rN || p.Kc % 16 || p.Kc < p.P2 + (p.P2 & 1) || p.H2 != p.P2 / 2 + 1 || p.H2 > 128 ||
        p.K < 1 || p.K > 256 || p.nlines < 1 || (reinterpret_cast<uintptr_t>(p.spec) & 15u) ||
        (reinterpret_cast<uintptr_t>(p.C) & 15u))
        return fail(SFW_ERR_SHAPE, "certificate tail on the tensor cores: n2=%d Kc=%d P2=%d H2=%d", p.n2, p.Kc, p.P2,
                    p.H2);
    const size_t smem = tc_c2r_smem_bytes(p.Kc);
    if (smem > 226u * 1024u) return fail(SFW_ERR_SHAPE, "certificate tail on the tensor cores: shared memory");
    // kernels per item: the fewest steps on the busiest CTA, then the fewest key merges; all
    // kernels in one item when per-voxel keys are wanted (stored once, without atomics)
    const long long ntiles = (p.nlines + kC2rRows - 1) / kC2rRows;
    int best_kg = 1;
    long long best_steps = -1;
    for (int kg = p.vox_key ? p.K : 1; kg <= p.K; ++kg) {
        const long long items = ntiles * ((p.K + kg - 1) / kg);
        const long long per = (items + num_sms - 1) / num_sms;
        const long long steps = per * kg;
        if (best_steps < 0 || steps <= best_steps) {
            best_steps = steps;
            best_kg = kg;
        }
    }
    p.kgroup = best_kg;
    const long long items = ntiles * ((p.K + best_kg - 1) / best_kg);
    const int grid = (int)(items < num_sms ? items : num_sms);
    static int configured = 0;
    if ((int)smem > configured) {
        SFW_CUDA(cudaFuncSetAttribute(k_c2r_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = (int)smem;
    }
    SFW_LAUNCH(st, "k_c2r_tc", k_c2r_tc<<<grid, kC2rThreads, smem, st>>>(p));
    return launch_check("k_c2r_tc");
}

}  // namespace sfw
