// The certificate's last stage on the tensor cores (tf32 operands, FP32 accumulation in
// tensor memory): the real inverse along axis 2 with the maximum over the kernels.
//
// After the axes 0 and 1 every line L = (i0, i1) of kernel k holds the half spectrum
// V_k[L, h2], h2 < H2 = P2 / 2 + 1, of a real line, and Eq. 5's certificate is
//     eta_k(i0, i1, i2) = (1 / lambda) sum_h2 c_h2 (Re V cos(2 pi h2 i2 / P2) - Im V sin(...))
// (c_h2 = 1 at h2 = 0 and P2 / 2, else 2; the 1 / |P| of the inverse is in the table).  Read as
// 2 H2 real numbers (Re, Im interleaved, exactly as the spectra lie in memory), a line times
// the fixed matrix C^T (2 H2 x n2; the coefficients of Im V[0] and Im V[P2 / 2] are sin 0 = 0)
// gives its n2 outputs, so over 128 lines this is one GEMM per kernel,
//     D (128 lines x n2) = A (128 x 2 H2) . C^T,
// with A loaded by the tensor-memory accelerator straight from the FP32 spectra into the
// swizzled operand layout and multiplied as tf32: no conversion pass.  A CTA takes a tile of
// 128 lines and a group of kernels; its epilogue warps keep each output's running maximum and
// its kernel in registers, then fold them into the per-voxel and grid-maximum candidate keys
// (value, then lowest flat index k V + lin(m)).
#include <math.h>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "sfw_internal.cuh"
#include "tc_sm100.cuh"

namespace sfw {

constexpr int kC2rRows = 128;      // lines per tile (M)
constexpr int kC2rN = 128;         // outputs per line (N), n2 <= 128
constexpr int kC2rChunk = 32;      // tf32 columns per 128-byte swizzle atom (one A stage)
constexpr uint32_t kC2rAtom = kC2rRows * 128u;   // bytes of a 128-row x 32-column atom
constexpr int kC2rEpiWarps = 16;   // warps 0-15: four per tensor-memory lane quadrant
constexpr int kC2rCols = kC2rN / (kC2rEpiWarps / 4);             // columns (outputs) per epilogue thread
constexpr int kC2rProdWarp = kC2rEpiWarps, kC2rMmaWarp = kC2rEpiWarps + 1;
constexpr int kC2rThreads = 32 * (kC2rEpiWarps + 2);
constexpr int kC2rMaxStages = 8;

// Columns of C (and of a line's A row): 2 h2 + part, part 0 = Re, 1 = Im; chunks of 32.
int tc_c2r_chunks(int H2) { return (2 * H2 + kC2rChunk - 1) / kC2rChunk; }

// C^T's rows as the MMA's B operand: row i2 < n2, column 2 h2 + part = c_h2 (cos, -sin)
// (2 pi h2 i2 / P2), zero elsewhere; FP32, atoms of 128 rows x 32 columns with the 128-byte
// swizzle (16-byte unit u of row r at unit u ^ (r mod 8)).
__global__ void k_tc_c2r_matrix(int P2, int H2, int n2, int nch, float* __restrict__ C) {
    const int total = kC2rN * nch * kC2rChunk;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int i2 = i / (nch * kC2rChunk), c = i - i2 * nch * kC2rChunk;
        const int h2 = c >> 1, part = c & 1;
        float v = 0.f;
        if (i2 < n2 && h2 < H2) {
            const long long r = ((long long)h2 * i2) % P2;
            double sn, cs;
            sincospi(2.0 * (double)r / (double)P2, &sn, &cs);
            const double w = (h2 == 0 || 2 * h2 == P2) ? 1.0 : 2.0;
            v = (float)(part ? -w * sn : w * cs);
        }
        const int cc = c & (kC2rChunk - 1);
        const uint32_t off = (uint32_t)(c / kC2rChunk) * kC2rAtom + (uint32_t)(i2 >> 3) * 1024u +
                             (uint32_t)(i2 & 7) * 128u + ((((uint32_t)cc >> 2) ^ (uint32_t)(i2 & 7)) << 4) +
                             (uint32_t)(cc & 3) * 4u;
        *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(C) + off) = v;
    }
}

sfw_status launch_tc_c2r_matrix(int P2, int H2, int n2, float* C, cudaStream_t st) {
    const int nch = tc_c2r_chunks(H2);
    SFW_LAUNCH(st, "k_tc_c2r_matrix", k_tc_c2r_matrix<<<64, 256, 0, st>>>(P2, H2, n2, nch, C));
    return launch_check("k_tc_c2r_matrix");
}

// Dynamic shared memory: C (nch atoms, resident), then a ring of A stages (one atom each).
static int c2r_stages(int nch) {
    const long long room = 226LL * 1024 - 1024 - (long long)nch * kC2rAtom;
    const long long s = room / kC2rAtom;
    return (int)(s > kC2rMaxStages ? kC2rMaxStages : s);
}
size_t tc_c2r_smem_bytes(int H2) {
    const int nch = tc_c2r_chunks(H2);
    return (size_t)(nch + c2r_stages(nch)) * kC2rAtom + 1024u;
}
bool tc_c2r_fits(int H2) { return c2r_stages(tc_c2r_chunks(H2)) >= 2; }

// The spectra as FP32 numbers (Re, Im interleaved): x = 2 h2 + part (2 H2 of them, row pitch
// 2 H2p), y = line, z = kernel; boxes of 32 x 128 x 1 with the 128-byte swizzle.
bool make_c2r_tmap(const float2* spec, int H2, int H2p, long long nlines, int K, void* tmap_out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    });
    if (!encode || (H2p & 1) || H2p < H2 || nlines < 1 || K < 1 || (reinterpret_cast<uintptr_t>(spec) & 15u))
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * H2), (cuuint64_t)nlines, (cuuint64_t)K};
    const cuuint64_t strides[2] = {(cuuint64_t)H2p * 8u, (cuuint64_t)nlines * (cuuint64_t)H2p * 8u};
    const cuuint32_t box[3] = {(cuuint32_t)kC2rChunk, (cuuint32_t)kC2rRows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap* tm = static_cast<CUtensorMap*>(tmap_out);
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(spec), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One CTA per (tile of 128 lines, group of kernels), persistent over such items; a step is one
// (item, kernel) and consists of nch chunks of 32 columns.  One lane of warp 16 loads the
// chunks of A (tensor-map boxes) into a ring of stages; one lane of warp 17 issues the
// 128 x 128 x 8 tf32 MMAs of each chunk against the resident C (two tensor-memory buffers);
// warps 0-15 fold each kernel's D into the running maxima and, after the group's last kernel,
// into the candidate keys.  mbarriers: full / empty per stage (box landed / its MMAs done),
// done (MMAs of a step finished), acc_empty (D read, 16 arrivals), C landed.  Every wait is
// bounded; a wait that runs out sets p.err.
__global__ void __launch_bounds__(kC2rThreads, 1) k_c2r_tc(C2rTcPass p, const __grid_constant__ CUtensorMap tm) {
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nch = p.nch, S = p.stages;
    unsigned char* Cs = base;                                   // C, resident: nch atoms
    unsigned char* ring = base + (uint32_t)nch * kC2rAtom;      // A stages
    __shared__ __align__(8) unsigned long long s_full[kC2rMaxStages], s_empty[kC2rMaxStages], s_done[2], s_acce[2],
        s_cbar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (p.nlines + kC2rRows - 1) / kC2rRows;
    const int ngroups = (p.K + p.kgroup - 1) / p.kgroup;
    const long long items = (long long)ntiles * ngroups;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            tc::mbar_init(tc::smem_addr(&s_full[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(tc::smem_addr(&s_done[i]), 1);
            tc::mbar_init(tc::smem_addr(&s_acce[i]), kC2rEpiWarps);
        }
        tc::mbar_init(tc::smem_addr(&s_cbar), 1);
        tc::mbar_init_fence();
        s_abort = 0;
    }
    if (warp == kC2rProdWarp) tc::tmem_alloc(&s_tmem, 256);
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

    if (warp == kC2rProdWarp) {
        // ---------------- producer: C once, then the chunks of every step into the ring
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];\n" :: "l"(&tm) : "memory");
            const uint32_t cbytes = (uint32_t)nch * kC2rAtom;
            tc::mbar_expect_tx(tc::smem_addr(&s_cbar), cbytes);
            tc::bulk_g2s(tc::smem_addr(Cs), p.C, cbytes, tc::smem_addr(&s_cbar));
            // ring position of the next chunk; its use count's parity flips at every wrap
            uint32_t slot = 0, ph = 0;
            bool wrapped = false;
            for (long long it = blockIdx.x; it < items && !s_abort; it += gridDim.x) {
                int k0, k1;
                item_k(it, &k0, &k1);
                const int y = (int)(it / ngroups) * kC2rRows;
                for (int k = k0; k < k1 && !s_abort; ++k) {
                    for (int c = 0; c < nch; ++c) {
                        // the stage is free once the MMAs of its previous chunk are done
                        if (wrapped && !tc::mbar_wait(tc::smem_addr(&s_empty[slot]), ph ^ 1u)) {
                            s_abort = 1;
                            break;
                        }
                        tc::mbar_expect_tx(tc::smem_addr(&s_full[slot]), kC2rAtom);
                        tc::tma_load_3d(tc::smem_addr(ring + slot * kC2rAtom), &tm, c * kC2rChunk, y, k,
                                        tc::smem_addr(&s_full[slot]));
                        if (++slot == (uint32_t)S) {
                            slot = 0;
                            ph ^= 1u;
                            wrapped = true;
                        }
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == kC2rMmaWarp) {
        // ---------------- MMA lane.  This one thread's instruction latency paces the MMAs: the
        // descriptors are built once and advanced by adding to their address field (16-byte
        // units), the ring position is tracked without divisions, a chunk's MMAs are unrolled.
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32_f32(kC2rRows, kC2rN);
            const uint64_t dA0 = tc::desc_kmajor_sw128(tc::smem_addr(ring));
            const uint64_t dB0 = tc::desc_kmajor_sw128(tc::smem_addr(Cs));
            constexpr uint64_t kAtomStep = kC2rAtom >> 4, kKStep = 32u >> 4;   // atom, K = 8 slice
            // K = 8 slices of the last chunk holding columns < 2 H2 (the rest is zero)
            const int nks_last = min(4, (2 * p.H2 - (nch - 1) * kC2rChunk + 7) / 8);
            if (!tc::mbar_wait(tc::smem_addr(&s_cbar), 0)) s_abort = 1;
            uint32_t slot = 0, ph = 0, t = 0;
            for (long long it = blockIdx.x; it < items && !s_abort; it += gridDim.x) {
                int k0, k1;
                item_k(it, &k0, &k1);
                for (int k = k0; k < k1 && !s_abort; ++k, ++t) {
                    const int s = (int)(t & 1);
                    // D[s] is free once the epilogue has read step t - 2
                    if (t >= 2 && !tc::mbar_wait(tc::smem_addr(&s_acce[s]), ((t - 2) >> 1) & 1u)) {
                        s_abort = 1;
                        break;
                    }
                    const uint32_t d = tmem + (uint32_t)(s * kC2rN);
                    for (int c = 0; c < nch; ++c) {
                        if (!tc::mbar_wait(tc::smem_addr(&s_full[slot]), ph)) {
                            s_abort = 1;
                            break;
                        }
                        tc::fence_after_sync();
                        const uint64_t a = dA0 + slot * kAtomStep, b = dB0 + (uint64_t)c * kAtomStep;
                        const uint32_t acc0 = c > 0 ? 1u : 0u;
                        if (c + 1 < nch) {
                            tc::mma_tf32(d, a, b, idesc, acc0);
                            tc::mma_tf32(d, a + kKStep, b + kKStep, idesc, 1u);
                            tc::mma_tf32(d, a + 2 * kKStep, b + 2 * kKStep, idesc, 1u);
                            tc::mma_tf32(d, a + 3 * kKStep, b + 3 * kKStep, idesc, 1u);
                        } else {
                            tc::mma_tf32(d, a, b, idesc, acc0);
                            for (int ks = 1; ks < nks_last; ++ks)
                                tc::mma_tf32(d, a + ks * kKStep, b + ks * kKStep, idesc, 1u);
                        }
                        tc::mma_commit(tc::smem_addr(&s_empty[slot]));
                        if (++slot == (uint32_t)S) {
                            slot = 0;
                            ph ^= 1u;
                        }
                    }
                    if (s_abort) break;
                    tc::mma_commit(tc::smem_addr(&s_done[s]));
                }
            }
        }
        __syncwarp();
    } else {
        // ---------------- running maxima: TMEM lane = line, kC2rCols columns (outputs i2) per thread
        const int quad = warp & 3, part = warp >> 2;
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
            for (int i = 0; i < S; ++i) tc::mbar_wait(tc::smem_addr(&s_full[i]), 0, 1 << 16);
            tc::mbar_wait(tc::smem_addr(&s_cbar), 0, 1 << 16);
        }
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == kC2rProdWarp) tc::tmem_dealloc(tmem, 256);
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

sfw_status launch_c2r_tc(const C2rTcPass& p0, const void* tmap, int num_sms, cudaStream_t st) {
    C2rTcPass p = p0;
    if (!tmap || p.n2 < 1 || p.n2 > kC2rN || p.H2 != p.P2 / 2 + 1 || !tc_c2r_fits(p.H2) || p.K < 1 || p.K > 256 ||
        p.nlines < 1 || (reinterpret_cast<uintptr_t>(p.C) & 15u))
        return fail(SFW_ERR_SHAPE, "certificate tail on the tensor cores: n2=%d P2=%d H2=%d", p.n2, p.P2, p.H2);
    p.nch = tc_c2r_chunks(p.H2);
    p.stages = c2r_stages(p.nch);
    const size_t smem = tc_c2r_smem_bytes(p.H2);
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
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tmap);
    SFW_LAUNCH(st, "k_c2r_tc", k_c2r_tc<<<grid, kC2rThreads, smem, st>>>(p, *tm));
    return launch_check("k_c2r_tc");
}

}  // namespace sfw
