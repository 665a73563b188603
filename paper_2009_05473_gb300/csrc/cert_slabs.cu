// The grid certificate's passes along axes 1 and 2 (Eq. 5; Algorithm 1 step 1) done
// per i0 slab, one CTA per slab, so the slab stays in shared memory between the two
// axes: the head (forward: real transform of the residual's rows along axis 2, then
// the columns along axis 1) and the tail (per kernel k: the columns' inverse along
// axis 1, the rows' real inverse along axis 2, and the running max / argmax over the
// CTA's kernels).
//
// Both use the register-resident transform (lengths 64 / 128).  Columns: each warp
// transforms 4 columns 8 apart, so that the two columns a half-warp reads sit in
// distinct banks (the complex row pitch H2 is 1 mod 16 float2).  Rows: complex line c
// carries real rows c (real part) and c + rows/2 (imaginary part).  The tail's slab
// in[k][i0] (P1 x H2 complex, contiguous) arrives by 16-byte cp.async; the head's
// result leaves by one bulk copy from shared to global memory.  Neither intermediate
// of the per-axis form, (n0, n1, H2) or (K, n0, n1, H2), is written.
#include <map>
#include <mutex>
#include <tuple>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "fft_core.cuh"

namespace sfw {

constexpr int kTailThreads = 256;
constexpr int kTailWarps = kTailThreads / 32;

template <int P1, int P2>
struct TailGeom {
    static constexpr int H2 = P2 / 2 + 1;
    static constexpr int SLAB = P1 * H2;                      // float2
    static constexpr int XS = RegFFT<P1>::XS > RegFFT<P2>::XS ? RegFFT<P1>::XS : RegFFT<P2>::XS;
    static constexpr int XL = 4;                              // exchange rows per warp
    static constexpr int NC = P1 / 4;                         // complex lines of axis 2
    static constexpr int NT1 = (P2 / 2) / 4 + 1;              // axis-1 tasks (4 columns each)
    static constexpr int NT2 = NC / RegFFT<P2>::LPW;          // axis-2 tasks
    // slab capacity (float2): a whole number of TMA boxes may overrun the slab
    __host__ __device__ static int cap(int boxg, int nbox) {
        const int c = boxg * nbox * 4 > SLAB ? boxg * nbox * 4 : SLAB;
        return (c + 15) & ~15;
    }
    static size_t smem(int slab_cap) {
        return 128 + sizeof(float2) * ((size_t)slab_cap + RegFFT<P1>::TWN + RegFFT<P2>::TWN +
                                       (size_t)kTailWarps * XL * XS);
    }
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Wait (bounded) for the phase of parity `phase` of the barrier at bar to complete.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase) {
    for (int it = 0; it < (1 << 16); ++it) {
        unsigned done = 0;
        asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, q;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

template <int P1, int P2, bool TMA>
__global__ void __launch_bounds__(kTailThreads) k_cert_tail(CertTailPass p,
                                                            const __grid_constant__ CUtensorMap tmap) {
    using G = TailGeom<P1, P2>;
    static_assert(RegFFT<P1>::T == 8 && RegFFT<P2>::T == 8, "4 lines per warp on both axes");
    static_assert(G::NT2 <= kTailWarps, "one axis-2 task per warp");
    constexpr int H2 = G::H2;
    constexpr int R1a = RegGeom<P1>::R1, R1b = RegGeom<P2>::R1;
    constexpr int MH = R1b / 2;                 // kept outputs per lane and real row
    extern __shared__ float4 smem_raw[];
    // the slab starts 128-byte aligned (TMA destination)
    float2* S = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    float2* TW1 = S + (TMA ? G::cap(p.boxg, p.nbox) : G::cap(0, 0));
    float2* TW2 = TW1 + RegFFT<P1>::TWN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* XW = TW2 + RegFFT<P2>::TWN + warp * (G::XL * G::XS);
    const int t = lane & 7, li = lane >> 3;
    float2* xl = XW + li * G::XS;
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_late;
    if (TMA && threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" :: "r"(smem_u32(&s_bar)) : "memory");
        s_late = 0;
    }
    reg_twiddles<P1, kTailThreads>(p.tw1, TW1);
    reg_twiddles<P2, kTailThreads>(p.tw2, TW2);
    const int i0 = blockIdx.x;
    const int k0 = (int)blockIdx.y * p.nspec;
    const int nk = min(p.nspec, p.ktotal - k0);

    // axis-2 task of this warp: complex line c = warp + (NC / 4) li, rows c and c + NC
    const bool has2 = warp < G::NT2;
    const int cA = warp + (G::NC / 4) * li, cB = cA + G::NC;
    float mx[2][MH];
    int ak[2][MH];
#pragma unroll
    for (int m = 0; m < MH; ++m) {
        mx[0][m] = mx[1][m] = -INFINITY;
        ak[0][m] = ak[1][m] = 0;
    }
    bool saw_nan = false;

    __syncthreads();
    for (int s = 0; s < nk; ++s) {
        const int kk = k0 + s;
        if constexpr (TMA) {
            // the slab's line groups: nbox box copies {4, 1, boxg, 1} at (0, i0, b boxg, kk)
            const unsigned bar = smem_u32(&s_bar);
            if (threadIdx.x == 0) {
                const unsigned bytes = (unsigned)(p.nbox * p.boxg * 32);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                             :: "r"(bar), "r"(bytes) : "memory");
                for (int b = 0; b < p.nbox; ++b)
                    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
                                 :: "r"(smem_u32(S + b * p.boxg * 4)), "l"(&tmap), "r"(0), "r"(i0),
                                    "r"(b * p.boxg), "r"(kk), "r"(bar)
                                 : "memory");
            }
            if (!mbar_wait(bar, (unsigned)(s & 1))) s_late = 1;
            __syncthreads();
            if (s_late) {
                // the copies did not land in time: flag it, wait once more for them, stop
                if (threadIdx.x == 0) atomicExch(p.err, 1);
                mbar_wait(bar, (unsigned)(s & 1));
                break;
            }
        } else {
            const float2* src = p.in + ((long long)kk * p.n0 + i0) * G::SLAB;
            for (int e = threadIdx.x; e < G::SLAB / 2; e += kTailThreads) cp_async16(S + 2 * e, src + 2 * e);
            cp_async_commit();
            cp_async_wait0();
            __syncthreads();
        }
        // axis 1: columns (P2 / 2 of them in groups of 32, then the last one, P2 / 2)
        for (int task = warp; task < G::NT1; task += kTailWarps) {
            const int main_tasks = G::NT1 - 1;
            const int col = task < main_tasks ? (task >> 3) * 32 + (task & 7) + 8 * li : P2 / 2;
            const bool cv = task < main_tasks || li == 0;
            float2 v[R1a];
#pragma unroll
            for (int m = 0; m < R1a; ++m) v[m] = cv ? S[(t + 8 * m) * H2 + col] : make_float2(0.f, 0.f);
            reg_fft<P1, 1>(v, TW1, xl, t);
            if (cv) {
#pragma unroll
                for (int m = 0; m < R1a / 2; ++m) S[(t + 8 * m) * H2 + col] = v[m];
            }
        }
        __syncthreads();
        // axis 2: real inverse of rows cA (real part) and cB (imaginary part)
        if (has2) {
            const float2* ra = S + cA * H2;
            const float2* rb = S + cB * H2;
            float2 v[R1b];
#pragma unroll
            for (int m = 0; m < R1b; ++m) {
                const int j = t + 8 * m;
                const bool lo = 2 * j <= P2;
                const int k = lo ? j : P2 - j;
                const float2 a = ra[k], b = rb[k];
                v[m] = lo ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, b.x - a.y);
            }
            reg_fft<P2, 1>(v, TW2, xl, t);
#pragma unroll
            for (int m = 0; m < MH; ++m) {
                const int i2 = t + 8 * m;
                if (i2 < p.n2) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = h ? cB : cA;
                        if (row < p.n1) {
                            const float val = (h ? v[m].y : v[m].x) * p.scale;
                            if (p.eta_out)
                                p.eta_out[(long long)kk * p.V + ((long long)i0 * p.n1 + row) * p.n2 + i2] = val;
                            saw_nan = saw_nan || val != val;
                            if (val > mx[h][m]) {
                                mx[h][m] = val;
                                ak[h][m] = kk;
                            }
                        }
                    }
                }
            }
        }
        // the slab is reloaded for the next kernel: order this kernel's shared-memory
        // accesses before the copy engine's writes
        if constexpr (TMA) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
    }

    unsigned long long best = 0ull;
    if (has2 && nk > 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = h ? cB : cA;
            if (row >= p.n1) continue;
#pragma unroll
            for (int m = 0; m < MH; ++m) {
                const int i2 = t + 8 * m;
                if (i2 < p.n2) {
                    const long long o = ((long long)i0 * p.n1 + row) * p.n2 + i2;
                    const unsigned long long key = candidate_key(mx[h][m], (unsigned long long)ak[h][m] * p.V + o);
                    if (p.vox_key) atomicMax(p.vox_key + o, key);
                    if (key > best) best = key;
                }
            }
        }
    }
    if (saw_nan) best = ~0ull;
    if (p.best_key) {
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o2 = __shfl_down_sync(0xffffffffu, best, off);
            if (o2 > best) best = o2;
        }
        if (lane == 0 && best) atomicMax(p.best_key, best);
        __syncthreads();
        // the last CTA decodes the key and re-arms it (0) for the next call
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

// 18 warps: the 17 column tasks (P2 = 128) of the head run in one round.
constexpr int kHeadWarps = 18;
constexpr int kHeadThreads = 32 * kHeadWarps;

template <int P1, int P2>
struct HeadGeom {
    static constexpr int RSN = (P1 / 2) * (P2 / 2 + 1);        // real slab bound (floats)
    static size_t smem() {
        using G = TailGeom<P1, P2>;
        return sizeof(float2) * ((size_t)G::SLAB + RegFFT<P1>::TWN + RegFFT<P2>::TWN +
                                 (size_t)kHeadWarps * G::XL * G::XS) + sizeof(float) * (size_t)RSN;
    }
};

template <int P1, int P2>
__global__ void __launch_bounds__(kHeadThreads) k_cert_head(CertHeadPass p) {
    using G = TailGeom<P1, P2>;
    static_assert(RegFFT<P1>::T == 8 && RegFFT<P2>::T == 8, "4 lines per warp on both axes");
    constexpr int H2 = G::H2;
    constexpr int R1a = RegGeom<P1>::R1, R1b = RegGeom<P2>::R1;
    constexpr int NCH = P1 / 4;                  // complex lines of axis 2 (rows c, c + NCH)
    extern __shared__ float4 smem_raw[];
    float2* S = reinterpret_cast<float2*>(smem_raw);
    float2* TW1 = S + G::SLAB;
    float2* TW2 = TW1 + RegFFT<P1>::TWN;
    float2* XW0 = TW2 + RegFFT<P2>::TWN;
    float* RS = reinterpret_cast<float*>(XW0 + kHeadWarps * G::XL * G::XS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = lane & 7, li = lane >> 3;
    float2* xl = XW0 + warp * (G::XL * G::XS) + li * G::XS;
    const int i0 = blockIdx.x;
    const int n1 = p.n1, n2 = p.n2;
    const int NP = n2 | 1;                       // odd row pitch of the real slab
    {   // every element in flight at once (asynchronous copies)
        const float* src = p.r + (long long)i0 * n1 * n2;
        for (int e = threadIdx.x; e < n1 * n2; e += kHeadThreads) {
            const int i1 = e / n2;
            cp_async(RS + i1 * NP + (e - i1 * n2), src + e, 4);
        }
        cp_async_commit();
    }
    reg_twiddles<P1, kHeadThreads>(p.tw1, TW1);
    reg_twiddles<P2, kHeadThreads>(p.tw2, TW2);
    cp_async_wait0();
    __syncthreads();
    // axis 2: rows c and c + NCH as one complex line, forward, then split the two spectra
    if (warp < NCH / 4) {
        const int ra = warp + (NCH / 4) * li, rb = ra + NCH;
        float2 v[R1b];
#pragma unroll
        for (int m = 0; m < R1b; ++m) {
            const int j = t + 8 * m;
            const float a = (ra < n1 && j < n2) ? RS[ra * NP + j] : 0.f;
            const float b = (rb < n1 && j < n2) ? RS[rb * NP + j] : 0.f;
            v[m] = make_float2(a, b);
        }
        reg_fft<P2, -1>(v, TW2, xl, t);
#pragma unroll
        for (int m = 0; m < R1b; ++m) xl[t + 8 * m] = v[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < (H2 + 7) / 8; ++m) {
            const int k = t + 8 * m;
            if (k < H2) {
                const float2 z = xl[k], zm = xl[(P2 - k) & (P2 - 1)];
                S[ra * H2 + k] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
                S[rb * H2 + k] = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            }
        }
        __syncwarp();
    }
    __syncthreads();
    // axis 1: columns, rows [0, n1) zero-padded to P1, all P1 outputs in place
    for (int task = warp; task < G::NT1; task += kHeadWarps) {
        const int main_tasks = G::NT1 - 1;
        const int col = task < main_tasks ? (task >> 3) * 32 + (task & 7) + 8 * li : P2 / 2;
        const bool cv = task < main_tasks || li == 0;
        float2 v[R1a];
#pragma unroll
        for (int m = 0; m < R1a; ++m)
            v[m] = (cv && t + 8 * m < n1) ? S[(t + 8 * m) * H2 + col] : make_float2(0.f, 0.f);
        reg_fft<P1, -1>(v, TW1, xl, t);
        if (cv) {
#pragma unroll
            for (int m = 0; m < R1a; ++m) S[(t + 8 * m) * H2 + col] = v[m];
        }
    }
    // the slab leaves in one bulk copy (shared -> global), issued once its writes are
    // visible to the copy engine
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        float2* dst = p.out + (long long)i0 * G::SLAB;
        const unsigned src = (unsigned)__cvta_generic_to_shared(S);
        const unsigned bytes = (unsigned)(sizeof(float2) * G::SLAB);
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                     :: "l"(dst), "r"(src), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
    }
}

template <int P1, int P2>
static sfw_status run_head(const CertHeadPass& p, cudaStream_t st) {
    const size_t smem = HeadGeom<P1, P2>::smem();
    SFW_TRY(prepare(k_cert_head<P1, P2>, smem));
    SFW_LAUNCH(st, "k_cert_head", (k_cert_head<P1, P2><<<p.n0, kHeadThreads, smem, st>>>(p)));
    return launch_check("k_cert_head");
}

sfw_status launch_cert_head(const CertHeadPass& p0, cudaStream_t st) {
    CertHeadPass p = p0;
    if (!cert_tail_supported(p.P1, p.P2, p.n1, p.n2) || p.H2 != p.P2 / 2 + 1)
        return fail(SFW_ERR_SHAPE, "fused certificate head: unsupported lengths %d x %d", p.P1, p.P2);
    if (p.n0 < 1) return SFW_OK;
    SFW_TRY(twiddle_table(p.P1, p.P1 == 64 ? 8 : 16, &p.tw1));
    SFW_TRY(twiddle_table(p.P2, p.P2 == 64 ? 8 : 16, &p.tw2));
    if (p.P1 == 64 && p.P2 == 64) return run_head<64, 64>(p, st);
    if (p.P1 == 64) return run_head<64, 128>(p, st);
    if (p.P2 == 64) return run_head<128, 64>(p, st);
    return run_head<128, 128>(p, st);
}

bool cert_tail_supported(int P1, int P2, int n1, int n2) {
    return (P1 == 64 || P1 == 128) && (P2 == 64 || P2 == 128) && 2 * n1 <= P1 && 2 * n2 <= P2;
}

template <int P1, int P2, bool TMA>
static sfw_status run_tail(CertTailPass p, const CUtensorMap& tm, int groups, cudaStream_t st) {
    using G = TailGeom<P1, P2>;
    const size_t smem = G::smem(TMA ? G::cap(p.boxg, p.nbox) : G::cap(0, 0));
    auto kern = k_cert_tail<P1, P2, TMA>;
    SFW_TRY(prepare(kern, smem));
    int dev = 0;
    SFW_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int>, int> chosen;  // (dev, P1, P2, TMA, n0, K) -> groups
    const auto key = std::make_tuple(dev, P1, P2, (int)TMA, p.n0, p.ktotal);
    if (groups <= 0) {
        std::lock_guard<std::mutex> lk(mu);
        auto it = chosen.find(key);
        if (it != chosen.end()) groups = it->second;
    }
    if (groups <= 0) {
        // kernels per CTA: the fewest rounds of resident CTAs, then the most kernels per CTA
        int sms = 1, per = 1;
        SFW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        SFW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kTailThreads, smem));
        const long long slots = (long long)(per > 0 ? per : 1) * sms;
        long long best_cost = -1;
        for (int ns = 1; ns <= p.ktotal; ++ns) {
            const long long g = (p.ktotal + ns - 1) / ns;
            const long long rounds = (p.n0 * g + slots - 1) / slots;
            const long long cost = rounds * ns;
            if (best_cost < 0 || cost <= best_cost) {
                best_cost = cost;
                groups = (int)g;
            }
        }
        std::lock_guard<std::mutex> lk(mu);
        chosen[key] = groups;
    }
    p.nspec = (p.ktotal + groups - 1) / groups;
    groups = (p.ktotal + p.nspec - 1) / p.nspec;
    p.ntiles = p.n0 * groups;
    const dim3 grid((unsigned)p.n0, (unsigned)groups);
    SFW_LAUNCH(st, "k_cert_tail", (kern<<<grid, kTailThreads, smem, st>>>(p, tm)));
    return launch_check("k_cert_tail");
}

bool make_tail_tmap(const void* in, int n0, long long ngroups, int K, int boxg, void* tmap_out) {
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
    if (!encode || boxg < 1 || boxg > 256 || n0 < 1 || K < 1) return false;
    const cuuint64_t dims[4] = {4, (cuuint64_t)n0, (cuuint64_t)ngroups, (cuuint64_t)K};
    const cuuint64_t strides[3] = {32, (cuuint64_t)n0 * 32, (cuuint64_t)ngroups * n0 * 32};
    const cuuint32_t box[4] = {4, 1, (cuuint32_t)boxg, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUtensorMap* tm = static_cast<CUtensorMap*>(tmap_out);
    return encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<void*>(in), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

sfw_status launch_cert_tail(const CertTailPass& p0, const void* tmap, int groups, cudaStream_t st) {
    CertTailPass p = p0;
    if (!cert_tail_supported(p.P1, p.P2, p.n1, p.n2) || p.H2 != p.P2 / 2 + 1)
        return fail(SFW_ERR_SHAPE, "fused certificate tail: unsupported lengths %d x %d", p.P1, p.P2);
    if (p.n0 < 1 || p.ktotal < 1) return SFW_OK;
    if (tmap && (p.boxg < 4 || p.boxg > 256 || p.boxg % 4 || p.nbox < 1 || !p.err ||
                 (long long)p.boxg * p.nbox * 4 < (long long)p.P1 * p.H2))
        return fail(SFW_ERR_ARG, "fused certificate tail: bad box geometry");
    SFW_TRY(twiddle_table(p.P1, p.P1 == 64 ? 8 : 16, &p.tw1));
    SFW_TRY(twiddle_table(p.P2, p.P2 == 64 ? 8 : 16, &p.tw2));
    CUtensorMap tm;
    if (tmap) memcpy(&tm, tmap, sizeof(tm));
    else memset(&tm, 0, sizeof(tm));
#define SFW_TAIL(A, B) return tmap ? run_tail<A, B, true>(p, tm, groups, st) : run_tail<A, B, false>(p, tm, groups, st)
    if (p.P1 == 64 && p.P2 == 64) SFW_TAIL(64, 64);
    if (p.P1 == 64) SFW_TAIL(64, 128);
    if (p.P2 == 64) SFW_TAIL(128, 64);
    SFW_TAIL(128, 128);
#undef SFW_TAIL
}

}  // namespace sfw
