// Reductions and layout kernels: arg-maximum / top-k of the certificate (the
// grid maximum that seeds the local ascent of step 1, Algorithms 1 and 2),
// circular placement of the PSF and of the kernel family on FFT grids, and
// the conversions of the kernel-family table (Section 2's lookup table).
#include <math.h>

#include "sfw_internal.cuh"

namespace sfw {

// ------------------------------------------------------------------ circular placement

// out[p] = H(u) with u_a = p_a if p_a <= R_a, p_a - P_a if p_a >= P_a - R_a, else 0.
__global__ void k_wrap_psf(const float* psf, int R0, int R1, int R2, int P0, int P1, int P2,
                           float* out) {
    const long long total = (long long)P0 * P1 * P2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int p2 = (int)(i % P2);
        const long long r = i / P2;
        const int p1 = (int)(r % P1);
        const int p0 = (int)(r / P1);
        const int u0 = p0 <= R0 ? p0 : (p0 >= P0 - R0 ? p0 - P0 : 1 << 30);
        const int u1 = p1 <= R1 ? p1 : (p1 >= P1 - R1 ? p1 - P1 : 1 << 30);
        const int u2 = p2 <= R2 ? p2 : (p2 >= P2 - R2 ? p2 - P2 : 1 << 30);
        float v = 0.f;
        if (u0 != (1 << 30) && u1 != (1 << 30) && u2 != (1 << 30))
            v = psf[((long long)(u0 + R0) * (2 * R1 + 1) + (u1 + R1)) * (2 * R2 + 1) + (u2 + R2)];
        out[i] = v;
    }
}

sfw_status launch_wrap_psf(const float* psf, const int R[3], const int P[3], float* out,
                           cudaStream_t st) {
    SFW_LAUNCH(st, "k_wrap_psf", k_wrap_psf<<<1024, 256, 0, st>>>(psf, R[0], R[1], R[2], P[0], P[1], P[2], out));
    return launch_check("k_wrap_psf");
}

// kx holds K(x) for |x_a| <= n_a - 1 at index x + (n - 1) (dense (2n-1)^3).
// out[p] = K(-x) with x_a = p_a (p_a <= h_a) or p_a - P_a (p_a >= P_a - h_a), else 0:
// the correlation kernel, kept on the box |x_a| <= h_a (h_a <= n_a - 1, outside which it
// vanishes), placed for a circular convolution on P (P_a >= n_a + h_a: no wrap-around
// reaches a grid displacement).
__global__ void k_wrap_kernel(const float* kx, int n0, int n1, int n2, int h0, int h1, int h2, int P0,
                              int P1, int P2, float* out) {
    const long long total = (long long)P0 * P1 * P2;
    const int D1 = 2 * n1 - 1, D2 = 2 * n2 - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int p2 = (int)(i % P2);
        const long long r = i / P2;
        const int p1 = (int)(r % P1);
        const int p0 = (int)(r / P1);
        const int x0 = p0 <= h0 ? p0 : (p0 >= P0 - h0 ? p0 - P0 : 1 << 30);
        const int x1 = p1 <= h1 ? p1 : (p1 >= P1 - h1 ? p1 - P1 : 1 << 30);
        const int x2 = p2 <= h2 ? p2 : (p2 >= P2 - h2 ? p2 - P2 : 1 << 30);
        float v = 0.f;
        if (x0 != (1 << 30) && x1 != (1 << 30) && x2 != (1 << 30))
            v = kx[((long long)(-x0 + n0 - 1) * D1 + (-x1 + n1 - 1)) * D2 + (-x2 + n2 - 1)];
        out[i] = v;
    }
}

sfw_status launch_wrap_kernel(const float* kx, const int n[3], const int h[3], const int P[3], float* out,
                              cudaStream_t st) {
    for (int a = 0; a < 3; ++a)
        if (h[a] < 0 || h[a] > n[a] - 1 || P[a] < n[a] + h[a])
            return fail(SFW_ERR_SHAPE, "kernel placement: h[%d]=%d, P=%d, n=%d", a, h[a], P[a], n[a]);
    SFW_LAUNCH(st, "k_wrap_kernel", k_wrap_kernel<<<1024, 256, 0, st>>>(kx, n[0], n[1], n[2], h[0], h[1], h[2],
                                                                      P[0], P[1], P[2], out));
    return launch_check("k_wrap_kernel");
}

// ------------------------------------------------------------------ arg-maximum (top-1)

constexpr int kRedThreads = 256;

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_down_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    return v;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v) {
    __shared__ unsigned long long s[kRedThreads / 32];
    v = warp_max_u64(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long r = 0ull;
    if (threadIdx.x == 0)
        for (int q = 0; q < kRedThreads / 32; ++q) r = s[q] > r ? s[q] : r;
    return r;
}

// Pass 1: per-block max of candidate keys of v[i] (value, then lowest index).
__global__ void __launch_bounds__(kRedThreads)
k_argmax_keys(const float* __restrict__ v, long long count, unsigned long long* partial) {
    unsigned long long best = 0ull;
    for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < count;
         i += (long long)gridDim.x * kRedThreads) {
        const unsigned long long k = candidate_key(v[i], (unsigned long long)i);
        best = k > best ? k : best;
    }
    best = block_max_u64(best);
    if (threadIdx.x == 0) partial[blockIdx.x] = best;
}

// Pass 2: max over the partial keys, then decode.
__global__ void __launch_bounds__(kRedThreads)
k_argmax_final(const unsigned long long* partial, int n, float* val, int64_t* idx) {
    unsigned long long best = 0ull;
    for (int i = threadIdx.x; i < n; i += kRedThreads) best = partial[i] > best ? partial[i] : best;
    best = block_max_u64(best);
    if (threadIdx.x == 0) {
        if (best == ~0ull || best == 0ull) {
            *val = __int_as_float(0x7fc00000);
            *idx = -1;
        } else {
            *val = float_from_order_key((unsigned int)(best >> 32));
            *idx = (int64_t)(0xffffffffu - (unsigned int)(best & 0xffffffffu));
        }
    }
}

sfw_status launch_argmax_keys(const float* v, long long count, unsigned long long* partial,
                              int nblocks, cudaStream_t st) {
    SFW_LAUNCH(st, "k_argmax_keys", k_argmax_keys<<<nblocks, kRedThreads, 0, st>>>(v, count, partial));
    return launch_check("k_argmax_keys");
}

sfw_status launch_argmax_final(const unsigned long long* partial, int n, float* val, int64_t* idx,
                               cudaStream_t st) {
    SFW_LAUNCH(st, "k_argmax_final", k_argmax_final<<<1, kRedThreads, 0, st>>>(partial, n, val, idx));
    return launch_check("k_argmax_final");
}

// ------------------------------------------------------------------ top-k (k <= 64)

constexpr int kSortN = 4096;  // keys sorted per block

// Sort kSortN keys descending in shared memory (bitonic network).
__device__ void bitonic_desc(unsigned long long* s) {
    for (int size = 2; size <= kSortN; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < kSortN / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool desc = ((lo & size) == 0);
                const unsigned long long a = s[lo], b = s[hi];
                if ((a < b) == desc) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
        }
    }
    __syncthreads();
}

// Each block takes kSortN consecutive inputs (values -> keys when `v` is set,
// else keys from `kin`), sorts them and writes its top `k` keys.
__global__ void __launch_bounds__(kRedThreads)
k_topk_block(const float* v, const unsigned long long* kin, long long count, int k,
             unsigned long long* kout) {
    __shared__ unsigned long long s[kSortN];
    const long long base = (long long)blockIdx.x * kSortN;
    for (int i = threadIdx.x; i < kSortN; i += kRedThreads) {
        const long long g = base + i;
        unsigned long long key = 0ull;
        if (g < count) key = v ? candidate_key(v[g], (unsigned long long)g) : kin[g];
        s[i] = key;
    }
    bitonic_desc(s);
    for (int i = threadIdx.x; i < k; i += kRedThreads) kout[(long long)blockIdx.x * k + i] = s[i];
}

__global__ void k_topk_decode(const unsigned long long* keys, int k, float* val, int64_t* idx) {
    const int i = threadIdx.x;
    if (i >= k) return;
    const unsigned long long key = keys[i];
    bool nan_seen = keys[0] == ~0ull;
    if (nan_seen || key == 0ull) {
        val[i] = __int_as_float(0x7fc00000);
        idx[i] = -1;
    } else {
        val[i] = float_from_order_key((unsigned int)(key >> 32));
        idx[i] = (int64_t)(0xffffffffu - (unsigned int)(key & 0xffffffffu));
    }
}

// ---- top-k of many values by radix selection: the order keys (float_order_key) of the k-th
// largest value t are found 12 + 12 + 8 bits at a time from histograms, then the values above t
// and the lowest-index values equal to t are gathered and sorted.  The result equals the sort of
// all candidate keys (value, then lowest index); a NaN anywhere makes every output NaN / -1.
constexpr int kSelGrid = 256;          // blocks of the passes over the values (contiguous chunks)
constexpr int kSelBins = 4096;
// scratch layout (64-bit slots)
constexpr long long kSelHist = 0;                      // kSelBins counters (32-bit)
constexpr long long kSelState = kSelHist + kSelBins / 2;   // 32 counters (32-bit)
constexpr long long kSelAbove = kSelState + 16;        // <= 64 keys above t
constexpr long long kSelBlkCnt = kSelAbove + 64;       // ties kept per block
constexpr long long kSelBlkTies = kSelBlkCnt + kSelGrid;   // <= 64 tie keys per block, in index order
constexpr long long kSelOut = kSelBlkTies + (long long)kSelGrid * 64;
constexpr long long kSelScratch = kSelOut + 64;
// state words: prefix of t's order key fixed so far, count above the current bin range,
// NaN seen, keys gathered above t, ties wanted (k - above)
enum { kStPrefix = 0, kStAbove = 1, kStNan = 2, kStNa = 3, kStM = 4 };

// level 0: bits 31..20 of every value's order key; level 1: bits 19..8 of those whose bits 31..20
// equal the prefix; level 2: bits 7..0 of those whose bits 31..8 do
__device__ __forceinline__ int sel_shift(int level) { return level == 0 ? 20 : level == 1 ? 8 : 0; }

__global__ void __launch_bounds__(kRedThreads) k_sel_hist(const float* __restrict__ v, long long count, int level,
                                                          unsigned long long* scratch) {
    __shared__ unsigned int h[kSelBins];
    unsigned int* gh = reinterpret_cast<unsigned int*>(scratch + kSelHist);
    unsigned int* stw = reinterpret_cast<unsigned int*>(scratch + kSelState);
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    const unsigned int prefix = stw[kStPrefix];
    const int sh = sel_shift(level), hi = level == 0 ? 32 : sel_shift(level - 1);
    const unsigned int mask = level == 2 ? 0xFFu : 0xFFFu;
    bool nan = false;
    // four loads in flight per thread
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; g0 < count; g0 += 4 * stride) {
        float x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = g0 + j * stride < count ? v[g0 + j * stride] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (g0 + j * stride >= count) continue;
            if (x[j] != x[j]) {
                nan = true;
                continue;
            }
            const unsigned int o = float_order_key(x[j]);
            if (hi < 32 && (o >> hi) != (prefix >> hi)) continue;
            atomicAdd(&h[(o >> sh) & mask], 1u);
        }
    }
    if (nan) stw[kStNan] = 1u;
    __syncthreads();
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
        if (h[i]) atomicAdd(&gh[i], h[i]);
}

// One block: the bin of the k-th largest key at this level (counting from the top, after the
// keys already known to lie above), its bits into the prefix; the histogram is cleared.
__global__ void __launch_bounds__(kRedThreads) k_sel_pick(int level, int k, unsigned long long* scratch) {
    __shared__ unsigned int hs[kSelBins];
    __shared__ unsigned int wsum[kRedThreads / 32];
    __shared__ int s_found;
    unsigned int* gh = reinterpret_cast<unsigned int*>(scratch + kSelHist);
    unsigned int* stw = reinterpret_cast<unsigned int*>(scratch + kSelState);
    const int nb = level == 2 ? 256 : kSelBins;
    const int per = nb / kRedThreads;                  // bins per thread; thread 0 the top ones
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < kSelBins; i += blockDim.x) {
        hs[i] = gh[i];
        gh[i] = 0u;
    }
    if (t == 0) s_found = 0;
    __syncthreads();
    unsigned int part = 0;
    for (int j = 0; j < per; ++j) part += hs[nb - 1 - (t * per + j)];
    // inclusive scan over threads (from the top bins down)
    unsigned int incl = part;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    for (int w = 0; w < warp; ++w) incl += wsum[w];
    const unsigned int above = stw[kStAbove];
    const unsigned int excl = incl - part;
    if (above + excl < (unsigned int)k && above + incl >= (unsigned int)k) {
        unsigned int acc = above + excl;
        int bin = nb - 1 - t * per;
        for (int j = 0; j < per; ++j) {
            const int b = nb - 1 - (t * per + j);
            if (acc + hs[b] >= (unsigned int)k) {
                bin = b;
                break;
            }
            acc += hs[b];
        }
        s_found = 1;
        stw[kStPrefix] |= (unsigned int)bin << sel_shift(level);
        stw[kStAbove] = acc;
        if (level == 2) stw[kStM] = (unsigned int)k - acc;
    }
    __syncthreads();
    // fewer than k values that are not NaN: leave the prefix (the output is NaN / -1 anyway)
    if (t == 0 && !s_found && level == 2) stw[kStM] = 0u;
}

// The keys above t (at most k - 1, any order) and, per block, the first m keys equal to t in
// index order (blocks take contiguous chunks).
__global__ void __launch_bounds__(kRedThreads) k_sel_gather(const float* __restrict__ v, long long count,
                                                            unsigned long long* scratch) {
    __shared__ unsigned int warp_cnt[kRedThreads / 32];
    __shared__ unsigned int s_taken;
    unsigned int* stw = reinterpret_cast<unsigned int*>(scratch + kSelState);
    const unsigned int tkey = stw[kStPrefix], m = stw[kStM];
    unsigned long long* above = scratch + kSelAbove;
    unsigned long long* ties = scratch + kSelBlkTies + (long long)blockIdx.x * 64;
    const long long chunk = (count + gridDim.x - 1) / gridDim.x;
    const long long b0 = (long long)blockIdx.x * chunk, b1 = min(count, b0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_taken = 0;
    __syncthreads();
    constexpr int U = 4;
    for (long long base = b0; base < b1; base += U * blockDim.x) {
        float x[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const long long g = base + j * blockDim.x + threadIdx.x;
            x[j] = g < b1 ? v[g] : __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const long long g = base + j * blockDim.x + threadIdx.x;
            bool tie = false;
            unsigned long long key = 0ull;
            if (x[j] == x[j]) {   // beyond the chunk: NaN, never taken
                const unsigned int o = float_order_key(x[j]);
                key = candidate_key(x[j], (unsigned long long)g);
                if (o > tkey) {
                    const unsigned int pos = atomicAdd(&stw[kStNa], 1u);
                    if (pos < 64u) above[pos] = key;
                }
                tie = o == tkey;
            }
            // ties in index order (rank in the warp, then the warps before); skipped when this
            // group of the block holds none
            if (__syncthreads_or(tie)) {
                const unsigned int bal = __ballot_sync(0xffffffffu, tie);
                if (lane == 0) warp_cnt[warp] = __popc(bal);
                __syncthreads();
                unsigned int before = s_taken;
                for (int w = 0; w < warp; ++w) before += warp_cnt[w];
                const unsigned int r = before + __popc(bal & ((1u << lane) - 1u));
                if (tie && r < m) ties[r] = key;
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned int tot = 0;
                    for (int w = 0; w < kRedThreads / 32; ++w) tot += warp_cnt[w];
                    s_taken += tot;
                }
                __syncthreads();
            }
        }
    }
    if (threadIdx.x == 0) scratch[kSelBlkCnt + blockIdx.x] = min(s_taken, m);
}

// One block: the keys above t, then ties block by block until k keys, sorted descending.
__global__ void __launch_bounds__(64) k_sel_final(int k, int nblocks, unsigned long long* scratch) {
    __shared__ unsigned long long s[64];
    __shared__ unsigned int cnt[kSelGrid];
    unsigned int* stw = reinterpret_cast<unsigned int*>(scratch + kSelState);
    const int t = threadIdx.x;
    const unsigned int na = min(stw[kStNa], 64u);
    s[t] = (unsigned int)t < na ? scratch[kSelAbove + t] : 0ull;
    for (int b = t; b < nblocks; b += 64) cnt[b] = (unsigned int)scratch[kSelBlkCnt + b];
    __syncthreads();
    if (t == 0) {
        unsigned int n = na;
        for (int b = 0; b < nblocks && n < (unsigned int)k; ++b)
            for (unsigned int j = 0; j < cnt[b] && n < (unsigned int)k; ++j)
                s[n++] = scratch[kSelBlkTies + (long long)b * 64 + j];
    }
    __syncthreads();
    // bitonic sort of 64 keys, descending
    for (int size = 2; size <= 64; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int partner = t ^ stride;
            const unsigned long long a = s[t], b = s[partner];
            __syncthreads();
            if (partner > t) {
                const bool desc = (t & size) == 0;
                if ((a < b) == desc) {
                    s[t] = b;
                    s[partner] = a;
                }
            }
            __syncthreads();
        }
    }
    unsigned long long* out = scratch + kSelOut;
    if (t < k) out[t] = (stw[kStNan] && t == 0) ? ~0ull : s[t];
}

static sfw_status launch_topk_select(const float* v, long long count, int topk, unsigned long long* scratch,
                                     float* val_out, int64_t* idx_out, cudaStream_t st) {
    SFW_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)(kSelBlkCnt + kSelGrid), st));
    for (int level = 0; level < 3; ++level) {
        SFW_LAUNCH(st, "k_sel_hist", k_sel_hist<<<4 * kSelGrid, kRedThreads, 0, st>>>(v, count, level, scratch));
        SFW_TRY(launch_check("k_sel_hist"));
        SFW_LAUNCH(st, "k_sel_pick", k_sel_pick<<<1, kRedThreads, 0, st>>>(level, topk, scratch));
        SFW_TRY(launch_check("k_sel_pick"));
    }
    SFW_LAUNCH(st, "k_sel_gather", k_sel_gather<<<kSelGrid, kRedThreads, 0, st>>>(v, count, scratch));
    SFW_TRY(launch_check("k_sel_gather"));
    SFW_LAUNCH(st, "k_sel_final", k_sel_final<<<1, 64, 0, st>>>(topk, kSelGrid, scratch));
    SFW_TRY(launch_check("k_sel_final"));
    SFW_LAUNCH(st, "k_topk_decode", k_topk_decode<<<1, 64, 0, st>>>(scratch + kSelOut, topk, val_out, idx_out));
    return launch_check("k_topk_decode");
}

long long topk_scratch_keys(long long count, int topk) {
    const long long blocks = (count + kSortN - 1) / kSortN;
    const long long sorts = 2 * (blocks * topk + 64);
    return count > 65536 && sorts < kSelScratch ? kSelScratch : sorts;
}

sfw_status launch_topk(const float* v, long long count, int topk, unsigned long long* scratch,
                       long long scratch_len, float* val_out, int64_t* idx_out, cudaStream_t st) {
    // many values: radix selection (a few passes over the values instead of block sorts)
    if (count > 65536 && topk <= 64 && scratch_len >= kSelScratch)
        return launch_topk_select(v, count, topk, scratch, val_out, idx_out, st);
    // ping-pong halves of scratch
    long long blocks = (count + kSortN - 1) / kSortN;
    long long half = scratch_len / 2;
    if (blocks * topk > half) return fail(SFW_ERR_SHAPE, "topk scratch too small");
    unsigned long long* a = scratch;
    unsigned long long* b = scratch + half;
    SFW_LAUNCH(st, "k_topk_block", k_topk_block<<<(unsigned)blocks, kRedThreads, 0, st>>>(v, nullptr, count, topk, a));
    SFW_TRY(launch_check("k_topk_block"));
    long long n = blocks * topk;
    while (n > kSortN) {
        blocks = (n + kSortN - 1) / kSortN;
        SFW_LAUNCH(st, "k_topk_block", k_topk_block<<<(unsigned)blocks, kRedThreads, 0, st>>>(nullptr, a, n, topk, b));
        SFW_TRY(launch_check("k_topk_block"));
        n = blocks * topk;
        unsigned long long* t = a;
        a = b;
        b = t;
    }
    SFW_LAUNCH(st, "k_topk_block", k_topk_block<<<1, kRedThreads, 0, st>>>(nullptr, a, n, topk, b));
    SFW_TRY(launch_check("k_topk_block"));
    SFW_LAUNCH(st, "k_topk_decode", k_topk_decode<<<1, 64, 0, st>>>(b, topk, val_out, idx_out));
    return launch_check("k_topk_decode");
}

// ------------------------------------------------------------------ table statistics / conversion

__global__ void k_spec_stats(const float2* s, long long count, float* stats) {
    float re = 0.f, im = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        re = fmaxf(re, fabsf(s[i].x));
        im = fmaxf(im, fabsf(s[i].y));
    }
    for (int off = 16; off > 0; off >>= 1) {
        re = fmaxf(re, __shfl_down_sync(0xffffffffu, re, off));
        im = fmaxf(im, __shfl_down_sync(0xffffffffu, im, off));
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<unsigned int*>(stats), __float_as_uint(re));
        atomicMax(reinterpret_cast<unsigned int*>(stats) + 1, __float_as_uint(im));
    }
}

sfw_status launch_spec_stats(const float2* s, long long count, float* stats, cudaStream_t st) {
    SFW_LAUNCH(st, "k_spec_stats", k_spec_stats<<<1024, 256, 0, st>>>(s, count, stats));
    return launch_check("k_spec_stats");
}

__global__ void k_spec_convert(const float2* s, long long count, int kind, void* out, int rows,
                               long long nl, int group) {
    const long long per = (long long)rows * nl;
    const long long ng = group > 0 ? (nl + group - 1) / group : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = s[i];
        long long o = i;
        if (group > 0) {
            const long long k = i / per, rem = i - k * per;
            const long long j = rem / nl, l = rem - j * nl;
            o = ((k * ng + l / group) * rows + j) * group + l % group;
        }
        if (kind == SPEC_R32) reinterpret_cast<float*>(out)[o] = v.x;
        else if (kind == SPEC_CBF16) reinterpret_cast<__nv_bfloat162*>(out)[o] = __float22bfloat162_rn(v);
        else if (kind == SPEC_RBF16) reinterpret_cast<__nv_bfloat16*>(out)[o] = __float2bfloat16_rn(v.x);
        else reinterpret_cast<float2*>(out)[o] = v;
    }
}

sfw_status launch_spec_convert(const float2* s, long long count, int kind, void* out, int rows,
                               long long nl, int group, cudaStream_t st) {
    if (rows < 1 || nl < 1 || count % ((long long)rows * nl) != 0)
        return fail(SFW_ERR_SHAPE, "spec_convert: %lld values are not whole %d x %lld spectra", count, rows, nl);
    SFW_LAUNCH(st, "k_spec_convert", k_spec_convert<<<1024, 256, 0, st>>>(s, count, kind, out, rows, nl, group));
    return launch_check("k_spec_convert");
}

}  // namespace sfw
