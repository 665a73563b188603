// The blur Phi (Eq. 3) and its transpose (Eq. 5) with the passes along axes 1 and 2 done
// per slab of axis 0, so a slab stays on chip between the two axes (Section 2:
// convolutions in the Fourier domain).  Each slab belongs to a cluster of two CTAs that
// split its lines between them and exchange the transposed half through distributed
// shared memory: one CTA per slab would leave half of the SMs idle.
//
// Head (forward along axes 2 then 1): each CTA reads its half of the real slab's rows
// (odd row pitch); rows 2c and 2c + 1 form complex line c of the axis-2 transform
// (zero-padded to P2 at column offset o2); the two half spectra are split and written
// column-major into the CTA that owns the column (rank 0: columns [0, ceil(H2 / 2)),
// rank 1 the rest), so the axis-1 transform of every column (zero-padded to P1 at row
// offset o1) reads a contiguous line; each CTA stores its columns of the P1 x H2 result.
//
// Tail (inverse along axes 1 then 2): each CTA fetches its columns of the P1 x H2 slab
// (cp.async), inverts them along axis 1 and sends the kept rows [o1, o1 + m1) to the
// CTA that owns the row pair (rank 0: pairs [0, ceil(pairs / 2)), rank 1 the rest);
// pairs of rows are inverted along axis 2 as one complex line (Hermitian extension at
// the load); each CTA stores its rows' kept columns [o2, o2 + m2) (coalesced), or turns
// them into the residual r = y - value and the criterion C = 1/2 sum r^2 + lambda sum w
// (Eq. 4) by a last-block reduction over all CTAs; the y rows are fetched while the
// rows are transformed.
//
// The transforms are the shared-memory Stockham stages of the per-axis passes (two
// lines per warp); the slab form saves, per blur, two launches and the write and
// re-read of two (slabs, P1, H2)-sized intermediates.
#include <cooperative_groups.h>

#include "fft_core.cuh"

namespace sfw {

namespace cg = cooperative_groups;

// Warps per CTA: enough that every phase takes one round of two lines per warp, at
// most kSlabMaxWarps (the block size is chosen per launch).
constexpr int kSlabMaxWarps = 16;
constexpr int kSlabMaxThreads = 32 * kSlabMaxWarps;

__host__ __device__ inline int ev(int x) { return (x + 1) & ~1; }
// The two CTAs of a slab split a count n: rank 0 takes [0, ceil(n / 2)), rank 1 the rest.
__host__ __device__ inline int half_lo(int n, int r) { return r ? (n + 1) / 2 : 0; }
__host__ __device__ inline int half_hi(int n, int r) { return r ? n : (n + 1) / 2; }

// Complex line li of the axis-2 transform: local rows 2 li (real part) and 2 li + 1
// (imaginary part) of the real rows held, columns placed at [off, off + cols).
struct RowPairLoad {
    const float* RS;
    int NP, rows, cols, off;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        const int jj = j - off;
        if (jj < 0 || jj >= cols) return make_float2(0.f, 0.f);
        const int r0 = 2 * li, r1 = r0 + 1;
        return make_float2(r0 < rows ? RS[r0 * NP + jj] : 0.f, r1 < rows ? RS[r1 * NP + jj] : 0.f);
    }
};

// Column li of the column-major buffer, rows placed at [off, off + rows).
struct ColLoad {
    const float2* CB;
    int LS, off, rows;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        const int jj = j - off;
        return (jj >= 0 && jj < rows) ? CB[li * LS + phy(jj)] : make_float2(0.f, 0.f);
    }
};

// Column li (< n) of a row-major block of pitch `pitch`.
struct SlabColLoad {
    const float2* IS;
    int pitch, n;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        return li < n ? IS[j * pitch + li] : make_float2(0.f, 0.f);
    }
};

// Shared-memory layout of one CTA (the same in both CTAs of a slab: every buffer is
// sized for the larger half).
struct SlabLayout {
    int LS1, LS2, NP, NCA, NCAh, Hh, NC2, NC2h, HS, buf;
    size_t tw1, tw2, ba, bb, cb, rs, is, rb, total;   // float2 offsets and total
};

__host__ __device__ inline SlabLayout slab_layout(const SlabPass& p) {
    SlabLayout q;
    q.LS1 = pitch(p.P1);
    q.LS2 = pitch(p.P2);
    q.NP = p.cols | 1;
    q.NCA = (p.rows + 1) / 2;
    q.NCAh = (q.NCA + 1) / 2;
    q.Hh = (p.H2 + 1) / 2;
    q.NC2 = (p.m1 + 1) / 2;
    q.NC2h = (q.NC2 + 1) / 2;
    q.HS = (p.H2 + 1) | 1;
    if (p.mode == SLAB_HEAD) {
        // warps transform lines in pairs: every line buffer holds an even count
        const int a = ev(q.NCAh) * q.LS2, b = ev(q.Hh) * q.LS1;
        q.buf = a > b ? a : b;
        q.tw1 = 0;
        q.tw2 = q.tw1 + p.P1;
        q.ba = q.tw2 + p.P2;
        q.bb = q.ba + q.buf;
        q.cb = q.bb + q.buf;
        q.rs = q.cb + (size_t)ev(q.Hh) * q.LS1;
        q.is = q.rb = 0;
        q.total = q.rs + ((size_t)2 * q.NCAh * q.NP + 1) / 2;
    } else {
        const int a = ev(q.Hh) * q.LS1, b = ev(q.NC2h) * q.LS2;
        q.buf = a > b ? a : b;
        // the input columns, later the observation rows (2 NC2h x m2 floats)
        const size_t in_el = (size_t)p.P1 * q.Hh, y_el = (size_t)q.NC2h * p.m2;
        q.is = 0;
        q.tw1 = q.is + (in_el > y_el ? in_el : y_el);
        q.tw2 = q.tw1 + p.P1;
        q.ba = q.tw2 + p.P2;
        q.bb = q.ba + q.buf;
        q.rb = q.bb + q.buf;
        q.cb = q.rs = 0;
        q.total = q.rb + (size_t)2 * ev(q.NC2h) * q.HS;
    }
    return q;
}

template <int LL1, int LL2>
__device__ __forceinline__ void slab_head_body(const SlabPass& p, int slab, int rank) {
    const int L1 = LL1 > 0 ? LL1 : p.P1, L2 = LL2 > 0 ? LL2 : p.P2;
    const int H2 = p.H2, rows = p.rows, cols = p.cols;
    const SlabLayout q = slab_layout(p);
    extern __shared__ float4 smem_raw[];
    float2* base = reinterpret_cast<float2*>(smem_raw);
    float2* TW1 = base + q.tw1;
    float2* TW2 = base + q.tw2;
    float2* BA = base + q.ba;
    float2* BB = base + q.bb;
    float2* CB = base + q.cb;
    float* RS = reinterpret_cast<float*>(base + q.rs);
    __shared__ int s_res;
    cg::cluster_group cluster = cg::this_cluster();
    float2* CBp = cluster.map_shared_rank(CB, rank ^ 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5, nt = blockDim.x;
    const int c_lo = half_lo(q.NCA, rank), nc = half_hi(q.NCA, rank) - c_lo;   // complex lines
    const int k_lo = half_lo(H2, rank), nk = half_hi(H2, rank) - k_lo;         // columns
    const int h0 = half_hi(H2, 0);                                             // rank 1's first column
    const int r_lo = 2 * c_lo;
    const int nrows = max(0, min(rows, r_lo + 2 * nc) - r_lo);
    for (int j = threadIdx.x; j < L1; j += nt) TW1[j] = p.tw1[j];
    for (int j = threadIdx.x; j < L2; j += nt) TW2[j] = p.tw2[j];
    {   // every element in flight at once (asynchronous copies)
        const float* src = p.rin + ((long long)slab * rows + r_lo) * cols;
        for (int e = threadIdx.x; e < nrows * cols; e += nt) {
            const int i = e / cols;
            cp_async(RS + i * q.NP + (e - i * cols), src + e, 4);
        }
        cp_async_commit();
    }
    cp_async_wait0();
    cluster.sync();   // also: the other CTA has started before its shared memory is written
    // axis 2: two real rows per complex line; their half spectra go to the column's owner
    for (int lc0 = 2 * warp; lc0 < nc; lc0 += 2 * nwarps) {
        const float2* res = line_fft<-1, LL2, 2>(BA, BB, L2, q.LS2, lc0, p.fac2, TW2,
                                                 RowPairLoad{RS, q.NP, nrows, cols, p.o2});
        for (int e = lane; e < 2 * H2; e += 32) {
            const int h = e / H2, k = e - h * H2;
            const int lc = lc0 + h;
            if (lc >= nc) continue;
            const int c = c_lo + lc;
            const float2 z = res[lc * q.LS2 + phy(k)];
            const float2 zm = res[lc * q.LS2 + phy((L2 - k) % L2)];
            const bool hi = k >= h0;
            float2* dst = (hi == (rank == 1)) ? CB : CBp;
            const int kk = hi ? k - h0 : k;
            dst[kk * q.LS1 + phy(2 * c)] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            if (2 * c + 1 < rows)
                dst[kk * q.LS1 + phy(2 * c + 1)] = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
        }
    }
    cluster.sync();
    // axis 1: this CTA's columns (rows at [o1, o1 + rows), zero elsewhere)
    const float2* res1 = BA;
    for (int lk0 = 2 * warp; lk0 < nk; lk0 += 2 * nwarps)
        res1 = line_fft<-1, LL1, 2>(BA, BB, L1, q.LS1, lk0, p.fac1, TW1, ColLoad{CB, q.LS1, p.o1, rows});
    if (threadIdx.x == 0) s_res = (res1 == BA) ? 0 : 1;   // warp 0 always has a column
    __syncthreads();
    const float2* R = s_res ? BB : BA;
    float2* dst = p.cout + (long long)slab * L1 * H2 + k_lo;
    for (int e = threadIdx.x; e < L1 * nk; e += nt) {
        const int p1 = e / nk, kk = e - p1 * nk;
        dst[(long long)p1 * H2 + kk] = R[kk * q.LS1 + phy(p1)];
    }
}

template <int LL1, int LL2, int MODE>
__device__ __forceinline__ void slab_tail_body(const SlabPass& p, int slab, int rank) {
    const int L1 = LL1 > 0 ? LL1 : p.P1, L2 = LL2 > 0 ? LL2 : p.P2;
    const int H2 = p.H2, m1 = p.m1, m2 = p.m2;
    const SlabLayout q = slab_layout(p);
    extern __shared__ float4 smem_raw[];
    float2* base = reinterpret_cast<float2*>(smem_raw);
    float2* IS = base + q.is;
    float2* TW1 = base + q.tw1;
    float2* TW2 = base + q.tw2;
    float2* BA = base + q.ba;
    float2* BB = base + q.bb;
    float2* RB = base + q.rb;
    float* YS = reinterpret_cast<float*>(IS);   // the observation rows, once IS is consumed
    __shared__ double s_red[32];
    __shared__ int s_res;
    cg::cluster_group cluster = cg::this_cluster();
    float2* RBp = cluster.map_shared_rank(RB, rank ^ 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5, nt = blockDim.x;
    const int k_lo = half_lo(H2, rank), nk = half_hi(H2, rank) - k_lo;         // columns
    const int c_lo = half_lo(q.NC2, rank), nc = half_hi(q.NC2, rank) - c_lo;   // row pairs
    const int p0 = half_hi(q.NC2, 0);                                          // rank 1's first pair
    const int r_lo = 2 * c_lo;
    const int nrows = max(0, min(m1, r_lo + 2 * nc) - r_lo);
    {
        const float2* src = p.cin + (long long)slab * L1 * H2 + k_lo;
        for (int e = threadIdx.x; e < L1 * nk; e += nt) {
            const int j = e / nk, kk = e - j * nk;
            cp_async(IS + j * q.Hh + kk, src + (long long)j * H2 + kk, 8);
        }
        cp_async_commit();
    }
    for (int j = threadIdx.x; j < L1; j += nt) TW1[j] = p.tw1[j];
    for (int j = threadIdx.x; j < L2; j += nt) TW2[j] = p.tw2[j];
    if ((m1 & 1) && nc > 0 && c_lo + nc == q.NC2)   // the second row of the last pair
        for (int k = threadIdx.x; k < H2; k += nt) RB[(m1 - r_lo) * q.HS + k] = make_float2(0.f, 0.f);
    cp_async_wait0();
    cluster.sync();   // also: the other CTA has started before its shared memory is written
    // axis 1 inverse of this CTA's columns; row i of [o1, o1 + m1) goes to its pair's owner
    for (int lk0 = 2 * warp; lk0 < nk; lk0 += 2 * nwarps) {
        const float2* res = line_fft<1, LL1, 2>(BA, BB, L1, q.LS1, lk0, p.fac1, TW1,
                                                SlabColLoad{IS, q.Hh, nk});
        for (int e = lane; e < 2 * m1; e += 32) {
            const int h = e / m1, i = e - h * m1;
            const int lk = lk0 + h;
            if (lk >= nk) continue;
            const bool hi = (i >> 1) >= p0;
            float2* dst = (hi == (rank == 1)) ? RB : RBp;
            dst[(hi ? i - 2 * p0 : i) * q.HS + k_lo + lk] = res[lk * q.LS1 + phy(i + p.o1)];
        }
    }
    cluster.sync();
    if constexpr (MODE == SLAB_RESIDUAL) {   // y travels while the rows are transformed
        const float* ys = p.y + ((long long)slab * m1 + r_lo) * m2;
        for (int e = threadIdx.x; e < nrows * m2; e += nt) cp_async(YS + e, ys + e, 4);
        cp_async_commit();
    }
    // axis 2 real inverse of this CTA's row pairs (every pair keeps its own line of BA / BB)
    const float2* z = BA;
    for (int lc0 = 2 * warp; lc0 < nc; lc0 += 2 * nwarps)
        z = line_fft<1, LL2, 2>(BA, BB, L2, q.LS2, lc0, p.fac2, TW2, HermLoad{RB, q.HS, L2});
    if (threadIdx.x == 0) s_res = (z == BA) ? 0 : 1;   // warp 0 has pair 0 whenever nc > 0
    if constexpr (MODE == SLAB_RESIDUAL) cp_async_wait0();
    __syncthreads();
    // kept columns [o2, o2 + m2) of this CTA's rows, coalesced
    const float2* Z = s_res ? BB : BA;
    double acc = 0.0;
    const long long o0 = ((long long)slab * m1 + r_lo) * m2;
    for (int e = threadIdx.x; e < nrows * m2; e += nt) {
        const int lr = e / m2, j = e - lr * m2;
        const float2 zz = Z[(lr >> 1) * q.LS2 + phy(j + p.o2)];
        const float v = (lr & 1) ? zz.y : zz.x;
        if constexpr (MODE == SLAB_STORE) {
            p.rout[o0 + e] = v;
        } else {
            const float r = YS[e] - v;
            if (p.rout) p.rout[o0 + e] = r;
            acc += (double)r * (double)r;
        }
    }
    if constexpr (MODE == SLAB_RESIDUAL) {
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) s_red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            p.partials[2 * slab + rank] = t;
        }
        // the last CTA to finish forms C = 1/2 sum r^2 + lambda sum w (fixed order)
        const int nparts = 2 * p.nslab;
        if (p.loss_out && last_block(p.counter, nparts)) {
            double a = 0.0;
            for (int i = threadIdx.x; i < nparts; i += nt) a += __ldcg(p.partials + i);
            double ws = 0.0;
            for (int i = threadIdx.x; i < p.nw; i += nt) ws += (double)__ldg(p.w + (long long)i * p.w_stride);
            double v = 0.5 * a + p.lambda * ws;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) s_red[warp] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int w = 0; w < nwarps; ++w) t += s_red[w];
                *p.loss_out = t;
                *p.counter = 0u;
            }
        }
    }
}

template <int LL1, int LL2>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kSlabMaxThreads) k_slab_head(SlabPass p) {
    slab_head_body<LL1, LL2>(p, blockIdx.x >> 1, (int)cg::this_cluster().block_rank());
}

template <int LL1, int LL2, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kSlabMaxThreads) k_slab_tail(SlabPass p) {
    slab_tail_body<LL1, LL2, MODE>(p, blockIdx.x >> 1, (int)cg::this_cluster().block_rank());
}

// Grouped launches (batches): cluster t runs slab t - start[q] of pass q (both CTAs of a
// cluster take the same slabs, so their cluster barriers match).
template <int LL1, int LL2>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kSlabMaxThreads)
    k_slab_head_g(const SlabPass* __restrict__ ps, const int* __restrict__ start, int n) {
    const int total = start[n], rank = (int)cg::this_cluster().block_rank();
    for (int t = blockIdx.x >> 1; t < total; t += gridDim.x >> 1) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        slab_head_body<LL1, LL2>(ps[q], t - start[q], rank);
        __syncthreads();
    }
}

template <int LL1, int LL2, int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kSlabMaxThreads)
    k_slab_tail_g(const SlabPass* __restrict__ ps, const int* __restrict__ start, int n) {
    const int total = start[n], rank = (int)cg::this_cluster().block_rank();
    for (int t = blockIdx.x >> 1; t < total; t += gridDim.x >> 1) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        slab_tail_body<LL1, LL2, MODE>(ps[q], t - start[q], rank);
        __syncthreads();
    }
}

int slab_warps(const SlabPass& p) {
    const SlabLayout q = slab_layout(p);
    const int lines = p.mode == SLAB_HEAD ? (q.NCAh > q.Hh ? q.NCAh : q.Hh) : (q.NC2h > q.Hh ? q.NC2h : q.Hh);
    const int warps = (lines + 1) / 2;
    return warps < 4 ? 4 : warps > kSlabMaxWarps ? kSlabMaxWarps : warps;
}

template <typename Single, typename Grouped>
static sfw_status run_slab(Single ks, Grouped kg, const SlabPass& p, size_t smem, cudaStream_t st,
                           GroupArgs* g) {
    const int warps = p.warps > 0 ? p.warps : slab_warps(p);
    if (!g) {
        SFW_TRY(prepare(ks, smem));
        SFW_LAUNCH(st, "k_slab", (ks<<<2 * p.nslab, 32 * warps, smem, st>>>(p)));
    } else {
        SFW_TRY(prepare(kg, smem));
        if (g->grid <= 0) g->grid = g->total;   // clusters: one per slab of the group
        if (g->total <= 0) return SFW_OK;
        SFW_LAUNCH(st, "k_slab", (kg<<<2 * g->grid, 32 * warps, smem, st>>>(
                                     reinterpret_cast<const SlabPass*>(g->passes), g->start, g->n)));
    }
    return launch_check("k_slab");
}

template <int LL1, int LL2>
static sfw_status run_slab_len(const SlabPass& p, size_t smem, cudaStream_t st, GroupArgs* g) {
    if (p.mode == SLAB_HEAD) return run_slab(k_slab_head<LL1, LL2>, k_slab_head_g<LL1, LL2>, p, smem, st, g);
    if (p.mode == SLAB_STORE)
        return run_slab(k_slab_tail<LL1, LL2, SLAB_STORE>, k_slab_tail_g<LL1, LL2, SLAB_STORE>, p, smem, st, g);
    return run_slab(k_slab_tail<LL1, LL2, SLAB_RESIDUAL>, k_slab_tail_g<LL1, LL2, SLAB_RESIDUAL>, p, smem, st, g);
}

size_t slab_smem(const SlabPass& p) {
    const SlabLayout q = slab_layout(p);
    const size_t bytes = sizeof(float2) * q.total;
    return bytes <= (size_t)220 * 1024 ? bytes : 0;
}

// Compile-time lengths: the 64^3 blur grid (80 x 96 on axes 1-2) and the 128^3 one (144 x 160).
bool slab_specialised(const SlabPass& p) { return (p.P1 == 80 && p.P2 == 96) || (p.P1 == 144 && p.P2 == 160); }

sfw_status launch_slab(const SlabPass& p0, cudaStream_t st, GroupArgs* g) {
    SlabPass p = p0;
    if (!g && p.nslab < 1) return SFW_OK;
    if (p.H2 != p.P2 / 2 + 1 || (p.P1 & 1)) return fail(SFW_ERR_SHAPE, "slab pass: bad lengths");
    size_t smem = slab_smem(p);
    if (!smem) return fail(SFW_ERR_SHAPE, "slab pass: %d x %d does not fit shared memory", p.P1, p.P2);
    if ((size_t)p.smem > smem) smem = (size_t)p.smem;
    if (!g) {   // factors and twiddles (a grouped launch takes every pass's own from its descriptor)
        const int mr1 = max_radix(p.P1, 2), mr2 = max_radix(p.P2, 2);
        if (!factorize(p.P1, &p.fac1, mr1) || !factorize(p.P2, &p.fac2, mr2))
            return fail(SFW_ERR_SHAPE, "slab pass: cannot factor %d x %d", p.P1, p.P2);
        SFW_TRY(twiddle_table(p.P1, mr1, &p.tw1));
        SFW_TRY(twiddle_table(p.P2, mr2, &p.tw2));
        if (g_recorder) return g_recorder->add(p);
    }
    if (p.P1 == 80 && p.P2 == 96) return run_slab_len<80, 96>(p, smem, st, g);
    if (p.P1 == 144 && p.P2 == 160) return run_slab_len<144, 160>(p, smem, st, g);
    return run_slab_len<0, 0>(p, smem, st, g);
}

}  // namespace sfw
