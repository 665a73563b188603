// The blur Phi (Eq. 3) and its transpose (Eq. 5) with the passes along axes 1 and 2 done
// per slab of axis 0, one CTA per slab, so a slab stays in shared memory between the
// two axes (Section 2: convolutions in the Fourier domain).
//
// Head (forward along axes 2 then 1): the real slab (rows x cols, odd row pitch) is read
// once; rows 2c and 2c + 1 form complex line c of the axis-2 transform (zero-padded to
// P2 at column offset o2); the two half spectra are split and written column-major, so
// the axis-1 transform of every column (zero-padded to P1 at row offset o1) reads a
// contiguous line; the P1 x H2 result leaves with coalesced stores.  Tail (inverse along
// axes 1 then 2): the P1 x H2 slab arrives by 16-byte cp.async; every column's inverse
// keeps rows [o1, o1 + m1) into a row buffer (odd pitch); pairs of rows are inverted
// along axis 2 as one complex line (Hermitian extension at the load); then the whole
// block stores the kept columns [o2, o2 + m2) row by row (coalesced), or turns them into
// the residual r = y - value and the criterion C = 1/2 sum r^2 + lambda sum w (Eq. 4) by
// a last-block reduction; the y slab is fetched into the consumed input buffer while
// the rows are transformed.
//
// The transforms are the shared-memory Stockham stages of the per-axis passes (two
// lines per warp); the slab form saves, per blur, two launches and the write and
// re-read of two (slabs, P1, H2)-sized intermediates.
#include "fft_core.cuh"

namespace sfw {

// Warps per CTA: enough that every phase takes one round of two lines per warp, at
// most kSlabMaxWarps (the block size is chosen per launch).
constexpr int kSlabMaxWarps = 25;
constexpr int kSlabMaxThreads = 32 * kSlabMaxWarps;

// Complex line li of the axis-2 transform: rows 2 li (real part) and 2 li + 1 (imaginary
// part) of the real slab, columns placed at [off, off + cols).
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

// Column li of a row-major slab of pitch H2.
struct SlabColLoad {
    const float2* IS;
    int H2;
    __device__ __forceinline__ float2 operator()(int li, int j) const {
        return li < H2 ? IS[j * H2 + li] : make_float2(0.f, 0.f);
    }
};

struct SlabLayout {
    int LS1, LS2, NP, NCA, NC2, HS, buf;
    size_t tw1, tw2, ba, bb, cb, rs, is, rb, total;   // float2 offsets and total
};

__host__ __device__ inline int ev(int x) { return (x + 1) & ~1; }

__host__ __device__ inline SlabLayout slab_layout(const SlabPass& p) {
    SlabLayout q;
    q.LS1 = pitch(p.P1);
    q.LS2 = pitch(p.P2);
    q.NP = p.cols | 1;
    q.NCA = (p.rows + 1) / 2;
    q.NC2 = (p.m1 + 1) / 2;
    q.HS = (p.H2 + 1) | 1;
    if (p.mode == SLAB_HEAD) {
        // warps transform lines in pairs: every line buffer holds an even count
        const int a = ev(q.NCA) * q.LS2, b = ev(p.H2) * q.LS1;
        q.buf = a > b ? a : b;
        q.tw1 = 0;
        q.tw2 = q.tw1 + p.P1;
        q.ba = q.tw2 + p.P2;
        q.bb = q.ba + q.buf;
        q.cb = q.bb + q.buf;
        q.rs = q.cb + (size_t)ev(p.H2) * q.LS1;
        q.is = q.rb = 0;
        q.total = q.rs + ((size_t)p.rows * q.NP + 1) / 2;
    } else {
        const int a = ev(p.H2) * q.LS1, b = ev(q.NC2) * q.LS2;
        q.buf = a > b ? a : b;
        q.is = 0;
        q.tw1 = q.is + (size_t)p.P1 * p.H2;
        q.tw2 = q.tw1 + p.P1;
        q.ba = q.tw2 + p.P2;
        q.bb = q.ba + q.buf;
        q.rb = q.bb + q.buf;
        q.cb = q.rs = 0;
        q.total = q.rb + (size_t)2 * ev(q.NC2) * q.HS;
    }
    return q;
}

template <int LL1, int LL2>
__device__ __forceinline__ void slab_head_body(const SlabPass& p, int slab) {
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
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5, nt = blockDim.x;
    for (int j = threadIdx.x; j < L1; j += nt) TW1[j] = p.tw1[j];
    for (int j = threadIdx.x; j < L2; j += nt) TW2[j] = p.tw2[j];
    {
        const float* src = p.rin + (long long)slab * rows * cols;
        for (int e = threadIdx.x; e < rows * cols; e += nt) {
            const int i = e / cols;
            RS[i * q.NP + (e - i * cols)] = __ldg(src + e);
        }
    }
    __syncthreads();
    // axis 2: two real rows per complex line, then their half spectra into columns of CB
    for (int c0 = 2 * warp; c0 < q.NCA; c0 += 2 * nwarps) {
        const float2* res = line_fft<-1, LL2, 2>(BA, BB, L2, q.LS2, c0, p.fac2, TW2,
                                                 RowPairLoad{RS, q.NP, rows, cols, p.o2});
        for (int e = lane; e < 2 * H2; e += 32) {
            const int h = e / H2, k = e - h * H2;
            const int c = c0 + h;
            if (c >= q.NCA) continue;
            const float2 z = res[c * q.LS2 + phy(k)];
            const float2 zm = res[c * q.LS2 + phy((L2 - k) % L2)];
            CB[k * q.LS1 + phy(2 * c)] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            if (2 * c + 1 < rows)
                CB[k * q.LS1 + phy(2 * c + 1)] = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
        }
    }
    __syncthreads();
    // axis 1: every column (rows at [o1, o1 + rows), zero elsewhere)
    const float2* res1 = BA;
    for (int k0 = 2 * warp; k0 < H2; k0 += 2 * nwarps)
        res1 = line_fft<-1, LL1, 2>(BA, BB, L1, q.LS1, k0, p.fac1, TW1, ColLoad{CB, q.LS1, p.o1, rows});
    if (threadIdx.x == 0) s_res = (res1 == BA) ? 0 : 1;   // warp 0 always has column 0
    __syncthreads();
    const float2* R = s_res ? BB : BA;
    float2* dst = p.cout + (long long)slab * L1 * H2;
    for (int e = threadIdx.x; e < L1 * H2; e += nt) {
        const int p1 = e / H2, k = e - p1 * H2;
        dst[e] = R[k * q.LS1 + phy(p1)];
    }
}

template <int LL1, int LL2, int MODE>
__device__ __forceinline__ void slab_tail_body(const SlabPass& p, int slab) {
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
    float* YS = reinterpret_cast<float*>(IS);   // the observation slab, once IS is consumed
    __shared__ double s_red[32];
    __shared__ int s_res;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5, nt = blockDim.x;
    {
        const float2* src = p.cin + (long long)slab * L1 * H2;
        for (int e = threadIdx.x; e < L1 * H2 / 2; e += nt) cp_async16(IS + 2 * e, src + 2 * e);
        cp_async_commit();
    }
    for (int j = threadIdx.x; j < L1; j += nt) TW1[j] = p.tw1[j];
    for (int j = threadIdx.x; j < L2; j += nt) TW2[j] = p.tw2[j];
    if (m1 & 1)   // the last row pair's second row
        for (int k = threadIdx.x; k < H2; k += nt) RB[m1 * q.HS + k] = make_float2(0.f, 0.f);
    cp_async_wait0();
    __syncthreads();
    // axis 1 inverse of every column, rows [o1, o1 + m1) into RB (row-major, pitch HS)
    for (int k0 = 2 * warp; k0 < H2; k0 += 2 * nwarps) {
        const float2* res = line_fft<1, LL1, 2>(BA, BB, L1, q.LS1, k0, p.fac1, TW1, SlabColLoad{IS, H2});
        for (int e = lane; e < 2 * m1; e += 32) {
            const int h = e / m1, i = e - h * m1;
            const int k = k0 + h;
            if (k < H2) RB[i * q.HS + k] = res[k * q.LS1 + phy(i + p.o1)];
        }
    }
    __syncthreads();
    if constexpr (MODE == SLAB_RESIDUAL) {   // y travels while the rows are transformed
        const float* ys = p.y + (long long)slab * m1 * m2;
        for (int e = threadIdx.x; e < m1 * m2; e += nt) cp_async(YS + e, ys + e, 4);
        cp_async_commit();
    }
    // axis 2 real inverse of row pairs (every pair keeps its own line of BA / BB)
    const float2* z = BA;
    for (int c0 = 2 * warp; c0 < q.NC2; c0 += 2 * nwarps)
        z = line_fft<1, LL2, 2>(BA, BB, L2, q.LS2, c0, p.fac2, TW2, HermLoad{RB, q.HS, L2});
    if (threadIdx.x == 0) s_res = (z == BA) ? 0 : 1;   // warp 0 always has pair 0
    if constexpr (MODE == SLAB_RESIDUAL) cp_async_wait0();
    __syncthreads();
    // kept columns [o2, o2 + m2) of every row, coalesced over the slab
    const float2* Z = s_res ? BB : BA;
    double acc = 0.0;
    const long long o0 = (long long)slab * m1 * m2;
    for (int e = threadIdx.x; e < m1 * m2; e += nt) {
        const int row = e / m2, j = e - row * m2;
        const float2 zz = Z[(row >> 1) * q.LS2 + phy(j + p.o2)];
        const float v = (row & 1) ? zz.y : zz.x;
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
            p.partials[slab] = t;
        }
        // the last slab to finish forms C = 1/2 sum r^2 + lambda sum w (fixed order)
        if (p.loss_out && last_block(p.counter, p.nslab)) {
            __syncthreads();
            double a = 0.0;
            for (int i = threadIdx.x; i < p.nslab; i += nt) a += __ldcg(p.partials + i);
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
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab_head(SlabPass p) {
    slab_head_body<LL1, LL2>(p, blockIdx.x);
}

template <int LL1, int LL2, int MODE>
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab_tail(SlabPass p) {
    slab_tail_body<LL1, LL2, MODE>(p, blockIdx.x);
}

// Grouped launches (batches): CTA t runs slab t - start[q] of pass q.
template <int LL1, int LL2>
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab_head_g(const SlabPass* __restrict__ ps,
                                                                 const int* __restrict__ start, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        slab_head_body<LL1, LL2>(ps[q], t - start[q]);
        __syncthreads();
    }
}

template <int LL1, int LL2, int MODE>
__global__ void __launch_bounds__(kSlabMaxThreads) k_slab_tail_g(const SlabPass* __restrict__ ps,
                                                                 const int* __restrict__ start, int n) {
    const int total = start[n];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int q = 0;
        while (start[q + 1] <= t) ++q;
        slab_tail_body<LL1, LL2, MODE>(ps[q], t - start[q]);
        __syncthreads();
    }
}

int slab_warps(const SlabPass& p) {
    const SlabLayout q = slab_layout(p);
    const int lines = p.mode == SLAB_HEAD ? (q.NCA > p.H2 ? q.NCA : p.H2) : (q.NC2 > p.H2 ? q.NC2 : p.H2);
    const int warps = (lines + 1) / 2;
    return warps < 8 ? 8 : warps > kSlabMaxWarps ? kSlabMaxWarps : warps;
}

template <typename Single, typename Grouped>
static sfw_status run_slab(Single ks, Grouped kg, const SlabPass& p, size_t smem, cudaStream_t st,
                           GroupArgs* g) {
    const int warps = p.warps > 0 ? p.warps : slab_warps(p);
    if (!g) {
        SFW_TRY(prepare(ks, smem));
        SFW_LAUNCH(st, "k_slab", (ks<<<p.nslab, 32 * warps, smem, st>>>(p)));
    } else {
        SFW_TRY(prepare(kg, smem));
        if (g->grid <= 0) g->grid = g->total;   // one CTA per slab of the group
        if (g->total <= 0) return SFW_OK;
        SFW_LAUNCH(st, "k_slab", (kg<<<g->grid, 32 * warps, smem, st>>>(
                                     reinterpret_cast<const SlabPass*>(g->passes), g->start, g->n)));
    }
    return launch_check("k_slab");
}

size_t slab_smem(const SlabPass& p) {
    const SlabLayout q = slab_layout(p);
    const size_t bytes = sizeof(float2) * q.total;
    return bytes <= (size_t)220 * 1024 ? bytes : 0;
}

bool slab_specialised(const SlabPass& p) { return p.P1 == 80 && p.P2 == 96; }

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
    const bool spec = slab_specialised(p);
    if (p.mode == SLAB_HEAD)
        return spec ? run_slab(k_slab_head<80, 96>, k_slab_head_g<80, 96>, p, smem, st, g)
                    : run_slab(k_slab_head<0, 0>, k_slab_head_g<0, 0>, p, smem, st, g);
    if (p.mode == SLAB_STORE)
        return spec ? run_slab(k_slab_tail<80, 96, SLAB_STORE>, k_slab_tail_g<80, 96, SLAB_STORE>, p, smem, st, g)
                    : run_slab(k_slab_tail<0, 0, SLAB_STORE>, k_slab_tail_g<0, 0, SLAB_STORE>, p, smem, st, g);
    return spec ? run_slab(k_slab_tail<80, 96, SLAB_RESIDUAL>, k_slab_tail_g<80, 96, SLAB_RESIDUAL>, p, smem, st, g)
                : run_slab(k_slab_tail<0, 0, SLAB_RESIDUAL>, k_slab_tail_g<0, 0, SLAB_RESIDUAL>, p, smem, st, g);
}

}  // namespace sfw
