// Batched 1-D FFT passes in shared memory (mixed radix 8/4/2/3/5, Stockham
// autosort), the building block of every convolution of the hot path:
// the blur Phi (Eq. 3), its transpose (Eq. 5) and the certificate
// correlation against the kernel-family table (Section 2: "convolutions are
// made in Fourier domain").
//
// A CTA owns a tile of W lines (W a multiple of 8).  Shared memory holds the
// tile line-major with one padding slot every 16 points and an odd line pitch
// (see phy / pitch), so strided stage writes and cross-line row accesses avoid
// bank conflicts.  Tiles arrive by cp.async (no register round trip).  The CTA
// loads and stores the tile cooperatively (rows of W lines for strided axes,
// whole lines for the contiguous axis); in between, each warp owns W / 8 lines
// and runs the butterfly stages on them alone, with __syncwarp between stages.
// Radix-R stages read R points L/R apart and write them Ns apart (Stockham), so
// no bit reversal is needed.  The first stage reads its inputs through a
// functor, which fuses the spectrum multiply of a convolution or the Hermitian
// rebuild of a real inverse transform into it.
#include <math.h>
#include <stdio.h>

#include <map>
#include <mutex>
#include <tuple>

#include "fft_core.cuh"

namespace sfw {

// ------------------------------------------------------------------ host helpers

// Largest power-of-two radix that still gives every lane of a warp a butterfly
// when a warp owns nl lines of length L: (L / R) nl >= 32.
int max_radix(int L, int nl) {
    int r = 16;
    while (r > 2 && (L / r) * nl < 32) r >>= 1;
    return r;
}

bool factorize(int L, Factors* f, int maxr) {
    f->n = 0;
    if (L < 1 || L > kMaxLen) return false;
    const int radices[6] = {16, 8, 4, 2, 3, 5};
    for (int q = 0; q < 6; ++q) {
        int r = radices[q];
        if (r <= 16 && (r & (r - 1)) == 0 && r > maxr) continue;
        while (L % r == 0 && L > 1) {
            if (f->n >= kMaxFactors) return false;
            f->r[f->n++] = r;
            L /= r;
        }
    }
    return L == 1;
}

int next_smooth_even(int x) {
    if (x < 2) x = 2;
    for (int v = x + (x & 1);; v += 2) {
        int t = v;
        while (t % 2 == 0) t /= 2;
        while (t % 3 == 0) t /= 3;
        while (t % 5 == 0) t /= 5;
        if (t == 1) return v;
    }
}

// Radix of the first stage of the register-resident transforms (0: not one of their lengths).
static int reg_first_radix(int L) { return L == 64 ? 8 : (L == 128 || L == 256) ? 16 : 0; }

namespace {
std::mutex g_tw_mu;
std::map<std::tuple<int, int, int>, float2*> g_tw;  // (device, L, max radix) -> table
}  // namespace

// Per-stage twiddles in the order of the Stockham stages of factorize(L, maxr):
// stage s (radix R, Ns = product of the earlier radices) stores
// exp(-2 pi i k r / (Ns R)) at (Ns - 1) + (r - 1) Ns + k, r = 1..R-1, k < Ns (the
// stages telescope to L - 1 entries), so that the lanes of a warp read
// consecutive entries.  Tables live until process exit.
sfw_status twiddle_table(int L, int maxr, const float2** out) {
    int dev = 0;
    SFW_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto key = std::make_tuple(dev, L, maxr);
    auto it = g_tw.find(key);
    if (it != g_tw.end()) {
        *out = it->second;
        return SFW_OK;
    }
    Factors fac;
    if (!factorize(L, &fac, maxr)) return fail(SFW_ERR_SHAPE, "cannot factor %d", L);
    std::vector<float2> h(L, make_float2(1.f, 0.f));
    const double two_pi = 6.283185307179586476925286766559;
    int Ns = 1;
    for (int st = 0; st < fac.n; ++st) {
        const int R = fac.r[st];
        for (int r = 1; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                const double a = -two_pi * (double)k * (double)r / ((double)Ns * (double)R);
                h[(Ns - 1) + (r - 1) * Ns + k] = make_float2((float)cos(a), (float)sin(a));
            }
        Ns *= R;
    }
    float2* d = nullptr;
    if (cudaMalloc(&d, sizeof(float2) * L) != cudaSuccess) {
        cudaGetLastError();
        return fail(SFW_ERR_ALLOC, "twiddle table");
    }
    cudaError_t e = cudaMemcpy(d, h.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "twiddle upload");
    }
    g_tw[key] = d;
    *out = d;
    return SFW_OK;
}

// Make the tables of length L for every tile width a pass of that length can
// use (so that launches, and stream captures, never allocate).
sfw_status TwiddleCache::get(int L, const float2** out) {
    if (reg_first_radix(L)) {
        const float2* t = nullptr;
        SFW_TRY(twiddle_table(L, reg_first_radix(L), &t));
    }
    const int ws[2] = {8, 16};
    for (int q = 0; q < 2; ++q) {
        const float2* t = nullptr;
        SFW_TRY(twiddle_table(L, max_radix(L, ws[q] / 8), &t));
        if (ws[q] == tile_width(L)) *out = t;
    }
    if (tile_width(L) != 8 && tile_width(L) != 16) return fail(SFW_ERR_SHAPE, "tile width");
    return SFW_OK;
}

void TwiddleCache::release() { tables.clear(); }

// The factors and twiddles of a pass follow the lines each warp owns (W / 8);
// passes on the register-resident path use the factorisation R1 x T.
static sfw_status fit_factors(int L, int W, Factors* fac, const float2** tw, bool reg = false) {
    const int mr = (reg && reg_first_radix(L)) ? reg_first_radix(L) : max_radix(L, W / 8);
    if (!factorize(L, fac, mr)) return fail(SFW_ERR_SHAPE, "cannot factor %d", L);
    return twiddle_table(L, mr, tw);
}

// ------------------------------------------------------------------ length dispatch

// Lengths with compile-time specialisations (fft_len_*.cu); others run generic code.
#define SFW_FFT_LENGTHS(X) X(64) X(80) X(96) X(128) X(144) X(160) X(192) X(256)
SFW_FFT_DECLARE(0)
#define SFW_DECL(LL) SFW_FFT_DECLARE(LL)
SFW_FFT_LENGTHS(SFW_DECL)
#undef SFW_DECL

bool fft_specialised(int L) {
    switch (L) {
#define SFW_CASE(LL) case LL: return true;
        SFW_FFT_LENGTHS(SFW_CASE)
#undef SFW_CASE
        default: return false;
    }
}

// Lines per CTA: 16 up to length 256, else 8 (shared memory).
int tile_width(int L) { return L <= 256 ? 16 : 8; }

int reg_line_group(int L) { return (L == 64 || L == 128) ? 4 : L == 256 ? 2 : 0; }

void pass_tiles(const C2CPass& p, int* W, int* nbx, int* nby) {
    *W = tile_width(p.L);
    *nbx = (int)((p.nlines + *W - 1) / *W);
    *nby = 1;
}

void pass_tiles(const MulPass& p, int* W, int* nbx, int* nby) {
    *W = tile_width(p.L);
    *nbx = (int)((p.nlines + *W - 1) / *W);
    *nby = (p.ktotal + p.nspec - 1) / p.nspec;
}

void pass_tiles(const R2CPass& p, int* W, int* nbx, int* nby) {
    *W = tile_width(p.L);
    *nbx = (int)((p.nlines + 2 * *W - 1) / (2 * *W));
    *nby = 1;
}

// The certificate epilogue keeps 2 (W / 8) * out_len running maxima per warp in
// registers (SLOTS per lane): its tiles are 8 lines wide; other modes use tile_width.
// On the register-resident path (c2r_on_reg) a tile is 16 complex = 32 real lines.
void pass_tiles(const C2RPass& p, int* W, int* nbx, int* nby) {
    *W = c2r_on_reg(p) ? 16 : p.mode == C2R_CERTMAX ? 8 : tile_width(p.L);
    *nbx = (int)((p.nlines + 2 * *W - 1) / (2 * *W));
    *nby = p.mode == C2R_CERTMAX ? (p.ktotal + p.nspec - 1) / p.nspec : 1;
}

sfw_status launch_c2c(const C2CPass& p0, cudaStream_t st, GroupArgs* g) {
    C2CPass p = p0;
    if (!g) {
        int W, nbx, nby;
        pass_tiles(p, &W, &nbx, &nby);
        SFW_TRY(fit_factors(p.L, W, &p.fac, &p.tw, true));
    }
    if (g_recorder && !g) return g_recorder->add(p);
    switch (p.L) {
#define SFW_CASE(LL) case LL: return run_c2c<LL>(p, st, g);
        SFW_FFT_LENGTHS(SFW_CASE)
#undef SFW_CASE
        default: return run_c2c<0>(p, st, g);
    }
}

sfw_status launch_mul(const MulPass& p0, cudaStream_t st, GroupArgs* g) {
    MulPass p = p0;
    if (!g) {
        int W, nbx, nby;
        pass_tiles(p, &W, &nbx, &nby);
        SFW_TRY(fit_factors(p.L, W, &p.fac, &p.tw, true));
    }
    if (g_recorder && !g) return g_recorder->add(p);
    switch (p.L) {
#define SFW_CASE(LL) case LL: return run_mul<LL>(p, st, g);
        SFW_FFT_LENGTHS(SFW_CASE)
#undef SFW_CASE
        default: return run_mul<0>(p, st, g);
    }
}

sfw_status launch_r2c(const R2CPass& p0, cudaStream_t st, GroupArgs* g) {
    R2CPass p = p0;
    if (!g) {
        int W, nbx, nby;
        pass_tiles(p, &W, &nbx, &nby);
        SFW_TRY(fit_factors(p.L, W, &p.fac, &p.tw));
    }
    if (g_recorder && !g) return g_recorder->add(p);
    switch (p.L) {
#define SFW_CASE(LL) case LL: return run_r2c<LL>(p, st, g);
        SFW_FFT_LENGTHS(SFW_CASE)
#undef SFW_CASE
        default: return run_r2c<0>(p, st, g);
    }
}

sfw_status launch_c2r(const C2RPass& p0, cudaStream_t st, int* blocks_out, GroupArgs* g) {
    C2RPass p = p0;
    if (!g) {
        int W, nbx, nby;
        pass_tiles(p, &W, &nbx, &nby);
        SFW_TRY(fit_factors(p.L, W, &p.fac, &p.tw, c2r_on_reg(p)));
        p.ntiles = nbx * nby;
    }
    if (g_recorder && !g) {
        int W, nbx, nby;
        pass_tiles(p, &W, &nbx, &nby);
        if (blocks_out) *blocks_out = nbx;
        return g_recorder->add(p);
    }
    switch (p.L) {
#define SFW_CASE(LL) case LL: return run_c2r<LL>(p, st, blocks_out, g);
        SFW_FFT_LENGTHS(SFW_CASE)
#undef SFW_CASE
        default: return run_c2r<0>(p, st, blocks_out, g);
    }
}

int c2r_blocks(const C2RPass& p) {
    int W, nbx, nby;
    pass_tiles(p, &W, &nbx, &nby);
    return nbx;
}

// Per-voxel keys -> max over k and its k.
__global__ void k_vox_decode(const unsigned long long* key, long long V, float* max_out,
                             int* argk_out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        float v;
        int a;
        if (k == ~0ull) {
            v = __int_as_float(0x7fc00000);
            a = 0;
        } else {
            v = float_from_order_key((unsigned int)(k >> 32));
            const unsigned long long flat = 0xffffffffu - (unsigned int)(k & 0xffffffffu);
            a = (int)(flat / V);
        }
        if (max_out) max_out[i] = v;
        if (argk_out) argk_out[i] = a;
    }
}

sfw_status launch_vox_decode(const unsigned long long* key, long long V, float* max_out,
                             int* argk_out, cudaStream_t st) {
    SFW_LAUNCH(st, "k_vox_decode", k_vox_decode<<<1024, 256, 0, st>>>(key, V, max_out, argk_out));
    return launch_check("k_vox_decode");
}

}  // namespace sfw
