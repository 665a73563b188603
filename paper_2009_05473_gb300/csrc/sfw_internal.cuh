// Internal declarations shared by the CUDA translation units of libsfw.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <vector>

#include "sfw.h"

namespace sfw {

// ------------------------------------------------------------------ errors
sfw_status fail(sfw_status st, const char* fmt, ...);
sfw_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define SFW_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e__ = (call);                             \
        if (e__ != cudaSuccess) return ::sfw::cuda_fail(e__, #call); \
    } while (0)

#define SFW_TRY(expr)                         \
    do {                                      \
        sfw_status s__ = (expr);              \
        if (s__ != SFW_OK) return s__;        \
    } while (0)

// Kernels launched by the library (process-wide counter).
extern std::atomic<int64_t> g_launches;
inline void counted_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Optional per-launch timing (sfw_profile_start): CUDA events recorded on the
// launching stream around every kernel, aggregated per tag.  The tag is the
// innermost active LaunchTag of this thread, else the kernel's own name.
void prof_begin(cudaStream_t st, const char* name);
bool prof_active();  // a profile is being recorded
void prof_end(cudaStream_t st);
struct LaunchTag {
    const char* prev;
    explicit LaunchTag(const char* tag);
    ~LaunchTag();
};

#define SFW_LAUNCH(st, name, ...)          \
    do {                                   \
        ::sfw::prof_begin((st), (name));   \
        __VA_ARGS__;                       \
        ::sfw::prof_end(st);               \
        ::sfw::counted_launch();           \
    } while (0)
// Check the launch that was just issued.
sfw_status launch_check(const char* what);

// ------------------------------------------------------------------ FFT plans
constexpr int kMaxFactors = 16;
constexpr int kMaxLen = 1024;

struct Factors {
    int n;
    int r[kMaxFactors];
};

// Split L into radices 16, 8, 4, 2, 3, 5 with power-of-two radices <= maxr
// (false if another prime divides L).
bool factorize(int L, Factors* f, int maxr = 16);
// Largest power-of-two radix that keeps all 32 lanes busy with nl lines per warp.
int max_radix(int L, int nl);
// Per-stage twiddles of factorize(L, maxr) (device table, cached per device).
sfw_status twiddle_table(int L, int maxr, const float2** out);
// Smallest 2-3-5 smooth even integer >= x.
int next_smooth_even(int x);

// Line addressing of a batched 1-D transform: line l -> a = l / B, b = l % B,
// base offset a * Sa + b * Sb; consecutive points of a line are Sj apart.
struct LineSet {
    long long Sa, Sb, Sj;
    long long B;
};

__host__ __device__ inline long long line_offset(const LineSet& s, long long l) {
    long long a = l / s.B;
    long long b = l - a * s.B;
    return a * s.Sa + b * s.Sb;
}

// Per-stage twiddle tables, one per length (device, float2; layout in fft_kernels.cu).
struct TwiddleCache {
    std::map<int, float2*> tables;
    sfw_status get(int L, const float2** out);
    void release();
};

// Spectrum element formats for the fused multiply.
enum SpecKind { SPEC_C64 = 0, SPEC_R32 = 1, SPEC_CBF16 = 2, SPEC_RBF16 = 3 };

// ---- pass descriptors (kernel parameters, by value) ----

// Complex-to-complex transform along a strided axis, zero-padded input rows
// [in_off, in_off + in_len), output rows [out_off, out_off + out_len).
struct C2CPass {
    const float2* in;
    float2* out;
    LineSet lin, lout;
    long long nlines;
    int L, in_off, in_len, out_off, out_len;
    int dir;  // -1 forward, +1 inverse
    float scale;
    Factors fac;
    const float2* tw;
};

// Forward transform along a strided axis, then for each of nspec spectra:
// multiply, inverse transform and write the cropped rows.
struct MulPass {
    const float2* in;
    LineSet lin;
    int in_off, in_len;
    long long nlines;
    int L;
    Factors fac;
    const float2* tw;
    const void* spec;
    LineSet lspec;
    long long spec_stride;  // elements between consecutive spectra
    int nspec;              // spectra per CTA (group size; grid.y = groups)
    int ktotal;             // number of spectra
    int spec_kind;
    int conj_spec;
    float2* out;
    LineSet lout;
    long long out_stride;   // elements between consecutive outputs
    int out_off, out_len;
};

// Real lines along the contiguous axis -> half spectra (L/2 + 1 points).
struct R2CPass {
    const float* in;
    LineSet lin;          // real lines, Sj = 1
    long long nlines;     // real lines
    int in_off, in_len;
    int L;
    Factors fac;
    const float2* tw;
    float2* out;
    LineSet lout;         // half-spectrum lines, Sj = 1
};

enum C2RMode { C2R_STORE = 0, C2R_RESIDUAL = 1, C2R_CERTMAX = 2 };

// Half spectra -> real lines along the contiguous axis, cropped rows, with an
// epilogue: store, residual + squared-norm partials, or certificate max.
struct C2RPass {
    const float2* in;
    LineSet lin;          // half-spectrum lines, Sj = 1
    long long nlines;     // real output lines
    long long in_spec_stride;
    int nspec;            // CERTMAX: spectra per CTA (group size); otherwise 1
    int L;
    Factors fac;
    const float2* tw;
    int out_off, out_len;
    LineSet lout;         // real lines, Sj = 1 (also voxel index for dense outputs)
    float scale;
    int mode;
    float* out;           // STORE: output; RESIDUAL: residual (may be NULL)
    const float* y;       // RESIDUAL: observation
    double* partials;     // RESIDUAL: one double per block
    float* eta_out;       // CERTMAX: K x V or NULL
    long long V;
    float* max_out;       // CERTMAX: V or NULL
    int* argk_out;        // unused by the kernel (decoded from vox_key)
    unsigned long long* best_key;  // CERTMAX: one key or NULL
    unsigned long long* vox_key;   // CERTMAX: V per-voxel keys (atomicMax) or NULL
    int ktotal;           // CERTMAX: number of spectra; grid.y groups them by nspec
    // last-tile epilogue (the tile that finishes last reduces and re-arms)
    int ntiles;           // tiles of this pass (set by the launcher)
    unsigned int* counter;  // zero between calls
    double* loss_out;     // RESIDUAL: C = 1/2 sum r^2 + lambda sum w, or NULL
    const float* w;       //   weights w[i * w_stride], i < nw
    int nw, w_stride;
    double lambda;
    float* best_val;      // CERTMAX: decoded best_key (best_key is reset to 0)
    int64_t* best_idx;
};

// Certificate tail fused in one pass (lengths P1 in {64, 128}, P2 in {64, 128, 256}):
// per (i0, kernel group) CTA and kernel k, the slab in[k][i0] (P1 x H2 complex,
// contiguous) -> inverse along axis 1 (keep n1 rows) -> real inverse along axis 2
// (keep n2) -> running max / argmax over the group, candidate keys as in C2RPass.
struct CertTailPass {
    const float2* in;           // (K, n0, P1, H2) complex; with a tensor map, line-group-major
                                // [k][l / 4][i0][l mod 4], l = p1 H2 + h2 (read by TMA)
    int boxg, nbox;             // TMA: line groups per box copy, box copies per slab
    int* err;                   // TMA: set to 1 if a slab's copies did not complete in time
    int n0, n1, n2, P1, P2, H2;
    int ktotal, nspec;          // kernels; kernels per CTA (grid.y = groups)
    const float2* tw1;          // twiddles of P1 (register factorisation)
    const float2* tw2;          // twiddles of P2
    float scale;                // 1 / lambda
    float* eta_out;             // K x V or NULL
    long long V;
    unsigned long long* best_key;
    unsigned long long* vox_key;
    int ntiles;
    unsigned int* counter;
    float* best_val;
    int64_t* best_idx;
};
// True when the fused tail handles these lengths (shared memory holds one slab).
bool cert_tail_supported(int P1, int P2, int n1, int n2);
// tmap: NULL (contiguous slabs, cp.async) or the 4-D tensor map of make_tail_tmap
// (line-group-major slabs, TMA box copies), an opaque 128-byte CUtensorMap.
sfw_status launch_cert_tail(const CertTailPass& p, const void* tmap, int groups, cudaStream_t st);
// Encode the tensor map {4, n0, P1 H2 / 4, K} (8-byte elements) of the line-group-major
// intermediate at in, boxes {4, 1, boxg, 1}; false if the driver entry point is missing.
bool make_tail_tmap(const void* in, int n0, long long ngroups, int K, int boxg, void* tmap_out);

// A blur slab pass (lengths of the blur grid, shared-memory transforms), one cluster of
// two CTAs per slab of axis 0.  Head: real slab rows x cols (rows placed at [o1, o1 + rows) of the P1
// transform, columns at [o2, o2 + cols) of P2) -> real forward along axis 2 -> forward
// along axis 1 -> out (nslab, P1, H2) complex.  Tail: in (nslab, P1, H2) -> inverse along
// axis 1 keeping rows [o1, o1 + m1) -> real inverse along axis 2 keeping [o2, o2 + m2) ->
// out (nslab, m1, m2) real: stored, or the residual y - value with the criterion
// C = 1/2 sum r^2 + lambda sum w (last-block reduction, as C2RPass).
struct SlabPass {
    int mode;                  // SLAB_HEAD, SLAB_STORE or SLAB_RESIDUAL
    int nslab, P1, P2, H2;
    int rows, cols;            // head: input slab shape
    int o1, m1, o2, m2;        // head: o1, o2 placement; tail: kept window
    const float* rin;          // head input (nslab, rows, cols)
    const float2* cin;         // tail input (nslab, P1, H2)
    float2* cout;              // head output (nslab, P1, H2)
    float* rout;               // tail output (nslab, m1, m2); RESIDUAL: may be NULL
    const float* y;            // RESIDUAL: observation (nslab, m1, m2)
    double* partials;          // RESIDUAL: one double per CTA (2 nslab)
    unsigned int* counter;
    double* loss_out;
    const float* w;
    int nw, w_stride;
    double lambda;
    Factors fac1, fac2;        // factors of P1 and P2 (two lines per warp)
    const float2* tw1;
    const float2* tw2;
    int warps;                 // warps per CTA (0: slab_warps)
    int smem;                  // dynamic shared memory at least this (grouped launches)
};
enum SlabMode { SLAB_HEAD = 0, SLAB_STORE = 1, SLAB_RESIDUAL = 2 };
struct GroupArgs;
// Dynamic shared memory of a slab pass (0: does not fit), its warps per CTA and
// whether it runs the (80, 96) specialisation.
size_t slab_smem(const SlabPass& p);
int slab_warps(const SlabPass& p);
bool slab_specialised(const SlabPass& p);
// One CTA per slab; with g, one grouped launch of g->n passes (g->passes) whose
// factors and twiddles were filled when they were recorded.
sfw_status launch_slab(const SlabPass& p, cudaStream_t st, GroupArgs* g = nullptr);

// Certificate head fused in one pass (same lengths as the tail): per i0 slab, the real
// forward transform of the residual rows along axis 2 (zero-padded n2 -> P2) and the
// forward transform of the columns along axis 1 (n1 -> P1): r (n0, n1, n2) -> out
// (n0, P1, H2) complex.
struct CertHeadPass {
    const float* r;
    float2* out;
    int n0, n1, n2, P1, P2, H2;
    const float2* tw1;
    const float2* tw2;
};
sfw_status launch_cert_head(const CertHeadPass& p, cudaStream_t st);

// A persistent grouped launch: n passes of one kernel variant, their
// descriptors and tile prefix sums in device memory.  Pass q owns tiles
// [start[q], start[q+1]); tile t of it maps to (t % nbx[q], t / nbx[q]).
struct GroupArgs {
    const void* passes;
    const int* start;
    const int* nbx;
    int n;
    int total;
    int grid;  // CTAs launched (0: resident CTAs of the kernel, computed on first use)
};

// Tile width W and tile grid (nbx, nby) of a pass (same rule for single and grouped launches).
int tile_width(int L);
// Lines per warp of the register-resident transforms of length L (0: other lengths).
int reg_line_group(int L);
void pass_tiles(const C2CPass& p, int* W, int* nbx, int* nby);
void pass_tiles(const MulPass& p, int* W, int* nbx, int* nby);
void pass_tiles(const R2CPass& p, int* W, int* nbx, int* nby);
void pass_tiles(const C2RPass& p, int* W, int* nbx, int* nby);
// Lengths with compile-time kernels (others run the generic code).
bool fft_specialised(int L);

// launchers (fft_kernels.cu); g != NULL launches the group instead of p
sfw_status launch_c2c(const C2CPass& p, cudaStream_t st, GroupArgs* g = nullptr);
sfw_status launch_mul(const MulPass& p, cudaStream_t st, GroupArgs* g = nullptr);
sfw_status launch_r2c(const R2CPass& p, cudaStream_t st, GroupArgs* g = nullptr);
// returns the number of blocks used (for the residual partials) via *blocks
sfw_status launch_c2r(const C2RPass& p, cudaStream_t st, int* blocks, GroupArgs* g = nullptr);
int c2r_blocks(const C2RPass& p);
sfw_status launch_vox_decode(const unsigned long long* key, long long V, float* max_out,
                             int* argk_out, cudaStream_t st);

// ------------------------------------------------------------------ atoms (atoms.cu)
struct AtomsDev {
    int N;
    const float* m;      // atom i at m[i * ms + a]
    const float* sigma;  // atom i at sigma[i * ps] (same for d, w)
    const float* d;
    const float* w;
    int ms = 3;
    int ps = 1;
};

// f on the box of shape E (dense), E index t <-> grid coordinate t - R.
sfw_status launch_render(const AtomsDev& a, const int E[3], const int R[3], float eps, float* f,
                         cudaStream_t st);
// Per-atom adjoint sums -> gradient (6N doubles) given b on E.  counters: N
// unsigned ints, zero between calls (the last chunk-block of an atom finalises it).
constexpr int kGradChunks = 32;   // blocks per atom of the adjoint sums
sfw_status launch_atom_grad(const AtomsDev& a, const int E[3], const int R[3], float eps,
                            const float* b, double lambda, double* partials, double* grad,
                            unsigned int* counters, cudaStream_t st);
// eta(theta_p) = <g_p, b>/lambda and its gradient for P parameter rows (m, sigma, d).
sfw_status launch_eta_points(const AtomsDev& pts, const int E[3], const int R[3], float eps,
                             const float* b, double lambda, double* partials, double* eta,
                             double* grad, unsigned int* counters, cudaStream_t st);
// Top-k voxels -> parameter rows (m0, m1, m2, sigma_k, d_k), k = argk of the voxel.
sfw_status launch_candidate_theta(const int64_t* vox, const int* argk, const float* grid_sd,
                                  int topk, const int n[3], float* theta, cudaStream_t st);
// Best of the FP32-summed candidates (ties -> first) and optional copies out.
sfw_status launch_candidate_select(const float* theta, const float* grid_val, const double* eta,
                                   int topk, float* theta_out, float* grid_out, double* eta_out,
                                   float* best_theta, double* best_eta, cudaStream_t st);
// Atom i with unit weight into a 6-float slot; Gram matrix and projections.
sfw_status launch_unit_atom(const AtomsDev& a, int i, float* slot, cudaStream_t st);
sfw_status launch_gram(const float* A, const float* y, int N, long long V, double* G, double* c,
                       cudaStream_t st);

// ------------------------------------------------------------------ tensor cores (cert_tc.cu)
// The certificate's axis-0 inverse for real bf16 tables on tcgen05: per line l,
// U_k[i0, l] = sum_p0 e^{2 pi i i0 p0 / P0} X[p0, l] T_k[p0, l] for all kernels k at once.
struct Axis0TcPass {
    const float2* X;            // forward axis-0 spectra (P0, nl): X[p0 * nl + l]
    const __nv_bfloat16* A;     // per half of the output rows: 128 x 2 Kp real form of the inverse DFT rows
    const __nv_bfloat16* Tb;    // per line: T_l as the Np x Kp bf16 B operand in the MMA layout
    float2* out;                // U_k[i0, l] at out + k * out_stride + line_offset(lout, l) + i0 * lout.Sj
    LineSet lout;
    long long out_stride;
    long long nl;               // lines (P1 * H2)
    int P0, Kp;                 // transform length, padded to a multiple of 16
    int n0;                     // kept output rows
    int K, Np;                  // kernels, padded to a multiple of 16 (<= 128)
    int* err;                   // set if a bounded wait ran out
};
sfw_status launch_tc_table(const float2* full, long long spec_elems, int K, int P0, long long nl, int Np,
                           int Kp, __nv_bfloat16* Tb, cudaStream_t st);
sfw_status launch_axis0_tc(const Axis0TcPass& p, int num_sms, cudaStream_t st);
// The A operands of launch_axis0_tc: ceil(n0 / 64) blocks of 128 x 2 Kp bf16.
sfw_status launch_tc_dft(int n0, int P0, int Kp, __nv_bfloat16* A, cudaStream_t st);
size_t tc_smem_bytes(int Kp, int Np, int P0);

// The certificate's real inverse along axis 2 with the max over kernels, on tcgen05
// (cert_tc_c2r.cu): per 128 lines (i0, i1) and kernel k, eta = A C^T with A the lines' half
// spectra read as 2 H2 FP32 numbers (tf32 MMAs) and C the fixed inverse matrix (n2 <= 128).
// The spectra come through the tensor map of make_c2r_tmap: (K, nlines, H2) complex, line pitch
// H2p (even).
struct C2rTcPass {
    const float* C;             // the inverse matrix (launch_tc_c2r_matrix): tc_c2r_chunks(H2) atoms
    int nlines, P2, H2, n2, K;
    int kgroup, nch, stages;    // set by the launcher
    float scale;                // 1 / lambda
    float* eta_out;             // K x V or NULL
    long long V;
    unsigned long long* vox_key;   // V per-voxel keys or NULL
    unsigned long long* best_key;  // one key or NULL; zero between calls
    unsigned int* counter;
    float* best_val;
    int64_t* best_idx;
    int* err;                   // set if a bounded wait ran out
};
int tc_c2r_chunks(int H2);                       // 32-column atoms of 2 H2 columns
bool tc_c2r_fits(int H2);                        // C and two A stages fit in shared memory
size_t tc_c2r_smem_bytes(int H2);
sfw_status launch_tc_c2r_matrix(int P2, int H2, int n2, float* C, cudaStream_t st);
bool make_c2r_tmap(const float2* spec, int H2, int H2p, long long nlines, int K, void* tmap_out);
sfw_status launch_c2r_tc(const C2rTcPass& p, const void* tmap, int num_sms, cudaStream_t st);

// ------------------------------------------------------------------ plain FP32 route (direct.cu)
// Direct sums without transforms (the route the transform route is measured against).
struct DirectBlur {
    const float* fE;          // rendered atoms on E = n + 2R
    const float* H;           // PSF (2R+1)^3, C order
    int n[3], R[3];
    float* out;               // store: H * f_E on the grid; residual: y - H * f_E (or NULL)
    const float* y;           // NULL: store mode; else the observation (residual mode)
    double* partials;         // residual: one double per block
    int partials_len;
    unsigned int* counter;    // residual: last-block counter, zero between calls
    double* loss_out;         // residual: C = 1/2 sum r^2 + lambda sum w, or NULL
    const float* w;
    int nw;
    double lambda;
    int num_sms;
};
sfw_status launch_direct_blur(const DirectBlur& p, cudaStream_t st);
// b_E = H^T r on the extended grid.
sfw_status launch_direct_transpose(const float* r, const float* H, const int n[3], const int R[3],
                                   float* bE, int num_sms, cudaStream_t st);
struct DirectCert {
    const float* bE;          // H^T r on E
    const float* gtab;        // unit atoms g_k on their boxes (2h_k + 1)^3
    const int2* kern;         // per k: (offset in gtab, h_k)
    int K;
    int n[3], R[3];
    float scale;              // 1 / lambda
    float* eta_out;           // K x V or NULL
    float* max_out;           // V or NULL
    int* argk_out;            // V or NULL
    unsigned long long* best_key;  // one key, zero between calls, or NULL
    unsigned int* counter;
    float* best_val;
    int64_t* best_idx;
    int num_sms;
};
sfw_status launch_direct_cert(const DirectCert& p, cudaStream_t st);

// ------------------------------------------------------------------ non-FFT ops as descriptors
// (one launch each, or grouped over the volumes of a batch)

struct RenderOp {
    AtomsDev a;
    int E[3], R[3];
    float eps;
    float* f;
};
// How the last chunk-block of an atom finalises its six adjoint sums.
struct AdjFin {
    int mode;                // 0: gradient of C (6N); 1: eta and d eta / d theta (P x 5 or NULL)
    double lambda;
    double* grad;
    double* eta;
    unsigned int* counters;  // one per atom, zero between calls
};
struct GradOp {
    AtomsDev a;
    int E[3], R[3];
    float eps;
    const float* b;
    double* partials;
    AdjFin fin;
};

// Grouped launches of the non-FFT ops (device arrays of n ops).
sfw_status launch_render_group(const RenderOp* ops, const int* start, const int* nbx, int n,
                               int total, int grid, cudaStream_t st);
sfw_status launch_grad_group(const GradOp* ops, const int* start, const int* nbx, int n, int total,
                             int grid, cudaStream_t st);
// tiles of one render / adjoint op
int render_tiles(const RenderOp& op, int* nbx);
int grad_tiles(const GradOp& op, int* nbx);

// ------------------------------------------------------------------ recording (batches)
// While g_recorder is set on this thread, every launcher appends its op here
// instead of launching; a batch replays the ops of all its volumes stage by stage.
enum OpKind {
    OP_R2C = 0, OP_C2C, OP_MUL, OP_C2R, OP_RENDER, OP_GRAD, OP_SLAB
};
struct RecOp {
    OpKind kind;
    R2CPass r2c;
    C2CPass c2c;
    MulPass mul;
    C2RPass c2r;
    RenderOp render;
    GradOp grad;
    SlabPass slab;
};
struct Recorder {
    std::vector<RecOp> ops;
    sfw_status add(const R2CPass& p) { RecOp o{}; o.kind = OP_R2C; o.r2c = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const C2CPass& p) { RecOp o{}; o.kind = OP_C2C; o.c2c = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const MulPass& p) { RecOp o{}; o.kind = OP_MUL; o.mul = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const C2RPass& p) { RecOp o{}; o.kind = OP_C2R; o.c2r = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const RenderOp& p) { RecOp o{}; o.kind = OP_RENDER; o.render = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const GradOp& p) { RecOp o{}; o.kind = OP_GRAD; o.grad = p; ops.push_back(o); return SFW_OK; }
    sfw_status add(const SlabPass& p) { RecOp o{}; o.kind = OP_SLAB; o.slab = p; ops.push_back(o); return SFW_OK; }
};
extern thread_local Recorder* g_recorder;

// ------------------------------------------------------------------ misc kernels (reduce.cu)
// dst[p] = src box value with circular placement (see definitions in reduce.cu)
sfw_status launch_wrap_psf(const float* psf, const int R[3], const int P[3], float* out,
                           cudaStream_t st);
sfw_status launch_wrap_kernel(const float* kx, const int n[3], const int h[3], const int P[3], float* out,
                              cudaStream_t st);
sfw_status launch_argmax_keys(const float* v, long long count, unsigned long long* partial,
                              int nblocks, cudaStream_t st);
sfw_status launch_argmax_final(const unsigned long long* partial, int n, float* val, int64_t* idx,
                               cudaStream_t st);
// Scratch keys launch_topk wants for `count` values (it falls back to block sorts with less).
long long topk_scratch_keys(long long count, int topk);
sfw_status launch_topk(const float* v, long long count, int topk, unsigned long long* scratch,
                       long long scratch_len, float* val_out, int64_t* idx_out, cudaStream_t st);
sfw_status launch_spec_stats(const float2* s, long long count, float* stats /*2 floats*/,
                             cudaStream_t st);
// Spectra (count / (rows * nl) of them, rows x nl lines) converted to `kind`.  group > 0
// stores them line-group-major: groups of `group` consecutive lines hold all their
// rows contiguously, [spectrum][line / group][row][line % group] (padding lines 0).
sfw_status launch_spec_convert(const float2* s, long long count, int kind, void* out, int rows,
                               long long nl, int group, cudaStream_t st);

#ifdef __CUDACC__
// True in every thread of the block that finishes last among `nblocks` blocks
// sharing `counter` (the block's global writes are made visible first).
__device__ __forceinline__ bool last_block(unsigned int* counter, int nblocks) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == (unsigned int)(nblocks - 1);
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}
#endif

// Monotone map of a float to an unsigned key (NaN handled by callers).
__host__ __device__ inline unsigned int float_order_key(float v) {
    unsigned int u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(v);
#else
    union { float f; unsigned int i; } c;
    c.f = v;
    u = c.i;
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ inline float float_from_order_key(unsigned int k) {
    unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    union { float f; unsigned int i; } c;
    c.i = u;
    return c.f;
#endif
}

// Candidate key: value order in the high word, inverted index in the low word,
// so that max(key) = largest value, then lowest index.  NaN -> all ones.
__host__ __device__ inline unsigned long long candidate_key(float v, unsigned long long idx) {
    if (v != v) return ~0ull;
    return ((unsigned long long)float_order_key(v) << 32) |
           (unsigned long long)(0xffffffffu - (unsigned int)idx);
}

}  // namespace sfw
