/*
 * sfw.h -- C ABI of the GB300 (sm_103a) hot path of the sliding Frank-Wolfe
 * solver for 3D deconvolution (Courbot & Colicchio, "Boosting the Sliding
 * Frank-Wolfe solver for 3D deconvolution", arXiv 2009.05473).
 *
 * Model (Section 1.1).  A measure mu = sum_n w_n delta_{theta_n} with w_n >= 0
 * and theta_n = (m_n, sigma_n, d_n) is observed through
 *     y = H * sum_n G(theta_n, w_n) + noise                       (Eqs. 1, 3)
 *     G(theta, w; s) = w exp(-|m - s|^d / (2 sigma^d))            (Eq. 2)
 * The criterion is C = 1/2 |y - Phi mu|^2 + lambda sum_n w_n     (Eq. 4)
 * and the certificate eta = Phi^T (y - Phi mu) / lambda           (Eq. 5).
 *
 * Discretisation (the paper is silent; this library fixes it):
 *   - a volume of shape n = (n0, n1, n2) is C-contiguous, axis 2 fastest,
 *     voxel centres at integer coordinates 0..n_a-1;
 *   - the PSF H has shape (2R0+1, 2R1+1, 2R2+1), centred at index R;
 *   - atoms are sampled at voxel centres of the extended grid E = n + 2R
 *     (E index t <-> grid coordinate t - R), blurred by the discrete linear
 *     convolution with H, and observed on the grid.  Phi is therefore an exact
 *     finite linear operator and Phi^T its transpose.
 *
 * Conventions of every call:
 *   - returns sfw_status; on failure sfw_last_error() (thread-local) holds a
 *     one-line message.  No C++ exception crosses the ABI.
 *   - "device" pointers are CUDA device memory owned by the caller; "host"
 *     pointers are ordinary host memory, read during the call only.
 *   - calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream) unless stated otherwise.
 *   - a plan owns its device workspace: calls that share a plan must be
 *     ordered on one stream (or otherwise serialised by the caller).
 *   - all floating-point data is IEEE binary32 unless the type says double.
 */
#ifndef SFW_H_
#define SFW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFW_OK = 0,
    SFW_ERR_ARG = 1,         /* NULL pointer, bad count, bad option */
    SFW_ERR_SHAPE = 2,       /* sizes outside the supported range */
    SFW_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SFW_ERR_NAN = 4,         /* a NaN reached a reduction that needs a total order */
    SFW_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
    SFW_ERR_ALLOC = 6,       /* device allocation failed */
    SFW_ERR_UNSUPPORTED = 7  /* option not built into this library */
} sfw_status;

enum { SFW_PREC_FP32 = 0, SFW_PREC_BF16 = 1 };

/* Algorithm of the convolutions (Eq. 3 and its transpose) and of the grid
 * certificate (Eq. 5).  FFT: Fourier-domain products on padded grids (Section 2:
 * "convolutions are made in Fourier domain"; the certificate against the
 * kernel-family table).  DIRECT: plain FP32 direct sums over the PSF taps and
 * over the unit atom's truncated box, one thread per output voxel (the
 * straightforward GPU form, kept as the comparison path).  AUTO: FFT until
 * sfw_autotune times both on the plan and keeps the faster one per operation. */
enum { SFW_ROUTE_AUTO = 0, SFW_ROUTE_FFT = 1, SFW_ROUTE_DIRECT = 2 };

/* Problem geometry, certificate grid and options of a plan (all HOST memory).
 *   n[3]      grid shape, each in [4, 1024]
 *   R[3]      PSF half-widths, each in [0, 64]
 *   psf       (2R0+1)(2R1+1)(2R2+1) values, C order, centred at index R
 *   n_sigma, n_d, sigmas, ds
 *             certificate grid (step 1 of Algorithms 1 and 2): kernels
 *             k = i_sigma * n_d + i_d, sigma in [0.25, 16], d in [0.5, 4];
 *             K = n_sigma * n_d in [0, 256] (0: no certificate grid) and
 *             K * n0 * n1 * n2 < 2^32 (flat candidate indices fit 32 bits)
 *   precision SFW_PREC_FP32 (complex64 kernel-family table) or SFW_PREC_BF16
 *             (bfloat16 table; tensor-core axis-0 stage for real tables, see
 *             sfw_certificate_grid)
 *   eps       atom truncation level for rendering and the adjoint: an atom is
 *             evaluated only where exp(-(rho/sigma)^d/2) >= eps; in [0, 0.1),
 *             0 selects 1e-9
 *   route     SFW_ROUTE_AUTO, SFW_ROUTE_FFT or SFW_ROUTE_DIRECT (above).  A
 *             DIRECT plan builds no kernel-family table; an AUTO plan builds
 *             what both routes need. */
typedef struct {
    int n[3];
    int R[3];
    const float* psf;
    int n_sigma;
    int n_d;
    const float* sigmas;
    const float* ds;
    int precision;
    float eps;
    int route;
} sfw_plan_desc;

typedef struct sfw_plan sfw_plan;

/* Sizes a plan chose (filled by sfw_plan_query). */
typedef struct {
    int E[3];               /* extended grid n + 2R */
    int P_conv[3];          /* FFT grid of the blur, >= E, 2-3-5 smooth */
    int P_cert[3];          /* FFT grid of the certificate, >= n + h (h: support half-width of
                               H * g_k, at most n - 1), 2-3-5 smooth; 0 on a DIRECT plan */
    int K;                  /* number of certificate kernels */
    int real_table;         /* 1 if the kernel-family spectra are real (even H) */
    size_t table_bytes;     /* device bytes of the kernel-family table */
    size_t workspace_bytes; /* device bytes of the plan workspace */
    int route_blur;         /* SFW_ROUTE_FFT or SFW_ROUTE_DIRECT: convolutions in use */
    int route_cert;         /* SFW_ROUTE_FFT or SFW_ROUTE_DIRECT: grid certificate in use */
    int tensor_cores;       /* 1 if the certificate's axis-0 stage runs on the tensor cores:
                               the default of SFW_PREC_BF16 plans with a real table, FFT
                               route and K <= 128; sfw_autotune may switch it off */
} sfw_plan_info;

/* Atom set (DEVICE memory, FP32, structure of arrays).
 *   N      number of atoms, 0 <= N <= 4096
 *   m      N x 3 positions in grid coordinates, row-major
 *   sigma  N widths (> 0), d  N shape exponents (> 0), w  N weights */
typedef struct {
    int N;
    const float* m;
    const float* sigma;
    const float* d;
    const float* w;
} sfw_atoms;

/* Create a plan: uploads H, computes its spectrum on P_conv and the table of
 * kernel-family spectra used by the certificate -- the "lookup table for
 * convolution in D computed once" of Section 2: for every grid kernel k,
 * K_k = H * g_{sigma_k, d_k} sampled at every grid displacement, transformed
 * on P_cert.  Synchronous (returns after the table is built).  *out receives
 * the plan.  Errors (checked before any CUDA call): SFW_ERR_SHAPE for n, R,
 * K or K * V outside the ranges above; SFW_ERR_ARG for NULL desc, out, psf or
 * grid arrays, negative grid sizes, grid values, precision, eps or route
 * outside theirs.  Then SFW_ERR_ALLOC or SFW_ERR_CUDA from the build. */
sfw_status sfw_plan_create(const sfw_plan_desc* desc, sfw_plan** out);

/* Engine choice by timing (no counterpart in the paper).  For an SFW_ROUTE_AUTO
 * plan: FFT or DIRECT, separately for the convolutions and for the grid
 * certificate.  For a plan whose certificate can run its axis-0 stage on the
 * tensor cores (SFW_PREC_BF16, real table): tensor cores or the FFT
 * arithmetic.  Each candidate is timed on the plan's own workspace (a zero
 * residual, one warm-up and three timed runs, CUDA events on stream) and the
 * faster one kept.  With cache_path (host string, may be NULL) the choice is
 * looked up in that text file first, keyed by the plan's shape, PSF support,
 * grid, precision and route, and appended to it after timing.  Synchronous;
 * not capturable.  A plan with nothing to choose returns SFW_OK at once. */
sfw_status sfw_autotune(sfw_plan* plan, const char* cache_path, void* stream);

/* Free a plan and its device memory (synchronises the device). NULL is a no-op. */
sfw_status sfw_plan_destroy(sfw_plan* plan);

/* Copy the plan's sizes into *info (host). */
sfw_status sfw_plan_query(const sfw_plan* plan, sfw_plan_info* info);

/* Device-side health of a plan (no counterpart in the paper).  Kernels that
 * wait on the copy engine or the tensor cores (the certificate tail's TMA slab
 * copies; the tensor-core axis-0 stage's bulk copies and MMA completions; the
 * tensor-core axis-2 tail's tensor-map loads and MMA completions) give
 * up after a bounded number of polls, leave their results unspecified and set
 * a flag of the plan instead of hanging.  This call synchronises the device,
 * returns SFW_ERR_TIMEOUT if the flag is set (and clears it), else SFW_OK. */
sfw_status sfw_plan_check(sfw_plan* plan);

/* Forward operator Phi mu (Eq. 3 without noise), Section 1.1.
 *   atoms  device atom set (m, sigma, d, w)
 *   y_out  device, n0*n1*n2 floats, receives (H * sum_n G(theta_n, w_n)) on the grid */
sfw_status sfw_forward(sfw_plan* plan, const sfw_atoms* atoms, float* y_out, void* stream);

/* Certificate of Eq. 5 on the grid (step 1 of Algorithms 1 and 2):
 *   eta_k(m) = (1/lambda) sum_{s in grid} r(s) (H * g_k)(s - m)
 *            = (1/lambda) <Phi G((m, sigma_k, d_k), 1), r>
 * for every voxel m and kernel k, by FFT correlation with the plan's table
 * (route FFT) or as (1/lambda) sum_t g_k(t - m) b(t), b = Phi^T r on E, by
 * direct sums (route DIRECT).
 *   residual  device, n0*n1*n2 floats (r = y - Phi mu; r = y for mu = 0)
 *   lambda    > 0
 *   eta_out   device K*n0*n1*n2 floats or NULL: eta in flat order k*V + lin(m)
 *   max_out   device n0*n1*n2 floats or NULL: max over k
 *   argk_out  device n0*n1*n2 int32 or NULL: the k of max_out (ties -> lowest k)
 *   best_val, best_idx
 *             device 1 float / 1 int64 or NULL: the grid maximum and its flat
 *             index k*V + lin(m), ties -> lowest flat index (the seed of the
 *             local ascent).  If any eta is NaN, best_idx = -1 and best_val =
 *             NaN (the call itself cannot see it: it does not synchronise).
 * With precision SFW_PREC_BF16 the table is read as bfloat16 (values carry
 * ~3 significant digits); with a real table (even PSF) the axis-0 stage of the
 * correlation then runs on the tensor cores: bf16 operands (the table and the
 * twiddled residual spectrum), FP32 accumulation; where the certificate takes
 * its per-axis tail and n2 <= 128, the axis-2 real inverse with the max over k
 * runs on them too (tf32 operands read straight from the FP32 spectra).
 * sfw_eta_points re-evaluates candidates in FP32. */
sfw_status sfw_certificate_grid(sfw_plan* plan, const float* residual, double lambda,
                                float* eta_out, float* max_out, int32_t* argk_out,
                                float* best_val, int64_t* best_idx, void* stream);

/* Grid certificate with FP32 re-scoring of the best candidates: the seed of
 * the local ascent of step 1 (Algorithms 1 and 2) when the grid correlation
 * runs on a reduced-precision table (SFW_PREC_BF16 plans).
 * Runs sfw_certificate_grid (per-voxel max over k), takes the topk voxels by
 * that value (ties -> lower voxel index), forms their parameter rows
 * (m = voxel position, sigma_k, d_k of the voxel's best k) and re-scores them
 * in FP32 by the direct sums of sfw_eta_points.
 *   residual   device n0*n1*n2 floats; lambda > 0; topk in [1, 64]
 *   cand_theta device topk x 5 floats or NULL: the candidate rows
 *   cand_grid  device topk floats or NULL: their grid values (table precision)
 *   cand_eta   device topk doubles or NULL: their re-scored certificates
 *   best_theta device 5 floats or NULL, best_eta device 1 double or NULL:
 *              the candidate with the largest re-scored value (ties -> first).
 * A NaN in the certificate makes the rows NaN.  Asynchronous. */
sfw_status sfw_certificate_topk(sfw_plan* plan, const float* residual, double lambda, int topk,
                                float* cand_theta, float* cand_grid, double* cand_eta,
                                float* best_theta, double* best_eta, void* stream);

/* Certificate of Eq. 5 at arbitrary (off-grid) parameters, with its
 * gradient: the objective of the local ascent of step 1 ("local ascent using
 * e.g. BFGS, starting from a maximum attained on a grid") and the FP32
 * re-scoring of grid candidates.
 *   eta(theta) = (1/lambda) sum_{t in E} g_theta(t) b(t),  b = Phi^T r on E
 *   residual  device n0*n1*n2 floats
 *   lambda    > 0
 *   P         number of rows, 1..4096
 *   theta     device P x 5 floats, rows (m0, m1, m2, sigma, d)
 *   eta_out   device P doubles
 *   grad_out  device P x 5 doubles or NULL: d eta / d (m0, m1, m2, sigma, d)
 * The atom profile is evaluated where g >= eps (plan option). */
sfw_status sfw_eta_points(sfw_plan* plan, const float* residual, double lambda, int P,
                          const float* theta, double* eta_out, double* grad_out, void* stream);

/* Arg-maximum / top-k of a device float array (the grid maximum that seeds
 * step 1).
 *   values   device, count floats, count in [1, 2^32 - 2] (the index of a
 *            value travels in the low 32 bits of a 64-bit comparison key;
 *            SFW_ERR_ARG outside that range)
 *   topk     1..64: the topk largest values, in decreasing order, ties ->
 *            lower index first
 *   val_out  device topk floats; idx_out device topk int64
 * A NaN anywhere makes idx_out[0] = -1 (checked on the device; the call does
 * not synchronise).  The key scratch is a library-owned device buffer,
 * allocated with cudaMalloc on first use and re-allocated (after a stream
 * synchronisation) when a larger count or topk needs more. */
sfw_status sfw_argmax(const float* values, int64_t count, int topk, float* val_out,
                      int64_t* idx_out, void* stream);

/* sfw_argmax without any device allocation.  (The paper has no counterpart:
 * this entry point exists for callers that cannot allocate.)
 * Same arguments, results and NaN reporting as sfw_argmax, same count range
 * [1, 2^32 - 2].  sfw_argmax allocates its key scratch with cudaMalloc on
 * first use; this variant uses a 2 MiB static device array of the library
 * instead and never calls cudaMalloc, cudaFree or an allocating library
 * routine -- for applications whose device memory belongs to another
 * allocator or a fixed budget, and for loops where the cudaFree of a
 * re-allocation would synchronise the device.
 * Limit: topk == 1 takes any count in the range above; topk > 1 needs
 * ceil(count / 4096) * topk <= 131072 (e.g. count <= 8 388 608 for topk = 64),
 * else SFW_ERR_SHAPE.  The first call on each device looks up the array's
 * address (make that first call before any stream capture).  All calls share
 * the array: calls whose kernels overlap on the GPU race and must be ordered
 * by the caller. */
sfw_status sfw_argmax_noalloc(const float* values, int64_t count, int topk, float* val_out,
                              int64_t* idx_out, void* stream);

/* Loss and analytic gradient of the sliding step (step 4 of Algorithm 1,
 * step 2b of Algorithm 2; Section 2: "grad C computed analytically").
 *   y         device n0*n1*n2 floats (observation)
 *   atoms     device atom set, N >= 1
 *   lambda    >= 0
 *   loss_out  device 1 double: C = 1/2 sum (y - Phi mu)^2 + lambda sum w
 *   grad_out  device 6N doubles or NULL (loss only: no back-projection and
 *             no adjoint): [dC/dm (N x 3, row-major) | dC/dsigma (N) |
 *             dC/dd (N) | dC/dw (N)], with b = Phi^T r on E,
 *               dC/dw_n = lambda - sum_t g_n(t) b(t),
 *               dC/dtheta_n = -w_n sum_t (d g_n / d theta)(t) b(t)
 *   residual_out  device n0*n1*n2 floats or NULL: r = y - Phi mu
 * The atom field is recomputed inside the call (never stored per atom). */
sfw_status sfw_slide_loss_grad(sfw_plan* plan, const float* y, const sfw_atoms* atoms,
                               double lambda, double* loss_out, double* grad_out,
                               float* residual_out, void* stream);

/* One SFW iteration's data-parallel work in one call: the sliding loss and
 * gradient of sfw_slide_loss_grad (Eq. 4; step 4 of Algorithm 1) and the grid
 * certificate maximum of sfw_certificate_grid (Eq. 5; step 1 of Algorithm 1)
 * for the same residual, so step 1 of the next iteration needs no extra pass.
 *   y, atoms, lambda (> 0), loss_out, grad_out (or NULL), residual_out (or
 *   NULL)  as for sfw_slide_loss_grad
 *   best_val, best_idx  device 1 float / 1 int64 or NULL: as for
 *             sfw_certificate_grid (max over k and voxels of eta_k, its flat
 *             index k V + lin(m); NaN / -1 if a NaN occurred)
 *   stream    the call's stream: it orders the call after earlier work and
 *             later work after the whole call
 *   aux_stream  another stream on the same device, or NULL.  Given, the
 *             certificate runs on it once the residual is ready (an event
 *             recorded on stream) while the back-projection and the adjoint
 *             sums continue on stream; stream then waits for aux_stream (a
 *             second event).  Both events belong to the plan: overlapping
 *             sfw_step calls on one plan are the caller's race.  Works under
 *             stream capture (the fork becomes a branch of the graph).
 * Results equal those of the two separate calls.  SFW_ERR_ARG on bad
 * arguments or a plan without certificate grid.
 * Graph: when a call has the same pointers, N and lambda as the call before
 * it (data may change in place), the call captures the step into a CUDA graph
 * of the plan (on two streams the plan owns; capturing runs nothing) and
 * launches it on stream; later identical calls only launch the graph.  A call
 * with other arguments drops the graph (after waiting for its last launch).
 * Calls made while stream is being captured by the caller, and calls while a
 * profile is recorded, launch their kernels directly. */
sfw_status sfw_step(sfw_plan* plan, const float* y, const sfw_atoms* atoms, double lambda,
                    double* loss_out, double* grad_out, float* residual_out, float* best_val,
                    int64_t* best_idx, void* stream, void* aux_stream);

/* The same iteration with the precision configuration's seed: the sliding
 * loss and gradient (Eq. 4; step 4 of Algorithm 1) and, for the same residual,
 * the grid certificate's top-k voxels re-scored in FP32 (sfw_certificate_topk:
 * the seed of step 1's local ascent).  One back-projection b = Phi^T r serves
 * both the adjoint sums of the gradient and the re-score.
 *   y, atoms, lambda (> 0), loss_out, grad_out (non-NULL), residual_out (or
 *   NULL)  as for sfw_slide_loss_grad
 *   topk, cand_theta, cand_grid, cand_eta, best_theta, best_eta  as for
 *             sfw_certificate_topk
 *   stream, aux_stream  as for sfw_step: given aux_stream, the grid
 *             certificate and the top-k selection run on it once the residual
 *             is ready, while the back-projection and the adjoint sums run on
 *             stream; the re-score follows on aux_stream once those are done
 *             (it shares their partial-sum scratch), and stream waits for it.
 *             Three events of the plan order the branches: overlapping calls
 *             on one plan are the caller's race.  Works under stream capture.
 * Results equal those of sfw_slide_loss_grad followed by
 * sfw_certificate_topk.  SFW_ERR_ARG on bad arguments or a plan without
 * certificate grid; no graph of its own (callers capture it). */
sfw_status sfw_step_topk(sfw_plan* plan, const float* y, const sfw_atoms* atoms, double lambda,
                         double* loss_out, double* grad_out, float* residual_out, int topk,
                         float* cand_theta, float* cand_grid, double* cand_eta, float* best_theta,
                         double* best_eta, void* stream, void* aux_stream);

/* Per-launch timing.  sfw_profile_start records a CUDA event pair on the
 * launching stream around each of the next max_launches kernels this library
 * launches (any thread) whose tag equals only_tag (host string; NULL = every
 * kernel).  The events are recorded as external events, so a
 * stream capture turns them into event-record nodes that time every replay
 * of the graph.  sfw_profile_collect waits for the recorded events and adds
 * their durations to per-tag totals (call it after each replay to time
 * replays); sfw_profile_stop ends recording (collecting once if collect was
 * never called) and writes a JSON object {"tag": [launches, total_ms], ...}
 * into json (host, len bytes, NUL-terminated).  Tags name the pass of the hot
 * path (e.g. "cert_axis0", "blur_tail", "k_atom_grad").  SFW_ERR_ARG if json
 * is too small or launches were dropped (pool full). */
sfw_status sfw_profile_start(int max_launches, const char* only_tag);
sfw_status sfw_profile_collect(void);
sfw_status sfw_profile_stop(char* json, size_t len);

/* Gram system of the non-negative LASSO of step 3 (Algorithm 1; step 3 of
 * Algorithm 2): with a_i = Phi G(theta_i, 1) the blurred unit atoms,
 *   G[i][j] = <a_i, a_j>,  c[i] = <a_i, y>   (sums in FP64 over the grid),
 * so that C(y, mu_{w,theta}, lambda) = 1/2 w^T G w - (c - lambda)^T w + |y|^2/2.
 *   atoms   device atom set, 1 <= N <= 256 (weights ignored)
 *   y       device n0*n1*n2 floats
 *   G_out   device N x N doubles (row-major), c_out device N doubles
 * The first call with N atoms allocates N*V floats in the plan (kept for
 * later calls; synchronises the stream when it grows).  Asynchronous
 * otherwise. */
sfw_status sfw_gram(sfw_plan* plan, const sfw_atoms* atoms, const float* y, double* G_out,
                    double* c_out, void* stream);

/* ---- Batches: many independent volumes (uneven shapes, PSFs, atom counts)
 * through one step of grouped launches.
 * At creation the batch records the launches of one SFW iteration's hot path
 * for every volume -- sfw_slide_loss_grad (loss, gradient, residual), then
 * sfw_certificate_grid of that residual (grid argmax only) -- and merges the
 * launches of each stage that use the same kernel variant into one
 * persistent launch whose CTAs stride over a device work list of (volume,
 * tile) items.  sfw_batch_step issues those launches only (no host
 * synchronisation, no allocation): capture it into a CUDA graph to run the
 * whole batch as one graph launch.  The first step computes the launch grids
 * (occupancy queries): run it once before any capture.
 *   count     number of volumes, 1..1024
 *   plans     host array of count distinct plans with a certificate grid; they
 *             must outlive the batch and not be used concurrently with a step
 *   vols      host array of count volume descriptions: device buffers owned by
 *             the caller, fixed for the batch's lifetime (the step reads y and
 *             the atoms and writes the outputs in place)
 *   lambdas   host array of count regularisation weights (> 0)
 * Errors: SFW_ERR_ARG for a NULL array, count outside its range, a NULL,
 * repeated or grid-less plan, N outside 1..4096, a NULL buffer or a lambda
 * not > 0 (all checked before any CUDA call); SFW_ERR_ALLOC, SFW_ERR_CUDA. */
typedef struct sfw_batch sfw_batch;

typedef struct {
    int N;               /* atoms of the volume, 1..4096 */
    const float* y;      /* device n0*n1*n2 (plan's grid): observation */
    const float* m;      /* device N x 3 atom positions; sigma, d, w: device N */
    const float* sigma;
    const float* d;
    const float* w;
    float* residual;     /* device n0*n1*n2: y - Phi mu (output) */
    double* grad;        /* device 6N: gradient of C (output, sfw_slide_loss_grad layout) */
    double* loss;        /* device 1: C (output) */
    float* best_val;     /* device 1: grid maximum of eta (output) */
    int64_t* best_idx;   /* device 1: its flat index k*V + lin(m) (output) */
} sfw_batch_volume;

sfw_status sfw_batch_create(int count, sfw_plan* const* plans, const sfw_batch_volume* vols,
                            const double* lambdas, sfw_batch** out);
sfw_status sfw_batch_destroy(sfw_batch* batch);
/* Number of grouped launches one sfw_batch_step issues. */
sfw_status sfw_batch_query(const sfw_batch* batch, int* launches_per_step);
/* One hot-path step for every volume of the batch, asynchronous on stream.
 * After the residual stages, the certificate stages run on a stream the batch
 * owns (an event forks it from stream) while the back-projection and
 * gradient stages continue on stream; stream then waits for the branch (a
 * second event), so work queued on stream afterwards sees the whole step.
 * Under stream capture the fork is a branch of the graph. */
sfw_status sfw_batch_step(sfw_batch* batch, void* stream);
/* Autotuner: for every grouped launch, time persistent grids of {resident
 * CTAs, 1, 2, 4, 8 x SMs, all tiles} on the batch's live buffers (after one
 * full step) and keep the fastest.  With cache_path (host string, may be
 * NULL) the choices are written there, keyed by the batch's launch list, and
 * read back by later calls with the same list instead of timing again.
 * Synchronous; not capturable (run it before capturing sfw_batch_step). */
sfw_status sfw_batch_autotune(sfw_batch* batch, const char* cache_path, void* stream);

/* Thread-local text of the last error of this thread ("" if none). */
const char* sfw_last_error(void);

/* Number of CUDA kernels this library has launched in this process. */
int64_t sfw_launch_count(void);

/* Library version string. */
const char* sfw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFW_H_ */
