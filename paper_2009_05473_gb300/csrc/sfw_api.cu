// C ABI of libsfw: plans and the hot-path entry points of the sliding
// Frank-Wolfe solver (arXiv 2009.05473).  Every step of the path runs in the
// kernels of this library; this file only checks arguments, owns device
// memory and sequences the launches on the caller's stream.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "sfw_internal.cuh"

namespace sfw {

// ------------------------------------------------------------------ errors

static thread_local char g_err[512] = "";
thread_local Recorder* g_recorder = nullptr;
std::atomic<int64_t> g_launches{0};

sfw_status fail(sfw_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

sfw_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? SFW_ERR_ALLOC : SFW_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

void clear_error() { g_err[0] = 0; }

sfw_status launch_check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SFW_OK;
}

// ------------------------------------------------------------------ profiler

namespace {
struct ProfRec {
    const char* tag;
    cudaEvent_t a, b;
};
struct ProfAcc {
    std::string tag;
    long long count;
    double ms;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof;      // event pool
size_t g_prof_used = 0;           // records in use
bool g_prof_dropped = false;
std::string g_prof_only;          // record only this tag ("" = all)
bool g_prof_collected = false;
std::vector<ProfAcc> g_prof_acc;  // per-tag totals
thread_local const char* t_tag = nullptr;
thread_local ProfRec* t_open = nullptr;

void prof_accumulate(const char* tag, double ms) {
    for (auto& a : g_prof_acc)
        if (a.tag == tag) {
            a.count += 1;
            a.ms += ms;
            return;
        }
    g_prof_acc.push_back(ProfAcc{tag, 1, ms});
}
}  // namespace

LaunchTag::LaunchTag(const char* tag) : prev(t_tag) { t_tag = tag; }
LaunchTag::~LaunchTag() { t_tag = prev; }

// Inside a stream capture the events are recorded with cudaEventRecordExternal, so
// that they become event-record nodes of the graph and time every replay; outside a
// capture they are plain event records (the external flag is refused there).
bool prof_active() { return g_prof_on.load(std::memory_order_relaxed); }

static void prof_record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void prof_begin(cudaStream_t st, const char* name) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_used >= g_prof.size()) {
        g_prof_dropped = true;
        return;
    }
    const char* tag = t_tag ? t_tag : name;
    if (!g_prof_only.empty() && g_prof_only != tag) return;
    ProfRec& r = g_prof[g_prof_used++];
    r.tag = tag;
    prof_record(r.a, st);
    t_open = &r;
}

void prof_end(cudaStream_t st) {
    if (!t_open) return;
    prof_record(t_open->b, st);
    t_open = nullptr;
}

static sfw_status prof_collect_locked() {
    for (size_t i = 0; i < g_prof_used; ++i) {
        ProfRec& r = g_prof[i];
        SFW_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        SFW_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        prof_accumulate(r.tag, t);
    }
    g_prof_collected = true;
    return SFW_OK;
}

// ------------------------------------------------------------------ geometry of a blur

// Transform grid of a blur whose input lives on the box E and whose output
// (the observation grid) is the sub-box [R, R + n) of E.
struct BlurGeom {
    int n[3], R[3], E[3], P[3], H2;
    Factors fac[3];
    const float2* tw[3];
};

static sfw_status make_blur_geom(TwiddleCache& tc, const int n[3], const int R[3], BlurGeom* g) {
    for (int a = 0; a < 3; ++a) {
        g->n[a] = n[a];
        g->R[a] = R[a];
        g->E[a] = n[a] + 2 * R[a];
        g->P[a] = next_smooth_even(g->E[a]);
        if (g->P[a] > kMaxLen) return fail(SFW_ERR_SHAPE, "FFT length %d > %d", g->P[a], kMaxLen);
        if (!factorize(g->P[a], &g->fac[a])) return fail(SFW_ERR_SHAPE, "cannot factor %d", g->P[a]);
        SFW_TRY(tc.get(g->P[a], &g->tw[a]));
    }
    g->H2 = g->P[2] / 2 + 1;
    return SFW_OK;
}

static size_t blur_buf_elems(const BlurGeom& g) {
    return (size_t)g.E[0] * g.P[1] * g.H2;  // >= every intermediate of forward and transpose
}

// Profiling tags of the five passes of a blur (or of its transpose).
struct PassTags {
    const char* r2c;
    const char* fwd1;
    const char* axis0;
    const char* inv1;
    const char* c2r;
    const char* head;   // r2c + fwd1 per slab
    const char* tail;   // inv1 + c2r per slab
};
static const PassTags kBlurTags = {"blur_r2c", "blur_c2c_fwd", "blur_axis0", "blur_c2c_inv", "blur_c2r",
                                   "blur_head", "blur_tail"};
static const PassTags kBackTags = {"bp_r2c", "bp_c2c_fwd", "bp_axis0", "bp_c2c_inv", "bp_c2r",
                                   "bp_head", "bp_tail"};
static const PassTags kTableTags = {"table_r2c", "table_c2c_fwd", "table_axis0", "table_c2c_inv", "table_c2r",
                                    "table_head", "table_tail"};
static const char* const kCertHeadTag = "cert_head";
static const char* const kCertTailTag = "cert_tail";
static const char* const kCertX0Tag = "cert_x0fwd";      // forward axis-0 spectrum (tensor-core path)
static const char* const kCertTcTag = "cert_axis0_tc";   // axis-0 inverse on the tensor cores
static const char* const kCertC2rTcTag = "cert_c2r_tc";  // axis-2 real inverse + max on the tensor cores
static const PassTags kCertTags = {"cert_r2c", "cert_c2c_fwd", "cert_axis0", "cert_c2c_inv", "cert_c2r_max",
                                   nullptr, nullptr};

// Axes 1 and 2 of a blur per slab of axis 0 (one CTA each) where the slab fits in
// shared memory.  A batch records the slab passes only if those of every volume fit
// (its volumes must record the same sequence of passes).
static thread_local bool g_slab_batch = false;
static bool use_slab(const SlabPass& s) {
    if (g_recorder) return g_slab_batch;
    return s.nslab > 0 && slab_smem(s) > 0;
}

static SlabPass slab_pass(const BlurGeom& g, int mode, int nslab) {
    SlabPass s;
    memset(&s, 0, sizeof(s));
    s.mode = mode;
    s.nslab = nslab;
    s.P1 = g.P[1];
    s.P2 = g.P[2];
    s.H2 = g.H2;
    return s;
}

// Whether all four slab passes of a blur and its transpose fit in shared memory.
static bool blur_slabs_fit(const BlurGeom& g) {
    SlabPass a = slab_pass(g, SLAB_HEAD, g.E[0]);
    a.rows = g.E[1];
    a.cols = g.E[2];
    SlabPass b = slab_pass(g, SLAB_RESIDUAL, g.n[0]);
    b.m1 = g.n[1];
    b.m2 = g.n[2];
    SlabPass c = slab_pass(g, SLAB_HEAD, g.n[0]);
    c.rows = g.n[1];
    c.cols = g.n[2];
    SlabPass d = slab_pass(g, SLAB_STORE, g.E[0]);
    d.m1 = g.E[1];
    d.m2 = g.E[2];
    return slab_smem(a) && slab_smem(b) && slab_smem(c) && slab_smem(d);
}

static LineSet ls(long long Sa, long long Sb, long long Sj, long long B) {
    LineSet s;
    s.Sa = Sa;
    s.Sb = Sb;
    s.Sj = Sj;
    s.B = B;
    return s;
}

// Blur forward: f on E (dense) -> observation grid through C2R epilogue `ep`
// (fields in/lin/nlines/L/fac/tw/out_off/out_len/lout filled here).
static sfw_status blur_forward(const BlurGeom& g, const float* f, const void* spec, int spec_kind,
                               float2* bufA, float2* bufB, C2RPass ep, cudaStream_t st,
                               int* c2r_blocks_out, const PassTags& tg = kBlurTags) {
    const int E0 = g.E[0], E1 = g.E[1], E2 = g.E[2];
    const int P0 = g.P[0], P1 = g.P[1], P2 = g.P[2], H2 = g.H2;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    SlabPass head = slab_pass(g, SLAB_HEAD, E0);
    head.rows = E1;
    head.cols = E2;
    head.rin = f;
    head.cout = bufB;
    if (use_slab(head)) {   // axes 2 and 1 forward per slab: f -> (E0, P1, H2)
        LaunchTag lt__(tg.head);
        SFW_TRY(launch_slab(head, st));
    } else {
    {   // axis 2: real lines of f -> half spectra (E0, E1, H2)
        R2CPass p;
        p.in = f;
        p.lin = ls((long long)E1 * E2, E2, 1, E1);
        p.nlines = (long long)E0 * E1;
        p.in_off = 0;
        p.in_len = E2;
        p.L = P2;
        p.fac = g.fac[2];
        p.tw = g.tw[2];
        p.out = bufA;
        p.lout = ls((long long)E1 * H2, H2, 1, E1);
        {
            LaunchTag lt__(tg.r2c);
            SFW_TRY(launch_r2c(p, st));
        }
    }
    {   // axis 1 forward: (E0, E1, H2) -> (E0, P1, H2)
        C2CPass p;
        p.in = bufA;
        p.out = bufB;
        p.lin = ls((long long)E1 * H2, 1, H2, H2);
        p.lout = ls((long long)P1 * H2, 1, H2, H2);
        p.nlines = (long long)E0 * H2;
        p.L = P1;
        p.in_off = 0;
        p.in_len = E1;
        p.out_off = 0;
        p.out_len = P1;
        p.dir = -1;
        p.scale = 1.f;
        p.fac = g.fac[1];
        p.tw = g.tw[1];
        {
            LaunchTag lt__(tg.fwd1);
            SFW_TRY(launch_c2c(p, st));
        }
    }
    }
    {   // axis 0: forward, times H^, inverse, keep rows [R0, R0 + n0) -> (n0, P1, H2)
        MulPass p;
        const long long nl = (long long)P1 * H2;
        p.in = bufB;
        p.lin = ls(0, 1, nl, nl);
        p.in_off = 0;
        p.in_len = E0;
        p.nlines = nl;
        p.L = P0;
        p.fac = g.fac[0];
        p.tw = g.tw[0];
        p.spec = spec;
        p.lspec = ls(0, 1, nl, nl);
        p.spec_stride = 0;
        p.nspec = 1;
        p.ktotal = 1;
        p.spec_kind = spec_kind;
        p.conj_spec = 0;
        p.out = bufA;
        p.lout = ls(0, 1, nl, nl);
        p.out_stride = 0;
        p.out_off = g.R[0];
        p.out_len = n0;
        {
            LaunchTag lt__(tg.axis0);
            SFW_TRY(launch_mul(p, st));
        }
    }
    if ((ep.mode == C2R_STORE || ep.mode == C2R_RESIDUAL) && ep.scale == 1.f) {
        // axes 1 and 2 inverse per slab with the store or residual epilogue
        SlabPass tail = slab_pass(g, ep.mode == C2R_STORE ? SLAB_STORE : SLAB_RESIDUAL, n0);
        tail.cin = bufA;
        tail.o1 = g.R[1];
        tail.m1 = n1;
        tail.o2 = g.R[2];
        tail.m2 = n2;
        tail.rout = ep.out;
        tail.y = ep.y;
        tail.partials = ep.partials;
        tail.counter = ep.counter;
        tail.loss_out = ep.loss_out;
        tail.w = ep.w;
        tail.nw = ep.nw;
        tail.w_stride = ep.w_stride;
        tail.lambda = ep.lambda;
        if (use_slab(tail)) {
            if (c2r_blocks_out) *c2r_blocks_out = 2 * n0;   // two CTAs per slab
            LaunchTag lt__(tg.tail);
            return launch_slab(tail, st);
        }
    }
    {   // axis 1 inverse: (n0, P1, H2) -> (n0, n1, H2), rows [R1, R1 + n1)
        C2CPass p;
        p.in = bufA;
        p.out = bufB;
        p.lin = ls((long long)P1 * H2, 1, H2, H2);
        p.lout = ls((long long)n1 * H2, 1, H2, H2);
        p.nlines = (long long)n0 * H2;
        p.L = P1;
        p.in_off = 0;
        p.in_len = P1;
        p.out_off = g.R[1];
        p.out_len = n1;
        p.dir = 1;
        p.scale = 1.f;
        p.fac = g.fac[1];
        p.tw = g.tw[1];
        {
            LaunchTag lt__(tg.inv1);
            SFW_TRY(launch_c2c(p, st));
        }
    }
    // axis 2 inverse with the epilogue: (n0, n1, H2) -> grid (n0, n1, n2)
    ep.in = bufB;
    ep.lin = ls((long long)n1 * H2, H2, 1, n1);
    ep.nlines = (long long)n0 * n1;
    ep.in_spec_stride = 0;
    if (ep.mode != C2R_CERTMAX) ep.nspec = 1;
    ep.L = P2;
    ep.fac = g.fac[2];
    ep.tw = g.tw[2];
    ep.out_off = g.R[2];
    ep.out_len = n2;
    ep.lout = ls((long long)n1 * n2, n2, 1, n1);
    LaunchTag lt__(tg.c2r);
    return launch_c2r(ep, st, c2r_blocks_out);
}

// Transpose of the blur: r on the grid -> b on E (dense), b(t) = sum_s H(s - t) r(s).
static sfw_status blur_transpose(const BlurGeom& g, const float* r, const void* spec,
                                 int spec_kind, float2* bufA, float2* bufB, float* b,
                                 cudaStream_t st, const PassTags& tg = kBackTags) {
    const int E0 = g.E[0], E1 = g.E[1], E2 = g.E[2];
    const int P0 = g.P[0], P1 = g.P[1], P2 = g.P[2], H2 = g.H2;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    SlabPass head = slab_pass(g, SLAB_HEAD, n0);
    head.rows = n1;
    head.cols = n2;
    head.o1 = g.R[1];
    head.o2 = g.R[2];
    head.rin = r;
    head.cout = bufB;
    if (use_slab(head)) {   // axes 2 and 1 forward per slab, r placed at [R1, R2): -> (n0, P1, H2)
        LaunchTag lt__(tg.head);
        SFW_TRY(launch_slab(head, st));
    } else {
    {   // axis 2: grid lines of r placed at rows [R2, R2 + n2) -> (n0, n1, H2)
        R2CPass p;
        p.in = r;
        p.lin = ls((long long)n1 * n2, n2, 1, n1);
        p.nlines = (long long)n0 * n1;
        p.in_off = g.R[2];
        p.in_len = n2;
        p.L = P2;
        p.fac = g.fac[2];
        p.tw = g.tw[2];
        p.out = bufA;
        p.lout = ls((long long)n1 * H2, H2, 1, n1);
        {
            LaunchTag lt__(tg.r2c);
            SFW_TRY(launch_r2c(p, st));
        }
    }
    {   // axis 1 forward, rows at [R1, R1 + n1): (n0, n1, H2) -> (n0, P1, H2)
        C2CPass p;
        p.in = bufA;
        p.out = bufB;
        p.lin = ls((long long)n1 * H2, 1, H2, H2);
        p.lout = ls((long long)P1 * H2, 1, H2, H2);
        p.nlines = (long long)n0 * H2;
        p.L = P1;
        p.in_off = g.R[1];
        p.in_len = n1;
        p.out_off = 0;
        p.out_len = P1;
        p.dir = -1;
        p.scale = 1.f;
        p.fac = g.fac[1];
        p.tw = g.tw[1];
        {
            LaunchTag lt__(tg.fwd1);
            SFW_TRY(launch_c2c(p, st));
        }
    }
    }
    {   // axis 0: forward (rows at [R0, R0 + n0)), times conj(H^), inverse -> (E0, P1, H2)
        MulPass p;
        const long long nl = (long long)P1 * H2;
        p.in = bufB;
        p.lin = ls(0, 1, nl, nl);
        p.in_off = g.R[0];
        p.in_len = n0;
        p.nlines = nl;
        p.L = P0;
        p.fac = g.fac[0];
        p.tw = g.tw[0];
        p.spec = spec;
        p.lspec = ls(0, 1, nl, nl);
        p.spec_stride = 0;
        p.nspec = 1;
        p.ktotal = 1;
        p.spec_kind = spec_kind;
        p.conj_spec = 1;
        p.out = bufA;
        p.lout = ls(0, 1, nl, nl);
        p.out_stride = 0;
        p.out_off = 0;
        p.out_len = E0;
        {
            LaunchTag lt__(tg.axis0);
            SFW_TRY(launch_mul(p, st));
        }
    }
    {
        SlabPass tail = slab_pass(g, SLAB_STORE, E0);
        tail.cin = bufA;
        tail.m1 = E1;
        tail.m2 = E2;
        tail.rout = b;
        if (use_slab(tail)) {   // axes 1 and 2 inverse per slab: -> b (E0, E1, E2)
            LaunchTag lt__(tg.tail);
            return launch_slab(tail, st);
        }
    }
    {   // axis 1 inverse: (E0, P1, H2) -> (E0, E1, H2)
        C2CPass p;
        p.in = bufA;
        p.out = bufB;
        p.lin = ls((long long)P1 * H2, 1, H2, H2);
        p.lout = ls((long long)E1 * H2, 1, H2, H2);
        p.nlines = (long long)E0 * H2;
        p.L = P1;
        p.in_off = 0;
        p.in_len = P1;
        p.out_off = 0;
        p.out_len = E1;
        p.dir = 1;
        p.scale = 1.f;
        p.fac = g.fac[1];
        p.tw = g.tw[1];
        {
            LaunchTag lt__(tg.inv1);
            SFW_TRY(launch_c2c(p, st));
        }
    }
    C2RPass p;
    memset(&p, 0, sizeof(p));
    p.in = bufB;
    p.lin = ls((long long)E1 * H2, H2, 1, E1);
    p.nlines = (long long)E0 * E1;
    p.nspec = 1;
    p.L = P2;
    p.fac = g.fac[2];
    p.tw = g.tw[2];
    p.out_off = 0;
    p.out_len = E2;
    p.lout = ls((long long)E1 * E2, E2, 1, E1);
    p.scale = 1.f;
    p.mode = C2R_STORE;
    p.out = b;
    LaunchTag lt__(tg.c2r);
    return launch_c2r(p, st, nullptr);
}

// Full forward transform of a dense real volume on the grid P (no padding):
// out (P0, P1, P2/2 + 1) complex, scaled by `scale`.  tmp holds P0*P1*H2.
static sfw_status fft3_forward(const int P[3], const Factors fac[3], const float2* const tw[3],
                               const float* in, float2* tmp, float2* out, float scale,
                               cudaStream_t st) {
    const int P0 = P[0], P1 = P[1], P2 = P[2], H2 = P2 / 2 + 1;
    {
        R2CPass p;
        p.in = in;
        p.lin = ls((long long)P1 * P2, P2, 1, P1);
        p.nlines = (long long)P0 * P1;
        p.in_off = 0;
        p.in_len = P2;
        p.L = P2;
        p.fac = fac[2];
        p.tw = tw[2];
        p.out = out;
        p.lout = ls((long long)P1 * H2, H2, 1, P1);
        {
            LaunchTag lt__("fft3_r2c");
            SFW_TRY(launch_r2c(p, st));
        }
    }
    {
        C2CPass p;
        p.in = out;
        p.out = tmp;
        p.lin = ls((long long)P1 * H2, 1, H2, H2);
        p.lout = p.lin;
        p.nlines = (long long)P0 * H2;
        p.L = P1;
        p.in_off = 0;
        p.in_len = P1;
        p.out_off = 0;
        p.out_len = P1;
        p.dir = -1;
        p.scale = 1.f;
        p.fac = fac[1];
        p.tw = tw[1];
        {
            LaunchTag lt__("fft3_c2c1");
            SFW_TRY(launch_c2c(p, st));
        }
    }
    {
        C2CPass p;
        const long long nl = (long long)P1 * H2;
        p.in = tmp;
        p.out = out;
        p.lin = ls(0, 1, nl, nl);
        p.lout = p.lin;
        p.nlines = nl;
        p.L = P0;
        p.in_off = 0;
        p.in_len = P0;
        p.out_off = 0;
        p.out_len = P0;
        p.dir = -1;
        p.scale = scale;
        p.fac = fac[0];
        p.tw = tw[0];
        {
            LaunchTag lt__("fft3_c2c0");
            SFW_TRY(launch_c2c(p, st));
        }
    }
    return SFW_OK;
}

}  // namespace sfw

using namespace sfw;

// ------------------------------------------------------------------ the plan

struct sfw_plan {
    int n[3], R[3], E[3];
    long long V, VE;
    float eps;
    int precision;
    TwiddleCache tw;
    BlurGeom blur;
    // certificate grid
    int K;
    std::vector<float> sigmas, ds;  // per kernel k
    int Pc[3], H2c;
    int hc[3];          // half-widths of the kernel family's support (K_k = 0 beyond, per axis)
    Factors facc[3];
    const float2* twc[3];
    void* table;        // K spectra of Pc0 rows x (Pc1 H2c) lines (layout: table_lines)
    LineSet table_lines;          // line -> offset within a spectrum (rows table_lines.Sj apart)
    long long table_stride;       // elements between spectra
    int table_kind;
    size_t table_bytes;
    int real_table;
    // device buffers
    float* psf;
    float2* Hspec;      // P0 x P1 x H2 (complex64), scaled by 1/|P|
    float2* bufA;
    float2* bufB;
    float* fE;          // rendered atoms on E
    float* bE;          // back-projected residual on E
    float* r;           // residual on the grid
    double* loss_parts;
    int loss_parts_len;
    double* grad_parts;
    int grad_parts_atoms;
    float2* cA;
    float2* cB;
    float2* cC;
    unsigned long long* best_key;
    unsigned int* ctr;            // last-block counters of the fused loss / argmax finalisers
    unsigned int* adj_ctr;        // one last-block counter per atom of the adjoint
    unsigned long long* vox_key;  // V per-voxel certificate keys
    float* grid_sd;               // 2K floats on the device: sigma_k, d_k
    float* vmax;                  // V: per-voxel max over k (top-k path)
    int* vargk;                   // V: its k
    float* cand_val;              // 64 grid values of the top-k voxels
    int64_t* cand_idx;            // their voxel indices
    float* cand_theta;            // 64 x 5 parameter rows
    double* cand_eta;             // 64 FP32-summed certificates
    float* gram_cols;             // N x V blurred unit atoms (grown on demand, sfw_gram)
    int gram_cap;                 // atoms gram_cols can hold
    float* unit_slot;             // one atom (m0, m1, m2, sigma, d, w = 1)
    int num_sms;
    cudaEvent_t ev_fork, ev_join;  // sfw_step: residual ready / certificate done
    cudaEvent_t ev_grad;           // sfw_step_topk: back-projection and adjoint sums done
    cudaEvent_t ev_graph;          // sfw_step: recorded after each launch of the cached graph
    cudaStream_t cap_own, aux_own; // sfw_step captures its graph on these (origin, branch)
    // certificate tail by TMA: tensor map of the line-group-major axis-0 output (opaque)
    alignas(64) unsigned char tail_tmap[128];
    bool tail_tma;
    int tail_boxg, tail_nbox;
    int* tail_err;                 // device flag: a tail CTA's copies did not land in time
    // sfw_step's own CUDA graph: captured at the second consecutive call with the same
    // arguments, replayed while they stay the same
    struct StepKey {
        const void* ptr[10];
        int N;
        double lambda;
        bool operator==(const StepKey& o) const {
            for (int i = 0; i < 10; ++i)
                if (ptr[i] != o.ptr[i]) return false;
            return N == o.N && lambda == o.lambda;
        }
    } step_key;
    bool step_seen;
    cudaGraphExec_t step_exec;
    unsigned long long* red_scratch;
    long long red_scratch_len;
    size_t ws_bytes;
    std::vector<void*> allocations;
    // routes: requested (AUTO, FFT, DIRECT) and in use (FFT or DIRECT) per operation
    int route;
    int route_blur, route_cert;
    bool fft_cert;                 // the kernel-family table and the certificate FFT buffers exist
    bool direct_ok;                // the direct-sum buffers exist
    float* gtab;                   // unit atoms g_k on their boxes (direct certificate)
    int2* gkern;                   // per k: (offset in gtab, half-width)
    float* bE_cert;                // H^T r of the direct certificate (bE belongs to the gradient)
    // tensor-core axis-0 pass (real bf16 tables): the table as per-line MMA operands and the
    // forward axis-0 spectrum of the residual
    bool tc_ready;                 // the tensor-core operands exist
    bool tc;                       // the certificate's axis-0 stage runs on the tensor cores
    __nv_bfloat16* tc_table;
    __nv_bfloat16* tc_dft;         // the inverse DFT rows (A operands), per half of the n0 rows
    int tc_Kp, tc_Np;
    float2* cX;
    // the real inverse along axis 2 on the tensor cores (per-axis tails): its matrix and the
    // tensor map of the spectra, whose lines then have the even pitch H2p
    float* tc_c2r_C;
    bool c2r_tma;
    int H2p;
    alignas(64) unsigned char c2r_tmap[128];
    double* dir_parts;             // criterion partials of the direct blur
    int dir_parts_len;
};

static sfw_status plan_alloc(sfw_plan* p, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SFW_ERR_ALLOC, "cudaMalloc(%zu bytes) failed", bytes);
    }
    p->allocations.push_back(*ptr);
    p->ws_bytes += bytes;
    return SFW_OK;
}

template <typename T>
static sfw_status plan_alloc_t(sfw_plan* p, T** ptr, size_t count) {
    void* v = nullptr;
    SFW_TRY(plan_alloc(p, &v, sizeof(T) * count));
    *ptr = static_cast<T*>(v);
    return SFW_OK;
}

static void plan_free(sfw_plan* p) {
    if (!p) return;
    if (p->step_exec) cudaGraphExecDestroy(p->step_exec);
    p->step_exec = nullptr;
    if (p->aux_own) cudaStreamDestroy(p->aux_own);
    if (p->cap_own) cudaStreamDestroy(p->cap_own);
    p->aux_own = p->cap_own = nullptr;
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->ev_grad) cudaEventDestroy(p->ev_grad);
    p->ev_grad = nullptr;
    if (p->ev_graph) cudaEventDestroy(p->ev_graph);
    p->ev_fork = p->ev_join = p->ev_graph = nullptr;
    if (p->gram_cols) cudaFree(p->gram_cols);
    p->gram_cols = nullptr;
    for (void* q : p->allocations) cudaFree(q);
    p->allocations.clear();
    p->tw.release();
}

// Build the kernel-family table: for each k, K_k = H * g_k at every grid
// displacement |x_a| <= n_a - 1 (a blur of one centred atom on the grid of
// shape 2n - 1), placed for correlation on Pc and transformed.
static sfw_status build_table(sfw_plan* p, cudaStream_t st) {
    const int K = p->K;
    if (K == 0) return SFW_OK;
    int n2[3];
    for (int a = 0; a < 3; ++a) n2[a] = 2 * p->n[a] - 1;
    BlurGeom g;
    SFW_TRY(make_blur_geom(p->tw, n2, p->R, &g));
    const long long Pc_tot = (long long)p->Pc[0] * p->Pc[1] * p->Pc[2];
    const long long spec_elems = (long long)p->Pc[0] * p->Pc[1] * p->H2c;
    const long long Pg_tot = (long long)g.P[0] * g.P[1] * g.P[2];
    const long long Eg_tot = (long long)g.E[0] * g.E[1] * g.E[2];
    const long long Ng_tot = (long long)n2[0] * n2[1] * n2[2];
    // temporaries
    std::vector<void*> tmp;
    auto talloc = [&](void** q, size_t bytes) -> sfw_status {
        cudaError_t e = cudaMalloc(q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SFW_ERR_ALLOC, "table build: cudaMalloc(%zu) failed", bytes);
        }
        tmp.push_back(*q);
        return SFW_OK;
    };
    sfw_status st_ret = SFW_OK;
    float2 *Hg = nullptr, *gA = nullptr, *gB = nullptr, *full = nullptr, *ftmp = nullptr;
    float *fE = nullptr, *kx = nullptr, *wrapped = nullptr, *stats = nullptr;
    float* atom = nullptr;
    do {
        const size_t gspec = (size_t)g.P[0] * g.P[1] * g.H2;
        const size_t gbuf = blur_buf_elems(g) > gspec ? blur_buf_elems(g) : gspec;
        if ((st_ret = talloc((void**)&Hg, sizeof(float2) * gspec))) break;
        if ((st_ret = talloc((void**)&gA, sizeof(float2) * gbuf))) break;
        if ((st_ret = talloc((void**)&gB, sizeof(float2) * gbuf))) break;
        if ((st_ret = talloc((void**)&fE, sizeof(float) * (size_t)(Eg_tot > Pg_tot ? Eg_tot : Pg_tot)))) break;
        if ((st_ret = talloc((void**)&kx, sizeof(float) * (size_t)Ng_tot))) break;
        if ((st_ret = talloc((void**)&wrapped, sizeof(float) * (size_t)Pc_tot))) break;
        if ((st_ret = talloc((void**)&full, sizeof(float2) * (size_t)K * spec_elems))) break;
        if ((st_ret = talloc((void**)&ftmp, sizeof(float2) * (size_t)spec_elems))) break;
        if ((st_ret = talloc((void**)&stats, sizeof(float) * 2))) break;
        if ((st_ret = talloc((void**)&atom, sizeof(float) * 6))) break;
        // H on the blur grid of the shape 2n - 1
        if ((st_ret = launch_wrap_psf(p->psf, p->R, g.P, fE, st))) break;
        if ((st_ret = fft3_forward(g.P, g.fac, g.tw, fE, gA, Hg, 1.0f / (float)Pg_tot, st))) break;
        for (int k = 0; k < K && st_ret == SFW_OK; ++k) {
            // one unit atom at the centre (n - 1) of the (2n - 1) grid
            float h_atom[6] = {(float)(p->n[0] - 1), (float)(p->n[1] - 1), (float)(p->n[2] - 1),
                               p->sigmas[k], p->ds[k], 1.0f};
            cudaError_t e = cudaMemcpyAsync(atom, h_atom, sizeof(h_atom), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) {
                st_ret = cuda_fail(e, "table atom upload");
                break;
            }
            AtomsDev a;
            a.N = 1;
            a.m = atom;
            a.sigma = atom + 3;
            a.d = atom + 4;
            a.w = atom + 5;
            if ((st_ret = launch_render(a, g.E, g.R, p->eps, fE, st))) break;
            C2RPass ep;
            memset(&ep, 0, sizeof(ep));
            ep.mode = C2R_STORE;
            ep.scale = 1.f;
            ep.out = kx;
            if ((st_ret = blur_forward(g, fE, Hg, SPEC_C64, gA, gB, ep, st, nullptr, kTableTags))) break;
            if ((st_ret = launch_wrap_kernel(kx, p->n, p->hc, p->Pc, wrapped, st))) break;
            if ((st_ret = fft3_forward(p->Pc, p->facc, p->twc, wrapped, ftmp, full + (size_t)k * spec_elems,
                                       1.0f / (float)Pc_tot, st)))
                break;
            e = cudaStreamSynchronize(st);  // the atom slot is rewritten next iteration
            if (e != cudaSuccess) {
                st_ret = cuda_fail(e, "table build");
                break;
            }
        }
        if (st_ret) break;
        // real spectra when the family is even (symmetric H): keep Re only
        cudaMemsetAsync(stats, 0, sizeof(float) * 2, st);
        if ((st_ret = launch_spec_stats(full, (long long)K * spec_elems, stats, st))) break;
        float h_stats[2];
        cudaError_t e = cudaMemcpyAsync(h_stats, stats, sizeof(h_stats), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            st_ret = cuda_fail(e, "table stats");
            break;
        }
        p->real_table = h_stats[1] <= 1e-6f * h_stats[0];
        int kind;
        size_t esz;
        if (p->precision == SFW_PREC_BF16) {
            kind = p->real_table ? SPEC_RBF16 : SPEC_CBF16;
            esz = p->real_table ? 2 : 4;
        } else {
            kind = p->real_table ? SPEC_R32 : SPEC_C64;
            esz = p->real_table ? 4 : 8;
        }
        p->table_kind = kind;
        // axis-0 lines of the certificate: Pc1 x H2c per spectrum, Pc0 rows.  For the
        // register-resident lengths each warp's lines sit together with all their rows.
        const long long nl = (long long)p->Pc[1] * p->H2c;
        const int grp = reg_line_group(p->Pc[0]);
        if (grp > 0) {
            const long long ng = (nl + grp - 1) / grp;
            p->table_lines = ls((long long)grp * p->Pc[0], 1, grp, grp);
            p->table_stride = ng * grp * p->Pc[0];
        } else {
            p->table_lines = ls(0, 1, nl, nl);
            p->table_stride = spec_elems;
        }
        p->table_bytes = esz * (size_t)K * (size_t)p->table_stride;
        if (p->precision == SFW_PREC_BF16 && p->real_table) {
            // the tensor-core axis-0 pass: T_l per line as the MMA's B operand (Np kernels x Kp
            // points, bf16); the plain bf16 table below stays for batches (recorded FFT passes)
            const int Kp = (p->Pc[0] + 63) / 64 * 64;
            const int Np = K <= 16 ? 16 : K <= 32 ? 32 : K <= 64 ? 64 : 128;
            if (K <= 128 && tc_smem_bytes(Kp, Np, p->Pc[0]) <= 227u * 1024u) {
                p->tc_Kp = Kp;
                p->tc_Np = Np;
                if ((st_ret = plan_alloc_t(p, &p->tc_table, (size_t)nl * Np * Kp))) break;
                if ((st_ret = plan_alloc_t(p, &p->cX, (size_t)nl * p->Pc[0]))) break;
                if ((st_ret = launch_tc_table(full, spec_elems, K, p->Pc[0], nl, Np, Kp, p->tc_table, st))) break;
                const size_t halves = (size_t)((p->n[0] + 63) / 64);
                if ((st_ret = plan_alloc_t(p, &p->tc_dft, halves * 128 * 2 * (size_t)Kp))) break;
                if ((st_ret = launch_tc_dft(p->n[0], p->Pc[0], Kp, p->tc_dft, st))) break;
                p->tc_ready = p->tc = true;
                // the tail's real inverse along axis 2 (per-axis tails only: the slab tails fuse
                // axes 1 and 2 already)
                if (!cert_tail_supported(p->Pc[1], p->Pc[2], p->n[1], p->n[2]) && p->n[2] <= 128 &&
                    p->H2c == p->Pc[2] / 2 + 1 && tc_c2r_fits(p->H2c)) {
                    const size_t cbytes = (size_t)tc_c2r_chunks(p->H2c) * 128 * 128;
                    if ((st_ret = plan_alloc(p, (void**)&p->tc_c2r_C, cbytes))) break;
                    if ((st_ret = launch_tc_c2r_matrix(p->Pc[2], p->H2c, p->n[2], p->tc_c2r_C, st))) break;
                    p->c2r_tma = make_c2r_tmap(p->cA, p->H2c, p->H2p, (long long)p->n[0] * p->n[1], K, p->c2r_tmap);
                }
            }
        }
        if ((st_ret = plan_alloc(p, &p->table, p->table_bytes))) break;
        if (cudaMemsetAsync(p->table, 0, p->table_bytes, st) != cudaSuccess) {
            st_ret = cuda_fail(cudaGetLastError(), "table clear");
            break;
        }
        if ((st_ret = launch_spec_convert(full, (long long)K * spec_elems, kind, p->table, p->Pc[0], nl,
                                          grp, st)))
            break;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) st_ret = cuda_fail(e, "table build");
    } while (0);
    cudaStreamSynchronize(st);
    for (void* q : tmp) cudaFree(q);
    return st_ret;
}

// Buffers of the direct-sum route: the criterion partials and, with a certificate
// grid, every unit atom g_k tabulated on the cube of its cut-off radius (rendered by the
// atom kernel itself, so the truncation g >= eps is the rendering's) plus a
// back-projection buffer of its own.  Boxes beyond 2^28 values in total leave the
// direct certificate out of an AUTO plan (SFW_ERR_SHAPE for a DIRECT plan).
static sfw_status build_direct(sfw_plan* p, cudaStream_t st) {
    p->dir_parts_len = 8 * p->num_sms;
    SFW_TRY(plan_alloc_t(p, &p->dir_parts, (size_t)p->dir_parts_len));
    const int K = p->K;
    if (K == 0) return SFW_OK;
    int emax = p->E[0];
    for (int a = 1; a < 3; ++a) emax = p->E[a] > emax ? p->E[a] : emax;
    const double L = 2.0 * log(1.0 / (double)p->eps);
    std::vector<int2> kern(K);
    std::vector<float> hm(3 * (size_t)K), hs(K), hd(K), hw(K, 1.0f);
    long long total = 0;
    for (int k = 0; k < K; ++k) {
        const double rho = (double)p->sigmas[k] * pow(L, 1.0 / (double)p->ds[k]);
        int h = (int)ceil(rho) + 1;
        if (h > emax - 1) h = emax - 1;
        kern[k] = make_int2((int)total, h);
        total += (long long)(2 * h + 1) * (2 * h + 1) * (2 * h + 1);
        for (int a = 0; a < 3; ++a) hm[3 * k + a] = (float)h;
        hs[k] = p->sigmas[k];
        hd[k] = p->ds[k];
    }
    if (total > (1LL << 28)) {
        if (p->route == SFW_ROUTE_DIRECT)
            return fail(SFW_ERR_SHAPE, "direct certificate: unit-atom boxes need %lld values (> 2^28)", total);
        return SFW_OK;
    }
    SFW_TRY(plan_alloc_t(p, &p->gtab, (size_t)total));
    SFW_TRY(plan_alloc_t(p, &p->gkern, (size_t)K));
    SFW_TRY(plan_alloc_t(p, &p->bE_cert, (size_t)p->VE));
    SFW_CUDA(cudaMemcpy(p->gkern, kern.data(), sizeof(int2) * K, cudaMemcpyHostToDevice));
    float* dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, sizeof(float) * 6 * (size_t)K);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SFW_ERR_ALLOC, "direct certificate: atom upload");
    }
    sfw_status s = SFW_OK;
    do {
        float* dm = dev;
        float* dsg = dev + 3 * K;
        float* dd = dev + 4 * K;
        float* dw = dev + 5 * K;
        if ((e = cudaMemcpy(dm, hm.data(), sizeof(float) * 3 * K, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(dsg, hs.data(), sizeof(float) * K, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(dd, hd.data(), sizeof(float) * K, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(dw, hw.data(), sizeof(float) * K, cudaMemcpyHostToDevice)) != cudaSuccess) {
            s = cuda_fail(e, "direct certificate: atom upload");
            break;
        }
        const int R0[3] = {0, 0, 0};
        for (int k = 0; k < K && s == SFW_OK; ++k) {
            AtomsDev a;
            a.N = 1;
            a.m = dm + 3 * k;
            a.sigma = dsg + k;
            a.d = dd + k;
            a.w = dw + k;
            const int wd = 2 * kern[k].y + 1;
            const int box[3] = {wd, wd, wd};
            s = launch_render(a, box, R0, p->eps, p->gtab + kern[k].x, st);
        }
        if (s) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) s = cuda_fail(e, "direct certificate tables");
    } while (0);
    cudaStreamSynchronize(st);
    cudaFree(dev);
    return s;
}

// Phi f_E on the grid by the plan's convolution route.
static sfw_status plan_blur_store(sfw_plan* p, const float* fE, float* out, cudaStream_t st) {
    if (p->route_blur == SFW_ROUTE_DIRECT) {
        if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the FFT route only");
        DirectBlur b;
        memset(&b, 0, sizeof(b));
        b.fE = fE;
        b.H = p->psf;
        for (int a = 0; a < 3; ++a) {
            b.n[a] = p->n[a];
            b.R[a] = p->R[a];
        }
        b.out = out;
        b.num_sms = p->num_sms;
        return launch_direct_blur(b, st);
    }
    C2RPass ep;
    memset(&ep, 0, sizeof(ep));
    ep.mode = C2R_STORE;
    ep.scale = 1.f;
    ep.out = out;
    return blur_forward(p->blur, fE, p->Hspec, SPEC_C64, p->bufA, p->bufB, ep, st, nullptr);
}

// b = Phi^T r on E by the plan's convolution route.
static sfw_status plan_transpose(sfw_plan* p, const float* r, float* bE, cudaStream_t st) {
    if (p->route_blur == SFW_ROUTE_DIRECT) {
        if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the FFT route only");
        return launch_direct_transpose(r, p->psf, p->n, p->R, bE, p->num_sms, st);
    }
    return blur_transpose(p->blur, r, p->Hspec, SPEC_C64, p->bufA, p->bufB, bE, st);
}

// Median of three timed runs of fn on st (after one untimed run), in ms; < 0 on error.
template <typename F>
static float time_route(F fn, cudaStream_t st) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        cudaGetLastError();
        return -1.f;
    }
    float t[3] = {-1.f, -1.f, -1.f};
    bool ok = fn() == SFW_OK;
    for (int i = 0; i < 3 && ok; ++i) {
        ok = cudaEventRecord(a, st) == cudaSuccess && fn() == SFW_OK && cudaEventRecord(b, st) == cudaSuccess &&
             cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t[i], a, b) == cudaSuccess;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) return -1.f;
    if (t[0] > t[1]) std::swap(t[0], t[1]);
    if (t[1] > t[2]) std::swap(t[1], t[2]);
    if (t[0] > t[1]) std::swap(t[0], t[1]);
    return t[1];
}

static sfw_status check_atoms(const sfw_atoms* a, bool need_nonempty) {
    if (!a) return fail(SFW_ERR_ARG, "atoms is NULL");
    if (a->N < 0 || a->N > 4096) return fail(SFW_ERR_ARG, "atom count %d outside [0, 4096]", a->N);
    if (need_nonempty && a->N == 0) return fail(SFW_ERR_ARG, "atom count must be >= 1");
    if (a->N > 0 && (!a->m || !a->sigma || !a->d || !a->w))
        return fail(SFW_ERR_ARG, "atom arrays must be non-NULL");
    return SFW_OK;
}

static AtomsDev to_dev(const sfw_atoms* a) {
    AtomsDev d;
    d.N = a->N;
    d.m = a->m;
    d.sigma = a->sigma;
    d.d = a->d;
    d.w = a->w;
    return d;
}

extern "C" {

const char* sfw_last_error(void) { return g_err; }

sfw_status sfw_profile_start(int max_launches, const char* only_tag) {
    clear_error();
    if (max_launches < 1 || max_launches > (1 << 20)) return fail(SFW_ERR_ARG, "max_launches outside [1, 2^20]");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    while ((int)g_prof.size() < max_launches) {
        ProfRec r;
        r.tag = nullptr;
        SFW_CUDA(cudaEventCreate(&r.a));
        cudaError_t e = cudaEventCreate(&r.b);
        if (e != cudaSuccess) {
            cudaEventDestroy(r.a);
            return cuda_fail(e, "cudaEventCreate");
        }
        g_prof.push_back(r);
    }
    g_prof_used = 0;
    g_prof_dropped = false;
    g_prof_collected = false;
    g_prof_acc.clear();
    g_prof_only = only_tag ? only_tag : "";
    g_prof_on = true;
    return SFW_OK;
}

sfw_status sfw_profile_collect(void) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return prof_collect_locked();
}

sfw_status sfw_profile_stop(char* json, size_t len) {
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    if (!g_prof_collected) SFW_TRY(prof_collect_locked());
    std::string out = "{";
    for (size_t k = 0; k < g_prof_acc.size(); ++k) {
        char buf[200];
        snprintf(buf, sizeof(buf), "%s\"%s\": [%lld, %.6f]", k ? ", " : "", g_prof_acc[k].tag.c_str(),
                 g_prof_acc[k].count, g_prof_acc[k].ms);
        out += buf;
    }
    out += "}";
    const bool dropped = g_prof_dropped;
    g_prof_used = 0;
    g_prof_acc.clear();
    g_prof_collected = false;
    if (json && len) {
        if (out.size() + 1 > len) return fail(SFW_ERR_ARG, "profile report needs %zu bytes", out.size() + 1);
        memcpy(json, out.c_str(), out.size() + 1);
    }
    if (dropped) return fail(SFW_ERR_ARG, "profile buffer full: some launches were not recorded");
    return SFW_OK;
}

int64_t sfw_launch_count(void) { return g_launches.load(); }

const char* sfw_version(void) { return "sfw-gb300 0.1 (sm_103a)"; }

sfw_status sfw_plan_create(const sfw_plan_desc* desc, sfw_plan** out) {
    clear_error();
    if (!desc || !out) return fail(SFW_ERR_ARG, "desc and out must be non-NULL");
    *out = nullptr;
    for (int a = 0; a < 3; ++a) {
        if (desc->n[a] < 4 || desc->n[a] > 1024) return fail(SFW_ERR_SHAPE, "n[%d]=%d outside [4, 1024]", a, desc->n[a]);
        if (desc->R[a] < 0 || desc->R[a] > 64) return fail(SFW_ERR_SHAPE, "R[%d]=%d outside [0, 64]", a, desc->R[a]);
    }
    if (!desc->psf) return fail(SFW_ERR_ARG, "psf is NULL");
    if (desc->n_sigma < 0 || desc->n_d < 0) return fail(SFW_ERR_ARG, "negative grid size");
    const int K = desc->n_sigma * desc->n_d;
    if (K > 0 && (!desc->sigmas || !desc->ds)) return fail(SFW_ERR_ARG, "grid arrays are NULL");
    if (K > 256) return fail(SFW_ERR_SHAPE, "K=%d > 256 kernels", K);
    for (int i = 0; i < desc->n_sigma; ++i)
        if (!(desc->sigmas[i] >= 0.25f && desc->sigmas[i] <= 16.f)) return fail(SFW_ERR_ARG, "grid sigma outside [0.25, 16]");
    for (int i = 0; i < desc->n_d; ++i)
        if (!(desc->ds[i] >= 0.5f && desc->ds[i] <= 4.f)) return fail(SFW_ERR_ARG, "grid d outside [0.5, 4]");
    if (desc->precision != SFW_PREC_FP32 && desc->precision != SFW_PREC_BF16)
        return fail(SFW_ERR_ARG, "unknown precision %d", desc->precision);
    if (!(desc->eps >= 0.f && desc->eps < 0.1f)) return fail(SFW_ERR_ARG, "eps outside [0, 0.1)");
    if (desc->route != SFW_ROUTE_AUTO && desc->route != SFW_ROUTE_FFT && desc->route != SFW_ROUTE_DIRECT)
        return fail(SFW_ERR_ARG, "unknown route %d", desc->route);

    sfw_plan* p = new (std::nothrow) sfw_plan();
    if (!p) return fail(SFW_ERR_ALLOC, "host allocation");
    p->eps = desc->eps > 0.f ? desc->eps : 1e-9f;
    p->precision = desc->precision;
    p->route = desc->route;
    p->route_blur = p->route_cert = desc->route == SFW_ROUTE_DIRECT ? SFW_ROUTE_DIRECT : SFW_ROUTE_FFT;
    p->fft_cert = K > 0 && desc->route != SFW_ROUTE_DIRECT;
    p->direct_ok = desc->route != SFW_ROUTE_FFT;
    for (int a = 0; a < 3; ++a) {
        p->n[a] = desc->n[a];
        p->R[a] = desc->R[a];
        p->E[a] = desc->n[a] + 2 * desc->R[a];
    }
    p->V = (long long)p->n[0] * p->n[1] * p->n[2];
    p->VE = (long long)p->E[0] * p->E[1] * p->E[2];
    p->K = K;
    for (int i = 0; i < desc->n_sigma; ++i)
        for (int j = 0; j < desc->n_d; ++j) {
            p->sigmas.push_back(desc->sigmas[i]);
            p->ds.push_back(desc->ds[j]);
        }
    if ((long long)K * p->V >= 0xffffffffll) {
        delete p;
        return fail(SFW_ERR_SHAPE, "K * V must stay below 2^32");
    }
    cudaStream_t st = nullptr;
    sfw_status s = SFW_OK;
    do {
        if ((s = make_blur_geom(p->tw, p->n, p->R, &p->blur))) break;
        if (p->fft_cert) {
            // Support of K_k = H * g_k: the rendered atom vanishes beyond its cut-off radius
            // rho_k = sigma_k (2 ln(1/eps))^(1/d_k) and H beyond R, so K_k(x) = 0 once
            // |x_a| > R_a + ceil(max_k rho_k).  A circular correlation on P_a >= n_a + h_a
            // then equals the linear one at every grid displacement.
            double rho = 0.0;
            const double L = 2.0 * log(1.0 / (double)p->eps);
            for (int k = 0; k < K; ++k) {
                const double r = (double)p->sigmas[k] * pow(L, 1.0 / (double)p->ds[k]);
                rho = r > rho ? r : rho;
            }
            for (int a = 0; a < 3; ++a) {
                const double h = (double)p->R[a] + ceil(rho);
                p->hc[a] = h >= (double)(p->n[a] - 1) ? p->n[a] - 1 : (int)h;
                // the smallest 2-3-5 smooth length, unless a register-resident length (64, 128,
                // 256) is within 25 % of it or a compile-time specialised one within 10 %
                const int m = p->n[a] + p->hc[a];
                const int sm = next_smooth_even(m);
                int pick = sm;
                const int reg[3] = {64, 128, 256};
                const int spec[7] = {64, 80, 96, 128, 160, 192, 256};
                int best_spec = 0;
                for (int q = 0; q < 7 && !best_spec; ++q)
                    if (spec[q] >= m) best_spec = spec[q];
                if (best_spec && best_spec <= sm + sm / 10) pick = best_spec;
                for (int q = 0; q < 3; ++q)
                    if (reg[q] >= m && reg[q] <= sm + sm / 4) {
                        pick = reg[q];
                        break;
                    }
                p->Pc[a] = pick;
                if (p->Pc[a] > kMaxLen) {
                    s = fail(SFW_ERR_SHAPE, "certificate FFT length %d > %d", p->Pc[a], kMaxLen);
                    break;
                }
                if (!factorize(p->Pc[a], &p->facc[a])) {
                    s = fail(SFW_ERR_SHAPE, "cannot factor %d", p->Pc[a]);
                    break;
                }
                if ((s = p->tw.get(p->Pc[a], &p->twc[a]))) break;
            }
            if (s) break;
            if (p->n[2] > 256) {
                s = fail(SFW_ERR_SHAPE, "certificate needs n[2] <= 256");
                break;
            }
            p->H2c = p->Pc[2] / 2 + 1;
        }
        const int nh = (2 * p->R[0] + 1) * (2 * p->R[1] + 1) * (2 * p->R[2] + 1);
        if ((s = plan_alloc_t(p, &p->psf, nh))) break;
        cudaError_t e = cudaMemcpy(p->psf, desc->psf, sizeof(float) * nh, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "psf upload");
            break;
        }
        const BlurGeom& g = p->blur;
        const long long Ptot = (long long)g.P[0] * g.P[1] * g.P[2];
        const size_t hs = (size_t)g.P[0] * g.P[1] * g.H2;
        const size_t bb = blur_buf_elems(g);
        if ((s = plan_alloc_t(p, &p->Hspec, hs))) break;
        if ((s = plan_alloc_t(p, &p->bufA, bb > hs ? bb : hs))) break;
        if ((s = plan_alloc_t(p, &p->bufB, bb > hs ? bb : hs))) break;
        if ((s = plan_alloc_t(p, &p->fE, (size_t)(p->VE > Ptot ? p->VE : Ptot)))) break;
        if ((s = plan_alloc_t(p, &p->bE, (size_t)p->VE))) break;
        if ((s = plan_alloc_t(p, &p->r, (size_t)p->V))) break;
        // one partial per residual tile (per-axis passes) or two per slab (slab passes)
        p->loss_parts_len = (int)(((long long)p->n[0] * p->n[1] + 15) / 16) + 16 + 2 * p->n[0];
        if ((s = plan_alloc_t(p, &p->loss_parts, (size_t)p->loss_parts_len))) break;
        p->grad_parts_atoms = 4096;
        if ((s = plan_alloc_t(p, &p->grad_parts, (size_t)p->grad_parts_atoms * kGradChunks * 6))) break;
        if ((s = plan_alloc_t(p, &p->best_key, 2))) break;
        if ((s = plan_alloc_t(p, &p->ctr, 16))) break;
        if ((s = plan_alloc_t(p, &p->adj_ctr, (size_t)p->grad_parts_atoms))) break;
        // the fused finalisers re-arm these themselves after every use
        if (cudaMemset(p->best_key, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMemset(p->ctr, 0, 16 * sizeof(unsigned int)) != cudaSuccess ||
            cudaMemset(p->adj_ctr, 0, (size_t)p->grad_parts_atoms * sizeof(unsigned int)) != cudaSuccess) {
            s = cuda_fail(cudaGetLastError(), "counter reset");
            break;
        }
        if ((s = plan_alloc_t(p, &p->vox_key, (size_t)p->V))) break;
        if ((s = plan_alloc_t(p, &p->unit_slot, 8))) break;
        if (K > 0) {
            if ((s = plan_alloc_t(p, &p->grid_sd, 2 * (size_t)K))) break;
            std::vector<float> sd(2 * (size_t)K);
            for (int k = 0; k < K; ++k) {
                sd[2 * k] = p->sigmas[k];
                sd[2 * k + 1] = p->ds[k];
            }
            e = cudaMemcpy(p->grid_sd, sd.data(), sizeof(float) * sd.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "grid upload");
                break;
            }
            if ((s = plan_alloc_t(p, &p->vmax, (size_t)p->V))) break;
            if ((s = plan_alloc_t(p, &p->vargk, (size_t)p->V))) break;
            if ((s = plan_alloc_t(p, &p->cand_val, 64))) break;
            if ((s = plan_alloc_t(p, &p->cand_idx, 64))) break;
            if ((s = plan_alloc_t(p, &p->cand_theta, 64 * 5))) break;
            if ((s = plan_alloc_t(p, &p->cand_eta, 64))) break;
        }
        {
            int dev = 0;
            cudaGetDevice(&dev);
            p->num_sms = 0;
            cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev);
            if (p->num_sms <= 0) p->num_sms = 1;
        }
        p->red_scratch_len = 1 << 20;
        if ((s = plan_alloc_t(p, &p->red_scratch, (size_t)p->red_scratch_len))) break;
        if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_grad, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_graph, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->aux_own, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&p->cap_own, cudaStreamNonBlocking) != cudaSuccess) {
            s = cuda_fail(cudaGetLastError(), "plan events");
            break;
        }
        if (p->fft_cert) {
            // lines of H2p = H2 rounded up to even complex values (a pitch of whole 16-byte
            // units, as the tensor-core tail's tensor map wants)
            p->H2p = (p->H2c + 1) & ~1;
            const size_t a_el = (size_t)K * p->n[0] * p->n[1] * p->H2p;
            const size_t b_el = (size_t)p->n[0] * p->Pc[1] * p->H2c;
            const size_t c_el = (size_t)K * p->n[0] * p->Pc[1] * p->H2c;
            if ((s = plan_alloc_t(p, &p->cA, a_el))) break;
            if ((s = plan_alloc_t(p, &p->cB, b_el))) break;
            if ((s = plan_alloc_t(p, &p->cC, c_el))) break;
            if ((s = plan_alloc_t(p, &p->tail_err, 1))) break;
            if (cudaMemset(p->tail_err, 0, sizeof(int)) != cudaSuccess) {
                s = cuda_fail(cudaGetLastError(), "tail flag");
                break;
            }
            if (cert_tail_supported(p->Pc[1], p->Pc[2], p->n[1], p->n[2])) {
                // line groups of 4 per slab, fetched in nbox box copies of boxg groups
                const long long ng = (long long)p->Pc[1] * p->H2c / 4;
                const int nbox = (int)((ng + 255) / 256);
                const int boxg = (int)(((ng + nbox - 1) / nbox + 3) / 4 * 4);
                p->tail_boxg = boxg;
                p->tail_nbox = nbox;
                p->tail_tma = make_tail_tmap(p->cC, p->n[0], ng, K, boxg, p->tail_tmap);
            }
        }
        // H^ on the blur grid, scaled by 1/|P| (folds the inverse normalisation)
        if ((s = launch_wrap_psf(p->psf, p->R, g.P, p->fE, st))) break;
        if ((s = fft3_forward(g.P, g.fac, g.tw, p->fE, p->bufA, p->Hspec, 1.0f / (float)Ptot, st))) break;
        if (p->fft_cert && (s = build_table(p, st))) break;
        if (p->direct_ok && (s = build_direct(p, st))) break;
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) s = cuda_fail(e, "plan create");
    } while (0);
    if (s != SFW_OK) {
        cudaDeviceSynchronize();
        plan_free(p);
        delete p;
        return s;
    }
    *out = p;
    return SFW_OK;
}

sfw_status sfw_plan_destroy(sfw_plan* plan) {
    clear_error();
    if (!plan) return SFW_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    delete plan;
    return SFW_OK;
}

sfw_status sfw_plan_query(const sfw_plan* p, sfw_plan_info* info) {
    clear_error();
    if (!p || !info) return fail(SFW_ERR_ARG, "plan and info must be non-NULL");
    for (int a = 0; a < 3; ++a) {
        info->E[a] = p->E[a];
        info->P_conv[a] = p->blur.P[a];
        info->P_cert[a] = p->fft_cert ? p->Pc[a] : 0;
    }
    info->route_blur = p->route_blur;
    info->tensor_cores = p->tc ? 1 : 0;
    info->route_cert = p->K ? p->route_cert : 0;
    info->K = p->K;
    info->real_table = p->real_table;
    info->table_bytes = p->table_bytes;
    info->workspace_bytes = p->ws_bytes - p->table_bytes;
    return SFW_OK;
}

sfw_status sfw_forward(sfw_plan* p, const sfw_atoms* atoms, float* y_out, void* stream) {
    clear_error();
    if (!p || !y_out) return fail(SFW_ERR_ARG, "plan and y_out must be non-NULL");
    SFW_TRY(check_atoms(atoms, false));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AtomsDev a = to_dev(atoms);
    SFW_TRY(launch_render(a, p->E, p->R, p->eps, p->fE, st));
    return plan_blur_store(p, p->fE, y_out, st);
}

// Rendering, blur, residual r = y - Phi mu and the criterion C (Eq. 4), on st.
static sfw_status residual_and_loss(sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                                    double* loss_out, float* r, cudaStream_t st) {
    AtomsDev a = to_dev(atoms);
    SFW_TRY(launch_render(a, p->E, p->R, p->eps, p->fE, st));
    if (p->route_blur == SFW_ROUTE_DIRECT) {
        if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the FFT route only");
        DirectBlur b;
        memset(&b, 0, sizeof(b));
        b.fE = p->fE;
        b.H = p->psf;
        for (int q = 0; q < 3; ++q) {
            b.n[q] = p->n[q];
            b.R[q] = p->R[q];
        }
        b.out = r;
        b.y = y;
        b.partials = p->dir_parts;
        b.partials_len = p->dir_parts_len;
        b.counter = p->ctr + 0;
        b.loss_out = loss_out;
        b.w = atoms->w;
        b.nw = atoms->N;
        b.lambda = lambda;
        b.num_sms = p->num_sms;
        return launch_direct_blur(b, st);
    }
    C2RPass ep;
    memset(&ep, 0, sizeof(ep));
    ep.mode = C2R_RESIDUAL;
    ep.scale = 1.f;
    ep.out = r;
    ep.y = y;
    ep.partials = p->loss_parts;
    ep.loss_out = loss_out;
    ep.counter = p->ctr + 0;
    ep.w = atoms->w;
    ep.nw = atoms->N;
    ep.w_stride = 1;
    ep.lambda = lambda;
    int blocks = 0;
    SFW_TRY(blur_forward(p->blur, p->fE, p->Hspec, SPEC_C64, p->bufA, p->bufB, ep, st, &blocks));
    if (blocks > p->loss_parts_len) return fail(SFW_ERR_SHAPE, "loss partial buffer too small");
    return SFW_OK;
}

// Back-projection b = Phi^T r and the analytic gradient of C (Eq. 4), on st.
static sfw_status loss_gradient(sfw_plan* p, const sfw_atoms* atoms, double lambda, const float* r,
                                double* grad_out, cudaStream_t st) {
    AtomsDev a = to_dev(atoms);
    SFW_TRY(plan_transpose(p, r, p->bE, st));
    return launch_atom_grad(a, p->E, p->R, p->eps, p->bE, lambda, p->grad_parts, grad_out,
                            p->adj_ctr, st);
}

static sfw_status slide_args(const sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                             const double* loss_out) {
    if (!p || !y || !loss_out) return fail(SFW_ERR_ARG, "plan, y, loss_out must be non-NULL");
    SFW_TRY(check_atoms(atoms, true));
    if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(SFW_ERR_ARG, "lambda must be finite and >= 0");
    if (atoms->N > p->grad_parts_atoms) return fail(SFW_ERR_ARG, "too many atoms");
    return SFW_OK;
}

sfw_status sfw_slide_loss_grad(sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                               double* loss_out, double* grad_out, float* residual_out,
                               void* stream) {
    clear_error();
    SFW_TRY(slide_args(p, y, atoms, lambda, loss_out));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* r = residual_out ? residual_out : p->r;
    SFW_TRY(residual_and_loss(p, y, atoms, lambda, loss_out, r, st));
    if (!grad_out) return SFW_OK;  // loss only
    return loss_gradient(p, atoms, lambda, r, grad_out, st);
}

static sfw_status certificate_impl(sfw_plan* p, const float* residual, double lambda, float* eta_out,
                                   float* max_out, int32_t* argk_out, float* best_val,
                                   int64_t* best_idx, cudaStream_t st);

static sfw_status certificate_args(const sfw_plan* p, const float* residual, double lambda) {
    if (!p || !residual) return fail(SFW_ERR_ARG, "plan and residual must be non-NULL");
    if (p->K == 0) return fail(SFW_ERR_ARG, "plan has no certificate grid");
    if (!(lambda > 0.0) || !isfinite(lambda)) return fail(SFW_ERR_ARG, "lambda must be finite and > 0");
    return SFW_OK;
}

static sfw_status step_body(sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                            double* loss_out, double* grad_out, float* r, float* best_val,
                            int64_t* best_idx, cudaStream_t st, cudaStream_t aux) {
    SFW_TRY(residual_and_loss(p, y, atoms, lambda, loss_out, r, st));
    if (aux != st) {
        SFW_CUDA(cudaEventRecord(p->ev_fork, st));
        SFW_CUDA(cudaStreamWaitEvent(aux, p->ev_fork, 0));
    }
    SFW_TRY(certificate_impl(p, r, lambda, nullptr, nullptr, nullptr, best_val, best_idx, aux));
    if (grad_out) SFW_TRY(loss_gradient(p, atoms, lambda, r, grad_out, st));
    if (aux != st) {
        SFW_CUDA(cudaEventRecord(p->ev_join, aux));
        SFW_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0));
    }
    return SFW_OK;
}

sfw_status sfw_step(sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                    double* loss_out, double* grad_out, float* residual_out, float* best_val,
                    int64_t* best_idx, void* stream, void* aux_stream) {
    clear_error();
    SFW_TRY(slide_args(p, y, atoms, lambda, loss_out));
    if (!p->K) return fail(SFW_ERR_ARG, "plan has no certificate grid");
    if (!(lambda > 0.0)) return fail(SFW_ERR_ARG, "lambda must be > 0 for the certificate");
    if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the single calls");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t aux = aux_stream ? static_cast<cudaStream_t>(aux_stream) : st;
    float* r = residual_out ? residual_out : p->r;

    sfw_plan::StepKey key;
    const void* ptrs[10] = {y, atoms->m, atoms->sigma, atoms->d, atoms->w, loss_out, grad_out, r,
                            best_val, best_idx};
    for (int i = 0; i < 10; ++i) key.ptr[i] = ptrs[i];
    key.N = atoms->N;
    key.lambda = lambda;
    // under a caller's capture or the profiler's events: launch directly and leave the
    // cached graph alone
    bool graphable = !prof_active();
    if (graphable) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            cudaGetLastError();
            graphable = false;
        } else {
            graphable = cs == cudaStreamCaptureStatusNone;
        }
    }
    if (!graphable) return step_body(p, y, atoms, lambda, loss_out, grad_out, r, best_val, best_idx, st, aux);
    const bool same = p->step_seen && key == p->step_key;
    if (same && p->step_exec) {
        SFW_CUDA(cudaGraphLaunch(p->step_exec, st));
        SFW_CUDA(cudaEventRecord(p->ev_graph, st));
        return SFW_OK;
    }
    if (same) {
        // second identical call in a row: capture the step on the plan's streams (capturing
        // runs nothing), then launch the graph on the caller's stream
        SFW_CUDA(cudaStreamBeginCapture(p->cap_own, cudaStreamCaptureModeThreadLocal));
        const sfw_status sb = step_body(p, y, atoms, lambda, loss_out, grad_out, r, best_val, best_idx,
                                        p->cap_own, p->aux_own);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(p->cap_own, &g);
        cudaGraphExec_t ex = nullptr;
        cudaError_t ei = cudaErrorUnknown;
        if (sb == SFW_OK && ec == cudaSuccess && g) ei = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        if (sb != SFW_OK) return sb;
        if (ec != cudaSuccess) return cuda_fail(ec, "sfw_step capture");
        if (ei != cudaSuccess) return cuda_fail(ei, "sfw_step graph instantiate");
        p->step_exec = ex;
        SFW_CUDA(cudaGraphLaunch(p->step_exec, st));
        SFW_CUDA(cudaEventRecord(p->ev_graph, st));
        return SFW_OK;
    }
    if (p->step_exec) {
        // the arguments changed: the cached graph is dropped once its last launch is done
        // (an event after each launch: no device-wide synchronisation)
        SFW_CUDA(cudaEventSynchronize(p->ev_graph));
        cudaGraphExecDestroy(p->step_exec);
        p->step_exec = nullptr;
    }
    p->step_key = key;
    p->step_seen = true;
    return step_body(p, y, atoms, lambda, loss_out, grad_out, r, best_val, best_idx, st, aux);
}

sfw_status sfw_certificate_grid(sfw_plan* p, const float* residual, double lambda, float* eta_out,
                                float* max_out, int32_t* argk_out, float* best_val,
                                int64_t* best_idx, void* stream) {
    clear_error();
    SFW_TRY(certificate_args(p, residual, lambda));
    return certificate_impl(p, residual, lambda, eta_out, max_out, argk_out, best_val, best_idx,
                            static_cast<cudaStream_t>(stream));
}

static sfw_status certificate_impl(sfw_plan* p, const float* residual, double lambda, float* eta_out,
                                   float* max_out, int32_t* argk_out, float* best_val,
                                   int64_t* best_idx, cudaStream_t st) {
    if (p->route_cert == SFW_ROUTE_DIRECT) {
        // b = Phi^T r on E, then eta_k(m) = (1/lambda) sum_t g_k(t - m) b(t) by direct sums
        if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the FFT route only");
        SFW_TRY(launch_direct_transpose(residual, p->psf, p->n, p->R, p->bE_cert, p->num_sms, st));
        DirectCert c;
        memset(&c, 0, sizeof(c));
        c.bE = p->bE_cert;
        c.gtab = p->gtab;
        c.kern = p->gkern;
        c.K = p->K;
        for (int a = 0; a < 3; ++a) {
            c.n[a] = p->n[a];
            c.R[a] = p->R[a];
        }
        c.scale = (float)(1.0 / lambda);
        c.eta_out = eta_out;
        c.max_out = max_out;
        c.argk_out = argk_out;
        c.best_key = (best_val || best_idx) ? p->best_key : nullptr;
        c.counter = p->ctr + 1;
        c.best_val = best_val;
        c.best_idx = best_idx;
        c.num_sms = p->num_sms;
        return launch_direct_cert(c, st);
    }
    const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
    const int P0 = p->Pc[0], P1 = p->Pc[1], P2 = p->Pc[2], H2 = p->H2c;
    const int K = p->K;
    const bool slabs = cert_tail_supported(P1, P2, n1, n2) && !g_recorder;
    if (slabs) {
        // axis-2 real forward and axis-1 forward in one pass per i0 slab -> cB
        CertHeadPass h;
        memset(&h, 0, sizeof(h));
        h.r = residual;
        h.out = p->cB;
        h.n0 = n0;
        h.n1 = n1;
        h.n2 = n2;
        h.P1 = P1;
        h.P2 = P2;
        h.H2 = H2;
        LaunchTag lt__(kCertHeadTag);
        SFW_TRY(launch_cert_head(h, st));
    } else {
        {   // axis 2 forward of r: (n0, n1, n2) -> (n0, n1, H2)
            R2CPass q;
            q.in = residual;
            q.lin = ls((long long)n1 * n2, n2, 1, n1);
            q.nlines = (long long)n0 * n1;
            q.in_off = 0;
            q.in_len = n2;
            q.L = P2;
            q.fac = p->facc[2];
            q.tw = p->twc[2];
            q.out = p->cA;
            q.lout = ls((long long)n1 * H2, H2, 1, n1);
            {
                LaunchTag lt__(kCertTags.r2c);
                SFW_TRY(launch_r2c(q, st));
            }
        }
        {   // axis 1 forward: -> (n0, P1, H2)
            C2CPass q;
            q.in = p->cA;
            q.out = p->cB;
            q.lin = ls((long long)n1 * H2, 1, H2, H2);
            q.lout = ls((long long)P1 * H2, 1, H2, H2);
            q.nlines = (long long)n0 * H2;
            q.L = P1;
            q.in_off = 0;
            q.in_len = n1;
            q.out_off = 0;
            q.out_len = P1;
            q.dir = -1;
            q.scale = 1.f;
            q.fac = p->facc[1];
            q.tw = p->twc[1];
            {
                LaunchTag lt__(kCertTags.fwd1);
                SFW_TRY(launch_c2c(q, st));
            }
        }
    }
    if (p->tc && !g_recorder) {
        // axis 0 on the tensor cores: forward transform of the (n0, P1, H2) lines into X
        // (P0, P1 H2), then U_k = W diag(X) T_k for all kernels as one bf16 GEMM per line
        const long long nl = (long long)P1 * H2;
        C2CPass f;
        f.in = p->cB;
        f.out = p->cX;
        f.lin = ls(0, 1, nl, nl);
        f.lout = ls(0, 1, nl, nl);
        f.nlines = nl;
        f.L = P0;
        f.in_off = 0;
        f.in_len = n0;
        f.out_off = 0;
        f.out_len = P0;
        f.dir = -1;
        f.scale = 1.f;
        f.fac = p->facc[0];
        f.tw = p->twc[0];
        {
            LaunchTag lt__(kCertX0Tag);
            SFW_TRY(launch_c2c(f, st));
        }
        Axis0TcPass a;
        memset(&a, 0, sizeof(a));
        a.X = p->cX;
        a.A = p->tc_dft;
        a.Tb = p->tc_table;
        a.out = p->cC;
        a.lout = (slabs && p->tail_tma) ? ls(4LL * n0, 1, 4, 4) : ls(0, 1, nl, nl);
        a.out_stride = (long long)n0 * nl;
        a.nl = nl;
        a.P0 = P0;
        a.Kp = p->tc_Kp;
        a.n0 = n0;
        a.K = K;
        a.Np = p->tc_Np;
        a.err = p->tail_err;
        LaunchTag lt__(kCertTcTag);
        SFW_TRY(launch_axis0_tc(a, p->num_sms, st));
    } else {   // axis 0: forward once, then for each kernel k: times table_k, inverse -> (K, n0, P1, H2)
        MulPass q;
        const long long nl = (long long)P1 * H2;
        q.in = p->cB;
        q.lin = ls(0, 1, nl, nl);
        q.in_off = 0;
        q.in_len = n0;
        q.nlines = nl;
        q.L = P0;
        q.fac = p->facc[0];
        q.tw = p->twc[0];
        q.spec = p->table;
        q.lspec = p->table_lines;
        q.spec_stride = p->table_stride;
        q.ktotal = K;
        {   // split the kernels so that the launch holds about 8 CTAs per SM
            const long long tiles = (nl + 15) / 16;
            long long groups = (8LL * p->num_sms + tiles - 1) / tiles;
            if (groups < 1) groups = 1;
            if (groups > K) groups = K;
            q.nspec = (int)((K + groups - 1) / groups);
        }
        q.spec_kind = p->table_kind;
        q.conj_spec = 0;
        q.out = p->cC;
        // the TMA tail reads it line-group-major, [k][l / 4][i0][l mod 4]: a warp's 4 lines
        // and all its rows form one contiguous block
        q.lout = (slabs && p->tail_tma) ? ls(4LL * n0, 1, 4, 4) : ls(0, 1, nl, nl);
        q.out_stride = (long long)n0 * nl;
        q.out_off = 0;
        q.out_len = n0;
        {
            LaunchTag lt__(kCertTags.axis0);
            SFW_TRY(launch_mul(q, st));
        }
    }
    const bool want_vox = max_out || argk_out;
    if (want_vox) {
        if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the argmax-only certificate");
        cudaError_t e = cudaMemsetAsync(p->vox_key, 0, sizeof(unsigned long long) * (size_t)p->V, st);
        if (e != cudaSuccess) return cuda_fail(e, "memset");
    }
    if (slabs) {
        // axis-1 inverse, real axis-2 inverse and the max over k in one pass per i0 slab
        CertTailPass t;
        memset(&t, 0, sizeof(t));
        t.in = p->cC;
        t.n0 = n0;
        t.n1 = n1;
        t.n2 = n2;
        t.P1 = P1;
        t.P2 = P2;
        t.H2 = H2;
        t.ktotal = K;
        t.scale = (float)(1.0 / lambda);
        t.eta_out = eta_out;
        t.V = p->V;
        t.vox_key = want_vox ? p->vox_key : nullptr;
        t.best_key = (best_val || best_idx) ? p->best_key : nullptr;
        t.best_val = best_val;
        t.best_idx = best_idx;
        t.counter = p->ctr + 1;
        t.boxg = p->tail_boxg;
        t.nbox = p->tail_nbox;
        t.err = p->tail_err;
        LaunchTag lt__(kCertTailTag);
        SFW_TRY(launch_cert_tail(t, p->tail_tma ? p->tail_tmap : nullptr, 0, st));
    } else {
        // the axis-2 stage on the tensor cores reads the spectra with the line pitch H2p
        const bool tc_tail = p->tc && p->tc_c2r_C && p->c2r_tma && !g_recorder;
        {   // axis 1 inverse over all kernels: (K n0, P1, H2) -> (K n0, n1, H2)
            C2CPass q;
            q.in = p->cC;
            q.out = p->cA;
            q.lin = ls((long long)P1 * H2, 1, H2, H2);
            q.lout = tc_tail ? ls((long long)n1 * p->H2p, 1, p->H2p, H2) : ls((long long)n1 * H2, 1, H2, H2);
            q.nlines = (long long)K * n0 * H2;
            q.L = P1;
            q.in_off = 0;
            q.in_len = P1;
            q.out_off = 0;
            q.out_len = n1;
            q.dir = 1;
            q.scale = 1.f;
            q.fac = p->facc[1];
            q.tw = p->twc[1];
            {
                LaunchTag lt__(kCertTags.inv1);
                SFW_TRY(launch_c2c(q, st));
            }
        }
        if (tc_tail) {
            // real inverse along axis 2 and the max over k on the tensor cores
            C2rTcPass c;
            memset(&c, 0, sizeof(c));
            c.C = p->tc_c2r_C;
            c.nlines = n0 * n1;
            c.P2 = P2;
            c.H2 = H2;
            c.n2 = n2;
            c.K = K;
            c.scale = (float)(1.0 / lambda);
            c.eta_out = eta_out;
            c.V = p->V;
            c.vox_key = want_vox ? p->vox_key : nullptr;
            c.best_key = (best_val || best_idx) ? p->best_key : nullptr;
            c.counter = p->ctr + 1;
            c.best_val = best_val;
            c.best_idx = best_idx;
            c.err = p->tail_err;
            {
                LaunchTag lt__(kCertC2rTcTag);
                SFW_TRY(launch_c2r_tc(c, p->c2r_tmap, p->num_sms, st));
            }
            if (want_vox) SFW_TRY(launch_vox_decode(p->vox_key, p->V, max_out, argk_out, st));
            return SFW_OK;
        }
        C2RPass q;
        memset(&q, 0, sizeof(q));
        q.in = p->cA;
        q.lin = ls((long long)n1 * H2, H2, 1, n1);
        q.nlines = (long long)n0 * n1;
        q.in_spec_stride = (long long)n0 * n1 * H2;
        q.ktotal = K;
        q.L = P2;
        q.fac = p->facc[2];
        q.tw = p->twc[2];
        q.out_off = 0;
        q.out_len = n2;
        q.lout = ls((long long)n1 * n2, n2, 1, n1);
        q.scale = (float)(1.0 / lambda);
        q.mode = C2R_CERTMAX;
        q.eta_out = eta_out;
        q.V = p->V;
        q.vox_key = want_vox ? p->vox_key : nullptr;
        q.best_key = (best_val || best_idx) ? p->best_key : nullptr;
        q.best_val = best_val;
        q.best_idx = best_idx;
        q.counter = p->ctr + 1;
        // split the kernels into groups so that the launch fills the GPU (about 3 CTAs per SM)
        q.nspec = K;
        {
            const int tiles = c2r_blocks(q);
            int groups = (8 * p->num_sms + tiles - 1) / tiles;
            if (groups < 1) groups = 1;
            if (groups > K) groups = K;
            q.nspec = (K + groups - 1) / groups;
        }
        {
            LaunchTag lt__(kCertTags.c2r);
            SFW_TRY(launch_c2r(q, st, nullptr));
        }
    }
    if (want_vox) SFW_TRY(launch_vox_decode(p->vox_key, p->V, max_out, argk_out, st));
    return SFW_OK;
}

sfw_status sfw_gram(sfw_plan* p, const sfw_atoms* atoms, const float* y, double* G_out,
                    double* c_out, void* stream) {
    clear_error();
    if (!p || !y || !G_out || !c_out) return fail(SFW_ERR_ARG, "plan, y, G_out, c_out must be non-NULL");
    SFW_TRY(check_atoms(atoms, true));
    if (atoms->N > 256) return fail(SFW_ERR_ARG, "sfw_gram takes at most 256 atoms");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = atoms->N;
    if (p->gram_cap < N) {
        // the only allocation of the hot path's API: the N blurred atoms, kept for reuse
        SFW_CUDA(cudaStreamSynchronize(st));
        if (p->gram_cols) cudaFree(p->gram_cols);
        p->gram_cols = nullptr;
        p->gram_cap = 0;
        const int cap = N < 16 ? 16 : N;
        cudaError_t e = cudaMalloc(&p->gram_cols, sizeof(float) * (size_t)cap * (size_t)p->V);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SFW_ERR_ALLOC, "sfw_gram: %d blurred atoms do not fit", cap);
        }
        p->gram_cap = cap;
    }
    AtomsDev a = to_dev(atoms);
    AtomsDev unit;
    unit.N = 1;
    unit.m = p->unit_slot;
    unit.sigma = p->unit_slot + 3;
    unit.d = p->unit_slot + 4;
    unit.w = p->unit_slot + 5;
    for (int i = 0; i < N; ++i) {
        SFW_TRY(launch_unit_atom(a, i, p->unit_slot, st));
        SFW_TRY(launch_render(unit, p->E, p->R, p->eps, p->fE, st));
        SFW_TRY(plan_blur_store(p, p->fE, p->gram_cols + (size_t)i * (size_t)p->V, st));
    }
    return launch_gram(p->gram_cols, y, N, p->V, G_out, c_out, st);
}

static sfw_status topk_rescore(sfw_plan* p, double lambda, int topk, float* cand_theta, float* cand_grid,
                               double* cand_eta, float* best_theta, double* best_eta, cudaStream_t st);

static sfw_status topk_args(const sfw_plan* p, const float* residual, double lambda, int topk) {
    if (!p || !residual) return fail(SFW_ERR_ARG, "plan and residual must be non-NULL");
    if (p->K == 0) return fail(SFW_ERR_ARG, "plan has no certificate grid");
    if (topk < 1 || topk > 64 || topk > p->V) return fail(SFW_ERR_ARG, "topk must be in [1, min(64, V)]");
    if (!(lambda > 0.0) || !isfinite(lambda)) return fail(SFW_ERR_ARG, "lambda must be finite and > 0");
    return SFW_OK;
}

// Steps 1-3 of the top-k seed without the re-score: the grid certificate's per-voxel maximum
// over k and its k, the topk voxels by that maximum, their parameter rows.
static sfw_status topk_select(sfw_plan* p, const float* residual, double lambda, int topk, cudaStream_t st) {
    SFW_TRY(certificate_impl(p, residual, lambda, nullptr, p->vmax, p->vargk, nullptr, nullptr, st));
    SFW_TRY(launch_topk(p->vmax, p->V, topk, p->red_scratch, p->red_scratch_len, p->cand_val,
                        p->cand_idx, st));
    return launch_candidate_theta(p->cand_idx, p->vargk, p->grid_sd, topk, p->n, p->cand_theta, st);
}

sfw_status sfw_certificate_topk(sfw_plan* p, const float* residual, double lambda, int topk,
                                float* cand_theta, float* cand_grid, double* cand_eta,
                                float* best_theta, double* best_eta, void* stream) {
    clear_error();
    SFW_TRY(topk_args(p, residual, lambda, topk));
    if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the argmax-only certificate");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // 1.-3. grid certificate -> per-voxel max over k, the topk voxels, their parameter rows
    SFW_TRY(topk_select(p, residual, lambda, topk, st));
    // 4. their FP32 re-score against b = Phi^T r, and the best
    SFW_TRY(plan_transpose(p, residual, p->bE, st));
    return topk_rescore(p, lambda, topk, cand_theta, cand_grid, cand_eta, best_theta, best_eta, st);
}

sfw_status sfw_step_topk(sfw_plan* p, const float* y, const sfw_atoms* atoms, double lambda,
                         double* loss_out, double* grad_out, float* residual_out, int topk,
                         float* cand_theta, float* cand_grid, double* cand_eta, float* best_theta,
                         double* best_eta, void* stream, void* aux_stream) {
    clear_error();
    SFW_TRY(slide_args(p, y, atoms, lambda, loss_out));
    if (!grad_out) return fail(SFW_ERR_ARG, "grad_out must be non-NULL");
    if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "batches record the single calls");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t aux = aux_stream ? static_cast<cudaStream_t>(aux_stream) : st;
    float* r = residual_out ? residual_out : p->r;
    SFW_TRY(topk_args(p, r, lambda, topk));
    SFW_TRY(residual_and_loss(p, y, atoms, lambda, loss_out, r, st));
    if (aux != st) {
        SFW_CUDA(cudaEventRecord(p->ev_fork, st));
        SFW_CUDA(cudaStreamWaitEvent(aux, p->ev_fork, 0));
    }
    // the certificate and the selection on aux; b = Phi^T r and the adjoint sums on st
    SFW_TRY(topk_select(p, r, lambda, topk, aux));
    SFW_TRY(loss_gradient(p, atoms, lambda, r, grad_out, st));
    if (aux != st) {
        SFW_CUDA(cudaEventRecord(p->ev_grad, st));
        SFW_CUDA(cudaStreamWaitEvent(aux, p->ev_grad, 0));
    }
    // the re-score reads b and the adjoint sums' scratch: after both branches
    SFW_TRY(topk_rescore(p, lambda, topk, cand_theta, cand_grid, cand_eta, best_theta, best_eta, aux));
    if (aux != st) {
        SFW_CUDA(cudaEventRecord(p->ev_join, aux));
        SFW_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0));
    }
    return SFW_OK;
}

// The FP32 re-score of the topk candidate rows against b = Phi^T r (already in p->bE) and the
// best of them.
static sfw_status topk_rescore(sfw_plan* p, double lambda, int topk, float* cand_theta, float* cand_grid,
                               double* cand_eta, float* best_theta, double* best_eta, cudaStream_t st) {
    AtomsDev pts;
    pts.N = topk;
    pts.m = p->cand_theta;
    pts.sigma = p->cand_theta + 3;
    pts.d = p->cand_theta + 4;
    pts.w = p->cand_theta + 3;
    pts.ms = 5;
    pts.ps = 5;
    SFW_TRY(launch_eta_points(pts, p->E, p->R, p->eps, p->bE, lambda, p->grad_parts, p->cand_eta,
                              nullptr, p->adj_ctr, st));
    // 4. the best re-scored candidate and the requested copies
    return launch_candidate_select(p->cand_theta, p->cand_val, p->cand_eta, topk, cand_theta,
                                   cand_grid, cand_eta, best_theta, best_eta, st);
}

sfw_status sfw_eta_points(sfw_plan* p, const float* residual, double lambda, int P,
                          const float* theta, double* eta_out, double* grad_out, void* stream) {
    clear_error();
    if (!p || !residual || !theta || !eta_out) return fail(SFW_ERR_ARG, "plan, residual, theta, eta_out must be non-NULL");
    if (P < 1 || P > p->grad_parts_atoms) return fail(SFW_ERR_ARG, "P must be in [1, %d]", p->grad_parts_atoms);
    if (!(lambda > 0.0) || !isfinite(lambda)) return fail(SFW_ERR_ARG, "lambda must be finite and > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SFW_TRY(plan_transpose(p, residual, p->bE, st));
    AtomsDev pts;
    pts.N = P;
    pts.m = theta;
    pts.sigma = theta + 3;
    pts.d = theta + 4;
    pts.w = theta + 3;  // unused by the sums
    pts.ms = 5;
    pts.ps = 5;
    return launch_eta_points(pts, p->E, p->R, p->eps, p->bE, lambda, p->grad_parts, eta_out,
                             grad_out, p->adj_ctr, st);
}

sfw_status sfw_plan_check(sfw_plan* p) {
    clear_error();
    if (!p) return fail(SFW_ERR_ARG, "plan is NULL");
    if (!p->tail_err) return SFW_OK;
    int flag = 0;
    SFW_CUDA(cudaDeviceSynchronize());
    SFW_CUDA(cudaMemcpy(&flag, p->tail_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!flag) return SFW_OK;
    SFW_CUDA(cudaMemset(p->tail_err, 0, sizeof(int)));
    return fail(SFW_ERR_TIMEOUT, "a certificate kernel gave up a bounded wait (slab copies or tensor-core MMAs)");
}

sfw_status sfw_autotune(sfw_plan* p, const char* cache_path, void* stream) {
    clear_error();
    if (!p) return fail(SFW_ERR_ARG, "plan is NULL");
    const bool tune_routes = p->route == SFW_ROUTE_AUTO;
    const bool tune_tc = p->tc_ready;
    if (!tune_routes && !tune_tc) return SFW_OK;
    if (g_recorder) return fail(SFW_ERR_UNSUPPORTED, "not while a batch records");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        SFW_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone) return fail(SFW_ERR_ARG, "sfw_autotune cannot be captured");
    }
    if (p->step_exec) {
        // sfw_step's cached graph holds the launches of the routes in use: drop it
        SFW_CUDA(cudaEventSynchronize(p->ev_graph));
        cudaGraphExecDestroy(p->step_exec);
        p->step_exec = nullptr;
    }
    p->step_seen = false;
    // cache key: shape, PSF support, certificate grid, precision, requested route
    std::string key;
    {
        char buf[112];
        snprintf(buf, sizeof(buf), "n=%d,%d,%d R=%d,%d,%d prec=%d route=%d K=%d", p->n[0], p->n[1], p->n[2],
                 p->R[0], p->R[1], p->R[2], p->precision, p->route, p->K);
        key = buf;
        for (int k = 0; k < p->K; ++k) {
            snprintf(buf, sizeof(buf), " %.7g/%.7g", p->sigmas[k], p->ds[k]);
            key += buf;
        }
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            char line[8192];
            while (fgets(line, sizeof(line), f)) {
                const size_t kl = key.size();
                int rb = 0, rc = 0, tcu = 0;
                if (strncmp(line, key.c_str(), kl) == 0 && line[kl] == '|' &&
                    sscanf(line + kl + 1, "%d %d %d", &rb, &rc, &tcu) == 3 &&
                    (rb == SFW_ROUTE_FFT || (rb == SFW_ROUTE_DIRECT && p->direct_ok)) &&
                    (rc == SFW_ROUTE_FFT ? p->fft_cert || p->K == 0 : rc == SFW_ROUTE_DIRECT && p->gtab) &&
                    (!tcu || p->tc_ready)) {
                    fclose(f);
                    p->route_blur = rb;
                    p->route_cert = rc;
                    p->tc = tcu != 0;
                    return SFW_OK;
                }
            }
            fclose(f);
        }
    }
    // a zero residual and a zero atom field on the plan's own buffers
    SFW_CUDA(cudaMemsetAsync(p->r, 0, sizeof(float) * (size_t)p->V, st));
    SFW_CUDA(cudaMemsetAsync(p->fE, 0, sizeof(float) * (size_t)p->VE, st));
    auto time_cert = [&]() {
        return time_route([&]() -> sfw_status {
            return certificate_impl(p, p->r, 1.0, nullptr, nullptr, nullptr, p->cand_val, p->cand_idx, st);
        }, st);
    };
    if (tune_routes) {
        float t_blur[3] = {-1.f, -1.f, -1.f};   // indexed by route
        for (int rt = SFW_ROUTE_FFT; rt <= SFW_ROUTE_DIRECT; ++rt) {
            if (rt == SFW_ROUTE_DIRECT && !p->direct_ok) continue;
            p->route_blur = rt;
            // the convolutions of one sliding-step evaluation: Phi on the grid, Phi^T on E
            t_blur[rt] = time_route([&]() -> sfw_status {
                SFW_TRY(plan_blur_store(p, p->fE, p->r, st));
                return plan_transpose(p, p->r, p->bE, st);
            }, st);
        }
        p->route_blur = (t_blur[SFW_ROUTE_DIRECT] >= 0.f && t_blur[SFW_ROUTE_DIRECT] < t_blur[SFW_ROUTE_FFT])
                            ? SFW_ROUTE_DIRECT : SFW_ROUTE_FFT;
        if (p->K > 0) {
            float t_cert[3] = {-1.f, -1.f, -1.f};
            for (int rt = SFW_ROUTE_FFT; rt <= SFW_ROUTE_DIRECT; ++rt) {
                if (rt == SFW_ROUTE_FFT && !p->fft_cert) continue;
                if (rt == SFW_ROUTE_DIRECT && !p->gtab) continue;
                p->route_cert = rt;
                t_cert[rt] = time_cert();
            }
            const bool direct = t_cert[SFW_ROUTE_DIRECT] >= 0.f &&
                                (t_cert[SFW_ROUTE_FFT] < 0.f || t_cert[SFW_ROUTE_DIRECT] < t_cert[SFW_ROUTE_FFT]);
            p->route_cert = direct ? SFW_ROUTE_DIRECT : SFW_ROUTE_FFT;
        }
    }
    if (tune_tc && p->route_cert == SFW_ROUTE_FFT) {
        // the certificate's axis-0 stage: tensor cores against the FP32-arithmetic transform
        p->tc = false;
        const float t_fft = time_cert();
        p->tc = true;
        const float t_tc = time_cert();
        p->tc = t_tc >= 0.f && (t_fft < 0.f || t_tc < t_fft);
    }
    SFW_CUDA(cudaStreamSynchronize(st));
    if (cache_path) {
        FILE* f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s|%d %d %d\n", key.c_str(), p->route_blur, p->route_cert, p->tc ? 1 : 0);
            fclose(f);
        }
    }
    return SFW_OK;
}

// Test hook (not part of the public header): raise the plan's timeout flag from the host,
// as a certificate-tail CTA whose bounded wait ran out would, so that the flag -> status
// path of sfw_plan_check is exercised without any device wait running out.
sfw_status sfw_test_raise_timeout_flag(sfw_plan* p) {
    clear_error();
    if (!p) return fail(SFW_ERR_ARG, "plan is NULL");
    if (!p->tail_err) return fail(SFW_ERR_UNSUPPORTED, "plan has no certificate tail flag");
    const int one = 1;
    SFW_CUDA(cudaMemcpy(p->tail_err, &one, sizeof(int), cudaMemcpyHostToDevice));
    return SFW_OK;
}

sfw_status sfw_argmax(const float* values, int64_t count, int topk, float* val_out,
                      int64_t* idx_out, void* stream) {
    clear_error();
    if (!values || !val_out || !idx_out) return fail(SFW_ERR_ARG, "pointers must be non-NULL");
    if (count < 1 || count >= 0xffffffffll) return fail(SFW_ERR_ARG, "count must be in [1, 2^32 - 2]");
    if (topk < 1 || topk > 64 || topk > count) return fail(SFW_ERR_ARG, "topk must be in [1, min(64, count)]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // scratch: a small per-device buffer owned by the library (grown on demand)
    static thread_local unsigned long long* scratch = nullptr;
    static thread_local long long scratch_len = 0;
    static thread_local int scratch_dev = -1;
    int dev = 0;
    SFW_CUDA(cudaGetDevice(&dev));
    const long long need = topk == 1 ? 1024 : topk_scratch_keys(count, topk);
    if (scratch_len < need || scratch_dev != dev) {
        if (scratch) {
            cudaStreamSynchronize(st);
            cudaFree(scratch);
        }
        scratch = nullptr;
        scratch_len = 0;
        cudaError_t e = cudaMalloc(&scratch, sizeof(unsigned long long) * (size_t)need);
        if (e != cudaSuccess) return cuda_fail(e, "argmax scratch");
        scratch_len = need;
        scratch_dev = dev;
    }
    if (topk == 1) {
        int nb = (int)((count + 255) / 256);
        if (nb > 1024) nb = 1024;
        SFW_TRY(launch_argmax_keys(values, count, scratch, nb, st));
        return launch_argmax_final(scratch, nb, val_out, idx_out, st);
    }
    return launch_topk(values, count, topk, scratch, scratch_len, val_out, idx_out, st);
}

}  // extern "C"

// ------------------------------------------------------------------ batches of volumes

namespace {

// One grouped launch of a batch step.
struct BatchLaunch {
    OpKind kind;
    RecOp proto;         // prototype pass (largest length of the group) for the FFT kinds
    GroupArgs g;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Key of the kernel variant an op launches (ops with equal keys share a launch).
std::string variant_key(const RecOp& o) {
    char b[128];
    int W, nbx, nby;
    switch (o.kind) {
        case OP_R2C:
            pass_tiles(o.r2c, &W, &nbx, &nby);
            snprintf(b, sizeof(b), "r2c/%d/%d", fft_specialised(o.r2c.L) ? o.r2c.L : 0, W);
            break;
        case OP_C2C:
            pass_tiles(o.c2c, &W, &nbx, &nby);
            snprintf(b, sizeof(b), "c2c/%d/%d/%d", fft_specialised(o.c2c.L) ? o.c2c.L : 0, W, o.c2c.dir);
            break;
        case OP_MUL:
            pass_tiles(o.mul, &W, &nbx, &nby);
            snprintf(b, sizeof(b), "mul/%d/%d/%d", fft_specialised(o.mul.L) ? o.mul.L : 0, W, o.mul.spec_kind);
            break;
        case OP_C2R: {
            pass_tiles(o.c2r, &W, &nbx, &nby);
            const int need = (2 * (W / 8) * o.c2r.out_len + 31) / 32;
            const int slots = o.c2r.mode != C2R_CERTMAX ? 1 : need <= 4 ? 4 : need <= 8 ? 8 : 16;
            snprintf(b, sizeof(b), "c2r/%d/%d/%d/%d", fft_specialised(o.c2r.L) ? o.c2r.L : 0, W, o.c2r.mode, slots);
            break;
        }
        case OP_SLAB:
            // compile-time lengths are part of the variant; runtime-length slabs group together
            snprintf(b, sizeof(b), "slab/%d/%d/%d", o.slab.mode, slab_specialised(o.slab) ? o.slab.P1 : 0,
                     slab_specialised(o.slab) ? o.slab.P2 : 0);
            break;
        default:
            snprintf(b, sizeof(b), "op/%d", (int)o.kind);
    }
    return b;
}

int op_length(const RecOp& o) {
    switch (o.kind) {
        case OP_R2C: return o.r2c.L;
        case OP_C2C: return o.c2c.L;
        case OP_MUL: return o.mul.L;
        case OP_C2R: return o.c2r.L;
        case OP_SLAB: return (int)slab_smem(o.slab);   // the group's prototype needs the most
        default: return 0;
    }
}

// Tiles of an op in a grouped launch: (x tiles, total tiles).
void op_tiles(const RecOp& o, int* nbx, int* total) {
    int W, nby;
    switch (o.kind) {
        case OP_R2C: pass_tiles(o.r2c, &W, nbx, &nby); *total = *nbx * nby; break;
        case OP_C2C: pass_tiles(o.c2c, &W, nbx, &nby); *total = *nbx * nby; break;
        case OP_MUL: pass_tiles(o.mul, &W, nbx, &nby); *total = *nbx * nby; break;
        case OP_C2R: pass_tiles(o.c2r, &W, nbx, &nby); *total = *nbx * nby; break;
        case OP_RENDER: *total = render_tiles(o.render, nbx); break;
        case OP_GRAD: *total = grad_tiles(o.grad, nbx); break;
        case OP_SLAB: *nbx = 1; *total = o.slab.nslab; break;
        default: *nbx = 1; *total = 1;
    }
}

template <class T>
const T& op_payload(const RecOp& o);
template <> const R2CPass& op_payload<R2CPass>(const RecOp& o) { return o.r2c; }
template <> const C2CPass& op_payload<C2CPass>(const RecOp& o) { return o.c2c; }
template <> const MulPass& op_payload<MulPass>(const RecOp& o) { return o.mul; }
template <> const C2RPass& op_payload<C2RPass>(const RecOp& o) { return o.c2r; }
template <> const RenderOp& op_payload<RenderOp>(const RecOp& o) { return o.render; }
template <> const GradOp& op_payload<GradOp>(const RecOp& o) { return o.grad; }
template <> const SlabPass& op_payload<SlabPass>(const RecOp& o) { return o.slab; }

template <class T>
void append_payloads(const std::vector<const RecOp*>& ops, std::vector<unsigned char>& blob) {
    for (const RecOp* o : ops) {
        const T& t = op_payload<T>(*o);
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&t);
        blob.insert(blob.end(), b, b + sizeof(T));
    }
}

}  // namespace

struct sfw_batch {
    int count;
    int num_sms;
    std::vector<sfw_plan*> plans;
    std::vector<BatchLaunch> launches;
    std::vector<int> branch;   // per launch: 0 before the fork, 1 certificate, 2 back-projection
    void* blob;           // device descriptors of every grouped launch
    cudaStream_t aux;     // the certificate branch of a step
    cudaEvent_t ev_fork, ev_join;
};

static void batch_free(sfw_batch* b) {
    if (b->blob) cudaFree(b->blob);
    b->blob = nullptr;
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->aux) cudaStreamDestroy(b->aux);
    b->ev_fork = b->ev_join = nullptr;
    b->aux = nullptr;
}

// One grouped launch of a batch step (also timed alone by the autotuner).
static sfw_status batch_launch(sfw_batch* b, BatchLaunch& L, cudaStream_t st) {
    GroupArgs& g = L.g;
    switch (L.kind) {
        case OP_R2C: {
            LaunchTag t("batch_r2c");
            SFW_TRY(launch_r2c(L.proto.r2c, st, &g));
            break;
        }
        case OP_C2C: {
            LaunchTag t("batch_c2c");
            SFW_TRY(launch_c2c(L.proto.c2c, st, &g));
            break;
        }
        case OP_MUL: {
            LaunchTag t(L.proto.mul.ktotal > 1 ? "batch_cert_axis0" : "batch_axis0");
            SFW_TRY(launch_mul(L.proto.mul, st, &g));
            break;
        }
        case OP_C2R: {
            LaunchTag t(L.proto.c2r.mode == C2R_CERTMAX ? "batch_cert_c2r_max" : "batch_c2r");
            SFW_TRY(launch_c2r(L.proto.c2r, st, nullptr, &g));
            break;
        }
        case OP_RENDER: {
            if (g.grid <= 0) g.grid = g.total < 8 * b->num_sms ? g.total : 8 * b->num_sms;
            LaunchTag t("batch_render");
            SFW_TRY(launch_render_group(static_cast<const RenderOp*>(g.passes), g.start, g.nbx, g.n, g.total, g.grid, st));
            break;
        }
        case OP_SLAB: {
            LaunchTag t(L.proto.slab.mode == SLAB_HEAD ? "batch_slab_head" : "batch_slab_tail");
            SFW_TRY(launch_slab(L.proto.slab, st, &g));
            break;
        }
        case OP_GRAD: {
            if (g.grid <= 0) g.grid = g.total < 8 * b->num_sms ? g.total : 8 * b->num_sms;
            LaunchTag t("batch_atom_grad");
            SFW_TRY(launch_grad_group(static_cast<const GradOp*>(g.passes), g.start, g.nbx, g.n, g.total, g.grid, st));
            break;
        }
        default:
            return fail(SFW_ERR_UNSUPPORTED, "unknown batch op");
    }
    return SFW_OK;
}

extern "C" {

sfw_status sfw_batch_create(int count, sfw_plan* const* plans, const sfw_batch_volume* vols,
                            const double* lambdas, sfw_batch** out) {
    clear_error();
    if (!out || !plans || !vols || !lambdas) return fail(SFW_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (count < 1 || count > 1024) return fail(SFW_ERR_ARG, "count must be in [1, 1024]");
    for (int v = 0; v < count; ++v) {
        const sfw_batch_volume& bv = vols[v];
        if (!plans[v]) return fail(SFW_ERR_ARG, "plan %d is NULL", v);
        if (plans[v]->K == 0) return fail(SFW_ERR_ARG, "plan %d has no certificate grid", v);
        if (plans[v]->route_blur != SFW_ROUTE_FFT || plans[v]->route_cert != SFW_ROUTE_FFT || !plans[v]->fft_cert)
            return fail(SFW_ERR_UNSUPPORTED, "plan %d: batches run the FFT route only", v);
        if (bv.N < 1 || bv.N > 4096) return fail(SFW_ERR_ARG, "volume %d: atoms outside [1, 4096]", v);
        if (!bv.y || !bv.m || !bv.sigma || !bv.d || !bv.w || !bv.residual || !bv.grad || !bv.loss ||
            !bv.best_val || !bv.best_idx)
            return fail(SFW_ERR_ARG, "volume %d: every buffer must be non-NULL", v);
        if (!(lambdas[v] > 0.0) || !isfinite(lambdas[v])) return fail(SFW_ERR_ARG, "volume %d: lambda must be > 0", v);
        for (int u = 0; u < v; ++u)
            if (plans[u] == plans[v]) return fail(SFW_ERR_ARG, "plans %d and %d are the same plan", u, v);
    }
    sfw_batch* b = new (std::nothrow) sfw_batch();
    if (!b) return fail(SFW_ERR_ALLOC, "host allocation");
    b->count = count;
    b->blob = nullptr;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        b->num_sms = 0;
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (b->num_sms <= 0) b->num_sms = 1;
    }
    sfw_status s = SFW_OK;
    std::vector<Recorder> rec(count);
    std::vector<size_t> n_fork(count), n_cert(count);
    do {
        if (cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            s = cuda_fail(cudaGetLastError(), "batch streams");
            break;
        }
        // record one step per volume through the single-volume code path, in the order
        // residual + loss | certificate | back-projection + gradient (the two last
        // branches run on two streams)
        g_slab_batch = true;
        for (int v = 0; v < count; ++v) g_slab_batch = g_slab_batch && blur_slabs_fit(plans[v]->blur);
        for (int v = 0; v < count && !s; ++v) {
            sfw_plan* p = plans[v];
            const sfw_batch_volume& bv = vols[v];
            b->plans.push_back(p);
            sfw_atoms at;
            at.N = bv.N;
            at.m = bv.m;
            at.sigma = bv.sigma;
            at.d = bv.d;
            at.w = bv.w;
            float* r = bv.residual ? bv.residual : p->r;
            s = slide_args(p, bv.y, &at, lambdas[v], bv.loss);
            if (!s) s = certificate_args(p, r, lambdas[v]);
            if (s) break;
            g_recorder = &rec[v];
            s = residual_and_loss(p, bv.y, &at, lambdas[v], bv.loss, r, nullptr);
            n_fork[v] = rec[v].ops.size();
            if (!s) s = certificate_impl(p, r, lambdas[v], nullptr, nullptr, nullptr, bv.best_val,
                                         bv.best_idx, nullptr);
            n_cert[v] = rec[v].ops.size();
            if (!s && bv.grad) s = loss_gradient(p, &at, lambdas[v], r, bv.grad, nullptr);
            g_recorder = nullptr;
        }
        if (s) break;
        const size_t nops = rec[0].ops.size();
        for (int v = 1; v < count && !s; ++v) {
            if (rec[v].ops.size() != nops || n_fork[v] != n_fork[0] || n_cert[v] != n_cert[0])
                s = fail(SFW_ERR_UNSUPPORTED, "volumes record different steps");
            for (size_t i = 0; i < nops && !s; ++i)
                if (rec[v].ops[i].kind != rec[0].ops[i].kind) s = fail(SFW_ERR_UNSUPPORTED, "volumes record different steps");
        }
        if (s) break;
        // group the ops of every stage by kernel variant; lay out their descriptors
        std::vector<unsigned char> blob;
        struct Pending {
            BatchLaunch L;
            size_t off_passes, off_start, off_nbx;
        };
        std::vector<Pending> pend;
        for (size_t i = 0; i < nops; ++i) {
            std::vector<std::string> keys;
            std::vector<std::vector<const RecOp*>> groups;
            for (int v = 0; v < count; ++v) {
                const RecOp* o = &rec[v].ops[i];
                std::string k = variant_key(*o);
                size_t gi = 0;
                while (gi < keys.size() && keys[gi] != k) ++gi;
                if (gi == keys.size()) {
                    keys.push_back(k);
                    groups.emplace_back();
                }
                groups[gi].push_back(o);
            }
            for (auto& grp : groups) {
                Pending P;
                memset(&P.L, 0, sizeof(P.L));
                P.L.kind = grp[0]->kind;
                const RecOp* proto = grp[0];
                for (const RecOp* o : grp)
                    if (op_length(*o) > op_length(*proto)) proto = o;
                P.L.proto = *proto;
                if (P.L.kind == OP_SLAB) {   // block size and shared memory of the largest slab
                    for (const RecOp* o : grp) {
                        const int w = slab_warps(o->slab), m = (int)slab_smem(o->slab);
                        if (w > P.L.proto.slab.warps) P.L.proto.slab.warps = w;
                        if (m > P.L.proto.slab.smem) P.L.proto.slab.smem = m;
                    }
                }
                P.L.g.n = (int)grp.size();
                std::vector<int> start(grp.size() + 1, 0), nbx(grp.size(), 1);
                for (size_t q = 0; q < grp.size(); ++q) {
                    int nx, tot;
                    op_tiles(*grp[q], &nx, &tot);
                    nbx[q] = nx;
                    start[q + 1] = start[q] + tot;
                }
                P.L.g.total = start.back();
                P.L.g.grid = 0;
                blob.resize(align16(blob.size()));
                P.off_passes = blob.size();
                switch (P.L.kind) {
                    case OP_R2C: append_payloads<R2CPass>(grp, blob); break;
                    case OP_C2C: append_payloads<C2CPass>(grp, blob); break;
                    case OP_MUL: append_payloads<MulPass>(grp, blob); break;
                    case OP_C2R: append_payloads<C2RPass>(grp, blob); break;
                    case OP_RENDER: append_payloads<RenderOp>(grp, blob); break;
                    case OP_GRAD: append_payloads<GradOp>(grp, blob); break;
                    case OP_SLAB: append_payloads<SlabPass>(grp, blob); break;
                    default: break;
                }
                blob.resize(align16(blob.size()));
                P.off_start = blob.size();
                blob.insert(blob.end(), reinterpret_cast<unsigned char*>(start.data()),
                            reinterpret_cast<unsigned char*>(start.data() + start.size()));
                blob.resize(align16(blob.size()));
                P.off_nbx = blob.size();
                blob.insert(blob.end(), reinterpret_cast<unsigned char*>(nbx.data()),
                            reinterpret_cast<unsigned char*>(nbx.data() + nbx.size()));
                pend.push_back(P);
                b->branch.push_back(i < n_fork[0] ? 0 : i < n_cert[0] ? 1 : 2);
            }
        }
        cudaError_t e = cudaMalloc(&b->blob, blob.size() ? blob.size() : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = fail(SFW_ERR_ALLOC, "batch descriptors");
            break;
        }
        e = cudaMemcpy(b->blob, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "batch descriptors");
            break;
        }
        unsigned char* base = static_cast<unsigned char*>(b->blob);
        for (auto& P : pend) {
            P.L.g.passes = base + P.off_passes;
            P.L.g.start = reinterpret_cast<const int*>(base + P.off_start);
            P.L.g.nbx = reinterpret_cast<const int*>(base + P.off_nbx);
            b->launches.push_back(P.L);
        }
    } while (0);
    g_recorder = nullptr;
    g_slab_batch = false;
    if (s) {
        batch_free(b);
        delete b;
        return s;
    }
    *out = b;
    return SFW_OK;
}

sfw_status sfw_batch_destroy(sfw_batch* b) {
    clear_error();
    if (!b) return SFW_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    delete b;
    return SFW_OK;
}

sfw_status sfw_batch_query(const sfw_batch* b, int* launches_per_step) {
    clear_error();
    if (!b || !launches_per_step) return fail(SFW_ERR_ARG, "NULL argument");
    *launches_per_step = (int)b->launches.size();
    return SFW_OK;
}

sfw_status sfw_batch_step(sfw_batch* b, void* stream) {
    clear_error();
    if (!b) return fail(SFW_ERR_ARG, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n = b->launches.size();
    for (size_t i = 0; i < n; ++i)
        if (b->branch[i] == 0) SFW_TRY(batch_launch(b, b->launches[i], st));
    // the certificates on the batch's stream while the back-projections continue
    SFW_CUDA(cudaEventRecord(b->ev_fork, st));
    SFW_CUDA(cudaStreamWaitEvent(b->aux, b->ev_fork, 0));
    for (size_t i = 0; i < n; ++i)
        if (b->branch[i] == 1) SFW_TRY(batch_launch(b, b->launches[i], b->aux));
    for (size_t i = 0; i < n; ++i)
        if (b->branch[i] == 2) SFW_TRY(batch_launch(b, b->launches[i], st));
    SFW_CUDA(cudaEventRecord(b->ev_join, b->aux));
    SFW_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
    return SFW_OK;
}

sfw_status sfw_batch_autotune(sfw_batch* b, const char* cache_path, void* stream) {
    clear_error();
    if (!b) return fail(SFW_ERR_ARG, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // signature of the launch list: kind, group size, total tiles of every launch
    std::string sig = "sfw-batch-v1";
    for (const BatchLaunch& L : b->launches) {
        char t[64];
        snprintf(t, sizeof(t), " %d.%d.%d", (int)L.kind, L.g.n, L.g.total);
        sig += t;
    }
    if (cache_path) {
        FILE* f = fopen(cache_path, "r");
        if (f) {
            std::string text;
            char buf[4096];
            size_t got;
            while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
            fclose(f);
            // {"signature": "<sig>", "grids": [g0, g1, ...]}
            const std::string want = "\"signature\": \"" + sig + "\"";
            const size_t at = text.find("\"grids\": [");
            if (text.find(want) != std::string::npos && at != std::string::npos) {
                std::vector<int> grids;
                const char* c = text.c_str() + at + 10;
                char* end = nullptr;
                while (true) {
                    while (*c == ' ' || *c == ',') ++c;
                    long v = strtol(c, &end, 10);
                    if (end == c) break;
                    grids.push_back((int)v);
                    c = end;
                }
                if (grids.size() == b->launches.size()) {
                    for (size_t i = 0; i < grids.size(); ++i) b->launches[i].g.grid = grids[i];
                    return SFW_OK;
                }
            }
        }
    }
    // a full step first: every launch then re-runs idempotently on live buffers
    SFW_TRY(sfw_batch_step(b, stream));
    SFW_CUDA(cudaStreamSynchronize(st));
    cudaEvent_t e0, e1;
    SFW_CUDA(cudaEventCreate(&e0));
    SFW_CUDA(cudaEventCreate(&e1));
    sfw_status s = SFW_OK;
    for (BatchLaunch& L : b->launches) {
        const bool tunable = L.kind == OP_R2C || L.kind == OP_C2C || L.kind == OP_MUL || L.kind == OP_C2R ||
                             L.kind == OP_RENDER || L.kind == OP_GRAD || L.kind == OP_SLAB;
        if (!tunable || L.g.total <= 1) continue;
        const int resident = L.g.grid;  // default chosen by the first step
        const int cand[6] = {resident, b->num_sms, 2 * b->num_sms, 4 * b->num_sms, 8 * b->num_sms, L.g.total};
        int best = resident;
        float best_ms = 1e30f;
        for (int c = 0; c < 6 && !s; ++c) {
            int gsz = cand[c] < L.g.total ? cand[c] : L.g.total;
            if (gsz < 1) continue;
            L.g.grid = gsz;
            if ((s = batch_launch(b, L, st))) break;  // warm
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && !s; ++r) s = batch_launch(b, L, st);
            cudaEventRecord(e1, st);
            if (s) break;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                s = cuda_fail(e, "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = gsz;
            }
        }
        L.g.grid = best;
        if (s) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    if (cache_path) {
        FILE* f = fopen(cache_path, "w");
        if (!f) return fail(SFW_ERR_ARG, "cannot write %s", cache_path);
        fprintf(f, "{\"signature\": \"%s\", \"grids\": [", sig.c_str());
        for (size_t i = 0; i < b->launches.size(); ++i) fprintf(f, "%s%d", i ? ", " : "", b->launches[i].g.grid);
        fprintf(f, "]}\n");
        fclose(f);
    }
    return SFW_OK;
}

}  // extern "C"
