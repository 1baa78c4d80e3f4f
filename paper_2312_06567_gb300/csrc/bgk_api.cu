// libbgk C-ABI: context, host-side operator construction, stage sequencing.
// See include/bgk.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <random>
#include <cstdio>
#include <cstring>
#include <string>
#include <limits>
#include <vector>

#include "../../include/bgk.h"
#include "bgk_internal.cuh"

struct bgk_ctx {
    // problem
    int p, q, Ns, Ne, Nu, C, P;
    int vn[3];
    int precision;
    MeshInfo mesh;
    FROps fr;
    GasInfo gas;
    VelGrid vg;                       // the velocities this context holds (a slab of the third axis if sharded)
    VelGrid vg_q;                     // the whole velocity grid: the Q' solve's sums run over it
    int Nu_q;                         // its size
    double *vtab_q;                   // its tables (the same arrays as vtab / vtab32 unless sharded)
    float4 *vtab32_q;
    bool shard;                       // holds third-axis velocity planes [slab_lo, slab_hi) of the grid
    int slab_lo, slab_hi;
    double jac;                       // |J_e|
    double lo[3];                     // mesh box corner
    double bc[6][5];
    std::vector<double> vtab_h;       // [Nu][BGK_VTAB]
    // curvilinear path (node coordinates given, or diffuse / closed faces)
    bool curved;
    std::vector<double> xyz_h;        // [P][3] node coordinates
    std::vector<double> geo_h;        // [P][BGK_NGEO]
    double *geo, *fvec;               // FP64 metric terms and face vectors
    float *geo32, *fvec32;            // their FP32 copies (mixed form)
    double *rho_w;                    // [Ne][6][q*q] diffuse-wall densities
    CurvOps32 cops;                   // FP32 tables of the mixed-form curvilinear stage
    int *wall_ef;                     // [n_wall][2] (element, face) pairs on diffuse faces
    int n_wall;
    // device
    cudaStream_t stream;
    int device;
    size_t elem;                      // bytes per state element
    void *f[3];                       // state (f^n) and two stage buffers
    double *part;                     // [n_vblk][NMOM][P]
    double *mom;                      // [P][NMOM]
    double *eq;                       // [P][NEQ]
    float *eq32;                      // [P][NEQ32] (mixed form)
    double *qp;                       // [P][5]
    double *vtab;                     // [Nu][VTAB]
    float4 *vtab32;                   // [Nu] FP32 velocity nodes
    double *bcval;                    // [6][C][Nu]
    unsigned int *status;
    NewtonStats *stats;
    int *iters;
    int Kblk, n_vblk;
    int lines, n_vblk_cap;            // first-axis velocity lines; most velocity blocks the partials hold
    bool part_valid;
    double tol;
    int max_iter;
    int qp_fp32;                      // Q' velocity sums on the FP32 pipe (mixed form default)
    int es_tensor;                    // tensor variant of the discrete ES equilibrium (delta = 0)
    int stage_variant, stage_depth;   // FP32 stage kernel choice and copy-ring depth
    int ring_limit;                   // test hook (bgk_test_ring_stall): velocities a ring delivers, 0 = all
    unsigned long long wait_ns;       // bounded-wait limit of the ring kernels, 0 = about 2 s
    // CUDA graphs of one SSP-RK3 step, one per buffer parity (f[0] alternates
    // between two buffers); recaptured when a launch parameter changes
    bool graphs_on;
    cudaStream_t cap_stream;          // private stream the graphs are captured on
    // pipelined host-to-host stepping (bgk_step_host): a fourth state buffer,
    // copy streams in each direction, and per buffer the event of its last
    // device-to-host copy
    struct HostPipe {
        void *extra[2] = {nullptr, nullptr};   // one or two more state buffers
        int n_extra = 0;
        cudaStream_t s_in = nullptr, s_out = nullptr;
        cudaEvent_t ev_in = nullptr, ev_comp = nullptr;
        void *buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        cudaEvent_t ev_out[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        bool out_pending[5] = {false, false, false, false, false};
        void *older[2] = {nullptr, nullptr};   // earlier results, oldest first: the next inputs' buffers
        bool active = false;
    } pipe;
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        void *f[3] = {nullptr, nullptr, nullptr};
        std::vector<double> sig;
    } graph[2];
    std::string err;
    // profiling: event pairs around launches, accumulated per kernel kind
    bool prof_on;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[BGK_NKINDS];
    long long launches[BGK_NKINDS];
    // learned guess
    float *mlp_w, *mlp_norm, *mlp_m, *mlp_v, *mlp_grad;
    float *mlp_w16;                   // BF16-rounded copy of mlp_w (refreshed when the weights change)
    double *mlp_loss;
    bool mlp_ready;
    int guess_mode, mlp_bf16;
    float *log;
    unsigned long long *log_count, *fallbacks;
    long long log_max;
    bool log_on;
};

namespace {

bgk_status fail(bgk_ctx *ctx, bgk_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

#define CU(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? BGK_ENOMEM : BGK_ECUDA,  \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                     \
    } while (0)

// ---- host-side FR operators (section "Numerical method") -------------------
// Legendre P_n and P_n' by the three-term recurrence.
void legendre(int n, double x, double &pn, double &dpn) {
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) { pn = 1.0; dpn = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        const double d2 = d0 + (2 * k + 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    pn = p1; dpn = d1;
}

void build_fr(int p, FROps &fr) {
    const int q = p + 1;
    fr.q = q;
    std::vector<double> x(q), lam(q);
    for (int i = 0; i < q; ++i) {        // Newton on P_q from cosine estimates
        double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre(q, t, pn, dpn);
            const double dt = pn / dpn;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double pn, dpn;
        legendre(q, t, pn, dpn);
        x[i] = t;
        fr.wq[i] = 2.0 / ((1.0 - t * t) * dpn * dpn);
        fr.xi[i] = t;
    }
    // barycentric weights lambda_j = 1 / prod_{m != j}(x_j - x_m)
    for (int j = 0; j < q; ++j) {
        double pr = 1.0;
        for (int m = 0; m < q; ++m)
            if (m != j) pr *= (x[j] - x[m]);
        lam[j] = 1.0 / pr;
    }
    // D_ij = (lambda_j / lambda_i) / (x_i - x_j), D_ii = -sum_{j != i} D_ij
    for (int i = 0; i < q; ++i) {
        double diag = 0.0;
        for (int j = 0; j < q; ++j) {
            if (j == i) continue;
            fr.D[i][j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            diag -= fr.D[i][j];
        }
        fr.D[i][i] = diag;
    }
    // l_j(t) at t = -1, +1 by the barycentric formula of the second kind
    for (int side = 0; side < 2; ++side) {
        const double t = side ? 1.0 : -1.0;
        double den = 0.0;
        for (int j = 0; j < q; ++j) den += lam[j] / (t - x[j]);
        for (int j = 0; j < q; ++j) {
            const double v = (lam[j] / (t - x[j])) / den;
            if (side) fr.lp[j] = v; else fr.lm[j] = v;
        }
    }
    // DG-recovering correction: g_L = (-1)^(p+1)/2 (P_{p+1} - P_p), g_R = (P_{p+1} + P_p)/2
    const double sL = (p % 2 == 0) ? -0.5 : 0.5;
    for (int i = 0; i < q; ++i) {
        double a, da, b, db;
        legendre(p + 1, x[i], a, da);
        legendre(p, x[i], b, db);
        fr.dgL[i] = sL * (da - db);
        fr.dgR[i] = 0.5 * (da + db);
    }
}

double maxwellian_value(double u1, double u2, double u3, const double *st) {
    const double rho = st[0], th = st[4];
    const double c1 = u1 - st[1], c2 = u2 - st[2], c3 = u3 - st[3];
    return rho / std::pow(2.0 * M_PI * th, 1.5) * std::exp(-(c1 * c1 + c2 * c2 + c3 * c3) / (2.0 * th));
}

cudaEvent_t pool_event(bgk_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one kernel launch: counts it and, when profiling, records events.
struct LaunchScope {
    bgk_ctx *ctx;
    int kind;
    cudaEvent_t b = nullptr;
    LaunchScope(bgk_ctx *c, int k) : ctx(c), kind(k) {
        ctx->launches[kind]++;
        if (ctx->prof_on) {
            cudaEvent_t a = pool_event(ctx);
            b = pool_event(ctx);
            cudaEventRecord(a, ctx->stream);
            ctx->prof_pending.push_back({kind, a, b});
        }
    }
    ~LaunchScope() {
        if (b) cudaEventRecord(b, ctx->stream);
    }
};

bgk_status check_device_status(bgk_ctx *ctx) {
    unsigned int st = 0;
    CU(cudaMemcpyAsync(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (st) {
        CU(cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), ctx->stream));
        if (st & BGK_DEV_TIMEOUT)
            return fail(ctx, BGK_ETIMEOUT, "a bounded wait in the stage kernel gave up (device status 0x%x)", st);
        if (st & BGK_DEV_NOCONV)
            return fail(ctx, BGK_ENOCONV, "Q' Newton iteration did not converge at some point");
        return fail(ctx, BGK_ENOCONV, "device status 0x%x", st);
    }
    return BGK_OK;
}

// Moment partials of a state.  The FP32 state's stepping path (resum =
// false) uses the stage epilogue's error-free FP32 accumulation; the
// diagnostic entry points (resum = true) re-sum in FP64, independently of it.
bgk_status run_moments(bgk_ctx *ctx, const void *f, bool resum = false) {
    LaunchScope ls(ctx, BGK_K_MOMENTS);
    if (ctx->precision == BGK_FP64) {
        MomentArgs64 a{(const double *)f, ctx->part, ctx->vtab, ctx->Nu, ctx->P, ctx->Kblk, ctx->C};
        CU(launch_moments_f64(a, ctx->n_vblk, ctx->stream));
    } else if (resum) {
        CU(launch_moments_f32((const float *)f, ctx->part, ctx->vtab, ctx->Nu, ctx->P, ctx->Kblk,
                              ctx->C, ctx->n_vblk, ctx->stream));
    } else {
        CU(launch_moments_f32_exact((const float *)f, ctx->part, ctx->vg, ctx->Nu, ctx->P, ctx->Kblk, ctx->C,
                                    ctx->n_vblk, ctx->stream));
    }
    return BGK_OK;
}

bgk_status run_qprime(bgk_ctx *ctx, const double *part, int n_vblk, int P, double *eq, double *qp,
                      int *iters, const double *guess) {
    QPrimeArgs a{};
    a.part = part; a.n_vblk = n_vblk; a.vtab = ctx->vtab_q; a.vtab32 = ctx->vtab32_q; a.guess = guess; a.eq = eq; a.qp = qp;
    a.eq32 = (eq && eq == ctx->eq) ? ctx->eq32 : nullptr;
    a.iters = iters; a.status = ctx->status; a.stats = ctx->stats; a.P = P; a.Nu = ctx->Nu_q;
    a.tol = ctx->tol; a.tol32 = 1e-6; a.max_iter = ctx->max_iter; a.gas = ctx->gas; a.vg = ctx->vg_q;
    a.mixed = ctx->precision == BGK_MIXED ? 1 : 0;
    a.mlp.w = ctx->mlp_w; a.mlp.norm = ctx->mlp_norm; a.mlp.w16 = ctx->mlp_w16;
    a.guess_mode = (ctx->guess_mode == 1 && ctx->mlp_ready) ? 1 : 0;
    a.mlp_bf16 = ctx->mlp_bf16;
    a.log = ctx->log_on ? ctx->log : nullptr;
    a.log_count = ctx->log_count; a.log_max = ctx->log_max; a.fallbacks = ctx->fallbacks;
    LaunchScope ls(ctx, BGK_K_QPRIME);
    if (ctx->es_tensor && a.eq) {
        // the d+2 solve gives the start; the refinement records the statistics
        QPrimeArgs a5 = a;
        a5.stats = nullptr;
        a5.log = nullptr;
        a5.eq32 = nullptr;
        CU(launch_qprime(a5, ctx->qp_fp32 != 0, ctx->stream));
        a.log = nullptr;
        CU(launch_qprime_tensor(a, ctx->qp_fp32 != 0, ctx->stream));
        return BGK_OK;
    }
    CU(launch_qprime(a, ctx->qp_fp32 != 0, ctx->stream));
    return BGK_OK;
}

template <typename T>
void set_geometry(bgk_ctx *ctx, StageArgs<T> &s);
template <>
void set_geometry<double>(bgk_ctx *ctx, StageArgs<double> &s) {
    s.geo = ctx->geo; s.fvec = ctx->fvec; s.rho_w = ctx->rho_w;
}
template <>
void set_geometry<float>(bgk_ctx *ctx, StageArgs<float> &s) {
    s.geo = ctx->geo32; s.fvec = ctx->fvec32; s.rho_w = ctx->rho_w;
    s.cops = ctx->cops;
}

// The FP32 tables of the curvilinear mixed-form stage (see CurvOps32): the
// rounded D, l(+1), g_R'; their mirror images for l(-1), g_L'; and the
// column-sum defects of the rounded D measured in FP64.
void build_curv_ops32(const FROps &fr, CurvOps32 &c) {
    const int q = fr.q;
    std::memset(&c, 0, sizeof c);
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j < q; ++j) c.D[i][j] = (float)fr.D[i][j];
        c.lp[i] = (float)fr.lp[i];
        c.dgR[i] = (float)fr.dgR[i];
    }
    for (int i = 0; i < q; ++i) {
        c.lm[i] = c.lp[q - 1 - i];
        c.dgL[i] = -c.dgR[q - 1 - i];
    }
    // column sums of the deviation-form operator: off-diagonal D (c'_j), the
    // own-value terms of each row (-W_j rho'_j), the lifted traces, and the
    // implicit (1 - sum l) weight of the exact-for-constants traces
    double sigR = 0.0, sigL = 0.0, wsum = 0.0, slp = 0.0, slm = 0.0;
    for (int i = 0; i < q; ++i) {
        sigR += fr.wq[i] * (double)c.dgR[i];
        sigL += fr.wq[i] * (double)c.dgL[i];
        wsum += fr.wq[i];
        slp += (double)c.lp[i];
        slm += (double)c.lm[i];
    }
    for (int j = 0; j < q; ++j) {
        double col = 0.0, row = 0.0;
        for (int i = 0; i < q; ++i)
            if (i != j) {
                col += fr.wq[i] * (double)c.D[i][j];
                row += (double)c.D[j][i];
            }
        const double dj = col - fr.wq[j] * row - sigR * (double)c.lp[j] - sigL * (double)c.lm[j] -
                          (1.0 - slp) * fr.wq[j] * (double)c.dgR[j] - (1.0 - slm) * fr.wq[j] * (double)c.dgL[j];
        c.def[j] = (float)(dj / wsum);
    }
}

template <typename T>
StageArgs<T> stage_args(bgk_ctx *ctx, const void *fn, const void *fs, void *fo, double a, double b,
                        double c, bool moments) {
    StageArgs<T> s{};
    s.f_n = (const T *)fn; s.f_s = (const T *)fs; s.f_out = (T *)fo;
    s.eq = ctx->eq; s.vtab = ctx->vtab; s.vtab32 = ctx->vtab32; s.bcval = ctx->bcval;
    s.part = moments ? ctx->part : nullptr;
    s.eq32 = ctx->eq32;
    s.status = ctx->status;
    s.a = a; s.b = b; s.c = c; s.Nu = ctx->Nu; s.P = ctx->P; s.Kblk = ctx->Kblk;
    s.vg = ctx->vg; s.fr = ctx->fr; s.mesh = ctx->mesh;
    s.a32 = (float)a; s.ab32 = (float)(a + b); s.c32 = (float)c;
    s.wait_ns = ctx->wait_ns;
    s.ring_limit = ctx->ring_limit;
    for (int d = 0; d < 3; ++d) s.toh32[d] = (float)ctx->mesh.two_over_h[d];
    if (ctx->curved) set_geometry<T>(ctx, s);
    return s;
}

bgk_status run_stage(bgk_ctx *ctx, const void *fn, const void *fs, void *fo, double a, double b,
                     double c, bool moments) {
    if (ctx->n_wall > 0) {            // diffuse-wall densities of the stage's input
        LaunchScope lw(ctx, BGK_K_WALL);
        if (ctx->precision == BGK_FP64)
            CU(launch_wall_density<double>((const double *)fs, ctx->fvec, ctx->bcval, ctx->vtab, ctx->wall_ef,
                                           ctx->n_wall, ctx->q, ctx->Ne, ctx->Nu, ctx->C, ctx->fr, ctx->rho_w,
                                           ctx->stream));
        else
            CU(launch_wall_density<float>((const float *)fs, ctx->fvec32, ctx->bcval, ctx->vtab, ctx->wall_ef,
                                          ctx->n_wall, ctx->q, ctx->Ne, ctx->Nu, ctx->C, ctx->fr, ctx->rho_w,
                                          ctx->stream));
    }
    LaunchScope ls(ctx, BGK_K_STAGE);
    if (ctx->precision == BGK_FP64)
        CU(launch_stage_f64(stage_args<double>(ctx, fn, fs, fo, a, b, c, moments), ctx->C, ctx->n_vblk,
                            ctx->stream));
    else {
        const StageArgs<float> sa = stage_args<float>(ctx, fn, fs, fo, a, b, c, moments);
        // caller buffers that a chosen variant cannot take (alignment) run on the plain kernel
        const int v = stage_f32_variant_supported(sa, ctx->C, ctx->stage_variant, ctx->stage_depth) ? ctx->stage_variant
                                                                                                   : BGK_STAGE_AUTO;
        CU(launch_stage_f32(sa, ctx->C, ctx->n_vblk, v, ctx->stage_depth, ctx->stream));
    }
    return BGK_OK;
}

// One full stage on device arrays: moments of fs must be in ctx->part.
bgk_status stage_from_partials(bgk_ctx *ctx, const void *fn, const void *fs, void *fo, double a,
                               double b, double c, bool moments_out) {
    bgk_status st = run_qprime(ctx, ctx->part, ctx->n_vblk, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr);
    if (st) return st;
    return run_stage(ctx, fn, fs, fo, a, b, c, moments_out);
}

// The three stages of one SSP-RK3 step (Shu--Osher form) on the context's
// buffers: f[0] = f^n, f[1], f[2] stage buffers; the result lands in f[1].
bgk_status enqueue_step(bgk_ctx *ctx, double dt) {
    void *f0 = ctx->f[0], *f1 = ctx->f[1], *f2 = ctx->f[2];
    bgk_status st;
    if ((st = stage_from_partials(ctx, nullptr, f0, f1, 0.0, 1.0, dt, true))) return st;
    if ((st = stage_from_partials(ctx, f0, f1, f2, 0.75, 0.25, 0.25 * dt, true))) return st;
    return stage_from_partials(ctx, f0, f2, f1, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt, true);
}

// Everything a captured step bakes into its kernel arguments.
std::vector<double> step_signature(const bgk_ctx *ctx, double dt) {
    return {dt,
            ctx->tol,
            (double)ctx->max_iter,
            (double)((ctx->guess_mode == 1 && ctx->mlp_ready) ? 1 : 0),
            (double)ctx->mlp_bf16,
            (double)(ctx->log_on ? 1 : 0),
            (double)(uintptr_t)ctx->log,
            (double)ctx->log_max,
            (double)ctx->stage_variant,
            (double)ctx->Kblk,
            (double)ctx->ring_limit,
            (double)ctx->wait_ns,
            (double)ctx->stage_depth,
            (double)ctx->qp_fp32,
            (double)ctx->es_tensor};
}

void drop_graphs(bgk_ctx *ctx) {
    for (auto &g : ctx->graph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = bgk_ctx::StepGraph{};
    }
}

// Launch one step as a CUDA graph, capturing it first if there is no graph
// for these buffers and parameters.
bgk_status replay_step(bgk_ctx *ctx, double dt) {
    const int slot = ctx->graph[0].f[0] == nullptr || ctx->graph[0].f[0] == ctx->f[0] ? 0 : 1;
    bgk_ctx::StepGraph &g = ctx->graph[slot];
    const std::vector<double> sig = step_signature(ctx, dt);
    if (!g.exec || g.sig != sig || g.f[0] != ctx->f[0] || g.f[1] != ctx->f[1] || g.f[2] != ctx->f[2]) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = bgk_ctx::StepGraph{};
        // capture on a private stream (the context's stream may be the legacy
        // default stream, which cannot be captured); replay on the context's
        if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        const cudaStream_t user = ctx->stream;
        CU(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
        ctx->stream = ctx->cap_stream;
        const bgk_status st = enqueue_step(ctx, dt);
        ctx->stream = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CU(e);
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CU(ei);
        g.f[0] = ctx->f[0]; g.f[1] = ctx->f[1]; g.f[2] = ctx->f[2];
        g.sig = sig;
    }
    CU(cudaGraphLaunch(g.exec, ctx->stream));
    return BGK_OK;
}

// Node coordinates of the uniform box mesh: x[P][3].
void box_node_coords(const bgk_ctx *ctx, double *x) {
    const int q = ctx->q, n1 = ctx->mesh.n[0], n2 = ctx->mesh.n[1];
    for (int e = 0; e < ctx->Ne; ++e) {
        const int c[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
        for (int s = 0; s < ctx->Ns; ++s) {
            const int id[3] = {s % q, (s / q) % q, s / (q * q)};
            for (int d = 0; d < 3; ++d) {
                const double hd = 2.0 / ctx->mesh.two_over_h[d];
                x[((size_t)e * ctx->Ns + s) * 3 + d] = ctx->lo[d] + (c[d] + 0.5 * (ctx->fr.xi[id[d]] + 1.0)) * hd;
            }
        }
    }
}

}  // namespace

void fr_build_host(int p, FROps &fr) { build_fr(p, fr); }

extern "C" {

}  // extern "C"
namespace {
// A context over the velocity planes [s_lo, s_hi) of the grid's third axis
// (the whole grid: 0, n[2]).
bgk_status create_ctx(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vg,
                      const bgk_gas_desc *gas, int precision, void *stream, int s_lo, int s_hi);
}  // namespace
extern "C" {

bgk_status bgk_create(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vg,
                      const bgk_gas_desc *gas, int precision, void *stream) {
    if (!out || !mesh || !vg || !gas) return BGK_EINVAL;
    return create_ctx(out, mesh, vg, gas, precision, stream, 0, vg->n[2]);
}

bgk_status bgk_create_shard(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vg,
                            const bgk_gas_desc *gas, int precision, void *stream, int slab_lo, int slab_hi) {
    if (!out || !mesh || !vg || !gas) return BGK_EINVAL;
    *out = nullptr;
    if (slab_lo < 0 || slab_hi > vg->n[2] || slab_hi - slab_lo < 2) {
        bgk_ctx *ctx = new bgk_ctx();
        ctx->err = "a shard holds third-axis velocity planes [slab_lo, slab_hi) with 0 <= slab_lo, "
                   "slab_hi <= n[2] and at least two planes";
        *out = ctx;
        return BGK_EINVAL;
    }
    for (int f = 0; f < 6; ++f)
        if (!mesh->periodic[f / 2] && mesh->face_type[f] != BGK_FACE_DIRICHLET) {
            bgk_ctx *ctx = new bgk_ctx();
            ctx->err = "a velocity shard supports periodic and Dirichlet faces only (specular faces mirror "
                       "velocities across shards, diffuse walls and closed faces sum over all velocities)";
            *out = ctx;
            return BGK_ENOTSUP;
        }
    return create_ctx(out, mesh, vg, gas, precision, stream, slab_lo, slab_hi);
}

}  // extern "C"
namespace {
bgk_status create_ctx(bgk_ctx **out, const bgk_mesh_desc *mesh, const bgk_vgrid_desc *vg,
                      const bgk_gas_desc *gas, int precision, void *stream, int s_lo, int s_hi) {
    *out = nullptr;
    bgk_ctx *ctx = new bgk_ctx();
    auto bad = [&](const char *msg) {
        ctx->err = msg;
        *out = ctx;   // keep the context so the caller can read the message
        return BGK_EINVAL;
    };
    if (mesh->order < 1 || mesh->order > 4) return bad("order must be in 1..4");
    for (int d = 0; d < 3; ++d) {
        if (mesh->n[d] < 1) return bad("mesh n[d] must be >= 1");
        if (!mesh->node_xyz && !(mesh->hi[d] > mesh->lo[d])) return bad("mesh hi must exceed lo");
        if (vg->n[d] < 2 || vg->n[d] > BGK_MAXV) return bad("velocity grid needs 2..128 nodes per axis");
        if (!(vg->hi[d] > vg->lo[d])) return bad("velocity hi must exceed lo");
    }
    if (!(gas->delta >= 0.0)) return bad("delta must be >= 0");
    if (!(gas->Pr >= 2.0 / 3.0 - 1e-12)) return bad("Pr must be >= 2/3");
    if (!(gas->mu_ref > 0.0) || !(gas->theta_ref > 0.0)) return bad("mu_ref, theta_ref must be > 0");
    if (precision != BGK_FP64 && precision != BGK_MIXED) return bad("unknown precision");
    for (int d = 0; d < 3; ++d)
        if (!mesh->periodic[d])
            for (int s = 0; s < 2; ++s) {
                const int ft = mesh->face_type[2 * d + s];
                const double *b = mesh->bc_state[2 * d + s];
                if (ft == BGK_FACE_DIRICHLET && (!(b[0] > 0.0) || !(b[4] > 0.0)))
                    return bad("Dirichlet state needs rho, theta > 0");
                if (ft == BGK_FACE_DIFFUSE && !(b[4] > 0.0)) return bad("a diffuse wall needs theta_w > 0");
            }
    const long long Ne = (long long)mesh->n[0] * mesh->n[1] * mesh->n[2];
    const long long Nu_full = (long long)vg->n[0] * vg->n[1] * vg->n[2];
    const long long Nu = (long long)vg->n[0] * vg->n[1] * (s_hi - s_lo);     // the planes this context holds
    const long long Ns = (long long)(mesh->order + 1) * (mesh->order + 1) * (mesh->order + 1);
    if (Ne * Ns > (1ll << 30) || Nu_full > (1ll << 30)) return bad("problem too large");
    bool curved = mesh->node_xyz != nullptr, any_specular = false;
    for (int f = 0; f < 6; ++f) {
        const int d = f / 2;
        if (mesh->face_type[f] < BGK_FACE_DIRICHLET || mesh->face_type[f] > BGK_FACE_CLOSED)
            return bad("face_type must be one of BGK_FACE_DIRICHLET, _SPECULAR, _DIFFUSE, _CLOSED");
        if (!mesh->periodic[d] && (mesh->face_type[f] == BGK_FACE_DIFFUSE || mesh->face_type[f] == BGK_FACE_CLOSED))
            curved = true;
        if (!mesh->periodic[d] && mesh->face_type[f] == BGK_FACE_SPECULAR) any_specular = true;
        if (mesh->face_type[f] == BGK_FACE_SPECULAR) {
            if (mesh->periodic[d]) return bad("a specular face must be non-periodic");
            if (std::fabs(vg->lo[d] + vg->hi[d]) > 1e-12 * (std::fabs(vg->lo[d]) + std::fabs(vg->hi[d])))
                return bad("a specular face needs a velocity grid symmetric in its axis");
        }
    }

    if (curved && any_specular) {
        ctx->err = "specular faces are supported on the uniform box mesh only (no node_xyz, no diffuse or closed faces)";
        *out = ctx;
        return BGK_ENOTSUP;
    }

    ctx->p = mesh->order; ctx->q = mesh->order + 1; ctx->Ns = (int)Ns; ctx->Ne = (int)Ne;
    ctx->Nu = (int)Nu; ctx->C = gas->delta > 0.0 ? 2 : 1; ctx->P = (int)(Ne * Ns);
    ctx->precision = precision;
    ctx->stream = (cudaStream_t)stream;
    ctx->tol = 1e-13;
    ctx->max_iter = 50;
    ctx->qp_fp32 = precision == BGK_MIXED ? 1 : 0;
    ctx->es_tensor = 0;
    ctx->stage_variant = BGK_STAGE_AUTO;
    ctx->stage_depth = 6;
    ctx->graphs_on = false;
    ctx->cap_stream = nullptr;
    ctx->shard = s_lo != 0 || s_hi != vg->n[2];
    ctx->slab_lo = s_lo;
    ctx->slab_hi = s_hi;
    for (int d = 0; d < 3; ++d) {
        const double h = (vg->hi[d] - vg->lo[d]) / (vg->n[d] - 1);
        ctx->vg_q.n[d] = vg->n[d];
        ctx->vg_q.lo[d] = vg->lo[d];
        ctx->vg_q.h[d] = h;
        ctx->vn[d] = d == 2 ? s_hi - s_lo : vg->n[d];
        ctx->vg.n[d] = ctx->vn[d];
        ctx->vg.lo[d] = d == 2 ? std::fma((double)s_lo, h, vg->lo[d]) : vg->lo[d];
        ctx->vg.h[d] = h;
        ctx->mesh.n[d] = mesh->n[d];
        ctx->mesh.periodic[d] = mesh->periodic[d] ? 1 : 0;
        ctx->mesh.two_over_h[d] = 2.0 * mesh->n[d] / (mesh->hi[d] - mesh->lo[d]);
    }
    ctx->vg_q.w3lo = ctx->vg_q.w3hi = 1;
    ctx->vg.w3lo = s_lo == 0 ? 1 : 0;            // interior slab ends carry full trapezoid weight
    ctx->vg.w3hi = s_hi == vg->n[2] ? 1 : 0;
    ctx->Nu_q = (int)Nu_full;
    ctx->mesh.Ne = ctx->Ne; ctx->mesh.Ns = ctx->Ns;
    for (int f = 0; f < 6; ++f) {
        ctx->mesh.specular[f] = !mesh->periodic[f / 2] && mesh->face_type[f] == BGK_FACE_SPECULAR;
        ctx->mesh.face_kind[f] = mesh->periodic[f / 2] ? BGK_FK_DIRICHLET : mesh->face_type[f];
    }
    ctx->jac = 1.0;
    for (int d = 0; d < 3; ++d) {
        ctx->jac *= 0.5 * (mesh->hi[d] - mesh->lo[d]) / mesh->n[d];
        ctx->lo[d] = mesh->lo[d];
    }
    std::memcpy(ctx->bc, mesh->bc_state, sizeof ctx->bc);
    build_fr(ctx->p, ctx->fr);
    ctx->curved = curved;
    ctx->geo = ctx->fvec = nullptr; ctx->geo32 = ctx->fvec32 = nullptr;
    ctx->rho_w = nullptr; ctx->wall_ef = nullptr; ctx->n_wall = 0;
    std::vector<double> fvec_h;
    std::vector<int> wall_h;
    if (curved) {
        ctx->xyz_h.resize((size_t)ctx->P * 3);
        if (mesh->node_xyz) {
            std::memcpy(ctx->xyz_h.data(), mesh->node_xyz, ctx->xyz_h.size() * sizeof(double));
        } else {
            box_node_coords(ctx, ctx->xyz_h.data());
        }
        std::string gerr;
        if (!build_curved_geometry(ctx->fr, mesh->n, ctx->mesh.periodic, ctx->xyz_h.data(), ctx->geo_h, fvec_h, gerr))
            return bad(gerr.c_str());
        build_curv_ops32(ctx->fr, ctx->cops);
        if (precision == BGK_MIXED) {
            // the mixed form divides by the FP32 1/J: its totals weigh the nodes
            // with W_s / (1/J)_32, so the quadrature the stage conserves is the
            // one the totals measure
            for (int p = 0; p < ctx->P; ++p) {
                double *g = &ctx->geo_h[(size_t)p * BGK_NGEO];
                const int s = p % ctx->Ns, q = ctx->q;
                const double W = ctx->fr.wq[s % q] * ctx->fr.wq[(s / q) % q] * ctx->fr.wq[s / (q * q)];
                g[10] = W / (double)(float)g[9];
            }
        }
        for (int e = 0; e < ctx->Ne; ++e) {
            const int ec[3] = {e % mesh->n[0], (e / mesh->n[0]) % mesh->n[1], e / (mesh->n[0] * mesh->n[1])};
            for (int f = 0; f < 6; ++f) {
                const int d = f / 2;
                const bool edge = (f % 2 == 0) ? ec[d] == 0 : ec[d] == mesh->n[d] - 1;
                if (edge && !mesh->periodic[d] && mesh->face_type[f] == BGK_FACE_DIFFUSE) {
                    wall_h.push_back(e);
                    wall_h.push_back(f);
                }
            }
        }
        ctx->n_wall = (int)(wall_h.size() / 2);
    }
    ctx->gas.delta = gas->delta; ctx->gas.Pr = gas->Pr; ctx->gas.mu_ref = gas->mu_ref;
    ctx->gas.theta_ref = gas->theta_ref; ctx->gas.theta_S = gas->theta_S;
    ctx->gas.gamma = (5.0 + gas->delta) / (3.0 + gas->delta);

    // velocity table: nodes, trapezoid weights, |u|^2/2
    std::vector<double> ax[3], wt[3];
    for (int d = 0; d < 3; ++d) {
        const double h = (vg->hi[d] - vg->lo[d]) / (vg->n[d] - 1);
        for (int j = 0; j < vg->n[d]; ++j) {
            ax[d].push_back(std::fma((double)j, h, vg->lo[d]));
            wt[d].push_back((j == 0 || j == vg->n[d] - 1) ? 0.5 * h : h);
        }
    }
    // the table of velocities k3 in [k3_from, k3_from + n_k / (n0 n1)), weights of the whole grid
    auto fill_vtab = [&](std::vector<double> &tab, long long n_k, int k3_from) {
        tab.assign((size_t)n_k * BGK_VTAB, 0.0);
        for (long long k = 0; k < n_k; ++k) {
            const int k1 = (int)(k % vg->n[0]), k2 = (int)((k / vg->n[0]) % vg->n[1]);
            const int k3 = k3_from + (int)(k / ((long long)vg->n[0] * vg->n[1]));
            double *v = &tab[(size_t)k * BGK_VTAB];
            v[0] = ax[0][k1]; v[1] = ax[1][k2]; v[2] = ax[2][k3];
            v[3] = wt[0][k1] * wt[1][k2] * wt[2][k3];
            v[4] = 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            v[5] = v[3] * v[0];
            v[6] = v[3] * v[0] * v[0];
            v[7] = 2.0 * mesh->n[0] / (mesh->hi[0] - mesh->lo[0]) * v[0];   // (2/h_1) u_1
        }
    };
    fill_vtab(ctx->vtab_h, Nu, s_lo);
    std::vector<double> vtab_q_h;
    if (ctx->shard) fill_vtab(vtab_q_h, Nu_full, 0);
    // Dirichlet exterior states per face and velocity
    std::vector<double> bcv((size_t)6 * ctx->C * Nu, 0.0);
    for (int face = 0; face < 6; ++face) {
        if (mesh->periodic[face / 2] || ctx->mesh.specular[face] || mesh->face_type[face] == BGK_FACE_CLOSED) continue;
        double st[5];
        std::memcpy(st, mesh->bc_state[face], sizeof st);
        if (mesh->face_type[face] == BGK_FACE_DIFFUSE) st[0] = 1.0;   // unit density; rho_w per flux node
        for (int k = 0; k < Nu; ++k) {
            const double *v = &ctx->vtab_h[(size_t)k * BGK_VTAB];
            const double F = maxwellian_value(v[0], v[1], v[2], st);
            bcv[((size_t)face * ctx->C + 0) * Nu + k] = F;
            if (ctx->C == 2) bcv[((size_t)face * ctx->C + 1) * Nu + k] = 0.5 * gas->delta * st[4] * F;
        }
    }
    // velocity blocking: enough CTAs to fill the GPU, bounded partial buffer
    {
        const int n_pb = (ctx->P + 255) / 256;
        const int lines = (int)(Nu / vg->n[0]);
        int want = (2432 + n_pb - 1) / n_pb;
        if (want > 64) want = 64;
        if (want > lines) want = lines;
        if (want < 1) want = 1;
        const int lines_per_blk = (lines + want - 1) / want;
        ctx->Kblk = lines_per_blk * vg->n[0];
        ctx->n_vblk = (int)((Nu + ctx->Kblk - 1) / ctx->Kblk);
        ctx->lines = lines;
        ctx->n_vblk_cap = std::max(ctx->n_vblk, std::min(64, lines));   // room for bgk_set_velocity_blocks
    }

    bgk_status st = BGK_OK;
    auto cu = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == BGK_OK) {
            st = e == cudaErrorMemoryAllocation ? BGK_ENOMEM : BGK_ECUDA;
            ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    cu(cudaGetDevice(&ctx->device), "cudaGetDevice");
    ctx->elem = precision == BGK_FP64 ? sizeof(double) : sizeof(float);
    const size_t fbytes = (size_t)ctx->C * Nu * ctx->P * ctx->elem;
    for (int i = 0; i < 3; ++i) {
        ctx->f[i] = nullptr;
        if (st == BGK_OK) cu(cudaMalloc(&ctx->f[i], fbytes), "cudaMalloc(state)");
    }
    const size_t P = ctx->P;
    if (st == BGK_OK) cu(cudaMalloc(&ctx->part, (size_t)ctx->n_vblk_cap * BGK_NMOM * P * sizeof(double)), "cudaMalloc(part)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mom, P * BGK_NMOM * sizeof(double)), "cudaMalloc(mom)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->eq, P * BGK_NEQ * sizeof(double)), "cudaMalloc(eq)");
    ctx->eq32 = nullptr;
    if (st == BGK_OK && precision == BGK_MIXED)
        cu(cudaMalloc(&ctx->eq32, P * BGK_NEQ32 * sizeof(float)), "cudaMalloc(eq32)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->qp, P * 5 * sizeof(double)), "cudaMalloc(qp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->iters, P * sizeof(int)), "cudaMalloc(iters)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->vtab, ctx->vtab_h.size() * sizeof(double)), "cudaMalloc(vtab)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->bcval, bcv.size() * sizeof(double)), "cudaMalloc(bcval)");
    std::vector<float4> v32(Nu);
    for (int k = 0; k < Nu; ++k) {
        const double *v = &ctx->vtab_h[(size_t)k * BGK_VTAB];
        v32[k] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
    }
    if (st == BGK_OK) cu(cudaMalloc(&ctx->vtab32, v32.size() * sizeof(float4)), "cudaMalloc(vtab32)");
    if (st == BGK_OK) cu(cudaMemcpyAsync(ctx->vtab32, v32.data(), v32.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream), "upload vtab32");
    // the whole grid's tables for the Q' solve of a shard
    ctx->vtab_q = ctx->vtab;
    ctx->vtab32_q = ctx->vtab32;
    std::vector<float4> v32q;
    if (st == BGK_OK && ctx->shard) {
        ctx->vtab_q = nullptr;
        ctx->vtab32_q = nullptr;
        v32q.resize((size_t)Nu_full);
        for (long long k = 0; k < Nu_full; ++k) {
            const double *v = &vtab_q_h[(size_t)k * BGK_VTAB];
            v32q[k] = make_float4((float)v[0], (float)v[1], (float)v[2], 0.f);
        }
        cu(cudaMalloc(&ctx->vtab_q, vtab_q_h.size() * sizeof(double)), "cudaMalloc(vtab_q)");
        if (st == BGK_OK) cu(cudaMalloc(&ctx->vtab32_q, v32q.size() * sizeof(float4)), "cudaMalloc(vtab32_q)");
        if (st == BGK_OK)
            cu(cudaMemcpyAsync(ctx->vtab_q, vtab_q_h.data(), vtab_q_h.size() * sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream), "upload vtab_q");
        if (st == BGK_OK)
            cu(cudaMemcpyAsync(ctx->vtab32_q, v32q.data(), v32q.size() * sizeof(float4), cudaMemcpyHostToDevice,
                               ctx->stream), "upload vtab32_q");
    }
    if (st == BGK_OK && curved) {
        const size_t ng = ctx->geo_h.size(), nf = fvec_h.size();
        const int q = ctx->q, Ns = ctx->Ns;
        // FP32 node records: S, 1/J, and S_face - S^d_node per face (in FP64)
        std::vector<float> g32((size_t)ctx->P * BGK_NGEO32, 0.f), f32(nf);
        for (int p = 0; p < ctx->P; ++p) {
            const double *g = &ctx->geo_h[(size_t)p * BGK_NGEO];
            float *o = &g32[(size_t)p * BGK_NGEO32];
            for (int i = 0; i < 10; ++i) o[i] = (float)g[i];
            const int e = p / Ns, s = p % Ns;
            const int id[3] = {s % q, (s / q) % q, s / (q * q)};
            const int fpi[3] = {id[1] + q * id[2], id[0] + q * id[2], id[0] + q * id[1]};
            for (int fc = 0; fc < 6; ++fc) {
                const int d = fc / 2;
                const double *fv = &fvec_h[(((size_t)e * 6 + fc) * q * q + fpi[d]) * 3];
                for (int c = 0; c < 3; ++c) o[10 + 3 * fc + c] = (float)(fv[c] - g[3 * d + c]);
            }
            // geometric remainder H (CurvOps32): the f_i-proportional terms of the
            // three directions' operators, with the FP32 coefficients, in FP64
            const CurvOps32 &co = ctx->cops;
            const int stride[3] = {1, q, q * q};
            double H[3] = {0.0, 0.0, 0.0};
            for (int d = 0; d < 3; ++d) {
                const int i = id[d];
                const int base = s - i * stride[d];
                const double *Si = &ctx->geo_h[((size_t)e * Ns + s) * BGK_NGEO + 3 * d];
                const double *FL = &fvec_h[(((size_t)e * 6 + 2 * d) * q * q + fpi[d]) * 3];
                const double *FR = &fvec_h[(((size_t)e * 6 + 2 * d + 1) * q * q + fpi[d]) * 3];
                for (int c = 0; c < 3; ++c) {
                    double vol = 0.0, trL = 0.0, trR = 0.0;
                    for (int j = 0; j < q; ++j) {
                        const double dS = ctx->geo_h[((size_t)e * Ns + base + j * stride[d]) * BGK_NGEO + 3 * d + c] - Si[c];
                        if (j != i) vol += (double)co.D[i][j] * dS;
                        vol -= (double)co.def[j] * dS;
                        trL += (double)co.lm[j] * dS;
                        trR += (double)co.lp[j] * dS;
                    }
                    H[c] += vol + (double)co.dgR[i] * (FR[c] - Si[c] - trR) + (double)co.dgL[i] * (FL[c] - Si[c] - trL);
                }
            }
            for (int c = 0; c < 3; ++c) o[28 + c] = (float)H[c];
        }
        for (size_t i = 0; i < nf; ++i) f32[i] = (float)fvec_h[i];
        cu(cudaMalloc(&ctx->geo, ng * sizeof(double)), "cudaMalloc(geo)");
        if (st == BGK_OK) cu(cudaMalloc(&ctx->fvec, nf * sizeof(double)), "cudaMalloc(fvec)");
        if (st == BGK_OK) cu(cudaMalloc(&ctx->geo32, g32.size() * sizeof(float)), "cudaMalloc(geo32)");
        if (st == BGK_OK) cu(cudaMalloc(&ctx->fvec32, nf * sizeof(float)), "cudaMalloc(fvec32)");
        if (st == BGK_OK) cu(cudaMalloc(&ctx->rho_w, (size_t)ctx->Ne * 6 * ctx->q * ctx->q * sizeof(double)), "cudaMalloc(rho_w)");
        if (st == BGK_OK && ctx->n_wall) cu(cudaMalloc(&ctx->wall_ef, wall_h.size() * sizeof(int)), "cudaMalloc(wall)");
        if (st == BGK_OK) cu(cudaMemcpy(ctx->geo, ctx->geo_h.data(), ng * sizeof(double), cudaMemcpyHostToDevice), "upload geo");
        if (st == BGK_OK) cu(cudaMemcpy(ctx->fvec, fvec_h.data(), nf * sizeof(double), cudaMemcpyHostToDevice), "upload fvec");
        if (st == BGK_OK) cu(cudaMemcpy(ctx->geo32, g32.data(), g32.size() * sizeof(float), cudaMemcpyHostToDevice), "upload geo32");
        if (st == BGK_OK) cu(cudaMemcpy(ctx->fvec32, f32.data(), nf * sizeof(float), cudaMemcpyHostToDevice), "upload fvec32");
        if (st == BGK_OK) cu(cudaMemset(ctx->rho_w, 0, (size_t)ctx->Ne * 6 * ctx->q * ctx->q * sizeof(double)), "memset rho_w");
        if (st == BGK_OK && ctx->n_wall)
            cu(cudaMemcpy(ctx->wall_ef, wall_h.data(), wall_h.size() * sizeof(int), cudaMemcpyHostToDevice), "upload wall");
    }
    if (st == BGK_OK) cu(cudaMalloc(&ctx->status, sizeof(unsigned int)), "cudaMalloc(status)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->stats, sizeof(NewtonStats)), "cudaMalloc(stats)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_w, MLP_NPARAM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_norm, MLP_NNORM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_w16, MLP_NPARAM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_m, MLP_NPARAM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_v, MLP_NPARAM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_grad, MLP_NPARAM * sizeof(float)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->mlp_loss, sizeof(double)), "cudaMalloc(mlp)");
    if (st == BGK_OK) cu(cudaMalloc(&ctx->log_count, 2 * sizeof(unsigned long long)), "cudaMalloc(log)");
    if (st == BGK_OK) {
        ctx->fallbacks = ctx->log_count + 1;
        cu(cudaMemsetAsync(ctx->log_count, 0, 2 * sizeof(unsigned long long), ctx->stream), "memset log");
    }
    if (st == BGK_OK) cu(cudaMemcpyAsync(ctx->vtab, ctx->vtab_h.data(), ctx->vtab_h.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload vtab");
    if (st == BGK_OK) cu(cudaMemcpyAsync(ctx->bcval, bcv.data(), bcv.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload bc");
    if (st == BGK_OK) cu(cudaMemsetAsync(ctx->status, 0, sizeof(unsigned int), ctx->stream), "memset status");
    if (st == BGK_OK) cu(cudaMemsetAsync(ctx->stats, 0, sizeof(NewtonStats), ctx->stream), "memset stats");
    if (st == BGK_OK) cu(cudaMemsetAsync(ctx->f[0], 0, fbytes, ctx->stream), "memset state");
    if (st == BGK_OK) cu(cudaStreamSynchronize(ctx->stream), "sync");
    ctx->part_valid = false;
    *out = ctx;
    return st;
}
}  // namespace
extern "C" {

bgk_status bgk_fr_tables(int order, double *fr_out, float *curv32_out) {
    if (order < 1 || order > 4 || !fr_out || !curv32_out) return BGK_EINVAL;
    FROps fr{};
    build_fr(order, fr);
    CurvOps32 c;
    build_curv_ops32(fr, c);
    const int q = order + 1;
    double *o = fr_out;
    for (int i = 0; i < q; ++i) *o++ = fr.xi[i];
    for (int i = 0; i < q; ++i) *o++ = fr.wq[i];
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) *o++ = fr.D[i][j];
    for (int i = 0; i < q; ++i) *o++ = fr.lm[i];
    for (int i = 0; i < q; ++i) *o++ = fr.lp[i];
    for (int i = 0; i < q; ++i) *o++ = fr.dgL[i];
    for (int i = 0; i < q; ++i) *o++ = fr.dgR[i];
    float *f = curv32_out;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) *f++ = c.D[i][j];
    for (int i = 0; i < q; ++i) *f++ = c.lp[i];
    for (int i = 0; i < q; ++i) *f++ = c.lm[i];
    for (int i = 0; i < q; ++i) *f++ = c.dgL[i];
    for (int i = 0; i < q; ++i) *f++ = c.dgR[i];
    for (int i = 0; i < q; ++i) *f++ = c.def[i];
    return BGK_OK;
}

bgk_status bgk_curved_metrics(const bgk_mesh_desc *mesh, double *S, double *J, double *fvec) {
    if (!mesh || !mesh->node_xyz || !S || !J || !fvec) return BGK_EINVAL;
    if (mesh->order < 1 || mesh->order > 4) return BGK_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (mesh->n[d] < 1) return BGK_EINVAL;
    FROps fr{};
    build_fr(mesh->order, fr);
    int periodic[3];
    for (int d = 0; d < 3; ++d) periodic[d] = mesh->periodic[d] ? 1 : 0;
    std::vector<double> geo, fv;
    std::string err;
    if (!build_curved_geometry(fr, mesh->n, periodic, mesh->node_xyz, geo, fv, err)) return BGK_EINVAL;
    const size_t P = geo.size() / BGK_NGEO;
    for (size_t p = 0; p < P; ++p) {
        for (int i = 0; i < 9; ++i) S[p * 9 + i] = geo[p * BGK_NGEO + i];
        J[p] = 1.0 / geo[p * BGK_NGEO + 9];
    }
    std::memcpy(fvec, fv.data(), fv.size() * sizeof(double));
    return BGK_OK;
}

bgk_status bgk_destroy(bgk_ctx *ctx) {
    if (!ctx) return BGK_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    {
        bgk_ctx::HostPipe &hp = ctx->pipe;
        if (hp.s_in) { cudaStreamSynchronize(hp.s_in); cudaStreamDestroy(hp.s_in); }
        if (hp.s_out) { cudaStreamSynchronize(hp.s_out); cudaStreamDestroy(hp.s_out); }
        if (hp.ev_in) cudaEventDestroy(hp.ev_in);
        if (hp.ev_comp) cudaEventDestroy(hp.ev_comp);
        for (int i = 0; i < 5; ++i)
            if (hp.ev_out[i]) cudaEventDestroy(hp.ev_out[i]);
    }
    for (auto &r : ctx->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    // the state buffers: f[0..2], plus the host pipeline's fourth buffer,
    // which may have rotated into f[] (free each pointer once)
    {
        void *bufs[5] = {ctx->f[0], ctx->f[1], ctx->f[2], ctx->pipe.extra[0], ctx->pipe.extra[1]};
        for (int i = 0; i < 5; ++i) {
            bool seen = false;
            for (int j = 0; j < i; ++j) seen = seen || bufs[j] == bufs[i];
            if (bufs[i] && !seen) cudaFree(bufs[i]);
        }
    }
    cudaFree(ctx->part); cudaFree(ctx->mom); cudaFree(ctx->eq); cudaFree(ctx->qp);
    cudaFree(ctx->iters); cudaFree(ctx->eq32); cudaFree(ctx->vtab); cudaFree(ctx->vtab32); cudaFree(ctx->bcval); cudaFree(ctx->status);
    if (ctx->shard) { cudaFree(ctx->vtab_q); cudaFree(ctx->vtab32_q); }
    cudaFree(ctx->stats);
    cudaFree(ctx->geo); cudaFree(ctx->fvec); cudaFree(ctx->geo32); cudaFree(ctx->fvec32);
    cudaFree(ctx->rho_w); cudaFree(ctx->wall_ef);
    cudaFree(ctx->mlp_w); cudaFree(ctx->mlp_w16); cudaFree(ctx->mlp_norm); cudaFree(ctx->mlp_m); cudaFree(ctx->mlp_v);
    cudaFree(ctx->mlp_grad); cudaFree(ctx->mlp_loss); cudaFree(ctx->log); cudaFree(ctx->log_count);
    delete ctx;
    return BGK_OK;
}

bgk_status bgk_sizes(const bgk_ctx *ctx, int *n_elem, int *n_sol, int *n_vel, int *n_comp) {
    if (!ctx) return BGK_EINVAL;
    if (n_elem) *n_elem = ctx->Ne;
    if (n_sol) *n_sol = ctx->Ns;
    if (n_vel) *n_vel = ctx->Nu;
    if (n_comp) *n_comp = ctx->C;
    return BGK_OK;
}

const char *bgk_last_error(const bgk_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

bgk_status bgk_node_coords(const bgk_ctx *ctx_c, double *x, int on_device) {
    bgk_ctx *ctx = const_cast<bgk_ctx *>(ctx_c);
    if (!ctx || !x) return BGK_EINVAL;
    std::vector<double> h((size_t)ctx->P * 3);
    if (ctx->curved) h = ctx->xyz_h;
    else box_node_coords(ctx, h.data());
    CU(cudaMemcpyAsync(x, h.data(), h.size() * sizeof(double),
                       on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_set_state(bgk_ctx *ctx, const void *f, int on_device) {
    if (!ctx || !f) return BGK_EINVAL;
    if (ctx->pipe.active) {                 // host copies of bgk_step_host may still read the state
        bgk_status ps = bgk_step_host_sync(ctx);
        if (ps) return ps;
    }
    const size_t bytes = (size_t)ctx->C * ctx->Nu * ctx->P * ctx->elem;
    CU(cudaMemcpyAsync(ctx->f[0], f, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->part_valid = false;
    if (!on_device) CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_get_state(bgk_ctx *ctx, void *f, int on_device) {
    if (!ctx || !f) return BGK_EINVAL;
    if (ctx->pipe.active) {
        bgk_status ps = bgk_step_host_sync(ctx);
        if (ps) return ps;
    }
    const size_t bytes = (size_t)ctx->C * ctx->Nu * ctx->P * ctx->elem;
    CU(cudaMemcpyAsync(f, ctx->f[0], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (!on_device) CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_set_maxwellian(bgk_ctx *ctx, const double *q, int on_device) {
    if (!ctx || !q) return BGK_EINVAL;
    if (ctx->pipe.active) {
        bgk_status ps = bgk_step_host_sync(ctx);
        if (ps) return ps;
    }
    const double *dq = q;
    double *tmp = nullptr;
    if (!on_device) {
        CU(cudaMallocAsync((void **)&tmp, (size_t)ctx->P * 5 * sizeof(double), ctx->stream));
        CU(cudaMemcpyAsync(tmp, q, (size_t)ctx->P * 5 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        dq = tmp;
    }
    {
        LaunchScope ls(ctx, BGK_K_OTHER);
        if (ctx->precision == BGK_FP64)
            CU(launch_maxwellian_f64((double *)ctx->f[0], dq, ctx->vtab, ctx->Nu, ctx->P, ctx->C,
                                     ctx->gas.delta, ctx->stream));
        else
            CU(launch_maxwellian_f32((float *)ctx->f[0], dq, ctx->vtab, ctx->Nu, ctx->P, ctx->C,
                                     ctx->gas.delta, ctx->stream));
    }
    if (tmp) CU(cudaFreeAsync(tmp, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->part_valid = false;
    return BGK_OK;
}

bgk_status bgk_set_qprime_engine(bgk_ctx *ctx, int fp32_sums) {
    if (!ctx) return BGK_EINVAL;
    if (fp32_sums && ctx->precision != BGK_MIXED)
        return fail(ctx, BGK_EINVAL, "FP32 Q' sums are for the mixed form only");
    ctx->qp_fp32 = fp32_sums ? 1 : 0;
    return BGK_OK;
}

bgk_status bgk_set_es_tensor(bgk_ctx *ctx, int enable) {
    if (!ctx) return BGK_EINVAL;
    if (enable && ctx->C != 1)
        return fail(ctx, BGK_ENOTSUP, "the tensor variant of the ES equilibrium is for a monatomic gas (delta = 0)");
    ctx->es_tensor = enable ? 1 : 0;
    return BGK_OK;
}

bgk_status bgk_set_stage_kernel(bgk_ctx *ctx, int variant, int depth) {
    if (!ctx || variant < BGK_STAGE_AUTO || variant > BGK_STAGE_HALF_WIDE || depth < 2 || depth > BGK_MAX_DEPTH)
        return BGK_EINVAL;
    if (variant >= BGK_STAGE_ASYNC) {
        if (ctx->precision != BGK_MIXED)
            return fail(ctx, BGK_ENOTSUP, "the asynchronous-copy stage kernels are for the mixed form only");
        const StageArgs<float> a = stage_args<float>(ctx, ctx->f[0], ctx->f[1], ctx->f[2], 0.5, 0.5, 1.0, true);
        if (!stage_f32_variant_supported(a, ctx->C, variant, depth))
            return fail(ctx, BGK_ENOTSUP, "asynchronous-copy stage kernels need the uniform box mesh (no specular, "
                                          "diffuse or closed faces), p = 1 or 3 and fitting shared memory");
    }
    ctx->stage_variant = variant;
    ctx->stage_depth = depth;
    return BGK_OK;
}

}  // extern "C"
namespace {
// Velocity blocking: n blocks of whole first-axis lines (the last may be
// shorter); the cached partials and captured graphs no longer apply.
void set_blocking(bgk_ctx *ctx, int n) {
    const int lpb = (ctx->lines + n - 1) / n;
    ctx->Kblk = lpb * ctx->vg.n[0];
    ctx->n_vblk = (int)((ctx->Nu + ctx->Kblk - 1) / ctx->Kblk);
    ctx->part_valid = false;
    drop_graphs(ctx);
}
}  // namespace
extern "C" {

bgk_status bgk_set_velocity_blocks(bgk_ctx *ctx, int n) {
    if (!ctx || n < 1) return BGK_EINVAL;
    if (n > ctx->n_vblk_cap)
        return fail(ctx, BGK_EINVAL, "at most %d velocity blocks on this context", ctx->n_vblk_cap);
    bgk_status st;
    if (ctx->pipe.active && (st = bgk_step_host_sync(ctx))) return st;
    CU(cudaStreamSynchronize(ctx->stream));
    set_blocking(ctx, n);
    return BGK_OK;
}

bgk_status bgk_get_velocity_blocks(const bgk_ctx *ctx, int *n_blocks, int *per_block, int *max_blocks) {
    if (!ctx) return BGK_EINVAL;
    if (n_blocks) *n_blocks = ctx->n_vblk;
    if (per_block) *per_block = ctx->Kblk;
    if (max_blocks) *max_blocks = ctx->n_vblk_cap;
    return BGK_OK;
}

bgk_status bgk_test_ring_stall(bgk_ctx *ctx, int after, double wait_seconds) {
    if (!ctx || after < 0 || !(wait_seconds >= 0.0) || wait_seconds > 10.0) return BGK_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->ring_limit = after;
    ctx->wait_ns = after > 0 ? (unsigned long long)(wait_seconds * 1e9) : 0ull;
    return BGK_OK;
}

bgk_status bgk_tune_stage(bgk_ctx *ctx, double dt, int reps, int *variant_out, int *depth_out, double *ms_out) {
    if (!ctx || !(dt > 0.0) || reps < 1) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "tune on an unsharded context of the same problem (a shard's own moments are partial)");
    bgk_status st;
    if (ctx->precision != BGK_MIXED) {
        // one stage kernel: only the velocity blocking is chosen, by the
        // stage's time (the FP64 Q' solve does not depend on it)
        const int n0 = ctx->n_vblk;
        std::vector<int> nb{n0};
        for (int n = n0 + 1; n <= std::min(ctx->n_vblk_cap, 4 * n0); ++n)
            if (ctx->lines % n == 0) nb.push_back(n);
        if (!ctx->part_valid) {
            if ((st = run_moments(ctx, ctx->f[0]))) return st;
            ctx->part_valid = true;
        }
        if ((st = run_qprime(ctx, ctx->part, ctx->n_vblk, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr))) return st;
        cudaEvent_t ea = nullptr, eb = nullptr;
        CU(cudaEventCreate(&ea));
        CU(cudaEventCreate(&eb));
        cudaError_t err = cudaSuccess;
        double best = 1e300;
        int pick_nb = n0;
        for (int n : nb) {
            set_blocking(ctx, n);
            StageArgs<double> sd = stage_args<double>(ctx, ctx->f[0], ctx->f[0], ctx->f[2], 0.75, 0.25, 0.25 * dt, true);
            err = launch_stage_f64(sd, ctx->C, ctx->n_vblk, ctx->stream);                   // warm-up
            if (err == cudaSuccess) err = cudaEventRecord(ea, ctx->stream);
            for (int r = 0; r < reps && err == cudaSuccess; ++r) err = launch_stage_f64(sd, ctx->C, ctx->n_vblk, ctx->stream);
            if (err == cudaSuccess) err = cudaEventRecord(eb, ctx->stream);
            if (err == cudaSuccess) err = cudaEventSynchronize(eb);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ea, eb);
            if (err != cudaSuccess) break;
            if (ms / reps < best) { best = ms / reps; pick_nb = n; }
        }
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        set_blocking(ctx, pick_nb);
        CU(err);
        if ((st = check_device_status(ctx))) return st;
        if (variant_out) *variant_out = BGK_STAGE_PLAIN;
        if (depth_out) *depth_out = ctx->stage_depth;
        if (ms_out) *ms_out = best;
        return BGK_OK;
    }
    if (!ctx->part_valid) {
        if ((st = run_moments(ctx, ctx->f[0]))) return st;
        ctx->part_valid = true;
    }
    if ((st = run_qprime(ctx, ctx->part, ctx->n_vblk, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr))) return st;
    // candidates: the plain kernel and every ring depth of the asynchronous one;
    // each runs a full stage (with f^n and the moment epilogue) from the
    // current state into the scratch buffer, so the state itself is untouched
    const StageArgs<float> sa = stage_args<float>(ctx, ctx->f[0], ctx->f[0], ctx->f[2], 0.75, 0.25, 0.25 * dt, true);
    struct Cand { int v, d; };
    std::vector<Cand> cands{{BGK_STAGE_PLAIN, ctx->stage_depth}};
    for (int v : {BGK_STAGE_ASYNC, BGK_STAGE_LINE, BGK_STAGE_LINE_WIDE, BGK_STAGE_HALF, BGK_STAGE_HALF_WIDE})
        for (int d : {2, 3, 4, 6, 8, 12, 16})
            if (stage_f32_variant_supported(sa, ctx->C, v, d)) cands.push_back({v, d});
    cudaEvent_t ea = nullptr, eb = nullptr;
    CU(cudaEventCreate(&ea));
    CU(cudaEventCreate(&eb));
    double best = 1e300;
    Cand pick = cands[0];
    cudaError_t err = cudaSuccess;
    for (const Cand &c : cands) {
        err = launch_stage_f32(sa, ctx->C, ctx->n_vblk, c.v, c.d, ctx->stream);      // warm-up
        if (err == cudaSuccess) err = cudaEventRecord(ea, ctx->stream);
        for (int r = 0; r < reps && err == cudaSuccess; ++r)
            err = launch_stage_f32(sa, ctx->C, ctx->n_vblk, c.v, c.d, ctx->stream);
        if (err == cudaSuccess) err = cudaEventRecord(eb, ctx->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(eb);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ea, eb);
        if (err != cudaSuccess) break;
        if (ms / reps < best) { best = ms / reps; pick = c; }
    }
    ctx->part_valid = false;              // the partials now describe the scratch output
    if (err == cudaSuccess) {
        // then the velocity blocking for the chosen kernel: blocks of whole
        // lines, from the default count to four times it, splitting the lines
        // evenly; each candidate timed as Q' solve + stage (more blocks fill
        // the GPU's last wave of CTAs better and cost the Q' solve more
        // partial sums)
        const int n0 = ctx->n_vblk;
        std::vector<int> nb{n0};
        for (int n = n0 + 1; n <= std::min(ctx->n_vblk_cap, 4 * n0); ++n)
            if (ctx->lines % n == 0) nb.push_back(n);
        double best_nb = 1e300;
        int pick_nb = n0;
        const StageArgs<float> sp = stage_args<float>(ctx, ctx->f[0], ctx->f[0], ctx->f[2], 0.75, 0.25, 0.25 * dt, true);
        for (int n : nb) {
            set_blocking(ctx, n);
            if ((st = run_moments(ctx, ctx->f[0]))) break;
            StageArgs<float> sn = sp;
            sn.Kblk = ctx->Kblk;
            if ((st = run_qprime(ctx, ctx->part, ctx->n_vblk, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr))) break;
            err = launch_stage_f32(sn, ctx->C, ctx->n_vblk, pick.v, pick.d, ctx->stream);       // warm-up
            if (err == cudaSuccess) err = cudaEventRecord(ea, ctx->stream);
            for (int r = 0; r < reps && err == cudaSuccess && !st; ++r) {
                st = run_qprime(ctx, ctx->part, ctx->n_vblk, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr);
                if (!st) err = launch_stage_f32(sn, ctx->C, ctx->n_vblk, pick.v, pick.d, ctx->stream);
            }
            if (err == cudaSuccess && !st) err = cudaEventRecord(eb, ctx->stream);
            if (err == cudaSuccess && !st) err = cudaEventSynchronize(eb);
            float ms = 0.f;
            if (err == cudaSuccess && !st) err = cudaEventElapsedTime(&ms, ea, eb);
            if (err != cudaSuccess || st) break;
            if (ms / reps < best_nb) { best_nb = ms / reps; pick_nb = n; }
        }
        set_blocking(ctx, pick_nb);
        // then the ring depths of that kernel again, at the chosen blocking
        // (the first search timed them at the default one); stage time only
        if (!st && err == cudaSuccess && pick.v != BGK_STAGE_PLAIN) {
            StageArgs<float> sn = sp;
            sn.Kblk = ctx->Kblk;
            double best_d = 1e300;
            int pick_d = pick.d;
            for (int d : {2, 3, 4, 6, 8, 12, 16}) {
                if (!stage_f32_variant_supported(sn, ctx->C, pick.v, d)) continue;
                err = launch_stage_f32(sn, ctx->C, ctx->n_vblk, pick.v, d, ctx->stream);      // warm-up
                if (err == cudaSuccess) err = cudaEventRecord(ea, ctx->stream);
                for (int r = 0; r < reps && err == cudaSuccess; ++r)
                    err = launch_stage_f32(sn, ctx->C, ctx->n_vblk, pick.v, d, ctx->stream);
                if (err == cudaSuccess) err = cudaEventRecord(eb, ctx->stream);
                if (err == cudaSuccess) err = cudaEventSynchronize(eb);
                float ms = 0.f;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ea, eb);
                if (err != cudaSuccess) break;
                if (ms / reps < best_d) { best_d = ms / reps; pick_d = d; }
            }
            if (err == cudaSuccess) {
                pick.d = pick_d;
                best = best_d;
            }
        }
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (st) return st;
    CU(err);
    if ((st = check_device_status(ctx))) return st;
    ctx->stage_variant = pick.v;
    ctx->stage_depth = pick.d;
    if (variant_out) *variant_out = pick.v;
    if (depth_out) *depth_out = pick.d;
    if (ms_out) *ms_out = best;
    return BGK_OK;
}

bgk_status bgk_set_graphs(bgk_ctx *ctx, int enable) {
    if (!ctx) return BGK_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    if (!enable) drop_graphs(ctx);
    ctx->graphs_on = enable != 0;
    return BGK_OK;
}

bgk_status bgk_set_newton(bgk_ctx *ctx, double tol, int max_iter) {
    if (!ctx || !(tol > 0.0) || max_iter < 0) return BGK_EINVAL;
    ctx->tol = tol;
    ctx->max_iter = max_iter;
    return BGK_OK;
}

bgk_status bgk_step(bgk_ctx *ctx, double dt, int n_steps) {
    if (!ctx || !(dt > 0.0) || n_steps < 0) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "a velocity shard steps through bgk_shard_partials and bgk_shard_stage");
    bgk_status st;
    if (ctx->pipe.active && (st = bgk_step_host_sync(ctx))) return st;
    if (!ctx->part_valid) {
        if ((st = run_moments(ctx, ctx->f[0]))) return st;
        ctx->part_valid = true;
    }
    const bool graphs = ctx->graphs_on && !ctx->prof_on;
    for (int n = 0; n < n_steps; ++n) {
        void *f0 = ctx->f[0], *f1 = ctx->f[1];
        if (graphs) {
            if ((st = replay_step(ctx, dt))) return st;
        } else if ((st = enqueue_step(ctx, dt))) {
            return st;
        }
        ctx->f[0] = f1;
        ctx->f[1] = f0;
    }
    return check_device_status(ctx);
}

namespace {
// index of a state buffer among the pipeline's
int pipe_index(const bgk_ctx::HostPipe &hp, const void *b) {
    for (int i = 0; i < 5; ++i)
        if (hp.buf[i] && hp.buf[i] == b) return i;
    return -1;
}
}  // namespace

bgk_status bgk_step_host(bgk_ctx *ctx, const void *f_in, void *f_out, double dt, int n_steps) {
    if (!ctx || !f_in || !f_out || !(dt > 0.0) || n_steps < 1) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "a velocity shard steps through bgk_shard_partials and bgk_shard_stage");
    bgk_ctx::HostPipe &hp = ctx->pipe;
    const size_t bytes = (size_t)ctx->C * ctx->Nu * ctx->P * ctx->elem;
    if (!hp.active) {
        // set up: one or two more state buffers (two when the device has room:
        // then an input copy never waits for the output copy of the call before
        // last), the copy streams and events; the current state buffer counts
        // as the last result (no copy pending)
        if (hp.n_extra == 0) {
            size_t free_b = 0, total_b = 0;
            CU(cudaMemGetInfo(&free_b, &total_b));
            CU(cudaMalloc(&hp.extra[0], bytes));
            hp.n_extra = 1;
            if (free_b > 2 * bytes + ((size_t)8 << 30)) {
                if (cudaMalloc(&hp.extra[1], bytes) == cudaSuccess) hp.n_extra = 2;
                else { hp.extra[1] = nullptr; cudaGetLastError(); }
            }
        }
        if (!hp.s_in) CU(cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking));
        if (!hp.s_out) CU(cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking));
        if (!hp.ev_in) CU(cudaEventCreateWithFlags(&hp.ev_in, cudaEventDisableTiming));
        if (!hp.ev_comp) CU(cudaEventCreateWithFlags(&hp.ev_comp, cudaEventDisableTiming));
        for (int i = 0; i < 5; ++i)
            if (!hp.ev_out[i]) CU(cudaEventCreateWithFlags(&hp.ev_out[i], cudaEventDisableTiming));
        hp.buf[0] = ctx->f[0]; hp.buf[1] = ctx->f[1]; hp.buf[2] = ctx->f[2];
        hp.buf[3] = hp.extra[0]; hp.buf[4] = hp.extra[1];
        for (int i = 0; i < 5; ++i) hp.out_pending[i] = false;
        hp.older[0] = hp.extra[0];
        hp.older[1] = hp.extra[1];
        // the state buffer joins the queue of results: its next input copy
        // waits for whatever the context's stream still has in flight
        CU(cudaEventRecord(hp.ev_comp, ctx->stream));
        CU(cudaStreamWaitEvent(hp.s_in, hp.ev_comp, 0));
        hp.active = true;
    }
    // this call's input buffer: the oldest earlier result, once its
    // device-to-host copy (if any) has finished
    void *in = hp.older[0];
    const int ii = pipe_index(hp, in);
    if (ii < 0) return fail(ctx, BGK_ECUDA, "host pipeline lost track of its buffers");
    if (hp.out_pending[ii]) CU(cudaStreamWaitEvent(hp.s_in, hp.ev_out[ii], 0));
    CU(cudaMemcpyAsync(in, f_in, bytes, cudaMemcpyHostToDevice, hp.s_in));
    CU(cudaEventRecord(hp.ev_in, hp.s_in));
    // compute on the context's stream: the new input, the last call's free
    // buffer as the first stage buffer, the second stage buffer unchanged
    void *last_res = ctx->f[0];
    CU(cudaStreamWaitEvent(ctx->stream, hp.ev_in, 0));
    ctx->f[0] = in;
    ctx->part_valid = false;
    bgk_status st;
    if ((st = run_moments(ctx, ctx->f[0]))) return st;
    ctx->part_valid = true;
    for (int n = 0; n < n_steps; ++n) {
        void *f0 = ctx->f[0], *f1 = ctx->f[1];
        if ((st = enqueue_step(ctx, dt))) return st;
        ctx->f[0] = f1;
        ctx->f[1] = f0;
    }
    CU(cudaEventRecord(hp.ev_comp, ctx->stream));
    // the result's device-to-host copy after the compute, on its own stream
    const int ri = pipe_index(hp, ctx->f[0]);
    if (ri < 0) return fail(ctx, BGK_ECUDA, "host pipeline lost track of its buffers");
    CU(cudaStreamWaitEvent(hp.s_out, hp.ev_comp, 0));
    CU(cudaMemcpyAsync(f_out, ctx->f[0], bytes, cudaMemcpyDeviceToHost, hp.s_out));
    CU(cudaEventRecord(hp.ev_out[ri], hp.s_out));
    hp.out_pending[ri] = true;
    // the queue of earlier results: drop the one just used as input, append the last
    if (hp.n_extra == 2) {
        hp.older[0] = hp.older[1];
        hp.older[1] = last_res;
    } else {
        hp.older[0] = last_res;
    }
    return BGK_OK;
}

bgk_status bgk_step_host_sync(bgk_ctx *ctx) {
    if (!ctx) return BGK_EINVAL;
    bgk_ctx::HostPipe &hp = ctx->pipe;
    if (hp.s_in) CU(cudaStreamSynchronize(hp.s_in));
    CU(cudaStreamSynchronize(ctx->stream));
    if (hp.s_out) CU(cudaStreamSynchronize(hp.s_out));
    for (int i = 0; i < 5; ++i) hp.out_pending[i] = false;
    return check_device_status(ctx);
}

bgk_status bgk_stage(bgk_ctx *ctx, const void *f_n, const void *f_in, void *f_out, double a,
                     double b, double c) {
    if (!ctx || !f_in || !f_out || f_in == f_out) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "a velocity shard needs the summed moments: use bgk_shard_stage");
    if (a != 0.0 && !f_n) return BGK_EINVAL;
    bgk_status st;
    if ((st = run_moments(ctx, f_in))) return st;
    if ((st = stage_from_partials(ctx, f_n, f_in, f_out, a, b, c, false))) return st;
    ctx->part_valid = false;
    return check_device_status(ctx);
}

bgk_status bgk_rhs(bgk_ctx *ctx, const void *f_in, void *r_out, int on_device) {
    if (!ctx || !f_in || !r_out) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "a velocity shard needs the summed moments: use bgk_shard_stage");
    const size_t bytes = (size_t)ctx->C * ctx->Nu * ctx->P * ctx->elem;
    CU(cudaMemcpyAsync(ctx->f[1], f_in, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       ctx->stream));
    bgk_status st;
    if ((st = run_moments(ctx, ctx->f[1]))) return st;
    if ((st = stage_from_partials(ctx, nullptr, ctx->f[1], ctx->f[2], 0.0, 0.0, 1.0, false))) return st;
    ctx->part_valid = false;
    CU(cudaMemcpyAsync(r_out, ctx->f[2], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return check_device_status(ctx);
}

bgk_status bgk_shard_partials(bgk_ctx *ctx, double *m) {
    if (!ctx || !m) return BGK_EINVAL;
    bgk_status st;
    if (!ctx->part_valid) {
        if ((st = run_moments(ctx, ctx->f[0]))) return st;
        ctx->part_valid = true;
    }
    LaunchScope ls(ctx, BGK_K_OTHER);
    CU(launch_sum_partials(ctx->part, ctx->n_vblk, ctx->P, m, ctx->stream));
    return BGK_OK;
}

bgk_status bgk_shard_stage(bgk_ctx *ctx, const double *m, int stage, double dt) {
    if (!ctx || !m || stage < 0 || stage > 2 || !(dt > 0.0)) return BGK_EINVAL;
    if (!ctx->part_valid) return fail(ctx, BGK_EINVAL, "no partial moments of the stage input: call bgk_shard_partials first");
    void *f0 = ctx->f[0], *f1 = ctx->f[1], *f2 = ctx->f[2];
    bgk_status st = run_qprime(ctx, m, 1, ctx->P, ctx->eq, ctx->qp, nullptr, nullptr);
    if (st) return st;
    if (stage == 0) st = run_stage(ctx, nullptr, f0, f1, 0.0, 1.0, dt, true);
    else if (stage == 1) st = run_stage(ctx, f0, f1, f2, 0.75, 0.25, 0.25 * dt, true);
    else st = run_stage(ctx, f0, f2, f1, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt, true);
    if (st) return st;
    if (stage == 2) {
        ctx->f[0] = f1;
        ctx->f[1] = f0;
    }
    ctx->part_valid = true;           // the epilogue wrote the partials of the next stage's input
    return check_device_status(ctx);
}

bgk_status bgk_moments(bgk_ctx *ctx, double *m, int on_device) {
    if (!ctx || !m) return BGK_EINVAL;
    bgk_status st;
    if (!ctx->part_valid) {
        if ((st = run_moments(ctx, ctx->f[0], true))) return st;
        ctx->part_valid = true;
    }
    {
        LaunchScope ls(ctx, BGK_K_OTHER);
        CU(launch_reduce_moments(ctx->part, ctx->n_vblk, ctx->P, ctx->mom, ctx->stream));
    }
    CU(cudaMemcpyAsync(m, ctx->mom, (size_t)ctx->P * BGK_NMOM * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_macro(bgk_ctx *ctx, double *out, int on_device) {
    if (!ctx || !out) return BGK_EINVAL;
    if (ctx->shard) return fail(ctx, BGK_ENOTSUP, "macroscopic diagnostics need every velocity (not a shard)");
    bgk_status st;
    if (!ctx->part_valid) {
        if ((st = run_moments(ctx, ctx->f[0], true))) return st;
        ctx->part_valid = true;
    }
    const size_t bytes = (size_t)ctx->P * BGK_NMACRO * sizeof(double);
    double *dst = out;
    if (!on_device) CU(cudaMallocAsync((void **)&dst, bytes, ctx->stream));
    double face_rho[6];
    for (int f = 0; f < 6; ++f) face_rho[f] = ctx->bc[f][0];
    {
        LaunchScope ls(ctx, BGK_K_OTHER);
        CU(launch_reduce_moments(ctx->part, ctx->n_vblk, ctx->P, ctx->mom, ctx->stream));
        CU(launch_macro(ctx->mom, dst, ctx->P, ctx->mesh, ctx->fr, ctx->gas, face_rho, ctx->curved ? ctx->geo : nullptr,
                        ctx->stream));
    }
    if (!on_device) {
        CU(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaFreeAsync(dst, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_qprime(bgk_ctx *ctx, const double *m, int n_points, double *qp, int *iters,
                      int on_device) {
    if (!ctx || !m || !qp || n_points <= 0) return BGK_EINVAL;
    // moments laid out [P][NMOM] by the caller; the kernel reads [vb][NMOM][P]
    double *dm = nullptr, *dq = nullptr;
    int *di = nullptr;
    const size_t n = (size_t)n_points;
    CU(cudaMallocAsync((void **)&dm, n * BGK_NMOM * sizeof(double), ctx->stream));
    CU(cudaMallocAsync((void **)&dq, n * 5 * sizeof(double), ctx->stream));
    CU(cudaMallocAsync((void **)&di, n * sizeof(int), ctx->stream));
    std::vector<double> hm(n * BGK_NMOM), ht(n * BGK_NMOM);
    CU(cudaMemcpyAsync(hm.data(), m, hm.size() * sizeof(double),
                       on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (size_t p = 0; p < n; ++p)
        for (int j = 0; j < BGK_NMOM; ++j) ht[(size_t)j * n + p] = hm[p * BGK_NMOM + j];
    CU(cudaMemcpyAsync(dm, ht.data(), ht.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    bgk_status st = run_qprime(ctx, dm, 1, n_points, nullptr, dq, di, nullptr);
    if (st) return st;
    CU(cudaMemcpyAsync(qp, dq, n * 5 * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (iters)
        CU(cudaMemcpyAsync(iters, di, n * sizeof(int),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaFreeAsync(dm, ctx->stream));
    CU(cudaFreeAsync(dq, ctx->stream));
    CU(cudaFreeAsync(di, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return check_device_status(ctx);
}

bgk_status bgk_totals(bgk_ctx *ctx, double totals[5], double *entropy) {
    if (!ctx || !totals) return BGK_EINVAL;
    std::vector<double> m((size_t)ctx->P * BGK_NMOM);
    bgk_status st = bgk_moments(ctx, m.data(), 0);
    if (st) return st;
    std::vector<double> hp;
    unsigned int nonpos = 0;
    if (entropy) {
        // per-point sum_k w_k F ln F in FP64 (a velocity-block partial, then
        // the sum over blocks), weighed below with the totals' quadrature
        double *dpart = nullptr, *dh = nullptr;
        unsigned int *dbad = nullptr;
        CU(cudaMallocAsync((void **)&dpart, (size_t)ctx->n_vblk * ctx->P * sizeof(double), ctx->stream));
        CU(cudaMallocAsync((void **)&dh, (size_t)ctx->P * sizeof(double), ctx->stream));
        CU(cudaMallocAsync((void **)&dbad, sizeof(unsigned int), ctx->stream));
        CU(cudaMemsetAsync(dbad, 0, sizeof(unsigned int), ctx->stream));
        {
            LaunchScope ls(ctx, BGK_K_OTHER);
            if (ctx->precision == BGK_FP64)
                CU(launch_entropy<double>((const double *)ctx->f[0], ctx->vtab, ctx->Nu, ctx->P, ctx->Kblk,
                                          ctx->n_vblk, dpart, dh, dbad, ctx->stream));
            else
                CU(launch_entropy<float>((const float *)ctx->f[0], ctx->vtab, ctx->Nu, ctx->P, ctx->Kblk,
                                         ctx->n_vblk, dpart, dh, dbad, ctx->stream));
        }
        hp.resize(ctx->P);
        CU(cudaMemcpyAsync(hp.data(), dh, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(&nonpos, dbad, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaFreeAsync(dpart, ctx->stream));
        CU(cudaFreeAsync(dh, ctx->stream));
        CU(cudaFreeAsync(dbad, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
    }
    const int q = ctx->q;
    double t[5] = {0, 0, 0, 0, 0}, H = 0.0;
    for (int p = 0; p < ctx->P; ++p) {
        const int s = p % ctx->Ns;
        const double W = ctx->curved ? ctx->geo_h[(size_t)p * BGK_NGEO + 10]
                                     : ctx->fr.wq[s % q] * ctx->fr.wq[(s / q) % q] * ctx->fr.wq[s / (q * q)] * ctx->jac;
        const double *mm = &m[(size_t)p * BGK_NMOM];
        t[0] += W * mm[0]; t[1] += W * mm[1]; t[2] += W * mm[2]; t[3] += W * mm[3];
        t[4] += W * (0.5 * (mm[4] + mm[5] + mm[6]) + mm[10]);
        if (entropy) H += W * hp[p];
    }
    for (int j = 0; j < 5; ++j) totals[j] = t[j];
    if (entropy) *entropy = nonpos ? std::numeric_limits<double>::quiet_NaN() : H;
    return BGK_OK;
}

// ---- learned guess ---------------------------------------------------------
bgk_status bgk_set_guess(bgk_ctx *ctx, int mode, int bf16) {
    if (!ctx || mode < 0 || mode > 1) return BGK_EINVAL;
    if (mode == 1 && !ctx->mlp_ready) return fail(ctx, BGK_EINVAL, "no trained or loaded network");
    ctx->guess_mode = mode;
    ctx->mlp_bf16 = bf16 ? 1 : 0;
    return BGK_OK;
}

bgk_status bgk_mlp_log(bgk_ctx *ctx, int enable, long long max_pairs) {
    if (!ctx || (enable && max_pairs <= 0)) return BGK_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    if (enable) {
        if (max_pairs > ctx->log_max) {
            CU(cudaFree(ctx->log));
            ctx->log = nullptr;
            CU(cudaMalloc(&ctx->log, (size_t)max_pairs * MLP_LOG_STRIDE * sizeof(float)));
            ctx->log_max = max_pairs;
        }
        CU(cudaMemsetAsync(ctx->log_count, 0, sizeof(unsigned long long), ctx->stream));
    }
    ctx->log_on = enable != 0;
    return BGK_OK;
}

static bgk_status log_count(bgk_ctx *ctx, long long *n) {
    unsigned long long c = 0;
    CU(cudaMemcpyAsync(&c, ctx->log_count, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n = std::min((long long)c, ctx->log_max);
    return BGK_OK;
}

bgk_status bgk_mlp_log_read(bgk_ctx *ctx, float *out, long long max_pairs, long long *n_out) {
    if (!ctx || !out || !n_out || max_pairs < 0) return BGK_EINVAL;
    long long n;
    bgk_status st = log_count(ctx, &n);
    if (st) return st;
    n = std::min(n, max_pairs);
    if (n > 0)
        CU(cudaMemcpyAsync(out, ctx->log, (size_t)n * MLP_LOG_STRIDE * sizeof(float), cudaMemcpyDeviceToHost,
                           ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *n_out = n;
    return BGK_OK;
}

bgk_status bgk_mlp_weights(bgk_ctx *ctx, float *buf, int load) {
    if (!ctx || !buf) return BGK_EINVAL;
    if (load) {
        CU(cudaMemcpyAsync(ctx->mlp_w, buf, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->mlp_norm, buf + MLP_NPARAM, MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice,
                           ctx->stream));
        CU(launch_mlp_round(ctx->mlp_w, ctx->mlp_w16, MLP_NPARAM, ctx->stream));
        ctx->mlp_ready = true;
    } else {
        if (!ctx->mlp_ready) return fail(ctx, BGK_EINVAL, "no trained or loaded network");
        CU(cudaMemcpyAsync(buf, ctx->mlp_w, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(buf + MLP_NPARAM, ctx->mlp_norm, MLP_NNORM * sizeof(float), cudaMemcpyDeviceToHost,
                           ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

// Upload x[n][9], t[n][5] (host) and run the training kernel over all n samples.
static bgk_status mlp_batch_pass(bgk_ctx *ctx, const float *dx, const float *dt, const int *didx, int n,
                                 int bf16) {
    MlpParams p{ctx->mlp_w, ctx->mlp_norm, nullptr};   // training rounds the master weights itself
    LaunchScope ls(ctx, BGK_K_OTHER);
    CU(launch_mlp_train(p, dx, dt, didx, n, ctx->mlp_grad, ctx->mlp_loss, bf16, ctx->stream));
    return BGK_OK;
}

bgk_status bgk_mlp_grad(bgk_ctx *ctx, const float *x, const float *t, int n, int bf16, double *loss, float *grad) {
    if (!ctx || !x || !t || n <= 0 || !loss || !grad) return BGK_EINVAL;
    if (!ctx->mlp_ready) return fail(ctx, BGK_EINVAL, "no trained or loaded network");
    float *dx = nullptr, *dt = nullptr;
    int *didx = nullptr;
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    CU(cudaMallocAsync((void **)&dx, (size_t)n * MLP_IN * sizeof(float), ctx->stream));
    CU(cudaMallocAsync((void **)&dt, (size_t)n * MLP_OUT * sizeof(float), ctx->stream));
    CU(cudaMallocAsync((void **)&didx, (size_t)n * sizeof(int), ctx->stream));
    CU(cudaMemcpyAsync(dx, x, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(dt, t, (size_t)n * MLP_OUT * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(didx, idx.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_grad, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(double), ctx->stream));
    bgk_status st = mlp_batch_pass(ctx, dx, dt, didx, n, bf16);
    if (st) return st;
    CU(cudaMemcpyAsync(grad, ctx->mlp_grad, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(loss, ctx->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaFreeAsync(dx, ctx->stream));
    CU(cudaFreeAsync(dt, ctx->stream));
    CU(cudaFreeAsync(didx, ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_grad, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_mlp_infer(bgk_ctx *ctx, const float *x, long long n, float *delta, int on_device) {
    if (!ctx || !x || !delta || n <= 0 || n > (1ll << 31)) return BGK_EINVAL;
    if (!ctx->mlp_ready) return fail(ctx, BGK_EINVAL, "no trained or loaded network");
    const float *dx = x;
    float *dd = delta;
    if (!on_device) {
        float *bx = nullptr, *bd = nullptr;
        CU(cudaMallocAsync((void **)&bx, (size_t)n * MLP_IN * sizeof(float), ctx->stream));
        CU(cudaMallocAsync((void **)&bd, (size_t)n * MLP_OUT * sizeof(float), ctx->stream));
        CU(cudaMemcpyAsync(bx, x, (size_t)n * MLP_IN * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
        dx = bx;
        dd = bd;
    }
    MlpParams mp;
    mp.w = ctx->mlp_w; mp.norm = ctx->mlp_norm; mp.w16 = ctx->mlp_w16;
    {
        LaunchScope ls(ctx, BGK_K_OTHER);
        CU(launch_mlp_infer_tc(mp, dx, n, dd, ctx->status, ctx->stream));
    }
    if (!on_device) {
        CU(cudaMemcpyAsync(delta, dd, (size_t)n * MLP_OUT * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaFreeAsync((void *)dx, ctx->stream));
        CU(cudaFreeAsync(dd, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return check_device_status(ctx);
}

bgk_status bgk_mlp_train(bgk_ctx *ctx, int epochs, int batch, float lr, unsigned long long seed, int bf16,
                         double *final_loss) {
    if (!ctx || epochs <= 0 || batch <= 0 || !(lr > 0.f)) return BGK_EINVAL;
    long long n;
    bgk_status st = log_count(ctx, &n);
    if (st) return st;
    if (n < batch) return fail(ctx, BGK_EINVAL, "only %lld logged pairs for batch %d", n, batch);
    if (n > (1ll << 30)) n = 1ll << 30;
    // pairs to host: normalisation statistics and the split into x and t
    std::vector<float> pairs((size_t)n * MLP_LOG_STRIDE);
    CU(cudaMemcpyAsync(pairs.data(), ctx->log, pairs.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    std::vector<double> mean(MLP_LOG_STRIDE, 0.0), var(MLP_LOG_STRIDE, 0.0);
    for (long long i = 0; i < n; ++i)
        for (int j = 0; j < MLP_LOG_STRIDE; ++j) mean[j] += pairs[(size_t)i * MLP_LOG_STRIDE + j];
    for (int j = 0; j < MLP_LOG_STRIDE; ++j) mean[j] /= (double)n;
    for (long long i = 0; i < n; ++i)
        for (int j = 0; j < MLP_LOG_STRIDE; ++j) {
            const double d = pairs[(size_t)i * MLP_LOG_STRIDE + j] - mean[j];
            var[j] += d * d;
        }
    std::vector<float> norm(MLP_NNORM), hx((size_t)n * MLP_IN), ht((size_t)n * MLP_OUT);
    // Standard deviations get floors so that components that are constant up
    // to round-off (e.g. a velocity component that is zero in the whole flow)
    // are not blown up into unit-variance noise: 1e-6 of the feature's scale,
    // 1e-7 absolute for the (dimensionless) targets.
    for (int j = 0; j < MLP_LOG_STRIDE; ++j) {
        double sd = std::sqrt(var[j] / (double)n);
        const double floor = j < MLP_IN ? 1e-6 * std::max(std::fabs(mean[j]), 1.0) : 1e-7;
        if (!(sd > floor)) sd = floor;
        if (j < MLP_IN) { norm[j] = (float)mean[j]; norm[MLP_IN + j] = (float)sd; }
        else { norm[2 * MLP_IN + (j - MLP_IN)] = (float)mean[j]; norm[2 * MLP_IN + MLP_OUT + (j - MLP_IN)] = (float)sd; }
    }
    for (long long i = 0; i < n; ++i) {
        for (int j = 0; j < MLP_IN; ++j) hx[(size_t)i * MLP_IN + j] = pairs[(size_t)i * MLP_LOG_STRIDE + j];
        for (int j = 0; j < MLP_OUT; ++j) ht[(size_t)i * MLP_OUT + j] = pairs[(size_t)i * MLP_LOG_STRIDE + MLP_IN + j];
    }
    // He-normal initialisation, zero biases
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<float> w(MLP_NPARAM, 0.f);
    const int fan[3][2] = {{MLP_IN, MLP_H}, {MLP_H, MLP_H}, {MLP_H, MLP_OUT}};
    size_t off = 0;
    for (int l = 0; l < 3; ++l) {
        const double sc = std::sqrt(2.0 / fan[l][0]);
        for (int i = 0; i < fan[l][0] * fan[l][1]; ++i) w[off + i] = (float)(nd(rng) * sc);
        off += (size_t)fan[l][0] * fan[l][1] + fan[l][1];
    }
    float *dx = nullptr, *dt = nullptr;
    int *didx = nullptr;
    CU(cudaMalloc(&dx, hx.size() * sizeof(float)));
    CU(cudaMalloc(&dt, ht.size() * sizeof(float)));
    CU(cudaMalloc(&didx, (size_t)n * sizeof(int)));
    CU(cudaMemcpyAsync(dx, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(dt, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->mlp_w, w.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->mlp_norm, norm.data(), MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_m, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_v, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    CU(cudaMemsetAsync(ctx->mlp_grad, 0, MLP_NPARAM * sizeof(float), ctx->stream));
    ctx->mlp_ready = true;
    std::vector<int> perm((size_t)n);
    for (long long i = 0; i < n; ++i) perm[i] = (int)i;
    const long long nbatch = n / batch;
    const long long total = (long long)epochs * nbatch;
    long long step = 0;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        CU(cudaMemcpyAsync(didx, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(double), ctx->stream));
        for (long long b = 0; b < nbatch; ++b) {
            st = mlp_batch_pass(ctx, dx, dt, didx + b * batch, batch, bf16);
            if (st) break;
            ++step;
            const double frac = (double)(step - 1) / (double)std::max(1ll, total - 1);
            const float lr_t = (float)(lr * (0.1 + 0.45 * (1.0 + std::cos(M_PI * frac))));
            LaunchScope ls(ctx, BGK_K_OTHER);
            cudaError_t e = launch_mlp_adam(ctx->mlp_w, ctx->mlp_m, ctx->mlp_v, ctx->mlp_grad, MLP_NPARAM, lr_t,
                                            0.9f, 0.999f, 1e-8f, (int)step, ctx->stream);
            if (e != cudaSuccess) { st = fail(ctx, BGK_ECUDA, "adam: %s", cudaGetErrorString(e)); break; }
        }
        if (st) break;
        double ls_sum = 0.0;
        cudaMemcpyAsync(&ls_sum, ctx->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        last = ls_sum / (double)nbatch;
    }
    if (!st) {
        const cudaError_t e = launch_mlp_round(ctx->mlp_w, ctx->mlp_w16, MLP_NPARAM, ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, BGK_ECUDA, "mlp round: %s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(dx);
    cudaFree(dt);
    cudaFree(didx);
    if (st) return st;
    if (final_loss) *final_loss = last;
    return BGK_OK;
}

bgk_status bgk_mlp_stats(bgk_ctx *ctx, unsigned long long *fallbacks) {
    if (!ctx || !fallbacks) return BGK_EINVAL;
    CU(cudaMemcpyAsync(fallbacks, ctx->fallbacks, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemsetAsync(ctx->fallbacks, 0, sizeof(unsigned long long), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return BGK_OK;
}

bgk_status bgk_profile(bgk_ctx *ctx, int enable) {
    if (!ctx) return BGK_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    for (auto &r : ctx->prof_pending) { ctx->ev_pool.push_back(r.a); ctx->ev_pool.push_back(r.b); }
    ctx->prof_pending.clear();
    for (int k = 0; k < BGK_NKINDS; ++k) { ctx->prof_ms[k] = 0.0; ctx->launches[k] = 0; }
    ctx->prof_on = enable != 0;
    return BGK_OK;
}

bgk_status bgk_profile_read(bgk_ctx *ctx, double ms[BGK_NKINDS], long long launches[BGK_NKINDS]) {
    if (!ctx) return BGK_EINVAL;
    CU(cudaStreamSynchronize(ctx->stream));
    for (auto &r : ctx->prof_pending) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, r.a, r.b));
        ctx->prof_ms[r.kind] += t;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    for (int k = 0; k < BGK_NKINDS; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->launches[k];
    }
    return BGK_OK;
}

bgk_status bgk_stats(bgk_ctx *ctx, double *mean_iters, int *max_iters, double *max_residual) {
    if (!ctx) return BGK_EINVAL;
    NewtonStats s;
    CU(cudaMemcpyAsync(&s, ctx->stats, sizeof s, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemsetAsync(ctx->stats, 0, sizeof(NewtonStats), ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (mean_iters) *mean_iters = s.solves ? (double)s.iter_sum / (double)s.solves : 0.0;
    if (max_iters) *max_iters = s.iter_max;
    if (max_residual) {
        double r;
        long long bits = (long long)s.res_max_bits;
        std::memcpy(&r, &bits, sizeof r);
        *max_residual = r;
    }
    return BGK_OK;
}

}  // extern "C"
