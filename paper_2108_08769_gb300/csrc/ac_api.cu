// ac_api.cu -- host side of the C ABI declared in include/ac.h: validation,
// device memory, the captured pseudo-iteration loop, state transfer.
//
// Control flow of one physical step (Alg. 1):
//   begin_step_kernel            Q^n <- Q, control block reset
//   graph: WHILE (not done) {    one pseudo-iteration per body execution
//     [dtau_min_kernel]          global pseudo-time step option
//     stage_kernel  x s_max      fused stage sweeps (Eq. RK2)
//     end_iteration_kernel       norms, stopping test, buffer rotation,
//   }                            sets the WHILE condition on the device
//   one 160-byte device->host read of the control block.
// The loop therefore runs without any host round trip; the host waits once
// per physical step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdarg>
#include <algorithm>
#include <string>

#include "../../include/ac.h"
#include "ac_kernels.cuh"

using namespace acgb;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                        __LINE__);                                                          \
    } while (0)

constexpr int kTX = 32, kTY = 8;
constexpr int kEndThreads = 256;

bool valid_bc(int b) { return b >= AC_BC_WALL_SLIP && b <= AC_BC_PERIODIC; }

}  // namespace

struct ac_ctx {
    ac_grid grid;
    ac_fluids fluids;
    bool has_fluids;
    double beta;
    ac_bc bc;
    ac_options opt;
    int device;
    size_t N;
    // device memory (FP64 form)
    double *buf[3][4];
    double *lev[4];
    double *partials;
    Ctl *ctl;
    Ctl *hctl;            // pinned host mirror
    dim3 grid_dim;
    int nblocks;
    cudaStream_t stream;  // user stream (0 = default)
    cudaStream_t cap;     // private stream used for capture
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool has_state;
    int cur_host;
    long long launches;
    int last_iters;
    bool profiling;
    cudaEvent_t ev[5];
    double stage_ms;
    long long stage_launches;
};

namespace {

SweepArgs<double> make_args(const ac_ctx *c, int stage) {
    SweepArgs<double> a;
    memset(&a, 0, sizeof a);
    a.nx = c->grid.nx;
    a.ny = c->grid.ny;
    a.bc[0] = c->bc.xlo; a.bc[1] = c->bc.xhi; a.bc[2] = c->bc.ylo; a.bc[3] = c->bc.yhi;
    a.gradp = c->opt.gradp;
    a.limiter_k = c->opt.limiter_k;
    a.realtime = c->opt.realtime;
    a.local_dtau = c->opt.local_dtau;
    a.alpha_pi_p_row = c->opt.alpha_pi_p_row;
    a.stage = stage;
    a.s_max = c->opt.rk_stages;
    a.alpha = stage > 0 ? 1.0 / double(c->opt.rk_stages - stage + 1) : 0.0;
    const double dx = c->grid.lx / c->grid.nx, dy = c->grid.ly / c->grid.ny;
    a.dx = dx; a.dy = dy;
    a.half_dx = 0.5 * dx; a.half_dy = 0.5 * dy;
    a.inv_dx = 1.0 / dx; a.inv_dy = 1.0 / dy;
    a.dx_over_dy = dx / dy; a.dy_over_dx = dy / dx;
    a.beta = c->beta; a.inv_beta = 1.0 / c->beta;
    a.gx = c->grid.gx; a.gy = c->grid.gy;
    a.cfl_area = c->opt.cfl_tau * dx * dy;
    for (int b = 0; b < 3; ++b)
        for (int f = 0; f < 4; ++f) a.buf[b][f] = c->buf[b][f];
    for (int f = 0; f < 4; ++f) a.lev[f] = c->lev[f];
    a.partials = c->partials;
    a.ctl = c->ctl;
    return a;
}

size_t stage_smem() { return sizeof(StageSmem<double, kTX, kTY>); }

// Enqueue one pseudo-iteration on stream s (with events around the stage
// sweeps when `timed`).
int enqueue_iteration(ac_ctx *c, cudaStream_t s, unsigned long long cond, int use_cond, bool timed = false) {
    if (!c->opt.local_dtau) {
        SweepArgs<double> a = make_args(c, 0);
        int blocks = (int)std::min<size_t>((c->N + 255) / 256, 152 * 8);
        dtau_min_kernel<double><<<blocks, 256, 0, s>>>(a);
        CK(cudaGetLastError());
    }
    if (timed) CK(cudaEventRecord(c->ev[0], s));
    for (int st = 1; st <= c->opt.rk_stages; ++st) {
        SweepArgs<double> a = make_args(c, st);
        stage_kernel<double, kTX, kTY><<<c->grid_dim, kTX * kTY, stage_smem(), s>>>(a);
        CK(cudaGetLastError());
        if (timed) CK(cudaEventRecord(c->ev[st], s));
    }
    end_iteration_kernel<kEndThreads><<<1, kEndThreads, 0, s>>>(
        c->ctl, c->partials, c->nblocks, 1.0 / double(c->N), c->opt.rk_stages, cond, use_cond);
    CK(cudaGetLastError());
    return AC_OK;
}

int kernels_per_iteration(const ac_ctx *c) { return c->opt.rk_stages + 1 + (c->opt.local_dtau ? 0 : 1); }

int build_graph(ac_ctx *c) {
    if (c->exec) return AC_OK;
    CK(cudaGraphCreate(&c->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
    // (the params union has no usable default constructor: zero raw storage)
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(c, c->cap, (unsigned long long)h, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap, &captured);
    if (rc != AC_OK) return rc;
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
    return AC_OK;
}

int check_host_field(const double *a, size_t n, bool positive, const char *name) {
    if (!a) return fail(AC_ERR_ARG, "%s is NULL", name);
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(a[k])) return fail(AC_ERR_NONFINITE, "%s[%zu] is not finite", name, k);
        if (positive && !(a[k] > 0.0)) return fail(AC_ERR_ARG, "%s[%zu] = %g is not > 0", name, k, a[k]);
    }
    return AC_OK;
}

bool use_host_loop() {
    const char *e = getenv("AC_LAUNCH");
    return e && strcmp(e, "host") == 0;
}

}  // namespace

extern "C" {

int ac_default_options(ac_options *o) {
    if (!o) return fail(AC_ERR_ARG, "options pointer is NULL");
    memset(o, 0, sizeof *o);
    o->rk_stages = 3;
    o->riemann = AC_RIEMANN_OSHER;
    o->gradp = AC_GRADP_NEW;
    o->limiter_k = 1;
    o->local_dtau = 1;
    o->realtime = 1;
    o->alpha_pi_p_row = 1;
    o->precision = AC_PREC_FP64;
    o->cfl_tau = 0.45;
    return AC_OK;
}

double ac_beta_from_speed(double c0, double rho_ref) { return rho_ref * c0 * c0; }

const char *ac_last_error(void) { return g_err.c_str(); }

int ac_create(const ac_grid *grid, const ac_fluids *fluids, double beta, const ac_bc *bc,
              const ac_options *opt, ac_ctx **out) {
    g_err.clear();
    if (!out) return fail(AC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !bc) return fail(AC_ERR_ARG, "grid and bc must not be NULL");
    if (grid->nx < 1 || grid->ny < 1) return fail(AC_ERR_ARG, "nx, ny must be >= 1 (got %d, %d)", grid->nx, grid->ny);
    if ((long long)grid->nx * grid->ny > (1LL << 31))
        return fail(AC_ERR_ARG, "nx*ny = %lld exceeds 2^31 cells", (long long)grid->nx * grid->ny);
    if (!(grid->lx > 0.0) || !(grid->ly > 0.0) || !std::isfinite(grid->lx) || !std::isfinite(grid->ly))
        return fail(AC_ERR_ARG, "lx, ly must be finite and > 0");
    if (!std::isfinite(grid->gx) || !std::isfinite(grid->gy)) return fail(AC_ERR_ARG, "gravity must be finite");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(AC_ERR_ARG, "beta must be finite and > 0 (got %g)", beta);
    const int sides[4] = {bc->xlo, bc->xhi, bc->ylo, bc->yhi};
    for (int k = 0; k < 4; ++k)
        if (!valid_bc(sides[k])) return fail(AC_ERR_ARG, "boundary kind %d on side %d is unknown", sides[k], k);
    if ((bc->xlo == AC_BC_PERIODIC) != (bc->xhi == AC_BC_PERIODIC) ||
        (bc->ylo == AC_BC_PERIODIC) != (bc->yhi == AC_BC_PERIODIC))
        return fail(AC_ERR_ARG, "periodic boundaries must be set on both sides of an axis");
    if (fluids && (!(fluids->rho_light > 0.0) || !(fluids->rho_heavy >= fluids->rho_light)))
        return fail(AC_ERR_ARG, "fluids must satisfy 0 < rho_light <= rho_heavy");
    ac_options o;
    ac_default_options(&o);
    if (opt) o = *opt;
    if (o.rk_stages < 1 || o.rk_stages > 4) return fail(AC_ERR_ARG, "rk_stages must be 1..4");
    if (o.riemann != AC_RIEMANN_OSHER) return fail(AC_ERR_ARG, "riemann solver %d is not available", o.riemann);
    if (o.gradp < AC_GRADP_NEW || o.gradp > AC_GRADP_SUPERBEE) return fail(AC_ERR_ARG, "gradp %d is unknown", o.gradp);
    if (o.limiter_k != 1 && o.limiter_k != 2) return fail(AC_ERR_ARG, "limiter_k must be 1 or 2");
    if (o.precision != AC_PREC_FP64) return fail(AC_ERR_ARG, "precision %d is not available", o.precision);
    if (!(o.cfl_tau > 0.0) || !std::isfinite(o.cfl_tau)) return fail(AC_ERR_ARG, "cfl_tau must be > 0");
    for (int k = 0; k < 4; ++k)
        if (!(o.abs_tol[k] >= 0.0)) return fail(AC_ERR_ARG, "abs_tol[%d] must be >= 0", k);
    o.local_dtau = o.local_dtau ? 1 : 0;
    o.realtime = o.realtime ? 1 : 0;
    o.alpha_pi_p_row = o.alpha_pi_p_row ? 1 : 0;

    ac_ctx *c = new ac_ctx();
    memset(c, 0, sizeof *c);
    c->grid = *grid;
    if (fluids) { c->fluids = *fluids; c->has_fluids = true; }
    c->beta = beta;
    c->bc = *bc;
    c->opt = o;
    c->N = (size_t)grid->nx * grid->ny;
    c->grid_dim = dim3((grid->nx + kTX - 1) / kTX, (grid->ny + kTY - 1) / kTY);
    c->nblocks = c->grid_dim.x * c->grid_dim.y;
    int rc = AC_OK;
    auto bail = [&](int code) { ac_destroy(c); return code; };
#define CKC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_)));                                      \
    } while (0)
    CKC(cudaGetDevice(&c->device));
    const size_t bytes = c->N * sizeof(double);
    for (int b = 0; b < 3; ++b)
        for (int f = 0; f < 4; ++f) CKC(cudaMalloc(&c->buf[b][f], bytes));
    for (int f = 0; f < 4; ++f) CKC(cudaMalloc(&c->lev[f], bytes));
    CKC(cudaMalloc(&c->partials, (size_t)c->nblocks * 4 * sizeof(double)));
    CKC(cudaMalloc(&c->ctl, sizeof(Ctl)));
    CKC(cudaMallocHost(&c->hctl, sizeof(Ctl)));
    CKC(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) CKC(cudaEventCreate(&c->ev[k]));
    CKC(cudaFuncSetAttribute(stage_kernel<double, kTX, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_smem()));
    memset(c->hctl, 0, sizeof(Ctl));
    for (int k = 0; k < 4; ++k) c->hctl->abs_tol[k] = o.abs_tol[k];
    c->hctl->done = 1;
    CKC(cudaMemcpy(c->ctl, c->hctl, sizeof(Ctl), cudaMemcpyHostToDevice));
#undef CKC
    (void)rc;
    *out = c;
    return AC_OK;
}

void ac_destroy(ac_ctx *c) {
    if (!c) return;
    for (int k = 0; k < 5; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (int b = 0; b < 3; ++b)
        for (int f = 0; f < 4; ++f) cudaFree(c->buf[b][f]);
    for (int f = 0; f < 4; ++f) cudaFree(c->lev[f]);
    cudaFree(c->partials);
    cudaFree(c->ctl);
    if (c->hctl) cudaFreeHost(c->hctl);
    delete c;
}

int ac_set_stream(ac_ctx *c, void *stream) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    c->stream = (cudaStream_t)stream;
    return AC_OK;
}

int ac_set_state(ac_ctx *c, const double *rho, const double *rhou, const double *rhov, const double *p) {
    g_err.clear();
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    int rc;
    if ((rc = check_host_field(rho, c->N, true, "rho")) != AC_OK) return rc;
    if ((rc = check_host_field(rhou, c->N, false, "rhou")) != AC_OK) return rc;
    if ((rc = check_host_field(rhov, c->N, false, "rhov")) != AC_OK) return rc;
    if ((rc = check_host_field(p, c->N, false, "p")) != AC_OK) return rc;
    if (c->has_fluids) {
        for (size_t k = 0; k < c->N; ++k)
            if (rho[k] < 0.5 * c->fluids.rho_light || rho[k] > 2.0 * c->fluids.rho_heavy)
                return fail(AC_ERR_ARG, "rho[%zu] = %g lies outside [rho_light/2, 2 rho_heavy]", k, rho[k]);
    }
    const double *src[4] = {rho, rhou, rhov, p};
    const size_t bytes = c->N * sizeof(double);
    CK(cudaStreamSynchronize(c->stream));
    for (int f = 0; f < 4; ++f) {
        CK(cudaMemcpyAsync(c->buf[0][f], src[f], bytes, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->lev[f], src[f], bytes, cudaMemcpyHostToDevice, c->stream));
    }
    c->hctl->cur = 0;
    c->hctl->done = 1;
    c->hctl->iter = 0;
    CK(cudaMemcpyAsync(c->ctl, c->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->cur_host = 0;
    c->has_state = true;
    return AC_OK;
}

int ac_get_state(const ac_ctx *c, double *rho, double *rhou, double *rhov, double *p) {
    g_err.clear();
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    double *dst[4] = {rho, rhou, rhov, p};
    const size_t bytes = c->N * sizeof(double);
    for (int f = 0; f < 4; ++f)
        if (dst[f]) CK(cudaMemcpyAsync(dst[f], c->buf[c->cur_host][f], bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AC_OK;
}

int ac_physical_step(ac_ctx *c, double dt, double tol, int max_iters, int *iters_out) {
    g_err.clear();
    if (iters_out) *iters_out = 0;
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "ac_set_state must be called before ac_physical_step");
    if (max_iters < 1) return fail(AC_ERR_ARG, "max_iters must be >= 1 (got %d)", max_iters);
    if (!std::isfinite(tol)) return fail(AC_ERR_ARG, "tol must be finite");
    if (c->opt.realtime && !(dt > 0.0 && std::isfinite(dt))) return fail(AC_ERR_ARG, "dt must be finite and > 0");
    if (!c->opt.realtime) dt = 1.0;
    cudaStream_t s = c->stream;
    {
        SweepArgs<double> a = make_args(c, 0);
        int blocks = (int)std::min<size_t>((c->N + 255) / 256, 152 * 8);
        begin_step_kernel<double><<<blocks, 256, 0, s>>>(a, dt, tol, max_iters);
        CK(cudaGetLastError());
        c->launches += 1;
    }
    if (c->profiling) {
        // one iteration at a time, stage sweeps bracketed by events
        while (true) {
            int rc = enqueue_iteration(c, s, 0, 0, true);
            if (rc != AC_OK) return rc;
            CK(cudaMemcpyAsync(c->hctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int st = 1; st <= c->opt.rk_stages; ++st) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, c->ev[st - 1], c->ev[st]));
                c->stage_ms += ms;
            }
            c->stage_launches += c->opt.rk_stages;
            c->launches += kernels_per_iteration(c);
            if (c->hctl->done) break;
        }
    } else if (use_host_loop()) {
        // debugging aid: host-driven loop, one round trip per chunk of iterations
        int done_iters = 0, chunk = 4;
        while (true) {
            for (int k = 0; k < chunk; ++k) {
                int rc = enqueue_iteration(c, s, 0, 0);
                if (rc != AC_OK) return rc;
            }
            CK(cudaMemcpyAsync(c->hctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            done_iters += chunk;
            if (c->hctl->done) break;
            chunk = std::min(chunk * 2, 64);
        }
        c->launches += (long long)done_iters * kernels_per_iteration(c);
    } else {
        int rc = build_graph(c);
        if (rc != AC_OK) return rc;
        CK(cudaGraphLaunch(c->exec, s));
        CK(cudaMemcpyAsync(c->hctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        c->launches += (long long)c->hctl->iter * kernels_per_iteration(c);
    }
    c->last_iters = c->hctl->iter;
    if (iters_out) *iters_out = c->hctl->iter;
    if (c->hctl->status == -3) {
        // restore the state of the start of the step: Q <- Q^n (all four fields)
        const size_t bytes = c->N * sizeof(double);
        for (int f = 0; f < 4; ++f)
            CK(cudaMemcpyAsync(c->buf[c->hctl->cur][f], c->lev[f], bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
        c->cur_host = c->hctl->cur;
        return fail(AC_ERR_NONFINITE, "residual norm became non-finite at pseudo-iteration %d", c->hctl->iter);
    }
    c->cur_host = c->hctl->cur;
    return c->hctl->status == 0 ? AC_OK : AC_NOT_CONVERGED;
}

int ac_residual_norms(const ac_ctx *c, double out[4], double out0[4]) {
    if (!c || !out) return fail(AC_ERR_ARG, "NULL argument");
    for (int k = 0; k < 4; ++k) {
        out[k] = c->hctl->R[k];
        if (out0) out0[k] = c->hctl->R0[k];
    }
    return AC_OK;
}

int ac_get_levels(const ac_ctx *c, double *rho_n, double *rhou_n, double *rhov_n) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    double *dst[3] = {rho_n, rhou_n, rhov_n};
    for (int f = 0; f < 3; ++f)
        if (dst[f]) CK(cudaMemcpyAsync(dst[f], c->lev[f], c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AC_OK;
}

int ac_set_levels(ac_ctx *c, const double *rho_n, const double *rhou_n, const double *rhov_n) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    int rc;
    if ((rc = check_host_field(rho_n, c->N, true, "rho_n")) != AC_OK) return rc;
    if ((rc = check_host_field(rhou_n, c->N, false, "rhou_n")) != AC_OK) return rc;
    if ((rc = check_host_field(rhov_n, c->N, false, "rhov_n")) != AC_OK) return rc;
    const double *src[3] = {rho_n, rhou_n, rhov_n};
    for (int f = 0; f < 3; ++f)
        CK(cudaMemcpyAsync(c->lev[f], src[f], c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AC_OK;
}

long long ac_kernel_launches(const ac_ctx *c) { return c ? c->launches : 0; }

int ac_set_profiling(ac_ctx *c, int on) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    c->profiling = on != 0;
    c->stage_ms = 0.0;
    c->stage_launches = 0;
    return AC_OK;
}

int ac_stage_kernel_time(const ac_ctx *c, double *total_ms, long long *launches) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (total_ms) *total_ms = c->stage_ms;
    if (launches) *launches = c->stage_launches;
    return AC_OK;
}

}  // extern "C"
