// ac_api.cu -- host side of the C ABI declared in include/ac.h: validation,
// device memory, the captured pseudo-iteration loop, state transfer.
//
// Control flow of one physical step (Alg. 1):
//   begin-step kernel            Q^n <- Q, control block reset
//   graph: WHILE (not done) {    one pseudo-iteration per body execution
//     [global dtau kernel]       global pseudo-time step option
//     stage sweep  x s_max       fused stage sweeps (Eq. RK2)
//     end_iteration_kernel       norms, stopping test, buffer rotation;
//   }                            sets the WHILE condition on the device
//   one device->host read of the control block.
// The loop runs without host round trips; the host waits once per step.
//
// Two arithmetic forms share this control flow through the Backend
// interface: FP64 (every step in double precision) and mixed (FP32 sweep,
// FP64 time level, reference pressure and norms; see ac_kernels_mixed.cuh).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ac.h"
#include "ac_internal.h"
#include "ac_kernels_mixed.cuh"
#include "ac_mixed_host.h"

using namespace acgb;

namespace {
thread_local std::string g_err;
}  // namespace

int acgb::set_last_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

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

// Largest tile count any tile shape of either form produces on an nx x ny
// grid (sizes the residual partial sums).
size_t max_tiles(int nx, int ny) {
    static const int shapes[][2] = {{32, 8}, {32, 7}, {32, 6}, {32, 4}, {16, 8}, {16, 16},
                                    {32, 14}, {64, 7}, {32, 16}, {64, 8}, {64, 16}};
    size_t m = 0;
    for (const auto &sh : shapes)
        m = std::max(m, (size_t)((nx + sh[0] - 1) / sh[0]) * ((ny + sh[1] - 1) / sh[1]));
    return m;
}
constexpr int kGridStrideBlocks = 152 * 8;

bool valid_bc(int b) { return b >= AC_BC_WALL_SLIP && b <= AC_BC_PERIODIC; }

struct Backend;

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
    double dx, dy;
    Backend *be;
    double *partials;
    Ctl *ctl;
    Ctl *hctl;            // pinned host mirror
    cudaStream_t stream;  // user stream (0 = default)
    cudaStream_t cap;     // private stream used for capture
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool has_state;
    int cur_host;
    long long launches;
    bool profiling;
    cudaEvent_t ev[5];
    double stage_ms;
    long long stage_launches;
    unsigned long long *dt_word;   // device result of ac_realtime_dt
    bool pdl;             // launch the loop's kernels with programmatic dependencies
    int nhist;            // older real-time levels held (0..2) before the next step
    int order_now;        // backward-difference order of the current step
    int graph_order;      // order the captured graph was built for
};

namespace {

int grid_stride_blocks(size_t N) { return (int)std::min<size_t>((N + 255) / 256, kGridStrideBlocks); }

struct Backend {
    dim3 grid;        // stage-sweep grid of the chosen tile shape
    int nblocks = 0;  // its CTA count (residual partial sums)
    virtual ~Backend() {}
    virtual int tune(ac_ctx *c, cudaStream_t s) { (void)c; (void)s; return AC_OK; }
    virtual int alloc(ac_ctx *c) = 0;
    virtual void release() = 0;
    virtual int set_state(ac_ctx *c, const double *const f[4]) = 0;
    virtual int get_state(const ac_ctx *c, double *const out[4]) = 0;
    virtual int get_history(const ac_ctx *c, int k, double *const out[3]) = 0;
    virtual int set_history(ac_ctx *c, int k, const double *const in[3]) = 0;
    virtual int begin(ac_ctx *c, cudaStream_t s, double dt, double tol, int max_iters, double tau_end) = 0;
    virtual int dtau_min(ac_ctx *c, cudaStream_t s) = 0;
    virtual int stage(ac_ctx *c, cudaStream_t s, int st) = 0;
    virtual int restore(ac_ctx *c, cudaStream_t s) = 0;
    virtual int realtime_dt(ac_ctx *c, double cfl_area, unsigned long long *out) = 0;
    // kernels enqueued after the end of a pseudo-iteration (mixed form: the
    // pressure rebase, which runs when the end of the iteration asks for it),
    // and whether the end sets the rebase flag
    virtual int after_iteration(ac_ctx *c, cudaStream_t s) { (void)c; (void)s; return AC_OK; }
    virtual int kernels_after_iteration() const { return 0; }
    virtual bool rebases() const { return false; }
    // chosen variant (-1 before tuning) and its tile shape
    virtual int shape(int &tx, int &ty, int &nt) const = 0;
};

// Backward-difference coefficients B0..B3 (Table BDF).
const double kBDF[4][4] = {
    {0.0, 0.0, 0.0, 0.0},
    {1.0, -1.0, 0.0, 0.0},
    {1.5, -2.0, 0.5, 0.0},
    {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0},
};

// ------------------------------------------------------------------ FP64

// Tile shapes of the FP64 sweep (one thread per cell).  The FP64 pipe bounds
// this sweep, so the shapes differ mainly in how evenly the CTAs fill the
// SMs: small grids favour shapes whose CTA count is near a multiple of the
// SM count.
struct F64Variant {
    int tx, ty;
};
// 32x14 and 64x7 make one 448-cell tile per SM on a 256^2 grid (152 SMs)
constexpr F64Variant kF64Variants[] = {{32, 8}, {32, 7}, {32, 6}, {32, 4}, {16, 8}, {16, 16}, {32, 14}, {64, 7}};
constexpr int kNumF64Variants = sizeof(kF64Variants) / sizeof(kF64Variants[0]);

template <int TX, int TY, int RS = kOsher>
cudaError_t allow_f64_smem() {
    return cudaFuncSetAttribute(stage_kernel<double, TX, TY, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(StageSmem<double, TX, TY>));
}

template <int TX, int TY, int RS = kOsher>
cudaError_t launch_f64(const SweepArgs<double> &a, dim3 g, bool pdl, cudaStream_t s) {
    return launch_pdl(pdl, stage_kernel<double, TX, TY, RS>, g, dim3(TX * TY), sizeof(StageSmem<double, TX, TY>), s,
                      a);
}

std::vector<std::pair<std::pair<int, int>, int>> g_tuned_f64;

struct F64Backend : Backend {
    int variant = -1;
    double *buf[3][4] = {};
    double *lev[4] = {};
    double *lev1[3] = {}, *lev2[3] = {};   // Q^{n-1}, Q^{n-2} (BDF2, BDF3)
    double *aux[4] = {};                    // dtau and real-time terms kept from stage 1

    int shape(int &tx, int &ty, int &nt) const override {
        const F64Variant &m = kF64Variants[variant < 0 ? 0 : variant];
        tx = m.tx;
        ty = m.ty;
        nt = m.tx * m.ty;
        return variant;
    }

    void set_variant(const ac_ctx *c, int v) {
        variant = v;
        const F64Variant &m = kF64Variants[v];
        grid = dim3((c->grid.nx + m.tx - 1) / m.tx, (c->grid.ny + m.ty - 1) / m.ty);
        nblocks = grid.x * grid.y;
    }

    int launch(const ac_ctx *c, cudaStream_t s, int st, int v) const {
        const SweepArgs<double> a = args(c, st);
        const F64Variant &m = kF64Variants[v];
        const dim3 g((c->grid.nx + m.tx - 1) / m.tx, (c->grid.ny + m.ty - 1) / m.ty);
        cudaError_t e;
        // the Bassi and Roe fluxes are compiled for the first tile shape only
        if (c->opt.riemann == AC_RIEMANN_BASSI) e = launch_f64<32, 8, kBassi>(a, g, c->pdl, s);
        else if (c->opt.riemann == AC_RIEMANN_ROE) e = launch_f64<32, 8, kRoe>(a, g, c->pdl, s);
        else switch (v) {
            case 0: e = launch_f64<32, 8>(a, g, c->pdl, s); break;
            case 1: e = launch_f64<32, 7>(a, g, c->pdl, s); break;
            case 2: e = launch_f64<32, 6>(a, g, c->pdl, s); break;
            case 3: e = launch_f64<32, 4>(a, g, c->pdl, s); break;
            case 4: e = launch_f64<16, 8>(a, g, c->pdl, s); break;
            case 5: e = launch_f64<16, 16>(a, g, c->pdl, s); break;
            case 6: e = launch_f64<32, 14>(a, g, c->pdl, s); break;
            default: e = launch_f64<64, 7>(a, g, c->pdl, s); break;
        }
        if (e != cudaSuccess) return fail(AC_ERR_CUDA, "stage sweep launch failed: %s", cudaGetErrorString(e));
        return AC_OK;
    }

    // Autotuner: one pseudo-iteration's stages of every shape on this grid
    // (they write only the two scratch buffers and the residual partials,
    // all rewritten by the real iteration), fastest kept per grid size.
    int tune(ac_ctx *c, cudaStream_t s) override {
        if (variant >= 0) return AC_OK;
        if (c->opt.riemann != AC_RIEMANN_OSHER) { set_variant(c, 0); return AC_OK; }
        const char *env = getenv("AC_TILE_F64");
        if (env) {
            const int v = atoi(env);
            if (v >= 0 && v < kNumF64Variants) { set_variant(c, v); return AC_OK; }
        }
        for (auto &kv : g_tuned_f64)
            if (kv.first.first == c->grid.nx && kv.first.second == c->grid.ny) {
                set_variant(c, kv.second);
                return AC_OK;
            }
        // the scratch buffers start as copies of the state, so that every
        // timed stage sees real data
        for (int b = 0; b < 3; ++b)
            if (b != c->cur_host)
                for (int f = 0; f < 4; ++f)
                    CK(cudaMemcpyAsync(buf[b][f], buf[c->cur_host][f], c->N * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
        // two passes over the variants, each kept at its faster one (the
        // first pass also brings an idle GPU's clocks up)
        std::vector<float> tmin(kNumF64Variants, 1e30f);
        const int S = c->opt.rk_stages;
        for (int pass = 0; pass < 2; ++pass)
            for (int v = 0; v < kNumF64Variants; ++v) {
                int rc;
                // every stage of one pseudo-iteration (stages write only the two
                // scratch buffers; the level Q^m is untouched)
                for (int st = 1; st <= S; ++st)
                    if ((rc = launch(c, s, st, v)) != AC_OK) return rc;
                CK(cudaEventRecord(c->ev[0], s));
                for (int r = 0; r < 2; ++r)
                    for (int st = 1; st <= S; ++st)
                        if ((rc = launch(c, s, st, v)) != AC_OK) return rc;
                CK(cudaEventRecord(c->ev[1], s));
                CK(cudaEventSynchronize(c->ev[1]));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                c->launches += 3 * S;
                tmin[v] = std::min(tmin[v], ms);
            }
        const int best = int(std::min_element(tmin.begin(), tmin.end()) - tmin.begin());
        set_variant(c, best);
        g_tuned_f64.push_back({{c->grid.nx, c->grid.ny}, best});
        return AC_OK;
    }

    SweepArgs<double> args(const ac_ctx *c, int stage) const {
        SweepArgs<double> a;
        memset(&a, 0, sizeof a);
        a.nx = c->grid.nx; a.ny = c->grid.ny;
        a.bc[0] = c->bc.xlo; a.bc[1] = c->bc.xhi; a.bc[2] = c->bc.ylo; a.bc[3] = c->bc.yhi;
        a.gradp = c->opt.gradp; a.limiter_k = c->opt.limiter_k; a.realtime = c->opt.realtime;
        a.riemann = c->opt.riemann;
        a.local_dtau = c->opt.local_dtau; a.alpha_pi_p_row = c->opt.alpha_pi_p_row;
        a.stage = stage; a.s_max = c->opt.rk_stages;
        a.alpha = stage > 0 ? 1.0 / double(c->opt.rk_stages - stage + 1) : 0.0;
        const double dx = c->dx, dy = c->dy;
        a.dx = dx; a.dy = dy; a.half_dx = 0.5 * dx; a.half_dy = 0.5 * dy;
        a.inv_dx = 1.0 / dx; a.inv_dy = 1.0 / dy; a.dx_over_dy = dx / dy; a.dy_over_dx = dy / dx;
        a.beta = c->beta; a.inv_beta = 1.0 / c->beta; a.gx = c->grid.gx; a.gy = c->grid.gy;
        a.cfl_area = c->opt.cfl_tau * dx * dy;
        for (int b = 0; b < 3; ++b)
            for (int f = 0; f < 4; ++f) a.buf[b][f] = buf[b][f];
        for (int f = 0; f < 4; ++f) a.lev[f] = lev[f];
        for (int f = 0; f < 3; ++f) { a.lev1[f] = lev1[f]; a.lev2[f] = lev2[f]; }
        a.order = c->order_now;
        for (int q = 0; q < 4; ++q) a.B[q] = kBDF[c->order_now][q];
        a.partials = c->partials;
        a.ctl = c->ctl;
        for (int f = 0; f < 4; ++f) a.aux[f] = aux[f];
        a.reuse = (aux[0] != nullptr && c->opt.rk_stages > 1) ? 1 : 0;
        return a;
    }
    int alloc(ac_ctx *c) override {
        set_variant(c, 0);
        variant = -1;   // tuned at the first physical step
        const size_t bytes = c->N * sizeof(double);
        for (int b = 0; b < 3; ++b)
            for (int f = 0; f < 4; ++f) CK(cudaMalloc(&buf[b][f], bytes));
        for (int f = 0; f < 4; ++f) CK(cudaMalloc(&lev[f], bytes));
        if (c->opt.rk_stages > 1)
            for (int f = 0; f < 4; ++f) CK(cudaMalloc(&aux[f], bytes));
        for (int f = 0; f < 3; ++f) {
            if (c->opt.bdf_order >= 2) CK(cudaMalloc(&lev1[f], bytes));
            if (c->opt.bdf_order >= 3) CK(cudaMalloc(&lev2[f], bytes));
        }
        CK((allow_f64_smem<32, 8>()));
        CK((allow_f64_smem<32, 7>()));
        CK((allow_f64_smem<32, 6>()));
        CK((allow_f64_smem<32, 4>()));
        CK((allow_f64_smem<16, 8>()));
        CK((allow_f64_smem<16, 16>()));
        CK((allow_f64_smem<32, 14>()));
        CK((allow_f64_smem<64, 7>()));
        CK((allow_f64_smem<32, 8, kBassi>()));
        CK((allow_f64_smem<32, 8, kRoe>()));
        return AC_OK;
    }
    void release() override {
        for (int b = 0; b < 3; ++b)
            for (int f = 0; f < 4; ++f) cudaFree(buf[b][f]);
        for (int f = 0; f < 4; ++f) { cudaFree(lev[f]); cudaFree(aux[f]); }
        for (int f = 0; f < 3; ++f) { cudaFree(lev1[f]); cudaFree(lev2[f]); }
    }
    int set_state(ac_ctx *c, const double *const f[4]) override {
        const size_t bytes = c->N * sizeof(double);
        for (int k = 0; k < 4; ++k) {
            CK(cudaMemcpyAsync(buf[0][k], f[k], bytes, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(lev[k], f[k], bytes, cudaMemcpyHostToDevice, c->stream));
        }
        return AC_OK;
    }
    int get_state(const ac_ctx *c, double *const out[4]) override {
        for (int k = 0; k < 4; ++k)
            if (out[k])
                CK(cudaMemcpyAsync(out[k], buf[c->cur_host][k], c->N * sizeof(double), cudaMemcpyDeviceToHost,
                                   c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return AC_OK;
    }
    // Between steps, history k (the state k physical steps back) is in
    // lev (k = 1) and lev1 (k = 2); the step's begin shifts them to lev1, lev2.
    int get_history(const ac_ctx *c, int k, double *const out[3]) override {
        double *const *src = (k == 1) ? lev : lev1;
        for (int f = 0; f < 3; ++f)
            if (out[f])
                CK(cudaMemcpyAsync(out[f], src[f], c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return AC_OK;
    }
    int set_history(ac_ctx *c, int k, const double *const in[3]) override {
        double *const *dst = (k == 1) ? lev : lev1;
        for (int f = 0; f < 3; ++f)
            CK(cudaMemcpyAsync(dst[f], in[f], c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return AC_OK;
    }
    int begin(ac_ctx *c, cudaStream_t s, double dt, double tol, int max_iters, double tau_end) override {
        begin_step_kernel<double><<<grid_stride_blocks(c->N), 256, 0, s>>>(args(c, 0), dt, tol, max_iters,
                                                                            tau_end);
        CK(cudaGetLastError());
        return AC_OK;
    }
    int dtau_min(ac_ctx *c, cudaStream_t s) override {
        CK(launch_pdl(c->pdl, dtau_min_kernel<double>, dim3(grid_stride_blocks(c->N)), dim3(256), 0, s, args(c, 0)));
        return AC_OK;
    }
    int stage(ac_ctx *c, cudaStream_t s, int st) override { return launch(c, s, st, variant < 0 ? 0 : variant); }
    int realtime_dt(ac_ctx *c, double cfl_area, unsigned long long *out) override {
        realtime_dt_kernel<double><<<grid_stride_blocks(c->N), 256, 0, c->stream>>>(args(c, 0), c->cur_host,
                                                                                     cfl_area, out);
        CK(cudaGetLastError());
        return AC_OK;
    }
    int restore(ac_ctx *c, cudaStream_t s) override {
        // Q <- Q^n (all four fields hold the state of the start of the step)
        for (int f = 0; f < 4; ++f)
            CK(cudaMemcpyAsync(buf[c->hctl->cur][f], lev[f], c->N * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return AC_OK;
    }
};

// ------------------------------------------------------------------ mixed

// Tile shapes of the mixed sweep: TX x TY cells per CTA of NT threads, and
// the CTAs per SM the register allocation is asked to allow (1 = no limit).
struct MixedVariant {
    int tx, ty, nt, minb;
    bool pf;      // ring terms and update inputs prefetched (cp.async / early loads)
    bool sweep;   // column-strip sweep: tx = 28 output columns per warp, ty = rows per strip
};
// (Without a CTAs-per-SM hint the compiler spends ~63 registers on this
// sweep; 6 x 256 or 3 x 512 threads per SM hold it at 40 without spills.)
constexpr MixedVariant kMixedVariants[] = {
    {32, 8, 256, 6}, {32, 16, 256, 6}, {32, 16, 512, 3}, {64, 8, 256, 6}, {64, 8, 512, 3}, {64, 16, 512, 3},
    {16, 16, 256, 6}, {16, 16, 256, 7}, {32, 8, 256, 7}, {32, 16, 512, 1},
    {32, 8, 256, 6, true}, {16, 16, 256, 6, true}, {32, 16, 512, 3, true}, {32, 8, 256, 5, true},
    {16, 16, 256, 5, true},
    // column-strip sweeps (new pressure gradient only): 28 columns x H rows per warp, 4 warps per CTA,
    // 4 CTAs per SM (127 registers, no spills; tighter hints spill and lose)
    {28, 32, 128, 4, false, true}, {28, 64, 128, 4, false, true}, {28, 128, 128, 4, false, true},
    {28, 256, 128, 4, false, true}, {28, 64, 256, 2, false, true},
    // one 448-cell tile per SM on a 256x256 grid (a single wave of CTAs), with and without prefetching
    {32, 14, 448, 1, true}, {32, 14, 448, 1},
};
constexpr int kNumMixedVariants = sizeof(kMixedVariants) / sizeof(kMixedVariants[0]);

template <int TX, int TY, int NT, int MINB, int RS = kOsher, bool BDF = false, bool PF = false>
int launch_mixed(const MixedArgs &a, dim3 g, bool pdl, cudaStream_t s) {
    const cudaError_t e = launch_pdl(pdl, stage_kernel_mixed<TX, TY, NT, MINB, RS, BDF, PF>, g, dim3(NT),
                                     sizeof(MixedSmem<TX, TY>), s, a);
    return e == cudaSuccess ? AC_OK : AC_ERR_CUDA;
}

template <int H, int WPC, int MINB>
int launch_sweep(const MixedArgs &a, dim3 g, bool pdl, cudaStream_t s) {
    const int nstrips = (int)(g.x * g.y);
    // the default options have instances of their own for stage 1 (residual sums; its input is Q^{m}
    // itself) and for the later stages; other options run the general instance
    const dim3 grid((nstrips + WPC - 1) / WPC), block(WPC * 32);
    const size_t smem = WPC * sizeof(StripRing);
    const bool fast = a.limiter_k == 1 && a.realtime && a.local_dtau && a.alpha_pi_p_row;
    const cudaError_t e =
        !fast           ? launch_pdl(pdl, sweep_kernel_mixed<H, WPC, MINB, 0>, grid, block, smem, s, a, (int)g.x, nstrips)
        : a.stage == 1 ? launch_pdl(pdl, sweep_kernel_mixed<H, WPC, MINB, 1>, grid, block, smem, s, a, (int)g.x, nstrips)
                       : launch_pdl(pdl, sweep_kernel_mixed<H, WPC, MINB, 2>, grid, block, smem, s, a, (int)g.x, nstrips);
    return e == cudaSuccess ? AC_OK : AC_ERR_CUDA;
}

template <int TX, int TY, int NT, int MINB, int RS = kOsher, bool BDF = false, bool PF = false>
cudaError_t allow_mixed_smem() {
    return cudaFuncSetAttribute(stage_kernel_mixed<TX, TY, NT, MINB, RS, BDF, PF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MixedSmem<TX, TY>));
}

// chosen tile shape per grid size, shared by the contexts of this process
struct TuneKey {
    int nx, ny;
};
std::vector<std::pair<TuneKey, int>> g_tuned;

struct MixedBackend : Backend {
    int variant = -1;
    float4 *d[3] = {};   // per cell (dQ of rho, rho u, rho v; dp or p), three rotating buffers
    float4 *qn = nullptr;  // per cell (FP32 Q^n of rho, rho u, rho v; rho_ref)
    float2 *jmp = nullptr;   // per cell level jumps (west face, south face)
    float *dtau = nullptr;   // per cell local pseudo-time step (column-strip sweep, default options)
    float *lev_p = nullptr;
    float *D1[3] = {}, *D2[3] = {};   // Q^n - Q^{n-1}, Q^n - Q^{n-2} (BDF2, BDF3)
    double *q64[4] = {};   // FP64 levels of rho, rho u, rho v, p
    double *p64_step = nullptr;   // FP64 pressure level at the start of the step
    double *pref64 = nullptr;   // FP64 reference pressure (with a reference)
    bool use_ref = false, plevel = false;

    int shape(int &tx, int &ty, int &nt) const override {
        const MixedVariant &m = kMixedVariants[variant < 0 ? 0 : variant];
        tx = m.tx;
        ty = m.ty;
        nt = m.nt;
        return variant;
    }

    void set_variant(const ac_ctx *c, int v) {
        variant = v;
        const MixedVariant &m = kMixedVariants[v];
        grid = dim3((c->grid.nx + m.tx - 1) / m.tx, (c->grid.ny + m.ty - 1) / m.ty);
        nblocks = grid.x * grid.y;
    }

    int launch(const ac_ctx *c, cudaStream_t s, int st, int v) const {
        const MixedArgs a = args(c, st);
        const MixedVariant &m = kMixedVariants[v];
        const dim3 g((c->grid.nx + m.tx - 1) / m.tx, (c->grid.ny + m.ty - 1) / m.ty);
        // the Bassi and Roe fluxes are compiled for the first tile shape only
        const bool bdf = c->opt.bdf_order > 1;
        if (c->opt.riemann == AC_RIEMANN_BASSI) return launch_mixed<32, 8, 256, 6, kBassi, true>(a, g, c->pdl, s);
        if (c->opt.riemann == AC_RIEMANN_ROE) return launch_mixed<32, 8, 256, 6, kRoe, true>(a, g, c->pdl, s);
        if (bdf) return launch_mixed<32, 8, 256, 6, kOsher, true>(a, g, c->pdl, s);
        switch (v) {
            case 0: return launch_mixed<32, 8, 256, 6>(a, g, c->pdl, s);
            case 1: return launch_mixed<32, 16, 256, 6>(a, g, c->pdl, s);
            case 2: return launch_mixed<32, 16, 512, 3>(a, g, c->pdl, s);
            case 3: return launch_mixed<64, 8, 256, 6>(a, g, c->pdl, s);
            case 4: return launch_mixed<64, 8, 512, 3>(a, g, c->pdl, s);
            case 5: return launch_mixed<64, 16, 512, 3>(a, g, c->pdl, s);
            case 6: return launch_mixed<16, 16, 256, 6>(a, g, c->pdl, s);
            case 7: return launch_mixed<16, 16, 256, 7>(a, g, c->pdl, s);
            case 8: return launch_mixed<32, 8, 256, 7>(a, g, c->pdl, s);
            case 9: return launch_mixed<32, 16, 512, 1>(a, g, c->pdl, s);
            case 10: return launch_mixed<32, 8, 256, 6, kOsher, false, true>(a, g, c->pdl, s);
            case 11: return launch_mixed<16, 16, 256, 6, kOsher, false, true>(a, g, c->pdl, s);
            case 12: return launch_mixed<32, 16, 512, 3, kOsher, false, true>(a, g, c->pdl, s);
            case 13: return launch_mixed<32, 8, 256, 5, kOsher, false, true>(a, g, c->pdl, s);
            case 14: return launch_mixed<16, 16, 256, 5, kOsher, false, true>(a, g, c->pdl, s);
            case 15: return launch_sweep<32, 4, 4>(a, g, c->pdl, s);
            case 16: return launch_sweep<64, 4, 4>(a, g, c->pdl, s);
            case 17: return launch_sweep<128, 4, 4>(a, g, c->pdl, s);
            case 18: return launch_sweep<256, 4, 4>(a, g, c->pdl, s);
            case 19: return launch_sweep<64, 8, 2>(a, g, c->pdl, s);
            case 20: return launch_mixed<32, 14, 448, 1, kOsher, false, true>(a, g, c->pdl, s);
            default: return launch_mixed<32, 14, 448, 1>(a, g, c->pdl, s);
        }
    }

    // Autotuner: time one pseudo-iteration's stages with every variant on
    // this grid (they write only the two scratch buffers and the residual
    // partials, all rewritten by the real iteration) and keep the fastest.
    int tune(ac_ctx *c, cudaStream_t s) override {
        if (variant >= 0) return AC_OK;
        // other solvers and BDF2/BDF3 run one compiled shape (32 x 8)
        if (c->opt.riemann != AC_RIEMANN_OSHER || c->opt.bdf_order > 1) { set_variant(c, 0); return AC_OK; }
        // the column-strip sweeps implement the new pressure gradient only
        const bool sweep_ok = c->opt.gradp == AC_GRADP_NEW;
        const char *env = getenv("AC_TILE");
        if (env) {
            int v = atoi(env);
            if (v >= 0 && v < kNumMixedVariants) {
                set_variant(c, kMixedVariants[v].sweep && !sweep_ok ? 0 : v);
                return AC_OK;
            }
        }
        for (auto &kv : g_tuned)
            if (kv.first.nx == c->grid.nx && kv.first.ny == c->grid.ny && (sweep_ok || !kMixedVariants[kv.second].sweep)) {
                set_variant(c, kv.second);
                return AC_OK;
            }
        // the scratch buffers start as copies of the state, so that every
        // timed stage sees real data
        for (int b = 0; b < 3; ++b)
            if (b != c->cur_host)
                CK(cudaMemcpyAsync(d[b], d[c->cur_host], c->N * sizeof(float4), cudaMemcpyDeviceToDevice, s));
        // two passes over the variants, each kept at its faster one (the
        // first pass also brings an idle GPU's clocks up)
        std::vector<float> tmin(kNumMixedVariants, 1e30f);
        const int reps = c->N > (1u << 22) ? 2 : 5;
        const int S = c->opt.rk_stages;
        for (int pass = 0; pass < 2; ++pass)
            for (int v = 0; v < kNumMixedVariants; ++v) {
                if (kMixedVariants[v].sweep && !sweep_ok) continue;
                int rc;
                // every stage of one pseudo-iteration (stages write only the two
                // scratch buffers; the level Q^m is untouched)
                for (int st = 1; st <= S; ++st)
                    if ((rc = launch(c, s, st, v)) != AC_OK) return fail(rc, "tile variant %d failed to launch", v);
                CK(cudaEventRecord(c->ev[0], s));
                for (int r = 0; r < reps; ++r)
                    for (int st = 1; st <= S; ++st)
                        if ((rc = launch(c, s, st, v)) != AC_OK)
                            return fail(rc, "tile variant %d failed to launch", v);
                CK(cudaEventRecord(c->ev[1], s));
                CK(cudaEventSynchronize(c->ev[1]));
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                c->launches += (1 + reps) * S;
                tmin[v] = std::min(tmin[v], ms);
            }
        const int best = int(std::min_element(tmin.begin(), tmin.end()) - tmin.begin());
        set_variant(c, best);
        g_tuned.push_back({TuneKey{c->grid.nx, c->grid.ny}, best});
        return AC_OK;
    }

    MixedArgs args(const ac_ctx *c, int stage) const {
        MixedArgs a;
        memset(&a, 0, sizeof a);
        a.nx = c->grid.nx; a.ny = c->grid.ny;
        a.bc[0] = c->bc.xlo; a.bc[1] = c->bc.xhi; a.bc[2] = c->bc.ylo; a.bc[3] = c->bc.yhi;
        a.gradp = c->opt.gradp; a.limiter_k = c->opt.limiter_k; a.realtime = c->opt.realtime;
        a.riemann = c->opt.riemann;
        a.local_dtau = c->opt.local_dtau; a.alpha_pi_p_row = c->opt.alpha_pi_p_row;
        a.stage = stage; a.s_max = c->opt.rk_stages;
        a.alpha = stage > 0 ? float(1.0 / double(c->opt.rk_stages - stage + 1)) : 0.0f;
        const double dx = c->dx, dy = c->dy;
        a.dx = float(dx); a.dy = float(dy); a.half_dx = float(0.5 * dx); a.half_dy = float(0.5 * dy);
        a.inv_dx = float(1.0 / dx); a.inv_dy = float(1.0 / dy);
        a.nh_inv_dx = float(-0.5 / dx); a.nh_inv_dy = float(-0.5 / dy);
        a.dx_over_dy = float(dx / dy); a.dy_over_dx = float(dy / dx);
        a.beta = float(c->beta); a.inv_beta = float(1.0 / c->beta);
        a.gx = float(c->grid.gx); a.gy = float(c->grid.gy);
        a.cfl_area = float(c->opt.cfl_tau * dx * dy);
        a.plevel = plevel ? 1 : 0;
        for (int b = 0; b < 3; ++b) a.d[b] = d[b];
        a.qn = qn;
        for (int f = 0; f < 4; ++f) a.q64[f] = q64[f];
        a.p64_step = p64_step;
        a.pref64 = pref64;
        a.jmp = jmp; a.lev_p = lev_p; a.dtau = dtau;
        for (int f = 0; f < 3; ++f) { a.D1[f] = D1[f]; a.D2[f] = D2[f]; }
        a.order = c->order_now;
        a.B0 = float(kBDF[c->order_now][0]);
        a.B2 = float(kBDF[c->order_now][2]);
        a.B3 = float(kBDF[c->order_now][3]);
        a.partials = c->partials;
        a.ctl = c->ctl;
        return a;
    }
    int alloc(ac_ctx *c) override {
        const size_t fb = c->N * sizeof(float), db = c->N * sizeof(double), f4 = c->N * sizeof(float4);
        // the reference applies when both y sides are walls and the pressure
        // gradient comes from Eq. new_gradp; the pressure level with Eq. new_gradp
        use_ref = mixed_uses_reference(c->bc, c->opt.gradp);
        plevel = mixed_uses_level(c->opt.gradp);
        for (int b = 0; b < 3; ++b) CK(cudaMalloc(&d[b], f4));
        CK(cudaMalloc(&qn, f4));
        for (int f = 0; f < 4; ++f) CK(cudaMalloc(&q64[f], db));
        if (plevel) CK(cudaMalloc(&p64_step, db));
        if (use_ref) CK(cudaMalloc(&pref64, db));
        CK(cudaMalloc(&jmp, c->N * sizeof(float2)));
        CK(cudaMalloc(&lev_p, fb));
        CK(cudaMalloc(&dtau, fb));
        for (int f = 0; f < 3; ++f) {
            if (c->opt.bdf_order >= 2) CK(cudaMalloc(&D1[f], fb));
            if (c->opt.bdf_order >= 3) CK(cudaMalloc(&D2[f], fb));
        }
        CK((allow_mixed_smem<32, 8, 256, 6>()));
        CK((allow_mixed_smem<32, 16, 256, 6>()));
        CK((allow_mixed_smem<32, 16, 512, 3>()));
        CK((allow_mixed_smem<64, 8, 256, 6>()));
        CK((allow_mixed_smem<64, 8, 512, 3>()));
        CK((allow_mixed_smem<64, 16, 512, 3>()));
        CK((allow_mixed_smem<16, 16, 256, 6>()));
        CK((allow_mixed_smem<16, 16, 256, 7>()));
        CK((allow_mixed_smem<32, 8, 256, 7>()));
        CK((allow_mixed_smem<32, 16, 512, 1>()));
        CK((allow_mixed_smem<32, 8, 256, 6, kOsher, false, true>()));
        CK((allow_mixed_smem<16, 16, 256, 6, kOsher, false, true>()));
        CK((allow_mixed_smem<32, 16, 512, 3, kOsher, false, true>()));
        CK((allow_mixed_smem<32, 8, 256, 5, kOsher, false, true>()));
        CK((allow_mixed_smem<16, 16, 256, 5, kOsher, false, true>()));
        CK((allow_mixed_smem<32, 14, 448, 1, kOsher, false, true>()));
        CK((allow_mixed_smem<32, 14, 448, 1>()));
        // the 8-warp strip CTA holds 8 row rings (56 KB)
        CK(cudaFuncSetAttribute(sweep_kernel_mixed<64, 8, 2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(8 * sizeof(StripRing))));
        CK(cudaFuncSetAttribute(sweep_kernel_mixed<64, 8, 2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(8 * sizeof(StripRing))));
        CK(cudaFuncSetAttribute(sweep_kernel_mixed<64, 8, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(8 * sizeof(StripRing))));
        CK((allow_mixed_smem<32, 8, 256, 6, kBassi, true>()));
        CK((allow_mixed_smem<32, 8, 256, 6, kRoe, true>()));
        CK((allow_mixed_smem<32, 8, 256, 6, kOsher, true>()));
        set_variant(c, 0);
        variant = -1;   // tuned at the first physical step
        return AC_OK;
    }
    void release() override {
        for (int b = 0; b < 3; ++b) cudaFree(d[b]);
        cudaFree(qn);
        for (int f = 0; f < 4; ++f) cudaFree(q64[f]);
        cudaFree(p64_step);
        cudaFree(pref64);
        cudaFree(jmp);
        cudaFree(lev_p);
        cudaFree(dtau);
        for (int f = 0; f < 3; ++f) { cudaFree(D1[f]); cudaFree(D2[f]); }
    }
    int set_state(ac_ctx *c, const double *const f[4]) override {
        const size_t N = c->N;
        for (int q = 0; q < 3; ++q) {
            if (D1[q]) CK(cudaMemsetAsync(D1[q], 0, N * sizeof(float), c->stream));
            if (D2[q]) CK(cudaMemsetAsync(D2[q], 0, N * sizeof(float), c->stream));
        }
        MixedReference ref;
        build_mixed_reference(c->grid.nx, c->grid.ny, c->dy, c->grid.gy, use_ref, plevel, f, ref);
        cudaStream_t s = c->stream;
        const size_t fb = N * sizeof(float), db = N * sizeof(double);
        // the two per-cell records: (Q^n in FP32, rho_ref) and (dQ = 0, dp = 0 or p)
        std::vector<float4> hq(N), hd(N);
        for (size_t q = 0; q < N; ++q) {
            hq[q] = make_float4(float(f[0][q]), float(f[1][q]), float(f[2][q]), ref.rho_ref[q]);
            hd[q] = make_float4(0.0f, 0.0f, 0.0f, ref.p_record[q]);
        }
        for (int k = 0; k < 3; ++k) CK(cudaMemcpyAsync(q64[k], f[k], db, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(q64[3], ref.p_level.data(), db, cudaMemcpyHostToDevice, s));
        if (pref64) CK(cudaMemcpyAsync(pref64, ref.p_ref.data(), db, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(qn, hq.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d[0], hd.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(lev_p, ref.p_record.data(), fb, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return AC_OK;
    }
    int get_state(const ac_ctx *c, double *const out[4]) override {
        const size_t N = c->N;
        std::vector<float4> h(N);
        const int cur = c->cur_host;
        CK(cudaMemcpyAsync(h.data(), d[cur], N * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
        for (int k = 0; k < 4; ++k)
            if (out[k]) CK(cudaMemcpyAsync(out[k], q64[k], N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        // state = FP64 level + FP32 increment
        if (out[0]) for (size_t q = 0; q < N; ++q) out[0][q] += double(h[q].x);
        if (out[1]) for (size_t q = 0; q < N; ++q) out[1][q] += double(h[q].y);
        if (out[2]) for (size_t q = 0; q < N; ++q) out[2][q] += double(h[q].z);
        if (out[3]) for (size_t q = 0; q < N; ++q) out[3][q] += double(h[q].w);
        return AC_OK;
    }
    // Between steps, history 1 is the FP64 level q64 and history 2 is
    // q64 - D1 (D1 = difference of the last two levels).
    int get_history(const ac_ctx *c, int k, double *const out[3]) override {
        const size_t N = c->N;
        std::vector<float> h(N);
        for (int f = 0; f < 3; ++f) {
            if (!out[f]) continue;
            CK(cudaMemcpyAsync(out[f], q64[f], N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            if (k == 2) CK(cudaMemcpyAsync(h.data(), D1[f], N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (k == 2)
                for (size_t q = 0; q < N; ++q) out[f][q] -= double(h[q]);
        }
        return AC_OK;
    }
    int set_history(ac_ctx *c, int k, const double *const in[3]) override {
        const size_t N = c->N;
        std::vector<double> old(N);
        std::vector<float> h(N);
        std::vector<float4> hd, hq;   // the per-cell records (k == 1)
        const int cur = c->cur_host;
        if (k == 1) {
            hd.resize(N);
            hq.resize(N);
            CK(cudaMemcpyAsync(hd.data(), d[cur], N * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(hq.data(), qn, N * sizeof(float4), cudaMemcpyDeviceToHost, c->stream));
        }
        for (int f = 0; f < 3; ++f) {
            CK(cudaMemcpyAsync(old.data(), q64[f], N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (k == 1) {
                // the state Q = q64 + dQ stays; the level and dQ change
                auto at = [f](float4 &v) -> float & { return f == 0 ? v.x : (f == 1 ? v.y : v.z); };
                for (size_t q = 0; q < N; ++q) {
                    at(hd[q]) = float((old[q] - in[f][q]) + double(at(hd[q])));
                    at(hq[q]) = float(in[f][q]);
                }
                CK(cudaMemcpyAsync(q64[f], in[f], N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            } else {
                for (size_t q = 0; q < N; ++q) h[q] = float(old[q] - in[f][q]);
                CK(cudaMemcpyAsync(D1[f], h.data(), N * sizeof(float), cudaMemcpyHostToDevice, c->stream));
            }
            CK(cudaStreamSynchronize(c->stream));
        }
        if (k == 1) {
            CK(cudaMemcpyAsync(d[cur], hd.data(), N * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(qn, hq.data(), N * sizeof(float4), cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        return AC_OK;
    }
    int begin(ac_ctx *c, cudaStream_t s, double dt, double tol, int max_iters, double tau_end) override {
        begin_step_kernel_mixed<<<grid_stride_blocks(c->N), 256, 0, s>>>(args(c, 0), dt, tol, max_iters, tau_end);
        CK(cudaGetLastError());
        level_jumps_kernel_mixed<<<grid_stride_blocks(c->N), 256, 0, s>>>(args(c, 0));
        CK(cudaGetLastError());
        c->launches += 1;
        return AC_OK;
    }
    int dtau_min(ac_ctx *c, cudaStream_t s) override {
        CK(launch_pdl(c->pdl, dtau_min_kernel_mixed, dim3(grid_stride_blocks(c->N)), dim3(256), 0, s, args(c, 0)));
        return AC_OK;
    }
    int stage(ac_ctx *c, cudaStream_t s, int st) override {
        const int rc = launch(c, s, st, variant < 0 ? 0 : variant);
        if (rc != AC_OK) return fail(rc, "stage sweep launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        return AC_OK;
    }
    int realtime_dt(ac_ctx *c, double cfl_area, unsigned long long *out) override {
        realtime_dt_kernel_mixed<<<grid_stride_blocks(c->N), 256, 0, c->stream>>>(args(c, 0), c->cur_host,
                                                                                   cfl_area, out);
        CK(cudaGetLastError());
        return AC_OK;
    }
    int restore(ac_ctx *c, cudaStream_t s) override {
        restore_kernel_mixed<<<grid_stride_blocks(c->N), 256, 0, s>>>(args(c, 0));
        CK(cudaGetLastError());
        level_jumps_kernel_mixed<<<grid_stride_blocks(c->N), 256, 0, s>>>(args(c, 0));
        CK(cudaGetLastError());
        return AC_OK;
    }
    int after_iteration(ac_ctx *c, cudaStream_t s) override {
        if (!plevel) return AC_OK;
        const dim3 g(grid_stride_blocks(c->N));
        CK(launch_pdl(c->pdl, rebase_shift_kernel_mixed, g, dim3(256), 0, s, args(c, 0)));
        CK(launch_pdl(c->pdl, rebase_jumps_kernel_mixed, g, dim3(256), 0, s, args(c, 0)));
        return AC_OK;
    }
    int kernels_after_iteration() const override { return plevel ? 2 : 0; }
    bool rebases() const override { return plevel; }
};

// ------------------------------------------------------------------ loop

// Enqueue one pseudo-iteration on stream s (events around the stage sweeps
// when `timed`); `after` adds the kernels that follow the end of an
// iteration (they act only when its end asks for them).
int enqueue_iteration(ac_ctx *c, cudaStream_t s, unsigned long long cond, int use_cond, bool timed = false,
                      bool after = true) {
    int rc;
    IterEnd e{};
    e.rebase_pow2 = c->be->rebases() ? 1 : 0;
    e.nparts = c->be->nblocks;
    e.s_max = c->opt.rk_stages;
    e.use_cond = use_cond;
    e.inv_cells = 1.0 / double(c->N);
    e.cond = cond;
    if (!c->opt.local_dtau && (rc = c->be->dtau_min(c, s)) != AC_OK) return rc;
    if (timed) CK(cudaEventRecord(c->ev[0], s));
    for (int st = 1; st <= c->opt.rk_stages; ++st) {
        if ((rc = c->be->stage(c, s, st)) != AC_OK) return rc;
        if (timed) CK(cudaEventRecord(c->ev[st], s));
    }
    CK(launch_pdl(c->pdl, end_iteration_kernel, dim3(1), dim3(kEndLanes), 0, s, c->ctl, c->partials, e));
    return after ? c->be->after_iteration(c, s) : AC_OK;
}

// Pressure rebases in a physical step of `iters` pseudo-iterations (those
// after iterations 1, 2, 4, 8 that are not the last).
long long rebases_in(int iters) {
    long long n = 0;
    for (int m = 1; m < iters; ++m) n += rebase_after(m);
    return n;
}

int kernels_per_iteration(const ac_ctx *c) {
    return c->opt.rk_stages + 1 + (c->opt.local_dtau ? 0 : 1) + c->be->kernels_after_iteration();
}

int build_graph(ac_ctx *c) {
    if (c->exec && c->graph_order == c->order_now) return AC_OK;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        cudaGraphDestroy(c->graph);
        c->exec = nullptr;
        c->graph = nullptr;
    }
    c->graph_order = c->order_now;
    CK(cudaGraphCreate(&c->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
    // With a pressure rebase (mixed form) the first kRebaseLast pseudo-iterations
    // run in line ahead of the loop, the rebase kernels after iterations 1, 2,
    // 4, 8 only, so that the loop body itself carries no per-iteration node
    // for them.  Each of these iterations sets the loop's condition; once
    // the step is done their kernels return at once.
    std::vector<cudaGraphNode_t> pro;
    if (c->be->rebases()) {
        CK(cudaStreamBeginCaptureToGraph(c->cap, c->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        int rc = AC_OK;
        for (int m = 1; m <= kRebaseLast && rc == AC_OK; ++m)
            rc = enqueue_iteration(c, c->cap, (unsigned long long)h, 1, false, rebase_after(m));
        cudaStreamCaptureStatus st;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(c->cap, &st, nullptr, &g, &deps, nullptr, &nd);
        if (e == cudaSuccess) pro.assign(deps, deps + nd);
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &captured);
        if (rc != AC_OK) return rc;
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(AC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    // (the params union has no usable default constructor: zero raw storage)
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, c->graph, pro.empty() ? nullptr : pro.data(), nullptr, pro.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(c, c->cap, (unsigned long long)h, 1, false, false);
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
    o->bdf_order = 1;
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
    if (o.riemann < AC_RIEMANN_OSHER || o.riemann > AC_RIEMANN_ROE)
        return fail(AC_ERR_ARG, "riemann solver %d is unknown", o.riemann);
    if (o.gradp < AC_GRADP_NEW || o.gradp > AC_GRADP_SPLIT_SUPERBEE) return fail(AC_ERR_ARG, "gradp %d is unknown", o.gradp);
    if (o.limiter_k != 1 && o.limiter_k != 2) return fail(AC_ERR_ARG, "limiter_k must be 1 or 2");
    if (o.precision != AC_PREC_FP64 && o.precision != AC_PREC_MIXED)
        return fail(AC_ERR_ARG, "precision %d is unknown", o.precision);
    if (!(o.cfl_tau > 0.0) || !std::isfinite(o.cfl_tau)) return fail(AC_ERR_ARG, "cfl_tau must be > 0");
    if (o.bdf_order < 1 || o.bdf_order > 3) return fail(AC_ERR_ARG, "bdf_order must be 1, 2 or 3");
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
    c->order_now = 1;
    c->dx = grid->lx / grid->nx;
    c->dy = grid->ly / grid->ny;
    if (o.precision == AC_PREC_MIXED) c->be = new MixedBackend();
    else c->be = new F64Backend();
    auto bail = [&](int code) { ac_destroy(c); return code; };
#define CKC(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_)));                                      \
    } while (0)
    CKC(cudaGetDevice(&c->device));
    int rc = c->be->alloc(c);
    if (rc != AC_OK) return bail(rc);
    CKC(cudaMalloc(&c->partials, max_tiles(grid->nx, grid->ny) * 4 * sizeof(double)));
    CKC(cudaMalloc(&c->ctl, sizeof(Ctl)));
    CKC(cudaMalloc(&c->dt_word, sizeof(unsigned long long)));
    CKC(cudaMallocHost(&c->hctl, sizeof(Ctl)));
    CKC(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) CKC(cudaEventCreate(&c->ev[k]));
    memset(c->hctl, 0, sizeof(Ctl));
    for (int k = 0; k < 4; ++k) c->hctl->abs_tol[k] = o.abs_tol[k];
    c->hctl->done = 1;
    CKC(cudaMemcpy(c->ctl, c->hctl, sizeof(Ctl), cudaMemcpyHostToDevice));
#undef CKC
    *out = c;
    return AC_OK;
}

void ac_destroy(ac_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 5; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->be) { c->be->release(); delete c->be; }
    cudaFree(c->partials);
    cudaFree(c->ctl);
    cudaFree(c->dt_word);
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
    CK(cudaStreamSynchronize(c->stream));
    if ((rc = c->be->set_state(c, src)) != AC_OK) return rc;
    c->hctl->cur = 0;
    c->hctl->done = 1;
    c->hctl->iter = 0;
    CK(cudaMemcpyAsync(c->ctl, c->hctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->cur_host = 0;
    c->nhist = 0;
    c->has_state = true;
    return AC_OK;
}

int ac_get_state(const ac_ctx *c, double *rho, double *rhou, double *rhov, double *p) {
    g_err.clear();
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    double *dst[4] = {rho, rhou, rhov, p};
    return c->be->get_state(c, dst);
}

// One physical step (Alg. 1), or with a finite tau_end a pure pseudo-time
// run that stops when the pseudo-time reaches tau_end.
static int physical_step_impl(ac_ctx *c, double dt, double tol, int max_iters, int *iters_out,
                              double tau_end = INFINITY) {
    g_err.clear();
    if (iters_out) *iters_out = 0;
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "ac_set_state must be called before ac_physical_step");
    if (max_iters < 1) return fail(AC_ERR_ARG, "max_iters must be >= 1 (got %d)", max_iters);
    if (!std::isfinite(tol)) return fail(AC_ERR_ARG, "tol must be finite");
    if (c->opt.realtime && !(dt > 0.0 && std::isfinite(dt))) return fail(AC_ERR_ARG, "dt must be finite and > 0");
    if (!c->opt.realtime) dt = 1.0;
    cudaStream_t s = c->stream;
    int rc;
    // the first real-time step can only be Backward-Euler, the second at
    // most BDF2, and so on (Sec. 2.2.2)
    c->order_now = c->opt.realtime ? std::min(c->opt.bdf_order, c->nhist + 1) : 1;
    if ((rc = c->be->begin(c, s, dt, tol, max_iters, tau_end)) != AC_OK) return rc;
    c->launches += 1;
    c->pdl = false;   // the tuner times launches one after another
    if ((rc = c->be->tune(c, s)) != AC_OK) return rc;
    c->pdl = pdl_enabled() && !c->profiling;
    if (c->profiling) {
        // one iteration at a time, stage sweeps bracketed by events
        while (true) {
            if ((rc = enqueue_iteration(c, s, 0, 0, true)) != AC_OK) return rc;
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
        int launched = 0, chunk = 4;
        while (true) {
            for (int k = 0; k < chunk; ++k)
                if ((rc = enqueue_iteration(c, s, 0, 0)) != AC_OK) return rc;
            CK(cudaMemcpyAsync(c->hctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            launched += chunk;
            if (c->hctl->done) break;
            chunk = std::min(chunk * 2, 64);
        }
        c->launches += (long long)launched * kernels_per_iteration(c);
    } else {
        if ((rc = build_graph(c)) != AC_OK) return rc;
        CK(cudaGraphLaunch(c->exec, s));
        CK(cudaMemcpyAsync(c->hctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        // with a rebase the graph's in-line prologue always launches its
        // kRebaseLast iterations and four rebase pairs (returning at once
        // once the step is done); the loop runs the rest
        const int ka = c->be->kernels_after_iteration();
        if (c->be->rebases())
            c->launches += (long long)std::max(c->hctl->iter, kRebaseLast) * (kernels_per_iteration(c) - ka) +
                           rebases_in(kRebaseLast + 1) * ka;
        else
            c->launches += (long long)c->hctl->iter * kernels_per_iteration(c);
    }
    if (iters_out) *iters_out = c->hctl->iter;
    if (c->hctl->status == -3) {
        if ((rc = c->be->restore(c, s)) != AC_OK) return rc;
        CK(cudaStreamSynchronize(s));
        c->cur_host = c->hctl->cur;
        c->nhist = 0;   // the levels were shifted: restart from Backward-Euler
        return fail(AC_ERR_NONFINITE, "residual norm became non-finite at pseudo-iteration %d", c->hctl->iter);
    }
    c->cur_host = c->hctl->cur;
    c->nhist = std::min(c->nhist + 1, 2);
    return c->hctl->status == 0 ? AC_OK : AC_NOT_CONVERGED;
}

// The public step: an NVTX range around the whole call, for timeline
// profilers, and the AC_LOG line (iterations, status, R0 and R per field).
int ac_physical_step(ac_ctx *c, double dt, double tol, int max_iters, int *iters_out) {
    nvtxRangePushA("ac_physical_step");
    int its = 0;
    const int rc = physical_step_impl(c, dt, tol, max_iters, &its);
    nvtxRangePop();
    if (iters_out) *iters_out = its;
    if (c && c->hctl && acgb::log_enabled()) {
        const Ctl &h = *c->hctl;
        std::fprintf(stderr,
                     "ac_physical_step: %dx%d %s rc=%d iters=%d R0=(%.3e %.3e %.3e %.3e) "
                     "R=(%.3e %.3e %.3e %.3e)\n",
                     c->grid.nx, c->grid.ny, c->opt.precision == AC_PREC_MIXED ? "mixed" : "fp64", rc, its,
                     h.R0[0], h.R0[1], h.R0[2], h.R0[3], h.R[0], h.R[1], h.R[2], h.R[3]);
    }
    return rc;
}

int ac_pseudo_time_run(ac_ctx *c, double tau_end, int max_iters, int *iters_out) {
    nvtxRangePushA("ac_pseudo_time_run");
    int rc;
    if (!c) rc = fail(AC_ERR_ARG, "ctx is NULL");
    else if (c->opt.realtime || c->opt.local_dtau)
        rc = fail(AC_ERR_ARG, "a pure pseudo-time run needs the real-time term off and the global pseudo-time step");
    else if (!(tau_end > 0.0) || !std::isfinite(tau_end)) rc = fail(AC_ERR_ARG, "tau_end must be finite and > 0");
    else rc = physical_step_impl(c, 1.0, -1.0, max_iters, iters_out, tau_end);
    nvtxRangePop();
    return rc;
}

int ac_residual_norms(const ac_ctx *c, double out[4], double out0[4]) {
    if (!c || !out) return fail(AC_ERR_ARG, "NULL argument");
    for (int k = 0; k < 4; ++k) {
        out[k] = c->hctl->R[k];
        if (out0) out0[k] = c->hctl->R0[k];
    }
    return AC_OK;
}

int ac_get_history(const ac_ctx *c, int k, double *rho, double *rhou, double *rhov) {
    g_err.clear();
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (k < 1 || k > 2) return fail(AC_ERR_ARG, "history level must be 1 or 2 (got %d)", k);
    if (!c->has_state || c->nhist < k) return fail(AC_ERR_STATE, "history level %d is not available", k);
    if (k == 2 && c->opt.bdf_order < 2) return fail(AC_ERR_STATE, "history level 2 is kept only for bdf_order >= 2");
    double *dst[3] = {rho, rhou, rhov};
    return c->be->get_history(c, k, dst);
}

int ac_set_history(ac_ctx *c, int k, const double *rho, const double *rhou, const double *rhov) {
    g_err.clear();
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    if (k < 1 || k > 2) return fail(AC_ERR_ARG, "history level must be 1 or 2 (got %d)", k);
    if (k == 2 && c->opt.bdf_order < 2) return fail(AC_ERR_ARG, "history level 2 is kept only for bdf_order >= 2");
    if (k == 2 && c->nhist < 1) return fail(AC_ERR_STATE, "set history level 1 before level 2");
    int rc;
    if ((rc = check_host_field(rho, c->N, true, "rho")) != AC_OK) return rc;
    if ((rc = check_host_field(rhou, c->N, false, "rhou")) != AC_OK) return rc;
    if ((rc = check_host_field(rhov, c->N, false, "rhov")) != AC_OK) return rc;
    const double *src[3] = {rho, rhou, rhov};
    if ((rc = c->be->set_history(c, k, src)) != AC_OK) return rc;
    c->nhist = k;
    return AC_OK;
}

int ac_realtime_dt(ac_ctx *c, double cfl_t, double *dt_out) {
    g_err.clear();
    if (!c || !dt_out) return fail(AC_ERR_ARG, "ctx and dt_out must not be NULL");
    if (!c->has_state) return fail(AC_ERR_STATE, "no state has been set");
    if (!(cfl_t > 0.0) || !std::isfinite(cfl_t)) return fail(AC_ERR_ARG, "cfl_t must be finite and > 0");
    const unsigned long long inf_bits = 0x7ff0000000000000ull;
    CK(cudaMemcpyAsync(c->dt_word, &inf_bits, sizeof inf_bits, cudaMemcpyHostToDevice, c->stream));
    int rc = c->be->realtime_dt(c, cfl_t * c->dx * c->dy, c->dt_word);
    if (rc != AC_OK) return rc;
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, c->dt_word, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->launches += 1;
    memcpy(dt_out, &bits, sizeof bits);
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

// FP64 FMA rate probe: every thread runs eight independent fused
// multiply-add chains (x <- x m + c with |m| < 1, so values stay bounded), so
// the FP64 pipe, not dependency latency, sets the pace.  One double per
// thread is written, to the grid-sized buffer, so nothing is optimised away.
static __global__ void fp64_fma_probe_kernel(double *out, int iters) {
    const double m = 0.9999999, k = 1e-9;
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1e-3 * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fma(x[j], m, k);
    }
    double sum = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) sum += x[j];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

int ac_probe_fp64_fma_tflops(double *tflops) {
    g_err.clear();
    if (!tflops) return fail(AC_ERR_ARG, "tflops is NULL");
    *tflops = 0.0;
    int dev = 0, sms = 0;
    cudaError_t e0_ = cudaGetDevice(&dev);
    if (e0_ == cudaSuccess) e0_ = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0_ != cudaSuccess) return fail(AC_ERR_CUDA, "FP64 probe: %s", cudaGetErrorString(e0_));
    const int blocks = 4 * sms, threads = 256, iters = 4096;
    double *out = nullptr;
    e0_ = cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
    if (e0_ != cudaSuccess)
        return fail(e0_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA, "FP64 probe: %s",
                    cudaGetErrorString(e0_));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // the first launch warms up
        if ((e = cudaEventRecord(e0, 0)) != cudaSuccess) break;
        fp64_fma_probe_kernel<<<blocks, threads>>>(out, iters);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, 0)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "FP64 probe: %s", cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return AC_OK;
}

int ac_tile_shape(const ac_ctx *c, int *tx, int *ty, int *threads, int *variant) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    int x, y, n;
    const int v = c->be->shape(x, y, n);
    if (tx) *tx = x;
    if (ty) *ty = y;
    if (threads) *threads = n;
    if (variant) *variant = v;
    return v < 0 ? AC_ERR_STATE : AC_OK;
}

int ac_stage_kernel_time(const ac_ctx *c, double *total_ms, long long *launches) {
    if (!c) return fail(AC_ERR_ARG, "ctx is NULL");
    if (total_ms) *total_ms = c->stage_ms;
    if (launches) *launches = c->stage_launches;
    return AC_OK;
}

}  // extern "C"
