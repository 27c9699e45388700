// ac_batch.cu -- many independent tanks of uneven size advanced together in
// the mixed form (declared in include/ac.h, ac_batch_*).
//
// Every stage of every tank is one launch over the flattened list of all
// tanks' tiles: CTA b looks up its tank in a tile -> tank map, reads the
// tank's descriptor for this stage from global memory and runs the same
// tile sweep as the single-tank kernel (mixed_tile), so a tank's numbers do
// not depend on what else is in the batch.  Each tank has its own control block: its own
// pseudo-iteration count, residual norms, stopping test, convergence flag
// and buffer rotation; the tiles of a tank that has converged return at
// once.  The end-of-iteration kernel runs one CTA per tank; the last CTA to
// arrive (an atomic counter, no waiting) sets the graph's WHILE condition
// to "some tank still iterating".  The whole pseudo-iteration loop of one
// physical step is one graph launch.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/ac.h"
#include "ac_internal.h"
#include "ac_kernels_mixed.cuh"
#include "ac_mixed_host.h"

using namespace acgb;

#define fail acgb::set_last_error
#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA, "%s failed: %s", #call, \
                        cudaGetErrorString(e_));                                                        \
    } while (0)

namespace {

struct BatchTank {
    MixedArgs a;   // the tank's arrays, scalars and control block (stage fields unset)
    int tile0;     // its first tile in the flattened list
    int tiles_x;   // tiles along x
    int ntiles;
    int pad;
};

struct BatchSync {
    unsigned int arrive;       // end-of-iteration CTAs arrived
    unsigned int still_active; // tanks still iterating after this iteration
};

// Descriptors of batches that fit, in constant memory: a CTA's loads of its
// tank's sizes, beta and pointers are then uniform constant-cache reads.  A
// batch owns a contiguous range of slots (first fit); larger batches, or
// batches created while the table is full, read their descriptors from
// global memory.
constexpr int kConstTanks = 160;
__constant__ BatchTank c_tanks[kConstTanks];

// Stage `stage` (coefficient alpha_s) of every active tank; blockIdx.x runs
// over the flattened tiles.  CD: the tank's descriptor is c_tanks[slot0 + k],
// else tanks[k].  PF: the prefetching tile sweep (see mixed_tile).  (The CTAs-per-SM hint keeps the sweep at 40 registers, see
// ac_api.cu.)
template <int TX, int TY, int NT, int RS = kOsher, bool BDF = false, bool CD = false, bool PF = false>
__global__ void __launch_bounds__(NT, NT == 512 ? 3 : 6)
batch_stage_kernel(const BatchTank *__restrict__ tanks, const int *__restrict__ tile_tank, int stage, float alpha,
                   int slot0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    pdl_wait();
    const int k = tile_tank[blockIdx.x];
    if constexpr (CD) {
        const BatchTank &t = c_tanks[slot0 + k];
        if (t.a.ctl->done) return;
        const int local = blockIdx.x - t.tile0;
        const int by = local / t.tiles_x, bx = local - by * t.tiles_x;
        mixed_tile<TX, TY, NT, RS, BDF, PF>(t.a, stage, alpha, bx, by, t.a.partials + (size_t)local * 4, smem_raw);
    } else {
        const BatchTank &t = tanks[k];
        if (t.a.ctl->done) return;
        const int local = blockIdx.x - t.tile0;
        const int by = local / t.tiles_x, bx = local - by * t.tiles_x;
        mixed_tile<TX, TY, NT, RS, BDF, PF>(t.a, stage, alpha, bx, by, t.a.partials + (size_t)local * 4, smem_raw);
    }
}

// Column-strip form over the flattened strips of all tanks: warp w takes
// strip w (see mixed_strip); CD as above; SK: 0 for any stage and options,
// 1 and 2 for stage 1 and the later stages with the default options.
template <int H, int WPC, int MINB, bool CD, int SK>
__global__ void __launch_bounds__(WPC * 32, MINB)
batch_sweep_kernel(const BatchTank *__restrict__ tanks, const int *__restrict__ strip_tank, int nstrips, int stage,
                   float alpha, int slot0) {
    extern __shared__ __align__(16) unsigned char strip_smem[];
    StripRing *ring = reinterpret_cast<StripRing *>(strip_smem) + (threadIdx.x >> 5);
    pdl_trigger();
    pdl_wait();
    const int w = blockIdx.x * WPC + (threadIdx.x >> 5);
    if (w >= nstrips) return;   // whole warps only
    const int k = strip_tank[w];
    if constexpr (CD) {
        const BatchTank &t = c_tanks[slot0 + k];
        if (t.a.ctl->done) return;
        const int local = w - t.tile0;
        const int sy = local / t.tiles_x, sx = local - sy * t.tiles_x;
        mixed_strip<H, 1, SK>(t.a, stage, alpha, sx, sy, t.a.partials + (size_t)local * 4, ring);
    } else {
        const BatchTank &t = tanks[k];
        if (t.a.ctl->done) return;
        const int local = w - t.tile0;
        const int sy = local / t.tiles_x, sx = local - sy * t.tiles_x;
        mixed_strip<H, 1, SK>(t.a, stage, alpha, sx, sy, t.a.partials + (size_t)local * 4, ring);
    }
}

// Start of a physical step for every tank (blockIdx.y = tank): level shift
// in FP64 and control-block reset (Alg. 1).
__global__ void batch_begin_kernel(BatchTank *tanks, BatchSync *sync, const double *dt, double tol,
                                   int max_iters) {
    const MixedArgs &a = tanks[blockIdx.y].a;
    Ctl *ctl = a.ctl;
    const int cur = ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_shift(a, cur, g);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double h = dt[blockIdx.y];
        ctl->iter = 0;
        ctl->done = 0;
        ctl->status = 1;
        ctl->max_iters = max_iters;
        ctl->fixed = tol < 0.0;
        ctl->tol = tol;
        ctl->dt = h;
        ctl->inv_dt = 1.0 / h;
        ctl->dtau_bits = 0x7ff0000000000000ull;
        ctl->rebase = 0;
        ctl->tau = 0.0;
        ctl->tau_end = INFINITY;
        if (blockIdx.y == 0) {
            sync->arrive = 0;
            sync->still_active = 0;
        }
    }
}

// Level jumps of every tank (blockIdx.y = tank), after the level shift.
__global__ void batch_jumps_kernel(const BatchTank *tanks) {
    const MixedArgs &a = tanks[blockIdx.y].a;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_jumps(a, g);
}

// Pressure rebase within a step (see mixed_rebase_shift), every tank whose
// end of iteration asked for one (blockIdx.y = tank); the jumps follow in a
// second launch.
__global__ void batch_rebase_shift_kernel(const BatchTank *tanks) {
    pdl_trigger();
    pdl_wait();
    const MixedArgs &a = tanks[blockIdx.y].a;
    if (!a.ctl->rebase) return;
    const int cur = a.ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_rebase_shift(a, cur, g);
}

__global__ void batch_rebase_jumps_kernel(const BatchTank *tanks) {
    pdl_trigger();
    pdl_wait();
    const MixedArgs &a = tanks[blockIdx.y].a;
    if (!a.ctl->rebase) return;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_jumps(a, g);
}

// End of a pseudo-iteration for every tank (blockIdx.x = tank): its norms
// from its own tiles' partial sums (the fixed order of sum_partials_fixed,
// as for a tank run alone), its stopping test and buffer rotation; the last
// CTA sets the WHILE condition.
template <int NT>
__global__ void __launch_bounds__(NT)
batch_end_kernel(BatchTank *tanks, BatchSync *sync, int ntanks, unsigned long long cond, int use_cond) {
    static_assert(NT >= kEndLanes, "sum_partials_fixed needs kEndLanes threads");
    const int tid = threadIdx.x;
    pdl_trigger();
    pdl_wait();
    const BatchTank &t = tanks[blockIdx.x];
    Ctl *ctl = t.a.ctl;
    const bool was_done = ctl->done != 0;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    if (!was_done) sum_partials_fixed(t.a.partials, t.ntiles, sums);
    if (tid == 0) {
        int active = 0;
        if (!was_done) {
            const double inv_cells = 1.0 / ((double)t.a.nx * t.a.ny);
            const int it = ctl->iter + 1;
            ctl->iter = it;
            bool finite = true, conv = true;
            for (int f = 0; f < 4; ++f) {
                const double R = sqrt(sums[f] * inv_cells);
                ctl->R[f] = R;
                if (it == 1) ctl->R0[f] = R;
                if (!isfinite(R)) finite = false;
                if (!(R <= fmax(ctl->tol * ctl->R0[f], ctl->abs_tol[f]))) conv = false;
            }
            ctl->cur = final_buffer(ctl->cur, t.a.s_max);
            int done = 0;
            if (!finite) { ctl->status = -3; done = 1; }
            else if (!ctl->fixed && conv) { ctl->status = 0; done = 1; }
            else if (it >= ctl->max_iters) { ctl->status = ctl->fixed ? 0 : 1; done = 1; }
            ctl->done = done;
            // pressure rebase after iterations 1, 2, 4, 8 (see mixed_rebase_shift)
            ctl->rebase = (t.a.plevel && !done && rebase_after(it)) ? 1 : 0;
            active = !done;
        }
        if (active) atomicAdd(&sync->still_active, 1u);
        __threadfence();
        const unsigned int prev = atomicAdd(&sync->arrive, 1u);
        if (prev == (unsigned int)ntanks - 1) {
            __threadfence();
            const unsigned int left = atomicExch(&sync->still_active, 0u);
            sync->arrive = 0;
            if (use_cond) cudaGraphSetConditional(cond, left ? 1u : 0u);
        }
    }
}

// After a non-finite residual in some tanks: those tanks back to the start
// of the step.
__global__ void batch_restore_kernel(BatchTank *tanks) {
    const MixedArgs &a = tanks[blockIdx.y].a;
    if (a.ctl->status != -3) return;
    const int cur = a.ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_restore(a, cur, g);
}

struct Variant {
    int tx, ty, nt;
    bool pf;      // prefetching tile sweep
    bool sweep;   // column-strip sweep: 28 columns x ty rows per warp (new pressure gradient only)
};
constexpr Variant kVariants[] = {
    {32, 8, 256},  {32, 16, 256}, {32, 16, 512}, {64, 8, 256},        {64, 8, 512},
    {64, 16, 512}, {16, 16, 256}, {32, 8, 256, true}, {16, 16, 256, true},
    {28, 32, 128, false, true}, {28, 64, 128, false, true}, {28, 128, 128, false, true},
    // the same strips held to 3 CTAs per SM (room for the descriptor reads without spills)
    {28, 32, 128, false, true}, {28, 64, 128, false, true}, {28, 128, 128, false, true},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

template <int TX, int TY, int NT, int RS = kOsher, bool BDF = false, bool PF = false>
cudaError_t allow_smem() {
    cudaError_t e = cudaFuncSetAttribute(batch_stage_kernel<TX, TY, NT, RS, BDF, false, PF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MixedSmem<TX, TY>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batch_stage_kernel<TX, TY, NT, RS, BDF, true, PF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MixedSmem<TX, TY>));
}

// slot0 < 0: descriptors in global memory
template <int H, int WPC, int MINB, int SK>
cudaError_t launch_sweep_sk(const BatchTank *tanks, const int *map, int nstrips, int stage, float alpha, int slot0,
                            bool pdl, cudaStream_t s) {
    const dim3 g((nstrips + WPC - 1) / WPC);
    const size_t smem = WPC * sizeof(StripRing);
    const dim3 b(WPC * 32);
    if (slot0 >= 0)
        return launch_pdl(pdl, batch_sweep_kernel<H, WPC, MINB, true, SK>, g, b, smem, s, tanks, map, nstrips, stage,
                          alpha, slot0);
    return launch_pdl(pdl, batch_sweep_kernel<H, WPC, MINB, false, SK>, g, b, smem, s, tanks, map, nstrips, stage,
                      alpha, 0);
}
// fast: the batch runs the default options (see mixed_strip)
template <int H, int WPC, int MINB>
cudaError_t launch_sweep(const BatchTank *tanks, const int *map, int nstrips, int stage, float alpha, int slot0,
                         bool fast, bool pdl, cudaStream_t s) {
    if (!fast) return launch_sweep_sk<H, WPC, MINB, 0>(tanks, map, nstrips, stage, alpha, slot0, pdl, s);
    if (stage == 1) return launch_sweep_sk<H, WPC, MINB, 1>(tanks, map, nstrips, stage, alpha, slot0, pdl, s);
    return launch_sweep_sk<H, WPC, MINB, 2>(tanks, map, nstrips, stage, alpha, slot0, pdl, s);
}

template <int TX, int TY, int NT, int RS = kOsher, bool BDF = false, bool PF = false>
cudaError_t launch_stage(const BatchTank *tanks, const int *map, int ntiles, int stage, float alpha, int slot0,
                         bool pdl, cudaStream_t s) {
    if (slot0 >= 0)
        return launch_pdl(pdl, batch_stage_kernel<TX, TY, NT, RS, BDF, true, PF>, dim3(ntiles), dim3(NT),
                          sizeof(MixedSmem<TX, TY>), s, tanks, map, stage, alpha, slot0);
    return launch_pdl(pdl, batch_stage_kernel<TX, TY, NT, RS, BDF, false, PF>, dim3(ntiles), dim3(NT),
                      sizeof(MixedSmem<TX, TY>), s, tanks, map, stage, alpha, 0);
}

// First-fit allocator over the constant descriptor table (process-wide).
std::mutex g_slot_mu;
std::vector<char> g_slot_used(kConstTanks, 0);

int acquire_slots(int n) {
    if (getenv("AC_BATCH_GLOBAL_DESC")) return -1;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int s = 0; s + n <= kConstTanks; ++s) {
        bool free_run = true;
        for (int q = s; q < s + n && free_run; ++q) free_run = !g_slot_used[q];
        if (free_run) {
            for (int q = s; q < s + n; ++q) g_slot_used[q] = 1;
            return s;
        }
    }
    return -1;
}

void release_slots(int s, int n) {
    if (s < 0) return;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int q = s; q < s + n; ++q) g_slot_used[q] = 0;
}

constexpr size_t kAlign = 64;   // cells: each tank's arrays start on a 256-byte boundary

}  // namespace

struct ac_batch {
    int n;
    std::vector<ac_grid> grids;
    std::vector<ac_bc> bcs;
    std::vector<double> betas;
    ac_options opt;
    std::vector<size_t> off;            // first cell of each tank in the pooled arrays
    size_t total;                       // pooled cells (with alignment padding)
    // pooled device arrays
    float4 *d[3];                       // per cell (dQ of rho, rho u, rho v; dp or p), three rotating pools
    float4 *qn;                         // per cell (FP32 Q^n of rho, rho u, rho v; rho_ref)
    float2 *jmp;                        // per cell level jumps (west face, south face)
    float *lev_p;                       // restore copy of p (without a level)
    float *dtau;                        // local pseudo-time steps (column-strip sweep, default options)
    float *D1[3], *D2[3];               // BDF2/BDF3 level differences (pools)
    double *q64[4];                     // FP64 levels of rho, rho u, rho v, p
    double *p64_step;                   // FP64 pressure levels at the start of the step
    double *pref64;                     // FP64 reference pressures (tanks with a reference)
    double *partials;
    Ctl *ctl;
    BatchSync *sync;
    BatchTank *tanks_dev;
    int *tile_map;                      // per variant: flattened tile -> tank
    double *dt_dev;
    std::vector<BatchTank> tanks_host;
    int slot0;                          // first constant-table slot, -1: descriptors in global memory
    bool pdl;                           // launch the loop's kernels with programmatic dependencies
    std::vector<char> use_ref;
    bool plevel;                        // pressure carried over an FP64 level (every tank)
    dim3 rebase_grid;                   // per-cell kernels over all tanks: (blocks per tank, tanks)
    Ctl *hctl;                          // pinned mirror of all control blocks
    int variant;
    int ntiles;
    std::vector<int> map_host;
    cudaStream_t stream, cap;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool has_state;
    int nhist;                          // older real-time levels held before the next step
    int order_now;                      // backward-difference order in the descriptors
    long long launches;
    bool profiling;
    cudaEvent_t ev[5];
    double stage_ms;
    long long stage_launches;
};

namespace {

// Device descriptors (global memory, and the constant table when the batch
// holds slots there), stream-ordered before the next launch that reads them.
int upload_tanks(ac_batch *b, cudaStream_t s) {
    CK(cudaMemcpyAsync(b->tanks_dev, b->tanks_host.data(), b->n * sizeof(BatchTank), cudaMemcpyHostToDevice, s));
    if (b->slot0 >= 0)
        CK(cudaMemcpyToSymbolAsync(c_tanks, b->tanks_host.data(), b->n * sizeof(BatchTank),
                                   b->slot0 * sizeof(BatchTank), cudaMemcpyHostToDevice, s));
    return AC_OK;
}

int build_tiles(ac_batch *b, int v) {
    const Variant &m = kVariants[v];
    b->map_host.clear();
    for (int k = 0; k < b->n; ++k) {
        const int tx = (b->grids[k].nx + m.tx - 1) / m.tx, ty = (b->grids[k].ny + m.ty - 1) / m.ty;
        BatchTank &t = b->tanks_host[k];
        t.tile0 = (int)b->map_host.size();
        t.tiles_x = tx;
        t.ntiles = tx * ty;
        for (int q = 0; q < tx * ty; ++q) b->map_host.push_back(k);
    }
    b->ntiles = (int)b->map_host.size();
    b->variant = v;
    CK(cudaMemcpyAsync(b->tile_map, b->map_host.data(), b->map_host.size() * sizeof(int), cudaMemcpyHostToDevice,
                       b->stream));
    int rc = upload_tanks(b, b->stream);
    if (rc != AC_OK) return rc;
    CK(cudaStreamSynchronize(b->stream));
    return AC_OK;
}

// Launch arguments of one batch stage.
struct StageLaunch {
    const BatchTank *tanks;
    const int *map;
    int ntiles, stage;
    float alpha;
    int slot0;
    bool fast, pdl;
    template <int TX, int TY, int NT, int RS = kOsher, bool BDF = false, bool PF = false>
    cudaError_t go(cudaStream_t s) const {
        return launch_stage<TX, TY, NT, RS, BDF, PF>(tanks, map, ntiles, stage, alpha, slot0, pdl, s);
    }
    template <int H, int MINB = 4>
    cudaError_t strips(cudaStream_t s) const {
        return launch_sweep<H, 4, MINB>(tanks, map, ntiles, stage, alpha, slot0, fast, pdl, s);
    }
};

int stage_launch(ac_batch *b, cudaStream_t s, int stage, int v) {
    cudaError_t e;
    const float alpha = float(1.0 / double(b->opt.rk_stages - stage + 1));   // alpha_s
    // the batch's tanks all use the pseudo-time step of their own cells
    const bool fast = b->opt.limiter_k == 1 && b->opt.realtime && b->opt.alpha_pi_p_row;
    const StageLaunch L{b->tanks_dev, b->tile_map, b->ntiles, stage, alpha, b->slot0, fast, b->pdl};
    // the Bassi and Roe fluxes are compiled for the first tile shape only
    if (b->opt.riemann == AC_RIEMANN_BASSI) e = L.go<32, 8, 256, kBassi, true>(s);
    else if (b->opt.riemann == AC_RIEMANN_ROE) e = L.go<32, 8, 256, kRoe, true>(s);
    else if (b->opt.bdf_order > 1) e = L.go<32, 8, 256, kOsher, true>(s);
    else switch (v) {
        case 0: e = L.go<32, 8, 256>(s); break;
        case 1: e = L.go<32, 16, 256>(s); break;
        case 2: e = L.go<32, 16, 512>(s); break;
        case 3: e = L.go<64, 8, 256>(s); break;
        case 4: e = L.go<64, 8, 512>(s); break;
        case 5: e = L.go<64, 16, 512>(s); break;
        case 6: e = L.go<16, 16, 256>(s); break;
        case 7: e = L.go<32, 8, 256, kOsher, false, true>(s); break;
        case 8: e = L.go<16, 16, 256, kOsher, false, true>(s); break;
        case 9: e = L.strips<32>(s); break;
        case 10: e = L.strips<64>(s); break;
        case 11: e = L.strips<128>(s); break;
        case 12: e = L.strips<32, 3>(s); break;
        case 13: e = L.strips<64, 3>(s); break;
        default: e = L.strips<128, 3>(s); break;
    }
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "batch stage launch failed: %s", cudaGetErrorString(e));
    return AC_OK;
}

// Autotuner for the batch: one pseudo-iteration's stages with every variant
// over all tanks (scratch buffers and partials only), fastest kept.
int tune(ac_batch *b, cudaStream_t s) {
    if (b->variant >= 0) return AC_OK;
    if (b->opt.riemann != AC_RIEMANN_OSHER || b->opt.bdf_order > 1) return build_tiles(b, 0);
    // the column-strip sweeps implement the new pressure gradient only
    const bool sweep_ok = b->opt.gradp == AC_GRADP_NEW;
    const char *env = getenv("AC_BATCH_TILE");
    if (env) {
        const int v = atoi(env);
        if (v >= 0 && v < kNumVariants) return build_tiles(b, kVariants[v].sweep && !sweep_ok ? 0 : v);
    }
    // the scratch buffers start as copies of the state (every tank holds
    // it in buffer 0 before its first step), so that every timed stage sees
    // real data
    bool all_first = true;
    for (int k = 0; k < b->n; ++k) all_first = all_first && b->hctl[k].cur == 0;
    if (all_first)
        for (int x = 1; x < 3; ++x)
            CK(cudaMemcpyAsync(b->d[x], b->d[0], b->total * sizeof(float4), cudaMemcpyDeviceToDevice, s));
    // two passes over the variants, each kept at its faster one (the first
    // pass also brings an idle GPU's clocks up)
    std::vector<float> tmin(kNumVariants, 1e30f);
    for (int pass = 0; pass < 2; ++pass)
        for (int v = 0; v < kNumVariants; ++v) {
            if (kVariants[v].sweep && !sweep_ok) continue;
            int rc = build_tiles(b, v);
            if (rc != AC_OK) return rc;
            // every stage of one pseudo-iteration (scratch buffers only)
            const int S = b->opt.rk_stages;
            for (int st = 1; st <= S; ++st)
                if ((rc = stage_launch(b, s, st, v)) != AC_OK) return rc;
            CK(cudaEventRecord(b->ev[0], s));
            for (int r = 0; r < 2; ++r)
                for (int st = 1; st <= S; ++st)
                    if ((rc = stage_launch(b, s, st, v)) != AC_OK) return rc;
            CK(cudaEventRecord(b->ev[1], s));
            CK(cudaEventSynchronize(b->ev[1]));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
            b->launches += 3 * S;
            tmin[v] = std::min(tmin[v], ms);
        }
    return build_tiles(b, int(std::min_element(tmin.begin(), tmin.end()) - tmin.begin()));
}

int enqueue_iteration(ac_batch *b, cudaStream_t s, unsigned long long cond, int use_cond, bool timed) {
    int rc;
    if (timed) CK(cudaEventRecord(b->ev[0], s));
    for (int st = 1; st <= b->opt.rk_stages; ++st) {
        if ((rc = stage_launch(b, s, st, b->variant)) != AC_OK) return rc;
        if (timed) CK(cudaEventRecord(b->ev[st], s));
    }
    CK(launch_pdl(b->pdl, batch_end_kernel<256>, dim3(b->n), dim3(256), 0, s, b->tanks_dev, b->sync, b->n, cond,
                  use_cond));
    CK(cudaGetLastError());
    if (b->plevel) {
        CK(launch_pdl(b->pdl, batch_rebase_shift_kernel, b->rebase_grid, dim3(256), 0, s, b->tanks_dev));
        CK(launch_pdl(b->pdl, batch_rebase_jumps_kernel, b->rebase_grid, dim3(256), 0, s, b->tanks_dev));
    }
    return AC_OK;
}

int build_graph(ac_batch *b) {
    if (b->exec) return AC_OK;
    CK(cudaGraphCreate(&b->graph, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, b->graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_iteration(b, b->cap, (unsigned long long)h, 1, false);
    cudaGraph_t captured = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &captured);
    if (rc != AC_OK) return rc;
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return AC_OK;
}

int check_field(const double *a, size_t n, bool positive, const char *name) {
    if (!a) return fail(AC_ERR_ARG, "%s is NULL", name);
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(a[k])) return fail(AC_ERR_NONFINITE, "%s[%zu] is not finite", name, k);
        if (positive && !(a[k] > 0.0)) return fail(AC_ERR_ARG, "%s[%zu] = %g is not > 0", name, k, a[k]);
    }
    return AC_OK;
}

}  // namespace

extern "C" {

void ac_batch_destroy(ac_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);   // (0: the default stream) nothing of this batch still runs
    for (int k = 0; k < 5; ++k)
        if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int x = 0; x < 3; ++x) cudaFree(b->d[x]);
    cudaFree(b->qn);
    for (int f = 0; f < 3; ++f) { cudaFree(b->D1[f]); cudaFree(b->D2[f]); }
    for (int f = 0; f < 4; ++f) cudaFree(b->q64[f]);
    cudaFree(b->p64_step);
    cudaFree(b->pref64);
    cudaFree(b->jmp);
    cudaFree(b->lev_p);
    cudaFree(b->dtau);
    cudaFree(b->partials);
    cudaFree(b->ctl);
    cudaFree(b->sync);
    cudaFree(b->tanks_dev);
    cudaFree(b->tile_map);
    cudaFree(b->dt_dev);
    if (b->hctl) cudaFreeHost(b->hctl);
    release_slots(b->slot0, b->n);
    delete b;
}

int ac_batch_create(int n, const ac_grid *grids, const double *beta, const ac_bc *bcs, const ac_options *opt,
                    ac_batch **out) {
    set_last_error(AC_OK, "%s", "");
    if (!out) return fail(AC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 65535) return fail(AC_ERR_ARG, "the batch needs 1..65535 tanks (got %d)", n);
    if (!grids || !beta || !bcs) return fail(AC_ERR_ARG, "grids, beta and bcs must not be NULL");
    ac_options o;
    ac_default_options(&o);
    o.precision = AC_PREC_MIXED;
    if (opt) o = *opt;
    if (o.precision != AC_PREC_MIXED) return fail(AC_ERR_ARG, "batched tanks run in the mixed form (AC_PREC_MIXED)");
    if (o.rk_stages < 1 || o.rk_stages > 4) return fail(AC_ERR_ARG, "rk_stages must be 1..4");
    if (o.riemann < AC_RIEMANN_OSHER || o.riemann > AC_RIEMANN_ROE)
        return fail(AC_ERR_ARG, "riemann solver %d is unknown", o.riemann);
    if (o.gradp < AC_GRADP_NEW || o.gradp > AC_GRADP_SPLIT_SUPERBEE) return fail(AC_ERR_ARG, "gradp %d is unknown", o.gradp);
    if (o.limiter_k != 1 && o.limiter_k != 2) return fail(AC_ERR_ARG, "limiter_k must be 1 or 2");
    if (!o.local_dtau) return fail(AC_ERR_ARG, "batched tanks use the local pseudo-time step");
    if (!(o.cfl_tau > 0.0)) return fail(AC_ERR_ARG, "cfl_tau must be > 0");
    if (o.bdf_order < 1 || o.bdf_order > 3) return fail(AC_ERR_ARG, "bdf_order must be 1, 2 or 3");
    size_t total = 0;
    for (int k = 0; k < n; ++k) {
        const ac_grid &g = grids[k];
        if (g.nx < 1 || g.ny < 1 || !(g.lx > 0.0) || !(g.ly > 0.0))
            return fail(AC_ERR_ARG, "tank %d: invalid grid", k);
        if (!(beta[k] > 0.0) || !std::isfinite(beta[k])) return fail(AC_ERR_ARG, "tank %d: beta must be > 0", k);
        const ac_bc &c = bcs[k];
        const int sides[4] = {c.xlo, c.xhi, c.ylo, c.yhi};
        for (int q = 0; q < 4; ++q)
            if (sides[q] < AC_BC_WALL_SLIP || sides[q] > AC_BC_PERIODIC)
                return fail(AC_ERR_ARG, "tank %d: boundary kind %d is unknown", k, sides[q]);
        if ((c.xlo == AC_BC_PERIODIC) != (c.xhi == AC_BC_PERIODIC) ||
            (c.ylo == AC_BC_PERIODIC) != (c.yhi == AC_BC_PERIODIC))
            return fail(AC_ERR_ARG, "tank %d: periodic boundaries must be set on both sides", k);
        total += ((size_t)g.nx * g.ny + kAlign - 1) / kAlign * kAlign;
    }
    if (total > (size_t)1 << 31) return fail(AC_ERR_ARG, "the batch holds more than 2^31 cells");
    ac_batch *b = new ac_batch();
    b->n = n;
    b->grids.assign(grids, grids + n);
    b->bcs.assign(bcs, bcs + n);
    b->betas.assign(beta, beta + n);
    b->opt = o;
    b->total = total;
    b->variant = -1;
    b->order_now = 1;
    b->slot0 = acquire_slots(n);
    b->off.resize(n);
    b->use_ref.resize(n);
    b->plevel = mixed_uses_level(o.gradp);
    bool any_ref = false;
    for (int k = 0; k < n; ++k) any_ref = any_ref || mixed_uses_reference(bcs[k], o.gradp);
    b->tanks_host.resize(n);
#define CKB(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            int c_ = fail(e_ == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA, "%s: %s", #call,   \
                          cudaGetErrorString(e_));                                                       \
            ac_batch_destroy(b);                                                                         \
            return c_;                                                                                   \
        }                                                                                                \
    } while (0)
    const size_t fb = total * sizeof(float), db = total * sizeof(double), f4 = total * sizeof(float4);
    for (int x = 0; x < 3; ++x) CKB(cudaMalloc(&b->d[x], f4));
    CKB(cudaMalloc(&b->qn, f4));
    for (int f = 0; f < 4; ++f) CKB(cudaMalloc(&b->q64[f], db));
    if (b->plevel) CKB(cudaMalloc(&b->p64_step, db));
    if (any_ref) CKB(cudaMalloc(&b->pref64, db));
    CKB(cudaMalloc(&b->jmp, total * sizeof(float2)));
    CKB(cudaMalloc(&b->lev_p, fb));
    CKB(cudaMalloc(&b->dtau, fb));
    for (int f = 0; f < 3; ++f) {
        if (o.bdf_order >= 2) CKB(cudaMalloc(&b->D1[f], fb));
        if (o.bdf_order >= 3) CKB(cudaMalloc(&b->D2[f], fb));
    }
    // tiles of the smallest shape (16 x 8 cells) bound every variant's tile count
    size_t max_tiles = 0;
    for (int k = 0; k < n; ++k) max_tiles += (size_t)((grids[k].nx + 15) / 16) * ((grids[k].ny + 7) / 8);
    CKB(cudaMalloc(&b->partials, max_tiles * 4 * sizeof(double)));
    CKB(cudaMalloc(&b->tile_map, max_tiles * sizeof(int)));
    CKB(cudaMalloc(&b->ctl, n * sizeof(Ctl)));
    CKB(cudaMalloc(&b->sync, sizeof(BatchSync)));
    CKB(cudaMalloc(&b->tanks_dev, n * sizeof(BatchTank)));
    CKB(cudaMalloc(&b->dt_dev, n * sizeof(double)));
    CKB(cudaMallocHost(&b->hctl, n * sizeof(Ctl)));
    CKB(cudaMemset(b->sync, 0, sizeof(BatchSync)));
    CKB(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) CKB(cudaEventCreate(&b->ev[k]));
    CKB((allow_smem<32, 8, 256>()));
    CKB((allow_smem<32, 16, 256>()));
    CKB((allow_smem<32, 16, 512>()));
    CKB((allow_smem<64, 8, 256>()));
    CKB((allow_smem<64, 8, 512>()));
    CKB((allow_smem<64, 16, 512>()));
    CKB((allow_smem<16, 16, 256>()));
    CKB((allow_smem<32, 8, 256, kOsher, false, true>()));
    CKB((allow_smem<16, 16, 256, kOsher, false, true>()));
    CKB((allow_smem<32, 8, 256, kBassi, true>()));
    CKB((allow_smem<32, 8, 256, kRoe, true>()));
    CKB((allow_smem<32, 8, 256, kOsher, true>()));
    // per-tank descriptors: arrays offset into the pools, scalars, control block
    size_t pos = 0, tpos = 0;
    memset(b->hctl, 0, n * sizeof(Ctl));
    for (int k = 0; k < n; ++k) {
        const ac_grid &g = grids[k];
        b->off[k] = pos;
        MixedArgs &a = b->tanks_host[k].a;
        memset(&a, 0, sizeof a);
        a.nx = g.nx; a.ny = g.ny;
        a.bc[0] = bcs[k].xlo; a.bc[1] = bcs[k].xhi; a.bc[2] = bcs[k].ylo; a.bc[3] = bcs[k].yhi;
        a.gradp = o.gradp; a.limiter_k = o.limiter_k; a.realtime = o.realtime ? 1 : 0;
        a.riemann = o.riemann;
        a.local_dtau = 1; a.alpha_pi_p_row = o.alpha_pi_p_row ? 1 : 0;
        a.s_max = o.rk_stages;
        const double dx = g.lx / g.nx, dy = g.ly / g.ny;
        a.dx = float(dx); a.dy = float(dy); a.half_dx = float(0.5 * dx); a.half_dy = float(0.5 * dy);
        a.inv_dx = float(1.0 / dx); a.inv_dy = float(1.0 / dy);
        a.nh_inv_dx = float(-0.5 / dx); a.nh_inv_dy = float(-0.5 / dy);
        a.dx_over_dy = float(dx / dy); a.dy_over_dx = float(dy / dx);
        a.beta = float(beta[k]); a.inv_beta = float(1.0 / beta[k]);
        a.gx = float(g.gx); a.gy = float(g.gy);
        a.cfl_area = float(o.cfl_tau * dx * dy);
        a.plevel = b->plevel ? 1 : 0;
        b->use_ref[k] = mixed_uses_reference(bcs[k], o.gradp);
        for (int x = 0; x < 3; ++x) a.d[x] = b->d[x] + pos;
        a.qn = b->qn + pos;
        for (int f = 0; f < 4; ++f) a.q64[f] = b->q64[f] + pos;
        a.p64_step = b->p64_step ? b->p64_step + pos : nullptr;
        a.pref64 = b->use_ref[k] ? b->pref64 + pos : nullptr;
        a.jmp = b->jmp + pos;
        a.dtau = b->dtau + pos;
        a.lev_p = b->lev_p + pos;
        for (int f = 0; f < 3; ++f) {
            a.D1[f] = b->D1[f] ? b->D1[f] + pos : nullptr;
            a.D2[f] = b->D2[f] ? b->D2[f] + pos : nullptr;
        }
        a.order = 1;
        a.B0 = 1.0f;
        a.partials = b->partials + tpos * 4;
        a.ctl = b->ctl + k;
        for (int q = 0; q < 4; ++q) b->hctl[k].abs_tol[q] = o.abs_tol[q];
        b->hctl[k].done = 1;
        pos += ((size_t)g.nx * g.ny + kAlign - 1) / kAlign * kAlign;
        tpos += (size_t)((g.nx + 15) / 16) * ((g.ny + 7) / 8);
    }
    CKB(cudaMemcpy(b->ctl, b->hctl, n * sizeof(Ctl), cudaMemcpyHostToDevice));
    size_t maxN = 0;
    for (int k = 0; k < n; ++k) maxN = std::max(maxN, (size_t)grids[k].nx * grids[k].ny);
    b->rebase_grid = dim3((unsigned)std::min<size_t>((maxN + 255) / 256, 64), n);
    if (int rc = build_tiles(b, 0)) { ac_batch_destroy(b); return rc; }
    b->variant = -1;
#undef CKB
    *out = b;
    return AC_OK;
}

int ac_batch_set_stream(ac_batch *b, void *stream) {
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    b->stream = (cudaStream_t)stream;
    return AC_OK;
}

int ac_batch_set_state(ac_batch *b, int k, const double *rho, const double *rhou, const double *rhov,
                       const double *p) {
    set_last_error(AC_OK, "%s", "");
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    if (k < 0 || k >= b->n) return fail(AC_ERR_ARG, "tank index %d out of range", k);
    const size_t N = (size_t)b->grids[k].nx * b->grids[k].ny;
    int rc;
    if ((rc = check_field(rho, N, true, "rho")) != AC_OK) return rc;
    if ((rc = check_field(rhou, N, false, "rhou")) != AC_OK) return rc;
    if ((rc = check_field(rhov, N, false, "rhov")) != AC_OK) return rc;
    if ((rc = check_field(p, N, false, "p")) != AC_OK) return rc;
    const double *f[4] = {rho, rhou, rhov, p};
    const ac_grid &g = b->grids[k];
    MixedReference ref;
    build_mixed_reference(g.nx, g.ny, g.ly / g.ny, g.gy, b->use_ref[k] != 0, b->plevel, f, ref);
    cudaStream_t s = b->stream;
    CK(cudaStreamSynchronize(s));
    // the tank's control block: buffer 0 holds its state from now on
    Ctl hc;
    CK(cudaMemcpy(&hc, b->ctl + k, sizeof(Ctl), cudaMemcpyDeviceToHost));
    hc.cur = 0;
    hc.done = 1;
    hc.iter = 0;
    const size_t o = b->off[k], fb = N * sizeof(float), db = N * sizeof(double);
    // the two per-cell records: (Q^n in FP32, rho_ref) and (dQ = 0, dp = 0 or p)
    std::vector<float4> hq(N), hd(N);
    for (size_t i = 0; i < N; ++i) {
        hq[i] = make_float4(float(f[0][i]), float(f[1][i]), float(f[2][i]), ref.rho_ref[i]);
        hd[i] = make_float4(0.0f, 0.0f, 0.0f, ref.p_record[i]);
    }
    for (int q = 0; q < 3; ++q) CK(cudaMemcpyAsync(b->q64[q] + o, f[q], db, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->q64[3] + o, ref.p_level.data(), db, cudaMemcpyHostToDevice, s));
    if (b->use_ref[k]) CK(cudaMemcpyAsync(b->pref64 + o, ref.p_ref.data(), db, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->qn + o, hq.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->d[0] + o, hd.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s));
    for (int q = 0; q < 3; ++q) {
        if (b->D1[q]) CK(cudaMemsetAsync(b->D1[q] + o, 0, fb, s));
        if (b->D2[q]) CK(cudaMemsetAsync(b->D2[q] + o, 0, fb, s));
    }
    CK(cudaMemcpyAsync(b->lev_p + o, ref.p_record.data(), fb, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(b->ctl + k, &hc, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    b->hctl[k] = hc;
    b->has_state = true;
    b->nhist = 0;   // the batch's levels restart with any tank's new state
    return AC_OK;
}

int ac_batch_get_state(const ac_batch *b, int k, double *rho, double *rhou, double *rhov, double *p) {
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    if (k < 0 || k >= b->n) return fail(AC_ERR_ARG, "tank index %d out of range", k);
    const size_t N = (size_t)b->grids[k].nx * b->grids[k].ny, o = b->off[k];
    const int cur = b->hctl[k].cur;
    double *out[4] = {rho, rhou, rhov, p};
    std::vector<float4> h(N);
    CK(cudaMemcpyAsync(h.data(), b->d[cur] + o, N * sizeof(float4), cudaMemcpyDeviceToHost, b->stream));
    for (int q = 0; q < 4; ++q)
        if (out[q]) CK(cudaMemcpyAsync(out[q], b->q64[q] + o, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    // state = FP64 level + FP32 increment
    if (rho) for (size_t i = 0; i < N; ++i) rho[i] += double(h[i].x);
    if (rhou) for (size_t i = 0; i < N; ++i) rhou[i] += double(h[i].y);
    if (rhov) for (size_t i = 0; i < N; ++i) rhov[i] += double(h[i].z);
    if (p) for (size_t i = 0; i < N; ++i) p[i] += double(h[i].w);
    return AC_OK;
}

static int batch_step_impl(ac_batch *b, const double *dt, double tol, int max_iters, int *iters_out,
                           int *status_out) {
    set_last_error(AC_OK, "%s", "");
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    if (!b->has_state) return fail(AC_ERR_STATE, "ac_batch_set_state must be called before a step");
    if (!dt) return fail(AC_ERR_ARG, "dt is NULL");
    if (max_iters < 1) return fail(AC_ERR_ARG, "max_iters must be >= 1");
    if (!std::isfinite(tol)) return fail(AC_ERR_ARG, "tol must be finite");
    std::vector<double> h(b->n);
    for (int k = 0; k < b->n; ++k) {
        h[k] = b->opt.realtime ? dt[k] : 1.0;
        if (!(h[k] > 0.0) || !std::isfinite(h[k])) return fail(AC_ERR_ARG, "dt[%d] must be finite and > 0", k);
    }
    cudaStream_t s = b->stream;
    // backward-difference order of this step (the first step can only be
    // Backward-Euler, Sec. 2.2.2); the kernels read it from the descriptors
    static const double bdf[4][4] = {{0, 0, 0, 0}, {1.0, -1.0, 0, 0}, {1.5, -2.0, 0.5, 0},
                                     {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0}};
    const int order = b->opt.realtime ? std::min(b->opt.bdf_order, b->nhist + 1) : 1;
    if (order != b->order_now) {
        for (int k = 0; k < b->n; ++k) {
            MixedArgs &a = b->tanks_host[k].a;
            a.order = order;
            a.B0 = float(bdf[order][0]);
            a.B2 = float(bdf[order][2]);
            a.B3 = float(bdf[order][3]);
        }
        const int urc = upload_tanks(b, s);
        if (urc != AC_OK) return urc;
        b->order_now = order;
    }
    CK(cudaMemcpyAsync(b->dt_dev, h.data(), b->n * sizeof(double), cudaMemcpyHostToDevice, s));
    size_t maxN = 0;
    for (int k = 0; k < b->n; ++k) maxN = std::max(maxN, (size_t)b->grids[k].nx * b->grids[k].ny);
    const dim3 bg((unsigned)std::min<size_t>((maxN + 255) / 256, 64), b->n);
    batch_begin_kernel<<<bg, 256, 0, s>>>(b->tanks_dev, b->sync, b->dt_dev, tol, max_iters);
    CK(cudaGetLastError());
    batch_jumps_kernel<<<bg, 256, 0, s>>>(b->tanks_dev);
    CK(cudaGetLastError());
    b->launches += 2;
    b->pdl = false;   // the tuner times launches one after another
    int rc = tune(b, s);
    if (rc != AC_OK) return rc;
    b->pdl = pdl_enabled() && !b->profiling;
    long long iters_run = 0;
    if (b->profiling) {
        while (true) {
            if ((rc = enqueue_iteration(b, s, 0, 0, true)) != AC_OK) return rc;
            CK(cudaMemcpyAsync(b->hctl, b->ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int st = 1; st <= b->opt.rk_stages; ++st) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, b->ev[st - 1], b->ev[st]));
                b->stage_ms += ms;
            }
            b->stage_launches += b->opt.rk_stages;
            ++iters_run;
            bool all = true;
            for (int k = 0; k < b->n; ++k) all = all && b->hctl[k].done;
            if (all) break;
        }
    } else {
        if ((rc = build_graph(b)) != AC_OK) return rc;
        CK(cudaGraphLaunch(b->exec, s));
        CK(cudaMemcpyAsync(b->hctl, b->ctl, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < b->n; ++k) iters_run = std::max<long long>(iters_run, b->hctl[k].iter);
    }
    b->launches += iters_run * (b->opt.rk_stages + 1 + (b->plevel ? 2 : 0));
    int ret = AC_OK;
    bool any_nonfinite = false;
    for (int k = 0; k < b->n; ++k) {
        if (iters_out) iters_out[k] = b->hctl[k].iter;
        const int st = b->hctl[k].status;
        if (status_out) status_out[k] = st == -3 ? AC_ERR_NONFINITE : (st == 0 ? AC_OK : AC_NOT_CONVERGED);
        if (st == -3) any_nonfinite = true;
        else if (st == 1 && ret == AC_OK) ret = AC_NOT_CONVERGED;
    }
    if (any_nonfinite) {
        batch_restore_kernel<<<dim3(bg.x, b->n), 256, 0, s>>>(b->tanks_dev);
        CK(cudaGetLastError());
        batch_jumps_kernel<<<bg, 256, 0, s>>>(b->tanks_dev);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        b->nhist = 0;
        return fail(AC_ERR_NONFINITE, "a residual norm became non-finite; those tanks are back at the step's start");
    }
    b->nhist = std::min(b->nhist + 1, 2);
    return ret;
}

// The public batch step: an NVTX range around the call and, with AC_LOG=1,
// one line per step on stderr (tanks, status, iteration range, how many
// tanks converged).
int ac_batch_physical_step(ac_batch *b, const double *dt, double tol, int max_iters, int *iters_out,
                           int *status_out) {
    nvtxRangePushA("ac_batch_physical_step");
    const bool log = b && acgb::log_enabled();
    std::vector<int> its_log, st_log;
    if (log && !iters_out) its_log.assign(b->n, 0), iters_out = its_log.data();
    if (log && !status_out) st_log.assign(b->n, 0), status_out = st_log.data();
    const int rc = batch_step_impl(b, dt, tol, max_iters, iters_out, status_out);
    nvtxRangePop();
    if (log) {
        int lo = max_iters, hi = 0, conv = 0;
        for (int k = 0; k < b->n; ++k) {
            lo = std::min(lo, iters_out[k]);
            hi = std::max(hi, iters_out[k]);
            conv += status_out[k] == AC_OK;
        }
        std::fprintf(stderr, "ac_batch_physical_step: %d tanks rc=%d iters=%d..%d converged=%d\n", b->n, rc, lo, hi,
                     conv);
    }
    return rc;
}

int ac_batch_residual_norms(const ac_batch *b, int k, double out[4], double out0[4]) {
    if (!b || !out) return fail(AC_ERR_ARG, "NULL argument");
    if (k < 0 || k >= b->n) return fail(AC_ERR_ARG, "tank index %d out of range", k);
    for (int q = 0; q < 4; ++q) {
        out[q] = b->hctl[k].R[q];
        if (out0) out0[q] = b->hctl[k].R0[q];
    }
    return AC_OK;
}

int ac_batch_tile_shape(const ac_batch *b, int *tx, int *ty, int *threads) {
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    const Variant &m = kVariants[b->variant < 0 ? 0 : b->variant];
    if (tx) *tx = m.tx;
    if (ty) *ty = m.ty;
    if (threads) *threads = m.nt;
    return b->variant < 0 ? AC_ERR_STATE : AC_OK;
}

int ac_batch_set_profiling(ac_batch *b, int on) {
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    b->profiling = on != 0;
    b->stage_ms = 0.0;
    b->stage_launches = 0;
    return AC_OK;
}

int ac_batch_stage_kernel_time(const ac_batch *b, double *total_ms, long long *launches) {
    if (!b) return fail(AC_ERR_ARG, "batch is NULL");
    if (total_ms) *total_ms = b->stage_ms;
    if (launches) *launches = b->stage_launches;
    return AC_OK;
}

long long ac_batch_kernel_launches(const ac_batch *b) { return b ? b->launches : 0; }

}  // extern "C"
