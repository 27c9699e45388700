// ac_noalloc.cu -- one stage sweep on caller-owned device buffers that
// performs no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// they do not own, a sandbox or plug-in host that forbids allocation after
// start-up, or a real-time loop where an allocation could stall or fail.
// They pass device pointers for every input and output; the scratch space
// the sweep needs (its control block and the per-tile residual partial
// sums) lives in a fixed-size array compiled into this library.
//
// The scratch array is a file-scope __device__ variable: every GPU that
// loads the library holds it (1 MiB) until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it is only a
// stand-in); its device address is looked up with cudaGetSymbolAddress on
// the current device at every call (a host-side lookup that allocates
// nothing), so no address outlives a device reset.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "../../include/ac.h"
#include "ac_internal.h"
#include "ac_kernels.cuh"

using namespace acgb;

namespace {

constexpr int kTX = 32, kTY = 8;
constexpr size_t kScratchBytes = size_t(1) << 20;       // AC_NOALLOC_SCRATCH_BYTES
constexpr size_t kCtlBytes = 256;                       // control block, 256-byte slot
constexpr size_t kMaxTiles = (kScratchBytes - kCtlBytes) / (4 * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

#define fail acgb::set_last_error

// Set-up on the current device, at every call: the scratch array's device
// address and the sweep kernels' shared-memory limit.  Both are host-side
// calls that allocate nothing; on a device's first call they may load the
// library's kernels, which is why that first call should come before any
// stream capture.
int setup_device(unsigned char **scratch) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    const int smem = (int)sizeof(StageSmem<double, kTX, kTY>);
    e = cudaFuncSetAttribute(stage_kernel<double, kTX, kTY, kOsher>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stage_kernel<double, kTX, kTY, kBassi>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stage_kernel<double, kTX, kTY, kRoe>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return fail(AC_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    *scratch = static_cast<unsigned char *>(p);
    return AC_OK;
}

// Reset the control block for one sweep: not done, Q^{m} in buffer slot 0,
// the real-time step, and an empty global pseudo-time step.
__global__ void noalloc_init_kernel(Ctl *ctl, double inv_dt) {
    ctl->iter = 0;
    ctl->done = 0;
    ctl->cur = 0;
    ctl->status = 1;
    ctl->inv_dt = inv_dt;
    ctl->dt = inv_dt > 0.0 ? 1.0 / inv_dt : 0.0;
    ctl->dtau_bits = 0x7ff0000000000000ull;
    ctl->tau = 0.0;
    ctl->tau_end = INFINITY;
}

// R_k = sqrt(sum of the tiles' partial sums / cells), summed in a fixed order.
__global__ void noalloc_norms_kernel(const double *partials, int ntiles, double inv_cells, double *norms) {
    __shared__ double red[4][256];
    const int tid = threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < ntiles; b += 256)
        for (int f = 0; f < 4; ++f) s[f] += partials[(size_t)b * 4 + f];
    for (int f = 0; f < 4; ++f) red[f][tid] = s[f];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
            for (int f = 0; f < 4; ++f) red[f][tid] += red[f][tid + w];
        __syncthreads();
    }
    if (tid < 4) norms[tid] = sqrt(red[tid][0] * inv_cells);
}

}  // namespace

extern "C" int ac_stage_sweep_noalloc(const ac_grid *grid, double beta, const ac_bc *bc, const ac_options *opt,
                                      int stage, double dt, const double *const q_prev[4],
                                      const double *const q0[4], const double *const qn[3],
                                      double *const q_out[4], double *norms, void *stream) {
    set_last_error(AC_OK, "%s", "");
    if (!grid || !bc || !opt || !q0 || !q_out) return fail(AC_ERR_ARG, "grid, bc, opt, q0 and q_out are required");
    if (grid->nx < 1 || grid->ny < 1) return fail(AC_ERR_ARG, "nx, ny must be >= 1");
    if (!(grid->lx > 0.0) || !(grid->ly > 0.0)) return fail(AC_ERR_ARG, "lx, ly must be > 0");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(AC_ERR_ARG, "beta must be finite and > 0");
    const int sides[4] = {bc->xlo, bc->xhi, bc->ylo, bc->yhi};
    for (int k = 0; k < 4; ++k)
        if (sides[k] < AC_BC_WALL_SLIP || sides[k] > AC_BC_PERIODIC)
            return fail(AC_ERR_ARG, "boundary kind %d on side %d is unknown", sides[k], k);
    if ((bc->xlo == AC_BC_PERIODIC) != (bc->xhi == AC_BC_PERIODIC) ||
        (bc->ylo == AC_BC_PERIODIC) != (bc->yhi == AC_BC_PERIODIC))
        return fail(AC_ERR_ARG, "periodic boundaries must be set on both sides of an axis");
    // the grid must fit the fixed scratch; checked before anything else is
    // looked at, so an oversized grid never reaches a launch
    const dim3 g((grid->nx + kTX - 1) / kTX, (grid->ny + kTY - 1) / kTY);
    const size_t tiles = (size_t)g.x * g.y;
    if (tiles > kMaxTiles)
        return fail(AC_ERR_ARG,
                    "grid %dx%d needs %zu tiles of %dx%d cells; the no-allocation scratch holds at most %zu "
                    "(about %zu cells)",
                    grid->nx, grid->ny, tiles, kTX, kTY, kMaxTiles, kMaxTiles * kTX * kTY);

    if (opt->precision != AC_PREC_FP64) return fail(AC_ERR_ARG, "only the FP64 sweep has a no-allocation variant");
    if (opt->rk_stages < 1 || opt->rk_stages > 4) return fail(AC_ERR_ARG, "rk_stages must be 1..4");
    if (stage < 1 || stage > opt->rk_stages) return fail(AC_ERR_ARG, "stage must be 1..rk_stages (got %d)", stage);
    if (opt->gradp < AC_GRADP_NEW || opt->gradp > AC_GRADP_SPLIT_SUPERBEE) return fail(AC_ERR_ARG, "gradp is unknown");
    if (opt->riemann < AC_RIEMANN_OSHER || opt->riemann > AC_RIEMANN_ROE) return fail(AC_ERR_ARG, "riemann is unknown");
    if (opt->limiter_k != 1 && opt->limiter_k != 2) return fail(AC_ERR_ARG, "limiter_k must be 1 or 2");
    if (!(opt->cfl_tau > 0.0)) return fail(AC_ERR_ARG, "cfl_tau must be > 0");
    if (opt->bdf_order > 1) return fail(AC_ERR_ARG, "the no-allocation sweep uses the Backward-Euler real-time term");
    if (opt->realtime && !(dt > 0.0 && std::isfinite(dt))) return fail(AC_ERR_ARG, "dt must be finite and > 0");
    if (stage > 1 && !q_prev) return fail(AC_ERR_ARG, "q_prev is required for stage > 1");
    if (opt->realtime && !qn) return fail(AC_ERR_ARG, "qn is required when the real-time term is on");
    for (int f = 0; f < 4; ++f)
        if (!q0[f] || !q_out[f] || (stage > 1 && !q_prev[f]))
            return fail(AC_ERR_ARG, "field pointer %d is NULL", f);
    cudaError_t e;
    unsigned char *scratch = nullptr;
    int rc = setup_device(&scratch);
    if (rc != AC_OK) return rc;
    Ctl *ctl = reinterpret_cast<Ctl *>(scratch);
    double *partials = reinterpret_cast<double *>(scratch + kCtlBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Buffer slots as the sweep kernel expects them (Q^{m} in slot 0).
    SweepArgs<double> a;
    memset(&a, 0, sizeof a);
    int in = 0, out = 0;
    {
        const int o1 = 1, o2 = 2;
        out = (stage & 1) ? o1 : o2;
        in = (stage == 1) ? 0 : (((stage - 1) & 1) ? o1 : o2);
    }
    for (int f = 0; f < 4; ++f) {
        a.buf[0][f] = const_cast<double *>(q0[f]);
        a.buf[out][f] = q_out[f];
        if (stage > 1) a.buf[in][f] = const_cast<double *>(q_prev[f]);
    }
    for (int f = 0; f < 3; ++f) a.lev[f] = qn ? const_cast<double *>(qn[f]) : nullptr;
    a.order = 1;                     // Backward-Euler real-time term
    a.B[0] = 1.0;
    a.B[1] = -1.0;
    a.nx = grid->nx; a.ny = grid->ny;
    for (int k = 0; k < 4; ++k) a.bc[k] = sides[k];
    a.gradp = opt->gradp; a.limiter_k = opt->limiter_k; a.realtime = opt->realtime ? 1 : 0;
    a.riemann = opt->riemann;
    a.local_dtau = opt->local_dtau ? 1 : 0; a.alpha_pi_p_row = opt->alpha_pi_p_row ? 1 : 0;
    a.stage = stage; a.s_max = opt->rk_stages;
    a.alpha = 1.0 / double(opt->rk_stages - stage + 1);
    const double dx = grid->lx / grid->nx, dy = grid->ly / grid->ny;
    a.dx = dx; a.dy = dy; a.half_dx = 0.5 * dx; a.half_dy = 0.5 * dy;
    a.inv_dx = 1.0 / dx; a.inv_dy = 1.0 / dy; a.dx_over_dy = dx / dy; a.dy_over_dx = dy / dx;
    a.beta = beta; a.inv_beta = 1.0 / beta; a.gx = grid->gx; a.gy = grid->gy;
    a.cfl_area = opt->cfl_tau * dx * dy;
    a.partials = partials;
    a.ctl = ctl;

    noalloc_init_kernel<<<1, 1, 0, s>>>(ctl, opt->realtime ? 1.0 / dt : 0.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(AC_ERR_CUDA, "init launch: %s", cudaGetErrorString(e));
    if (!a.local_dtau) {
        const size_t N = (size_t)grid->nx * grid->ny;
        const int blocks = (int)((N + 255) / 256 < 1216 ? (N + 255) / 256 : 1216);
        dtau_min_kernel<double><<<blocks, 256, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(AC_ERR_CUDA, "dtau launch: %s", cudaGetErrorString(e));
    }
    const size_t smem = sizeof(StageSmem<double, kTX, kTY>);
    if (opt->riemann == AC_RIEMANN_BASSI) stage_kernel<double, kTX, kTY, kBassi><<<g, kTX * kTY, smem, s>>>(a);
    else if (opt->riemann == AC_RIEMANN_ROE) stage_kernel<double, kTX, kTY, kRoe><<<g, kTX * kTY, smem, s>>>(a);
    else stage_kernel<double, kTX, kTY, kOsher><<<g, kTX * kTY, smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(AC_ERR_CUDA, "sweep launch: %s", cudaGetErrorString(e));
    if (stage == 1 && norms) {
        noalloc_norms_kernel<<<1, 256, 0, s>>>(partials, (int)tiles, 1.0 / ((double)grid->nx * grid->ny), norms);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(AC_ERR_CUDA, "norms launch: %s", cudaGetErrorString(e));
    }
    return AC_OK;
}
