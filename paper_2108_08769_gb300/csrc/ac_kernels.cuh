// ac_kernels.cuh -- the fused pseudo-time stage sweep and its control kernels.
//
// One launch of stage_kernel performs Runge-Kutta stage s of one
// pseudo-iteration (Alg. 1, Eq. RK2) over the whole grid:
//   ghost synthesis (Sec. 2.5) -> limited gradients of rho, u, v (Sec. 2.3.1)
//   -> pressure gradient (Eq. new_gradp, or a limiter on p) -> MUSCL face
//   states (Eqs. muscl1-2) -> Osher flux on every x- and y-face (Sec. 2.4.3,
//   y-faces through the rotation of Alg. 2) -> flux divergence + real-time
//   term + body force (Sec. 2.2.1) -> point-implicit stage update
//   (Eqs. RK2, point_implicit) -> stage-1 residual partial sums.
// Each CTA owns a TX x TY tile; the tile plus a two-cell halo is staged in
// shared memory, so every field of every cell is read from HBM once per
// stage (halo re-reads hit L2).
//
// Which of the three state buffers holds Q^{m}, the stage inputs and the
// stage outputs is decided on the device from ctl->cur, so one captured
// graph serves every pseudo-iteration.
#pragma once

#include "ac_device.cuh"

namespace acgb {

// Device-resident control block of one physical step.
struct Ctl {
    int iter;        // pseudo-iterations completed
    int done;        // 1: stop iterating
    int cur;         // buffer index (0..2) holding Q^{m}
    int status;      // 0 converged / 1 not converged / -3 non-finite
    int max_iters;
    int fixed;       // 1: tol < 0, run exactly max_iters
    double tol;
    double dt, inv_dt;
    double R[4], R0[4];
    double abs_tol[4];
    unsigned long long dtau_bits;  // global pseudo-time step (bit pattern of a positive double)
    int rebase;      // mixed form: fold the pressure increment into its FP64 level before the next iteration
    double tau, tau_end;  // pure pseudo-time run: pseudo-time reached and its end (+inf in a physical step)
};

// The global pseudo-time step of the current iteration, shortened so that a
// pure pseudo-time run lands on its end (tau_end is +inf otherwise).
__device__ __forceinline__ double global_dtau(const Ctl *ctl) {
    return fmin(__longlong_as_double((long long)ctl->dtau_bits), ctl->tau_end - ctl->tau);
}

// What the end of a pseudo-iteration needs (see end_iteration).
// The mixed form rebases its pressure level after these pseudo-iterations of
// a step (1, 2, 4, ..., kRebaseLast): the first ones are where a step that
// starts from an unbalanced state moves the pressure the most.
constexpr int kRebaseLast = 8;
__host__ __device__ __forceinline__ bool rebase_after(int it) { return it <= kRebaseLast && (it & (it - 1)) == 0; }

struct IterEnd {
    int rebase_pow2;           // mixed form with a pressure level: rebase after iterations 1, 2, 4, 8
    int nparts;                // residual partial slots written by stage 1
    int s_max;
    int use_cond;              // set the graph's while-condition
    double inv_cells;
    unsigned long long cond;   // its handle
};
constexpr int kEndLanes = 128;  // threads that take part in end_iteration

template <typename T>
struct SweepArgs {
    int nx, ny;
    int bc[4];
    int gradp, limiter_k, realtime, local_dtau, alpha_pi_p_row;
    int riemann;                   // kOsher / kBassi / kRoe
    int stage, s_max;
    T alpha;                       // alpha_s of this stage
    T dx, dy, half_dx, half_dy, inv_dx, inv_dy, dx_over_dy, dy_over_dx;
    T beta, inv_beta, gx, gy;
    T cfl_area;                    // CFL_tau * |Omega|
    T *buf[3][4];                  // three state buffers: rho, rho u, rho v, p
    T *lev[4];                     // real-time level Q^n (rho, rho u, rho v, p)
    T *lev1[3], *lev2[3];          // Q^{n-1}, Q^{n-2} (rho, rho u, rho v) for BDF2/BDF3
    int order;                     // backward-difference order used in this step (1..3)
    T B[4];                        // its coefficients B0..B3 (Table BDF)
    double *partials;              // per-CTA residual partial sums [nblocks][4]
    Ctl *ctl;
    // Per-cell values that stay fixed through a pseudo-iteration (they come
    // from Q^{m} and the real-time levels): local dtau and the real-time
    // terms of rho, rho u, rho v.  With reuse set, stage 1 writes them and
    // later stages read them back instead of recomputing; null otherwise.
    T *aux[4];
    int reuse;
};

// Frozen real-time term (Eq. bdf) of field f at index s, Q^{m} value qm:
// (B0 Q^{m} + B1 Q^n + B2 Q^{n-1} + B3 Q^{n-2}) / dt, always in this order.
template <typename T>
__device__ __forceinline__ T realtime_term(const SweepArgs<T> &a, T qm, int f, size_t s, T inv_dt) {
    T r = fma(a.B[1], a.lev[f][s], a.B[0] * qm);
    if (a.order >= 2) r = fma(a.B[2], a.lev1[f][s], r);
    if (a.order >= 3) r = fma(a.B[3], a.lev2[f][s], r);
    return r * inv_dt;
}

// Buffer roles within a pseudo-iteration: stage s reads `in` and writes
// `out`; Q^{m} (stage 0) stays in `cur` until the iteration ends.
__device__ __forceinline__ void stage_buffers(int cur, int s, int &in, int &out) {
    const int o1 = (cur + 1) % 3, o2 = (cur + 2) % 3;
    out = (s & 1) ? o1 : o2;
    in = (s == 1) ? cur : (((s - 1) & 1) ? o1 : o2);
}
__host__ __device__ __forceinline__ int final_buffer(int cur, int s_max) {
    return (s_max & 1) ? (cur + 1) % 3 : (cur + 2) % 3;
}

// Sum of the stage-1 residual partials (4 per slot, nparts slots) in a fixed
// order: 128 strided sums, a shuffle tree in each of four warps, the four
// warp sums left to right.  Called by every thread of a CTA of at least
// kEndLanes threads; the sums are valid in thread 0.  The single-tank end of
// iteration and the batch's per-tank end both use it, so a tank's norms do
// not depend on which of them ran.
__device__ __forceinline__ void sum_partials_fixed(const double *partials, int nparts, double out[4]) {
    __shared__ double wsum[kEndLanes / 32][4];
    const int tid = threadIdx.x;
    if (tid < kEndLanes) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = tid; b < nparts; b += kEndLanes) {
#pragma unroll
            for (int f = 0; f < 4; ++f) s[f] += partials[(size_t)b * 4 + f];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int f = 0; f < 4; ++f) s[f] += __shfl_down_sync(0xffffffffu, s[f], o);
        }
        if ((tid & 31) == 0) {
#pragma unroll
            for (int f = 0; f < 4; ++f) wsum[tid >> 5][f] = s[f];
        }
    }
    __syncthreads();
    if (tid == 0) {
        for (int f = 0; f < 4; ++f) {
            double sum = wsum[0][f];
            for (int w = 1; w < kEndLanes / 32; ++w) sum += wsum[w][f];
            out[f] = sum;
        }
    }
}

// End of a pseudo-iteration: the residual norms from the stage-1 partials,
// the stopping test (Alg. 1), the buffer rotation and, inside a captured
// loop, the while-condition.  Called by every thread of one CTA of at least
// kEndLanes threads.
__device__ __forceinline__ void end_iteration(Ctl *ctl, const double *partials, const IterEnd &e) {
    double sums[4];
    sum_partials_fixed(partials, e.nparts, sums);
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int it = ctl->iter + 1;
        ctl->iter = it;
        bool finite = true, conv = true;
        for (int f = 0; f < 4; ++f) {
            const double R = sqrt(sums[f] * e.inv_cells);
            ctl->R[f] = R;
            if (it == 1) ctl->R0[f] = R;
            if (!isfinite(R)) finite = false;
            const double thr = fmax(ctl->tol * ctl->R0[f], ctl->abs_tol[f]);
            if (!(R <= thr)) conv = false;
        }
        ctl->cur = final_buffer(ctl->cur, e.s_max);
        bool reached = false;   // a pure pseudo-time run reached its end
        if (ctl->tau_end < INFINITY) {
            ctl->tau += global_dtau(ctl);
            reached = ctl->tau >= ctl->tau_end;
        }
        int done = 0;
        if (!finite) { ctl->status = -3; done = 1; }
        else if (reached) { ctl->status = 0; done = 1; }
        else if (!ctl->fixed && conv) { ctl->status = 0; done = 1; }
        else if (it >= ctl->max_iters) {
            // a fixed iteration count is complete; a pseudo-time run short of its end is not
            ctl->status = (ctl->fixed && !(ctl->tau_end < INFINITY)) ? 0 : 1;
            done = 1;
        }
        ctl->done = done;
        ctl->rebase = (e.rebase_pow2 && !done && rebase_after(it)) ? 1 : 0;
        ctl->dtau_bits = 0x7ff0000000000000ull;
        if (e.use_cond) cudaGraphSetConditional(e.cond, done ? 0u : 1u);
    }
}

template <typename T>
__device__ __forceinline__ T wall_ghost_sign(int gi, int gj, int nx, int ny, const int bc[4]) {
    const bool w = (gi < 0 && is_wall(bc[0])) || (gi >= nx && is_wall(bc[1])) ||
                   (gj < 0 && is_wall(bc[2])) || (gj >= ny && is_wall(bc[3]));
    return w ? T(-1) : T(1);
}

// Programmatic dependent launch: let the next kernel in the stream be
// scheduled (its CTAs then wait in pdl_wait), and wait until the previous
// kernel has finished and its writes are visible.  No-ops for a kernel
// launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T, int TX, int TY>
struct StageSmem {
    static constexpr int RW = TX + 4, RH = TY + 4;   // tile + 2-cell halo
    static constexpr int GW = TX + 2, GH = TY + 2;   // tile + 1-cell ring
    static constexpr int NXF = (TX + 1) * TY;        // x-faces
    static constexpr int NYF = TX * (TY + 1);        // y-faces
    T w[4][RW * RH];      // rho, u, v, p
    T wir[RW * RH];       // 1/rho of w (stage 1's local pseudo-time step takes it, with u and v)
    T rt[2][GW * GH];     // frozen real-time term of rho u, rho v on the ring
    T gx[4][GW * GH];     // whole slopes along x: rho, u, v, p (the face states take half of each)
    T gy[4][GW * GH];     // whole slopes along y
    T fx[4][NXF];         // x-face fluxes: mass, x-mom, y-mom, p/beta
    T fy[4][NYF];         // y-face fluxes
    double red[4][TX * TY / 32];
};

// Tiles of 448 cells are sized to run one per SM: they may take the whole
// register file (ptxas otherwise budgets for two CTAs per SM and recomputes
// products to stay inside it).  Other shapes keep the compiler's choice.
constexpr int f64_min_blocks(int nt) { return nt >= 448 ? 1 : 0; }

template <typename T, int TX, int TY, int RS = kOsher>
__global__ void __launch_bounds__(TX * TY, f64_min_blocks(TX * TY))
stage_kernel(const SweepArgs<T> a) {
    using S = StageSmem<T, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    constexpr int NT = TX * TY;
    constexpr int RW = S::RW, RH = S::RH, GW = S::GW, GH = S::GH;

    pdl_trigger();
    pdl_wait();
    const Ctl *ctl = a.ctl;
    if (ctl->done) return;
    int in, out;
    const int cur = ctl->cur;
    stage_buffers(cur, a.stage, in, out);
    const T *const *qin = a.buf[in];
    const T *const *q0 = a.buf[cur];
    T *const *qout = a.buf[out];
    const T inv_dt = a.realtime ? T(ctl->inv_dt) : T(0);

    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    // ---- 1. stage Q^{s-1} (+ two-cell halo, ghosts synthesised) as W ----
    for (int k = tid; k < RW * RH; k += NT) {
        const int gi = x0 + (k % RW) - 2, gj = y0 + (k / RW) - 2;
        int nfx, tfx, nfy, tfy;
        const int si = fold_axis(gi, nx, a.bc[0], a.bc[1], nfx, tfx);
        const int sj = fold_axis(gj, ny, a.bc[2], a.bc[3], nfy, tfy);
        const size_t s = (size_t)sj * nx + si;
        const T r = qin[0][s];
        T m = qin[1][s], n = qin[2][s];
        if ((nfx + tfy) & 1) m = -m;
        if ((nfy + tfx) & 1) n = -n;
        const T ir = Ar<T>::rcp(r);
        sm.w[0][k] = r;
        sm.w[1][k] = m * ir;
        sm.w[2][k] = n * ir;
        sm.w[3][k] = qin[3][s];
        sm.wir[k] = ir;
    }
    // ---- frozen real-time term of the momenta on the ring (Eq. bdf, BE) ----
    const bool need_rt = (a.gradp == kGradNew) && a.realtime;
    const bool reuse_now = a.reuse && a.stage > 1;   // fixed per-cell values from stage 1
    if (need_rt) {
        for (int k = tid; k < GW * GH; k += NT) {
            const int gi = x0 + (k % GW) - 1, gj = y0 + (k / GW) - 1;
            int nfx, tfx, nfy, tfy;
            const int si = fold_axis(gi, nx, a.bc[0], a.bc[1], nfx, tfx);
            const int sj = fold_axis(gj, ny, a.bc[2], a.bc[3], nfy, tfy);
            const size_t s = (size_t)sj * nx + si;
            T rx, ry;
            if (reuse_now) {
                rx = a.aux[2][s];
                ry = a.aux[3][s];
            } else {
                rx = realtime_term(a, q0[1][s], 1, s, inv_dt);
                ry = realtime_term(a, q0[2][s], 2, s, inv_dt);
            }
            if ((nfx + tfy) & 1) rx = -rx;
            if ((nfy + tfx) & 1) ry = -ry;
            sm.rt[0][k] = rx;
            sm.rt[1][k] = ry;
        }
    }
    __syncthreads();

    // ---- 2. limited slopes and pressure gradient on the ring ----
    // Whole slopes (the limited difference across one cell, dx d_x rho and
    // so on); the face states take half of each with one FMA.  Halving is
    // exact, so these are the half slopes of the limiter's definition to
    // the last bit, formed with fewer FP64 instructions.
    const T klim = T(a.limiter_k);
    const T kp = (a.gradp == kGradSuperbee || a.gradp == kGradSplitSuperbee) ? T(2) : T(1);
    for (int k = tid; k < GW * GH; k += NT) {
        const int li = k % GW, lj = k / GW;            // ring coords (cell li-1, lj-1)
        const int c = (lj + 1) * RW + (li + 1);
        const int e = c + 1, wv = c - 1, nn = c + RW, ss = c - RW;
        const T *R = sm.w[0], *U = sm.w[1], *V = sm.w[2], *P = sm.w[3];
        T srx, sry, sux, suy, svx, svy;
        if (a.limiter_k == 1) {
            srx = minmod_bits(R[e] - R[c], R[c] - R[wv]);
            sry = minmod_bits(R[nn] - R[c], R[c] - R[ss]);
            sux = minmod_bits(U[e] - U[c], U[c] - U[wv]);
            suy = minmod_bits(U[nn] - U[c], U[c] - U[ss]);
            svx = minmod_bits(V[e] - V[c], V[c] - V[wv]);
            svy = minmod_bits(V[nn] - V[c], V[c] - V[ss]);
        } else {
            srx = limiter(R[e] - R[c], R[c] - R[wv], klim);
            sry = limiter(R[nn] - R[c], R[c] - R[ss], klim);
            sux = limiter(U[e] - U[c], U[c] - U[wv], klim);
            suy = limiter(U[nn] - U[c], U[c] - U[ss], klim);
            svx = limiter(V[e] - V[c], V[c] - V[wv], klim);
            svy = limiter(V[nn] - V[c], V[c] - V[ss], klim);
        }
        T spx, spy;
        if (a.gradp == kGradNew) {
            // Eq. new_gradp times dx, with dx d_x rho = srx etc.
            const int gi = x0 + li - 1, gj = y0 + lj - 1;
            const T rho = R[c], u = U[c], v = V[c];
            // the body force with gravity reversed in wall ghosts: a sign, not a product
            const T rho_g = wall_ghost_sign<T>(gi, gj, nx, ny, a.bc) < T(0) ? -rho : rho;
            const T rtx = need_rt ? sm.rt[0][k] : T(0);
            const T rty = need_rt ? sm.rt[1][k] : T(0);
            const T ru = rho * u, rv = rho * v, uv = u * v;
            spx = a.dx * fma(rho_g, a.gx, -rtx) - (u * u * srx + T(2) * ru * sux) -
                  a.dx_over_dy * (uv * sry + ru * svy + rv * suy);
            spy = a.dy * fma(rho_g, a.gy, -rty) - (v * v * sry + T(2) * rv * svy) -
                  a.dy_over_dx * (uv * srx + rv * sux + ru * svx);
        } else if (a.gradp == kGradSplitMinmod || a.gradp == kGradSplitSuperbee) {
            // Qian et al. split (Sec. 2.3.2): limit the kinematic part of the
            // one-sided pressure differences, add the cell's hydrostatic
            // slope back; gravity reversed in wall ghosts as for Eq. new_gradp
            const int gi = x0 + li - 1, gj = y0 + lj - 1;
            const T sg = wall_ghost_sign<T>(gi, gj, nx, ny, a.bc);
            const T gxs = a.gx * sg, gys = a.gy * sg;
            spx = limiter(P[e] - P[c] - a.half_dx * (R[c] + R[e]) * gxs,
                          P[c] - P[wv] - a.half_dx * (R[wv] + R[c]) * gxs, kp) + a.dx * R[c] * gxs;
            spy = limiter(P[nn] - P[c] - a.half_dy * (R[c] + R[nn]) * gys,
                          P[c] - P[ss] - a.half_dy * (R[ss] + R[c]) * gys, kp) + a.dy * R[c] * gys;
        } else {
            spx = limiter(P[e] - P[c], P[c] - P[wv], kp);
            spy = limiter(P[nn] - P[c], P[c] - P[ss], kp);
        }
        sm.gx[0][k] = srx; sm.gx[1][k] = sux; sm.gx[2][k] = svx; sm.gx[3][k] = spx;
        sm.gy[0][k] = sry; sm.gy[1][k] = suy; sm.gy[2][k] = svy; sm.gy[3][k] = spy;
    }
    __syncthreads();

    // ---- 3. face states and Osher fluxes ----
    // The faces are dealt out so that the four SM sub-partitions get equal
    // numbers of warp-passes (the FP64 pipe, not issue, bounds this loop, and
    // a pass costs the same with idle lanes).  The warps of a CTA sit on
    // contiguous slots, so warps w and w + 4 share a sub-partition; group
    // w mod 4 takes faces [32 P g, 32 P (g + 1)), P = ceil(F / 128), in
    // passes of 32 shared round-robin by its warps.  The plain strided loop
    // gives the first warps an extra pass when the warp count is not a
    // multiple of 4 (32x14 tiles: 9 warp-passes on two sub-partitions
    // against 8 here).
    constexpr int NF = S::NXF + S::NYF, NW = NT / 32, FP = (NF + 127) / 128;
    static_assert(NW >= 4, "face schedule needs four warps");
    const int fw = tid >> 5, fgrp = fw & 3;
    const int fwarps = (NW - fgrp + 3) >> 2;
    const int fbeg = fgrp * 32 * FP, fend = min(NF, fbeg + 32 * FP);
    for (int fq = fw >> 2; fbeg + 32 * fq < fend; fq += fwarps) {
        const int k = fbeg + 32 * fq + (tid & 31);
        if (k >= fend) continue;
        const bool isx = k < S::NXF;
        // face states: density, normal and tangential velocity (rotation,
        // Alg. 2: (u, v) on x-faces, (v, u) on y-faces), pressure
        T rL, nL, tL, pL, rR, nR, tR, pR;
        int fo;   // face index within its kind
        if (isx) {
            const int fi = k % (TX + 1), fj = k / (TX + 1);  // face between cells fi-1 and fi
            const int ga = (fj + 1) * GW + fi, gb = ga + 1;
            const int ca = (fj + 2) * RW + fi + 1, cb = ca + 1;
            rL = fma(T(0.5), sm.gx[0][ga], sm.w[0][ca]); rR = fma(T(-0.5), sm.gx[0][gb], sm.w[0][cb]);
            nL = fma(T(0.5), sm.gx[1][ga], sm.w[1][ca]); nR = fma(T(-0.5), sm.gx[1][gb], sm.w[1][cb]);
            tL = fma(T(0.5), sm.gx[2][ga], sm.w[2][ca]); tR = fma(T(-0.5), sm.gx[2][gb], sm.w[2][cb]);
            pL = fma(T(0.5), sm.gx[3][ga], sm.w[3][ca]); pR = fma(T(-0.5), sm.gx[3][gb], sm.w[3][cb]);
            fo = k;
        } else {
            const int kk = k - S::NXF;
            const int fi = kk % TX, fj = kk / TX;            // face between cells fj-1 and fj
            const int ga = fj * GW + fi + 1, gb = ga + GW;
            const int ca = (fj + 1) * RW + fi + 2, cb = ca + RW;
            rL = fma(T(0.5), sm.gy[0][ga], sm.w[0][ca]); rR = fma(T(-0.5), sm.gy[0][gb], sm.w[0][cb]);
            tL = fma(T(0.5), sm.gy[1][ga], sm.w[1][ca]); tR = fma(T(-0.5), sm.gy[1][gb], sm.w[1][cb]);
            nL = fma(T(0.5), sm.gy[2][ga], sm.w[2][ca]); nR = fma(T(-0.5), sm.gy[2][gb], sm.w[2][cb]);
            pL = fma(T(0.5), sm.gy[3][ga], sm.w[3][ca]); pR = fma(T(-0.5), sm.gy[3][gb], sm.w[3][cb]);
            fo = kk;
        }
        // one flux call for both kinds: no divergence where a warp holds both
        // (2F: the divergence below takes the 1/2)
        T F[4];
        riemann_flux<RS, T, true>(rL, nL, tL, pL, rR, nR, tR, pR, a.beta, a.inv_beta, F);
        T *fd = isx ? &sm.fx[0][fo] : &sm.fy[0][fo];
        const int fs = isx ? S::NXF : S::NYF;
        fd[0] = F[0];
        fd[fs] = isx ? F[1] : F[2];
        fd[2 * fs] = isx ? F[2] : F[1];
        fd[3 * fs] = F[3];
    }
    __syncthreads();

    // ---- 4. divergence + sources + point-implicit stage update ----
    const int li = tid % TX, lj = tid / TX;
    const int gi = x0 + li, gj = y0 + lj;
    const bool inside = (gi < nx) && (gj < ny);
    double sq[4] = {0.0, 0.0, 0.0, 0.0};
    if (inside) {
        const size_t g = (size_t)gj * nx + gi;
        const int fw = lj * (TX + 1) + li, fe = fw + 1;
        const int fs = lj * TX + li, fn = fs + TX;
        // fluxes are stored doubled: (2Fe - 2Fw) (1/(2 dx)) is (Fe - Fw)/dx exactly
        const T hidx = T(0.5) * a.inv_dx, hidy = T(0.5) * a.inv_dy;
        T div[4];
#pragma unroll
        for (int f = 0; f < 4; ++f)
            div[f] = (sm.fx[f][fe] - sm.fx[f][fw]) * hidx + (sm.fy[f][fn] - sm.fy[f][fs]) * hidy;
        const T r0 = q0[0][g], m0 = q0[1][g], n0 = q0[2][g], p0 = q0[3][g];
        // At stage 1 the input Q^{s-1} is Q^{m} itself, so the cell's W (never
        // a folded ghost here) holds the 1/rho, u and v of Q^{m}, and the ring
        // already holds its momenta's real-time terms: taken as they are, the
        // same values to the last bit.
        const bool from_tile = a.stage == 1;
        const int ct = (lj + 2) * RW + (li + 2), cr = (lj + 1) * GW + (li + 1);
        T rt0 = T(0), rt1 = T(0), rt2 = T(0);
        if (a.realtime) {
            if (reuse_now) {
                rt0 = a.aux[1][g];
                rt1 = a.aux[2][g];
                rt2 = a.aux[3][g];
            } else {
                rt0 = realtime_term(a, r0, 0, g, inv_dt);
                if (from_tile && need_rt) {
                    rt1 = sm.rt[0][cr];
                    rt2 = sm.rt[1][cr];
                } else {
                    rt1 = realtime_term(a, m0, 1, g, inv_dt);
                    rt2 = realtime_term(a, n0, 2, g, inv_dt);
                }
                if (a.reuse) {
                    a.aux[1][g] = rt0;
                    a.aux[2][g] = rt1;
                    a.aux[3][g] = rt2;
                }
            }
        }
        const T b0 = -div[0] - rt0;
        const T b1 = -div[1] - rt1 + r0 * a.gx;
        const T b2 = -div[2] - rt2 + r0 * a.gy;
        const T b3 = -div[3];
        // pseudo-time step from Q^{m} (Sec. 2.2.3)
        T dtau;
        if (a.local_dtau && reuse_now) {
            dtau = a.aux[0][g];
        } else if (a.local_dtau) {
            T ir, u, v;
            if (from_tile) {
                ir = sm.wir[ct];
                u = sm.w[1][ct];
                v = sm.w[2][ct];
            } else {
                ir = Ar<T>::rcp(r0);
                u = m0 * ir;
                v = n0 * ir;
            }
            const T fb = T(4) * a.beta * ir;
            // square roots as x / sqrt(x) and quotients as products with a
            // rounded reciprocal: a few ulps, far inside the 1e-11 bar
            T cx, cy, unused;
            Ar<T>::sqrt_rsqrt(u * u + fb, cx, unused);
            Ar<T>::sqrt_rsqrt(v * v + fb, cy, unused);
            const T den = T(0.5) * (fabs(u) + cx) * a.dy + T(0.5) * (fabs(v) + cy) * a.dx;
            dtau = a.cfl_area * Ar<T>::rcp(den);
            if (a.reuse) a.aux[0][g] = dtau;
        } else {
            dtau = T(global_dtau(ctl));
        }
        const T api = T(1) + a.B[0] * a.alpha * dtau * inv_dt;   // Eq. point_implicit
        const T coef = (a.alpha * dtau) * Ar<T>::rcp(api);
        const T coef_p = a.alpha_pi_p_row ? coef : a.alpha * dtau;
        qout[0][g] = r0 + coef * b0;
        qout[1][g] = m0 + coef * b1;
        qout[2][g] = n0 + coef * b2;
        qout[3][g] = p0 + a.beta * coef_p * b3;
        if (a.stage == 1) {
            const double pb = double(a.beta) * double(b3);
            sq[0] = double(b0) * double(b0);
            sq[1] = double(b1) * double(b1);
            sq[2] = double(b2) * double(b2);
            sq[3] = pb * pb;
        }
    }
    if (a.stage == 1) {
        // deterministic block reduction of the squared bracket (FP64)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            double v = sq[f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) sm.red[f][tid >> 5] = v;
        }
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += sm.red[tid][w];
            a.partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + tid] = s;
        }
    }
}

// Global pseudo-time step option: min over cells of the local step
// (Sec. 2.2.3), from Q^{m}.  Positive doubles order like their bit patterns.
template <typename T>
__global__ void dtau_min_kernel(const SweepArgs<T> a) {
    pdl_trigger();
    pdl_wait();
    const Ctl *ctl = a.ctl;
    if (ctl->done) return;
    const T *const *q = a.buf[ctl->cur];
    const size_t N = (size_t)a.nx * a.ny;
    double mn = INFINITY;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        const T r0 = q[0][g];
        const T ir = Ar<T>::rcp(r0);
        const T u = q[1][g] * ir, v = q[2][g] * ir, fb = T(4) * a.beta * ir;
        const T cx = Ar<T>::sqrt_(u * u + fb), cy = Ar<T>::sqrt_(v * v + fb);
        const T den = T(0.5) * (fabs(u) + cx) * a.dy + T(0.5) * (fabs(v) + cy) * a.dx;
        mn = fmin(mn, double(Ar<T>::div(a.cfl_area, den)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0)
        atomicMin(&a.ctl->dtau_bits, (unsigned long long)__double_as_longlong(mn));
}

// Global real-time step (Sec. 2.2.4): min over cells of
// CFL_t |Omega| / (|u| dS_x + |v| dS_y), from buffer `cur`; +inf at rest.
template <typename T>
__global__ void realtime_dt_kernel(const SweepArgs<T> a, int cur, double cfl_area, unsigned long long *out) {
    const T *const *q = a.buf[cur];
    const size_t N = (size_t)a.nx * a.ny;
    double mn = INFINITY;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        const double ir = 1.0 / double(q[0][g]);
        const double u = double(q[1][g]) * ir, v = double(q[2][g]) * ir;
        const double den = fabs(u) * double(a.dy) + fabs(v) * double(a.dx);
        mn = fmin(mn, cfl_area / den);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, (unsigned long long)__double_as_longlong(mn));
}

// Start of a physical step: Q^n <- Q (Alg. 1) and reset of the control block.
template <typename T>
__global__ void begin_step_kernel(const SweepArgs<T> a, double dt, double tol, int max_iters, double tau_end) {
    Ctl *ctl = a.ctl;
    const int cur = ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        // older levels move back one step: Q^{n-2} <- Q^{n-1} <- Q^n
        if (a.lev2[0])
#pragma unroll
            for (int f = 0; f < 3; ++f) a.lev2[f][g] = a.lev1[f][g];
        if (a.lev1[0])
#pragma unroll
            for (int f = 0; f < 3; ++f) a.lev1[f][g] = a.lev[f][g];
#pragma unroll
        for (int f = 0; f < 4; ++f) a.lev[f][g] = a.buf[cur][f][g];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iter = 0;
        ctl->done = 0;
        ctl->status = 1;
        ctl->max_iters = max_iters;
        ctl->fixed = tol < 0.0;
        ctl->tol = tol;
        ctl->dt = dt;
        ctl->inv_dt = 1.0 / dt;
        ctl->dtau_bits = 0x7ff0000000000000ull;  // +inf
        ctl->tau = 0.0;
        ctl->tau_end = tau_end;
    }
}

// End of a pseudo-iteration (kEndLanes threads, one CTA).  Sets the graph's
// while-condition when launched inside a captured loop.
static __global__ void __launch_bounds__(kEndLanes)
end_iteration_kernel(Ctl *ctl, const double *partials, const IterEnd e) {
    pdl_trigger();
    pdl_wait();
    if (ctl->done) {
        if (e.use_cond && threadIdx.x == 0) cudaGraphSetConditional(e.cond, 0);
        return;
    }
    end_iteration(ctl, partials, e);
}

}  // namespace acgb
