// ac_kernels_mixed.cuh -- the fused stage sweep in the mixed form:
// FP32 flux, reconstruction and update arithmetic; FP64 real-time level,
// hydrostatic reference pressure and residual sums.
//
// Storage (per cell):
//   qn32[3]   FP32 copy of the real-time level Q^n = (rho, rho u, rho v)
//   d[b][4]   three rotating FP32 buffers: dQ = Q - Q^n for rho, rho u, rho v
//             and p' = p - p_ref
//   rho_ref   FP32 reference density; p_ref (FP64, host side) is its discrete
//             hydrostatic column integral along y
//   dref      FP32 jump p_ref(i) - p_ref(i-1) across the west x-face
//   q64[3]    FP64 real-time level, advanced once per physical step
//             (Q^{n+1} = Q^n + dQ in FP64: the level accumulation)
//
// Why this is exact algebra and not an approximation of the scheme:
//   * The real-time term of Eq. bdf (Backward-Euler) is (Q^{m} - Q^n)/dt =
//     dQ^{m}/dt: no cancellation between two large FP32 numbers.
//   * Every Riemann flux here is affine in a pressure offset common to the
//     two face states (|A| does not depend on p), so each face may be solved
//     with p'' = p - P_f for any face constant P_f, adding P_f back to the
//     normal momentum flux.  On y-faces P_f is the hydrostatic face value of
//     the reference, which the cells on both sides agree on (wall ghosts
//     mirror p_ref and reverse gravity, Sec. 2.5); the divergence of those
//     face values is exactly -rho_ref g_y, which cancels the reference part
//     of the body force, leaving (rho - rho_ref) g_y.  On x-faces P_f is the
//     mean of the two cells' references and the jump dref enters the face
//     states; the divergence of the means is -(dref_e + dref_w)/(2 dx).
//   * The new pressure gradient (Eq. new_gradp) does not depend on p; only
//     its gravity term changes to (rho - rho_ref) g_y once the reference
//     slope rho_ref g_y is moved into P_f.
// With zero rho_ref and dref (used when the y sides are not both walls or
// the pressure gradient is limited from p) this is the plain FP32 sweep.
#pragma once

#include "ac_kernels.cuh"

namespace acgb {

struct MixedArgs {
    int nx, ny;
    int bc[4];
    int gradp, limiter_k, realtime, local_dtau, alpha_pi_p_row;
    int stage, s_max;
    float alpha;
    float dx, dy, half_dx, half_dy, inv_dx, inv_dy, dx_over_dy, dy_over_dx;
    float beta, inv_beta, gx, gy;
    float cfl_area;
    float *d[3][4];        // dQ (rho, rho u, rho v) and p'
    float *qn32[3];        // FP32 copy of Q^n
    const float *rho_ref;  // reference density
    const float *dref;     // reference jump across the west x-face
    float *lev_p;          // p' at the start of the physical step
    double *q64[3];        // FP64 real-time level
    double *partials;
    Ctl *ctl;
};

template <int TX, int TY>
struct MixedSmem {
    static constexpr int RW = TX + 4, RH = TY + 4;
    static constexpr int GW = TX + 2, GH = TY + 2;
    static constexpr int NXF = (TX + 1) * TY;
    static constexpr int NYF = TX * (TY + 1);
    float w[4][RW * RH];       // rho, u, v, p'
    float rt[2][GW * GH];      // frozen real-time term of rho u, rho v
    float rr[GW * GH];         // reference density on the ring
    float gx[4][GW * GH];      // half slopes along x
    float gy[4][GW * GH];      // half slopes along y (p: of p - p_ref)
    float fx[4][NXF];
    float fy[4][NYF];
    float dxf[NXF];            // reference jump on each x-face
    double red[4][32];
};

// Gather Q^{s-1} = Q^n + dQ^{s-1} of one cell into W (interior or folded).
struct CellLoad {
    const float *__restrict__ qn0, *__restrict__ qn1, *__restrict__ qn2;
    const float *__restrict__ d0, *__restrict__ d1, *__restrict__ d2, *__restrict__ d3;
    __device__ __forceinline__ void operator()(int s, bool fx, bool fy, float &r, float &u, float &v,
                                               float &p) const {
        r = __ldg(qn0 + s) + d0[s];
        float m = __ldg(qn1 + s) + d1[s];
        float n = __ldg(qn2 + s) + d2[s];
        m = fx ? -m : m;
        n = fy ? -n : n;
        const float ir = Ar<float>::rcp(r);
        u = m * ir;
        v = n * ir;
        p = d3[s];
    }
};

// One TX x TY tile (tile coordinates bx, by) of one stage of one tank, by
// a CTA of NT threads (NT divides TX*TY; several cells per thread in the
// update when NT < TX*TY).  `partial` receives the tile's four residual
// partial sums at stage 1.  Shared by the single-tank and batched kernels.
template <int TX, int TY, int NT>
__device__ __forceinline__ void mixed_tile(const MixedArgs &a, int bx, int by, double *partial,
                                           unsigned char *smem_raw) {
    using S = MixedSmem<TX, TY>;
    static_assert((TX * TY) % NT == 0 && NT % 32 == 0, "tile/thread shape");
    S &sm = *reinterpret_cast<S *>(smem_raw);
    constexpr int RW = S::RW, RH = S::RH, GW = S::GW, GH = S::GH;

    const Ctl *ctl = a.ctl;
    int in, out;
    const int cur = ctl->cur;
    stage_buffers(cur, a.stage, in, out);
    const float *const *din = a.d[in];
    const float *const *d0 = a.d[cur];
    float *const *dout = a.d[out];
    const float inv_dt = a.realtime ? float(ctl->inv_dt) : 0.0f;

    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    // halo entirely inside the domain: no ghost folding for this tile
    const bool interior = (x0 >= 2) && (x0 + TX + 2 <= nx) && (y0 >= 2) && (y0 + TY + 2 <= ny);
    const CellLoad ld{a.qn32[0], a.qn32[1], a.qn32[2], din[0], din[1], din[2], din[3]};

    // ---- 1. stage Q^{s-1} = Q^n + dQ^{s-1} (+ halo) as W = (rho, u, v, p') ----
    if (interior) {
        const int base = (y0 - 2) * nx + (x0 - 2);
        for (int k = tid; k < RW * RH; k += NT) {
            const int rr = k / RW, cc = k - rr * RW;
            float r, u, v, p;
            ld(base + rr * nx + cc, false, false, r, u, v, p);
            sm.w[0][k] = r; sm.w[1][k] = u; sm.w[2][k] = v; sm.w[3][k] = p;
        }
    } else {
        for (int k = tid; k < RW * RH; k += NT) {
            const int rr = k / RW, cc = k - rr * RW;
            int nfx, tfx, nfy, tfy;
            const int si = fold_axis(x0 + cc - 2, nx, a.bc[0], a.bc[1], nfx, tfx);
            const int sj = fold_axis(y0 + rr - 2, ny, a.bc[2], a.bc[3], nfy, tfy);
            float r, u, v, p;
            ld(sj * nx + si, (nfx + tfy) & 1, (nfy + tfx) & 1, r, u, v, p);
            sm.w[0][k] = r; sm.w[1][k] = u; sm.w[2][k] = v; sm.w[3][k] = p;
        }
    }
    const bool new_gradp = (a.gradp == kGradNew);
    const bool need_rt = new_gradp && a.realtime;
    if (new_gradp) {
        const float *__restrict__ e1 = d0[1];
        const float *__restrict__ e2 = d0[2];
        const float *__restrict__ rref = a.rho_ref;
        for (int k = tid; k < GW * GH; k += NT) {
            const int rr = k / GW, cc = k - rr * GW;
            int s, fx = 0, fy = 0;
            if (interior) {
                s = (y0 + rr - 1) * nx + (x0 + cc - 1);
            } else {
                int nfx, tfx, nfy, tfy;
                const int si = fold_axis(x0 + cc - 1, nx, a.bc[0], a.bc[1], nfx, tfx);
                const int sj = fold_axis(y0 + rr - 1, ny, a.bc[2], a.bc[3], nfy, tfy);
                s = sj * nx + si;
                fx = (nfx + tfy) & 1;
                fy = (nfy + tfx) & 1;
            }
            if (need_rt) {
                const float rx = e1[s] * inv_dt;   // (Q^{m} - Q^n)/dt of rho u
                const float ry = e2[s] * inv_dt;
                sm.rt[0][k] = fx ? -rx : rx;
                sm.rt[1][k] = fy ? -ry : ry;
            }
            sm.rr[k] = __ldg(rref + s);
        }
    }
    __syncthreads();

    // ---- 2. limited half slopes and pressure gradient on the ring ----
    const float klim = float(a.limiter_k);
    const float kp = (a.gradp == kGradSuperbee) ? 2.0f : 1.0f;
    for (int k = tid; k < GW * GH; k += NT) {
        const int lj = k / GW, li = k - lj * GW;
        const int c = (lj + 1) * RW + (li + 1);
        const int e = c + 1, wv = c - 1, nn = c + RW, ss = c - RW;
        const float *R = sm.w[0], *U = sm.w[1], *V = sm.w[2], *P = sm.w[3];
        float hrx, hry, hux, huy, hvx, hvy;
        if (a.limiter_k == 1) {
            hrx = half_minmod(R[e] - R[c], R[c] - R[wv]);
            hry = half_minmod(R[nn] - R[c], R[c] - R[ss]);
            hux = half_minmod(U[e] - U[c], U[c] - U[wv]);
            huy = half_minmod(U[nn] - U[c], U[c] - U[ss]);
            hvx = half_minmod(V[e] - V[c], V[c] - V[wv]);
            hvy = half_minmod(V[nn] - V[c], V[c] - V[ss]);
        } else {
            hrx = 0.5f * limiter(R[e] - R[c], R[c] - R[wv], klim);
            hry = 0.5f * limiter(R[nn] - R[c], R[c] - R[ss], klim);
            hux = 0.5f * limiter(U[e] - U[c], U[c] - U[wv], klim);
            huy = 0.5f * limiter(U[nn] - U[c], U[c] - U[ss], klim);
            hvx = 0.5f * limiter(V[e] - V[c], V[c] - V[wv], klim);
            hvy = 0.5f * limiter(V[nn] - V[c], V[c] - V[ss], klim);
        }
        float hpx, hpy;
        if (new_gradp) {
            float sg = 1.0f;
            if (!interior) sg = wall_ghost_sign<float>(x0 + li - 1, y0 + lj - 1, nx, ny, a.bc);
            const float rho = R[c], u = U[c], v = V[c];
            const float rtx = need_rt ? sm.rt[0][k] : 0.0f;
            const float rty = need_rt ? sm.rt[1][k] : 0.0f;
            const float ru = rho * u, rv = rho * v, uv = u * v;
            hpx = -a.half_dx * rtx - (u * u * hrx + 2.0f * ru * hux) -
                  a.dx_over_dy * (uv * hry + ru * hvy + rv * huy) + a.half_dx * rho * a.gx * sg;
            // slope of p - p_ref: the reference slope rho_ref g_y is removed
            hpy = -a.half_dy * rty - (v * v * hry + 2.0f * rv * hvy) -
                  a.dy_over_dx * (uv * hrx + rv * hux + ru * hvx) + a.half_dy * (rho - sm.rr[k]) * a.gy * sg;
        } else {
            hpx = 0.5f * limiter(P[e] - P[c], P[c] - P[wv], kp);
            hpy = 0.5f * limiter(P[nn] - P[c], P[c] - P[ss], kp);
        }
        sm.gx[0][k] = hrx; sm.gx[1][k] = hux; sm.gx[2][k] = hvx; sm.gx[3][k] = hpx;
        sm.gy[0][k] = hry; sm.gy[1][k] = huy; sm.gy[2][k] = hvy; sm.gy[3][k] = hpy;
    }
    __syncthreads();

    // ---- 3. face states and Osher fluxes (pressures relative to P_f) ----
    const bool per_x = (a.bc[0] == kPeriodic);
    for (int k = tid; k < S::NXF + S::NYF; k += NT) {
        float F[4];
        if (k < S::NXF) {
            const int fj = k / (TX + 1), fi = k - fj * (TX + 1);
            const int gi = x0 + fi, gj = y0 + fj;
            float jump = 0.0f;
            if (gj < ny) {
                if (gi < nx) jump = __ldg(a.dref + gj * nx + gi);
                else if (gi == nx && per_x) jump = __ldg(a.dref + gj * nx);
            }
            sm.dxf[k] = jump;
            const int ga = (fj + 1) * GW + fi, gb = ga + 1;
            const int ca = (fj + 2) * RW + fi + 1, cb = ca + 1;
            const float rL = sm.w[0][ca] + sm.gx[0][ga], rR = sm.w[0][cb] - sm.gx[0][gb];
            const float uL = sm.w[1][ca] + sm.gx[1][ga], uR = sm.w[1][cb] - sm.gx[1][gb];
            const float vL = sm.w[2][ca] + sm.gx[2][ga], vR = sm.w[2][cb] - sm.gx[2][gb];
            const float pL = sm.w[3][ca] + sm.gx[3][ga] - 0.5f * jump;
            const float pR = sm.w[3][cb] - sm.gx[3][gb] + 0.5f * jump;
            osher_flux<float>(rL, uL, vL, pL, rR, uR, vR, pR, a.beta, a.inv_beta, F);
            sm.fx[0][k] = F[0]; sm.fx[1][k] = F[1]; sm.fx[2][k] = F[2]; sm.fx[3][k] = F[3];
        } else {
            const int kk = k - S::NXF;
            const int fj = kk / TX, fi = kk - fj * TX;
            const int ga = fj * GW + fi + 1, gb = ga + GW;
            const int ca = (fj + 1) * RW + fi + 2, cb = ca + RW;
            const float rL = sm.w[0][ca] + sm.gy[0][ga], rR = sm.w[0][cb] - sm.gy[0][gb];
            const float uL = sm.w[1][ca] + sm.gy[1][ga], uR = sm.w[1][cb] - sm.gy[1][gb];
            const float vL = sm.w[2][ca] + sm.gy[2][ga], vR = sm.w[2][cb] - sm.gy[2][gb];
            const float pL = sm.w[3][ca] + sm.gy[3][ga], pR = sm.w[3][cb] - sm.gy[3][gb];
            osher_flux<float>(rL, vL, uL, pL, rR, vR, uR, pR, a.beta, a.inv_beta, F);
            sm.fy[0][kk] = F[0]; sm.fy[1][kk] = F[2]; sm.fy[2][kk] = F[1]; sm.fy[3][kk] = F[3];
        }
    }
    __syncthreads();

    // ---- 4. divergence + sources + point-implicit update of dQ and p' ----
    float sq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int cell = tid; cell < TX * TY; cell += NT) {
        const int lj = cell / TX, li = cell - lj * TX;
        const int gi = x0 + li, gj = y0 + lj;
        if (gi >= nx || gj >= ny) continue;
        const int g = gj * nx + gi;
        const int fw = lj * (TX + 1) + li, fe = fw + 1;
        const int fs = cell, fn = fs + TX;
        float div[4];
#pragma unroll
        for (int f = 0; f < 4; ++f)
            div[f] = (sm.fx[f][fe] - sm.fx[f][fw]) * a.inv_dx + (sm.fy[f][fn] - sm.fy[f][fs]) * a.inv_dy;
        const float e0 = d0[0][g], e1 = d0[1][g], e2 = d0[2][g], p0 = d0[3][g];
        const float r0 = __ldg(a.qn32[0] + g) + e0;
        const float m0 = __ldg(a.qn32[1] + g) + e1;
        const float n0 = __ldg(a.qn32[2] + g) + e2;
        const float rt0 = e0 * inv_dt, rt1 = e1 * inv_dt, rt2 = e2 * inv_dt;
        // reference force: -(divergence of the x-face reference means)
        const float sref = -0.5f * (sm.dxf[fe] + sm.dxf[fw]) * a.inv_dx;
        const float b0 = -div[0] - rt0;
        const float b1 = -div[1] - rt1 + r0 * a.gx + sref;
        const float b2 = -div[2] - rt2 + (r0 - __ldg(a.rho_ref + g)) * a.gy;
        const float b3 = -div[3];
        float dtau;
        if (a.local_dtau) {
            const float ir = Ar<float>::rcp(r0);
            const float u = m0 * ir, v = n0 * ir, fb = 4.0f * a.beta * ir;
            const float u2 = u * u + fb, v2 = v * v + fb;
            const float cx = u2 * rsqrtf(u2), cy = v2 * rsqrtf(v2);
            const float den = 0.5f * (fabsf(u) + cx) * a.dy + 0.5f * (fabsf(v) + cy) * a.dx;
            dtau = __fdividef(a.cfl_area, den);
        } else {
            dtau = float(__longlong_as_double((long long)ctl->dtau_bits));
        }
        const float adt = a.alpha * dtau;
        const float coef = __fdividef(adt, 1.0f + adt * inv_dt);   // Eq. point_implicit, B0 = 1
        const float coef_p = a.alpha_pi_p_row ? coef : adt;
        dout[0][g] = e0 + coef * b0;
        dout[1][g] = e1 + coef * b1;
        dout[2][g] = e2 + coef * b2;
        dout[3][g] = p0 + a.beta * coef_p * b3;
        if (a.stage == 1) {
            const float pb = a.beta * b3;
            sq[0] += b0 * b0; sq[1] += b1 * b1; sq[2] += b2 * b2; sq[3] += pb * pb;
        }
    }
    if (a.stage == 1) {
        // per-warp sums in FP32, block and grid sums in FP64
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            float v = sq[f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) sm.red[f][tid >> 5] = double(v);
        }
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += sm.red[tid][w];
            partial[tid] = s;
        }
    }
}

template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
stage_kernel_mixed(const MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.ctl->done) return;
    mixed_tile<TX, TY, NT>(a, blockIdx.x, blockIdx.y,
                           a.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4, smem_raw);
}

// Global pseudo-time step option for the mixed form.
static __global__ void dtau_min_kernel_mixed(const MixedArgs a) {
    const Ctl *ctl = a.ctl;
    if (ctl->done) return;
    const float *const *d = a.d[ctl->cur];
    const size_t N = (size_t)a.nx * a.ny;
    double mn = INFINITY;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        const float r0 = a.qn32[0][g] + d[0][g];
        const float ir = Ar<float>::rcp(r0);
        const float u = (a.qn32[1][g] + d[1][g]) * ir, v = (a.qn32[2][g] + d[2][g]) * ir;
        const float fb = 4.0f * a.beta * ir;
        const float cx = sqrtf(u * u + fb), cy = sqrtf(v * v + fb);
        const float den = 0.5f * (fabsf(u) + cx) * a.dy + 0.5f * (fabsf(v) + cy) * a.dx;
        mn = fmin(mn, double(a.cfl_area / den));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0)
        atomicMin(&a.ctl->dtau_bits, (unsigned long long)__double_as_longlong(mn));
}

// Start of a physical step in the mixed form: the FP64 level absorbs the
// increments (Q^n <- Q^n + dQ, Alg. 1), its FP32 copy is refreshed, the
// increments restart from zero, and p' is kept for a restore.
static __global__ void begin_step_kernel_mixed(const MixedArgs a, double dt, double tol, int max_iters) {
    Ctl *ctl = a.ctl;
    const int cur = ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const double q = a.q64[f][g] + double(a.d[cur][f][g]);
            a.q64[f][g] = q;
            a.qn32[f][g] = float(q);
            a.d[cur][f][g] = 0.0f;
        }
        a.lev_p[g] = a.d[cur][3][g];
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
        ctl->dtau_bits = 0x7ff0000000000000ull;
    }
}

// After a non-finite residual: back to the state at the start of the step.
static __global__ void restore_kernel_mixed(const MixedArgs a) {
    const int cur = a.ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        a.d[cur][0][g] = 0.0f;
        a.d[cur][1][g] = 0.0f;
        a.d[cur][2][g] = 0.0f;
        a.d[cur][3][g] = a.lev_p[g];
    }
}

}  // namespace acgb
