// ac_kernels_mixed.cuh -- the fused stage sweep in the mixed form:
// FP32 flux, reconstruction and update arithmetic; FP64 real-time levels,
// hydrostatic reference pressure and residual sums.
//
// Storage (per cell; the two 16-byte records are read with one vector load):
//   qn        (FP32 copy of the real-time level Q^n = (rho, rho u, rho v),
//             reference density rho_ref)
//   d[b]      three rotating buffers of (dQ = Q - Q^n for rho, rho u, rho v,
//             dp = p - p^n), FP32: every field is an increment over its
//             level, small within a physical step
//   q64[4]    FP64 levels Q^n and p^n, advanced once per physical step
//             (Q^{n+1} = Q^n + dQ in FP64: the level accumulation)
//   pref64    FP64 static reference pressure: the discrete hydrostatic
//             column of rho_ref (none: zero)
//   jmp       FP32 jumps of the level across each cell's west and south
//             faces, (jx, jy) in one 8-byte record: jx = p^n(i) - p^n(i-1),
//             jy = q^n(j) - q^n(j-1) with q^n = p^n - p_ref, formed in FP64
//             at the start of each step (and at each rebase)
//
// Why this is exact algebra and not an approximation of the scheme:
//   * The real-time term of Eq. bdf is (B0 Q^{m} + B1 Q^n + B2 Q^{n-1} +
//     B3 Q^{n-2})/dt; the coefficients sum to zero, so it equals
//     (B0 dQ^{m} - B2 D1 - B3 D2)/dt with D1 = Q^n - Q^{n-1}, D2 = Q^n -
//     Q^{n-2}: small FP32 differences, no cancellation between large FP32
//     numbers (Backward-Euler: dQ^{m}/dt).
//   * Every Riemann flux here is affine in a pressure offset common to the
//     two face states (|A| does not depend on p), so each face may be solved
//     with p'' = p - P_f for any face constant P_f, adding P_f back to the
//     normal momentum flux.  On x-faces P_f is the mean of the two cells'
//     levels p^n; the states then carry dp -+ jx/2 and the divergence of
//     the means is -(jx_e + jx_w)/(2 dx).  On y-faces P_f is the reference's
//     hydrostatic face value, which the cells on both sides agree on (wall
//     ghosts mirror p_ref and reverse gravity, Sec. 2.5) and whose divergence
//     is exactly -rho_ref g_y, cancelling the reference part of the body
//     force and leaving (rho - rho_ref) g_y, plus the mean of the two cells'
//     q^n, whose divergence is -(jy_n + jy_s)/(2 dy).
//   * The new pressure gradient (Eq. new_gradp) does not depend on p; only
//     its gravity term changes to (rho - rho_ref) g_y once the reference
//     slope rho_ref g_y is moved into P_f.
// FP32 then holds only increments and cell-to-cell jumps, never a pressure
// of the size of the tank's hydrostatic head.  With a limited pressure
// gradient (Sec. 2.3.1-2.3.2) the slopes need pressure differences, so there
// the FP32 record holds p itself (plevel = 0: no level, zero jumps).
#pragma once

#include "ac_kernels.cuh"

namespace acgb {

struct MixedArgs {
    int nx, ny;
    int bc[4];
    int gradp, limiter_k, realtime, local_dtau, alpha_pi_p_row;
    int riemann;           // kOsher / kBassi / kRoe
    int stage, s_max;
    float alpha;
    float dx, dy, half_dx, half_dy, inv_dx, inv_dy, dx_over_dy, dy_over_dx;
    float nh_inv_dx, nh_inv_dy;   // -1/(2 dx), -1/(2 dy)
    float beta, inv_beta, gx, gy;
    float cfl_area;
    int plevel;            // 1: pressure as dp over the FP64 level p^n; 0: the record holds p
    float4 *d[3];          // per cell (dQ of rho, rho u, rho v; dp or p), three rotating buffers
    float4 *qn;            // per cell (FP32 Q^n of rho, rho u, rho v; rho_ref)
    float2 *jmp;           // per cell (level jump across the west face, across the south face)
    float *lev_p;          // p at the start of the physical step (plevel = 0, for a restore)
    float *dtau;           // per cell local pseudo-time step of the pseudo-iteration: written by stage 1 of
                           // the column-strip sweep with the default options, read by its later stages
    float *D1[3], *D2[3];  // Q^n - Q^{n-1}, Q^n - Q^{n-2} (rho, rho u, rho v) for BDF2/BDF3
    int order;             // backward-difference order used in this step (1..3)
    float B0, B2, B3;      // its coefficients (Table BDF); B1 = -(B0 + B2 + B3)
    double *q64[4];        // FP64 real-time levels of rho, rho u, rho v and p (p: zero when plevel = 0)
    double *p64_step;      // FP64 pressure level at the start of the physical step (for a restore)
    const double *pref64;  // FP64 reference pressure (null: none)
    double *partials;
    Ctl *ctl;
};

// Exact FP32 -> FP64 conversion with integer instructions (exponent rebias,
// mantissa shift), off GB300's FP64 unit, which runs at 1/64 of the FP32
// rate.  FP32 subnormals (below 1.2e-38) become 0; infinities and NaNs stay
// what they are, so a non-finite residual is still seen.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
    const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
    const unsigned long long ex = e == 0u ? 0ull : (e == 255u ? 0x7ffull : (unsigned long long)(e + 896u));
    return __longlong_as_double((long long)(sgn | (ex << 52) | (e == 0u ? 0ull : m)));
}

// Residual partial sums of the tile sweep (one or two cells per thread):
// each cell's stage-1 squares in FP32, and every sum from the warp's up in
// FP64 (the thread's values converted exactly).
struct SqTile {
    float x = 0.0f, y = 0.0f, z = 0.0f, w = 0.0f;
    __device__ __forceinline__ void add(float b0, float b1, float b2, float b3) {
        x = fmaf(b0, b0, x);
        y = fmaf(b1, b1, y);
        z = fmaf(b2, b2, z);
        w = fmaf(b3, b3, w);
    }
    __device__ __forceinline__ double get(int f) const {
        return f32_to_f64_exact(f == 0 ? x : f == 1 ? y : f == 2 ? z : w);
    }
};

// Residual partial sums of the column-strip sweep, where one lane adds the
// squares of up to 256 cells: compensated (Kahan) FP32 summation per lane,
// whose error stays within about two FP32 roundings of the lane's total
// whatever the number of cells (a plain FP32 sum of n squares can be off by
// n roundings), and FP64 for every sum across lanes, strips and the grid
// (lane_sum()).  On GB300 the FP64 unit runs at 1/64 of the FP32 rate; one
// FP64 accumulation per cell cost 18 % of a stage-1 strip launch.
struct SqKahan {
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    __device__ __forceinline__ void add(float b0, float b1, float b2, float b3) {
        const float q[4] = {b0 * b0, b1 * b1, b2 * b2, b3 * b3};
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const float y = __fsub_rn(q[f], c[f]);
            const float t = __fadd_rn(s[f], y);
            c[f] = __fsub_rn(__fsub_rn(t, s[f]), y);
            s[f] = t;
        }
    }
    // the lane's sum of field f, the compensation folded in FP64
    __device__ __forceinline__ double lane_sum(int f) const { return double(s[f]) - double(c[f]); }
};

template <int TX, int TY>
struct MixedSmem {
    static constexpr int RW = TX + 4, RH = TY + 4;
    static constexpr int GW = TX + 2, GH = TY + 2;
    static constexpr int NXF = (TX + 1) * TY;
    static constexpr int NYF = TX * (TY + 1);
    // one 16-byte vector per cell or face: a face or a cell reads all four
    // components with one shared-memory instruction
    float4 w[RW * RH];       // (rho, u, v, dp) of the tile + two-cell halo
    union {                  // aux is dead once the slopes exist; fx reuses it
        float4 aux[GW * GH]; // (RT of rho u, RT of rho v, rho_ref, -) on the ring
        float4 fx[NXF];      // x-face fluxes: (mass, x-mom, y-mom, p/beta)
    };
    float4 gx[GW * GH];      // half slopes along x: (rho, u, v, p)
    float4 gy[GW * GH];      // half slopes along y: (rho, u, v, p - p_ref)
    float4 fy[NYF];          // y-face fluxes
    float dxf[NXF];          // level jump on each x-face
    float dyf[NYF];          // level jump on each y-face
    double red[4][32];
};

// Gather Q^{s-1} = Q^n + dQ^{s-1} of one cell as W = (rho, u, v, dp).
struct CellLoad {
    const float4 *__restrict__ qn;
    const float4 *__restrict__ d;
    __device__ __forceinline__ float4 operator()(int s, bool fx, bool fy) const {
        const float4 q = __ldg(qn + s), e = d[s];
        const float r = q.x + e.x;
        float m = q.y + e.y;
        float n = q.z + e.z;
        m = fx ? -m : m;
        n = fy ? -n : n;
        const float ir = Ar<float>::rcp(r);
        return make_float4(r, m * ir, n * ir, e.w);
    }
};

__device__ __forceinline__ void limit_slopes(const float4 &c, const float4 &e, const float4 &w, const float4 &n,
                                             const float4 &s, int k, float klim, float &hrx, float &hry,
                                             float &hux, float &huy, float &hvx, float &hvy) {
    if (k == 1) {
        hrx = half_minmod(e.x - c.x, c.x - w.x);
        hry = half_minmod(n.x - c.x, c.x - s.x);
        hux = half_minmod(e.y - c.y, c.y - w.y);
        huy = half_minmod(n.y - c.y, c.y - s.y);
        hvx = half_minmod(e.z - c.z, c.z - w.z);
        hvy = half_minmod(n.z - c.z, c.z - s.z);
    } else {
        hrx = 0.5f * limiter(e.x - c.x, c.x - w.x, klim);
        hry = 0.5f * limiter(n.x - c.x, c.x - s.x, klim);
        hux = 0.5f * limiter(e.y - c.y, c.y - w.y, klim);
        huy = 0.5f * limiter(n.y - c.y, c.y - s.y, klim);
        hvx = 0.5f * limiter(e.z - c.z, c.z - w.z, klim);
        hvy = 0.5f * limiter(n.z - c.z, c.z - s.z, klim);
    }
}

// minmod(a, b) as the median of a, b and 0: zero where the signs differ,
// else the argument of smaller magnitude; min and max only (the ALU pipe, not
// the FMA pipe).
__device__ __forceinline__ float minmod_median(float a, float b) {
    return fmaxf(fminf(a, b), fminf(fmaxf(a, b), 0.0f));
}

// The column-strip sweep's limiter on whole slopes (the face states take
// half of a slope in one FMA; halving is exact, so the states equal those
// from half slopes), from the differences themselves: east/west along x,
// north/south along y (the sweep forms each difference once and passes it on
// to the neighbour that needs it as its other side).
__device__ __forceinline__ void limit_diffs(float er, float wr, float nr, float sr, float eu, float wu, float nu,
                                            float su, float ev, float wv, float nv, float sv, int k, float klim,
                                            float &srx, float &sry, float &sux, float &suy, float &svx, float &svy) {
    if (k == 1) {
        srx = minmod_median(er, wr); sry = minmod_median(nr, sr);
        sux = minmod_median(eu, wu); suy = minmod_median(nu, su);
        svx = minmod_median(ev, wv); svy = minmod_median(nv, sv);
    } else {
        srx = limiter(er, wr, klim); sry = limiter(nr, sr, klim);
        sux = limiter(eu, wu, klim); suy = limiter(nu, su, klim);
        svx = limiter(ev, wv, klim); svy = limiter(nv, sv, klim);
    }
}

// ---------------------------------------------------------------------------
// Per-cell and per-face arithmetic shared by the tile sweep and the
// column-strip sweep, so that both compute every value the same way.
// ---------------------------------------------------------------------------

// Half slope of p from the new pressure gradient (Eq. new_gradp) at a cell
// with W = Wc, the half slopes of rho, u, v, the frozen real-time terms of
// rho u, rho v (rtx, rty), the reference density and the ghost gravity sign.
__device__ __forceinline__ void new_gradp_half_slopes(const MixedArgs &a, const float4 &Wc, float hrx, float hry,
                                                      float hux, float huy, float hvx, float hvy, float rtx,
                                                      float rty, float rref, float sg, float &hpx, float &hpy) {
    const float rho = Wc.x, u = Wc.y, v = Wc.z;
    const float ru = rho * u, rv = rho * v, uv = u * v;
    hpx = -a.half_dx * rtx - (u * u * hrx + 2.0f * ru * hux) -
          a.dx_over_dy * (uv * hry + ru * hvy + rv * huy) + a.half_dx * rho * a.gx * sg;
    // slope of p - p_ref: the reference slope rho_ref g_y is removed
    hpy = -a.half_dy * rty - (v * v * hry + 2.0f * rv * hvy) -
          a.dy_over_dx * (uv * hrx + rv * hux + ru * hvx) + a.half_dy * (rho - rref) * a.gy * sg;
}

// The same, whole slope of p - p_ref (twice the above, exactly: every term is
// scaled by 2, with dx = 2 half_dx), from whole slopes of rho, u, v.
__device__ __forceinline__ void new_gradp_whole_slopes(const MixedArgs &a, const float4 &Wc, float srx, float sry,
                                                       float sux, float suy, float svx, float svy, float rtx,
                                                       float rty, float rref, float sg, float &spx, float &spy) {
    const float rho = Wc.x, u = Wc.y, v = Wc.z;
    const float ru = rho * u, rv = rho * v, uv = u * v;
    spx = -a.dx * rtx - (u * u * srx + 2.0f * ru * sux) -
          a.dx_over_dy * (uv * sry + ru * svy + rv * suy) + a.dx * rho * a.gx * sg;
    spy = -a.dy * rty - (v * v * sry + 2.0f * rv * svy) -
          a.dy_over_dx * (uv * srx + rv * sux + ru * svx) + a.dy * (rho - rref) * a.gy * sg;
}

// Face states between cells A (left/below) and B with half slopes SA, SB
// along the face normal: density, normal and tangential velocity (rotation,
// Alg. 2: (u, v) on x-faces, (v, u) on y-faces), pressure relative to the
// face constant; jump = level jump across the face.
struct FaceStates {
    float rL, nL, tL, pL, rR, nR, tR, pR;
};
__device__ __forceinline__ void x_face_states(const float4 &A, const float4 &B, const float4 &SA, const float4 &SB,
                                              float jump, FaceStates &f) {
    f.rL = A.x + SA.x; f.nL = A.y + SA.y; f.tL = A.z + SA.z; f.pL = A.w + SA.w - 0.5f * jump;
    f.rR = B.x - SB.x; f.nR = B.y - SB.y; f.tR = B.z - SB.z; f.pR = B.w - SB.w + 0.5f * jump;
}
__device__ __forceinline__ void y_face_states(const float4 &A, const float4 &B, const float4 &SA, const float4 &SB,
                                              float jump, FaceStates &f) {
    f.rL = A.x + SA.x; f.nL = A.z + SA.z; f.tL = A.y + SA.y; f.pL = A.w + SA.w - 0.5f * jump;
    f.rR = B.x - SB.x; f.nR = B.z - SB.z; f.tR = B.y - SB.y; f.pR = B.w - SB.w + 0.5f * jump;
}
// The same from whole slopes SA, SB (half of each taken in one FMA).
__device__ __forceinline__ void x_face_states_whole(const float4 &A, const float4 &B, const float4 &SA,
                                                    const float4 &SB, float jump, FaceStates &f) {
    f.rL = fmaf(0.5f, SA.x, A.x); f.nL = fmaf(0.5f, SA.y, A.y); f.tL = fmaf(0.5f, SA.z, A.z);
    f.pL = fmaf(0.5f, SA.w, A.w) - 0.5f * jump;
    f.rR = fmaf(-0.5f, SB.x, B.x); f.nR = fmaf(-0.5f, SB.y, B.y); f.tR = fmaf(-0.5f, SB.z, B.z);
    f.pR = fmaf(-0.5f, SB.w, B.w) + 0.5f * jump;
}
__device__ __forceinline__ void y_face_states_whole(const float4 &A, const float4 &B, const float4 &SA,
                                                    const float4 &SB, float jump, FaceStates &f) {
    f.rL = fmaf(0.5f, SA.x, A.x); f.nL = fmaf(0.5f, SA.z, A.z); f.tL = fmaf(0.5f, SA.y, A.y);
    f.pL = fmaf(0.5f, SA.w, A.w) - 0.5f * jump;
    f.rR = fmaf(-0.5f, SB.x, B.x); f.nR = fmaf(-0.5f, SB.z, B.z); f.tR = fmaf(-0.5f, SB.y, B.y);
    f.pR = fmaf(-0.5f, SB.w, B.w) + 0.5f * jump;
}

// The face flux from its states: (mass, x-momentum, y-momentum, p/beta).
template <int RS>
__device__ __forceinline__ float4 face_flux(const MixedArgs &a, bool isx, const FaceStates &f) {
    float F[4];
    riemann_flux<RS, float>(f.rL, f.nL, f.tL, f.pL, f.rR, f.nR, f.tR, f.pR, a.beta, a.inv_beta, F);
    return make_float4(F[0], isx ? F[1] : F[2], isx ? F[2] : F[1], F[3]);
}

// Divergence, sources and the point-implicit update of one cell (Eqs. RK2,
// point_implicit): writes dQ^s and dp^s at g and adds the stage-1 squared
// bracket to sq.  Fw, Fe, Fs, Fn: face fluxes, scaled by s_f (1 or 2), and
// fdx, fdy = 1/(s_f dx), 1/(s_f dy); jw, je, js, jn: level jumps of the
// west, east, south and north faces; src.cell(cell, g, ...) gives dQ^{m},
// dp^{m}, Q^n and rho_ref of the cell.  live = false: the arithmetic runs
// (a halo lane of the column-strip sweep, on a real cell's values) but
// nothing is stored or summed.  FAST: the default options (local pseudo-time
// step, alpha_PI on the p row) are compiled in rather than read.  DTM: 0
// forms the local pseudo-time step from Q^{m}; 1 forms it and stores it in
// a.dtau (stage 1); 2 takes it from dt_in, as stage 1 stored it (the later
// stages: Q^{m} is the same for every stage of a pseudo-iteration).
template <bool BDF, bool FAST = false, int DTM = 0, typename Src, typename Sq>
__device__ __forceinline__ void cell_update(const MixedArgs &a, float alpha, float inv_dt, float b0dt, bool stage1,
                                            float4 *dout, int cell, int g, const float4 &Fw, const float4 &Fe,
                                            const float4 &Fs, const float4 &Fn, float fdx, float fdy, float jw,
                                            float je, float js, float jn, const Src &src, Sq &sq,
                                            bool live = true, float dt_in = 0.0f) {
    const float div0 = (Fe.x - Fw.x) * fdx + (Fn.x - Fs.x) * fdy;
    const float div1 = (Fe.y - Fw.y) * fdx + (Fn.y - Fs.y) * fdy;
    const float div2 = (Fe.z - Fw.z) * fdx + (Fn.z - Fs.z) * fdy;
    const float div3 = (Fe.w - Fw.w) * fdx + (Fn.w - Fs.w) * fdy;
    float e0, e1, e2, p0, q0, q1, q2, rref;
    src.cell(cell, g, e0, e1, e2, p0, q0, q1, q2, rref);
    const float r0 = q0 + e0;
    const float m0 = q1 + e1;
    const float n0 = q2 + e2;
    // real-time terms (B0 Q^{m} - ...)/dt, for Backward-Euler B0/dt (b0dt) times Q^{m} - Q^n
    float rt0, rt1, rt2;
    if constexpr (BDF) {
        rt0 = a.B0 * e0;
        rt1 = a.B0 * e1;
        rt2 = a.B0 * e2;
        if (a.order >= 2) {
            rt0 -= a.B2 * a.D1[0][g];
            rt1 -= a.B2 * a.D1[1][g];
            rt2 -= a.B2 * a.D1[2][g];
        }
        if (a.order >= 3) {
            rt0 -= a.B3 * a.D2[0][g];
            rt1 -= a.B3 * a.D2[1][g];
            rt2 -= a.B3 * a.D2[2][g];
        }
        rt0 *= inv_dt;
        rt1 *= inv_dt;
        rt2 *= inv_dt;
    } else {
        rt0 = b0dt * e0;
        rt1 = b0dt * e1;
        rt2 = b0dt * e2;
    }
    // with the level force -(divergence of the face constants' level parts),
    // -(je + jw)/(2 dx) and -(jn + js)/(2 dy)
    const float b0 = -div0 - rt0;
    const float b1 = fmaf(je + jw, a.nh_inv_dx, fmaf(r0, a.gx, -div1 - rt1));
    const float b2 = fmaf(jn + js, a.nh_inv_dy, fmaf(r0 - rref, a.gy, -div2 - rt2));
    const float b3 = -div3;
    float dtau;
    if constexpr (DTM == 2) {
        dtau = dt_in;
    } else if (FAST || a.local_dtau) {
        const float ir = Ar<float>::rcp(r0);
        const float u = m0 * ir, v = n0 * ir, fb = 4.0f * a.beta * ir;
        const float u2 = u * u + fb, v2 = v * v + fb;
        const float cx = u2 * rsqrtf(u2), cy = v2 * rsqrtf(v2);
        const float den = 0.5f * (fabsf(u) + cx) * a.dy + 0.5f * (fabsf(v) + cy) * a.dx;
        dtau = __fdividef(a.cfl_area, den);
        if constexpr (DTM == 1) {
            if (live) a.dtau[g] = dtau;
        }
    } else {
        dtau = float(global_dtau(a.ctl));
    }
    const float adt = alpha * dtau;
    const float coef = __fdividef(adt, fmaf(adt, b0dt, 1.0f));   // Eq. point_implicit
    const float coef_p = (FAST || a.alpha_pi_p_row) ? coef : adt;
    if (live) dout[g] = make_float4(e0 + coef * b0, e1 + coef * b1, e2 + coef * b2, p0 + a.beta * coef_p * b3);
    if (stage1) {
        if (live) sq.add(b0, b1, b2, a.beta * b3);   // the p row in pressure units
    }
}

// 4-byte global -> shared copy that completes asynchronously (cp.async);
// cp_async_wait_all() makes this thread's copies visible to itself, a
// barrier after it to the block.
__device__ __forceinline__ void cp_async4(void *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Level jump of the x-face west of cell (gi, gj) (gi = nx: the east face of
// the last column) and of the y-face south of it (gj = ny: the north face
// of the top row); zero on faces that are not the domain's, and on
// boundary faces unless the axis is periodic.
__device__ __forceinline__ float x_face_jump(const MixedArgs &a, int gi, int gj, bool per_x) {
    float j = 0.0f;
    if (gj < a.ny) {
        if (gi < a.nx) j = __ldg(&a.jmp[gj * a.nx + gi].x);
        else if (gi == a.nx && per_x) j = __ldg(&a.jmp[gj * a.nx].x);
    }
    return j;
}
__device__ __forceinline__ float y_face_jump(const MixedArgs &a, int gi, int gj, bool per_y) {
    float j = 0.0f;
    if (gi < a.nx) {
        if (gj < a.ny) j = __ldg(&a.jmp[gj * a.nx + gi].y);
        else if (gj == a.ny && per_y) j = __ldg(&a.jmp[gi].y);
    }
    return j;
}

// Inputs of phases 3-4 read straight from global memory when used.
struct DirectSrc {
    static constexpr bool kJumpsStaged = false;
    const MixedArgs &a;
    const float4 *d0;
    __device__ __forceinline__ void prefetch(int, int) {}
    // (dQ^{m} of rho, rho u, rho v, dp^{m}; Q^n of rho, rho u, rho v; rho_ref) of cell g
    __device__ __forceinline__ void cell(int cell, int g, float &e0, float &e1, float &e2, float &p0, float &q0,
                                         float &q1, float &q2, float &rr) const {
        (void)cell;
        const float4 e = d0[g], q = __ldg(a.qn + g);
        e0 = e.x; e1 = e.y; e2 = e.z; p0 = e.w;
        q0 = q.x; q1 = q.y; q2 = q.z; rr = q.w;
    }
};

// Inputs of phase 4 loaded into registers at the start of phase 3, so that
// their latency overlaps the face fluxes (one cell per thread); the face
// level jumps are already in shared memory (staged with cp.async).
struct PrefetchSrc {
    static constexpr bool kJumpsStaged = true;
    const MixedArgs &a;
    const float4 *d0;
    float v[8];
    __device__ __forceinline__ void prefetch(int gi, int gj) {
        if (gi < a.nx && gj < a.ny) {
            const int g = gj * a.nx + gi;
            const float4 e = d0[g], q = __ldg(a.qn + g);
            v[0] = e.x; v[1] = e.y; v[2] = e.z; v[3] = e.w;
            v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
        }
    }
    __device__ __forceinline__ void cell(int, int, float &e0, float &e1, float &e2, float &p0, float &q0,
                                         float &q1, float &q2, float &rr) const {
        e0 = v[0]; e1 = v[1]; e2 = v[2]; p0 = v[3]; q0 = v[4]; q1 = v[5]; q2 = v[6]; rr = v[7];
    }
};

// Phases 2-4 of one tile, on W and the ring terms already in shared memory.
// RAW_AUX: the ring holds (dQ of rho u, dQ of rho v, rho_ref, fold bits) as
// copied, and the real-time terms are formed here (Backward-Euler only).
template <int TX, int TY, int NT, int RS, bool BDF, bool RAW_AUX, typename Src>
__device__ __forceinline__ void mixed_tile_compute(const MixedArgs &a, int stage, float alpha, int x0, int y0,
                                                   bool interior, double *partial, MixedSmem<TX, TY> &sm, Src &src) {
    static_assert(!(RAW_AUX && BDF), "raw ring terms are Backward-Euler only");
    using S = MixedSmem<TX, TY>;
    constexpr int RW = S::RW, GW = S::GW, GH = S::GH;
    const Ctl *ctl = a.ctl;
    int in, out;
    stage_buffers(ctl->cur, stage, in, out);
    float4 *dout = a.d[out];
    const float inv_dt = a.realtime ? float(ctl->inv_dt) : 0.0f;
    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const bool new_gradp = (a.gradp == kGradNew);

    // ---- 2. limited half slopes and pressure gradient on the ring ----
    const bool need_rt = new_gradp && a.realtime;
    const float klim = float(a.limiter_k);
    const float kp = (a.gradp == kGradSuperbee || a.gradp == kGradSplitSuperbee) ? 2.0f : 1.0f;
    for (int k = tid; k < GW * GH; k += NT) {
        const int lj = k / GW, li = k - lj * GW;
        const int c = (lj + 1) * RW + (li + 1);
        const float4 Wc = sm.w[c], We = sm.w[c + 1], Ww = sm.w[c - 1], Wn = sm.w[c + RW], Ws = sm.w[c - RW];
        float hrx, hry, hux, huy, hvx, hvy;
        limit_slopes(Wc, We, Ww, Wn, Ws, a.limiter_k, klim, hrx, hry, hux, huy, hvx, hvy);
        float hpx, hpy;
        if (new_gradp) {
            float sg = 1.0f;
            if (!interior) sg = wall_ghost_sign<float>(x0 + li - 1, y0 + lj - 1, nx, ny, a.bc);
            float4 ax = sm.aux[k];
            if constexpr (RAW_AUX) {
                float rx = 0.0f, ry = 0.0f;
                if (need_rt) {
                    rx = (a.B0 * ax.x) * inv_dt;
                    ry = (a.B0 * ax.y) * inv_dt;
                    if (!interior) {
                        const int f = __float_as_int(ax.w);
                        rx = (f & 1) ? -rx : rx;
                        ry = (f & 2) ? -ry : ry;
                    }
                }
                ax.x = rx;
                ax.y = ry;
            }
            new_gradp_half_slopes(a, Wc, hrx, hry, hux, huy, hvx, hvy, ax.x, ax.y, ax.z, sg, hpx, hpy);
        } else if (a.gradp == kGradSplitMinmod || a.gradp == kGradSplitSuperbee) {
            // Qian et al. split (Sec. 2.3.2); the record holds p here (no level)
            float sg = 1.0f;
            if (!interior) sg = wall_ghost_sign<float>(x0 + li - 1, y0 + lj - 1, nx, ny, a.bc);
            const float gxs = a.gx * sg, gys = a.gy * sg;
            hpx = 0.5f * limiter(We.w - Wc.w - a.half_dx * (Wc.x + We.x) * gxs,
                                 Wc.w - Ww.w - a.half_dx * (Ww.x + Wc.x) * gxs, kp) + a.half_dx * Wc.x * gxs;
            hpy = 0.5f * limiter(Wn.w - Wc.w - a.half_dy * (Wc.x + Wn.x) * gys,
                                 Wc.w - Ws.w - a.half_dy * (Ws.x + Wc.x) * gys, kp) + a.half_dy * Wc.x * gys;
        } else {
            hpx = 0.5f * limiter(We.w - Wc.w, Wc.w - Ww.w, kp);
            hpy = 0.5f * limiter(Wn.w - Wc.w, Wc.w - Ws.w, kp);
        }
        sm.gx[k] = make_float4(hrx, hux, hvx, hpx);
        sm.gy[k] = make_float4(hry, huy, hvy, hpy);
    }
    __syncthreads();

    // ---- 3. face states and Osher fluxes (pressures relative to P_f) ----
    const bool per_x = (a.bc[0] == kPeriodic), per_y = (a.bc[2] == kPeriodic);
    src.prefetch(x0 + tid % TX, y0 + tid / TX);
    for (int k = tid; k < S::NXF + S::NYF; k += NT) {
        const bool isx = k < S::NXF;
        FaceStates f;
        float4 *dst;
        if (isx) {
            const int fj = k / (TX + 1), fi = k - fj * (TX + 1);
            float jump;
            if constexpr (Src::kJumpsStaged) {
                jump = sm.dxf[k];
            } else {
                jump = x_face_jump(a, x0 + fi, y0 + fj, per_x);
                sm.dxf[k] = jump;
            }
            const int ga = (fj + 1) * GW + fi;
            const int ca = (fj + 2) * RW + fi + 1;
            x_face_states(sm.w[ca], sm.w[ca + 1], sm.gx[ga], sm.gx[ga + 1], jump, f);
            dst = &sm.fx[k];
        } else {
            const int kk = k - S::NXF;
            const int fj = kk / TX, fi = kk - fj * TX;
            float jump;
            if constexpr (Src::kJumpsStaged) {
                jump = sm.dyf[kk];
            } else {
                jump = y_face_jump(a, x0 + fi, y0 + fj, per_y);
                sm.dyf[kk] = jump;
            }
            const int ga = fj * GW + fi + 1;
            const int ca = (fj + 1) * RW + fi + 2;
            y_face_states(sm.w[ca], sm.w[ca + RW], sm.gy[ga], sm.gy[ga + GW], jump, f);
            dst = &sm.fy[kk];
        }
        // one flux call for both kinds: no divergence where a warp holds both
        *dst = face_flux<RS>(a, isx, f);
    }
    __syncthreads();

    // ---- 4. divergence + sources + point-implicit update of dQ and dp ----
    SqTile sq;
#pragma unroll
    for (int cell = tid; cell < TX * TY; cell += NT) {
        const int lj = cell / TX, li = cell - lj * TX;
        const int gi = x0 + li, gj = y0 + lj;
        if (gi >= nx || gj >= ny) continue;
        const int g = gj * nx + gi;
        const int fw = lj * (TX + 1) + li;
        cell_update<BDF>(a, alpha, inv_dt, a.B0 * inv_dt, stage == 1, dout, cell, g, sm.fx[fw], sm.fx[fw + 1],
                         sm.fy[cell], sm.fy[cell + TX], a.inv_dx, a.inv_dy, sm.dxf[fw], sm.dxf[fw + 1], sm.dyf[cell],
                         sm.dyf[cell + TX], src, sq);
    }
    if (stage == 1) {
        // warp, block and grid sums in FP64
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            double v = sq.get(f);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) sm.red[f][tid >> 5] = v;
        }
        __syncthreads();
        if (tid < 4) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += sm.red[tid][w];
            partial[tid] = s;
        }
    }
}


// One TX x TY tile (tile coordinates bx, by) of one stage of one tank, by
// a CTA of NT threads (NT divides TX*TY; several cells per thread in the
// update when NT < TX*TY).  `partial` receives the tile's four residual
// partial sums at stage 1.  Shared by the single-tank and batched kernels.
// PF (one cell per thread, Backward-Euler): the ring terms and the x-face
// reference jumps are copied with cp.async while the halo is being loaded,
// and the update's own-cell inputs are prefetched at the start of phase 3.
template <int TX, int TY, int NT, int RS, bool BDF, bool PF = false>
__device__ __forceinline__ void mixed_tile(const MixedArgs &a, int stage, float alpha, int bx, int by,
                                           double *partial, unsigned char *smem_raw) {
    using S = MixedSmem<TX, TY>;
    static_assert((TX * TY) % NT == 0 && NT % 32 == 0, "tile/thread shape");
    static_assert(!PF || (NT == TX * TY && !BDF), "prefetch: one cell per thread, Backward-Euler");
    S &sm = *reinterpret_cast<S *>(smem_raw);
    constexpr int RW = S::RW, RH = S::RH, GW = S::GW, GH = S::GH;

    const Ctl *ctl = a.ctl;
    int in, out;
    const int cur = ctl->cur;
    stage_buffers(cur, stage, in, out);
    const float4 *din = a.d[in];
    const float4 *d0 = a.d[cur];
    const float inv_dt = a.realtime ? float(ctl->inv_dt) : 0.0f;

    const int nx = a.nx, ny = a.ny;
    const int tid = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    // halo entirely inside the domain: no ghost folding for this tile
    const bool interior = (x0 >= 2) && (x0 + TX + 2 <= nx) && (y0 >= 2) && (y0 + TY + 2 <= ny);
    const CellLoad ld{a.qn, din};
    const bool new_gradp = (a.gradp == kGradNew);
    const bool need_rt = new_gradp && a.realtime;

    if constexpr (PF) {
        // face level jumps (zero outside the domain, as x_face_jump, y_face_jump)
        const bool per_x = (a.bc[0] == kPeriodic), per_y = (a.bc[2] == kPeriodic);
        for (int k = tid; k < S::NXF; k += NT) {
            const int fj = k / (TX + 1), fi = k - fj * (TX + 1);
            const int gi = x0 + fi, gj = y0 + fj;
            if (gj < ny && gi < nx) cp_async4(&sm.dxf[k], &a.jmp[gj * nx + gi].x);
            else if (gj < ny && gi == nx && per_x) cp_async4(&sm.dxf[k], &a.jmp[gj * nx].x);
            else sm.dxf[k] = 0.0f;
        }
        for (int k = tid; k < S::NYF; k += NT) {
            const int fj = k / TX, fi = k - fj * TX;
            const int gi = x0 + fi, gj = y0 + fj;
            if (gi < nx && gj < ny) cp_async4(&sm.dyf[k], &a.jmp[gj * nx + gi].y);
            else if (gi < nx && gj == ny && per_y) cp_async4(&sm.dyf[k], &a.jmp[gi].y);
            else sm.dyf[k] = 0.0f;
        }
        // ring: (dQ of rho u, dQ of rho v, rho_ref, fold bits)
        if (new_gradp) {
            for (int k = tid; k < GW * GH; k += NT) {
                const int rr = k / GW, cc = k - rr * GW;
                int s, fl = 0;
                if (interior) {
                    s = (y0 + rr - 1) * nx + (x0 + cc - 1);
                } else {
                    int nfx, tfx, nfy, tfy;
                    const int si = fold_axis(x0 + cc - 1, nx, a.bc[0], a.bc[1], nfx, tfx);
                    const int sj = fold_axis(y0 + rr - 1, ny, a.bc[2], a.bc[3], nfy, tfy);
                    s = sj * nx + si;
                    fl = ((nfx + tfy) & 1) | (((nfy + tfx) & 1) << 1);
                }
                float *dst = reinterpret_cast<float *>(&sm.aux[k]);
                if (need_rt) {
                    cp_async4(dst, &d0[s].y);
                    cp_async4(dst + 1, &d0[s].z);
                }
                cp_async4(dst + 2, &a.qn[s].w);
                dst[3] = __int_as_float(fl);
            }
        }
    }

    // ---- 1. stage Q^{s-1} = Q^n + dQ^{s-1} (+ halo) as W = (rho, u, v, dp) ----
    if (interior) {
        const int base = (y0 - 2) * nx + (x0 - 2);
        for (int k = tid; k < RW * RH; k += NT) {
            const int rr = k / RW, cc = k - rr * RW;
            sm.w[k] = ld(base + rr * nx + cc, false, false);
        }
    } else {
        for (int k = tid; k < RW * RH; k += NT) {
            const int rr = k / RW, cc = k - rr * RW;
            int nfx, tfx, nfy, tfy;
            const int si = fold_axis(x0 + cc - 2, nx, a.bc[0], a.bc[1], nfx, tfx);
            const int sj = fold_axis(y0 + rr - 2, ny, a.bc[2], a.bc[3], nfy, tfy);
            sm.w[k] = ld(sj * nx + si, (nfx + tfy) & 1, (nfy + tfx) & 1);
        }
    }
    if (!PF && new_gradp) {
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
            float rx = 0.0f, ry = 0.0f;
            if (need_rt) {
                rx = a.B0 * d0[s].y;   // B0 (Q^{m} - Q^n) of rho u, ...
                ry = a.B0 * d0[s].z;
                if constexpr (BDF) {
                    if (a.order >= 2) {
                        rx -= a.B2 * a.D1[1][s];
                        ry -= a.B2 * a.D1[2][s];
                    }
                    if (a.order >= 3) {
                        rx -= a.B3 * a.D2[1][s];
                        ry -= a.B3 * a.D2[2][s];
                    }
                }
                rx *= inv_dt;
                ry *= inv_dt;
                rx = fx ? -rx : rx;
                ry = fy ? -ry : ry;
            }
            sm.aux[k] = make_float4(rx, ry, __ldg(&a.qn[s].w), 0.0f);
        }
    }
    if constexpr (PF) {
        cp_async_wait_all();
        __syncthreads();
        PrefetchSrc src{a, d0, {}};
        mixed_tile_compute<TX, TY, NT, RS, BDF, true>(a, stage, alpha, x0, y0, interior, partial, sm, src);
    } else {
        __syncthreads();
        DirectSrc src{a, d0};
        mixed_tile_compute<TX, TY, NT, RS, BDF, false>(a, stage, alpha, x0, y0, interior, partial, sm, src);
    }
}

template <int TX, int TY, int NT, int MINB = 1, int RS = kOsher, bool BDF = false, bool PF = false>
__global__ void __launch_bounds__(NT, MINB)
stage_kernel_mixed(const MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_trigger();
    pdl_wait();
    if (a.ctl->done) return;
    mixed_tile<TX, TY, NT, RS, BDF, PF>(a, a.stage, a.alpha, blockIdx.x, blockIdx.y,
                           a.partials + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4, smem_raw);
}

// ---------------------------------------------------------------------------
// Column-strip form of the stage sweep (Osher flux, Backward-Euler, the new
// pressure gradient; either limiter).  Each warp owns 32 adjacent columns, of which the middle 28 are
// output, and walks up a strip of H rows with a rolling window in registers:
// the y-direction stencil lives in each lane's registers, x-neighbours come
// from warp shuffles, and each lane's row records arrive through its own
// slots of a shared-memory ring (StripRing), so there is no block barrier.  At
// the row it ingests, k, the warp forms W(k); with W(k-2..k) it forms the
// slopes and pressure gradient of row k-1, the x-face fluxes of row k-1 and
// the y-face flux between rows k-2 and k-1, and it updates row k-2.  Lanes
// 0, 1, 30, 31 are halo (their slopes or fluxes feed the output lanes'
// faces; they run the update's arithmetic too, storing nothing, so that the
// warp does not branch around it).  Every per-cell value uses the same functions as the tile sweep;
// a lane's x- and y-face fluxes go through the face-pair form of the Osher
// flux (osher_flux_pair), which returns 2F.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 shfl_down4(const float4 &v, int d) {
    return make_float4(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d),
                       __shfl_down_sync(0xffffffffu, v.z, d), __shfl_down_sync(0xffffffffu, v.w, d));
}
__device__ __forceinline__ float4 shfl_up4(const float4 &v, int d) {
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                       __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
}

constexpr int kStripOut = 28;   // output columns per warp

// One warp's rows in flight: each lane's records of four rows (slot k & 3
// holds row k), copied from global memory by cp.async one row ahead of use
// and read back by the same lane, so that no register holds a row before it
// is needed and none is copied from row to row.
struct StripRing {
    float4 q[4][32];   // Q^n of rho, rho u, rho v; rho_ref
    float4 d[4][32];   // dQ^{s-1} of rho, rho u, rho v; dp
    float4 e[4][32];   // dQ^{m}, dp^{m} (the ring terms)
    float jx[4][32];   // level jump across the east x-face (0 off the tank's rows)
    float jy[4][32];   // level jump across the south y-face (0 off the tank's faces)
    float dt[4][32];   // local pseudo-time step that stage 1 stored (later stages, default options)
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// The same 4-byte copy of n = 4 or 0 source bytes (0: the slot is filled with
// zero; the source address must still be valid).
__device__ __forceinline__ void cp_async4_zf(void *smem, const float *gmem, unsigned n) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// all but the most recent group of this thread's copies have landed
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// The update's inputs of one cell, held in registers.
struct HeldSrc {
    float e0, e1, e2, p0, q0, q1, q2, rr;
    __device__ __forceinline__ void cell(int, int, float &a0, float &a1, float &a2, float &a3, float &b0,
                                         float &b1, float &b2, float &c0) const {
        a0 = e0; a1 = e1; a2 = e2; a3 = p0; b0 = q0; b1 = q1; b2 = q2; c0 = rr;
    }
};

// One strip (strip coordinates sx, sy) of stage `stage` (coefficient alpha)
// of one tank, by one warp; `partial` receives the strip's four residual
// partial sums at stage 1.  Shared by the single-tank and batched kernels.
// The per-column parts of the boundary logic are formed once per strip and
// interior rows skip the fold.  Every row's records go through the warp's
// ring (StripRing): row k + 1 is copied in while row k is worked on, and
// the later uses of a row (its ring terms, reference density and level
// jumps one row on, the update's records two rows on) read it back from
// shared memory.  UNROLL: row-loop unrolling (2 lets the compiler keep the
// rolling rows' registers in place instead of moving them each row).  SK = 0
// compiles any stage and any of the sweep's options, read at run time; SK =
// 1 and 2 compile the default options (minmod limiter, real-time term,
// local pseudo-time step, alpha_PI on the p row) in, for stage 1 (whose
// input Q^{s-1} is Q^{m}, so one record serves both and the ring's e slots
// stay unused) and for the later stages (no residual sums).  The first four
// rows (y0 - 2 .. y0 + 1) run in a loop of their own, where part of the row's
// work is not needed yet, and so do the rows near the tank's top, whose
// windows reach ghost rows; the main loop then tests neither the row number
// nor the fold of ghost rows.
template <int H, int UNROLL = 1, int SK = 0>
__device__ __forceinline__ void mixed_strip(const MixedArgs &a, int stage, float alpha, int sx, int sy,
                                            double *partial, StripRing *ring) {
    constexpr bool FAST = SK != 0;
    const bool st1 = SK == 0 ? (stage == 1) : (SK == 1);
    const Ctl *ctl = a.ctl;
    const int lane = threadIdx.x & 31;
    const int nx = a.nx, ny = a.ny;
    const int c = sx * kStripOut + lane - 2;   // this lane's column
    const int y0 = sy * H, y1 = min(y0 + H, ny);
    int in, out;
    const int cur = ctl->cur;
    stage_buffers(cur, stage, in, out);
    const float4 *din = a.d[in];
    const float4 *d0 = a.d[cur];
    float4 *dout = a.d[out];
    const bool need_rt = FAST || a.realtime != 0;
    const float inv_dt = need_rt ? float(ctl->inv_dt) : 0.0f;
    const float b0dt = a.B0 * inv_dt;
    const int klim = FAST ? 1 : a.limiter_k;
    const bool per_x = (a.bc[0] == kPeriodic);
    // the column's source (ghost columns fold onto interior ones)
    int nfx, tfx;
    const int scol = fold_axis(c, nx, a.bc[0], a.bc[1], nfx, tfx);
    const bool out_lane = lane >= 2 && lane < 30 && c < nx;
    // the face pairs come as 2F: (2Fe - 2Fw) (1/(2 dx)) is (Fe - Fw)/dx exactly
    const float hidx = 0.5f * a.inv_dx, hidy = 0.5f * a.inv_dy;

    // Per-column parts of the boundary logic, fixed for the whole strip, in
    // one word: the fold bits of an interior row (bits 0-1), whether the
    // column is a wall ghost (bit 2), whether the low and high y sides are
    // walls (bits 3, 4); and the column of the east x-face's reference jump
    // (-1: none).
    const int gi = c + 1;   // the east x-face's column
    const int jcol = (gi >= 0 && gi < nx) ? gi : ((gi == nx && per_x) ? 0 : -1);
    const bool own_col = c >= 0 && c < nx;   // the south y-face of this column is the tank's
    // a tank row's jump copies: source columns (clamped into the tank) and byte counts
    const int jxc = jcol >= 0 ? jcol : 0, jyc = own_col ? c : 0;
    const unsigned jxn = jcol >= 0 ? 4u : 0u, jyn = own_col ? 4u : 0u;
    const bool per_y = (a.bc[2] == kPeriodic);
    const int colbits = (nfx & 1) | ((tfx & 1) << 1) |
                        (((c < 0 && is_wall(a.bc[0])) || (c >= nx && is_wall(a.bc[1]))) ? 4 : 0) |
                        (is_wall(a.bc[2]) ? 8 : 0) | (is_wall(a.bc[3]) ? 16 : 0);
    // fold bits of row k in this column (ghost rows fold onto tank rows); the
    // edge flag (a std::bool_constant) is false where k is known to be a tank row
    auto row_flags = [&](int k, auto edge) {
        if (!decltype(edge)::value || (k >= 0 && k < ny)) return colbits & 3;   // the same for the whole warp
        int nfy, tfy;
        fold_axis(k, ny, a.bc[2], a.bc[3], nfy, tfy);
        return ((nfx + tfy) & 1) | (((nfy + tfx) & 1) << 1);
    };
    // copies of row k's records into ring slot k & 3, as one group (edge as
    // above)
    auto stage_row = [&](int k, auto edge) {
        constexpr bool E = decltype(edge)::value;
        int nfy, tfy;
        const int srow = (!E || (k >= 0 && k < ny)) ? k : fold_axis(k, ny, a.bc[2], a.bc[3], nfy, tfy);
        const int s = srow * nx + scol, sl = k & 3;
        cp_async16(&ring->q[sl][lane], a.qn + s);
        cp_async16(&ring->d[sl][lane], din + s);
        if (SK != 1) cp_async16(&ring->e[sl][lane], d0 + s);
        if (SK == 2) cp_async4(&ring->dt[sl][lane], a.dtau + s);
        if (!E) {
            // a tank row: whether its faces are the tank's depends on the lane
            // only, so every lane copies (a zero where the face is not the tank's)
            cp_async4_zf(&ring->jx[sl][lane], &a.jmp[k * nx + jxc].x, jxn);
            cp_async4_zf(&ring->jy[sl][lane], &a.jmp[k * nx + jyc].y, jyn);
        } else {
            if (k >= 0 && k < ny && jcol >= 0)
                cp_async4(&ring->jx[sl][lane], &a.jmp[k * nx + jcol].x);
            else
                ring->jx[sl][lane] = 0.0f;
            // row ny: the north face of the top row (periodic: the south face of row 0)
            if (own_col && k >= 0 && (k < ny || (k == ny && per_y)))
                cp_async4(&ring->jy[sl][lane], &a.jmp[(k < ny ? k : 0) * nx + c].y);
            else
                ring->jy[sl][lane] = 0.0f;
        }
        cp_async_commit();
    };

    // the ring terms (dQ^{m}, dp^{m}) of the row in slot sl
    auto ering = [&](int sl) -> float4 { return SK == 1 ? ring->d[sl][lane] : ring->e[sl][lane]; };
    float4 Wm2 = make_float4(0.f, 0.f, 0.f, 0.f), Wm1 = Wm2;   // W at rows k-2, k-1
    float4 Dp = Wm2;                                         // W(k-1) - W(k-2) (rho, u, v)
    float4 Sym2 = Wm2;                                       // whole y slopes of row k-2
    float4 Fxm2 = Wm2;                                       // east x-face flux of row k-2
    float4 Fyp = Wm2;                                        // y-face flux between rows k-3 and k-2
    float Jm2 = 0.0f;                                        // east x-face level jump of row k-2
    float Jyp = 0.0f;                                        // level jump of the y-face below row k-2
    SqKahan sq;
    stage_row(y0 - 2, std::true_type{});
    // row k of the sweep; first: one of the strip's first four rows; edge:
    // rows k - 2 .. k + 1 may include ghost rows
    auto row = [&](int k, auto first, auto edge) {
        constexpr bool FIRST = decltype(first)::value, EDGE = decltype(edge)::value;
        // prefetch: the next row's records; then row k's own copies have landed
        stage_row(k + 1, edge);
        cp_async_wait_1();
        const int sk = k & 3, s1 = (k - 1) & 3, s2 = (k - 2) & 3;
        // ---- W = (rho, u, v, dp) of Q^{s-1} at row k ----
        float4 W0;
        {
            const float4 q = ring->q[sk][lane], d = ring->d[sk][lane];
            const int fl = row_flags(k, edge);
            const float r = q.x + d.x;
            float mm = q.y + d.y;
            float nn = q.z + d.z;
            mm = (fl & 1) ? -mm : mm;
            nn = (fl & 2) ? -nn : nn;
            const float ir = Ar<float>::rcp(r);
            W0 = make_float4(r, mm * ir, nn * ir, d.w);
        }
        if (!FIRST || k >= y0) {
            // ---- slopes and pressure gradient of row r = k-1 ----
            const int r = k - 1;
            // differences of rho, u, v across the east face (the west one is
            // the west neighbour's east difference) and the north face (the
            // south one was the north difference of the row before)
            const float4 We = shfl_down4(Wm1, 1);
            const float exr = We.x - Wm1.x, exu = We.y - Wm1.y, exv = We.z - Wm1.z;
            const float wxr = __shfl_up_sync(0xffffffffu, exr, 1), wxu = __shfl_up_sync(0xffffffffu, exu, 1),
                        wxv = __shfl_up_sync(0xffffffffu, exv, 1);
            float hrx, hry, hux, huy, hvx, hvy;
            limit_diffs(exr, wxr, W0.x - Wm1.x, Dp.x, exu, wxu, W0.y - Wm1.y, Dp.y, exv, wxv, W0.z - Wm1.z, Dp.z,
                        klim, float(klim), hrx, hry, hux, huy, hvx, hvy);
            float rx = 0.0f, ry = 0.0f;
            if (need_rt) {
                const float4 e1 = ering(s1);
                const int fl = row_flags(r, edge);
                rx = b0dt * e1.y;
                ry = b0dt * e1.z;
                rx = (fl & 1) ? -rx : rx;
                ry = (fl & 2) ? -ry : ry;
            }
            // gravity reversed in wall ghosts (as wall_ghost_sign)
            const bool wall_ghost =
                (colbits & 4) || (EDGE && ((r < 0 && (colbits & 8)) || (r >= ny && (colbits & 16))));
            const float sg = wall_ghost ? -1.0f : 1.0f;
            float hpx, hpy;
            new_gradp_whole_slopes(a, Wm1, hrx, hry, hux, huy, hvx, hvy, rx, ry, ring->q[s1][lane].w, sg, hpx, hpy);
            const float4 Sx = make_float4(hrx, hux, hvx, hpx), Sy = make_float4(hry, huy, hvy, hpy);
            // (on the strip's first slope row, r = y0 - 1, neither face is
            // needed: only its y slopes are, by the y-face above it)
            if (!FIRST || k >= y0 + 1) {
                // ---- east x-face of row r (between columns c and c + 1) ----
                const float4 &Wn = We;
                const float4 Sn = shfl_down4(Sx, 1);
                const float jump = ring->jx[s1][lane];
                const float jy1 = ring->jy[s1][lane];   // below row r
                // ---- and the y-face between rows r - 1 and r: both fluxes as one packed pair ----
                FaceStates f, fy;
                x_face_states_whole(Wm1, Wn, Sx, Sn, jump, f);
                y_face_states_whole(Wm2, Wm1, Sym2, Sy, jy1, fy);
                float2 Fp[4];
                osher_flux_pair(make_float2(f.rL, fy.rL), make_float2(f.nL, fy.nL), make_float2(f.tL, fy.tL),
                                make_float2(f.pL, fy.pL), make_float2(f.rR, fy.rR), make_float2(f.nR, fy.nR),
                                make_float2(f.tR, fy.tR), make_float2(f.pR, fy.pR), a.beta, a.inv_beta, Fp);
                const float4 Fx = make_float4(Fp[0].x, Fp[1].x, Fp[2].x, Fp[3].x);
                // the y-face's normal momentum is rho v
                const float4 Fy = make_float4(Fp[0].y, Fp[2].y, Fp[1].y, Fp[3].y);
                if (!FIRST || k >= y0 + 2) {
                    // ---- update of row k - 2 ----
                    const float4 Fw = shfl_up4(Fxm2, 1);
                    const float jw = __shfl_up_sync(0xffffffffu, Jm2, 1);
                    // row k - 2 is a tank row, so its slot holds this column's records
                    const float4 ue = ering(s2), uq = ring->q[s2][lane];
                    const HeldSrc Uk{ue.x, ue.y, ue.z, ue.w, uq.x, uq.y, uq.z, uq.w};
                    cell_update<false, FAST, SK>(a, alpha, inv_dt, b0dt, st1, dout, 0, (k - 2) * nx + c, Fw, Fxm2,
                                                 Fyp, Fy, hidx, hidy, jw, Jm2, Jyp, jy1, Uk, sq, out_lane,
                                                 SK == 2 ? ring->dt[s2][lane] : 0.0f);
                }
                Fyp = Fy;
                Jyp = jy1;
                Fxm2 = Fx;
                Jm2 = jump;
            }
            Sym2 = Sy;
        }
        Dp = make_float4(W0.x - Wm1.x, W0.y - Wm1.y, W0.z - Wm1.z, 0.0f);
        Wm2 = Wm1;
        Wm1 = W0;
    };
    // the strip's first four rows, the rows whose window holds tank rows only
    // (row k + 1 is copied ahead, so k <= ny - 2), and the top strip's last rows
    int k = y0 - 2;
#pragma unroll 1
    for (; k < y0 + 2; ++k) row(k, std::true_type{}, std::true_type{});
    const int kin = min(y1 + 1, ny - 2);
#pragma unroll UNROLL
    for (; k <= kin; ++k) row(k, std::false_type{}, std::false_type{});
#pragma unroll 1
    for (; k <= y1 + 1; ++k) row(k, std::false_type{}, std::true_type{});
    cp_async_wait_all();   // the copies past the strip's last row
    if (st1) {
        // the strip's sums across lanes, in FP64
        double v0 = sq.lane_sum(0), v1 = sq.lane_sum(1), v2 = sq.lane_sum(2), v3 = sq.lane_sum(3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_down_sync(0xffffffffu, v0, o);
            v1 += __shfl_down_sync(0xffffffffu, v1, o);
            v2 += __shfl_down_sync(0xffffffffu, v2, o);
            v3 += __shfl_down_sync(0xffffffffu, v3, o);
        }
        if (lane == 0) {
            partial[0] = v0; partial[1] = v1; partial[2] = v2; partial[3] = v3;
        }
    }
}

// SK: 0 for any stage and options, 1 and 2 for stage 1 and the later stages
// with the default options (see mixed_strip); the stage-1 instance runs its
// row loop plain (unrolled by 2 it spills and gains nothing measurable), the
// others unroll it by 2, which keeps the rolling rows' registers in place.
template <int H, int WPC, int MINB, int SK>
__global__ void __launch_bounds__(WPC * 32, MINB)
sweep_kernel_mixed(const MixedArgs a, int strips_x, int nstrips) {
    pdl_trigger();
    pdl_wait();
    if (a.ctl->done) return;
    extern __shared__ __align__(16) unsigned char strip_smem[];
    const int warp = blockIdx.x * WPC + (threadIdx.x >> 5);
    if (warp >= nstrips) return;   // whole warps only
    const int sy = warp / strips_x, sx = warp - sy * strips_x;
    mixed_strip<H, SK == 1 ? 1 : 2, SK>(a, a.stage, a.alpha, sx, sy, a.partials + (size_t)warp * 4,
                      reinterpret_cast<StripRing *>(strip_smem) + (threadIdx.x >> 5));
}

// Global pseudo-time step option for the mixed form.
static __global__ void dtau_min_kernel_mixed(const MixedArgs a) {
    pdl_trigger();
    pdl_wait();
    const Ctl *ctl = a.ctl;
    if (ctl->done) return;
    const float4 *d = a.d[ctl->cur];
    const size_t N = (size_t)a.nx * a.ny;
    double mn = INFINITY;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        const float4 e = d[g], q = a.qn[g];
        const float r0 = q.x + e.x;
        const float ir = Ar<float>::rcp(r0);
        const float u = (q.y + e.y) * ir, v = (q.z + e.z) * ir;
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

// Global real-time step (Sec. 2.2.4) in the mixed form, Q = Q^n + dQ.
static __global__ void realtime_dt_kernel_mixed(const MixedArgs a, int cur, double cfl_area,
                                                unsigned long long *out) {
    const float4 *d = a.d[cur];
    const size_t N = (size_t)a.nx * a.ny;
    double mn = INFINITY;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x) {
        const float4 e = d[g], q4 = a.qn[g];
        const double r = double(q4.x) + double(e.x);
        const double u = (double(q4.y) + double(e.y)) / r;
        const double v = (double(q4.z) + double(e.z)) / r;
        mn = fmin(mn, cfl_area / (fabs(u) * double(a.dy) + fabs(v) * double(a.dx)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, (unsigned long long)__double_as_longlong(mn));
}

// Start of a physical step in the mixed form, one cell: the FP64 levels
// absorb the increments (Q^n <- Q^n + dQ, p^n <- p^n + dp, Alg. 1), the FP32
// copy of Q^n is refreshed and the increments restart from zero.  Without a
// pressure level the record keeps p, and p is kept for a restore.
__device__ __forceinline__ void mixed_level_shift(const MixedArgs &a, int cur, size_t g) {
    const float4 e = a.d[cur][g];
    float4 q4 = a.qn[g];   // .w (rho_ref) stays
    const float dqs[3] = {e.x, e.y, e.z};
    float qs[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const float dq = dqs[f];
        const double q = a.q64[f][g] + double(dq);
        // differences to the older levels, relative to the new Q^n
        if (a.D2[0]) a.D2[f][g] = float(double(a.D1[f][g]) + double(dq));
        if (a.D1[0]) a.D1[f][g] = dq;
        a.q64[f][g] = q;
        qs[f] = float(q);
    }
    q4.x = qs[0]; q4.y = qs[1]; q4.z = qs[2];
    a.qn[g] = q4;
    if (a.plevel) {
        const double p = a.q64[3][g] + double(e.w);
        a.q64[3][g] = p;
        a.p64_step[g] = p;
        a.d[cur][g] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
        a.d[cur][g] = make_float4(0.0f, 0.0f, 0.0f, e.w);
        a.lev_p[g] = e.w;
    }
}

// Jumps of the pressure level across the west and south faces of cell g,
// differenced in FP64 and rounded once: jx = p^n(i) - p^n(i-1),
// jy = q^n(j) - q^n(j-1), q^n = p^n - p_ref.  Boundary faces carry zero (a
// wall or transmissive ghost repeats its cell's level) unless the axis is
// periodic.  Without a pressure level p^n is zero and so are the jumps.
__device__ __forceinline__ void mixed_level_jumps(const MixedArgs &a, size_t g) {
    const int nx = a.nx, ny = a.ny;
    const int j = (int)(g / nx), i = (int)(g - (size_t)j * nx);
    const double *P = a.q64[3], *R = a.pref64;
    const double p = P[g];
    float jx = 0.0f, jy = 0.0f;
    if (i > 0) jx = float(p - P[g - 1]);
    else if (a.bc[0] == kPeriodic) jx = float(p - P[g + nx - 1]);
    size_t s = g;   // the cell below across the south face
    bool has_s = false;
    if (j > 0) { s = g - nx; has_s = true; }
    else if (a.bc[2] == kPeriodic) { s = g + (size_t)(ny - 1) * nx; has_s = true; }
    if (has_s) jy = R ? float((p - R[g]) - (P[s] - R[s])) : float(p - P[s]);
    a.jmp[g] = make_float2(jx, jy);
}

static __global__ void begin_step_kernel_mixed(const MixedArgs a, double dt, double tol, int max_iters,
                                               double tau_end) {
    Ctl *ctl = a.ctl;
    const int cur = ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_shift(a, cur, g);
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
        ctl->rebase = 0;
        ctl->tau = 0.0;
        ctl->tau_end = tau_end;
    }
}

// After the level shift (a separate launch: it reads the neighbours' new
// levels).
static __global__ void level_jumps_kernel_mixed(const MixedArgs a) {
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_jumps(a, g);
}

// Back to the state at the start of the step, one cell (after a
// non-finite residual): the levels hold it, the pressure level as it was
// before any rebase of the step (the jumps are formed again afterwards).
__device__ __forceinline__ void mixed_restore(const MixedArgs &a, int cur, size_t g) {
    if (a.plevel) a.q64[3][g] = a.p64_step[g];
    a.d[cur][g] = make_float4(0.0f, 0.0f, 0.0f, a.plevel ? 0.0f : a.lev_p[g]);
}

// Rebase of the pressure within a physical step, one cell: the FP64 level
// absorbs the current increment, which restarts from zero (the pressure has
// no real-time term, so its level may move at any time; the sum is exact up
// to one FP64 rounding).  FP32 then holds only the change since the rebase:
// in the first iterations of a step that starts from an unbalanced state
// (a collapsing column) the pressure moves by as much as the hydrostatic
// head.  The jumps are formed again by a second launch (mixed_level_jumps).
__device__ __forceinline__ void mixed_rebase_shift(const MixedArgs &a, int cur, size_t g) {
    float4 *r = a.d[cur] + g;
    a.q64[3][g] += double(r->w);
    r->w = 0.0f;
}

// The end of iteration m sets ctl->rebase after m = 1, 2, 4, 8 (not on the
// last iteration); otherwise these return at once.
static __global__ void rebase_shift_kernel_mixed(const MixedArgs a) {
    pdl_trigger();
    pdl_wait();
    const Ctl *ctl = a.ctl;
    if (!ctl->rebase) return;
    const int cur = ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_rebase_shift(a, cur, g);
}

static __global__ void rebase_jumps_kernel_mixed(const MixedArgs a) {
    pdl_trigger();
    pdl_wait();
    if (!a.ctl->rebase) return;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_level_jumps(a, g);
}

static __global__ void restore_kernel_mixed(const MixedArgs a) {
    const int cur = a.ctl->cur;
    const size_t N = (size_t)a.nx * a.ny;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < N; g += (size_t)gridDim.x * blockDim.x)
        mixed_restore(a, cur, g);
}

}  // namespace acgb
