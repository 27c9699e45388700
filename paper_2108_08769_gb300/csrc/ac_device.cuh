// ac_device.cuh -- device-side building blocks of the fused pseudo-time stage
// sweep: boundary mapping, k-limiter, the rank-2 Osher flux, pseudo-time step.
//
// Method: Leakey, Glenis & Hewett (arXiv 2108.08769).  Everything here is
// written for GB300 (sm_103a): one thread per cell, tiles staged in shared
// memory, no library calls.
#pragma once

#include <cstring>
#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

namespace acgb {

enum BcKind { kSlip = 0, kNoSlip = 1, kTransmissive = 2, kPeriodic = 3 };
enum GradP { kGradNew = 0, kGradMinmod = 1, kGradSuperbee = 2, kGradSplitMinmod = 3, kGradSplitSuperbee = 4 };
enum Riemann { kOsher = 0, kBassi = 1, kRoe = 2 };

// ---------------------------------------------------------------------------
// Arithmetic traits.  FP64 uses IEEE division and square root; FP32 uses
// the fast reciprocal / reciprocal-square-root instructions (about 1 ulp),
// which is far below the FP32 rounding of the stored state.
// ---------------------------------------------------------------------------
template <typename T> struct Ar;
template <> struct Ar<double> {
    // correctly rounded reciprocal (the division routine's numerator handling is not needed)
    static __device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
    // returns sqrt(x) and 1/sqrt(x): one reciprocal square root (<= 1 ulp) and
    // a product, in place of a square root and a division
    static __device__ __forceinline__ void sqrt_rsqrt(double x, double &s, double &rs) {
        rs = rsqrt(x);
        s = x * rs;
    }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};
template <> struct Ar<float> {
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ void sqrt_rsqrt(float x, float &s, float &rs) {
        rs = rsqrtf(x);
        s = x * rs;
    }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
};

// ---------------------------------------------------------------------------
// Ghost cells (Sec. 2.5).  A ghost index along one axis is folded back onto
// the interior cell it copies; every wall reflection flips the normal
// momentum, a no-slip reflection also the tangential one.  Indices reach at
// most a few cells past the domain, so the loop is short; the final clamp
// keeps every access in bounds whatever the input.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fold_axis(int i, int n, int lo, int hi, int &nflip, int &tflip) {
    nflip = 0;
    tflip = 0;
#pragma unroll 1
    for (int g = 0; g < 8 && (i < 0 || i >= n); ++g) {
        if (i < 0) {
            if (lo == kPeriodic) i += n;
            else if (lo == kTransmissive) i = 0;
            else { i = -1 - i; ++nflip; tflip += (lo == kNoSlip); }
        } else {
            if (hi == kPeriodic) i -= n;
            else if (hi == kTransmissive) i = n - 1;
            else { i = 2 * n - 1 - i; ++nflip; tflip += (hi == kNoSlip); }
        }
    }
    return min(max(i, 0), n - 1);
}

__device__ __forceinline__ bool is_wall(int bc) { return bc == kSlip || bc == kNoSlip; }

// ---------------------------------------------------------------------------
// k-limiter G(a, b) = s max(0, min(k|b|, s a), min(|b|, k s a)), s = sgn(b)
// (Sec. 2.3.1); a forward, b backward difference.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T limiter(T a, T b, T k) {
    T s = (b > T(0)) ? T(1) : ((b < T(0)) ? T(-1) : T(0));
    T t = s * a;
    T ab = fabs(b);
    T m = fmax(fmin(k * ab, t), fmin(ab, k * t));
    return s * fmax(T(0), m);
}

// Half of the k = 1 limiter (minmod), branch-free:
//   G(a, b)/2 = (sgn a + sgn b)/4 * min(|a|, |b|),
// which is 0 for opposite signs or a zero argument and +-min(|a|,|b|)/2
// otherwise -- the same value, bit for bit (the factors are powers of two).
template <typename T>
__device__ __forceinline__ T half_minmod(T a, T b) {
    return (copysign(T(0.25), a) + copysign(T(0.25), b)) * fmin(fabs(a), fabs(b));
}

// The whole k = 1 limiter, G(a, b) = 2 half_minmod(a, b), from the bit
// patterns: zero where the sign bits differ, else the argument of smaller
// magnitude (finite magnitudes order like their patterns with the sign bit
// cleared).  Integer instructions only, for sweeps that the FP64 pipe
// bounds; the same value, signed zeros included, and, like fmin, the other
// argument in place of a NaN.
__device__ __forceinline__ double minmod_bits(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    const long long m = (ma < mb) ? ia : ib;
    return ((ia ^ ib) < 0) ? 0.0 : __longlong_as_double(m);
}

// ---------------------------------------------------------------------------
// Osher flux of Dumbser & Toro along the straight path in Q, 3-point
// Gauss-Legendre (Sec. 2.4.3), in the face-normal frame.  States are given
// as primitive (rho, un, ut, p); Q = (rho, rho un, rho ut, p/beta).
//
// |A| has the triple eigenvalue u and the acoustic pair (u +- c)/2, so with
// sum_k r_k l_k = I it collapses to the exact rank-2 form
//   |A| dQ = |u| dQ + (|l4| - |u|) r4 (l4.dQ) + (|l5| - |u|) r5 (l5.dQ),
// with r4, r5, l4, l5 the acoustic columns/rows of R_x, L_x (Sec. 2.1.3).
// Writing a = (d(rho un) - un d(rho))/beta and dq = d(p/beta):
//   l4.dQ =  (rho/c)(l4 a + dq),   l5.dQ = -(rho/c)(l5 a + dq),
// and since l4 > 0 > l5: |l4| - |u| = l4 - |u|, |l5| - |u| = -l5 - |u|.
// Output F = (mass, normal momentum, tangential momentum, p/beta flux), or
// 2F with TWICE (the caller folds the 1/2 into its divergence; a factor of
// two is exact, so the divergence is the same to the last bit).
// ---------------------------------------------------------------------------
template <typename T, bool TWICE = false>
__device__ __forceinline__ void osher_flux(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR,
                                           T beta, T inv_beta, T F[4]) {
    const T mL = rL * uL, nL = rL * vL;
    const T mR = rR * uR, nR = rR * vR;
    const T dr = rR - rL, dm = mR - mL, dn = nR - nL, dp = pR - pL;
    const T dq = dp * inv_beta;   // the jump of Q's last component p/beta
    const T four_beta = T(4) * beta;
    // Gauss-Legendre points mapped to [0,1]: (xi + 1)/2, weights w/2
    const T tq[3] = {T(0.11270166537925831148), T(0.5), T(0.88729833462074168852)};
    const T wq[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
    // D = sum_j w_j |A_j| dQ, accumulated as
    //   D0 = dr Sau + Se,  D1 = dm Sau + Sue + beta Sg,
    //   D2 = dn Sau + Sve, D3 = dq Sau - Sh
    // with, at point j, G4 = (l4 - |u|) (l4 beta a + dp), G5 = (l5 + |u|)
    // (l5 beta a + dp) and k = w_j / (beta c): e = rho k (G4 l4 + G5 l5)
    // enters Se and, times u and v, Sue and Sve (rho u = m, rho v = n), and
    // Sg, Sh take k (G4 + G5) and k (G4 l5 + G5 l4) (the acoustic terms of
    // |A| dQ over rho times rho: the density cancels).  Since l4 + l5 = u,
    // G4 l5 + G5 l4 = (G4 + G5) u - (G4 l4 + G5 l5).
    T Sau, Se, Sue, Sve, Sg, Sh;
    // the three densities' reciprocals from one reciprocal of their product
    // (1 reciprocal + 6 products in place of 3 reciprocals)
    T rq[3], irq[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) rq[j] = rL + tq[j] * dr;
    {
        const T r01 = rq[0] * rq[1];
        const T inv = Ar<T>::rcp(r01 * rq[2]);
        const T inv01 = rq[2] * inv;   // 1 / (r0 r1)
        irq[2] = r01 * inv;
        irq[0] = rq[1] * inv01;
        irq[1] = rq[0] * inv01;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T r = rq[j];
        const T m = mL + tq[j] * dm;
        const T n = nL + tq[j] * dn;
        const T ir = irq[j];
        const T u = m * ir;
        const T c2 = u * u + four_beta * ir;
        T c, ic;
        Ar<T>::sqrt_rsqrt(c2, c, ic);
        // l4 = u/2 + c/2, l5 = u/2 - c/2 (c/2 is exact: one rounding each)
        const T hu = T(0.5) * u;
        const T l4 = fma(T(0.5), c, hu), l5 = fma(T(-0.5), c, hu);
        const T au = fabs(u);
        const T ba = dm - u * dr;   // beta a
        const T w = wq[j];
        const T k = (w * inv_beta) * ic;
        const T G4 = (l4 - au) * (l4 * ba + dp);
        const T G5 = (l5 + au) * (l5 * ba + dp);
        const T Gs = G4 + G5;
        const T Ep = G4 * l4 + G5 * l5;
        const T Hp = Gs * u - Ep;        // G4 l5 + G5 l4
        const T E = k * Ep;              // e / rho
        if (j == 0) {
            Sau = w * au; Se = r * E; Sue = m * E; Sve = n * E; Sg = k * Gs; Sh = k * Hp;
        } else {
            Sau += w * au; Se += r * E; Sue += m * E; Sve += n * E; Sg += k * Gs; Sh += k * Hp;
        }
    }
    // central part 1/2 (F(Q_L) + F(Q_R)); dissipation 1/2 * D (D already
    // carries the 1/2 of the [0,1] quadrature)
    const T hf = TWICE ? T(1) : T(0.5);
    F[0] = hf * ((mL + mR) - (dr * Sau + Se));
    F[1] = hf * ((mL * uL + pL + mR * uR + pR) - (dm * Sau + Sue + beta * Sg));
    F[2] = hf * ((mL * vL + mR * vR) - (dn * Sau + Sve));
    F[3] = hf * ((uL + uR) - (dq * Sau - Sh));
}

// ---------------------------------------------------------------------------
// Roe flux with the Roe averages of Sec. 2.4.2 (no entropy fix, none being
// needed here): F = 1/2 (F(Q_L) + F(Q_R) - |A(Q~)| dQ), |A| dQ in the same
// rank-2 form as one Osher quadrature point with weight 1.
// ---------------------------------------------------------------------------
template <typename T, bool TWICE = false>
__device__ __forceinline__ void roe_flux(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR, T beta, T inv_beta,
                                         T F[4]) {
    const T mL = rL * uL, nL = rL * vL, qL = pL * inv_beta;
    const T mR = rR * uR, nR = rR * vR, qR = pR * inv_beta;
    const T dr = rR - rL, dm = mR - mL, dn = nR - nL, dq = qR - qL;
    const T sL = Ar<T>::sqrt_(rL), sR = Ar<T>::sqrt_(rR);
    const T isum = Ar<T>::rcp(sL + sR);
    const T r = sL * sR;
    const T u = (sL * uL + sR * uR) * isum, v = (sL * vL + sR * vR) * isum;
    const T ir = Ar<T>::rcp(r);
    const T c2 = u * u + T(4) * beta * ir;
    T c, ic;
    Ar<T>::sqrt_rsqrt(c2, c, ic);
    const T hu = T(0.5) * u, hc = T(0.5) * c;
    const T l4 = hu + hc, l5 = hu - hc;
    const T au = fabs(u);
    const T a = (dm - u * dr) * inv_beta;
    const T k = r * ic;
    const T g4 = (l4 - au) * k * (l4 * a + dq);
    const T g5 = (l5 + au) * k * (l5 * a + dq);
    const T e = g4 * l4 + g5 * l5;
    const T hf = TWICE ? T(1) : T(0.5);   // 2F with TWICE, as osher_flux
    F[0] = hf * ((mL + mR) - (au * dr + e));
    F[1] = hf * ((mL * uL + pL + mR * uR + pR) - (au * dm + u * e + beta * ir * (g4 + g5)));
    F[2] = hf * ((mL * vL + mR * vR) - (au * dn + v * e));
    F[3] = hf * ((uL + uR) - (au * dq - (g4 * l5 + g5 * l4) * ir));
}

// ---------------------------------------------------------------------------
// Flux of the exact (non-iterative) Riemann solution of Bassi et al.
// (Sec. 2.4.1): acoustic speeds S_L = (u_L - c_L)/2, S_R = (u_R + c_R)/2, the
// star values u*, p*, rho*_L, rho*_R, and the state at x/tau = 0 sampled as
// left (0 <= S_L), left star (0 <= u*), right star (0 <= S_R) or right.
// ---------------------------------------------------------------------------
template <typename T, bool TWICE = false>
__device__ __forceinline__ void bassi_flux(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR, T beta, T inv_beta,
                                           T F[4]) {
    const T cL = Ar<T>::sqrt_(uL * uL + T(4) * beta * Ar<T>::rcp(rL));
    const T cR = Ar<T>::sqrt_(uR * uR + T(4) * beta * Ar<T>::rcp(rR));
    const T l4L = T(0.5) * (uL + cL), l5L = T(0.5) * (uL - cL);
    const T l4R = T(0.5) * (uR + cR), l5R = T(0.5) * (uR - cR);
    const T SL = l5L, SR = l4R;
    T r, u, v, p;
    if (T(0) <= SL) {
        r = rL; u = uL; v = vL; p = pL;
    } else {
        const T us = Ar<T>::div(pR - pL + rR * uR * l5R - rL * uL * l4L, rR * l5R - rL * l4L);
        const T ps = pR + rR * l5R * (uR - us);
        if (T(0) <= us) {
            r = Ar<T>::div(rL * l4L, us - l5L); u = us; v = vL; p = ps;
        } else if (T(0) <= SR) {
            r = Ar<T>::div(rR * l5R, us - l4R); u = us; v = vR; p = ps;
        } else {
            r = rR; u = uR; v = vR; p = pR;
        }
    }
    const T m = r * u;
    const T s = TWICE ? T(2) : T(1);   // 2F with TWICE, as osher_flux
    F[0] = s * m;
    F[1] = s * (m * u + p);
    F[2] = s * (m * v);
    F[3] = s * u;
}

// FP32 form of osher_flux for sm_100-class parts: the two outer Gauss points
// (same weight 5/18, positions 1/2 -+ sqrt(15)/10) run as the two lanes of
// packed FP32x2 instructions (__ffma2_rn, __fmul2_rn, __fadd2_rn: one issue
// slot for two operations, per-lane rounding as the scalar forms), the
// middle point in scalar code.  Same quadrature and the same terms as
// osher_flux; only the order of the three point sums differs.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// a - b as one packed FP32x2 subtraction (the same value as a + (-b),
// without separate sign flips of b's halves)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}

__device__ __forceinline__ void osher_flux_x2(float rL, float uL, float vL, float pL, float rR, float uR,
                                              float vR, float pR, float beta, float inv_beta, float F[4]) {
    const float mL = rL * uL, nL = rL * vL, qL = pL * inv_beta;
    const float mR = rR * uR, nR = rR * vR, qR = pR * inv_beta;
    const float dr = rR - rL, dm = mR - mL, dn = nR - nL, dq = qR - qL;
    const float four_beta = 4.0f * beta;
    const float w13 = 5.0f / 18.0f, w2 = 8.0f / 18.0f;
    // ---- points 1 and 3 ----
    const float2 t = make_float2(0.11270166537925831148f, 0.88729833462074168852f);
    const float2 r = __ffma2_rn(t, dup2(dr), dup2(rL));
    const float2 mm = __ffma2_rn(t, dup2(dm), dup2(mL));
    const float2 nn = __ffma2_rn(t, dup2(dn), dup2(nL));
    const float2 ir = make_float2(Ar<float>::rcp(r.x), Ar<float>::rcp(r.y));
    const float2 u = __fmul2_rn(mm, ir);
    const float2 c2 = __ffma2_rn(u, u, __fmul2_rn(dup2(four_beta), ir));
    const float2 ic = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));
    const float2 c = __fmul2_rn(c2, ic);
    const float2 hu = __fmul2_rn(dup2(0.5f), u), hc = __fmul2_rn(dup2(0.5f), c);
    const float2 l4 = __fadd2_rn(hu, hc), l5 = sub2(hu, hc);
    const float2 au = make_float2(fabsf(u.x), fabsf(u.y));
    const float2 a = __fmul2_rn(__ffma2_rn(neg2(u), dup2(dr), dup2(dm)), dup2(inv_beta));
    // k = 1/c, taken out of G4, G5 as in osher_flux (the density cancels)
    const float2 G4 = __fmul2_rn(sub2(l4, au), __ffma2_rn(l4, a, dup2(dq)));
    const float2 G5 = __fmul2_rn(__fadd2_rn(l5, au), __ffma2_rn(l5, a, dup2(dq)));
    const float2 Gs = __fadd2_rn(G4, G5);
    const float2 Ep = __ffma2_rn(G5, l5, __fmul2_rn(G4, l4));
    const float2 E = __fmul2_rn(ic, Ep);
    const float2 gs = __fmul2_rn(ic, Gs);
    const float2 h = __fmul2_rn(ic, sub2(__fmul2_rn(Gs, u), Ep));   // G4 l5 + G5 l4, times k
    // lane sums of (|u|, rho E, m E, n E, k (G4 + G5), k (G4 l5 + G5 l4)), times w13
    const float2 re = __fmul2_rn(r, E), me = __fmul2_rn(mm, E), ne = __fmul2_rn(nn, E);
    float Sau = w13 * (au.x + au.y), Se = w13 * (re.x + re.y), Sue = w13 * (me.x + me.y);
    float Sve = w13 * (ne.x + ne.y), Sg = w13 * (gs.x + gs.y), Sh = w13 * (h.x + h.y);
    // ---- point 2 ----
    {
        const float r2 = rL + 0.5f * dr, m2 = mL + 0.5f * dm, n2 = nL + 0.5f * dn;
        const float ir2 = Ar<float>::rcp(r2);
        const float u2 = m2 * ir2;
        const float c22 = u2 * u2 + four_beta * ir2;
        const float ic2 = rsqrtf(c22), cc = c22 * ic2;
        const float hu2 = 0.5f * u2, hc2 = 0.5f * cc;
        const float l42 = hu2 + hc2, l52 = hu2 - hc2;
        const float au2 = fabsf(u2);
        const float a2 = (dm - u2 * dr) * inv_beta;
        const float G42 = (l42 - au2) * (l42 * a2 + dq);
        const float G52 = (l52 + au2) * (l52 * a2 + dq);
        const float Gs2 = G42 + G52;
        const float Ep2 = G42 * l42 + G52 * l52;
        const float k2 = w2 * ic2;
        const float E2 = k2 * Ep2;
        Sau += w2 * au2;
        Se += r2 * E2;
        Sue += m2 * E2;
        Sve += n2 * E2;
        Sg += k2 * Gs2;
        Sh += k2 * (Gs2 * u2 - Ep2);   // G42 l52 + G52 l42
    }
    F[0] = 0.5f * ((mL + mR) - (dr * Sau + Se));
    F[1] = 0.5f * ((mL * uL + pL + mR * uR + pR) - (dm * Sau + Sue + beta * Sg));
    F[2] = 0.5f * ((mL * vL + mR * vR) - (dn * Sau + Sve));
    F[3] = 0.5f * ((uL + uR) - (dq * Sau - Sh));
}

// Osher fluxes of two faces at once (Sec. 2.4.3), for a thread that owns an
// x-face and a y-face: lane x of every packed FP32x2 instruction carries one
// face and lane y the other, and each lane takes the three Gauss points in
// turn.  Every operation of the flux is then a packed one (the reciprocal
// and reciprocal square root excepted) and no lane sums are needed.  Same
// quadrature and terms as osher_flux, per lane; the weight of a point rides
// on k = w / c (1/beta stays on the jump term, where it costs no register
// held across a caller's loop).  Inputs are (rho, un, ut, p) per
// lane; returns 2F per lane (the caller's divergence takes the 1/2).
__device__ __forceinline__ void osher_flux_pair(float2 rL, float2 uL, float2 vL, float2 pL, float2 rR, float2 uR,
                                                float2 vR, float2 pR, float beta, float inv_beta, float2 F[4]) {
    const float2 ib = dup2(inv_beta);
    const float2 mL = __fmul2_rn(rL, uL), nL = __fmul2_rn(rL, vL);
    const float2 mR = __fmul2_rn(rR, uR), nR = __fmul2_rn(rR, vR);
    const float2 dr = sub2(rR, rL), dm = sub2(mR, mL), dn = sub2(nR, nL), dp = sub2(pR, pL);
    const float2 dq = __fmul2_rn(dp, ib);   // the jump of Q's last component p/beta
    const float2 ndr = sub2(rL, rR);        // -dr, exactly
    // central parts F(Q_L) + F(Q_R) first, so that the face states die here
    const float2 c0 = __fadd2_rn(mL, mR);
    const float2 c1 = __fadd2_rn(__ffma2_rn(mR, uR, __ffma2_rn(mL, uL, pL)), pR);
    const float2 c2c = __ffma2_rn(mR, vR, __fmul2_rn(mL, vL));
    const float2 c3 = __fadd2_rn(uL, uR);
    const float2 fb = dup2(4.0f * beta);
    const float tq[3] = {0.11270166537925831148f, 0.5f, 0.88729833462074168852f};
    const float wq[3] = {5.0f / 18.0f, 8.0f / 18.0f, 5.0f / 18.0f};
    float2 Sau, Se, Sue, Sve, Sg, Sh, SE;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float2 t = dup2(tq[j]), w = dup2(wq[j]);
        const float2 r = __ffma2_rn(t, dr, rL), m = __ffma2_rn(t, dm, mL), n = __ffma2_rn(t, dn, nL);
        const float2 ir = make_float2(Ar<float>::rcp(r.x), Ar<float>::rcp(r.y));
        const float2 u = __fmul2_rn(m, ir);
        const float2 c2 = __ffma2_rn(u, u, __fmul2_rn(fb, ir));
        const float2 ic = make_float2(rsqrtf(c2.x), rsqrtf(c2.y));
        const float2 c = __fmul2_rn(c2, ic);
        // l4 = u/2 + c/2, l5 = u/2 - c/2 (c/2 is exact, so one rounding each)
        const float2 hu = __fmul2_rn(dup2(0.5f), u);
        const float2 l4 = __ffma2_rn(dup2(0.5f), c, hu), l5 = __ffma2_rn(dup2(-0.5f), c, hu);
        const float2 au = make_float2(fabsf(u.x), fabsf(u.y));
        const float2 a = __fmul2_rn(__ffma2_rn(u, ndr, dm), ib);
        // k = w / c, taken out of G4, G5 as in osher_flux (the density cancels)
        const float2 k = __fmul2_rn(w, ic);
        const float2 G4 = __fmul2_rn(sub2(l4, au), __ffma2_rn(l4, a, dq));
        const float2 G5 = __fmul2_rn(__fadd2_rn(l5, au), __ffma2_rn(l5, a, dq));
        const float2 KG = __fmul2_rn(k, __fadd2_rn(G4, G5));
        const float2 E = __fmul2_rn(k, __ffma2_rn(G5, l5, __fmul2_rn(G4, l4)));
        // k (G4 l5 + G5 l4) = k (G4 + G5) u - E: Sh takes KG u and, after the
        // loop, minus the sum of E (there is no packed negation)
        if (j == 0) {
            Sau = __fmul2_rn(w, au);
            Se = __fmul2_rn(r, E);
            Sue = __fmul2_rn(m, E);
            Sve = __fmul2_rn(n, E);
            Sg = KG;
            Sh = __fmul2_rn(KG, u);
            SE = E;
        } else {
            Sau = __ffma2_rn(w, au, Sau);
            Se = __ffma2_rn(r, E, Se);
            Sue = __ffma2_rn(m, E, Sue);
            Sve = __ffma2_rn(n, E, Sve);
            Sg = __fadd2_rn(Sg, KG);
            Sh = __ffma2_rn(KG, u, Sh);
            SE = __fadd2_rn(SE, E);
        }
    }
    // 2F = F(Q_L) + F(Q_R) - D, D as in osher_flux
    F[0] = sub2(c0, __ffma2_rn(dr, Sau, Se));
    F[1] = sub2(c1, __ffma2_rn(dup2(beta), Sg, __ffma2_rn(dm, Sau, Sue)));
    F[2] = sub2(c2c, __ffma2_rn(dn, Sau, Sve));
    Sh = sub2(Sh, SE);
    F[3] = sub2(c3, sub2(__fmul2_rn(dq, Sau), Sh));
}

// Face flux of the solver RS, chosen at compile time so that a kernel built
// for one solver carries none of the others' registers.  The FP32 Osher flux
// of one face is always the packed form above, so every FP32 tile sweep (any
// tile shape, single tank or batch) evaluates a face's flux with the same
// rounded operations (the face states around it are plain arithmetic that
// the compiler may contract differently in different kernels); the
// column-strip sweep takes its faces in pairs (osher_flux_pair).
// With TWICE (FP64 only) every solver returns 2F.
template <int RS, typename T, bool TWICE = false>
__device__ __forceinline__ void riemann_flux(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR, T beta,
                                             T inv_beta, T F[4]) {
    static_assert(!TWICE || std::is_same<T, double>::value, "2F form is FP64 only");
    if constexpr (RS == kRoe) roe_flux<T, TWICE>(rL, uL, vL, pL, rR, uR, vR, pR, beta, inv_beta, F);
    else if constexpr (RS == kBassi) bassi_flux<T, TWICE>(rL, uL, vL, pL, rR, uR, vR, pR, beta, inv_beta, F);
    else if constexpr (std::is_same<T, float>::value) osher_flux_x2(rL, uL, vL, pL, rR, uR, vR, pR, beta, inv_beta, F);
    else osher_flux<T, TWICE>(rL, uL, vL, pL, rR, uR, vR, pR, beta, inv_beta, F);
}

}  // namespace acgb
