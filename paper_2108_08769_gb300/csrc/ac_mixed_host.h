// ac_mixed_host.h -- host-side set-up of the mixed form's reference pressure
// (shared by the single-tank and batched contexts).
#pragma once

#include <cstddef>
#include <vector>

#include "../../include/ac.h"

namespace acgb {

inline bool is_wall_side(int b) { return b == AC_BC_WALL_SLIP || b == AC_BC_WALL_NOSLIP; }

// The hydrostatic reference applies when both y sides are walls and the
// pressure gradient comes from the rearranged momentum equation.
inline bool mixed_uses_reference(const ac_bc &bc, int gradp) {
    return is_wall_side(bc.ylo) && is_wall_side(bc.yhi) && gradp == AC_GRADP_NEW;
}

// From host fields f = (rho, rho u, rho v, p) of an nx x ny grid: the FP32
// reference density, its FP64 discrete hydrostatic columns p_ref (anchored at
// each column's top cell), the FP32 jump of p_ref across each cell's west
// x-face, and p' = p - p_ref in FP32.  Without a reference all are zero and
// p' = p.
struct MixedReference {
    std::vector<float> rho_ref, dref, p_prime;
    std::vector<double> p_ref;
};

inline void build_mixed_reference(int nx, int ny, double dy, double gy, const ac_bc &bc, bool use_ref,
                                  const double *const f[4], MixedReference &r) {
    const size_t N = (size_t)nx * ny;
    r.rho_ref.assign(N, 0.0f);
    r.dref.assign(N, 0.0f);
    r.p_prime.resize(N);
    r.p_ref.assign(N, 0.0);
    if (use_ref) {
        for (size_t k = 0; k < N; ++k) r.rho_ref[k] = float(f[0][k]);
        for (int i = 0; i < nx; ++i) {
            const size_t top = (size_t)(ny - 1) * nx + i;
            r.p_ref[top] = f[3][top];
            for (int j = ny - 2; j >= 0; --j) {
                const size_t k = (size_t)j * nx + i;
                r.p_ref[k] = r.p_ref[k + nx] - (double(r.rho_ref[k]) + double(r.rho_ref[k + nx])) * gy * dy / 2.0;
            }
        }
        const bool per_x = bc.xlo == AC_BC_PERIODIC;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const size_t k = (size_t)j * nx + i;
                if (i > 0) r.dref[k] = float(r.p_ref[k] - r.p_ref[k - 1]);
                else if (per_x) r.dref[k] = float(r.p_ref[k] - r.p_ref[k + nx - 1]);
            }
    }
    for (size_t k = 0; k < N; ++k) r.p_prime[k] = float(f[3][k] - r.p_ref[k]);
}

}  // namespace acgb
