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

// The pressure is carried as an FP32 increment over an FP64 level when the
// pressure gradient comes from the rearranged momentum equation; a limited
// pressure gradient needs pressure differences, so there the FP32 record
// holds p itself.
inline bool mixed_uses_level(int gradp) { return gradp == AC_GRADP_NEW; }

// From host fields f = (rho, rho u, rho v, p) of an nx x ny grid: the FP32
// reference density, its FP64 discrete hydrostatic columns p_ref (anchored at
// each column's top cell; empty without a reference), and the initial
// pressure record and level: (FP32 dp = 0, FP64 p^n = p) with a pressure
// level, (FP32 p, 0) without.
struct MixedReference {
    std::vector<float> rho_ref, p_record;
    std::vector<double> p_ref, p_level;
};

inline void build_mixed_reference(int nx, int ny, double dy, double gy, bool use_ref, bool plevel,
                                  const double *const f[4], MixedReference &r) {
    const size_t N = (size_t)nx * ny;
    r.rho_ref.assign(N, 0.0f);
    r.p_ref.clear();
    if (use_ref) {
        r.p_ref.assign(N, 0.0);
        for (size_t k = 0; k < N; ++k) r.rho_ref[k] = float(f[0][k]);
        for (int i = 0; i < nx; ++i) {
            const size_t top = (size_t)(ny - 1) * nx + i;
            r.p_ref[top] = f[3][top];
            for (int j = ny - 2; j >= 0; --j) {
                const size_t k = (size_t)j * nx + i;
                r.p_ref[k] = r.p_ref[k + nx] - (double(r.rho_ref[k]) + double(r.rho_ref[k + nx])) * gy * dy / 2.0;
            }
        }
    }
    r.p_record.resize(N);
    r.p_level.resize(N);
    for (size_t k = 0; k < N; ++k) {
        r.p_record[k] = plevel ? 0.0f : float(f[3][k]);
        r.p_level[k] = plevel ? f[3][k] : 0.0;
    }
}

}  // namespace acgb
