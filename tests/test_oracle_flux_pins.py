"""Pins of the oracle's Roe and Bassi fluxes (Sec. 2.4.1, 2.4.2) against
what the mathematics fixes, independently of the oracle's own formulas.

Roe.  The paper's Roe averages are the state Q~ at which the Jacobian
satisfies Roe's property  A(Q~) (Q_R - Q_L) = F(Q_R) - F(Q_L).  The tests
find that state numerically from the property alone (scipy root finding
on finite-difference Jacobians of the flux), take |A~| from numpy's
eigen-decomposition and compare the whole flux.  A consequence is pinned
too: across a single discontinuity that satisfies the jump conditions the
Roe flux is the upwind flux of that wave.

Bassi.  The flux is F_x,inv of the exact solution at x/tau = 0.  The star
states are pinned by the Rankine-Hugoniot relations (test_oracle_pins.py);
here the state at the interface is picked from the ordered wave speeds of
the fan, and the flux compared with F_x,inv of it.

Planted mistakes: each test is also run against copies of the oracle built
with one deliberate slip (a swapped sqrt(rho) weight, an arithmetic-mean
density, a flipped dissipation sign, the wrong side of the contact, the
tangential velocity from the wrong side); every copy must fail at least one
of the pins.  The copies are compiled from oracle/ac_oracle.c into a
temporary directory on the CPU.
"""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.optimize import fsolve

import oracle
from paper_2108_08769_gb300 import workloads as W

_D = C.POINTER(C.c_double)
SRC = os.path.join(os.path.dirname(oracle.__file__), "ac_oracle.c")


class Flux:
    """The oracle's x-direction solvers from one build of ac_oracle.c."""

    def __init__(self, L):
        self.L = L
        for name in ("orc_flux_x",):
            getattr(L, name).argtypes = [_D, C.c_double, _D]
        for name in ("orc_roe_x", "orc_bassi_x"):
            getattr(L, name).argtypes = [_D, _D, C.c_double, _D]
        L.orc_bassi_star.argtypes = [_D, _D, C.c_double, _D]

    @staticmethod
    def _v(x, n):
        return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))

    def flux(self, Q, beta):
        Q = self._v(Q, 5)
        F = np.zeros(5)
        self.L.orc_flux_x(Q.ctypes.data_as(_D), beta, F.ctypes.data_as(_D))
        return F

    def solver(self, kind, QL, QR, beta):
        QL, QR = self._v(QL, 5), self._v(QR, 5)
        F = np.zeros(5)
        fn = self.L.orc_roe_x if kind == "roe" else self.L.orc_bassi_x
        fn(QL.ctypes.data_as(_D), QR.ctypes.data_as(_D), beta, F.ctypes.data_as(_D))
        return F

    def star(self, WL, WR, beta):
        WL, WR = self._v(WL, 4), self._v(WR, 4)
        out = np.zeros(6)
        self.L.orc_bassi_star(WL.ctypes.data_as(_D), WR.ctypes.data_as(_D), beta, out.ctypes.data_as(_D))
        return out


def _oracle_flux():
    return Flux(oracle.lib())


_MUTANT_DIR = tempfile.mkdtemp(prefix="orc_mutants_")


def _mutant(name, old, new):
    """A copy of the oracle with `old` replaced by `new` (exactly once)."""
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path_c = os.path.join(_MUTANT_DIR, f"{name}.c")
    path_so = os.path.join(_MUTANT_DIR, f"{name}.so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                           f"-I{os.path.dirname(SRC)}", "-o", path_so, path_c, "-lm"])
    return Flux(C.CDLL(path_so))


# ----------------------------------------------------------------- inputs

def _pairs(n, seed):
    """Random face-state pairs in Q = (rho, rho u, rho v, rho w, p/beta) with
    all velocity components different on the two sides."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        beta = rng.uniform(0.5, 3.0)
        qs = []
        for _side in range(2):
            rho = rng.uniform(0.2, 3.0)
            u, v, w = rng.uniform(-1.0, 1.0, 3)
            p = rng.uniform(-1.0, 1.0)
            qs.append(np.array([rho, rho * u, rho * v, rho * w, p / beta]))
        out.append((qs[0], qs[1], beta))
    return out


def _fd_jacobian(fx, Q, beta, h=1e-7):
    cols = []
    for e in np.eye(5):
        cols.append((fx.flux(Q + h * e, beta) - fx.flux(Q - h * e, beta)) / (2 * h))
    return np.array(cols).T


# ----------------------------------------------------------------- Roe

def _roe_state_from_property_u(fx, QL, QR, beta):
    """(rho~, u~, v~, w~) with A(Q~) dQ = dF (rows 2-5; the mass row holds
    for any state), found by root finding from the arithmetic means.  Of the
    two roots of the quadratic in u~, Roe's is the one between u_L and u_R."""
    dQ, dF = QR - QL, fx.flux(QR, beta) - fx.flux(QL, beta)

    def g(x):
        r, u, v, w = x
        Qt = np.array([r, r * u, r * v, r * w, 0.0])
        return (_fd_jacobian(fx, Qt, beta) @ dQ - dF)[1:]

    uL, uR = QL[1] / QL[0], QR[1] / QR[0]
    x0 = [0.5 * (QL[0] + QR[0]), 0.5 * (uL + uR), 0.5 * (QL[2] / QL[0] + QR[2] / QR[0]),
          0.5 * (QL[3] / QL[0] + QR[3] / QR[0])]
    x, info, ier, msg = fsolve(g, x0, full_output=True, xtol=1e-10)
    # (the finite-difference Jacobians limit the attainable residual to ~1e-9)
    assert np.abs(g(x)).max() < 1e-7 * max(np.abs(dF).max(), 1.0), msg
    assert min(uL, uR) - 1e-9 <= x[1] <= max(uL, uR) + 1e-9
    return x


def _numpy_roe(fx, QL, QR, beta):
    r, u, v, w = _roe_state_from_property_u(fx, QL, QR, beta)
    Qt = np.array([r, r * u, r * v, r * w, 0.0])
    ev, V = np.linalg.eig(_fd_jacobian(fx, Qt, beta))
    absA = (V @ np.diag(np.abs(ev)) @ np.linalg.inv(V)).real
    return 0.5 * (fx.flux(QL, beta) + fx.flux(QR, beta) - absA @ (QR - QL))


def _pin_roe_property_u(fx):
    for QL, QR, beta in _pairs(20, 11):
        expect = _numpy_roe(fx, QL, QR, beta)
        got = fx.solver("roe", QL, QR, beta)
        if not np.allclose(got, expect, rtol=1e-6, atol=1e-6):
            return False
    return True


def _single_waves(fx, n, seed):
    """Pairs of states joined by one wave of the exact solution, with its
    speed: left acoustic wave, contact, right acoustic wave (star states
    from the exact solver, whose jump conditions test_oracle_pins.py pins)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        beta = rng.uniform(0.5, 3.0)
        WL = [rng.uniform(0.2, 3.0), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)]
        WR = [rng.uniform(0.2, 3.0), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)]
        SL, SR, us, ps, rsL, rsR = fx.star(WL, WR, beta)

        def Q(r, u, v, p):
            return np.array([r, r * u, r * v, 0.0, p / beta])

        QL, QR = Q(*WL), Q(*WR)
        QsL, QsR = Q(rsL, us, WL[2], ps), Q(rsR, us, WR[2], ps)
        out += [(QL, QsL, SL, beta), (QsL, QsR, us, beta), (QsR, QR, SR, beta)]
    return out


def _pin_roe_upwind_on_single_waves(fx):
    """Across one discontinuity dF = S dQ, so Roe's property makes dQ an
    eigenvector of A~ with eigenvalue S: the flux is F(Q_L) for S > 0 and
    F(Q_R) for S < 0."""
    for QL, QR, S, beta in _single_waves(fx, 12, 5):
        up = fx.flux(QL, beta) if S > 0 else fx.flux(QR, beta)
        got = fx.solver("roe", QL, QR, beta)
        if not np.allclose(got, up, rtol=1e-10, atol=1e-10 * max(np.abs(up).max(), 1.0)):
            return False
    return True


def test_roe_averages_satisfy_property_u():
    """Sec. 2.4.2: the flux equals 1/2 (F_L + F_R - |A~| dQ) with Q~ found from
    Roe's property alone and |A~| from numpy's eigen-decomposition."""
    assert _pin_roe_property_u(_oracle_flux())


def test_roe_is_upwind_across_a_single_wave():
    fx = _oracle_flux()
    waves = _single_waves(fx, 12, 5)
    assert any(S > 0 for _, _, S, _ in waves) and any(S < 0 for _, _, S, _ in waves)
    assert _pin_roe_upwind_on_single_waves(fx)


# ----------------------------------------------------------------- Bassi

def _fan_state_at_interface(fx, QL, QR, beta):
    """State at x/tau = 0 of the exact solution: the waves are ordered
    S_L < u* < S_R and the state between the two speeds around 0 is taken;
    tangential velocities change only across the contact."""
    WL = [QL[0], QL[1] / QL[0], QL[2] / QL[0], beta * QL[4]]
    WR = [QR[0], QR[1] / QR[0], QR[2] / QR[0], beta * QR[4]]
    wL, wR = QL[3] / QL[0], QR[3] / QR[0]
    SL, SR, us, ps, rsL, rsR = fx.star(WL, WR, beta)
    if not SL < us < SR:
        return None, us   # the contact overtakes an acoustic wave: outside the solver's assumption
    regions = [  # (upper speed of the region, state in it)
        (SL, (WL[0], WL[1], WL[2], wL, WL[3])),
        (us, (rsL, us, WL[2], wL, ps)),
        (SR, (rsR, us, WR[2], wR, ps)),
        (np.inf, (WR[0], WR[1], WR[2], wR, WR[3])),
    ]
    for upper, (r, u, v, w, p) in regions:
        if 0.0 <= upper:   # x/tau = 0 lies at or below this region's upper edge
            return np.array([r, r * u, r * v, r * w, p / beta]), us


def _pin_bassi_fan_state(fx):
    signs = set()
    used = 0
    for QL, QR, beta in _pairs(40, 13):
        Q0, us = _fan_state_at_interface(fx, QL, QR, beta)
        if Q0 is None:
            continue
        used += 1
        signs.add(us > 0)
        got = fx.solver("bassi", QL, QR, beta)
        if not np.allclose(got, fx.flux(Q0, beta), rtol=1e-12, atol=1e-12):
            return False
    assert used >= 20 and signs == {True, False}   # both star regions sampled
    return True


def test_bassi_flux_is_the_flux_of_the_fan_state_at_the_interface():
    """Sec. 2.4.1: the Bassi flux is F_x,inv of the exact solution at x/tau = 0,
    from random pairs landing in both star regions (the acoustic speeds
    (u -+ c)/2 always straddle 0 here, as c > |u|).  Pairs whose contact
    would overtake an acoustic wave, where the paper notes the solver's
    assumption breaks down, are left out."""
    assert _pin_bassi_fan_state(_oracle_flux())


# ----------------------------------------------------------------- planted mistakes

MUTANTS = [
    ("roe_swapped_sqrt_weight", "double ut = (sL * uL + sR * uR) / (sL + sR);",
     "double ut = (sR * uL + sL * uR) / (sL + sR);"),
    ("roe_v_weight_swapped", "double vt = (sL * vL + sR * vR) / (sL + sR);",
     "double vt = (sR * vL + sL * vR) / (sL + sR);"),
    ("roe_arithmetic_mean_density", "double rt = sqrt(rL * rR);", "double rt = 0.5 * (rL + rR);"),
    ("roe_dissipation_sign", "F[r] = 0.5 * (FL[r] + FR[r] - d);", "F[r] = 0.5 * (FL[r] + FR[r] + d);"),
    ("bassi_wrong_star_side", "} else if (xi <= st[2]) {", "} else if (xi >= st[2]) {"),
    ("bassi_tangential_from_right", "W[0] = st[4]; W[1] = st[2]; W[2] = WL[2]; W[3] = st[3];",
     "W[0] = st[4]; W[1] = st[2]; W[2] = WR[2]; W[3] = st[3];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_flux_mistake_fails_a_pin(name, old, new):
    fx = _mutant(name, old, new)
    if name.startswith("roe"):
        caught = not _pin_roe_property_u(fx) or not _pin_roe_upwind_on_single_waves(fx)
    else:
        try:
            caught = not _pin_bassi_fan_state(fx)
        except AssertionError:
            caught = True
    assert caught, f"{name} passed every flux pin"


# ----------------------------------------------------------------- Riemann problems

@pytest.mark.parametrize("kind", ["bassi", "roe"])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_other_solvers_converge_on_riemann_problems(kind, k):
    """Sec. 3.1: on RP1-RP4 all three solvers perform almost identically; with
    the Bassi and Roe fluxes the L1 error against the exact solution falls
    under refinement 100 -> 200 -> 400 cells, and at 400 cells the profile
    is within a few per cent of Osher's."""
    rL, rR, uL, uR, pL, pR, beta, tau = W.RIEMANN_TABLE[k]
    errs, gaps = [], []
    for nx in (100, 200, 400):
        rp = W.riemann_problem(k, nx)
        rp.options.riemann = kind
        q, status, its = oracle.pseudo_time_run(rp, rp.state(), rp.tau_end)
        assert status == oracle.OK
        ro = W.riemann_problem(k, nx)
        qo, *_ = oracle.pseudo_time_run(ro, ro.state(), ro.tau_end)
        ex = np.array([oracle.bassi_sample([rL, uL, 0, pL], [rR, uR, 0, pR], beta, x / tau) for x in rp.x])
        scale = np.abs(ex).max(axis=0) + 1e-30
        e, g = [], []
        for f, (a, b) in enumerate(((q[0][0], qo[0][0]), (q[1][0] / q[0][0], qo[1][0] / qo[0][0]),
                                    (q[3][0], qo[3][0]))):
            col = (0, 1, 3)[f]
            s = max(scale[col], 1e-3)
            e.append(np.abs(a - ex[:, col]).mean() / s)
            g.append(np.abs(a - b).mean() / s)
        errs.append(e)
        gaps.append(g)
    errs = np.array(errs)
    for f in range(3):
        if errs[0, f] < 1e-12:
            assert errs[2, f] < 1e-12
            continue
        assert errs[1, f] < errs[0, f] and errs[2, f] < errs[1, f], errs
        assert errs[2, f] < 0.15
    assert max(gaps[-1]) < 0.05, gaps
