"""Batched tanks (ac_batch_*) through the C ABI.

A tank's numbers must not depend on the rest of the batch: the same tank
gives the same bits whatever other tanks share its batch.  Against a
single-tank context in the mixed form, a batched tank agrees bit for bit in
the column-strip sweep (same iteration counts and residual norms under the
stopping test too), and to round-off in the tile sweep.  The batch and
single-tank kernels share their arithmetic but not their compiled code, and
the compiler may fuse a product and a sum into one FMA in one kernel and not
in the other; in the tile sweep it does.  Against the FP64 oracle each tank
stays within the mixed form's 1e-5 relative field error.
"""
import numpy as np
import pytest

import oracle
from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def uneven_cases():
    cases = W.batched_tanks(count=6, nmin=20, nmax=90, seed=11)
    # add tanks of other kinds: ragged rectangle, open sides, periodic x
    cases.append(W.random_two_fluid(37, 19, ratio=300.0, c0=8.0, seed=3))
    cases.append(W.random_two_fluid(45, 21, ratio=50.0, c0=5.0, seed=4,
                                    bc=("transmissive", "slip", "noslip", "slip")))
    cases.append(W.random_two_fluid(33, 17, ratio=20.0, c0=4.0, seed=5,
                                    bc=("periodic", "periodic", "slip", "slip")))
    return cases


# batch against single tank where the compiled forms may differ: far below
# the 1e-5 bar against the oracle, far above FP32 round-off of a few steps
ROUND_OFF = 1e-6


def assert_same(got, ref, bitwise, what):
    if bitwise:
        for x, y in zip(got, ref):
            assert np.array_equal(x, y), what
    else:
        errs = rel_errors(got, ref)
        assert max(errs) <= ROUND_OFF, (what, errs)


def single_mixed(case, dt, tol, iters):
    t = ac.Tank.from_case(case, precision="mixed")
    rc, n = t.physical_step(dt, tol, iters)
    s = t.get_state()
    R, _ = t.residual_norms()
    t.close()
    return s, n, R


# single-tank variant of the same form as each batch variant: the tile
# sweep (32x8) for the tile variants, the strip sweep of the same strip
# height (32, 64, 128 rows) for the strip variants
SINGLE_OF_BATCH = {9: 15, 10: 16, 11: 17}
STRIP_BATCH, STRIP_SINGLE = "10", "16"   # 64-row strips in both


@pytest.mark.parametrize("form", ["tile", "strip"])
def test_batch_equals_single_tanks_fixed_iterations(monkeypatch, form):
    strip = form == "strip"
    monkeypatch.setenv("AC_BATCH_TILE", STRIP_BATCH if strip else "0")
    monkeypatch.setenv("AC_TILE", STRIP_SINGLE if strip else "0")
    cases = uneven_cases()
    b = ac.Batch.from_cases(cases)
    rc, its, st = b.physical_step(1e-3, -1.0, 7)
    assert its == [7] * len(cases) and st == [ac.AC_OK] * len(cases)
    for k, c in enumerate(cases):
        ref, _, _ = single_mixed(c, 1e-3, -1.0, 7)
        assert_same(b.get_state(k), ref, strip, k)
    assert b.tile_shape()[0] > 0
    b.close()


@pytest.mark.parametrize("v", [0, 10])
def test_tank_does_not_depend_on_the_rest_of_the_batch(monkeypatch, v):
    """The same tanks in a batch of their own, in another order, and next to
    other tanks: bit for bit the same."""
    monkeypatch.setenv("AC_BATCH_TILE", str(v))
    cases = uneven_cases()
    full = ac.Batch.from_cases(cases)
    full.physical_step(1e-3, -1.0, 6)
    picked = [8, 2, 6]
    others = W.batched_tanks(count=3, nmin=40, nmax=100, seed=77)
    mixed_in = [cases[8], others[0], cases[2], others[1], cases[6], others[2]]
    for sub_cases, where in (([cases[k] for k in picked], (0, 1, 2)), (mixed_in, (0, 2, 4))):
        b = ac.Batch.from_cases(sub_cases)
        b.physical_step(1e-3, -1.0, 6)
        for k, j in zip(picked, where):
            for x, y in zip(b.get_state(j), full.get_state(k)):
                assert np.array_equal(x, y), (k, j)
        b.close()
    full.close()


N_BATCH_VARIANTS = 15


@pytest.mark.parametrize("v", range(N_BATCH_VARIANTS))
def test_every_batch_variant_equals_single_tanks(monkeypatch, v):
    """Each compiled batch variant (tile shape, direct or prefetching
    loads, column strips), forced in place of the autotuner's pick, against
    single tanks run with the same form: bit for bit for the strips, to
    round-off for the tiles."""
    monkeypatch.setenv("AC_BATCH_TILE", str(v))
    monkeypatch.setenv("AC_TILE", str(SINGLE_OF_BATCH.get(v, 0)))
    cases = uneven_cases()
    b = ac.Batch.from_cases(cases)
    b.physical_step(1e-3, -1.0, 5)
    for k, c in enumerate(cases):
        ref, _, _ = single_mixed(c, 1e-3, -1.0, 5)
        assert_same(b.get_state(k), ref, v in SINGLE_OF_BATCH, k)
    b.close()


def test_batch_against_oracle():
    cases = uneven_cases()[:4] + uneven_cases()[6:]
    b = ac.Batch.from_cases(cases)
    b.physical_step(1e-3, -1.0, 8)
    for k, c in enumerate(cases):
        ref, *_ = oracle.physical_step(c, c.state(), dt=1e-3, tol=-1.0, max_iters=8)
        errs = rel_errors(b.get_state(k), ref)
        assert max(errs) <= 1e-5, (k, errs)
    b.close()


def test_per_tank_convergence_flags_and_counts(monkeypatch):
    """Each tank stops on its own test; counts, norms and states equal the
    tank run alone (the strip sweep in both, whose arithmetic compiles alike,
    and one partial-sum order for the norms).  Absolute residual floors, as
    the paper's own stopping rules are (the relative drop cannot pass here:
    the first iteration's rho v residual is round-off in columns that start
    in vertical balance)."""
    monkeypatch.setenv("AC_TILE", STRIP_SINGLE)
    monkeypatch.setenv("AC_BATCH_TILE", STRIP_BATCH)
    cases = W.batched_tanks(count=5, nmin=16, nmax=48, seed=21)
    for c in cases:
        c.options.abs_tol = (0.03, 0.3, 0.3, 100.0)
    b = ac.Batch.from_cases(cases)
    rc, its, st = b.physical_step(1e-3, 0.0, 2500)
    assert rc == ac.AC_OK and st == [ac.AC_OK] * len(cases), (rc, st)
    assert len(set(its)) == len(cases), its    # each tank stops at its own count
    for k, c in enumerate(cases):
        ref, n, R = single_mixed(c, 1e-3, 0.0, 2500)
        assert its[k] == n, (k, its[k], n)
        for x, y in zip(b.get_state(k), ref):
            assert np.array_equal(x, y)
        bR, _ = b.residual_norms(k)
        assert np.array_equal(bR, R)
    b.close()


def test_two_physical_steps_and_levels(monkeypatch):
    monkeypatch.setenv("AC_TILE", STRIP_SINGLE)
    monkeypatch.setenv("AC_BATCH_TILE", STRIP_BATCH)
    cases = W.batched_tanks(count=3, nmin=30, nmax=60, seed=5)
    b = ac.Batch.from_cases(cases)
    singles = [ac.Tank.from_case(c, precision="mixed") for c in cases]
    for step in range(2):
        b.physical_step([1e-3, 2e-3, 5e-4], -1.0, 5)
        for t, dt in zip(singles, [1e-3, 2e-3, 5e-4]):
            t.physical_step(dt, -1.0, 5)
    for k, t in enumerate(singles):
        for x, y in zip(b.get_state(k), t.get_state()):
            assert np.array_equal(x, y)
        t.close()
    b.close()


def test_nonfinite_tank_is_restored_alone():
    """A pseudo-CFL far beyond stability blows up the dynamic tank; the
    hydrostatic tank beside it is an exact steady state in the mixed form
    (zero residual, so any CFL leaves it put) and runs all its iterations."""
    rest = W.hydrostatic_tank(32)
    bad = W.random_two_fluid(32, 16, ratio=1000.0, c0=20.0, seed=2)
    o = ac.options_from(bad.options, "mixed")
    o.cfl_tau = 40.0
    b = ac.Batch.from_cases([rest, bad], options=o)
    before = b.get_state(1)
    with pytest.raises(ac.ACError) as e:
        b.physical_step(1e-3, -1.0, 300)
    assert e.value.code == ac.AC_ERR_NONFINITE
    for x, y in zip(before, b.get_state(1)):
        assert np.array_equal(x, y)
    got = b.get_state(0)
    assert np.abs(got[2]).max() == 0.0 and np.array_equal(got[0], rest.rho)
    b.close()


def test_bdf2_batch_equals_single_tanks():
    """BDF2 runs the tile sweep only: round-off agreement."""
    cases = W.batched_tanks(count=3, nmin=24, nmax=56, seed=8)
    for c in cases:
        c.options.bdf_order = 2
    b = ac.Batch.from_cases(cases)
    singles = [ac.Tank.from_case(c, precision="mixed") for c in cases]
    for step in range(3):
        b.physical_step(1e-3, -1.0, 6)
        for t in singles:
            t.physical_step(1e-3, -1.0, 6)
    for k, t in enumerate(singles):
        assert_same(b.get_state(k), t.get_state(), False, k)
        t.close()
    b.close()


def test_two_batches_alive_at_once(monkeypatch):
    """Two batches hold separate ranges of the constant descriptor table;
    stepping them in turn leaves each equal to its tanks run alone."""
    monkeypatch.setenv("AC_BATCH_TILE", STRIP_BATCH)
    monkeypatch.setenv("AC_TILE", STRIP_SINGLE)
    ca = uneven_cases()[:4]
    cb = W.batched_tanks(count=5, nmin=24, nmax=70, seed=31)
    a = ac.Batch.from_cases(ca)
    b = ac.Batch.from_cases(cb)
    for _ in range(2):
        a.physical_step(1e-3, -1.0, 4)
        b.physical_step(1e-3, -1.0, 4)
    for batch, cases in ((a, ca), (b, cb)):
        for k, c in enumerate(cases):
            t = ac.Tank.from_case(c, precision="mixed")
            t.physical_step(1e-3, -1.0, 4)
            t.physical_step(1e-3, -1.0, 4)
            ref = t.get_state()
            t.close()
            for x, y in zip(batch.get_state(k), ref):
                assert np.array_equal(x, y), k
    a.close()
    b.close()


def test_batch_larger_than_the_constant_table(monkeypatch):
    """170 small tanks do not fit the 160-slot constant table: the batch
    reads its descriptors from global memory, with the same results."""
    monkeypatch.setenv("AC_BATCH_TILE", STRIP_BATCH)
    monkeypatch.setenv("AC_TILE", STRIP_SINGLE)
    cases = W.batched_tanks(count=170, nmin=8, nmax=20, seed=41)
    b = ac.Batch.from_cases(cases)
    b.physical_step(1e-3, -1.0, 3)
    for k in (0, 1, 97, 169):
        ref, _, _ = single_mixed(cases[k], 1e-3, -1.0, 3)
        for x, y in zip(b.get_state(k), ref):
            assert np.array_equal(x, y), k
    b.close()
