"""Pins for the fixed-point emulation of the paper's methods (oracle/fixedpoint.py,
Sec. IV.C / Fig. 1).  CPU only.

  - in IEEE binary64 the Python restatement reproduces the pinned C oracle bit
    for bit (Cholesky, the proposed inverse, Equation Solving, Triangular
    Matrix Operations in both counting variants);
  - integer and power-of-two inputs are inverted exactly in fixed point by
    every method and both accumulation modes;
  - the error falls as 2^-F with the fraction bits F, and with 64 fraction
    bits it is below the binary64 oracle's own error;
  - values outside the word's range are counted as saturations;
  - Equation Solving and the proposed method agree bit for bit;
  - the stored study table (tests/golden/fixedpoint_study.json) is
    reproduced by re-running one of its rows.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fixedpoint as fp
from paper_1111_4144_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fixedpoint_study.json")


def rand_spd(rng, n):
    B = rng.standard_normal((n, n))
    return B @ B.T + n * np.eye(n)


def as_lists(M):
    return [list(map(float, row)) for row in M]


@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_float_restatement_matches_c_oracle(orc, n):
    rng = np.random.default_rng(300 + n)
    A = rand_spd(rng, n)
    ar = fp.FloatArith()
    R, info = fp.chol(ar, as_lists(A))
    Rc, infoc = orc.chol(A)
    assert info == infoc == 0
    R = np.array(R)
    assert np.array_equal(R, Rc)
    assert np.array_equal(np.array(fp.inv_proposed(ar, as_lists(R))), orc.inv_rows(Rc))
    assert np.array_equal(np.array(fp.inv_es(ar, as_lists(R))), orc.es(Rc))
    for ex in (False, True):
        assert np.array_equal(np.array(fp.inv_tmo(ar, as_lists(R), exploit=ex)), orc.tmo(Rc, exploit=ex))


@pytest.mark.parametrize("acc", ["round", "wide"])
@pytest.mark.parametrize("method", list(fp.METHODS))
def test_integer_inputs_exact(method, acc):
    """a_ij = min(i, j) (1-based): R is all ones, X = tridiag(-1, 2, -1) with
    x_NN = 1; every intermediate is an integer, so Q(4.8) is exact."""
    n = 6
    A = [[float(min(i, j) + 1) for j in range(n)] for i in range(n)]
    ar = fp.FixedArith(8, 4, acc)
    X, info = fp.invert(ar, A, method)
    assert info == 0 and ar.saturations == 0
    want = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1)
    want[-1, -1] = 1.0
    assert np.array_equal(np.triu(np.array(X)), want)


@pytest.mark.parametrize("acc", ["round", "wide"])
@pytest.mark.parametrize("method", list(fp.METHODS))
def test_powers_of_two_exact(method, acc):
    """A = diag(2^-2, 2^-4, 2^-6): R = diag(2^-1, 2^-2, 2^-3) and
    X = diag(4, 16, 64), all representable in Q(8.12)."""
    A = np.diag([2.0 ** -2, 2.0 ** -4, 2.0 ** -6])
    ar = fp.FixedArith(12, 8, acc)
    X, info = fp.invert(ar, as_lists(A), method)
    assert info == 0 and ar.saturations == 0
    assert np.array_equal(np.array(X), np.diag([4.0, 16.0, 64.0]))


def test_primitives_round_to_nearest():
    """Products, quotients and square roots against exact rationals: the
    result is the nearest representable value (ties away from zero)."""
    from fractions import Fraction
    F = 10
    ar = fp.FixedArith(F, 20, "round")
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a, b = (int(x) for x in rng.integers(-(1 << 18), 1 << 18, size=2))
        exact = Fraction(a * b, 1 << F)              # in units of 2^-F
        got = ar.mul(a, b)
        assert abs(Fraction(got) - exact) <= Fraction(1, 2)
        if abs(Fraction(got) - exact) == Fraction(1, 2):
            assert abs(got) > abs(exact)
        if b != 0:
            exact = Fraction(a << F, b)
            got = ar.div(a, b)
            assert abs(Fraction(got) - exact) <= Fraction(1, 2)
            if abs(Fraction(got) - exact) == Fraction(1, 2):
                assert abs(got) > abs(exact)
        v = abs(a)
        r = ar.sqrt(v)                               # nearest to sqrt(v 2^-F) 2^F = sqrt(v 2^F)
        assert (2 * r - 1) ** 2 <= 4 * (v << F) <= (2 * r + 1) ** 2
    assert ar.saturations == 0


def _mean_err(F, acc, method, mats, ibits):
    errs = []
    for A in mats:
        ar = fp.FixedArith(F, ibits, acc)
        Aq = np.array(fp.from_arith(ar, fp.to_arith(ar, as_lists(A))))
        Aq = np.triu(Aq) + np.triu(Aq, 1).T
        ref = np.triu(np.linalg.inv(Aq))
        X, info = fp.invert(ar, A, method)
        assert info == 0 and ar.saturations == 0
        errs.append(np.linalg.norm(np.triu(np.array(X)) - ref) / np.linalg.norm(ref))
    return float(np.mean(errs))


@pytest.mark.parametrize("acc", ["round", "wide"])
@pytest.mark.parametrize("method", list(fp.METHODS))
def test_error_halves_per_fraction_bit(method, acc):
    """Eight more fraction bits divide the mean error by about 2^8."""
    kappa, N = 1e2, 8
    mats = wl.fixed_kappa(12, N, kappa, seed=77, layout=wl.LAYOUT_DENSE).A.reshape(12, N, N) / kappa
    ibits = int(math.ceil(math.log2(kappa))) + 2
    e16 = _mean_err(16, acc, method, mats, ibits)
    e24 = _mean_err(24, acc, method, mats, ibits)
    ratio = e24 / e16
    assert 2.0 ** -10 <= ratio <= 2.0 ** -6, ratio


@pytest.mark.parametrize("method", list(fp.METHODS))
def test_wide_words_agree_with_binary64(orc, method):
    """With 64 fraction bits the fixed-point result differs from the binary64
    oracle by about the oracle's own rounding error."""
    kappa, N = 1e2, 10
    A = wl.fixed_kappa(1, N, kappa, seed=78, layout=wl.LAYOUT_DENSE).A.reshape(N, N) / kappa
    ar = fp.FixedArith(64, 9, "round")
    X, info = fp.invert(ar, as_lists(A), method)
    assert info == 0 and ar.saturations == 0
    Aq = np.array(fp.from_arith(ar, fp.to_arith(ar, as_lists(A))))
    Rc, _ = orc.chol(np.triu(Aq) + np.triu(Aq, 1).T)
    ref = orc.inv_rows(Rc)
    err = np.linalg.norm(np.triu(np.array(X)) - ref) / np.linalg.norm(ref)
    assert err <= 1e-14 * kappa, err


@pytest.mark.parametrize("method", list(fp.METHODS))
def test_out_of_range_values_saturate(method):
    """kappa = 1e3 needs about 10 integer bits for X; with 2 they saturate."""
    kappa, N = 1e3, 6
    A = wl.fixed_kappa(1, N, kappa, seed=79, layout=wl.LAYOUT_DENSE).A.reshape(N, N) / kappa
    ar = fp.FixedArith(16, 2, "round")
    fp.invert(ar, as_lists(A), method)
    assert ar.saturations > 0


@pytest.mark.parametrize("acc", ["round", "wide"])
def test_equation_solving_equals_proposed(acc):
    """Equation Solving's forward solve gives b_i = 0 (i < j) and b_j = 1/r_jj,
    exactly the s_ij of Eq. 24, and its back solve then takes the proposed
    method's steps: the two agree bit for bit in fixed point too."""
    kappa, N = 1e2, 9
    mats = wl.fixed_kappa(6, N, kappa, seed=80, layout=wl.LAYOUT_DENSE).A.reshape(6, N, N) / kappa
    for A in mats:
        Xs = []
        for m in ("proposed", "equation_solving"):
            ar = fp.FixedArith(14, 9, acc)
            Xs.append(fp.invert(ar, as_lists(A), m)[0])
        assert Xs[0] == Xs[1]


def test_stored_study_reproduces():
    with open(GOLDEN) as f:
        rec = json.load(f)
    rows = rec["rows"]
    assert len(rows) == len(rec["params"]["sizes"]) * len(rec["params"]["kappas"]) * \
        len(rec["params"]["frac_bits"]) * len(rec["params"]["accumulate"])
    pick = [r for r in rows if r["N"] == 4 and r["kappa"] == 100.0 and r["frac_bits"] == 16]
    assert len(pick) == 2
    for r in pick:
        again = fp.study(sizes=(4,), kappas=(100.0,), frac_bits=(16,), accumulate=(r["accumulate"],),
                         count=rec["params"]["count"], seed=rec["params"]["seed"])[0]
        for m in fp.METHODS:
            assert again[f"{m}_mean_err"] == pytest.approx(r[f"{m}_mean_err"], rel=1e-9)
            assert again[f"{m}_saturations"] == r[f"{m}_saturations"]
