"""Fixed-point emulation of the paper's inversion methods (Sec. IV.C, Fig. 1).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: nothing in the CUDA
library calls it.  The paper compares the numerical accuracy of the proposed
method (Sec. IV.A, Eqs. 20-24) with Equation Solving (Sec. III.A, Eq. 15) and
Triangular Matrix Operations (Sec. III.B, Eqs. 16-19) by fixed-point
simulation, and reports in Fig. 1 that the proposed method has the lowest
average norm error.  The figure and the word lengths behind it are not in the
text, so Fig. 1 itself is parity unpinned; this module restates the three
methods over a pluggable scalar arithmetic so that the comparison can be run
for stated word lengths:

  FloatArith   IEEE binary64, the same operations in the same order as the C
               oracle (oracle.c), so the two agree bit for bit (a pin of this
               restatement against the pinned C code).
  FixedArith   signed Q(I.F) numbers held as Python integers (value q 2^-F,
               I integer bits, word length 1 + I + F), round to nearest on
               every product, quotient and square root, saturation at the
               word's range (counted).  Dot products either round every
               product ("round", a plain fixed-point datapath) or keep the
               exact products in a wide accumulator and round once ("wide",
               a DSP multiply-accumulate unit).

Real matrices only.  Every function follows the loop order of its C
counterpart: orc_chol_d (Sec. II, Eqs. 3-4), orc_inv_rows_d (Sec. IV.A),
orc_es_d (Sec. III.A), orc_tmo_d (Sec. III.B).
"""
from __future__ import annotations

import math


class FloatArith:
    """IEEE binary64 with the C oracle's operation order."""
    name = "float64"

    def __init__(self):
        self.zero, self.one = 0.0, 1.0

    def q(self, x):
        return float(x)

    def val(self, r):
        return float(r)

    def sub(self, a, b):
        return a - b

    def div(self, a, b):
        return a / b

    def sqrt(self, a):
        return math.sqrt(a)

    def positive(self, a):
        return a > 0.0 and math.isfinite(a)

    def msub(self, init, pairs):
        """init - sum a*b, the terms subtracted one at a time in order."""
        s = init
        for a, b in pairs:
            s -= a * b
        return s

    def madd(self, init, pairs):
        """init + sum a*b, the terms added one at a time in order."""
        s = init
        for a, b in pairs:
            s += a * b
        return s


def _round_shift(v: int, f: int) -> int:
    """v / 2^f rounded to nearest (ties away from zero)."""
    if f == 0:
        return v
    h = 1 << (f - 1)
    return (v + h) >> f if v >= 0 else -((-v + h) >> f)


def _round_div(a: int, b: int) -> int:
    """a / b rounded to nearest (ties away from zero); b != 0."""
    neg = (a < 0) != (b < 0)
    a, b = abs(a), abs(b)
    q = (2 * a + b) // (2 * b)
    return -q if neg else q


class FixedArith:
    """Signed Q(I.F): values q 2^-F with |q| < 2^(I+F), rounded to nearest."""

    def __init__(self, frac_bits: int, int_bits: int, accumulate: str = "round"):
        if accumulate not in ("round", "wide"):
            raise ValueError("accumulate is 'round' or 'wide'")
        self.F, self.I, self.acc = int(frac_bits), int(int_bits), accumulate
        self.max = (1 << (self.I + self.F)) - 1
        self.min = -(1 << (self.I + self.F))
        self.saturations = 0
        self.zero, self.one = 0, self._sat(1 << self.F)
        self.name = f"Q{self.I}.{self.F}/{accumulate}"

    def _sat(self, v: int) -> int:
        if v > self.max:
            self.saturations += 1
            return self.max
        if v < self.min:
            self.saturations += 1
            return self.min
        return v

    def q(self, x):
        return self._sat(int(round(float(x) * (1 << self.F))))

    def val(self, r):
        return r / float(1 << self.F)

    def sub(self, a, b):
        return self._sat(a - b)

    def mul(self, a, b):
        return self._sat(_round_shift(a * b, self.F))

    def div(self, a, b):
        if b == 0:
            self.saturations += 1
            return self.max if a >= 0 else self.min
        return self._sat(_round_div(a << self.F, b))

    def sqrt(self, a):
        """sqrt of a value >= 0, rounded to nearest: isqrt(a 2^F) corrected
        upward when the remainder exceeds r (then (r + 1/2)^2 < a 2^F)."""
        v = a << self.F
        r = math.isqrt(v)
        if v - r * r > r:
            r += 1
        return self._sat(r)

    def positive(self, a):
        return a > 0

    def msub(self, init, pairs):
        if self.acc == "round":
            s = init
            for a, b in pairs:
                s = self._sat(s - self.mul(a, b))
            return s
        acc = init << self.F
        for a, b in pairs:
            acc -= a * b
        return self._sat(_round_shift(acc, self.F))

    def madd(self, init, pairs):
        if self.acc == "round":
            s = init
            for a, b in pairs:
                s = self._sat(s + self.mul(a, b))
            return s
        acc = init << self.F
        for a, b in pairs:
            acc += a * b
        return self._sat(_round_shift(acc, self.F))


# ---------------------------------------------------------------------------
# The methods.  A, R, X, M are lists of rows of arithmetic values; only the
# upper triangle of A is read, and X is returned with its upper half filled
# (zeros below), like the C oracle.
# ---------------------------------------------------------------------------

def chol(ar, A):
    """Sec. II, Eqs. 3-4, row by row (orc_chol_d).  Returns (R, info)."""
    n = len(A)
    R = [[ar.zero] * n for _ in range(n)]
    for i in range(n):
        t = ar.msub(A[i][i], [(R[k][i], R[k][i]) for k in range(i)])
        if not ar.positive(t):
            return R, i + 1
        rii = ar.sqrt(t)
        R[i][i] = rii
        for j in range(i + 1, n):
            s = ar.msub(A[i][j], [(R[k][i], R[k][j]) for k in range(i)])
            R[i][j] = ar.div(s, rii)
    return R, 0


def inv_proposed(ar, R):
    """Sec. IV.A, Eqs. 20-24: R X = S with s_ii = 1/r_ii, rows N..1, within a
    row j = N..i+1 then the diagonal (orc_inv_rows_d)."""
    n = len(R)
    X = [[ar.zero] * n for _ in range(n)]
    for i in range(n - 1, -1, -1):
        rii = R[i][i]
        for j in range(n - 1, i, -1):
            s = ar.madd(ar.zero, [(R[i][k], X[k][j] if k <= j else X[j][k]) for k in range(i + 1, n)])
            X[i][j] = ar.div(ar.sub(ar.zero, s), rii)
        s = ar.madd(ar.zero, [(R[i][k], X[i][k]) for k in range(i + 1, n)])
        X[i][i] = ar.div(ar.sub(ar.div(ar.one, rii), s), rii)
    return X


def inv_es(ar, R):
    """Sec. III.A, Eq. 15: R^* b = e_j forward, then R x_j = b backward for
    rows i <= j, columns j = N..1 (orc_es_d)."""
    n = len(R)
    X = [[ar.zero] * n for _ in range(n)]
    for j in range(n - 1, -1, -1):
        b = [ar.zero] * n
        for k in range(j, n):
            s = ar.msub(ar.one if k == j else ar.zero, [(R[l][k], b[l]) for l in range(k)])
            b[k] = ar.div(s, R[k][k])
        for i in range(j, -1, -1):
            s = ar.madd(ar.zero, [(R[i][l], X[l][j] if l <= j else X[j][l]) for l in range(i + 1, n)])
            X[i][j] = ar.div(ar.sub(b[i], s), R[i][i])
    return X


def inv_tmo(ar, R, exploit=False):
    """Sec. III.B, Eqs. 16-19: M = R^{-1} from R m_i = e_i, then X = M M^*,
    upper half (orc_tmo_d)."""
    n = len(R)
    M = [[ar.zero] * n for _ in range(n)]
    for i in range(n):
        for k in range(i, -1, -1):
            lend = i + 1 if exploit else n
            s = ar.msub(ar.one if k == i else ar.zero, [(R[k][l], M[l][i]) for l in range(k + 1, lend)])
            M[k][i] = ar.div(s, R[k][k])
    X = [[ar.zero] * n for _ in range(n)]
    for i in range(n):
        for j in range(i, n):
            X[i][j] = ar.madd(ar.zero, [(M[i][l], M[j][l]) for l in range(j, n)])
    return X


METHODS = {"proposed": inv_proposed, "equation_solving": inv_es, "triangular_ops": inv_tmo}


def to_arith(ar, A):
    return [[ar.q(x) for x in row] for row in A]


def from_arith(ar, X):
    return [[ar.val(x) for x in row] for row in X]


def invert(ar, A_float, method):
    """Quantise A (nested lists or a 2-D array of floats), factor, invert by
    `method`; returns (X as floats, upper half, info)."""
    A = to_arith(ar, [list(map(float, row)) for row in A_float])
    R, info = chol(ar, A)
    if info:
        return None, info
    return from_arith(ar, METHODS[method](ar, R)), 0


def study(sizes=(4, 8, 16), kappas=(1e1, 1e2, 1e3), frac_bits=(12, 16, 20, 24), accumulate=("round", "wide"),
          count=100, seed=2024):
    """Mean relative Frobenius error (upper half of X against the FP64 inverse
    of the quantised A) of each method, for A = Q diag(lambda) Q^T / kappa with
    lambda log-uniform on [1, kappa] (lambda_1 = 1, lambda_N = kappa), so that
    |a_ij| <= 1 and |x_ij| <= kappa.  I = ceil(log2 kappa) + 2 integer bits.
    Returns a list of dict rows."""
    import numpy as np

    from paper_1111_4144_gb300 import workloads as wl

    rows = []
    for N in sizes:
        for kappa in kappas:
            b = wl.fixed_kappa(count, N, kappa, seed=seed + N, layout=wl.LAYOUT_DENSE)
            mats = b.A.reshape(count, N, N) / kappa
            ibits = int(math.ceil(math.log2(kappa))) + 2
            for F in frac_bits:
                for acc in accumulate:
                    errs = {m: [] for m in METHODS}
                    sats = {m: 0 for m in METHODS}
                    fails = 0
                    for k in range(count):
                        ar0 = FixedArith(F, ibits, acc)
                        A = mats[k]
                        Aq = np.triu(np.array(from_arith(ar0, to_arith(ar0, A.tolist()))))
                        Aq = Aq + np.triu(Aq, 1).T
                        ref = np.triu(np.linalg.inv(Aq))
                        for m in METHODS:
                            ar = FixedArith(F, ibits, acc)
                            X, info = invert(ar, A, m)
                            if info:
                                fails += 1
                                continue
                            errs[m].append(float(np.linalg.norm(np.triu(np.array(X)) - ref) / np.linalg.norm(ref)))
                            sats[m] += ar.saturations
                    row = {"N": N, "kappa": kappa, "int_bits": ibits, "frac_bits": F, "accumulate": acc,
                           "matrices": count, "factor_failures": fails}
                    for m in METHODS:
                        row[f"{m}_mean_err"] = float(np.mean(errs[m])) if errs[m] else None
                        row[f"{m}_saturations"] = sats[m]
                    best = min(METHODS, key=lambda m: row[f"{m}_mean_err"] if row[f"{m}_mean_err"] is not None
                               else math.inf)
                    row["lowest"] = best
                    rows.append(row)
    return rows
