"""Pins for the oracle's tables and window entropy (Sec. 2.1, Eq. 1-3).

Nothing here re-types the oracle's formula: the tables are checked against
an independent 200-bit evaluation, the entropy against the paper's closed
form (Eq. 2) and its monotonicity claim (Eq. 3), against -sum p ln p in
high precision, and against the special cases H = 0 and H = ln B.
"""
import os

import mpmath as mp
import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "eq2_mixture.txt")


def _rn(x):
    """Nearest binary64 to an mpmath value (mpmath rounds to nearest)."""
    return float(x)


def test_tables_correctly_rounded(ko):
    mp.mp.prec = 200
    T, L = ko.tables(137065)
    assert T[0] == 0.0 and T[1] == 0.0 and L[1] == 0.0
    rng = np.random.default_rng(11)
    cs = list(range(2, 3001)) + sorted(set(rng.integers(3001, 137066, size=1500).tolist())) + [137065]
    for c in cs:
        mc = mp.mpf(c)
        lc = mp.log(mc)
        assert T[c] == _rn(mc * lc), c
        assert L[c] == _rn(lc), c


def test_entropy_constant_window_is_zero(ko):
    # Sec. 2.1: alpha = 0 (window entirely in the homogeneous background) gives H = 0.
    for B in (16, 32, 64):
        for n in (1, 2, 7, 4169, 137065):
            c = np.zeros(B, np.int64)
            c[B // 3] = n
            assert ko.entropy(c, nmax=137065) == 0.0


def test_entropy_uniform_fill_is_log_B(ko):
    # Sec. 2.1: alpha = 1 (uniform over M bins) gives H = log M.
    for B in (2, 16, 32, 64):
        for k in (1, 3, 100, 2000):
            c = np.full(B, k, np.int64)
            assert abs(ko.entropy(c, nmax=B * k) - np.log(B)) <= 1e-13 * np.log(B)


def test_entropy_matches_eq2_mixture(ko):
    # Eq. 2: window = background delta (n0 voxels) + uniform over M bins (n1 each).
    rows = [l.split() for l in open(GOLD) if not l.startswith("#")]
    assert len(rows) >= 20
    for M, n0, n1, H in rows:
        M, n0, n1, H = int(M), int(n0), int(n1), float(H)
        c = np.full(M, n1, np.int64)
        c[0] += n0
        got = ko.entropy(c, nmax=int(c.sum()))
        assert abs(got - H) <= 1e-12 * max(1.0, abs(H)), (M, n0, n1, got, H)


def test_entropy_monotone_in_overlap_eq3(ko):
    # Eq. 3: dH/dalpha > 0 on (0, 1).  Hold N fixed and move voxels from the
    # background into the uniform part: H must increase strictly.
    for M in (4, 16, 64):
        N = M * 60
        prev = -1.0
        for n1 in range(0, 61):
            c = np.full(M, n1, np.int64)
            c[0] += N - M * n1
            h = ko.entropy(c, nmax=N)
            assert h > prev
            prev = h
        assert abs(prev - np.log(M)) < 1e-12


def test_eq3_derivative_is_the_derivative_of_eq2():
    # Cross-check the paper's two formulas against each other (and so our
    # reading of Eq. 2 used above): central difference of Eq. 2 vs Eq. 3.
    mp.mp.dps = 50
    for M in (2, 8, 64):
        for a in (0.05, 0.3, 0.7, 0.95):
            Mm, am = mp.mpf(M), mp.mpf(a)

            def H(x):
                g = x / Mm + 1 - x
                return -(g * mp.log(g)) - x * (Mm - 1) / Mm * mp.log(x / Mm)

            h = mp.mpf("1e-20")
            fd = (H(am + h) - H(am - h)) / (2 * h)
            eq3 = (Mm - 1) / Mm * mp.log((am + Mm * (1 - am)) / am)
            assert abs(fd - eq3) < mp.mpf("1e-15")
            assert eq3 > 0


def test_entropy_vs_high_precision_definition(ko):
    # Eq. 1 with p_b = c_b / N, evaluated at 200 bits.
    mp.mp.prec = 200
    rng = np.random.default_rng(5)
    for _ in range(300):
        B = int(rng.choice([16, 32, 64]))
        c = rng.integers(0, 50, size=B) * (rng.random(B) < 0.5)
        c = c.astype(np.int64)
        N = int(c.sum())
        if N == 0:
            continue
        ref = -mp.fsum(mp.mpf(int(x)) / N * mp.log(mp.mpf(int(x)) / N) for x in c if x > 0)
        got = ko.entropy(c, nmax=max(N, 1))
        assert abs(got - float(ref)) <= 1e-13 * max(1.0, np.log(N)), (got, ref)


@pytest.mark.parametrize("B", [16, 64])
def test_entropy_bin_permutation_invariance_is_not_assumed(ko, B):
    # The sum order is fixed (bin order), so a permuted histogram may differ
    # by rounding only; both must agree with the definition to 1e-13.
    rng = np.random.default_rng(B)
    c = rng.integers(0, 1000, size=B).astype(np.int64)
    p = rng.permutation(c)
    assert abs(ko.entropy(c) - ko.entropy(p)) <= 1e-13 * np.log(c.sum())
