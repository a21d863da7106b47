"""Pins for the oracle's binning, window histograms, inter-scale weight and
dense Kadir-Brady sweep (Sec. 1, Sec. 2.1, Sec. 2.2 post-filter).

References used here are independent of the oracle's code: pure-Python
enumeration of Ball(r), exact rational arithmetic (fractions) for W, 200-bit
logarithms for H, numpy float32 for the affine binning, and exhaustive
enumeration of every uint8 / int16 input value.
"""
from fractions import Fraction
import math

import mpmath as mp
import numpy as np
import pytest

from paper_1310_6736_b300 import synth


# ----------------------------------------------------------------- binning
def test_bin_u8_exhaustive(ko):
    v = np.arange(256, dtype=np.uint8)
    for bins, shift in ((16, 4), (32, 3), (64, 2)):
        got = ko.bin_volume(v, {"kind": 0, "bins": bins, "shift": shift, "lo": 0, "hi": 255})
        assert got.tolist() == [(x >> shift) + 1 for x in range(256)]


def test_bin_i16_exhaustive(ko):
    v = np.arange(-32768, 32768, dtype=np.int32).astype(np.int16)
    for bins, shift in ((32, 6), (64, 5)):
        got = ko.bin_volume(v, {"kind": 0, "bins": bins, "shift": shift, "lo": 0, "hi": 2047})
        ref = (np.clip(v.astype(np.int64), 0, 2047) >> shift) + 1
        assert np.array_equal(got, ref.astype(np.uint8))


def test_bin_window_excludes_outside(ko):
    v = np.arange(-100, 3000, dtype=np.int32).astype(np.int16)
    got = ko.bin_volume(v, {"kind": 2, "bins": 32, "shift": 5, "lo": 100, "hi": 1123})
    vv = v.astype(np.int64)
    ref = np.where((vv < 100) | (vv > 1123), 0, ((vv - 100) >> 5) + 1)
    assert np.array_equal(got, ref.astype(np.uint8))


def test_bin_f32_matches_numpy_float32(ko):
    vol = synth.workload("pet128").volume
    got = ko.bin_volume(vol, {"kind": 1, "bins": 32, "shift": 0, "lo": 0, "hi": 0})
    v = vol.astype(np.float32)
    vmin, vmax = np.float32(v.min()), np.float32(v.max())
    d = np.float32(np.float32(vmax - vmin) + np.float32(1e-6))
    q = (np.float32(32.0) * (v - vmin)) / d
    ref = np.clip(np.floor(q).astype(np.int64), 0, 31) + 1
    assert q.dtype == np.float32
    assert np.array_equal(got, ref.astype(np.uint8))
    assert got.min() == 1 and got.max() == 32


# -------------------------------------------------------------- histograms
def _ball(r):
    return [(dx, dy, dz) for dz in range(-r, r + 1) for dy in range(-r, r + 1)
            for dx in range(-r, r + 1) if dx * dx + dy * dy + dz * dz <= r * r]


def _py_counts(bins, B, p, r):
    nz, ny, nx = bins.shape
    c = [0] * B
    for dx, dy, dz in _ball(r):
        x, y, z = p[0] + dx, p[1] + dy, p[2] + dz
        if 0 <= x < nx and 0 <= y < ny and 0 <= z < nz and bins[z, y, x]:
            c[bins[z, y, x] - 1] += 1
    return c


def test_ball_sizes_by_enumeration(ko):
    for r in range(0, 11):
        assert ko.ball_size(r) == len(_ball(r))
    assert [ko.ball_size(r) for r in (10, 20, 32)] == [4169, 33401, 137065]


def test_window_counts_brute_force_tiny(ko):
    rng = np.random.default_rng(3)
    B = 5
    bins = rng.integers(0, B + 1, size=(6, 7, 8)).astype(np.uint8)  # 0 = not counted
    for z in range(6):
        for y in range(7):
            for x in range(8):
                for r in (0, 1, 2, 4):
                    got = ko.window_counts(bins, B, (x, y, z), r)
                    assert got.tolist() == _py_counts(bins, B, (x, y, z), r)


def test_interior_window_total_is_ball_size(ko):
    bins = np.ones((30, 30, 30), np.uint8)
    for r in range(0, 13):
        assert ko.window_counts(bins, 4, (15, 15, 15), r).sum() == ko.ball_size(r)


# ----------------------------------------------------------------- weight W
def _frac_weight(c, cp, r, w_norm=0):
    N, Np = sum(c), sum(cp)
    if N == 0 or Np == 0:
        return Fraction(0)
    s = sum(abs(Fraction(a, N) - Fraction(b, Np)) for a, b in zip(c, cp))
    f = Fraction(1) if w_norm == 1 else Fraction(r * r, 2 * r - 1)
    return f * s


def test_weight_exact_rational(ko):
    rng = np.random.default_rng(7)
    for _ in range(500):
        B = int(rng.choice([3, 16, 64]))
        cp = rng.integers(0, 30, size=B)
        c = cp + rng.integers(0, 30, size=B)
        r = int(rng.integers(2, 33))
        for wn in (0, 1):
            ref = _frac_weight(c.tolist(), cp.tolist(), r, wn)
            got = ko.weight(c, cp, r, wn)
            # two roundings (the quotient, then the product with f)
            assert abs(Fraction(got) - ref) <= abs(ref) * Fraction(1, 2 ** 51), (got, float(ref))


def test_weight_zero_for_identical_pdfs(ko):
    c = np.array([3, 0, 9, 12], np.int64)
    assert ko.weight(4 * c, c, 5) == 0.0
    assert ko.weight(c, c, 9) == 0.0


# ---------------------------------------------------------------- dense KB
def _py_kb(bins, B, p, r_min, r_max, w_norm=0):
    """Kadir-Brady at one centre from pure-Python counts, 200-bit H and
    rational W; returns (H list, W list, candidate peak list)."""
    mp.mp.prec = 200
    counts = [_py_counts(bins, B, p, r) for r in range(r_min, r_max + 1)]
    H = []
    for c in counts:
        N = sum(c)
        H.append(mp.mpf(0) if N <= 1 else
                 -mp.fsum(mp.mpf(x) / N * mp.log(mp.mpf(x) / N) for x in c if x))
    W = [Fraction(0)] + [_frac_weight(counts[i], counts[i - 1], r_min + i, w_norm)
                         for i in range(1, len(counts))]
    return H, W


def test_dense_brute_vs_python_tiny(ko):
    rng = np.random.default_rng(9)
    B, r_min, r_max = 4, 1, 4
    bins = rng.integers(1, B + 1, size=(7, 8, 9)).astype(np.uint8)
    bins[rng.random(bins.shape) < 0.1] = 0
    Y, s, Hs, Ws = ko.dense(bins, B, r_min, r_max, want_hw=True)
    Hs = Hs.reshape(7, 8, 9, -1)
    Ws = Ws.reshape(7, 8, 9, -1)
    checked = 0
    for z in range(7):
        for y in range(8):
            for x in range(9):
                H, W = _py_kb(bins, B, (x, y, z), r_min, r_max)
                for i in range(len(H)):
                    assert abs(Hs[z, y, x, i] - float(H[i])) <= 1e-13
                    assert abs(Fraction(Ws[z, y, x, i]) - W[i]) <= abs(W[i]) * Fraction(1, 2 ** 51)
                # peak decision where no near-tie could flip it
                margins = [abs(H[i] - H[i + 1]) for i in range(len(H) - 1)]
                if min(margins) < 1e-9:
                    continue
                best, sb = None, 0
                for i in range(1, len(H) - 1):
                    if H[i - 1] < H[i] and H[i] >= H[i + 1]:
                        yv = H[i] * mp.mpf(W[i].numerator) / W[i].denominator
                        if sb == 0 or yv > best:
                            best, sb = yv, r_min + i
                assert s[z, y, x] == sb
                if sb:
                    assert abs(Y[z, y, x] - float(best)) <= 1e-12 * max(1.0, float(best))
                else:
                    assert Y[z, y, x] == 0.0
                checked += 1
    assert checked > 300


def test_dense_shell_incremental_equals_brute(ko):
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)[10:26, 12:30, 5:25].copy()
    Y0, s0, H0, W0 = ko.dense(bins, 16, 2, 10, want_hw=True, brute=False)
    Y1, s1, H1, W1 = ko.dense(bins, 16, 2, 10, want_hw=True, brute=True)
    assert np.array_equal(H0, H1) and np.array_equal(W0, W1)
    assert np.array_equal(Y0, Y1) and np.array_equal(s0, s1)


def test_dense_constant_volume_has_no_peaks(ko):
    bins = np.full((12, 12, 12), 3, np.uint8)
    Y, s = ko.dense(bins, 16, 2, 6)
    assert (Y == 0).all() and (s == 0).all()


def test_dense_centre_list_matches_full_sweep(ko):
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    Y, s = ko.dense(bins, 16, 2, 10)
    rng = np.random.default_rng(1)
    cen = np.stack([rng.integers(0, 48, 200) for _ in range(3)], axis=1)
    Yc, sc = ko.dense(bins, 16, 2, 10, centres=cen)
    assert np.array_equal(Yc, Y[cen[:, 2], cen[:, 1], cen[:, 0]])
    assert np.array_equal(sc, s[cen[:, 2], cen[:, 1], cen[:, 0]])


def test_dense_sphere_centres_peak_near_radius(ko):
    # Sanity (not parity): at a planted sphere's centre the best scale is the
    # sphere's own radius give or take a voxel or two.
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    cen = np.array([c for c, r in w.meta["spheres"]], np.int32)
    Y, s = ko.dense(bins, 16, 2, 10, centres=cen)
    for (c, r), sb in zip(w.meta["spheres"], s):
        if 2 < r < 10:
            assert abs(int(sb) - r) <= 2, (c, r, sb)
