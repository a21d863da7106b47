"""Pins for the oracle's seed grid, octant hill-climbing (Sec. 2.2, Alg. 1)
and uniform-target mean shift (Sec. 2.3, Eq. 4-6).

References: pure-Python enumeration of closed octants, 200-bit entropies
with an argmax/rounding re-evaluation of one climbing step, the per-voxel
form of Eq. 6 at 200 bits (the oracle regroups it per bin), symmetry and
special-case invariants.
"""
from fractions import Fraction

import mpmath as mp
import numpy as np
import pytest

from paper_1310_6736_b300 import synth


def _ball(r):
    return [(dx, dy, dz) for dz in range(-r, r + 1) for dy in range(-r, r + 1)
            for dx in range(-r, r + 1) if dx * dx + dy * dy + dz * dz <= r * r]


def _in_octant(j, o):
    sg = [(-1 if (j >> a) & 1 else 1) for a in range(3)]
    return all(o[a] * sg[a] >= 0 for a in range(3))


def _H(c):
    N = sum(c)
    if N <= 1:
        return mp.mpf(0)
    return -mp.fsum(mp.mpf(x) / N * mp.log(mp.mpf(x) / N) for x in c if x)


def test_seed_grid_counts(ko):
    assert ko.seed_grid((48, 48, 48), 6).shape[0] == 512
    assert ko.seed_grid((128, 128, 64), 8).shape[0] == 2048
    assert ko.seed_grid((256, 256, 160), 12).shape[0] == 5733
    g = ko.seed_grid((48, 48, 48), 6)
    assert g[0].tolist() == [3, 3, 3] and g[1].tolist() == [9, 3, 3] and g[-1].tolist() == [45] * 3


def test_octant_counts_brute_force(ko):
    rng = np.random.default_rng(4)
    B = 6
    bins = rng.integers(0, B + 1, size=(9, 9, 9)).astype(np.uint8)
    for p in ((4, 4, 4), (0, 3, 8), (8, 8, 1)):
        for r in (1, 2, 3, 5):
            for j in range(8):
                ref = [0] * B
                for o in _ball(r):
                    if not _in_octant(j, o):
                        continue
                    x, y, z = p[0] + o[0], p[1] + o[1], p[2] + o[2]
                    if 0 <= x < 9 and 0 <= y < 9 and 0 <= z < 9 and bins[z, y, x]:
                        ref[bins[z, y, x] - 1] += 1
                assert ko.octant_counts(bins, B, p, r, j).tolist() == ref


def _py_octant_step(ko, bins, B, r_min, r_max, p):
    """Alg. 1 in 3D from brute-force octant counts and 200-bit entropies.
    Returns the step, or None when a near-tie makes the FP64 decision
    legitimately ambiguous."""
    mp.mp.prec = 200
    eps, kopt = [], []
    for j in range(8):
        hs = [_H(ko.octant_counts(bins, B, p, r, j).tolist()) for r in range(r_min, r_max + 1)]
        m = max(hs)
        k = hs.index(m)
        near = [h for i, h in enumerate(hs) if i != k and abs(h - m) < 1e-9 and hs[i] != hs[k]]
        if near:
            return None
        eps.append(m)
        kopt.append(r_min + k)
    den = mp.fsum(eps)
    if den == 0:
        return [0, 0, 0]
    step = []
    for a in range(3):
        num = mp.fsum(eps[j] * kopt[j] * (-1 if (j >> a) & 1 else 1) for j in range(8))
        d = num / den
        frac = abs(d) - mp.floor(abs(d))
        if abs(frac - mp.mpf(0.5)) < 1e-9:
            return None
        step.append(int(mp.sign(d) * mp.floor(abs(d) + mp.mpf(0.5))))
    return step


def test_octant_step_vs_python_reevaluation(ko):
    rng = np.random.default_rng(8)
    checked = 0
    for trial in range(12):
        B = 8
        bins = rng.integers(1, B + 1, size=(14, 14, 14)).astype(np.uint8)
        # a high-entropy blob on a two-bin background
        bins[:] = rng.choice([2, 3], size=bins.shape, p=[0.9, 0.1])
        c = rng.integers(3, 11, size=3)
        zz, yy, xx = np.mgrid[0:14, 0:14, 0:14]
        blob = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= 9
        bins[blob] = rng.integers(1, B + 1, size=int(blob.sum()))
        p = tuple(int(v) for v in rng.integers(2, 12, size=3))
        ref = _py_octant_step(ko, bins, B, 1, 4, p)
        if ref is None:
            continue
        assert ko.octant_one_step(bins, B, 1, 4, p).tolist() == ref
        checked += 1
    assert checked >= 8


def test_octant_constant_volume_converges_immediately(ko):
    bins = np.full((20, 20, 20), 5, np.uint8)
    seeds = ko.seed_grid((20, 20, 20), 6)
    out = ko.octant_climb(bins, 16, 2, 6, seeds)
    assert (out["iters"] == 1).all() and (out["converged"] == 1).all()
    assert np.array_equal(out["xyz"], seeds)
    assert (out["s"] == 0).all()


def test_octant_mirror_symmetric_volume_gives_zero_step(ko):
    rng = np.random.default_rng(2)
    q = rng.integers(1, 9, size=(11, 11, 11)).astype(np.uint8)
    a = np.abs(np.arange(21) - 10)
    b2 = q[a[:, None, None], a[None, :, None], a[None, None, :]]   # mirror about (10,10,10)
    assert np.array_equal(b2, b2[:, :, ::-1]) and np.array_equal(b2, b2[:, ::-1, :]) \
        and np.array_equal(b2, b2[::-1])
    assert ko.octant_one_step(b2, 8, 2, 8, (10, 10, 10)).tolist() == [0, 0, 0]


def test_octant_seed_moves_toward_lone_sphere(ko):
    # Sanity: a seed a few voxels off a lone high-entropy sphere climbs towards it.
    rng = np.random.default_rng(6)
    bins = np.full((40, 40, 40), 3, np.uint8)
    zz, yy, xx = np.mgrid[0:40, 0:40, 0:40]
    sph = (xx - 20) ** 2 + (yy - 20) ** 2 + (zz - 20) ** 2 <= 36
    bins[sph] = rng.integers(1, 17, size=int(sph.sum()))
    seeds = np.array([[14, 20, 20], [20, 26, 21], [24, 17, 20]], np.int32)
    out = ko.octant_climb(bins, 16, 2, 8, seeds)
    for s0, s1 in zip(seeds, out["xyz"]):
        assert np.abs(s1 - 20).sum() < np.abs(s0 - 20).sum()


def test_octant_trajectory_bookkeeping(ko):
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    seeds = ko.seed_grid(w.dims, 6)[:64]
    out = ko.octant_climb(bins, 16, 2, 10, seeds, want_traj=True)
    for i in range(len(seeds)):
        t = out["traj"][i]
        assert np.array_equal(t[0], seeds[i]) and np.array_equal(t[-1], out["xyz"][i])
        moves = int((np.abs(np.diff(t, axis=0)).sum(axis=1) > 0).sum())
        assert moves == out["iters"][i] - out["converged"][i]


# ------------------------------------------------------------- mean shift
def _py_ms_delta(bins, B, p, r):
    """Eq. 6 per voxel at 200 bits: sum_s w(s) o_s / sum_s w(s) with
    w(s) = sqrt(q_b / p_b) (Eq. 5), q_b = 1/B, p_b = c_b / N (Eq. 4, flat)."""
    mp.mp.prec = 200
    nz, ny, nx = bins.shape
    vox = []
    for o in _ball(r):
        x, y, z = p[0] + o[0], p[1] + o[1], p[2] + o[2]
        if 0 <= x < nx and 0 <= y < ny and 0 <= z < nz and bins[z, y, x]:
            vox.append((o, int(bins[z, y, x]) - 1))
    N = len(vox)
    c = [0] * B
    for _, b in vox:
        c[b] += 1
    if N == 0:
        return [mp.mpf(0)] * 3, c
    w = [mp.sqrt((mp.mpf(1) / B) / (mp.mpf(c[b]) / N)) for _, b in vox]
    den = mp.fsum(w)
    return [mp.fsum(wi * o[a] for wi, (o, _) in zip(w, vox)) / den for a in range(3)], c


def test_meanshift_moments_brute_force(ko):
    rng = np.random.default_rng(12)
    B = 7
    bins = rng.integers(0, B + 1, size=(10, 11, 12)).astype(np.uint8)
    for p in ((5, 5, 5), (0, 0, 0), (11, 10, 9)):
        for r in (1, 3, 4):
            c, m = ko.ms_window(bins, B, p, r)
            rc, rm = [0] * B, [[0, 0, 0] for _ in range(B)]
            for o in _ball(r):
                x, y, z = p[0] + o[0], p[1] + o[1], p[2] + o[2]
                if 0 <= x < 12 and 0 <= y < 11 and 0 <= z < 10 and bins[z, y, x]:
                    b = bins[z, y, x] - 1
                    rc[b] += 1
                    for a in range(3):
                        rm[b][a] += o[a]
            assert c.tolist() == rc and m.tolist() == rm


def test_meanshift_first_step_vs_per_voxel_eq6(ko):
    rng = np.random.default_rng(13)
    checked = 0
    for trial in range(20):
        B = 8
        bins = rng.choice([2, 3], size=(16, 16, 16), p=[0.85, 0.15]).astype(np.uint8)
        c = rng.integers(4, 12, size=3)
        zz, yy, xx = np.mgrid[0:16, 0:16, 0:16]
        blob = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= 9
        bins[blob] = rng.integers(1, B + 1, size=int(blob.sum()))
        p = [int(v) for v in rng.integers(3, 13, size=3)]
        r = int(rng.integers(2, 6))
        delta, _ = _py_ms_delta(bins, B, p, r)
        if any(abs(abs(d) - mp.floor(abs(d)) - mp.mpf(0.5)) < 1e-9 for d in delta):
            continue
        step = [int(mp.sign(d) * mp.floor(abs(d) + mp.mpf(0.5))) for d in delta]
        exp = [min(max(p[a] + step[a], 0), 15) for a in range(3)]
        out = ko.meanshift(bins, B, r, r, np.array([p], np.int32), max_iter=1)
        assert out["xyz"][0].tolist() == exp
        checked += 1
    assert checked >= 15


def test_meanshift_single_bin_interior_does_not_move(ko):
    # One bin: every weight equal, Eq. 6 gives the window centroid = P.
    bins = np.full((30, 30, 30), 4, np.uint8)
    seeds = np.array([[15, 15, 15], [10, 12, 20]], np.int32)
    out = ko.meanshift(bins, 16, 2, 8, seeds)
    assert (out["iters"] == 1).all() and (out["converged"] == 1).all()
    assert np.array_equal(out["xyz"], np.repeat(seeds, 7, axis=0))
    # rho of a single-bin window against U[1..B] is sqrt(1/B); H = 0
    assert np.allclose(out["rho"], np.sqrt(1 / 16), rtol=0, atol=1e-15)
    assert (out["H"] == 0).all()


def test_meanshift_uniform_histogram_rho_is_one(ko):
    # A window whose histogram is exactly uniform over all B bins: rho = 1.
    B = 4
    bins = np.zeros((9, 9, 9), np.uint8)
    pts = _ball(1)                     # 7 voxels -> not divisible; use r=0 + pattern
    bins[4, 4, 4] = 1
    out = ko.meanshift(bins, 1, 0, 0, np.array([[4, 4, 4]], np.int32))
    assert out["rho"][0] == 1.0
    # 8 voxels of a 2x2x2 block, 2 per bin, seen by a ball of radius 1 plus
    # nothing else: build counts directly through the window view instead.
    bins = np.zeros((5, 5, 5), np.uint8)
    for k, o in enumerate(pts[1:]):     # the 6 face neighbours
        bins[2 + o[2], 2 + o[1], 2 + o[0]] = 1 + (k % 3)
    c, _ = ko.ms_window(bins, 3, (2, 2, 2), 1)
    assert c.tolist() == [2, 2, 2]
    out = ko.meanshift(bins, 3, 1, 1, np.array([[2, 2, 2]], np.int32), max_iter=0)
    assert abs(out["rho"][0] - 1.0) <= 4e-16


def test_meanshift_item_order_and_final_H(ko):
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    seeds = ko.seed_grid(w.dims, 6)[:20]
    out = ko.meanshift(bins, 16, 2, 10, seeds)
    S = 9
    for i in range(len(seeds) * S):
        r = 2 + i % S
        c = ko.window_counts(bins, 16, out["xyz"][i], r)
        assert out["H"][i] == ko.entropy(c, nmax=4169)
