"""Pins of the oracle's quadrant climb: Alg. 1 as printed, in 2D (Sec. 2.2),
run in each seed's z-slice with disk windows."""
import math

import numpy as np


def _brute_step(bins, B, r_min, r_max, p):
    """One quadrant step written out from Alg. 1: closed quadrants of the
    disk of radius k in P's slice, entropy -sum p ln p of each, eps_j = max
    over k (smallest k on ties), delta = sum_j eps_j k_j sigma_j / sum eps."""
    nz, ny, nx = bins.shape
    x0, y0, z0 = p
    eps, kopt = [0.0] * 4, [r_min] * 4
    for k in range(r_min, r_max + 1):
        for j in range(4):
            sx, sy = (-1 if j & 1 else 1), (-1 if j & 2 else 1)
            c = [0] * B
            for dy in range(-k, k + 1):
                for dx in range(-k, k + 1):
                    if dx * dx + dy * dy > k * k or dx * sx < 0 or dy * sy < 0:
                        continue
                    x, y = x0 + dx, y0 + dy
                    if 0 <= x < nx and 0 <= y < ny and bins[z0, y, x]:
                        c[bins[z0, y, x] - 1] += 1
            n = sum(c)
            h = 0.0 if sum(1 for v in c if v) <= 1 else -sum(v / n * math.log(v / n) for v in c if v)
            if k == r_min or h > eps[j] + 1e-12:
                eps[j], kopt[j] = h, k
    den = sum(eps)
    if den == 0.0:
        return [0, 0, 0]
    out = []
    for a in range(2):
        num = sum(eps[j] * kopt[j] * (-1 if j & (1 << a) else 1) for j in range(4))
        d = num / den
        out.append(int(math.copysign(math.floor(abs(d) + 0.5), d)))
    return out + [0]


def test_quadrant_step_equals_brute_force(ko):
    rng = np.random.default_rng(3)
    bins = rng.integers(0, 6, size=(5, 23, 21)).astype(np.uint8)
    bins[:, 8:14, 5:12] = rng.integers(1, 6, size=(5, 6, 7))
    for p in [(10, 11, 2), (3, 4, 0), (18, 20, 4), (7, 12, 1), (0, 0, 3)]:
        got = ko.octant_one_step(bins, 5, 2, 5, p, planar=True)
        assert list(got) == _brute_step(bins, 5, 2, 5, p), p


def test_quadrant_climb_stays_in_its_slice_and_ignores_the_others(ko):
    rng = np.random.default_rng(8)
    bins = rng.integers(1, 9, size=(6, 30, 30)).astype(np.uint8)
    seeds = np.array([[7, 7, 2], [20, 15, 2], [15, 25, 2]], np.int32)
    a = ko.octant_climb(bins, 8, 2, 7, seeds, planar=True, want_traj=True)
    assert (a["xyz"][:, 2] == 2).all() and (a["traj"][:, :, 2] == 2).all()
    other = bins.copy()
    other[[0, 1, 3, 4, 5]] = rng.integers(0, 9, size=(5, 30, 30))
    b = ko.octant_climb(other, 8, 2, 7, seeds, planar=True, want_traj=True)
    for k in ("xyz", "iters", "converged", "s", "traj"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["Y"], b["Y"])


def test_mirror_symmetric_slice_gives_no_step(ko):
    rng = np.random.default_rng(4)
    q = rng.integers(1, 7, size=(9, 9)).astype(np.uint8)
    half = np.concatenate([q[:, ::-1], q[:, :1], q], axis=1)          # symmetric in x
    sl = np.concatenate([half[::-1], half[:1], half], axis=0)          # and in y
    bins = np.stack([sl, sl[::-1, ::-1]]).astype(np.uint8)
    assert list(ko.octant_one_step(bins, 6, 2, 7, (9, 9, 0), planar=True)) == [0, 0, 0]
