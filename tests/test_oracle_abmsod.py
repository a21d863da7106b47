"""Pins of the oracle's adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3,
Alg. 2, Eq. 7) against closed forms, a plain fp64 evaluation of one
iteration, and symmetries of the definition."""
import math

import numpy as np
import pytest

import oracle as ko


def _lattice_ball(r):
    """Integer offsets with |o|^2 <= r^2 (the first window of an item with
    H = r^2 I when 1/r^2 is exact in binary32, i.e. r a power of two)."""
    pts = []
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                if dx * dx + dy * dy + dz * dz <= r * r:
                    pts.append((dx, dy, dz))
    return np.array(pts, dtype=np.int64)


def test_kernel_is_exp_of_minus_half_d():
    """k(d) = exp(-d/2) (Alg. 2) to within two binary32 ulps on [0, 1]."""
    assert ko.ab_kernel(0.0) == 1.0
    for d in np.linspace(0.0, 1.0, 4001, dtype=np.float32):
        want = math.exp(-0.5 * float(d))
        got = ko.ab_kernel(float(d))
        assert abs(got - want) <= 2 * np.spacing(np.float32(want)), (d, got, want)


@pytest.mark.parametrize("r", [2, 4, 8])
def test_homogeneous_region_closed_form(r):
    """One bin everywhere: HP = e_b, so rho = sqrt(1/B) every iteration; the
    window is symmetric about an integer centre, so the centre never moves;
    rho never rises after the first iteration, so the best bandwidth is the
    first update, 5 (E[o o^T] + I/12) over the lattice ball
    = diag(5 S2 / N + 5/12)."""
    B = 4
    n = 2 * r + 24
    bins = np.full((n, n, n), 2, np.uint8)
    seed = np.array([[n // 2, n // 2 + 1, n // 2 - 1]], np.int32)
    res = ko.abmsod(bins, B, r, r + 1, seed, max_iter=6)
    pts = _lattice_ball(r)
    S2 = float((pts[:, 0] ** 2).sum())
    N = float(len(pts))
    i = 0   # the r item
    assert res["rho"][i] == 0.5
    assert res["iters"][i] == 6 and res["stopped"][i] == 0
    assert np.array_equal(res["x"][i], seed[0].astype(float))
    H = res["H"][i]
    for k in (1, 2, 4):
        assert H[k] == 0.0
    for k in (0, 3, 5):
        assert H[k] == pytest.approx(5.0 * S2 / N + 5.0 / 12.0, rel=1e-14)
    # the r + 1 item sees the same region: same rho and a fixed centre
    assert res["rho"][1] == 0.5
    assert np.array_equal(res["x"][1], seed[0].astype(float))
    # one iteration evaluates the ball twice (at x and at x' = x)
    one = ko.abmsod(bins, B, r, r + 1, seed, max_iter=1)
    assert one["voxels"][0] == 2 * len(pts)


@pytest.mark.parametrize("e", [(2, 1, 0), (-1, 0, 3), (0, -2, -2)])
def test_single_odd_voxel_shift(e):
    """A homogeneous window with one voxel of the other bin at offset e:
    with w_b = sqrt(HQ_b / HP_b) the odd voxel weighs more, and the Eq. 6
    step is (w_o - w_m) k_e e / (w_m (K - k_e) + w_o k_e), K the kernel sum
    of the ball, k_e = exp(-|e|^2 / (2 r^2))."""
    r, B, n = 4, 2, 24
    bins = np.full((n, n, n), 1, np.uint8)
    c = np.array([12, 11, 13])
    bins[c[2] + e[2], c[1] + e[1], c[0] + e[0]] = 2
    res = ko.abmsod(bins, B, r, r + 1, c[None, :].astype(np.int32), max_iter=1)
    pts = _lattice_ball(r)
    k = np.exp(-(pts ** 2).sum(1) / (2.0 * r * r))
    K = k.sum()
    ke = math.exp(-sum(v * v for v in e) / (2.0 * r * r))
    wo = math.sqrt((1.0 / B) / (ke / K))
    wm = math.sqrt((1.0 / B) / ((K - ke) / K))
    step = (wo - wm) * ke * np.array(e, float) / (wm * (K - ke) + wo * ke)
    got = res["x"][0] - c
    assert np.all(np.abs(got - step) < 5e-5), (got, step)
    assert res["iters"][0] == 1


def _fp64_iteration(bins, B, seed, r):
    """One iteration of Alg. 2 in fp64 with the exact Gaussian profile and
    no fixed-point sums; returns (x_new, H_new, rho, min |d - 1| of the
    second window)."""
    nz, ny, nx = bins.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(float)
    v = bins.ravel().astype(int)
    Hinv = np.eye(3) / (r * r)

    def window(x):
        o = s - x
        d = np.einsum("ia,ab,ib->i", o, Hinv, o)
        m = (d <= 1.0) & (v > 0)
        return o[m], d[m], v[m] - 1, np.abs(d - 1.0).min()

    def weights(d, b):
        kk = np.exp(-0.5 * d)
        hp = np.bincount(b, weights=kk, minlength=B) / kk.sum()
        return kk, hp, np.where(hp > 0, np.sqrt((1.0 / B) / np.where(hp > 0, hp, 1.0)), 0.0)

    x = np.array(seed, float)
    o, d, b, _ = window(x)
    kk, _, w = weights(d, b)
    t = kk * w[b]
    xn = x + (t[:, None] * o).sum(0) / t.sum()
    o2, d2, b2, gap = window(xn)
    _, hp2, w2 = weights(d2, b2)
    ww = w2[b2]
    Hn = 5.0 * (np.einsum("i,ia,ib->ab", ww, o2, o2) / ww.sum() + np.eye(3) / 12.0)
    for a in range(3):
        Hn[a, a] = max(Hn[a, a], 1.0)
    rho = np.sqrt(hp2 / B).sum()
    return xn, Hn, rho, gap


def _blob_volume(seed=7):
    """Background bin 1, an oblique ellipsoid of bin 3, 10% of voxels set
    to bins 2 / 4 at random."""
    rng = np.random.default_rng(seed)
    n = 28
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.stack([xx - 13.3, yy - 14.1, zz - 12.7], -1).astype(float)
    R = np.array([[0.8, 0.6, 0.0], [-0.6, 0.8, 0.0], [0.0, 0.0, 1.0]])
    q = u @ R.T
    inside = (q[..., 0] / 6.0) ** 2 + (q[..., 1] / 3.0) ** 2 + (q[..., 2] / 4.0) ** 2 <= 1.0
    bins = np.where(inside, 3, 1).astype(np.uint8)
    noise = rng.random(bins.shape) < 0.1
    bins[noise] = rng.choice([2, 4], size=int(noise.sum())).astype(np.uint8)
    return bins


def test_one_iteration_matches_fp64_evaluation():
    """The fixed-point / binary32 evaluation of one iteration agrees with a
    plain fp64 evaluation of Alg. 2 and Eq. 7 within the rounding of the
    sums (r = 4: the first window is the exact lattice ball)."""
    bins = _blob_volume()
    B, r = 4, 4
    seeds = [(10, 12, 11), (16, 15, 13), (13, 9, 12), (18, 17, 14), (9, 16, 12), (14, 14, 8)]
    checked = 0
    for sd in seeds:
        xn, Hn, rho, gap = _fp64_iteration(bins, B, sd, r)
        if gap < 1e-4:
            continue   # a voxel on the second window's boundary: membership is rounding-decided
        res = ko.abmsod(bins, B, r, r + 1, np.array([sd], np.int32), max_iter=1)
        H = res["H"][0]
        Hm = np.array([[H[0], H[1], H[2]], [H[1], H[3], H[4]], [H[2], H[4], H[5]]])
        assert np.all(np.abs(res["x"][0] - xn) < 1e-4), (sd, res["x"][0], xn)
        assert np.all(np.abs(Hm - Hn) < 2e-3 + 1e-4 * np.abs(Hn)), (sd, Hm, Hn)
        assert abs(res["rho"][0] - rho) < 1e-6, (sd, res["rho"][0], rho)
        checked += 1
    assert checked >= 4


def test_axis_swap_symmetry():
    """Swapping x and y in the volume and the seeds swaps the centre and the
    H entries (00 <-> 11, 02 <-> 12); rho and the iteration count agree.
    The evaluation walks x-rows, so the swap changes the rounding only:
    agreement to rounding level, with a rare item allowed to take another
    path."""
    bins = _blob_volume(11)
    B = 4
    rng = np.random.default_rng(3)
    seeds = rng.integers(4, 24, size=(40, 3)).astype(np.int32)
    a = ko.abmsod(bins, B, 3, 6, seeds, max_iter=8)
    bt = np.ascontiguousarray(bins.transpose(0, 2, 1))
    st = seeds[:, [1, 0, 2]].copy()
    b = ko.abmsod(bt, B, 3, 6, st, max_iter=8)
    same = ((np.abs(a["x"] - b["x"][:, [1, 0, 2]]) < 1e-4).all(1) &
            (np.abs(a["H"] - b["H"][:, [3, 1, 4, 0, 2, 5]]) < 1e-3 * (1 + np.abs(a["H"]))).all(1) &
            (np.abs(a["rho"] - b["rho"]) < 1e-6) & (a["iters"] == b["iters"]))
    assert same.mean() >= 0.95, same.mean()


def test_stopping_rule_and_best_tracking():
    """Alg. 2's loop: an item stopped by a fall of rho gives the same result
    under any larger iteration limit; the best rho never falls as the limit
    grows; every bandwidth stays within [1, 32^2] on the diagonal."""
    bins = _blob_volume(5)
    B = 4
    rng = np.random.default_rng(9)
    seeds = rng.integers(3, 25, size=(30, 3)).astype(np.int32)
    prev = None
    for it in (1, 2, 4, 8, 16):
        res = ko.abmsod(bins, B, 3, 7, seeds, max_iter=it)
        assert np.all(res["iters"] <= it)
        assert np.all((res["stopped"] == 1) | (res["iters"] == it))
        for k in (0, 3, 5):
            assert np.all(res["H"][:, k] >= 1.0) and np.all(res["H"][:, k] <= 1024.0)
        if prev is not None:
            assert np.all(res["rho"] >= prev["rho"])
            done = prev["stopped"] == 1
            for key in ("x", "H", "rho", "iters"):
                assert np.array_equal(res[key][done], prev[key][done])
        prev = res
    assert prev["stopped"].sum() > 0


def test_uncounted_region_is_empty_window():
    """No counted voxel in the window: the item stops before its first
    iteration at its seed with H = r^2 I and rho = 0."""
    bins = np.zeros((20, 20, 20), np.uint8)
    bins[:2] = 1
    res = ko.abmsod(bins, 3, 2, 4, np.array([[10, 10, 12]], np.int32), max_iter=5)
    for i, r in enumerate((2, 3, 4)):
        assert res["iters"][i] == 0 and res["rho"][i] == 0.0
        assert np.array_equal(res["x"][i], [10.0, 10.0, 12.0])
        assert np.array_equal(res["H"][i], [r * r, 0, 0, r * r, 0, r * r])


def test_thin_structures_keep_the_search_well_defined():
    """Counted voxels only on an oblique plane or along a line: the voxel
    second moments are (nearly) singular, and the unit-voxel term I/12
    keeps every bandwidth positive definite (smallest eigenvalue >= 5/12
    up to the scaling to 32^2); rho stays in [0, 1] (Cauchy-Schwarz), H
    finite with diagonal in [1, 32^2]."""
    n = 40
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    plane = np.abs(3 * xx - 2 * yy + zz - 40) <= 1
    rng = np.random.default_rng(2)
    bins = np.where(plane, rng.integers(1, 5, size=plane.shape), 0).astype(np.uint8)
    pts = np.argwhere(plane)[::97][:, ::-1].astype(np.int32)
    line = np.zeros_like(bins)
    for t in range(-12, 13):
        line[20 + t // 2, 20 - t, 20 + t] = 1 + (t & 3)
    lpts = np.array([[20 + t, 20 - t, 20 + t // 2] for t in range(-9, 10, 3)], np.int32)
    for vol, sd in ((bins, pts), (line, lpts)):
        res = ko.abmsod(vol, 4, 6, 14, sd, max_iter=12)
        assert np.all(np.isfinite(res["rho"]))
        assert np.all(res["rho"] >= 0) and np.all(res["rho"] <= 1)
        assert np.all(np.isfinite(res["H"])) and np.all(np.isfinite(res["x"]))
        for k in (0, 3, 5):
            assert np.all(res["H"][:, k] >= 1.0) and np.all(res["H"][:, k] <= 1024.0)
        assert np.all(res["iters"] >= 1)
        for H in res["H"]:
            Hm = np.array([[H[0], H[1], H[2]], [H[1], H[3], H[4]], [H[2], H[4], H[5]]])
            scale = min(1.0, 1024.0 / max(H[0], H[3], H[5]))
            assert np.linalg.eigvalsh(Hm).min() >= 5.0 / 12.0 * scale * (1 - 1e-9) - 1e-9


def test_row_spans_hold_every_window_voxel():
    """The row span (the root interval of d <= 1 + 1/16 along x) contains
    every voxel of the bounding box with 0 <= d <= 1, for round, flat,
    elongated and oblique bandwidths (condition numbers up to ~2500)."""
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(300):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.exp(rng.uniform(np.log(5.0 / 12.0), np.log(1024.0), 3))
        Hm = Q @ np.diag(lam) @ Q.T
        scale = min(1.0, 1024.0 / Hm.diagonal().max())
        Hm = Hm * scale
        H = np.array([Hm[0, 0], Hm[0, 1], Hm[0, 2], Hm[1, 1], Hm[1, 2], Hm[2, 2]])
        x = rng.uniform(40.0, 60.0, 3)
        box, span = ko.ab_window_check(x, H)
        assert box == span and box > 0, (x, H, box, span)
        checked += 1
    assert checked == 300
