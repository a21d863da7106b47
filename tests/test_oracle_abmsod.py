"""Pins of the oracle's adaptive-bandwidth mean shift (ABMSOD; Sec. 2.3,
Alg. 2, Eq. 6 and 7), the plain binary64 statement `oracle.abmsod`, against
closed forms, an independent numpy evaluation of whole searches, and
symmetries of the definition; and bounds between it and the kernel's stated
arithmetic (`oracle.abmsod_fixed`, binary32 terms on fixed-point grids),
which the CUDA kernel reproduces bit for bit."""
import math

import numpy as np
import pytest

import abmsod_chain
import oracle as ko


def _lattice_ball(r):
    """Integer offsets with |o|^2 <= r^2: the first window of an item with
    H = r^2 I at an integer centre (boundary voxels included)."""
    g = np.arange(-r, r + 1)
    o = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return o[(o ** 2).sum(1) <= r * r][:, ::-1].astype(np.int64)


def test_fixed_model_kernel_is_exp_of_minus_half_d():
    """The kernel's k(d): a binary32 polynomial for exp(-d/2) (Alg. 2),
    within two binary32 ulps of exp on [0, 1]."""
    assert ko.ab_kernel(0.0) == 1.0
    for d in np.linspace(0.0, 1.0, 4001, dtype=np.float32):
        want = math.exp(-0.5 * float(d))
        got = ko.ab_kernel(float(d))
        assert abs(got - want) <= 2 * np.spacing(np.float32(want)), (d, got, want)


@pytest.mark.parametrize("r", [2, 3, 5, 8])
def test_homogeneous_region_closed_form(r):
    """One bin everywhere: HP = e_b, so rho = sqrt(1/B) every iteration; the
    window is symmetric about an integer centre, so the centre never moves;
    rho never rises after the first iteration, so the best bandwidth is the
    first update, 5 (E[o o^T] + I/12) over the lattice ball
    = diag(5 S2 / N + 5/12); every window is the whole lattice ball."""
    B = 4
    n = 2 * r + 24
    bins = np.full((n, n, n), 2, np.uint8)
    seed = np.array([[n // 2, n // 2 + 1, n // 2 - 1]], np.int32)
    res = ko.abmsod(bins, B, r, r + 1, seed, max_iter=6)
    pts = _lattice_ball(r)
    S2 = float((pts[:, 0] ** 2).sum())
    N = len(pts)
    assert res["rho"][0] == 0.5
    assert res["iters"][0] == 6 and res["stopped"][0] == 0
    assert np.array_equal(res["x"][0], seed[0].astype(float))
    H = res["H"][0]
    assert H[1] == H[2] == H[4] == 0.0
    for k in (0, 3, 5):
        assert H[k] == pytest.approx(5.0 * S2 / N + 5.0 / 12.0, rel=1e-14)
    assert res["rho"][1] == 0.5
    assert np.array_equal(res["x"][1], seed[0].astype(float))
    one = ko.abmsod(bins, B, r, r + 1, seed, max_iter=1)
    assert one["voxels"][0] == 2 * N


@pytest.mark.parametrize("e", [(2, 1, 0), (-1, 0, 3), (0, -2, -2), (4, 0, 0)])
def test_single_odd_voxel_shift(e):
    """A homogeneous window with one voxel of the other bin at offset e:
    with w_b = sqrt(HQ_b / HP_b) the odd voxel weighs more, and the Eq. 6
    step is (w_o - w_m) k_e e / (w_m (K - k_e) + w_o k_e), K the kernel sum
    of the ball, k_e = exp(-|e|^2 / (2 r^2)); e = (4, 0, 0) lies on the
    boundary of the r = 4 window and is counted."""
    r, B, n = 4, 2, 24
    bins = np.full((n, n, n), 1, np.uint8)
    c = np.array([12, 11, 13])
    bins[c[2] + e[2], c[1] + e[1], c[0] + e[0]] = 2
    res = ko.abmsod(bins, B, r, r + 1, c[None, :].astype(np.int32), max_iter=1)
    pts = _lattice_ball(r)
    K = np.exp(-(pts ** 2).sum(1) / (2.0 * r * r)).sum()
    ke = math.exp(-sum(v * v for v in e) / (2.0 * r * r))
    wo = math.sqrt((1.0 / B) / (ke / K))
    wm = math.sqrt((1.0 / B) / ((K - ke) / K))
    step = (wo - wm) * ke * np.array(e, float) / (wm * (K - ke) + wo * ke)
    assert np.allclose(res["x"][0] - c, step, rtol=1e-12, atol=1e-13), (res["x"][0] - c, step)
    assert res["iters"][0] == 1


# ---------------------------------------------------------------- numpy Alg. 2
def _np_search(bins, B, x, H, max_iter):
    """Alg. 2 with Eq. 6 and 7 as read (factor 5, I/12, diagonal in
    [1, 32^2]) in numpy: whole-volume masks, np.linalg.solve for d, np.exp,
    numpy's own summation order.  A voxel counts when d <= 1 + 1e-12 (the
    closed ellipsoid; ties of the integer first window are inside).
    Returns (x_opt, H_opt, best, iters, stopped)."""
    nz, ny, nx = bins.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(float)
    v = bins.ravel().astype(int)
    dim = np.array([nx, ny, nz], float)

    def mat(h):
        return np.array([[h[0], h[1], h[2]], [h[1], h[3], h[4]], [h[2], h[4], h[5]]])

    def window(c, h):
        o = s - c
        d = np.einsum("ia,ia->i", o, np.linalg.solve(mat(h), o.T).T)
        m = (d <= 1.0 + 1e-12) & (v > 0)
        return o[m], d[m], v[m] - 1

    def hist(d, b):
        k = np.exp(-0.5 * d)
        P = np.bincount(b, weights=k, minlength=B)
        p = P / k.sum()
        w = np.zeros(B)
        w[p > 0] = np.sqrt((1.0 / B) / p[p > 0])
        return k, p, w

    x = np.array(x, float)
    H = np.array(H, float)
    xo, Ho, best = x.copy(), H.copy(), 0.0
    it, stopped = 0, 0
    while it < max_iter:
        o, d, b = window(x, H)
        if len(o) == 0:
            break
        k, _, w = hist(d, b)
        t = k * w[b]
        xn = np.clip(x + (t[:, None] * o).sum(0) / t.sum(), 0.0, dim - 1)
        o2, d2, b2 = window(xn, H)
        it += 1
        if len(o2) == 0:
            break
        _, p2, w2 = hist(d2, b2)
        ww = w2[b2]
        M = 5.0 * (np.einsum("i,ia,ib->ab", ww, o2, o2) / ww.sum() + np.eye(3) / 12.0)
        for a in range(3):
            M[a, a] = max(M[a, a], 1.0)
        M *= min(1.0, 1024.0 / M.diagonal().max())
        Hn = np.array([M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]])
        rho = np.sqrt(p2 / B).sum()
        fell = rho < best
        if rho > best:
            best, xo, Ho = rho, xn, Hn
        if fell:
            stopped = 1
            break
        x, H = xn, Hn
    return xo, Ho, best, it, stopped


def _blob_volume(seed=7, n=28):
    """Background bin 1, an oblique ellipsoid of bin 3, 10% of voxels set
    to bins 2 / 4 at random."""
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.stack([xx - 13.3, yy - 14.1, zz - 12.7], -1).astype(float)
    R = np.array([[0.8, 0.6, 0.0], [-0.6, 0.8, 0.0], [0.0, 0.0, 1.0]])
    q = u @ R.T
    inside = (q[..., 0] / 6.0) ** 2 + (q[..., 1] / 3.0) ** 2 + (q[..., 2] / 4.0) ** 2 <= 1.0
    bins = np.where(inside, 3, 1).astype(np.uint8)
    noise = rng.random(bins.shape) < 0.1
    bins[noise] = rng.choice([2, 4], size=int(noise.sum())).astype(np.uint8)
    return bins


def test_whole_searches_match_numpy_evaluation():
    """Whole searches (up to 8 iterations: position steps, bandwidth updates,
    best-rho tracking, the stop at the first fall of rho, the diagonal
    bounds) against the numpy statement, items seeded around an oblique
    blob.  Items whose decisions the oracle itself reports within 1e-9 of a
    tie (a voxel on the window's boundary, or rho equal to the best) are
    left out; they must be rare."""
    bins = _blob_volume()
    B = 4
    rng = np.random.default_rng(5)
    seeds = rng.integers(5, 23, size=(10, 3)).astype(np.int32)
    res = ko.abmsod(bins, B, 2, 5, seeds, max_iter=8)
    x0, H0 = abmsod_chain.seed_items(seeds, 2, 5)
    checked = 0
    for i in range(len(x0)):
        if res["edge"][i] < 1e-9 or res["rho_gap"][i] < 1e-9:
            continue
        xo, Ho, best, it, stopped = _np_search(bins, B, x0[i], H0[i], 8)
        assert res["iters"][i] == it and res["stopped"][i] == stopped, i
        assert np.allclose(res["x"][i], xo, rtol=0, atol=1e-9), (i, res["x"][i], xo)
        assert np.allclose(res["H"][i], Ho, rtol=1e-9, atol=1e-9), (i, res["H"][i], Ho)
        assert abs(res["rho"][i] - best) <= 1e-12, (i, res["rho"][i], best)
        checked += 1
    assert checked >= 0.9 * len(x0)
    assert (res["stopped"] == 1).sum() >= 5 and (res["iters"] > 1).sum() >= 20


def test_axis_swap_symmetry():
    """Swapping x and y in the volume and the seeds swaps the centre and the
    H entries (00 <-> 11, 02 <-> 12); rho and the iteration count agree.
    Only the order of the binary64 sums changes, so every item agrees to
    rounding level, except where the oracle reports a tie in the stopping
    test (|rho' - best| < 1e-12), whose outcome rounding decides."""
    bins = _blob_volume(11)
    B = 4
    rng = np.random.default_rng(3)
    seeds = rng.integers(4, 24, size=(40, 3)).astype(np.int32)
    a = ko.abmsod(bins, B, 3, 6, seeds, max_iter=8)
    bt = np.ascontiguousarray(bins.transpose(0, 2, 1))
    b = ko.abmsod(bt, B, 3, 6, seeds[:, [1, 0, 2]].copy(), max_iter=8)
    tie = (a["rho_gap"] < 1e-12) | (b["rho_gap"] < 1e-12)
    assert tie.sum() <= 2
    ok = ~tie
    assert np.array_equal(a["iters"][ok], b["iters"][ok])
    assert np.array_equal(a["stopped"][ok], b["stopped"][ok])
    assert np.allclose(a["x"][ok], b["x"][ok][:, [1, 0, 2]], rtol=0, atol=1e-9)
    assert np.allclose(a["H"][ok], b["H"][ok][:, [3, 1, 4, 0, 2, 5]], rtol=1e-9, atol=1e-9)
    assert np.allclose(a["rho"][ok], b["rho"][ok], rtol=0, atol=1e-12)


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


def _thin_volumes():
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
    return ((bins, pts), (line, lpts))


@pytest.mark.parametrize("search,slack", [(ko.abmsod, 1e-9), (ko.abmsod_fixed, 1e-3)])
def test_thin_structures_keep_the_search_well_defined(search, slack):
    """Counted voxels only on an oblique plane or along a line: the voxel
    second moments are (nearly) singular, and the unit-voxel term I/12
    keeps every bandwidth positive definite (smallest eigenvalue >= 5/12
    up to the scaling to 32^2, less the rounding of the moment sums: 1e-9
    in binary64, 1e-3 on the kernel's fixed-point grids); rho stays in
    [0, 1] (Cauchy-Schwarz), H finite with diagonal in [1, 32^2]."""
    for vol, sd in _thin_volumes():
        res = search(vol, 4, 6, 14, sd, max_iter=12)
        assert np.all(np.isfinite(res["rho"]))
        assert np.all(res["rho"] >= 0) and np.all(res["rho"] <= 1)
        assert np.all(np.isfinite(res["H"])) and np.all(np.isfinite(res["x"]))
        for k in (0, 3, 5):
            assert np.all(res["H"][:, k] >= 1.0) and np.all(res["H"][:, k] <= 1024.0)
        assert np.all(res["iters"] >= 1)
        for H in res["H"]:
            Hm = np.array([[H[0], H[1], H[2]], [H[1], H[3], H[4]], [H[2], H[4], H[5]]])
            scale = min(1.0, 1024.0 / max(H[0], H[3], H[5]))
            assert np.linalg.eigvalsh(Hm).min() >= 5.0 / 12.0 * scale - slack


def test_fixed_model_row_spans_hold_every_window_voxel():
    """The kernel's row span (the root interval of d <= 1 + 1/16 along x)
    contains every voxel of the bounding box with 0 <= d <= 1, for round,
    flat, elongated and oblique bandwidths (condition numbers to ~2500)."""
    rng = np.random.default_rng(4)
    for _ in range(300):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        lam = np.exp(rng.uniform(np.log(5.0 / 12.0), np.log(1024.0), 3))
        Hm = Q @ np.diag(lam) @ Q.T
        Hm = Hm * min(1.0, 1024.0 / Hm.diagonal().max())
        H = np.array([Hm[0, 0], Hm[0, 1], Hm[0, 2], Hm[1, 1], Hm[1, 2], Hm[2, 2]])
        x = rng.uniform(40.0, 60.0, 3)
        box, span = ko.ab_window_check(x, H)
        assert box == span and box > 0, (x, H, box, span)


# ----------------------------------------- kernel arithmetic against the oracle
def test_fixed_model_per_iteration_bounds_spheres48():
    """Every iteration of every item of the spheres workload (48^3, 16 bins,
    r = 2..10, stride 6, 4608 items): one iteration of the kernel's
    arithmetic from each state the oracle visits agrees with the oracle's
    iteration within the bounds of tests/abmsod_chain.py."""
    from paper_1310_6736_b300 import synth
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    B = w.binning["bins"]
    x0, H0 = abmsod_chain.seed_items(ko.seed_grid(w.dims, w.stride), w.r_min, w.r_max)
    st = abmsod_chain.oracle_states(ko, bins, B, x0, H0, w.max_iter)
    got = ko.abmsod_fixed(bins, B, 0, 0, None, 1, cand=(st["x"], st["H"]))
    far, near = abmsod_chain.compare(st, got)
    assert far >= 0.8 * (far + near)


def test_fixed_model_whole_searches_agree_statistically():
    """Whole searches in the kernel's arithmetic and in the oracle's take the
    same path for most items; where a tie in the stopping test (rho flat to
    1e-7 near convergence) or a boundary voxel sends them apart, both still
    end at nearby optima.  Sanity bounds over the 4608 spheres items."""
    from paper_1310_6736_b300 import synth
    w = synth.workload("spheres48")
    bins = ko.bin_volume(w.volume, w.binning)
    B = w.binning["bins"]
    sd = ko.seed_grid(w.dims, w.stride)
    a = ko.abmsod(bins, B, w.r_min, w.r_max, sd, w.max_iter)
    f = ko.abmsod_fixed(bins, B, w.r_min, w.r_max, sd, w.max_iter)
    same = (a["iters"] == f["iters"]) & (a["stopped"] == f["stopped"])
    assert same.mean() >= 0.9
    dr = np.abs(a["rho"] - f["rho"])
    assert np.median(dr) <= 1e-7 and np.mean(dr <= 1e-4) >= 0.95
    assert np.median(np.abs(a["x"] - f["x"]).max(1)) <= 1e-4
    assert abs(a["rho"].mean() - f["rho"].mean()) <= 1e-3
