"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bar: integer results bit-exact (bins, scale indices, seed positions,
iteration counts, trajectories); FP64 results (H, W, Y, rho) within
|gpu - oracle| <= 1e-12 * max(1, |oracle|), the entropy tolerance of the
method's statement.  Both sides evaluate one fixed operation order on
correctly rounded tables, so the observed difference is expected to be 0;
the tests also report how many values are bit-identical.
"""
import numpy as np
import pytest

import abmsod_chain
import oracle_checks
from paper_1310_6736_b300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    bad = np.abs(a - b) > RTOL * np.maximum(1.0, np.abs(b))
    assert not bad.any(), f"{bad.sum()} of {bad.size} differ; first at {np.argwhere(bad)[:3]}"
    return int((a == b).sum())


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1310_6736_b300 import build, ks
    build.build()
    c = ks.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def ks_mod():
    from paper_1310_6736_b300 import ks
    return ks


def _params(ks, w):
    return ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)


# ------------------------------------------------------------------ tables
def test_tables_bit_exact(ctx, ko):
    T, L = ctx.tables(137065)
    To, Lo = ko.tables(137065)
    assert np.array_equal(T.view(np.uint64), To[:137066].view(np.uint64))
    assert np.array_equal(L.view(np.uint64), Lo[:137066].view(np.uint64))


# ----------------------------------------------------------------- binning
@pytest.mark.parametrize("name", ["spheres48", "pet128", "mr256"])
def test_binning_bit_exact(ctx, ko, name):
    w = synth.workload(name)
    v = ctx.create_volume(w.volume, w.binning)
    got = ctx.volume_bins(v, w.volume.shape)
    ctx.release_volume(v)
    assert np.array_equal(got, ko.bin_volume(w.volume, w.binning))


@pytest.mark.parametrize("dims,dtype", [((37, 23, 19), np.uint8), ((33, 5, 7), np.int16),
                                        ((17, 16, 3), np.float32), ((1, 1, 1), np.uint8),
                                        ((64, 2, 2), np.int16), ((128, 3, 2), np.uint8),
                                        ((192, 2, 3), np.int16)])
def test_binning_ragged_and_kinds(ctx, ko, dims, dtype):
    rng = np.random.default_rng(sum(dims))
    nx, ny, nz = dims
    if dtype == np.float32:
        vol = rng.normal(3.0, 2.0, size=(nz, ny, nx)).astype(np.float32)
        bins = [{"kind": 1, "bins": 32}]
    elif dtype == np.int16:
        vol = rng.integers(-200, 2300, size=(nz, ny, nx)).astype(np.int16)
        bins = [{"kind": 0, "bins": 64, "shift": 5, "lo": 0, "hi": 2047},
                {"kind": 2, "bins": 40, "shift": 5, "lo": 100, "hi": 1300}]
    else:
        vol = rng.integers(0, 256, size=(nz, ny, nx)).astype(np.uint8)
        # rows of 64-voxel multiples take the four-run path; the first three
        # there take the bytewise form (lo = 0, hi >= 255: the clamp never
        # applies), the next two the general one (hi < 255; lo > 0)
        bins = [{"kind": 0, "bins": 16, "shift": 4, "lo": 0, "hi": 255},
                {"kind": 0, "bins": 32, "shift": 3, "lo": 0, "hi": 255},
                {"kind": 0, "bins": 64, "shift": 2, "lo": 0, "hi": 255},
                {"kind": 0, "bins": 32, "shift": 3, "lo": 0, "hi": 200},
                {"kind": 0, "bins": 16, "shift": 4, "lo": 10, "hi": 255},
                {"kind": 2, "bins": 7, "shift": 4, "lo": 30, "hi": 140}]
    for b in bins:
        v = ctx.create_volume(vol, b)
        got = ctx.volume_bins(v, vol.shape)
        ctx.release_volume(v)
        assert np.array_equal(got, ko.bin_volume(vol, b)), b


# ------------------------------------------------------------------- dense
def _dense_vs_oracle(ctx, ko, ks, bins_vol_raw, binning, r_min, r_max, w_norm=0, hw=True):
    v = ctx.create_volume(bins_vol_raw, binning)
    p = ks.make_params(r_min, r_max, 8, 20, w_norm)
    if hw:
        Y, s, H, W = ctx.dense_saliency(v, p, bins_vol_raw.shape, want_hw=True)
    else:
        Y, s = ctx.dense_saliency(v, p, bins_vol_raw.shape)
    ctx.release_volume(v)
    b = ko.bin_volume(bins_vol_raw, binning)
    B = binning["bins"]
    if hw:
        Yo, so, Ho, Wo = ko.dense(b, B, r_min, r_max, w_norm=w_norm, want_hw=True)
        close(H, Ho)
        close(W, Wo)
    else:
        Yo, so = ko.dense(b, B, r_min, r_max, w_norm=w_norm)
    assert np.array_equal(s, so)
    return close(Y, Yo)


@pytest.mark.parametrize("cfg", [None, (0, 16, 4, 4), (0, 8, 2, 4), (0, 4, 4, 1), (1, 16, 4, 4),
                                 (1, 8, 8, 1), (2, 8, 4, 2), (2, 4, 1, 4), (3, 4, 2, 2),
                                 (3, 1, 1, 1), (3, 8, 2, 4), (4, 4, 2, 2), (4, 1, 1, 1),
                                 (4, 8, 2, 4), (4, 2, 1, 2), (5, 1, 1, 16), (5, 1, 1, 48),
                                 (5, 1, 1, 7)])
def test_dense_spheres48_full_volume(ctx, ko, ks_mod, cfg):
    ks = ks_mod
    try:
        if cfg is not None:
            ks.force_dense_config(*cfg)
        w = synth.workload("spheres48")
        _dense_vs_oracle(ctx, ko, ks, w.volume, w.binning, w.r_min, w.r_max)
    finally:
        ks.force_dense_config(-1)


@pytest.mark.parametrize("case", [
    ((37, 23, 19), 5, 1, 6, 0),      # ragged tiles, odd bin count, r_min = 1
    ((45, 9, 30), 33, 3, 9, 1),      # bins between template sizes, w_norm ONE
    ((20, 20, 20), 64, 2, 7, 0),
    ((1, 1, 1), 16, 1, 3, 0),        # one voxel
    ((70, 3, 2), 16, 2, 12, 0),      # thin slab, radius larger than the volume
    ((75, 6, 4), 8, 24, 28, 0),      # r_max > 25: global offset table, 32-bit previous counts
])
@pytest.mark.parametrize("path", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_dense_random_volumes(ctx, ko, ks_mod, case, path):
    """Every launch path forced on random volumes (a shape that does not fit
    the path, e.g. paths 6 to 8 below r_max = 26, falls back to the
    autotuner)."""
    ks = ks_mod
    dims, B, r_min, r_max, wn = case
    nx, ny, nz = dims
    rng = np.random.default_rng(nx * 7 + B)
    # blobs of high entropy over a two-level background, plus excluded voxels
    vol = rng.choice([40, 41, 90], size=(nz, ny, nx), p=[0.6, 0.3, 0.1]).astype(np.int16)
    blob = rng.random((nz, ny, nx)) < 0.25
    vol[blob] = rng.integers(0, 2048, size=int(blob.sum()))
    shift = max(0, int(np.ceil(np.log2(2048 / B))))
    binning = {"kind": 2, "bins": B, "shift": shift, "lo": 30, "hi": min(2047, (B << shift) - 1)}
    try:
        ks.force_dense_config(*((5, 1, 1, 8) if path == 5 else (path, 8, 4, 2)))
        _dense_vs_oracle(ctx, ko, ks, vol, binning, r_min, r_max, wn)
    finally:
        ks.force_dense_config(-1)


@pytest.mark.parametrize("case", [
    ((41, 9, 6), 16, 20, 27, (6, 4, 4, 1)),     # 16 bins, ragged x tile
    ((37, 8, 8), 40, 24, 30, (6, 8, 4, 2)),     # 40 bins (64-bin template), 8 warps
    ((66, 5, 4), 64, 26, 32, (6, 4, 2, 2)),     # 64 bins, r_max = 32, two x tiles
    ((35, 12, 5), 33, 22, 28, (6, 16, 4, 4)),   # 16 warps: 4 TMEM column groups
    ((41, 9, 6), 16, 20, 27, (7, 4, 4, 1)),     # two centres per lane, one ragged x tile
    ((70, 5, 4), 64, 26, 32, (7, 4, 2, 2)),     # 64 bins, r_max = 32, a 6-centre second tile
    ((37, 8, 8), 40, 24, 30, (7, 8, 4, 2)),     # 8 warps: 2 TMEM column groups of 128
    ((130, 3, 3), 32, 25, 26, (7, 8, 2, 4)),    # 32 bins, three x tiles
    ((41, 9, 6), 16, 20, 27, (8, 4, 4, 1)),     # 16-bit wrapping counters, one ragged x tile
    ((70, 5, 4), 64, 26, 32, (8, 4, 2, 2)),     # r_min > 25: the first scale recovered at 25
    ((37, 8, 8), 40, 31, 32, (8, 8, 4, 2)),     # r_min = 31: 59 220 voxels after the recovery
    ((130, 3, 3), 32, 4, 32, (8, 4, 4, 1)),     # every scale from 4 to 32
    ((41, 9, 6), 16, 20, 27, (9, 4, 4, 1)),     # four centres per lane, one ragged x tile
    ((140, 5, 4), 64, 26, 32, (9, 4, 2, 2)),    # r_min > 25, a 12-centre second tile
    ((37, 8, 8), 40, 31, 32, (9, 8, 4, 2)),     # r_min = 31, 8 warps
    ((130, 3, 3), 32, 4, 32, (9, 4, 4, 1)),     # every scale from 4 to 32
])
def test_dense_wide_tmem_path(ctx, ko, ks_mod, case):
    """Launch paths 6 to 9 (r_max > 25): the 32-bit previous-scale counts
    in TMEM, one, two or four centres per lane (paths 8 and 9: 16-bit
    counters modulo 2^16, recovered from the previous counts).  Every H, W, Y and s_best of
    random volumes equals the oracle's.  Each forced shape fits its path
    (r_max > 25, a 16-, 32- or 64-bin template, 4, 8 or 16 warps, at most 8
    for paths 7 to 9), so it is the one that runs."""
    ks = ks_mod
    dims, B, r_min, r_max, cfg = case
    nx, ny, nz = dims
    rng = np.random.default_rng(B * 5 + r_max)
    vol = rng.choice([40, 41, 90], size=(nz, ny, nx), p=[0.6, 0.3, 0.1]).astype(np.int16)
    blob = rng.random((nz, ny, nx)) < 0.3
    vol[blob] = rng.integers(0, 2048, size=int(blob.sum()))
    shift = max(0, int(np.ceil(np.log2(2048 / B))))
    binning = {"kind": 2, "bins": B, "shift": shift, "lo": 30, "hi": min(2047, (B << shift) - 1)}
    try:
        ks.force_dense_config(*cfg)
        _dense_vs_oracle(ctx, ko, ks, vol, binning, r_min, r_max)
    finally:
        ks.force_dense_config(-1)


def test_dense_mr256_full_volume_sampled(ctx, ko, ks_mod):
    """The MR-shaped volume at full size (256x256x160 int16, 64 bins, r =
    4..32), as the serving loop sweeps it: the autotuned wide launch gives
    the same Y and s_best as launch path 6 everywhere, and the oracle's at
    sampled centres (corners, x-tile edges and random ones)."""
    ks = ks_mod
    w = synth.workload("mr256")
    p = _params(ks, w)
    nz, ny, nx = w.volume.shape
    v = ctx.create_volume(w.volume, w.binning)
    Y, s = ctx.dense_saliency(v, p, (nz, ny, nx))
    try:
        ks.force_dense_config(6, 4, 2, 2)
        Y6, s6 = ctx.dense_saliency(v, p, (nz, ny, nx))
    finally:
        ks.force_dense_config(-1)
    ctx.release_volume(v)
    assert np.array_equal(s, s6) and np.array_equal(Y.view(np.uint64), Y6.view(np.uint64))
    rng = np.random.default_rng(256)
    n = 240
    cen = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)],
                   1).astype(np.int32)
    edges = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [31, 7, 80], [32, 7, 80], [63, 100, 3],
             [64, 100, 3], [95, 128, 159], [96, 128, 159], [127, 255, 0], [128, 0, 77],
             [200, 130, 79], [255, 131, 80]]
    cen = np.concatenate([np.array(edges, np.int32), cen])
    Yo, so = ko.dense(ko.bin_volume(w.volume, w.binning), w.binning["bins"], w.r_min, w.r_max,
                      centres=cen)
    x, y, z = cen[:, 0], cen[:, 1], cen[:, 2]
    assert np.array_equal(s[z, y, x], so)
    close(Y[z, y, x], Yo)
    assert int((so > 0).sum()) > n // 4       # peaks in scale were found


def test_dense_wrap_counts_past_16_bits(ctx, ko, ks_mod):
    """Launch paths 8 and 9 count modulo 2^16: on a 72^3 volume that is 95% one
    value, a centre's Ball(32) holds about 130 000 voxels of one bin, so the
    counts wrap twice.  H, W, Y and s_best equal path 7's (32-bit counters)
    everywhere and the oracle's at sampled centres, the middle ones (whole
    balls inside the volume) included."""
    ks = ks_mod
    rng = np.random.default_rng(72)
    n = 72
    vol = np.full((n, n, n), 700, np.int16)
    noise = rng.random((n, n, n)) < 0.05
    vol[noise] = rng.integers(0, 2048, size=int(noise.sum()))
    binning = {"kind": 2, "bins": 64, "shift": 5, "lo": 0, "hi": 2047}
    p = ks.make_params(4, 32, 8, 20)
    out = {}
    for path in (7, 8, 9):
        try:
            ks.force_dense_config(path, 4, 4, 1)
            v = ctx.create_volume(vol, binning)
            out[path] = ctx.dense_saliency(v, p, vol.shape, want_hw=True)
            ctx.release_volume(v)
        finally:
            ks.force_dense_config(-1)
    for path in (8, 9):
        for a7, ap in zip(out[7], out[path]):
            assert np.array_equal(a7, ap)
    Y, s, H, W = out[8]
    cen = np.concatenate([np.array([[36, 36, 36], [35, 37, 36], [32, 32, 39], [39, 39, 32]]),
                          rng.integers(0, n, size=(60, 3))]).astype(np.int32)
    b = ko.bin_volume(vol, binning)
    Yo, so, Ho, Wo = ko.dense(b, 64, 4, 32, centres=cen, want_hw=True)
    x, y, z = cen[:, 0], cen[:, 1], cen[:, 2]
    flat = (z * n + y) * n + x
    assert np.array_equal(s[z, y, x], so)
    close(Y[z, y, x], Yo)
    close(H[flat], Ho)
    close(W[flat], Wo)
    # the middle centres' dominant bin passed 2^17 at r = 32
    assert int((b[4:69, 4:69, 4:69] == b[36, 36, 36]).sum()) > 2 * 65536


def test_host_out_into_pinned_arrays_equals_default_outputs(ctx, ks_mod):
    """The end-to-end path: the raw volume in pinned host memory and every
    result written into caller-owned pinned arrays gives the same records and
    maps as the binding's own host outputs."""
    import torch
    ks = ks_mod
    w = synth.workload("spheres48")
    p = _params(ks, w)
    nz, ny, nx = w.volume.shape

    def pinned(nbytes):
        return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()

    vol = pinned(w.volume.nbytes).view(w.volume.dtype).reshape(w.volume.shape)
    vol[...] = w.volume
    v = ctx.create_volume(w.volume, w.binning)
    Y0, s0 = ctx.dense_saliency(v, p, (nz, ny, nx))
    o0, m0 = ctx.seed_climb(v, p), ctx.meanshift(v, p)
    ctx.release_volume(v)
    Y = pinned(nx * ny * nz * 8).view(np.float64).reshape(nz, ny, nx)
    s = pinned(nx * ny * nz).reshape(nz, ny, nx)
    o = pinned(len(o0) * ks.SEED_RESULT.itemsize).view(ks.SEED_RESULT)
    m = pinned(len(m0) * ks.MS_RESULT.itemsize).view(ks.MS_RESULT)
    v = ctx.create_volume(vol, w.binning)
    ctx.dense_saliency(v, p, (nz, ny, nx), host_out=(Y, s))
    got_o = ctx.seed_climb(v, p, host_out=o)
    got_m = ctx.meanshift(v, p, host_out=m)
    ctx.release_volume(v)
    assert np.array_equal(Y, Y0) and np.array_equal(s, s0)
    assert np.array_equal(got_o, o0) and np.array_equal(got_m, m0)
    with pytest.raises(ValueError):
        ctx.dense_saliency(v, p, (nz, ny, nx), host_out=(Y[:, :, :-1], s))


@pytest.mark.parametrize("name", ["spheres48", "pet128"])
def test_saliency_call_equals_the_three_calls(ctx, ks_mod, name):
    """ks_saliency (dense sweep on a high-priority stream, seed searches
    beside it on a low-priority one) gives the three separate calls' results
    bit for bit, with host and with device outputs."""
    import torch
    ks = ks_mod
    w = synth.workload(name)
    p = _params(ks, w)
    shape = w.volume.shape
    v = ctx.create_volume(w.volume, w.binning)
    try:
        Y0, s0 = ctx.dense_saliency(v, p, shape)
        o0, m0 = ctx.seed_climb(v, p), ctx.meanshift(v, p)
        Y1, s1, o1, m1 = ctx.saliency(v, p, shape)
        assert np.array_equal(Y1, Y0) and np.array_equal(s1, s0)
        assert np.array_equal(o1, o0) and np.array_equal(m1, m0)
        Yd = torch.empty(shape, dtype=torch.float64, device="cuda")
        sd = torch.empty(shape, dtype=torch.uint8, device="cuda")
        od = torch.empty(len(o0) * ks.SEED_RESULT.itemsize, dtype=torch.uint8, device="cuda")
        md = torch.empty(len(m0) * ks.MS_RESULT.itemsize, dtype=torch.uint8, device="cuda")
        assert ctx.saliency(v, p, shape, out=(Yd, sd, od, md)) == (len(o0), len(m0))
        torch.cuda.synchronize()
        assert np.array_equal(Yd.cpu().numpy(), Y0) and np.array_equal(sd.cpu().numpy(), s0)
        assert np.array_equal(od.cpu().numpy().view(ks.SEED_RESULT), o0)
        assert np.array_equal(md.cpu().numpy().view(ks.MS_RESULT), m0)
        with pytest.raises(ValueError):
            ctx.saliency(v, p, shape, out=(Yd, sd, od[:64], md))
    finally:
        ctx.release_volume(v)


def test_saliency_reports_a_small_capacity(ctx, ks_mod):
    """Through the C ABI: a record buffer that is too small gives KS_EINVAL
    with the needed counts written, and the context stays usable."""
    import ctypes as C
    ks = ks_mod
    w = synth.workload("spheres48")
    p = _params(ks, w)
    nz, ny, nx = w.volume.shape
    v = ctx.create_volume(w.volume, w.binning)
    try:
        n = ctx.seed_count(v, p)
        S = p.r_max - p.r_min + 1
        Y = np.empty((nz, ny, nx), np.float64)
        s = np.empty((nz, ny, nx), np.uint8)
        o = np.zeros(n, ks.SEED_RESULT)
        m = np.zeros(n * S - 1, ks.MS_RESULT)          # one record short
        n_oct, n_ms = C.c_int64(-1), C.c_int64(-1)
        st = ks.lib().ks_saliency(ctx.h, int(v), C.byref(p), C.c_void_p(Y.ctypes.data),
                                  C.c_void_p(s.ctypes.data), C.c_void_p(o.ctypes.data), n,
                                  C.byref(n_oct), C.c_void_p(m.ctypes.data), len(m),
                                  C.byref(n_ms), 0)
        assert st == ks.KS_EINVAL
        assert n_oct.value == n and n_ms.value == n * S
        _, _, o2, m2 = ctx.saliency(v, p, (nz, ny, nx))      # still usable
        assert len(o2) == n and len(m2) == n * S
    finally:
        ctx.release_volume(v)


@pytest.mark.parametrize("cfg", [None, (5, 1, 1, 64), (1, 8, 8, 1), (3, 4, 2, 2)])
def test_dense_pet128_full_size_sampled(ctx, ko, ks_mod, cfg):
    """The bench workload (128x128x64 float32, 32 bins, r=4..20) at full size,
    in the autotuned launch configuration, the sliding-window path, the
    one-centre-per-lane path and the shared-memory four-centre path;
    checked on three whole z-planes (first, middle, last: 49 152 centres)
    and 3000 random centres."""
    ks = ks_mod
    w = synth.workload("pet128")
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    try:
        if cfg is not None:
            ks.force_dense_config(*cfg)
        Y, s = ctx.dense_saliency(v, p, w.volume.shape)
    finally:
        ks.force_dense_config(-1)
    ctx.release_volume(v)
    b = ko.bin_volume(w.volume, w.binning)
    rng = np.random.default_rng(0)
    nz, ny, nx = w.volume.shape
    cen = np.stack([rng.integers(0, nx, 3000), rng.integers(0, ny, 3000),
                    rng.integers(0, nz, 3000)], axis=1)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    planes = [np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, z)], 1) for z in (0, nz // 2, nz - 1)]
    cen = np.concatenate([cen] + planes).astype(np.int32)
    Yo, so = ko.dense(b, 32, w.r_min, w.r_max, centres=cen)
    got_Y = Y[cen[:, 2], cen[:, 1], cen[:, 0]]
    got_s = s[cen[:, 2], cen[:, 1], cen[:, 0]]
    assert np.array_equal(got_s, so)
    close(got_Y, Yo)
    # properties that hold at every voxel: s in {0} u (r_min, r_max), Y >= 0, Y = 0 iff no peak
    assert set(np.unique(s)) <= {0} | set(range(w.r_min + 1, w.r_max))
    assert (Y >= 0).all() and ((Y > 0) <= (s > 0)).all()


# ------------------------------------------------------------------- seeds
def _oct_vs_oracle(ctx, ko, ks, w, seeds=None, traj=True):
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    if traj:
        got, gtraj = ctx.seed_climb(v, p, seeds=seeds, want_traj=True)
    else:
        got = ctx.seed_climb(v, p, seeds=seeds)
    ctx.release_volume(v)
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride) if seeds is None else np.asarray(seeds, np.int32)
    ref = ko.octant_climb(b, w.binning["bins"], w.r_min, w.r_max, sd, w.max_iter,
                          want_traj=traj)
    assert np.array_equal(np.stack([got["seed_x"], got["seed_y"], got["seed_z"]], 1), sd)
    assert np.array_equal(np.stack([got["x"], got["y"], got["z"]], 1), ref["xyz"])
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])
    assert np.array_equal(got["s_best"], ref["s"])
    if traj:
        assert np.array_equal(gtraj, ref["traj"])
    close(got["Y_best"], ref["Y"])
    close(got["H_best"], ref["H"])
    close(got["W_best"], ref["W"])
    return got


def _ms_vs_oracle(ctx, ko, ks, w, seeds=None):
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    got = ctx.meanshift(v, p, seeds=seeds)
    ctx.release_volume(v)
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride) if seeds is None else np.asarray(seeds, np.int32)
    ref = ko.meanshift(b, w.binning["bins"], w.r_min, w.r_max, sd, w.max_iter)
    S = w.r_max - w.r_min + 1
    assert np.array_equal(got["seed"], np.repeat(np.arange(len(sd)), S))
    assert np.array_equal(got["r"], np.tile(np.arange(w.r_min, w.r_max + 1), len(sd)))
    assert np.array_equal(np.stack([got["x"], got["y"], got["z"]], 1), ref["xyz"])
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])
    close(got["rho"], ref["rho"])
    close(got["H"], ref["H"])
    return got


def test_octant_spheres48_all_seeds(ctx, ko, ks_mod):
    _oct_vs_oracle(ctx, ko, ks_mod, synth.workload("spheres48"))


def test_meanshift_spheres48_all_items(ctx, ko, ks_mod):
    _ms_vs_oracle(ctx, ko, ks_mod, synth.workload("spheres48"))


def test_octant_pet128_all_seeds(ctx, ko, ks_mod):
    _oct_vs_oracle(ctx, ko, ks_mod, synth.workload("pet128"), traj=True)


@pytest.mark.parametrize("max_iter", [5, 9, 14])
def test_octant_cycles_jump_to_max_iter(ctx, ko, ks_mod, max_iter):
    """Searches whose centres repeat with a period of 2..8 are finished by
    a jump to max_iter.  Several max_iter values put the final centre at
    different phases of each cycle, so both the reuse of the last pass and a
    final pass at another centre of the cycle are taken; records and
    trajectories equal the oracle's, which runs every iteration."""
    w = synth.workload("pet128")
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride)
    ref = ko.octant_climb(b, w.binning["bins"], w.r_min, w.r_max, sd, max_iter, want_traj=True)
    # per cycling search: does the final centre equal the last pass's centre?
    reuse = extra = 0
    for i in np.nonzero(ref["converged"] == 0)[0]:
        tr = ref["traj"][i]
        hit = [(t, p) for t in range(2, max_iter + 1) for p in range(2, min(t, 8) + 1)
               if (tr[t] == tr[t - p]).all()]
        if hit:
            t, p = hit[0]
            if (tr[t - p + (max_iter - t) % p] == tr[t - 1]).all():
                reuse += 1
            else:
                extra += 1
    assert reuse >= 10 and extra >= 10
    v = ctx.create_volume(w.volume, w.binning)
    p = ks_mod.make_params(w.r_min, w.r_max, w.stride, max_iter)
    got, traj = ctx.seed_climb(v, p, want_traj=True)
    assert np.array_equal(np.stack([got["x"], got["y"], got["z"]], 1), ref["xyz"])
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])
    assert np.array_equal(traj, ref["traj"])
    assert np.array_equal(got["s_best"], ref["s"])
    close(got["Y_best"], ref["Y"])
    close(got["H_best"], ref["H"])
    close(got["W_best"], ref["W"])
    ctx.release_volume(v)


def test_meanshift_pet128_all_items(ctx, ko, ks_mod):
    _ms_vs_oracle(ctx, ko, ks_mod, synth.workload("pet128"))


def test_seeds_mr256_full_grid_and_edges(ctx, ko, ks_mod):
    """The MR-shaped workload at full size (256x256x160 int16, 64 bins,
    r = 4..32): the octant climb on all 5733 grid seeds (trajectories
    included) plus volume corners and faces; mean shift on 1024 grid seeds
    at all 29 radii (29 696 items, every one of them on the block path:
    more than 32 bins) plus the corners."""
    w = synth.workload("mr256")
    grid = ko.seed_grid(w.dims, w.stride)
    edge = np.array([[0, 0, 0], [255, 255, 159], [128, 0, 80], [255, 130, 0]], np.int32)
    seeds = np.concatenate([grid, edge]).astype(np.int32)
    _oct_vs_oracle(ctx, ko, ks_mod, w, seeds=seeds, traj=True)
    rng = np.random.default_rng(3)
    pick = grid[np.sort(rng.choice(len(grid), 1024, replace=False))]
    _ms_vs_oracle(ctx, ko, ks_mod, w, seeds=np.concatenate([pick, edge]).astype(np.int32))


def test_meanshift_radii_across_warp_and_block_paths(ctx, ko, ks_mod):
    """Radii 17..23: items with r <= 20 run one per warp, the others one per
    block, in one launch; 5 bins (not a multiple of 8), ragged last ticket."""
    rng = np.random.default_rng(11)
    vol = rng.integers(0, 5, size=(30, 36, 40)).astype(np.uint8)
    vol[:, :, :13] = 2                       # a flat slab beside the noise
    w = synth.Workload("mixed", vol, {"kind": 0, "bins": 5, "shift": 0, "lo": 0, "hi": 4},
                       17, 23, 9, 12)
    _ms_vs_oracle(ctx, ko, ks_mod, w)


@pytest.mark.parametrize("B", [33, 47])
def test_meanshift_block_only_bin_counts(ctx, ko, ks_mod, B):
    """More than 32 bins: every mean-shift item runs on the block path, in
    the launch compiled without the warp path (the B words at a fixed
    offset; column sums by groups of 4 threads per bin).  Radii 18..23,
    bins that are neither a power of two nor a multiple of 8."""
    rng = np.random.default_rng(B)
    vol = rng.integers(0, 8 * B, size=(28, 33, 37)).astype(np.int16)
    vol[:, :12, :] = 8 * (B // 2)            # a flat slab beside the noise
    w = synth.Workload("block-only", vol, {"kind": 0, "bins": B, "shift": 3, "lo": 0,
                                           "hi": 8 * B - 1}, 18, 23, 9, 12)
    _ms_vs_oracle(ctx, ko, ks_mod, w)
    _oct_vs_oracle(ctx, ko, ks_mod, w)


def test_seed_edge_cases(ctx, ko, ks_mod):
    ks = ks_mod
    # constant volume: every seed converges at once; excluded voxels only: N = 0
    vol = np.full((20, 21, 22), 77, np.uint8)
    w = synth.Workload("const", vol, {"kind": 0, "bins": 16, "shift": 4, "lo": 0, "hi": 255},
                       2, 6, 5, 20)
    g = _oct_vs_oracle(ctx, ko, ks, w)
    assert (g["iters"] == 1).all() and (g["s_best"] == 0).all()
    _ms_vs_oracle(ctx, ko, ks, w)
    w2 = synth.Workload("empty", vol, {"kind": 2, "bins": 8, "shift": 4, "lo": 200, "hi": 255},
                        1, 4, 7, 3)
    _oct_vs_oracle(ctx, ko, ks, w2)
    _ms_vs_oracle(ctx, ko, ks, w2)
    # max_iter = 0: no move, evaluation at the seed
    w3 = synth.workload("spheres48")
    w3.max_iter = 0
    _oct_vs_oracle(ctx, ko, ks, w3)
    _ms_vs_oracle(ctx, ko, ks, w3)


def test_seed_device_outputs_equal_host_outputs(ctx, ks_mod):
    """out= (device tensors) gives the same records as the host-output calls."""
    import torch
    ks = ks_mod
    w = synth.workload("spheres48")
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    o, m = ctx.seed_climb(v, p), ctx.meanshift(v, p)
    od = torch.zeros(len(o) * ks.SEED_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    md = torch.zeros(len(m) * ks.MS_RESULT.itemsize + 48, dtype=torch.uint8, device="cuda")
    assert ctx.seed_climb(v, p, out=od) == len(o)
    assert ctx.meanshift(v, p, out=md) == len(m)
    ctx.release_volume(v)
    assert np.array_equal(od.cpu().numpy().view(ks.SEED_RESULT), o)
    assert np.array_equal(md.cpu().numpy()[:len(m) * ks.MS_RESULT.itemsize].view(ks.MS_RESULT), m)
    with pytest.raises(ValueError):
        ctx.meanshift(ctx.create_volume(w.volume, w.binning), p, out=od[:16])


def test_released_volume_memory_is_reused_cleanly(ks_mod, ko):
    """A released volume's allocation is reused by the next volume of the same
    size: its halo must still read as not counted, and volumes of other sizes
    (and a tight budget) must still work."""
    ks = ks_mod
    a = synth.workload("spheres48")
    rng = np.random.default_rng(2)
    other = rng.integers(0, 256, size=a.volume.shape).astype(np.uint8)   # every bin occupied
    pa = _params(ks, a)
    budget = 3 * (56 + 64) ** 2 * (48 + 64) + (64 << 20)    # tables + a few volumes
    c = ks.Context(hbm_budget_bytes=budget)
    try:
        first = None
        for vol in (other, a.volume, other, a.volume):
            v = c.create_volume(vol, a.binning)
            Y, s = c.dense_saliency(v, pa, vol.shape)
            c.release_volume(v)
            if vol is a.volume:
                if first is None:
                    first = (Y, s)
                else:
                    assert np.array_equal(s, first[1]) and np.array_equal(Y, first[0])
        Yo, so = ko.dense(ko.bin_volume(a.volume, a.binning), a.binning["bins"], a.r_min, a.r_max)
        assert np.array_equal(first[1], so)
        close(first[0], Yo)
        # a different size after the pool holds the first one
        small = a.volume[:20, :30, :40].copy()
        v = c.create_volume(small, a.binning)
        assert np.array_equal(c.volume_bins(v, small.shape), ko.bin_volume(small, a.binning))
        c.release_volume(v)
    finally:
        c.close()


# ---------------------------------------------------- batched and serving
def test_batch_equals_plain_calls_and_oracle(ctx, ko, ks_mod):
    """The batched launch gives the plain calls' records bit for bit, and
    every volume's records equal the oracle's.  The batch mixes uint8
    sphere volumes (r = 2..10) with int16 MR-like volumes (r = 4..32, one
    of them with 64 bins), so mean shift takes both its warp path and its
    block path (r > 20 or more than 32 bins)."""
    ks = ks_mod
    ws = synth.batch_volumes(seed=5, count=6, hi=96)
    assert any(w.volume.dtype == np.int16 and w.binning["bins"] == 64 for w in ws)
    vols = [ctx.create_volume(w.volume, w.binning) for w in ws]
    ps = [_params(ks, w) for w in ws]
    for use_graph in (1, 0, 1):
        octs, mss = ctx.batch_seeds(vols, ps, kinds=3, use_graph=use_graph)
        for v, p, o, m in zip(vols, ps, octs, mss):
            assert np.array_equal(o, ctx.seed_climb(v, p))
            assert np.array_equal(m, ctx.meanshift(v, p))
    for w, o, m in zip(ws, octs, mss):
        oracle_checks.octant_records(ko, w, o)
        oracle_checks.meanshift_records(ko, w, m)
    for v in vols:
        ctx.release_volume(v)


def test_serving_results_alone_equal_mixed(ko, ks_mod):
    ks = ks_mod
    ws = synth.batch_volumes(seed=9, count=5, hi=80)
    c1 = ks.Context()
    alone = []
    for i, w in enumerate(ws):
        kind = ks.KS_REQ_DENSE if i % 3 == 2 else ks.KS_REQ_SEEDS
        rid = c1.submit(w.volume, w.binning, _params(ks, w), kind=kind)
        st, res = c1.poll(rid, -1)
        assert st == ks.KS_OK
        alone.append(res)
    mixed_ids = []
    for i, w in enumerate(ws):
        kind = ks.KS_REQ_DENSE if i % 3 == 2 else ks.KS_REQ_SEEDS
        mixed_ids.append(c1.submit(w.volume, w.binning, _params(ks, w), kind=kind))
    for rid, a in zip(mixed_ids, alone):
        st, res = c1.poll(rid, -1)
        assert st == ks.KS_OK
        for k in ("oct", "ms", "Y", "s"):
            assert (k in a) == (k in res)
            if k in a:
                assert np.array_equal(a[k], res[k]), k
    # seed items advance 1 iteration per wave, or whole searches per wave:
    # the same records
    for iters in (1, 0):
        c1.set_serve_wave_iters(iters)
        ids = [c1.submit(w.volume, w.binning, _params(ks, w),
                         kind=ks.KS_REQ_DENSE if i % 3 == 2 else ks.KS_REQ_SEEDS)
               for i, w in enumerate(ws)]
        for rid, a in zip(ids, alone):
            st, res = c1.poll(rid, -1)
            assert st == ks.KS_OK
            for k in ("oct", "ms", "Y", "s"):
                if k in a:
                    assert np.array_equal(a[k], res[k]), (iters, k)
    c1.set_serve_wave_iters(4)
    # the plain path gives the same numbers, and so does the oracle
    v = c1.create_volume(ws[0].volume, ws[0].binning)
    assert np.array_equal(alone[0]["oct"], c1.seed_climb(v, _params(ks, ws[0])))
    c1.close()
    for w, a in zip(ws, alone):
        if "oct" in a:
            oracle_checks.octant_records(ko, w, a["oct"])
            oracle_checks.meanshift_records(ko, w, a["ms"])
        else:
            oracle_checks.dense_maps(ko, w, a["Y"], a["s"])


def test_errors_are_reported_not_raised_across_abi(ctx, ks_mod):
    ks = ks_mod
    w = synth.workload("spheres48")
    with pytest.raises(ks.KsError) as e:
        ctx.create_volume(w.volume, {"kind": 0, "bins": 16, "shift": 2, "lo": 0, "hi": 255})
    assert e.value.status == ks.KS_EINVAL
    v = ctx.create_volume(w.volume, w.binning)
    with pytest.raises(ks.KsError) as e:
        ctx.seed_climb(v, ks.make_params(5, 40, 6))
    assert e.value.status == ks.KS_EINVAL
    with pytest.raises(ks.KsError) as e:
        ctx.seed_climb(v, ks.make_params(2, 10, 6), seeds=[[48, 0, 0]])
    assert e.value.status == ks.KS_EINVAL
    ctx.release_volume(v)
    with pytest.raises(ks.KsError) as e:
        ctx.seed_climb(v, ks.make_params(2, 10, 6))
    assert e.value.status == ks.KS_ENOTFOUND
    small = ks.Context(hbm_budget_bytes=64 << 20)
    big = np.zeros((300, 300, 300), np.uint8)
    with pytest.raises(ks.KsError) as e:
        small.create_volume(big, w.binning)
    assert e.value.status == ks.KS_ENOMEM
    small.close()


# ------------------------------------------------ points and selection
def test_dense_points_equal_oracle_centres(ctx, ko, ks_mod):
    ks = ks_mod
    for name, n in (("pet128", 700), ("mr256", 120), ("spheres48", 300)):
        w = synth.workload(name)
        v = ctx.create_volume(w.volume, w.binning)
        p = _params(ks, w)
        rng = np.random.default_rng(len(name))
        nx, ny, nz = w.dims
        cen = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)],
                       1).astype(np.int32)
        cen[:4] = [[0, 0, 0], [nx - 1, ny - 1, nz - 1], [0, ny - 1, nz // 2], [nx - 1, 0, 0]]
        Y, s, H, W = ctx.dense_points(v, p, cen, want_hw=True)
        b = ko.bin_volume(w.volume, w.binning)
        Yo, so, Ho, Wo = ko.dense(b, w.binning["bins"], w.r_min, w.r_max, centres=cen, want_hw=True)
        assert np.array_equal(s, so)
        close(Y, Yo)
        close(H, Ho)
        close(W, Wo)
        with pytest.raises(ks.KsError):
            ctx.dense_points(v, p, np.array([[nx, 0, 0]], np.int32))
        ctx.dense_points(v, p, cen[:3])            # the context is usable afterwards
        ctx.release_volume(v)


def _cand_list(arr):
    return [dict(x=int(c["x"]), y=int(c["y"]), z=int(c["z"]), r=int(c["r"]),
                 source=int(c["source"]), H=float(c["H"]), W=float(c["W"])) for c in arr]


def _same_cands(got, ref):
    got = _cand_list(got)
    assert [(c["x"], c["y"], c["z"], c["r"], c["source"]) for c in got] == \
        [(c["x"], c["y"], c["z"], c["r"], c["source"]) for c in ref]
    close([c["H"] for c in got], [c["H"] for c in ref])
    close([c["W"] for c in got], [c["W"] for c in ref])


def test_candidates_and_selection_equal_oracle(ctx, ko, ks_mod):
    ks = ks_mod
    w = synth.workload("pet128")
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    b = ko.bin_volume(w.volume, w.binning)
    B = w.binning["bins"]
    sd = ko.seed_grid(w.dims, w.stride)
    # octant: candidates from the GPU results equal the oracle's
    o = ctx.seed_climb(v, p)
    oref = ko.octant_climb(b, B, w.r_min, w.r_max, sd, w.max_iter)
    oc = ctx.octant_candidates(o)
    _same_cands(oc, ko.octant_candidates(oref))
    # mean shift: every item's final centre and radius, W evaluated there
    m = ctx.meanshift(v, p)
    mref = ko.meanshift(b, B, w.r_min, w.r_max, sd, w.max_iter)
    mc = ctx.meanshift_candidates(v, p, m)
    _same_cands(mc, ko.meanshift_candidates(b, B, w.r_min, w.r_max, mref, m["r"]))
    # the item's H at its own radius is the mean-shift kernel's final H
    close(mc["H"], m["H"])
    for cands in (oc, mc):
        ref_all = _cand_list(cands)
        for h_min, top_k in ((0.0, 20), (2.5, 20), (0.0, 1), (0.0, 256)):
            got = ctx.select_salient(cands, h_min=h_min, top_k=top_k)
            _same_cands(got, ko.select_salient(ref_all, h_min=h_min, top_k=top_k))
    ctx.release_volume(v)


def test_selection_many_ties_and_duplicates(ctx, ko, ks_mod):
    ks = ks_mod
    rng = np.random.default_rng(17)
    n = 50000                                        # several rounds of 1024-entry sorts
    c = np.zeros(n, ks.CANDIDATE)
    c["x"] = rng.integers(0, 6, n)
    c["y"] = rng.integers(0, 6, n)
    c["z"] = rng.integers(0, 40, n)
    c["r"] = rng.integers(0, 4, n)
    c["source"] = rng.permutation(n)
    key = ((c["z"] * 6 + c["y"]) * 6 + c["x"]) * 4 + c["r"]
    # H and W are functions of the region, with many equal values
    c["W"] = (key % 7) * 0.125
    c["H"] = (key % 5) * 0.5
    ref_all = _cand_list(c)
    for h_min, top_k in ((0.0, 256), (0.75, 20), (-1.0, 7)):
        got = ctx.select_salient(c, h_min=h_min, top_k=top_k)
        _same_cands(got, ko.select_salient(ref_all, h_min=h_min, top_k=top_k))
    assert len(ctx.select_salient(c[:0], top_k=5)) == 0
    with pytest.raises(ks.KsError):
        ctx.select_salient(c[:10], top_k=257)


def test_window_level_workload_equals_oracle(ctx, ko, ks_mod):
    """The MR workload with the tumour window level (voxels outside [800,
    2047] not counted): binning, both seed schemes on sampled seeds and the
    Kadir-Brady quantities at sampled centres equal the oracle's."""
    ks = ks_mod
    w = synth.workload("mr256w")
    v = ctx.create_volume(w.volume, w.binning)
    b = ko.bin_volume(w.volume, w.binning)
    assert np.array_equal(ctx.volume_bins(v, w.volume.shape), b)
    assert (b == 0).mean() > 0.5                      # most voxels fall outside the window
    ctx.release_volume(v)
    grid = ko.seed_grid(w.dims, w.stride)
    rng = np.random.default_rng(5)
    seeds = grid[rng.choice(len(grid), 40, replace=False)].astype(np.int32)
    _oct_vs_oracle(ctx, ko, ks, w, seeds=seeds, traj=True)
    _ms_vs_oracle(ctx, ko, ks, w, seeds=seeds[:12])
    v = ctx.create_volume(w.volume, w.binning)
    nx, ny, nz = w.dims
    cen = np.stack([rng.integers(0, nx, 200), rng.integers(0, ny, 200), rng.integers(0, nz, 200)],
                   1).astype(np.int32)
    Y, s, H, W = ctx.dense_points(v, _params(ks, w), cen, want_hw=True)
    ctx.release_volume(v)
    Yo, so, Ho, Wo = ko.dense(b, w.binning["bins"], w.r_min, w.r_max, centres=cen, want_hw=True)
    assert np.array_equal(s, so)
    close(Y, Yo)
    close(H, Ho)
    close(W, Wo)


@pytest.mark.parametrize("name", ["spheres48", "pet128"])
def test_quadrant_climb_equals_oracle(ctx, ko, ks_mod, name):
    """Alg. 1 as printed (2D quadrants, disks in each seed's slice): every
    grid seed, final centres, iterations, trajectories and the disk
    Kadir-Brady evaluation bit-exact against the oracle."""
    ks = ks_mod
    w = synth.workload(name)
    v = ctx.create_volume(w.volume, w.binning)
    got, gtraj = ctx.seed_climb(v, _params(ks, w), want_traj=True, planar=True)
    ctx.release_volume(v)
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride)
    ref = ko.octant_climb(b, w.binning["bins"], w.r_min, w.r_max, sd, w.max_iter,
                          want_traj=True, planar=True)
    assert np.array_equal(np.stack([got["x"], got["y"], got["z"]], 1), ref["xyz"])
    assert np.array_equal(got["z"], sd[:, 2])                      # stays in its slice
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])
    assert np.array_equal(got["s_best"], ref["s"])
    assert np.array_equal(gtraj, ref["traj"])
    close(got["Y_best"], ref["Y"])
    close(got["H_best"], ref["H"])
    close(got["W_best"], ref["W"])


# ----------------------------------------------------------------- ABMSOD
def _ab_vs_oracle(ctx, ko, ks, w, seeds=None, max_iter=None):
    """Adaptive-bandwidth mean shift (Alg. 2, Eq. 7) against the kernel's
    stated arithmetic (oracle.abmsod_fixed: binary32 voxel terms, exact
    membership, exact fixed-point sums): every item's best centre,
    bandwidth, rho, iteration count, stop flag and window voxels bit for
    bit.  The distance of that arithmetic from the plain binary64 oracle is
    bounded by the per-iteration tests below."""
    v = ctx.create_volume(w.volume, w.binning)
    it = w.max_iter if max_iter is None else max_iter
    p = ks.make_params(w.r_min, w.r_max, w.stride, it)
    got = ctx.abmsod(v, p, seeds=seeds)
    ctx.release_volume(v)
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride) if seeds is None else np.asarray(seeds, np.int32)
    ref = ko.abmsod_fixed(b, w.binning["bins"], w.r_min, w.r_max, sd, it)
    S = w.r_max - w.r_min + 1
    assert np.array_equal(got["seed"], np.repeat(np.arange(len(sd)), S))
    assert np.array_equal(got["r"], np.tile(np.arange(w.r_min, w.r_max + 1), len(sd)))
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["stopped"], ref["stopped"])
    assert np.array_equal(got["voxels"], ref["voxels"])
    assert np.array_equal(got["x"].view(np.uint64), ref["x"].view(np.uint64))
    assert np.array_equal(got["H"].view(np.uint64), ref["H"].view(np.uint64))
    assert np.array_equal(got["rho"].view(np.uint64), ref["rho"].view(np.uint64))
    return got, ref


def test_abmsod_spheres48_all_items(ctx, ko, ks_mod):
    got, _ = _ab_vs_oracle(ctx, ko, ks_mod, synth.workload("spheres48"))
    assert (got["stopped"] == 1).any() and (got["iters"] == 20).any()


def test_abmsod_pet128_sampled_seeds(ctx, ko, ks_mod):
    """pet128 at its full size: every 8th grid seed at all 17 radii (the
    launch shape of the full grid, fewer items for the oracle)."""
    w = synth.workload("pet128")
    grid = ko.seed_grid(w.dims, w.stride)
    _ab_vs_oracle(ctx, ko, ks_mod, w, seeds=grid[::8].copy())


def test_abmsod_64_bins_and_edges(ctx, ko, ks_mod):
    """mr256 (64 bins: two bins per lane), radii up to 32 (windows up to 65
    voxels wide, at the halo), seeds on the volume's corners and faces."""
    w = synth.workload("mr256")
    grid = ko.seed_grid(w.dims, w.stride)
    rng = np.random.default_rng(5)
    pick = grid[rng.choice(len(grid), 6, replace=False)]
    edge = np.array([[0, 0, 0], [255, 255, 159], [128, 0, 80], [255, 130, 0]], np.int32)
    seeds = np.concatenate([pick, edge]).astype(np.int32)
    w.r_min, w.r_max = 22, 32
    _ab_vs_oracle(ctx, ko, ks_mod, w, seeds=seeds, max_iter=6)


def test_abmsod_window_level_and_edge_cases(ctx, ko, ks_mod):
    """Uncounted voxels (window level), a constant volume (HP = e_b every
    iteration), an all-uncounted volume (empty windows), ragged small
    volumes, max_iter 0 and 1, a single seed."""
    ks = ks_mod
    w = synth.workload("mr256w")
    grid = ko.seed_grid(w.dims, w.stride)
    _ab_vs_oracle(ctx, ko, ks, w, seeds=grid[::97].copy(), max_iter=5)
    vol = np.full((20, 21, 22), 77, np.uint8)
    wc = synth.Workload("const", vol, {"kind": 0, "bins": 16, "shift": 4, "lo": 0, "hi": 255},
                        2, 6, 5, 7)
    got, _ = _ab_vs_oracle(ctx, ko, ks, wc)
    assert (got["rho"] == 0.25).all()
    we = synth.Workload("empty", vol, {"kind": 2, "bins": 8, "shift": 4, "lo": 200, "hi": 255},
                        1, 4, 7, 3)
    got, _ = _ab_vs_oracle(ctx, ko, ks, we)
    assert (got["iters"] == 0).all() and (got["rho"] == 0.0).all()
    rng = np.random.default_rng(8)
    vr = rng.integers(0, 7, size=(9, 13, 31)).astype(np.uint8)
    wr = synth.Workload("ragged", vr, {"kind": 0, "bins": 7, "shift": 0, "lo": 0, "hi": 6},
                        1, 5, 4, 9)
    _ab_vs_oracle(ctx, ko, ks, wr)
    _ab_vs_oracle(ctx, ko, ks, wr, max_iter=0)
    _ab_vs_oracle(ctx, ko, ks, wr, max_iter=1)
    _ab_vs_oracle(ctx, ko, ks, synth.workload("spheres48"), seeds=np.array([[24, 20, 30]]))


def test_abmsod_device_output_equals_host(ctx, ks_mod):
    import torch
    ks = ks_mod
    w = synth.workload("spheres48")
    v = ctx.create_volume(w.volume, w.binning)
    p = _params(ks, w)
    a = ctx.abmsod(v, p)
    d = torch.zeros(len(a) * ks.AB_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    assert ctx.abmsod(v, p, out=d) == len(a)
    ctx.release_volume(v)
    assert np.array_equal(d.cpu().numpy().view(ks.AB_RESULT), a)


def test_abmsod_team_split_does_not_change_results(ctx, ko, ks_mod):
    """Every item on one warp, every item on a whole block, and the default
    split give the same records (and equal the oracle)."""
    ks = ks_mod
    w = synth.workload("spheres48")
    grid = ko.seed_grid(w.dims, w.stride)[::5].copy()
    outs = []
    try:
        for rt in (33, 1, 6, 0):
            ks.set_abmsod_team_radius(rt)
            outs.append(_ab_vs_oracle(ctx, ko, ks, w, seeds=grid)[0])
    finally:
        ks.set_abmsod_team_radius(0)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    with pytest.raises(ks.KsError):
        ks.set_abmsod_team_radius(34)
    # radii up to 20: large windows on one warp and on whole blocks
    w = synth.workload("pet128")
    grid = ko.seed_grid(w.dims, w.stride)[::16].copy()
    outs = []
    try:
        for rt in (33, 1):
            ks.set_abmsod_team_radius(rt)
            outs.append(_ab_vs_oracle(ctx, ko, ks, w, seeds=grid, max_iter=8)[0])
    finally:
        ks.set_abmsod_team_radius(0)
    assert np.array_equal(outs[0], outs[1])


# ------------------------------- ABMSOD against the plain binary64 oracle
def _ab_per_iteration(ctx, ko, w, seeds):
    """Every iteration of the oracle's searches from `seeds` at every radius,
    replayed one at a time: the GPU runs one iteration (through
    ks_abmsod_candidates) from each state the oracle visits, and the
    results are compared at the bounds of tests/abmsod_chain.py."""
    b = ko.bin_volume(w.volume, w.binning)
    B = w.binning["bins"]
    x0, H0 = abmsod_chain.seed_items(seeds, w.r_min, w.r_max)
    st = abmsod_chain.oracle_states(ko, b, B, x0, H0, w.max_iter)
    v = ctx.create_volume(w.volume, w.binning)
    got = ctx.abmsod_candidates(v, st["x"], st["H"], max_iter=1)
    ctx.release_volume(v)
    assert np.array_equal(got["seed"], np.arange(len(st["x"])))
    assert (got["r"] == 0).all()
    far, near = abmsod_chain.compare(st, got)
    return far, near


def test_abmsod_per_iteration_vs_plain_oracle_spheres48(ctx, ko):
    """All 4608 items of the spheres workload, every iteration."""
    w = synth.workload("spheres48")
    far, near = _ab_per_iteration(ctx, ko, w, ko.seed_grid(w.dims, w.stride))
    assert far >= 0.8 * (far + near)


def test_abmsod_per_iteration_vs_plain_oracle_pet128(ctx, ko):
    """pet128 at full size (128 x 128 x 64 float32, 32 bins, r = 4..20):
    every 16th grid seed at all 17 radii, every iteration."""
    w = synth.workload("pet128")
    far, near = _ab_per_iteration(ctx, ko, w, ko.seed_grid(w.dims, w.stride)[::16])
    assert far >= 0.6 * (far + near)


def test_abmsod_per_iteration_vs_plain_oracle_mr256_large_windows(ctx, ko):
    """mr256 (64 bins, windows to r = 32 at the halo, corner seeds)."""
    w = synth.workload("mr256")
    grid = ko.seed_grid(w.dims, w.stride)
    rng = np.random.default_rng(5)
    seeds = np.concatenate([grid[rng.choice(len(grid), 5, replace=False)],
                            np.array([[0, 0, 0], [255, 255, 159], [128, 0, 80]])]).astype(np.int32)
    w.r_min, w.r_max, w.max_iter = 24, 32, 6
    far, near = _ab_per_iteration(ctx, ko, w, seeds)
    assert far + near > 100


def test_abmsod_whole_searches_vs_plain_oracle(ctx, ko, ks_mod):
    """Whole GPU searches against whole oracle searches: most items take the
    same path; the others part where the stopping test meets a tie of rho
    (flat to ~1e-7 near convergence) or a boundary voxel, and still end at
    nearby optima.  Every record is valid: rho in [0, 1], the diagonal of
    H in [1, 32^2], the centre in the volume, iterations within the limit,
    a stop flag only before the limit."""
    ks = ks_mod
    for name, step in (("spheres48", 1), ("pet128", 8)):
        w = synth.workload(name)
        sd = ko.seed_grid(w.dims, w.stride)[::step].copy()
        v = ctx.create_volume(w.volume, w.binning)
        got = ctx.abmsod(v, _params(ks, w), seeds=sd)
        ctx.release_volume(v)
        ref = ko.abmsod(ko.bin_volume(w.volume, w.binning), w.binning["bins"], w.r_min,
                        w.r_max, sd, w.max_iter)
        same = (got["iters"] == ref["iters"]) & (got["stopped"] == ref["stopped"])
        assert same.mean() >= 0.9, (name, same.mean())
        dr = np.abs(got["rho"] - ref["rho"])
        assert np.median(dr) <= 1e-6 and np.mean(dr <= 1e-4) >= 0.9, name
        assert np.median(np.abs(got["x"] - ref["x"]).max(1)) <= 1e-3, name
        assert abs(got["rho"].mean() - ref["rho"].mean()) <= 1e-3, name
        assert ((got["rho"] >= 0) & (got["rho"] <= 1)).all()
        for k in (0, 3, 5):
            assert ((got["H"][:, k] >= 1) & (got["H"][:, k] <= 1024)).all()
        assert ((got["x"] >= 0) & (got["x"] <= np.array(w.dims, float) - 1)).all()
        assert ((got["iters"] >= 0) & (got["iters"] <= w.max_iter)).all()
        assert not ((got["stopped"] == 1) & (got["iters"] == 0)).any()


def test_abmsod_candidates_entry_point(ctx, ko, ks_mod):
    """ks_abmsod_candidates from (seed, r^2 I) gives ks_abmsod's records;
    device inputs give the host inputs' records; given oblique candidates
    equal the fixed-point model; bad candidates are refused."""
    import torch
    ks = ks_mod
    w = synth.workload("spheres48")
    sd = ko.seed_grid(w.dims, w.stride)[::7].copy()
    v = ctx.create_volume(w.volume, w.binning)
    a = ctx.abmsod(v, _params(ks, w), seeds=sd)
    x0, H0 = abmsod_chain.seed_items(sd, w.r_min, w.r_max)
    c = ctx.abmsod_candidates(v, x0, H0, max_iter=w.max_iter)
    for k in ("x", "H", "rho", "iters", "stopped", "voxels"):
        assert np.array_equal(c[k], a[k]), k
    rng = np.random.default_rng(4)
    n = 300
    xs = rng.uniform(0, 47, size=(n, 3))
    Hs = np.zeros((n, 6))
    for i in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        M = Q @ np.diag(np.exp(rng.uniform(np.log(2.0), np.log(90.0), 3))) @ Q.T
        Hs[i] = [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]]
    c = ctx.abmsod_candidates(v, xs, Hs, max_iter=6)
    ref = ko.abmsod_fixed(ko.bin_volume(w.volume, w.binning), w.binning["bins"], 0, 0, None, 6,
                          cand=(xs, Hs))
    for k in ("x", "H", "rho", "iters", "stopped", "voxels"):
        assert np.array_equal(c[k], ref[k]), k
    d = ctx.abmsod_candidates(v, torch.from_numpy(xs).cuda(), torch.from_numpy(Hs).cuda(),
                              max_iter=6)
    assert np.array_equal(d.cpu().numpy().view(ks.AB_RESULT), c)
    for bx, bH in (([[48.0, 1.0, 1.0]], [[4, 0, 0, 4, 0, 4]]),
                   ([[5.0, 5.0, 5.0]], [[1100, 0, 0, 4, 0, 4]]),
                   ([[5.0, 5.0, 5.0]], [[0.5, 0, 0, 4, 0, 4]])):
        with pytest.raises(ks.KsError) as e:
            ctx.abmsod_candidates(v, np.array(bx), np.array(bH, float))
        assert e.value.status == ks.KS_EINVAL
        with pytest.raises(ks.KsError) as e:
            ctx.abmsod_candidates(v, torch.tensor(bx, dtype=torch.float64, device="cuda"),
                                  torch.tensor(bH, dtype=torch.float64, device="cuda"))
        assert e.value.status == ks.KS_EINVAL
    assert len(ctx.abmsod_candidates(v, x0, H0, max_iter=1)) == len(x0)   # context still usable
    ctx.release_volume(v)


# ------------------------------------------- dense sweep in z-slabs (GPU)
def test_stored_bins_and_dense_range_equal_the_whole_sweep(ctx, ko, ks_mod):
    """A volume made from stored bins (KS_BIN_STORED) reproduces them
    (values above `bins` are not counted); the sweep of planes [z0, z1)
    equals the whole sweep's planes; three z-slabs with their r_max halos,
    each swept on the GPU, merge into the whole sweep (the per-rank work of
    the sharded dense sweep, run here in one process)."""
    from paper_1310_6736_b300 import shard
    ks = ks_mod
    w = synth.workload("pet128")
    p = _params(ks, w)
    v = ctx.create_volume(w.volume, w.binning)
    Y, s = ctx.dense_saliency(v, p, w.volume.shape)
    bins = ctx.volume_bins(v, w.volume.shape)
    Yr, sr = ctx.dense_saliency_range(v, p, w.volume.shape, 20, 44)
    ctx.release_volume(v)
    assert np.array_equal(sr, s[20:44]) and np.array_equal(Yr, Y[20:44])
    noisy = bins.copy()
    noisy[::7, 3, 5] = 250                                   # above bins: not counted
    vs = ctx.create_volume(noisy, {"kind": ks.KS_BIN_STORED, "bins": 32, "shift": 0, "lo": 0,
                                   "hi": 0})
    want = np.where(noisy <= 32, noisy, 0)
    assert np.array_equal(ctx.volume_bins(vs, w.volume.shape), want)
    ctx.release_volume(vs)
    ex = shard.gpu_slab_executor(ctx, 32, p)
    parts = [shard.dense_slab(bins, w.r_max, z0, z1, ex) for z0, z1 in shard.z_slabs(64, 3)]
    Ym, sm = shard.merge_slabs(parts, 64)
    assert np.array_equal(sm, s) and np.array_equal(Ym, Y)
    Yo, so = ko.dense(bins, 32, w.r_min, w.r_max,
                      centres=np.array([[5, 7, 21], [64, 64, 22], [127, 0, 43]], np.int32))
    assert np.array_equal(sm[[21, 22, 43], [7, 64, 0], [5, 64, 127]], so)
    with pytest.raises(ks.KsError):
        ctx.create_volume(w.volume, {"kind": ks.KS_BIN_STORED, "bins": 32, "shift": 0, "lo": 0,
                                     "hi": 0})                # float32 data: refused
