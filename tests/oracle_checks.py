"""Comparisons of CUDA-path records with the CPU oracle, shared by the GPU
tests of the plain, batched and serving forms.

Bar (the method's statement): integers exact (centres, iterations,
convergence flags, scale indices, bins); FP64 values within
|gpu - oracle| <= 1e-12 * max(1, |oracle|)."""
import numpy as np

RTOL = 1e-12


def close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape
    bad = np.abs(a - b) > RTOL * np.maximum(1.0, np.abs(b))
    assert not bad.any(), f"{bad.sum()} of {bad.size} differ; first at {np.argwhere(bad)[:3]}"
    return int((a == b).sum())


def octant_records(ko, w, got, seeds=None):
    """Octant-climb records (SEED_RESULT) of workload w against
    oracle.octant_climb on the same binned volume and seeds."""
    b = ko.bin_volume(w.volume, w.binning)
    sd = ko.seed_grid(w.dims, w.stride) if seeds is None else np.asarray(seeds, np.int32)
    ref = ko.octant_climb(b, w.binning["bins"], w.r_min, w.r_max, sd, w.max_iter)
    assert len(got) == len(sd)
    assert np.array_equal(np.stack([got["seed_x"], got["seed_y"], got["seed_z"]], 1), sd)
    assert np.array_equal(np.stack([got["x"], got["y"], got["z"]], 1), ref["xyz"])
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])
    assert np.array_equal(got["s_best"], ref["s"])
    close(got["Y_best"], ref["Y"])
    close(got["H_best"], ref["H"])
    close(got["W_best"], ref["W"])


def meanshift_records(ko, w, got, seeds=None):
    """Mean-shift records (MS_RESULT, one per (seed, r) item) of workload w
    against oracle.meanshift."""
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


def dense_maps(ko, w, Y, s, sample=None, seed=0):
    """Dense Y_best / s_best maps (flat or shaped like the volume) of
    workload w against oracle.dense: every voxel when sample is None, else
    `sample` random voxels plus the eight corners."""
    b = ko.bin_volume(w.volume, w.binning)
    nz, ny, nx = w.volume.shape
    Y = np.asarray(Y).reshape(-1)
    s = np.asarray(s).reshape(-1)
    if sample is None:
        Yo, so = ko.dense(b, w.binning["bins"], w.r_min, w.r_max)
        assert np.array_equal(s, so.reshape(-1))
        close(Y, Yo.reshape(-1))
        return
    rng = np.random.default_rng(seed)
    idx = rng.choice(Y.size, min(sample, Y.size), replace=False)
    corners = [((z * ny) + y) * nx + x for z in (0, nz - 1) for y in (0, ny - 1)
               for x in (0, nx - 1)]
    idx = np.unique(np.concatenate([idx, corners]))
    xyz = np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], 1).astype(np.int32)
    Yo, so = ko.dense(b, w.binning["bins"], w.r_min, w.r_max, centres=xyz)
    assert np.array_equal(s[idx], so)
    close(Y[idx], Yo)
