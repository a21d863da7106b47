"""Seeded synthetic volumes shaped like the paper's workloads.

The paper evaluates on PET volumes (128x128x34, Sec. 3.1) and FLAIR MR brain
volumes (256x256x176, Sec. 3.2); neither dataset ships here, so these
generators stand in for them with the shapes, value ranges and structure of
those workloads (a homogeneous background with compact high-entropy regions,
as in the toy model of Sec. 2.1).

This module holds only random-number generation and geometry.  It contains
none of the method's arithmetic (no binning, histograms or entropies), so the
CUDA path and the CPU oracle can both draw their inputs from it.

Volumes are numpy arrays of shape (nz, ny, nx): x is the fastest axis and the
voxel index is (z*ny + y)*nx + x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload", "spheres_u8", "pet_f32", "mr_i16", "batch_volumes",
    "request_stream", "workload", "WORKLOADS",
]


@dataclass
class Workload:
    """One synthetic volume plus the method parameters it is evaluated with."""
    name: str
    volume: np.ndarray            # (nz, ny, nx)
    binning: dict                 # kind, bins, shift, lo, hi
    r_min: int
    r_max: int
    stride: int
    max_iter: int = 20
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        nz, ny, nx = self.volume.shape
        return nx, ny, nz


def _grid(nx, ny, nz):
    """Broadcastable coordinate arrays (x: (1,1,nx), y: (1,ny,1), z: (nz,1,1))."""
    return (np.arange(nx, dtype=np.float64)[None, None, :],
            np.arange(ny, dtype=np.float64)[None, :, None],
            np.arange(nz, dtype=np.float64)[:, None, None])


def spheres_u8(seed=0, dims=(48, 48, 48), radii=(10, 7, 4)):
    """uint8 volume: Gaussian(40, 5) background, spheres of uniform [0,255].

    Spheres are placed in the given order at integer centres drawn so that
    each sphere lies fully inside the volume and no two spheres touch
    (centre distance > r1 + r2).  Radii that do not fit are clipped to
    (min(dims) - 1) // 2.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    vol = np.clip(np.rint(rng.normal(40.0, 5.0, size=(nz, ny, nx))), 0, 255).astype(np.uint8)
    x, y, z = _grid(nx, ny, nz)
    placed = []
    rcap = max(1, (min(dims) - 1) // 2)
    for r0 in radii:
        r = min(r0, rcap)
        for _attempt in range(10000):
            c = (int(rng.integers(r, nx - r)), int(rng.integers(r, ny - r)),
                 int(rng.integers(r, nz - r)))
            if all(math.dist(c, pc) > r + pr for pc, pr in placed):
                break
        else:   # crowded small volume: accept overlap rather than loop forever
            pass
        placed.append((c, r))
        inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= r * r
        vol[inside] = rng.integers(0, 256, size=int(inside.sum()), dtype=np.uint8)
    return vol, {"spheres": [(list(c), r) for c, r in placed]}


def pet_f32(seed=1, dims=(128, 128, 64), semi=(18, 14, 16), thick=3, sigma=1.5):
    """float32 PET-like volume: Gamma(2,1) background, Gamma(9,1) ellipsoidal
    shell (semi-axes `semi`, thickness `thick`) at a random fully-inside
    centre, then an isotropic Gaussian blur (sigma 1.5, reflect, truncate 4).
    """
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    vol = rng.gamma(2.0, 1.0, size=(nz, ny, nx)).astype(np.float32)
    c = [int(rng.integers(s, n - s)) for s, n in zip(semi, dims)]
    x, y, z = _grid(nx, ny, nz)

    def inside(a):
        return (((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2
                + ((z - c[2]) / a[2]) ** 2) <= 1.0

    shell = inside(semi) & ~inside([s - thick for s in semi])
    vol[shell] = rng.gamma(9.0, 1.0, size=int(shell.sum())).astype(np.float32)
    vol = gaussian_filter(vol, sigma=sigma, mode="reflect", truncate=4.0).astype(np.float32)
    return np.ascontiguousarray(vol), {"shell_centre": c}


def mr_i16(seed=2, dims=(256, 256, 160), n_tumours=None):
    """int16 MR-brain-like volume.

    A centred ellipsoidal brain (semi-axes 0.40, 0.45, 0.42 of each dim)
    holds 600 + N(0, 40) under a multiplicative linear bias field
    1 + 0.15 (u . v), u a random unit vector and v the normalised ellipsoid
    coordinate, so the bias spans +-15%.  Air outside is 0.  1-4 tumours are
    ellipsoids with per-axis radii U[8, 25] centred inside the brain, with an
    interior drawn uniformly from {200..1400} and an outer rim of thickness 2
    at 900 + N(0, 40).  Values are clipped to [0, 2047].
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    x, y, z = _grid(nx, ny, nz)
    c = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    a = np.array([0.40 * nx, 0.45 * ny, 0.42 * nz])
    vx, vy, vz = (x - c[0]) / a[0], (y - c[1]) / a[1], (z - c[2]) / a[2]
    brain = vx * vx + vy * vy + vz * vz <= 1.0
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    bias = np.broadcast_to(1.0 + 0.15 * (u[0] * vx + u[1] * vy + u[2] * vz), brain.shape)
    vol = np.zeros((nz, ny, nx), dtype=np.float32)
    vol[brain] = (600.0 + rng.normal(0.0, 40.0, size=int(brain.sum()))) * bias[brain]
    nt = int(rng.integers(1, 5)) if n_tumours is None else n_tumours
    tumours = []
    scale = min(dims) / 160.0          # keep blobs proportionate on small volumes
    for _ in range(nt):
        rad = np.maximum(3.0, rng.uniform(8.0, 25.0, size=3) * min(1.0, scale))
        for _attempt in range(1000):
            t = c + (rng.uniform(-1.0, 1.0, size=3) * a * 0.6)
            if (((t - c) / a) ** 2).sum() <= 0.36:
                break
        tumours.append((t.tolist(), rad.tolist()))
        # work inside the blob's bounding box only
        lo_ = [max(0, int(math.floor(t[k] - rad[k]))) for k in range(3)]
        hi_ = [min(n, int(math.ceil(t[k] + rad[k])) + 1) for k, n in enumerate(dims)]
        bx, by, bz = x[..., lo_[0]:hi_[0]], y[:, lo_[1]:hi_[1], :], z[lo_[2]:hi_[2]]
        q = (((bx - t[0]) / rad[0]) ** 2 + ((by - t[1]) / rad[1]) ** 2
             + ((bz - t[2]) / rad[2]) ** 2)
        inner_rad = np.maximum(rad - 2.0, 0.5)
        qi = (((bx - t[0]) / inner_rad[0]) ** 2 + ((by - t[1]) / inner_rad[1]) ** 2
              + ((bz - t[2]) / inner_rad[2]) ** 2)
        body = qi <= 1.0
        rim = (q <= 1.0) & ~body
        sub = vol[lo_[2]:hi_[2], lo_[1]:hi_[1], lo_[0]:hi_[0]]
        sub[body] = rng.integers(200, 1401, size=int(body.sum()))
        sub[rim] = 900.0 + rng.normal(0.0, 40.0, size=int(rim.sum()))
    np.rint(vol, out=vol)
    np.clip(vol, 0, 2047, out=vol)
    vol = vol.astype(np.int16)
    return vol, {"tumours": tumours, "bias_dir": u.tolist()}


# Binning descriptors (interpreted by the library and by the oracle).
KS_BIN_CLAMP_SHIFT = 0
KS_BIN_AFFINE_F32 = 1
KS_BIN_WINDOW = 2


def _u8_binning(bins):
    return {"kind": KS_BIN_CLAMP_SHIFT, "bins": bins, "shift": {16: 4, 32: 3, 64: 2}[bins],
            "lo": 0, "hi": 255}


def _i16_binning(bins):
    return {"kind": KS_BIN_CLAMP_SHIFT, "bins": bins, "shift": {32: 6, 64: 5}[bins],
            "lo": 0, "hi": 2047}


def batch_volumes(seed=3, count=64, lo=48, hi=256, zcap=160, max_dim=None):
    """Uneven-size batch: every dim log-uniform in [lo, hi] (z capped at zcap).
    Even entries are uint8 sphere volumes (radii r=2..10), odd entries are
    int16 MR-like volumes (radii r=4..32).  Stride is drawn from {8..12}
    and the bin count from {32, 64}.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3)]
        d[2] = min(d[2], zcap)
        if max_dim is not None:
            d = [min(v, max_dim) for v in d]
        stride = int(rng.integers(8, 13))
        bins = int(rng.choice([32, 64]))
        sub = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            vol, meta = spheres_u8(sub, tuple(d))
            out.append(Workload(f"batch{i}-u8", vol, _u8_binning(bins), 2, 10, stride, 20, meta))
        else:
            vol, meta = mr_i16(sub, tuple(d))
            out.append(Workload(f"batch{i}-i16", vol, _i16_binning(bins), 4, 32, stride, 20, meta))
    return out


def request_stream(seed=4, count=2000, rate=50.0, dense_frac=0.3, max_dim=None):
    """Poisson request stream: exponential inter-arrival times at `rate`
    per second; each request carries a volume drawn as in `batch_volumes`
    (generated lazily by the caller from `vol_seed`) and asks for the seed
    schemes (70%) or the dense sweep (30%)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    kinds = np.where(rng.random(count) < dense_frac, "dense", "seeds")
    vol_seeds = rng.integers(0, 2**31 - 1, size=count)
    return [{"t": float(t[i]), "kind": str(kinds[i]), "vol_seed": int(vol_seeds[i]),
             "max_dim": max_dim} for i in range(count)]


def workload(name, **kw):
    """The named workloads: 'spheres48' (48^3 uint8, 16 bins, r=2..10,
    stride 6), 'pet128' (128x128x64 float32, 32 bins, r=4..20, stride 8),
    'mr256' (256x256x160 int16, 64 bins, r=4..32, stride 12)."""
    if name == "spheres48":
        vol, meta = spheres_u8(kw.get("seed", 0), kw.get("dims", (48, 48, 48)))
        return Workload(name, vol, _u8_binning(16), 2, 10, 6, 20, meta)
    if name == "pet128":
        vol, meta = pet_f32(kw.get("seed", 1), kw.get("dims", (128, 128, 64)))
        return Workload(name, vol, {"kind": KS_BIN_AFFINE_F32, "bins": 32, "shift": 0,
                                    "lo": 0, "hi": 0}, 4, 20, 8, 20, meta)
    if name == "mr256":
        vol, meta = mr_i16(kw.get("seed", 2), kw.get("dims", (256, 256, 160)))
        return Workload(name, vol, _i16_binning(64), 4, 32, 12, 20, meta)
    if name == "mr256w":
        # the same MR volume with a tumour window level: only intensities in
        # [800, 2047] are counted (normal tissue, 600 +- 40 under a +-15%
        # bias, and air fall outside), 39 bins of 32 levels
        vol, meta = mr_i16(kw.get("seed", 2), kw.get("dims", (256, 256, 160)))
        return Workload(name, vol, dict(MR_TUMOUR_WINDOW), 4, 32, 12, 20, meta)
    raise KeyError(name)


# Window-level binning of the MR workloads (Sec. 3.2: entropy over the
# intensity range of a tumour-specific window level)
MR_TUMOUR_WINDOW = {"kind": 2, "bins": 39, "shift": 5, "lo": 800, "hi": 2047}


def in_tumour(meta, xyz):
    """True for each xyz (n, 3) inside one of the MR volume's tumour
    ellipsoids (meta as mr_i16 returns it)."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    hit = np.zeros(len(xyz), bool)
    for t, rad in meta.get("tumours", []):
        q = (((xyz - np.asarray(t)) / np.asarray(rad)) ** 2).sum(axis=1)
        hit |= q <= 1.0
    return hit


WORKLOADS = ("spheres48", "pet128", "mr256", "mr256w")
