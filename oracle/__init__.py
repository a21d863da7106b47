"""CPU oracle for the Kadir-Brady saliency hot path -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg (and its
`--impl reference` arm) may import this package.  The product path (the
C-ABI library and its Python binding) never imports it, and the two share no
code: this package is plain C (ks_oracle.c, built with gcc -O2
-ffp-contract=off) behind ctypes, plus numpy marshalling.

Every function follows a passage of arXiv 1310.6736 (cited in ks_oracle.c)
and is pinned by tests/test_oracle_*.py against brute force, closed forms
(Eq. 2-3) and invariants.  Parity unpinned: none of the functions here; the
paper's accuracy experiments (Table 1, Jaccard indices) need datasets that
are not available and are out of scope.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ks_oracle.c")
_SRC_FIXED = os.path.join(_HERE, "ks_abmsod_fixed.c")
_LIB = os.path.join(_HERE, "libks_oracle.so")
_lock = threading.Lock()
_lib = None

BIN_CLAMP_SHIFT, BIN_AFFINE_F32, BIN_WINDOW, BIN_STORED = 0, 1, 2, 3


def build(force=False):
    """Compile ks_oracle.c and ks_abmsod_fixed.c into libks_oracle.so (gcc,
    OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and all(
            os.path.getmtime(_LIB) >= os.path.getmtime(f) for f in (_SRC, _SRC_FIXED)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
           "-fPIC", "-o", tmp, _SRC, _SRC_FIXED, "-lquadmath", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
            sig = {
                "ko_tables": (None, [I64, P, P]),
                "ko_bin_int": (None, [P, I64, I32, I32, I32, I32, I32, P]),
                "ko_bin_f32": (None, [P, I64, I32, P, P, P]),
                "ko_window_counts": (None, [P, I32, I32, I32, I32, I32, I32, I32, I32, P]),
                "ko_entropy": (D, [P, I32, P, P]),
                "ko_weight": (D, [P, P, I32, I32, I32]),
                "ko_dense": (None, [P, I32, I32, I32, I32, I32, I32, I32, P, P, P, I64, I32,
                                    I32, P, P, P, P]),
                "ko_seed_grid": (I64, [I32, I32, I32, I32, P]),
                "ko_octant_climb": (None, [P, I32, I32, I32, I32, I32, I32, I32, I32, P, P,
                                           P, I64, I32, P, P, P, P, P, P, P, P]),
                "ko_quadrant_climb": (None, [P, I32, I32, I32, I32, I32, I32, I32, I32, P, P,
                                             P, I64, I32, P, P, P, P, P, P, P, P]),
                "ko_meanshift": (None, [P, I32, I32, I32, I32, I32, I32, I32, P, P, P, I64,
                                        I32, P, P, P, P, P]),
                "ko_octant_counts": (None, [P, I32, I32, I32, I32, I32, I32, I32, I32, I32, P]),
                "ko_octant_one_step": (None, [P, I32, I32, I32, I32, I32, I32, P, P, I32, I32,
                                              I32, I32, P]),
                "ko_ms_window": (None, [P, I32, I32, I32, I32, I32, I32, I32, I32, P, P]),
                "ko_ab_kernel": (C.c_float, [C.c_float]),
                "ko_ab_window_check": (None, [P, P, P]),
                "ko_abmsod": (None, [P, I32, I32, I32, I32, I32, I32, I32, P, I64, P, P, I32, P,
                                     P, P, P, P, P, P, P]),
                "ko_abmsod_fixed": (None, [P, I32, I32, I32, I32, I32, I32, I32, P, I64, P, P,
                                           I32, P, P, P, P, P, P]),
                "ko_max_threads": (I32, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


_tables = {"n": -1, "T": None, "L": None}


def tables(nmax):
    """(T, L) with T[c] = c ln c and L[n] = ln n, correctly rounded, c,n <= nmax."""
    with _lock:
        if _tables["n"] < nmax:
            n = max(nmax, 1)
            T = np.empty(n + 1, np.float64)
            Lt = np.empty(n + 1, np.float64)
            _tables.update(n=n, T=T, L=Lt)
            build_needed = True
        else:
            build_needed = False
    if build_needed:
        lib().ko_tables(_tables["n"], _p(_tables["T"]), _p(_tables["L"]))
    return _tables["T"], _tables["L"]


def ball_size(r):
    """|Ball(r)| = number of integer offsets with |o|^2 <= r^2."""
    r = int(r)
    if r < 0:
        return 0
    d = np.arange(-r, r + 1)
    return int(((d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
                <= r * r).sum())


def bin_volume(vol, binning):
    """Stored-bin volume (uint8, b+1; 0 = not counted) for a raw volume."""
    vol = np.ascontiguousarray(vol)
    out = np.empty(vol.shape, np.uint8)
    kind = binning["kind"]
    if kind == BIN_AFFINE_F32:
        v = np.ascontiguousarray(vol, dtype=np.float32)
        lo = np.zeros(1, np.float32)
        hi = np.zeros(1, np.float32)
        lib().ko_bin_f32(_p(v), v.size, binning["bins"], _p(out), _p(lo), _p(hi))
        return out
    v = np.ascontiguousarray(vol, dtype=np.int32)
    lib().ko_bin_int(_p(v), v.size, kind, binning["bins"], binning["shift"],
                     binning["lo"], binning["hi"], _p(out))
    return out


def _dims(bins):
    nz, ny, nx = bins.shape
    return nx, ny, nz


def window_counts(bins, B, p, r):
    nx, ny, nz = _dims(bins)
    c = np.zeros(B, np.int64)
    lib().ko_window_counts(_p(np.ascontiguousarray(bins)), nx, ny, nz, B, int(p[0]), int(p[1]),
                           int(p[2]), int(r), _p(c))
    return c


def octant_counts(bins, B, p, r, j):
    nx, ny, nz = _dims(bins)
    c = np.zeros(B, np.int64)
    lib().ko_octant_counts(_p(np.ascontiguousarray(bins)), nx, ny, nz, B, int(p[0]), int(p[1]),
                           int(p[2]), int(r), int(j), _p(c))
    return c


def entropy(counts, nmax=None):
    c = np.ascontiguousarray(counts, dtype=np.int64)
    T, L = tables(max(int(c.sum()), int(c.max(initial=0)), 1) if nmax is None else nmax)
    return lib().ko_entropy(_p(c), c.size, _p(T), _p(L))


def weight(counts, prev_counts, r, w_norm=0):
    c = np.ascontiguousarray(counts, dtype=np.int64)
    cp = np.ascontiguousarray(prev_counts, dtype=np.int64)
    return lib().ko_weight(_p(c), _p(cp), c.size, int(r), int(w_norm))


def dense(bins, B, r_min, r_max, w_norm=0, centres=None, brute=False, nthreads=0,
          want_hw=False):
    """Dense Kadir-Brady: (Y_best, s_best[, H, W]) per centre.

    centres=None evaluates every voxel and returns arrays shaped like `bins`;
    otherwise `centres` is an (n, 3) int array of xyz and outputs are flat."""
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    nx, ny, nz = _dims(bins)
    S = r_max - r_min + 1
    T, L = tables(ball_size(r_max))
    if centres is None:
        n = bins.size
        cp = None
    else:
        cen = np.ascontiguousarray(centres, dtype=np.int32).reshape(-1, 3)
        n = cen.shape[0]
        cp = _p(cen)
    Y = np.zeros(n, np.float64)
    s = np.zeros(n, np.uint8)
    H = np.zeros((n, S), np.float64) if want_hw else None
    W = np.zeros((n, S), np.float64) if want_hw else None
    lib().ko_dense(_p(bins), nx, ny, nz, B, r_min, r_max, w_norm, _p(T), _p(L), cp, n,
                   int(brute), int(nthreads), _p(Y), _p(s),
                   _p(H) if want_hw else None, _p(W) if want_hw else None)
    if centres is None:
        Y = Y.reshape(bins.shape)
        s = s.reshape(bins.shape)
    return (Y, s, H, W) if want_hw else (Y, s)


def seed_grid(dims, stride):
    nx, ny, nz = dims
    n = lib().ko_seed_grid(nx, ny, nz, stride, None)
    out = np.zeros((n, 3), np.int32)
    lib().ko_seed_grid(nx, ny, nz, stride, _p(out))
    return out


def octant_climb(bins, B, r_min, r_max, seeds, max_iter=20, w_norm=0, nthreads=0,
                 want_traj=False, planar=False):
    """Octant climb (3D form of Alg. 1); planar=True: the quadrant climb of
    Alg. 1 as printed, with disk windows in each seed's z-slice."""
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    nx, ny, nz = _dims(bins)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32).reshape(-1, 3)
    n = seeds.shape[0]
    T, L = tables(ball_size(r_max))
    out = {
        "xyz": np.zeros((n, 3), np.int32), "iters": np.zeros(n, np.int32),
        "converged": np.zeros(n, np.int32), "Y": np.zeros(n), "s": np.zeros(n, np.int32),
        "H": np.zeros(n), "W": np.zeros(n),
    }
    traj = np.zeros((n, max_iter + 1, 3), np.int32) if want_traj else None
    fn = lib().ko_quadrant_climb if planar else lib().ko_octant_climb
    fn(_p(bins), nx, ny, nz, B, r_min, r_max, max_iter, w_norm, _p(T), _p(L),
                          _p(seeds), n, int(nthreads), _p(out["xyz"]), _p(out["iters"]),
                          _p(out["converged"]), _p(traj) if want_traj else None, _p(out["Y"]),
                          _p(out["s"]), _p(out["H"]), _p(out["W"]))
    if want_traj:
        out["traj"] = traj
    return out


def octant_one_step(bins, B, r_min, r_max, p, planar=False):
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    nx, ny, nz = _dims(bins)
    T, L = tables(ball_size(r_max))
    st = np.zeros(3, np.int32)
    lib().ko_octant_one_step(_p(bins), nx, ny, nz, B, r_min, r_max, _p(T), _p(L), int(p[0]),
                             int(p[1]), int(p[2]), int(planar), _p(st))
    return st


def meanshift(bins, B, r_min, r_max, seeds, max_iter=20, nthreads=0):
    """Items are (seed, r) seed-major: item = seed*S + (r - r_min)."""
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    nx, ny, nz = _dims(bins)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32).reshape(-1, 3)
    S = r_max - r_min + 1
    n = seeds.shape[0] * S
    T, L = tables(ball_size(r_max))
    out = {
        "xyz": np.zeros((n, 3), np.int32), "iters": np.zeros(n, np.int32),
        "converged": np.zeros(n, np.int32), "rho": np.zeros(n), "H": np.zeros(n),
    }
    lib().ko_meanshift(_p(bins), nx, ny, nz, B, r_min, r_max, max_iter, _p(T), _p(L), _p(seeds),
                       seeds.shape[0], int(nthreads), _p(out["xyz"]), _p(out["iters"]),
                       _p(out["converged"]), _p(out["rho"]), _p(out["H"]))
    return out


def ms_window(bins, B, p, r):
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    nx, ny, nz = _dims(bins)
    c = np.zeros(B, np.int64)
    m = np.zeros((B, 3), np.int64)
    lib().ko_ms_window(_p(bins), nx, ny, nz, B, int(p[0]), int(p[1]), int(p[2]), int(r), _p(c),
                       _p(m))
    return c, m


def max_threads():
    return lib().ko_max_threads()


# ----------------------------------------------------------------- selection
# Selection of salient regions among converged seeds (Sec. 2.3, end: maxima
# whose entropy is above a threshold are kept and ranked by the change of
# the pdf at their scale; Sec. 3.1: the 20 with the highest pdf difference).
# Candidates are records with fields x, y, z, r, source, H, W (r = 0: no
# scale).  Readings: "above" is strict (H > h_min); candidates with the same
# (x, y, z, r) are one region, represented by the smallest source; the order
# is W descending, then H descending, then z, y, x, r ascending.

def octant_candidates(res):
    """One candidate per octant seed result: the final centre with r = s,
    H and W of the Kadir-Brady evaluation there (`res` as octant_climb
    returns it); source = the seed's index."""
    xyz = np.asarray(res["xyz"])
    n = len(xyz)
    return [dict(x=int(xyz[i, 0]), y=int(xyz[i, 1]), z=int(xyz[i, 2]), r=int(res["s"][i]),
                 source=i, H=float(res["H"][i]), W=float(res["W"][i])) for i in range(n)]


def meanshift_candidates(bins, B, r_min, r_max, res, radii, w_norm=0):
    """One candidate per mean-shift item: its final centre and radius, with
    H(r) and W(r) of the dense definition evaluated there (`res` as
    meanshift returns it, `radii` the item radii); source = the item index."""
    xyz = np.asarray(res["xyz"], np.int32).reshape(-1, 3)
    _, _, H, W = dense(bins, B, r_min, r_max, w_norm=w_norm, centres=xyz, want_hw=True)
    out = []
    for i in range(len(xyz)):
        si = int(radii[i]) - r_min
        out.append(dict(x=int(xyz[i, 0]), y=int(xyz[i, 1]), z=int(xyz[i, 2]), r=int(radii[i]),
                        source=i, H=float(H[i, si]), W=float(W[i, si])))
    return out


def select_salient(cands, h_min=0.0, top_k=20):
    """The selection, step by step: threshold, merge, order, take top_k."""
    kept = [c for c in cands if c["r"] > 0 and c["H"] > h_min]
    regions = {}
    for c in kept:
        key = (c["x"], c["y"], c["z"], c["r"])
        if key not in regions or c["source"] < regions[key]["source"]:
            regions[key] = c
    ordered = sorted(regions.values(),
                     key=lambda c: (-c["W"], -c["H"], c["z"], c["y"], c["x"], c["r"]))
    return ordered[:top_k]


# -------------------------------------------------------------------- ABMSOD
def ab_kernel(d):
    """exp(-d/2) as the kernel's stated arithmetic evaluates it (binary32
    polynomial; ks_abmsod_fixed.c)."""
    return float(lib().ko_ab_kernel(float(d)))


def _ab_out(n):
    return {"x": np.zeros((n, 3)), "H": np.zeros((n, 6)), "rho": np.zeros(n),
            "iters": np.zeros(n, np.int32), "stopped": np.zeros(n, np.int32),
            "voxels": np.zeros(n, np.int64)}


def _ab_inputs(bins, r_min, r_max, seeds, cand):
    bins = np.ascontiguousarray(bins, dtype=np.uint8)
    if cand is None:
        seeds = np.ascontiguousarray(seeds, dtype=np.int32).reshape(-1, 3)
        return bins, seeds, seeds.shape[0], seeds.shape[0] * (r_max - r_min + 1), None, None
    cx = np.ascontiguousarray(cand[0], dtype=np.float64).reshape(-1, 3)
    cH = np.ascontiguousarray(cand[1], dtype=np.float64).reshape(-1, 6)
    assert cx.shape[0] == cH.shape[0]
    dummy = np.zeros((1, 3), np.int32)
    return bins, dummy, cx.shape[0], cx.shape[0], cx, cH


def abmsod(bins, B, r_min, r_max, seeds, max_iter=20, nthreads=0, cand=None):
    """Adaptive-bandwidth mean shift (Alg. 2, Eq. 6-7), the plain binary64
    statement, for every (seed, r) item (seed-major), or for given candidate
    ellipsoids cand = (x (n, 3), H (n, 6)): best centre x, its bandwidth H
    (00 01 02 11 12 22), best Bhattacharyya coefficient rho, iterations,
    whether the search stopped at a fall of rho, the window voxels of every
    kernel histogram evaluated, and the item's decision margins: edge
    (smallest |d - 1| of a counted box voxel) and rho_gap (smallest
    |rho' - best| of an iteration after the first; inf if none).  See
    ks_oracle.c."""
    bins, seeds, ns, n, cx, cH = _ab_inputs(bins, r_min, r_max, seeds, cand)
    nx, ny, nz = _dims(bins)
    out = _ab_out(n)
    out["edge"] = np.zeros(n)
    out["rho_gap"] = np.zeros(n)
    lib().ko_abmsod(_p(bins), nx, ny, nz, B, r_min, r_max, max_iter, _p(seeds), ns,
                    None if cx is None else _p(cx), None if cH is None else _p(cH),
                    int(nthreads), _p(out["x"]), _p(out["H"]), _p(out["rho"]), _p(out["iters"]),
                    _p(out["stopped"]), _p(out["voxels"]), _p(out["edge"]), _p(out["rho_gap"]))
    return out


def abmsod_fixed(bins, B, r_min, r_max, seeds, max_iter=20, nthreads=0, cand=None):
    """The same search in the kernel's stated arithmetic (binary32 window
    geometry, polynomial exp, fixed-point sums; ks_abmsod_fixed.c).  Not the
    oracle of record: a model of the kernel for a bit-exact regression
    check, bounded against abmsod() by the tolerance tests."""
    bins, seeds, ns, n, cx, cH = _ab_inputs(bins, r_min, r_max, seeds, cand)
    nx, ny, nz = _dims(bins)
    out = _ab_out(n)
    lib().ko_abmsod_fixed(_p(bins), nx, ny, nz, B, r_min, r_max, max_iter, _p(seeds), ns,
                          None if cx is None else _p(cx), None if cH is None else _p(cH),
                          int(nthreads), _p(out["x"]), _p(out["H"]), _p(out["rho"]),
                          _p(out["iters"]), _p(out["stopped"]), _p(out["voxels"]))
    return out


def ab_window_check(x, H):
    """Kernel arithmetic (ks_abmsod_fixed.c): (box voxels with 0 <= d <= 1,
    those inside their row's span) for the window (x, H) in a volume of
    counted voxels."""
    x = np.ascontiguousarray(x, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    out = np.zeros(2, np.int64)
    lib().ko_ab_window_check(_p(x), _p(H), _p(out))
    return int(out[0]), int(out[1])
