"""Python binding of the C ABI in include/ks.h (libks.so).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  There is no CPU fallback; a missing or unloadable library raises.
Host arrays are numpy; device arrays are torch CUDA tensors (torch is used
for device memory and streams only).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libks.so")

KS_OK, KS_PENDING, KS_EINVAL, KS_ENOMEM, KS_ECUDA, KS_ETIMEDOUT, KS_ECANCELED, \
    KS_ENOTFOUND, KS_ENODEV = 0, 1, -1, -2, -3, -4, -5, -6, -7
KS_U8, KS_I16, KS_F32 = 0, 1, 2
KS_BIN_CLAMP_SHIFT, KS_BIN_AFFINE_F32, KS_BIN_WINDOW, KS_BIN_STORED = 0, 1, 2, 3
KS_WNORM_KB, KS_WNORM_ONE = 0, 1
KS_REQ_SEEDS, KS_REQ_DENSE = 0, 1


class KsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ks_binning(C.Structure):
    _fields_ = [("kind", C.c_int32), ("bins", C.c_int32), ("shift", C.c_int32),
                ("lo", C.c_int32), ("hi", C.c_int32)]


class ks_params(C.Structure):
    _fields_ = [("r_min", C.c_int32), ("r_max", C.c_int32), ("stride", C.c_int32),
                ("max_iter", C.c_int32), ("w_norm", C.c_int32)]


class ks_request(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("nx", C.c_int32),
                ("ny", C.c_int32), ("nz", C.c_int32), ("binning", ks_binning),
                ("params", ks_params), ("kind", C.c_int32), ("seed_kinds", C.c_int32)]


class ks_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("n_seeds", C.c_int64),
                ("n_items", C.c_int64), ("n_voxels", C.c_int64), ("oct", C.c_void_p),
                ("ms", C.c_void_p), ("Y_best", C.c_void_p), ("s_best", C.c_void_p),
                ("t_submit_us", C.c_double), ("t_admit_us", C.c_double),
                ("t_done_us", C.c_double)]


SEED_RESULT = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("seed_x", "<i4"),
                        ("seed_y", "<i4"), ("seed_z", "<i4"), ("iters", "<i4"),
                        ("converged", "<i4"), ("s_best", "<i4"), ("reserved", "<i4"),
                        ("Y_best", "<f8"), ("H_best", "<f8"), ("W_best", "<f8")])
MS_RESULT = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("r", "<i4"), ("seed", "<i4"),
                      ("iters", "<i4"), ("converged", "<i4"), ("reserved", "<i4"),
                      ("rho", "<f8"), ("H", "<f8")])
CANDIDATE = np.dtype([("x", "<i4"), ("y", "<i4"), ("z", "<i4"), ("r", "<i4"),
                      ("source", "<i4"), ("reserved", "<i4"), ("H", "<f8"), ("W", "<f8")])
AB_RESULT = np.dtype([("x", "<f8", (3,)), ("H", "<f8", (6,)), ("rho", "<f8"), ("seed", "<i4"),
                      ("r", "<i4"), ("iters", "<i4"), ("stopped", "<i4"), ("voxels", "<i8")])
assert SEED_RESULT.itemsize == 64 and MS_RESULT.itemsize == 48 and CANDIDATE.itemsize == 40
assert AB_RESULT.itemsize == 104

# Every symbol include/ks.h declares, with (restype, argtypes).
_P, _I, _I64, _D, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
_PP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "ks_init": (_I, [_PP, _SZ, _P, _I]),
    "ks_destroy": (_I, [_P]),
    "ks_strerror": (C.c_char_p, [_I]),
    "ks_last_error": (C.c_char_p, [_P]),
    "ks_sync": (_I, [_P]),
    "ks_create_volume": (_I, [_P, _P, _I, _I, _I, _I, _I, C.POINTER(ks_binning),
                              C.POINTER(C.c_int64)]),
    "ks_release_volume": (_I, [_P, _I64]),
    "ks_volume_bins": (_I, [_P, _I64, _P, _I]),
    "ks_dense_saliency": (_I, [_P, _I64, C.POINTER(ks_params), _P, _P, _I]),
    "ks_dense_saliency_ex": (_I, [_P, _I64, C.POINTER(ks_params), _P, _P, _P, _P, _I]),
    "ks_dense_saliency_range": (_I, [_P, _I64, C.POINTER(ks_params), _I, _I, _P, _P, _I]),
    "ks_seed_count": (_I, [_P, _I64, C.POINTER(ks_params), C.POINTER(C.c_int64)]),
    "ks_seed_climb": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _I64,
                           C.POINTER(C.c_int64), _P, _I]),
    "ks_quadrant_climb": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _I64,
                               C.POINTER(C.c_int64), _P, _I]),
    "ks_meanshift": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _I64,
                          C.POINTER(C.c_int64), _I]),
    "ks_abmsod": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _I64,
                       C.POINTER(C.c_int64), _I]),
    "ks_abmsod_candidates": (_I, [_P, _I64, _P, _P, _I64, _I, _P, _I]),
    "ks_saliency": (_I, [_P, _I64, C.POINTER(ks_params), _P, _P, _P, _I64, C.POINTER(C.c_int64),
                         _P, _I64, C.POINTER(C.c_int64), _I]),
    "ks_dense_points": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _P, _P, _P, _I]),
    "ks_octant_candidates": (_I, [_P, _P, _I64, _P, _I]),
    "ks_meanshift_candidates": (_I, [_P, _I64, C.POINTER(ks_params), _P, _I64, _P, _I]),
    "ks_select_salient": (_I, [_P, _P, _I64, _D, _I, _P, C.POINTER(C.c_int64), _I]),
    "ks_batch_seeds": (_I, [_P, _P, _P, _I, _I, _P, _P, _I]),
    "ks_submit": (_I, [_P, C.POINTER(ks_request), C.POINTER(C.c_int64)]),
    "ks_poll": (_I, [_P, _I64, _I64, C.POINTER(ks_result)]),
    "ks_cancel": (_I, [_P, _I64]),
    "ks_release_result": (_I, [_P, _I64]),
    "ks_set_serve_wave_iters": (_I, [_P, _I]),
    "ks_tables": (_I, [_P, _I64, _P, _P]),
    "ks_launch_count": (_I64, [_P]),
    "ks_set_profiling": (_I, [_P, _I]),
    "ks_kernel_time": (_I, [_P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "ks_measure_smem_peak": (_I, [_P, C.POINTER(C.c_double)]),
    "ks_measure_smem_red_rate": (_I, [_P, C.POINTER(C.c_double)]),
    "ks_measure_fp64_rate": (_I, [_P, C.POINTER(C.c_double)]),
    "ks_dense_config": (_I, [_P, _I, _I, C.POINTER(C.c_int), C.POINTER(C.c_int),
                             C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ks_force_dense_config": (_I, [_I, _I, _I, _I]),
    "ks_set_abmsod_team_radius": (_I, [_I]),
    "ks_bin_f32_noalloc": (_I, [_P, _I, _I, _I, _I, _P, _P]),
    "ks_selftest_wait_timeout": (_I, [_P, _I]),
}

_lib = None


def lib():
    """Load libks.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; run paper_1310_6736_b300.build first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dtype_code(a):
    dt = np.dtype(str(a.dtype).replace("torch.", ""))
    if dt == np.uint8:
        return KS_U8
    if dt == np.int16:
        return KS_I16
    if dt == np.float32:
        return KS_F32
    raise TypeError(f"unsupported volume dtype {a.dtype}")


def _is_torch_cuda(a):
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def make_binning(b):
    if isinstance(b, ks_binning):
        return b
    return ks_binning(int(b["kind"]), int(b["bins"]), int(b.get("shift", 0)),
                      int(b.get("lo", 0)), int(b.get("hi", 0)))


def make_params(r_min, r_max, stride=8, max_iter=20, w_norm=KS_WNORM_KB):
    return ks_params(int(r_min), int(r_max), int(stride), int(max_iter), int(w_norm))


class Context:
    """One ks_ctx: a device, a stream (torch's current stream by default)."""

    def __init__(self, hbm_budget_bytes=0, stream=None, device=0, use_torch_stream=True):
        if stream is None and use_torch_stream:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = C.c_void_p()
        st = lib().ks_init(C.byref(h), int(hbm_budget_bytes), C.c_void_p(stream or 0),
                           int(device))
        if st != KS_OK:
            raise KsError(st, f"ks_init: {lib().ks_strerror(st).decode()}")
        self.h = h

    # ------------------------------------------------------------ plumbing
    def _check(self, st, what):
        if st != KS_OK:
            msg = lib().ks_last_error(self.h).decode(errors="replace")
            raise KsError(st, f"{what}: {msg or lib().ks_strerror(st).decode()}")
        return st

    def close(self):
        if getattr(self, "h", None):
            lib().ks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        return self._check(lib().ks_sync(self.h), "ks_sync")

    # ------------------------------------------------------------- volumes
    def create_volume(self, vol, binning):
        """vol: (nz, ny, nx) numpy array or torch CUDA tensor (uint8 / int16 / float32)."""
        nz, ny, nx = vol.shape
        dev = _is_torch_cuda(vol)
        if dev:
            vol = vol.contiguous()
            ptr = vol.data_ptr()
        else:
            vol = np.ascontiguousarray(vol)
            ptr = vol.ctypes.data
        out = C.c_int64()
        b = make_binning(binning)
        self._check(lib().ks_create_volume(self.h, C.c_void_p(ptr), int(dev), _dtype_code(vol),
                                           nx, ny, nz, C.byref(b), C.byref(out)),
                    "ks_create_volume")
        self._keep = vol   # keep the source alive until the call returned
        return out.value

    def release_volume(self, v):
        return self._check(lib().ks_release_volume(self.h, int(v)), "ks_release_volume")

    def volume_bins(self, v, shape):
        out = np.empty(shape, np.uint8)
        self._check(lib().ks_volume_bins(self.h, int(v), C.c_void_p(out.ctypes.data), 0),
                    "ks_volume_bins")
        return out

    # ------------------------------------------------------------ hot path
    def dense_saliency(self, v, params, shape, want_hw=False, out=None, host_out=None):
        """Dense sweep.  out=None: host numpy outputs, written into host_out =
        (Y, s) when given (caller-owned, e.g. pinned, C-contiguous float64 and
        uint8 arrays of the volume's shape).  out=(Y, s) torch CUDA tensors:
        results stay on the device."""
        nz, ny, nx = shape
        S = params.r_max - params.r_min + 1
        if out is not None:
            Y, s = out
            self._check(lib().ks_dense_saliency(self.h, int(v), C.byref(params),
                                                C.c_void_p(Y.data_ptr()), C.c_void_p(s.data_ptr()),
                                                1), "ks_dense_saliency")
            return Y, s
        if host_out is not None:
            Y, s = host_out
            if (Y.shape != tuple(shape) or s.shape != tuple(shape) or Y.dtype != np.float64
                    or s.dtype != np.uint8 or not Y.flags.c_contiguous
                    or not s.flags.c_contiguous):
                raise ValueError("host_out: C-contiguous float64 and uint8 arrays of the volume's shape")
        else:
            Y = np.empty(shape, np.float64)
            s = np.empty(shape, np.uint8)
        H = np.empty((nz * ny * nx, S), np.float64) if want_hw else None
        W = np.empty((nz * ny * nx, S), np.float64) if want_hw else None
        self._check(lib().ks_dense_saliency_ex(
            self.h, int(v), C.byref(params), C.c_void_p(Y.ctypes.data), C.c_void_p(s.ctypes.data),
            C.c_void_p(H.ctypes.data) if want_hw else None,
            C.c_void_p(W.ctypes.data) if want_hw else None, 0), "ks_dense_saliency")
        return (Y, s, H, W) if want_hw else (Y, s)

    def dense_saliency_range(self, v, params, shape, z0, z1):
        """Dense sweep for the centres of planes [z0, z1): host (Y, s) of
        shape (z1 - z0, ny, nx), equal to the whole sweep's planes."""
        nz, ny, nx = shape
        Y = np.empty((z1 - z0, ny, nx), np.float64)
        s = np.empty((z1 - z0, ny, nx), np.uint8)
        self._check(lib().ks_dense_saliency_range(self.h, int(v), C.byref(params), int(z0),
                                                  int(z1), C.c_void_p(Y.ctypes.data),
                                                  C.c_void_p(s.ctypes.data), 0),
                    "ks_dense_saliency_range")
        return Y, s

    def seed_count(self, v, params):
        n = C.c_int64()
        self._check(lib().ks_seed_count(self.h, int(v), C.byref(params), C.byref(n)),
                    "ks_seed_count")
        return n.value

    def _seeds_arg(self, seeds):
        if seeds is None:
            return None, 0, None
        s = np.ascontiguousarray(seeds, dtype=np.int32).reshape(-1, 3)
        return C.c_void_p(s.ctypes.data), s.shape[0], s

    @staticmethod
    def _host_records(host_out, n, dtype):
        """A caller-owned record array of at least n entries, or a new one."""
        if host_out is None:
            return np.zeros(max(n, 1), dtype)
        if host_out.dtype != dtype or not host_out.flags.c_contiguous or len(host_out) < max(n, 1):
            raise ValueError(f"host_out: a C-contiguous array of at least {n} {dtype} records")
        return host_out

    def seed_climb(self, v, params, seeds=None, want_traj=False, out=None, planar=False,
                   host_out=None):
        """Octant climb (planar=True: the quadrant climb of Alg. 1 as printed,
        disks in each seed's z-slice).  out=None: host SEED_RESULT array (and
        trajectories when want_traj), written into host_out when given.  out=a CUDA tensor of at least n * 64
        bytes: the records stay on the device; returns their count n."""
        fn, name = ((lib().ks_quadrant_climb, "ks_quadrant_climb") if planar else
                    (lib().ks_seed_climb, "ks_seed_climb"))
        sp, ns, keep = self._seeds_arg(seeds)
        n = ns if seeds is not None else self.seed_count(v, params)
        if out is not None:
            if want_traj:
                raise ValueError("trajectories are returned with host outputs only")
            return self._seeds_to_device(fn, name, v, params, sp, ns,
                                         out, n * SEED_RESULT.itemsize, SEED_RESULT.itemsize,
                                         extra=(None,))
        out = self._host_records(host_out, n, SEED_RESULT)
        traj = np.zeros((max(n, 1), params.max_iter + 1, 3), np.int32) if want_traj else None
        got = C.c_int64()
        self._check(fn(self.h, int(v), C.byref(params), sp, ns,
                       C.c_void_p(out.ctypes.data), out.shape[0], C.byref(got),
                       C.c_void_p(traj.ctypes.data) if want_traj else None, 0), name)
        out = out[:got.value]
        return (out, traj[:got.value]) if want_traj else out

    def meanshift(self, v, params, seeds=None, out=None, host_out=None):
        """Mean shift for every (seed, r).  out=None: host MS_RESULT array
        (written into host_out when given).
        out=a CUDA tensor of at least n * S * 48 bytes: the records stay on
        the device; returns their count n * S."""
        sp, ns, keep = self._seeds_arg(seeds)
        n = ns if seeds is not None else self.seed_count(v, params)
        S = params.r_max - params.r_min + 1
        if out is not None:
            return self._seeds_to_device(lib().ks_meanshift, "ks_meanshift", v, params, sp, ns,
                                         out, n * S * MS_RESULT.itemsize, MS_RESULT.itemsize)
        out = self._host_records(host_out, n * S, MS_RESULT)
        got = C.c_int64()
        self._check(lib().ks_meanshift(self.h, int(v), C.byref(params), sp, ns,
                                       C.c_void_p(out.ctypes.data), out.shape[0], C.byref(got), 0),
                    "ks_meanshift")
        return out[:got.value]

    def abmsod(self, v, params, seeds=None, out=None):
        """Adaptive-bandwidth mean shift for every (seed, r).  out=None: host
        AB_RESULT array.  out=a CUDA tensor of at least n * S * 104 bytes: the
        records stay on the device; returns their count n * S."""
        sp, ns, keep = self._seeds_arg(seeds)
        n = ns if seeds is not None else self.seed_count(v, params)
        S = params.r_max - params.r_min + 1
        if out is not None:
            return self._seeds_to_device(lib().ks_abmsod, "ks_abmsod", v, params, sp, ns,
                                         out, n * S * AB_RESULT.itemsize, AB_RESULT.itemsize)
        out = np.zeros(max(n * S, 1), AB_RESULT)
        got = C.c_int64()
        self._check(lib().ks_abmsod(self.h, int(v), C.byref(params), sp, ns,
                                    C.c_void_p(out.ctypes.data), out.shape[0], C.byref(got), 0),
                    "ks_abmsod")
        return out[:got.value]

    def abmsod_candidates(self, v, x, H, max_iter=20):
        """Adaptive-bandwidth mean shift from given candidate ellipsoids:
        x (n, 3) centres and H (n, 6) bandwidths (00 01 02 11 12 22), as
        numpy arrays (host AB_RESULT records returned) or CUDA float64
        tensors (returns a CUDA uint8 tensor of n records)."""
        if _is_torch_cuda(x):
            import torch
            n = x.shape[0]
            assert x.dtype == torch.float64 and H.dtype == torch.float64
            assert x.is_contiguous() and H.is_contiguous() and H.shape[0] == n
            out = torch.empty(max(n, 1) * AB_RESULT.itemsize, dtype=torch.uint8, device=x.device)
            self._check(lib().ks_abmsod_candidates(self.h, int(v), C.c_void_p(x.data_ptr()),
                                                   C.c_void_p(H.data_ptr()), n, int(max_iter),
                                                   C.c_void_p(out.data_ptr()), 1),
                        "ks_abmsod_candidates")
            return out[:n * AB_RESULT.itemsize]
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        H = np.ascontiguousarray(H, np.float64).reshape(-1, 6)
        if H.shape[0] != x.shape[0]:
            raise ValueError("x and H must list the same number of candidates")
        n = x.shape[0]
        out = np.zeros(max(n, 1), AB_RESULT)
        self._check(lib().ks_abmsod_candidates(self.h, int(v), C.c_void_p(x.ctypes.data),
                                               C.c_void_p(H.ctypes.data), n, int(max_iter),
                                               C.c_void_p(out.ctypes.data), 0),
                    "ks_abmsod_candidates")
        return out[:n]

    def _seeds_to_device(self, fn, name, v, params, sp, ns, out, need, rec, extra=()):
        if not out.is_cuda or out.numel() * out.element_size() < need:
            raise ValueError(f"{name}: out must be a CUDA tensor of at least {need} bytes")
        got = C.c_int64()
        cap = out.numel() * out.element_size() // rec
        self._check(fn(self.h, int(v), C.byref(params), sp, ns, C.c_void_p(out.data_ptr()), cap,
                       C.byref(got), *extra, 1), name)
        return got.value

    def saliency(self, v, params, shape, out=None, host_out=None):
        """Dense sweep, octant climb and mean shift of one volume in one call
        (the dense sweep on a high-priority stream, the seed searches beside
        it on a low-priority one; results equal the three separate calls).
        out=(Y, s, oct, ms) torch CUDA tensors (oct and ms as bytes): results
        stay on the device; returns the record counts.  Otherwise host
        outputs, written into host_out=(Y, s, oct, ms) when given; returns
        (Y, s, SEED_RESULT array, MS_RESULT array)."""
        nz, ny, nx = shape
        n = self.seed_count(v, params)
        S = params.r_max - params.r_min + 1
        n_oct, n_ms = C.c_int64(), C.c_int64()
        if out is not None:
            Y, s, o, m = out
            need = [(Y, nx * ny * nz * 8), (s, nx * ny * nz), (o, n * SEED_RESULT.itemsize),
                    (m, n * S * MS_RESULT.itemsize)]
            if any(not t.is_cuda or t.numel() * t.element_size() < b for t, b in need):
                raise ValueError("saliency: out must be CUDA tensors large enough for every result")
            self._check(lib().ks_saliency(
                self.h, int(v), C.byref(params), C.c_void_p(Y.data_ptr()), C.c_void_p(s.data_ptr()),
                C.c_void_p(o.data_ptr()), o.numel() * o.element_size() // SEED_RESULT.itemsize,
                C.byref(n_oct), C.c_void_p(m.data_ptr()),
                m.numel() * m.element_size() // MS_RESULT.itemsize, C.byref(n_ms), 1), "ks_saliency")
            return n_oct.value, n_ms.value
        if host_out is not None:
            Y, s, o, m = host_out
            if (Y.shape != tuple(shape) or s.shape != tuple(shape) or Y.dtype != np.float64
                    or s.dtype != np.uint8 or not Y.flags.c_contiguous
                    or not s.flags.c_contiguous):
                raise ValueError("host_out: C-contiguous float64 and uint8 arrays of the volume's shape")
        else:
            Y, s, o, m = np.empty(shape, np.float64), np.empty(shape, np.uint8), None, None
        o = self._host_records(o, n, SEED_RESULT)
        m = self._host_records(m, n * S, MS_RESULT)
        self._check(lib().ks_saliency(
            self.h, int(v), C.byref(params), C.c_void_p(Y.ctypes.data), C.c_void_p(s.ctypes.data),
            C.c_void_p(o.ctypes.data), len(o), C.byref(n_oct), C.c_void_p(m.ctypes.data), len(m),
            C.byref(n_ms), 0), "ks_saliency")
        return Y, s, o[:n_oct.value], m[:n_ms.value]

    def dense_points(self, v, params, xyz, want_hw=False):
        """Kadir-Brady at listed centres ((n, 3) int xyz): (Y_best, s_best[, H, W])."""
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        n = xyz.shape[0]
        S = params.r_max - params.r_min + 1
        Y = np.zeros(n, np.float64)
        s = np.zeros(n, np.uint8)
        H = np.zeros((n, S), np.float64) if want_hw else None
        W = np.zeros((n, S), np.float64) if want_hw else None
        self._check(lib().ks_dense_points(
            self.h, int(v), C.byref(params), C.c_void_p(xyz.ctypes.data), n,
            C.c_void_p(Y.ctypes.data), C.c_void_p(s.ctypes.data),
            C.c_void_p(H.ctypes.data) if want_hw else None,
            C.c_void_p(W.ctypes.data) if want_hw else None, 0), "ks_dense_points")
        return (Y, s, H, W) if want_hw else (Y, s)

    def octant_candidates(self, res):
        res = np.ascontiguousarray(res, dtype=SEED_RESULT)
        out = np.zeros(max(len(res), 1), CANDIDATE)
        self._check(lib().ks_octant_candidates(self.h, C.c_void_p(res.ctypes.data), len(res),
                                               C.c_void_p(out.ctypes.data), 0),
                    "ks_octant_candidates")
        return out[:len(res)]

    def meanshift_candidates(self, v, params, res):
        res = np.ascontiguousarray(res, dtype=MS_RESULT)
        out = np.zeros(max(len(res), 1), CANDIDATE)
        self._check(lib().ks_meanshift_candidates(self.h, int(v), C.byref(params),
                                                  C.c_void_p(res.ctypes.data), len(res),
                                                  C.c_void_p(out.ctypes.data), 0),
                    "ks_meanshift_candidates")
        return out[:len(res)]

    def select_salient(self, cands, h_min=0.0, top_k=20):
        cands = np.ascontiguousarray(cands, dtype=CANDIDATE)
        out = np.zeros(top_k, CANDIDATE)
        got = C.c_int64()
        self._check(lib().ks_select_salient(self.h, C.c_void_p(cands.ctypes.data), len(cands),
                                            float(h_min), int(top_k), C.c_void_p(out.ctypes.data),
                                            C.byref(got), 0), "ks_select_salient")
        return out[:got.value]

    def batch_seeds(self, vols, params, kinds=3, use_graph=True):
        n = len(vols)
        hv = (C.c_int64 * n)(*[int(v) for v in vols])
        hp = (ks_params * n)(*params)
        octs, mss = [], []
        for v, p in zip(vols, params):
            ns = self.seed_count(v, p)
            S = p.r_max - p.r_min + 1
            octs.append(np.zeros(max(ns, 1), SEED_RESULT)[:ns] if kinds & 1 else None)
            mss.append(np.zeros(max(ns * S, 1), MS_RESULT)[:ns * S] if kinds & 2 else None)
        po = (C.c_void_p * n)(*[a.ctypes.data if a is not None and a.size else None for a in octs])
        pm = (C.c_void_p * n)(*[a.ctypes.data if a is not None and a.size else None for a in mss])
        self._check(lib().ks_batch_seeds(self.h, hv, hp, n, int(kinds), po, pm, int(use_graph)),
                    "ks_batch_seeds")
        return octs, mss

    # ------------------------------------------------------------- serving
    def submit(self, vol, binning, params, kind=KS_REQ_SEEDS, seed_kinds=3):
        vol = np.ascontiguousarray(vol)
        nz, ny, nx = vol.shape
        r = ks_request(C.c_void_p(vol.ctypes.data), _dtype_code(vol), nx, ny, nz,
                       make_binning(binning), params, int(kind), int(seed_kinds))
        out = C.c_int64()
        self._check(lib().ks_submit(self.h, C.byref(r), C.byref(out)), "ks_submit")
        return out.value

    def poll(self, req, timeout_us=-1):
        """Returns (status, result dict or None).  Arrays are copied out."""
        res = ks_result()
        st = lib().ks_poll(self.h, int(req), int(timeout_us), C.byref(res))
        if st in (KS_PENDING, KS_ETIMEDOUT, KS_ENOTFOUND):
            return st, None
        d = {"status": res.status, "kind": res.kind, "t_submit_us": res.t_submit_us,
             "t_admit_us": res.t_admit_us, "t_done_us": res.t_done_us}
        if res.oct:
            d["oct"] = np.frombuffer((C.c_char * (res.n_seeds * 64)).from_address(res.oct),
                                     SEED_RESULT).copy()
        if res.ms:
            d["ms"] = np.frombuffer((C.c_char * (res.n_items * 48)).from_address(res.ms),
                                    MS_RESULT).copy()
        if res.Y_best:
            d["Y"] = np.frombuffer((C.c_char * (res.n_voxels * 8)).from_address(res.Y_best),
                                   np.float64).copy()
            d["s"] = np.frombuffer((C.c_char * res.n_voxels).from_address(res.s_best),
                                   np.uint8).copy()
        return st, d

    def cancel(self, req):
        return lib().ks_cancel(self.h, int(req))

    def set_serve_wave_iters(self, iters):
        """Iterations per seed item and serving wave (0 = whole searches)."""
        self._check(lib().ks_set_serve_wave_iters(self.h, int(iters)), "ks_set_serve_wave_iters")

    def release_result(self, req):
        return lib().ks_release_result(self.h, int(req))

    # --------------------------------------------------------- diagnostics
    def tables(self, nmax):
        T = np.empty(nmax + 1, np.float64)
        L = np.empty(nmax + 1, np.float64)
        self._check(lib().ks_tables(self.h, int(nmax), C.c_void_p(T.ctypes.data),
                                    C.c_void_p(L.ctypes.data)), "ks_tables")
        return T, L

    def launch_count(self):
        return lib().ks_launch_count(self.h)

    def set_profiling(self, on):
        return self._check(lib().ks_set_profiling(self.h, int(on)), "ks_set_profiling")

    def kernel_time(self, prefix):
        ms, n = C.c_double(), C.c_int64()
        self._check(lib().ks_kernel_time(self.h, prefix.encode(), C.byref(ms), C.byref(n)),
                    "ks_kernel_time")
        return ms.value, n.value

    def measure_smem_peak(self):
        r = C.c_double()
        self._check(lib().ks_measure_smem_peak(self.h, C.byref(r)), "ks_measure_smem_peak")
        return r.value

    def measure_smem_red_rate(self):
        """Shared-memory reductions per second with nothing else issued."""
        r = C.c_double()
        self._check(lib().ks_measure_smem_red_rate(self.h, C.byref(r)), "ks_measure_smem_red_rate")
        return r.value

    def measure_fp64_rate(self):
        """FP64 additions (lane operations) per second of this device."""
        r = C.c_double()
        self._check(lib().ks_measure_fp64_rate(self.h, C.byref(r)), "ks_measure_fp64_rate")
        return r.value

    def dense_config(self, bins, r_max):
        vals = [C.c_int() for _ in range(4)]
        st = lib().ks_dense_config(self.h, int(bins), int(r_max), *[C.byref(v) for v in vals])
        return None if st != KS_OK else tuple(v.value for v in vals)


def set_abmsod_team_radius(r_team):
    """Items with starting radius >= r_team run on a whole block (0: default)."""
    st = lib().ks_set_abmsod_team_radius(int(r_team))
    if st:
        raise KsError(st, "ks_set_abmsod_team_radius")


def force_dense_config(path, warps=0, ty=0, tz=0):
    st = lib().ks_force_dense_config(int(path), int(warps), int(ty), int(tz))
    if st != KS_OK:
        raise KsError(st, "ks_force_dense_config")
