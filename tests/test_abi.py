"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/ks.h declares, and its structs match the binding's layouts.
No compute call is made here (no GPU on the build host)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1310_6736_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ks.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|int64_t|const char \*)\s*\**\s*(ks_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libks():
    path = build.build()
    from paper_1310_6736_b300 import ks
    return ks, C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ks_init", "ks_destroy", "ks_create_volume", "ks_dense_saliency",
                 "ks_seed_climb", "ks_meanshift", "ks_submit", "ks_poll", "ks_cancel",
                 "ks_batch_seeds", "ks_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(libks):
    ks, L = libks
    for name in _declared():
        assert hasattr(L, name), name
        assert name in ks.SIGNATURES, f"binding lacks {name}"
    ks.lib()   # the binding loads and types every symbol


def test_struct_layouts_match_binding(tmp_path):
    from paper_1310_6736_b300 import ks
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ks.h"\nint main(){'
                    'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ks_seed_result),'
                    'sizeof(ks_ms_result), sizeof(ks_request), sizeof(ks_result),'
                    'offsetof(ks_seed_result, Y_best), offsetof(ks_ms_result, rho),'
                    'offsetof(ks_request, kind), sizeof(ks_candidate),'
                    'offsetof(ks_candidate, H), sizeof(ks_abmsod_result),'
                    'offsetof(ks_abmsod_result, rho), offsetof(ks_abmsod_result, voxels));}')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)],
                   check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    assert got == [ks.SEED_RESULT.itemsize, ks.MS_RESULT.itemsize, C.sizeof(ks.ks_request),
                   C.sizeof(ks.ks_result), ks.SEED_RESULT.fields["Y_best"][1],
                   ks.MS_RESULT.fields["rho"][1], ks.ks_request.kind.offset,
                   ks.CANDIDATE.itemsize, ks.CANDIDATE.fields["H"][1],
                   ks.AB_RESULT.itemsize, ks.AB_RESULT.fields["rho"][1],
                   ks.AB_RESULT.fields["voxels"][1]]


def test_error_strings_and_no_device_path(libks):
    ks, L = libks
    lib = ks.lib()
    assert lib.ks_strerror(ks.KS_EINVAL) == b"invalid argument"
    assert lib.ks_strerror(12345) == b"unknown status"
    assert lib.ks_destroy(None) == ks.KS_OK
    assert lib.ks_force_dense_config(0, 3, 2, 2) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(5, 8, 4, 2) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(4, 4, 2, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(4, 16, 4, 4) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(3, 16, 4, 4) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(3, 4, 2, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(2, 16, 4, 4) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(2, 8, 4, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(6, 8, 4, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(6, 2, 2, 1) == ks.KS_EINVAL   # not whole warpgroups
    assert lib.ks_force_dense_config(6, 12, 4, 3) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(7, 4, 2, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(7, 16, 4, 4) == ks.KS_EINVAL  # two centres per lane: <= 8 warps
    assert lib.ks_force_dense_config(8, 4, 2, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(8, 16, 4, 4) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(9, 4, 2, 2) == ks.KS_OK
    assert lib.ks_force_dense_config(9, 16, 4, 4) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(10, 4, 2, 2) == ks.KS_EINVAL
    assert lib.ks_force_dense_config(-1, 0, 0, 0) == ks.KS_OK
    import torch
    if not torch.cuda.is_available():
        h = C.c_void_p()
        assert lib.ks_init(C.byref(h), 0, None, 0) == ks.KS_ENODEV


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_1310_6736_b300 import ks
    monkeypatch.setattr(ks, "_lib", None)
    monkeypatch.setattr(ks, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        ks.lib()


def test_host_record_arrays_are_checked():
    """host_out= takes a caller-owned record array (e.g. in pinned memory):
    the right dtype, C-contiguous, and room for every record."""
    from paper_1310_6736_b300 import ks
    ok = np.zeros(5, ks.SEED_RESULT)
    assert ks.Context._host_records(ok, 5, ks.SEED_RESULT) is ok
    assert len(ks.Context._host_records(None, 3, ks.MS_RESULT)) == 3
    with pytest.raises(ValueError):
        ks.Context._host_records(np.zeros(4, ks.SEED_RESULT), 5, ks.SEED_RESULT)
    with pytest.raises(ValueError):
        ks.Context._host_records(np.zeros(5, ks.MS_RESULT), 5, ks.SEED_RESULT)
    with pytest.raises(ValueError):
        ks.Context._host_records(np.zeros(10, ks.SEED_RESULT)[::2], 5, ks.SEED_RESULT)
