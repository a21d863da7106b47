"""ks_bin_f32_noalloc: float32 binning without any device allocation.

Some users of this library cannot let it call cudaMalloc: their framework's
caching allocator owns every byte of device memory, or their serving loop
must not take the device-wide synchronisation an allocation can cause, or
their memory budget is already fully spent.  For them the library offers
one entry point that works only in the caller's input and output buffers
plus a fixed scratch array compiled into the library.  This test calls it
through the C ABI several times in a row (the scratch keeps the previous
call's contents) and checks each output byte for byte against the
allocating path, ks_create_volume + ks_volume_bins, and checks that the
calls leave the device's free memory and the torch allocator untouched.
It lives in its own file, collected last, and passes alone in a fresh
process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_binning_matches_allocating_path():
    import torch

    from paper_1310_6736_b300 import build, ks, synth

    assert torch.cuda.is_available()
    build.build()
    lib = ks.lib()
    ctx = ks.Context()
    stream = torch.cuda.current_stream()
    binning = {"kind": ks.KS_BIN_AFFINE_F32, "bins": 32}
    cases = [
        (synth.workload("pet128").volume, 0),               # aligned rows: vector path
        (synth.pet_f32(seed=11, dims=(41, 33, 35))[0], 0),   # ragged rows
        (synth.pet_f32(seed=12)[0], 1),                      # output not 16-byte aligned
    ]
    for vol, shift in cases:
        nz, ny, nx = vol.shape
        n = vol.size
        d_in = torch.from_numpy(vol).cuda()
        d_buf = torch.full((n + 16,), 255, dtype=torch.uint8, device="cuda")
        out_ptr = d_buf.data_ptr() + shift
        st = lib.ks_bin_f32_noalloc(ctypes.c_void_p(d_in.data_ptr()), nx, ny, nz, 32,
                                    ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream.cuda_stream))
        assert st == ks.KS_OK
        torch.cuda.synchronize()
        got = d_buf[shift:shift + n].cpu().numpy().reshape(vol.shape)
        v = ctx.create_volume(vol, binning)
        ref = ctx.volume_bins(v, vol.shape)
        ctx.release_volume(v)
        assert np.array_equal(got, ref)
        assert got.min() >= 1 and got.max() <= 32
    # dims beyond the library's per-axis limit: refused before any launch
    st = lib.ks_bin_f32_noalloc(ctypes.c_void_p(d_in.data_ptr()), 4097, 4, 4, 32,
                                ctypes.c_void_p(d_buf.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
    assert st == ks.KS_EINVAL
    assert lib.ks_bin_f32_noalloc(None, 4, 4, 4, 32, ctypes.c_void_p(d_buf.data_ptr()),
                                  None) == ks.KS_EINVAL
    ctx.close()


def test_noalloc_binning_allocates_nothing():
    """After a first call, further calls leave the device's free memory and
    the torch allocator's counters unchanged, and give the same bytes."""
    import torch

    from paper_1310_6736_b300 import build, ks, synth

    assert torch.cuda.is_available()
    build.build()
    lib = ks.lib()
    stream = torch.cuda.current_stream()
    vol = synth.pet_f32(seed=13, dims=(96, 80, 72))[0]
    nz, ny, nx = vol.shape
    d_in = torch.from_numpy(vol).cuda()
    d_out = torch.zeros(vol.size, dtype=torch.uint8, device="cuda")

    def call():
        return lib.ks_bin_f32_noalloc(ctypes.c_void_p(d_in.data_ptr()), nx, ny, nz, 32,
                                      ctypes.c_void_p(d_out.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))

    assert call() == ks.KS_OK                  # first call: may load the module
    torch.cuda.synchronize()
    first = d_out.cpu()
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        assert call() == ks.KS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    allocs1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0
    assert allocs1 == allocs0
    assert torch.equal(d_out.cpu(), first)
