"""Serving loop and failure handling on the GPU, without faulting it.

Failures are made on the host (bad requests, a budget too small, a
cancelled request, a poll that runs out of time) or by a device wait that
gives up after a bounded number of polls (ks_selftest_wait_timeout): the
kernel records the timeout in a status word that the host reads back, and
the context stays usable."""
import numpy as np
import pytest

import oracle_checks
from paper_1310_6736_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ks_mod():
    import torch
    assert torch.cuda.is_available()
    from paper_1310_6736_b300 import build, ks
    build.build()
    return ks


def _params(ks, w):
    return ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)


def test_bounded_device_wait_reports_timeout_and_context_survives(ks_mod):
    ks = ks_mod
    ctx = ks.Context()
    st = ks.lib().ks_selftest_wait_timeout(ctx.h, 1000)
    assert st == ks.KS_ETIMEDOUT
    assert ks.lib().ks_sync(ctx.h) == ks.KS_OK          # status was consumed
    w = synth.workload("spheres48")
    v = ctx.create_volume(w.volume, w.binning)           # the context still works
    out = ctx.seed_climb(v, _params(ks, w))
    assert len(out) == 512
    ctx.close()


def test_many_requests_match_plain_calls_and_oracle(ko, ks_mod):
    """Eight requests in flight at once: each result equals the plain call's
    and the oracle's (seed requests in full; dense sweeps of the int16
    volumes, r = 4..32, on 1500 sampled voxels and the corners)."""
    ks = ks_mod
    ctx = ks.Context()
    ws = synth.batch_volumes(seed=21, count=8, hi=72)
    ids = []
    for i, w in enumerate(ws):
        kind = ks.KS_REQ_DENSE if i % 4 == 3 else ks.KS_REQ_SEEDS
        ids.append((ctx.submit(w.volume, w.binning, _params(ks, w), kind=kind), kind, w))
    for rid, kind, w in ids:
        st, res = ctx.poll(rid, -1)
        assert st == ks.KS_OK
        assert res["t_submit_us"] <= res["t_admit_us"] <= res["t_done_us"]
        v = ctx.create_volume(w.volume, w.binning)
        p = _params(ks, w)
        if kind == ks.KS_REQ_DENSE:
            Y, s = ctx.dense_saliency(v, p, w.volume.shape)
            assert np.array_equal(res["Y"], Y.ravel()) and np.array_equal(res["s"], s.ravel())
            oracle_checks.dense_maps(ko, w, res["Y"], res["s"], sample=1500, seed=rid)
        else:
            assert np.array_equal(res["oct"], ctx.seed_climb(v, p))
            assert np.array_equal(res["ms"], ctx.meanshift(v, p))
            oracle_checks.octant_records(ko, w, res["oct"])
            oracle_checks.meanshift_records(ko, w, res["ms"])
        ctx.release_volume(v)
        assert ctx.release_result(rid) == ks.KS_OK
    ctx.close()


def test_poll_timeout_cancel_and_admission(ks_mod):
    ks = ks_mod
    # a small HBM budget: a request whose footprint exceeds it is refused
    ctx = ks.Context(hbm_budget_bytes=96 << 20)
    big = np.zeros((600, 600, 600), np.int16)
    with pytest.raises(ks.KsError) as e:
        ctx.submit(big, {"kind": 0, "bins": 64, "shift": 5, "lo": 0, "hi": 2047},
                   ks.make_params(4, 20, 12))
    assert e.value.status == ks.KS_ENOMEM
    vol, _ = synth.mr_i16(5, (100, 100, 100))
    b = {"kind": 0, "bins": 64, "shift": 5, "lo": 0, "hi": 2047}
    p = ks.make_params(4, 24, 10)
    first = ctx.submit(vol, b, p, kind=ks.KS_REQ_DENSE)
    queued = [ctx.submit(vol, b, p, kind=ks.KS_REQ_SEEDS) for _ in range(3)]
    st, _ = ctx.poll(queued[-1], 0)
    assert st in (ks.KS_PENDING, ks.KS_OK)
    assert ctx.cancel(queued[-1]) == ks.KS_OK
    st, res = ctx.poll(queued[-1], -1)
    assert st in (ks.KS_ECANCELED, ks.KS_OK)            # it may have finished first
    for rid in [first] + queued[:-1]:
        st, res = ctx.poll(rid, -1)
        assert st == ks.KS_OK
    # a poll that gives up: a fresh dense request polled for 1 microsecond
    rid = ctx.submit(vol, b, p, kind=ks.KS_REQ_DENSE)
    st, _ = ctx.poll(rid, 1)
    assert st in (ks.KS_ETIMEDOUT, ks.KS_OK)
    st, _ = ctx.poll(rid, -1)
    assert st == ks.KS_OK
    assert ctx.poll(987654, 0)[0] == ks.KS_ENOTFOUND
    with pytest.raises(ks.KsError):
        ctx.submit(vol, {"kind": 0, "bins": 64, "shift": 1, "lo": 0, "hi": 2047}, p)
    ctx.close()
