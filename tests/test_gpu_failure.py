"""Failure detection without a GPU fault.  A device wait given a deadline far below a bulk copy's
latency runs out: the scan sets its error word, still waits (bounded) for its own copies in flight,
and returns; the host reports FPS_ERR_TIMEOUT, resets the scan state, and the same library and stream
answer as before the failure (the answer itself is pinned to the oracle by the parity tests).

The library (20 M records, 480 MB) streams from HBM over ~70 tiles per warp, so some wait is still
pending once the deadline (1 ns after the kernel starts) has passed, whatever the timer's resolution."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_device_wait_timeout_is_reported_and_recovered(gpu_lib):
    fps = gpu_lib
    n, k = 20_000_000, 30
    lib = fps.fps_library_load(packed=synth.packed(n, 30))
    try:
        q = synth.packed(1, 1030)[0]
        before_i, before_d = fps.fps_search_packed(lib, q, k)
        assert len(before_i) == k
        # host form: the error comes back from the call
        with pytest.raises(fps.FpsError) as e:
            fps.fps_search_packed(lib, q, k, timeout_s=1e-9)
        assert e.value.status == fps.FPS_ERR_TIMEOUT
        # device form: the call only enqueues; the error comes back from fps_sync
        qd = torch.from_numpy(q.view(np.int64).copy()).cuda()
        fps.fps_search_packed(lib, qd, k, timeout_s=1e-9)
        with pytest.raises(fps.FpsError) as e:
            fps.fps_sync(lib)
        assert e.value.status == fps.FPS_ERR_TIMEOUT
        # the context, the library and the stream's workspace answer as before, in both forms
        gi, gd = fps.fps_search_packed(lib, q, k)
        assert np.array_equal(gi, before_i) and np.array_equal(gd, before_d)
        oi, od, oc = fps.fps_search_packed(lib, qd, k)
        fps.fps_sync(lib)
        assert int(oc.item()) == k
        assert np.array_equal(oi.cpu().numpy(), before_i) and np.array_equal(od.cpu().numpy(), before_d)
    finally:
        fps.fps_release(lib)


def test_tensor_core_wait_timeout_is_reported_and_recovered(gpu_lib):
    """The tensor-core batch: with a 1 ns bound every pipeline wait (copy landed, stage free,
    accumulator full or free, hand-off ring room) gives up at its first miss.  Each warp then
    stops issuing; the copy producer waits (at least 1 s) for its bulk copies in flight and the
    MMA thread for its MMAs before the CTA frees its TMEM.  The call reports FPS_ERR_TIMEOUT in
    both forms, and the same library and stream return the same results afterwards."""
    fps = gpu_lib
    n, Q = 5_000_000, 512
    lib = fps.fps_library_load(packed=synth.packed(n, 31), flags=fps.FPS_LOAD_TC_OPERAND)
    try:
        qs = synth.packed(Q, 1031)
        ks = synth.k_mix(Q, seed=31)
        bi, bd, bc, _ = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_TC_FP8, flat=True)
        assert np.array_equal(bc, np.minimum(ks, n))
        with pytest.raises(fps.FpsError) as e:
            fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_TC_FP8, timeout_s=1e-9)
        assert e.value.status == fps.FPS_ERR_TIMEOUT
        qd = torch.from_numpy(qs.view(np.int64).copy()).cuda()
        with pytest.raises(fps.FpsError) as e:
            fps.fps_search_batch(lib, qd, ks, path=fps.FPS_PATH_TC_FP8, timeout_s=1e-9)
            fps.fps_sync(lib)
        assert e.value.status == fps.FPS_ERR_TIMEOUT
        for _ in range(2):
            ai, ad, ac, _ = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_TC_FP8, flat=True)
            assert np.array_equal(ac, bc) and np.array_equal(ai, bi) and np.array_equal(ad, bd)
        oi, od, oc, off = fps.fps_search_batch(lib, qd, ks, path=fps.FPS_PATH_TC_FP8)
        fps.fps_sync(lib)
        assert np.array_equal(oc.cpu().numpy(), bc)
        assert np.array_equal(oi.cpu().numpy()[: off[-1]], bi[: off[-1]])
        assert np.array_equal(od.cpu().numpy()[: off[-1]], bd[: off[-1]])
    finally:
        fps.fps_release(lib)
