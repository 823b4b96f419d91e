"""The allocation-free single-query search against the regular one.

fps_search_noalloc serves callers that cannot allocate device memory while
searching (their device memory is owned by another allocator, or an
allocation's synchronisation would break their latency budget, or they search
on many short-lived streams).  It keeps its scratch in a fixed array inside the
library.  Its results must equal fps_search_packed's exactly (integer outputs),
call after call, since consecutive calls reuse that array.  This file is named
to be collected last.
"""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_search_on_consecutive_calls(gpu_lib):
    fps = gpu_lib
    n = 300_000
    lib = fps.fps_library_load(packed=synth.packed(n, 21))
    try:
        qs = torch.from_numpy(synth.packed(4, 1021).view(np.int64).copy()).cuda()
        for k in (30, 1, 128):
            for j in (0, 1, 1, 2):                   # two different queries in a row, then a repeat
                want_i, want_d, want_c = fps.fps_search_packed(lib, qs[j], k)
                oi = torch.full((k,), -7, dtype=torch.int32, device="cuda")
                od = torch.full((k,), -7, dtype=torch.int32, device="cuda")
                oc = torch.full((1,), -7, dtype=torch.int32, device="cuda")
                fps.fps_search_noalloc(lib, qs[j], k, oi, od, oc)
                torch.cuda.synchronize()
                fps.fps_sync(lib)
                c = int(want_c.item())
                assert int(oc.item()) == c == min(k, n)
                assert torch.equal(oi[:c], want_i[:c]) and torch.equal(od[:c], want_d[:c])
        with pytest.raises(fps.FpsError) as e:
            fps.fps_search_noalloc(lib, qs[0], fps.FPS_NOALLOC_K_MAX + 1, oi, od, oc)
        assert e.value.status == fps.FPS_ERR_UNSUPPORTED
    finally:
        fps.fps_release(lib)
