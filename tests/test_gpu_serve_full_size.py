"""The serving loop at the benchmarked sizes: three resident libraries of 1,000,000 / 20,000,000 /
95,417,114 generated records (seeds 10 / 11 / 12, with FP8 operands), Poisson arrivals at 5000 req/s
(seed 5), k from {10, 30, 100}, dynamic batches of up to 512 requests.  Every served result equals the
single-query scan's (exact at full size by tests/test_gpu_full_size.py); a sample of requests is checked
element by element against the plain PyTorch brute force, and each result's distances by the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from torch_brute import brute_topk

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SIZES = {"1M": (1_000_000, 10), "20M": (20_000_000, 11), "95M": (95_417_114, 12)}


def test_serving_full_size(gpu_lib):
    fps = gpu_lib
    from paper_1906_06170_gb300 import serve

    packed = {nm: synth.packed(n, s) for nm, (n, s) in SIZES.items()}
    libs = {nm: fps.fps_library_load(packed=p, flags=fps.FPS_LOAD_TC_OPERAND) for nm, p in packed.items()}
    try:
        nreq = 3000
        arr = serve.poisson_arrivals(nreq, 5000.0, seed=5)
        qs = synth.packed(nreq, 1004)
        names = list(SIZES)
        reqs = [serve.Request(float(t), names[synth.draw(5, i, 1) % 3], qs[i], [10, 30, 100][synth.draw(5, i, 2) % 3])
                for i, t in enumerate(arr)]
        srv = serve.Server(libs, has_tc={nm: True for nm in names}, max_batch=512)
        done = srv.run(reqs)
        assert len(done) == nreq and max(srv.batch_sizes) > 1          # dynamic batches were formed
        for r in done:
            wi, wd = fps.fps_search_packed(libs[r.lib], r.query, r.k)
            assert np.array_equal(r.result[0], wi) and np.array_equal(r.result[1], wd)
        # a sample of requests per library against the brute force and the oracle
        rng = np.random.default_rng(17)
        for nm in names:
            mine = [r for r in done if r.lib == nm]
            pick = [mine[i] for i in rng.choice(len(mine), size=min(8, len(mine)), replace=False)]
            raw = torch.from_numpy(packed[nm].view(np.uint8).reshape(-1, 24)).cuda()
            want = brute_topk(raw, np.stack([r.query for r in pick]), 100)
            del raw
            for r, w in zip(pick, want):
                gi, gd = r.result
                assert np.array_equal((gd.astype(np.int64) << 32) | gi, w[: r.k]), (nm, r.k)
                text = synth.strings_to_text(synth.packed_to_strings(packed[nm][gi]))
                assert np.array_equal(oracle.distances(text, synth.packed_to_strings(r.query.reshape(1, 3))[0]), gd)
    finally:
        for lib in libs.values():
            fps.fps_release(lib)
        torch.cuda.empty_cache()
