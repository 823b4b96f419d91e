"""The learned-threshold search path (FPS_PATH_LEARNED): exact whatever the predictor does.

A query whose predicted bound is below its true k-th distance has fewer than
k records under the bound and is re-run exactly; a bound far above simply
accepts more candidates.  The results must equal the oracle's in every case.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def qstrs(p):
    return synth.packed_to_strings(np.asarray(p).reshape(-1, 3))


def run_learned(fps, lib, qs, ks, tau):
    stats = fps.fps_search_stats()
    got = fps.fps_search_batch(lib, qs, ks, path=fps.FPS_PATH_LEARNED, tau=np.asarray(tau, np.float32), stats=stats)
    return got, stats


@pytest.mark.parametrize("tc", [False, True])
def test_learned_path_exact_with_bad_predictors(gpu_lib, tc):
    fps = gpu_lib
    n = 200000
    text = synth.text(n, 51)
    lib = fps.fps_library_load(text=text, flags=fps.FPS_LOAD_TC_OPERAND if tc else 0)
    try:
        qs = np.concatenate([synth.packed(150, 1051), synth.packed_at([7, 777], 51)])
        ks = np.array([[1, 10, 30, 100, 1000][i % 5] for i in range(len(qs))], np.int32)
        want = oracle.topk_many(text, qstrs(qs), ks)
        tk = np.array([w[1][-1] for w in want], np.float32)           # exact k-th distances (oracle)
        rng = np.random.default_rng(3)
        cases = {"zero": np.zeros(len(qs)), "max": np.full(len(qs), 166.0), "random": rng.uniform(0, 60, len(qs)),
                 "exact": tk, "one_below": tk - 1.0, "fractional": tk - 0.5}
        for name, tau in cases.items():
            got, st = run_learned(fps, lib, qs, ks, tau)
            for q, ((gi, gd), (wi, wd)) in enumerate(zip(got, want)):
                assert np.array_equal(gi, wi) and np.array_equal(gd, wd), (name, q)
            if name in ("exact", "fractional"):
                assert st.fallbacks == 0, name                         # ceil(T - 0.5) = T: enough records
            if name == "one_below":   # fewer than k records under T - 1 by definition (bounds clamp at 0)
                assert st.fallbacks == int(np.sum(tk > 0)), name
    finally:
        fps.fps_release(lib)


def test_trained_network_gains_over_sampled_bound(gpu_lib):
    """Train on exact labels of one library, then search another: fewer accepted candidates, same results."""
    fps = gpu_lib
    from paper_1906_06170_gb300 import learn
    from oracle import mlp as ref

    k = 30
    lib_train = fps.fps_library_load(packed=synth.packed(400000, 52), flags=fps.FPS_LOAD_TC_OPERAND)
    lib_eval = fps.fps_library_load(packed=synth.packed(400000, 53), flags=fps.FPS_LOAD_TC_OPERAND)
    m = fps.fps_mlp_create(0)
    try:
        qtr = torch.from_numpy(synth.packed(60000, 1052).view(np.int64).copy()).cuda()
        ttr = learn.exact_kth(lib_train, qtr, k)
        fps.fps_mlp_set_params(m, ref.init_params(21))
        learn.train(m, qtr, ttr, epochs=10, batch=2048, lr=2e-3, quantile=0.9)
        qcal = torch.from_numpy(synth.packed(4096, 1053).view(np.int64).copy()).cuda()
        offset = learn.calibrate_offset(m, qcal, learn.exact_kth(lib_eval, qcal, k), max_fallback=0.01)
        qe = synth.packed(2048, 1054)
        qed = torch.from_numpy(qe.view(np.int64).copy()).cuda()
        ks = np.full(len(qe), k, np.int32)
        s_pilot = fps.fps_search_stats()
        base = fps.fps_search_batch(lib_eval, qe, ks, path=fps.FPS_PATH_TC_FP8, stats=s_pilot)
        tau = learn.predict_tau(m, qed, offset).cpu().numpy()
        s_learn = fps.fps_search_stats()
        got = fps.fps_search_batch(lib_eval, qe, ks, path=fps.FPS_PATH_LEARNED, tau=tau, stats=s_learn)
        for (gi, gd), (bi, bd) in zip(got, base):
            assert np.array_equal(gi, bi) and np.array_equal(gd, bd)
        assert s_learn.fallbacks <= 0.05 * len(qe), s_learn.fallbacks
        assert s_learn.candidates < 0.8 * s_pilot.candidates, (s_learn.candidates, s_pilot.candidates)
    finally:
        fps.fps_mlp_release(m)
        fps.fps_release(lib_train)
        fps.fps_release(lib_eval)
