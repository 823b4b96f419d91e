"""n-bit fingerprints and the Tanimoto measure on the GPU (fps_wide_*) against oracle.wide_topk."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def lines(rows):
    return ("\n".join(rows) + "\n").encode() if rows else b""


def check(fps, lib, text, n_bits, queries, ks, metric):
    for q, k in zip(queries, ks):
        qs = synth.wide_to_strings(q, n_bits)[0]
        wi, wn, wd = oracle.wide_topk(text, n_bits, qs, int(k), metric)
        gi, gn, gd = fps.fps_wide_search(lib, q, int(k), metric)
        assert gi.tolist() == wi.tolist(), (n_bits, metric, k, gi[:6], wi[:6])
        assert gn.tolist() == wn.tolist() and gd.tolist() == wd.tolist(), (n_bits, metric, k)


@pytest.mark.parametrize("n_bits,n", [(64, 1), (64, 129), (166, 20000), (300, 50003), (1024, 70001), (2048, 9000)])
@pytest.mark.parametrize("metric", [0, 1])
def test_wide_matches_oracle(gpu_lib, n_bits, n, metric):
    fps = gpu_lib
    packed = synth.wide_packed(n, n_bits, 90 + n_bits)
    packed[n // 3] = 0                                          # empty records: Tanimoto 0/0 with an empty query
    text = lines(synth.wide_to_strings(packed, n_bits))
    lib = fps.fps_wide_load(text=text, n_bits=n_bits)
    try:
        W = synth.wide_words(n_bits)
        ones = np.zeros((1, W), np.uint64)
        for j in range(n_bits):
            ones[0, j // 64] |= np.uint64(1) << np.uint64(j % 64)
        qs = np.concatenate([synth.wide_packed(4, n_bits, 7000 + n_bits), packed[[0, n - 1]],
                             np.zeros((1, W), np.uint64), ones])
        ks = [1, 30, 128, 129, 1000, 1920, 30, 10][: len(qs)]
        check(fps, lib, text, n_bits, qs, ks, metric)
    finally:
        fps.fps_wide_release(lib)


@pytest.mark.parametrize("metric", [0, 1])
def test_wide_ties_and_device_form(gpu_lib, metric):
    fps = gpu_lib
    n_bits = 512
    base = synth.wide_packed(30000, n_bits, 95)
    dup = np.repeat(base[5:6], 20000, axis=0)                  # 20,000 equal records: ties broken by index
    packed = np.concatenate([base[:12000], dup, base[12000:]])
    text = lines(synth.wide_to_strings(packed, n_bits))
    lib = fps.fps_wide_load(packed=packed, n_bits=n_bits)
    try:
        q = base[5]
        for k in (1, 300, 1920):
            qs = synth.wide_to_strings(q, n_bits)[0]
            wi, wn, wd = oracle.wide_topk(text, n_bits, qs, k, metric)
            qd = torch.from_numpy(q.view(np.int64).copy()).cuda()
            oi, on, od, oc = fps.fps_wide_search(lib, qd, k, metric)
            torch.cuda.synchronize()
            c = int(oc.item())
            assert c == len(wi)
            assert oi[:c].cpu().tolist() == wi.tolist()
            assert on[:c].cpu().tolist() == wn.tolist() and od[:c].cpu().tolist() == wd.tolist()
    finally:
        fps.fps_wide_release(lib)


def test_wide_manhattan_at_166_bits_equals_the_main_path(gpu_lib):
    fps = gpu_lib
    packed = synth.packed(200000, 96)                           # 3 words, bits past 166 zero: the same records
    main = fps.fps_library_load(packed=packed)
    wide = fps.fps_wide_load(packed=packed, n_bits=166)
    try:
        qs = synth.packed(12, 1096)
        ks = synth.k_mix(12, seed=3)
        got = fps.fps_search_batch(main, qs, ks, path=fps.FPS_PATH_POPC)
        for q, k, (mi, md) in zip(qs, ks, got):
            wi, wn, wd = fps.fps_wide_search(wide, q, int(k), fps.FPS_METRIC_MANHATTAN)
            assert wi.tolist() == mi.tolist() and wn.tolist() == md.tolist() and set(wd.tolist()) <= {1}
    finally:
        fps.fps_release(main)
        fps.fps_wide_release(wide)


def test_wide_argument_errors(gpu_lib):
    fps = gpu_lib
    for nb in (0, 2049):
        with pytest.raises(fps.FpsError) as e:
            fps.fps_wide_load(packed=np.zeros((2, 33), np.uint64), n_bits=nb)
        assert e.value.status == fps.FPS_ERR_INVALID_ARG
    bad = np.zeros((3, 2), np.uint64)
    bad[1, 1] = np.uint64(1) << np.uint64(40)                   # bit 104 of a 100-bit record
    with pytest.raises(fps.FpsError) as e:
        fps.fps_wide_load(packed=bad, n_bits=100)
    assert e.value.status == fps.FPS_ERR_INVALID_ARG
    rows = synth.wide_to_strings(synth.wide_packed(5, 100, 1), 100)
    with pytest.raises(fps.FpsError) as e:
        fps.fps_wide_load(text=lines(rows[:3] + [rows[3] + "0"] + rows[4:]), n_bits=100)
    assert e.value.status == fps.FPS_ERR_PARSE and e.value.line == 4
    lib = fps.fps_wide_load(text=lines(rows), n_bits=100)
    try:
        with pytest.raises(fps.FpsError) as e:
            fps.fps_wide_search(lib, synth.wide_packed(1, 100, 2)[0], fps.FPS_K_MAX + 1)
        assert e.value.status == fps.FPS_ERR_UNSUPPORTED
        gi, gn, gd = fps.fps_wide_search(lib, synth.wide_packed(1, 100, 2)[0], 0)
        assert len(gi) == 0
        gi, gn, gd = fps.fps_wide_search(lib, synth.wide_packed(1, 100, 2)[0], 50)
        assert len(gi) == 5
    finally:
        fps.fps_wide_release(lib)
