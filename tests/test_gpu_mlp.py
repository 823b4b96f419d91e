"""GPU MLP kernels against the CPU reference (oracle/mlp.py).

Parameters and data are generated on the host (seeded) and given to both
sides.  Tolerances follow from the arithmetic: both sides use the same
bf16-rounded weights and layer inputs; the GPU accumulates in FP32 and the
reference in FP64, which can flip a bf16 rounding of an activation, so
gradients are compared per tensor by relative L2 error (<= 2e-2) and cosine
similarity (>= 0.999).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def dev_batch(n, seed):
    q = synth.packed(n, seed)
    return q, torch.from_numpy(q.view(np.int64).copy()).cuda()


def per_tensor(g):
    out, i = {}, 0
    for name, shape in ref.SHAPES:
        k = int(np.prod(shape))
        out[name] = g[i: i + k]
        i += k
    return out


def test_gradients_match_reference(gpu_lib):
    fps = gpu_lib
    flat = ref.init_params(11)
    m = fps.fps_mlp_create(0)
    try:
        fps.fps_mlp_set_params(m, flat)
        q, qd = dev_batch(1024, 2001)
        t = np.random.default_rng(5).uniform(5, 40, 1024).astype(np.float32)
        loss_g, g_gpu = fps.fps_mlp_grad(m, qd, torch.from_numpy(t).cuda(), 0.9)
        loss_c, g_cpu, _ = ref.loss_and_grad(flat.astype(np.float64), q, t.astype(np.float64), 0.9)
        assert abs(loss_g - loss_c) <= 1e-3 * max(1.0, abs(loss_c))
        G, C = per_tensor(g_gpu.astype(np.float64)), per_tensor(g_cpu)
        for name, _ in ref.SHAPES:
            a, b = G[name], C[name]
            nb = np.linalg.norm(b)
            if nb == 0:
                assert np.linalg.norm(a) < 1e-6
                continue
            rel = np.linalg.norm(a - b) / nb
            cos = float(a @ b / (np.linalg.norm(a) * nb))
            assert rel <= 2e-2 and cos >= 0.999, (name, rel, cos)
    finally:
        fps.fps_mlp_release(m)


def test_forward_matches_reference(gpu_lib):
    fps = gpu_lib
    flat = ref.init_params(12)
    m = fps.fps_mlp_create(0)
    try:
        fps.fps_mlp_set_params(m, flat)
        q, qd = dev_batch(2000, 2002)
        y = fps.fps_mlp_predict(m, qd).cpu().numpy()[:2000]
        yc, _ = ref.forward(ref.unflatten(flat.astype(np.float64)), ref.features(q))
        assert np.all(np.abs(y - yc) <= 0.05 + 1e-2 * np.abs(yc)), np.max(np.abs(y - yc))
        assert np.array_equal(fps.fps_mlp_get_params(m), flat)
    finally:
        fps.fps_mlp_release(m)


def test_adam_step_matches_reference(gpu_lib):
    fps = gpu_lib
    flat = ref.init_params(13)
    m = fps.fps_mlp_create(0)
    try:
        fps.fps_mlp_set_params(m, flat)
        q, qd = dev_batch(512, 2003)
        t = np.random.default_rng(6).uniform(5, 40, 512).astype(np.float32)
        lr = 1e-3
        fps.fps_mlp_train_step(m, qd, torch.from_numpy(t).cuda(), 0.9, lr)
        p_gpu = fps.fps_mlp_get_params(m)
        _, g_cpu, _ = ref.loss_and_grad(flat.astype(np.float64), q, t.astype(np.float64), 0.9)
        p_cpu, _, _ = ref.adam(flat, g_cpu, np.zeros_like(flat), np.zeros_like(flat), step=1, lr=lr)
        close = np.abs(p_gpu - p_cpu) <= 1e-6 + 0.05 * lr
        assert close.mean() >= 0.99, close.mean()           # first Adam step ~ lr * sign(g)
        assert np.abs(p_gpu - flat).max() <= 1.01 * lr + 1e-7
    finally:
        fps.fps_mlp_release(m)


def test_training_reduces_loss_on_a_learnable_target(gpu_lib):
    fps = gpu_lib
    from paper_1906_06170_gb300 import learn

    m = fps.fps_mlp_create(0)
    try:
        fps.fps_mlp_set_params(m, ref.init_params(14))
        q, qd = dev_batch(32768, 2004)
        bits = np.unpackbits(q.view(np.uint8), axis=1, bitorder="little")[:, :166].astype(np.float32)
        t = 0.5 * bits.sum(1) + 3.0 * bits[:, 10] + 2.0                 # a function of the bits, computed on the host
        td = torch.from_numpy(t).cuda()
        l0, _ = fps.fps_mlp_grad(m, qd, td, 0.5)
        hist = learn.train(m, qd, td, epochs=6, batch=1024, lr=2e-3, quantile=0.5)
        l1, _ = fps.fps_mlp_grad(m, qd, td, 0.5)
        assert l1 < 0.2 * l0, (l0, l1, hist)
    finally:
        fps.fps_mlp_release(m)
