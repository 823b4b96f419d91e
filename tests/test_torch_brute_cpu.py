"""The plain-PyTorch brute force used at the paper's library size, pinned to the oracle on the CPU."""
import numpy as np
import torch

import oracle
import synth
from torch_brute import brute_topk


def test_brute_force_equals_oracle():
    n, k = 30000, 40
    packed = synth.packed(n, 0)
    raw = torch.from_numpy(packed.view(np.uint8).reshape(n, 24))
    qs = np.concatenate([synth.packed(4, 1001), np.zeros((1, 3), np.uint64), synth.packed_at([77, n - 1], 0)])
    want = brute_topk(raw, qs, k, chunk=7001)       # chunks that do not divide n
    text = synth.text(n, 0)
    for i, q in enumerate(qs):
        wi, wd, _ = oracle.topk(text, synth.packed_to_strings(q.reshape(1, 3))[0], k)
        assert np.array_equal((wd.astype(np.int64) << 32) | wi, want[i]), i
