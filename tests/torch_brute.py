"""Exact top-k by brute force in plain PyTorch: an independent check of completeness for
libraries too large for the oracle.  Uses no kernel of this project.

d(q, x) = popc(q) + popc(x) - 2 q.x over the 192 bits of the packed records (bits past 166
are zero), as a 0/1 FP16 matrix product: every product is 0 or 1 and every sum an integer
<= 192, which FP16 represents exactly, so d is exact whatever the summation order.
"""
import numpy as np
import torch


def brute_topk(raw, q_rows, kmax, chunk=1 << 21):
    """k smallest keys (d << 32 | index) per query over the whole library, plain PyTorch."""
    dev = raw.device
    shifts = torch.arange(8, device=dev, dtype=torch.uint8)

    def bits(u8):
        return ((u8[:, :, None] >> shifts) & 1).reshape(u8.shape[0], -1).to(torch.float16)

    qb = bits(torch.from_numpy(np.ascontiguousarray(q_rows).view(np.uint8).reshape(-1, 24)).to(dev))
    pq = qb.float().sum(1)
    best = None
    for s in range(0, raw.shape[0], chunk):
        xb = bits(raw[s: s + chunk])
        px = xb.float().sum(1)
        d = (pq[:, None] + px[None, :] - 2.0 * (qb @ xb.T).float()).to(torch.int64)
        key = (d << 32) | torch.arange(s, s + xb.shape[0], device=dev, dtype=torch.int64)[None, :]
        top = torch.topk(key, min(kmax, key.shape[1]), dim=1, largest=False).values
        best = top if best is None else torch.topk(torch.cat([best, top], 1), min(kmax, best.shape[1] + top.shape[1]),
                                                   dim=1, largest=False).values
    return best.cpu().numpy()
