"""Write tests/golden/topk_seed0_n20000.txt from the CPU oracle only.

The file pins the seeded generator and the oracle together on one small
workload so that a run on another machine (another CPU architecture, another
libm) can check that it regenerates exactly the same library and results.
Expected values come from ``oracle`` alone, never from the CUDA path.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

N, K, QSEED, NQ = 20000, 30, 1001, 3


def main():
    text = synth.text(N, 0)
    queries = synth.packed_to_strings(synth.packed(NQ, QSEED))
    lines = [
        "# Exact top-30 by the CPU oracle (Fig. 3 steps 1-6, ties by ascending index).",
        f"# library: synth seed 0, chemistry seed 0, N = {N}; queries: synth seed {QSEED}, first {NQ}.",
        "# columns: query | rank | index | distance",
    ]
    for qi, q in enumerate(queries):
        idx, dist, _ = oracle.topk(text, q, K)
        for r, (i, d) in enumerate(zip(idx.tolist(), dist.tolist())):
            lines.append(f"{qi} {r} {i} {d}")
    with open(os.path.join(HERE, "topk_seed0_n20000.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
