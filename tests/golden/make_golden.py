"""Write the seeded fixtures of tests/golden/ from the CPU oracle only.

topk_seed0_n20000.txt   166-bit top-30 (Fig. 3 steps 1-6)
wide_seed21_n3000.txt   1024-bit top-20, Manhattan and Tanimoto (the n-bit extension)
cluster_seed1400.txt    batch clustering of 120 queries, counts 2..6 (the batch clustering search)

Each file pins the seeded generator and the oracle together on one small
workload so that a run on another machine (another CPU architecture, another
libm) can check that it regenerates exactly the same inputs and results.
Expected values come from ``oracle`` alone, never from the CUDA path.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle import cluster  # noqa: E402

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
    write_wide()
    write_cluster()


WIDE_N, WIDE_BITS, WIDE_K, WIDE_SEED, WIDE_QSEED, WIDE_NQ = 3000, 1024, 20, 21, 1021, 2


def write_wide():
    text = synth.wide_text(WIDE_N, WIDE_BITS, WIDE_SEED)
    queries = synth.wide_to_strings(synth.wide_packed(WIDE_NQ, WIDE_BITS, WIDE_QSEED), WIDE_BITS)
    lines = [
        "# Exact top-20 of 1024-bit records by the CPU oracle: Manhattan (ascending d) and Tanimoto",
        "# (descending c / u, compared exactly); ties by ascending index.",
        f"# library: synth wide seed {WIDE_SEED}, N = {WIDE_N}; queries: synth wide seed {WIDE_QSEED}, first {WIDE_NQ}.",
        "# columns: metric (0 Manhattan, 1 Tanimoto) | query | rank | index | num | den",
    ]
    for metric in (oracle.MANHATTAN, oracle.TANIMOTO):
        for qi, q in enumerate(queries):
            idx, num, den = oracle.wide_topk(text, WIDE_BITS, q, WIDE_K, metric)
            for r, (i, a, b) in enumerate(zip(idx.tolist(), num.tolist(), den.tolist())):
                lines.append(f"{metric} {qi} {r} {i} {a} {b}")
    with open(os.path.join(HERE, "wide_seed21_n3000.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


CL_Q, CL_SEED, CL_CMIN, CL_CMAX = 120, 1400, 2, 6


def write_cluster():
    queries = synth.packed_to_strings(synth.packed(CL_Q, CL_SEED))
    res = cluster.cluster_batch(queries, CL_CMIN, CL_CMAX)
    lines = [
        "# Batch clustering by the CPU oracle: k-medoids per count, silhouette sum floor(s * 2^32),",
        "# the best count (ties: smaller), its medoids and labels.",
        f"# queries: synth seed {CL_SEED}, first {CL_Q}; counts {CL_CMIN}..{CL_CMAX}.",
        "# lines: 'score <c> <sum>', 'best <c>', 'medoids <i> ...', 'labels <l> ...'",
    ]
    for c in sorted(res["scores"]):
        lines.append(f"score {c} {res['scores'][c]}")
    lines.append(f"best {res['c']}")
    lines.append("medoids " + " ".join(str(int(m)) for m in res["medoids"]))
    lines.append("labels " + " ".join(str(int(v)) for v in res["labels"]))
    with open(os.path.join(HERE, "cluster_seed1400.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
