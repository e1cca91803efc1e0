"""Writes random_pairs_n100_digest.json from the CPU oracle (only oracle/ is called).

The n=100 random-pairs workload (100,000 random H/S/CNOT gates and 20 RZ gates,
seed 1, eps = 1e-14 pruning after every one-qubit operator) is propagated in
plan mode by the oracle.  Its full result is too large to store, so the
digest keeps, per generator: the term count, the SHA-256 of the sorted list of
its strings, the sum of squared weights, the pruned squared weight, the
number of strings within a factor 10 of eps (where a rounding tie could
decide pruning), and every 50th term's exact weight (hex float).

Run: python tests/golden/make_random_pairs_digest.py  (about 7 minutes on 8 cores)
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2505_03307_gb300 import workloads as W  # noqa: E402

EPS = 1e-14
SAMPLE_EVERY = 50


def main():
    n, instrs = W.random_pairs(1)
    res = O.propagate(n, instrs, mode="plan", eps=EPS, threads=os.cpu_count() or 1)
    gens = []
    for g in res:
        strings = g["strings"]  # base-4 order already
        h = hashlib.sha256("\n".join(strings).encode()).hexdigest()
        w = g["re"]
        near = int(sum(1 for v in w if abs(v) < 10 * EPS))
        sample = [[strings[i], float(w[i]).hex()] for i in range(0, len(strings), SAMPLE_EVERY)]
        gens.append({"nterms": len(strings), "sha256": h, "sumsq": float((w * w).sum()),
                     "pruned_sumsq": float(g["pruned_sumsq"]), "near_eps": near,
                     "sample": sample})
    out = {"workload": "random_pairs_n100", "seed": 1, "eps": EPS, "mode": "plan",
           "generators": gens}
    with open(os.path.join(HERE, "random_pairs_n100_digest.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
