"""Write the stored exact histograms under tests/golden/ by running the CPU oracle.

Every stored value comes from ``oracle/`` alone (the CUDA path is never
imported here). Each file records the SHA-256 of the generated input so a
test can tell a generator drift from a counting mismatch.

    python tests/golden/make_golden.py [--threads N] [names...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2209_10241_gb300 import synth  # noqa: E402

CASES = {
    # name: (workload, seed, scale, orders)
    "uniform-200": ("uniform-200", 0, 1.0, (3, 4)),
    "f2f-330": ("f2f-330", 0, 1.0, (3, 4)),
    "coauth-1m-s001": ("coauth-1m", 0, 0.01, (3, 4)),
    "coauth-1m-s005": ("coauth-1m", 0, 0.05, (3, 4)),
    "comm-5m-s001": ("comm-5m", 0, 0.01, (3, 4)),
}

# Stub-shuffled null models (Sec. 6.3) of the smallest null-batch base:
# name: (base hyperedges, base seed, shuffle seed, model index, orders). Model
# t of a batch with shuffle seed s is oracle.stub_shuffle(base, seed=s,
# model=t), normalised and counted like any input.
NULL_CASES = {
    "null-50k-m0": (50_000, 100, 1, 0, (3, 4)),
    "null-50k-m1": (50_000, 100, 1, 1, (3, 4)),
}


def input_digest(h) -> str:
    d = hashlib.sha256()
    d.update(h.members.astype("<i4").tobytes())
    d.update(h.offsets.astype("<i8").tobytes())
    d.update(str(h.num_nodes).encode())
    return d.hexdigest()


def make(name: str, threads: int) -> dict:
    if name in NULL_CASES:
        H, base_seed, null_seed, model, orders = NULL_CASES[name]
        h = synth.null_base(H, seed=base_seed)
        shuffled = oracle.stub_shuffle(h.members, h.offsets, seed=null_seed, model=model)
        g = oracle.Graph(shuffled, h.offsets, h.num_nodes, 4)
        head = {"case": name, "workload": "null_base", "base_hyperedges": H,
                "base_seed": base_seed, "null_seed": null_seed, "model": model}
    else:
        wl, seed, scale, orders = CASES[name]
        h = synth.workload(wl, seed=seed, scale=scale)
        g = oracle.Graph.from_hypergraph(h, 4)
        head = {"case": name, "workload": wl, "seed": seed, "scale": scale}
    rec = {
        **head,
        "num_nodes": h.num_nodes, "num_hyperedges": h.num_hyperedges,
        "input_sha256": input_digest(h),
        "distinct_per_size": {str(s): g.count(s) for s in (2, 3, 4)},
        "larger_than_4": g.count(5),
        "hist": {},
        "oracle_seconds": {},
    }
    for k in orders:
        t = time.time()
        hist, cand = g.census(k, threads=threads)
        rec["hist"][str(k)] = [int(x) for x in hist]
        rec["oracle_seconds"][str(k)] = round(time.time() - t, 2)
        rec.setdefault("esu_candidates", {})[str(k)] = cand
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("names", nargs="*", default=list(CASES) + list(NULL_CASES))
    a = ap.parse_args()
    for name in a.names:
        rec = make(name, a.threads)
        path = os.path.join(HERE, f"census_{name}.json")
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)
        print(name, rec["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main()
