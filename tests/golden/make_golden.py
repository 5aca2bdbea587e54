"""Write the stored hashes under tests/golden/ (calls only graphgen and oracle).

    python tests/golden/make_golden.py

* graphgen_hashes.json -- SHA-256 of each named workload's (src, dst, w)
  arrays and of its seeded sources: pins the input recipe.
* oracle_hashes.json   -- SHA-256 of the oracle's outputs on small named
  workloads: any later change of the oracle's results shows up here.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


GEN_WORKLOADS = {
    "er-16384-131072": lambda: gg.er(),
    "rmat-12": lambda: gg.rmat(12),
    "rmat-22": lambda: gg.rmat(22),
    "grid-64": lambda: gg.grid(64),
    "grid-4096": lambda: gg.grid(4096),
}

ORACLE_WORKLOADS = {
    "er-16384-131072": lambda: gg.er(),
    "rmat-12": lambda: gg.rmat(12),
    "grid-64": lambda: gg.grid(64),
}


def gen_hashes():
    out = {}
    for name, make in GEN_WORKLOADS.items():
        g = make()
        out[name] = {"n": g.n, "m": g.m, "edges": sha(g.src, g.dst, g.w),
                     "sources8": sha(gg.sources(g, 8))}
    return out


def oracle_hashes():
    out = {}
    for name, make in ORACLE_WORKLOADS.items():
        g = make()
        srcs = [0] if name.startswith("er") else [int(s) for s in gg.sources(g, 2)]
        rec = {}
        for s in srcs:
            rc, d = oracle.sssp(g.n, g.src, g.dst, g.w, s)
            assert rc == oracle.OK
            rec[f"sssp/{s}"] = sha(d)
            rc, lv = oracle.bfs(g.n, g.src, g.dst, s)
            rec[f"bfs/{s}"] = sha(lv)
            r, _ = oracle.jacobi_rounds(g.n, g.src, g.dst, g.w, s)
            rec[f"sssp_sync_rounds/{s}"] = r
        rc, lab = oracle.cc(g.n, g.src, g.dst)
        rec["cc"] = sha(lab)
        out[name] = rec
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "graphgen_hashes.json"), "w") as f:
        json.dump(gen_hashes(), f, indent=1, sort_keys=True)
    with open(os.path.join(HERE, "oracle_hashes.json"), "w") as f:
        json.dump(oracle_hashes(), f, indent=1, sort_keys=True)
    print("written")
