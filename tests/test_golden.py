"""The oracle against the hand-derived fixtures and the stored hashes under tests/golden/."""
import glob
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = oracle.UNREACHED


def parse_fixture(path):
    spec = {"edges": []}
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        if key == "edge":
            spec["edges"].append(tuple(int(v) for v in vals))
        elif key in ("n", "source", "sssp_sync_rounds", "bfs_sync_rounds"):
            spec[key] = int(vals[0])
        else:
            spec[key] = [INF if v == "INF" else int(v) for v in vals]
    e = np.array(spec["edges"], np.int64).reshape(-1, 3)
    spec["src"], spec["dst"], spec["w"] = e[:, 0], e[:, 1], e[:, 2]
    return spec


HAND = sorted(glob.glob(os.path.join(GOLDEN, "hand_*.txt")))


@pytest.mark.parametrize("path", HAND, ids=[os.path.basename(p) for p in HAND])
def test_hand_fixture(path):
    f = parse_fixture(path)
    n, s = f["n"], f["source"]
    rc, d = oracle.sssp(n, f["src"], f["dst"], f["w"], s)
    assert rc == oracle.OK and d.tolist() == f["sssp"]
    rc, lv = oracle.bfs(n, f["src"], f["dst"], s)
    assert rc == oracle.OK and lv.tolist() == f["bfs"]
    rc, lab = oracle.cc(n, f["src"], f["dst"])
    assert rc == oracle.OK and lab.tolist() == f["cc"]
    r, _ = oracle.jacobi_rounds(n, f["src"], f["dst"], f["w"], s)
    assert r == f["sssp_sync_rounds"]
    r, _ = oracle.jacobi_rounds(n, f["src"], f["dst"], f["w"], s, unit=True)
    assert r == f["bfs_sync_rounds"]


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_oracle_hashes():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    stored = json.load(open(os.path.join(GOLDEN, "oracle_hashes.json")))
    assert mg.oracle_hashes() == stored
