"""The bench's algorithmic-byte model on hand-made counters (host logic, no
GPU): each variant's bytes per query, written out term by term from the byte
model of the measurement design, so that a dropped or misplaced term in
bench.algorithmic_bytes fails here."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

INFO = {"n": 1000}


def stats(S=0, Va=0, Ea=0, U=0, P=0, jumps=0):
    return {"scanned": S, "vertices_processed": Va, "edges_relaxed": Ea, "updates": U, "pushes": P,
            "jump_passes": jumps}


def test_sync_modes():
    st = stats(S=500, Va=40, Ea=300, U=7)
    # SSSP: 4 per activity word, 16 per expanded vertex, 12 per edge, 12 per update
    assert bench.algorithmic_bytes(0, 0, st, INFO) == 4 * 500 + 16 * 40 + 12 * 300 + 12 * 7
    assert bench.algorithmic_bytes(0, 2, st, INFO) == 4 * 500 + 16 * 40 + 12 * 300 + 12 * 7
    # BFS: 8 per vertex, 8 per edge, 4 per update
    assert bench.algorithmic_bytes(1, 0, st, INFO) == 4 * 500 + 8 * 40 + 8 * 300 + 4 * 7
    # CC: 8 per edge, plus 8 bytes per vertex per pointer-jumping pass
    st_cc = stats(S=500, Va=40, Ea=300, U=7, jumps=3)
    assert bench.algorithmic_bytes(2, 2, st_cc, INFO) == 4 * 500 + 16 * 40 + 8 * 300 + 12 * 7 + 3 * 1000 * 8


def test_async_modes():
    st = stats(Va=40, Ea=300, U=7, P=5)
    # vertex-async SSSP: 16 per item, 12 per edge, 12 per update, 8 per push
    assert bench.algorithmic_bytes(0, 1, st, INFO) == 16 * 40 + 12 * 300 + 12 * 7 + 8 * 5
    # BFS items and claims are smaller
    assert bench.algorithmic_bytes(1, 1, st, INFO) == 12 * 40 + 8 * 300 + 8 * 7 + 8 * 5
    # edge-async: + 16 per item for the degree prefix ...
    assert bench.algorithmic_bytes(0, 3, st, INFO) == 32 * 40 + 12 * 300 + 12 * 7 + 8 * 5
    # ... and the edge sources its dense generations stream
    st_dense = stats(S=2000, Va=40, Ea=300, U=7, P=5)
    assert bench.algorithmic_bytes(0, 3, st_dense, INFO) == 4 * 2000 + 32 * 40 + 12 * 300 + 12 * 7 + 8 * 5
    # vertex-async ignores the scan counter (its dense generations read no edge sources)
    assert bench.algorithmic_bytes(0, 1, st_dense, INFO) == 16 * 40 + 12 * 300 + 12 * 7 + 8 * 5


def test_model_grows_with_every_counter():
    base = stats(S=10, Va=10, Ea=10, U=10, P=10, jumps=1)
    for algo, mode in [(0, 0), (0, 1), (0, 2), (0, 3), (1, 0), (1, 3), (2, 0), (2, 1)]:
        b0 = bench.algorithmic_bytes(algo, mode, base, INFO)
        for key in ("vertices_processed", "edges_relaxed", "updates"):
            more = dict(base)
            more[key] += 1
            assert bench.algorithmic_bytes(algo, mode, more, INFO) > b0, (algo, mode, key)


def rstats(R=0, Va=0, Ea=0, U=0, P=0, jumps=0):
    d = stats(Va=Va, Ea=Ea, U=U, P=P, jumps=jumps)
    d["rounds"] = R
    return d


def test_measurement_plan_formula_term_by_term():
    """roofline.frac uses the measurement plan's per-round formulas: V = n per
    round for the sync modes, 12 (vertex) or 20 (edge) bytes per relaxed SSSP
    edge, 4 per update; async 16 per processed vertex, 12 per edge, 4 per push
    and per update; 4 bytes less per edge without weights; CC + 8 n per jump."""
    st = rstats(R=5, Va=40, Ea=300, U=7, P=9)
    n = INFO["n"]
    assert bench.plan_bytes(0, 0, st, INFO) == 16 * n * 5 + 12 * 300 + 4 * 7
    assert bench.plan_bytes(0, 5, st, INFO) == 16 * n * 5 + 12 * 300 + 4 * 7
    assert bench.plan_bytes(0, 2, st, INFO) == 8 * n * 5 + 20 * 300 + 4 * 7
    assert bench.plan_bytes(1, 2, st, INFO) == 8 * n * 5 + 16 * 300 + 4 * 7
    for mode in (1, 3, 6):
        assert bench.plan_bytes(0, mode, st, INFO) == 16 * 40 + 12 * 300 + 4 * 9 + 4 * 7
        assert bench.plan_bytes(1, mode, st, INFO) == 16 * 40 + 8 * 300 + 4 * 9 + 4 * 7
    st_cc = rstats(R=5, Va=40, Ea=300, U=7, jumps=3)
    assert bench.plan_bytes(2, 0, st_cc, INFO) == 16 * n * 5 + 8 * 300 + 4 * 7 + 8 * n * 3


def test_measurement_plan_formula_matches_the_full_sweep_figures():
    """One all-active round on R-MAT 22 (n = 2^22, m = 16 n, every edge
    relaxed, no update): 872 MB vertex-sync, 1376 MB edge-sync, the
    headline figures of the measurement plan."""
    n, m = 1 << 22, 16 << 22
    st = rstats(R=1, Ea=m)
    assert abs(bench.plan_bytes(0, 0, st, {"n": n}) / 1e6 - 872.4) < 0.1
    assert abs(bench.plan_bytes(0, 2, st, {"n": n}) / 1e6 - 1375.7) < 0.1


def test_host_info_states_cores_and_model():
    h = bench.host_info()
    assert h["host_cores"] >= 1 and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_compact_serving_keeps_both_arms_per_rate():
    row = {"rate_per_s": 1000,
           "batched": {"p50_ms": 1.04, "p99_ms": 9.96, "completed_per_s": 870.0, "all_ok": True},
           "one_at_a_time": {"p50_ms": 2.0, "p99_ms": 20.0, "completed_per_s": 750.0, "all_ok": True}}
    c = bench.compact_serving({"resident_graphs": ["a", "b"], "resident_device_gb": 4.0,
                               "requests_per_rate": 2000, "rates": [row]})
    r = c["rates"]["1000"]
    assert r["qps"] == [870.0, 750.0] and r["p50"] == [1.0, 2.0] and r["p99"] == [10.0, 20.0] and r["ok"]


def test_cpu_baseline_legs_on_a_small_graph():
    """The CPU-baseline leg (host only): the oracle's single-thread figure with
    the host it ran on, and the multi-core OpenMP figure beside it, both in
    GTEPS of the same edge-counting convention; the OpenMP leg reports its
    thread count and sample, or why it is unavailable."""
    import numpy as np
    import graphgen as gg
    g = gg.rmat(12)
    srcs = gg.sources(g, 8)
    deg = np.bincount(g.src, minlength=g.n).astype(np.int64)
    out = bench.cpu_baseline_sample(g, srcs, deg, "rmat22")
    assert out["kind"] == "oracle" and out["cores"] == 1 and out["unit"] == "GTEPS"
    assert out["value"] > 0 and out["host_cores"] >= 1 and out["cpu_model"]
    omp = out["omp"]
    if "unavailable" not in omp:
        assert omp["value"] > 0 and omp["cores"] >= 1
        assert omp["sample"].startswith("1 build + 8 SSSP + 8 BFS + 1 CC")
