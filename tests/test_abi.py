"""The C ABI without a GPU: the library loads, exports every function that
include/fg.h declares, the binding's struct layouts match a C compiler's, and
host-side argument checks fail before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1903_01665_gb300 as fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fg_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fg_graph_create_csr", "fg_graph_create_coo", "fg_graph_destroy", "fg_sssp",
                     "fg_bfs", "fg_cc", "fg_select_mode", "fg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = fg.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", fg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fg_[a-z_]+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "fg.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("fg_options %zu\nfg_stats %zu\nfg_graph_info_t %zu\n", sizeof(fg_options), sizeof(fg_stats), sizeof(fg_graph_info_t));
  P(fg_options, stream); P(fg_options, max_rounds); P(fg_options, wait_timeout_ms);
  P(fg_options, blocks_per_sm); P(fg_options, inject_missing_arrival); P(fg_options, round_trace);
  P(fg_options, round_trace_cap); P(fg_options, delta); P(fg_stats, barriers);
  P(fg_stats, mode); P(fg_stats, rounds); P(fg_stats, jump_passes); P(fg_stats, grid_blocks);
  P(fg_stats, vertices_processed); P(fg_stats, edges_relaxed); P(fg_stats, updates);
  P(fg_stats, pushes); P(fg_stats, scanned); P(fg_stats, kernel_ms);
  P(fg_stats, pull_rounds); P(fg_stats, edges_pulled);
  P(fg_graph_info_t, n); P(fg_graph_info_t, m); P(fg_graph_info_t, m_sym);
  P(fg_graph_info_t, max_out_degree); P(fg_graph_info_t, n_zero_out); P(fg_graph_info_t, n_low);
  P(fg_graph_info_t, n_mid); P(fg_graph_info_t, n_high); P(fg_graph_info_t, n_high_chunks);
  P(fg_graph_info_t, n_isolated);
  P(fg_graph_info_t, device_bytes); P(fg_graph_info_t, relabelled); P(fg_graph_info_t, in_degree_gini);
  printf("fg_query %zu\nfg_batch_options %zu\nfg_batch_stats %zu\n", sizeof(fg_query), sizeof(fg_batch_options), sizeof(fg_batch_stats));
  P(fg_query, g); P(fg_query, algo); P(fg_query, src); P(fg_query, out); P(fg_query, mode);
  P(fg_batch_options, stream); P(fg_batch_options, use_cuda_graph); P(fg_batch_options, wait_timeout_ms);
  P(fg_batch_options, fuse_same_graph);
  P(fg_batch_stats, kernel_ms); P(fg_batch_stats, launches); P(fg_batch_stats, teams); P(fg_batch_stats, ctas);
  printf("fg_server_options %zu\nfg_completion %zu\n", sizeof(fg_server_options), sizeof(fg_completion));
  P(fg_server_options, hbm_budget_bytes); P(fg_server_options, max_inflight); P(fg_server_options, max_wave);
  P(fg_server_options, one_at_a_time); P(fg_server_options, wait_timeout_ms); P(fg_server_options, exclusive_edges);
  P(fg_server_options, no_fusion);
  P(fg_completion, ticket); P(fg_completion, status); P(fg_completion, wave_size); P(fg_completion, latency_ms);
  printf("fg_plan %zu\n", sizeof(fg_plan));
  P(fg_plan, mode); P(fg_plan, blocks_per_sm); P(fg_plan, delta); P(fg_plan, tuned); P(fg_plan, depth_est);
  P(fg_plan, degree_gini);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    c = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        k, v = line.split()
        c[k] = int(v)
    for cls in (fg.fg_options, fg.fg_stats, fg.fg_graph_info_t, fg.fg_query, fg.fg_batch_options,
                fg.fg_batch_stats, fg.fg_server_options, fg.fg_completion, fg.fg_plan):
        assert ctypes.sizeof(cls) == c[cls.__name__]
        for name, _ in cls._fields_:
            assert getattr(cls, name).offset == c[f"{cls.__name__}.{name}"], (cls.__name__, name)


def test_host_side_argument_checks():
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    st, g = fg.fg_graph_create_coo(0, src, dst)
    assert st == fg.FG_ERR_INVALID_ARG and g is None
    assert "positive" in fg.fg_last_error()
    st = fg.load().fg_graph_create_coo(3, 2, None, dst.ctypes.data, None, ctypes.byref(ctypes.c_void_p()))
    assert st == fg.FG_ERR_INVALID_ARG
    st = fg.load().fg_graph_create_csr(3, 2, None, dst.ctypes.data, None, ctypes.byref(ctypes.c_void_p()))
    assert st == fg.FG_ERR_INVALID_ARG
    st = fg.load().fg_graph_create_coo(3, -1, src.ctypes.data, dst.ctypes.data, None,
                                       ctypes.byref(ctypes.c_void_p()))
    assert st == fg.FG_ERR_INVALID_ARG
    st = fg.load().fg_graph_create_coo(3, 1 << 31, src.ctypes.data, dst.ctypes.data, None,
                                       ctypes.byref(ctypes.c_void_p()))
    assert st == fg.FG_ERR_INVALID_ARG
    for bad_flags in (8, 0x80000000, 2 | 4):   # unknown bits; renumber and keep ids together
        st, g = fg.fg_graph_create_coo(3, src, dst, flags=bad_flags)
        assert st == fg.FG_ERR_INVALID_ARG and g is None and "flags" in fg.fg_last_error()
        st, g = fg.fg_graph_create_csr(3, np.array([0, 1, 2, 2], np.int64), dst, flags=bad_flags)
        assert st == fg.FG_ERR_INVALID_ARG and g is None
    out = np.zeros(3, np.int32)
    assert fg.fg_sssp(None, 0, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_cc(None, out) == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_select_mode(None, fg.FG_ALGO_BFS)
    assert st == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_select_plan(None, fg.FG_ALGO_BFS)
    assert st == fg.FG_ERR_INVALID_ARG
    assert fg.fg_graph_destroy(None) == fg.FG_OK
    st, _, _, _ = fg.fg_run_batch([(None, 0, 0, out, 0)])
    assert st == fg.FG_ERR_INVALID_ARG and "graph is NULL" in fg.fg_last_error()
    st, _, _ = fg.fg_autotune(None, 0)
    assert st == fg.FG_ERR_INVALID_ARG
    st, _, _ = fg.fg_run_multi(None, fg.FG_ALGO_SSSP, [0], [out])
    assert st == fg.FG_ERR_INVALID_ARG and "graph is NULL" in fg.fg_last_error()
    assert fg.fg_status_string(fg.FG_ERR_OVERFLOW) == "FG_ERR_OVERFLOW"
    assert fg.fg_status_string(fg.FG_ERR_TIMEOUT) == "FG_ERR_TIMEOUT"


def test_binding_rejects_wrong_dtypes():
    with pytest.raises(TypeError):
        fg.fg_graph_create_coo(3, np.array([0], np.int64), np.array([1], np.int32))
    with pytest.raises(TypeError):
        fg.fg_sssp(None, 0, np.zeros(3, np.float32))
