"""The C-ABI library loads without a GPU, exports every entry point that
include/dsssp.h declares, and its structs have the same layout as the binding's."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsssp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dsssp_\w+)\s*\(", text)))


def test_library_exports_every_declared_entry_point():
    import paper_1911_06895_gb300 as ds
    lib = ctypes.CDLL(ds.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ds.EXPORTED)


def test_status_strings_and_defaults():
    import paper_1911_06895_gb300 as ds
    for s in range(13):
        assert ds.dsssp_status_string(s) != b"unknown status"
    assert ds.dsssp_status_string(999) == b"unknown status"
    o = ds.make_options()
    assert o.struct_size == ctypes.sizeof(ds.dsssp_options)
    assert o.block_size == 512 and o.solo_work == 2048 and o.timeout_ns == 2_000_000_000
    assert ds.dsssp_options_default(None) == ds.DSSSP_ERR_INVALID_ARG


def test_null_arguments_rejected_without_gpu():
    import paper_1911_06895_gb300 as ds
    h = ctypes.c_void_p()
    assert ds.dsssp_graph_create(0, 0, None, None, None, 0, 0, None, ctypes.byref(h)) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_graph_create(4, 2, None, None, None, 0, 0, None, ctypes.byref(h)) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_graph_create(4, 0, ctypes.c_void_p(8), None, None, 7, 0, None,
                                 ctypes.byref(h)) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_solve(None, 0, 1.0, None, None, None, None, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_prepare(None, 1.0, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_graph_destroy(None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_graph_sync(None, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_graph_info(None, None, None, None) == ds.DSSSP_ERR_INVALID_ARG
    b = ctypes.c_void_p()
    assert ds.dsssp_batch_create(None, 1, None, 1, None, None, None, None, 0, None, None,
                                 ctypes.byref(b)) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_batch_create(None, 0, None, 0, None, None, None, None, 0, None, None,
                                 None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_batch_run(None, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_batch_sync(None, None, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_batch_destroy(None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_backward(None, None, None, 0, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_solve_batched(None, 1, None, 1, None, None, None, None, None, None,
                                  None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_autotune(None, 1, None, 1, None, None, None, None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_tune_team_blocks(None, 1, None, 1, None, None, None, None, None, None,
                                     None) == ds.DSSSP_ERR_INVALID_ARG
    assert ds.dsssp_tune_solo_work(None, None, 1, 1.0, None, None, None) == ds.DSSSP_ERR_INVALID_ARG


def test_struct_layout_matches_header():
    import paper_1911_06895_gb300 as ds
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "dsssp.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(dsssp_options), sizeof(dsssp_stats),
             offsetof(dsssp_options, max_phases), offsetof(dsssp_options, test_hook),
             offsetof(dsssp_stats, block_size), sizeof(dsssp_batch_stats),
             offsetof(dsssp_batch_stats, team));
      printf("%zu %zu %zu\n", sizeof(dsssp_tune_options), offsetof(dsssp_tune_options, candidates),
             offsetof(dsssp_options, team_blocks));
      return 0;
    }'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    want = [ctypes.sizeof(ds.dsssp_options), ctypes.sizeof(ds.dsssp_stats),
            ds.dsssp_options.max_phases.offset, ds.dsssp_options.test_hook.offset,
            ds.dsssp_stats.block_size.offset, ctypes.sizeof(ds.dsssp_batch_stats),
            ds.dsssp_batch_stats.team.offset, ctypes.sizeof(ds.dsssp_tune_options),
            ds.dsssp_tune_options.candidates.offset, ds.dsssp_options.team_blocks.offset]
    assert [int(x) for x in out] == want
