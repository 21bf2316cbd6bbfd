"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function that include/bgpc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bgpc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("bgpc_", "d2gc_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_02628_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["bgpc_ctx_create", "bgpc_ctx_destroy", "bgpc_color", "d2gc_color",
              "bgpc_validate", "bgpc_color_sets", "bgpc_strerror", "bgpc_opts_default"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    import paper_1701_02628_gb300 as bg
    assert sorted(bg.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    """bgpc_opts_default and bgpc_strerror touch no device."""
    import paper_1701_02628_gb300 as bg
    o = bg.bgpc_opts_default()
    assert (o.policy, o.chunk, o.waves, o.big_net, o.max_rounds) == (0, 64, 16, 64, 1000)
    assert bg.bgpc_strerror(bg.BGPC_EUNSORTED).startswith("adjacency")
    assert ctypes.sizeof(bg.bgpc_stats_t) == (4 + 4 + 8 * 64 * 2 + 8 + 4 * 4 + 8 * 2 + 8 * 4
                                               + 8 * 4 + 8 * 5 + 8 * 3 + 8 + 4 * 2)


def test_struct_layout_matches_header():
    """The ctypes mirrors follow the C struct layout (field offsets)."""
    import paper_1701_02628_gb300 as bg
    assert bg.bgpc_opts_t.rank.offset == 16
    assert bg.bgpc_opts_t.stop_after_waves.offset == 32
    assert bg.bgpc_opts_t.W_out.offset == 40
    assert bg.bgpc_graph_t.a_ptr.offset == 16


def test_ctx_create_without_gpu_fails_cleanly(lib):
    """With no device visible the context constructor returns an error code."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.bgpc_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    assert lib.bgpc_ctx_create(ctypes.byref(h), 0) < 0


def test_struct_layout_against_the_c_compiler(tmp_path):
    """sizeof / offsetof of every ABI struct, from gcc on include/bgpc.h,
    equal the ctypes mirrors of the binding."""
    import subprocess
    import paper_1701_02628_gb300 as bg
    fields = {"bgpc_graph_t": ["n_a", "n_b", "nnz", "a_ptr", "a_idx", "b_ptr", "b_idx"],
              "bgpc_ugraph_t": ["n", "nnz", "ptr", "idx"],
              "bgpc_opts_t": [f for f, _ in bg.bgpc_opts_t._fields_],
              "bgpc_stats_t": [f for f, _ in bg.bgpc_stats_t._fields_],
              "bgpc_mlp_t": ["w", "w_bf16", "adam_m", "adam_v", "step"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    for st in fields:
        cls = getattr(bg, st)
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
