"""Host checks of the C ABI: the library loads, exports every function that
the headers under include/ declare, and its structs have the layout the
binding assumes.
No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2510_15271_b300 import ba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("ba.h", "ba_pose_graph.h", "ba_rig.h")]


@pytest.fixture(scope="module")
def built():
    from paper_2510_15271_b300 import build
    build.build()
    return ba.lib()


def _declared_functions():
    src = "".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:ba_status|void|const char\s*\*)\s+(ba_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ("ba_create", "ba_set_problem", "ba_solve", "ba_get_state", "ba_submit",
                     "ba_poll", "ba_destroy", "ba_solve_batch", "ba_last_error",
                     "ba_pg_create", "ba_pg_set_graph", "ba_pg_solve", "ba_pg_get_state",
                     "ba_rig_create", "ba_rig_set_problem", "ba_rig_solve", "ba_rig_get_state"):
        assert required in names


def test_library_exports_every_declared_function(built):
    out = subprocess.run(["nm", "-D", "--defined-only", ba.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(ba_\w+)", out))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    for n in _declared_functions():
        assert hasattr(built, n)
    assert set(ba.EXPORTS) == set(_declared_functions())


def test_struct_layouts_match_the_c_compiler(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "ba.h"\n'
        "int main(void){\n"
        'printf("%zu %zu %zu %zu %zu\\n", sizeof(ba_options), sizeof(ba_report), '
        "sizeof(ba_problem), sizeof(ba_result), sizeof(ba_intrinsics));\n"
        'printf("%zu %zu %zu %zu %zu\\n", offsetof(ba_options, cuda_stream), '
        "offsetof(ba_options, serve_arena_bytes), offsetof(ba_report, rmse_px), "
        "offsetof(ba_problem, K), offsetof(ba_options, prior_abs_weight));\n"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    a, b = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    sizes = [int(v) for v in a.split()]
    offs = [int(v) for v in b.split()]
    assert sizes == [ctypes.sizeof(ba.Options), ctypes.sizeof(ba.Report),
                     ctypes.sizeof(ba.Problem), ctypes.sizeof(ba.Result),
                     ctypes.sizeof(ba.Intrinsics)]
    assert offs == [ba.Options.cuda_stream.offset, ba.Options.serve_arena_bytes.offset,
                    ba.Report.rmse_px.offset, ba.Problem.K.offset,
                    ba.Options.prior_abs_weight.offset]


def test_option_defaults(built):
    o = ba.ba_options_default()
    assert (o.precision, o.solver, o.max_lm_iters, o.pcg_max_iters) == (ba.BA_FP64, ba.BA_SOLVER_AUTO, 10, 100)
    assert o.pcg_tol == 1e-6 and o.mu0 == 1e-4 and o.use_graph == 1 and o.refine_max == 5
    assert o.mu_min == -1.0 and o.pcg_variant == 0 and o.serve_tick_ms == 4.0
    assert o.serve_split_ms == 10.0
    assert o.prior_seq_weight == 0.0 and o.prior_abs_weight == 0.0


def test_invalid_calls_fail_cleanly_without_a_device(built):
    L = built
    assert L.ba_solve(None, None) == ba.BA_ERR_INVALID_ARG
    assert L.ba_set_problem(None, 1, 1, 1, None, None, None, None, None, None, None, 0) == ba.BA_ERR_INVALID_ARG
    assert L.ba_get_state(None, None, None, 0) == ba.BA_ERR_INVALID_ARG
    L.ba_destroy(None)
    o = ba.ba_options_default(max_lm_iters=0)
    h = ctypes.c_void_p()
    assert L.ba_create(ctypes.byref(o), ctypes.byref(h)) == ba.BA_ERR_INVALID_ARG
    assert "max_lm_iters" in ba.ba_last_error(None)
    o = ba.ba_options_default(precision=7)
    assert L.ba_create(ctypes.byref(o), ctypes.byref(h)) == ba.BA_ERR_INVALID_ARG


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(ba, "_LIB", None)
    monkeypatch.setattr(ba, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ba.lib()
