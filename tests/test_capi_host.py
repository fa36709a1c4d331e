"""The C-ABI library loads and exports what include/saamg.h declares (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "saamg.h")


@pytest.fixture(scope="module")
def S():
    from paper_0907_4863_gb300 import build
    build.build()
    from paper_0907_4863_gb300 import saamg
    saamg.lib()
    return saamg


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(saamg_[a-z0-9_]+)\s*\(", text)) - {"saamg_alloc_fn", "saamg_free_fn"})


def test_every_declared_symbol_is_exported(S):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIBPATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (saamg_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = S.lib()
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layouts_match_header(S, tmp_path):
    """Sizes and offsets of the ctypes mirrors equal what a C compiler makes of the header."""
    structs = {"saamg_domain": S.Domain, "saamg_grid": S.Grid, "saamg_params": S.Params,
               "saamg_solve_info": S.SolveInfo, "saamg_hierarchy_info": S.HierarchyInfo,
               "saamg_stencil_config": S.StencilConfig}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "saamg.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_params_default(S):
    p = S.params_default()
    assert (p.cheb_degree, p.cheb_ratio, p.cheb_safety, p.max_coarse, p.max_levels, p.power_iters,
            p.precision, p.beta_rule, p.maxit, p.device_loop) == (2, 30.0, 1.1, 1000, 10, 10, 0, 0,
                                                                1000, 1)
    assert S.lib().saamg_params_default(None) == S.EINVAL


def test_invalid_arguments_are_rejected_before_any_device_work(S):
    L = S.lib()
    out = C.c_void_p()
    g = S.Grid()
    d = S.Domain(0.45, 0.45, 1.0, 0.0, 0.0, 0, 1)
    assert L.saamg_build_operator(None, C.byref(g), 1, None, C.byref(out)) == S.EINVAL
    assert "NULL" in S.last_error()
    for n, h in [((0, 4, 4), (0.1, 0.1, 0.1)), ((4, 4, 1), (0.1, 0.1, 0.1)),
                 ((4, 4, 4), (0.0, 0.1, 0.1)), ((4, 4, 4), (float("nan"), 0.1, 0.1))]:
        g = S.Grid()
        for k in range(3):
            g.n[k], g.h[k], g.origin[k] = n[k], h[k], -0.5
        assert L.saamg_build_operator(C.byref(d), C.byref(g), 1, None, C.byref(out)) == S.EINVAL
    g = S.Grid()
    for k in range(3):
        g.n[k], g.h[k], g.origin[k] = 4, 0.25, -0.5
    assert L.saamg_build_operator(C.byref(d), C.byref(g), 7, None, C.byref(out)) == S.EINVAL
    bad = S.Domain(-1.0, 0.45, 1.0, 0.0, 0.0, 0, 1)
    assert L.saamg_build_operator(C.byref(bad), C.byref(g), 1, None, C.byref(out)) == S.EINVAL
    dz = S.Domain(0.45, 0.45, 1.0, 0.0, 0.0, 5, 1)
    assert L.saamg_build_operator(C.byref(dz), C.byref(g), 1, None, C.byref(out)) == S.EINVAL
    assert L.saamg_setup(None, None, None, C.byref(out)) == S.EINVAL
    assert L.saamg_solve(None, None, None, 1e-8, None, None) == S.EINVAL
    assert L.saamg_vcycle(None, None, None, None) == S.EINVAL
    n_agg = C.c_int(-1)
    assert L.saamg_mis2_aggregate(-1, None, None, None, 0, None, None, C.byref(n_agg), None) == S.EINVAL
    assert L.saamg_mis2_aggregate(0, None, None, None, 0, None, None, C.byref(n_agg), None) == S.OK
    assert n_agg.value == 0
    # a garbage handle is recognised by its tag and ignored by saamg_free
    buf = (C.c_uint32 * 16)()
    L.saamg_free(C.cast(buf, C.c_void_p))
    L.saamg_free(None)


def test_allocator_hook_pairing(S):
    L = S.lib()
    assert L.saamg_set_allocator(S.ALLOC_FN(), S.FREE_FN(), None) == S.OK
    f = S.ALLOC_FN(lambda n, s, c: None)
    assert L.saamg_set_allocator(f, S.FREE_FN(), None) == S.EINVAL
