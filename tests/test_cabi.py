"""Host-side checks of the C-ABI library: it loads, exports every declared symbol,
and validates arguments before touching the GPU."""
import ctypes as C
import os

import numpy as np
import pytest

import __graft_entry__  # noqa: F401  (build helper)


@pytest.fixture(scope="module")
def bmg():
    __graft_entry__.build_library()
    from paper_1511_07042_gb300 import bmg as b
    return b


def test_every_declared_symbol_is_exported(bmg):
    names = bmg.header_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(bmg.LIB, n)]
    assert not missing, missing


def test_default_options(bmg):
    o = bmg.options()
    assert (o.smoother, o.nu, o.form, o.cycles_intermediate, o.max_cycles) == (0, 2, 0, 6, 200)
    assert abs(o.omega - 2.0 / 3.0) < 1e-16
    assert (o.stop_after_cycles, o.resume) == (0, 0)


def test_argument_errors_are_reported_without_gpu(bmg):
    h = C.c_void_p()
    code = bmg.LIB.bmg_assemble(None, 12, None, 20, 2, 0.0, None, None, C.byref(h))
    assert code == 1 and h.value is None
    assert b"null mesh" in bmg.LIB.bmg_last_error() or b"empty" in bmg.LIB.bmg_last_error()
    v = np.zeros((12, 3)); t = np.zeros((20, 3), np.int32)
    code = bmg.LIB.bmg_assemble(v.ctypes.data, 12, t.ctypes.data, 20, 11, 0.0, None, None, C.byref(h))
    assert code == 1
    t[0, 0] = 99
    code = bmg.LIB.bmg_assemble(v.ctypes.data, 12, t.ctypes.data, 20, 1, 0.0, None, None, C.byref(h))
    assert code == 7                                  # BMG_ERR_MESH
    assert bmg.LIB.bmg_hierarchy(None, 2) == 1
    assert bmg.LIB.bmg_solve(None, 4, 2, 0.0, 1e-8, None, None, 0, None, None, 0, None, None) == 1
    assert bmg.LIB.bmg_dense_eig(None, None, 4, 0.0, 2, None, None, None, None) == 1
    assert bmg.LIB.bmg_gram(None, None, 4, 2, 2, None, None) == 1
    used = C.c_size_t(0)
    assert bmg.LIB.bmg_get_state(None, 4, None, 0, C.byref(used)) == 1
    assert bmg.LIB.bmg_set_state(None, 4, None, 0) == 1
    bmg.LIB.bmg_destroy(None)


def test_struct_layouts_match_the_header(bmg, tmp_path):
    """The ctypes mirrors of bmg_options and bmg_solve_info have the C layout: every
    field's offset and the struct sizes, compiled from include/bmg.h by the host C
    compiler."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"bmg_options": bmg.Options, "bmg_solve_info": bmg.SolveInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bmg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(out[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)
