"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, and exports every entry point declared in include/*.h."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(mc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_05458_gb300 import build
    build.build_library()
    from paper_1808_05458_gb300 import mincut
    return mincut.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("mc_graph_create", "mc_min_cut", "mc_batch_min_cut", "mc_graph_destroy",
              "mc_strerror"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f"{f} declared in include/ but not exported"


def test_binding_covers_exports():
    from paper_1808_05458_gb300 import mincut
    assert set(declared_functions()) <= set(mincut.EXPORTS)


def test_strerror_and_defaults_without_gpu(lib):
    from paper_1808_05458_gb300 import mincut
    assert "invalid" in mincut.strerror(mincut.MC_EINVAL)
    o = mincut.options()
    assert o.pr_level == 4 and o.pq_order == mincut.MC_PQ_LIFO


def test_invalid_arguments_rejected_without_gpu(lib):
    # n < 2 and NULL outputs are rejected before any CUDA call
    h = ctypes.c_void_p()
    import numpy as np
    rp = np.zeros(2, dtype=np.int32)
    assert lib.mc_graph_create(1, rp.ctypes.data, None, None, 0, ctypes.byref(h)) == -1
    assert lib.mc_min_cut(None, None, None, None, None) == -1
    assert lib.mc_graph_destroy(None) == -1
    # the batched-kernel shape selector: indices -1 .. count - 1 only
    count = lib.mc_batch_shape_count()
    assert count >= 1
    assert lib.mc_batch_set_shape(count) == -1 and lib.mc_batch_set_shape(-2) == -1
    assert lib.mc_batch_set_shape(count - 1) == 0 and lib.mc_batch_set_shape(-1) == 0


def test_binding_struct_layouts_match_header(tmp_path):
    # the ctypes structures of the binding against the C compiler's view of
    # include/mc.h: size and every field offset
    import shutil
    import subprocess
    from paper_1808_05458_gb300 import mincut
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"mc_options": mincut.McOptions, "mc_stats": mincut.McStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, fname, val = line.split()
        got[(cname, fname)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_constants_match_header():
    # every #define MC_* integer of include/mc.h that the binding mirrors
    from paper_1808_05458_gb300 import mincut
    text = open(os.path.join(ROOT, "include", "mc.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(MC_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", text)}
    alias = {"MC_PROPOSER_PARAMS": "PROPOSER_PARAMS"}
    mirrored = 0
    for k, v in defs.items():
        name = alias.get(k, k)
        if hasattr(mincut, name):
            assert getattr(mincut, name) == v, k
            mirrored += 1
    for k in ("MC_OK", "MC_EINVAL", "MC_ENOMEM", "MC_EOVERFLOW", "MC_PQ_FIFO", "MC_BOUND_LP",
              "MC_DEVICE_PTRS", "MC_PROPOSER_PARAMS"):
        assert k in defs and hasattr(mincut, alias.get(k, k)), k
    assert mirrored >= 15
