"""The C ABI library builds, loads without a GPU and exports every entry point
declared in include/mpg.h; the Python binding carries the same names."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_12818_gb300 import build
    return build.build()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("mpg_sample_seeds", "mpg_manifold_walk", "mpg_chain_contribution", "mpg_guide_update",
              "mpg_walk_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    assert set(_declared()) <= exported


def test_python_binding_names_match(libpath):
    from paper_2311_12818_gb300 import mpg
    for n in ("mpg_sample_seeds", "mpg_manifold_walk", "mpg_chain_contribution", "mpg_guide_update",
              "mpg_walk_adjoint", "mpg_guide_records", "mpg_trace_rays"):
        assert callable(getattr(mpg, n))
    assert set(mpg.EXPORTS) <= set(_declared())
    assert mpg.lib().mpg_version() >= 1


def test_error_path_without_arguments(libpath):
    from paper_2311_12818_gb300 import mpg
    L = mpg.lib()
    assert L.mpg_manifold_walk(None, None, None, None, None) == -1
    assert b"NULL" in L.mpg_last_error()
    assert L.mpg_ctx_sync(None, None) == -1


def test_params_struct_layout_matches_header():
    from paper_2311_12818_gb300 import mpg
    src = open(os.path.join(ROOT, "include", "mpg.h")).read()
    body = src[src.index("typedef struct mpg_params"):src.index("} mpg_params;")]
    fields = re.findall(r"\b(?:float|int32_t)\s+([a-z_0-9]+);", body)
    assert fields == [f for f, _ in mpg.mpg_params._fields_]
    body = src[src.index("typedef struct mpg_chains"):src.index("} mpg_chains;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-zA-Z_]+)[;,]", body.replace("B, Q, spq", "B; Q; spq"))
    assert fields == [f for f, _ in mpg.mpg_chains._fields_]
