"""CPU-only checks of the C ABI library: it builds for sm_103a, loads without
a GPU, and exports every entry point include/cbfs.h declares (no compute
calls are made here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "cbfs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbfs_\w+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2410_17226_gb300 import build as B

    lib = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(cbfs_\w+)", out))
    want = declared_symbols()
    assert len(want) >= 12
    missing = [s for s in want if s not in exported]
    assert not missing, missing


def test_ctypes_signatures_cover_header():
    from paper_2410_17226_gb300 import cbfs

    assert sorted(cbfs.SIGNATURES) == declared_symbols()
    L = cbfs.lib()  # loads without a GPU
    for name in cbfs.SIGNATURES:
        assert hasattr(L, name)
    assert cbfs.status_string(-2).startswith("CBFS_E_DIAMETER")


def test_built_for_sm103a_only():
    from paper_2410_17226_gb300 import build as B

    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    objs = subprocess.run(["cuobjdump", "--list-elf", B.build()], capture_output=True, text=True)
    if objs.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in objs.stdout


def test_product_path_has_no_cpu_fallback():
    """The binding must not import the oracle and must raise without CUDA."""
    import ast

    for fn in ("cbfs.py", "serve.py", "tune.py", "__init__.py"):
        p = os.path.join(ROOT, "paper_2410_17226_gb300", fn)
        if not os.path.exists(p):
            continue
        tree = ast.parse(open(p).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("oracle") for a in node.names), fn
            if isinstance(node, ast.ImportFrom):
                assert not (node.module or "").startswith("oracle"), fn
    import torch

    if not torch.cuda.is_available():
        from paper_2410_17226_gb300 import cbfs

        with pytest.raises(RuntimeError):
            cbfs.Graph([0, 0], [])


def _struct_fields(name):
    """(type, field) pairs of a typedef'd struct in include/cbfs.h, in order."""
    with open(os.path.join(ROOT, "include", "cbfs.h")) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    body = re.search(r"typedef struct \w*\s*\{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    return re.findall(r"(\w+)\s+(\w+)\s*;", body)


def test_python_structs_match_the_header_field_by_field():
    import ctypes

    from paper_2410_17226_gb300 import cbfs

    ctype = {"float": ctypes.c_float, "int": ctypes.c_int, "uint64_t": ctypes.c_uint64}
    for py, c in ((cbfs.Tune, "cbfs_tune_t"), (cbfs.ClusterStats, "cbfs_cluster_stats_t")):
        want = [(f, ctype[t]) for t, f in _struct_fields(c)]
        assert [(f, t) for f, t in py._fields_] == want, c
