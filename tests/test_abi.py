"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/oem.h declares; argument errors come back before any launch;
the oracle and the product share no code."""
import ast
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "oem.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(oem_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (oem_[a-z0-9_]+)", out))
    declared = _declared()
    assert len(declared) >= 12
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(lib_path):
    import paper_1801_09661_gb300 as oem
    for name in _declared():
        assert hasattr(oem.lib, name)
    for name in oem.EXPORTED:
        assert name in _declared()


def test_options_default_values(lib_path):
    import paper_1801_09661_gb300 as oem
    o = oem.make_options()
    assert o.nlambda == 100 and o.lambda_min_ratio == 1e-3 and o.tol == 1e-7
    assert o.max_iter == 10000 and o.gram_mode == oem.OEM_GRAM_AUTO


def test_argument_errors_return_before_launch(lib_path):
    """Bad arguments are rejected on the host with OEM_EINVAL; no context or
    device is needed for that (a NULL context is rejected first)."""
    import ctypes as C
    import paper_1801_09661_gb300 as oem
    L = oem.lib
    assert L.oem_gram(None, None, 1, 10, 5, 8, None, 0, None, None, None, None) == oem.OEM_EINVAL
    assert L.oem_destroy(None) == oem.OEM_EINVAL
    assert L.oem_sync(None, None) == oem.OEM_EINVAL
    o = oem.make_options()
    assert L.oem_fit_path(None, None, None, 5, 0.0, None, 1, C.byref(o), None, None, None, None,
                          None) == oem.OEM_EINVAL


def test_noalloc_rejects_sizes_beyond_its_maximum(lib_path):
    """oem_gram_noalloc refuses p > 1024 (OEM_EBUDGET) and bad strides
    (OEM_EINVAL) on the host, before touching the device."""
    import paper_1801_09661_gb300 as oem
    L = oem.lib
    fake = 4096  # aligned, never dereferenced on these paths
    assert L.oem_gram_noalloc(fake, oem.OEM_F32, 1000, 2000, 2000, fake, oem.OEM_GRAM_FP32,
                              fake, fake, fake, None) == oem.OEM_EBUDGET
    assert L.oem_gram_noalloc(fake, oem.OEM_F32, 1000, 10, 10, fake, oem.OEM_GRAM_FP32,
                              fake, fake, fake, None) == oem.OEM_EINVAL
    assert L.oem_gram_noalloc(fake, oem.OEM_F64, 1000, 10, 10, fake, oem.OEM_GRAM_FP32,
                              fake, fake, fake, None) == oem.OEM_EINVAL


def _imports(path):
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def test_oracle_and_product_share_no_code():
    for d, banned in (("oracle", "paper_1801_09661_gb300"), ("paper_1801_09661_gb300", "oracle")):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith(".py"):
                assert banned not in _imports(os.path.join(ROOT, d, f)), (d, f)
    for f in os.listdir(os.path.join(ROOT, "synthgen")):
        if f.endswith(".py"):
            mods = _imports(os.path.join(ROOT, "synthgen", f))
            assert "oracle" not in mods and "paper_1801_09661_gb300" not in mods
