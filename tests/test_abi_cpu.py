"""The C-ABI library builds, loads and exports every symbol include/pwk.h declares (no GPU;
only pure host functions are called)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_01695_gb300 import build, pwk
    if not os.path.exists(pwk.LIB_PATH):
        build.build()
    return pwk.load()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pwk_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2412_01695_gb300 import pwk
    declared = _declared()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(pwk.EXPORTS) == declared


def test_pure_host_functions(lib):
    from paper_2412_01695_gb300 import pwk
    assert pwk.version().startswith("pwk")
    assert lib.pwk_strerror(0) == b"success"
    assert lib.pwk_strerror(-4).startswith(b"plan HBM budget")
    assert pwk.supported_grid(24) and pwk.supported_grid(36) and pwk.supported_grid(20)
    assert not pwk.supported_grid(23) and not pwk.supported_grid(7)


def test_null_arguments_rejected_without_gpu(lib):
    """Argument checks run before any CUDA call: a NULL plan is an error, not a crash."""
    import ctypes
    assert lib.pwk_hpsi_batched(None, 0, None, None, 1, None) == -1
    assert lib.pwk_plan_create(None, None, 24, 24, 24, 1, None, None, 1, None, 0, None, None, None, 0) == -1
    h = ctypes.c_void_p()
    assert lib.pwk_plan_create(ctypes.byref(h), None, 24, 24, 24, 1, None, None, 1, None, 0, None,
                               None, None, 0) == -1
    lib.pwk_plan_destroy(None)
