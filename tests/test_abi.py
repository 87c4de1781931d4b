"""The C ABI library builds for sm_103a, loads, and exports every symbol include/glm.h declares.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(glm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_04993_gb300 import build as b
    import paper_1502_04993_gb300 as glm
    path = b.build()
    assert os.path.exists(path)
    return glm.load_library(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("glm_create", "glm_destroy", "glm_set_problem", "glm_filter", "glm_loglik_grad",
                     "glm_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1502_04993_gb300 as glm
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert sorted(glm.SIGNATURES) == names


def test_status_strings(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10, 12345]:
        s = lib.glm_strerror(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.glm_version() >= 100


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.glm_create(ctypes.byref(h), 0, 0, None)
    assert rc == -5 and not h.value
