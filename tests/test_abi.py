"""CPU checks of the C ABI: the library builds, loads without a GPU, and exports every
function declared in include/adept.h; the binding refuses to run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "adept.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adept_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("adept_init", "adept_build_tables", "adept_submit", "adept_transport", "adept_get_scoring",
              "adept_last_error", "adept_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2209_15445_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(lib, n), n


def test_null_arguments_are_rejected_without_touching_the_gpu():
    from paper_2209_15445_gb300 import adept as A
    L = A.load()
    assert L.adept_init(None, None, None, 0, None, None, None, 0, None) == A.EINVAL
    assert L.adept_build_tables(None) == A.EINVAL
    assert L.adept_transport(None, 0) == A.EINVAL
    assert L.adept_poll(None, 1) == A.EINVAL
    assert A.adept_last_error(None) == "null context"


def test_transport_wrapper_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2209_15445_gb300 import adept as A
    from paper_2209_15445_gb300 import workloads as W
    with pytest.raises(RuntimeError):
        A.Transport(W.slab_calorimeter())
