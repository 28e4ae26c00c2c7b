"""Helpers shared by the GPU tests (no test functions here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2209_15445_gb300 import build
    build.build()
    return torch


def make(geom, **kw):
    from paper_2209_15445_gb300 import adept as A
    kw.setdefault("arena_bytes", 512 << 20)
    return A.Transport(geom, **kw)


def ledger(edep, leaked, killed):
    return edep.sum(axis=1) + leaked + killed
