"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol
that include/me.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_07439_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    import paper_2503_07439_gb300 as me
    names = me.declared_symbols()
    assert "me_init" in names and "me_submit" in names and "me_poll" in names
    for n in names:
        assert hasattr(lib, n), n


def test_header_cites_the_paper_and_documents_errors():
    text = open(os.path.join(ROOT, "include", "me.h")).read()
    for code in ("ME_ERR_ARG", "ME_ERR_OOM", "ME_ERR_PROCESS", "ME_ERR_TIMEOUT", "ME_ERR_CUDA", "ME_ERR_BUSY"):
        assert code in text
    assert re.search(r"Sec\. 4\.3, Algorithm 2", text)


def test_default_params_without_gpu(lib):
    import paper_2503_07439_gb300 as me
    p = me.default_params()
    assert p.version == me.ME_PARAMS_VERSION and p.precision == me.ME_PREC_FP64 and p.queued_rescue == 0
    assert abs(p.alpha_s - 0.118) < 1e-15 and abs(p.mt - 173.0) < 1e-12


def test_binding_has_no_cpu_fallback():
    """The package exposes only the ctypes binding: no numpy/torch compute path."""
    src = open(os.path.join(ROOT, "paper_2503_07439_gb300", "_capi.py")).read()
    assert "oracle" not in src and "synth" not in src


def test_noalloc_buffer_rule_refuses_other_devices(lib):
    """The allocation-free entry point accepts device memory of the requested GPU and
    managed memory, and refuses device memory of another GPU (no peer access is set up,
    so its kernels could not read it) and host memory.  The rule is checked here through
    its exported helper, so that no second GPU is needed."""
    f = lib.me_internal_buffer_usable
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    unregistered, host, device, managed = 0, 1, 2, 3  # cudaMemoryType
    assert f(device, 0, 0) == 1 and f(device, 3, 3) == 1
    assert f(device, 1, 0) == 0 and f(device, 0, 1) == 0
    assert f(managed, 0, 1) == 1
    assert f(host, 0, 0) == 0 and f(unregistered, 0, 0) == 0
