"""Host-side checks of the C-ABI library: it builds, loads, and exports
every entry point declared in include/cvsadc.h.  No compute calls (there
is no GPU here)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "cvsadc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cvsadc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_27451_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("cvsadc_create", "cvsadc_destroy", "cvsadc_solve",
                 "cvsadc_strerror", "cvsadc_sigma", "cvsadc_prepare"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_2604_27451_gb300 import _lib

    assert sorted(_lib.exported_names()) == _declared()


def test_strerror_and_null_arguments(lib):
    assert lib.cvsadc_strerror(0) == b"ok"
    assert lib.cvsadc_strerror(-2).startswith(b"input matrix")
    assert lib.cvsadc_create(None, 0, None) == -1
    # NULL context is rejected without touching the device
    assert lib.cvsadc_solve(None, None, None, None, None, None, None, None, None) == -1
    assert lib.cvsadc_sigma(None, 0, 0, None, None, 1) == -1
    lib.cvsadc_destroy(None)


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.cvsadc_create(ctypes.byref(h), 0, None)
    assert rc in (-1, -4)
    assert not h.value


def test_estimate_bytes_without_gpu():
    """The footprint estimate is host arithmetic: it bounds the stored
    tensors from below and grows with every dimension and the root count."""
    import paper_2604_27451_gb300 as pkg

    def est(nc, nw, nv, L, k=4, prec="fp64"):
        return pkg.estimate_bytes(nc, nw, nv, L, nroots=k, precision=prec)

    nc, nw, nv, L = 6, 50, 250, 1250
    n, o = nc + nw + nv, nc + nw
    N = nc * nv + nc * nw * nv * (nv - 1) // 2
    floor = 16 * L * n * n + 32 * o * o * nv * nv + 16 * N * 48 * 2
    assert est(nc, nw, nv, L) >= floor
    assert est(nc, nw, nv, L) < 4 * floor
    assert est(nc, nw, nv + 10, L) > est(nc, nw, nv, L)
    assert est(nc, nw + 2, nv, L) > est(nc, nw, nv, L)
    assert est(nc, nw, nv, L + 100) > est(nc, nw, nv, L)
    assert est(nc, nw, nv, L, k=16) > est(nc, nw, nv, L, k=4)
    # the preconditioner packs 4-slice operands in every precision
    assert est(nc, nw, nv, L, prec="slice4") >= est(nc, nw, nv, L)
    with pytest.raises(pkg.CvsadcError):
        est(0, nw, nv, L)


def test_estimate_bytes_large_shape_without_gpu():
    """The large shape (12/120/600/3000, 16 roots): a full-space subspace of
    4.14 GB vectors does not fit one GPU, the doubles-folded solver does;
    its estimate still covers B^P, the t2 bands and the sigma
    intermediates of one vector."""
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L, k = 12, 120, 600, 3000, 16
    n = nc + nw + nv
    full = pkg.estimate_bytes(nc, nw, nv, L, nroots=k, precision="slice4")
    fold = pkg.estimate_bytes(nc, nw, nv, L, nroots=k, precision="slice4", solver="folded")
    assert full > 1e12
    assert fold < 284208 * 2**20  # one GB300's HBM (nvidia-smi total)
    floor = 16 * L * n * n + 16e9 + 2 * 16 * nc * nv * nw * nv
    assert fold > floor


def test_batched_and_bytes_reject_null_without_gpu():
    from paper_2604_27451_gb300 import _lib

    lib = _lib.load()
    assert lib.cvsadc_solve_batched(None, 1, None, None, None, None, None, None, None,
                                    None, None, 0) == -1
    assert lib.cvsadc_device_bytes(None, None) == -1
    assert lib.cvsadc_estimate_bytes(None, None) == -1
