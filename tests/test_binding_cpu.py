"""The Python binding is argument marshalling only; its rules hold without a
GPU: host arrays must be C-contiguous numpy arrays, NULL maps to None, and
precision names map to the C ABI's codes."""

import numpy as np
import pytest


def test_pointer_marshalling_rules():
    import paper_2604_27451_gb300 as pkg

    assert pkg._ptr(None) == (None, None)
    a = np.zeros(5, dtype=np.complex128)
    p, dev = pkg._ptr(a)
    assert dev is False and p.value == a.ctypes.data
    with pytest.raises(ValueError):
        pkg._ptr(np.zeros((4, 4), dtype=np.complex128)[:, ::2])
    with pytest.raises(ValueError):
        pkg._ptr([1.0, 2.0])


def test_precision_codes_match_the_header():
    import re
    from pathlib import Path

    import paper_2604_27451_gb300 as pkg

    hdr = (Path(__file__).resolve().parents[1] / "include" / "cvsadc.h").read_text()
    codes = {m.group(1): int(m.group(2))
             for m in re.finditer(r"#define CVSADC_(FP64|MIXED_BF16X3|MIXED_SLICE4|FP64_SLICE7) (\d+)", hdr)}
    assert pkg.PRECISIONS == {"fp64": codes["FP64"], "bf16x3": codes["MIXED_BF16X3"],
                              "slice4": codes["MIXED_SLICE4"], "fp64_slice7": codes["FP64_SLICE7"]}
    flags = {m.group(1): int(m.group(2))
             for m in re.finditer(r"#define CVSADC_FLAG_(\w+) (\d+)", hdr)}
    from paper_2604_27451_gb300 import _lib
    for name, val in flags.items():
        assert getattr(_lib, "CVSADC_FLAG_" + name) == val
