"""The C-ABI library loads without a GPU, exports every function include/*.h declares,
and rejects bad plan descriptions on the host before any CUDA call."""
import ctypes
import glob
import os
import re

import pytest

from paper_2311_18737_gb300 import isr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(isr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    lib = isr.load_library()
    declared = _declared()
    assert {"isr_plan_create", "isr_integrate", "isr_spectra", "isr_destroy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared but not exported"
    assert set(isr.EXPORTS) == declared


def _desc(**kw):
    d = isr.IsrPlanDesc()
    d.nfft, d.code_len, d.n_ranges, d.range_start, d.range_step = 1024, 1024, 4, 0, 25
    d.tx_type, d.echo_stride, d.tx_stride, d.ipp_chunk, d.max_chunks = isr.ISR_TX_PM1, 2048, 0, 0, 0
    d.device, d.flags, d.stream = -1, 0, None
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,status", [
    (dict(nfft=1000), isr.ISR_ERR_UNSUPPORTED),
    (dict(nfft=32768, code_len=1024), isr.ISR_ERR_UNSUPPORTED),
    (dict(nfft=4), isr.ISR_ERR_UNSUPPORTED),
    (dict(tx_type=7), isr.ISR_ERR_UNSUPPORTED),
    (dict(code_len=0), isr.ISR_ERR_INVALID_ARG),
    (dict(code_len=2048), isr.ISR_ERR_INVALID_ARG),
    (dict(n_ranges=0), isr.ISR_ERR_INVALID_ARG),
    (dict(range_step=0), isr.ISR_ERR_INVALID_ARG),
    (dict(echo_stride=2050), isr.ISR_ERR_INVALID_ARG),
    (dict(tx_stride=100), isr.ISR_ERR_INVALID_ARG),
    (dict(flags=1), isr.ISR_ERR_INVALID_ARG),
    (dict(max_chunks=70000), isr.ISR_ERR_INVALID_ARG),
    (dict(n_ranges=50), isr.ISR_ERR_OUT_OF_RANGE),     # 49*25 + 1024 > 2048
    (dict(range_start=1100), isr.ISR_ERR_OUT_OF_RANGE),
])
def test_bad_descriptions_rejected_on_host(kw, status):
    with pytest.raises(isr.IsrError) as ei:
        isr.isr_plan_create(_desc(**kw))
    assert ei.value.status == status
    assert isr.isr_last_error()


def test_null_arguments():
    lib = isr.load_library()
    assert lib.isr_plan_create(None, None) == isr.ISR_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.isr_plan_create(ctypes.byref(h), None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_integrate(None, None, None, 1, None, 1024) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_spectra(None, None, 0, None) == isr.ISR_ERR_INVALID_ARG
    lib.isr_destroy(None)  # NULL is safe


def test_fp32_peak_rejects_bad_arguments_on_host():
    lib = isr.load_library()
    assert lib.isr_fp32_peak(0, 0, None, None) == isr.ISR_ERR_INVALID_ARG
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.isr_fp32_peak(0, 2, ctypes.byref(tf), ctypes.byref(ms)) == isr.ISR_ERR_INVALID_ARG
