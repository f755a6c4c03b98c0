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


def test_phase_cycles_rejects_null_on_host():
    lib = isr.load_library()
    assert lib.isr_plan_phase_cycles(None, None) == isr.ISR_ERR_INVALID_ARG


def test_tc05_rate_rejects_bad_arguments_on_host():
    lib = isr.load_library()
    tf, cyc = ctypes.c_double(), ctypes.c_double()
    assert lib.isr_tc05_rate(0, 32, None, None) == isr.ISR_ERR_INVALID_ARG
    for n in (0, 16, 48, 512):
        assert lib.isr_tc05_rate(0, n, ctypes.byref(tf), ctypes.byref(cyc)) == isr.ISR_ERR_INVALID_ARG


def _status(fn, *args, msg=None):
    """Status of a call that must fail; msg: a fragment its error text must contain (so that
    the intended check, not an earlier one, fired)."""
    with pytest.raises(isr.IsrError) as ei:
        fn(*args)
    text = isr.isr_last_error()
    assert text
    if msg is not None:
        assert msg in text, text
    return ei.value.status


FAKE = 0x10000   # a non-NULL address; every call below fails its host checks before using it


def test_peak_fit_rejects_bad_arguments_on_host():
    lib = isr.load_library()
    assert lib.isr_peak_fit(None, 4, 1024, 0, 10, None, None, None) == isr.ISR_ERR_INVALID_ARG
    for n_ranges, nfft, lo, hi in [(0, 1024, 0, 10), (4, 4, 0, 2), (4, 1024, 10, 10), (4, 1024, -1, 10),
                                   (4, 1024, 0, 1025)]:
        assert _status(isr.isr_peak_fit, FAKE, n_ranges, nfft, lo, hi, FAKE, FAKE,
                       msg="band_lo < band_hi") == isr.ISR_ERR_INVALID_ARG


def test_estimator_rejects_bad_arguments_on_host():
    lib = isr.load_library()
    assert lib.isr_est_create(None, 16384, 320, 4608, 128, isr.ISR_EST_BF16, -1, None) == isr.ISR_ERR_INVALID_ARG
    for nfft, lo, ln, mb in [(16384, 320, 8, 128), (16384, 16000, 4608, 128), (16384, -1, 4608, 128),
                             (16384, 320, 4608, 0), (4, 0, 16, 1)]:
        assert _status(isr.isr_est_create, nfft, lo, ln, mb, msg="band_len >= 16") == isr.ISR_ERR_INVALID_ARG
    assert _status(isr.isr_est_create, 16384, 320, 4608, 128, 9, msg="precision") == isr.ISR_ERR_UNSUPPORTED
    assert lib.isr_est_set_params(None, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_est_get_params(None, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_est_features(None, None, 1, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_est_predict(None, None, 1, None, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_est_grad(None, None, 1, None, None, None, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_est_train_step(None, None, 1, None, None, 1e-3, None) == isr.ISR_ERR_INVALID_ARG
    lib.isr_est_destroy(None)  # NULL is safe


def _window(**kw):
    w = isr.IsrWindow()
    w.echo, w.tx_code, w.out = FAKE, FAKE, FAKE
    w.echo_stride, w.tx_stride, w.nfft, w.code_len = 8192, 0, 4096, 4096
    w.n_ranges, w.range_start, w.range_step, w.n_ipp, w.order, w.reserved = 10, 0, 25, 100, -1, 0
    for k, v in kw.items():
        setattr(w, k, v)
    return w


@pytest.mark.parametrize("kw,status,msg", [
    (dict(nfft=1024, code_len=1024), isr.ISR_ERR_UNSUPPORTED, "nfft"),     # batched windows: nfft 2048..16384
    (dict(nfft=3000), isr.ISR_ERR_UNSUPPORTED, "nfft"),
    (dict(code_len=0), isr.ISR_ERR_INVALID_ARG, "geometry"),
    (dict(n_ipp=0), isr.ISR_ERR_INVALID_ARG, "geometry"),
    (dict(echo_stride=8190), isr.ISR_ERR_INVALID_ARG, "geometry"),
    (dict(order=9), isr.ISR_ERR_INVALID_ARG, "geometry"),
    (dict(tx_stride=100), isr.ISR_ERR_INVALID_ARG, "geometry"),
    (dict(n_ranges=200), isr.ISR_ERR_OUT_OF_RANGE, "past the echo row"),   # 199 * 25 + 4096 > 8192
    (dict(echo=0), isr.ISR_ERR_INVALID_ARG, "NULL or misaligned"),
    (dict(echo=FAKE + 4), isr.ISR_ERR_INVALID_ARG, "NULL or misaligned"),  # echo must be 16-byte aligned
])
def test_batch_rejects_bad_windows_on_host(kw, status, msg):
    # windows are checked in order and a good window's device-pointer query needs a GPU, so
    # the bad window is the only one
    assert _status(isr.isr_batch_create, [_window(**kw)], msg=msg) == status


def test_batch_rejects_bad_calls_on_host():
    lib = isr.load_library()
    h = ctypes.c_void_p()
    arr = (isr.IsrWindow * 1)(_window())
    assert lib.isr_batch_create(None, arr, 1, 0, -1, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_batch_create(ctypes.byref(h), None, 1, 0, -1, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_batch_create(ctypes.byref(h), arr, 0, 0, -1, None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_batch_create(ctypes.byref(h), arr, 1, 64, -1, None) == isr.ISR_ERR_INVALID_ARG   # unknown flag
    assert lib.isr_batch_run(None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_batch_wait(None) == isr.ISR_ERR_INVALID_ARG
    assert lib.isr_batch_query(None, None) == isr.ISR_ERR_INVALID_ARG
    lib.isr_batch_destroy(None)  # NULL is safe


def test_allocation_free_call_rejects_bad_arguments_on_host():
    lib = isr.load_library()
    assert lib.isr_integrate_static(None, None, None, 1, None) == isr.ISR_ERR_INVALID_ARG
    assert _status(isr.isr_integrate_static, _desc(nfft=1000), FAKE, FAKE, 1, FAKE,
                   msg="power of two") == isr.ISR_ERR_UNSUPPORTED
    assert _status(isr.isr_integrate_static, _desc(n_ranges=50), FAKE, FAKE, 1, FAKE) == isr.ISR_ERR_OUT_OF_RANGE
    # 4097 gates x 1024 bins exceed the 4 Mi-float static scratch (geometry itself is valid)
    big = _desc(n_ranges=4097, range_step=1, echo_stride=8192)
    assert _status(isr.isr_integrate_static, big, FAKE, FAKE, 1, FAKE,
                   msg="static scratch") == isr.ISR_ERR_INVALID_ARG
