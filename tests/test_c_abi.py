"""The C ABI as a C program sees it.

* CPU: a C file compiled with gcc against include/isr.h prints the size and field offsets of
  every struct in the header; they must equal the ctypes mirror in the Python binding (a
  field added to the header but not to the binding would garble every call).
* GPU: a plain C client (create -> integrate host buffers in two calls -> spectra into host
  memory -> destroy), linked against the library, against the FP64 oracle.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2311_18737_gb300 import isr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi")
INCLUDE = os.path.join(ROOT, "include")

MIRRORS = {"isr_plan_desc": isr.IsrPlanDesc, "isr_ranges": isr.IsrRanges, "isr_plan_info": isr.IsrPlanInfo,
           "isr_window": isr.IsrWindow, "isr_batch_info": isr.IsrBatchInfo}


def _gcc(src, out, *extra):
    cmd = ["gcc", "-std=c11", "-O1", "-Wall", "-Werror", f"-I{INCLUDE}", src, "-o", out, *extra]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, f"gcc failed: {' '.join(cmd)}\n{r.stderr}"


def test_struct_layouts_match_the_binding(tmp_path):
    exe = str(tmp_path / "abi_layout")
    _gcc(os.path.join(SRC, "abi_layout.c"), exe)
    lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    c_size, c_off = {}, {}
    for ln in filter(None, lines):
        name, value = ln.rsplit(" ", 1)
        if name.endswith(" size"):
            c_size[name[:-5]] = int(value)
        else:
            c_off[name] = int(value)
    assert set(c_size) == set(MIRRORS)
    for cname, py in MIRRORS.items():
        assert ctypes.sizeof(py) == c_size[cname], f"sizeof({cname}): C {c_size[cname]}, ctypes {ctypes.sizeof(py)}"
        fields = [f for f, _ in py._fields_]
        c_fields = [k.split(".", 1)[1] for k in c_off if k.startswith(cname + ".")]
        assert fields == c_fields, f"{cname}: C fields {c_fields}, ctypes fields {fields}"
        for f in fields:
            assert getattr(py, f).offset == c_off[f"{cname}.{f}"], f"offsetof({cname}, {f}) differs"


def test_constants_match_the_binding(tmp_path):
    src = tmp_path / "consts.c"
    names = ["ISR_OK", "ISR_ERR_INVALID_ARG", "ISR_ERR_UNSUPPORTED", "ISR_ERR_OUT_OF_RANGE", "ISR_ERR_NO_MEMORY",
             "ISR_ERR_CUDA", "ISR_ERR_TIMEOUT", "ISR_TX_CI16", "ISR_TX_C32", "ISR_TX_PM1", "ISR_RESET_AFTER",
             "ISR_MEAN", "ISR_PREC_FP32", "ISR_PREC_TC_BF16_SPLIT", "ISR_PREC_TC_FP16_SPLIT", "ISR_PREC_TC_BF16",
             "ISR_PREC_TC_FP16", "ISR_PREC_TC05_BF16_SPLIT", "ISR_PREC_TC05_FP16_SPLIT",
             "ISR_PREC_TC05_BF16", "ISR_PREC_TC05_FP16", "ISR_STATIC_SCRATCH_FLOATS", "ISR_EST_N_PARAMS", "ISR_EST_FP32", "ISR_EST_BF16", "ISR_EST_BF16_MMASYNC",
             "ISR_BATCH_GRAPH", "ISR_BATCH_AUTOTUNE"]
    body = "\n".join(f'    printf("{n} %lld\\n", (long long)({n}));' for n in names)
    src.write_text(f'#include <stdio.h>\n#include "isr.h"\nint main(void)\n{{\n{body}\n    return 0;\n}}\n')
    exe = str(tmp_path / "consts")
    _gcc(str(src), exe)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in filter(None, out):
        n, v = ln.split()
        assert getattr(isr, n) == int(v), f"{n}: C {v}, binding {getattr(isr, n)}"


@pytest.mark.gpu
def test_c_client_against_oracle(tmp_path):
    import oracle
    import synth
    from gpu_helpers import RTOL, assert_parity

    exe = str(tmp_path / "c_client")
    libdir = os.path.dirname(isr.LIB_PATH)
    _gcc(os.path.join(SRC, "c_client.c"), exe, f"-L{libdir}", "-lisr", f"-Wl,-rpath,{libdir}")
    w = synth.small(n_ipp=45, n_ranges=40, seed=41)
    echo, code = w.echo_host(), w.code()
    (tmp_path / "echo.bin").write_bytes(np.ascontiguousarray(echo).tobytes())
    (tmp_path / "code.bin").write_bytes(np.ascontiguousarray(code).tobytes())
    out = tmp_path / "out.bin"
    r = subprocess.run([exe, str(tmp_path / "echo.bin"), str(tmp_path / "code.bin"), str(out), str(w.nfft),
                        str(w.n_ranges), str(w.range_step), str(w.n_ipp), str(w.echo_stride)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, f"c_client exit {r.returncode}: {r.stderr}"
    got = np.fromfile(out, dtype=np.float32).reshape(w.n_ranges, w.nfft).astype(np.float64)
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    assert_parity(got, ref, rtol=RTOL, what="C client")
