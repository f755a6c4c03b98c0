"""The debug build of the library (-DISR_DEBUG): every gate of every fused kernel checks that
its staged window copy lies inside its echo row and fits the stage buffer before it issues
the copy, and reports a failed check as ISR_ERR_OUT_OF_RANGE (never a trap or a fault).

* CPU: the debug library compiles for sm_103a and exports every declared entry point.
* GPU: with valid inputs only, the debug build gives the same spectra as the oracle for
  every kernel family (several gates per warp, per-gate named barriers, one gate per CTA in
  each radix order), i.e. no check fires on a valid geometry; its phase-cycle tracing
  (isr_plan_phase_cycles) reports every phase of the Stockham kernels, and the release build
  refuses the call.
"""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_2311_18737_gb300 import _build, isr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_library_builds_and_exports():
    lib_path = _build.build(debug=True)
    assert lib_path.endswith("libisr_debug.so") and os.path.exists(lib_path)
    lib = ctypes.CDLL(lib_path)
    for name in isr.EXPORTS:
        assert hasattr(lib, name), f"{name} missing from the debug build"


CHILD = r"""
import numpy as np
import oracle, synth
from gpu_helpers import RTOL, assert_parity, gpu_integrate
from paper_2311_18737_gb300 import isr
assert isr.LIB_PATH.endswith("libisr_debug.so"), isr.LIB_PATH
cases = [(256, 24, 0), (1024, 20, 0), (4096, 9, 0), (16384, 3, 0), (16384, 3, 1), (16384, 3, 3), (16384, 3, 5)]
for nfft, n_ranges, order in cases:
    w = synth.small(nfft=nfft, code_len=nfft, n_ranges=n_ranges, n_ipp=9, range_start=3, seed=51 + nfft,
                    echo_stride=((3 + (n_ranges - 1) * 25 + nfft + 127) // 128) * 128)
    echo, code = w.echo_host(), w.code()
    ref = oracle.integrate(echo, code, nfft=nfft, n_ranges=n_ranges, range_start=3, range_step=25)
    import torch
    dev = torch.device("cuda:0")
    with isr.Plan(nfft=nfft, n_ranges=n_ranges, echo_stride=w.echo_stride, range_start=3, range_step=25,
                  tx_type=isr.ISR_TX_PM1, device=0) as plan:
        if order:
            isr.isr_plan_set_order(plan.handle, order)
        plan.integrate(torch.from_numpy(echo).to(dev), torch.from_numpy(code).to(dev), w.n_ipp)
        out = torch.empty((n_ranges, nfft), dtype=torch.float32, device=dev)
        plan.spectra(out)
        cyc = isr.isr_plan_phase_cycles(plan.handle)
    # the Stockham kernels record their phases (thread 0 of each CTA); the warp-local and paired
    # orders do not
    stockham = order in (0, 1, 2) or nfft < 16384
    if stockham:
        assert cyc[4] > 0 and min(cyc[:2]) > 0 and cyc[3] > 0, (nfft, order, cyc)
        assert sum(cyc[:4]) / cyc[4] < 1e7, (nfft, order, cyc)   # cycles per IPP and CTA, sane
    else:
        assert cyc == [0, 0, 0, 0, 0], (nfft, order, cyc)
    assert_parity(out.cpu().numpy().astype(np.float64), ref, rtol=RTOL, what=f"debug build nfft {nfft} order {order}")
print("debug build parity ok")
"""


@pytest.mark.gpu
def test_debug_build_parity_on_valid_inputs():
    lib_path = _build.build(debug=True)
    env = dict(os.environ, ISR_LIBRARY=lib_path)
    env["PYTHONPATH"] = os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), env.get("PYTHONPATH", "")])
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, timeout=900, cwd=ROOT)
    assert r.returncode == 0, f"debug-build child failed:\n{r.stdout[-2000:]}\n{r.stderr[-4000:]}"
    assert "debug build parity ok" in r.stdout


@pytest.mark.gpu
def test_release_build_refuses_phase_cycles():
    torch = pytest.importorskip("torch")
    with isr.Plan(nfft=256, n_ranges=4, echo_stride=384, range_step=25, tx_type=isr.ISR_TX_PM1, device=0) as plan:
        out = (ctypes.c_uint64 * 5)()
        assert isr.load_library().isr_plan_phase_cycles(plan.handle, out) == isr.ISR_ERR_UNSUPPORTED
