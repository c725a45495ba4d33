"""The integer-issue microbenchmark (ts_int_issue_peak), which gives the
roofline's denominator: every instruction kind runs, and its rate is
physically possible, at most 128 lane operations per clock per SM at the
GPU's maximum SM clock (4 SM sub-partitions x 32 lanes), within 5 %."""
import subprocess

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09221_gb300 import build
    build.build()
    import paper_2604_09221_gb300 as e
    e.library()
    return e


def max_sm_mhz():
    out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm",
                          "--format=csv,noheader,nounits"], stdout=subprocess.PIPE, text=True)
    return float(out.stdout.split()[0])


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_int_peak_kind_is_plausible(eng, kind):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * max_sm_mhz() * 1e6
    rate, ms = eng.int_issue_peak(kind, 1 << 12)
    assert ms > 0
    assert 0.05 * bound < rate <= 1.05 * bound, (eng.INT_PEAK_KINDS[kind], rate / bound)


def test_int_peak_rejects_bad_arguments(eng):
    import ctypes
    r = ctypes.c_double()
    assert eng.library().ts_int_issue_peak(4, 16, ctypes.byref(r), None, None) == 1
    assert eng.library().ts_int_issue_peak(0, 0, ctypes.byref(r), None, None) == 1
