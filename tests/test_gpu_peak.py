"""The FP64 FMA-rate probe behind the plain FP64 roofline: a plausible rate
(between a third of and 1.2x the nominal 2 FMA per clock per SM at the maximum
clock), repeatable, and refusing bad arguments."""
import ctypes

import pytest

import paper_2105_12764_gb300 as mgr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def test_fp64_fma_rate_is_plausible_and_repeatable():
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 2 * 2.07e9
    rates = [mgr.fp64_fma_rate(0) for _ in range(3)]
    for r in rates:
        assert nominal / 3 < r < 1.2 * nominal, (r, nominal)
    assert max(rates) / min(rates) < 1.2


def test_fp64_fma_rate_arguments():
    v = ctypes.c_double()
    assert mgr.lib.mgr_fp64_fma_rate(-1, ctypes.byref(v)) == mgr.MGR_EINVAL
    assert mgr.lib.mgr_fp64_fma_rate(torch.cuda.device_count(), ctypes.byref(v)) == mgr.MGR_EINVAL
    assert mgr.lib.mgr_fp64_fma_rate(0, None) == mgr.MGR_EINVAL
