"""The rate probes behind the rooflines (needs a GPU): the FMA-rate probe (the execute
kernels' arithmetic bound) and the distributed-shared-memory probe (the cross stage's bound)
return plausible figures and reject bad arguments."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdh():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1604_07486_gb300 as m
    from paper_1604_07486_gb300 import build
    build.build()
    return m


def test_fma_rate(tdh):
    """FP32 above FP64, both positive and below what 2 flops x 256 lanes x 3 GHz per SM
    could give."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = tdh.measure_fma_rate("fp32")
    f64 = tdh.measure_fma_rate("fp64")
    cap = 2 * 256 * 3.0e9 * sms / 1e12
    assert 0 < f64 < f32 < cap, (f32, f64, cap)
    with pytest.raises(tdh.TdhError):
        tdh.measure_fma_rate(7)


def test_dsmem_rate(tdh):
    """Remote shared-memory throughput per SM and cycle: positive and below 128 bytes (the
    width of one shared-memory access per cycle) in each direction."""
    r = tdh.measure_dsmem_rate()
    for key in ("loads", "stores", "loads_one_cluster"):
        assert 0 < r[key] < 128, r
    assert 0 < r["both"] < 256, r
    assert tdh.lib().tdh_measure_dsmem_rate(None, None) == -1
