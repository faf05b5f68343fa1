"""The FP32 throughput probe behind the FMA-bound roofline (bench.py reports the
dominant launch against it beside the nominal FP32 peak): one launch through the
C ABI, timed with CUDA events on its stream.  A rate within the physically
possible range shows that the chains really execute (a probe the compiler had
emptied would report an impossible rate).  No paper counterpart."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peak_probe_runs_at_a_plausible_rate():
    import torch
    from paper_1411_3656_gb300 import build, ppf
    build.build()
    ppf.load()
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    stream = torch.cuda.current_stream()
    blocks = 2 * props.multi_processor_count
    st, lanes = ppf.ppf_fma_peak(blocks, 20000, stream)
    assert st == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, lanes = ppf.ppf_fma_peak(blocks, 20000, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    assert st == 0 and lanes == blocks * 512 * 20000 * 8 * 2
    rate = lanes / (e0.elapsed_time(e1) / 1e3)
    # 128 FP32 lanes per SM and clock at most; at least a fifth of that at any clock above 400 MHz
    upper = props.multi_processor_count * 128 * 2.2e9
    lower = props.multi_processor_count * 128 * 0.4e9 / 5
    assert lower < rate < upper, (rate, lower, upper)
