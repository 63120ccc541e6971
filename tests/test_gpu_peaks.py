"""The arithmetic throughput loops behind the measured ALU peaks (gr_peak_alu): a launch reports the
floating-point operations it performs, and the GPU's FP32 rate is far above its FP64 rate."""
import pytest

from paper_2311_04989_gb300 import grstage as G

pytestmark = pytest.mark.gpu


def test_peak_loops_count_and_rank_the_pipes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_04989_gb300 import build as B
    B.build()
    sink = torch.zeros(64, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    rates = {}
    for kind, per_fma in ((0, 2), (1, 4), (2, 2)):
        iters = 1 << (14 if kind < 2 else 10)
        fl = G.gr_peak_alu(kind, 64, 128, iters, sink, s)
        assert fl == 64 * 128 * iters * 16 * per_fma
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        G.gr_peak_alu(kind, 64, 128, iters, sink, s)
        e1.record(s)
        torch.cuda.synchronize()
        rates[kind] = fl / e0.elapsed_time(e1)
    assert float(sink.abs().sum()) == 0.0      # the guarded store never fires
    assert rates[0] > 8 * rates[2] and rates[1] > 8 * rates[2], rates
    with pytest.raises(G.GrstageError):
        G.gr_peak_alu(3, 64, 128, 1, sink, s)
