"""The arithmetic-pipe probes (include/egn_probe.h) that give the integrator's
roofline its measured denominators.  A probe whose work the compiler dropped
would report rates far above what the hardware can do, so every rate must lie
below the GB300's nominal per-SM width at its maximum clock (FP32 FMA: 128 lanes
x 2 FLOP; FP64 FMA: 2 lanes x 2 FLOP; MUFU: 16 operations per SM per clock,
32 for the base-2 exponential, whose unit GB300 doubles; the mix of packed and
scalar FP32 FMAs: twice the FP32 width, the most two separate pipes could give)
and above a quarter of it, and the sinks must hold finite chain values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_MHZ = 2070.0
SLACK = 1.05  # clock reading and event resolution


@pytest.fixture(scope="module")
def egn():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2412_11614_gb300 import _build
    _build.build()
    from paper_2412_11614_gb300 import egn as E
    E.lib()
    return E


@pytest.mark.parametrize("kind,per_sm_clk,iters", [("ffma", 256, 20000), ("ffma2", 256, 10000),
                                                   ("dfma", 4, 300), ("mufu_sin", 16, 4000),
                                                   ("mufu_ex2", 32, 4000), ("mufu_rcp", 16, 4000),
                                                   ("fma_mix", 512, 6000)])
def test_probe_rate_is_physical(egn, kind, per_sm_clk, iters):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.full((blocks * threads,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    egn.probe_launch(kind, blocks, threads, iters, sink, st.cuda_stream)  # warm-up
    best = None
    with torch.cuda.stream(st):
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            egn.probe_launch(kind, blocks, threads, iters, sink, st.cuda_stream)
            e1.record(st)
            e1.synchronize()
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
    rate = egn.probe_ops(kind, blocks, threads, iters) / (best * 1e-3)
    ceiling = sms * per_sm_clk * MAX_MHZ * 1e6
    assert rate < SLACK * ceiling, (kind, rate, ceiling)
    assert rate > 0.25 * ceiling, (kind, rate, ceiling)
    assert np.all(np.isfinite(sink.cpu().numpy()))


def test_probe_refuses_bad_arguments(egn):
    import torch
    sink = torch.empty(32, dtype=torch.float64, device="cuda")
    for kind, blocks, threads, iters in (("ffma", 1, 48, 1), ("ffma", 0, 32, 1), ("ffma", 1, 2048, 1),
                                         ("ffma", 1, 32, 0)):
        with pytest.raises(egn.EgnError) as ei:
            egn.probe_launch(kind, blocks, threads, iters, torch.empty(blocks * max(threads, 1) + 32,
                                                                       dtype=torch.float64, device="cuda"))
        assert ei.value.status == egn.EGN_E_INVALID_ARG
    with pytest.raises(ValueError):
        egn.probe_launch("ffma", 2, 32, 1, sink)  # sink smaller than blocks x threads doubles
