"""The allocation-free entry point, egn_nli_eta_static, through the C ABI.

It exists for callers that cannot call cudaMalloc (device memory owned by another
allocator, online control loops that cannot take the implied synchronisation,
plugin hosts that forbid device allocation); its scratch is a fixed array
compiled into the library.  Its output must equal the output of the existing
entry point, egn_nli_eta_device, with a caller workspace, within the tolerances of
the parity tests (FP64: 1e-9 relative; FP32C: 1e-3 dB), on two calls in a row --
the second call reuses the array with the first call's contents still in it.
"Allocates nothing" is checked with the library's own allocation counter
(egn_allocation_count), which other processes on the GPU cannot disturb, and,
as a second check, with the device's free memory.
This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _reference(egn, ln, opts, n):
    import torch
    ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
    eta = torch.empty(n, dtype=torch.float64, device="cuda")
    pn = torch.empty(n, dtype=torch.float64, device="cuda")
    ln.nli_eta_device(opts, ws, eta, pn)
    torch.cuda.synchronize()
    return eta.cpu().numpy(), pn.cpu().numpy()


def _close(a, b, precision, egn):
    if precision == egn.EGN_PREC_FP64:
        return np.allclose(a, b, rtol=1e-9, atol=0)
    return np.max(np.abs(10 * np.log10(a / b))) < 1e-3


def _typed_link(workloads, n_ch, gl):
    """Spans of three types (60, 67 and 74 km): the shared-table path of Eq. 22."""
    wl = workloads.config_small(n_ch=n_ch, gl_order=gl, n_spans=3)
    for i, s in enumerate(wl.spans):
        s.length_m = (60 + 7 * i) * 1e3
    return wl


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_static_matches_device_api_two_calls(egn, workloads, prec):
    import torch
    precision = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    stream = torch.cuda.Stream()
    # a larger comb first, then a smaller one, then spans of three types: each
    # evaluation runs on scratch that still holds the previous one's islands,
    # terms and tables
    for wl in (workloads.config_small(n_ch=7, gl_order=16, n_spans=3), workloads.config_small(n_ch=4, gl_order=16),
               _typed_link(workloads, 3, 16)):
        n_ch = wl.n_ch
        ln = egn.link_from_workload(wl)
        opts = egn.make_opts(gl_order=16, precision=precision, stream=stream.cuda_stream)
        want_eta, want_pn = _reference(egn, ln, opts, n_ch)
        for call in range(2):
            eta = torch.full((n_ch,), float("nan"), dtype=torch.float64, device="cuda")
            pn = torch.full((n_ch,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            allocs_before = egn.allocation_count()
            free_before = torch.cuda.mem_get_info()[0]
            ln.nli_eta_static(opts, eta, pn)
            stream.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            assert egn.allocation_count() == allocs_before  # the library allocated nothing
            got_eta, got_pn = eta.cpu().numpy(), pn.cpu().numpy()
            assert np.all(np.isfinite(got_eta)), (n_ch, call)
            assert _close(got_eta, want_eta, precision, egn), (n_ch, call, got_eta, want_eta)
            assert _close(got_pn, want_pn, precision, egn), (n_ch, call)
            if call == 1:
                assert free_after >= free_before  # and the device's free memory did not shrink
        ln.close()


def test_static_refuses_oversized_evaluation(egn, workloads):
    import torch
    wl = workloads.config_cl()  # about 97 MB of workspace, beyond the static scratch
    ln = egn.link_from_workload(wl)
    eta = torch.empty(wl.n_ch, dtype=torch.float64, device="cuda")
    pn = torch.empty(wl.n_ch, dtype=torch.float64, device="cuda")
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta_static(egn.make_opts(gl_order=32), eta, pn)
    assert ei.value.status == egn.EGN_E_CAPACITY
    assert "static scratch" in str(ei.value)
    ln.close()


def test_static_refuses_many_span_types(egn, workloads):
    import torch
    wl = workloads.config_small(n_ch=2, gl_order=8, n_spans=5)
    for i, s in enumerate(wl.spans):
        s.length_m = (60 + 7 * i) * 1e3
    ln = egn.link_from_workload(wl)
    eta = torch.empty(2, dtype=torch.float64, device="cuda")
    pn = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta_static(egn.make_opts(gl_order=8), eta, pn)
    assert ei.value.status == egn.EGN_E_UNSUPPORTED
    ln.close()
