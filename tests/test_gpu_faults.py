"""Failure detection without a device fault: host-side injected failures
(EGN_FAULT=alloc|h2d|launch) and the host wait limit (opts.timeout_ms).

Every failure is made on the host before anything reaches the device, or is a
wait that gives up while the device work completes normally, so no test faults,
traps or hangs the GPU.  Each test checks the status, then clears the cause and
checks that the same link evaluates bit for bit like one that never failed."""
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


def _wl(workloads):
    return workloads.config_small(n_ch=4, gl_order=16, n_spans=2)


def _opts(egn, **kw):
    kw.setdefault("gl_order", 16)
    kw.setdefault("precision", egn.EGN_PREC_FP32C)
    return egn.make_opts(**kw)


@pytest.fixture(scope="module")
def want(egn, workloads):
    """Reference results of links that never saw a failure, at dz 1 and 0.5 km."""
    ln = egn.link_from_workload(_wl(workloads))
    out = {dz: ln.nli_eta(_opts(egn, dz_km=dz)) for dz in (1.0, 0.5)}
    ln.close()
    return out


def _set_wdm(egn, ln, wl):
    mom = [egn.egn_format_moments(f) for f in wl.formats]
    ln.set_wdm(wl.centre_hz, wl.symbol_rate_baud, wl.launch_power_w, [m[0] for m in mom], [m[1] for m in mom],
               wl.rolloff)


def _expect(egn, status, fn, *args):
    with pytest.raises(egn.EgnError) as ei:
        fn(*args)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


def _same(got, ref):
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("kind,status", [("alloc", 3), ("h2d", 4)])
def test_set_wdm_failure_leaves_link_reusable(egn, workloads, want, monkeypatch, kind, status):
    wl = _wl(workloads)
    ln = egn.Link(wl.spans)
    monkeypatch.setenv("EGN_FAULT", kind)
    _expect(egn, status, _set_wdm, egn, ln, wl)
    _expect(egn, egn.EGN_E_STATE, ln.nli_eta, _opts(egn))  # no WDM set
    monkeypatch.delenv("EGN_FAULT")
    _set_wdm(egn, ln, wl)
    _same(ln.nli_eta(_opts(egn)), want[1.0])
    ln.close()


@pytest.mark.parametrize("kind,status", [("alloc", 3), ("h2d", 4)])
def test_table_rebuild_failure_keeps_link(egn, workloads, want, monkeypatch, kind, status):
    """A new dz needs larger segment tables (K = 160 instead of 80): the
    allocation or the upload fails, the link keeps working afterwards."""
    ln = egn.link_from_workload(_wl(workloads))
    _same(ln.nli_eta(_opts(egn, dz_km=1.0)), want[1.0])
    monkeypatch.setenv("EGN_FAULT", kind)
    msg = _expect(egn, status, ln.nli_eta, _opts(egn, dz_km=0.5))
    assert ("ensure" in msg) if kind == "alloc" else ("h2d" in msg)
    if kind == "alloc":  # the dz 1 km tables fit the buffer that was kept: nothing to allocate
        _same(ln.nli_eta(_opts(egn, dz_km=1.0)), want[1.0])
    else:  # the tables were invalidated and must be uploaded again
        _expect(egn, status, ln.nli_eta, _opts(egn, dz_km=1.0))
    monkeypatch.delenv("EGN_FAULT")
    _same(ln.nli_eta(_opts(egn, dz_km=0.5)), want[0.5])
    _same(ln.nli_eta(_opts(egn, dz_km=1.0)), want[1.0])
    ln.close()


def test_launch_failure(egn, workloads, want, monkeypatch):
    ln = egn.link_from_workload(_wl(workloads))
    monkeypatch.setenv("EGN_FAULT", "launch")
    msg = _expect(egn, egn.EGN_E_CUDA, ln.nli_eta, _opts(egn))
    assert "EGN_LAUNCH_GATE" in msg or "inject" in msg
    _expect(egn, egn.EGN_E_CUDA, ln.island_terms, _opts(egn), np.array([[0, 0, 0, 0]], dtype=np.int32))
    _expect(egn, egn.EGN_E_CUDA, egn.Batch, [ln], _opts(egn))
    monkeypatch.setenv("EGN_FAULT", "launch,alloc")
    _expect(egn, egn.EGN_E_CUDA, ln.nli_eta, _opts(egn))  # the workspace is kept, so launch fails first
    monkeypatch.delenv("EGN_FAULT")
    _same(ln.nli_eta(_opts(egn)), want[1.0])
    b = egn.Batch([ln], _opts(egn))
    b.launch()
    [(eta, pnli)] = b.read()
    _same((eta, pnli), want[1.0])
    b.close()
    ln.close()


def test_unknown_fault_names_are_ignored(egn, workloads, want, monkeypatch):
    ln = egn.link_from_workload(_wl(workloads))
    monkeypatch.setenv("EGN_FAULT", "none,,allocx")
    _same(ln.nli_eta(_opts(egn)), want[1.0])
    ln.close()


def test_timeout_then_reuse(egn, workloads):
    """A 120-channel evaluation (about 20 ms of device work) with a 1 ms host
    wait limit returns EGN_E_TIMEOUT while the device work completes normally;
    the next call on the same stream is ordered after it and returns the same
    result as a call that never timed out."""
    wl = workloads.config_cl(n_ch=120)
    ln = egn.link_from_workload(wl)
    opts = _opts(egn, gl_order=32, terms=egn.EGN_TERMS_GN)
    ref = ln.nli_eta(opts)
    _expect(egn, egn.EGN_E_TIMEOUT, ln.nli_eta, _opts(egn, gl_order=32, terms=egn.EGN_TERMS_GN, timeout_ms=1))
    _same(ln.nli_eta(opts), ref)
    ln.close()
