"""Batches of links (egn_batch_* / egn_nli_eta_batch): the same kernels as the
single-link path, so every channel must equal the single-link result bit for
bit; the batch is a snapshot of its links; graph replays are repeatable; and
seeded heterogeneous links evaluated inside a batch agree with the FP64 CPU
oracle (FP64 within 1e-9 relative, FP32C within 1e-3 dB)."""
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


def _workloads(workloads):
    a = workloads.config_small(n_ch=5, gl_order=16)
    b = workloads.config_small(n_ch=3, gl_order=16, n_spans=3)
    c = workloads.table1(n_spans=2, cr=1.12, fmt="16QAM", gl_order=16, n_ch=9)
    d = workloads.config_small(n_ch=4, gl_order=16, n_spans=3)  # spans that differ (Eq. 22 span by span)
    d.spans[1].alpha_db_km = 0.16
    d.spans[1].D_ps_nm_km = 21.0
    d.spans[2].length_m = 57e3
    e = workloads.config_small(n_ch=1, gl_order=16)
    f = workloads.config_small(n_ch=3, gl_order=16, n_spans=6)  # six span types: the span-by-span path
    for i, s in enumerate(f.spans):
        s.length_m = (60 + 7 * i) * 1e3
    return [a, b, c, d, e, f]


@pytest.mark.parametrize("prec", ["fp32c", "fp64"])
def test_batch_equals_single_links(egn, workloads, prec):
    p = egn.EGN_PREC_FP32C if prec == "fp32c" else egn.EGN_PREC_FP64
    opts = egn.make_opts(gl_order=16, precision=p)
    links = [egn.link_from_workload(w) for w in _workloads(workloads)]
    want = [ln.nli_eta(opts) for ln in links]
    b = egn.Batch(links, opts)
    assert list(np.diff(b.offsets)) == [ln.n_ch for ln in links]
    first = b.read()  # the validating run of egn_batch_create
    b.launch()
    got = b.read()
    for (ge, gp), (fe, fp), (we, wp) in zip(got, first, want):
        assert np.array_equal(ge, we) and np.array_equal(gp, wp)
        assert np.array_equal(fe, we)
    one = egn.nli_eta_batch(links, opts)
    for (oe, op), (we, wp) in zip(one, want):
        assert np.array_equal(oe, we) and np.array_equal(op, wp)
    b.close()


def test_batch_is_a_snapshot(egn, workloads):
    import torch
    opts = egn.make_opts(gl_order=16)
    wls = _workloads(workloads)
    links = [egn.link_from_workload(w) for w in wls]
    want = [ln.nli_eta(opts) for ln in links]
    b = egn.Batch(links, opts)
    # change link 0's comb (new powers) and destroy link 1: the batch keeps its copies
    w0 = wls[0]
    links[0].set_wdm(w0.centre_hz, w0.symbol_rate_baud, [2 * x for x in w0.launch_power_w],
                     *zip(*[egn.egn_format_moments(f) for f in w0.formats]), w0.rolloff)
    links[1].close()
    s = torch.cuda.Stream()
    for _ in range(3):
        b.launch(s.cuda_stream)
    got = b.read(s.cuda_stream)
    for (ge, gp), (we, wp) in zip(got, want):
        assert np.array_equal(ge, we) and np.array_equal(gp, wp)
    # the changed link itself now gives a different answer
    e0, _ = links[0].nli_eta(opts)
    assert not np.allclose(e0, want[0][0])
    b.close()


class _DeviceArray:
    """A float64 device array at a raw address, viewable by torch.as_tensor."""

    def __init__(self, addr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (addr, False), "version": 3}


def test_batch_device_outputs(egn, workloads):
    import torch
    opts = egn.make_opts(gl_order=16)
    links = [egn.link_from_workload(w) for w in _workloads(workloads)[:3]]
    want = [ln.nli_eta(opts) for ln in links]
    b = egn.Batch(links, opts)
    s = torch.cuda.Stream()
    b.launch(s.cuda_stream)
    s.synchronize()
    n = int(b.offsets[-1])
    eta_addr, pnli_addr = b.outputs()
    eta = torch.as_tensor(_DeviceArray(eta_addr, n), device="cuda").cpu().numpy()
    pnli = torch.as_tensor(_DeviceArray(pnli_addr, n), device="cuda").cpu().numpy()
    assert np.array_equal(eta, np.concatenate([w[0] for w in want]))
    assert np.array_equal(pnli, np.concatenate([w[1] for w in want]))
    b.close()


def test_batch_errors(egn, workloads):
    opts = egn.make_opts(gl_order=16)
    with pytest.raises(egn.EgnError) as ei:
        egn.Batch([], opts)
    assert ei.value.status == egn.EGN_E_INVALID_ARG
    bare = egn.Link(workloads.config_small().spans)  # no comb yet
    ok = egn.link_from_workload(workloads.config_small(n_ch=2, gl_order=16))
    with pytest.raises(egn.EgnError) as ei:
        egn.Batch([ok, bare], opts)
    assert ei.value.status == egn.EGN_E_STATE
    with pytest.raises(egn.EgnError) as ei:
        egn.nli_eta_batch([ok], egn.make_opts(gl_order=16, precision=egn.EGN_PREC_FP32C, mu_form=egn.EGN_MU_INTEGRAL))
    assert ei.value.status == egn.EGN_E_UNSUPPORTED


def _cut(wl, n_ch, gl):
    """The first n_ch channels of a workload at a gl x gl rule."""
    import copy
    w = copy.deepcopy(wl)
    w.centre_hz, w.symbol_rate_baud = w.centre_hz[:n_ch], w.symbol_rate_baud[:n_ch]
    w.launch_power_w, w.formats = w.launch_power_w[:n_ch], w.formats[:n_ch]
    w.gl_order = gl
    return w


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_batch_of_random_links_against_oracle(egn, oracle_mod, workloads, prec):
    """Seeded random links (tilted rippled powers, mixed formats) in one batch: 29
    SSMF/PSCF spans of 26 types (span-by-span path), 2 and 3 span types (shared
    c_k tables) and one span (phased-array closed form), cut to 8-12 channels at
    8 x 8 nodes; three channels of each against the oracle."""
    gl = 8
    wls = [_cut(workloads.random_link(2), 10, gl), _cut(workloads.random_link(4), 8, gl),
           _cut(workloads.random_link(19), 12, gl), _cut(workloads.random_link(3), 9, gl)]
    p = egn.EGN_PREC_FP32C if prec == "fp32c" else egn.EGN_PREC_FP64
    opts = egn.make_opts(gl_order=gl, precision=p)
    links = [egn.link_from_workload(w) for w in wls]
    b = egn.Batch(links, opts)
    b.launch()
    got = b.read()
    for w, (eta, _) in zip(wls, got):
        cois = [0, w.n_ch // 2, w.n_ch - 1]
        want, _ = oracle_mod.Problem(w, gl_order=gl).eta(cois)
        if prec == "fp64":
            assert np.allclose(eta[cois], want, rtol=1e-9, atol=0), (w.name, eta[cois], want)
        else:
            assert np.max(np.abs(10 * np.log10(eta[cois] / want))) < 1e-3, (w.name, eta[cois], want)
    b.close()
