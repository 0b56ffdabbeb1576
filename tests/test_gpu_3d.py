"""f-integrated (3-D) EGN through egn_nli_eta_3d against the oracle's eta_3d: the
integral over f of Eq. 17-21 by an n_f-point Gauss-Legendre rule, each node a
full evaluation with the islands planned at that COI frequency.

Bars: FP64 within 1e-9 relative (as every FP64 parity test), FP32C within
1e-3 dB (as the small FP32C cases); n_f = 1 is the white-NLI evaluation bit for
bit (the COI frequency arrays then equal the centres)."""
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


PRECS = [("fp64", 0), ("fp32c", 1)]


def _mixed_rates(workloads):
    """Gaussian-format channels of 32 and 64 GBd on an irregular grid (GN terms)."""
    wl = workloads.config_small(n_ch=4, gl_order=16, fmt="GAUSS")
    c = wl.centre_hz[2]
    wl.centre_hz = [c - 120e9, c - 62e9, c, c + 49e9]
    wl.symbol_rate_baud = [64e9, 32e9, 64e9, 32e9]
    wl.launch_power_w = [1e-3, 0.5e-3, 1.2e-3, 0.8e-3]
    return wl


@pytest.mark.parametrize("name,prec", PRECS)
def test_one_node_equals_white_nli(egn, workloads, name, prec):
    ln = egn.link_from_workload(workloads.config_small(n_ch=3, gl_order=16, n_spans=2))
    opts = egn.make_opts(gl_order=16, precision=prec)
    e2, p2 = ln.nli_eta(opts)
    e1, p1 = ln.nli_eta_3d(opts, 1)
    assert np.array_equal(e1, e2) and np.array_equal(p1, p2)
    ln.close()


@pytest.mark.parametrize("name,prec", PRECS)
@pytest.mark.parametrize("case", ["qam_3ch", "mixed_rates"])
def test_against_oracle(egn, oracle_mod, workloads, name, prec, case):
    if case == "qam_3ch":
        wl, n_f, terms = workloads.config_small(n_ch=3, gl_order=16, n_spans=2), 3, 1
    else:
        wl, n_f, terms = _mixed_rates(workloads), 4, 0
    want, _ = oracle_mod.Problem(wl, gl_order=16, terms=terms).eta_3d(n_f)
    ln = egn.link_from_workload(wl)
    got, _ = ln.nli_eta_3d(egn.make_opts(gl_order=16, precision=prec, terms=terms), n_f)
    if prec == 0:
        assert np.allclose(got, want, rtol=1e-9, atol=0), got / want - 1
    else:
        assert np.max(np.abs(10 * np.log10(got / want))) < 1e-3
    # the link's own plan is restored: the white-NLI call afterwards is unchanged
    white, _ = ln.nli_eta(egn.make_opts(gl_order=16, precision=prec, terms=terms))
    want2, _ = oracle_mod.Problem(wl, gl_order=16, terms=terms).eta()
    if prec == 0:
        assert np.allclose(white, want2, rtol=1e-9, atol=0)
    else:
        assert np.max(np.abs(10 * np.log10(white / want2))) < 1e-3
    ln.close()


def test_refused_node_counts(egn, workloads):
    ln = egn.link_from_workload(workloads.config_small(n_ch=2, gl_order=8))
    for nf in (0, 65):
        with pytest.raises(egn.EgnError) as ei:
            ln.nli_eta_3d(egn.make_opts(gl_order=8), nf)
        assert ei.value.status == egn.EGN_E_INVALID_ARG
    ln.close()
