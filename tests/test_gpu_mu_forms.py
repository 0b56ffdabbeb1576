"""GPU parity of the three forms of the FWM efficiency mu (FP64 path) against the
oracle's independent routines:
  * Maclaurin closed form, Eq. 4-6;
  * integral form, Eq. 23 integrated numerically (the paper's reference);
  * segment closed form, Eq. 7-10 (covered in test_gpu_parity.py).

Tolerance: 1e-9 relative for the closed forms (both sides FP64).  The integral
form uses the same piece layout on both sides (equal pieces of at most a
quarter period) but a fixed 10-point rule per piece on the GPU against the
oracle's adaptive bisection to 1e-10: 1e-9 relative as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-9


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


def _opts(egn, gl, form, terms=1):
    return egn.make_opts(gl_order=gl, precision=egn.EGN_PREC_FP64, terms=terms, mu_form=form)


@pytest.mark.parametrize("terms", [0, 1])
def test_maclaurin_eta_small(egn, oracle_mod, workloads, terms):
    wl = workloads.config_small(gl_order=32)
    ln = egn.link_from_workload(wl)
    got, gp = ln.nli_eta(_opts(egn, 32, egn.EGN_MU_MACLAURIN, terms))
    want, wp = oracle_mod.Problem(wl, gl_order=32, terms=terms, mu_form=oracle_mod.MU_MACLAURIN).eta()
    assert np.allclose(got, want, rtol=RTOL, atol=0), got / want - 1
    assert np.allclose(gp, wp, rtol=RTOL, atol=0)


def test_maclaurin_strong_isrs_multispan(egn, oracle_mod, workloads):
    """Table I at Cr = 1.12 (the paper's high-ISRS case), 3 spans, 7 channels of
    the 101-channel grid around the centre."""
    wl = workloads.table1(n_spans=3, cr=1.12, fmt="QPSK", gl_order=12, n_ch=7)
    ln = egn.link_from_workload(wl)
    got, _ = ln.nli_eta(_opts(egn, 12, egn.EGN_MU_MACLAURIN))
    want, _ = oracle_mod.Problem(wl, gl_order=12, mu_form=oracle_mod.MU_MACLAURIN).eta()
    assert np.allclose(got, want, rtol=RTOL, atol=0), got / want - 1


def test_maclaurin_heterogeneous_spans(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=3, gl_order=10, n_spans=3)
    wl.spans[1].alpha_db_km = 0.16
    wl.spans[1].D_ps_nm_km = 21.0
    wl.spans[2].length_m = 61e3
    ln = egn.link_from_workload(wl)
    got, _ = ln.nli_eta(_opts(egn, 10, egn.EGN_MU_MACLAURIN))
    want, _ = oracle_mod.Problem(wl, gl_order=10, mu_form=oracle_mod.MU_MACLAURIN).eta()
    assert np.allclose(got, want, rtol=RTOL, atol=0), got / want - 1


def test_integral_island_terms(egn, oracle_mod, workloads):
    """Every term on every island of a 3-channel comb, 6 x 6 nodes."""
    wl = workloads.config_small(n_ch=3, gl_order=6)
    ln = egn.link_from_workload(wl)
    pb = oracle_mod.Problem(wl, gl_order=6, mu_form=oracle_mod.MU_INTEGRAL)
    isl = np.array([(n, *t) for n in range(3) for t in pb.islands(n)], dtype=np.int32)
    got = ln.island_terms(_opts(egn, 6, egn.EGN_MU_INTEGRAL), isl, all_terms=True)
    want = np.array([pb.island_terms(*row, all_terms=True) for row in isl])
    assert np.allclose(got, want, rtol=RTOL, atol=1e-300), np.max(np.abs(got / np.where(want == 0, 1, want) - 1))


def test_integral_eta_two_spans(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=2, gl_order=6, n_spans=2)
    ln = egn.link_from_workload(wl)
    got, _ = ln.nli_eta(_opts(egn, 6, egn.EGN_MU_INTEGRAL))
    want, _ = oracle_mod.Problem(wl, gl_order=6, mu_form=oracle_mod.MU_INTEGRAL).eta()
    assert np.allclose(got, want, rtol=RTOL, atol=0), got / want - 1


def test_forms_agree_without_isrs(egn, workloads):
    """Cr = 0: the segment sum telescopes to the lossy closed form (Eq. 6), the
    Maclaurin correction vanishes and the integral is that closed form too."""
    wl = workloads.config_small(n_ch=3, gl_order=8, n_spans=2)
    for s in wl.spans:
        s.cr_per_w_km_thz = 0.0
    ln = egn.link_from_workload(wl)
    seg, _ = ln.nli_eta(_opts(egn, 8, egn.EGN_MU_SEGMENT))
    mac, _ = ln.nli_eta(_opts(egn, 8, egn.EGN_MU_MACLAURIN))
    itg, _ = ln.nli_eta(_opts(egn, 8, egn.EGN_MU_INTEGRAL))
    assert np.allclose(mac, seg, rtol=1e-11, atol=0)
    assert np.allclose(itg, seg, rtol=RTOL, atol=0)


def test_closed_forms_fp32c_unsupported(egn, workloads):
    wl = workloads.config_small(n_ch=2, gl_order=8)
    ln = egn.link_from_workload(wl)
    for form in (egn.EGN_MU_MACLAURIN, egn.EGN_MU_INTEGRAL):
        with pytest.raises(egn.EgnError) as ei:
            ln.nli_eta(egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP32C, mu_form=form))
        assert ei.value.status == egn.EGN_E_UNSUPPORTED
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP64, mu_form=7))
    assert ei.value.status == egn.EGN_E_INVALID_ARG
