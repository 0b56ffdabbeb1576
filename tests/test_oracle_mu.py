"""Pins of the FWM efficiency factor mu (Eq. 2-10, 23-25) and the link function
(Eq. 22) in the oracle."""
import cmath
import math

import numpy as np
import pytest
from scipy import integrate

A = 0.2 * math.log(10) / 10  # 1/km


def known_mu_lin(chi, alpha, L):
    """Textbook FWM efficiency without ISRS: |mu|^2 = |1 - e^{(-alpha + i chi) L}|^2 / |alpha - i chi|^2."""
    return (1 - cmath.exp((-alpha + 1j * chi) * L)) / (alpha - 1j * chi)


@pytest.fixture
def span(oracle_mod):
    def mk(cr=0.0, L=80.0, alpha=A):
        return oracle_mod.make_span(alpha, -21.68, 0.1447, 1.3, cr, L)
    return mk


@pytest.mark.parametrize("chi", [0.0, 0.37, 3.7, 55.0, 1700.0])
def test_cr0_all_forms_reduce_to_known_closed_form(oracle_mod, span, chi):
    s = span(cr=0.0)
    ref = known_mu_lin(chi, A, 80.0)
    assert abs(oracle_mod.mu_lin(chi, A, 80.0) - ref) <= 1e-13 * abs(ref) + 1e-15
    for K in (1, 7, 80, 333):
        assert abs(oracle_mod.mu_segment(chi, 1.3, s, 0.19, 9.0, K) - ref) <= 1e-11 * abs(ref) + 1e-14
    assert abs(oracle_mod.mu_maclaurin(chi, 1.3, s, 0.19) - ref) <= 1e-13 * abs(ref) + 1e-15
    if chi < 100:
        assert abs(oracle_mod.mu_integral(chi, 1.3, s, 0.19, 9.0) - ref) <= 1e-9 * abs(ref)


def test_peak_is_effective_length(oracle_mod, span):
    # Fig. 3: at f1 = f2 = f and Cr = 0 the efficiency factor mu / L_eff is 1
    s = span(cr=0.0)
    mu = oracle_mod.mu_segment(0.0, 0.0, s, 0.19, 9.0, 80)
    assert mu.real / oracle_mod.leff(A, 80.0) == pytest.approx(1.0, rel=1e-14)
    assert abs(mu.imag) < 1e-15


def integral_by_scipy(chi, f3, alpha, ptot, cr, btot, L):
    """Eq. 23 by scipy's QUADPACK (an integrator independent of the oracle's)."""
    def rho(z):
        zeta = ptot * cr * (-math.expm1(-alpha * z) / alpha)
        x = btot * zeta
        g = 1.0 if x == 0 else x * math.exp(-zeta * f3) / (2 * math.sinh(x / 2))
        return g * math.exp(-alpha * z)
    lim = 2000
    re, _ = integrate.quad(lambda z: rho(z), 0, L, weight="cos", wvar=chi, limit=lim) if chi else integrate.quad(rho, 0, L)
    im, _ = integrate.quad(lambda z: rho(z), 0, L, weight="sin", wvar=chi, limit=lim) if chi else (0.0, 0.0)
    return complex(re, im)


@pytest.mark.parametrize("chi,f3,cr", [(0.0, 2.3, 0.028), (0.9, -3.1, 0.028), (3.7, 2.3, 0.028),
                                       (40.0, 0.45, 1.12 * 0.0794 / 0.19), (150.0, -4.0, 0.028)])
def test_integral_form_matches_independent_quadrature(oracle_mod, span, chi, f3, cr):
    s = span(cr=cr)
    got = oracle_mod.mu_integral(chi, f3, s, 0.19, 9.0)
    ref = integral_by_scipy(chi, f3, A, 0.19, cr, 9.0, 80.0)
    assert abs(got - ref) <= 1e-8 * abs(ref)


def test_chi0_integral_by_change_of_variables(oracle_mod, span):
    """At chi = 0, int rho dz = (1/(P Cr)) int_0^{zeta_L} B zeta e^{-zeta f}/(2 sinh(B zeta / 2)) dzeta
    (substituting zeta = P Cr L_eff(z), d zeta = P Cr e^{-alpha z} dz)."""
    p, cr, B, f3 = 0.19, 0.028, 9.0, 3.3
    s = span(cr=cr)
    zL = p * cr * oracle_mod.leff(A, 80.0)
    val, _ = integrate.quad(lambda x: B * x * math.exp(-x * f3) / (2 * math.sinh(B * x / 2)) if x else 1.0, 0, zL)
    assert oracle_mod.mu_integral(0.0, f3, s, p, B).real == pytest.approx(val / (p * cr), rel=1e-10)


def test_segment_telescopes_at_cr0(oracle_mod, span):
    # sum_k I_k = mu_lin for any K (Eq. 9)
    s = span(cr=0.0)
    for chi in (0.2, 12.0, 400.0):
        ref = oracle_mod.mu_lin(chi, A, 80.0)
        for K in (2, 3, 80, 1000):
            assert abs(oracle_mod.mu_segment(chi, -2.0, s, 0.19, 9.0, K) - ref) <= 1e-11 * abs(ref)


def test_segment_converges_second_order_at_small_phase_step(oracle_mod, span):
    """Midpoint-envelope segments: error O(K^-2) while chi L / K is small."""
    s = span(cr=0.028)
    chi, f3 = 0.3, 3.0
    ref = oracle_mod.mu_integral(chi, f3, s, 0.19, 9.0, 1e-12)
    errs = [abs(oracle_mod.mu_segment(chi, f3, s, 0.19, 9.0, K) - ref) for K in (40, 80, 160, 320)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    for r in ratios:
        assert 3.6 < r < 4.4, ratios


def test_segment_converges_to_integral(oracle_mod, span):
    s = span(cr=0.028)
    for chi, f3 in [(3.7, 2.3), (150.0, -4.0)]:
        ref = oracle_mod.mu_integral(chi, f3, s, 0.19, 9.0, 1e-12)
        e1 = abs(oracle_mod.mu_segment(chi, f3, s, 0.19, 9.0, 80) - ref)
        e2 = abs(oracle_mod.mu_segment(chi, f3, s, 0.19, 9.0, 8000) - ref)
        assert e2 < 0.02 * e1


def test_maclaurin_error_is_second_order_in_cr(oracle_mod, span):
    """Eq. 3 keeps first order in zeta f and second order of the sinh: the error vs the
    exact integral scales as Cr^2."""
    chi, f3 = 0.0, 3.0
    errs = []
    for cr in (0.014, 0.007, 0.0035):
        s = span(cr=cr)
        ref = oracle_mod.mu_integral(chi, f3, s, 0.19, 9.0, 1e-12)
        errs.append(abs(oracle_mod.mu_maclaurin(chi, f3, s, 0.19) - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, (r1, r2)


def test_maclaurin_first_order_in_cr_exact(oracle_mod, span):
    # d mu / d Cr at Cr = 0 of the Maclaurin form equals that of the integral form
    chi, f3, h = 2.0, 1.7, 1e-6
    s0, s1 = span(cr=0.0), span(cr=h)
    dm = (oracle_mod.mu_maclaurin(chi, f3, s1, 0.19) - oracle_mod.mu_maclaurin(chi, f3, s0, 0.19)) / h
    di = (oracle_mod.mu_integral(chi, f3, s1, 0.19, 9.0, 1e-13) - oracle_mod.mu_integral(chi, f3, s0, 0.19, 9.0, 1e-13)) / h
    assert abs(dm - di) <= 1e-4 * abs(di)


# --------------------------------------------------------------------------- Eq. 22

def _link_problem(oracle_mod, workloads, n_spans, **kw):
    wl = workloads.config_small(n_ch=3, n_spans=n_spans)
    for s in wl.spans:
        for k, v in kw.items():
            setattr(s, k, v)
    return oracle_mod.Problem(wl)


@pytest.mark.parametrize("n_spans", [1, 2, 5, 10, 30])
def test_identical_spans_phased_array(oracle_mod, workloads, n_spans):
    """For identical spans Eq. 22 is a geometric series:
    Y = gamma mu e^{i (N-1) phi / 2} sin(N phi / 2) / sin(phi / 2), phi = chi L."""
    pb1 = _link_problem(oracle_mod, workloads, 1)
    pbN = _link_problem(oracle_mod, workloads, n_spans)
    sp = pb1.spans[0]
    rng = np.random.default_rng(1)
    for _ in range(20):
        f1, f2, f = rng.uniform(-0.1, 0.1, 3)
        y1 = pb1.upsilon(f1, f2, f)
        chi = oracle_mod.chi(f1, f2, f, sp.beta2, sp.beta3)
        phi = chi * sp.L
        af = cmath.exp(1j * (n_spans - 1) * phi / 2) * math.sin(n_spans * phi / 2) / math.sin(phi / 2)
        yN = pbN.upsilon(f1, f2, f)
        assert abs(yN - y1 * af) <= 1e-8 * abs(y1) * max(1.0, abs(af))


def test_phased_array_peak(oracle_mod, workloads):
    # phi -> 0: array factor -> N
    pb1 = _link_problem(oracle_mod, workloads, 1)
    pb7 = _link_problem(oracle_mod, workloads, 7)
    y1 = pb1.upsilon(0.03, 0.0, 0.0)
    y7 = pb7.upsilon(0.03, 0.0, 0.0)
    assert abs(y7 - 7 * y1) <= 1e-14 * abs(y7)


def test_heterogeneous_spans_sum(oracle_mod, workloads):
    """Two different spans: Y = g1 mu1 + g2 mu2 e^{i chi1 L1} (Eq. 22 written out)."""
    from oracle.oracle import OrSpan
    wl = workloads.config_small(n_ch=3, n_spans=2)
    wl.spans[1].length_m = 55e3
    wl.spans[1].alpha_db_km = 0.16
    wl.spans[1].D_ps_nm_km = 21.0
    wl.spans[1].gamma_per_w_km = 0.8
    pb = oracle_mod.Problem(wl)
    s1, s2 = pb.spans
    f1, f2, f = 0.041, -0.03, 0.0
    f3 = f1 + f2 - f
    mu = []
    for s in (s1, s2):
        c = oracle_mod.chi(f1, f2, f, s.beta2, s.beta3)
        mu.append((c, oracle_mod.mu_segment(c, f3, OrSpan(s.alpha, s.beta2, s.beta3, s.gamma, s.cr, s.L),
                                            pb.ptot, pb.btot, oracle_mod.segments(s.L, 1.0))))
    ref = s1.gamma * mu[0][1] + s2.gamma * mu[1][1] * cmath.exp(1j * mu[0][0] * s1.L)
    assert abs(pb.upsilon(f1, f2, f) - ref) <= 1e-13 * abs(ref)


def test_upsilon_symmetric_in_f1_f2(oracle_mod, workloads):
    pb = _link_problem(oracle_mod, workloads, 3)
    for f1, f2, f in [(0.01, 0.07, 0.02), (-0.2, 0.13, 0.0)]:
        assert abs(pb.upsilon(f1, f2, f) - pb.upsilon(f2, f1, f)) <= 1e-14 * abs(pb.upsilon(f1, f2, f))
