"""Pins of the ridge-resolving node rule of the oracle (oracle/ridge_rule.py), the
estimate of Eq. 17's converged value where doubling the Gauss-Legendre order is
out of reach: exact areas, the dispersionless closed form, the exact
single-channel integral, and the converged level of the configured rule on an
island with a narrow ridge."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def RR():
    from oracle import ridge_rule
    return ridge_rule


def test_raised_cosine_is_the_oracles(RR, oracle_mod):
    R, beta = 0.064, 0.01
    x = np.linspace(-0.6 * R, 0.6 * R, 2001)
    got = RR.raised_cosine(x, R, beta)
    want = np.array([oracle_mod.rc(float(t), R, beta) for t in x])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("isl", [(0, 0, 0), (0, 4, 4), (1, 2, 3), (0, 1, 0), (2, 2, 4)])
def test_weights_sum_to_the_island_area(RR, oracle_mod, workloads, isl):
    """The island is a polygon; both rules integrate 1 over it exactly, in each of
    the three evaluation orders (the (u, v) -> (w, u) and (v, u) maps have unit
    Jacobian)."""
    pb = oracle_mod.Problem(workloads.config_small(), gl_order=8)
    rules = [RR.RidgeRule(pb), RR.RidgeRule(pb, knees=False)]
    for n in (0, 2):
        plain = pb.island_nodes(n, *isl)
        for rule in rules:
            for ordering in (0, 1, 2):
                r = rule.rows(n, *isl, ordering, 8)
                if r is None:
                    assert len(plain) == 0
                    continue
                area = sum(wo * wt.sum() for _, wo, _, wt in r[0])
                assert area == pytest.approx(plain[:, 2].sum(), rel=1e-12)
                assert all(np.all(wt > 0) and wo > 0 for _, wo, _, wt in r[0])


def test_dispersionless_closed_form(RR, oracle_mod, workloads):
    """beta2 = beta3 = 0, Cr = 0, rectangular spectra: Y = gamma L_eff, so D of the
    SCI island is (16/27) R^-2 (gamma L_eff)^2 times the hexagon's area 3 R^2 / 4."""
    wl = workloads.config_small(n_ch=3, gl_order=8)
    s = wl.spans[0]
    s.D_ps_nm_km = s.S_ps_nm2_km = s.cr_per_w_km_thz = 0.0
    wl.rolloff = 0.0
    pb = oracle_mod.Problem(wl, gl_order=8)
    sp = pb.spans[0]
    Y = sp.gamma * oracle_mod.leff(sp.alpha, sp.L)
    got, _ = RR.RidgeRule(pb).d_term(1, 1, 1, 1, 8)
    assert got == pytest.approx(16 / 27 / pb.R[1] ** 2 * Y * Y * 0.75 * pb.R[1] ** 2, rel=1e-12)


def test_single_channel_integral(RR, oracle_mod, workloads):
    """The long single channel (Cr = 0, beta3 = 0, one segment): the ridges f1 = f and
    f2 = f cross at the centre.  The error falls geometrically with the nodes per
    piece (2e-3 at 8, 7e-8 at 32, 1e-12 at 64)."""
    from scipy import integrate
    wl = workloads.config_small(n_ch=1, gl_order=8)
    wl.rolloff = 0.0
    s = wl.spans[0]
    s.length_m = 1500e3
    s.cr_per_w_km_thz = 0.0
    s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0
    pb = oracle_mod.Problem(wl, gl_order=8, terms=0, dz_km=1500.0)
    sp = pb.spans[0]
    R, a, g = pb.R[0], sp.alpha, sp.gamma
    c = 4 * math.pi ** 2 * abs(sp.beta2)

    def inner(u):
        lo, hi = max(-R / 2, -R / 2 - u), min(R / 2, R / 2 - u)
        if u == 0:
            return (hi - lo) / a ** 2
        k = c * abs(u) / a
        return (math.atan(k * hi) - math.atan(k * lo)) / (a * c * abs(u))

    val, _ = integrate.quad(inner, -R / 2, R / 2, points=[0.0], limit=400, epsabs=0, epsrel=1e-12)
    want = 16 / 27 / R ** 2 * g * g * val
    rule = RR.RidgeRule(pb)
    assert rule.d_term(0, 0, 0, 0, 32)[0] == pytest.approx(want, rel=1e-6)
    assert rule.d_term(0, 0, 0, 0, 64)[0] == pytest.approx(want, rel=1e-10)
    assert abs(pb.island_terms(0, 0, 0, 0)[0] / want - 1) > 0.1  # the plain 8 x 8 rule: 14 % high


def test_narrow_ridge_island(RR, oracle_mod, workloads):
    """XCI island (0, 4, 4) of the 5-channel link: a ridge 0.4 GHz wide along f1 = f.
    32 nodes per piece come within 1e-3 of the converged plain rule (256 x 256),
    where the plain 32 x 32 rule is 40 % off."""
    wl = workloads.config_small()
    want = oracle_mod.Problem(wl, gl_order=256, terms=0).island_terms(0, 0, 4, 4)[0]
    pb = oracle_mod.Problem(wl, gl_order=32, terms=0)
    got, npts = RR.RidgeRule(pb).d_term(0, 0, 4, 4, 32)
    assert abs(got / want - 1) < 1e-3 and npts < 4096
    assert abs(pb.island_terms(0, 0, 4, 4)[0] / want - 1) > 0.3


def test_gn_sum_converges_where_the_plain_rule_swings(RR, oracle_mod, workloads):
    """The finding on the 5-channel link, as a pin: the GN part of Eq. 15 for the
    edge and centre COIs settles within 0.02 dB between 8 and 16 nodes per piece
    of the ridge rule, while the configured rule moves by more than 0.1 dB between
    16 x 16 and 32 x 32 nodes (the ridges are not resolved)."""
    wl = workloads.config_small()
    pb = oracle_mod.Problem(wl, gl_order=8, terms=0)
    rule = RR.RidgeRule(pb)
    for n in (0, 2):
        r8, r16 = rule.pnli_gn(n, 8), rule.pnli_gn(n, 16)
        p16 = oracle_mod.Problem(wl, gl_order=16, terms=0).island_contribs(n)[1].sum()
        p32 = oracle_mod.Problem(wl, gl_order=32, terms=0).island_contribs(n)[1].sum()
        assert abs(10 * np.log10(r8 / r16)) < 0.02, (n, r8, r16)
        assert abs(10 * np.log10(p16 / p32)) > 0.1, (n, p16, p32)


def test_all_terms_dispersionless_exact(RR, oracle_mod, workloads):
    """beta2 = beta3 = 0, Cr = 0, rectangular spectra: Y is constant, every inner
    integral is Y times a length linear in the outer variable, so both rules give
    D..H exactly on SCI, XCI and MCI islands of a 5-channel comb."""
    wl = workloads.config_small(n_ch=5, gl_order=16)
    s = wl.spans[0]
    s.D_ps_nm_km = s.S_ps_nm2_km = s.cr_per_w_km_thz = 0.0
    wl.rolloff = 0.0
    pb = oracle_mod.Problem(wl, gl_order=16)
    rule = RR.RidgeRule(pb)
    for n, isl in ((2, (2, 2, 2)), (2, (1, 1, 0)), (2, (2, 3, 3)), (0, (0, 1, 1)), (1, (0, 2, 1)), (2, (1, 3, 2))):
        want = pb.island_terms(n, *isl, all_terms=True)
        got = rule.terms(n, *isl, 8)
        assert np.allclose(got, want, rtol=1e-12, atol=0), (isl, got / want - 1)


def test_e_f_mirror(RR, oracle_mod, workloads):
    """E of (n1, n2, n1) and F of (n2, n1, n1) integrate mirrored structures (f1 <-> f2)
    on mirrored nodes: equal up to their printed coefficients."""
    pb = oracle_mod.Problem(workloads.config_small(), gl_order=16)
    rule = RR.RidgeRule(pb)
    for n, a, b in ((2, 1, 3), (0, 0, 2), (4, 3, 4)):
        e = rule.terms(n, a, b, a, 16)[1] / (16 / 27)
        f = rule.terms(n, b, a, a, 16)[2] / (32 / 81)
        assert e == pytest.approx(f, rel=1e-12)


def test_all_terms_narrow_ridge(RR, oracle_mod, workloads):
    """XCI island (0, 4, 4) of the 5-channel link: all five terms at 32 nodes per
    piece within 6e-3 of the converged plain rule (256 x 256), where the plain
    32 x 32 rule is 6 % to 67 % off."""
    wl = workloads.config_small()
    want = oracle_mod.Problem(wl, gl_order=256).island_terms(0, 0, 4, 4, all_terms=True)
    pb = oracle_mod.Problem(wl, gl_order=32)
    got = RR.RidgeRule(pb).terms(0, 0, 4, 4, 32)
    assert np.max(np.abs(got / want - 1)) < 6e-3
    assert np.min(np.abs(pb.island_terms(0, 0, 4, 4, all_terms=True) / want - 1)) > 0.05


def test_shifted_coi_single_channel(RR, oracle_mod, workloads):
    """At a COI frequency moved by delta inside the band the ridges move with it;
    the rule reaches the arctan closed form of the shifted single channel (64 nodes
    per piece: 1e-10 at delta = 0.3 R/2, 5e-7 at -0.8 R/2, near the band edge)."""
    from scipy import integrate
    wl = workloads.config_small(n_ch=1, gl_order=8)
    wl.rolloff = 0.0
    s = wl.spans[0]
    s.length_m = 1500e3
    s.cr_per_w_km_thz = 0.0
    s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0
    pb = oracle_mod.Problem(wl, gl_order=8, terms=0, dz_km=1500.0)
    sp = pb.spans[0]
    R, a, g = pb.R[0], sp.alpha, sp.gamma
    c = 4 * math.pi ** 2 * abs(sp.beta2)
    rule = RR.RidgeRule(pb)
    for frac in (0.3, -0.8):
        delta = frac * R / 2

        def inner(p):
            lo = max(-R / 2 - delta, -R / 2 - delta - p)
            hi = min(R / 2 - delta, R / 2 - delta - p)
            if hi <= lo:
                return 0.0
            if p == 0.0:
                return (hi - lo) / a ** 2
            k = c * abs(p) / a
            return (math.atan(k * hi) - math.atan(k * lo)) / (a * c * abs(p))

        val, _ = integrate.quad(inner, -R / 2 - delta, R / 2 - delta, points=[0.0, -delta], limit=400,
                                epsabs=0, epsrel=1e-12)
        want = 16 / 27 / R ** 2 * g * g * val
        pb.set_coi_offsets(np.array([delta]))
        try:
            got = rule.d_term(0, 0, 0, 0, 64)[0]
        finally:
            pb.set_coi_offsets(None)
        assert got == pytest.approx(want, rel=1e-6), (frac, got / want - 1)


def test_f_integral_matches_the_oracle_dispersionless(RR, oracle_mod, workloads):
    """Without dispersion the integrand is constant on every island, both rules are
    exact at every COI frequency, and the f-integrated sums agree (the island sets
    change with f inside the band)."""
    wl = workloads.config_small(n_ch=3, gl_order=8)
    s = wl.spans[0]
    s.D_ps_nm_km = s.S_ps_nm2_km = s.cr_per_w_km_thz = 0.0
    wl.rolloff = 0.0
    pb = oracle_mod.Problem(wl, gl_order=8)
    want = pb.eta_3d(4, coi=[1])[1][0]
    got = RR.RidgeRule(pb).pnli_3d(1, 8, 4)
    assert got == pytest.approx(want, rel=1e-12)
