"""Pins of the oracle's island integrals D, E, F, G, H (Eq. 17-21): closed-form
geometry in the dispersionless limit, brute-force midpoint grids, symmetries, and
the single-channel GN integral."""
import math

import numpy as np
import pytest
from scipy import integrate


def test_gauss_legendre_exactness(oracle_mod):
    for n in (1, 2, 5, 16, 32, 64):
        x, w = oracle_mod.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=1e-14, rtol=0) and np.allclose(w, wr, atol=1e-14, rtol=0)
        for k in range(2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.dot(w, x ** k) - exact) < 1e-13


def _dispersionless(workloads, oracle_mod, n_ch=5, n_spans=1, spacing=75e9):
    """beta2 = beta3 = 0, Cr = 0, rectangular spectra: Y = N gamma L_eff everywhere."""
    wl = workloads.config_small(n_ch=n_ch, n_spans=n_spans, gl_order=16)
    for s in wl.spans:
        s.D_ps_nm_km = 0.0
        s.S_ps_nm2_km = 0.0
        s.cr_per_w_km_thz = 0.0
    wl.rolloff = 0.0
    c = wl.centre_hz[n_ch // 2]
    wl.centre_hz = [c + (k - n_ch // 2) * spacing for k in range(n_ch)]
    pb = oracle_mod.Problem(wl, gl_order=16)
    a = pb.spans[0].alpha
    Y = n_spans * pb.spans[0].gamma * oracle_mod.leff(a, pb.spans[0].L)
    return pb, Y


@pytest.mark.parametrize("n_spans", [1, 3])
def test_dispersionless_sci_closed_form(oracle_mod, workloads, n_spans):
    """SCI island, d = 0: hexagon |u|, |v|, |u + v| <= R/2 of area 3R^2/4; each inner
    integral of E, F, G has length R - |outer| and int (R - |x|)^2 dx = 7 R^3 / 12."""
    pb, Y = _dispersionless(workloads, oracle_mod, n_spans=n_spans)
    t = pb.island_terms(2, 2, 2, 2, all_terms=True)
    Y2 = Y * Y
    want = [16 / 27 * 3 / 4 * Y2, 16 / 27 * 7 / 12 * Y2, 32 / 81 * 7 / 12 * Y2,
            16 / 81 * 7 / 12 * Y2, 16 / 81 * 9 / 16 * Y2]
    assert np.allclose(t, want, rtol=1e-12, atol=0)


def test_dispersionless_xci_d0_closed_form(oracle_mod, workloads):
    # (n1, n2, n3) = (n, m, m): d = 0, same hexagon in local coordinates
    pb, Y = _dispersionless(workloads, oracle_mod)
    t = pb.island_terms(2, 2, 4, 4, all_terms=True)
    Y2 = Y * Y
    want = [16 / 27 * 3 / 4, 16 / 27 * 7 / 12, 32 / 81 * 7 / 12, 16 / 81 * 7 / 12, 16 / 81 * 9 / 16]
    assert np.allclose(t, np.array(want) * Y2, rtol=1e-12, atol=0)


def test_dispersionless_l1_triangle_closed_form(oracle_mod, workloads):
    """(n1, n2, n3) = (n, n, n - 1): d = +spacing; the domain is the triangle
    u, v >= -R/2, u + v <= R/2 - d - R/2 with legs a = 3R/2 - d.  Area a^2/2, and every
    inner integral has length t in [0, a]: int t^2 = a^3 / 3."""
    pb, Y = _dispersionless(workloads, oracle_mod)
    R = pb.R[0]
    d = pb.nu[2] - pb.nu[1]
    a = 1.5 * R - d
    t = pb.island_terms(2, 2, 2, 1, all_terms=True)
    Y2 = Y * Y
    want = [16 / 27 / R ** 2 * a * a / 2, 16 / 27 / R ** 3 * a ** 3 / 3, 32 / 81 / R ** 3 * a ** 3 / 3,
            16 / 81 / R ** 3 * a ** 3 / 3, 16 / 81 / R ** 4 * (a * a / 2) ** 2]
    assert np.allclose(t, np.array(want) * Y2, rtol=1e-12, atol=0)


def test_d_symmetric_in_n1_n2(oracle_mod, workloads):
    """f1 <-> f2 symmetry of the integrand; with equal widths the swapped island's
    nodes are the mirror image, so D agrees to rounding."""
    pb = oracle_mod.Problem(workloads.config_small(gl_order=16), gl_order=16)
    for n in range(5):
        for n1, n2, n3 in pb.islands(n):
            if n1 < n2:
                a = pb.island_terms(n, n1, n2, n3)[0]
                b = pb.island_terms(n, n2, n1, n3)[0]
                assert a == pytest.approx(b, rel=1e-11)


def test_e_f_mirror(oracle_mod, workloads):
    """E of (n1, n2, n1) and F of (n2, n1, n1) are the same integral after f1 <-> f2,
    up to their printed coefficients 16/27 and 32/81."""
    pb = oracle_mod.Problem(workloads.config_small(gl_order=16), gl_order=16)
    checked = 0
    for n in range(5):
        for n1, n2, n3 in pb.islands(n):
            if n1 == n3 and n1 != n2:
                e = pb.island_terms(n, n1, n2, n3)[1]
                f = pb.island_terms(n, n2, n1, n3)[2]
                assert e / (16 / 27) == pytest.approx(f / (32 / 81), rel=1e-11)
                checked += 1
    assert checked > 5


def test_node_rule_vs_dense_midpoint(oracle_mod, workloads):
    """Gauss-Legendre node rule (panels at kinks) against a brute-force midpoint grid
    over the bounding rectangle (no panels): the two independent rules converge to
    the same five integrals."""
    wl = workloads.config_small(n_ch=3)
    wl.spans[0].length_m = 20e3
    pb = oracle_mod.Problem(wl, gl_order=128)
    for isl in [(1, 1, 1), (1, 0, 0), (0, 1, 0), (1, 2, 1)]:
        a = pb.island_terms(1, *isl, all_terms=True)
        b = pb.island_terms_midpoint(1, *isl, 400)
        assert np.allclose(a, b, rtol=6e-4, atol=0), (isl, (b - a) / a)


def test_single_channel_gn_integral(oracle_mod, workloads):
    """Single rectangular channel, Cr = 0, beta3 = 0, one very long span: |mu|^2 =
    1/(alpha^2 + chi^2) with chi = 4 pi^2 beta2 u v.  D is then (16/27) R^-2 gamma^2
    times the integral over the hexagon, which has the inner integral in closed form
    (arctan); the outer one is done by scipy."""
    wl = workloads.config_small(n_ch=1, gl_order=128)
    wl.rolloff = 0.0
    s = wl.spans[0]
    s.length_m = 1500e3
    s.cr_per_w_km_thz = 0.0
    s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0  # makes beta3 = (lambda^2/2pi c)^2 (S + 2D/lambda) = 0
    pb = oracle_mod.Problem(wl, gl_order=128, terms=0)
    sp = pb.spans[0]
    assert abs(sp.beta3) < 1e-15
    R, a, b2, g = pb.R[0], sp.alpha, sp.beta2, sp.gamma
    c = 4 * math.pi ** 2 * abs(b2)

    def inner(u):
        lo, hi = max(-R / 2, -R / 2 - u), min(R / 2, R / 2 - u)
        if u == 0:
            return (hi - lo) / a ** 2
        k = c * abs(u) / a
        return (math.atan(k * hi) - math.atan(k * lo)) / (a * c * abs(u))

    val, _ = integrate.quad(inner, -R / 2, R / 2, points=[0.0], limit=400, epsabs=0, epsrel=1e-11)
    want = 16 / 27 / R ** 2 * g * g * val
    got = pb.island_terms(0, 0, 0, 0)[0]
    assert got == pytest.approx(want, rel=1e-4)
    eta, _ = pb.eta()
    assert eta[0] == pytest.approx(want, rel=1e-4)


def _single_channel_k1(workloads, oracle_mod, gl):
    """The long single channel of the test above with one segment per span (Cr = 0:
    the segment form is exact for any K) and its integral by the arctan inner form."""
    wl = workloads.config_small(n_ch=1, gl_order=gl)
    wl.rolloff = 0.0
    s = wl.spans[0]
    s.length_m = 1500e3
    s.cr_per_w_km_thz = 0.0
    s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0
    pb = oracle_mod.Problem(wl, gl_order=gl, terms=0, dz_km=1500.0)
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
    return pb, 16 / 27 / R ** 2 * g * g * val


def test_converged_level_reaches_the_integral(oracle_mod, workloads):
    """Doubling the order from 8 until eta moves by < 1e-4 dB lands within 1e-4 dB
    of the exact single-channel integral, with the order-8 value well off it."""
    pb, want = _single_channel_k1(workloads, oracle_mod, 8)
    eta, order, hist = pb.eta_converged(tol_db=1e-4, max_order=1024)
    assert order > 8 and sorted(hist) == [8 * 2 ** i for i in range(len(hist))]
    assert abs(10 * math.log10(eta[0] / want)) < 1e-4
    assert abs(10 * math.log10(hist[8][0] / want)) > 1e-3
    assert pb.c.gl_order == 8  # the problem's own order is restored
    with pytest.raises(RuntimeError):
        pb.eta_converged(tol_db=1e-12, max_order=32)


def test_orders_beyond_512(oracle_mod, workloads):
    """Node buffers are sized by the rule: a 600 x 600 rule (above any fixed buffer of
    512) integrates the single channel to the closed form, and the node list has
    600 x 600 weights summing to the hexagon's area."""
    pb, want = _single_channel_k1(workloads, oracle_mod, 600)
    assert pb.island_terms(0, 0, 0, 0)[0] == pytest.approx(want, rel=1e-8)
    nodes = pb.island_nodes(0, 0, 0, 0)
    R = pb.R[0]
    assert len(nodes) == 600 * 600 and nodes[:, 2].sum() == pytest.approx(0.75 * R * R, rel=1e-12)
    with pytest.raises(ValueError):
        oracle_mod.Problem(workloads.config_small(n_ch=1), gl_order=0)


def test_single_channel_gn_closed_form_soft(oracle_mod, workloads):
    """The incoherent-GN closed form (8/27) gamma^2 L_eff^2 asinh(pi^2/2 |b2| L_eff R^2)
    / (pi |b2| L_eff R^2) approximates the single-channel eta to a few percent."""
    wl = workloads.config_small(n_ch=1, gl_order=64)
    wl.spans[0].length_m = 1000e3
    wl.spans[0].cr_per_w_km_thz = 0.0
    pb = oracle_mod.Problem(wl, terms=0)
    sp = pb.spans[0]
    L = 1 / sp.alpha
    R = pb.R[0]
    x = math.pi ** 2 / 2 * abs(sp.beta2) * L * R * R
    cf = 8 / 27 * sp.gamma ** 2 * L * L * math.asinh(x) / (math.pi * abs(sp.beta2) * L * R * R)
    eta, _ = pb.eta()
    assert abs(10 * math.log10(eta[0] / cf)) < 0.3


def test_quadrature_order_convergence(oracle_mod, workloads):
    """Converged-rule check.  The SCI island converges quickly with the order; an XCI
    island with a distant interferer has a ridge of |mu|^2 along f1 = f only
    ~ alpha / (4 pi^2 |beta2| |f2 - f|) wide (0.4 GHz here), which 32 or 64 nodes
    across a 64 GHz channel do not resolve: there the low orders are tens of percent
    off while high orders converge."""
    wl = workloads.config_small()
    sci = [oracle_mod.Problem(wl, gl_order=g).island_terms(0, 0, 0, 0)[0] for g in (64, 128)]
    assert sci[1] == pytest.approx(sci[0], rel=1e-3)
    xci = [oracle_mod.Problem(wl, gl_order=g).island_terms(0, 0, 4, 4)[0] for g in (32, 256, 384)]
    assert xci[2] == pytest.approx(xci[1], rel=1e-5)
    assert abs(xci[0] / xci[2] - 1) > 0.2


def test_d_rate_normalisation_split_channel(oracle_mod, workloads):
    """D carries R_n / (R1 R2 R3) so that P_i / R_i is each channel's PSD: with
    rectangular spectra, no dispersion and no ISRS, replacing an interferer of rate
    2R and power 2P by two adjacent channels of rate R and power P (the same PSD)
    leaves the COI's GN eta unchanged."""
    def comb(split):
        wl = workloads.config_small(n_ch=2, gl_order=8)
        for s in wl.spans:
            s.D_ps_nm_km = 0.0
            s.S_ps_nm2_km = 0.0
            s.cr_per_w_km_thz = 0.0
        wl.rolloff = 0.0
        c = 1.93e14
        R = 40e9
        if split:
            wl.centre_hz = [c, c + 2.5 * R, c + 3.5 * R]
            wl.symbol_rate_baud = [R, R, R]
            wl.launch_power_w = [1e-3, 1e-3, 1e-3]
            wl.formats = ["GAUSS"] * 3
        else:
            wl.centre_hz = [c, c + 3.0 * R]
            wl.symbol_rate_baud = [R, 2 * R]
            wl.launch_power_w = [1e-3, 2e-3]
            wl.formats = ["GAUSS"] * 2
        return wl
    e1, p1 = oracle_mod.Problem(comb(False), gl_order=8, terms=0).eta([0])
    e2, p2 = oracle_mod.Problem(comb(True), gl_order=8, terms=0).eta([0])
    assert p1[0] == pytest.approx(p2[0], rel=1e-12)


def test_dispersionless_mixed_widths_kinks(oracle_mod, workloads):
    """Island with three different widths and d != 0 whose inner limits switch
    inside the outer range: with Upsilon constant each term is a polygon area or the
    integral of a squared piecewise-linear inner length, integrated here by scipy
    from the supports alone (no panels)."""
    wl = workloads.config_small(n_ch=4, gl_order=8)
    for s in wl.spans:
        s.D_ps_nm_km = 0.0
        s.S_ps_nm2_km = 0.0
        s.cr_per_w_km_thz = 0.0
    wl.rolloff = 0.0
    c = 1.93e14
    wl.centre_hz = [c - 100e9, c, c + 100e9, c + 190e9]
    wl.symbol_rate_baud = [40e9, 60e9, 30e9, 50e9]
    wl.formats = ["GAUSS"] * 4
    pb = oracle_mod.Problem(wl, gl_order=8)
    Y = pb.spans[0].gamma * oracle_mod.leff(pb.spans[0].alpha, pb.spans[0].L)
    n, n1, n2, n3 = 0, 1, 2, 3
    W1, W2, W3 = pb.R[n1], pb.R[n2], pb.R[n3]
    d = (pb.nu[n1] - pb.nu[n]) + (pb.nu[n2] - pb.nu[n3])
    assert abs(d - 0.010) < 1e-12

    def length(lo1, hi1, lo2, hi2):
        return max(0.0, min(hi1, hi2) - max(lo1, lo2))

    # inner lengths of the three evaluation orders, from the supports
    lw = lambda w: length(-W1 / 2, W1 / 2, w - d - W2 / 2, w - d + W2 / 2)        # inner u at fixed w
    lv = lambda v: length(-W1 / 2, W1 / 2, -W3 / 2 - v - d, W3 / 2 - v - d)      # inner u at fixed v
    lu = lambda u: length(-W2 / 2, W2 / 2, -W3 / 2 - u - d, W3 / 2 - u - d)      # inner v at fixed u
    q = lambda f, a, b: integrate.quad(f, a, b, limit=200, epsabs=0, epsrel=1e-13)[0]
    area = q(lw, -W3 / 2, W3 / 2)
    e_int = q(lambda v: lv(v) ** 2, -W2 / 2, W2 / 2)
    f_int = q(lambda u: lu(u) ** 2, -W1 / 2, W1 / 2)
    g_int = q(lambda w: lw(w) ** 2, -W3 / 2, W3 / 2)
    R = pb.R[n]
    want = np.array([16 / 27 * R / (W1 * W2 * W3) * area, 16 / 27 / R ** 3 * e_int, 32 / 81 / R ** 3 * f_int,
                     16 / 81 / R ** 3 * g_int, 16 / 81 / R ** 4 * area ** 2]) * Y * Y
    got = pb.island_terms(n, n1, n2, n3, all_terms=True)
    assert np.allclose(got, want, rtol=1e-10, atol=0), (got / want - 1)
