"""Pins of the oracle's f-integrated (3-D) EGN: the integral over f of Eq. 17-21
taken literally, each COI evaluated at shifted frequencies f = f_n + delta.

The shifted 2-D integral is pinned to a closed-form inner integral (single
rectangular channel, one very long span, Cr = 0, beta3 = 0: |mu|^2 = 1/(alpha^2 +
chi^2)), to a brute-force midpoint grid, and to the reflection symmetry f -> -f of
a symmetric comb; the f-integral is pinned to scipy's adaptive quadrature of the
same closed form, and n_f = 1 reduces to the white-NLI value."""
import math

import numpy as np
import pytest
from scipy import integrate


def _long_single(workloads, oracle_mod):
    wl = workloads.config_small(n_ch=1, gl_order=128)
    wl.rolloff = 0.0
    s = wl.spans[0]
    s.length_m = 1500e3
    s.cr_per_w_km_thz = 0.0
    s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0  # beta3 = (lambda^2/2pi c)^2 (S + 2D/lambda) = 0
    pb = oracle_mod.Problem(wl, gl_order=128, terms=0)
    assert abs(pb.spans[0].beta3) < 1e-15
    return pb


def _closed_form_d(pb, delta):
    """D of the single channel evaluated at f = delta: with p = f1 - f, q = f2 - f the
    region is |p + delta|, |q + delta|, |p + q + delta| <= R/2 and the integrand
    1/(alpha^2 + c^2 p^2 q^2), c = 4 pi^2 |beta2|; the q integral is an arctan."""
    sp = pb.spans[0]
    R, a, g = pb.R[0], sp.alpha, sp.gamma
    c = 4 * math.pi ** 2 * abs(sp.beta2)

    def inner(p):
        lo = max(-R / 2 - delta, -R / 2 - delta - p)
        hi = min(R / 2 - delta, R / 2 - delta - p)
        if hi <= lo:
            return 0.0
        if p == 0.0:
            return (hi - lo) / a ** 2
        k = c * abs(p) / a
        return (math.atan(k * hi) - math.atan(k * lo)) / (a * c * abs(p))

    plo, phi = -R / 2 - delta, R / 2 - delta
    pts = [x for x in (0.0, -delta) if plo < x < phi] or None
    val, _ = integrate.quad(inner, plo, phi, points=pts, limit=400, epsabs=0, epsrel=1e-11)
    return 16 / 27 / R ** 2 * g * g * val


def test_one_node_is_the_white_nli_value(oracle_mod, workloads):
    pb = oracle_mod.Problem(workloads.config_small(n_ch=3, gl_order=16), gl_order=16)
    e2, p2 = pb.eta()
    e1, p1 = pb.eta_3d(1)
    assert np.array_equal(e1, e2) and np.array_equal(p1, p2)


@pytest.mark.parametrize("frac", [0.3, -0.6, 0.9])
def test_shifted_single_channel_closed_form(oracle_mod, workloads, frac):
    pb = _long_single(workloads, oracle_mod)
    d = frac * pb.R[0] / 2
    pb.set_coi_offsets(np.array([d]))
    got = pb.island_terms(0, 0, 0, 0)[0]
    pb.set_coi_offsets(None)
    assert got == pytest.approx(_closed_form_d(pb, d), rel=1e-7)


def test_f_integral_single_channel(oracle_mod, workloads):
    """eta_3d = (1/R) int G(delta) d delta over the band; scipy integrates the closed
    form over delta.  The f-integrated value is about 0.7 dB below the white-NLI one."""
    pb = _long_single(workloads, oracle_mod)
    R = pb.R[0]
    val, _ = integrate.quad(lambda d: _closed_form_d(pb, d), -R / 2, R / 2, points=[0.0], limit=200, epsrel=1e-9)
    want = val / R
    got = pb.eta_3d(16)[1][0] / pb.P[0] ** 3
    assert got == pytest.approx(want, rel=1e-4)
    white = pb.eta()[0][0]
    assert -0.8 < 10 * math.log10(want / white) < -0.6


def _symmetric_comb(workloads, oracle_mod, beta3_zero=True):
    wl = workloads.config_small(n_ch=3, gl_order=24)
    for s in wl.spans:
        s.cr_per_w_km_thz = 0.0
        if beta3_zero:
            s.S_ps_nm2_km = -2 * s.D_ps_nm_km / 1550.0
    return oracle_mod.Problem(wl, gl_order=24)


def test_reflection_symmetry_of_the_shift(oracle_mod, workloads):
    """Centre COI of a symmetric comb, beta3 = 0, Cr = 0: f -> -f maps the comb and
    its islands onto themselves, so P_NLI(+delta) = P_NLI(-delta).  With beta3 != 0
    the symmetry is broken (the test sees the sign of the shift)."""
    for beta3_zero, same in ((True, True), (False, False)):
        pb = _symmetric_comb(workloads, oracle_mod, beta3_zero)
        R = pb.R[1]
        out = []
        for sgn in (1.0, -1.0):
            pb.set_coi_offsets(np.array([0.0, sgn * 0.55 * R / 2, 0.0]))
            out.append(pb.eta(coi=[1])[1][0])
        pb.set_coi_offsets(None)
        rel = abs(out[0] / out[1] - 1)
        assert (rel < 1e-10) if same else (rel > 1e-6), rel


def test_shifted_node_rule_vs_dense_midpoint(oracle_mod, workloads):
    """At a shifted COI frequency the island offsets, panels and kinks move; the node
    rule still agrees with the brute-force midpoint grid (no panels)."""
    wl = workloads.config_small(n_ch=3)
    wl.spans[0].length_m = 20e3
    pb = oracle_mod.Problem(wl, gl_order=128)
    pb.set_coi_offsets(np.array([0.0, 0.5 * pb.R[1] / 2, 0.0]))
    for isl in [(1, 1, 1), (1, 0, 0), (0, 1, 0), (1, 2, 1)]:
        assert pb.island_exists(1, *isl)
        a = pb.island_terms(1, *isl, all_terms=True)
        b = pb.island_terms_midpoint(1, *isl, 400)
        assert np.allclose(a, b, rtol=6e-4, atol=0), (isl, (b - a) / a)
    pb.set_coi_offsets(None)


def test_islands_follow_the_shift(oracle_mod, workloads):
    """Near the band edge the f3 range of a pair leaves the next channel: with a
    66 GHz grid of 64.64 GHz supports, the offset d = m 66 GHz - delta of an m = -1
    island exceeds the 97 GHz half-sum of the supports once delta > 31 GHz.  The
    island set at such a shift is the brute-force set of positive-area overlaps,
    and it is smaller than the set at the centre."""
    wl = workloads.config_small(n_ch=5, gl_order=8)
    wl.centre_hz = [wl.centre_hz[2] + (k - 2) * 66e9 for k in range(5)]  # guard band 1.4 GHz
    pb = oracle_mod.Problem(wl, gl_order=8)
    at_centre = {tuple(int(x) for x in t) for t in pb.islands(2)}
    pb.set_coi_offsets(np.full(5, 0.495 * pb.R[2]))
    shifted = {tuple(int(x) for x in t) for t in pb.islands(2)}
    nu, W = pb.nu, pb.R * (1 + wl.rolloff)
    f = nu[2] + 0.495 * pb.R[2]
    brute = {(a, b, c) for a in range(5) for b in range(5) for c in range(5)
             if abs((nu[a] - f) + (nu[b] - nu[c])) < 0.5 * (W[a] + W[b] + W[c])}
    pb.set_coi_offsets(None)
    assert shifted == brute and shifted < at_centre
