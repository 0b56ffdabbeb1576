"""Pins of the EGN assembly (Eq. 11, 15): modulation-format moments, the GN limit,
scaling laws, and the paper's closed-form-vs-numerical accuracy findings."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def pam_moments(m):
    """Moments of the square QAM from its 1-D PAM components (x, y independent):
    E|a|^2 = 2 E x^2, E|a|^4 = 2 E x^4 + 2 (E x^2)^2, E|a|^6 = 2 E x^6 + 6 E x^4 E x^2."""
    lv = np.arange(-(m - 1), m, 2, dtype=float)
    e2, e4, e6 = (lv ** 2).mean(), (lv ** 4).mean(), (lv ** 6).mean()
    a2 = 2 * e2
    a4 = 2 * e4 + 2 * e2 * e2
    a6 = 2 * e6 + 6 * e4 * e2
    mu4, mu6 = a4 / a2 ** 2, a6 / a2 ** 3
    return mu4 - 2, mu6 - 9 * mu4 + 12


@pytest.mark.parametrize("name,m,phi,psi", [("QPSK", 2, -1.0, 4.0), ("16QAM", 4, -0.68, 2.08),
                                            ("64QAM", 8, -13 / 21, None), ("GAUSS", 0, 0.0, 0.0)])
def test_format_moments(oracle_mod, name, m, phi, psi):
    p, s = oracle_mod.format_moments(name)
    if m:
        pp, ss = pam_moments(m)
        assert p == pytest.approx(pp, abs=1e-14) and s == pytest.approx(ss, abs=1e-13)
    assert p == pytest.approx(phi, abs=1e-14)
    if psi is not None:
        assert s == pytest.approx(psi, abs=1e-13)


def test_gaussian_egn_equals_gn(oracle_mod, workloads):
    wl = workloads.config_small(gl_order=16)
    wl.formats = ["GAUSS"] * 5
    e_egn, _ = oracle_mod.Problem(wl, gl_order=16, terms=1).eta()
    e_gn, _ = oracle_mod.Problem(wl, gl_order=16, terms=0).eta()
    assert np.array_equal(e_egn, e_gn)


def test_qam_lowers_eta(oracle_mod, workloads):
    wl = workloads.config_small(gl_order=16)
    etas = {}
    for f in ("QPSK", "16QAM", "64QAM", "GAUSS"):
        wl.formats = [f] * 5
        etas[f], _ = oracle_mod.Problem(wl, gl_order=16).eta()
    assert np.all(etas["QPSK"] < etas["16QAM"])
    assert np.all(etas["16QAM"] < etas["64QAM"])
    assert np.all(etas["64QAM"] < etas["GAUSS"])


def test_scaling_laws(oracle_mod, workloads):
    wl = workloads.config_small(gl_order=16)
    wl.spans[0].cr_per_w_km_thz = 0.0
    e0, p0 = oracle_mod.Problem(wl, gl_order=16).eta()
    wl.launch_power_w = [2 * p for p in wl.launch_power_w]
    e1, p1 = oracle_mod.Problem(wl, gl_order=16).eta()
    assert np.allclose(e1, e0, rtol=1e-12)           # Cr = 0: eta independent of power
    assert np.allclose(p1, 8 * p0, rtol=1e-12)       # P_NLI ~ P^3
    wl.spans[0].gamma_per_w_km *= 2
    e2, _ = oracle_mod.Problem(wl, gl_order=16).eta()
    assert np.allclose(e2, 4 * e0, rtol=1e-12)       # eta ~ gamma^2


def test_isrs_tilts_eta(oracle_mod, workloads):
    """With ISRS on the same link, the high-frequency channel (which loses power along
    the span) sees less NLI than the low-frequency one; without ISRS and with beta3 = 0
    the mirror-image edge channels match."""
    wl = workloads.config_small(gl_order=16)
    wl.spans[0].cr_per_w_km_thz = 0.5
    wl.launch_power_w = [0.02] * 5
    e, _ = oracle_mod.Problem(wl, gl_order=16).eta([0, 4])
    assert e[0] > e[1]
    wl.spans[0].cr_per_w_km_thz = 0.0
    wl.spans[0].S_ps_nm2_km = -2 * wl.spans[0].D_ps_nm_km / 1550.0  # beta3 = 0
    wl.centre_hz = [wl.centre_hz[2] + (k - 2) * 75e9 for k in range(5)]
    e, _ = oracle_mod.Problem(wl, gl_order=16).eta([0, 4])
    assert e[0] == pytest.approx(e[1], rel=1e-9)


def test_kronecker_selection(oracle_mod, workloads):
    pb = oracle_mod.Problem(workloads.config_small(gl_order=8), gl_order=8)
    for n1, n2, n3 in pb.islands(2):
        t = pb.island_terms(2, n1, n2, n3)
        assert (t[1] != 0) == (n1 == n3)
        assert (t[2] != 0) == (n2 == n3)
        assert (t[3] != 0) == (n1 == n2)
        assert (t[4] != 0) == (n1 == n2 == n3)


def _reduced_table1(workloads, cr_full, n_ch=21, n_spans=1):
    """Table I with fewer channels: the same per-channel rate, spacing, total launch
    power and span; Cr scaled by 101/n_ch so that Delta rho (Eq. 12, ~ P Cr B) is the
    101-channel value."""
    wl = workloads.table1(n_spans=n_spans, cr=cr_full, gl_order=4, n_ch=n_ch)
    for s in wl.spans:
        s.cr_per_w_km_thz = cr_full * 101.0 / n_ch
    return wl


def test_paper_closed_form_accuracy(oracle_mod, workloads):
    """Sec. III-C / Fig. 8: against the integral form, the segment form (dz = 1 km) errs
    by < 0.001 dB MAE (max 0.0027 dB) at both ISRS levels; the Maclaurin form errs by
    ~ +-0.01 dB at Cr = 0.28 and by an order of magnitude more at Cr = 1.12."""
    g = json.load(open(GOLDEN))["closed_form_errors"]
    for cr in (0.28, 1.12):
        wl = _reduced_table1(workloads, cr)
        cois = [10, 5, 0]
        ref, _ = oracle_mod.Problem(wl, mu_form=2, int_tol=1e-8).eta(cois)
        seg, _ = oracle_mod.Problem(wl, mu_form=0).eta(cois)
        mac, _ = oracle_mod.Problem(wl, mu_form=1).eta(cois)
        es = 10 * np.log10(seg / ref)
        em = 10 * np.log10(mac / ref)
        assert np.mean(np.abs(es)) < g["segment_mae_db_bound"]
        assert np.max(np.abs(es)) < g["segment_cr112_max_abs_db"]
        if cr == 0.28:
            lo, hi = g["maclaurin_cr028_range_db"]
            assert np.max(np.abs(em)) < 2 * max(-lo, hi)
        else:
            assert np.max(np.abs(em)) > 0.05
            assert np.max(np.abs(em)) > 20 * np.max(np.abs(es))


def test_segment_error_does_not_accumulate_over_spans(oracle_mod, workloads):
    """Sec. III-C / Fig. 9(b): the segment error stays < 0.001 dB MAE at 10 spans."""
    wl = _reduced_table1(workloads, 1.12, n_spans=10)
    cois = [10, 0]
    ref, _ = oracle_mod.Problem(wl, mu_form=2, int_tol=1e-8).eta(cois)
    seg, _ = oracle_mod.Problem(wl, mu_form=0).eta(cois)
    assert np.mean(np.abs(10 * np.log10(seg / ref))) < 1e-3


def test_interferer_format_enters_xci_corrections(oracle_mod, workloads):
    """Two channels narrower than 2/3 of their spacing (only l = 0 islands), no
    ISRS: the COI's own format changes only its SCI island, so the change of P_NLI
    with the COI's Phi/Psi equals that of the COI alone; the interferer's format
    enters only through the XCI islands where it appears twice (its Phi)."""
    def problem(n_ch, phi, psi):
        wl = workloads.config_small(n_ch=2, gl_order=16)
        wl.centre_hz = wl.centre_hz[:n_ch]  # the COI sits at the same frequency in both combs
        wl.symbol_rate_baud = [40e9] * n_ch
        wl.launch_power_w = wl.launch_power_w[:n_ch]
        wl.formats = wl.formats[:n_ch]
        wl.spans[0].cr_per_w_km_thz = 0.0
        return oracle_mod.Problem(wl, gl_order=16, phi=phi, psi=psi)
    _, alone0 = problem(1, [0.0], [0.0]).eta([0])
    _, alone1 = problem(1, [-1.0], [4.0]).eta([0])
    _, both0 = problem(2, [0.0, 0.0], [0.0, 0.0]).eta([0])
    _, coi1 = problem(2, [-1.0, 0.0], [4.0, 0.0]).eta([0])
    _, int1 = problem(2, [0.0, -1.0], [0.0, 4.0]).eta([0])
    assert coi1[0] - both0[0] == pytest.approx(alone1[0] - alone0[0], rel=1e-10)
    # interferer format: the (B, A, B) E-island and (A, B, B) F-island of COI A
    pb = problem(2, [0.0, -1.0], [0.0, 4.0])
    t_e = pb.island_terms(0, 1, 0, 1, all_terms=True)[1]
    t_f = pb.island_terms(0, 0, 1, 1, all_terms=True)[2]
    P = 1e-3
    assert int1[0] - both0[0] == pytest.approx(-1.0 * P ** 3 * (t_e + t_f), rel=1e-10)


def test_each_correction_uses_its_repeated_channel(oracle_mod, workloads):
    """d P_NLI / d Phi_m (finite difference of the oracle's eta) equals the sum of
    the correction terms of the islands in which channel m appears twice: E where
    n1 = n3 = m, F where n2 = n3 = m, G where n1 = n2 = m."""
    wl = workloads.config_small(n_ch=5, gl_order=8)
    base = [0.0] * 5
    p0 = oracle_mod.Problem(wl, gl_order=8, phi=base, psi=base)
    _, pn0 = p0.eta([2])
    for m in range(5):
        phi = list(base)
        phi[m] = 1.0
        pb = oracle_mod.Problem(wl, gl_order=8, phi=phi, psi=base)
        _, pn1 = pb.eta([2])
        want = 0.0
        for n1, n2, n3 in pb.islands(2):
            t = pb.island_terms(2, n1, n2, n3, all_terms=True)
            w = wl.launch_power_w[n1] * wl.launch_power_w[n2] * wl.launch_power_w[n3]
            if n1 == n3 == m:
                want += w * t[1]
            if n2 == n3 == m:
                want += w * t[2]
            if n1 == n2 == m:
                want += w * t[3]
        assert pn1[0] - pn0[0] == pytest.approx(want, rel=1e-9), m
