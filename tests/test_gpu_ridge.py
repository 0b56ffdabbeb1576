"""The ridge-resolving node rule on the GPU (egn_set_node_rule(EGN_RULE_RIDGE),
FP64 and FP32C paths) against the oracle's ridge rule (oracle/ridge_rule.py) at
the same node counts, through the C ABI.

The two sides share no code: the oracle's rule is numpy around the oracle's C
integrand; the kernel forms the same cuts, pieces and sinh-graded nodes on the
device.  Bars: every term of every island within 1e-9 of the oracle's (relative
to the largest term of its kind in the COI), eta within 1e-9 relative (the GPU
evaluates the half list and counts each mirror island twice; the oracle sums
every island; the two differ by rounding).  The rule converges where the
configured one does not: on the 5-channel link 16 and 32 nodes per piece agree
within 0.003 dB for the GN part and 0.04 dB with the EGN corrections, where the
configured rule moves by more than 0.3 dB from 32 x 32 to 64 x 64 (the narrow
ridges of |mu|^2).  FP32C (links of identical spans): every term within 3e-4
of the oracle's relative to itself plus 3e-5 of the largest term of its kind in
the COI, the bars of the configured rule's FP32C parity, and eta within 1e-3 dB."""
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


@pytest.fixture(scope="module")
def RR():
    from oracle import ridge_rule
    return ridge_rule


def _ridge_link(egn, wl, n_min=4):
    ln = egn.link_from_workload(wl)
    ln.set_node_rule(egn.EGN_RULE_RIDGE, n_min)
    return ln


@pytest.mark.parametrize("order", [8, 16])
def test_ridge_island_terms_match_oracle(egn, oracle_mod, workloads, RR, order):
    """All five terms of every island of the edge and centre COIs of the 5-channel
    link (SCI, XCI with the ridges inside, MCI)."""
    wl = workloads.config_small(gl_order=order)
    ln = _ridge_link(egn, wl)
    pb = oracle_mod.Problem(wl, gl_order=order)
    rule = RR.RidgeRule(pb)
    opts = egn.make_opts(gl_order=order, precision=egn.EGN_PREC_FP64)
    for n in (0, 2):
        isl = [(n, int(a), int(b), int(c)) for a, b, c in pb.islands(n)]
        got = ln.island_terms(opts, isl, all_terms=True)
        want = np.array([rule.terms(*t, order) for t in isl])
        scale = np.max(np.abs(want), axis=0) + 1e-300
        assert np.all(np.abs(got - want) <= 1e-9 * scale), (n, np.max(np.abs(got - want) / scale, axis=0))
    ln.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_ridge_sampled_islands_of_the_benchmark_link(egn, oracle_mod, workloads, RR, prec):
    """The full-size 120-channel C+L link (ten spans): all five terms of sampled
    islands of COIs 0, 59 and 119 -- the SCI island, XCI islands with the nearest
    and the farthest interferer, and four seeded random islands each -- against
    the oracle's rule at 16 nodes per piece.  FP64 within 1e-9 of the largest term
    of its kind among the sampled islands; FP32C within 3e-4 of the term plus 3e-5
    of that largest term."""
    wl = workloads.config_cl()
    ln = _ridge_link(egn, wl)
    pb = oracle_mod.Problem(wl, gl_order=16)
    rule = RR.RidgeRule(pb)
    rng = np.random.default_rng(11)
    isl = []
    for n in (0, 59, 119):
        near, far = (n + 1, 119) if n < 119 else (118, 0)
        isl += [(n, n, n, n), (n, n, near, near), (n, n, far, far)]
        cand = pb.islands(n)
        for k in rng.choice(len(cand), 4, replace=False):
            a, b, c = (int(v) for v in cand[k])
            isl.append((n, a, b, c))
    for t in isl:
        assert pb.island_exists(*t), t
    pr = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got = ln.island_terms(egn.make_opts(gl_order=16, dz_km=wl.dz_km, precision=pr), isl, all_terms=True)
    want = np.array([rule.terms(*t, 16) for t in isl])
    scale = np.max(np.abs(want), axis=0) + 1e-300
    err = np.abs(got - want)
    if prec == "fp64":
        assert np.all(err <= 1e-9 * scale), np.max(err / scale, axis=0)
    else:
        assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * scale), np.max(err / (np.abs(want) + 1e-300), axis=0)
    ln.close()


@pytest.mark.parametrize("case", ["5ch", "8ch_3spans", "4ch_3types", "3ch_6types"])
def test_ridge_eta_matches_oracle(egn, oracle_mod, workloads, RR, case):
    """eta of every channel; the last two cases are links whose spans differ (three
    span types: per-type c_k tables; six: span by span), where the ridge widths
    take the first span's fibre and the integrand is Eq. 22's explicit span sum."""
    if case == "5ch":
        wl, order = workloads.config_small(gl_order=16), 16
    elif case == "8ch_3spans":
        wl, order = workloads.config_small(n_ch=8, gl_order=8, n_spans=3), 8
        wl.formats = ["QPSK", "16QAM", "64QAM", "GAUSS"] * 2
    else:
        n_ch, n_spans = (4, 3) if case == "4ch_3types" else (3, 6)
        wl, order = workloads.config_small(n_ch=n_ch, gl_order=8, n_spans=n_spans), 8
        for i, sp in enumerate(wl.spans):
            sp.length_m = (60 + 7 * i) * 1e3
        wl.spans[1].alpha_db_km = 0.16
        wl.spans[1].D_ps_nm_km = 21.0
    ln = _ridge_link(egn, wl)
    eta, pnli = ln.nli_eta(egn.make_opts(gl_order=order, precision=egn.EGN_PREC_FP64))
    pb = oracle_mod.Problem(wl, gl_order=order)
    rule = RR.RidgeRule(pb)
    want = np.array([rule.pnli(n, order) for n in range(wl.n_ch)])
    assert np.allclose(pnli, want, rtol=1e-9, atol=0), (pnli, want)
    assert np.allclose(eta, want / np.asarray(wl.launch_power_w) ** 3, rtol=1e-9, atol=0)
    ln.close()


@pytest.mark.parametrize("order", [8, 16])
def test_ridge_fp32c_island_terms_match_oracle(egn, oracle_mod, workloads, RR, order):
    wl = workloads.config_small(gl_order=order)
    ln = _ridge_link(egn, wl)
    pb = oracle_mod.Problem(wl, gl_order=order)
    rule = RR.RidgeRule(pb)
    opts = egn.make_opts(gl_order=order, precision=egn.EGN_PREC_FP32C)
    for n in (0, 2):
        isl = [(n, int(a), int(b), int(c)) for a, b, c in pb.islands(n)]
        got = ln.island_terms(opts, isl, all_terms=True)
        want = np.array([rule.terms(*t, order) for t in isl])
        scale = np.max(np.abs(want), axis=0) + 1e-300
        err = np.abs(got - want)
        assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * scale), (n, np.max(err / (np.abs(want) + 1e-300), axis=0))
    ln.close()


@pytest.mark.parametrize("case", ["5ch", "8ch_3spans", "16ch_beta0", "4ch_3types", "6ch_4types"])
def test_ridge_fp32c_eta_matches_oracle(egn, oracle_mod, workloads, RR, case):
    """eta of every channel in FP32C; 8 channels over three identical spans with
    four modulation formats; 16 channels without roll-off; links of three and
    four span types (lengths, attenuation and dispersion differ; Eq. 22 summed
    span by span)."""
    if case == "5ch":
        wl, order = workloads.config_small(gl_order=16), 16
    elif case == "8ch_3spans":
        wl, order = workloads.config_small(n_ch=8, gl_order=8, n_spans=3), 8
        wl.formats = ["QPSK", "16QAM", "64QAM", "GAUSS"] * 2
    elif case == "16ch_beta0":
        wl, order = workloads.config_small(n_ch=16, gl_order=8), 8
        wl.rolloff = 0.0
    else:
        n_ch, n_spans = (4, 3) if case == "4ch_3types" else (6, 5)
        wl, order = workloads.config_small(n_ch=n_ch, gl_order=8, n_spans=n_spans), 8
        for i, sp in enumerate(wl.spans):
            sp.length_m = (60 + 7 * (i % 4)) * 1e3
        wl.spans[1].alpha_db_km = 0.16
        wl.spans[1].D_ps_nm_km = 21.0
    ln = _ridge_link(egn, wl)
    eta, _ = ln.nli_eta(egn.make_opts(gl_order=order, precision=egn.EGN_PREC_FP32C))
    pb = oracle_mod.Problem(wl, gl_order=order)
    rule = RR.RidgeRule(pb)
    want = np.array([rule.pnli(n, order) for n in range(wl.n_ch)]) / np.asarray(wl.launch_power_w) ** 3
    db = np.abs(10 * np.log10(eta / want))
    assert np.max(db) < 1e-3, db
    ln.close()


def test_ridge_fp32c_matches_fp64_on_a_link_of_span_types(egn, workloads):
    """30 channels of the C+L grid over six spans of three types (80, 70 and 90 km,
    the second with 0.17 dB/km and 20 ps/nm/km): FP32C against the FP64 ridge
    kernel on every channel within 1e-3 dB."""
    wl = workloads.config_cl(n_ch=30, n_spans=6)
    for i, sp in enumerate(wl.spans):
        sp.length_m = (80e3, 70e3, 90e3)[i % 3]
        if i % 3 == 1:
            sp.alpha_db_km = 0.17
            sp.D_ps_nm_km = 20.0
    ln = _ridge_link(egn, wl)
    o = lambda pr: egn.make_opts(gl_order=8, dz_km=wl.dz_km, precision=pr)  # noqa: E731
    e64, _ = ln.nli_eta(o(egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(o(egn.EGN_PREC_FP32C))
    db = np.abs(10 * np.log10(e32 / e64))
    assert np.max(db) < 1e-3, db
    ln.close()


def test_ridge_fp32c_matches_fp64_on_a_wide_link(egn, workloads):
    """40 channels of the 75 GHz C+L grid (2.9 THz wide) over ten spans: FP32C
    against the FP64 ridge kernel on every channel within 1e-3 dB (the narrowest
    ridges: their half-widths fall as 1 / |f2 - f|)."""
    wl = workloads.config_cl(n_ch=40)
    ln = _ridge_link(egn, wl)
    o = lambda pr: egn.make_opts(gl_order=8, dz_km=wl.dz_km, precision=pr)  # noqa: E731
    e64, _ = ln.nli_eta(o(egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(o(egn.EGN_PREC_FP32C))
    db = np.abs(10 * np.log10(e32 / e64))
    assert np.max(db) < 1e-3, db
    ln.close()


def test_ridge_rule_converges_where_the_configured_rule_does_not(egn, workloads):
    """GN part: 16 and 32 nodes per piece within 0.003 dB; with the EGN corrections
    (which need more nodes) within 0.04 dB; the configured rule moves by more than
    0.3 dB from 32 x 32 to 64 x 64."""
    wl = workloads.config_small(gl_order=16)
    ln = egn.link_from_workload(wl)
    o = lambda n, t: egn.make_opts(gl_order=n, precision=egn.EGN_PREC_FP64, terms=t)  # noqa: E731
    plain32, _ = ln.nli_eta(o(32, egn.EGN_TERMS_EGN))
    plain64, _ = ln.nli_eta(o(64, egn.EGN_TERMS_EGN))
    ln.set_node_rule(egn.EGN_RULE_RIDGE, 4)
    db = lambda a, b: np.abs(10 * np.log10(a / b))  # noqa: E731
    for terms, bar in ((egn.EGN_TERMS_GN, 3e-3), (egn.EGN_TERMS_EGN, 0.04)):
        r16, _ = ln.nli_eta(o(16, terms))
        r32, _ = ln.nli_eta(o(32, terms))
        assert np.max(db(r16, r32)) < bar, (terms, db(r16, r32))
    assert np.max(db(plain32, plain64)) > 0.3, db(plain32, plain64)
    ln.set_node_rule(egn.EGN_RULE_GL)  # back to the configured rule: the same results as before
    again, _ = ln.nli_eta(o(32, egn.EGN_TERMS_EGN))
    assert np.array_equal(again, plain32)
    ln.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_ridge_rule_in_a_batch_equals_single_links(egn, workloads, prec):
    opts = egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C)
    wh = workloads.config_small(n_ch=3, gl_order=8, n_spans=3)  # two span types
    wh.spans[1].length_m = 65e3
    wls = [workloads.config_small(n_ch=4, gl_order=8), workloads.config_small(n_ch=3, gl_order=8, n_spans=2), wh]
    links = [_ridge_link(egn, w) for w in wls]
    want = [ln.nli_eta(opts) for ln in links]
    b = egn.Batch(links, opts)
    b.launch()
    for (ge, gp), (we, wp) in zip(b.read(), want):
        assert np.array_equal(ge, we) and np.array_equal(gp, wp)
    b.close()


def test_ridge_rule_refusals(egn, workloads):
    import torch
    wh = workloads.config_small(n_ch=2, gl_order=8, n_spans=5)
    for i, sp in enumerate(wh.spans):
        sp.length_m = (60 + 5 * i) * 1e3
    lh = _ridge_link(egn, wh)  # five span types: FP64 only
    with pytest.raises(egn.EgnError) as ei:
        lh.nli_eta(egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP32C))
    assert ei.value.status == egn.EGN_E_UNSUPPORTED
    lh.close()
    wl = workloads.config_small(n_ch=2, gl_order=8)
    ln = _ridge_link(egn, wl)
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts(gl_order=65, precision=egn.EGN_PREC_FP32C))
    assert ei.value.status == egn.EGN_E_INVALID_ARG
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts(gl_order=65, precision=egn.EGN_PREC_FP64))
    assert ei.value.status == egn.EGN_E_INVALID_ARG
    eta = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta_static(egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP64), eta, eta)
    assert ei.value.status == egn.EGN_E_UNSUPPORTED
    for rule, n_min in ((7, 4), (egn.EGN_RULE_RIDGE, 0)):
        with pytest.raises(egn.EgnError) as ei:
            ln.set_node_rule(rule, n_min)
        assert ei.value.status == egn.EGN_E_INVALID_ARG
    ln.close()
