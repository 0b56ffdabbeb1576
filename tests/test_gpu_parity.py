"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on the
same seeded inputs.

Tolerances (stated per test):
  * island lists: bit-exact (the same set, in the same order);
  * FP64 path: eta and per-island terms within 1e-9 relative (both sides FP64;
    differences come from Horner vs term-by-term summation and node rounding);
  * FP32C path: every channel within 0.01 dB of the oracle (the accuracy target),
    and within 1e-3 dB on the small workloads.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-9


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


def _pair(egn, oracle_mod, wl, gl=None, terms=1):
    ln = egn.link_from_workload(wl)
    pb = oracle_mod.Problem(wl, gl_order=gl or wl.gl_order, terms=terms)
    return ln, pb


def _db(a, b):
    return np.abs(10 * np.log10(np.asarray(a) / np.asarray(b)))


# --------------------------------------------------------------------------- planner

@pytest.mark.parametrize("n_ch", [1, 2, 5, 11])
def test_island_list_bit_exact(egn, oracle_mod, workloads, n_ch):
    wl = workloads.config_small(n_ch=n_ch, gl_order=8)
    ln, pb = _pair(egn, oracle_mod, wl)
    got = ln.plan_islands()
    want = np.array([(n, *t) for n in range(n_ch) for t in pb.islands(n)], dtype=np.int32).reshape(-1, 4)
    assert np.array_equal(got, want)
    tot, per, nh, ne, nf = ln.island_count()
    assert tot == len(want)
    n1, n2, n3 = want[:, 1], want[:, 2], want[:, 3]
    assert nh == int(np.sum(n1 <= n2))
    assert ne == int(np.sum((n1 == n3) & (n1 <= n2))) and nf == int(np.sum((n2 == n3) & (n1 < n2)))
    # every island's mirror (n2, n1, n3) is an island too
    s = {tuple(r) for r in want}
    assert all((c, b, a, d) in s for c, a, b, d in s)


def test_island_list_irregular_comb(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=6, gl_order=8)
    base = wl.centre_hz[0]
    wl.centre_hz = [base, base + 61e9, base + 140e9, base + 197e9, base + 262e9, base + 400e9]
    wl.symbol_rate_baud = [40e9, 60e9, 32e9, 50e9, 64e9, 96e9]
    wl.formats = ["GAUSS"] * 6
    ln, pb = _pair(egn, oracle_mod, wl)
    got = ln.plan_islands()
    want = np.array([(n, *t) for n in range(6) for t in pb.islands(n)], dtype=np.int32).reshape(-1, 4)
    assert np.array_equal(got, want)


def test_island_count_config_cl(egn, workloads):
    # 120 ch on a 75 GHz grid with 64.64 GHz supports: Eq. 16 counts
    wl = workloads.config_cl()
    ln = egn.link_from_workload(wl)
    tot, per, nh, ne, nf = ln.island_count()
    M = 120
    want = 0
    for n in range(M):
        for l in (-1, 0, 1):
            for n1 in range(M):
                lo, hi = max(0, n - l - n1), min(M - 1, M - 1 + n - l - n1)
                want += max(0, hi - lo + 1)
    assert tot == want == 3455880


# --------------------------------------------------------------------------- FP64 path

@pytest.mark.parametrize("terms", [0, 1])
def test_fp64_eta_small(egn, oracle_mod, workloads, terms):
    wl = workloads.config_small(gl_order=64)
    ln, pb = _pair(egn, oracle_mod, wl, terms=terms)
    got, gp = ln.nli_eta(egn.make_opts(gl_order=64, precision=egn.EGN_PREC_FP64, terms=terms))
    want, wp = pb.eta()
    assert np.allclose(got, want, rtol=FP64_RTOL, atol=0), (got / want - 1)
    assert np.allclose(gp, wp, rtol=FP64_RTOL, atol=0)


@pytest.mark.parametrize("gl", [1, 7, 13, 32])
def test_fp64_island_terms_all(egn, oracle_mod, workloads, gl):
    """All five terms on every island (ragged outer panels: ceil(n/2) nodes)."""
    wl = workloads.config_small(gl_order=gl, n_ch=3)
    ln, pb = _pair(egn, oracle_mod, wl, gl=gl)
    isl = np.array([(n, *t) for n in range(3) for t in pb.islands(n)], dtype=np.int32)
    got = ln.island_terms(egn.make_opts(gl_order=gl, precision=egn.EGN_PREC_FP64), isl, all_terms=True)
    want = np.array([pb.island_terms(*row, all_terms=True) for row in isl])
    assert np.allclose(got, want, rtol=FP64_RTOL, atol=1e-300)


def test_fp64_multispan_and_mixed_widths(egn, oracle_mod, workloads):
    """5 spans (phased array), irregular comb with three different widths (three
    outer panels on some islands), GN terms (mixed rates)."""
    wl = workloads.config_small(n_ch=4, gl_order=12, n_spans=5)
    base = wl.centre_hz[0]
    wl.centre_hz = [base, base + 61e9, base + 140e9, base + 197e9]
    wl.symbol_rate_baud = [40e9, 60e9, 32e9, 50e9]
    ln, pb = _pair(egn, oracle_mod, wl, terms=0)
    got, _ = ln.nli_eta(egn.make_opts(gl_order=12, precision=egn.EGN_PREC_FP64, terms=0))
    want, _ = pb.eta()
    assert np.allclose(got, want, rtol=FP64_RTOL, atol=0)


def test_fp64_single_channel_and_dz(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=1, gl_order=16)
    ln = egn.link_from_workload(wl)
    for dz in (1.0, 0.7, 7.0):
        pb = oracle_mod.Problem(wl, dz_km=dz)
        got, _ = ln.nli_eta(egn.make_opts(gl_order=16, dz_km=dz, precision=egn.EGN_PREC_FP64))
        want, _ = pb.eta()
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=0), dz


def test_fp64_config_cl_sampled_islands(egn, oracle_mod, workloads):
    """Full C+L workload (120 ch, 10 x 80 km, 32 x 32): per-island terms of a seeded
    sample of islands (all COIs, all kinds) against the oracle one by one."""
    wl = workloads.config_cl()
    ln, pb = _pair(egn, oracle_mod, wl)
    plan = ln.plan_islands()
    rng = np.random.default_rng(7)
    pick = np.concatenate([rng.choice(len(plan), 40, replace=False),
                           np.flatnonzero(plan[:, 1] == plan[:, 3])[:: 5000],
                           np.flatnonzero((plan[:, 1] == plan[:, 2]) & (plan[:, 2] == plan[:, 3]))[:: 40]])
    isl = plan[pick]
    got = ln.island_terms(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP64), isl)
    want = np.array([pb.island_terms(*row) for row in isl])
    assert np.allclose(got, want, rtol=1e-8, atol=1e-300)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_200_channel_link_sampled_islands(egn, oracle_mod, workloads, prec):
    """The largest comb of the seeded random links: 200 channels x 32 GBd on a 50 GHz
    grid (10 THz), 6 x 80 km; per-island terms of a seeded sample (all kinds) against
    the oracle one by one, and the planned list's size against the island count."""
    wl = workloads.config_small(n_ch=200, gl_order=12, n_spans=6)
    base = wl.centre_hz[100]
    wl.centre_hz = [base + (k - 99.5) * 50e9 for k in range(200)]
    wl.symbol_rate_baud = [32e9] * 200
    rng = np.random.default_rng(3)
    wl.formats = [("QPSK", "16QAM", "64QAM", "GAUSS")[i] for i in rng.integers(0, 4, 200)]
    ln, pb = _pair(egn, oracle_mod, wl, gl=12)
    plan = ln.plan_islands()
    assert len(plan) == ln.island_count()[0] and len(plan) > 4_000_000
    pick = np.concatenate([rng.choice(len(plan), 30, replace=False),
                           np.flatnonzero(plan[:, 1] == plan[:, 3])[:: 20000],
                           np.flatnonzero(plan[:, 1] == plan[:, 2])[:: 20000],
                           np.flatnonzero((plan[:, 1] == plan[:, 2]) & (plan[:, 2] == plan[:, 3]))[:: 50]])
    isl = plan[pick]
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got = ln.island_terms(egn.make_opts(gl_order=12, precision=p), isl)
    want = np.array([pb.island_terms(*row) for row in isl])
    if prec == "fp64":
        assert np.allclose(got, want, rtol=1e-8, atol=1e-300)
    else:
        err = np.abs(got - want)
        assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * np.abs(want[:, :1]))


def test_device_api_matches_host_api(egn, workloads):
    import torch
    wl = workloads.config_small(gl_order=16)
    ln = egn.link_from_workload(wl)
    s = torch.cuda.Stream()
    opts = egn.make_opts(gl_order=16, precision=egn.EGN_PREC_FP64, stream=s.cuda_stream)
    ws = torch.empty(ln.workspace_size(opts), dtype=torch.uint8, device="cuda")
    eta = torch.empty(5, dtype=torch.float64, device="cuda")
    pn = torch.empty(5, dtype=torch.float64, device="cuda")
    ln.nli_eta_device(opts, ws, eta, pn)
    s.synchronize()
    h_eta, h_pn = ln.nli_eta(egn.make_opts(gl_order=16, precision=egn.EGN_PREC_FP64))
    assert np.array_equal(eta.cpu().numpy(), h_eta)
    assert np.array_equal(pn.cpu().numpy(), h_pn)


def test_repeatable_bitwise(egn, workloads):
    wl = workloads.config_small(gl_order=16)
    ln = egn.link_from_workload(wl)
    o = egn.make_opts(gl_order=16, precision=egn.EGN_PREC_FP64)
    a, _ = ln.nli_eta(o)
    b, _ = ln.nli_eta(o)
    assert np.array_equal(a, b)


def test_workspace_too_small_is_rejected(egn, workloads):
    import torch
    wl = workloads.config_small(gl_order=8)
    ln = egn.link_from_workload(wl)
    o = egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP64)
    ws = torch.empty(ln.workspace_size(o) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta_device(o, ws)
    assert ei.value.status == egn.EGN_E_CAPACITY


def _mixed_link(workloads, n_ch=3, gl=12):
    """Four spans of two fibre types and three lengths (three span types)."""
    wl = workloads.config_small(n_ch=n_ch, gl_order=gl, n_spans=4)
    pscf = dict(alpha_db_km=0.16, D_ps_nm_km=21.0, gamma_per_w_km=0.8)
    for k, v in pscf.items():
        setattr(wl.spans[1], k, v)
        setattr(wl.spans[3], k, v)
    wl.spans[2].length_m = 55e3
    wl.spans[3].length_m = 101e3
    return wl


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_heterogeneous_spans_eta(egn, oracle_mod, workloads, prec):
    """Eq. 22 as an explicit coherent sum over spans of different fibres and lengths."""
    wl = _mixed_link(workloads)
    ln, pb = _pair(egn, oracle_mod, wl)
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got, _ = ln.nli_eta(egn.make_opts(gl_order=12, precision=p))
    want, _ = pb.eta()
    if prec == "fp64":
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=0), got / want - 1
    else:
        assert np.max(_db(got, want)) < 1e-3, _db(got, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_heterogeneous_spans_island_terms(egn, oracle_mod, workloads, prec):
    wl = _mixed_link(workloads, gl=9)
    ln, pb = _pair(egn, oracle_mod, wl, gl=9)
    isl = np.array([(n, *t) for n in range(3) for t in pb.islands(n)], dtype=np.int32)
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got = ln.island_terms(egn.make_opts(gl_order=9, precision=p), isl, all_terms=True)
    want = np.array([pb.island_terms(*row, all_terms=True) for row in isl])
    if prec == "fp64":
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=1e-300)
    else:
        err = np.abs(got - want)
        assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * np.abs(want[:, :1]))


def _many_types_link(workloads, n_ch=3, gl=10):
    """Seven spans of six types: lengths 55..115 km, SSMF and PSCF, the first
    type again at the end (a type that recurs after others)."""
    wl = workloads.config_small(n_ch=n_ch, gl_order=gl, n_spans=7)
    for i, s in enumerate(wl.spans[:6]):
        s.length_m = (55 + 12 * i) * 1e3
        if i % 2:
            s.alpha_db_km, s.D_ps_nm_km, s.gamma_per_w_km = 0.16, 21.0, 0.8
    last = wl.spans[6]
    for k, v in wl.spans[0].__dict__.items():
        setattr(last, k, v)
    return wl


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_sixty_three_span_types_four_fibres(egn, oracle_mod, workloads, prec):
    """63 spans of 63 types on four fibres (attenuations 0.16..0.22 dB/km, lengths
    60..122 km): the span-by-span path with the most types and fibre tables its
    shared memory holds, where the fewest rows per chunk (an odd number) fit; eta
    of every channel against the oracle."""
    wl = workloads.config_small(n_ch=3, gl_order=6, n_spans=63)
    for i, sp in enumerate(wl.spans):
        sp.length_m = (60 + i) * 1e3
        sp.alpha_db_km = (0.16, 0.18, 0.20, 0.22)[i % 4]
    ln, pb = _pair(egn, oracle_mod, wl)
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got, _ = ln.nli_eta(egn.make_opts(gl_order=6, precision=p))
    want, _ = pb.eta()
    if prec == "fp64":
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=0), (got, want)
    else:
        assert np.max(_db(got, want)) < 1e-3, _db(got, want)
    ln.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_many_span_types_eta(egn, oracle_mod, workloads, prec):
    """More than four span types: Eq. 22 walked span by span (c_k on the fly)."""
    wl = _many_types_link(workloads)
    ln, pb = _pair(egn, oracle_mod, wl)
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got, _ = ln.nli_eta(egn.make_opts(gl_order=10, precision=p))
    want, _ = pb.eta()
    if prec == "fp64":
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=0), got / want - 1
    else:
        assert np.max(_db(got, want)) < 1e-3, _db(got, want)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_many_span_types_island_terms(egn, oracle_mod, workloads, prec):
    wl = _many_types_link(workloads, gl=7)
    ln, pb = _pair(egn, oracle_mod, wl, gl=7)
    isl = np.array([(n, *t) for n in range(3) for t in pb.islands(n)], dtype=np.int32)
    p = egn.EGN_PREC_FP64 if prec == "fp64" else egn.EGN_PREC_FP32C
    got = ln.island_terms(egn.make_opts(gl_order=7, precision=p), isl, all_terms=True)
    want = np.array([pb.island_terms(*row, all_terms=True) for row in isl])
    if prec == "fp64":
        assert np.allclose(got, want, rtol=FP64_RTOL, atol=1e-300)
    else:
        err = np.abs(got - want)
        assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * np.abs(want[:, :1]))


@pytest.mark.parametrize("seed", [1, 2, 5])
def test_random_link_spans(egn, oracle_mod, workloads, seed):
    """The spans of the seeded random links (up to 30, each length drawn) on a
    4-channel comb of the link's rate, FP32C against the oracle."""
    rl = workloads.random_link(seed)
    wl = workloads.config_small(n_ch=4, gl_order=8)
    wl.spans = rl.spans
    ln, pb = _pair(egn, oracle_mod, wl)
    got, _ = ln.nli_eta(egn.make_opts(gl_order=8, precision=egn.EGN_PREC_FP32C))
    want, _ = pb.eta()
    assert np.max(_db(got, want)) < 1e-3, (len(rl.spans), _db(got, want))


def test_more_than_64_differing_spans_unsupported(egn, workloads):
    wl = workloads.config_small(n_spans=65)
    for i, s in enumerate(wl.spans):
        s.length_m = (50 + i) * 1e3
    ln = egn.link_from_workload(wl)
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts())
    assert ei.value.status == egn.EGN_E_UNSUPPORTED


def test_more_than_2_32_islands_refused(egn, workloads):
    """1700 channels on a 75 GHz grid hold about 2 x 1700^3 = 9.8e9 islands: the
    planner's 64-bit totals exceed the 32-bit island indices, so egn_set_wdm refuses
    the comb (and leaves the link without a WDM); 1200 channels (3.5e9) are counted."""
    wl = workloads.config_small(n_ch=1700, gl_order=8)
    ln = egn.Link(wl.spans)
    n = len(wl.centre_hz)
    phi = np.zeros(n)
    with pytest.raises(egn.EgnError) as ei:
        ln.set_wdm(wl.centre_hz, wl.symbol_rate_baud, wl.launch_power_w, phi, phi, wl.rolloff)
    assert ei.value.status == egn.EGN_E_UNSUPPORTED and "2^32" in str(ei.value)
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts(gl_order=8))
    assert ei.value.status == egn.EGN_E_STATE
    wl2 = workloads.config_small(n_ch=1200, gl_order=8)
    ln.set_wdm(wl2.centre_hz, wl2.symbol_rate_baud, wl2.launch_power_w, np.zeros(1200), np.zeros(1200), wl2.rolloff)
    total = ln.island_count()[0]
    assert 3.0e9 < total < 2 ** 32
    ln.close()


# --------------------------------------------------------------------------- FP32C path

FP32C_DB = 1e-3      # small workloads
TARGET_DB = 0.01     # the accuracy target at full size


@pytest.mark.parametrize("terms", [0, 1])
def test_fp32c_eta_small(egn, oracle_mod, workloads, terms):
    wl = workloads.config_small(gl_order=64)
    ln, pb = _pair(egn, oracle_mod, wl, terms=terms)
    got, gp = ln.nli_eta(egn.make_opts(gl_order=64, precision=egn.EGN_PREC_FP32C, terms=terms))
    want, wp = pb.eta()
    assert np.max(_db(got, want)) < FP32C_DB, _db(got, want)
    assert np.max(_db(gp, wp)) < FP32C_DB


@pytest.mark.parametrize("gl", [1, 7, 13, 32])
def test_fp32c_island_terms_all(egn, oracle_mod, workloads, gl):
    wl = workloads.config_small(gl_order=gl, n_ch=3, n_spans=3)
    ln, pb = _pair(egn, oracle_mod, wl, gl=gl)
    isl = np.array([(n, *t) for n in range(3) for t in pb.islands(n)], dtype=np.int32)
    got = ln.island_terms(egn.make_opts(gl_order=gl, precision=egn.EGN_PREC_FP32C), isl, all_terms=True)
    want = np.array([pb.island_terms(*row, all_terms=True) for row in isl])
    scale = np.abs(want[:, :1])  # |D| of the island bounds every term's rounding
    err = np.abs(got - want)
    assert np.all(err <= 3e-4 * np.abs(want) + 3e-5 * scale), np.max(err / (np.abs(want) + 1e-300))


def test_fp32c_multispan_mixed_widths(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=4, gl_order=12, n_spans=5)
    base = wl.centre_hz[0]
    wl.centre_hz = [base, base + 61e9, base + 140e9, base + 197e9]
    wl.symbol_rate_baud = [40e9, 60e9, 32e9, 50e9]
    ln, pb = _pair(egn, oracle_mod, wl, terms=0)
    got, _ = ln.nli_eta(egn.make_opts(gl_order=12, precision=egn.EGN_PREC_FP32C, terms=0))
    want, _ = pb.eta()
    assert np.max(_db(got, want)) < FP32C_DB


@pytest.mark.parametrize("dz", [1.0, 0.7, 7.0, 80.0])
def test_fp32c_segment_counts(egn, oracle_mod, workloads, dz):
    """K = 80, 115 (K mod 4 = 3), 12, 1 segments."""
    wl = workloads.config_small(n_ch=3, gl_order=16, n_spans=2)
    ln = egn.link_from_workload(wl)
    got, _ = ln.nli_eta(egn.make_opts(gl_order=16, dz_km=dz, precision=egn.EGN_PREC_FP32C))
    want, _ = oracle_mod.Problem(wl, dz_km=dz).eta()
    assert np.max(_db(got, want)) < FP32C_DB, dz


def test_fp32c_single_channel(egn, oracle_mod, workloads):
    wl = workloads.config_small(n_ch=1, gl_order=32)
    ln, pb = _pair(egn, oracle_mod, wl)
    got, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C))
    want, _ = pb.eta()
    assert np.max(_db(got, want)) < FP32C_DB


def test_fp32c_config_cl_sampled_islands(egn, oracle_mod, workloads):
    wl = workloads.config_cl()
    ln, pb = _pair(egn, oracle_mod, wl)
    plan = ln.plan_islands()
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(len(plan), 40, replace=False),
                           np.flatnonzero(plan[:, 1] == plan[:, 3])[:: 5000],
                           np.flatnonzero(plan[:, 2] == plan[:, 3])[:: 5000],
                           np.flatnonzero((plan[:, 1] == plan[:, 2]) & (plan[:, 2] == plan[:, 3]))[:: 40]])
    isl = plan[pick]
    got = ln.island_terms(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C), isl)
    want = np.array([pb.island_terms(*row) for row in isl])
    scale = np.abs(want[:, :1])
    err = np.abs(got - want)
    assert np.all(err <= 1e-3 * np.abs(want) + 1e-4 * scale), np.max(err / (np.abs(want) + 1e-300))


def test_config_cl_full_size_sampled_channels(egn, oracle_mod, workloads):
    """The benchmarked launch (120 ch, 10 x 80 km, 32 x 32, EGN) for all channels on
    the GPU in both precisions; the oracle evaluates two full channels (edge and
    centre), which it can do one by one."""
    wl = workloads.config_cl()
    ln, pb = _pair(egn, oracle_mod, wl)
    e64, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C))
    assert np.max(_db(e32, e64)) < TARGET_DB
    cois = [0, 59]
    want, _ = pb.eta(cois)
    assert np.allclose(e64[cois], want, rtol=1e-8, atol=0)
    assert np.max(_db(e32[cois], want)) < TARGET_DB


def test_config_cl_thirty_spans(egn, workloads):
    """The 120-channel C+L link over 30 identical spans (the longest links of the
    batch workload): N phi / 2 of the phased array is largest here, so the FP32
    small-angle series near its poles and the double-float phase are most exposed.
    FP32C against FP64 on every channel within 0.01 dB."""
    wl = workloads.config_cl(n_spans=30)
    ln = egn.link_from_workload(wl)
    e64, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C))
    assert np.all(np.isfinite(e32)) and np.max(_db(e32, e64)) < TARGET_DB, np.max(_db(e32, e64))
    ln.close()


def test_random_link_full_size(egn, oracle_mod, workloads):
    """A seeded link of the batch workload at full size: random_link(2), 50
    channels of 37 GBd on a 116 GHz grid, tilted rippled powers, 29 SSMF/PSCF spans
    of 26 types (the span-by-span path), 16 x 16 nodes.  FP32C against FP64 on
    every channel within 0.01 dB; FP64 against the oracle on the centre channel
    within 1e-8."""
    wl = workloads.random_link(2)
    ln, pb = _pair(egn, oracle_mod, wl)
    e64, _ = ln.nli_eta(egn.make_opts(gl_order=wl.gl_order, precision=egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(egn.make_opts(gl_order=wl.gl_order, precision=egn.EGN_PREC_FP32C))
    assert np.max(_db(e32, e64)) < TARGET_DB, np.max(_db(e32, e64))
    coi = [wl.n_ch // 2]
    want, _ = pb.eta(coi)
    assert np.allclose(e64[coi], want, rtol=1e-8, atol=0), (e64[coi], want)
    ln.close()


@pytest.mark.parametrize("p_dbm", [-2.0, 4.0])
def test_config3_power_sweep(egn, oracle_mod, workloads, p_dbm):
    """The benchmark link at the ends of the launch-power sweep, -2 and +4 dBm/ch
    (the strongest ISRS: P_tot 24.8 dBm, about 6.9 dB of power transfer across the
    band per span by Eq. 12), where the FP32C design (double-float phase, FP32
    phased-array series near its poles) is most exposed.  FP32C against the plain
    FP64 path on every channel within the 0.01 dB accuracy target; FP64 against the
    oracle on the edge and a centre channel within 1e-8 relative."""
    wl = workloads.config_cl(p_dbm=p_dbm)
    ln, pb = _pair(egn, oracle_mod, wl)
    e64, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP64))
    e32, _ = ln.nli_eta(egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C))
    assert np.all(np.isfinite(e32)) and np.all(e32 > 0)
    assert np.max(_db(e32, e64)) < TARGET_DB, (p_dbm, int(np.argmax(_db(e32, e64))), np.max(_db(e32, e64)))
    cois = [0, 59]
    want, _ = pb.eta(cois)
    assert np.allclose(e64[cois], want, rtol=1e-8, atol=0)
    assert np.max(_db(e32[cois], want)) < TARGET_DB
    ln.close()


def test_fp32c_launch_shapes_agree(egn, oracle_mod, workloads):
    """2, 4 and 8 points per thread in the FP32C D/G/H pass: same terms up to rounding."""
    wl = workloads.config_small(n_ch=5, gl_order=32, n_spans=3)
    ln, pb = _pair(egn, oracle_mod, wl)
    o = egn.make_opts(gl_order=32, precision=egn.EGN_PREC_FP32C)
    a, _ = ln.nli_eta(o)
    want, _ = pb.eta()
    for kp in (8, 2):
        ln.set_tuning(egn.EGN_TUNE_FP32C_POINTS_PER_THREAD, kp)
        b, _ = ln.nli_eta(o)
        assert np.max(_db(a, b)) < 1e-4, kp
        assert np.max(_db(b, want)) < FP32C_DB, kp
