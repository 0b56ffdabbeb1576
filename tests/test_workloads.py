"""The seeded input generators (no GPU): the splitmix64 stream against its published
outputs, and the workloads' grids, powers and ranges against the values they are
built from (Table I and II of Sec. III-A and App. C, the C+L link, the random
heterogeneous links of the batched path)."""
import math

import numpy as np


def test_splitmix64_published_outputs(workloads):
    # first outputs of splitmix64 (Steele, Lea, Flood 2014) for seeds 0 and 1234567
    r = workloads.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]
    r = workloads.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                                9817491932198370423]


def test_splitmix64_derived_draws(workloads):
    r = workloads.SplitMix64(11)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    k = np.array([r.randint(3, 7) for _ in range(20000)])
    assert set(k.tolist()) == {3, 4, 5, 6, 7}
    g = np.array([r.normal() for _ in range(20000)])
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.03


def test_grid_and_power_units(workloads):
    c = workloads.grid(4, 75e9, 193e12)
    assert np.allclose(np.diff(c), 75e9) and math.isclose(0.5 * (c[0] + c[-1]), 193e12)
    assert math.isclose(workloads.dbm_to_w(0.0), 1e-3) and math.isclose(workloads.dbm_to_w(30.0), 1.0)


def test_tables_of_the_paper(workloads):
    t1 = workloads.table1()
    assert t1.n_ch == 101 and np.allclose(np.diff(t1.centre_hz), 10.1e9)
    assert math.isclose(sum(t1.launch_power_w), workloads.dbm_to_w(19.0))
    assert t1.spans[0].length_m == 100e3 and t1.spans[0].S_ps_nm2_km == 0.0
    t2 = workloads.table2()
    assert t2.n_ch == 101 and np.allclose(np.diff(t2.centre_hz), 101e9)
    assert math.isclose(sum(t2.launch_power_w), workloads.dbm_to_w(25.0))
    assert set(t2.symbol_rate_baud) == {100e9} and len(t2.spans) == 1


def test_cl_link(workloads):
    w = workloads.config_cl()
    c = np.asarray(w.centre_hz)
    assert w.n_ch == 120 and np.allclose(np.diff(c), 75e9)
    assert c[-1] - c[0] == 119 * 75e9 and len(w.spans) == 10
    lo, hi = workloads.C_M_PER_S / 1605e-9, workloads.C_M_PER_S / 1530e-9
    assert lo < c[0] and c[-1] < hi
    assert w.formats == workloads.config_cl().formats and w.formats != workloads.config_cl(seed=1).formats
    assert set(w.formats) == set(workloads.FORMATS)


def test_random_links_are_seeded_and_in_range(workloads):
    a, b = workloads.random_link(5), workloads.random_link(5)
    assert a.launch_power_w == b.launch_power_w and a.formats == b.formats and a.spans == b.spans
    fibres = {(f["alpha_db_km"], f["gamma_per_w_km"]) for f in (workloads.SSMF, workloads.PSCF)}
    for seed in range(300):
        w = workloads.random_link(seed)
        R = w.symbol_rate_baud[0]
        assert set(w.symbol_rate_baud) == {R} and 32e9 <= R <= 96e9
        sp = np.diff(w.centre_hz)
        spacing = sp[0]
        assert np.allclose(sp, spacing)
        assert max(50e9, math.ceil(1.01 * R / 1e9) * 1e9) - 1 <= spacing <= 150e9 + 1
        assert 1 <= w.n_ch <= 200 and w.n_ch * spacing <= 12e12 + 1
        assert spacing >= R * (1 + w.rolloff)   # no two channels' supports overlap
        assert 1 <= len(w.spans) <= 30
        for s in w.spans:
            assert 50e3 <= s.length_m <= 120e3 and (s.alpha_db_km, s.gamma_per_w_km) in fibres
        p_dbm = 10 * np.log10(np.asarray(w.launch_power_w) / 1e-3)
        assert np.all(np.isfinite(p_dbm)) and -8.0 < p_dbm.min() and p_dbm.max() < 10.0
        assert set(w.formats) <= set(workloads.FORMATS) and len(w.formats) == w.n_ch


def test_tables_match_the_printed_parameters(workloads):
    """table1 / table2 carry the parameters printed in Table I and Table II (the
    golden fixture quotes them with their citation)."""
    import json
    import pathlib
    gold = json.loads((pathlib.Path(__file__).parent / "golden" / "paper_values.json").read_text())
    for name in ("table1", "table2"):
        g = gold[name]
        n_sp = g["n_spans"] if isinstance(g["n_spans"], list) else [g["n_spans"]]
        cr = g["cr"] if isinstance(g["cr"], list) else [g["cr"]]
        for ns in n_sp:
            for c in cr:
                w = workloads.table1(n_spans=ns, cr=c) if name == "table1" else workloads.table2()
                s = w.spans[0]
                assert w.n_ch == g["n_ch"] and len(w.spans) == ns
                assert s.length_m == g["span_km"] * 1e3 and s.alpha_db_km == g["alpha_db_km"]
                assert s.D_ps_nm_km == g["D"] and s.S_ps_nm2_km == g["S"] and s.gamma_per_w_km == g["gamma"]
                assert s.cr_per_w_km_thz == c
                assert math.isclose(w.symbol_rate_baud[0], g["R_gbd"] * 1e9)
                assert math.isclose(w.centre_hz[1] - w.centre_hz[0], g["spacing_ghz"] * 1e9, rel_tol=1e-9)
                assert math.isclose(10 * math.log10(sum(w.launch_power_w) / 1e-3), g["ptot_dbm"], abs_tol=1e-9)
