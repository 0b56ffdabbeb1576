"""Pins of the oracle's island enumeration (Eq. 15-16) and node rule geometry."""
import itertools
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def t_kappa(M, kappa):
    """Eq. 16 written out as a set comprehension."""
    return {(k1, k2, l) for k1 in range(-M, M + 1) for k2 in range(-M, M + 1) for l in (-1, 0, 1)
            if -M <= k1 + k2 - kappa + l <= M}


def oracle_set(pb, M, n):
    isl = pb.islands(n)
    out = set()
    for n1, n2, n3 in isl:
        k1, k2, kappa = n1 - M, n2 - M, n - M
        l = (n3 - M) - (k1 + k2 - kappa)
        out.add((k1, k2, l))
    return out


@pytest.mark.parametrize("n_ch", [5, 7, 11])
def test_islands_equal_eq16_uniform_grid(oracle_mod, workloads, n_ch):
    # 64 GBd * 1.01 on a 75 GHz grid: 2/3 spacing < channel width < spacing
    wl = workloads.config_small(n_ch=n_ch)
    pb = oracle_mod.Problem(wl)
    M = (n_ch - 1) // 2
    for n in range(n_ch):
        assert oracle_set(pb, M, n) == t_kappa(M, n - M)


def test_island_count_small_config(oracle_mod, workloads):
    pb = oracle_mod.Problem(workloads.config_small())
    counts = [len(pb.islands(n)) for n in range(5)]
    assert sum(counts) == 245
    l0 = sum(1 for n in range(5) for n1, n2, n3 in pb.islands(n) if n3 == n1 + n2 - n)
    assert l0 == 85


def test_narrow_channels_only_l0(oracle_mod, workloads):
    """Sec. II-B: with B_ch <= 2/3 of the spacing only l = 0 islands exist."""
    wl = workloads.config_small(n_ch=7)
    wl.symbol_rate_baud = [40e9] * 7  # 40.4 GHz support on a 75 GHz grid
    pb = oracle_mod.Problem(wl)
    M = 3
    for n in range(7):
        want = {t for t in t_kappa(M, n - M) if t[2] == 0}
        assert oracle_set(pb, M, n) == want


def test_no_island_when_supports_only_touch(oracle_mod, workloads):
    # width == spacing: |d| = 1.5 W islands would touch in a single point -> excluded
    wl = workloads.config_small(n_ch=5)
    wl.symbol_rate_baud = [50e9] * 5
    wl.rolloff = 0.0
    wl.centre_hz = [wl.centre_hz[2] + (k - 2) * 50e9 for k in range(5)]
    pb = oracle_mod.Problem(wl)
    for n in range(5):
        for n1, n2, n3 in pb.islands(n):
            assert abs((n1 + n2 - n) - n3) <= 1


def test_islands_nonuniform_grid_brute_force(oracle_mod, workloads):
    """Mixed widths and irregular spacing: the island set is exactly the set of
    (n1, n2, n3) whose three supports admit a 2-D region of positive area,
    checked by sampling a fine (u, v) grid."""
    wl = workloads.config_small(n_ch=4)
    wl.centre_hz = [1.93e14, 1.93e14 + 61e9, 1.93e14 + 140e9, 1.93e14 + 197e9]
    wl.symbol_rate_baud = [40e9, 60e9, 32e9, 50e9]
    wl.rolloff = 0.0
    pb = oracle_mod.Problem(wl)
    nu, W = pb.nu, pb.R
    for n in range(4):
        got = {tuple(t) for t in pb.islands(n)}
        want = set()
        for n1, n2, n3 in itertools.product(range(4), repeat=3):
            u = np.linspace(-W[n1] / 2, W[n1] / 2, 161)[1:-1]
            v = np.linspace(-W[n2] / 2, W[n2] / 2, 161)[1:-1]
            uu, vv = np.meshgrid(u, v)
            w = nu[n1] + nu[n2] - nu[n] - nu[n3] + uu + vv
            if np.any(np.abs(w) < W[n3] / 2 * (1 - 1e-9)):
                want.add((n1, n2, n3))
        assert got == want, n


def test_max_phase_product_over_domain(oracle_mod, workloads):
    """Sec. II-C: max |(f1 - f)(f2 - f)| over the domain is B^2/4 for the centre and
    the edge COI and 3 B^2/16 for the quarter COI (101 ch, 1 THz)."""
    g = json.load(open(GOLDEN))["max_abs_f1f_f2f"]["coi_offset_fraction"]
    wl = workloads.table1(gl_order=4)
    pb = oracle_mod.Problem(wl, gl_order=4)
    B = pb.btot
    for off, frac in g.items():
        n = 50 + int(off)
        f = pb.nu[n]
        best = 0.0
        for n1, n2, n3 in pb.islands(n):
            nodes = pb.island_nodes(n, n1, n2, n3)
            f1 = pb.nu[n1] + nodes[:, 0]
            f2 = pb.nu[n2] + nodes[:, 1]
            best = max(best, float(np.max(np.abs((f1 - f) * (f2 - f)))))
        assert best / B ** 2 == pytest.approx(frac, rel=0.03), (off, best / B ** 2)


def test_node_rule_panels(oracle_mod, workloads):
    """l = 0 islands of equal widths split the outer range once (2 x n/2 outer nodes);
    l = +-1 islands are one panel (n outer nodes); every node lies inside the
    three supports."""
    wl = workloads.config_small(gl_order=8)
    pb = oracle_mod.Problem(wl, gl_order=8)
    W = pb.R[0] * 1.01
    for n in range(5):
        for n1, n2, n3 in pb.islands(n):
            nodes = pb.island_nodes(n, n1, n2, n3)
            assert len(nodes) == 64
            d = (pb.nu[n1] - pb.nu[n]) + (pb.nu[n2] - pb.nu[n3])
            u, v = nodes[:, 0], nodes[:, 1]
            assert np.all(np.abs(u) < W / 2) and np.all(np.abs(v) < W / 2)
            assert np.all(np.abs(u + v + d) < W / 2 * (1 + 1e-12))
