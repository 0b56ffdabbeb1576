"""Seeded synthetic link/WDM descriptions (SI units), shared by the CUDA path's
tests/bench and by the oracle.

This module only describes inputs: fibre parameters as printed in the paper's
tables, channel grids, launch powers and modulation-format *names*.  It holds
none of the method's arithmetic (no unit conversion to beta2/beta3, no ISRS
profile, no format moments): each side of a parity test derives those itself.

Workloads:
  * ``config_small``  5 ch x 64 GBd, 1 x 80 km SSMF, 64x64 Gauss-Legendre
  * ``config_cl``     120 ch x 64 GBd C+L (9 THz), 10 x 80 km SSMF, 2 dBm/ch,
                      formats drawn from a splitmix64 stream, 32x32 GL
  * ``table1``        101 ch x 10 GBd at 10.1 GHz, N x 100 km (Table I, Sec. III-A)
  * ``table2``        101 ch x 100 GBd at 101 GHz, 1 x 100 km (Table II, App. C)
  * ``random_link``   seeded heterogeneous links for the batched path
  * ``surrogate_link`` seeded 120-channel C+L links with identical spans, the
                      training and held-out sets of the MLP surrogate
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

C_M_PER_S = 299792458.0

FORMATS = ("QPSK", "16QAM", "64QAM", "GAUSS")

# Fibre types.  SSMF as quoted for the C+L workloads; PSCF for mixed links.
SSMF = dict(alpha_db_km=0.2, D_ps_nm_km=17.0, S_ps_nm2_km=0.067, lambda_ref_m=1550e-9,
            gamma_per_w_km=1.3, cr_per_w_km_thz=0.028)
PSCF = dict(alpha_db_km=0.16, D_ps_nm_km=21.0, S_ps_nm2_km=0.067, lambda_ref_m=1550e-9,
            gamma_per_w_km=0.8, cr_per_w_km_thz=0.028)


class SplitMix64:
    """splitmix64 counter-based generator (Steele, Lea, Flood 2014)."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.next_u64() % (hi - lo + 1)

    def normal(self) -> float:
        """Standard normal by Box-Muller."""
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def dbm_to_w(p_dbm: float) -> float:
    return 1e-3 * 10.0 ** (p_dbm / 10.0)


@dataclass
class Span:
    alpha_db_km: float
    D_ps_nm_km: float
    S_ps_nm2_km: float
    lambda_ref_m: float
    gamma_per_w_km: float
    cr_per_w_km_thz: float
    length_m: float


@dataclass
class Workload:
    name: str
    spans: List[Span]
    centre_hz: List[float]
    symbol_rate_baud: List[float]
    launch_power_w: List[float]
    formats: List[str]
    rolloff: float
    gl_order: int
    dz_km: float = 1.0
    notes: dict = field(default_factory=dict)

    @property
    def n_ch(self) -> int:
        return len(self.centre_hz)


def _spans(fibre: dict, length_km: float, n: int) -> List[Span]:
    return [Span(length_m=length_km * 1e3, **fibre) for _ in range(n)]


def grid(n_ch: int, spacing_hz: float, centre_hz: float) -> List[float]:
    """n_ch channel centres on a uniform grid symmetric about centre_hz."""
    return [centre_hz + (k - 0.5 * (n_ch - 1)) * spacing_hz for k in range(n_ch)]


def config_small(gl_order: int = 64, n_ch: int = 5, p_dbm: float = 0.0,
                 fmt: str = "16QAM", n_spans: int = 1) -> Workload:
    """5 ch x 64 GBd on a 75 GHz grid at 1550 nm, 1 x 80 km SSMF, 0 dBm/ch,
    raised-cosine roll-off 0.01, 16QAM, 64x64 GL per island."""
    centre = C_M_PER_S / 1550e-9
    return Workload(
        name=f"{n_ch}ch x 64GBd @75GHz, {n_spans}x80km SSMF, {p_dbm:g} dBm/ch, {fmt}, {gl_order}x{gl_order} GL",
        spans=_spans(SSMF, 80.0, n_spans),
        centre_hz=grid(n_ch, 75e9, centre),
        symbol_rate_baud=[64e9] * n_ch,
        launch_power_w=[dbm_to_w(p_dbm)] * n_ch,
        formats=[fmt] * n_ch,
        rolloff=0.01,
        gl_order=gl_order,
    )


def config_cl(gl_order: int = 32, p_dbm: float = 2.0, seed: int = 0, n_spans: int = 10,
              n_ch: int = 120) -> Workload:
    """120 ch x 64 GBd on a 75 GHz grid spanning 9 THz between 1530 and 1605 nm,
    10 x 80 km SSMF, 2 dBm/ch, formats drawn per channel from a splitmix64 stream."""
    f_hi = C_M_PER_S / 1530e-9
    f_lo = C_M_PER_S / 1605e-9
    centre = 0.5 * (f_hi + f_lo)
    rng = SplitMix64(seed)
    fmts = [FORMATS[rng.next_u64() % 4] for _ in range(n_ch)]
    return Workload(
        name=f"{n_ch}ch x 64GBd C+L @75GHz, {n_spans}x80km SSMF, {p_dbm:g} dBm/ch, {gl_order}x{gl_order} GL",
        spans=_spans(SSMF, 80.0, n_spans),
        centre_hz=grid(n_ch, 75e9, centre),
        symbol_rate_baud=[64e9] * n_ch,
        launch_power_w=[dbm_to_w(p_dbm)] * n_ch,
        formats=fmts,
        rolloff=0.01,
        gl_order=gl_order,
        notes={"seed": seed},
    )


def table1(n_spans: int = 1, cr: float = 0.28, fmt: str = "QPSK", gl_order: int = 16,
           n_ch: int = 101, dz_km: float = 1.0) -> Workload:
    """Table I (Sec. III-A): 101 ch x 10 GBd at 10.1 GHz, N x 100 km, alpha 0.2,
    D 17, S 0, gamma 1.2, total launch power 19 dBm, Cr 0.28 or 1.12."""
    fibre = dict(alpha_db_km=0.2, D_ps_nm_km=17.0, S_ps_nm2_km=0.0, lambda_ref_m=1550e-9,
                 gamma_per_w_km=1.2, cr_per_w_km_thz=cr)
    centre = C_M_PER_S / 1550e-9
    p_ch = dbm_to_w(19.0) / n_ch
    return Workload(
        name=f"Table I: {n_ch}ch x 10GBd @10.1GHz, {n_spans}x100km, Cr={cr}, {fmt}",
        spans=_spans(fibre, 100.0, n_spans),
        centre_hz=grid(n_ch, 10.1e9, centre),
        symbol_rate_baud=[10e9] * n_ch,
        launch_power_w=[p_ch] * n_ch,
        formats=[fmt] * n_ch,
        rolloff=0.01,
        gl_order=gl_order,
        dz_km=dz_km,
    )


def table2(fmt: str = "QPSK", gl_order: int = 16, dz_km: float = 1.0) -> Workload:
    """Table II (App. C): 101 ch x 100 GBd at 101 GHz, 1 x 100 km, alpha 0.2, D 17,
    S 0.067, gamma 1.2, total launch power 25 dBm, Cr 0.028."""
    fibre = dict(alpha_db_km=0.2, D_ps_nm_km=17.0, S_ps_nm2_km=0.067, lambda_ref_m=1550e-9,
                 gamma_per_w_km=1.2, cr_per_w_km_thz=0.028)
    n_ch = 101
    centre = C_M_PER_S / 1550e-9
    p_ch = dbm_to_w(25.0) / n_ch
    return Workload(
        name="Table II: 101ch x 100GBd @101GHz, 1x100km, Cr=0.028",
        spans=_spans(fibre, 100.0, 1),
        centre_hz=grid(n_ch, 101e9, centre),
        symbol_rate_baud=[100e9] * n_ch,
        launch_power_w=[p_ch] * n_ch,
        formats=[fmt] * n_ch,
        rolloff=0.01,
        gl_order=gl_order,
        dz_km=dz_km,
    )


def random_link(seed: int, gl_order: int = 16) -> Workload:
    """Seeded heterogeneous link: n_ch in 20..200, one symbol rate per link in
    32..96 GBd, spacing in [max(50, ceil(1.01 R)), 150] GHz with n_ch * spacing
    capped at 12 THz, 1..30 spans of 50..120 km each SSMF or PSCF, mean power
    U[-2, 4] dBm with a +-3 dB linear tilt and N(0, 0.5 dB) ripple, formats drawn
    per channel."""
    rng = SplitMix64(0xE6A0000 + seed)
    n_ch = rng.randint(20, 200)
    R_gbd = rng.randint(32, 96)
    sp_lo = max(50, int(math.ceil(1.01 * R_gbd)))
    spacing = rng.randint(sp_lo, 150)
    n_ch = min(n_ch, int(12000 // spacing))
    n_spans = rng.randint(1, 30)
    spans = []
    for _ in range(n_spans):
        fibre = SSMF if rng.next_u64() % 2 == 0 else PSCF
        spans.append(Span(length_m=rng.randint(50, 120) * 1e3, **fibre))
    p0 = -2.0 + 6.0 * rng.uniform()
    tilt = -3.0 + 6.0 * rng.uniform()
    centre = C_M_PER_S / 1567.5e-9
    cen = grid(n_ch, spacing * 1e9, centre)
    f_min, f_max = cen[0], cen[-1]
    powers = []
    for f in cen:
        rel = (f - 0.5 * (f_min + f_max)) / max(f_max - f_min, 1.0)
        powers.append(dbm_to_w(p0 + tilt * rel + 0.5 * rng.normal()))
    fmts = [FORMATS[rng.next_u64() % 4] for _ in range(n_ch)]
    return Workload(
        name=f"random link {seed}: {n_ch}ch x {R_gbd}GBd @{spacing}GHz, {n_spans} spans",
        spans=spans,
        centre_hz=cen,
        symbol_rate_baud=[R_gbd * 1e9] * n_ch,
        launch_power_w=powers,
        formats=fmts,
        rolloff=0.01,
        gl_order=gl_order,
        notes={"seed": seed},
    )


def surrogate_link(seed: int, gl_order: int = 32, n_ch: int = 120) -> Workload:
    """Seeded C+L link for the surrogate: the 120-channel, 64 GBd, 75 GHz grid of
    config_cl (or its n_ch central channels' grid of the same spacing, centred at
    the same frequency); N_s ~ U{1..30} identical SSMF spans of L ~ U[50, 120] km with
    Cr ~ U[0.014, 0.042] 1/(W km THz); mean launch power U[-2, 4] dBm with a
    linear tilt U[-3, 3] dB across the band and N(0, 0.5 dB) ripple per
    channel; formats drawn per channel.  Training seeds 1, 2, ...; held-out
    seeds from 1,000,001."""
    rng = SplitMix64(0x5A770000 + seed)
    n_spans = rng.randint(1, 30)
    length_km = 50.0 + 70.0 * rng.uniform()
    cr = 0.014 + 0.028 * rng.uniform()
    p0 = -2.0 + 6.0 * rng.uniform()
    tilt = -3.0 + 6.0 * rng.uniform()
    base = config_cl(gl_order=gl_order, n_spans=1, n_ch=n_ch)
    cen = base.centre_hz
    f_min, f_max = cen[0], cen[-1]
    powers = []
    for f in cen:
        rel = (f - 0.5 * (f_min + f_max)) / (f_max - f_min)
        powers.append(dbm_to_w(p0 + tilt * rel + 0.5 * rng.normal()))
    fmts = [FORMATS[rng.next_u64() % 4] for _ in cen]
    fibre = dict(SSMF)
    fibre["cr_per_w_km_thz"] = cr
    return Workload(
        name=f"surrogate link {seed}: {n_ch}ch C+L, {n_spans}x{length_km:.1f}km, Cr {cr:.4f}, {p0:.2f} dBm, tilt {tilt:.2f} dB",
        spans=_spans(fibre, length_km, n_spans),
        centre_hz=list(cen),
        symbol_rate_baud=[64e9] * len(cen),
        launch_power_w=powers,
        formats=fmts,
        rolloff=0.01,
        gl_order=gl_order,
        notes={"seed": seed, "n_spans": n_spans, "length_km": length_km, "cr": cr, "p0_dbm": p0, "tilt_db": tilt},
    )
