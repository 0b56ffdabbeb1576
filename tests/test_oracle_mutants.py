"""Mutation check of the oracle's pins: each plausible mistake (a dropped term, a
wrong sign, index or coefficient) is planted in a copy of the oracle's C source on
the CPU, built into a temporary library, and the pin suite must fail on it.

Opt-in (several minutes): EGN_RUN_MUTANTS=1 python -m pytest tests/test_oracle_mutants.py
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "egn_oracle.c")

MUTANTS = {
    "leff_sign": ("return -expm1(-alpha * z) / alpha;", "return expm1(-alpha * z) / alpha;"),
    "srs_half": ("return x * exp(-zeta * f) / (2.0 * sinh(x / 2.0));", "return x * exp(-zeta * f) / (2.0 * sinh(x));"),
    "srs_sign": ("return x * exp(-zeta * f) / (2.0 * sinh(x / 2.0));", "return x * exp(zeta * f) / (2.0 * sinh(x / 2.0));"),
    "chi_beta3": ("(beta2 + OR_PI * beta3 * (f1 + f2))", "(beta2 + OR_PI * beta3 * (f1 - f2))"),
    "chi_factor": ("return 4.0 * OR_PI * OR_PI * (f1 - f)", "return 2.0 * OR_PI * OR_PI * (f1 - f)"),
    "segment_mid": ("double zk = (k + 0.5) / K * s->L;", "double zk = (k + 0.0) / K * s->L;"),
    "segment_edge": ("double za = (double)(k + 1) / K * s->L;", "double za = (double)(k + 2) / K * s->L;"),
    "maclaurin_2a": ("cplx g2 = I * chi - 2.0 * s->alpha;", "cplx g2 = I * chi - s->alpha;"),
    "upsilon_phase": ("Y += sp->gamma * mu * cexp(I * acc);", "Y += sp->gamma * mu * cexp(-I * acc);"),
    "upsilon_beta3": ("(sp->beta2 * sp->L + OR_PI * (f1 + f2) * sp->beta3 * sp->L)", "(sp->beta2 * sp->L)"),
    "rc_knee": ("return 0.5 * (1.0 + cos(OR_PI / (beta * R) * (ax - a)));", "return 0.5 * (1.0 + cos(OR_PI / (beta * R) * (ax + a)));"),
    "offset_sign": ("return (pb->nu[n1] - or_fcoi(pb, n)) + (pb->nu[n2] - pb->nu[n3]);", "return (pb->nu[n1] - or_fcoi(pb, n)) - (pb->nu[n2] - pb->nu[n3]);"),
    "coi_offset_sign": ("return pb->nu[n] + (pb->f_off ? pb->f_off[n] : 0.0);", "return pb->nu[n] - (pb->f_off ? pb->f_off[n] : 0.0);"),
    "coi_offset_not_in_upsilon": ("    double f = or_fcoi(pb, n);\n    for (int p = 0; p < np; ++p) {", "    double f = pb->nu[n];\n    for (int p = 0; p < np; ++p) {"),
    "coef_D": ("cf[OR_T_D] = (16.0 / 27.0) * R / (pb->R[n1] * pb->R[n2] * pb->R[n3]);", "cf[OR_T_D] = (16.0 / 27.0) / (pb->R[n1] * pb->R[n2]);"),
    "coef_F": ("cf[OR_T_F] = (32.0 / 81.0) / (R * R * R);", "cf[OR_T_F] = (16.0 / 27.0) / (R * R * R);"),
    "coef_H": ("cf[OR_T_H] = (16.0 / 81.0) / (R * R * R * R);", "cf[OR_T_H] = (16.0 / 81.0) / (R * R * R);"),
    "g_inner": ("inner += wi * sqrt(h1 * h2) * Y;          /* G inner", "inner += wi * sqrt(h1 * h3) * Y;          /* G inner"),
    "e_inner": ("inner += wi * sqrt(h1 * h3) * Y;          /* E inner", "inner += wi * sqrt(h2 * h3) * Y;          /* E inner"),
    "pnli_F_phi": ("if (n2 == n3) s += pb->phi[n2] * t[OR_T_F];", "if (n2 == n3) s += pb->phi[n1] * t[OR_T_F];"),
    "pnli_G_flag": ("if (n1 == n2) s += pb->phi[n1] * t[OR_T_G];", "if (n1 == n3) s += pb->phi[n1] * t[OR_T_G];"),
    "psi_moment": ("*psi = mu6 - 9.0 * mu4 + 12.0;", "*psi = mu6 - 6.0 * mu4 + 12.0;"),
    "panel_kink": ("double k1 = s * ((C - B) - c);", "double k1 = s * ((C - B) + c);"),
    "units_beta3": ("double b3_si = a * a * (S_si + 2.0 * D_si / lam);", "double b3_si = a * a * (S_si + D_si / lam);"),
    "units_shift": ("*beta2 = b2 + 2.0 * OR_PI * b3 * (fc_thz - f_ref_thz);", "*beta2 = b2 - 2.0 * OR_PI * b3 * (fc_thz - f_ref_thz);"),
    "gl_weight": ("w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);", "w[n - 1 - i] = 2.0 / ((1.0 + t * t) * dp * dp);"),
}


@pytest.mark.skipif(os.environ.get("EGN_RUN_MUTANTS") != "1", reason="opt-in: EGN_RUN_MUTANTS=1")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/found: {name}"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                        "-o", so, c, "-lm"], check=True)
        env = dict(os.environ, EGN_ORACLE_LIB=so, EGN_RUN_MUTANTS="0")
        # fast pins first; a pin that runs away on a mutant counts as failing (per-test timeout)
        order = ["test_oracle_isrs.py", "test_oracle_mu.py", "test_oracle_quadrature.py", "test_oracle_islands.py",
                 "test_oracle_egn.py", "test_oracle_3d.py"]
        pins = [os.path.join(ROOT, "tests", f) for f in order]
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--timeout", "120"]
                           + pins, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
        assert r.returncode != 0, f"mutant {name} survived the pins"
