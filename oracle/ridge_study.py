"""Discretisation error of Eq. 15 per COI (its GN part, or with --egn all of it): the configured
Gauss-Legendre rule at several orders against the ridge-resolving rule of
ridge_rule.py at several orders (the oracle only; CPU; minutes per COI of the
120-channel link).

    python oracle/ridge_study.py small 0,1,2,3,4 --plain 32,64,512 --ridge 8,16,32
    python oracle/ridge_study.py cl 0 --plain 16,32,64 --ridge 16,32,64

Prints one line per COI and rule: the sum over islands of P1 P2 P3 D (with
--egn, plus the EGN corrections; with --f3d N, integrated over the COI band by N
nodes) and its ratio in dB to the last ridge-rule order."""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import oracle as O  # noqa: E402
from oracle.ridge_rule import RidgeRule  # noqa: E402
from paper_2412_11614_gb300 import workloads  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=["small", "cl"])
    ap.add_argument("coi", help="comma-separated channel indices")
    ap.add_argument("--plain", default="32,64")
    ap.add_argument("--ridge", default="16,32")
    ap.add_argument("--egn", action="store_true", help="include the EGN corrections (E, F, G, H)")
    ap.add_argument("--no-knees", action="store_true", help="ridge rule without the cuts at the spectral knees")
    ap.add_argument("--f3d", type=int, default=0,
                    help="integrate over the COI band with this many Gauss-Legendre nodes (0: white NLI)")
    a = ap.parse_args(argv)
    wl = workloads.config_small() if a.workload == "small" else workloads.config_cl()
    plain = [int(x) for x in a.plain.split(",") if x]
    ridge = [int(x) for x in a.ridge.split(",") if x]
    for n in (int(x) for x in a.coi.split(",")):
        res = []
        terms = 1 if a.egn else 0
        pb = O.Problem(wl, gl_order=8, terms=terms)
        rule = RidgeRule(pb, knees=not a.no_knees)
        n_isl = len(pb.islands(n))
        for q in ridge:
            t0 = time.time()
            v = rule.pnli_3d(n, q, a.f3d, egn=a.egn) if a.f3d else rule.pnli(n, q, egn=a.egn)
            res.append((f"ridge {q}", v, time.time() - t0))
        for q in plain:
            t0 = time.time()
            pq = O.Problem(wl, gl_order=q, terms=terms)
            s = pq.eta_3d(a.f3d, coi=[n])[1][0] if a.f3d else pq.island_contribs(n)[1].sum()
            res.append((f"plain {q}x{q}", s, time.time() - t0))
        ref = res[len(ridge) - 1][1] if ridge else res[-1][1]
        for name, s, t in res:
            print(f"COI {n} ({n_isl} islands) {name:>14}: {s:.6e} W  {10 * math.log10(s / ref):+8.4f} dB  {t:6.1f} s",
                  flush=True)


if __name__ == "__main__":
    main()
