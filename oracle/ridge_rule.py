"""A node rule for the island integrals (Eq. 17-21) that resolves the ridges of |mu|^2.

TEST INFRASTRUCTURE, like the rest of oracle/: only tests/ may import it.  It
shares no code with the CUDA path and is not a parity target of it; it estimates
the converged value of Eq. 15 on links where doubling the Gauss-Legendre order of
the configured node rule (Problem.eta_converged) is out of reach.

Why a different rule.  With chi = 4 pi^2 (f1 - f)(f2 - f)[beta2 + pi beta3 (f1 + f2)]
(Eq. 5, 24), |mu|^2 of Eq. 8-10 is about 1/(alpha^2 + chi^2), so along f1 at fixed
f2 it is a Lorentzian centred on f1 = f of half-width alpha / (4 pi^2 |beta2| |f2 - f|),
and likewise along f2.  For an interferer 1 THz from the COI that is about 54 MHz,
against node gaps of gigahertz in a Gauss-Legendre rule over a 64 GHz channel.
The spectral shapes add kinks: the raised cosine h(x) is smooth inside
|x| < (1 - beta) R / 2 and on the roll-off, but not across the knee between them.

The rule.  In each evaluation order, e.g. (outer w, inner u) with w = u + v + d:
  * the outer range is cut at the knees of the outer shape and wherever two inner
    break points cross (which includes the island's own kinks, where the active
    inner limit switches, and the point where both ridges meet, f1 = f2 = f), and
    at a ridge of the outer variable;
  * each inner interval is cut at the knees of the other two shapes and at the
    ridge points f1 = f and f2 = f that fall inside it;
  * a piece that does not end on a ridge gets ceil(n * length / total) nodes, at
    least n_min, placed by Gauss-Legendre;
  * a piece that ends on a ridge gets n nodes, placed by the sinh transformation
    x = x_r + h sinh(tau) with tau uniform-Gauss-Legendre on [0, asinh(L / h)]
    (Johnston and Elliott's transformation for nearly singular integrands), h the
    ridge half-width; a piece with a ridge at both ends is halved first.
The integrand is the oracle's own Upsilon (Eq. 22) and raised-cosine shapes."""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O


def _gl(n, cache={}):
    if n not in cache:
        cache[n] = O.gauss_legendre(n)
    return cache[n]


def _piece(a, b, n, ha, hb):
    """Nodes and weights on [a, b]; ha / hb the ridge half-width at a / b (None: no ridge)."""
    if ha is not None and hb is not None:
        m = 0.5 * (a + b)
        x1, w1 = _piece(a, m, n, ha, None)
        x2, w2 = _piece(m, b, n, None, hb)
        return np.concatenate([x1, x2]), np.concatenate([w1, w2])
    x, w = _gl(n)
    if ha is None and hb is None:
        return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w
    h = ha if ha is not None else hb
    T = math.asinh((b - a) / h)
    tau = 0.5 * T * (x + 1.0)
    off, jac = h * np.sinh(tau), 0.5 * T * w * h * np.cosh(tau)
    return (a + off, jac) if ha is not None else (b - off, jac)


def _interval(lo, hi, points, n, n_min):
    """Nodes on [lo, hi] cut at the break points (x, h) inside it; h is a ridge
    half-width or None for a plain cut (a knee or a kink)."""
    eps = 1e-12
    cand = sorted([(p, h) for p, h in points if lo + eps < p < hi - eps], key=lambda t: t[0])
    cuts = []
    for p, h in cand:
        if cuts and p - cuts[-1][0] < eps:
            if h is not None:
                cuts[-1] = (cuts[-1][0], h)
            continue
        cuts.append((p, h))
    ends = [(lo, None)] + cuts + [(hi, None)]
    for p, h in points:  # a ridge exactly on an end of the interval
        if h is not None and abs(p - lo) <= eps:
            ends[0] = (lo, h)
        if h is not None and abs(p - hi) <= eps:
            ends[-1] = (hi, h)
    X, W = [], []
    for (a, ha), (b, hb) in zip(ends[:-1], ends[1:]):
        if not b > a:
            continue
        m = n if (ha is not None or hb is not None) else max(n_min, math.ceil(n * (b - a) / (hi - lo)))
        x, w = _piece(a, b, m, ha, hb)
        X.append(x)
        W.append(w)
    return np.concatenate(X), np.concatenate(W)


def raised_cosine(x, R, beta):
    """h(x): 1 for |x| <= (1 - beta) R/2, a half cosine down to 0 at (1 + beta) R/2."""
    ax = np.abs(x)
    k = (1 - beta) * R / 2
    if beta == 0.0:
        return np.where(ax <= k, 1.0, 0.0)
    taper = 0.5 * (1 + np.cos(math.pi / (beta * R) * np.clip(ax - k, 0.0, beta * R)))
    return np.where(ax <= k, 1.0, np.where(ax <= (1 + beta) * R / 2, taper, 0.0))


class RidgeRule:
    """The rule above for the islands of an oracle Problem (identical spans: the
    ridge half-widths take the first span's alpha, beta2 and beta3).

    The three evaluation orders of Eq. 17-21 are those of the configured rule:
    order 0 (outer w, inner u; D, G, H), order 1 (outer v, inner u; E) and
    order 2 (outer u, inner v; F).  In each, the outer variable o and the inner t
    are coupled by |y| <= C with y = +-(t - (s o + c)) the third variable; every
    break point of the inner interval is a line t = a o + b (a = 0 or s), and the
    outer range is cut wherever two such lines of different slope cross, at the
    knees of the outer shape, and at a ridge of the outer variable."""

    def __init__(self, pb: O.Problem, n_min: int = 4, knees: bool = True):
        """knees=False leaves out the cuts at the raised-cosine knees (the ridge and
        kink cuts stay), the simpler form a GPU planner would start from."""
        self.pb = pb
        sp = pb.spans[0]
        self.alpha, self.beta2, self.beta3 = sp.alpha, sp.beta2, sp.beta3
        self.rolloff = pb.c.rolloff
        self.n_min = n_min
        self.knees = knees

    def fcoi(self, n):
        """The frequency at which COI n is evaluated: its centre plus the problem's
        COI offset (Problem.set_coi_offsets), if any."""
        off = getattr(self.pb, "_f_off", None)
        return self.pb.nu[n] + (off[n] if off is not None else 0.0)

    def rows(self, n, n1, n2, n3, ordering, order):
        """The rule's rows for one evaluation order: a list of (o, wo, t, wt) with the
        outer node and weight and the inner nodes and weights, and a function
        mapping (o, t) to (u, v, w); None if the island has zero area."""
        pb, be = self.pb, self.rolloff
        nu, R = pb.nu, pb.R
        W = R * (1 + be)
        f = self.fcoi(n)
        d = (nu[n1] - f) + (nu[n2] - nu[n3])
        k = [(1 - be) * R[m] / 2 for m in (n1, n2, n3)]   # knees of h1, h2, h3
        half = [0.5 * W[m] for m in (n1, n2, n3)]
        cc = 4 * math.pi ** 2 * abs(self.beta2 + 2 * math.pi * self.beta3 * f)
        us, vs = f - nu[n1], f - nu[n2]                    # ridges u = us (f1 = f), v = vs (f2 = f)
        if ordering == 0:   # o = w, t = u, v = (o - d) - t
            A, B, s, c, C = half[2], half[0], 1.0, -d, half[1]
            ko, kt, ky = k[2], k[0], k[1]
            uvw = lambda o, t: (t, (s * o + c) - t, o)
        elif ordering == 1:  # o = v, t = u, w = t + o + d
            A, B, s, c, C = half[1], half[0], -1.0, -d, half[2]
            ko, kt, ky = k[1], k[0], k[2]
            uvw = lambda o, t: (t, o, t - (s * o + c))
        else:                # o = u, t = v, w = t + o + d
            A, B, s, c, C = half[0], half[1], -1.0, -d, half[2]
            ko, kt, ky = k[0], k[1], k[2]
            uvw = lambda o, t: (o, t, t - (s * o + c))
        p_, q_ = s * (-(B + C) - c), s * ((B + C) - c)
        lo, hi = max(-A, min(p_, q_)), min(A, max(p_, q_))
        if not hi > lo:
            return None
        ridges = cc > 0  # no dispersion: chi = 0 everywhere, no ridges
        hmax = self.alpha / (cc * max(half[0], half[1])) if ridges else None
        # inner break lines t = a o + b: limits, knees, ridges
        flat = [-B, B] + ([-kt, kt] if self.knees else [])
        slant = [c - C, c + C] + ([c - ky, c + ky] if self.knees else [])
        ridge_flat = ridge_slant = None
        if ridges:
            if ordering == 0:
                ridge_flat, ridge_slant = us, c - vs      # u = us; v = vs
            elif ordering == 1:
                ridge_flat = us
            else:
                ridge_flat = vs
        outer = [(-ko, None), (ko, None)] if self.knees else []
        for b0 in flat + ([ridge_flat] if ridge_flat is not None else []):
            for b1 in slant + ([ridge_slant] if ridge_slant is not None else []):
                both = (b0 == ridge_flat and ridge_flat is not None and b1 == ridge_slant
                        and ridge_slant is not None)
                outer.append(((b0 - b1) / s, hmax if both else None))
        if ridges and ordering == 1:
            outer.append((vs, hmax))
        if ridges and ordering == 2:
            outer.append((us, hmax))
        xo, wo = _interval(lo, hi, outer, order, self.n_min)
        out = []
        for o, ww in zip(xo, wo):
            m = s * o + c
            tlo, thi = max(-B, m - C), min(B, m + C)
            if not thi > tlo:
                continue
            pts = [(-kt, None), (kt, None), (m - ky, None), (m + ky, None)] if self.knees else []
            if ridges:
                if ordering == 0:
                    x2 = nu[n2] + (m - us) - f            # f2 - f on the ridge f1 = f
                    if x2 != 0:
                        pts.append((us, self.alpha / (cc * abs(x2))))
                    tr = m - vs                           # ridge f2 = f
                    x1 = nu[n1] + tr - f
                    if x1 != 0:
                        pts.append((tr, self.alpha / (cc * abs(x1))))
                elif ordering == 1:
                    x2 = nu[n2] + o - f
                    if x2 != 0:
                        pts.append((us, self.alpha / (cc * abs(x2))))
                else:
                    x1 = nu[n1] + o - f
                    if x1 != 0:
                        pts.append((vs, self.alpha / (cc * abs(x1))))
            t, wt = _interval(tlo, thi, pts, order, self.n_min)
            out.append((o, ww, t, wt))
        return out, uvw

    def _eval(self, n, n1, n2, n3, ordering, order):
        r = self.rows(n, n1, n2, n3, ordering, order)
        if r is None or not r[0]:
            return None
        rows, uvw = r
        pb, R, nu, be = self.pb, self.pb.R, self.pb.nu, self.rolloff
        o = np.concatenate([np.full(len(t), oo) for oo, _, t, _ in rows])
        t = np.concatenate([t for _, _, t, _ in rows])
        wi = np.concatenate([wt for _, _, _, wt in rows])
        wo = np.array([ww for _, ww, _, _ in rows])
        starts = np.cumsum([0] + [len(tt) for _, _, tt, _ in rows])[:-1]
        u, v, w = uvw(o, t)
        Y = pb.upsilon_many(nu[n1] + u, nu[n2] + v, self.fcoi(n))
        h = (raised_cosine(u, R[n1], be), raised_cosine(v, R[n2], be), raised_cosine(w, R[n3], be))
        return o, wo, wi, starts, Y, h

    def terms(self, n, n1, n2, n3, order, which="DEFGH"):
        """(D, E, F, G, H) of Eq. 17-21 for island (n1, n2, n3) of COI n with the
        coefficients of the configured rule; terms not in `which` are 0."""
        Rn, R = self.pb.R[n], self.pb.R
        out = np.zeros(5)
        if any(x in which for x in "DGH"):
            e = self._eval(n, n1, n2, n3, 0, order)
            if e is not None:
                o, wo, wi, st, Y, (h1, h2, h3) = e
                wrow = np.repeat(wo, np.diff(np.append(st, len(wi))))
                out[0] = 16 / 27 * Rn / (R[n1] * R[n2] * R[n3]) * np.sum(wrow * wi * h1 * h2 * h3 * np.abs(Y) ** 2)
                inner = np.add.reduceat(wi * np.sqrt(h1 * h2) * Y, st)
                out[3] = 16 / 81 / Rn ** 3 * np.sum(wo * raised_cosine(o[st], R[n3], self.rolloff) * np.abs(inner) ** 2)
                out[4] = 16 / 81 / Rn ** 4 * abs(np.sum(wrow * wi * np.sqrt(h1 * h2 * h3) * Y)) ** 2
        for idx, ordering, coef, key in ((1, 1, 16 / 27, "E"), (2, 2, 32 / 81, "F")):
            if key not in which:
                continue
            e = self._eval(n, n1, n2, n3, ordering, order)
            if e is None:
                continue
            o, wo, wi, st, Y, (h1, h2, h3) = e
            a, ho = (np.sqrt(h1 * h3), h2) if ordering == 1 else (np.sqrt(h2 * h3), h1)
            inner = np.add.reduceat(wi * a * Y, st)
            out[idx] = coef / Rn ** 3 * np.sum(wo * ho[st] * np.abs(inner) ** 2)
        return out

    def d_term(self, n, n1, n2, n3, order):
        """D of Eq. 17 (with the coefficient of the configured rule) and the node count."""
        r = self.rows(n, n1, n2, n3, 0, order)
        if r is None:
            return 0.0, 0
        return float(self.terms(n, n1, n2, n3, order, "D")[0]), sum(len(t) for _, _, t, _ in r[0])

    def pnli(self, n, order, egn=True):
        """Eq. 15 for COI n: the sum over its islands of P1 P2 P3 (D + the EGN
        corrections selected by the Kronecker deltas, if egn)."""
        pb = self.pb
        P, phi, psi = pb.P, pb.phi, pb.psi
        s = 0.0
        for a, b, c in pb.islands(n):
            a, b, c = int(a), int(b), int(c)
            which = "D"
            if egn:
                which += ("E" if a == c else "") + ("F" if b == c else "") + ("G" if a == b else "") + \
                    ("H" if a == b == c else "")
            t = self.terms(n, a, b, c, order, which)
            v = t[0]
            if egn:
                v += (phi[a] * t[1] if a == c else 0) + (phi[b] * t[2] if b == c else 0) + \
                    (phi[a] * t[3] if a == b else 0) + (psi[a] * t[4] if a == b == c else 0)
            s += P[a] * P[b] * P[c] * v
        return s

    def pnli_3d(self, n, order, n_f, egn=True):
        """Eq. 15 with the integral over f of Eq. 17-21 taken literally (the oracle's
        eta_3d reading): an n_f-point Gauss-Legendre rule over f in
        [f_n - R_n/2, f_n + R_n/2], each node the island sum at that COI frequency."""
        pb = self.pb
        x, w = O.gauss_legendre(int(n_f))
        total = 0.0
        try:
            for xj, wj in zip(x, w):
                off = np.zeros(pb.n_ch)
                off[n] = 0.5 * xj * pb.R[n]
                pb.set_coi_offsets(off)
                total += 0.5 * wj * self.pnli(n, order, egn)
        finally:
            pb.set_coi_offsets(None)
        return total

    def pnli_gn(self, n, order):
        """The GN part of Eq. 15 for COI n: sum over its islands of P1 P2 P3 D."""
        return self.pnli(n, order, egn=False)
