"""A node rule for the D integral (Eq. 17) that resolves the ridges of |mu|^2.

TEST INFRASTRUCTURE, like the rest of oracle/: only tests/ may import it.  It
shares no code with the CUDA path and is not a parity target of it; it estimates
the converged value of Eq. 17 on links where doubling the Gauss-Legendre order of
the configured node rule (Problem.eta_converged) is out of reach.

Why a different rule.  With chi = 4 pi^2 (f1 - f)(f2 - f)[beta2 + pi beta3 (f1 + f2)]
(Eq. 5, 24), |mu|^2 of Eq. 8-10 is about 1/(alpha^2 + chi^2), so along f1 at fixed
f2 it is a Lorentzian centred on f1 = f of half-width alpha / (4 pi^2 |beta2| |f2 - f|),
and likewise along f2.  For an interferer 1 THz from the COI that is about 54 MHz,
against node gaps of gigahertz in a Gauss-Legendre rule over a 64 GHz channel.
The spectral shapes add kinks: the raised cosine h(x) is smooth inside
|x| < (1 - beta) R / 2 and on the roll-off, but not across the knee between them.

The rule.  In the (outer w, inner u) order of the island (w = u + v + d):
  * the outer range is cut at the island's own kinks (where the active inner limit
    switches), at the knees of h3, where two inner break points cross, and at the
    point where both ridges meet (f1 = f2 = f);
  * each inner interval is cut at the knees of h1 and h2 and at the ridge points
    f1 = f and f2 = f;
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
    ridge half-widths take the first span's alpha, beta2 and beta3)."""

    def __init__(self, pb: O.Problem, n_min: int = 4):
        self.pb = pb
        sp = pb.spans[0]
        self.alpha, self.beta2, self.beta3 = sp.alpha, sp.beta2, sp.beta3
        self.rolloff = pb.c.rolloff
        self.n_min = n_min

    def nodes(self, n, n1, n2, n3, order):
        """(u, v, w, weight) of every node of island (n1, n2, n3) of COI n, or None
        if the island has zero area."""
        pb, be = self.pb, self.rolloff
        nu, R = pb.nu, pb.R
        W = R * (1 + be)
        f = nu[n]
        d = (nu[n1] - f) + (nu[n2] - nu[n3])
        A, B, C = 0.5 * W[n3], 0.5 * W[n1], 0.5 * W[n2]
        lo, hi = max(-A, d - (B + C)), min(A, d + (B + C))
        if not hi > lo:
            return None
        c = 4 * math.pi ** 2 * abs(self.beta2 + 2 * math.pi * self.beta3 * f)
        k1, k2, k3 = (1 - be) * R[n1] / 2, (1 - be) * R[n2] / 2, (1 - be) * R[n3] / 2
        outer = [(d + C - B, None), (d + B - C, None), (-k3, None), (k3, None)]
        for ku in (k1, B):
            for kv in (k2, C):
                for su in (-1, 1):
                    for sv in (-1, 1):
                        outer.append((su * ku + sv * kv + d, None))
        ridges = c > 0  # no dispersion: chi = 0 everywhere, no ridges
        if ridges:
            outer.append(((f - nu[n1]) + (f - nu[n2]) + d, self.alpha / (c * max(B, C))))
        xo, wo = _interval(lo, hi, outer, order, self.n_min)
        U, V, Wt, WW = [], [], [], []
        for w, ww in zip(xo, wo):
            ilo, ihi = max(-B, w - d - C), min(B, w - d + C)
            if not ihi > ilo:
                continue
            pts = [(-k1, None), (k1, None), (w - d - k2, None), (w - d + k2, None)]
            if ridges:
                u1 = f - nu[n1]                   # ridge f1 = f
                x2 = nu[n2] + (w - u1 - d) - f
                if x2 != 0:
                    pts.append((u1, self.alpha / (c * abs(x2))))
                u2 = w - d - (f - nu[n2])         # ridge f2 = f
                x1 = nu[n1] + u2 - f
                if x1 != 0:
                    pts.append((u2, self.alpha / (c * abs(x1))))
            x, wi = _interval(ilo, ihi, pts, order, self.n_min)
            U.append(x)
            V.append(w - x - d)
            Wt.append(np.full_like(x, w))
            WW.append(ww * wi)
        return tuple(map(np.concatenate, (U, V, Wt, WW)))

    def d_term(self, n, n1, n2, n3, order):
        """D of Eq. 17 (with the coefficient of the configured rule) and the node count."""
        nd = self.nodes(n, n1, n2, n3, order)
        if nd is None:
            return 0.0, 0
        u, v, w, wt = nd
        pb, R, nu, be = self.pb, self.pb.R, self.pb.nu, self.rolloff
        Y = pb.upsilon_many(nu[n1] + u, nu[n2] + v, nu[n])
        h = raised_cosine(u, R[n1], be) * raised_cosine(v, R[n2], be) * raised_cosine(w, R[n3], be)
        cf = 16.0 / 27.0 * R[n] / (R[n1] * R[n2] * R[n3])
        return cf * float(np.sum(wt * h * np.abs(Y) ** 2)), len(u)

    def pnli_gn(self, n, order):
        """The GN part of Eq. 15 for COI n: sum over its islands of P1 P2 P3 D."""
        P = self.pb.P
        s = 0.0
        for a, b, c in self.pb.islands(n):
            a, b, c = int(a), int(b), int(c)
            s += P[a] * P[b] * P[c] * self.d_term(n, a, b, c, order)[0]
        return s
