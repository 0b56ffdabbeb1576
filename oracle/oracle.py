"""ctypes front end of the FP64 CPU oracle (oracle/egn_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference leg may import this module.  It shares no code with the
CUDA path (paper_2412_11614_gb300/); the only common input is the seeded
workload description of paper_2412_11614_gb300/workloads.py, which carries no
method arithmetic.

Besides the C routines, this file holds the oracle's own reading of the WDM
bookkeeping (all in FP64):
  * spectral centre f_c = (f_max + f_min)/2 of the channel centres, the origin of
    both the ISRS profile (Eq. 25) and of beta2/beta3 (Eq. 24);
  * B_tot = (f_max - f_min) * N/(N - 1) (= N * spacing on a uniform grid, i.e. the
    (2M + 1) R of Appendix B), and B_tot = R for a single channel;
  * P_tot = sum of the launch powers.

Levels: Problem.eta is the node rule at the problem's order (the parity target of
the GPU path); Problem.eta_converged doubles that order until the per-channel
change is below a tolerance (the rule's own discretisation error); mu_form
MU_INTEGRAL replaces the segment form by the adaptive integral of Eq. 23.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import build as _build  # noqa: E402

MU_SEGMENT, MU_MACLAURIN, MU_INTEGRAL = 0, 1, 2
FORMAT_POINTS = {"QPSK": 2, "16QAM": 4, "64QAM": 8, "GAUSS": 0}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class OrSpan(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta2", C.c_double), ("beta3", C.c_double),
                ("gamma", C.c_double), ("cr", C.c_double), ("L", C.c_double)]


class OrProblem(C.Structure):
    _fields_ = [("n_ch", C.c_int), ("nu", _dp), ("R", _dp), ("P", _dp), ("phi", _dp),
                ("psi", _dp), ("rolloff", C.c_double), ("ptot", C.c_double),
                ("btot", C.c_double), ("n_spans", C.c_int), ("spans", C.POINTER(OrSpan)),
                ("gl_order", C.c_int), ("mu_form", C.c_int), ("dz", C.c_double),
                ("int_tol", C.c_double), ("terms", C.c_int), ("f_off", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # EGN_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = os.environ.get("EGN_ORACLE_LIB") or _build.build()
        _lib = C.CDLL(path)
        L = _lib
        L.or_units.argtypes = [C.c_double] * 5 + [_dp] * 3
        L.or_leff.restype = C.c_double
        L.or_leff.argtypes = [C.c_double, C.c_double]
        for fn in ("or_srs_gain", "or_rho"):
            getattr(L, fn).restype = C.c_double
            getattr(L, fn).argtypes = [C.c_double] * 6
        L.or_delta_rho_db.restype = C.c_double
        L.or_delta_rho_db.argtypes = [C.c_double] * 5
        L.or_chi.restype = C.c_double
        L.or_chi.argtypes = [C.c_double] * 5
        L.or_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
        L.or_segments.restype = C.c_int
        L.or_segments.argtypes = [C.c_double, C.c_double]
        L.or_mu_lin_out.argtypes = [C.c_double] * 3 + [_dp]
        L.or_mu_segment_out.argtypes = [C.c_double, C.c_double, C.POINTER(OrSpan), C.c_double,
                                        C.c_double, C.c_int, _dp]
        L.or_mu_maclaurin_out.argtypes = [C.c_double, C.c_double, C.POINTER(OrSpan), C.c_double, _dp]
        L.or_mu_integral_out.argtypes = [C.c_double, C.c_double, C.POINTER(OrSpan), C.c_double,
                                         C.c_double, C.c_double, _dp]
        L.or_upsilon_out.argtypes = [C.POINTER(OrProblem), C.c_double, C.c_double, C.c_double, _dp]
        L.or_upsilon_many.argtypes = [C.POINTER(OrProblem), C.c_long, _dp, _dp, C.c_double, _dp]
        L.or_rc.restype = C.c_double
        L.or_rc.argtypes = [C.c_double] * 3
        L.or_island_exists.restype = C.c_int
        L.or_island_exists.argtypes = [C.POINTER(OrProblem)] + [C.c_int] * 4
        L.or_islands.restype = C.c_long
        L.or_islands.argtypes = [C.POINTER(OrProblem), C.c_int, _ip, C.c_long]
        L.or_island_terms.argtypes = [C.POINTER(OrProblem)] + [C.c_int] * 5 + [_dp]
        L.or_island_terms_midpoint.argtypes = [C.POINTER(OrProblem)] + [C.c_int] * 5 + [_dp]
        L.or_eta.restype = C.c_int
        L.or_eta.argtypes = [C.POINTER(OrProblem), _ip, C.c_int, _dp, _dp]
        L.or_island_contribs.restype = C.c_long
        L.or_island_contribs.argtypes = [C.POINTER(OrProblem), C.c_int, _ip, _dp, C.c_long]
        L.or_island_nodes.restype = C.c_long
        L.or_island_nodes.argtypes = [C.POINTER(OrProblem)] + [C.c_int] * 4 + [_dp, C.c_long]
        L.or_format_moments.restype = C.c_int
        L.or_format_moments.argtypes = [C.c_int, _dp, _dp]
        L.or_num_threads.restype = C.c_int
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


# --------------------------------------------------------------------------- scalars

def units(alpha_db_km, D, S, lambda_ref_m, fc_hz):
    a, b2, b3 = C.c_double(), C.c_double(), C.c_double()
    lib().or_units(alpha_db_km, D, S, lambda_ref_m, fc_hz, C.byref(a), C.byref(b2), C.byref(b3))
    return a.value, b2.value, b3.value


def leff(alpha, z):
    return lib().or_leff(alpha, z)


def srs_gain(z, f, alpha, ptot, cr, btot):
    return lib().or_srs_gain(z, f, alpha, ptot, cr, btot)


def rho(z, f, alpha, ptot, cr, btot):
    return lib().or_rho(z, f, alpha, ptot, cr, btot)


def delta_rho_db(alpha, L, ptot, cr, btot):
    return lib().or_delta_rho_db(alpha, L, ptot, cr, btot)


def chi(f1, f2, f, beta2, beta3):
    return lib().or_chi(f1, f2, f, beta2, beta3)


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, _ptr(x), _ptr(w))
    return x, w


def segments(L, dz):
    return lib().or_segments(L, dz)


def rc(x, R, beta):
    return lib().or_rc(x, R, beta)


def _cx(out):
    return complex(out[0], out[1])


def mu_lin(chi_, alpha, L):
    o = np.zeros(2)
    lib().or_mu_lin_out(chi_, alpha, L, _ptr(o))
    return _cx(o)


def make_span(alpha, beta2, beta3, gamma, cr, L):
    return OrSpan(alpha, beta2, beta3, gamma, cr, L)


def mu_segment(chi_, f3, span: OrSpan, ptot, btot, K):
    o = np.zeros(2)
    lib().or_mu_segment_out(chi_, f3, C.byref(span), ptot, btot, K, _ptr(o))
    return _cx(o)


def mu_maclaurin(chi_, f3, span: OrSpan, ptot):
    o = np.zeros(2)
    lib().or_mu_maclaurin_out(chi_, f3, C.byref(span), ptot, _ptr(o))
    return _cx(o)


def mu_integral(chi_, f3, span: OrSpan, ptot, btot, rel_tol=1e-10):
    o = np.zeros(2)
    lib().or_mu_integral_out(chi_, f3, C.byref(span), ptot, btot, rel_tol, _ptr(o))
    return _cx(o)


def format_moments(name: str):
    phi, psi = C.c_double(), C.c_double()
    rc_ = lib().or_format_moments(FORMAT_POINTS[name], C.byref(phi), C.byref(psi))
    if rc_ != 0:
        raise ValueError(name)
    return phi.value, psi.value


def num_threads():
    return lib().or_num_threads()


# --------------------------------------------------------------------------- problems

class Problem:
    """A workload in the oracle's internal units, kept alive for the C struct."""

    def __init__(self, wl, gl_order=None, mu_form=MU_SEGMENT, dz_km=None, terms=1,
                 int_tol=1e-10, phi=None, psi=None):
        cen = np.asarray(wl.centre_hz, dtype=np.float64)
        n = len(cen)
        fmin, fmax = float(cen.min()), float(cen.max())
        self.fc_hz = 0.5 * (fmin + fmax)
        self.nu = (cen - self.fc_hz) * 1e-12
        self.R = np.asarray(wl.symbol_rate_baud, dtype=np.float64) * 1e-12
        self.P = np.asarray(wl.launch_power_w, dtype=np.float64)
        if phi is None or psi is None:
            mom = [format_moments(f) for f in wl.formats]
            phi = [m[0] for m in mom]
            psi = [m[1] for m in mom]
        self.phi = np.asarray(phi, dtype=np.float64)
        self.psi = np.asarray(psi, dtype=np.float64)
        self.ptot = float(self.P.sum())
        self.btot = (fmax - fmin) * 1e-12 * n / (n - 1) if n > 1 else float(self.R[0])
        spans = []
        for s in wl.spans:
            a, b2, b3 = units(s.alpha_db_km, s.D_ps_nm_km, s.S_ps_nm2_km, s.lambda_ref_m, self.fc_hz)
            spans.append(OrSpan(a, b2, b3, s.gamma_per_w_km, s.cr_per_w_km_thz, s.length_m * 1e-3))
        self.span_arr = (OrSpan * len(spans))(*spans)
        self.n_ch = n
        gl = int(gl_order if gl_order is not None else wl.gl_order)
        if gl < 1:
            raise ValueError(f"gl_order {gl} < 1")
        self.c = OrProblem(
            n, _ptr(self.nu), _ptr(self.R), _ptr(self.P), _ptr(self.phi), _ptr(self.psi),
            float(wl.rolloff), self.ptot, self.btot, len(spans), self.span_arr,
            gl, int(mu_form),
            float(dz_km if dz_km is not None else wl.dz_km), float(int_tol), int(terms))

    @property
    def spans(self):
        return list(self.span_arr)

    def eta(self, coi=None):
        """(eta [1/W^2], P_NLI [W]) for the listed COIs (all if None)."""
        if coi is None:
            idx = np.arange(self.n_ch, dtype=np.int32)
        else:
            idx = np.asarray(coi, dtype=np.int32).ravel()
        eta = np.zeros(len(idx))
        pn = np.zeros(len(idx))
        rc_ = lib().or_eta(C.byref(self.c), idx.ctypes.data_as(_ip), len(idx), _ptr(eta), _ptr(pn))
        if rc_ != 0:
            raise RuntimeError(f"or_eta failed: {rc_}")
        return eta, pn

    def eta_converged(self, coi=None, tol_db=1e-4, max_order=1024):
        """The converged level of the node rule: the Gauss-Legendre order per island
        side is doubled from this problem's order until no listed channel's eta
        changes by tol_db or more between two orders.  Returns (eta, order, history)
        with history the eta of every order tried; raises RuntimeError when
        max_order is passed first."""
        g0 = self.c.gl_order
        hist = {}
        try:
            g = g0
            prev = hist[g] = self.eta(coi)[0]
            while 2 * g <= max_order:
                g *= 2
                self.c.gl_order = g
                cur = hist[g] = self.eta(coi)[0]
                if np.max(np.abs(10 * np.log10(cur / prev))) < tol_db:
                    return cur, g, hist
                prev = cur
        finally:
            self.c.gl_order = g0
        raise RuntimeError(f"not converged to {tol_db} dB by order {g}")

    def set_coi_offsets(self, off=None):
        """Evaluate each COI n at f = its centre + off[n] [THz] (None: at the centre)."""
        if off is None:
            self._f_off = None
            self.c.f_off = _dp()
        else:
            self._f_off = np.ascontiguousarray(off, dtype=np.float64)
            assert self._f_off.shape == (self.n_ch,)
            self.c.f_off = _ptr(self._f_off)

    def eta_3d(self, n_f, coi=None):
        """(eta, P_NLI) with the integral over f of Eq. 17-21 taken literally:
        f over [-R_n/2, R_n/2] of COI n by an n_f-point Gauss-Legendre rule, the
        2-D island integrals evaluated at each node (n_f = 1: the white-NLI
        value R_n x G(f_n))."""
        x, w = gauss_legendre(int(n_f))
        pn = None
        try:
            for xj, wj in zip(x, w):
                self.set_coi_offsets(0.5 * xj * self.R)
                _, p = self.eta(coi)
                pn = 0.5 * wj * p if pn is None else pn + 0.5 * wj * p
        finally:
            self.set_coi_offsets(None)
        idx = np.arange(self.n_ch) if coi is None else np.asarray(coi).ravel()
        return pn / self.P[idx] ** 3, pn

    def islands(self, n):
        cap = 3 * self.n_ch * self.n_ch + 16
        tri = np.zeros(3 * cap, dtype=np.int32)
        k = lib().or_islands(C.byref(self.c), int(n), tri.ctypes.data_as(_ip), cap)
        if k > cap:
            raise RuntimeError("island buffer too small")
        return tri[: 3 * k].reshape(k, 3)

    def island_exists(self, n, n1, n2, n3):
        return bool(lib().or_island_exists(C.byref(self.c), n, n1, n2, n3))

    def island_terms(self, n, n1, n2, n3, all_terms=False):
        o = np.zeros(5)
        lib().or_island_terms(C.byref(self.c), n, n1, n2, n3, int(all_terms), _ptr(o))
        return o

    def island_terms_midpoint(self, n, n1, n2, n3, M):
        o = np.zeros(5)
        lib().or_island_terms_midpoint(C.byref(self.c), n, n1, n2, n3, int(M), _ptr(o))
        return o

    def island_contribs(self, n):
        cap = 3 * self.n_ch * self.n_ch + 16
        tri = np.zeros(3 * cap, dtype=np.int32)
        con = np.zeros(cap)
        k = lib().or_island_contribs(C.byref(self.c), int(n), tri.ctypes.data_as(_ip), _ptr(con), cap)
        if k < 0:
            raise RuntimeError("island buffer too small")
        return tri[: 3 * k].reshape(k, 3), con[:k]

    def island_nodes(self, n, n1, n2, n3):
        g = self.c.gl_order
        cap = 4 * g * g
        buf = np.zeros(3 * cap)
        k = lib().or_island_nodes(C.byref(self.c), n, n1, n2, n3, _ptr(buf), cap)
        return buf[: 3 * k].reshape(k, 3)

    def upsilon(self, f1, f2, f):
        o = np.zeros(2)
        lib().or_upsilon_out(C.byref(self.c), f1, f2, f, _ptr(o))
        return _cx(o)

    def upsilon_many(self, f1, f2, f):
        f1 = np.ascontiguousarray(f1, dtype=np.float64)
        f2 = np.ascontiguousarray(f2, dtype=np.float64)
        out = np.zeros(2 * len(f1))
        lib().or_upsilon_many(C.byref(self.c), len(f1), _ptr(f1), _ptr(f2), float(f), _ptr(out))
        return out[0::2] + 1j * out[1::2]
