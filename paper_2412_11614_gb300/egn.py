"""Python binding of libegn.so (include/egn.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  PyTorch is
used for device memory (workspace and output tensors) and streams.  If the
shared library is missing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

EGN_OK, EGN_E_INVALID_ARG, EGN_E_UNSUPPORTED, EGN_E_NOMEM, EGN_E_CUDA, EGN_E_TIMEOUT, EGN_E_STATE, EGN_E_CAPACITY = range(8)
EGN_MU_SEGMENT = 0
EGN_MU_MACLAURIN = 1
EGN_MU_INTEGRAL = 2
EGN_PREC_FP64, EGN_PREC_FP32C = 0, 1
EGN_TERMS_GN, EGN_TERMS_EGN = 0, 1
EGN_FMT = {"GAUSS": 0, "QPSK": 1, "16QAM": 2, "64QAM": 3}
EGN_TUNE_FP32C_POINTS_PER_THREAD = 1
EGN_RULE_GL, EGN_RULE_RIDGE = 0, 1
STATUS_NAMES = {0: "EGN_OK", 1: "EGN_E_INVALID_ARG", 2: "EGN_E_UNSUPPORTED", 3: "EGN_E_NOMEM", 4: "EGN_E_CUDA",
                5: "EGN_E_TIMEOUT", 6: "EGN_E_STATE", 7: "EGN_E_CAPACITY"}


class EgnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class egn_span(C.Structure):
    _fields_ = [("alpha_db_per_km", C.c_double), ("D_ps_nm_km", C.c_double), ("S_ps_nm2_km", C.c_double),
                ("lambda_ref_m", C.c_double), ("gamma_per_w_km", C.c_double), ("cr_per_w_km_thz", C.c_double),
                ("length_m", C.c_double)]


class egn_tune_result(C.Structure):
    _fields_ = [("dz_km", C.c_double), ("points_per_thread", C.c_int), ("max_err_db", C.c_double), ("ms", C.c_double)]


class egn_rule_result(C.Structure):
    _fields_ = [("rule", C.c_int), ("nodes", C.c_int), ("max_err_db", C.c_double), ("reference_nodes", C.c_int),
                ("last_change_db", C.c_double), ("configured_err_db", C.c_double), ("ms", C.c_double)]


class egn_opts(C.Structure):
    _fields_ = [("gl_order", C.c_int), ("dz_km", C.c_double), ("mu_form", C.c_int), ("precision", C.c_int),
                ("terms", C.c_int), ("timeout_ms", C.c_int), ("stream", C.c_void_p)]


_dp = C.POINTER(C.c_double)
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libegn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2412_11614_gb300._build.build() "
                               "(the CUDA extension is required; there is no CPU fallback)")
        L = C.CDLL(path)
        L.egn_link_create.argtypes = [C.POINTER(egn_span), C.c_int, C.POINTER(C.c_void_p)]
        L.egn_link_destroy.argtypes = [C.c_void_p]
        L.egn_link_destroy.restype = None
        L.egn_set_wdm.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_double]
        L.egn_workspace_size.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.POINTER(C.c_size_t)]
        L.egn_island_count.argtypes = [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.egn_nli_eta.argtypes = [C.c_void_p, C.POINTER(egn_opts), _dp, _dp]
        L.egn_nli_eta_3d.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_int, _dp, _dp]
        L.egn_nli_eta_device.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_void_p, C.c_size_t, C.c_void_p,
                                         C.c_void_p]
        L.egn_nli_eta_static.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_void_p, C.c_void_p]
        L.egn_island_terms.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_int, C.POINTER(C.c_int), C.c_int, _dp]
        L.egn_plan_islands.argtypes = [C.c_void_p, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
        L.egn_format_moments.argtypes = [C.c_int, _dp, _dp]
        L.egn_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
        L.egn_set_profiling.argtypes = [C.c_void_p, C.c_int]
        L.egn_set_tuning.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.egn_set_node_rule.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.egn_autotune_rule.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_double, C.c_int,
                                        C.POINTER(egn_rule_result)]
        L.egn_last_timings.argtypes = [C.c_void_p, _dp, C.c_int, C.POINTER(C.c_int)]
        L.egn_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(egn_opts), C.POINTER(C.c_void_p)]
        L.egn_batch_launch.argtypes = [C.c_void_p, C.c_void_p]
        L.egn_batch_outputs.argtypes = [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.POINTER(C.c_longlong))]
        L.egn_batch_read.argtypes = [C.c_void_p, C.c_void_p, _dp, _dp]
        L.egn_batch_destroy.argtypes = [C.c_void_p]
        L.egn_batch_destroy.restype = None
        L.egn_nli_eta_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(egn_opts), C.POINTER(_dp),
                                        C.POINTER(_dp)]
        L.egn_autotune.argtypes = [C.c_void_p, C.POINTER(egn_opts), C.c_double, _dp, C.c_int, C.c_double,
                                   C.POINTER(egn_tune_result)]
        L.egn_probe_launch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.egn_probe_ops.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp]
        L.egn_allocation_count.argtypes = [C.POINTER(C.c_longlong)]
        L.egn_last_error.restype = C.c_char_p
        L.egn_version.restype = C.c_char_p
        for fn in ("egn_link_create", "egn_set_wdm", "egn_workspace_size", "egn_island_count", "egn_nli_eta",
                   "egn_nli_eta_device", "egn_island_terms", "egn_plan_islands", "egn_format_moments",
                   "egn_gauss_legendre", "egn_set_profiling", "egn_last_timings", "egn_nli_eta_static", "egn_set_tuning",
                   "egn_batch_create", "egn_batch_launch", "egn_batch_outputs", "egn_batch_read", "egn_nli_eta_batch",
                   "egn_autotune", "egn_nli_eta_3d", "egn_probe_launch", "egn_probe_ops",
                   "egn_allocation_count", "egn_set_node_rule", "egn_autotune_rule"):
            getattr(L, fn).restype = C.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != EGN_OK:
        raise EgnError(status, lib().egn_last_error().decode())


def _arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def egn_version() -> str:
    return lib().egn_version().decode()


def allocation_count() -> int:
    """Device and pinned-host allocations the library has made in this process."""
    n = C.c_longlong()
    _check(lib().egn_allocation_count(C.byref(n)))
    return n.value


def egn_format_moments(fmt) -> tuple:
    code = EGN_FMT[fmt] if isinstance(fmt, str) else int(fmt)
    phi, psi = C.c_double(), C.c_double()
    _check(lib().egn_format_moments(code, C.byref(phi), C.byref(psi)))
    return phi.value, psi.value


def egn_gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(lib().egn_gauss_legendre(n, x.ctypes.data_as(_dp), w.ctypes.data_as(_dp)))
    return x, w


EGN_PROBE = {"ffma": 0, "ffma2": 1, "dfma": 2, "mufu_sin": 3, "mufu_ex2": 4, "mufu_rcp": 5, "fma_mix": 6}


def probe_ops(kind: str, blocks: int, threads: int, iters: int) -> float:
    """Operations of one probe launch (egn_probe_ops): FLOP for the FMA probes,
    special-function operations for the MUFU probes."""
    ops = C.c_double()
    _check(lib().egn_probe_ops(EGN_PROBE[kind], int(blocks), int(threads), int(iters), C.byref(ops)))
    return ops.value


def probe_launch(kind: str, blocks: int, threads: int, iters: int, sink, stream: Optional[int] = None):
    """One throughput-probe launch (egn_probe_launch) into a device tensor `sink`
    of at least blocks * threads * 8 bytes, on `stream`."""
    if sink.numel() * sink.element_size() < blocks * threads * 8:
        raise ValueError("probe sink too small")
    _check(lib().egn_probe_launch(EGN_PROBE[kind], int(blocks), int(threads), int(iters),
                                  C.c_void_p(sink.data_ptr()), C.c_void_p(stream) if stream else None))


def make_opts(gl_order=32, dz_km=1.0, precision=EGN_PREC_FP32C, terms=EGN_TERMS_EGN, timeout_ms=0,
              stream: Optional[int] = None, mu_form=EGN_MU_SEGMENT) -> egn_opts:
    return egn_opts(int(gl_order), float(dz_km), int(mu_form), int(precision), int(terms), int(timeout_ms),
                    C.c_void_p(stream) if stream else None)


class Link:
    """An egn_link handle (egn_link_create / egn_set_wdm / egn_link_destroy)."""

    def __init__(self, spans: Sequence):
        arr = (egn_span * len(spans))()
        for i, s in enumerate(spans):
            arr[i] = egn_span(s.alpha_db_km, s.D_ps_nm_km, s.S_ps_nm2_km, s.lambda_ref_m, s.gamma_per_w_km,
                              s.cr_per_w_km_thz, s.length_m)
        h = C.c_void_p()
        _check(lib().egn_link_create(arr, len(spans), C.byref(h)))
        self.h = h
        self.n_ch = 0

    def close(self):
        if self.h:
            lib().egn_link_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wdm(self, centre_hz, symbol_rate_baud, launch_power_w, phi, psi, rolloff):
        c, r, p, f, s = (_arr(x) for x in (centre_hz, symbol_rate_baud, launch_power_w, phi, psi))
        ptr = lambda a: a.ctypes.data_as(_dp)  # noqa: E731
        _check(lib().egn_set_wdm(self.h, len(c), ptr(c), ptr(r), ptr(p), ptr(f), ptr(s), float(rolloff)))
        self.n_ch = len(c)

    def island_count(self):
        """(total, per-COI counts, half-list size, E-list size, F-list size)."""
        tot, nh, ne, nf = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        per = (C.c_longlong * self.n_ch)()
        _check(lib().egn_island_count(self.h, C.byref(tot), per, C.byref(nh), C.byref(ne), C.byref(nf)))
        return tot.value, np.array(per[:], dtype=np.int64), nh.value, ne.value, nf.value

    def workspace_size(self, opts: egn_opts) -> int:
        b = C.c_size_t()
        _check(lib().egn_workspace_size(self.h, C.byref(opts), C.byref(b)))
        return b.value

    def nli_eta(self, opts: egn_opts):
        """Host API: returns (eta [1/W^2], P_NLI [W]) as numpy arrays."""
        eta = np.zeros(self.n_ch)
        pn = np.zeros(self.n_ch)
        _check(lib().egn_nli_eta(self.h, C.byref(opts), eta.ctypes.data_as(_dp), pn.ctypes.data_as(_dp)))
        return eta, pn

    def nli_eta_3d(self, opts: egn_opts, n_f: int):
        """f-integrated (3-D) EGN: (eta, P_NLI) with the COI band integrated by an
        n_f-point Gauss-Legendre rule (n_f = 1: the white-NLI value)."""
        eta = np.zeros(self.n_ch)
        pn = np.zeros(self.n_ch)
        _check(lib().egn_nli_eta_3d(self.h, C.byref(opts), int(n_f), eta.ctypes.data_as(_dp),
                                    pn.ctypes.data_as(_dp)))
        return eta, pn

    def nli_eta_device(self, opts: egn_opts, workspace, eta_dev=None, pnli_dev=None):
        """Device API on opts.stream with a torch-allocated workspace (uint8 tensor)
        and optional float64 device output tensors."""
        _check(lib().egn_nli_eta_device(self.h, C.byref(opts), C.c_void_p(workspace.data_ptr()),
                                        workspace.numel() * workspace.element_size(),
                                        C.c_void_p(eta_dev.data_ptr()) if eta_dev is not None else None,
                                        C.c_void_p(pnli_dev.data_ptr()) if pnli_dev is not None else None))

    def nli_eta_static(self, opts: egn_opts, eta_dev, pnli_dev):
        """Allocation-free evaluation (scratch compiled into the library) on
        opts.stream into float64 device tensors of n_ch entries."""
        _check(lib().egn_nli_eta_static(self.h, C.byref(opts), C.c_void_p(eta_dev.data_ptr()),
                                        C.c_void_p(pnli_dev.data_ptr())))

    def island_terms(self, opts: egn_opts, islands, all_terms=False) -> np.ndarray:
        isl = np.ascontiguousarray(np.asarray(islands, dtype=np.int32).reshape(-1, 4))
        out = np.zeros((len(isl), 5))
        _check(lib().egn_island_terms(self.h, C.byref(opts), len(isl), isl.ctypes.data_as(C.POINTER(C.c_int)),
                                      int(bool(all_terms)), out.ctypes.data_as(_dp)))
        return out

    def autotune(self, opts: egn_opts, target_db: float, dz_candidates, dz_ref_km: float) -> dict:
        """egn_autotune: coarsest segment bound within target_db of the reference,
        and the faster FP32C launch shape (set on the link)."""
        cand = _arr(dz_candidates)
        r = egn_tune_result()
        _check(lib().egn_autotune(self.h, C.byref(opts), float(target_db), cand.ctypes.data_as(_dp), len(cand),
                                  float(dz_ref_km), C.byref(r)))
        return {"dz_km": r.dz_km, "points_per_thread": r.points_per_thread, "max_err_db": r.max_err_db, "ms": r.ms}

    def autotune_rule(self, opts: egn_opts, target_db: float, max_nodes: int = 64) -> dict:
        """egn_autotune_rule: the ridge rule's order within target_db of its converged
        value (set on the link), and the configured rule's error against it."""
        r = egn_rule_result()
        _check(lib().egn_autotune_rule(self.h, C.byref(opts), float(target_db), int(max_nodes), C.byref(r)))
        return {f: getattr(r, f) for f, _ in egn_rule_result._fields_}

    def set_tuning(self, param: int, value: int):
        _check(lib().egn_set_tuning(self.h, int(param), int(value)))

    def set_node_rule(self, rule: int, n_min: int = 4):
        """egn_set_node_rule: EGN_RULE_GL (default) or EGN_RULE_RIDGE (FP64 on any link, FP32C on links
        of at most four span types)."""
        _check(lib().egn_set_node_rule(self.h, int(rule), int(n_min)))

    def set_profiling(self, on: bool):
        _check(lib().egn_set_profiling(self.h, int(bool(on))))

    def last_timings(self) -> dict:
        """Device ms of the last evaluation per stage (needs set_profiling(True))."""
        ms = np.zeros(5)
        n = C.c_int()
        _check(lib().egn_last_timings(self.h, ms.ctypes.data_as(_dp), 5, C.byref(n)))
        return dict(zip(("plan", "integrate_dgh", "integrate_e", "integrate_f", "assemble"), ms[: n.value]))

    def plan_islands(self) -> np.ndarray:
        tot = self.island_count()[0]
        out = np.zeros((max(tot, 1), 4), dtype=np.int32)
        cnt = C.c_longlong()
        _check(lib().egn_plan_islands(self.h, tot, out.ctypes.data_as(C.POINTER(C.c_int)), C.byref(cnt)))
        return out[: cnt.value]


def _handles(links) -> "C.Array":
    arr = (C.c_void_p * len(links))()
    for i, ln in enumerate(links):
        arr[i] = ln.h
    return arr


class Batch:
    """An egn_batch handle: links snapshotted for repeated evaluation by one CUDA
    graph (egn_batch_create / egn_batch_launch / egn_batch_read)."""

    def __init__(self, links: Sequence[Link], opts: egn_opts):
        h = C.c_void_p()
        _check(lib().egn_batch_create(_handles(links), len(links), C.byref(opts), C.byref(h)))
        self.h = h
        off = C.POINTER(C.c_longlong)()
        _check(lib().egn_batch_outputs(self.h, None, None, C.byref(off)))
        self.offsets = np.array(off[: len(links) + 1], dtype=np.int64)

    def launch(self, stream: Optional[int] = None):
        _check(lib().egn_batch_launch(self.h, C.c_void_p(stream) if stream else None))

    def outputs(self):
        """Device addresses of eta and P_NLI of all channels (link after link)."""
        e, p = C.c_void_p(), C.c_void_p()
        _check(lib().egn_batch_outputs(self.h, C.byref(e), C.byref(p), None))
        return e.value, p.value

    def read(self, stream: Optional[int] = None):
        """Wait for the work on `stream`, then [(eta, P_NLI) per link] on the host."""
        n = int(self.offsets[-1])
        eta, pn = np.zeros(n), np.zeros(n)
        _check(lib().egn_batch_read(self.h, C.c_void_p(stream) if stream else None, eta.ctypes.data_as(_dp),
                                    pn.ctypes.data_as(_dp)))
        o = self.offsets
        return [(eta[o[i]:o[i + 1]], pn[o[i]:o[i + 1]]) for i in range(len(o) - 1)]

    def close(self):
        if self.h:
            lib().egn_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nli_eta_batch(links: Sequence[Link], opts: egn_opts):
    """One evaluation of several links (egn_nli_eta_batch): [(eta, P_NLI) per link]."""
    outs = [(np.zeros(ln.n_ch), np.zeros(ln.n_ch)) for ln in links]
    ep = (_dp * len(links))(*[o[0].ctypes.data_as(_dp) for o in outs])
    pp = (_dp * len(links))(*[o[1].ctypes.data_as(_dp) for o in outs])
    _check(lib().egn_nli_eta_batch(_handles(links), len(links), C.byref(opts), ep, pp))
    return outs


def link_from_workload(wl, phi=None, psi=None) -> Link:
    """Create a Link from a workloads.Workload (format moments from the library)."""
    ln = Link(wl.spans)
    if phi is None or psi is None:
        mom = [egn_format_moments(f) for f in wl.formats]
        phi = [m[0] for m in mom]
        psi = [m[1] for m in mom]
    ln.set_wdm(wl.centre_hz, wl.symbol_rate_baud, wl.launch_power_w, phi, psi, wl.rolloff)
    return ln
