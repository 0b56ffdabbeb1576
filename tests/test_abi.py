"""CPU checks of the C ABI: the library builds and loads, exports every entry
point the headers under include/ declare, and its host-only logic (argument
validation, format moments, Gauss-Legendre nodes) is right.  No compute call
needs a GPU here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def egn():
    from paper_2412_11614_gb300 import _build
    _build.build()
    from paper_2412_11614_gb300 import egn as E
    E.lib()
    return E


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            src = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(egn_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("egn_link_create", "egn_set_wdm", "egn_nli_eta", "egn_link_destroy", "egn_last_error",
                 "egn_format_moments", "egn_nli_eta_device", "egn_workspace_size", "egn_batch_create",
                 "egn_autotune", "egn_mlp_gemm", "egn_mlp_adam"):
        assert must in names


def test_every_declared_symbol_is_exported(egn):
    L = egn.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_library_is_in_tree(egn):
    assert os.path.commonpath([egn.library_path(), ROOT]) == ROOT


def test_format_moments_match_oracle(egn, oracle_mod):
    for f in ("QPSK", "16QAM", "64QAM", "GAUSS"):
        a = egn.egn_format_moments(f)
        b = oracle_mod.format_moments(f)
        assert a == pytest.approx(b, abs=1e-13)


def test_gauss_legendre_nodes(egn):
    for n in (1, 2, 3, 11, 16, 32, 64, 128):
        x, w = egn.egn_gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, xr, atol=2e-15, rtol=0)
        assert np.allclose(w, wr, atol=1e-14, rtol=0)


def _bad_span(workloads, **kw):
    s = workloads.config_small().spans[0]
    for k, v in kw.items():
        setattr(s, k, v)
    return s


@pytest.mark.parametrize("field,value", [("alpha_db_km", 0.0), ("alpha_db_km", float("nan")), ("length_m", -1.0),
                                         ("cr_per_w_km_thz", -0.1), ("lambda_ref_m", 0.0),
                                         ("gamma_per_w_km", float("inf"))])
def test_link_create_rejects_bad_spans(egn, workloads, field, value):
    with pytest.raises(egn.EgnError) as ei:
        egn.Link([_bad_span(workloads, **{field: value})])
    assert ei.value.status == egn.EGN_E_INVALID_ARG


def test_link_create_rejects_empty(egn):
    import ctypes as C
    h = C.c_void_p()
    assert egn.lib().egn_link_create(None, 0, C.byref(h)) == egn.EGN_E_INVALID_ARG
    assert egn.lib().egn_link_create(None, 1, None) == egn.EGN_E_INVALID_ARG


def test_set_wdm_rejects_bad_combs_before_touching_the_device(egn, workloads):
    wl = workloads.config_small()
    ln = egn.Link(wl.spans)
    phi = [0.0] * 5
    bad = [
        dict(centre_hz=wl.centre_hz[::-1]),                                 # not increasing
        dict(centre_hz=[wl.centre_hz[0] + 30e9 * k for k in range(5)]),     # overlapping
        dict(symbol_rate_baud=[64e9, 64e9, -1.0, 64e9, 64e9]),
        dict(launch_power_w=[1e-3, 1e-3, float("nan"), 1e-3, 1e-3]),
    ]
    for b in bad:
        args = dict(centre_hz=wl.centre_hz, symbol_rate_baud=wl.symbol_rate_baud, launch_power_w=wl.launch_power_w)
        args.update(b)
        with pytest.raises(egn.EgnError) as ei:
            ln.set_wdm(args["centre_hz"], args["symbol_rate_baud"], args["launch_power_w"], phi, phi, 0.01)
        assert ei.value.status == egn.EGN_E_INVALID_ARG
    with pytest.raises(egn.EgnError):
        ln.set_wdm(wl.centre_hz, wl.symbol_rate_baud, wl.launch_power_w, phi, phi, 1.5)  # roll-off > 1


def test_eta_before_set_wdm_is_a_state_error(egn, workloads):
    ln = egn.Link(workloads.config_small().spans)
    with pytest.raises(egn.EgnError) as ei:
        ln.nli_eta(egn.make_opts())
    assert ei.value.status == egn.EGN_E_STATE


def test_last_error_is_informative(egn, workloads):
    with pytest.raises(egn.EgnError) as ei:
        egn.Link([_bad_span(workloads, length_m=0.0)])
    assert "length" in str(ei.value)


def test_new_entry_points_validate_before_launching(egn):
    """Bad shapes and null arguments are refused before any device work (no GPU here)."""
    import ctypes as C
    from paper_2412_11614_gb300 import mlp
    L = mlp._lib()
    fake = C.c_void_p(0x10000)  # never dereferenced: validation fails first
    # k not a multiple of 64, n not a multiple of 32, splits without the FP32 epilogue, misaligned A
    assert L.egn_mlp_gemm(64, 32, 96, 1, fake, fake, mlp.EPI_F32, None, None, fake, fake, None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_gemm(64, 40, 64, 1, fake, fake, mlp.EPI_F32, None, None, fake, fake, None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_gemm(64, 32, 128, 2, fake, fake, mlp.EPI_BIAS, fake, None, fake, fake, None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_gemm(64, 32, 64, 1, C.c_void_p(0x10004), fake, mlp.EPI_F32, None, None, fake, fake,
                          None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_gemm(64, 32, 64, 1, fake, fake, mlp.EPI_RELU_GRAD, None, None, fake, fake, None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_adam(None, None, None, None, 4, 1e-3, 0.9, 0.999, 1e-8, 1, None, None, 1, 4, None) == egn.EGN_E_INVALID_ARG
    assert L.egn_mlp_head(fake, 10, 40, fake, fake, fake, None, None, None, None, None, None, None, None) == \
        egn.EGN_E_INVALID_ARG  # hid not a multiple of 32
    # batches and the autotuner
    lib = egn.lib()
    opts = egn.make_opts()
    out = C.c_void_p()
    assert lib.egn_batch_create((C.c_void_p * 1)(), 0, C.byref(opts), C.byref(out)) == egn.EGN_E_INVALID_ARG
    res = egn.egn_tune_result()
    cand = (C.c_double * 1)(1.0)
    assert lib.egn_autotune(None, C.byref(opts), 0.01, cand, 1, 0.5, C.byref(res)) == egn.EGN_E_INVALID_ARG
    assert "null" in lib.egn_last_error().decode()
    # pipe probes: kind, launch shape and the sink are checked before any launch
    ops = C.c_double()
    assert lib.egn_probe_ops(0, 4, 256, 10, C.byref(ops)) == egn.EGN_OK and ops.value == 2 * 4 * 256 * 8 * 10
    assert lib.egn_probe_ops(1, 4, 256, 10, C.byref(ops)) == egn.EGN_OK and ops.value == 4 * 4 * 256 * 8 * 10
    assert lib.egn_probe_ops(3, 4, 256, 10, C.byref(ops)) == egn.EGN_OK and ops.value == 4 * 256 * 8 * 10
    assert lib.egn_probe_ops(6, 4, 256, 10, C.byref(ops)) == egn.EGN_OK and ops.value == 6 * 4 * 256 * 8 * 10
    assert lib.egn_probe_ops(9, 4, 256, 10, C.byref(ops)) == egn.EGN_E_INVALID_ARG
    assert lib.egn_probe_launch(0, 4, 48, 10, fake, None) == egn.EGN_E_INVALID_ARG
    assert lib.egn_probe_launch(0, 4, 256, 10, None, None) == egn.EGN_E_INVALID_ARG
    # the allocation counter: a count, and refuses a null output
    assert egn.allocation_count() >= 0
    assert lib.egn_allocation_count(None) == egn.EGN_E_INVALID_ARG
