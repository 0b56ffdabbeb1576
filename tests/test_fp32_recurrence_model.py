"""Error model of the FP32C segment sum (no GPU): sum_k c_k w^k evaluated by the
second-order real recurrence b_k = c_k + 2 Re(w) b_{k+1} - |w|^2 b_{k+2},
sum = b_0 - conj(w) b_1, in FP32 with fused multiply-adds, against the FP64
polynomial, on the benchmark fibre's c_k (K = 80, alpha 0.2 dB/km, 1 km segments,
P_tot Cr of the 120-channel link) for random segment phases and phases near 0 and
pi, where the recurrence's two roots nearly coincide.  The FP32C integrator's
accuracy budget (1e-3 dB on small links, 0.01 dB at full size) leaves room for
the bound checked here by two orders of magnitude."""
import numpy as np

f32 = np.float32


def _fma32(a, b, c):
    # FP32 operands: the product is exact in FP64, one rounding of the sum to FP64
    # and one to FP32 (a faithful model of fma.rn.f32 for these magnitudes)
    return f32(float(a) * float(b) + float(c))


def _recurrence32(c, w):
    p, q = f32(2.0 * w.real), f32(abs(w) ** 2)
    b1 = b2 = f32(0.0)
    for k in range(len(c) - 1, -1, -1):
        b0 = _fma32(p, b1, _fma32(-q, b2, c[k]))  # p b_{k+1} + (c_k - q b_{k+2})
        b2, b1 = b1, b0
    wr, wi = f32(w.real), f32(w.imag)
    return complex(_fma32(-wr, b2, b1), f32(wi * b2))


def test_fp32_recurrence_error_bound():
    K, dz = 80, 1.0
    a = 0.2 * np.log(10) / 10
    r = np.exp(-a * dz)
    ptot, cr, btot = 0.19, 0.028, 9.0
    z = (np.arange(K) + 0.5) * dz
    zeta = ptot * cr * (-np.expm1(-a * z) / a)
    ck = btot * zeta / (2 * np.sinh(btot * zeta / 2))
    rng = np.random.default_rng(0)
    thetas = np.concatenate([rng.uniform(-np.pi, np.pi, 200), rng.uniform(-1e-3, 1e-3, 100),
                             np.pi - rng.uniform(0, 1e-3, 100)])
    worst = 0.0
    for th in thetas:
        c = (ck * np.exp(-zeta * rng.uniform(-4.5, 4.5))).astype(np.float32)
        w = r * np.exp(1j * th)
        ref = np.polyval(c[::-1].astype(np.float64), w)
        worst = max(worst, abs(_recurrence32(c, w) - ref) / abs(ref))
    assert worst < 1e-4, worst
