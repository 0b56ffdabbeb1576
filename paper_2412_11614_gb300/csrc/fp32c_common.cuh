// fp32c_common.cuh -- device helpers of the FP32 integrators: double-float
// ("df", an unevaluated FP32 head + tail) arithmetic, packed FP32x2 FMA, exact
// rounding to an integer, hardware-approximation wrappers, small-angle sine,
// the raised-cosine shape, and a row's phase polynomial and its exact per-point
// reduction.
#pragma once

#include "egn_internal.h"

namespace egn {
namespace fp32c {

struct Df {
  float hi, lo;
};

__device__ __forceinline__ Df df_of(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ Df quick(float s, float e) {
  float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ Df dadd(Df a, Df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return quick(s, e);
}
__device__ __forceinline__ Df dneg(Df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ Df dsub(Df a, Df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ Df dmul(Df a, Df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return quick(p, e);
}
__device__ __forceinline__ Df dhalf(Df a) { return {0.5f * a.hi, 0.5f * a.lo}; }
__device__ __forceinline__ bool dgt(Df a, Df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ Df dmax(Df a, Df b) { return dgt(a, b) ? a : b; }
__device__ __forceinline__ Df dmin(Df a, Df b) { return dgt(a, b) ? b : a; }
__device__ __forceinline__ float dval(Df a) { return a.hi + a.lo; }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32x2: two lanes of FP32 in one 64-bit register, one FMA instruction
// for both (fma.rn.f32x2), which halves the issue slots of the segment recurrence.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Round to nearest (ties to even) by adding and subtracting 1.5 * 2^23; exact for
// |x| < 2^22, two FP32 additions on the FMA pipe.
__device__ __forceinline__ float rint_fast(float x) {
  const float M = 12582912.0f;
  return (x + M) - M;
}

// The same rounding by cvt.rni (exact at any magnitude); it leaves the FMA pipe,
// which the per-point arithmetic keeps busy, to the conversion unit.
__device__ __forceinline__ float rint_cvt(float x) {
  float y;
  asm("cvt.rni.f32.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// sin(x) for |x| < 0.05 by its Taylor series to x^5 (relative error < 4e-12).
__device__ __forceinline__ float sin_small(float x) {
  const float x2 = x * x;
  return x * fmaf(x2, fmaf(x2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
}

// Phased-array sines of Eq. 22: sd = sin(x), sn = sin(N x) for x = pi phi,
// |x| <= pi / 2, so that the ratio is sn / sd.  Hardware sines (absolute error
// ~4e-7) away from zero; within |.| < 0.05 the Taylor series keeps the relative
// error small where the ratio peaks at N.  Both forms are evaluated and
// selected, so the warp does not diverge.  Below |x| = 1e-12 the pair is
// (1, N): the ratio is N to within (N x)^2 and no reciprocal of a vanishing
// sine is taken.
__device__ __forceinline__ void array_sines(float x, float N, float& sd, float& sn) {
  const float Nx = N * x;
  const float d = fabsf(x) < 0.05f ? sin_small(x) : __sinf(x);
  const float nn = fabsf(Nx) < 0.05f ? sin_small(Nx) : __sinf(Nx);
  const bool z = fabsf(x) < 1e-12f;
  sd = z ? 1.0f : d;
  sn = z ? N : nn;
}
__device__ __forceinline__ float array_ratio(float x, float N) {
  float sd, sn;
  array_sines(x, N, sd, sn);
  return sn * rcp_approx(sd);
}

// Raised-cosine shape in FP32 without branches: a = (1 - beta) R / 2 is the knee
// and inv = 1 / (beta R) (0 when beta = 0, where every node lies in the flat
// part).  t = clamp((|x| - a) / (beta R), 0, 1), h = (1 + cos(pi t)) / 2.
__device__ __forceinline__ float rc_f(float x, float a, float inv) {
  const float t = __saturatef((fabsf(x) - a) * inv);
  return fmaf(0.5f, __cosf(3.14159265f * t), 0.5f);
}

// Per-link constants of the identical-spans passes: K, the segment factor
// r = e^{-alpha dz} and its combinations, the span count N and gamma.
struct DwConsts {
  int K;
  float Kf, invK, alpha, alpha2, r, one_m_r, q, m2r, c2r, c4r, omr2, N, gam, g2;
};

__device__ __forceinline__ DwConsts dw_consts(const LinkParams& p) {
  DwConsts c;
  c.K = p.seg.K;
  c.Kf = (float)c.K;
  c.invK = 1.0f / (float)c.K;
  c.alpha = (float)p.alpha;
  c.alpha2 = c.alpha * c.alpha;
  c.r = (float)p.r;
  c.one_m_r = (float)(-expm1(-p.alpha * p.dz));
  c.q = c.r * c.r;
  c.m2r = -2.0f * c.r;
  c.c2r = 2.0f * c.r;
  c.c4r = 4.0f * c.r;
  c.omr2 = c.one_m_r * c.one_m_r;
  c.N = (float)p.n_spans;
  c.gam = (float)p.gamma;
  c.g2 = c.gam * c.gam;
  return c;
}

// Row geometry in double-float: outer node o, inner interval im +- ih and the
// linear forms f1 - f = a0 + a1 x, f2 - f = b0 + b1 x, f1 + f2 = s0 + s1 x of the
// inner Gauss-Legendre coordinate x (frequencies relative to the spectral centre).
struct RowGeo {
  Df o, im, ih, a0, a1, b0, b1, s0, s1, ph;
};

// Phase polynomial of a row for one span type, in turns of that span:
// Theta(x) = Q0 + Q1 x + Q2 x^2 + Q3 x^3 with Q0 reduced modulo K.
// G0 = 2 pi L beta2, G1 = 2 pi^2 L beta3 (double-floats).
struct RowPhase {
  Df Q0r, Q1, Q2;
  float Q3;
};

__device__ __forceinline__ RowPhase row_phase(const RowGeo& r, Df G0, Df G1, float Kf, float invK) {
  const Df g0 = dadd(G0, dmul(G1, r.s0));   // 2 pi L (beta2 + pi beta3 s0)
  const Df g1 = dmul(G1, r.s1);             // 2 pi L pi beta3 s1
  const Df ab0 = dmul(r.a0, r.b0);
  const Df ab1 = dadd(dmul(r.a0, r.b1), dmul(r.a1, r.b0));
  const Df ab2 = dmul(r.a1, r.b1);
  const Df Q0 = dmul(g0, ab0);
  RowPhase q;
  q.Q1 = dadd(dmul(g0, ab1), dmul(g1, ab0));
  q.Q2 = dadd(dmul(g0, ab2), dmul(g1, ab1));
  q.Q3 = dval(g1) * dval(ab2);
  const float r0 = fmaf(-Kf, rint_fast(Q0.hi * invK), Q0.hi);  // the FMA residual is exact
  q.Q0r = quick(r0, Q0.lo);
  return q;
}

// Phase of one point of a row: theta (turns of one segment, chi L / (2 pi K))
// and phi (turns of the span, chi L / (2 pi)), both reduced to [-1/2, 1/2].
// qa = {q0h, q0l, q1h, q1l}, qb = {q2h, q2l, q3, frac(q0h)}, x4 = {x, x tail,
// x^2, x^2 tail}, xc = x^3.  Q1 x and Q2 x^2 are exact FP32 products (head by
// FMA residual, tails by the cross terms); Q1 x is reduced modulo K exactly.
__device__ __forceinline__ void point_phase(const float4& qa, const float4& qb, const float4& x4, float xc, float Kf,
                                            float invK, float& th, float& ph) {
  const float p1 = qa.z * x4.x, e1 = fmaf(qa.z, x4.x, -p1);
  const float t1 = fmaf(qa.z, x4.y, fmaf(qa.w, x4.x, e1));
  const float p2 = qb.x * x4.z, e2 = fmaf(qb.x, x4.z, -p2);
  const float t2 = fmaf(qb.x, x4.w, fmaf(qb.y, x4.z, e2));
  const float r1 = fmaf(-Kf, rint_cvt(p1 * invK), p1);
  const float tail = (qa.y + t1) + fmaf(qb.z, xc, t2);
  th = fmaf((qa.x + r1) + p2, invK, tail * invK);
  th -= rint_cvt(th);
  ph = (qb.w + (r1 - rint_cvt(r1))) + ((p2 - rint_cvt(p2)) + tail);
  ph -= rint_cvt(ph);
}

}  // namespace fp32c
}  // namespace egn
