// island_geom.cuh -- node rule of one island, shared by the FP64 and FP32C
// integrators (device code).
//
// An island (COI n; n1, n2, n3) lives in local coordinates u, v, w (offsets of
// f1, f2, f3 = f1 + f2 - f from the centres of channels n1, n2, n3), with
// w = u + v + d, d = (nu_n1 - nu_n) + (nu_n2 - nu_n3), and supports |u| <= W1/2,
// |v| <= W2/2, |w| <= W3/2.  Each evaluation order has one outer variable o with
// |o| <= A and one inner variable t with |t| <= B, coupled by |t - (s o + c)| <= C:
//   DW (D, G, H): o = w, t = u, s = +1, c = -d, C = W2/2   (Eq. 17, 20, 21)
//   E           : o = v, t = u, s = -1, c = -d, C = W3/2   (Eq. 18: inner over f1)
//   F           : o = u, t = v, s = -1, c = -d, C = W3/2   (Eq. 19: inner over f2)
// The inner interval is [max(-B, m - C), min(B, m + C)], m = s o + c; the outer
// range is where it is non-empty, split at the kinks m = C - B and m = B - C that
// lie strictly inside.  P panels of ceil(n/P) Gauss-Legendre nodes each, n inner
// nodes per outer node.
#pragma once

#include "egn_internal.h"

namespace egn {

enum { ORD_DW = 0, ORD_E = 1, ORD_F = 2 };

struct Ordering {
  double A, B, s, c, C;
};

__device__ __forceinline__ Ordering make_ordering(int ord, double W1, double W2, double W3, double d) {
  Ordering g;
  g.c = -d;
  if (ord == ORD_DW) { g.A = 0.5 * W3; g.B = 0.5 * W1; g.s = 1.0; g.C = 0.5 * W2; }
  else if (ord == ORD_E) { g.A = 0.5 * W2; g.B = 0.5 * W1; g.s = -1.0; g.C = 0.5 * W3; }
  else { g.A = 0.5 * W1; g.B = 0.5 * W2; g.s = -1.0; g.C = 0.5 * W3; }
  return g;
}

// Outer panel edges e[0..P]; returns P (0 when the island has zero area).
__device__ __forceinline__ int outer_panels(const Ordering& g, double e[4]) {
  double p = g.s * (-(g.B + g.C) - g.c);
  double q = g.s * ((g.B + g.C) - g.c);
  double lo = fmax(-g.A, fmin(p, q));
  double hi = fmin(g.A, fmax(p, q));
  if (!(hi > lo)) return 0;
  double k1 = g.s * ((g.C - g.B) - g.c);
  double k2 = g.s * ((g.B - g.C) - g.c);
  if (k1 > k2) { double t = k1; k1 = k2; k2 = t; }
  int np = 0;
  e[np++] = lo;
  if (k1 > lo && k1 < hi) e[np++] = k1;
  if (k2 > lo && k2 < hi && k2 != k1) e[np++] = k2;
  e[np++] = hi;
  return np - 1;
}

__device__ __forceinline__ void inner_limits(const Ordering& g, double o, double& lo, double& hi) {
  double m = g.s * o + g.c;
  lo = fmax(-g.B, m - g.C);
  hi = fmin(g.B, m + g.C);
}

// Raised-cosine power shape h(x), unit in band, support |x| <= (1 + beta) R / 2.
__device__ __forceinline__ double rc_shape(double x, double R, double beta) {
  double ax = fabs(x);
  double a = 0.5 * (1.0 - beta) * R, b = 0.5 * (1.0 + beta) * R;
  if (ax <= a) return 1.0;
  if (ax >= b) return 0.0;
  return 0.5 * (1.0 + cospi((ax - a) / (beta * R)));
}

// Term coefficients after |S|^2 = h / R^2 and the COI integral -> R x value at
// the COI centre: D (16/27) R / (R1 R2 R3), E (16/27) R^-3, F (32/81) R^-3,
// G (16/81) R^-3, H (16/81) R^-4 (Eq. 17-21).
__device__ __forceinline__ void term_coefs(double R, double R1, double R2, double R3, double cf[5]) {
  cf[0] = (16.0 / 27.0) * R / (R1 * R2 * R3);
  cf[1] = (16.0 / 27.0) / (R * R * R);
  cf[2] = (32.0 / 81.0) / (R * R * R);
  cf[3] = (16.0 / 81.0) / (R * R * R);
  cf[4] = (16.0 / 81.0) / (R * R * R * R);
}

}  // namespace egn
