// ridge_rule.cuh -- geometry of the ridge-resolving node rule
// (egn_set_node_rule(EGN_RULE_RIDGE)), shared by the FP64 and FP32C integrators.
//
// With chi of Eq. 5/24, |mu|^2 of Eq. 8-10 is close to 1 / (alpha^2 + chi^2):
// along f1 at fixed f2 a Lorentzian centred on f1 = f of half-width alpha /
// (4 pi^2 |beta2 + 2 pi beta3 f| |f2 - f|), and likewise along f2 -- tens of MHz
// for interferers a THz away, inside channels of tens of GHz.  The raised-cosine
// shapes add kinks at their knees.  In each evaluation order (outer o, inner t,
// coupled by |t - (s o + c)| <= C, see island_geom.cuh):
//   * the outer range is cut at the knees of the outer shape, wherever two inner
//     break lines t = const and t = s o + const cross (which includes the
//     island's kinks), and at a ridge of the outer variable;
//   * each inner interval is cut at the knees of the other two shapes and at the
//     ridge points f1 = f and f2 = f inside it;
//   * cuts closer than 1e-12 THz merge (a ridge wins); a piece that ends on a
//     ridge gets n nodes placed by x = x_r + h sinh(tau), tau on an n-point
//     Gauss-Legendre rule over [0, asinh(length / h)] (h the ridge half-width; a
//     piece with a ridge at both ends is halved first); another piece gets
//     max(n_min, ceil(n length / interval)) Gauss-Legendre nodes.
// The ridge half-widths take one span's alpha, beta2 and beta3 (the first span's).
// Everything here is FP64: the rule's cuts and pieces are per island and per row.
#pragma once

#include "egn_internal.h"
#include "island_geom.cuh"

namespace egn {

struct RCut {
  double x, h;  // h > 0: a ridge of half-width h; otherwise a plain cut
};
struct RPiece {
  double a, b, ha, hb;  // ends and their ridge half-widths (<= 0: none)
  int m;                // nodes
};
constexpr int kOuterCuts = 30;  // 2 knees + 5 x 5 crossings + 1 ridge of the outer variable
constexpr int kInnerCuts = 6;   // 4 knees + 2 ridges
constexpr int kOuterPieces = 2 * (kOuterCuts + 1);
constexpr int kInnerPieces = 2 * (kInnerCuts + 1);

__device__ __forceinline__ void sort_cuts(RCut* c, int n) {  // stable, ascending x
  for (int i = 1; i < n; ++i) {
    const RCut v = c[i];
    int j = i;
    while (j > 0 && c[j - 1].x > v.x) {
      c[j] = c[j - 1];
      --j;
    }
    c[j] = v;
  }
}

// Pieces of [lo, hi] cut at the points of `pts` inside it; returns their number.
template <int MAXC>
__device__ int ridge_pieces(double lo, double hi, const RCut* pts, int np, int n, int n_min, RPiece* out) {
  const double eps = 1e-12;
  RCut cand[MAXC];
  int nc = 0;
  for (int i = 0; i < np; ++i)
    if (lo + eps < pts[i].x && pts[i].x < hi - eps) cand[nc++] = pts[i];
  sort_cuts(cand, nc);
  RCut e[MAXC + 2];
  int ne = 0;
  e[ne++] = {lo, -1.0};
  for (int i = 0; i < nc; ++i) {
    if (ne > 1 && cand[i].x - e[ne - 1].x < eps) {  // merges into the previous cut
      if (cand[i].h > 0.0) e[ne - 1].h = cand[i].h;
      continue;
    }
    e[ne++] = cand[i];
  }
  e[ne++] = {hi, -1.0};
  for (int i = 0; i < np; ++i) {  // a ridge on an end of the interval
    if (pts[i].h > 0.0 && fabs(pts[i].x - lo) <= eps) e[0].h = pts[i].h;
    if (pts[i].h > 0.0 && fabs(pts[i].x - hi) <= eps) e[ne - 1].h = pts[i].h;
  }
  int k = 0;
  for (int i = 0; i + 1 < ne; ++i) {
    const double a = e[i].x, b = e[i + 1].x, ha = e[i].h, hb = e[i + 1].h;
    if (!(b > a)) continue;
    if (ha > 0.0 && hb > 0.0) {
      const double mid = 0.5 * (a + b);
      out[k++] = {a, mid, ha, -1.0, n};
      out[k++] = {mid, b, -1.0, hb, n};
    } else if (ha > 0.0 || hb > 0.0) {
      out[k++] = {a, b, ha, hb, n};
    } else {
      out[k++] = {a, b, -1.0, -1.0, max(n_min, (int)ceil((double)n * (b - a) / (hi - lo)))};
    }
  }
  return k;
}

// Node j and weight of a piece (Gauss-Legendre of order q.m, sinh-graded towards a ridge end).
__device__ __forceinline__ void piece_node(const RPiece& q, int j, const double* __restrict__ gx,
                                           const double* __restrict__ gw, double& x, double& w) {
  const size_t o = (size_t)q.m * (q.m - 1) / 2;
  const double xj = gx[o + j], wj = gw[o + j];
  if (q.ha > 0.0 || q.hb > 0.0) {
    const double h = q.ha > 0.0 ? q.ha : q.hb;
    const double T = asinh((q.b - q.a) / h);
    const double tau = 0.5 * T * (xj + 1.0);
    const double off = h * sinh(tau);
    w = 0.5 * T * wj * h * cosh(tau);
    x = q.ha > 0.0 ? q.a + off : q.b - off;
  } else {
    x = 0.5 * (q.a + q.b) + 0.5 * (q.b - q.a) * xj;
    w = 0.5 * (q.b - q.a) * wj;
  }
}

// One island in one evaluation order: its channels, the coupling of the outer
// and inner variables, the knees, the ridges and the outer range.
struct RidgeIsland {
  double f, nu1, nu2, nu3, R1, R2, R3, be;
  double A, B, sg, c, C, ko, kt, ky;  // ordering (island_geom.cuh) and the knees of the outer, inner, third shape
  double lo, hi;                      // outer range (hi > lo: the island has area)
  double cc, alpha, hmax, us, vs;     // ridge scale 4 pi^2 |beta2 + 2 pi beta3 f|; ridges u = us, v = vs
  bool ridges;
};

template <int ORD>
__device__ __forceinline__ RidgeIsland ridge_island(const ChannelTable& ch, int coi, int n1, int n2, int n3,
                                                    double rolloff, double alpha, double beta2, double beta3) {
  RidgeIsland g;
  g.f = ch.nu_coi[coi];
  g.nu1 = ch.nu[n1];
  g.nu2 = ch.nu[n2];
  g.nu3 = ch.nu[n3];
  g.R1 = ch.R[n1];
  g.R2 = ch.R[n2];
  g.R3 = ch.R[n3];
  g.be = rolloff;
  const double d = (g.nu1 - g.f) + (g.nu2 - g.nu3);
  const double k1 = (1.0 - g.be) * g.R1 / 2.0, k2 = (1.0 - g.be) * g.R2 / 2.0, k3 = (1.0 - g.be) * g.R3 / 2.0;
  const double h1w = 0.5 * ch.W[n1], h2w = 0.5 * ch.W[n2], h3w = 0.5 * ch.W[n3];
  g.cc = 4.0 * kPi * kPi * fabs(beta2 + 2.0 * kPi * beta3 * g.f);
  g.alpha = alpha;
  g.ridges = g.cc > 0.0;
  g.us = g.f - g.nu1;
  g.vs = g.f - g.nu2;
  g.c = -d;
  if (ORD == ORD_DW) { g.A = h3w; g.B = h1w; g.sg = 1.0; g.C = h2w; g.ko = k3; g.kt = k1; g.ky = k2; }
  else if (ORD == ORD_E) { g.A = h2w; g.B = h1w; g.sg = -1.0; g.C = h3w; g.ko = k2; g.kt = k1; g.ky = k3; }
  else { g.A = h1w; g.B = h2w; g.sg = -1.0; g.C = h3w; g.ko = k1; g.kt = k2; g.ky = k3; }
  const double pp = g.sg * (-(g.B + g.C) - g.c), qq = g.sg * ((g.B + g.C) - g.c);
  g.lo = fmax(-g.A, fmin(pp, qq));
  g.hi = fmin(g.A, fmax(pp, qq));
  g.hmax = g.ridges ? g.alpha / (g.cc * fmax(h1w, h2w)) : -1.0;
  return g;
}

// The island's outer pieces (0 when it has no area).
template <int ORD>
__device__ int ridge_outer_pieces(const RidgeIsland& g, int n, int n_min, RPiece* out) {
  if (!(g.hi > g.lo)) return 0;
  RCut cuts[kOuterCuts];
  int nc = 0;
  cuts[nc++] = {-g.ko, -1.0};
  cuts[nc++] = {g.ko, -1.0};
  // inner break lines t = b0 (flat) and t = s o + b1 (slant); the ridge lines last
  double flat[5] = {-g.B, g.B, -g.kt, g.kt, 0.0}, slant[5] = {g.c - g.C, g.c + g.C, g.c - g.ky, g.c + g.ky, 0.0};
  int nfl = 4, nsl = 4;
  const bool rfl = g.ridges, rsl = g.ridges && ORD == ORD_DW;
  const double ridge_flat = ORD == ORD_F ? g.vs : g.us, ridge_slant = g.c - g.vs;
  if (rfl) flat[nfl++] = ridge_flat;
  if (rsl) slant[nsl++] = ridge_slant;
  for (int i = 0; i < nfl; ++i)
    for (int j = 0; j < nsl; ++j) {
      const bool both = rfl && rsl && flat[i] == ridge_flat && slant[j] == ridge_slant;
      cuts[nc++] = {(flat[i] - slant[j]) / g.sg, both ? g.hmax : -1.0};
    }
  if (g.ridges && ORD == ORD_E) cuts[nc++] = {g.vs, g.hmax};
  if (g.ridges && ORD == ORD_F) cuts[nc++] = {g.us, g.hmax};
  return ridge_pieces<kOuterCuts>(g.lo, g.hi, cuts, nc, n, n_min, out);
}

// The inner pieces of the row at outer node o (0 when its interval is empty);
// m_out = s o + c, the centre line of the coupling.
template <int ORD>
__device__ int ridge_inner_pieces(const RidgeIsland& g, double o, int n, int n_min, RPiece* out, double& m_out) {
  const double m = g.sg * o + g.c;
  m_out = m;
  const double tlo = fmax(-g.B, m - g.C), thi = fmin(g.B, m + g.C);
  if (!(thi > tlo)) return 0;
  RCut pts[kInnerCuts];
  int npt = 0;
  pts[npt++] = {-g.kt, -1.0};
  pts[npt++] = {g.kt, -1.0};
  pts[npt++] = {m - g.ky, -1.0};
  pts[npt++] = {m + g.ky, -1.0};
  if (g.ridges) {
    if (ORD == ORD_DW) {
      const double x2 = g.nu2 + (m - g.us) - g.f;  // f2 - f on the ridge f1 = f
      if (x2 != 0.0) pts[npt++] = {g.us, g.alpha / (g.cc * fabs(x2))};
      const double tr = m - g.vs;                  // the ridge f2 = f
      const double x1 = g.nu1 + tr - g.f;
      if (x1 != 0.0) pts[npt++] = {tr, g.alpha / (g.cc * fabs(x1))};
    } else if (ORD == ORD_E) {
      const double x2 = g.nu2 + o - g.f;
      if (x2 != 0.0) pts[npt++] = {g.us, g.alpha / (g.cc * fabs(x2))};
    } else {
      const double x1 = g.nu1 + o - g.f;
      if (x1 != 0.0) pts[npt++] = {g.vs, g.alpha / (g.cc * fabs(x1))};
    }
  }
  return ridge_pieces<kInnerCuts>(tlo, thi, pts, npt, n, n_min, out);
}

}  // namespace egn
