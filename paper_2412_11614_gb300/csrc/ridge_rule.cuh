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
// The cuts and pieces are FP64 (per island and per row); the FP32C kernel may take
// the ridge half-widths in FP32 (ridge_width).
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
// Pieces: one more than the cuts inside the range, plus one for every piece with
// a ridge at both ends (halved).  Ridge ends are the range ends and the ridge
// cuts, at most two of each, so kOuterCuts + 6 bounds the outer pieces; the
// inner bound keeps the full margin.  pieces_of_ends never writes past max_p.
constexpr int kOuterPieces = kOuterCuts + 6;
constexpr int kInnerPieces = 2 * (kInnerCuts + 1);

// A cut or piece end is a ridge when its half-width is positive (plain: -1).  The
// test reads the sign and magnitude bits as an integer: no FP64 comparison.
__device__ __forceinline__ bool is_ridge(double h) { return __double_as_longlong(h) > 0; }

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

// Nodes of a plain piece: max(n_min, ceil(n len / interval)).  The ratio is
// first formed in FP32 (relative error below 4e-7 on a value of at most 64, so
// within 3e-5 of the FP64 ratio) and its ceiling taken where it lies more than
// 1e-4 from an integer, where it is the ceiling of the FP64 ratio; otherwise
// (and where FP32 over- or underflows) the ratio is formed in FP64.  GB300 runs
// an FP64 division at a small fraction of the FP32 rate.
__device__ __forceinline__ int plain_nodes(double len, double interval, int n, int n_min) {
  const float r = (float)n * __fdividef((float)len, (float)interval);
  const float c = ceilf(r);
  if (c - r > 1e-4f && r - (c - 1.0f) > 1e-4f && c <= 128.0f) return max(n_min, (int)c);
  return max(n_min, (int)ceil((double)n * len / interval));
}

// Pieces between consecutive ends e[0..ne) of an interval of length len (at most
// max_p of them).
__device__ __forceinline__ int pieces_of_ends(const RCut* e, int ne, double len, int n, int n_min, RPiece* out,
                                              int max_p) {
  int k = 0;
  for (int i = 0; i + 1 < ne; ++i) {
    const double a = e[i].x, b = e[i + 1].x, ha = e[i].h, hb = e[i + 1].h;
    if (!(b > a)) continue;
    const bool ra = is_ridge(ha), rb = is_ridge(hb);
    if (k + (ra && rb ? 2 : 1) > max_p) break;
    if (ra && rb) {
      const double mid = 0.5 * (a + b);
      out[k++] = {a, mid, ha, -1.0, n};
      out[k++] = {mid, b, -1.0, hb, n};
    } else if (ra || rb) {
      out[k++] = {a, b, ha, hb, n};
    } else {
      out[k++] = {a, b, -1.0, -1.0, plain_nodes(b - a, len, n, n_min)};
    }
  }
  return k;
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
      if (is_ridge(cand[i].h)) e[ne - 1].h = cand[i].h;
      continue;
    }
    e[ne++] = cand[i];
  }
  e[ne++] = {hi, -1.0};
  for (int i = 0; i < np; ++i) {  // a ridge on an end of the interval
    if (!is_ridge(pts[i].h)) continue;
    if (fabs(pts[i].x - lo) <= eps) e[0].h = pts[i].h;
    if (fabs(pts[i].x - hi) <= eps) e[ne - 1].h = pts[i].h;
  }
  return pieces_of_ends(e, ne, hi - lo, n, n_min, out, 2 * (MAXC + 1));
}

// Node j and weight of a piece (Gauss-Legendre of order q.m, sinh-graded towards a ridge end).
__device__ __forceinline__ void piece_node(const RPiece& q, int j, const double* __restrict__ gx,
                                           const double* __restrict__ gw, double& x, double& w) {
  const size_t o = (size_t)q.m * (q.m - 1) / 2;
  const double xj = gx[o + j], wj = gw[o + j];
  const bool ra = is_ridge(q.ha);
  if (ra || is_ridge(q.hb)) {
    const double h = ra ? q.ha : q.hb;
    const double T = asinh((q.b - q.a) / h);
    const double tau = 0.5 * T * (xj + 1.0);
    const double off = h * sinh(tau);
    w = 0.5 * T * wj * h * cosh(tau);
    x = ra ? q.a + off : q.b - off;
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

// The island's outer pieces (none when it has no area), formed by one warp (all
// 32 lanes call it): the cuts are computed, filtered to the range and checked
// against its ends one per lane, so that the FP64 work one lane does alone is the
// sort and merge of the few cuts inside the range (ridge_pieces' steps in the
// same order, with the same result).
// Writes out[0..np) and cum[0..np] (node prefix: cum[np] outer nodes in all)
// and returns np on every lane.  sx, sh: kOuterCuts doubles of shared scratch.
template <int ORD>
__device__ int ridge_outer_pieces_warp(const RidgeIsland& g, int n, int n_min, RPiece* out, int* cum, double* sx,
                                       double* sh, int lane) {
  const bool area = g.hi > g.lo;
  const double eps = 1e-12;
  const bool rfl = g.ridges, rsl = g.ridges && ORD == ORD_DW;
  const int nfl = rfl ? 5 : 4, nsl = rsl ? 5 : 4, ncr = nfl * nsl;
  const int nc = 2 + ncr + (g.ridges && ORD != ORD_DW ? 1 : 0);
  const double ridge_flat = ORD == ORD_F ? g.vs : g.us, ridge_slant = g.c - g.vs;
  double x = 0.0, h = -1.0;
  if (lane < 2) {
    x = lane == 0 ? -g.ko : g.ko;
  } else if (lane < 2 + ncr) {  // crossing of inner break lines t = fl (flat) and t = s o + sl (slant)
    const int i = (lane - 2) / nsl, j = (lane - 2) - i * nsl;
    const double fl = i == 0 ? -g.B : (i == 1 ? g.B : (i == 2 ? -g.kt : (i == 3 ? g.kt : ridge_flat)));
    const double sl = j == 0 ? g.c - g.C : (j == 1 ? g.c + g.C : (j == 2 ? g.c - g.ky : (j == 3 ? g.c + g.ky : ridge_slant)));
    const bool both = rfl && rsl && fl == ridge_flat && sl == ridge_slant;
    x = (fl - sl) * g.sg;  // sg = +-1: the quotient by sg
    h = both ? g.hmax : -1.0;
  } else if (lane < nc) {  // the ridge of the outer variable (E: v = vs, F: u = us)
    x = ORD == ORD_E ? g.vs : g.us;
    h = g.hmax;
  }
  const bool valid = area && lane < nc;
  const bool in = valid && g.lo + eps < x && x < g.hi - eps;
  const unsigned min_ = __ballot_sync(0xffffffffu, in);
  if (in) {
    const int k = __popc(min_ & ((1u << lane) - 1u));  // cut order kept
    sx[k] = x;
    sh[k] = h;
  }
  // a ridge on an end of the range: the last such cut in cut order sets its width
  const bool rdg = valid && is_ridge(h);
  const unsigned mlo = __ballot_sync(0xffffffffu, rdg && fabs(x - g.lo) <= eps);
  const unsigned mhi = __ballot_sync(0xffffffffu, rdg && fabs(x - g.hi) <= eps);
  const double hlo = __shfl_sync(0xffffffffu, h, mlo ? 31 - __clz(mlo) : 0);
  const double hhi = __shfl_sync(0xffffffffu, h, mhi ? 31 - __clz(mhi) : 0);
  __syncwarp();
  if (lane == 0) {
    int np = 0;
    if (area) {
      RCut cand[kOuterCuts];
      const int nin = __popc(min_);
      for (int i = 0; i < nin; ++i) cand[i] = {sx[i], sh[i]};
      sort_cuts(cand, nin);
      RCut e[kOuterCuts + 2];
      int ne = 0;
      e[ne++] = {g.lo, mlo ? hlo : -1.0};
      for (int i = 0; i < nin; ++i) {
        if (ne > 1 && cand[i].x - e[ne - 1].x < eps) {
          if (is_ridge(cand[i].h)) e[ne - 1].h = cand[i].h;
          continue;
        }
        e[ne++] = cand[i];
      }
      e[ne++] = {g.hi, mhi ? hhi : -1.0};
      np = pieces_of_ends(e, ne, g.hi - g.lo, n, n_min, out, kOuterPieces);
    }
    int c = 0;
    for (int q = 0; q < np; ++q) {
      cum[q] = c;
      c += out[q].m;
    }
    cum[np] = c;
    sx[0] = (double)np;  // broadcast through the scratch
  }
  __syncwarp();
  const int np = (int)sx[0];
  __syncwarp();  // the scratch may be rewritten by the next island
  return np;
}

// Ridge half-width alpha / (cc |x|) at a point whose other frequency lies x from
// the COI: FP64, or FP32 with FAST (the half-width only scales the grading).
template <bool FAST>
__device__ __forceinline__ double ridge_width(const RidgeIsland& g, double x) {
  if (FAST) return (double)__fdividef((float)g.alpha, (float)g.cc * fabsf((float)x));
  return g.alpha / (g.cc * fabs(x));
}

// The inner pieces of the row at outer node o (0 when its interval is empty);
// m_out = s o + c, the centre line of the coupling.  FAST: the half-widths in
// FP32 (ridge_width).
template <int ORD, bool FAST = false>
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
      if (x2 != 0.0) pts[npt++] = {g.us, ridge_width<FAST>(g, x2)};
      const double tr = m - g.vs;                  // the ridge f2 = f
      const double x1 = g.nu1 + tr - g.f;
      if (x1 != 0.0) pts[npt++] = {tr, ridge_width<FAST>(g, x1)};
    } else if (ORD == ORD_E) {
      const double x2 = g.nu2 + o - g.f;
      if (x2 != 0.0) pts[npt++] = {g.us, ridge_width<FAST>(g, x2)};
    } else {
      const double x1 = g.nu1 + o - g.f;
      if (x1 != 0.0) pts[npt++] = {g.vs, ridge_width<FAST>(g, x1)};
    }
  }
  return ridge_pieces<kInnerCuts>(tlo, thi, pts, npt, n, n_min, out);
}

}  // namespace egn
