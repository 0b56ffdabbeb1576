// integrate_fp64.cu -- the plain FP64 island integrators (the precision baseline),
// with the configured Gauss-Legendre rule and with the ridge-resolving rule.
//
// One warp per island, one lane per outer node ("row"); every lane walks the n
// inner nodes of its row.  Per quadrature point (f1, f2) at the COI centre f:
//   chi    = 4 pi^2 (f1 - f)(f2 - f) [beta2 + pi beta3 (f1 + f2)]         (Eq. 5, 24)
//   w      = e^{(i chi - alpha) L/K}
//   mu     = (w - 1)/(i chi - alpha) * sum_k c_k w^k,                       (Eq. 8-10)
//            c_k = C_k e^{-zeta_k f3}, the k-th midpoint SRS gain (Eq. 14),
//            summed by the second-order real recurrence (Goertzel's) from
//            k = K - 1 down to 0
//   Y      = gamma mu e^{i (N-1) phi/2} sin(N phi/2) / sin(phi/2), phi = chi L   (Eq. 22)
// The segment form is Eq. 8 exactly: I_k = w^k (w - 1)/(i chi - alpha).  Phases
// are reduced in turns (chi L/K / 2 pi and chi L / 2 pi modulo 1) before
// sincospi.  In the DW order f3 is constant along a row, so the row's c_k are
// tabulated once in shared memory; the E and F orders evaluate them per point.
#include "egn_internal.h"
#include "island_geom.cuh"
#include "ridge_rule.cuh"

namespace egn {
namespace {

struct Cd {
  double re, im;
};

__device__ __forceinline__ Cd cmul(Cd a, Cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// sum_k c_k w^k (k = 0 .. K-1, real c_k = ck(k), |w|^2 = r2) by the second-order
// real recurrence b_k = c_k + 2 Re(w) b_{k+1} - |w|^2 b_{k+2} from b_K = b_{K+1} = 0,
// then sum = b_0 - conj(w) b_1: two FMAs per segment instead of a complex product.
template <class C>
__device__ __forceinline__ Cd segment_sum(Cd w, double r2, int K, C&& ck) {
  const double p2 = 2.0 * w.re;
  double b1 = 0.0, b2 = 0.0;
  for (int k = K - 1; k >= 0; --k) {
    const double b0 = fma(p2, b1, fma(-r2, b2, ck(k)));
    b2 = b1;
    b1 = b0;
  }
  return {b1 - w.re * b2, w.im * b2};
}

// (e^{(i chi - a) L} - 1) / (i chi - a) with the span phase chi L given in turns
// reduced modulo 1 (tp), so that a large chi L loses no accuracy.
__device__ __forceinline__ Cd lossy_closed_form(double chi, double a, double L, double tp) {
  double s, c;
  sincospi(2.0 * tp, &s, &c);
  const double e = exp(-a * L);
  const double xr = e * c - 1.0, xi = e * s;
  const double den = a * a + chi * chi;
  // (x)(-a - i chi) / (a^2 + chi^2)
  return {(-a * xr + chi * xi) / den, (-chi * xr - a * xi) / den};
}

// Maclaurin closed form, Eq. 4-6: first order in e^{-zeta f} and second order in
// the sinh normalisation of Eq. 25 give
//   mu = eta_1 - (P_tot Cr f3 / alpha) (eta_1 - eta_2),
//   eta_m = (e^{(i chi - m alpha) L} - 1) / (i chi - m alpha).
__device__ __forceinline__ Cd mu_maclaurin(double chi, double f3, double alpha, double L, double pcr, double tp) {
  const Cd e1 = lossy_closed_form(chi, alpha, L, tp);
  const Cd e2 = lossy_closed_form(chi, 2.0 * alpha, L, tp);
  const double k = pcr * f3 / alpha;
  return {e1.re - k * (e1.re - e2.re), e1.im - k * (e1.im - e2.im)};
}

// Normalised ISRS power profile rho(z, f3) of Eq. 25 (with Eq. 14).
__device__ __forceinline__ double rho_isrs(double z, double f3, double alpha, double pcr, double btot) {
  const double zeta = pcr * (-expm1(-alpha * z) / alpha);
  const double x = btot * zeta;
  const double g = (x == 0.0) ? 1.0 : x * exp(-zeta * f3) / (2.0 * sinh(0.5 * x));
  return g * exp(-alpha * z);
}

// Integral form, Eq. 23: mu = int_0^L rho(z, f3) e^{i chi z} dz by Gauss-Legendre
// (order kMuGl) on npieces equal pieces, each at most a quarter period
// pi / (2 |chi|) of the phase factor long.  Phases are taken in turns, chi z /
// 2 pi, reduced modulo 1.
__device__ __forceinline__ Cd mu_integral(const LinkParams& p, double chi, double f3, double alpha, double L,
                                          double pcr) {
  const double quarter = (chi != 0.0) ? kPi / (2.0 * fabs(chi)) : L;
  long long np = (long long)ceil(L / quarter);
  if (np < 1) np = 1;
  const double h = L / (double)np, hh = 0.5 * h;
  const double cturn = chi / (2.0 * kPi);
  Cd sum = {0.0, 0.0};
  for (long long q = 0; q < np; ++q) {
    const double m = ((double)q + 0.5) * h;
    Cd ps = {0.0, 0.0};
    for (int j = 0; j < kMuGl; ++j) {
      const double z = m + hh * p.mgx[j];
      double t = cturn * z;
      t -= rint(t);
      double s, c;
      sincospi(2.0 * t, &s, &c);
      const double v = p.mgw[j] * rho_isrs(z, f3, alpha, pcr, p.btot);
      ps.re += v * c;
      ps.im += v * s;
    }
    sum.re += ps.re;
    sum.im += ps.im;
  }
  return {sum.re * hh, sum.im * hh};
}

// Upsilon at one point.  Segment form: ck points at this row's c_k (stride
// ck_stride) or is null, in which case c_k is formed from f3 on the fly.  The
// Maclaurin and integral forms use f3 directly.
__device__ __forceinline__ Cd upsilon_fp64(const LinkParams& p, double f1, double f2, double f, const double* ck,
                                           int ck_stride, double f3, double* af2_out, bool need_phase) {
  const int K = p.seg.K;
  double a = f1 - f, b = f2 - f;
  double bc = p.beta2 + kPi * p.beta3 * (f1 + f2);
  double chi = 4.0 * kPi * kPi * a * b * bc;
  // span phase chi L in turns (phased array, closed forms)
  double tp = chi * (p.L / (2.0 * kPi));
  tp -= rint(tp);
  Cd mu;
  if (p.mu_form == MU_MACLAURIN) {
    mu = mu_maclaurin(chi, f3, p.alpha, p.L, p.types[0].pcr, tp);
  } else if (p.mu_form == MU_INTEGRAL) {
    mu = mu_integral(p, chi, f3, p.alpha, p.L, p.types[0].pcr);
  } else {
    double tt = chi * (p.dz / (2.0 * kPi));
    tt -= rint(tt);
    double s, c;
    sincospi(2.0 * tt, &s, &c);
    Cd w = {p.r * c, p.r * s};
    const double r2 = p.r * p.r;
    Cd acc;
    if (ck) acc = segment_sum(w, r2, K, [&](int k) { return ck[k * ck_stride]; });
    else acc = segment_sum(w, r2, K, [&](int k) { return p.seg.ck[k] * exp(-p.seg.zeta[k] * f3); });
    // (w - 1)/(i chi - alpha) = (w - 1)(-alpha - i chi)/(alpha^2 + chi^2)
    double xr = w.re - 1.0, xi = w.im;
    double den = p.alpha * p.alpha + chi * chi;
    Cd q = {(-p.alpha * xr + chi * xi) / den, (-chi * xr - p.alpha * xi) / den};
    mu = cmul(acc, q);
  }
  // phased array of N identical spans
  double N = (double)p.n_spans;
  double ratio = (tp == 0.0) ? N : sinpi(N * tp) / sinpi(tp);
  *af2_out = ratio * ratio;
  if (!need_phase) return mu;
  double sp, cp;
  sincospi((N - 1.0) * tp, &sp, &cp);
  Cd y = cmul(mu, Cd{cp, sp});
  double g = p.gamma * ratio;
  return {g * y.re, g * y.im};
}

// gamma_t mu_t and e^{i phi_t} (phi_t = chi_t L_t) of span type t at one point.
// ck: this row's c_k of type t (stride 32) or null (c_k formed from f3).
__device__ __forceinline__ void type_mu(const LinkParams& p, const SpanType& ty, double a, double b, double f1,
                                        double f2, const double* ck, double f3, Cd& gmu, Cd& eph) {
  const double chi = 4.0 * kPi * kPi * a * b * (ty.beta2 + kPi * ty.beta3 * (f1 + f2));
  double tp = chi * (ty.L / (2.0 * kPi));
  tp -= rint(tp);
  double s, c;
  Cd m;
  if (p.mu_form == MU_MACLAURIN) {
    m = mu_maclaurin(chi, f3, ty.alpha, ty.L, ty.pcr, tp);
  } else if (p.mu_form == MU_INTEGRAL) {
    m = mu_integral(p, chi, f3, ty.alpha, ty.L, ty.pcr);
  } else {
    double tt = chi * (ty.dz / (2.0 * kPi));
    tt -= rint(tt);
    sincospi(2.0 * tt, &s, &c);
    const Cd w = {ty.r * c, ty.r * s};
    const Cd acc = segment_sum(w, ty.r * ty.r, ty.seg.K,
                               [&](int k) { return ck ? ck[k * 32] : ty.seg.ck[k] * exp(-ty.seg.zeta[k] * f3); });
    const double xr = w.re - 1.0, xi = w.im;
    const double den = ty.alpha * ty.alpha + chi * chi;
    const Cd q = {(-ty.alpha * xr + chi * xi) / den, (-chi * xr - ty.alpha * xi) / den};
    m = cmul(acc, q);
  }
  gmu = {ty.gamma * m.re, ty.gamma * m.im};
  sincospi(2.0 * tp, &s, &c);
  eph = {c, s};
}

// Upsilon of a link whose spans differ (Eq. 22 written out): mu_t and the span
// phase phi_t = chi_t L_t of every span type t, then the coherent sum
// Y = sum_s gamma_{t(s)} mu_{t(s)} e^{i Phi_s}, Phi_{s+1} = Phi_s + phi_{t(s)}.
// Up to kMaxTypes types: each type once per point, ck the row tables (stride
// 32, type t at offset koff[t]) or null.  More types: span by span, c_k formed
// on the fly, a type's mu reused while consecutive spans share it.
__device__ __forceinline__ Cd upsilon_fp64_general(const LinkParams& p, double f1, double f2, double f,
                                                   const double* ck, const int* koff, double f3) {
  const double a = f1 - f, b = f2 - f;
  Cd z = {1.0, 0.0}, Y = {0.0, 0.0};
  if (p.n_types > kMaxTypes) {
    Cd m = {0.0, 0.0}, e = {1.0, 0.0};
    int prev = -1;
    for (int sp = 0; sp < p.n_spans; ++sp) {
      const int t = p.span_type[sp];
      if (t != prev) type_mu(p, p.types_dev[t], a, b, f1, f2, nullptr, f3, m, e);
      prev = t;
      const Cd v = cmul(m, z);
      Y.re += v.re;
      Y.im += v.im;
      z = cmul(z, e);
    }
    return Y;
  }
  Cd mu[kMaxTypes], ph[kMaxTypes];
  for (int t = 0; t < p.n_types; ++t) type_mu(p, p.types[t], a, b, f1, f2, ck ? ck + koff[t] * 32 : nullptr, f3, mu[t], ph[t]);
  for (int sp = 0; sp < p.n_spans; ++sp) {
    const int t = p.span_type[sp];
    const Cd v = cmul(mu[t], z);
    Y.re += v.re;
    Y.im += v.im;
    z = cmul(z, ph[t]);
  }
  return Y;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ORD_DW: D, G, H.  ORD_E / ORD_F: E / F.  `list` maps work items to island
// indices (null: item i is island i).
template <int ORD>
__global__ void __launch_bounds__(32) integrate_fp64_kernel(LinkParams p, const uint64_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ list, long long n_items,
                                                            double* __restrict__ terms, long long n_isl) {
  extern __shared__ double ck_s[];  // [K][32] (DW order only); general links: types one after the other
  const int lane = threadIdx.x;
  // c_k row tables of up to kMaxTypes span types (more types form c_k on the fly)
  const bool tables = p.n_types <= kMaxTypes && p.mu_form == MU_SEGMENT;
  int koff[kMaxTypes];
  for (int t = 0, o = 0; t < kMaxTypes; ++t) {
    koff[t] = o;
    if (t < p.n_types && tables) o += p.types[t].seg.K;
  }
  const ChannelTable& ch = p.ch;
  const int n = p.gl.n;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    double nu = ch.nu_coi[coi], nu1 = ch.nu[n1], nu2 = ch.nu[n2], nu3 = ch.nu[n3];
    double R = ch.R[coi], R1 = ch.R[n1], R2 = ch.R[n2], R3 = ch.R[n3];
    double d = (nu1 - nu) + (nu2 - nu3);
    Ordering g = make_ordering(ORD, ch.W[n1], ch.W[n2], ch.W[n3], d);
    double e[4];
    int np = outer_panels(g, e);
    bool want_g = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_g(n1, n2, n3)));
    bool want_h = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_h(n1, n2, n3)));
    double dsum = 0.0, csum = 0.0;
    Cd hsum = {0.0, 0.0};
    if (np > 0) {
      const int no = p.gl.order[np];
      const double* ox = p.gl.x[np];
      const double* ow = p.gl.w[np];
      const double* ix = p.gl.x[1];
      const double* iw = p.gl.w[1];
      const int rows = np * no;
      for (int base = 0; base < rows; base += 32) {
        const int row = base + lane;
        const bool active = row < rows;
        int pi = active ? row / no : 0, i = active ? row % no : 0;
        double pm = 0.5 * (e[pi] + e[pi + 1]), ph = 0.5 * (e[pi + 1] - e[pi]);
        double o = pm + ph * ox[i];
        double wo = ph * ow[i];
        double lo, hi;
        inner_limits(g, o, lo, hi);
        double im = 0.5 * (lo + hi), ih = 0.5 * (hi - lo);
        const double* ckrow = nullptr;
        double outer_h;
        if (ORD == ORD_DW) {
          double f3 = nu3 + o;
          if (active && tables) {
            if (p.n_types == 1) {
              for (int k = 0; k < p.seg.K; ++k) ck_s[k * 32 + lane] = p.seg.ck[k] * exp(-p.seg.zeta[k] * f3);
            } else {
              for (int t = 0; t < p.n_types; ++t)
                for (int k = 0; k < p.types[t].seg.K; ++k)
                  ck_s[(koff[t] + k) * 32 + lane] = p.types[t].seg.ck[k] * exp(-p.types[t].seg.zeta[k] * f3);
            }
          }
          ckrow = ck_s + lane;
          outer_h = rc_shape(o, R3, p.rolloff);
        } else if (ORD == ORD_E) {
          outer_h = rc_shape(o, R2, p.rolloff);
        } else {
          outer_h = rc_shape(o, R1, p.rolloff);
        }
        Cd inner = {0.0, 0.0};
        if (active) {
          for (int j = 0; j < n; ++j) {
            double t = im + ih * ix[j];
            double wi = ih * iw[j];
            double u, v, w;
            if (ORD == ORD_DW) { w = o; u = t; v = w - u - d; }
            else if (ORD == ORD_E) { v = o; u = t; w = u + v + d; }
            else { u = o; v = t; w = u + v + d; }
            double h1 = rc_shape(u, R1, p.rolloff), h2 = rc_shape(v, R2, p.rolloff), h3 = rc_shape(w, R3, p.rolloff);
            double f1 = nu1 + u, f2 = nu2 + v;
            double af2;
            if (p.n_types == 1 && ORD == ORD_DW && !want_g && !want_h) {
              Cd mu = upsilon_fp64(p, f1, f2, nu, ckrow, 32, nu3 + w, &af2, false);
              double y2 = p.gamma * p.gamma * (mu.re * mu.re + mu.im * mu.im) * af2;
              dsum += wo * wi * h1 * h2 * h3 * y2;
            } else {
              Cd Y = p.n_types == 1 ? upsilon_fp64(p, f1, f2, nu, ckrow, 32, nu3 + w, &af2, true)
                                    : upsilon_fp64_general(p, f1, f2, nu, (ORD == ORD_DW && tables) ? ck_s + lane : nullptr,
                                                           koff, nu3 + w);
              if (ORD == ORD_DW) {
                dsum += wo * wi * h1 * h2 * h3 * (Y.re * Y.re + Y.im * Y.im);
                double a12 = wi * sqrt(h1 * h2);
                inner.re += a12 * Y.re;
                inner.im += a12 * Y.im;
                double a123 = wo * wi * sqrt(h1 * h2 * h3);
                hsum.re += a123 * Y.re;
                hsum.im += a123 * Y.im;
              } else {
                double a = wi * (ORD == ORD_E ? sqrt(h1 * h3) : sqrt(h2 * h3));
                inner.re += a * Y.re;
                inner.im += a * Y.im;
              }
            }
          }
          csum += wo * outer_h * (inner.re * inner.re + inner.im * inner.im);
        }
      }
    }
    dsum = warp_sum(dsum);
    csum = warp_sum(csum);
    hsum.re = warp_sum(hsum.re);
    hsum.im = warp_sum(hsum.im);
    if (lane == 0) {
      double cf[5];
      term_coefs(R, R1, R2, R3, cf);
      if (ORD == ORD_DW) {
        terms[isl] = cf[0] * dsum;
        if (want_g) terms[3 * n_isl + isl] = cf[3] * csum;
        if (want_h) terms[4 * n_isl + isl] = cf[4] * (hsum.re * hsum.re + hsum.im * hsum.im);
      } else if (ORD == ORD_E) {
        terms[1 * n_isl + isl] = cf[1] * csum;
      } else {
        terms[2 * n_isl + isl] = cf[2] * csum;
      }
    }
    __syncwarp();
  }
}

// one warp per island as in the configured rule: the warp forms the outer pieces,
// one warp per island as in the configured rule: lane 0 forms the outer pieces,
// every lane then takes outer nodes ("rows") and walks its row's inner pieces.
template <int ORD>
__global__ void __launch_bounds__(32) integrate_ridge_kernel(LinkParams p, const uint64_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ list, long long n_items,
                                                             double* __restrict__ terms, long long n_isl) {
  extern __shared__ double ck_s[];  // [K][32] c_k row tables (DW order), as in the configured rule
  __shared__ RPiece opc[kOuterPieces];
  __shared__ int ocum[kOuterPieces + 1];
  __shared__ double osx[kOuterCuts], osh[kOuterCuts];  // scratch of ridge_outer_pieces_warp
  const int lane = threadIdx.x;
  const bool tables = p.n_types <= kMaxTypes && p.mu_form == MU_SEGMENT;
  int koff[kMaxTypes];
  for (int t = 0, o = 0; t < kMaxTypes; ++t) {
    koff[t] = o;
    if (t < p.n_types && tables) o += p.types[t].seg.K;
  }
  const ChannelTable& ch = p.ch;
  const int n = p.gl.n, n_min = p.ridge_n_min;
  const double be = p.rolloff;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    const RidgeIsland g = ridge_island<ORD>(ch, coi, n1, n2, n3, p.rolloff, p.alpha, p.beta2, p.beta3);
    const double f = g.f, nu1 = g.nu1, nu2 = g.nu2, nu3 = g.nu3;
    const double R = ch.R[coi], R1 = g.R1, R2 = g.R2, R3 = g.R3;
    const int npc = ridge_outer_pieces_warp<ORD>(g, n, n_min, opc, ocum, osx, osh, lane);
    const int rows = ocum[npc];
    const bool want_g = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_g(n1, n2, n3)));
    const bool want_h = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_h(n1, n2, n3)));
    double dsum = 0.0, csum = 0.0;
    Cd hsum = {0.0, 0.0};
    for (int base = 0; base < rows; base += 32) {
      const int row = base + lane;
      if (row >= rows) continue;
      int q = 0;
      while (ocum[q + 1] <= row) ++q;
      double o, wo;
      piece_node(opc[q], row - ocum[q], p.glx_all, p.glw_all, o, wo);
      double m;
      RPiece ipc[kInnerPieces];
      const int nip = ridge_inner_pieces<ORD>(g, o, n, n_min, ipc, m);
      if (nip == 0) continue;
      double outer_h;
      if (ORD == ORD_DW) {
        const double f3 = nu3 + o;
        if (tables) {
          if (p.n_types == 1) {
            for (int k = 0; k < p.seg.K; ++k) ck_s[k * 32 + lane] = p.seg.ck[k] * exp(-p.seg.zeta[k] * f3);
          } else {
            for (int t = 0; t < p.n_types; ++t)
              for (int k = 0; k < p.types[t].seg.K; ++k)
                ck_s[(koff[t] + k) * 32 + lane] = p.types[t].seg.ck[k] * exp(-p.types[t].seg.zeta[k] * f3);
          }
        }
        outer_h = rc_shape(o, R3, be);
      } else if (ORD == ORD_E) {
        outer_h = rc_shape(o, R2, be);
      } else {
        outer_h = rc_shape(o, R1, be);
      }
      const double* ckrow = (ORD == ORD_DW && tables) ? ck_s + lane : nullptr;
      Cd inner = {0.0, 0.0};
      for (int ip = 0; ip < nip; ++ip) {
        for (int j = 0; j < ipc[ip].m; ++j) {
          double t, wi;
          piece_node(ipc[ip], j, p.glx_all, p.glw_all, t, wi);
          double u, v, w;
          if (ORD == ORD_DW) { u = t; v = m - t; w = o; }
          else if (ORD == ORD_E) { u = t; v = o; w = t - m; }
          else { u = o; v = t; w = t - m; }
          const double h1 = rc_shape(u, R1, be), h2 = rc_shape(v, R2, be), h3 = rc_shape(w, R3, be);
          const double f1 = nu1 + u, f2 = nu2 + v;
          double af2;
          if (p.n_types == 1 && ORD == ORD_DW && !want_g && !want_h) {
            const Cd mu = upsilon_fp64(p, f1, f2, f, ckrow, 32, nu3 + w, &af2, false);
            dsum += wo * wi * h1 * h2 * h3 * (p.gamma * p.gamma * (mu.re * mu.re + mu.im * mu.im) * af2);
          } else {
            const Cd Y = p.n_types == 1 ? upsilon_fp64(p, f1, f2, f, ckrow, 32, nu3 + w, &af2, true)
                                        : upsilon_fp64_general(p, f1, f2, f, ckrow, koff, nu3 + w);
            if (ORD == ORD_DW) {
              dsum += wo * wi * h1 * h2 * h3 * (Y.re * Y.re + Y.im * Y.im);
              const double a12 = wi * sqrt(h1 * h2);
              inner.re += a12 * Y.re;
              inner.im += a12 * Y.im;
              const double a123 = wo * wi * sqrt(h1 * h2 * h3);
              hsum.re += a123 * Y.re;
              hsum.im += a123 * Y.im;
            } else {
              const double a = wi * (ORD == ORD_E ? sqrt(h1 * h3) : sqrt(h2 * h3));
              inner.re += a * Y.re;
              inner.im += a * Y.im;
            }
          }
        }
      }
      csum += wo * outer_h * (inner.re * inner.re + inner.im * inner.im);
    }
    dsum = warp_sum(dsum);
    csum = warp_sum(csum);
    hsum.re = warp_sum(hsum.re);
    hsum.im = warp_sum(hsum.im);
    if (lane == 0) {
      double cf[5];
      term_coefs(R, R1, R2, R3, cf);
      if (ORD == ORD_DW) {
        terms[isl] = cf[0] * dsum;
        if (want_g) terms[3 * n_isl + isl] = cf[3] * csum;
        if (want_h) terms[4 * n_isl + isl] = cf[4] * (hsum.re * hsum.re + hsum.im * hsum.im);
      } else if (ORD == ORD_E) {
        terms[1 * n_isl + isl] = cf[1] * csum;
      } else {
        terms[2 * n_isl + isl] = cf[2] * csum;
      }
    }
    __syncwarp();  // the outer pieces are rewritten for the next island
  }
}

template <int ORD>
cudaError_t launch_ridge(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                         double* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  int ksum = 0;
  if (p.mu_form == MU_SEGMENT && p.n_types <= kMaxTypes)
    for (int t = 0; t < p.n_types; ++t) ksum += p.n_types == 1 ? p.seg.K : p.types[t].seg.K;
  const size_t smem = (ORD == ORD_DW) ? (size_t)ksum * 32 * sizeof(double) : 0;
  static std::atomic<unsigned long long> attr_done{0};  // per device
  if (smem > 40 * 1024)
    if (cudaError_t e = opt_in_smem(integrate_ridge_kernel<ORD>, (int)(kMaxK * 32 * sizeof(double)), attr_done)) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (long long)sms * 32;
  if (blocks > n_items) blocks = n_items;
  integrate_ridge_kernel<ORD><<<(unsigned)blocks, 32, smem, st>>>(p, keys, list, n_items, terms, n_isl);
  return cudaGetLastError();
}

template <int ORD>
cudaError_t launch_one(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                       double* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  int ksum = p.mu_form == MU_SEGMENT ? p.seg.K : 0;
  if (p.n_types > 1) {
    ksum = 0;
    if (p.n_types <= kMaxTypes && p.mu_form == MU_SEGMENT)
      for (int t = 0; t < p.n_types; ++t) ksum += p.types[t].seg.K;
  }
  size_t smem = (ORD == ORD_DW) ? (size_t)ksum * 32 * sizeof(double) : 0;
  static std::atomic<unsigned long long> attr_done{0};  // per device
  if (smem > 48 * 1024)
    if (cudaError_t e = opt_in_smem(integrate_fp64_kernel<ORD>, (int)(kMaxK * 32 * sizeof(double)), attr_done)) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (long long)sms * 32;
  if (blocks > n_items) blocks = n_items;
  integrate_fp64_kernel<ORD><<<(unsigned)blocks, 32, smem, st>>>(p, keys, list, n_items, terms, n_isl);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp64_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                             long long n_items, double* terms, long long n_isl, cudaStream_t st) {
  if (p.rule == RULE_RIDGE) {
    if (ord == ORD_DW) return launch_ridge<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
    if (ord == ORD_E) return launch_ridge<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
    return launch_ridge<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (ord == ORD_DW) return launch_one<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
  if (ord == ORD_E) return launch_one<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
  return launch_one<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
}

}  // namespace egn
