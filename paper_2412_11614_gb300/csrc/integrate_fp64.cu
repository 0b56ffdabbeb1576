// integrate_fp64.cu -- the plain FP64 island integrator (the precision baseline).
//
// One warp per island, one lane per outer node ("row"); every lane walks the n
// inner nodes of its row.  Per quadrature point (f1, f2) at the COI centre f:
//   chi    = 4 pi^2 (f1 - f)(f2 - f) [beta2 + pi beta3 (f1 + f2)]         (Eq. 5, 24)
//   w      = e^{(i chi - alpha) L/K}
//   mu     = (w - 1)/(i chi - alpha) * sum_k c_k w^k,                       (Eq. 8-10)
//            c_k = C_k e^{-zeta_k f3}, the k-th midpoint SRS gain (Eq. 14),
//            summed by Horner's rule from k = K - 1 down to 0
//   Y      = gamma mu e^{i (N-1) phi/2} sin(N phi/2) / sin(phi/2), phi = chi L   (Eq. 22)
// The segment form is Eq. 8 exactly: I_k = w^k (w - 1)/(i chi - alpha).  Phases
// are reduced in turns (chi L/K / 2 pi and chi L / 2 pi modulo 1) before
// sincospi.  In the DW order f3 is constant along a row, so the row's c_k are
// tabulated once in shared memory; the E and F orders evaluate them per point.
#include "egn_internal.h"
#include "island_geom.cuh"

namespace egn {
namespace {

struct Cd {
  double re, im;
};

__device__ __forceinline__ Cd cmul(Cd a, Cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

// Upsilon at one point.  ck points at this row's c_k (stride ck_stride) or is
// null, in which case c_k is formed from f3 on the fly.
__device__ __forceinline__ Cd upsilon_fp64(const LinkParams& p, double f1, double f2, double f, const double* ck,
                                           int ck_stride, double f3, double* af2_out, bool need_phase) {
  const int K = p.seg.K;
  double a = f1 - f, b = f2 - f;
  double bc = p.beta2 + kPi * p.beta3 * (f1 + f2);
  double chi = 4.0 * kPi * kPi * a * b * bc;
  double tt = chi * (p.dz / (2.0 * kPi));
  tt -= rint(tt);
  double s, c;
  sincospi(2.0 * tt, &s, &c);
  Cd w = {p.r * c, p.r * s};
  Cd acc = {0.0, 0.0};
  if (ck) {
    for (int k = K - 1; k >= 0; --k) {
      acc = cmul(acc, w);
      acc.re += ck[k * ck_stride];
    }
  } else {
    for (int k = K - 1; k >= 0; --k) {
      acc = cmul(acc, w);
      acc.re += p.seg.ck[k] * exp(-p.seg.zeta[k] * f3);
    }
  }
  // (w - 1)/(i chi - alpha) = (w - 1)(-alpha - i chi)/(alpha^2 + chi^2)
  double xr = w.re - 1.0, xi = w.im;
  double den = p.alpha * p.alpha + chi * chi;
  Cd q = {(-p.alpha * xr + chi * xi) / den, (-chi * xr - p.alpha * xi) / den};
  Cd mu = cmul(acc, q);
  // phased array of N identical spans
  double tp = chi * (p.L / (2.0 * kPi));
  tp -= rint(tp);
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
  extern __shared__ double ck_s[];  // [K][32] (DW order only)
  const int lane = threadIdx.x;
  const ChannelTable& ch = p.ch;
  const int n = p.gl.n;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    double nu = ch.nu[coi], nu1 = ch.nu[n1], nu2 = ch.nu[n2], nu3 = ch.nu[n3];
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
          if (active)
            for (int k = 0; k < p.seg.K; ++k) ck_s[k * 32 + lane] = p.seg.ck[k] * exp(-p.seg.zeta[k] * f3);
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
            if (ORD == ORD_DW && !want_g && !want_h) {
              Cd mu = upsilon_fp64(p, f1, f2, nu, ckrow, 32, 0.0, &af2, false);
              double y2 = p.gamma * p.gamma * (mu.re * mu.re + mu.im * mu.im) * af2;
              dsum += wo * wi * h1 * h2 * h3 * y2;
            } else {
              Cd Y = upsilon_fp64(p, f1, f2, nu, ckrow, 32, nu3 + w, &af2, true);
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

template <int ORD>
cudaError_t launch_one(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                       double* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  size_t smem = (ORD == ORD_DW) ? (size_t)p.seg.K * 32 * sizeof(double) : 0;
  static bool attr_set[3] = {false, false, false};
  if (smem > 48 * 1024 && !attr_set[ORD]) {
    cudaError_t e = cudaFuncSetAttribute(integrate_fp64_kernel<ORD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kMaxK * 32 * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr_set[ORD] = true;
  }
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
  if (ord == ORD_DW) return launch_one<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
  if (ord == ORD_E) return launch_one<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
  return launch_one<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
}

}  // namespace egn
