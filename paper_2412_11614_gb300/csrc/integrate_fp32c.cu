// integrate_fp32c.cu -- FP32 island integrator with exact phase reduction (the
// fast path).
//
// Arithmetic per quadrature point, all FP32 except where stated:
//  * Phase.  Along a row (fixed outer node) the phase in turns of one span,
//      Theta(x) = chi L / 2 pi = 2 pi L (f1 - f)(f2 - f) [beta2 + pi beta3 (f1 + f2)],
//    is a cubic in the inner Gauss-Legendre coordinate x (Eq. 5, 24).  Its
//    coefficients Q0..Q3 are formed per row in FP64 and stored as FP32 head/tail
//    pairs (Q0 already reduced modulo K).  Per point, Q1 x and Q2 x^2 are formed as
//    exact FP32 products (head * head by FMA error-free product, plus the tail
//    cross terms), reduced modulo K exactly (the FMA residual p - K n is exact),
//    and summed with error-free two-sums.  The reduced phase gives both
//    theta = chi L/K (turns, modulo 1) for the segment factor and phi = chi L
//    (turns, modulo 1) for the phased array, each to ~1e-7 turns.
//  * Segment sum (Eq. 8-10).  mu = (w - 1)/(i chi - alpha) sum_k c_k w^k with
//    w = r e^{i theta} and real c_k = C_k e^{-zeta_k f3}.  For real coefficients the
//    polynomial is evaluated by the second-order real recurrence
//      b_k = c_k + p b_{k+1} - q b_{k+2},  p = 2 Re w, q = |w|^2,
//      sum_k c_k w^k = b_0 - conj(w) b_1,
//    an exact rewriting of Horner's rule (2 FMA per segment instead of 4); the
//    attenuation |w| < 1 bounds its rounding-error growth.
//  * Phased array (Eq. 22): |Y|^2 = gamma^2 |mu|^2 [sin(N pi phi)/sin(pi phi)]^2 with
//    sinpif/cospif of the reduced phase (limit N at phi = 0).
// In the DW order (D, G, H) f3 is constant along a row and the row's c_k are
// tabulated in shared memory; the E and F orders form c_k per point with ex2.
// Island sums are FP32 per thread, then fixed-order shuffle/shared-memory trees.
#include "egn_internal.h"
#include "island_geom.cuh"

namespace egn {
namespace {

constexpr int kThreads = 128;
constexpr int kP = 4;           // points per thread (same row)
constexpr int kRowsMax = 64;    // rows per chunk held in shared memory
constexpr int kTabFloats = 10240;  // DW c_k table budget (40 KB)

struct RowSm {
  float q0h[kRowsMax], q0l[kRowsMax], q1h[kRowsMax], q1l[kRowsMax], q2h[kRowsMax], q2l[kRowsMax], q3[kRowsMax];
  float a0[kRowsMax], a1[kRowsMax], b0[kRowsMax], b1[kRowsMax];  // f1 - f, f2 - f = a0 + a1 x, b0 + b1 x
  float bc0[kRowsMax], bc1[kRowsMax];                            // beta2 + pi beta3 (f1 + f2) = bc0 + bc1 x
  float im[kRowsMax], ih[kRowsMax];                              // inner variable = im + ih x
  float o[kRowsMax];                                             // outer variable
  float wrow[kRowsMax];                                          // outer weight x inner half-width
  float wo[kRowsMax];                                            // outer weight
  float hout[kRowsMax];                                          // shape of the outer variable's channel
  float f30[kRowsMax], f31[kRowsMax];                            // f3 = f30 + f31 x (E, F orders)
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Raised-cosine shape in FP32.
__device__ __forceinline__ float rc_f(float x, float R, float beta) {
  float ax = fabsf(x);
  float a = 0.5f * (1.0f - beta) * R, b = 0.5f * (1.0f + beta) * R;
  if (ax <= a) return 1.0f;
  if (ax >= b) return 0.0f;
  return 0.5f * (1.0f + cospif((ax - a) / (beta * R)));
}

template <int ORD>
__global__ void __launch_bounds__(kThreads) integrate_fp32c_kernel(LinkParams p, const uint64_t* __restrict__ keys,
                                                                   const uint32_t* __restrict__ list,
                                                                   long long n_items, float* __restrict__ terms,
                                                                   long long n_isl, int rows_per_chunk, int kpad) {
  __shared__ RowSm rs;
  __shared__ float red[5][kThreads / 32];
  extern __shared__ float tab[];  // [rows_per_chunk][kpad] (DW only)

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const ChannelTable& ch = p.ch;
  const int n = p.gl.n;
  const int K = p.seg.K;
  const float Kf = (float)K, invK = 1.0f / (float)K;
  const float beta = (float)p.rolloff;
  const float alpha = (float)p.alpha;
  const float r = (float)p.r;
  const float one_m_r = (float)(-expm1(-p.alpha * p.dz));
  const float q = r * r;
  const float N = (float)p.n_spans;
  const float gam = (float)p.gamma;
  const float k4 = (float)(4.0 * kPi * kPi);
  // threads per row (power of two) and the row owned by this thread
  int tpr = 1;
  while (tpr * kP < n) tpr <<= 1;
  const int rows_per_pass = kThreads / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;
  const double twopiL = 2.0 * kPi * p.L;
  const double invKd = 1.0 / (double)K;

  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    const double nu = ch.nu[coi], nu1 = ch.nu[n1], nu2 = ch.nu[n2], nu3 = ch.nu[n3];
    const double R = ch.R[coi], R1 = ch.R[n1], R2 = ch.R[n2], R3 = ch.R[n3];
    const double d = (nu1 - nu) + (nu2 - nu3);
    const Ordering g = make_ordering(ORD, ch.W[n1], ch.W[n2], ch.W[n3], d);
    double e[4];
    const int np = outer_panels(g, e);
    const bool want_g = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_g(n1, n2, n3)));
    const bool want_h = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_h(n1, n2, n3)));
    const bool cplx = ORD != ORD_DW || want_g || want_h;
    const float R1f = (float)R1, R2f = (float)R2, R3f = (float)R3;
    float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
    const int no = np > 0 ? p.gl.order[np] : 0;
    const int rows = np * no;
    for (int c0 = 0; c0 < rows; c0 += rows_per_chunk) {
      const int rc = min(rows_per_chunk, rows - c0);
      // ---- row constants (FP64), one thread per row, rows spread across warps
      for (int rr = tid; rr < rc; rr += kThreads) {
        int row = c0 + rr;
        int pi = row / no, i = row % no;
        double pm = 0.5 * (e[pi] + e[pi + 1]), ph = 0.5 * (e[pi + 1] - e[pi]);
        double o = pm + ph * p.gl.x[np][i];
        double wo = ph * p.gl.w[np][i];
        double lo, hi;
        inner_limits(g, o, lo, hi);
        double im = 0.5 * (lo + hi), ih = 0.5 * (hi - lo);
        // f1 - f = a0 + a1 x, f2 - f = b0 + b1 x, f1 + f2 = s0 + s1 x (frequencies relative to f_c)
        double a0, a1, b0, b1, s0, s1, f30, f31;
        if (ORD == ORD_DW) {        // w = o, u = im + ih x, v = w - u - d
          a0 = (nu1 - nu) + im; a1 = ih;
          b0 = (nu2 - nu) + (o - im - d); b1 = -ih;
          s0 = nu1 + nu2 + (o - d); s1 = 0.0;
          f30 = nu3 + o; f31 = 0.0;
        } else if (ORD == ORD_E) {  // v = o, u = im + ih x, w = u + v + d
          a0 = (nu1 - nu) + im; a1 = ih;
          b0 = (nu2 - nu) + o; b1 = 0.0;
          s0 = nu1 + nu2 + im + o; s1 = ih;
          f30 = nu3 + (im + o + d); f31 = ih;
        } else {                    // u = o, v = im + ih x, w = u + v + d
          a0 = (nu1 - nu) + o; a1 = 0.0;
          b0 = (nu2 - nu) + im; b1 = ih;
          s0 = nu1 + nu2 + o + im; s1 = ih;
          f30 = nu3 + (o + im + d); f31 = ih;
        }
        double g0 = twopiL * (p.beta2 + kPi * p.beta3 * s0), g1 = twopiL * kPi * p.beta3 * s1;
        double ab0 = a0 * b0, ab1 = a0 * b1 + a1 * b0, ab2 = a1 * b1;
        double Q0 = g0 * ab0, Q1 = g0 * ab1 + g1 * ab0, Q2 = g0 * ab2 + g1 * ab1, Q3 = g1 * ab2;
        Q0 = fma(-(double)K, rint(Q0 * invKd), Q0);
        float h;
        h = (float)Q0; rs.q0h[rr] = h; rs.q0l[rr] = (float)(Q0 - (double)h);
        h = (float)Q1; rs.q1h[rr] = h; rs.q1l[rr] = (float)(Q1 - (double)h);
        h = (float)Q2; rs.q2h[rr] = h; rs.q2l[rr] = (float)(Q2 - (double)h);
        rs.q3[rr] = (float)Q3;
        rs.a0[rr] = (float)a0; rs.a1[rr] = (float)a1;
        rs.b0[rr] = (float)b0; rs.b1[rr] = (float)b1;
        rs.bc0[rr] = (float)(p.beta2 + kPi * p.beta3 * s0);
        rs.bc1[rr] = (float)(kPi * p.beta3 * s1);
        rs.im[rr] = (float)im; rs.ih[rr] = (float)ih;
        rs.o[rr] = (float)o;
        rs.wrow[rr] = (float)(wo * ih);
        rs.wo[rr] = (float)wo;
        rs.f30[rr] = (float)f30; rs.f31[rr] = (float)f31;
        float of = (float)o;
        rs.hout[rr] = ORD == ORD_DW ? rc_f(of, R3f, beta) : (ORD == ORD_E ? rc_f(of, R2f, beta) : rc_f(of, R1f, beta));
      }
      __syncthreads();
      // ---- c_k tables of the chunk's rows (DW): C_k 2^{-zeta_k log2(e) f3}
      if (ORD == ORD_DW) {
        for (int idx = tid; idx < rc * K; idx += kThreads) {
          int rr = idx / K, k = idx - rr * K;
          tab[rr * kpad + k] = p.seg.ck_f[k] * exp2f(-p.seg.zeta_f[k] * rs.f30[rr]);
        }
        __syncthreads();
      }
      // ---- points
      for (int rb = 0; rb < rc; rb += rows_per_pass) {
        const int rr = rb + rsub;
        const bool row_ok = rr < rc;
        const int rrc = row_ok ? rr : 0;
        float gre = 0.0f, gim = 0.0f;  // G inner sum of this thread's points
        float p_[kP], b1_[kP], b2_[kP], f3_[kP];
        float wr_[kP], wi_[kP], chi_[kP], phi_[kP], wgt_[kP], s12_[kP], s123_[kP];
        bool ok_[kP];
        const float q0h = rs.q0h[rrc], q0l = rs.q0l[rrc], q1h = rs.q1h[rrc], q1l = rs.q1l[rrc];
        const float q2h = rs.q2h[rrc], q2l = rs.q2l[rrc], q3 = rs.q3[rrc];
        const float a0 = rs.a0[rrc], a1 = rs.a1[rrc], b0 = rs.b0[rrc], b1 = rs.b1[rrc];
        const float bc0 = rs.bc0[rrc], bc1 = rs.bc1[rrc], im = rs.im[rrc], ih = rs.ih[rrc], of = rs.o[rrc];
        const float wrow = rs.wrow[rrc], f30 = rs.f30[rrc], f31 = rs.f31[rrc];
#pragma unroll
        for (int m = 0; m < kP; ++m) {
          const int j = lr + tpr * m;
          ok_[m] = row_ok && j < n;
          const int jj = ok_[m] ? j : 0;
          const float xh = p.gl.xh[1][jj], xl = p.gl.xl[1][jj], x2h = p.gl.x2h[1][jj], x2l = p.gl.x2l[1][jj];
          // phase modulo K: Q0 + Q1 x + Q2 x^2 + Q3 x^3 with exact products and sums
          float p1 = q1h * xh, e1 = fmaf(q1h, xh, -p1);
          float t1 = fmaf(q1h, xl, fmaf(q1l, xh, e1));
          float p2 = q2h * x2h, e2 = fmaf(q2h, x2h, -p2);
          float t2 = fmaf(q2h, x2l, fmaf(q2l, x2h, e2));
          float r1 = fmaf(-Kf, rintf(p1 * invK), p1);
          float r2 = fmaf(-Kf, rintf(p2 * invK), p2);
          float s1, s2, ea, eb;
          two_sum(q0h, r1, s1, ea);
          two_sum(s1, r2, s2, eb);
          float tail = ((ea + eb) + (q0l + t1 + t2)) + q3 * (xh * x2h);
          float th = fmaf(s2, invK, tail * invK);
          th -= rintf(th);                        // theta in turns, [-1/2, 1/2)
          float ph = (s2 - rintf(s2)) + tail;     // phi in turns
          ph -= rintf(ph);
          // w = r e^{2 pi i th}: half-angle sines keep w - 1 accurate
          float sh, chh;
          sincospif(th, &sh, &chh);
          float wr = r * fmaf(-2.0f * sh, sh, 1.0f);
          float wi = 2.0f * r * sh * chh;
          p_[m] = 2.0f * wr;
          wr_[m] = -one_m_r - 2.0f * r * sh * sh;  // Re(w - 1)
          wi_[m] = wi;
          phi_[m] = ph;
          // chi [rad/km] for (i chi - alpha), from the factors in FP32
          float x = xh;
          float a = fmaf(a1, x, a0), b = fmaf(b1, x, b0), bc = fmaf(bc1, x, bc0);
          chi_[m] = k4 * a * b * bc;
          // spectral shapes and weights
          float t = fmaf(ih, x, im);
          float u, v, h3;
          if (ORD == ORD_DW) { u = t; v = of - t - (float)d; h3 = rs.hout[rrc]; }
          else {
            if (ORD == ORD_E) { v = of; u = t; } else { u = of; v = t; }
            h3 = rc_f(u + v + (float)d, R3f, beta);
          }
          float h1 = rc_f(u, R1f, beta), h2 = rc_f(v, R2f, beta);
          float wij = wrow * p.gl.wf[1][jj];
          wgt_[m] = ok_[m] ? wij * h1 * h2 * h3 : 0.0f;
          if (ORD == ORD_DW) {
            s12_[m] = ok_[m] ? p.gl.wf[1][jj] * sqrtf(h1 * h2) : 0.0f;  // G: inner weight x s1 s2
            s123_[m] = ok_[m] ? wij * sqrtf(h1 * h2 * h3) : 0.0f;        // H
          } else if (ORD == ORD_E) {
            s12_[m] = ok_[m] ? p.gl.wf[1][jj] * ih * sqrtf(h1 * h3) : 0.0f;
            s123_[m] = 0.0f;
          } else {
            s12_[m] = ok_[m] ? p.gl.wf[1][jj] * ih * sqrtf(h2 * h3) : 0.0f;
            s123_[m] = 0.0f;
          }
          f3_[m] = fmaf(f31, x, f30);
          b1_[m] = 0.0f;
          b2_[m] = 0.0f;
        }
        // ---- segment sum by the real recurrence, k = K-1 .. 0
        if (ORD == ORD_DW) {
          const float* trow = tab + rrc * kpad;
          int k = K - 1;
          // peel K mod 4 steps so that the float4 loads below start on 16-byte boundaries
          for (int s = 0; s < (K & 3); ++s, --k) {
            float c = trow[k];
#pragma unroll
            for (int m = 0; m < kP; ++m) {
              float bn = fmaf(p_[m], b1_[m], c);
              bn = fmaf(-q, b2_[m], bn);
              b2_[m] = b1_[m];
              b1_[m] = bn;
            }
          }
          for (; k >= 3; k -= 4) {
            float4 c4 = *reinterpret_cast<const float4*>(trow + k - 3);
            float cc[4] = {c4.w, c4.z, c4.y, c4.x};
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
              for (int m = 0; m < kP; ++m) {
                float bn = fmaf(p_[m], b1_[m], cc[s]);
                bn = fmaf(-q, b2_[m], bn);
                b2_[m] = b1_[m];
                b1_[m] = bn;
              }
          }
        } else {
          for (int k = K - 1; k >= 0; --k) {
            float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
#pragma unroll
            for (int m = 0; m < kP; ++m) {
              float c = ck * exp2f(-zk * f3_[m]);
              float bn = fmaf(p_[m], b1_[m], c);
              bn = fmaf(-q, b2_[m], bn);
              b2_[m] = b1_[m];
              b1_[m] = bn;
            }
          }
        }
        // ---- mu, Upsilon and the sums
#pragma unroll
        for (int m = 0; m < kP; ++m) {
          // after the loop b1 = b_0 and b2 = b_1
          float wr = 0.5f * p_[m], wi = wi_[m];
          float sre = fmaf(-wr, b2_[m], b1_[m]);  // b_0 - conj(w) b_1
          float sim = wi * b2_[m];
          // (w - 1)/(i chi - alpha) = (w - 1)(-alpha - i chi)/(alpha^2 + chi^2)
          float xr = wr_[m], xi = wi;
          float chi = chi_[m];
          float inv = 1.0f / fmaf(chi, chi, alpha * alpha);
          float qr = (fmaf(-alpha, xr, chi * xi)) * inv;
          float qi = (fmaf(-chi, xr, -alpha * xi)) * inv;
          float mre = sre * qr - sim * qi;
          float mim = fmaf(sre, qi, sim * qr);
          float ph = phi_[m];
          float ratio = (ph == 0.0f) ? N : sinpif(N * ph) / sinpif(ph);
          if (!cplx) {
            dsum = fmaf(wgt_[m], gam * gam * (mre * mre + mim * mim) * ratio * ratio, dsum);
          } else {
            float sp, cp;
            sincospif((N - 1.0f) * ph, &sp, &cp);
            float gr = gam * ratio;
            float yre = gr * (mre * cp - mim * sp);
            float yim = gr * fmaf(mre, sp, mim * cp);
            if (ORD == ORD_DW) {
              dsum = fmaf(wgt_[m], yre * yre + yim * yim, dsum);
              gre = fmaf(s12_[m], yre, gre);
              gim = fmaf(s12_[m], yim, gim);
              hre = fmaf(s123_[m], yre, hre);
              him = fmaf(s123_[m], yim, him);
            } else {
              gre = fmaf(s12_[m], yre, gre);
              gim = fmaf(s12_[m], yim, gim);
            }
          }
        }
        if (cplx && (ORD != ORD_DW || want_g)) {
          // complete the row's inner sum over its tpr threads, then |.|^2 x outer weight
          for (int o = tpr >> 1; o > 0; o >>= 1) {
            gre += __shfl_xor_sync(0xffffffffu, gre, o);
            gim += __shfl_xor_sync(0xffffffffu, gim, o);
          }
          if (lr == 0 && row_ok) {
            float wo = rs.wo[rrc];
            float ih_ = (ORD == ORD_DW) ? rs.ih[rrc] : 1.0f;
            float gr_ = gre * ih_, gi_ = gim * ih_;
            csum = fmaf(wo * rs.hout[rrc], gr_ * gr_ + gi_ * gi_, csum);
          }
        }
      }
      __syncthreads();  // rows and tables are rewritten by the next chunk
    }
    // ---- block reduction of dsum, csum, hre, him (fixed order)
    float vals[4] = {dsum, csum, hre, him};
#pragma unroll
    for (int a = 0; a < 4; ++a)
      for (int o = 16; o > 0; o >>= 1) vals[a] += __shfl_xor_sync(0xffffffffu, vals[a], o);
    if (lane == 0)
#pragma unroll
      for (int a = 0; a < 4; ++a) red[a][wid] = vals[a];
    __syncthreads();
    if (tid == 0) {
      float t[4];
      for (int a = 0; a < 4; ++a) {
        float s = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) s += red[a][w];
        t[a] = s;
      }
      double cf[5];
      term_coefs(R, R1, R2, R3, cf);
      if (ORD == ORD_DW) {
        terms[isl] = (float)(cf[0] * (double)t[0]);
        if (want_g) terms[3 * n_isl + isl] = (float)(cf[3] * (double)t[1]);
        if (want_h) terms[4 * n_isl + isl] = (float)(cf[4] * ((double)t[2] * t[2] + (double)t[3] * t[3]));
      } else if (ORD == ORD_E) {
        terms[1 * n_isl + isl] = (float)(cf[1] * (double)t[1]);
      } else {
        terms[2 * n_isl + isl] = (float)(cf[2] * (double)t[1]);
      }
    }
    __syncthreads();
  }
}

template <int ORD>
cudaError_t launch_one(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items, float* terms,
                       long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const int K = p.seg.K;
  int kpad = (K + 3) & ~3;
  if ((kpad & 7) == 0) kpad += 4;  // row stride = 4 (mod 8) words: rows' float4 loads hit distinct banks
  int rows = kRowsMax;
  if (ORD == ORD_DW) {
    rows = kTabFloats / kpad;
    if (rows > kRowsMax) rows = kRowsMax;
    if (rows < 1) rows = 1;
  }
  size_t smem = ORD == ORD_DW ? (size_t)rows * kpad * sizeof(float) : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (long long)sms * 8;
  if (blocks > n_items) blocks = n_items;
  integrate_fp32c_kernel<ORD><<<(unsigned)blocks, kThreads, smem, st>>>(p, keys, list, n_items, terms, n_isl, rows,
                                                                       kpad);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp32c_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                              long long n_items, float* terms, long long n_isl, cudaStream_t st) {
  if (ord == ORD_DW) return launch_one<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
  if (ord == ORD_E) return launch_one<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
  return launch_one<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
}

}  // namespace egn
