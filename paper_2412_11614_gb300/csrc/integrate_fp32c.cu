// integrate_fp32c.cu -- FP32 island integrator with exact phase reduction (the
// fast path).
//
// Work decomposition.  A CTA of 128 threads takes islands in batches of 128.
//  1. Batch set-up (FP64, one island per thread): geometry of the node rule,
//     panel edges and the island constants, rounded to FP32 head/tail pairs
//     ("double-float", 48-bit significand).  GB300 runs FP64 at 1/64 of the FP32
//     rate, so FP64 appears only here, with every lane busy.
//  2. Per island, per chunk of outer nodes ("rows"): the row constants in
//     double-float arithmetic (FP32 only) -- the cubic phase polynomial in the
//     inner node, Q0 reduced modulo K -- and, in the DW order, the row's table
//     c_k = C_k e^{-zeta_k f3} in shared memory.
//  3. Per point (4 per thread, one row): phase, segment sum, Upsilon, weights.
//
// Arithmetic per point:
//  * Phase.  Theta(x) = chi L / 2 pi = 2 pi L (f1 - f)(f2 - f)[beta2 + pi beta3 (f1 + f2)]
//    (Eq. 5, 24) is a cubic in the inner Gauss-Legendre coordinate x along a row.
//    Q1 x and Q2 x^2 are exact FP32 products (error-free FMA product plus tail
//    cross terms), reduced modulo K exactly (the FMA residual p - K n is exact),
//    and summed with error-free two-sums; this yields theta = chi L/K and
//    phi = chi L, both in turns modulo 1, to ~1e-7 turns.
//  * Segment sum (Eq. 8-10).  mu = (w - 1)/(i chi - alpha) sum_k c_k w^k,
//    w = r e^{i theta}; the real-coefficient polynomial is evaluated by the
//    second-order real recurrence b_k = c_k + p b_{k+1} - q b_{k+2} (p = 2 Re w,
//    q = |w|^2), sum = b_0 - conj(w) b_1: Horner's rule rewritten exactly, 2 FMA
//    per segment instead of 4; |w| < 1 bounds its error growth.
//  * Phased array (Eq. 22): ratio sin(N pi phi)/sin(pi phi); near phi = 0 the
//    sines use their Taylor series (|argument| < 0.05, relative error < 1e-12).
//    Hardware sin/cos (MUFU, absolute error ~4e-7 on [-pi, pi]) elsewhere.
// Island sums: FP32 per thread, fixed-order shuffle and shared-memory trees.
#include "egn_internal.h"
#include "island_geom.cuh"

namespace egn {
namespace {

constexpr int kThreads = 128;
constexpr int kBatch = kThreads;   // islands per batch, one per thread in the set-up
constexpr int kP = 4;              // points per thread (same row)
constexpr int kRowsMax = 64;       // rows per chunk held in shared memory
constexpr int kTabFloats = 5376;   // DW c_k table budget (21 KB), each c_k stored twice (f32x2)

// ---------------------------------------------------------------- double-float
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

// sin(x) for |x| < 0.05 by its Taylor series to x^7 (relative error < 1e-12).
__device__ __forceinline__ float sin_small(float x) {
  float x2 = x * x;
  return x * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
}

// Raised-cosine shape in FP32.
__device__ __forceinline__ float rc_f(float x, float R, float beta) {
  float ax = fabsf(x);
  float a = 0.5f * (1.0f - beta) * R, b = 0.5f * (1.0f + beta) * R;
  if (ax <= a) return 1.0f;
  if (ax >= b) return 0.0f;
  return 0.5f * (1.0f + __cosf(3.14159265f * (ax - a) / (beta * R)));
}

// ---------------------------------------------------------------- shared state
struct BatchSm {  // one entry per island of the batch
  long long isl[kBatch];
  int np[kBatch];
  int flags[kBatch];  // bit0 G wanted, bit1 H wanted
  Df pm[3][kBatch], ph[3][kBatch];                      // panel midpoints and half-widths
  Df Bv[kBatch], Cv[kBatch], cv[kBatch];                // node-rule constants
  Df F1[kBatch], F2[kBatch], S12[kBatch], dd[kBatch];   // nu1 - nu, nu2 - nu, nu1 + nu2, d
  float R1[kBatch], R2[kBatch], R3[kBatch], nu3[kBatch];
  float cf0[kBatch], cf1[kBatch], cf2[kBatch];          // D, G, H (DW) or the E / F coefficient
};

struct RowSm {
  float q0h[kRowsMax], q0l[kRowsMax], q1h[kRowsMax], q1l[kRowsMax], q2h[kRowsMax], q2l[kRowsMax], q3[kRowsMax];
  float a0[kRowsMax], a1[kRowsMax], b0[kRowsMax], b1[kRowsMax];  // f1 - f, f2 - f = a0 + a1 x, b0 + b1 x
  float bc0[kRowsMax], bc1[kRowsMax];                            // beta2 + pi beta3 (f1 + f2) = bc0 + bc1 x
  float im[kRowsMax], ih[kRowsMax];                              // inner variable = im + ih x
  float o[kRowsMax];                                             // outer variable
  float wo[kRowsMax];                                            // outer weight
  float hout[kRowsMax];                                          // shape of the outer variable's channel
  float f30[kRowsMax], f31[kRowsMax];                            // f3 = f30 + f31 x
};

template <int ORD>
__global__ void __launch_bounds__(kThreads, 4)
integrate_fp32c_kernel(LinkParams p, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                       long long n_items, float* __restrict__ terms, long long n_isl, int rows_per_chunk, int kpad,
                       Df G0, Df G1) {
  __shared__ BatchSm bs;
  __shared__ RowSm rs;
  __shared__ float red[4][kThreads / 32];
  extern __shared__ __align__(16) float2 tab[];  // [rows_per_chunk][kpad] pairs (c_k, c_k) (DW only)

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = p.gl.n;
  const int K = p.seg.K;
  const float Kf = (float)K, invK = 1.0f / (float)K;
  const float beta = (float)p.rolloff;
  const float alpha = (float)p.alpha, alpha2 = alpha * alpha;
  const float r = (float)p.r;
  const float one_m_r = (float)(-expm1(-p.alpha * p.dz));
  const float q = r * r;
  const float N = (float)p.n_spans;
  const float gam = (float)p.gamma;
  const float g2 = gam * gam;
  const float k4 = (float)(4.0 * kPi * kPi);
  const float pib3 = (float)(kPi * p.beta3), b2f = (float)p.beta2;
  const float pi_f = 3.14159265358979f;
  // threads per row (power of two), row slot and point slot of this thread
  int tpr = 1;
  while (tpr * kP < n) tpr <<= 1;
  const int rows_per_pass = kThreads / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;
  // this thread's inner nodes (fixed for the whole launch)
  float nxh[kP], nxl[kP], nwf[kP];
  bool jok[kP];
#pragma unroll
  for (int m = 0; m < kP; ++m) {
    int j = lr + tpr * m;
    jok[m] = j < n;
    int jj = jok[m] ? j : 0;
    nxh[m] = p.gl.xh[1][jj];
    nxl[m] = p.gl.xl[1][jj];
    nwf[m] = jok[m] ? p.gl.wf[1][jj] : 0.0f;
  }

  for (long long b0 = (long long)blockIdx.x * kBatch; b0 < n_items; b0 += (long long)gridDim.x * kBatch) {
    // ---------------- 1. batch set-up, FP64, one island per thread
    {
      long long it = b0 + tid;
      int np = 0, flags = 0;
      long long isl = -1;
      if (it < n_items) {
        isl = list ? (long long)list[it] : it;
        int coi, n1, n2, n3;
        unpack_key(keys[isl], coi, n1, n2, n3);
        const ChannelTable& ch = p.ch;
        double nu = ch.nu[coi], nu1 = ch.nu[n1], nu2 = ch.nu[n2], nu3 = ch.nu[n3];
        double R = ch.R[coi], R1 = ch.R[n1], R2 = ch.R[n2], R3 = ch.R[n3];
        double d = (nu1 - nu) + (nu2 - nu3);
        Ordering g = make_ordering(ORD, ch.W[n1], ch.W[n2], ch.W[n3], d);
        double e[4];
        np = outer_panels(g, e);
        for (int q_ = 0; q_ < 3; ++q_) {
          double pm = 0.0, ph = 0.0;
          if (q_ < np) { pm = 0.5 * (e[q_] + e[q_ + 1]); ph = 0.5 * (e[q_ + 1] - e[q_]); }
          bs.pm[q_][tid] = df_of(pm);
          bs.ph[q_][tid] = df_of(ph);
        }
        bs.Bv[tid] = df_of(g.B);
        bs.Cv[tid] = df_of(g.C);
        bs.cv[tid] = df_of(g.c);
        bs.F1[tid] = df_of(nu1 - nu);
        bs.F2[tid] = df_of(nu2 - nu);
        bs.S12[tid] = df_of(nu1 + nu2);
        bs.dd[tid] = df_of(d);
        bs.R1[tid] = (float)R1;
        bs.R2[tid] = (float)R2;
        bs.R3[tid] = (float)R3;
        bs.nu3[tid] = (float)nu3;
        double cf[5];
        term_coefs(R, R1, R2, R3, cf);
        if (ORD == ORD_DW) {
          bool wg = p.all_terms || (p.terms && flag_g(n1, n2, n3));
          bool wh = p.all_terms || (p.terms && flag_h(n1, n2, n3));
          flags = (wg ? 1 : 0) | (wh ? 2 : 0);
          bs.cf0[tid] = (float)cf[0];
          bs.cf1[tid] = (float)cf[3];
          bs.cf2[tid] = (float)cf[4];
        } else {
          bs.cf0[tid] = (float)(ORD == ORD_E ? cf[1] : cf[2]);
        }
      }
      bs.isl[tid] = isl;
      bs.np[tid] = np;
      bs.flags[tid] = flags;
    }
    __syncthreads();
    const int nb = (int)min((long long)kBatch, n_items - b0);
    // ---------------- 2./3. the islands of the batch, one after the other
    for (int ib = 0; ib < nb; ++ib) {
      const int np = bs.np[ib];
      const int flags = bs.flags[ib];
      const bool want_g = flags & 1, want_h = flags & 2;
      const bool cplx = ORD != ORD_DW || flags != 0;
      const float R1f = bs.R1[ib], R2f = bs.R2[ib], R3f = bs.R3[ib];
      const float dfl = dval(bs.dd[ib]);
      float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
      const int no = np > 0 ? p.gl.order[np] : 0;
      const int rows = np * no;
      for (int c0 = 0; c0 < rows; c0 += rows_per_chunk) {
        const int rc = min(rows_per_chunk, rows - c0);
        // ---- row constants in double-float; rows spread over the four warps
        {
          // slot rr = 32 (tid mod 4) + tid / 4 (a bijection on 0..127): the first 32 rows
          // of a chunk go to 8 lanes of each warp, so all four warps share the work
          const int rr = (tid & 3) * 32 + (tid >> 2);
          if (rr < rc) {
            const int row = c0 + rr;
            const int pi = row / no, i = row - pi * no;
            const Df y = {p.gl.xh[np][i], p.gl.xl[np][i]};
            const Df pm = bs.pm[pi][ib], ph = bs.ph[pi][ib];
            const Df o = dadd(pm, dmul(ph, y));
            const Df m = (ORD == ORD_DW) ? dadd(o, bs.cv[ib]) : dsub(bs.cv[ib], o);
            const Df Bv = bs.Bv[ib], Cv = bs.Cv[ib];
            const Df lo = dmax(dneg(Bv), dsub(m, Cv));
            const Df hi = dmin(Bv, dadd(m, Cv));
            const Df im = dhalf(dadd(lo, hi)), ih = dhalf(dsub(hi, lo));
            const Df zero = {0.0f, 0.0f};
            Df a0, b0_, s0, a1 = zero, b1 = zero, s1 = zero;
            if (ORD == ORD_DW) {  // w = o, u = im + ih x, v = w - u - d
              a0 = dadd(bs.F1[ib], im); a1 = ih;
              b0_ = dadd(bs.F2[ib], dsub(dsub(o, im), bs.dd[ib])); b1 = dneg(ih);
              s0 = dadd(bs.S12[ib], dsub(o, bs.dd[ib]));
            } else if (ORD == ORD_E) {  // v = o, u = im + ih x
              a0 = dadd(bs.F1[ib], im); a1 = ih;
              b0_ = dadd(bs.F2[ib], o);
              s0 = dadd(bs.S12[ib], dadd(im, o)); s1 = ih;
            } else {  // u = o, v = im + ih x
              a0 = dadd(bs.F1[ib], o);
              b0_ = dadd(bs.F2[ib], im); b1 = ih;
              s0 = dadd(bs.S12[ib], dadd(o, im)); s1 = ih;
            }
            const Df g0 = dadd(G0, dmul(G1, s0));   // 2 pi L (beta2 + pi beta3 s0)
            const Df g1 = dmul(G1, s1);             // 2 pi L pi beta3 s1
            const Df ab0 = dmul(a0, b0_);
            const Df ab1 = dadd(dmul(a0, b1), dmul(a1, b0_));
            const Df ab2 = dmul(a1, b1);
            const Df Q0 = dmul(g0, ab0);
            const Df Q1 = dadd(dmul(g0, ab1), dmul(g1, ab0));
            const Df Q2 = dadd(dmul(g0, ab2), dmul(g1, ab1));
            const float Q3 = dval(g1) * dval(ab2);
            // Q0 modulo K (the FMA residual is exact)
            const float r0 = fmaf(-Kf, rintf(Q0.hi * invK), Q0.hi);
            const Df Q0r = quick(r0, Q0.lo);
            rs.q0h[rr] = Q0r.hi; rs.q0l[rr] = Q0r.lo;
            rs.q1h[rr] = Q1.hi; rs.q1l[rr] = Q1.lo;
            rs.q2h[rr] = Q2.hi; rs.q2l[rr] = Q2.lo;
            rs.q3[rr] = Q3;
            rs.a0[rr] = dval(a0); rs.a1[rr] = dval(a1);
            rs.b0[rr] = dval(b0_); rs.b1[rr] = dval(b1);
            const float s0f = dval(s0), s1f = dval(s1);
            rs.bc0[rr] = fmaf(pib3, s0f, b2f);
            rs.bc1[rr] = pib3 * s1f;
            const float imf = dval(im), ihf = dval(ih), of = dval(o);
            rs.im[rr] = imf; rs.ih[rr] = ihf; rs.o[rr] = of;
            rs.wo[rr] = dval(ph) * p.gl.wf[np][i];
            rs.hout[rr] = ORD == ORD_DW ? rc_f(of, R3f, beta) : (ORD == ORD_E ? rc_f(of, R2f, beta) : rc_f(of, R1f, beta));
            const float nu3 = bs.nu3[ib];
            if (ORD == ORD_DW) { rs.f30[rr] = nu3 + of; rs.f31[rr] = 0.0f; }
            else { rs.f30[rr] = nu3 + (imf + of + dfl); rs.f31[rr] = ihf; }
          }
        }
        __syncthreads();
        // ---- c_k tables of the chunk's rows (DW): C_k 2^{-zeta_k log2(e) f3}
        if (ORD == ORD_DW) {
          for (int k = tid; k < K; k += kThreads) {
            const float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
            for (int rr = 0; rr < rc; ++rr) {
              const float c = ck * ex2_approx(-zk * rs.f30[rr]);
              tab[rr * kpad + k] = make_float2(c, c);
            }
          }
          __syncthreads();
        }
        // ---- points
        for (int rb = 0; rb < rc; rb += rows_per_pass) {
          const int rr = rb + rsub;
          const bool row_ok = rr < rc;
          const int rrc = row_ok ? rr : 0;
          float gre = 0.0f, gim = 0.0f;
          float p_[kP], b1_[kP], b2_[kP], f3_[kP];
          float wm1_[kP], wi_[kP], chi_[kP], phi_[kP], wgt_[kP], s12_[kP], s123_[kP];
          const float q0h = rs.q0h[rrc], q0l = rs.q0l[rrc], q1h = rs.q1h[rrc], q1l = rs.q1l[rrc];
          const float q2h = rs.q2h[rrc], q2l = rs.q2l[rrc], q3 = rs.q3[rrc];
          const float a0 = rs.a0[rrc], a1 = rs.a1[rrc], b0 = rs.b0[rrc], b1 = rs.b1[rrc];
          const float bc0 = rs.bc0[rrc], bc1 = rs.bc1[rrc], im = rs.im[rrc], ih = rs.ih[rrc], of = rs.o[rrc];
          const float wo = rs.wo[rrc], hout = rs.hout[rrc], f30 = rs.f30[rrc], f31 = rs.f31[rrc];
#pragma unroll
          for (int m = 0; m < kP; ++m) {
            const bool ok = row_ok && jok[m];
            const float xh = nxh[m], xl = nxl[m];
            // x^2 as a double-float
            const float x2h = xh * xh, x2l = fmaf(xh, xh, -x2h) + 2.0f * xh * xl;
            // phase modulo K: Q0 + Q1 x + Q2 x^2 + Q3 x^3 with exact products and sums
            const float p1 = q1h * xh, e1 = fmaf(q1h, xh, -p1);
            const float t1 = fmaf(q1h, xl, fmaf(q1l, xh, e1));
            const float p2 = q2h * x2h, e2 = fmaf(q2h, x2h, -p2);
            const float t2 = fmaf(q2h, x2l, fmaf(q2l, x2h, e2));
            const float r1 = fmaf(-Kf, rintf(p1 * invK), p1);
            const float r2 = fmaf(-Kf, rintf(p2 * invK), p2);
            float s1, s2, ea, eb;
            two_sum(q0h, r1, s1, ea);
            two_sum(s1, r2, s2, eb);
            const float tail = ((ea + eb) + (q0l + t1 + t2)) + q3 * (xh * x2h);
            float th = fmaf(s2, invK, tail * invK);
            th -= rintf(th);                     // theta in turns, [-1/2, 1/2]
            float ph = (s2 - rintf(s2)) + tail;  // phi in turns
            ph -= rintf(ph);
            // w = r e^{2 pi i th} from the half angle: keeps w - 1 accurate
            const float ah = pi_f * th;
            const float sh = __sinf(ah), chh = __cosf(ah);
            const float wr = r * fmaf(-2.0f * sh, sh, 1.0f);
            p_[m] = 2.0f * wr;
            wm1_[m] = -one_m_r - 2.0f * r * sh * sh;  // Re(w - 1)
            wi_[m] = 2.0f * r * sh * chh;
            phi_[m] = ph;
            // chi [rad/km] for (i chi - alpha)
            const float a = fmaf(a1, xh, a0), b = fmaf(b1, xh, b0), bc = fmaf(bc1, xh, bc0);
            chi_[m] = k4 * a * b * bc;
            // spectral shapes and weights
            const float t = fmaf(ih, xh, im);
            float u, v, h3;
            if (ORD == ORD_DW) { u = t; v = of - t - dfl; h3 = hout; }
            else {
              if (ORD == ORD_E) { v = of; u = t; } else { u = of; v = t; }
              h3 = rc_f(u + v + dfl, R3f, beta);
            }
            const float h1 = rc_f(u, R1f, beta), h2 = rc_f(v, R2f, beta);
            const float wij = ok ? wo * ih * nwf[m] : 0.0f;
            wgt_[m] = wij * h1 * h2 * h3;
            s12_[m] = 0.0f;
            s123_[m] = 0.0f;
            if (cplx) {
              if (ORD == ORD_DW) {
                s12_[m] = ok ? nwf[m] * sqrtf(h1 * h2) : 0.0f;
                s123_[m] = wij * sqrtf(h1 * h2 * h3);
              } else {
                s12_[m] = ok ? nwf[m] * ih * sqrtf(ORD == ORD_E ? h1 * h3 : h2 * h3) : 0.0f;
              }
            }
            f3_[m] = fmaf(f31, xh, f30);
            b1_[m] = 0.0f;
            b2_[m] = 0.0f;
          }
          // ---- segment sum by the real recurrence, k = K-1 .. 0
          if (ORD == ORD_DW) {
            // points (0, 1) and (2, 3) as f32x2 pairs; the table holds (c_k, c_k)
            const float2* trow = tab + rrc * kpad;
            const f32x2 nq2 = pack2(-q, -q);
            const f32x2 pA = pack2(p_[0], p_[1]), pB = pack2(p_[2], p_[3]);
            f32x2 b1A = 0ull, b2A = 0ull, b1B = 0ull, b2B = 0ull;
            int k = K - 1;
            if (K & 1) {  // peel so that the 16-byte loads below are aligned
              const f32x2 c = *reinterpret_cast<const f32x2*>(trow + k);
              f32x2 nA = ffma2(nq2, b2A, ffma2(pA, b1A, c));
              f32x2 nB = ffma2(nq2, b2B, ffma2(pB, b1B, c));
              b2A = b1A; b1A = nA; b2B = b1B; b1B = nB;
              --k;
            }
            for (; k >= 1; k -= 2) {
              const ulonglong2 cc = *reinterpret_cast<const ulonglong2*>(trow + k - 1);  // (c_{k-1}, c_k) pairs
              f32x2 nA = ffma2(nq2, b2A, ffma2(pA, b1A, cc.y));
              f32x2 nB = ffma2(nq2, b2B, ffma2(pB, b1B, cc.y));
              b2A = b1A; b1A = nA; b2B = b1B; b1B = nB;
              nA = ffma2(nq2, b2A, ffma2(pA, b1A, cc.x));
              nB = ffma2(nq2, b2B, ffma2(pB, b1B, cc.x));
              b2A = b1A; b1A = nA; b2B = b1B; b1B = nB;
            }
            unpack2(b1A, b1_[0], b1_[1]);
            unpack2(b2A, b2_[0], b2_[1]);
            unpack2(b1B, b1_[2], b1_[3]);
            unpack2(b2B, b2_[2], b2_[3]);
          } else {
            for (int k = K - 1; k >= 0; --k) {
              const float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
#pragma unroll
              for (int m = 0; m < kP; ++m) {
                const float c = ck * ex2_approx(-zk * f3_[m]);
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
            // after the loop b1 = b_0 and b2 = b_1: sum = b_0 - conj(w) b_1
            const float wr = 0.5f * p_[m], wi = wi_[m];
            const float sre = fmaf(-wr, b2_[m], b1_[m]);
            const float sim = wi * b2_[m];
            // (w - 1)/(i chi - alpha) = (w - 1)(-alpha - i chi)/(alpha^2 + chi^2)
            const float xr = wm1_[m], chi = chi_[m];
            const float inv = rcp_approx(fmaf(chi, chi, alpha2));
            const float qr = fmaf(-alpha, xr, chi * wi) * inv;
            const float qi = fmaf(-chi, xr, -alpha * wi) * inv;
            const float mre = fmaf(sre, qr, -sim * qi);
            const float mim = fmaf(sre, qi, sim * qr);
            // phased array: sin(N pi phi) / sin(pi phi)
            const float x = pi_f * phi_[m];
            const float Nx = N * x;
            float ratio;
            if (fabsf(x) >= 0.05f) {
              ratio = __sinf(Nx) * rcp_approx(__sinf(x));
            } else {  // near the array-factor peak: series for the small sines
              const float snum = fabsf(Nx) < 0.05f ? sin_small(Nx) : __sinf(Nx);
              ratio = (x == 0.0f) ? N : snum * rcp_approx(sin_small(x));
            }
            if (!cplx) {
              dsum = fmaf(wgt_[m], (mre * mre + mim * mim) * (ratio * ratio), dsum);
            } else {
              const float ang = (N - 1.0f) * x;
              const float sp = __sinf(ang), cp = __cosf(ang);
              const float yre = ratio * fmaf(mre, cp, -mim * sp);  // Upsilon / gamma
              const float yim = ratio * fmaf(mre, sp, mim * cp);
              if (ORD == ORD_DW) {
                dsum = fmaf(wgt_[m], yre * yre + yim * yim, dsum);
                hre = fmaf(s123_[m], yre, hre);
                him = fmaf(s123_[m], yim, him);
              }
              gre = fmaf(s12_[m], yre, gre);
              gim = fmaf(s12_[m], yim, gim);
            }
          }
          if (ORD != ORD_DW || want_g) {
            // complete the row's inner sum over its tpr threads, then |.|^2 x outer weight
            for (int o_ = tpr >> 1; o_ > 0; o_ >>= 1) {
              gre += __shfl_xor_sync(0xffffffffu, gre, o_);
              gim += __shfl_xor_sync(0xffffffffu, gim, o_);
            }
            if (lr == 0 && row_ok) {
              const float ihr = (ORD == ORD_DW) ? ih : 1.0f;
              const float gr_ = gre * ihr, gi_ = gim * ihr;
              csum = fmaf(wo * hout, gr_ * gr_ + gi_ * gi_, csum);
            }
          }
        }
        __syncthreads();  // rows and tables are rewritten by the next chunk
      }
      // ---- island reduction (fixed order); every sum above is of Upsilon / gamma
      float vals[4] = {dsum, csum, hre, him};
#pragma unroll
      for (int a = 0; a < 4; ++a)
        for (int o_ = 16; o_ > 0; o_ >>= 1) vals[a] += __shfl_xor_sync(0xffffffffu, vals[a], o_);
      if (lane == 0)
#pragma unroll
        for (int a = 0; a < 4; ++a) red[a][wid] = vals[a];
      __syncthreads();
      if (tid == 0) {
        float t[4];
        for (int a = 0; a < 4; ++a) t[a] = (red[a][0] + red[a][1]) + (red[a][2] + red[a][3]);
        const long long isl = bs.isl[ib];
        if (ORD == ORD_DW) {
          terms[isl] = bs.cf0[ib] * g2 * t[0];
          if (want_g) terms[3 * n_isl + isl] = bs.cf1[ib] * g2 * t[1];
          if (want_h) terms[4 * n_isl + isl] = bs.cf2[ib] * g2 * (t[2] * t[2] + t[3] * t[3]);
        } else {
          terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = bs.cf0[ib] * g2 * t[1];
        }
      }
      __syncthreads();
    }
  }
}

template <int ORD>
cudaError_t launch_one(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items, float* terms,
                       long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const int K = p.seg.K;
  int kpad = (K + 3) & ~3;
  if ((kpad & 7) == 0) kpad += 4;  // row stride 2 kpad = 8 (mod 16) words: 4 rows' 16-byte loads hit distinct banks
  int rows = kRowsMax;
  if (ORD == ORD_DW) {
    rows = kTabFloats / (2 * kpad);
    if (rows > kRowsMax) rows = kRowsMax;
    if (rows < 1) rows = 1;
  }
  size_t smem = ORD == ORD_DW ? (size_t)rows * kpad * sizeof(float2) : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long batches = (n_items + kBatch - 1) / kBatch;
  long long blocks = (long long)sms * 4;
  if (blocks > batches) blocks = batches;
  // 2 pi L beta2 and 2 pi^2 L beta3 as double-floats
  double g0 = 2.0 * kPi * p.L * p.beta2, g1 = 2.0 * kPi * kPi * p.L * p.beta3;
  float g0h = (float)g0, g1h = (float)g1;
  Df G0 = {g0h, (float)(g0 - (double)g0h)}, G1 = {g1h, (float)(g1 - (double)g1h)};
  integrate_fp32c_kernel<ORD><<<(unsigned)blocks, kThreads, smem, st>>>(p, keys, list, n_items, terms, n_isl, rows,
                                                                       kpad, G0, G1);
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
