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
//  3. Per point (KP per thread, one row): phase, segment sum, Upsilon, weights.
//
// Arithmetic per point:
//  * Phase.  Theta(x) = chi L / 2 pi = 2 pi L (f1 - f)(f2 - f)[beta2 + pi beta3 (f1 + f2)]
//    (Eq. 5, 24) is a cubic in the inner Gauss-Legendre coordinate x along a row,
//    Theta = Q0 + Q1 x + Q2 x^2 + Q3 x^3 (turns of one span).  Q1 x and Q2 x^2 are
//    formed as exact FP32 products (error-free FMA product plus tail cross terms)
//    and Q1 x is reduced modulo K exactly (the FMA residual p - K n is exact).
//    phi = chi L modulo 1 is the sum of the exact fractional parts of the terms
//    (~1e-7 turns); theta = chi L / K modulo 1 takes the rounded sum of the
//    reduced terms divided by K (~1e-5 / K turns).
//  * Segment sum (Eq. 8-10).  mu = (w - 1)/(i chi - alpha) sum_k c_k w^k,
//    w = r e^{i theta}; the real-coefficient polynomial is evaluated by the
//    second-order real recurrence b_k = c_k + p b_{k+1} - q b_{k+2} (p = 2 Re w,
//    q = |w|^2), sum = b_0 - conj(w) b_1: Horner's rule rewritten exactly, 2 FMA
//    per segment instead of 4; |w| < 1 bounds its error growth.  In the DW order
//    two points share one fma.rn.f32x2 instruction.
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

// Row constants, four per float4 so that a point pass loads them with 16-byte loads.
struct RowSm {
  float4 qa[kRowsMax];  // q0h, q0l, q1h, q1l              (phase, turns; Q0 modulo K)
  float4 qb[kRowsMax];  // q2h, q2l, q3, frac(q0h)
  float4 ab[kRowsMax];  // a0, a1, b0, b1                  (f1 - f = a0 + a1 x, f2 - f = b0 + b1 x)
  float4 kc[kRowsMax];  // 4 pi^2 bc0, 4 pi^2 bc1, im, ih   (bc = beta2 + pi beta3 (f1 + f2); inner = im + ih x)
  float4 ow[kRowsMax];  // o - d (DW) or o, wo ih hout, wo ih, hout   (wo outer weight, hout outer shape)
  float4 f3[kRowsMax];  // f30, f31, wo, 0                  (f3 = f30 + f31 x)
};

// Inner Gauss-Legendre nodes of the launch: {x head, x tail, x^2 head, x^2 tail}, {x^3, w}.
struct NodeSm {
  float4 x4[kMaxGl];
  float2 x2[kMaxGl];
};

template <int ORD, int KP>
__global__ void __launch_bounds__(kThreads, KP == 8 ? 3 : 4)
integrate_fp32c_kernel(LinkParams p, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                       long long n_items, float* __restrict__ terms, long long n_isl, int rows_per_chunk, int kpad,
                       Df G0, Df G1) {
  static_assert(KP % 2 == 0, "points per thread come in f32x2 pairs");
  constexpr int NPAIR = KP / 2;
  __shared__ BatchSm bs;
  __shared__ RowSm rs;
  __shared__ NodeSm ns;
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
  const float m2r = -2.0f * r;
  const float N = (float)p.n_spans;
  const float gam = (float)p.gamma;
  const float g2 = gam * gam;
  const float k4 = (float)(4.0 * kPi * kPi);
  const float pib3 = (float)(kPi * p.beta3), b2f = (float)p.beta2;
  const float pi_f = 3.14159265358979f;
  // threads per row (power of two), row slot and point slot of this thread
  int tpr = 1;
  while (tpr * KP < n) tpr <<= 1;
  const int rows_per_pass = kThreads / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;

  for (int j = tid; j < n; j += kThreads) {
    const float xh = p.gl.xh[1][j], xl = p.gl.xl[1][j];
    ns.x4[j] = make_float4(xh, xl, p.gl.x2h[1][j], p.gl.x2l[1][j]);
    ns.x2[j] = make_float2(xh * p.gl.x2h[1][j], p.gl.wf[1][j]);
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
        // ---- row constants in double-float; slot rr = 32 (tid mod 4) + tid / 4 (a
        // bijection on 0..127) spreads the first 32 rows of a chunk over the four warps
        {
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
            const float s0f = dval(s0), s1f = dval(s1);
            const float imf = dval(im), ihf = dval(ih), of = dval(o);
            const float wo = dval(ph) * p.gl.wf[np][i];
            const float hout = ORD == ORD_DW ? rc_f(of, R3f, beta) : (ORD == ORD_E ? rc_f(of, R2f, beta) : rc_f(of, R1f, beta));
            rs.qa[rr] = make_float4(Q0r.hi, Q0r.lo, Q1.hi, Q1.lo);
            rs.qb[rr] = make_float4(Q2.hi, Q2.lo, Q3, Q0r.hi - rintf(Q0r.hi));
            rs.ab[rr] = make_float4(dval(a0), dval(a1), dval(b0_), dval(b1));
            rs.kc[rr] = make_float4(k4 * fmaf(pib3, s0f, b2f), k4 * pib3 * s1f, imf, ihf);
            rs.ow[rr] = make_float4(ORD == ORD_DW ? of - dfl : of, wo * ihf * hout, wo * ihf, hout);
            const float nu3 = bs.nu3[ib];
            if (ORD == ORD_DW) rs.f3[rr] = make_float4(nu3 + of, 0.0f, wo, 0.0f);
            else rs.f3[rr] = make_float4(nu3 + (imf + of + dfl), ihf, wo, 0.0f);
          }
        }
        __syncthreads();
        // ---- c_k tables of the chunk's rows (DW): C_k 2^{-zeta_k log2(e) f3}
        if (ORD == ORD_DW) {
          for (int k = tid; k < K; k += kThreads) {
            const float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
            for (int rr = 0; rr < rc; ++rr) {
              const float c = ck * ex2_approx(-zk * rs.f3[rr].x);
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
          const float4 qa = rs.qa[rrc], qb = rs.qb[rrc], ab = rs.ab[rrc], kc = rs.kc[rrc], ow = rs.ow[rrc];
          const float4 f3r = rs.f3[rrc];
          const float q0h = qa.x, q0l = qa.y, q1h = qa.z, q1l = qa.w;
          const float q2h = qb.x, q2l = qb.y, q3 = qb.z, fq0 = qb.w;
          const float im = kc.z, ih = kc.w;
          const float wrowh = row_ok ? ow.y : 0.0f, wrow = row_ok ? ow.z : 0.0f;
          float gre = 0.0f, gim = 0.0f;
          float p_[KP], b1_[KP], b2_[KP], f3_[KP];
          float wm1_[KP], wi_[KP], chi_[KP], phi_[KP], wgt_[KP], s12_[KP], s123_[KP];
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const int j = lr + tpr * m;
            const bool jok = j < n;
            const int jj = jok ? j : 0;
            const float4 x4 = ns.x4[jj];
            const float2 x2 = ns.x2[jj];
            const float xh = x4.x, xl = x4.y, x2h = x4.z, x2l = x4.w, xc = x2.x;
            const float wnode = jok ? x2.y : 0.0f;
            // phase: exact products, Q1 x reduced modulo K
            const float p1 = q1h * xh, e1 = fmaf(q1h, xh, -p1);
            const float t1 = fmaf(q1h, xl, fmaf(q1l, xh, e1));
            const float p2 = q2h * x2h, e2 = fmaf(q2h, x2h, -p2);
            const float t2 = fmaf(q2h, x2l, fmaf(q2l, x2h, e2));
            const float r1 = fmaf(-Kf, rintf(p1 * invK), p1);
            const float tail = (q0l + t1) + fmaf(q3, xc, t2);
            float th = fmaf((q0h + r1) + p2, invK, tail * invK);
            th -= rintf(th);                                           // theta (turns)
            float ph = (fq0 + (r1 - rintf(r1))) + ((p2 - rintf(p2)) + tail);
            ph -= rintf(ph);                                           // phi (turns)
            // w = r e^{2 pi i th} from the half angle (keeps w - 1 accurate)
            const float ah = pi_f * th;
            const float sh = __sinf(ah), chh = __cosf(ah);
            const float t2r = m2r * sh;
            const float wm1 = fmaf(t2r, sh, -one_m_r);                 // Re(w - 1)
            p_[m] = fmaf(2.0f, wm1, 2.0f);                            // 2 Re(w)
            wm1_[m] = wm1;
            wi_[m] = -t2r * chh;                                      // Im(w)
            phi_[m] = ph;
            // chi [rad/km] for (i chi - alpha)
            chi_[m] = fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z) * fmaf(kc.y, xh, kc.x);
            // spectral shapes and weights
            const float t = fmaf(ih, xh, im);
            float u, v, h3;
            if (ORD == ORD_DW) { u = t; v = ow.x - t; h3 = 1.0f; }  // h3(w) is folded into wrowh
            else {
              if (ORD == ORD_E) { v = ow.x; u = t; } else { u = ow.x; v = t; }
              h3 = rc_f(u + v + dfl, R3f, beta);
            }
            const float h1 = rc_f(u, R1f, beta), h2 = rc_f(v, R2f, beta);
            wgt_[m] = (ORD == ORD_DW ? wrowh : wrow) * wnode * h1 * h2 * h3;
            s12_[m] = 0.0f;
            s123_[m] = 0.0f;
            if (cplx) {
              if (ORD == ORD_DW) {
                s12_[m] = (row_ok ? wnode : 0.0f) * sqrtf(h1 * h2);
                s123_[m] = wrow * wnode * sqrtf(h1 * h2 * ow.w);
              } else {
                s12_[m] = (row_ok ? wnode : 0.0f) * ih * sqrtf(ORD == ORD_E ? h1 * h3 : h2 * h3);
              }
            }
            f3_[m] = fmaf(f3r.y, xh, f3r.x);
            b1_[m] = 0.0f;
            b2_[m] = 0.0f;
          }
          // ---- segment sum by the real recurrence, k = K-1 .. 0
          if (ORD == ORD_DW) {
            const float2* trow = tab + rrc * kpad;
            const f32x2 nq2 = pack2(-q, -q);
            f32x2 pp[NPAIR], b1p[NPAIR], b2p[NPAIR];
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) {
              pp[a] = pack2(p_[2 * a], p_[2 * a + 1]);
              b1p[a] = 0ull;
              b2p[a] = 0ull;
            }
            int k = K - 1;
            if (K & 1) {  // peel so that the 16-byte loads below are aligned
              const f32x2 c = *reinterpret_cast<const f32x2*>(trow + k);
#pragma unroll
              for (int a = 0; a < NPAIR; ++a) {
                const f32x2 nb = ffma2(nq2, b2p[a], ffma2(pp[a], b1p[a], c));
                b2p[a] = b1p[a];
                b1p[a] = nb;
              }
              --k;
            }
            for (; k >= 1; k -= 2) {
              const ulonglong2 cc = *reinterpret_cast<const ulonglong2*>(trow + k - 1);  // (c_{k-1}, c_k) pairs
#pragma unroll
              for (int a = 0; a < NPAIR; ++a) {
                const f32x2 nb = ffma2(nq2, b2p[a], ffma2(pp[a], b1p[a], cc.y));
                b2p[a] = b1p[a];
                b1p[a] = nb;
              }
#pragma unroll
              for (int a = 0; a < NPAIR; ++a) {
                const f32x2 nb = ffma2(nq2, b2p[a], ffma2(pp[a], b1p[a], cc.x));
                b2p[a] = b1p[a];
                b1p[a] = nb;
              }
            }
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) {
              unpack2(b1p[a], b1_[2 * a], b1_[2 * a + 1]);
              unpack2(b2p[a], b2_[2 * a], b2_[2 * a + 1]);
            }
          } else {
            for (int k = K - 1; k >= 0; --k) {
              const float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
#pragma unroll
              for (int m = 0; m < KP; ++m) {
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
          for (int m = 0; m < KP; ++m) {
            // after the loop b1 = b_0 and b2 = b_1: sum = b_0 - conj(w) b_1
            const float wm1 = wm1_[m], wi = wi_[m], chi = chi_[m];
            const float sre = fmaf(-(wm1 + 1.0f), b2_[m], b1_[m]);
            const float sim = wi * b2_[m];
            // (w - 1)/(i chi - alpha) = (w - 1)(-alpha - i chi)/(alpha^2 + chi^2)
            const float inv = rcp_approx(fmaf(chi, chi, alpha2));
            const float qr = fmaf(-alpha, wm1, chi * wi) * inv;
            const float qi = fmaf(-chi, wm1, -alpha * wi) * inv;
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
              dsum = fmaf(wgt_[m], fmaf(mre, mre, mim * mim) * (ratio * ratio), dsum);
            } else {
              const float ang = (N - 1.0f) * x;
              const float sp = __sinf(ang), cp = __cosf(ang);
              const float yre = ratio * fmaf(mre, cp, -mim * sp);  // Upsilon / gamma
              const float yim = ratio * fmaf(mre, sp, mim * cp);
              if (ORD == ORD_DW) {
                dsum = fmaf(wgt_[m], fmaf(yre, yre, yim * yim), dsum);
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
              csum = fmaf(f3r.z * ow.w, gr_ * gr_ + gi_ * gi_, csum);
            }
          }
        }
        __syncthreads();  // rows and tables are rewritten by the next chunk
      }
      // ---- island reduction (fixed order); every sum above is of Upsilon / gamma
      if (!cplx) {
        float v = dsum;
        for (int o_ = 16; o_ > 0; o_ >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o_);
        if (lane == 0) red[0][wid] = v;
      } else {
        float vals[4] = {dsum, csum, hre, him};
#pragma unroll
        for (int a = 0; a < 4; ++a)
          for (int o_ = 16; o_ > 0; o_ >>= 1) vals[a] += __shfl_xor_sync(0xffffffffu, vals[a], o_);
        if (lane == 0)
#pragma unroll
          for (int a = 0; a < 4; ++a) red[a][wid] = vals[a];
      }
      __syncthreads();
      if (tid == 0) {
        const long long isl = bs.isl[ib];
        const float t0 = (red[0][0] + red[0][1]) + (red[0][2] + red[0][3]);
        if (ORD == ORD_DW) {
          terms[isl] = bs.cf0[ib] * g2 * t0;
          if (cplx) {
            const float t1 = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
            const float t2 = (red[2][0] + red[2][1]) + (red[2][2] + red[2][3]);
            const float t3 = (red[3][0] + red[3][1]) + (red[3][2] + red[3][3]);
            if (want_g) terms[3 * n_isl + isl] = bs.cf1[ib] * g2 * t1;
            if (want_h) terms[4 * n_isl + isl] = bs.cf2[ib] * g2 * (t2 * t2 + t3 * t3);
          }
        } else {
          const float t1 = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
          terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = bs.cf0[ib] * g2 * t1;
        }
      }
      __syncthreads();
    }
  }
}

template <int ORD, int KP>
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
  // static shared memory + the c_k table exceed the 48 KB default: opt in once per device
  static unsigned long long attr_done = 0;
  if (!(attr_done >> (dev & 63) & 1ull)) {
    cudaError_t e = cudaFuncSetAttribute(integrate_fp32c_kernel<ORD, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTabFloats * (int)sizeof(float));
    if (e != cudaSuccess) return e;
    attr_done |= 1ull << (dev & 63);
  }
  long long batches = (n_items + kBatch - 1) / kBatch;
  long long blocks = (long long)sms * (KP == 8 ? 3 : 4);
  if (blocks > batches) blocks = batches;
  // 2 pi L beta2 and 2 pi^2 L beta3 as double-floats
  double g0 = 2.0 * kPi * p.L * p.beta2, g1 = 2.0 * kPi * kPi * p.L * p.beta3;
  float g0h = (float)g0, g1h = (float)g1;
  Df G0 = {g0h, (float)(g0 - (double)g0h)}, G1 = {g1h, (float)(g1 - (double)g1h)};
  integrate_fp32c_kernel<ORD, KP><<<(unsigned)blocks, kThreads, smem, st>>>(p, keys, list, n_items, terms, n_isl,
                                                                           rows, kpad, G0, G1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp32c_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                              long long n_items, float* terms, long long n_isl, cudaStream_t st) {
  if (ord == ORD_DW) {
    if (p.fp32c_kp == 8) return launch_one<ORD_DW, 8>(p, keys, list, n_items, terms, n_isl, st);
    return launch_one<ORD_DW, 4>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (ord == ORD_E) return launch_one<ORD_E, 4>(p, keys, list, n_items, terms, n_isl, st);
  return launch_one<ORD_F, 4>(p, keys, list, n_items, terms, n_isl, st);
}

}  // namespace egn
