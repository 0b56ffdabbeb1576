// integrate_ridge32.cu -- the ridge-resolving node rule (ridge_rule.cuh) in the
// FP32 arithmetic of the fast path (FP32C), for links of identical spans and of
// up to kMaxTypes span types.
//
// Work decomposition: one warp (a 32-thread CTA) per island, as in the FP64 form
// of the rule.  The warp forms the island's outer pieces (FP64).  The lanes then
// take outer nodes ("rows") 32 at a time, one lane per row, and an island's last
// rows L lanes per row (L a power of two, so that the batch fills the warp): the
// lanes of a row form its inner pieces (FP64) and, in the DW order, its c_k =
// C_k e^{-zeta_k f3} in the row's column of a [K][32] shared table, and walk its
// nodes in groups of four points (the row's groups dealt out to its L lanes), two
// per fma.rn.f32x2 in the segment recurrence.
//
// Per piece the inner coordinate is t = t0 + t1 y, with y the piece variable: the
// Gauss-Legendre node x_j on a plain piece (t0 its midpoint, t1 its half-length),
// the offset h sinh(tau_j) from the ridge end on a graded one (t1 = +1 or -1).
// f1 - f, f2 - f and f1 + f2 are linear in y, so the phase of Eq. 5/24 is a
// polynomial in y whose coefficients are formed per piece in double-float
// (row_phase, Q0 reduced modulo K), and every point's phase is reduced exactly as
// on the configured rule (point_phase).  On a graded piece f1 - f (or f2 - f) is
// the offset itself plus a constant that vanishes to double-float rounding, so chi
// near the ridge keeps full relative precision.  The graded offsets are formed in
// FP32 (sinh and cosh from one ex2 and its reciprocal), and so are the ridge
// half-widths that scale them: a node lies within a few 1e-7 of its FP64 offset
// from the ridge (or of h), a perturbation of the rule, not of the integrand.  The cuts, their order and the node counts are the
// FP64 rule's (plain_nodes takes a count from FP32 only where it is unambiguous);
// GB300 runs FP64 at 1/64 of the FP32 rate, so the per-row and per-piece
// arithmetic beyond the cuts is double-float.
//
// Everything past the node (w, the segment sum, mu, the phased array, the sums)
// is the arithmetic of the configured rule's FP32C passes.
#include "egn_internal.h"

#include "fp32c_common.cuh"
#include "island_geom.cuh"
#include "ridge_rule.cuh"

namespace egn {
namespace {

using namespace fp32c;

constexpr int kGroup = 4;  // points per lane and step of the node walk

// Constants of one inner piece of a lane's row.
struct PieceC {
  float4 qa, qb;         // phase polynomial in y (point_phase)
  float a0, a1, b0, b1;  // f1 - f = a0 + a1 y, f2 - f = b0 + b1 y
  float k0, k1;          // 4 pi^2 (beta2 + pi beta3 (f1 + f2)) = k0 + k1 y
  float u0, u1, v0, v1;  // shape coordinates u = u0 + u1 y, v = v0 + v1 y
  float w0, w1;          // w = w0 + w1 y (E and F; DW: the row's)
  float T2, h, wsc;      // graded: tau = T2 (x + 1), y = h sinh(tau), weight wsc w_j cosh(tau); plain: weight wsc w_j
  int m, goff;           // nodes; offset of the order-m rule in the node tables
  bool graded;
};

// The island's frequencies relative to the COI as double-floats: F1 = nu1 - f,
// F2 = nu2 - f, S12 = nu1 + nu2; the FP32 constants of chi.
struct IslandDf {
  Df F1, F2, S12;
  float k4, b2, pib3;  // 4 pi^2, beta2, pi beta3
};

// Type-independent constants of inner piece q of the row at outer node o (od,
// md: o and the coupling centre m as double-floats): the linear forms of f1 - f,
// f2 - f and f1 + f2 in y, the shape coordinates and the node map.  Per piece
// only the ends are converted from FP64; the rest is double-float and FP32.
struct PieceGeo {
  RowGeo r;              // a0, a1, b0, b1, s0, s1
  Df u0, u1, v0, v1, w0, w1;
  float T2, h, wsc;
  int m, goff;
  bool graded;
};

template <int ORD>
__device__ __forceinline__ PieceGeo piece_geom(const IslandDf& isd, const RPiece& q, Df od, Df md) {
  PieceGeo c;
  c.graded = q.ha > 0.0 || q.hb > 0.0;
  c.m = q.m;
  c.goff = q.m * (q.m - 1) / 2;
  Df t0, t1;
  if (c.graded) {
    const bool at_a = q.ha > 0.0;
    c.h = (float)(at_a ? q.ha : q.hb);
    t0 = df_of(at_a ? q.a : q.b);
    t1 = {at_a ? 1.0f : -1.0f, 0.0f};
    c.T2 = 0.5f * asinhf(__fdividef((float)(q.b - q.a), c.h));
    c.wsc = c.T2 * c.h;
  } else {
    const Df A = df_of(q.a), B = df_of(q.b);
    t0 = dhalf(dadd(A, B));
    t1 = dhalf(dsub(B, A));
    c.T2 = 0.0f;
    c.h = 0.0f;
    c.wsc = dval(t1);
  }
  const Df zero = {0.0f, 0.0f};
  if (ORD == ORD_DW) {  // u = t, v = m - t, w = o
    c.u0 = t0; c.u1 = t1; c.v0 = dsub(md, t0); c.v1 = dneg(t1); c.w0 = od; c.w1 = zero;
    c.r.s0 = dadd(isd.S12, md); c.r.s1 = zero;
  } else if (ORD == ORD_E) {  // u = t, v = o, w = t - m
    c.u0 = t0; c.u1 = t1; c.v0 = od; c.v1 = zero; c.w0 = dsub(t0, md); c.w1 = t1;
    c.r.s0 = dadd(isd.S12, dadd(od, t0)); c.r.s1 = t1;
  } else {  // u = o, v = t, w = t - m
    c.u0 = od; c.u1 = zero; c.v0 = t0; c.v1 = t1; c.w0 = dsub(t0, md); c.w1 = t1;
    c.r.s0 = dadd(isd.S12, dadd(od, t0)); c.r.s1 = t1;
  }
  c.r.a0 = dadd(isd.F1, c.u0); c.r.a1 = c.u1;
  c.r.b0 = dadd(isd.F2, c.v0); c.r.b1 = c.v1;
  return c;
}

// Constants of inner piece q for links of identical spans: the geometry and the
// phase polynomial of the span (G0 = 2 pi L beta2, G1 = 2 pi^2 L beta3).
template <int ORD>
__device__ __forceinline__ PieceC piece_consts(const IslandDf& isd, const RPiece& q, Df od, Df md, Df G0, Df G1,
                                               float Kf, float invK) {
  const PieceGeo gq = piece_geom<ORD>(isd, q, od, md);
  PieceC c;
  c.graded = gq.graded;
  c.m = gq.m;
  c.goff = gq.goff;
  c.T2 = gq.T2;
  c.h = gq.h;
  c.wsc = gq.wsc;
  const RowPhase ph = row_phase(gq.r, G0, G1, Kf, invK);
  c.qa = make_float4(ph.Q0r.hi, ph.Q0r.lo, ph.Q1.hi, ph.Q1.lo);
  c.qb = make_float4(ph.Q2.hi, ph.Q2.lo, ph.Q3, ph.Q0r.hi - rint_fast(ph.Q0r.hi));
  c.a0 = dval(gq.r.a0); c.a1 = dval(gq.r.a1);
  c.b0 = dval(gq.r.b0); c.b1 = dval(gq.r.b1);
  c.k0 = isd.k4 * fmaf(isd.pib3, dval(gq.r.s0), isd.b2);
  c.k1 = isd.k4 * isd.pib3 * dval(gq.r.s1);
  c.u0 = dval(gq.u0); c.u1 = dval(gq.u1);
  c.v0 = dval(gq.v0); c.v1 = dval(gq.v1);
  c.w0 = dval(gq.w0); c.w1 = dval(gq.w1);
  return c;
}

template <int ORD>
__global__ void __launch_bounds__(32) integrate_ridge_fp32c_kernel(LinkParams p, const uint64_t* __restrict__ keys,
                                                                   const uint32_t* __restrict__ list,
                                                                   long long n_items, float* __restrict__ terms,
                                                                   long long n_isl, Df G0, Df G1) {
  extern __shared__ float ck_s[];  // DW: [K][32], the c_k of each lane's row
  __shared__ RPiece opc[kOuterPieces];
  __shared__ int ocum[kOuterPieces + 1];
  __shared__ double osx[kOuterCuts], osh[kOuterCuts];  // scratch of ridge_outer_pieces_warp
  const int lane = threadIdx.x;
  const DwConsts cst = dw_consts(p);
  const int K = cst.K;
  const float Kf = cst.Kf, invK = cst.invK, alpha = cst.alpha, alpha2 = cst.alpha2, one_m_r = cst.one_m_r;
  const float q = cst.q, m2r = cst.m2r, N = cst.N;
  const float pi_f = 3.14159265358979f;
  const int n = p.gl.n, n_min = p.ridge_n_min;
  const double be = p.rolloff;
  const ChannelTable& ch = p.ch;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    const RidgeIsland g = ridge_island<ORD>(ch, coi, n1, n2, n3, p.rolloff, p.alpha, p.beta2, p.beta3);
    const int npc = ridge_outer_pieces_warp<ORD>(g, n, n_min, opc, ocum, osx, osh, lane);
    const int rows = ocum[npc];
    const bool want_g = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_g(n1, n2, n3)));
    const bool want_h = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_h(n1, n2, n3)));
    const bool cplx = ORD != ORD_DW || want_g || want_h;
    // raised-cosine knees and 1/(beta R) of the three shapes (rc_f)
    const float ra1 = (float)(0.5 * (1.0 - be) * g.R1), ra2 = (float)(0.5 * (1.0 - be) * g.R2);
    const float ra3 = (float)(0.5 * (1.0 - be) * g.R3);
    const float ri1 = be > 0.0 ? (float)(1.0 / (be * g.R1)) : 0.0f, ri2 = be > 0.0 ? (float)(1.0 / (be * g.R2)) : 0.0f;
    const float ri3 = be > 0.0 ? (float)(1.0 / (be * g.R3)) : 0.0f;
    const float nu3f = (float)g.nu3;
    IslandDf isd;
    isd.F1 = df_of(g.nu1 - g.f);
    isd.F2 = df_of(g.nu2 - g.f);
    isd.S12 = df_of(g.nu1 + g.nu2);
    isd.k4 = (float)(4.0 * kPi * kPi);
    isd.b2 = (float)p.beta2;
    isd.pib3 = (float)(kPi * p.beta3);
    const float rao = ORD == ORD_DW ? ra3 : (ORD == ORD_E ? ra2 : ra1);
    const float rio = ORD == ORD_DW ? ri3 : (ORD == ORD_E ? ri2 : ri1);
    float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
    // Rows in batches of up to 32, L lanes per row: L = 1 while at least 32 rows
    // are left, else the largest power of two that keeps the batch within the warp
    // (an island's last rows get several lanes each, which take the node groups of
    // every piece in turn).
    for (int base = 0; base < rows;) {
      const int left = rows - base;
      int L = 1;
      while (L < 32 && 2 * L * left <= 32) L <<= 1;
      const int nrow = min(left, 32 / L);
      const int rsub = lane / L, lsub = lane & (L - 1);
      const int row = base + rsub;
      bool act = rsub < nrow;
      double o = 0.0, wod = 0.0, m = 0.0;
      RPiece ipc[kInnerPieces];
      int nip = 0;
      if (act) {
        int qo = 0;
        while (ocum[qo + 1] <= row) ++qo;
        piece_node(opc[qo], row - ocum[qo], p.glx_all, p.glw_all, o, wod);
        nip = ridge_inner_pieces<ORD, true>(g, o, n, n_min, ipc, m);
        act = nip > 0;
      }
      const float wo = (float)wod;
      const Df od = df_of(o), md = df_of(m);
      const float hout = rc_f(dval(od), rao, rio);
      const int colx = rsub * L;  // the row's column of the c_k table
      if (ORD == ORD_DW) {
        if (act) {
          const float f3 = nu3f + dval(od);
          for (int k = lsub; k < K; k += L) ck_s[k * 32 + colx] = p.seg.ck_f[k] * ex2_approx(-p.seg.zeta_f[k] * f3);
        }
        __syncwarp();
      }
      const float* col = ck_s + colx;
      float gre = 0.0f, gim = 0.0f;  // this lane's part of the row's inner sum (G of DW, E, F)
      for (int ip = 0; act && ip < nip; ++ip) {
        const PieceC pc = piece_consts<ORD>(isd, ipc[ip], od, md, G0, G1, Kf, invK);
        for (int j0 = lsub * kGroup; j0 < pc.m; j0 += L * kGroup) {
          float p_[kGroup], b1_[kGroup], b2_[kGroup], f3_[kGroup];
          float wm1_[kGroup], wi_[kGroup], chi_[kGroup], phi_[kGroup], wD_[kGroup], wG_[kGroup], wH_[kGroup];
#pragma unroll
          for (int e = 0; e < kGroup; ++e) {
            const int j = j0 + e;
            const bool valid = j < pc.m;
            const int jj = pc.goff + (valid ? j : pc.m - 1);  // a repeated node of weight 0 pads the group
            const float xh = p.glxh_all[jj], wj = p.glwf_all[jj];
            float yh, yl, wn;
            if (pc.graded) {
              const float tau = fmaf(pc.T2, xh, pc.T2);
              // sinh and cosh from one exponential: e^tau by ex2, e^-tau by rcp (absolute
              // error ~2e-7 e^tau: the offset moves by about 1e-7 h near the ridge and
              // by a few 1e-7 of itself far from it)
              const float ep = ex2_approx(tau * 1.44269504f), em = rcp_approx(ep);
              yh = pc.h * (0.5f * (ep - em));
              yl = 0.0f;
              wn = pc.wsc * wj * (0.5f * (ep + em));
            } else {
              yh = xh;
              yl = p.glxl_all[jj];
              wn = pc.wsc * wj;
            }
            wn = valid ? wn : 0.0f;
            const float y2h = yh * yh;
            const float y2l = fmaf(2.0f * yh, yl, fmaf(yh, yh, -y2h));
            float th, ph;
            point_phase(pc.qa, pc.qb, make_float4(yh, yl, y2h, y2l), y2h * yh, Kf, invK, th, ph);
            // w = r e^{2 pi i th} from the half angle (keeps w - 1 accurate)
            const float ah = pi_f * th;
            const float sh = __sinf(ah), chh = __cosf(ah);
            const float t2r = m2r * sh;
            const float wm1 = fmaf(t2r, sh, -one_m_r);
            p_[e] = fmaf(2.0f, wm1, 2.0f);
            wm1_[e] = wm1;
            wi_[e] = -t2r * chh;
            phi_[e] = ph;
            chi_[e] = fmaf(pc.a1, yh, pc.a0) * fmaf(pc.b1, yh, pc.b0) * fmaf(pc.k1, yh, pc.k0);
            const float u = fmaf(pc.u1, yh, pc.u0), v = fmaf(pc.v1, yh, pc.v0), w = fmaf(pc.w1, yh, pc.w0);
            const float h1 = rc_f(u, ra1, ri1), h2 = rc_f(v, ra2, ri2);
            const float h3 = ORD == ORD_DW ? hout : rc_f(w, ra3, ri3);
            wD_[e] = wo * wn * h1 * h2 * h3;
            wH_[e] = wo * wn * sqrtf(h1 * h2 * h3);
            wG_[e] = wn * (ORD == ORD_DW ? sqrtf(h1 * h2) : (ORD == ORD_E ? sqrtf(h1 * h3) : sqrtf(h2 * h3)));
            f3_[e] = nu3f + w;
            b1_[e] = 0.0f;
            b2_[e] = 0.0f;
          }
          // ---- segment sum, b_k = c_k + p b_{k+1} - q b_{k+2}, k = K-1 .. 0
          if (ORD == ORD_DW) {
            f32x2 pp[kGroup / 2], b1p[kGroup / 2], b2p[kGroup / 2];
#pragma unroll
            for (int a = 0; a < kGroup / 2; ++a) {
              pp[a] = pack2(p_[2 * a], p_[2 * a + 1]);
              b1p[a] = 0ull;
              b2p[a] = 0ull;
            }
            const f32x2 nq2 = pack2(-q, -q);
#pragma unroll 4
            for (int k = K - 1; k >= 0; --k) {
              const float c = col[k * 32];
              const f32x2 cc = pack2(c, c);
#pragma unroll
              for (int a = 0; a < kGroup / 2; ++a) {
                const f32x2 nb = ffma2(pp[a], b1p[a], ffma2(nq2, b2p[a], cc));
                b2p[a] = b1p[a];
                b1p[a] = nb;
              }
            }
#pragma unroll
            for (int a = 0; a < kGroup / 2; ++a) {
              unpack2(b1p[a], b1_[2 * a], b1_[2 * a + 1]);
              unpack2(b2p[a], b2_[2 * a], b2_[2 * a + 1]);
            }
          } else {
            // c_k per point (f3 varies along the row)
#pragma unroll 2
            for (int k = K - 1; k >= 0; --k) {
              const float ck = p.seg.ck_f[k], zk = p.seg.zeta_f[k];
#pragma unroll
              for (int e = 0; e < kGroup; ++e) {
                const float c = ck * ex2_approx(-zk * f3_[e]);
                const float bn = fmaf(p_[e], b1_[e], fmaf(-q, b2_[e], c));
                b2_[e] = b1_[e];
                b1_[e] = bn;
              }
            }
          }
          // ---- mu, Upsilon / gamma and the sums
#pragma unroll
          for (int e = 0; e < kGroup; ++e) {
            const float wm1 = wm1_[e], wi = wi_[e], chi = chi_[e];
            const float sre = fmaf(-(wm1 + 1.0f), b2_[e], b1_[e]);  // b_0 - conj(w) b_1
            const float sim = wi * b2_[e];
            const float inv = rcp_approx(fmaf(chi, chi, alpha2));    // (w - 1)/(i chi - alpha)
            const float qr = fmaf(-alpha, wm1, chi * wi) * inv;
            const float qi = fmaf(-chi, wm1, -alpha * wi) * inv;
            const float mre = fmaf(sre, qr, -sim * qi);
            const float mim = fmaf(sre, qi, sim * qr);
            const float x = pi_f * phi_[e];
            const float ratio = array_ratio(x, N);
            if (!cplx) {
              dsum = fmaf(wD_[e], fmaf(mre, mre, mim * mim) * (ratio * ratio), dsum);
            } else {
              const float ang = (N - 1.0f) * x;
              const float sp = __sinf(ang), cp = __cosf(ang);
              const float yre = ratio * fmaf(mre, cp, -mim * sp);
              const float yim = ratio * fmaf(mre, sp, mim * cp);
              if (ORD == ORD_DW) {
                dsum = fmaf(wD_[e], fmaf(yre, yre, yim * yim), dsum);
                hre = fmaf(wH_[e], yre, hre);
                him = fmaf(wH_[e], yim, him);
              }
              gre = fmaf(wG_[e], yre, gre);
              gim = fmaf(wG_[e], yim, gim);
            }
          }
        }
      }
      for (int o_ = 1; o_ < L; o_ <<= 1) {  // the row's inner sum over its L lanes
        gre += __shfl_xor_sync(0xffffffffu, gre, o_);
        gim += __shfl_xor_sync(0xffffffffu, gim, o_);
      }
      if (act && lsub == 0 && (ORD != ORD_DW || want_g)) csum = fmaf(wo * hout, fmaf(gre, gre, gim * gim), csum);
      if (ORD == ORD_DW) __syncwarp();  // the table is rewritten by the next batch
      base += nrow;
    }
    for (int o_ = 16; o_ > 0; o_ >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o_);
      csum += __shfl_xor_sync(0xffffffffu, csum, o_);
      hre += __shfl_xor_sync(0xffffffffu, hre, o_);
      him += __shfl_xor_sync(0xffffffffu, him, o_);
    }
    if (lane == 0) {
      double cf[5];
      term_coefs(ch.R[coi], g.R1, g.R2, g.R3, cf);
      const double g2 = (double)cst.g2;
      if (ORD == ORD_DW) {
        terms[isl] = (float)(cf[0] * g2 * dsum);
        if (want_g) terms[3 * n_isl + isl] = (float)(cf[3] * g2 * csum);
        if (want_h) terms[4 * n_isl + isl] = (float)(cf[4] * g2 * ((double)hre * hre + (double)him * him));
      } else {
        terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = (float)(cf[ORD == ORD_E ? 1 : 2] * g2 * csum);
      }
    }
    __syncwarp();  // the outer pieces are rewritten for the next island
  }
}

// Links of 2..kMaxTypes span types (Eq. 22 summed span by span): per point and
// type the phase, mu_t and e^{2 pi i phi_t}, then the coherent sum over the spans
// in their order, as in the configured rule's general passes.  Two points per
// group; each lane keeps its current piece's per-type phase polynomials in its
// own shared-memory slots.  In the DW order the c_k of every type for each lane's
// row sit in a [K_1 + .. + K_T][32] shared table.
constexpr int kGroupT = 2;

template <int ORD>
__global__ void __launch_bounds__(32) integrate_ridge_fp32c_types_kernel(LinkParams p, const uint64_t* __restrict__ keys,
                                                                         const uint32_t* __restrict__ list,
                                                                         long long n_items, float* __restrict__ terms,
                                                                         long long n_isl) {
  extern __shared__ float ck_s[];  // DW: [sum of K_t][32]
  __shared__ RPiece opc[kOuterPieces];
  __shared__ int ocum[kOuterPieces + 1];
  __shared__ double osx[kOuterCuts], osh[kOuterCuts];  // scratch of ridge_outer_pieces_warp
  __shared__ float4 qa_s[kMaxTypes][32], qb_s[kMaxTypes][32];  // each lane's current piece, per type
  __shared__ float2 kk_s[kMaxTypes][32];                       // 4 pi^2 (beta2_t + pi beta3_t (f1 + f2)) = x + y y
  __shared__ float tyf[kMaxTypes][8];                          // K, 1/K, alpha, r, 1 - r, gamma, beta2, pi beta3
  __shared__ Df tyg[kMaxTypes][2];                             // 2 pi L beta2, 2 pi^2 L beta3
  __shared__ int koff[kMaxTypes];
  const int lane = threadIdx.x;
  const int T = p.n_types;
  if (lane < T) {
    const SpanType& ty = p.types[lane];
    tyf[lane][0] = (float)ty.seg.K;
    tyf[lane][1] = 1.0f / (float)ty.seg.K;
    tyf[lane][2] = (float)ty.alpha;
    tyf[lane][3] = (float)ty.r;
    tyf[lane][4] = (float)(-expm1(-ty.alpha * ty.dz));
    tyf[lane][5] = (float)ty.gamma;
    tyf[lane][6] = (float)ty.beta2;
    tyf[lane][7] = (float)(kPi * ty.beta3);
    const double g0 = 2.0 * kPi * ty.L * ty.beta2, g1 = 2.0 * kPi * kPi * ty.L * ty.beta3;
    tyg[lane][0] = df_of(g0);
    tyg[lane][1] = df_of(g1);
  }
  if (lane == 0) {
    int o = 0;
    for (int t = 0; t < T; ++t) {
      koff[t] = o;
      o += p.types[t].seg.K;
    }
  }
  __syncwarp();
  const float pi_f = 3.14159265358979f, k4 = (float)(4.0 * kPi * kPi);
  const int n = p.gl.n, n_min = p.ridge_n_min;
  const double be = p.rolloff;
  const ChannelTable& ch = p.ch;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const long long isl = list ? (long long)list[it] : it;
    int coi, n1, n2, n3;
    unpack_key(keys[isl], coi, n1, n2, n3);
    const RidgeIsland g = ridge_island<ORD>(ch, coi, n1, n2, n3, p.rolloff, p.alpha, p.beta2, p.beta3);
    const int npc = ridge_outer_pieces_warp<ORD>(g, n, n_min, opc, ocum, osx, osh, lane);
    const int rows = ocum[npc];
    const bool want_g = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_g(n1, n2, n3)));
    const bool want_h = (ORD == ORD_DW) && (p.all_terms || (p.terms && flag_h(n1, n2, n3)));
    const float ra1 = (float)(0.5 * (1.0 - be) * g.R1), ra2 = (float)(0.5 * (1.0 - be) * g.R2);
    const float ra3 = (float)(0.5 * (1.0 - be) * g.R3);
    const float ri1 = be > 0.0 ? (float)(1.0 / (be * g.R1)) : 0.0f, ri2 = be > 0.0 ? (float)(1.0 / (be * g.R2)) : 0.0f;
    const float ri3 = be > 0.0 ? (float)(1.0 / (be * g.R3)) : 0.0f;
    const float nu3f = (float)g.nu3;
    IslandDf isd;
    isd.F1 = df_of(g.nu1 - g.f);
    isd.F2 = df_of(g.nu2 - g.f);
    isd.S12 = df_of(g.nu1 + g.nu2);
    isd.k4 = k4;
    isd.b2 = (float)p.beta2;
    isd.pib3 = (float)(kPi * p.beta3);
    const float rao = ORD == ORD_DW ? ra3 : (ORD == ORD_E ? ra2 : ra1);
    const float rio = ORD == ORD_DW ? ri3 : (ORD == ORD_E ? ri2 : ri1);
    float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
    for (int base = 0; base < rows;) {  // row batches and lanes per row as in the identical-spans kernel
      const int left = rows - base;
      int L = 1;
      while (L < 32 && 2 * L * left <= 32) L <<= 1;
      const int nrow = min(left, 32 / L);
      const int rsub = lane / L, lsub = lane & (L - 1);
      const int row = base + rsub;
      bool act = rsub < nrow;
      double o = 0.0, wod = 0.0, m = 0.0;
      RPiece ipc[kInnerPieces];
      int nip = 0;
      if (act) {
        int qo = 0;
        while (ocum[qo + 1] <= row) ++qo;
        piece_node(opc[qo], row - ocum[qo], p.glx_all, p.glw_all, o, wod);
        nip = ridge_inner_pieces<ORD, true>(g, o, n, n_min, ipc, m);
        act = nip > 0;
      }
      const float wo = (float)wod;
      const Df od = df_of(o), md = df_of(m);
      const float hout = rc_f(dval(od), rao, rio);
      const int colx = rsub * L;
      if (ORD == ORD_DW) {
        if (act) {
          const float f3 = nu3f + dval(od);
          for (int t = 0; t < T; ++t) {
            const SegmentTables& sg = p.types[t].seg;
            for (int k = lsub; k < sg.K; k += L)
              ck_s[(koff[t] + k) * 32 + colx] = sg.ck_f[k] * ex2_approx(-sg.zeta_f[k] * f3);
          }
        }
        __syncwarp();
      }
      float gre = 0.0f, gim = 0.0f;
      for (int ip = 0; act && ip < nip; ++ip) {
        const PieceGeo gq = piece_geom<ORD>(isd, ipc[ip], od, md);
        for (int t = 0; t < T; ++t) {
          const RowPhase ph = row_phase(gq.r, tyg[t][0], tyg[t][1], tyf[t][0], tyf[t][1]);
          qa_s[t][lane] = make_float4(ph.Q0r.hi, ph.Q0r.lo, ph.Q1.hi, ph.Q1.lo);
          qb_s[t][lane] = make_float4(ph.Q2.hi, ph.Q2.lo, ph.Q3, ph.Q0r.hi - rint_fast(ph.Q0r.hi));
          kk_s[t][lane] = make_float2(k4 * fmaf(tyf[t][7], dval(gq.r.s0), tyf[t][6]), k4 * tyf[t][7] * dval(gq.r.s1));
        }
        const float a0 = dval(gq.r.a0), a1 = dval(gq.r.a1), b0 = dval(gq.r.b0), b1 = dval(gq.r.b1);
        const float u0 = dval(gq.u0), u1 = dval(gq.u1), v0 = dval(gq.v0), v1 = dval(gq.v1);
        const float w0 = dval(gq.w0), w1 = dval(gq.w1);
        for (int j0 = lsub * kGroupT; j0 < gq.m; j0 += L * kGroupT) {
          float y4_[kGroupT][4], y3_[kGroupT], wD_[kGroupT], wG_[kGroupT], wH_[kGroupT], f3_[kGroupT];
          float yre_[kGroupT], yim_[kGroupT], ys_[kGroupT];
#pragma unroll
          for (int e = 0; e < kGroupT; ++e) {
            const int j = j0 + e;
            const bool valid = j < gq.m;
            const int jj = gq.goff + (valid ? j : gq.m - 1);  // a repeated node of weight 0 pads the group
            const float xh = p.glxh_all[jj], wj = p.glwf_all[jj];
            float yh, yl, wn;
            if (gq.graded) {
              const float tau = fmaf(gq.T2, xh, gq.T2);
              const float ep = ex2_approx(tau * 1.44269504f), em = rcp_approx(ep);
              yh = gq.h * (0.5f * (ep - em));
              yl = 0.0f;
              wn = gq.wsc * wj * (0.5f * (ep + em));
            } else {
              yh = xh;
              yl = p.glxl_all[jj];
              wn = gq.wsc * wj;
            }
            wn = valid ? wn : 0.0f;
            const float y2h = yh * yh;
            y4_[e][0] = yh;
            y4_[e][1] = yl;
            y4_[e][2] = y2h;
            y4_[e][3] = fmaf(2.0f * yh, yl, fmaf(yh, yh, -y2h));
            y3_[e] = y2h * yh;
            ys_[e] = yh;
            const float u = fmaf(u1, yh, u0), v = fmaf(v1, yh, v0), w = fmaf(w1, yh, w0);
            const float h1 = rc_f(u, ra1, ri1), h2 = rc_f(v, ra2, ri2);
            const float h3 = ORD == ORD_DW ? hout : rc_f(w, ra3, ri3);
            wD_[e] = wo * wn * h1 * h2 * h3;
            wH_[e] = wo * wn * sqrtf(h1 * h2 * h3);
            wG_[e] = wn * (ORD == ORD_DW ? sqrtf(h1 * h2) : (ORD == ORD_E ? sqrtf(h1 * h3) : sqrtf(h2 * h3)));
            f3_[e] = nu3f + w;
            yre_[e] = 0.0f;
            yim_[e] = 0.0f;
          }
          // per span type: gamma_t mu_t and e^{2 pi i phi_t}, kept for the span sum
          float mre_[kMaxTypes][kGroupT], mim_[kMaxTypes][kGroupT], ere_[kMaxTypes][kGroupT], eim_[kMaxTypes][kGroupT];
#pragma unroll
          for (int t = 0; t < kMaxTypes; ++t) {
            if (t >= T) break;
            const float4 qa = qa_s[t][lane], qb = qb_s[t][lane];
            const float2 kk = kk_s[t][lane];
            const float Kf = tyf[t][0], invK = tyf[t][1], alpha = tyf[t][2], r = tyf[t][3], omr = tyf[t][4],
                        gam = tyf[t][5];
            const int K = (int)Kf;
            const float q = r * r;
            float p_[kGroupT], wm1_[kGroupT], wi_[kGroupT], chi_[kGroupT], b1_[kGroupT], b2_[kGroupT];
#pragma unroll
            for (int e = 0; e < kGroupT; ++e) {
              float th, ph;
              point_phase(qa, qb, make_float4(y4_[e][0], y4_[e][1], y4_[e][2], y4_[e][3]), y3_[e], Kf, invK, th, ph);
              const float ah = pi_f * th;
              const float sh = __sinf(ah), chh = __cosf(ah);
              const float t2r = -2.0f * r * sh;
              wm1_[e] = fmaf(t2r, sh, -omr);
              p_[e] = fmaf(2.0f, wm1_[e], 2.0f);
              wi_[e] = -t2r * chh;
              const float yh = ys_[e];
              chi_[e] = fmaf(a1, yh, a0) * fmaf(b1, yh, b0) * fmaf(kk.y, yh, kk.x);
              const float ang = 2.0f * pi_f * ph;
              ere_[t][e] = __cosf(ang);
              eim_[t][e] = __sinf(ang);
              b1_[e] = 0.0f;
              b2_[e] = 0.0f;
            }
            if (ORD == ORD_DW) {
              const float* trow = ck_s + koff[t] * 32 + colx;
              for (int k = K - 1; k >= 0; --k) {
                const float c = trow[k * 32];
#pragma unroll
                for (int e = 0; e < kGroupT; ++e) {
                  const float bn = fmaf(p_[e], b1_[e], fmaf(-q, b2_[e], c));
                  b2_[e] = b1_[e];
                  b1_[e] = bn;
                }
              }
            } else {  // c_k per point (f3 varies along the row)
              const float* ckf = p.types[t].seg.ck_f;
              const float* zkf = p.types[t].seg.zeta_f;
              for (int k = K - 1; k >= 0; --k) {
                const float ck = ckf[k], zk = zkf[k];
#pragma unroll
                for (int e = 0; e < kGroupT; ++e) {
                  const float c = ck * ex2_approx(-zk * f3_[e]);
                  const float bn = fmaf(p_[e], b1_[e], fmaf(-q, b2_[e], c));
                  b2_[e] = b1_[e];
                  b1_[e] = bn;
                }
              }
            }
#pragma unroll
            for (int e = 0; e < kGroupT; ++e) {
              const float wm1 = wm1_[e], wi = wi_[e], chi = chi_[e];
              const float sre = fmaf(-(wm1 + 1.0f), b2_[e], b1_[e]);  // b_0 - conj(w) b_1
              const float sim = wi * b2_[e];
              const float inv = rcp_approx(fmaf(chi, chi, alpha * alpha)) * gam;
              const float qr = fmaf(-alpha, wm1, chi * wi) * inv;
              const float qi = fmaf(-chi, wm1, -alpha * wi) * inv;
              mre_[t][e] = fmaf(sre, qr, -sim * qi);  // gamma_t mu_t
              mim_[t][e] = fmaf(sre, qi, sim * qr);
            }
          }
          // coherent sum over the spans in their order: Y = sum_s gamma_t mu_t e^{i Phi_s}
          float zre_[kGroupT], zim_[kGroupT];
#pragma unroll
          for (int e = 0; e < kGroupT; ++e) {
            zre_[e] = 1.0f;
            zim_[e] = 0.0f;
          }
          for (int sp = 0; sp < p.n_spans; ++sp) {
            const int t = p.span_type[sp];
#pragma unroll
            for (int e = 0; e < kGroupT; ++e) {
              float mr = 0.0f, mi = 0.0f, er = 1.0f, ei = 0.0f;
#pragma unroll
              for (int u = 0; u < kMaxTypes; ++u)
                if (u == t) { mr = mre_[u][e]; mi = mim_[u][e]; er = ere_[u][e]; ei = eim_[u][e]; }
              yre_[e] = fmaf(mr, zre_[e], fmaf(-mi, zim_[e], yre_[e]));
              yim_[e] = fmaf(mr, zim_[e], fmaf(mi, zre_[e], yim_[e]));
              const float zr = fmaf(zre_[e], er, -zim_[e] * ei);
              zim_[e] = fmaf(zre_[e], ei, zim_[e] * er);
              zre_[e] = zr;
            }
          }
#pragma unroll
          for (int e = 0; e < kGroupT; ++e) {
            const float yre = yre_[e], yim = yim_[e];
            if (ORD == ORD_DW) {
              dsum = fmaf(wD_[e], fmaf(yre, yre, yim * yim), dsum);
              if (want_h) {
                hre = fmaf(wH_[e], yre, hre);
                him = fmaf(wH_[e], yim, him);
              }
            }
            gre = fmaf(wG_[e], yre, gre);
            gim = fmaf(wG_[e], yim, gim);
          }
        }
      }
      for (int o_ = 1; o_ < L; o_ <<= 1) {  // the row's inner sum over its L lanes
        gre += __shfl_xor_sync(0xffffffffu, gre, o_);
        gim += __shfl_xor_sync(0xffffffffu, gim, o_);
      }
      if (act && lsub == 0 && (ORD != ORD_DW || want_g)) csum = fmaf(wo * hout, fmaf(gre, gre, gim * gim), csum);
      if (ORD == ORD_DW) __syncwarp();  // the table is rewritten by the next batch
      base += nrow;
    }
    for (int o_ = 16; o_ > 0; o_ >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o_);
      csum += __shfl_xor_sync(0xffffffffu, csum, o_);
      hre += __shfl_xor_sync(0xffffffffu, hre, o_);
      him += __shfl_xor_sync(0xffffffffu, him, o_);
    }
    if (lane == 0) {  // every sum above is of Upsilon itself (gamma included)
      double cf[5];
      term_coefs(ch.R[coi], g.R1, g.R2, g.R3, cf);
      if (ORD == ORD_DW) {
        terms[isl] = (float)(cf[0] * dsum);
        if (want_g) terms[3 * n_isl + isl] = (float)(cf[3] * csum);
        if (want_h) terms[4 * n_isl + isl] = (float)(cf[4] * ((double)hre * hre + (double)him * him));
      } else {
        terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = (float)(cf[ORD == ORD_E ? 1 : 2] * csum);
      }
    }
    __syncwarp();  // the outer pieces are rewritten for the next island
  }
}

template <int ORD>
cudaError_t launch_types(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                         float* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  int ksum = 0;
  for (int t = 0; t < p.n_types; ++t) ksum += p.types[t].seg.K;
  const size_t smem = ORD == ORD_DW ? (size_t)ksum * 32 * sizeof(float) : 0;
  static std::atomic<unsigned long long> attr_done{0};  // per device
  if (smem > 32 * 1024)
    if (cudaError_t e = opt_in_smem(integrate_ridge_fp32c_types_kernel<ORD>, (int)(kMaxKSum * 32 * sizeof(float)),
                                    attr_done))
      return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrate_ridge_fp32c_types_kernel<ORD>,
                                                                    32, smem))
    return e;
  long long blocks = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > n_items) blocks = n_items;
  integrate_ridge_fp32c_types_kernel<ORD><<<(unsigned)blocks, 32, smem, st>>>(p, keys, list, n_items, terms, n_isl);
  return cudaGetLastError();
}

template <int ORD>
cudaError_t launch_ord(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                       float* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = ORD == ORD_DW ? (size_t)p.seg.K * 32 * sizeof(float) : 0;
  static std::atomic<unsigned long long> attr_done{0};  // per device
  if (smem > 40 * 1024)
    if (cudaError_t e = opt_in_smem(integrate_ridge_fp32c_kernel<ORD>, (int)(kMaxK * 32 * sizeof(float)), attr_done))
      return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (long long)sms * 16;
  if (blocks > n_items) blocks = n_items;
  const double g0 = 2.0 * kPi * p.L * p.beta2, g1 = 2.0 * kPi * kPi * p.L * p.beta3;
  const float g0h = (float)g0, g1h = (float)g1;
  const Df G0 = {g0h, (float)(g0 - (double)g0h)}, G1 = {g1h, (float)(g1 - (double)g1h)};
  integrate_ridge_fp32c_kernel<ORD><<<(unsigned)blocks, 32, smem, st>>>(p, keys, list, n_items, terms, n_isl, G0, G1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ridge_fp32c(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                               long long n_items, float* terms, long long n_isl, cudaStream_t st) {
  if (p.n_types < 1 || p.n_types > kMaxTypes || p.mu_form != MU_SEGMENT)
    return cudaErrorInvalidValue;  // refused by the option checks
  if (p.n_types > 1) {
    if (ord == ORD_DW) return launch_types<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
    if (ord == ORD_E) return launch_types<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
    return launch_types<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (ord == ORD_DW) return launch_ord<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
  if (ord == ORD_E) return launch_ord<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
  return launch_ord<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
}

}  // namespace egn
