// integrate_fp32c.cu -- FP32 island integrator with exact phase reduction (the
// fast path).
//
// Work decomposition.  Links of identical spans: 64-thread CTAs (10 per SM) take
// islands in batches of 16; links whose spans differ: 128-thread CTAs, batches of
// 128.
//  1. Batch set-up (FP64, one island per thread): geometry of the node rule,
//     panel edges and the island constants, rounded to FP32 head/tail pairs
//     ("double-float", 48-bit significand).  GB300 runs FP64 at 1/64 of the FP32
//     rate, so FP64 appears only here.
//  2. Per island, per chunk of outer nodes ("rows"): the row constants in
//     double-float arithmetic (FP32 only) -- the cubic phase polynomial in the
//     inner node, Q0 reduced modulo K -- one row per thread (the first warp forms
//     the island's rows, the second the next island's into a second buffer), and,
//     in the DW order, the rows' table c_k = C_k e^{-zeta_k f3} in shared memory,
//     kept while the rows' f3 are unchanged (the work list groups such islands).
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
//    sines use their Taylor series (|argument| < 0.05, relative error < 4e-12).
//    Hardware sin/cos (MUFU, absolute error ~4e-7 on [-pi, pi]) elsewhere.
// Island sums: FP32 per thread, fixed-order shuffle and shared-memory trees.
#include <algorithm>
#include <cstring>

#include "egn_internal.h"

#include "fp32c_common.cuh"
#include "island_geom.cuh"

namespace egn {
namespace {

using namespace fp32c;

constexpr int kThreads = 128;
constexpr int kDwThreads = 64;     // CTA size of the D/G/H, E and F passes
constexpr int kDwCtas = 10;        // resident CTAs per SM of the D/G/H pass
constexpr int kEfCtas = 10;        // and of the E and F passes
constexpr int kDwBatch = 16;       // islands per batch of the D/G/H pass
constexpr int kEfBatch = 16;       // and of the E and F passes (short lists: smaller
                                   // batches spread them over more CTAs)
constexpr int kBatch = kThreads;   // islands per batch, one per thread in the set-up
constexpr int kRowsMax = 64;       // rows per chunk held in shared memory
constexpr int kTabFloats = 2688;   // DW c_k table budget (10.5 KB): [rows][kpad] floats

// ---------------------------------------------------------------- shared state
template <int NB>
struct BatchSmT {  // one entry per island of the batch
  long long isl[NB];
  int np[NB];
  int flags[NB];  // bit0 G wanted, bit1 H wanted
  Df pm[3][NB], ph[3][NB];                      // panel midpoints and half-widths
  Df Bv[NB], Cv[NB], cv[NB];                    // node-rule constants
  Df F1[NB], F2[NB], S12[NB], dd[NB];           // nu1 - nu, nu2 - nu, nu1 + nu2, d
  float ra[3][NB], ri[3][NB];                   // raised-cosine knee and 1/(beta R) of n1, n2, n3
  float nu3[NB];
  float cf0[NB], cf1[NB], cf2[NB];              // D, G, H (DW) or the E / F coefficient
};
using BatchSm = BatchSmT<kBatch>;

// Row constants, four per float4 so that a point pass loads them with 16-byte loads.
template <int RM>
struct RowSm {
  float4 qa[RM];  // q0h, q0l, q1h, q1l              (phase, turns; Q0 modulo K)
  float4 qb[RM];  // q2h, q2l, q3, frac(q0h)
  float4 ab[RM];  // a0, a1, b0, b1                  (f1 - f = a0 + a1 x, f2 - f = b0 + b1 x)
  float4 kc[RM];  // 4 pi^2 bc0, 4 pi^2 bc1, im, ih   (bc = beta2 + pi beta3 (f1 + f2); inner = im + ih x)
  float4 ow[RM];  // o - d (DW) or o, wo ih hout, wo ih, hout   (wo outer weight, hout outer shape)
  float4 f3[RM];  // f30, f31, wo, 0                  (f3 = f30 + f31 x)
};

// Inner Gauss-Legendre nodes of the launch: {x head, x tail, x^2 head, x^2 tail}, {x^3, w}.
struct NodeSm {
  float4 x4[kMaxGl];
  float2 x2[kMaxGl];
};

// Batch set-up (FP64, one island per thread): node-rule geometry and island
// constants of item b0 + tid, rounded to double-floats.
template <int ORD, class BS>
__device__ __forceinline__ void batch_setup(const LinkParams& p, const uint64_t* __restrict__ keys,
                                            const uint32_t* __restrict__ list, long long n_items, long long b0,
                                            BS& bs, int tid) {
    long long it = b0 + tid;
    int np = 0, flags = 0;
    long long isl = -1;
    if (it < n_items) {
      isl = list ? (long long)list[it] : it;
      int coi, n1, n2, n3;
      unpack_key(keys[isl], coi, n1, n2, n3);
      const ChannelTable& ch = p.ch;
      double nu = ch.nu_coi[coi], nu1 = ch.nu[n1], nu2 = ch.nu[n2], nu3 = ch.nu[n3];
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
      const double Rs[3] = {R1, R2, R3};
      for (int q_ = 0; q_ < 3; ++q_) {
        bs.ra[q_][tid] = (float)(0.5 * (1.0 - p.rolloff) * Rs[q_]);
        bs.ri[q_][tid] = p.rolloff > 0.0 ? (float)(1.0 / (p.rolloff * Rs[q_])) : 0.0f;
      }
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

template <int ORD, class BS>
__device__ __forceinline__ RowGeo row_geometry(const LinkParams& p, const BS& bs, int ib, int np, int pi,
                                               int i) {
  RowGeo r;
  const Df y = {p.gl.xh[np][i], p.gl.xl[np][i]};
  const Df pm = bs.pm[pi][ib];
  r.ph = bs.ph[pi][ib];
  r.o = dadd(pm, dmul(r.ph, y));
  const Df m = (ORD == ORD_DW) ? dadd(r.o, bs.cv[ib]) : dsub(bs.cv[ib], r.o);
  const Df Bv = bs.Bv[ib], Cv = bs.Cv[ib];
  const Df lo = dmax(dneg(Bv), dsub(m, Cv));
  const Df hi = dmin(Bv, dadd(m, Cv));
  r.im = dhalf(dadd(lo, hi));
  r.ih = dhalf(dsub(hi, lo));
  const Df zero = {0.0f, 0.0f};
  r.a1 = zero;
  r.b1 = zero;
  r.s1 = zero;
  if (ORD == ORD_DW) {  // w = o, u = im + ih x, v = w - u - d
    r.a0 = dadd(bs.F1[ib], r.im); r.a1 = r.ih;
    r.b0 = dadd(bs.F2[ib], dsub(dsub(r.o, r.im), bs.dd[ib])); r.b1 = dneg(r.ih);
    r.s0 = dadd(bs.S12[ib], dsub(r.o, bs.dd[ib]));
  } else if (ORD == ORD_E) {  // v = o, u = im + ih x
    r.a0 = dadd(bs.F1[ib], r.im); r.a1 = r.ih;
    r.b0 = dadd(bs.F2[ib], r.o);
    r.s0 = dadd(bs.S12[ib], dadd(r.im, r.o)); r.s1 = r.ih;
  } else {  // u = o, v = im + ih x
    r.a0 = dadd(bs.F1[ib], r.o);
    r.b0 = dadd(bs.F2[ib], r.im); r.b1 = r.ih;
    r.s0 = dadd(bs.S12[ib], dadd(r.o, r.im)); r.s1 = r.ih;
  }
  return r;
}

// Row constants of row `row` of island jb of the batch into slot rr of R (the
// point passes' constants, see RowSm); returns the row's f3 (DW order).
template <int ORD, class BS, class RS>
__device__ __forceinline__ float form_row(const LinkParams& p, const BS& bs, RS& R, int jb, int np, int no, int row,
                                          int rr, Df G0, Df G1, float Kf, float invK) {
  const float k4 = (float)(4.0 * kPi * kPi);
  const float pib3 = (float)(kPi * p.beta3), b2f = (float)p.beta2;
  const int pi = row / no, i = row - pi * no;
  const RowGeo g = row_geometry<ORD>(p, bs, jb, np, pi, i);
  const RowPhase q = row_phase(g, G0, G1, Kf, invK);
  const float s0f = dval(g.s0), s1f = dval(g.s1);
  const float imf = dval(g.im), ihf = dval(g.ih), of = dval(g.o);
  const float wo = dval(g.ph) * p.gl.wf[np][i];
  const float dfl = dval(bs.dd[jb]);
  const float hout = ORD == ORD_DW ? rc_f(of, bs.ra[2][jb], bs.ri[2][jb])
                                   : (ORD == ORD_E ? rc_f(of, bs.ra[1][jb], bs.ri[1][jb]) : rc_f(of, bs.ra[0][jb], bs.ri[0][jb]));
  R.qa[rr] = make_float4(q.Q0r.hi, q.Q0r.lo, q.Q1.hi, q.Q1.lo);
  R.qb[rr] = make_float4(q.Q2.hi, q.Q2.lo, q.Q3, q.Q0r.hi - rint_fast(q.Q0r.hi));
  const float kx = k4 * fmaf(pib3, s0f, b2f);
  // DW: f1 + f2 is constant along a row (s1 = 0), so its factor of chi is folded
  // into f1 - f: chi = (a0' + a1' x)(b0 + b1 x) with a' = kx a
  R.ab[rr] = ORD == ORD_DW ? make_float4(kx * dval(g.a0), kx * dval(g.a1), dval(g.b0), dval(g.b1))
                           : make_float4(dval(g.a0), dval(g.a1), dval(g.b0), dval(g.b1));
  R.kc[rr] = make_float4(kx, k4 * pib3 * s1f, imf, ihf);
  R.ow[rr] = make_float4(ORD == ORD_DW ? of - dfl : of, wo * ihf * hout, wo * ihf, hout);
  const float nu3 = bs.nu3[jb];
  float f3v = 0.0f;
  if (ORD == ORD_DW) {
    f3v = nu3 + of;
    R.f3[rr] = make_float4(f3v, 0.0f, wo, 0.0f);
  } else {
    R.f3[rr] = make_float4(nu3 + (imf + of + dfl), ihf, wo, 0.0f);
  }
  return f3v;
}

// Segment sum of NPAIR point pairs of one row by the second-order real
// recurrence b_k = c_k + p b_{k+1} - q b_{k+2}, k = K-1 .. 0, two points per
// fma.rn.f32x2.  It is evaluated as p b_{k+1} + (c_k - q b_{k+2}): the inner FMA
// does not wait for the previous step, so one FMA per step is on the dependency
// chain.  trow holds the row's c_k, 16-byte aligned; each c_k is paired with
// itself in registers.  On return b1p = b_0 and b2p = b_1.
template <int NPAIR>
__device__ __forceinline__ void dw_step(float c, f32x2 nq2, const f32x2* pp, f32x2* b1p, f32x2* b2p) {
  const f32x2 cc = pack2(c, c);
#pragma unroll
  for (int a = 0; a < NPAIR; ++a) {
    const f32x2 nb = ffma2(pp[a], b1p[a], ffma2(nq2, b2p[a], cc));
    b2p[a] = b1p[a];
    b1p[a] = nb;
  }
}

template <int NPAIR>
__device__ __forceinline__ void dw_recurrence(const float* __restrict__ trow, int K, f32x2 nq2, const f32x2* pp,
                                              f32x2* b1p, f32x2* b2p) {
#pragma unroll
  for (int a = 0; a < NPAIR; ++a) {
    b1p[a] = 0ull;
    b2p[a] = 0ull;
  }
  int k = K - 1;
  for (int e = K & 3; e > 0; --e, --k) dw_step<NPAIR>(trow[k], nq2, pp, b1p, b2p);  // peel: k + 1 = 0 (mod 4)
#pragma unroll 2
  for (; k >= 3; k -= 4) {
    const float4 c4 = *reinterpret_cast<const float4*>(trow + k - 3);  // c_{k-3} .. c_k
    dw_step<NPAIR>(c4.w, nq2, pp, b1p, b2p);
    dw_step<NPAIR>(c4.z, nq2, pp, b1p, b2p);
    dw_step<NPAIR>(c4.y, nq2, pp, b1p, b2p);
    dw_step<NPAIR>(c4.x, nq2, pp, b1p, b2p);
  }
}

// Launch shape of the main kernel: NT threads (and NT islands per batch) per
// CTA, min_ctas resident CTAs per SM (the register budget follows from it) and
// rows_max rows of constants per chunk.
__host__ __device__ constexpr int min_ctas(int ord, int kp, int nt) {
  return nt == 64 ? (ord == ORD_DW ? kDwCtas : kEfCtas) : (kp == 8 ? 3 : (kp == 2 ? 8 : (ord == ORD_DW ? 5 : 4)));
}
// Islands per batch (FP64 set-up, one island per thread): fewer than NT keeps the
// batch arrays small enough for kDwCtas CTAs per SM.
__host__ __device__ constexpr int batch_of(int ord, int kp, int nt) {
  return nt == 64 ? (ord == ORD_DW ? kDwBatch : kEfBatch) : (kp == 2 ? kDwBatch : nt);
}
__host__ __device__ constexpr int rows_max(int nt) { return nt == 64 ? 32 : kRowsMax; }
// Floats of the inner-node arrays at the head of the main kernel's dynamic shared
// memory (6 per node, rounded up to 16 bytes).
__host__ __device__ constexpr int node_floats(int n) { return (6 * n + 3) & ~3; }
// Threads per row of the point passes: the smallest power of two whose kp point
// slots each cover n inner nodes.
__host__ __device__ inline int threads_per_row(int n, int kp) {
  int t = 1;
  while (t * kp < n) t <<= 1;
  return t;
}

// Fixed-order sum of the per-warp partial sums of a CTA.
template <int NW>
__device__ __forceinline__ float warp_sum(const float* r) {
  if (NW == 4) return (r[0] + r[1]) + (r[2] + r[3]);
  float t = r[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) t += r[w];
  return t;
}

// Shared state of the identical-spans passes (one CTA).
template <int ORD, int KP, int NT>
struct DwShared {
  BatchSmT<batch_of(ORD, KP, NT)> bs;
  RowSm<rows_max(NT)> rsb[2];  // the current island's rows and the next one's
  float red[4][NT / 32];
  // the rows the c_k table holds (DW): their f3 in FP32 and their number (-1: none)
  float tab_f3[rows_max(NT)];
  int tab_rows;
};

// Inner Gauss-Legendre nodes of the launch into dynamic shared memory:
// {x head, x tail, x^2 head, x^2 tail}[npad], {x^3, w}[npad]; nodes n..npad-1 are
// x = 0 with weight 0, so no point slot needs a bounds test.
template <int NT>
__device__ __forceinline__ void load_nodes(const LinkParams& p, int npad, float4* nx4, float2* nx2) {
  const int n = p.gl.n;
  for (int j = threadIdx.x; j < npad; j += NT) {
    if (j < n) {
      const float xh = p.gl.xh[1][j], xl = p.gl.xl[1][j];
      nx4[j] = make_float4(xh, xl, p.gl.x2h[1][j], p.gl.x2l[1][j]);
      nx2[j] = make_float2(xh * p.gl.x2h[1][j], p.gl.wf[1][j]);
    } else {
      nx4[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      nx2[j] = make_float2(0.0f, 0.0f);
    }
  }
}

// One batch of islands (work items b0 .. b0 + NB - 1 of `list`) of one link.
// cur and have_rows carry the row buffers from island to island.
template <int ORD, int KP, int NT>
__device__ __forceinline__ void dw_batch(const LinkParams& p, const DwConsts& cst, const uint64_t* __restrict__ keys,
                                         const uint32_t* __restrict__ list, long long n_items,
                                         float* __restrict__ terms, long long n_isl, int rows_per_chunk, int kpad,
                                         Df G0, Df G1, long long b0, DwShared<ORD, KP, NT>& sh,
                                         const float4* __restrict__ nx4, const float2* __restrict__ nx2,
                                         float* __restrict__ tab, int& cur, bool& have_rows) {
  constexpr int NPAIR = KP / 2;
  constexpr int NB = batch_of(ORD, KP, NT);
  constexpr int NW = NT / 32;
  auto& bs = sh.bs;
  auto& rsb = sh.rsb;
  auto& red = sh.red;
  auto& tab_f3 = sh.tab_f3;
  int& tab_rows = sh.tab_rows;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = p.gl.n;
  // threads per row (power of two), row slot and point slot of this thread; the
  // tpr x KP point slots of a row cover the n inner nodes
  const int tpr = threads_per_row(n, KP);
  const int rows_per_pass = NT / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;
  const int K = cst.K;
  const float Kf = cst.Kf, invK = cst.invK;
  const float alpha = cst.alpha, alpha2 = cst.alpha2;
  const float r = cst.r;
  const float one_m_r = cst.one_m_r;
  const float q = cst.q;
  const float m2r = cst.m2r;
  const float c2r = cst.c2r, c4r = cst.c4r, omr2 = cst.omr2;
  const float N = cst.N;
  const float g2 = cst.g2;
  const float pi_f = 3.14159265358979f;
  (void)r;
    // ---------------- 1. batch set-up, FP64, one island per thread
    if (tid < NB) batch_setup<ORD>(p, keys, list, n_items, b0, bs, tid);
    __syncthreads();
    const int nb = (int)min((long long)NB, n_items - b0);
    // ---------------- 2./3. the islands of the batch, one after the other
    for (int ib = 0; ib < nb; ++ib) {
      bool fetched = false;
      const int np = bs.np[ib];
      const int flags = bs.flags[ib];
      const bool want_g = flags & 1, want_h = flags & 2;
      const bool cplx = ORD != ORD_DW || flags != 0;
      const float sa1 = bs.ra[0][ib], sa2 = bs.ra[1][ib], sa3 = bs.ra[2][ib];
      const float si1 = bs.ri[0][ib], si2 = bs.ri[1][ib], si3 = bs.ri[2][ib];
      const float dfl = dval(bs.dd[ib]);
      float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
      const int no = np > 0 ? p.gl.order[np] : 0;
      const int rows = np * no;
      for (int c0 = 0; c0 < rows; c0 += rows_per_chunk) {
        const int rc = min(rows_per_chunk, rows - c0);
        // ---- row constants in double-float, one row per thread of the first half of
        // the CTA (rc <= NT / 2).  When this island and the next fit one chunk, the
        // second half forms the next island's rows into the other buffer meanwhile,
        // and the next island skips this phase.
        RowSm<rows_max(NT)>& rs = rsb[cur];
        bool same_row = true;  // DW: this row's f3 equals the table's row rr
        bool fetch = false;
        if (!have_rows) {
          const int nb1 = ib + 1 < nb ? bs.np[ib + 1] : 0;
          const int rows1 = nb1 > 0 ? nb1 * p.gl.order[nb1] : 0;
          fetch = rows <= NT / 2 && rows <= rows_per_chunk && rows1 > 0 && rows1 <= NT / 2 && rows1 <= rows_per_chunk;
          fetched = fetch;
          if (tid < rc) {
            const float f3v = form_row<ORD>(p, bs, rs, ib, np, no, c0 + tid, tid, G0, G1, Kf, invK);
            if (ORD == ORD_DW) same_row = tab_rows == rc && tab_f3[tid] == f3v;
          } else if (fetch && tid >= NT / 2 && tid - NT / 2 < rows1) {
            form_row<ORD>(p, bs, rsb[cur ^ 1], ib + 1, nb1, p.gl.order[nb1], tid - NT / 2, tid - NT / 2, G0, G1, Kf,
                          invK);
          }
        } else if (ORD == ORD_DW && tid < rc) {
          same_row = tab_rows == rc && tab_f3[tid] == rs.f3[tid].x;
        }
        // the c_k table depends only on the rows' f3 (and the launch's C_k, zeta_k):
        // when every row matches, the table already holds this chunk's values
        const bool keep = ORD == ORD_DW ? __syncthreads_and(same_row) != 0 : (__syncthreads(), false);
        // ---- c_k tables of the chunk's rows (DW): C_k 2^{-zeta_k log2(e) f3}
        // A task is four consecutive columns of one row (one 16-byte store); rounds
        // of up to NT column groups, and a round of gn < NT groups gives each group
        // NT / gn threads that split the rows.  The four C_k and zeta_k stay in
        // registers; columns K..kpad-1 (padding, never read) get C_k = 0.
        // It is rebuilt only when some row's f3 differs from the rows it holds (the
        // work list groups islands with equal outer nodes).
        if (ORD == ORD_DW && !keep) {
          const int ng = kpad >> 2;
          for (int g0 = 0; g0 < ng; g0 += NT) {
            const int gn = min(NT, ng - g0);
            const int rstep = NT / gn, g4 = g0 + tid % gn, r0 = tid / gn;
            if (r0 < rstep) {
              float c4[4], z4[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int k = 4 * g4 + e;
                c4[e] = k < K ? p.seg.ck_f[k] : 0.0f;
                z4[e] = k < K ? p.seg.zeta_f[k] : 0.0f;
              }
#pragma unroll 4
              for (int rr = r0; rr < rc; rr += rstep) {
                const float f3 = rs.f3[rr].x;
                float4 v;
                v.x = c4[0] * ex2_approx(-z4[0] * f3);
                v.y = c4[1] * ex2_approx(-z4[1] * f3);
                v.z = c4[2] * ex2_approx(-z4[2] * f3);
                v.w = c4[3] * ex2_approx(-z4[3] * f3);
                *reinterpret_cast<float4*>(tab + rr * kpad + 4 * g4) = v;
              }
            }
          }
          __syncthreads();
          // read again only in the next chunk's row phase, after the chunk's last barrier
          if (tid < rc) tab_f3[tid] = rs.f3[tid].x;
          if (tid == 0) tab_rows = rc;
        }
        // ---- points
        for (int rb = 0; rb < rc; rb += rows_per_pass) {
          const int rr = rb + rsub;
          const bool row_ok = rr < rc;
          const int rrc = row_ok ? rr : 0;
          const float4 qa = rs.qa[rrc], qb = rs.qb[rrc], ab = rs.ab[rrc], kc = rs.kc[rrc], ow = rs.ow[rrc];
          const float4 f3r = rs.f3[rrc];
          const float im = kc.z, ih = kc.w;
          const float wrowh = row_ok ? ow.y : 0.0f, wrow = row_ok ? ow.z : 0.0f;
          if (ORD == ORD_DW && !cplx) {
            // D only.  |Upsilon / gamma|^2 = |sum|^2 |w - 1|^2 / (alpha^2 + chi^2) * (sn / sd)^2
            // with 2 Re w = 2r - 4r sin^2(pi theta), |w - 1|^2 = (1 - r)^2 + 4r sin^2(pi theta)
            // and |sum|^2 = |b_0 - conj(w) b_1|^2 = b_0 (b_0 - 2 Re(w) b_1) + r^2 b_1^2.
            // Every factor but |sum|^2 is formed before the recurrence, so that one value
            // per point (with 2 Re w) stays live across it.
            float pv[KP], fac[KP];
#pragma unroll
            for (int m = 0; m < KP; ++m) {
              const int j = lr + tpr * m;
              const float4 x4 = nx4[j];
              const float2 x2 = nx2[j];
              float th, ph;
              point_phase(qa, qb, x4, x2.x, Kf, invK, th, ph);
              const float sh = __sinf(pi_f * th);
              const float s2 = sh * sh;
              pv[m] = fmaf(-c4r, s2, c2r);
              const float wa = fmaf(c4r, s2, omr2);
              const float xh = x4.x;
              const float chi = fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z);  // kx folded into ab.xy
              const float t = fmaf(ih, xh, im);
              const float wgt = x2.y * rc_f(t, sa1, si1) * rc_f(ow.x - t, sa2, si2);
              float sd, sn;
              array_sines(pi_f * ph, N, sd, sn);
              const float den = (sd * sd) * fmaf(chi, chi, alpha2);
              fac[m] = (wgt * wa) * ((sn * sn) * rcp_approx(den));
            }
            f32x2 pp[NPAIR], b1p[NPAIR], b2p[NPAIR];
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) pp[a] = pack2(pv[2 * a], pv[2 * a + 1]);
            dw_recurrence<NPAIR>(tab + rrc * kpad, K, pack2(-q, -q), pp, b1p, b2p);
            float acc = 0.0f;
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) {
              float b0v[2], b1v[2];
              unpack2(b1p[a], b0v[0], b0v[1]);
              unpack2(b2p[a], b1v[0], b1v[1]);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int m = 2 * a + e;
                const float s2sum = fmaf(b0v[e], fmaf(-pv[m], b1v[e], b0v[e]), q * b1v[e] * b1v[e]);
                acc = fmaf(fac[m], s2sum, acc);
              }
            }
            dsum = fmaf(wrowh, acc, dsum);
            continue;
          }
          float gre = 0.0f, gim = 0.0f;
          float p_[KP], b1_[KP], b2_[KP], f3_[KP];
          float wm1_[KP], wi_[KP], chi_[KP], phi_[KP], wgt_[KP], s12_[KP], s123_[KP];
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const int j = lr + tpr * m;
            const float4 x4 = nx4[j];
            const float2 x2 = nx2[j];
            const float xh = x4.x;
            const float wnode = x2.y;
            float th, ph;
            point_phase(qa, qb, x4, x2.x, Kf, invK, th, ph);
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
            chi_[m] = ORD == ORD_DW ? fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z)  // kx folded into ab.xy
                                    : fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z) * fmaf(kc.y, xh, kc.x);
            // spectral shapes and weights
            const float t = fmaf(ih, xh, im);
            float u, v, h3;
            if (ORD == ORD_DW) { u = t; v = ow.x - t; h3 = 1.0f; }  // h3(w) is folded into wrowh
            else {
              if (ORD == ORD_E) { v = ow.x; u = t; } else { u = ow.x; v = t; }
              h3 = rc_f(u + v + dfl, sa3, si3);
            }
            const float h1 = rc_f(u, sa1, si1), h2 = rc_f(v, sa2, si2);
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
            f32x2 pp[NPAIR], b1p[NPAIR], b2p[NPAIR];
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) pp[a] = pack2(p_[2 * a], p_[2 * a + 1]);
            dw_recurrence<NPAIR>(tab + rrc * kpad, K, pack2(-q, -q), pp, b1p, b2p);
#pragma unroll
            for (int a = 0; a < NPAIR; ++a) {
              unpack2(b1p[a], b1_[2 * a], b1_[2 * a + 1]);
              unpack2(b2p[a], b2_[2 * a], b2_[2 * a + 1]);
            }
          } else {
            // E and F: c_k per point (f3 varies along the row); four segments per
            // round from 16-byte loads of C_k and zeta_k, so that the ex2 of later
            // segments are issued ahead of the recurrence that waits on them
            auto step = [&](float ck, float zk) {
#pragma unroll
              for (int m = 0; m < KP; ++m) {
                const float c = ck * ex2_approx(-zk * f3_[m]);
                const float bn = fmaf(p_[m], b1_[m], fmaf(-q, b2_[m], c));
                b2_[m] = b1_[m];
                b1_[m] = bn;
              }
            };
            int k = K - 1;
            for (int e = K & 3; e > 0; --e, --k) step(p.seg.ck_f[k], p.seg.zeta_f[k]);  // peel: k + 1 = 0 (mod 4)
#pragma unroll 1
            for (; k >= 3; k -= 4) {
              const float4 c4 = *reinterpret_cast<const float4*>(p.seg.ck_f + k - 3);
              const float4 z4 = *reinterpret_cast<const float4*>(p.seg.zeta_f + k - 3);
              step(c4.w, z4.w);
              step(c4.z, z4.z);
              step(c4.y, z4.y);
              step(c4.x, z4.x);
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
            const float ratio = array_ratio(x, N);
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
        const float t0 = warp_sum<NW>(red[0]);
        if (ORD == ORD_DW) {
          terms[isl] = bs.cf0[ib] * g2 * t0;
          if (cplx) {
            const float t1 = warp_sum<NW>(red[1]);
            const float t2 = warp_sum<NW>(red[2]);
            const float t3 = warp_sum<NW>(red[3]);
            if (want_g) terms[3 * n_isl + isl] = bs.cf1[ib] * g2 * t1;
            if (want_h) terms[4 * n_isl + isl] = bs.cf2[ib] * g2 * (t2 * t2 + t3 * t3);
          }
        } else {
          const float t1 = warp_sum<NW>(red[1]);
          terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = bs.cf0[ib] * g2 * t1;
        }
      }
      __syncthreads();
      // the next island's rows are in the other buffer if they were formed here
      if (fetched) cur ^= 1;
      have_rows = fetched;
    }
}

template <int ORD, int KP, int NT>
__global__ void __launch_bounds__(NT, min_ctas(ORD, KP, NT))
integrate_fp32c_kernel(LinkParams p, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                       long long n_items, float* __restrict__ terms, long long n_isl, int rows_per_chunk, int kpad,
                       Df G0, Df G1) {
  static_assert(KP % 2 == 0, "points per thread come in f32x2 pairs");
  constexpr int NB = batch_of(ORD, KP, NT);
  __shared__ DwShared<ORD, KP, NT> sh;
  if (threadIdx.x == 0) sh.tab_rows = -1;  // read after the first batch barrier
  const int npad = threads_per_row(p.gl.n, KP) * KP;
  // dynamic: the inner nodes, then (DW only) the [rows_per_chunk][kpad] c_k of
  // the chunk's rows, 16-byte aligned
  extern __shared__ __align__(16) float dyn[];
  float4* const nx4 = reinterpret_cast<float4*>(dyn);
  float2* const nx2 = reinterpret_cast<float2*>(dyn + 4 * npad);
  float* const tab = dyn + node_floats(npad);
  const DwConsts cst = dw_consts(p);
  load_nodes<NT>(p, npad, nx4, nx2);
  int cur = 0;             // row buffer of the current island
  bool have_rows = false;  // its rows were formed with the previous island's
  for (long long b0 = (long long)blockIdx.x * NB; b0 < n_items; b0 += (long long)gridDim.x * NB)
    dw_batch<ORD, KP, NT>(p, cst, keys, list, n_items, terms, n_isl, rows_per_chunk, kpad, G0, G1, b0, sh, nx4, nx2,
                          tab, cur, have_rows);
}

template <int ORD, int KP, int NT>
cudaError_t launch_one(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items, float* terms,
                       long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const int K = p.seg.K;
  int kpad = (K + 3) & ~3;
  if ((kpad & 7) == 0) kpad += 4;  // row stride = 4 (mod 8) words: 4 rows' 16-byte loads hit distinct banks
  int rows = rows_max(NT);
  if (ORD == ORD_DW) {
    rows = kTabFloats / kpad;
    if (rows > rows_max(NT)) rows = rows_max(NT);
    if (rows < 1) rows = 1;
  }
  const int npad = threads_per_row(p.gl.n, KP) * KP;
  size_t smem = ((size_t)node_floats(npad) + (ORD == ORD_DW ? (size_t)rows * kpad : 0)) * sizeof(float);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // static shared memory + the c_k table exceed the 48 KB default: opt in once per device
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = opt_in_smem(integrate_fp32c_kernel<ORD, KP, NT>,
                                  (node_floats(2 * kMaxGl) + kTabFloats) * (int)sizeof(float), attr_done))
    return e;
  long long batches = (n_items + batch_of(ORD, KP, NT) - 1) / batch_of(ORD, KP, NT);
  long long blocks = (long long)sms * min_ctas(ORD, KP, NT);
  if (blocks > batches) blocks = batches;
  // 2 pi L beta2 and 2 pi^2 L beta3 as double-floats
  double g0 = 2.0 * kPi * p.L * p.beta2, g1 = 2.0 * kPi * kPi * p.L * p.beta3;
  float g0h = (float)g0, g1h = (float)g1;
  Df G0 = {g0h, (float)(g0 - (double)g0h)}, G1 = {g1h, (float)(g1 - (double)g1h)};
  integrate_fp32c_kernel<ORD, KP, NT><<<(unsigned)blocks, NT, smem, st>>>(p, keys, list, n_items, terms, n_isl,
                                                                             rows, kpad, G0, G1);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Links whose spans differ (Eq. 22 written out).  Same node rule, batch set-up
// and row geometry as above; per row and span type t the phase polynomial and
// the c_k table; per point mu_t, phi_t for every type and the coherent sum
// Y = sum_s gamma_t(s) mu_t(s) e^{i Phi_s}, Phi_{s+1} = Phi_s + phi_t(s) (turns,
// by complex multiplication with e^{2 pi i phi_t}).  Two points per thread,
// scalar recurrences.
// ---------------------------------------------------------------------------

constexpr int kGRows = 32;   // rows per chunk, general links
constexpr int kGTab = 10240; // c_k tables of all types, floats (40 KB)

struct GenTypes {
  Df G0[kMaxTypes], G1[kMaxTypes];  // 2 pi L_t beta2_t, 2 pi^2 L_t beta3_t
  int koff[kMaxTypes];              // offset of type t in a table row
  int ktot;                         // table row stride (floats)
};

struct GenRowSm {
  float4 qa[kMaxTypes][kGRows];  // q0h, q0l, q1h, q1l of type t
  float4 qb[kMaxTypes][kGRows];  // q2h, q2l, q3, frac(q0h)
  float2 kc[kMaxTypes][kGRows];  // 4 pi^2 (beta2_t + pi beta3_t s0), 4 pi^2 pi beta3_t s1
  float4 ab[kGRows];             // a0, a1, b0, b1
  float4 ow[kGRows];             // o - d (DW) or o, wo ih hout, wo ih, hout
  float4 f3[kGRows];             // f30, f31, wo, im
  float ih[kGRows];
};

// Shared state of the general-links passes (one CTA).
struct GenShared {
  BatchSm bs;
  GenRowSm rs;
  NodeSm ns;
  float red[4][kThreads / 32];
  float tyf[kMaxTypes][6];  // K, 1/K, alpha, r, 1 - r, gamma
};

// Inner Gauss-Legendre nodes of the launch (the first n slots).
__device__ __forceinline__ void load_node_sm(const LinkParams& p, NodeSm& ns) {
  for (int j = threadIdx.x; j < p.gl.n; j += kThreads) {
    const float xh = p.gl.xh[1][j], xl = p.gl.xl[1][j];
    ns.x4[j] = make_float4(xh, xl, p.gl.x2h[1][j], p.gl.x2l[1][j]);
    ns.x2[j] = make_float2(xh * p.gl.x2h[1][j], p.gl.wf[1][j]);
  }
}

// Per-type constants of a general link (the caller synchronises before use).
__device__ __forceinline__ void gen_types(const LinkParams& p, GenShared& sh) {
  const int tid = threadIdx.x;
  if (tid < p.n_types) {
    const SpanType& ty = p.types[tid];
    sh.tyf[tid][0] = (float)ty.seg.K;
    sh.tyf[tid][1] = 1.0f / (float)ty.seg.K;
    sh.tyf[tid][2] = (float)ty.alpha;
    sh.tyf[tid][3] = (float)ty.r;
    sh.tyf[tid][4] = (float)(-expm1(-ty.alpha * ty.dz));
    sh.tyf[tid][5] = (float)ty.gamma;
  }
}

// One batch of islands (items b0 .. b0 + kBatch - 1 of `list`) of one general link.
template <int ORD>
__device__ __forceinline__ void gen_batch(const LinkParams& p, const GenTypes& gt, const uint64_t* __restrict__ keys,
                                          const uint32_t* __restrict__ list, long long n_items,
                                          float* __restrict__ terms, long long n_isl, int rows_per_chunk,
                                          long long b0, GenShared& sh, float* __restrict__ tabg) {
  constexpr int KP = 2;
  auto& bs = sh.bs;
  auto& rs = sh.rs;
  auto& ns = sh.ns;
  auto& red = sh.red;
  auto& tyf = sh.tyf;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = p.gl.n;
  const int T = p.n_types;
  const float k4 = (float)(4.0 * kPi * kPi);
  const float pi_f = 3.14159265358979f;
  int tpr = 1;
  while (tpr * KP < n) tpr <<= 1;
  const int rows_per_pass = kThreads / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;
    batch_setup<ORD>(p, keys, list, n_items, b0, bs, tid);
    __syncthreads();
    const int nb = (int)min((long long)kBatch, n_items - b0);
    for (int ib = 0; ib < nb; ++ib) {
      const int np = bs.np[ib];
      const int flags = bs.flags[ib];
      const bool want_g = flags & 1, want_h = flags & 2;
      const float sa1 = bs.ra[0][ib], sa2 = bs.ra[1][ib], sa3 = bs.ra[2][ib];
      const float si1 = bs.ri[0][ib], si2 = bs.ri[1][ib], si3 = bs.ri[2][ib];
      const float dfl = dval(bs.dd[ib]);
      float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
      const int no = np > 0 ? p.gl.order[np] : 0;
      const int rows = np * no;
      for (int c0 = 0; c0 < rows; c0 += rows_per_chunk) {
        const int rc = min(rows_per_chunk, rows - c0);
        // ---- row constants: geometry once, phase per type (slot = row, type)
        for (int slot = tid; slot < rc * T; slot += kThreads) {
          const int rr = slot % rc, t = slot / rc;
          const int row = c0 + rr;
          const int pi = row / no, i = row - pi * no;
          const RowGeo g = row_geometry<ORD>(p, bs, ib, np, pi, i);
          const RowPhase q = row_phase(g, gt.G0[t], gt.G1[t], tyf[t][0], tyf[t][1]);
          rs.qa[t][rr] = make_float4(q.Q0r.hi, q.Q0r.lo, q.Q1.hi, q.Q1.lo);
          rs.qb[t][rr] = make_float4(q.Q2.hi, q.Q2.lo, q.Q3, q.Q0r.hi - rint_fast(q.Q0r.hi));
          const float pib3 = (float)(kPi * p.types[t].beta3);
          rs.kc[t][rr] = make_float2(k4 * fmaf(pib3, dval(g.s0), (float)p.types[t].beta2), k4 * pib3 * dval(g.s1));
          if (t == 0) {
            const float imf = dval(g.im), ihf = dval(g.ih), of = dval(g.o);
            const float wo = dval(g.ph) * p.gl.wf[np][i];
            const float hout =
                ORD == ORD_DW ? rc_f(of, sa3, si3) : (ORD == ORD_E ? rc_f(of, sa2, si2) : rc_f(of, sa1, si1));
            rs.ab[rr] = make_float4(dval(g.a0), dval(g.a1), dval(g.b0), dval(g.b1));
            rs.ow[rr] = make_float4(ORD == ORD_DW ? of - dfl : of, wo * ihf * hout, wo * ihf, hout);
            const float nu3 = bs.nu3[ib];
            if (ORD == ORD_DW) rs.f3[rr] = make_float4(nu3 + of, 0.0f, wo, imf);
            else rs.f3[rr] = make_float4(nu3 + (imf + of + dfl), ihf, wo, imf);
            rs.ih[rr] = ihf;
          }
        }
        __syncthreads();
        if (ORD == ORD_DW) {  // c_k tables, all types
          for (int t = 0; t < T; ++t) {
            const int K = p.types[t].seg.K;
            for (int k = tid; k < K; k += kThreads) {
              const float ck = p.types[t].seg.ck_f[k], zk = p.types[t].seg.zeta_f[k];
              for (int rr = 0; rr < rc; ++rr) tabg[rr * gt.ktot + gt.koff[t] + k] = ck * ex2_approx(-zk * rs.f3[rr].x);
            }
          }
          __syncthreads();
        }
        for (int rb = 0; rb < rc; rb += rows_per_pass) {
          const int rr = rb + rsub;
          const bool row_ok = rr < rc;
          const int rrc = row_ok ? rr : 0;
          const float4 ab = rs.ab[rrc], ow = rs.ow[rrc], f3r = rs.f3[rrc];
          const float im = f3r.w, ih = rs.ih[rrc];
          const float wrowh = row_ok ? ow.y : 0.0f, wrow = row_ok ? ow.z : 0.0f;
          float xh_[KP], wnode_[KP], yre_[KP], yim_[KP];
          float zre_[KP], zim_[KP];
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const int j = lr + tpr * m;
            const bool jok = j < n;
            xh_[m] = ns.x4[jok ? j : 0].x;
            wnode_[m] = jok ? ns.x2[j].y : 0.0f;
            yre_[m] = 0.0f;
            yim_[m] = 0.0f;
          }
          // per span type: mu_t and e^{2 pi i phi_t}, kept for the span sum
          float mre_[kMaxTypes][KP], mim_[kMaxTypes][KP], ere_[kMaxTypes][KP], eim_[kMaxTypes][KP];
#pragma unroll
          for (int t = 0; t < kMaxTypes; ++t) {
            if (t >= T) break;
            const float4 qa = rs.qa[t][rrc], qb = rs.qb[t][rrc];
            const float2 kc = rs.kc[t][rrc];
            const float Kf = tyf[t][0], invK = tyf[t][1], alpha = tyf[t][2], r = tyf[t][3], omr = tyf[t][4],
                        gam = tyf[t][5];
            const int K = (int)Kf;
            float p_[KP], wm1_[KP], wi_[KP], chi_[KP], b1_[KP], b2_[KP], f3_[KP];
#pragma unroll
            for (int m = 0; m < KP; ++m) {
              const int j = lr + tpr * m;
              const int jj = j < n ? j : 0;
              const float4 x4 = ns.x4[jj];
              const float xh = x4.x, xl = x4.y, x2h = x4.z, x2l = x4.w, xc = ns.x2[jj].x;
              const float p1 = qa.z * xh, e1 = fmaf(qa.z, xh, -p1);
              const float t1 = fmaf(qa.z, xl, fmaf(qa.w, xh, e1));
              const float p2 = qb.x * x2h, e2 = fmaf(qb.x, x2h, -p2);
              const float t2 = fmaf(qb.x, x2l, fmaf(qb.y, x2h, e2));
              const float r1 = fmaf(-Kf, rint_cvt(p1 * invK), p1);
              const float tail = (qa.y + t1) + fmaf(qb.z, xc, t2);
              float th = fmaf((qa.x + r1) + p2, invK, tail * invK);
              th -= rint_cvt(th);
              float ph = (qb.w + (r1 - rint_cvt(r1))) + ((p2 - rint_cvt(p2)) + tail);
              ph -= rint_cvt(ph);
              const float ah = pi_f * th;
              const float sh = __sinf(ah), chh = __cosf(ah);
              const float t2r = -2.0f * r * sh;
              wm1_[m] = fmaf(t2r, sh, -omr);
              p_[m] = fmaf(2.0f, wm1_[m], 2.0f);
              wi_[m] = -t2r * chh;
              chi_[m] = fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z) * fmaf(kc.y, xh, kc.x);
              const float ang = 2.0f * pi_f * ph;
              ere_[t][m] = __cosf(ang);
              eim_[t][m] = __sinf(ang);
              f3_[m] = fmaf(f3r.y, xh, f3r.x);
              b1_[m] = 0.0f;
              b2_[m] = 0.0f;
            }
            const float q = r * r;
            if (ORD == ORD_DW) {
              const float* trow = tabg + rrc * gt.ktot + gt.koff[t];
              for (int k = K - 1; k >= 0; --k) {
                const float c = trow[k];
#pragma unroll
                for (int m = 0; m < KP; ++m) {
                  const float bn = fmaf(p_[m], b1_[m], fmaf(-q, b2_[m], c));
                  b2_[m] = b1_[m];
                  b1_[m] = bn;
                }
              }
            } else {  // E, F: c_k per point, segments in rounds of four (16-byte loads)
              const float* ckf = p.types[t].seg.ck_f;
              const float* zkf = p.types[t].seg.zeta_f;
              auto step = [&](float ck, float zk) {
#pragma unroll
                for (int m = 0; m < KP; ++m) {
                  const float c = ck * ex2_approx(-zk * f3_[m]);
                  const float bn = fmaf(p_[m], b1_[m], fmaf(-q, b2_[m], c));
                  b2_[m] = b1_[m];
                  b1_[m] = bn;
                }
              };
              int k = K - 1;
              for (int e = K & 3; e > 0; --e, --k) step(ckf[k], zkf[k]);  // peel: k + 1 = 0 (mod 4)
#pragma unroll 1
              for (; k >= 3; k -= 4) {
                const float4 c4 = *reinterpret_cast<const float4*>(ckf + k - 3);
                const float4 z4 = *reinterpret_cast<const float4*>(zkf + k - 3);
                step(c4.w, z4.w);
                step(c4.z, z4.z);
                step(c4.y, z4.y);
                step(c4.x, z4.x);
              }
            }
#pragma unroll
            for (int m = 0; m < KP; ++m) {
              const float wm1 = wm1_[m], wi = wi_[m], chi = chi_[m];
              const float sre = fmaf(-(wm1 + 1.0f), b2_[m], b1_[m]);
              const float sim = wi * b2_[m];
              const float inv = rcp_approx(fmaf(chi, chi, alpha * alpha)) * gam;
              const float qr = fmaf(-alpha, wm1, chi * wi) * inv;
              const float qi = fmaf(-chi, wm1, -alpha * wi) * inv;
              mre_[t][m] = fmaf(sre, qr, -sim * qi);  // gamma_t mu_t
              mim_[t][m] = fmaf(sre, qi, sim * qr);
            }
          }
          // coherent sum over the spans
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            zre_[m] = 1.0f;
            zim_[m] = 0.0f;
          }
          for (int sp = 0; sp < p.n_spans; ++sp) {
            const int t = p.span_type[sp];
#pragma unroll
            for (int m = 0; m < KP; ++m) {
              float mr = 0.0f, mi = 0.0f, er = 1.0f, ei = 0.0f;
#pragma unroll
              for (int u = 0; u < kMaxTypes; ++u)
                if (u == t) { mr = mre_[u][m]; mi = mim_[u][m]; er = ere_[u][m]; ei = eim_[u][m]; }
              yre_[m] = fmaf(mr, zre_[m], fmaf(-mi, zim_[m], yre_[m]));
              yim_[m] = fmaf(mr, zim_[m], fmaf(mi, zre_[m], yim_[m]));
              const float zr = fmaf(zre_[m], er, -zim_[m] * ei);
              zim_[m] = fmaf(zre_[m], ei, zim_[m] * er);
              zre_[m] = zr;
            }
          }
          // weights and sums (Upsilon itself, gamma included)
          float gre = 0.0f, gim = 0.0f;
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const float xh = xh_[m];
            const float tt = fmaf(ih, xh, im);
            float u, v, h3;
            if (ORD == ORD_DW) { u = tt; v = ow.x - tt; h3 = 1.0f; }
            else {
              if (ORD == ORD_E) { v = ow.x; u = tt; } else { u = ow.x; v = tt; }
              h3 = rc_f(u + v + dfl, sa3, si3);
            }
            const float h1 = rc_f(u, sa1, si1), h2 = rc_f(v, sa2, si2);
            const float yre = yre_[m], yim = yim_[m];
            if (ORD == ORD_DW) {
              dsum = fmaf((wrowh * wnode_[m]) * (h1 * h2), fmaf(yre, yre, yim * yim), dsum);
              if (want_g) {
                const float a12 = (row_ok ? wnode_[m] : 0.0f) * sqrtf(h1 * h2);
                gre = fmaf(a12, yre, gre);
                gim = fmaf(a12, yim, gim);
              }
              if (want_h) {
                const float a123 = wrow * wnode_[m] * sqrtf(h1 * h2 * ow.w);
                hre = fmaf(a123, yre, hre);
                him = fmaf(a123, yim, him);
              }
            } else {
              const float a = (row_ok ? wnode_[m] : 0.0f) * ih * sqrtf(ORD == ORD_E ? h1 * h3 : h2 * h3);
              gre = fmaf(a, yre, gre);
              gim = fmaf(a, yim, gim);
            }
          }
          if (ORD != ORD_DW || want_g) {
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
        __syncthreads();
      }
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
          terms[isl] = bs.cf0[ib] * t[0];
          if (want_g) terms[3 * n_isl + isl] = bs.cf1[ib] * t[1];
          if (want_h) terms[4 * n_isl + isl] = bs.cf2[ib] * (t[2] * t[2] + t[3] * t[3]);
        } else {
          terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = bs.cf0[ib] * t[1];
        }
      }
      __syncthreads();
    }
}

template <int ORD>
__global__ void __launch_bounds__(kThreads, 3)
integrate_fp32c_general_kernel(LinkParams p, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                               long long n_items, float* __restrict__ terms, long long n_isl, int rows_per_chunk,
                               GenTypes gt) {
  __shared__ GenShared sh;
  extern __shared__ __align__(16) float tabg[];  // [rows_per_chunk][ktot]
  load_node_sm(p, sh.ns);
  gen_types(p, sh);
  __syncthreads();
  for (long long b0 = (long long)blockIdx.x * kBatch; b0 < n_items; b0 += (long long)gridDim.x * kBatch)
    gen_batch<ORD>(p, gt, keys, list, n_items, terms, n_isl, rows_per_chunk, b0, sh, tabg);
}

template <int ORD>
cudaError_t launch_general(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                           float* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  GenTypes gt{};
  int ktot = 0;
  for (int t = 0; t < p.n_types; ++t) {
    const SpanType& ty = p.types[t];
    double g0 = 2.0 * kPi * ty.L * ty.beta2, g1 = 2.0 * kPi * kPi * ty.L * ty.beta3;
    float g0h = (float)g0, g1h = (float)g1;
    gt.G0[t] = {g0h, (float)(g0 - (double)g0h)};
    gt.G1[t] = {g1h, (float)(g1 - (double)g1h)};
    gt.koff[t] = ktot;
    ktot += ty.seg.K;
  }
  gt.ktot = ktot;
  int rows = kGRows;
  if (ORD == ORD_DW) {
    rows = kGTab / ktot;
    if (rows > kGRows) rows = kGRows;
    if (rows < 1) rows = 1;
  }
  size_t smem = ORD == ORD_DW ? (size_t)rows * ktot * sizeof(float) : 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = opt_in_smem(integrate_fp32c_general_kernel<ORD>, kGTab * (int)sizeof(float), attr_done))
    return e;
  long long batches = (n_items + kBatch - 1) / kBatch;
  long long blocks = (long long)sms * 3;
  if (blocks > batches) blocks = batches;
  integrate_fp32c_general_kernel<ORD><<<(unsigned)blocks, kThreads, smem, st>>>(p, keys, list, n_items, terms, n_isl,
                                                                               rows, gt);
  return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// Links with more than kMaxTypes span types (Eq. 22 span by span).  The span
// types come from device memory; per row and type the phase polynomial lives in
// dynamic shared memory; per point the spans are walked in order and a type's
// gamma mu and e^{2 pi i phi} are recomputed only when the type changes from one
// span to the next, with c_k formed on the fly (one ex2 per segment).  Two
// points per thread, scalar recurrences.
// ---------------------------------------------------------------------------

constexpr int kSpanTypeFloats = 12;  // per type: G0 (df), G1 (df), K, 1/K, alpha, r, 1 - r, gamma, beta2, pi beta3

// Shared state of the span-by-span passes (one CTA); the per-type constants, row
// phases and fibre tables are in dynamic shared memory, laid out by spans_layout.
constexpr int kSpansBatch = 64;            // islands per batch of the span-by-span passes
constexpr int kSpansCtas = 4;              // resident CTAs per SM
constexpr int kSpansDynBytes = 40 * 1024;  // per-type constants, row phases and fibre c_k tables

struct SpansShared {
  BatchSmT<kSpansBatch> bs;
  float4 g_ab[kGRows], g_ow[kGRows], g_f3[kGRows];
  float g_ih[kGRows];
  NodeSm ns;
  float red[4][kThreads / 32];
};

struct SpansLayout {
  float4* sqa;  // [T][R]
  float4* sqb;  // [T][R]
  float2* skc;  // [T][R]
  float* tyc;   // [T][kSpanTypeFloats]
  float* tabf;  // DW with fibre groups: c_k of the chunk's rows per fibre, [n_fib][R][kfp]
};

// Floats of the dynamic layout before the fibre tables: the row phases (40 T R
// bytes) and the type constants, rounded up to a 16-byte boundary (the fibre
// rows are read with 16-byte loads; 40 T R + 48 T is a multiple of 16 only when T
// or R is even).
__host__ __device__ constexpr int spans_head_floats(int T, int R) { return (10 * T * R + kSpanTypeFloats * T + 3) & ~3; }

__device__ __forceinline__ SpansLayout spans_layout(float* dyn, int T, int R) {
  SpansLayout l;
  l.sqa = reinterpret_cast<float4*>(dyn);
  l.sqb = l.sqa + T * R;
  l.skc = reinterpret_cast<float2*>(l.sqb + T * R);
  l.tyc = reinterpret_cast<float*>(l.skc + T * R);
  l.tabf = dyn + spans_head_floats(T, R);
  return l;
}

// Per-type constants of a span-by-span link (the caller synchronises before use).
__device__ __forceinline__ void spans_types(const LinkParams& p, float* tyc) {
  for (int t = threadIdx.x; t < p.n_types; t += kThreads) {
    const SpanType& ty = p.types_dev[t];
    const double g0 = 2.0 * kPi * ty.L * ty.beta2, g1 = 2.0 * kPi * kPi * ty.L * ty.beta3;
    float* c = tyc + kSpanTypeFloats * t;
    c[0] = (float)g0;
    c[1] = (float)(g0 - (double)c[0]);
    c[2] = (float)g1;
    c[3] = (float)(g1 - (double)c[2]);
    c[4] = (float)ty.seg.K;
    c[5] = 1.0f / (float)ty.seg.K;
    c[6] = (float)ty.alpha;
    c[7] = (float)ty.r;
    c[8] = (float)(-expm1(-ty.alpha * ty.dz));
    c[9] = (float)ty.gamma;
    c[10] = (float)ty.beta2;
    c[11] = (float)(kPi * ty.beta3);
  }
}

// One batch of islands (items b0 .. b0 + kSpansBatch - 1 of `list`) of one link walked span by span.
template <int ORD>
__device__ __forceinline__ void spans_batch(const LinkParams& p, const uint64_t* __restrict__ keys,
                                            const uint32_t* __restrict__ list, long long n_items,
                                            float* __restrict__ terms, long long n_isl, int rows_per_chunk, int kfp,
                                            long long b0, SpansShared& sh, float* dyn) {
  constexpr int KP = 2;
  auto& bs = sh.bs;
  auto& g_ab = sh.g_ab;
  auto& g_ow = sh.g_ow;
  auto& g_f3 = sh.g_f3;
  auto& g_ih = sh.g_ih;
  auto& ns = sh.ns;
  auto& red = sh.red;
  const int T = p.n_types, R = rows_per_chunk;
  const SpansLayout lay = spans_layout(dyn, T, R);
  float4* const sqa = lay.sqa;
  float4* const sqb = lay.sqb;
  float2* const skc = lay.skc;
  const float* const tyc = lay.tyc;
  float* const tabf = lay.tabf;
  const bool fib_tab = ORD == ORD_DW && p.n_fib > 0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = p.gl.n;
  const float k4 = (float)(4.0 * kPi * kPi);
  const float pi_f = 3.14159265358979f;
  int tpr = 1;
  while (tpr * KP < n) tpr <<= 1;
  const int rows_per_pass = kThreads / tpr;
  const int lr = tid & (tpr - 1);
  const int rsub = tid / tpr;
    if (tid < kSpansBatch) batch_setup<ORD>(p, keys, list, n_items, b0, bs, tid);
    __syncthreads();
    const int nb = (int)min((long long)kSpansBatch, n_items - b0);
    for (int ib = 0; ib < nb; ++ib) {
      const int np = bs.np[ib];
      const int flags = bs.flags[ib];
      const bool want_g = flags & 1, want_h = flags & 2;
      const float sa1 = bs.ra[0][ib], sa2 = bs.ra[1][ib], sa3 = bs.ra[2][ib];
      const float si1 = bs.ri[0][ib], si2 = bs.ri[1][ib], si3 = bs.ri[2][ib];
      const float dfl = dval(bs.dd[ib]);
      float dsum = 0.0f, csum = 0.0f, hre = 0.0f, him = 0.0f;
      const int no = np > 0 ? p.gl.order[np] : 0;
      const int rows = np * no;
      for (int c0 = 0; c0 < rows; c0 += R) {
        const int rc = min(R, rows - c0);
        // ---- row constants: phase per (row, type); the geometry by the type-0 slots
        for (int slot = tid; slot < rc * T; slot += kThreads) {
          const int rr = slot % rc, t = slot / rc;
          const int row = c0 + rr;
          const int pi = row / no, i = row - pi * no;
          const RowGeo g = row_geometry<ORD>(p, bs, ib, np, pi, i);
          const float* c = tyc + kSpanTypeFloats * t;
          const RowPhase q = row_phase(g, Df{c[0], c[1]}, Df{c[2], c[3]}, c[4], c[5]);
          sqa[t * R + rr] = make_float4(q.Q0r.hi, q.Q0r.lo, q.Q1.hi, q.Q1.lo);
          sqb[t * R + rr] = make_float4(q.Q2.hi, q.Q2.lo, q.Q3, q.Q0r.hi - rint_fast(q.Q0r.hi));
          skc[t * R + rr] = make_float2(k4 * fmaf(c[11], dval(g.s0), c[10]), k4 * c[11] * dval(g.s1));
          if (t == 0) {
            const float imf = dval(g.im), ihf = dval(g.ih), of = dval(g.o);
            const float wo = dval(g.ph) * p.gl.wf[np][i];
            const float hout =
                ORD == ORD_DW ? rc_f(of, sa3, si3) : (ORD == ORD_E ? rc_f(of, sa2, si2) : rc_f(of, sa1, si1));
            g_ab[rr] = make_float4(dval(g.a0), dval(g.a1), dval(g.b0), dval(g.b1));
            g_ow[rr] = make_float4(ORD == ORD_DW ? of - dfl : of, wo * ihf * hout, wo * ihf, hout);
            const float nu3 = bs.nu3[ib];
            if (ORD == ORD_DW) g_f3[rr] = make_float4(nu3 + of, 0.0f, wo, imf);
            else g_f3[rr] = make_float4(nu3 + (imf + of + dfl), ihf, wo, imf);
            g_ih[rr] = ihf;
          }
        }
        __syncthreads();
        if (fib_tab) {  // c_k = C_k 2^{-zeta_k log2(e) f3} per fibre, row and segment
          for (int f = 0; f < p.n_fib; ++f) {
            const int Kfib = p.fib_K[f];
            for (int k = tid; k < Kfib; k += kThreads) {
              const float ck = p.fib_ck[f][k], zk = p.fib_zk[f][k];
              float* col = tabf + (size_t)f * R * kfp + k;
              for (int rr = 0; rr < rc; ++rr) col[rr * kfp] = ck * ex2_approx(-zk * g_f3[rr].x);
            }
          }
          __syncthreads();
        }
        for (int rb = 0; rb < rc; rb += rows_per_pass) {
          const int rr = rb + rsub;
          const bool row_ok = rr < rc;
          const int rrc = row_ok ? rr : 0;
          const float4 ab = g_ab[rrc], ow = g_ow[rrc], f3r = g_f3[rrc];
          const float im = f3r.w, ih = g_ih[rrc];
          const float wrowh = row_ok ? ow.y : 0.0f, wrow = row_ok ? ow.z : 0.0f;
          float xh_[KP], wnode_[KP], f3_[KP], yre_[KP], yim_[KP], zre_[KP], zim_[KP];
          float mre_[KP], mim_[KP], ere_[KP], eim_[KP];
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const int j = lr + tpr * m;
            const bool jok = j < n;
            xh_[m] = ns.x4[jok ? j : 0].x;
            wnode_[m] = jok ? ns.x2[j].y : 0.0f;
            f3_[m] = fmaf(f3r.y, xh_[m], f3r.x);
            yre_[m] = yim_[m] = 0.0f;
            zre_[m] = 1.0f;
            zim_[m] = 0.0f;
            mre_[m] = mim_[m] = 0.0f;
            ere_[m] = 1.0f;
            eim_[m] = 0.0f;
          }
          int prev = -1;
          for (int sp = 0; sp < p.n_spans; ++sp) {
            const int t = p.span_type[sp];
            if (t != prev) {  // gamma_t mu_t and e^{2 pi i phi_t} of this span's type
              prev = t;
              const float4 qa = sqa[t * R + rrc], qb = sqb[t * R + rrc];
              const float2 kc = skc[t * R + rrc];
              const float* c = tyc + kSpanTypeFloats * t;
              const float Kf = c[4], invK = c[5], alpha = c[6], r = c[7], omr = c[8], gam = c[9];
              const int K = (int)Kf;
              float p_[KP], wm1_[KP], wi_[KP], chi_[KP], b1_[KP], b2_[KP];
#pragma unroll
              for (int m = 0; m < KP; ++m) {
                const int j = lr + tpr * m;
                const int jj = j < n ? j : 0;
                float th, ph;
                point_phase(qa, qb, ns.x4[jj], ns.x2[jj].x, Kf, invK, th, ph);
                const float ah = pi_f * th;
                const float sh = __sinf(ah), chh = __cosf(ah);
                const float t2r = -2.0f * r * sh;
                wm1_[m] = fmaf(t2r, sh, -omr);
                p_[m] = fmaf(2.0f, wm1_[m], 2.0f);
                wi_[m] = -t2r * chh;
                const float xh = xh_[m];
                chi_[m] = fmaf(ab.y, xh, ab.x) * fmaf(ab.w, xh, ab.z) * fmaf(kc.y, xh, kc.x);
                const float ang = 2.0f * pi_f * ph;
                ere_[m] = __cosf(ang);
                eim_[m] = __sinf(ang);
                b1_[m] = 0.0f;
                b2_[m] = 0.0f;
              }
              const float q = r * r;
              if (fib_tab) {  // the type's c_k: the first K entries of its fibre's row
                static_assert(KP == 2, "one f32x2 pair of points per thread");
                const float* trow = tabf + ((size_t)p.type_fib[t] * R + rrc) * kfp;  // 16-byte aligned
                const f32x2 pp = pack2(p_[0], p_[1]);
                f32x2 bb1, bb2;
                dw_recurrence<1>(trow, K, pack2(-q, -q), &pp, &bb1, &bb2);
                unpack2(bb1, b1_[0], b1_[1]);
                unpack2(bb2, b2_[0], b2_[1]);
              } else {  // c_k per point, segments in rounds of four (16-byte loads)
                const float* ckf = p.types_dev[t].seg.ck_f;
                const float* zkf = p.types_dev[t].seg.zeta_f;
                auto step = [&](float ck, float zk) {
#pragma unroll
                  for (int m = 0; m < KP; ++m) {
                    const float cc = ck * ex2_approx(-zk * f3_[m]);
                    const float bn = fmaf(p_[m], b1_[m], fmaf(-q, b2_[m], cc));
                    b2_[m] = b1_[m];
                    b1_[m] = bn;
                  }
                };
                int k = K - 1;
                for (int e = K & 3; e > 0; --e, --k) step(ckf[k], zkf[k]);  // peel: k + 1 = 0 (mod 4)
#pragma unroll 1
                for (; k >= 3; k -= 4) {
                  const float4 c4 = *reinterpret_cast<const float4*>(ckf + k - 3);
                  const float4 z4 = *reinterpret_cast<const float4*>(zkf + k - 3);
                  step(c4.w, z4.w);
                  step(c4.z, z4.z);
                  step(c4.y, z4.y);
                  step(c4.x, z4.x);
                }
              }
#pragma unroll
              for (int m = 0; m < KP; ++m) {
                const float wm1 = wm1_[m], wi = wi_[m], chi = chi_[m];
                const float sre = fmaf(-(wm1 + 1.0f), b2_[m], b1_[m]);
                const float sim = wi * b2_[m];
                const float inv = rcp_approx(fmaf(chi, chi, alpha * alpha)) * gam;
                const float qr = fmaf(-alpha, wm1, chi * wi) * inv;
                const float qi = fmaf(-chi, wm1, -alpha * wi) * inv;
                mre_[m] = fmaf(sre, qr, -sim * qi);  // gamma_t mu_t
                mim_[m] = fmaf(sre, qi, sim * qr);
              }
            }
#pragma unroll
            for (int m = 0; m < KP; ++m) {
              yre_[m] = fmaf(mre_[m], zre_[m], fmaf(-mim_[m], zim_[m], yre_[m]));
              yim_[m] = fmaf(mre_[m], zim_[m], fmaf(mim_[m], zre_[m], yim_[m]));
              const float zr = fmaf(zre_[m], ere_[m], -zim_[m] * eim_[m]);
              zim_[m] = fmaf(zre_[m], eim_[m], zim_[m] * ere_[m]);
              zre_[m] = zr;
            }
          }
          // weights and sums (Upsilon itself, gamma included)
          float gre = 0.0f, gim = 0.0f;
#pragma unroll
          for (int m = 0; m < KP; ++m) {
            const float tt = fmaf(ih, xh_[m], im);
            float u, v, h3;
            if (ORD == ORD_DW) { u = tt; v = ow.x - tt; h3 = 1.0f; }
            else {
              if (ORD == ORD_E) { v = ow.x; u = tt; } else { u = ow.x; v = tt; }
              h3 = rc_f(u + v + dfl, sa3, si3);
            }
            const float h1 = rc_f(u, sa1, si1), h2 = rc_f(v, sa2, si2);
            const float yre = yre_[m], yim = yim_[m];
            if (ORD == ORD_DW) {
              dsum = fmaf((wrowh * wnode_[m]) * (h1 * h2), fmaf(yre, yre, yim * yim), dsum);
              if (want_g) {
                const float a12 = (row_ok ? wnode_[m] : 0.0f) * sqrtf(h1 * h2);
                gre = fmaf(a12, yre, gre);
                gim = fmaf(a12, yim, gim);
              }
              if (want_h) {
                const float a123 = wrow * wnode_[m] * sqrtf(h1 * h2 * ow.w);
                hre = fmaf(a123, yre, hre);
                him = fmaf(a123, yim, him);
              }
            } else {
              const float a = (row_ok ? wnode_[m] : 0.0f) * ih * sqrtf(ORD == ORD_E ? h1 * h3 : h2 * h3);
              gre = fmaf(a, yre, gre);
              gim = fmaf(a, yim, gim);
            }
          }
          if (ORD != ORD_DW || want_g) {
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
        __syncthreads();
      }
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
        for (int a = 0; a < 4; ++a) t[a] = warp_sum<kThreads / 32>(red[a]);
        const long long isl = bs.isl[ib];
        if (ORD == ORD_DW) {
          terms[isl] = bs.cf0[ib] * t[0];
          if (want_g) terms[3 * n_isl + isl] = bs.cf1[ib] * t[1];
          if (want_h) terms[4 * n_isl + isl] = bs.cf2[ib] * (t[2] * t[2] + t[3] * t[3]);
        } else {
          terms[(ORD == ORD_E ? 1 : 2) * n_isl + isl] = bs.cf0[ib] * t[1];
        }
      }
      __syncthreads();
    }
}

template <int ORD>
__global__ void __launch_bounds__(kThreads, kSpansCtas)
integrate_fp32c_spans_kernel(LinkParams p, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ list,
                             long long n_items, float* __restrict__ terms, long long n_isl, int rows_per_chunk,
                             int kfp) {
  __shared__ SpansShared sh;
  extern __shared__ __align__(16) float dyn[];
  load_node_sm(p, sh.ns);
  spans_types(p, spans_layout(dyn, p.n_types, rows_per_chunk).tyc);
  __syncthreads();
  for (long long b0 = (long long)blockIdx.x * kSpansBatch; b0 < n_items; b0 += (long long)gridDim.x * kSpansBatch)
    spans_batch<ORD>(p, keys, list, n_items, terms, n_isl, rows_per_chunk, kfp, b0, sh, dyn);
}

template <int ORD>
cudaError_t launch_spans(const LinkParams& p, const uint64_t* keys, const uint32_t* list, long long n_items,
                         float* terms, long long n_isl, cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  const int T = p.n_types;
  const int per_type = (int)(2 * sizeof(float4) + sizeof(float2));
  int kfp = 0;  // row stride of the fibre tables (DW): the longest fibre's K, 4 (mod 8)
  if (ORD == ORD_DW && p.n_fib > 0) {
    for (int f = 0; f < p.n_fib; ++f) kfp = std::max(kfp, p.fib_K[f]);
    kfp = (kfp + 3) & ~3;
    if ((kfp & 7) == 0) kfp += 4;
  }
  const int per_row = T * per_type + (ORD == ORD_DW ? p.n_fib * kfp * (int)sizeof(float) : 0);
  // 12 bytes of the budget reserved for the fibre tables' 16-byte alignment
  int rows = (kSpansDynBytes - 12 - T * kSpanTypeFloats * (int)sizeof(float)) / per_row;
  if (rows > kGRows) rows = kGRows;
  if (rows < 1) return cudaErrorInvalidValue;  // not reached: 64 types and 4 fibres of K 1024 leave 2 rows
  const size_t smem = (size_t)spans_head_floats(T, rows) * sizeof(float) +
                      (ORD == ORD_DW ? (size_t)p.n_fib * rows * kfp * sizeof(float) : 0);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = opt_in_smem(integrate_fp32c_spans_kernel<ORD>, kSpansDynBytes, attr_done)) return e;
  long long batches = (n_items + kSpansBatch - 1) / kSpansBatch;
  long long blocks = (long long)sms * kSpansCtas;
  if (blocks > batches) blocks = batches;
  integrate_fp32c_spans_kernel<ORD><<<(unsigned)blocks, kThreads, smem, st>>>(p, keys, list, n_items, terms, n_isl,
                                                                             rows, kfp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Multi-link passes (a batch of links, FP32C).  One pass of several links is one
// launch per kernel family: the island batches of the links' work lists are
// numbered across the links (link j owns batches first_batch_j ..
// first_batch_{j+1} - 1), a CTA takes batches gb = blockIdx.x, blockIdx.x +
// gridDim.x, ..., finds each one's link by binary search in the job table and
// evaluates it with that link's parameters exactly as the single-link kernels
// do; a CTA moving to another link forms that link's constants first.
// ---------------------------------------------------------------------------

struct LinkJob {
  LinkParams p;
  const uint64_t* keys;
  const uint32_t* list;
  long long n_items;
  float* terms;
  long long n_isl;
  long long first_batch;
  int rows;  // rows per chunk
  int kpad;  // identical spans: row stride of the c_k table
  int kfp;   // span by span: row stride of the fibre tables
  Df G0, G1; // identical spans: 2 pi L beta2, 2 pi^2 L beta3
  GenTypes gt;  // up to kMaxTypes span types
};

// The last job whose first batch is at most gb.
__device__ __forceinline__ int find_job(const LinkJob* __restrict__ jobs, int n_jobs, long long gb) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].first_batch <= gb) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int ORD>
__global__ void __launch_bounds__(kDwThreads, min_ctas(ORD, 4, kDwThreads))
integrate_fp32c_multi_kernel(const LinkJob* __restrict__ jobs, int n_jobs, long long batches) {
  constexpr int KP = 4, NT = kDwThreads, NB = batch_of(ORD, KP, NT);
  __shared__ DwShared<ORD, KP, NT> sh;
  const int npad = threads_per_row(jobs[0].p.gl.n, KP) * KP;  // every link of a batch has the same order
  extern __shared__ __align__(16) float dyn[];
  float4* const nx4 = reinterpret_cast<float4*>(dyn);
  float2* const nx2 = reinterpret_cast<float2*>(dyn + 4 * npad);
  float* const tab = dyn + node_floats(npad);
  load_nodes<NT>(jobs[0].p, npad, nx4, nx2);
  int cur = 0;
  bool have_rows = false;
  int job = -1;
  DwConsts cst{};
  for (long long gb = blockIdx.x; gb < batches; gb += gridDim.x) {
    const int j = find_job(jobs, n_jobs, gb);
    const LinkJob& J = jobs[j];
    if (j != job) {  // another link: its constants, and a c_k table that holds none of its rows
      job = j;
      cst = dw_consts(J.p);
      if (threadIdx.x == 0) sh.tab_rows = -1;  // read after the batch set-up's barrier
    }
    dw_batch<ORD, KP, NT>(J.p, cst, J.keys, J.list, J.n_items, J.terms, J.n_isl, J.rows, J.kpad, J.G0, J.G1,
                          (gb - J.first_batch) * NB, sh, nx4, nx2, tab, cur, have_rows);
  }
}

template <int ORD>
__global__ void __launch_bounds__(kThreads, 3)
integrate_fp32c_general_multi_kernel(const LinkJob* __restrict__ jobs, int n_jobs, long long batches) {
  __shared__ GenShared sh;
  extern __shared__ __align__(16) float tabg[];
  load_node_sm(jobs[0].p, sh.ns);
  int job = -1;
  for (long long gb = blockIdx.x; gb < batches; gb += gridDim.x) {
    const int j = find_job(jobs, n_jobs, gb);
    const LinkJob& J = jobs[j];
    if (j != job) {  // the previous batch ended on a barrier
      job = j;
      gen_types(J.p, sh);
      __syncthreads();
    }
    gen_batch<ORD>(J.p, J.gt, J.keys, J.list, J.n_items, J.terms, J.n_isl, J.rows, (gb - J.first_batch) * kBatch, sh,
                   tabg);
  }
}

template <int ORD>
__global__ void __launch_bounds__(kThreads, kSpansCtas)
integrate_fp32c_spans_multi_kernel(const LinkJob* __restrict__ jobs, int n_jobs, long long batches) {
  __shared__ SpansShared sh;
  extern __shared__ __align__(16) float dyn[];
  load_node_sm(jobs[0].p, sh.ns);
  int job = -1;
  for (long long gb = blockIdx.x; gb < batches; gb += gridDim.x) {
    const int j = find_job(jobs, n_jobs, gb);
    const LinkJob& J = jobs[j];
    if (j != job) {  // the previous batch ended on a barrier
      job = j;
      spans_types(J.p, spans_layout(dyn, J.p.n_types, J.rows).tyc);
      __syncthreads();
    }
    spans_batch<ORD>(J.p, J.keys, J.list, J.n_items, J.terms, J.n_isl, J.rows, J.kfp, (gb - J.first_batch) * kSpansBatch,
                     sh, dyn);
  }
}

// Launch shape of one link in a pass of its family, as the single-link launchers
// choose it: rows per chunk, table strides, the phase constants, the dynamic
// shared memory and the island batches.
struct JobShape {
  int rows = 0, kpad = 0, kfp = 0;
  Df G0{}, G1{};
  GenTypes gt{};
  size_t smem = 0;
  long long batches = 0;
};

JobShape job_shape(int ord, int family, const LinkParams& p, long long n_items) {
  JobShape s;
  if (family == 0) {
    const int K = p.seg.K;
    s.kpad = (K + 3) & ~3;
    if ((s.kpad & 7) == 0) s.kpad += 4;
    s.rows = rows_max(kDwThreads);
    if (ord == ORD_DW) s.rows = std::max(1, std::min(kTabFloats / s.kpad, rows_max(kDwThreads)));
    const int npad = threads_per_row(p.gl.n, 4) * 4;
    s.smem = ((size_t)node_floats(npad) + (ord == ORD_DW ? (size_t)s.rows * s.kpad : 0)) * sizeof(float);
    const double g0 = 2.0 * kPi * p.L * p.beta2, g1 = 2.0 * kPi * kPi * p.L * p.beta3;
    const float g0h = (float)g0, g1h = (float)g1;
    s.G0 = {g0h, (float)(g0 - (double)g0h)};
    s.G1 = {g1h, (float)(g1 - (double)g1h)};
    s.batches = (n_items + batch_of(ord, 4, kDwThreads) - 1) / batch_of(ord, 4, kDwThreads);
  } else if (family == 1) {
    int ktot = 0;
    for (int t = 0; t < p.n_types; ++t) {
      const SpanType& ty = p.types[t];
      const double g0 = 2.0 * kPi * ty.L * ty.beta2, g1 = 2.0 * kPi * kPi * ty.L * ty.beta3;
      const float g0h = (float)g0, g1h = (float)g1;
      s.gt.G0[t] = {g0h, (float)(g0 - (double)g0h)};
      s.gt.G1[t] = {g1h, (float)(g1 - (double)g1h)};
      s.gt.koff[t] = ktot;
      ktot += ty.seg.K;
    }
    s.gt.ktot = ktot;
    s.rows = kGRows;
    if (ord == ORD_DW) s.rows = std::max(1, std::min(kGTab / ktot, kGRows));
    s.smem = ord == ORD_DW ? (size_t)s.rows * ktot * sizeof(float) : 0;
    s.batches = (n_items + kBatch - 1) / kBatch;
  } else {
    const int T = p.n_types;
    const int per_type = (int)(2 * sizeof(float4) + sizeof(float2));
    if (ord == ORD_DW && p.n_fib > 0) {
      for (int f = 0; f < p.n_fib; ++f) s.kfp = std::max(s.kfp, p.fib_K[f]);
      s.kfp = (s.kfp + 3) & ~3;
      if ((s.kfp & 7) == 0) s.kfp += 4;
    }
    const int per_row = T * per_type + (ord == ORD_DW ? p.n_fib * s.kfp * (int)sizeof(float) : 0);
    s.rows = std::min((kSpansDynBytes - 12 - T * kSpanTypeFloats * (int)sizeof(float)) / per_row, kGRows);
    s.smem = (size_t)spans_head_floats(T, s.rows) * sizeof(float) +
             (ord == ORD_DW ? (size_t)p.n_fib * s.rows * s.kfp * sizeof(float) : 0);
    s.batches = (n_items + kSpansBatch - 1) / kSpansBatch;
  }
  return s;
}

template <int ORD>
cudaError_t launch_multi_ord(const MultiLaunch& m, const void* d_jobs, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const LinkJob* jobs = (const LinkJob*)d_jobs;
  if (m.family == 0) {
    static std::atomic<unsigned long long> done{0};
    e = opt_in_smem(integrate_fp32c_multi_kernel<ORD>, (node_floats(2 * kMaxGl) + kTabFloats) * (int)sizeof(float),
                    done);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((long long)sms * min_ctas(ORD, 4, kDwThreads), m.batches);
    integrate_fp32c_multi_kernel<ORD><<<(unsigned)blocks, kDwThreads, m.smem, st>>>(jobs, m.n_jobs, m.batches);
  } else if (m.family == 1) {
    static std::atomic<unsigned long long> done{0};
    e = opt_in_smem(integrate_fp32c_general_multi_kernel<ORD>, kGTab * (int)sizeof(float), done);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((long long)sms * 3, m.batches);
    integrate_fp32c_general_multi_kernel<ORD><<<(unsigned)blocks, kThreads, m.smem, st>>>(jobs, m.n_jobs, m.batches);
  } else {
    static std::atomic<unsigned long long> done{0};
    e = opt_in_smem(integrate_fp32c_spans_multi_kernel<ORD>, kSpansDynBytes, done);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((long long)sms * kSpansCtas, m.batches);
    integrate_fp32c_spans_multi_kernel<ORD><<<(unsigned)blocks, kThreads, m.smem, st>>>(jobs, m.n_jobs, m.batches);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fp32c_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                              long long n_items, float* terms, long long n_isl, cudaStream_t st) {
  if (p.rule == RULE_RIDGE) return launch_ridge_fp32c(ord, p, keys, list, n_items, terms, n_isl, st);
  if (p.n_types > kMaxTypes) {
    if (ord == ORD_DW) return launch_spans<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
    if (ord == ORD_E) return launch_spans<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
    return launch_spans<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (p.n_types > 1) {
    if (ord == ORD_DW) return launch_general<ORD_DW>(p, keys, list, n_items, terms, n_isl, st);
    if (ord == ORD_E) return launch_general<ORD_E>(p, keys, list, n_items, terms, n_isl, st);
    return launch_general<ORD_F>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (ord == ORD_DW) {
    if (p.fp32c_kp == 8) return launch_one<ORD_DW, 8, 128>(p, keys, list, n_items, terms, n_isl, st);
    if (p.fp32c_kp == 2) return launch_one<ORD_DW, 2, 128>(p, keys, list, n_items, terms, n_isl, st);
    return launch_one<ORD_DW, 4, kDwThreads>(p, keys, list, n_items, terms, n_isl, st);
  }
  if (ord == ORD_E) return launch_one<ORD_E, 4, kDwThreads>(p, keys, list, n_items, terms, n_isl, st);
  return launch_one<ORD_F, 4, kDwThreads>(p, keys, list, n_items, terms, n_isl, st);
}


int fp32c_family(const LinkParams& p) { return p.n_types > kMaxTypes ? 2 : (p.n_types > 1 ? 1 : 0); }

size_t fp32c_multi_bytes(int n_links) { return (size_t)std::max(n_links, 1) * sizeof(LinkJob); }

cudaError_t fp32c_multi_build(int ord, int family, const FlatPass* links, int n, void* image, MultiLaunch* out) {
  if (n < 1 || !links || !image || !out || ord < 0 || ord > 2 || family < 0 || family > 2) return cudaErrorInvalidValue;
  LinkJob* jobs = (LinkJob*)image;
  long long batches = 0;
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    const FlatPass& f = links[i];
    if (fp32c_family(*f.p) != family || (i > 0 && f.p->gl.n != links[0].p->gl.n)) return cudaErrorInvalidValue;
    const JobShape js = job_shape(ord, family, *f.p, f.n_items);
    if (js.rows < 1) return cudaErrorInvalidValue;  // not reached: the single-link checks hold for every link
    LinkJob& J = jobs[i];
    std::memset((void*)&J, 0, sizeof(LinkJob));
    J.p = *f.p;
    J.keys = f.keys;
    J.list = f.list;
    J.n_items = f.n_items;
    J.terms = f.terms;
    J.n_isl = f.n_isl;
    J.first_batch = batches;
    J.rows = js.rows;
    J.kpad = js.kpad;
    J.kfp = js.kfp;
    J.G0 = js.G0;
    J.G1 = js.G1;
    J.gt = js.gt;
    batches += js.batches;
    smem = std::max(smem, js.smem);
  }
  out->ord = ord;
  out->family = family;
  out->n_jobs = n;
  out->batches = batches;
  out->smem = smem;
  return cudaSuccess;
}

cudaError_t launch_fp32c_multi(const MultiLaunch& m, const void* d_jobs, cudaStream_t st) {
  if (m.batches <= 0) return cudaSuccess;
  if (m.ord == ORD_DW) return launch_multi_ord<ORD_DW>(m, d_jobs, st);
  if (m.ord == ORD_E) return launch_multi_ord<ORD_E>(m, d_jobs, st);
  return launch_multi_ord<ORD_F>(m, d_jobs, st);
}

}  // namespace egn
