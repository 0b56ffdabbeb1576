// api.cu -- C ABI of the ISRS EGN integrator: validation, unit conversion, link
// and segment tables, workspace management and the launch sequence
//   plan (A1) -> integrate (A3-A8) -> assemble (A9)
// on one CUDA stream.  See include/egn.h for the contract of every entry point.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "link.h"

namespace egn_host {

thread_local std::string g_last_error;
std::atomic<long long> g_alloc_count{0};

egn_status fail(egn_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

unsigned fault_mask() {
  const char* v = std::getenv("EGN_FAULT");
  if (!v || !*v) return 0;
  unsigned m = 0;
  const std::string s(v);
  for (size_t i = 0; i <= s.size();) {
    size_t j = s.find(',', i);
    if (j == std::string::npos) j = s.size();
    const std::string w = s.substr(i, j - i);
    if (w == "alloc") m |= kFaultAlloc;
    else if (w == "h2d") m |= kFaultH2D;
    else if (w == "launch") m |= kFaultLaunch;
    i = j + 1;
  }
  return m;
}

}  // namespace egn_host

using namespace egn_host;


namespace egn {

// Gauss-Legendre nodes and weights on [-1, 1] (gl_node), nodes ascending.
void gauss_legendre(int n, double* x, double* w) {
  for (int k = 1; k <= (n + 1) / 2; ++k) {
    double xk, wk;
    gl_node(n, k, &xk, &wk);
    // xk is the k-th largest node; mirror to the k-th smallest
    x[n - k] = xk;
    w[n - k] = wk;
    x[k - 1] = -xk;
    w[k - 1] = wk;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

size_t workspace_bytes(int n_ch, const PlanCounts& c, int precision) {
  size_t n_rows = (size_t)n_ch * n_ch;
  size_t tsz = precision == EGN_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t b = 0;
  b += align256((size_t)c.n_isl * sizeof(uint64_t));
  b += align256((size_t)c.n_half * sizeof(uint32_t));
  b += align256((size_t)c.n_e * sizeof(uint32_t));
  b += align256((size_t)c.n_f * sizeof(uint32_t));
  b += align256(4 * n_rows * sizeof(uint32_t));
  b += align256(4 * (n_rows + 1) * sizeof(uint32_t));
  b += align256(4 * sizeof(unsigned long long));
  b += align256((size_t)c.n_half * sizeof(uint32_t));
  b += align256(4 * (size_t)n_ch * kGroupBlocks * sizeof(uint32_t));
  b += align256(2 * 4 * (size_t)n_ch * sizeof(uint32_t));
  b += align256(5 * (size_t)c.n_isl * tsz);
  b += align256((size_t)n_ch * sizeof(double));
  b += align256((size_t)n_ch * sizeof(double));
  b += align256(sizeof(int));
  return b;
}

Workspace carve_workspace(void* base, int n_ch, const PlanCounts& c, int precision) {
  size_t n_rows = (size_t)n_ch * n_ch;
  size_t tsz = precision == EGN_PREC_FP64 ? sizeof(double) : sizeof(float);
  char* p = (char*)base;
  Workspace w{};
  w.keys = (uint64_t*)p;
  p += align256((size_t)c.n_isl * sizeof(uint64_t));
  w.h_idx = (uint32_t*)p;
  p += align256((size_t)c.n_half * sizeof(uint32_t));
  w.e_idx = (uint32_t*)p;
  p += align256((size_t)c.n_e * sizeof(uint32_t));
  w.f_idx = (uint32_t*)p;
  p += align256((size_t)c.n_f * sizeof(uint32_t));
  w.row_cnt = (uint32_t*)p;
  p += align256(4 * n_rows * sizeof(uint32_t));
  w.row_off = (uint32_t*)p;
  p += align256(4 * (n_rows + 1) * sizeof(uint32_t));
  w.row_tot = (unsigned long long*)p;
  p += align256(4 * sizeof(unsigned long long));
  w.d_idx = (uint32_t*)p;
  p += align256((size_t)c.n_half * sizeof(uint32_t));
  w.grp_cnt = (uint32_t*)p;
  p += align256(4 * (size_t)n_ch * kGroupBlocks * sizeof(uint32_t));
  w.grp_off = (uint32_t*)p;
  p += align256(2 * 4 * (size_t)n_ch * sizeof(uint32_t));
  w.terms = (void*)p;
  p += align256(5 * (size_t)c.n_isl * tsz);
  w.out_eta = (double*)p;
  p += align256((size_t)n_ch * sizeof(double));
  w.out_pnli = (double*)p;
  p += align256((size_t)n_ch * sizeof(double));
  w.status = (int*)p;
  w.cap_isl = c.n_isl;
  w.cap_half = c.n_half;
  w.cap_e = c.n_e;
  w.cap_f = c.n_f;
  return w;
}

}  // namespace egn

namespace egn_host {

using namespace egn;

// Span in internal units; beta2 moved to the spectral centre fc_hz (Eq. 24
// frequencies are relative to f_c).
Span to_internal(const egn_span& s, double fc_hz) {
  Span o;
  o.alpha = s.alpha_db_per_km * std::log(10.0) / 10.0;
  double lam = s.lambda_ref_m;
  double k = lam * lam / (2.0 * kPi * kC);                      // s m
  double b2 = -(s.D_ps_nm_km * 1e-6) * k * 1e27;               // ps^2/km
  double b3 = k * k * (s.S_ps_nm2_km * 1e3 + 2.0 * (s.D_ps_nm_km * 1e-6) / lam) * 1e39;  // ps^3/km
  double df_thz = (fc_hz - kC / lam) * 1e-12;
  o.beta2 = b2 + 2.0 * kPi * b3 * df_thz;
  o.beta3 = b3;
  o.gamma = s.gamma_per_w_km;
  o.cr = s.cr_per_w_km_thz;
  o.L = s.length_m * 1e-3;
  return o;
}

egn_status check_opts(const egn_link* l, const egn_opts* o) {
  if (!l || !o) return fail(EGN_E_INVALID_ARG, "null link or options");
  if (l->n_ch <= 0) return fail(EGN_E_STATE, "egn_set_wdm has not been called");
  if (o->gl_order < 1 || o->gl_order > kMaxGl) return fail(EGN_E_INVALID_ARG, "gl_order %d not in [1, %d]", o->gl_order, kMaxGl);
  if (!finite_pos(o->dz_km)) return fail(EGN_E_INVALID_ARG, "dz_km must be positive");
  if (o->mu_form != EGN_MU_SEGMENT && o->mu_form != EGN_MU_MACLAURIN && o->mu_form != EGN_MU_INTEGRAL)
    return fail(EGN_E_INVALID_ARG, "unknown mu_form %d", o->mu_form);
  if (o->precision != EGN_PREC_FP64 && o->precision != EGN_PREC_FP32C)
    return fail(EGN_E_INVALID_ARG, "unknown precision %d", o->precision);
  if (o->mu_form != EGN_MU_SEGMENT && o->precision != EGN_PREC_FP64)
    return fail(EGN_E_UNSUPPORTED, "the Maclaurin and integral forms of mu run in FP64 only");
  if (o->terms != EGN_TERMS_GN && o->terms != EGN_TERMS_EGN) return fail(EGN_E_INVALID_ARG, "unknown terms %d", o->terms);
  if (o->timeout_ms < 0) return fail(EGN_E_INVALID_ARG, "timeout_ms < 0");
  if (!l->identical && (int)l->spans_si.size() > kMaxSpans)
    return fail(EGN_E_UNSUPPORTED, "links whose spans differ are limited to %d spans", kMaxSpans);
  double ksum = 0.0;
  for (const egn_span& t : l->type_si) {
    double kk = std::ceil(t.length_m * 1e-3 / o->dz_km);
    if (kk > kMaxK) return fail(EGN_E_INVALID_ARG, "K = ceil(L/dz) = %.0f exceeds %d", kk, kMaxK);
    ksum += kk;
  }
  // up to kMaxTypes types keep every type's c_k table of a row in shared memory
  if (!l->identical && (int)l->type_si.size() <= kMaxTypes && ksum > kMaxKSum)
    return fail(EGN_E_INVALID_ARG, "the span types need %.0f segments in all, more than %d", ksum, kMaxKSum);
  if (o->terms == EGN_TERMS_EGN && l->mixed_rates && l->any_corr)
    return fail(EGN_E_UNSUPPORTED, "EGN corrections with mixed symbol rates are not defined");
  if (l->rule == RULE_RIDGE) {
    if (o->precision != EGN_PREC_FP64 && !l->identical && (int)l->type_si.size() > kMaxTypes)
      return fail(EGN_E_UNSUPPORTED, "the ridge-resolving rule in FP32C takes at most %d span types (FP64: any spans)",
                  kMaxTypes);
    if (o->gl_order > kRidgeMaxN)
      return fail(EGN_E_INVALID_ARG, "ridge rule: %d nodes per piece, at most %d", o->gl_order, kRidgeMaxN);
  }
  return EGN_OK;
}


// (Re)build the segment and Gauss-Legendre tables for these options.
egn_status ensure_tables(egn_link* l, const egn_opts* o) {
  if (l->tab_dz != o->dz_km) {
    l->tab_dz = -1.0;  // invalid until every table is uploaded
    const int nt = (int)l->type_si.size();
    std::vector<Span> sp(nt);
    std::vector<int> Ks(nt);
    size_t bytes = 0;
    for (int t = 0; t < nt; ++t) {
      sp[t] = to_internal(l->type_si[t], l->fc_hz);
      Ks[t] = std::max(1, (int)std::ceil(sp[t].L / o->dz_km));
      bytes += align256(Ks[t] * sizeof(double)) * 2 + align256(Ks[t] * sizeof(float)) * 2;
    }
    EGN_ALLOC(l->d_seg.ensure(bytes));
    // every type's tables staged on the host and copied in one transfer
    std::vector<char> host(bytes, 0);
    char* base = (char*)l->d_seg.p;
    size_t off = 0;
    l->types.assign(nt, SpanType{});
    for (int t = 0; t < nt; ++t) {
      const Span& s = sp[t];
      const int K = Ks[t];
      double* zeta = (double*)(host.data() + off);
      double* ck = (double*)(host.data() + off + align256(K * sizeof(double)));
      float* zf = (float*)(host.data() + off + 2 * align256(K * sizeof(double)));
      float* cf = (float*)(host.data() + off + 2 * align256(K * sizeof(double)) + align256(K * sizeof(float)));
      for (int k = 0; k < K; ++k) {
        segment_entry(k, K, s.L, s.alpha, l->ptot * s.cr, l->btot, &zeta[k], &ck[k]);
        zf[k] = (float)(zeta[k] * 1.4426950408889634);  // log2(e)
        cf[k] = (float)ck[k];
      }
      SpanType& ty = l->types[t];
      ty.alpha = s.alpha;
      ty.beta2 = s.beta2;
      ty.beta3 = s.beta3;
      ty.gamma = s.gamma;
      ty.L = s.L;
      ty.dz = s.L / K;
      ty.r = std::exp(-s.alpha * ty.dz);
      ty.pcr = l->ptot * s.cr;
      ty.seg.K = K;
      ty.seg.zeta = (const double*)(base + ((char*)zeta - host.data()));
      ty.seg.ck = (const double*)(base + ((char*)ck - host.data()));
      ty.seg.zeta_f = (const float*)(base + ((char*)zf - host.data()));
      ty.seg.ck_f = (const float*)(base + ((char*)cf - host.data()));
      off += align256(K * sizeof(double)) * 2 + align256(K * sizeof(float)) * 2;
    }
    EGN_CUDA(h2d(base, host.data(), bytes));
    if (nt > kMaxTypes) {
      EGN_ALLOC(l->d_types.ensure(nt * sizeof(SpanType)));
      EGN_CUDA(h2d(l->d_types.p, l->types.data(), nt * sizeof(SpanType)));
    }
    l->seg = l->types[0].seg;
    l->K = l->types[0].seg.K;
    l->span = sp[0];
    l->tab_dz = o->dz_km;
  }
  if (l->tab_gl != o->gl_order) {
    l->tab_gl = -1;
    int n = o->gl_order;
    std::vector<char> host;
    size_t off[4][7] = {};
    size_t total = 0;
    int ord[4] = {0, n, (n + 1) / 2, (n + 2) / 3};
    for (int p = 1; p <= 3; ++p) {
      int m = ord[p];
      for (int a = 0; a < 2; ++a) { off[p][a] = total; total += align256(m * sizeof(double)); }
      for (int a = 2; a < 7; ++a) { off[p][a] = total; total += align256(m * sizeof(float)); }
    }
    // the ridge rule's pieces take every order 1..max(n, n_min): order m at offset
    // m (m - 1) / 2, tabulated up to max(n, kRidgeMaxN)
    const int m_all = std::max(n, kRidgeMaxN);
    const size_t n_all = (size_t)m_all * (m_all + 1) / 2;
    const size_t off_allx = total, off_allw = total + align256(n_all * sizeof(double));
    total += 2 * align256(n_all * sizeof(double));
    const size_t off_allxh = total, off_allxl = total + align256(n_all * sizeof(float)),
                 off_allwf = total + 2 * align256(n_all * sizeof(float));
    total += 3 * align256(n_all * sizeof(float));
    host.assign(total, 0);
    for (int m = 1; m <= m_all; ++m)
      gauss_legendre(m, (double*)(host.data() + off_allx) + (size_t)m * (m - 1) / 2,
                     (double*)(host.data() + off_allw) + (size_t)m * (m - 1) / 2);
    for (size_t i = 0; i < n_all; ++i) {
      const double x = ((const double*)(host.data() + off_allx))[i];
      const float xh = (float)x;
      ((float*)(host.data() + off_allxh))[i] = xh;
      ((float*)(host.data() + off_allxl))[i] = (float)(x - (double)xh);
      ((float*)(host.data() + off_allwf))[i] = (float)((const double*)(host.data() + off_allw))[i];
    }
    for (int p = 1; p <= 3; ++p) {
      int m = ord[p];
      std::vector<double> x(m), w(m);
      gauss_legendre(m, x.data(), w.data());
      double* hx = (double*)(host.data() + off[p][0]);
      double* hw = (double*)(host.data() + off[p][1]);
      float* xh = (float*)(host.data() + off[p][2]);
      float* xl = (float*)(host.data() + off[p][3]);
      float* x2h = (float*)(host.data() + off[p][4]);
      float* x2l = (float*)(host.data() + off[p][5]);
      float* wf = (float*)(host.data() + off[p][6]);
      for (int i = 0; i < m; ++i) {
        hx[i] = x[i];
        hw[i] = w[i];
        xh[i] = (float)x[i];
        xl[i] = (float)(x[i] - (double)xh[i]);
        double x2 = x[i] * x[i];
        x2h[i] = (float)x2;
        x2l[i] = (float)(x2 - (double)x2h[i]);
        wf[i] = (float)w[i];
      }
    }
    EGN_ALLOC(l->d_gl.ensure(total));
    EGN_CUDA(h2d(l->d_gl.p, host.data(), total));
    char* b = (char*)l->d_gl.p;
    l->gl.n = n;
    for (int p = 1; p <= 3; ++p) {
      l->gl.order[p] = ord[p];
      l->gl.x[p] = (const double*)(b + off[p][0]);
      l->gl.w[p] = (const double*)(b + off[p][1]);
      l->gl.xh[p] = (const float*)(b + off[p][2]);
      l->gl.xl[p] = (const float*)(b + off[p][3]);
      l->gl.x2h[p] = (const float*)(b + off[p][4]);
      l->gl.x2l[p] = (const float*)(b + off[p][5]);
      l->gl.wf[p] = (const float*)(b + off[p][6]);
    }
    l->gl.order[0] = 0;
    l->gl_all_x = (const double*)(b + off_allx);
    l->gl_all_w = (const double*)(b + off_allw);
    l->gl_all_xh = (const float*)(b + off_allxh);
    l->gl_all_xl = (const float*)(b + off_allxl);
    l->gl_all_wf = (const float*)(b + off_allwf);
    l->tab_gl = n;
  }
  return EGN_OK;
}

ChannelTable channel_table(const egn_link* l) {
  ChannelTable t;
  const double* b = (const double*)l->d_ch.p;
  size_t s = align256(l->n_ch * sizeof(double)) / sizeof(double);
  t.n_ch = l->n_ch;
  t.wmax = *std::max_element(l->W.begin(), l->W.end());
  t.nu = b;
  t.R = b + s;
  t.W = b + 2 * s;
  t.P = b + 3 * s;
  t.phi = b + 4 * s;
  t.psi = b + 5 * s;
  t.nu_f = (const float*)(b + 6 * s);  // the seventh array holds nu_f[n_ch] then hw_f[n_ch]
  t.hw_f = t.nu_f + l->n_ch;
  t.nu_coi = t.nu;
  t.nu_coi_f = t.nu_f;
  if (l->coi_shift) {
    t.nu_coi = (const double*)l->d_coi.p;
    t.nu_coi_f = (const float*)((const char*)l->d_coi.p + align256(l->n_ch * sizeof(double)));
  }
  t.hwmax_f = 0.5f * (float)t.wmax;
  double numax = 0.0;  // COI frequencies lie within half a support of a centre
  for (double x : l->nu) numax = std::max(numax, std::fabs(x) + 0.5 * t.wmax);
  // FP32 rounding of four centres, three half supports and five operations on
  // values up to 3 numax + 1.5 wmax: well inside 4e-6 (numax + wmax)
  t.plan_margin = (float)(4e-6 * (numax + t.wmax)) + 1e-30f;
  return t;
}

// Form of mu and the constants of its Maclaurin and integral variants.
void set_mu_params(LinkParams& p, const egn_link* l, const egn_opts* o) {
  p.mu_form = o->mu_form;
  p.btot = l->btot;
  struct Rule {
    double x[kMuGl], w[kMuGl];
    Rule() { gauss_legendre(kMuGl, x, w); }
  };
  static const Rule rule;  // initialised once, thread-safe
  for (int j = 0; j < kMuGl; ++j) {
    p.mgx[j] = rule.x[j];
    p.mgw[j] = rule.w[j];
  }
}

LinkParams link_params(const egn_link* l, const egn_opts* o, int all_terms) {
  LinkParams p{};
  p.ch = channel_table(l);
  p.gl = l->gl;
  p.seg = l->seg;
  p.n_spans = (int)l->spans_si.size();
  p.alpha = l->span.alpha;
  p.beta2 = l->span.beta2;
  p.beta3 = l->span.beta3;
  p.gamma = l->span.gamma;
  p.L = l->span.L;
  p.dz = l->span.L / l->K;
  p.r = std::exp(-l->span.alpha * p.dz);
  p.rolloff = l->rolloff;
  p.terms = o->terms;
  p.all_terms = all_terms;
  p.fp32c_kp = l->fp32c_kp;
  p.rule = l->rule;
  p.ridge_n_min = l->ridge_n_min;
  p.glx_all = l->gl_all_x;
  p.glw_all = l->gl_all_w;
  p.glxh_all = l->gl_all_xh;
  p.glxl_all = l->gl_all_xl;
  p.glwf_all = l->gl_all_wf;
  set_mu_params(p, l, o);
  p.n_types = l->identical ? 1 : (int)l->type_si.size();
  for (int t = 0; t < p.n_types && t < kMaxTypes; ++t) p.types[t] = l->types[t];
  p.types_dev = p.n_types > kMaxTypes ? (const SpanType*)l->d_types.p : nullptr;
  for (int s = 0; s < (int)l->span_type.size() && s < kMaxSpans; ++s) p.span_type[s] = l->span_type[s];
  // fibre groups of the span types (used by the span-by-span path)
  p.n_fib = 0;
  if (p.n_types > kMaxTypes && (int)l->types.size() == p.n_types) {
    int nf = 0, rep[kMaxFibres] = {};
    bool ok = true;
    for (int t = 0; t < p.n_types && ok; ++t) {
      const SpanType& ty = l->types[t];
      int f = 0;
      while (f < nf && !(l->types[rep[f]].alpha == ty.alpha && l->types[rep[f]].pcr == ty.pcr &&
                         l->types[rep[f]].dz == ty.dz))
        ++f;
      if (f == nf) {
        if (nf == kMaxFibres) { ok = false; break; }
        rep[nf++] = t;
      } else if (ty.seg.K > l->types[rep[f]].seg.K) {
        rep[f] = t;  // the longest type of the fibre holds every prefix
      }
      p.type_fib[t] = (unsigned char)f;
    }
    if (ok) {
      p.n_fib = nf;
      for (int f = 0; f < nf; ++f) {
        p.fib_ck[f] = l->types[rep[f]].seg.ck_f;
        p.fib_zk[f] = l->types[rep[f]].seg.zeta_f;
        p.fib_K[f] = l->types[rep[f]].seg.K;
      }
    }
  }
  return p;
}

// Integrator passes: D/G/H over the half list in any order (the planner's grouped
// copy of it; every island of `keys` when h_idx is null), then E and F over their lists (or over every island when
// all_terms is set).  ev, if given, is recorded after each pass.
cudaError_t integrate(const LinkParams& p, int precision, const uint64_t* keys, long long n_isl,
                      const uint32_t* h_idx, long long n_half, const uint32_t* e_idx, long long n_e,
                      const uint32_t* f_idx, long long n_f, void* terms, cudaStream_t st, cudaEvent_t* ev) {
  auto pass = [&](int ord, const uint32_t* list, long long n) {
    return precision == EGN_PREC_FP64 ? launch_fp64_pass(ord, p, keys, list, n, (double*)terms, n_isl, st)
                                      : launch_fp32c_pass(ord, p, keys, list, n, (float*)terms, n_isl, st);
  };
  bool corr = p.all_terms || p.terms;
  const uint32_t* el = p.all_terms ? nullptr : e_idx;
  const uint32_t* fl = p.all_terms ? nullptr : f_idx;
  long long ne = p.all_terms ? n_isl : (corr ? n_e : 0);
  long long nf = p.all_terms ? n_isl : (corr ? n_f : 0);
  cudaError_t e = pass(0, h_idx, h_idx ? n_half : n_isl);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = pass(1, el, ne);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) e = pass(2, fl, nf);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
  return e;
}

// Per-row offsets of the half list inside the planner's offset arrays.
const uint32_t* half_offsets(const Workspace& ws, int n_ch) { return ws.row_off + ((size_t)n_ch * n_ch + 1); }

// The whole step on one stream: plan -> integrate -> assemble.
egn_status run_step(egn_link* l, const egn_opts* o, const Workspace& ws, double* eta, double* pnli) {
  NvtxRange range("egn::run_step");
  cudaStream_t st = (cudaStream_t)o->stream;
  ChannelTable ch = channel_table(l);
  cudaEvent_t* ev = nullptr;
  l->prof_valid = false;
  if (l->prof_on) {
    for (auto& e : l->prof_ev)
      if (!e) EGN_CUDA(cudaEventCreate(&e));
    ev = l->prof_ev;
    EGN_CUDA(cudaEventRecord(ev[0], st));
  }
  EGN_LAUNCH_GATE();
  EGN_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), st));
  EGN_CUDA(launch_plan(ch, ws, st));
  if (ev) EGN_CUDA(cudaEventRecord(ev[1], st));
  LinkParams p = link_params(l, o, 0);
  EGN_CUDA(integrate(p, o->precision, ws.keys, l->cnt.n_isl, ws.d_idx, l->cnt.n_half, ws.e_idx, l->cnt.n_e,
                     ws.f_idx, l->cnt.n_f, ws.terms, st, ev ? ev + 2 : nullptr));
  EGN_CUDA(launch_assemble(ch, half_offsets(ws, l->n_ch), ws.keys, ws.h_idx, l->cnt.n_isl, ws.terms, o->precision,
                           o->terms, eta, pnli, st));
  if (ev) {
    EGN_CUDA(cudaEventRecord(ev[5], st));
    l->prof_valid = true;
  }
  return EGN_OK;
}

// Island counts of the link's channel table (COI frequencies included) from the
// planner's count pass: totals of the four lists and, if asked, per COI.
egn_status count_islands(egn_link* l, PlanCounts* cnt, std::vector<long long>* per_coi) {
  const int n_ch = l->n_ch;
  size_t n_rows = (size_t)n_ch * n_ch;
  size_t cnt_b = align256(4 * n_rows * sizeof(uint32_t)), off_b = align256(4 * (n_rows + 1) * sizeof(uint32_t));
  DevBuf& tmp = l->d_count;  // kept by the link: no allocation when the comb size repeats
  cudaError_t e = tmp.ensure(cnt_b + off_b + 4 * sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
  Workspace w{};
  w.row_cnt = (uint32_t*)tmp.p;
  w.row_off = (uint32_t*)((char*)tmp.p + cnt_b);
  w.row_tot = (unsigned long long*)((char*)tmp.p + cnt_b + off_b);
  e = launch_plan_count(channel_table(l), w, 0);
  std::vector<uint32_t> off(4 * (n_rows + 1));
  unsigned long long tot[4] = {};
  if (e == cudaSuccess) e = cudaMemcpy(off.data(), w.row_off, off.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(tot, w.row_tot, sizeof tot, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(EGN_E_CUDA, "island count: %s", cudaGetErrorString(e));
  // island indices and list offsets are 32-bit
  if (tot[0] > 0xffffffffull)
    return fail(EGN_E_UNSUPPORTED, "%llu islands: more than 2^32 - 1 (too many channels for one evaluation)", tot[0]);
  cnt->n_isl = off[n_rows];
  cnt->n_half = off[(n_rows + 1) + n_rows];
  cnt->n_e = off[2 * (n_rows + 1) + n_rows];
  cnt->n_f = off[3 * (n_rows + 1) + n_rows];
  if (per_coi) {
    per_coi->resize(n_ch);
    for (int c = 0; c < n_ch; ++c) (*per_coi)[c] = (long long)off[(size_t)(c + 1) * n_ch] - off[(size_t)c * n_ch];
  }
  return EGN_OK;
}

egn_status wait_event(cudaEvent_t ev, int timeout_ms) {
  auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return EGN_OK;
    if (e != cudaErrorNotReady) return fail(EGN_E_CUDA, "device error: %s", cudaGetErrorString(e));
    if (timeout_ms > 0) {
      auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
      if (ms > timeout_ms) return fail(EGN_E_TIMEOUT, "device work not finished after %d ms", timeout_ms);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

// Closed-form moments of an equiprobable square QAM with m levels per dimension
// from its 1-D PAM levels +-1, +-3, ..., +-(m-1).
void qam_moments(int m, double* phi, double* psi) {
  double e2 = 0, e4 = 0, e6 = 0;
  for (int i = 0; i < m; ++i) {
    double a = 2.0 * i - (m - 1);
    e2 += a * a;
    e4 += a * a * a * a;
    e6 += a * a * a * a * a * a;
  }
  e2 /= m;
  e4 /= m;
  e6 /= m;
  // |x + iy|^{2k} moments with x, y independent PAM
  double s2 = 2 * e2, s4 = 2 * e4 + 2 * e2 * e2, s6 = 2 * e6 + 6 * e4 * e2;
  double mu4 = s4 / (s2 * s2), mu6 = s6 / (s2 * s2 * s2);
  *phi = mu4 - 2.0;
  *psi = mu6 - 9.0 * mu4 + 12.0;
}

}  // namespace egn_host

extern "C" {

const char* egn_last_error(void) { return g_last_error.c_str(); }

const char* egn_version(void) { return "egn-gb300 0.2 (sm_103a)"; }

egn_status egn_allocation_count(long long* count) {
  if (!count) return fail(EGN_E_INVALID_ARG, "null output");
  *count = g_alloc_count.load(std::memory_order_relaxed);
  return EGN_OK;
}

egn_status egn_format_moments(int fmt, double* phi, double* psi) {
  if (!phi || !psi) return fail(EGN_E_INVALID_ARG, "null output");
  switch (fmt) {
    case EGN_FMT_GAUSS: *phi = 0.0; *psi = 0.0; return EGN_OK;
    case EGN_FMT_QPSK: qam_moments(2, phi, psi); return EGN_OK;
    case EGN_FMT_16QAM: qam_moments(4, phi, psi); return EGN_OK;
    case EGN_FMT_64QAM: qam_moments(8, phi, psi); return EGN_OK;
    default: return fail(EGN_E_INVALID_ARG, "unknown format %d", fmt);
  }
}

egn_status egn_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > 4096 || !x || !w) return fail(EGN_E_INVALID_ARG, "bad Gauss-Legendre request");
  egn::gauss_legendre(n, x, w);
  return EGN_OK;
}

egn_status egn_link_create(const egn_span* spans, int n_spans, egn_link** out) {
  if (!out) return fail(EGN_E_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (!spans || n_spans < 1) return fail(EGN_E_INVALID_ARG, "need at least one span");
  for (int i = 0; i < n_spans; ++i) {
    const egn_span& s = spans[i];
    if (!finite_pos(s.alpha_db_per_km)) return fail(EGN_E_INVALID_ARG, "span %d: alpha must be > 0", i);
    if (!finite_pos(s.lambda_ref_m)) return fail(EGN_E_INVALID_ARG, "span %d: lambda_ref must be > 0", i);
    if (!finite_pos(s.length_m)) return fail(EGN_E_INVALID_ARG, "span %d: length must be > 0", i);
    if (!std::isfinite(s.D_ps_nm_km) || !std::isfinite(s.S_ps_nm2_km))
      return fail(EGN_E_INVALID_ARG, "span %d: D and S must be finite", i);
    if (!(s.gamma_per_w_km >= 0.0) || !std::isfinite(s.gamma_per_w_km))
      return fail(EGN_E_INVALID_ARG, "span %d: gamma must be >= 0", i);
    if (!(s.cr_per_w_km_thz >= 0.0) || !std::isfinite(s.cr_per_w_km_thz))
      return fail(EGN_E_INVALID_ARG, "span %d: Cr must be >= 0", i);
  }
  egn_link* l = new (std::nothrow) egn_link();
  if (!l) return fail(EGN_E_NOMEM, "out of host memory");
  l->spans_si.assign(spans, spans + n_spans);
  for (int i = 0; i < n_spans; ++i) {
    if (std::memcmp(&spans[i], &spans[0], sizeof(egn_span)) != 0) l->identical = false;
    int t = 0;
    while (t < (int)l->type_si.size() && std::memcmp(&spans[i], &l->type_si[t], sizeof(egn_span)) != 0) ++t;
    if (t == (int)l->type_si.size()) l->type_si.push_back(spans[i]);
    l->span_type.push_back((unsigned char)std::min(t, 255));
  }
  *out = l;
  return EGN_OK;
}

void egn_link_destroy(egn_link* link) {
  if (!link) return;
  DeviceGuard g(link->device);
  delete link;
}

egn_status egn_set_wdm(egn_link* l, int n_ch, const double* centre_hz, const double* rate, const double* power,
                       const double* phi, const double* psi, double rolloff) {
  egn_status s_ = EGN_OK;
  if (!l) return fail(EGN_E_INVALID_ARG, "null link");
  if (n_ch < 1 || n_ch > 4096) return fail(EGN_E_INVALID_ARG, "n_ch %d not in [1, 4096]", n_ch);
  if (!centre_hz || !rate || !power || !phi || !psi) return fail(EGN_E_INVALID_ARG, "null channel array");
  if (!(rolloff >= 0.0 && rolloff <= 1.0)) return fail(EGN_E_INVALID_ARG, "rolloff must be in [0, 1]");
  for (int i = 0; i < n_ch; ++i) {
    if (!finite_pos(centre_hz[i]) || !finite_pos(rate[i]) || !finite_pos(power[i]))
      return fail(EGN_E_INVALID_ARG, "channel %d: centre, rate and power must be positive and finite", i);
    if (!std::isfinite(phi[i]) || !std::isfinite(psi[i])) return fail(EGN_E_INVALID_ARG, "channel %d: Phi/Psi not finite", i);
    if (i > 0) {
      if (!(centre_hz[i] > centre_hz[i - 1])) return fail(EGN_E_INVALID_ARG, "channel centres must increase");
      double gap = centre_hz[i] - centre_hz[i - 1];
      double need = 0.5 * (rate[i] + rate[i - 1]) * (1.0 + rolloff);
      if (gap < need * (1.0 - 1e-9)) return fail(EGN_E_INVALID_ARG, "channels %d and %d overlap", i - 1, i);
    }
  }
  int dev = 0;
  EGN_CUDA(cudaGetDevice(&dev));
  if (l->device >= 0 && l->device != dev) return fail(EGN_E_STATE, "link is bound to device %d", l->device);
  l->device = dev;
  l->n_ch = 0;  // invalid until complete
  double fmin = centre_hz[0], fmax = centre_hz[n_ch - 1];
  l->fc_hz = 0.5 * (fmin + fmax);
  l->rolloff = rolloff;
  l->nu.resize(n_ch);
  l->R.resize(n_ch);
  l->W.resize(n_ch);
  l->P.assign(power, power + n_ch);
  l->phi.assign(phi, phi + n_ch);
  l->psi.assign(psi, psi + n_ch);
  l->ptot = 0.0;
  l->mixed_rates = false;
  l->any_corr = false;
  for (int i = 0; i < n_ch; ++i) {
    l->nu[i] = (centre_hz[i] - l->fc_hz) * 1e-12;
    l->R[i] = rate[i] * 1e-12;
    l->W[i] = l->R[i] * (1.0 + rolloff);
    l->ptot += power[i];
    if (rate[i] != rate[0]) l->mixed_rates = true;
    if (phi[i] != 0.0 || psi[i] != 0.0) l->any_corr = true;
  }
  l->btot = n_ch > 1 ? (fmax - fmin) * 1e-12 * n_ch / (n_ch - 1) : l->R[0];
  // channel table
  size_t s = align256(n_ch * sizeof(double));
  EGN_ALLOC(l->d_ch.ensure(7 * s));
  const std::vector<double>* arr[6] = {&l->nu, &l->R, &l->W, &l->P, &l->phi, &l->psi};
  for (int a = 0; a < 6; ++a)
    EGN_CUDA(h2d((char*)l->d_ch.p + a * s, arr[a]->data(), n_ch * sizeof(double)));
  {
    std::vector<float> f32(2 * (size_t)n_ch);
    for (int i = 0; i < n_ch; ++i) {
      f32[i] = (float)l->nu[i];
      f32[n_ch + i] = 0.5f * (float)l->W[i];
    }
    EGN_CUDA(h2d((char*)l->d_ch.p + 6 * s, f32.data(), f32.size() * sizeof(float)));
  }
  l->tab_dz = -1.0;  // P_tot and B_tot changed
  // count islands on the device
  l->n_ch = n_ch;
  s_ = count_islands(l, &l->cnt, &l->per_coi);
  if (s_ != EGN_OK) {
    l->n_ch = 0;
    return s_;
  }
  // pinned staging for host outputs
  const size_t stage_n = 2 * (size_t)n_ch + 2;  // kept while large enough (a comb changed in place)
  if (!l->h_stage || l->h_stage_n < stage_n) {
    if (l->h_stage) cudaFreeHost(l->h_stage);
    l->h_stage = nullptr;
    l->h_stage_n = 0;
    cudaError_t e = pinned_alloc((void**)&l->h_stage, stage_n * sizeof(double));
    if (e != cudaSuccess) {
      l->h_stage = nullptr;
      l->n_ch = 0;
      return fail(EGN_E_NOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
    }
    l->h_stage_n = stage_n;
  }
  return EGN_OK;
}

egn_status egn_island_count(const egn_link* l, long long* total, long long* per_coi, long long* n_half,
                            long long* n_e, long long* n_f) {
  if (!l) return fail(EGN_E_INVALID_ARG, "null link");
  if (l->n_ch <= 0) return fail(EGN_E_STATE, "egn_set_wdm has not been called");
  if (total) *total = l->cnt.n_isl;
  if (n_half) *n_half = l->cnt.n_half;
  if (n_e) *n_e = l->cnt.n_e;
  if (n_f) *n_f = l->cnt.n_f;
  if (per_coi) std::copy(l->per_coi.begin(), l->per_coi.end(), per_coi);
  return EGN_OK;
}

egn_status egn_workspace_size(const egn_link* l, const egn_opts* o, size_t* bytes) {
  if (!bytes) return fail(EGN_E_INVALID_ARG, "null output");
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  *bytes = workspace_bytes(l->n_ch, l->cnt, o->precision);
  return EGN_OK;
}

egn_status egn_nli_eta_device(egn_link* l, const egn_opts* o, void* workspace, size_t workspace_bytes_,
                              double* eta_dev, double* pnli_dev) {
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(EGN_E_INVALID_ARG, "workspace must be 256-byte aligned");
  size_t need = workspace_bytes(l->n_ch, l->cnt, o->precision);
  if (workspace_bytes_ < need) return fail(EGN_E_CAPACITY, "workspace %zu bytes < %zu needed", workspace_bytes_, need);
  DeviceGuard g(l->device);
  s = ensure_tables(l, o);
  if (s != EGN_OK) return s;
  Workspace ws = carve_workspace(workspace, l->n_ch, l->cnt, o->precision);
  return run_step(l, o, ws, eta_dev ? eta_dev : ws.out_eta, pnli_dev ? pnli_dev : ws.out_pnli);
}

egn_status egn_nli_eta(egn_link* l, const egn_opts* o, double* eta, double* pnli) {
  NvtxRange range("egn_nli_eta");
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  DeviceGuard g(l->device);
  size_t need = workspace_bytes(l->n_ch, l->cnt, o->precision);
  cudaError_t e = l->ws.ensure(need);
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "workspace cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
  s = egn_nli_eta_device(l, o, l->ws.p, l->ws.bytes, nullptr, nullptr);
  if (s != EGN_OK) return s;
  Workspace ws = carve_workspace(l->ws.p, l->n_ch, l->cnt, o->precision);
  cudaStream_t st = (cudaStream_t)o->stream;
  int n = l->n_ch;
  EGN_CUDA(cudaMemcpyAsync(l->h_stage, ws.out_eta, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  EGN_CUDA(cudaMemcpyAsync(l->h_stage + n, ws.out_pnli, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  EGN_CUDA(cudaMemcpyAsync(l->h_stage + 2 * n, ws.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  cudaEvent_t ev;
  EGN_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t re = cudaEventRecord(ev, st);
  if (re != cudaSuccess) { cudaEventDestroy(ev); return fail(EGN_E_CUDA, "cudaEventRecord: %s", cudaGetErrorString(re)); }
  s = wait_event(ev, o->timeout_ms);
  cudaEventDestroy(ev);
  if (s != EGN_OK) return s;
  int status = 0;
  std::memcpy(&status, l->h_stage + 2 * n, sizeof(int));
  if (status) return fail(EGN_E_CUDA, "device planner overflow (status %d)", status);
  if (eta) std::memcpy(eta, l->h_stage, n * sizeof(double));
  if (pnli) std::memcpy(pnli, l->h_stage + n, n * sizeof(double));
  return EGN_OK;
}

egn_status egn_nli_eta_3d(egn_link* l, const egn_opts* o, int n_f, double* eta, double* pnli) {
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  if (n_f < 1 || n_f > 64) return fail(EGN_E_INVALID_ARG, "n_f %d not in [1, 64]", n_f);
  DeviceGuard g(l->device);
  const int n = l->n_ch;
  const size_t dbytes = align256(n * sizeof(double));
  cudaStream_t st = (cudaStream_t)o->stream;
  EGN_CUDA(cudaStreamSynchronize(st));  // nothing queued by an earlier call may still read d_coi
  EGN_ALLOC(l->d_coi.ensure(dbytes + align256(n * sizeof(float))));
  std::vector<double> x(n_f), w(n_f), acc(n, 0.0), pj(n), nc(n);
  std::vector<float> ncf(n);
  gauss_legendre(n_f, x.data(), w.data());
  // every node is a full evaluation with the COI frequencies moved and the
  // islands counted for them; the link's own counts and tables are restored after
  struct Restore {
    egn_link* l;
    PlanCounts c;
    ~Restore() {
      l->cnt = c;
      l->coi_shift = false;
    }
  } restore{l, l->cnt};
  for (int j = 0; j < n_f; ++j) {
    for (int i = 0; i < n; ++i) {
      nc[i] = l->nu[i] + 0.5 * x[j] * l->R[i];
      ncf[i] = (float)nc[i];
    }
    l->coi_shift = false;
    EGN_CUDA(h2d(l->d_coi.p, nc.data(), n * sizeof(double)));
    EGN_CUDA(h2d((char*)l->d_coi.p + dbytes, ncf.data(), n * sizeof(float)));
    l->coi_shift = true;
    PlanCounts cnt{};
    s = count_islands(l, &cnt, nullptr);
    if (s != EGN_OK) return s;
    l->cnt = cnt;
    s = egn_nli_eta(l, o, nullptr, pj.data());
    if (s != EGN_OK) return s;
    for (int i = 0; i < n; ++i) acc[i] += 0.5 * w[j] * pj[i];
  }
  for (int i = 0; i < n; ++i) {
    if (pnli) pnli[i] = acc[i];
    if (eta) eta[i] = acc[i] / (l->P[i] * l->P[i] * l->P[i]);
  }
  return EGN_OK;
}

egn_status egn_set_tuning(egn_link* l, int param, int value) {
  if (!l) return fail(EGN_E_INVALID_ARG, "null link");
  switch (param) {
    case EGN_TUNE_FP32C_POINTS_PER_THREAD:
      if (value != 2 && value != 4 && value != 8) return fail(EGN_E_INVALID_ARG, "points per thread must be 2, 4 or 8");
      l->fp32c_kp = value;
      return EGN_OK;
    default:
      return fail(EGN_E_INVALID_ARG, "unknown tuning parameter %d", param);
  }
}

egn_status egn_set_node_rule(egn_link* l, int rule, int n_min) {
  if (!l) return fail(EGN_E_INVALID_ARG, "null link");
  if (rule != EGN_RULE_GL && rule != EGN_RULE_RIDGE) return fail(EGN_E_INVALID_ARG, "unknown node rule %d", rule);
  if (rule == EGN_RULE_RIDGE && (n_min < 1 || n_min > kRidgeMaxN))
    return fail(EGN_E_INVALID_ARG, "n_min %d not in [1, %d]", n_min, kRidgeMaxN);
  l->rule = rule == EGN_RULE_RIDGE ? RULE_RIDGE : RULE_GL;
  if (rule == EGN_RULE_RIDGE) l->ridge_n_min = n_min;
  return EGN_OK;
}

egn_status egn_set_profiling(egn_link* l, int enable) {
  if (!l) return fail(EGN_E_INVALID_ARG, "null link");
  l->prof_on = enable != 0;
  l->prof_valid = false;
  return EGN_OK;
}

egn_status egn_last_timings(egn_link* l, double* ms, int max, int* n) {
  if (!l || !ms || !n) return fail(EGN_E_INVALID_ARG, "null argument");
  if (!l->prof_valid) return fail(EGN_E_STATE, "no profiled evaluation since egn_set_profiling");
  DeviceGuard g(l->device);
  EGN_CUDA(cudaEventSynchronize(l->prof_ev[5]));
  *n = 0;
  for (int i = 0; i < 5 && i < max; ++i) {
    float t = 0.0f;
    EGN_CUDA(cudaEventElapsedTime(&t, l->prof_ev[i], l->prof_ev[i + 1]));
    ms[i] = t;
    *n = i + 1;
  }
  return EGN_OK;
}

egn_status egn_plan_islands(egn_link* l, long long max, int* out, long long* count) {
  if (!l || !count) return fail(EGN_E_INVALID_ARG, "null argument");
  if (l->n_ch <= 0) return fail(EGN_E_STATE, "egn_set_wdm has not been called");
  DeviceGuard g(l->device);
  size_t need = workspace_bytes(l->n_ch, l->cnt, EGN_PREC_FP64);
  cudaError_t e = l->ws.ensure(need);
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "workspace cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
  Workspace ws = carve_workspace(l->ws.p, l->n_ch, l->cnt, EGN_PREC_FP64);
  EGN_LAUNCH_GATE();
  EGN_CUDA(cudaMemset(ws.status, 0, sizeof(int)));
  EGN_CUDA(launch_plan(channel_table(l), ws, 0));
  std::vector<uint64_t> keys(l->cnt.n_isl);
  EGN_CUDA(cudaMemcpy(keys.data(), ws.keys, keys.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  *count = l->cnt.n_isl;
  long long m = std::min<long long>(max, l->cnt.n_isl);
  for (long long i = 0; out && i < m; ++i) {
    int c, a, b, d;
    unpack_key(keys[i], c, a, b, d);
    out[4 * i] = c;
    out[4 * i + 1] = a;
    out[4 * i + 2] = b;
    out[4 * i + 3] = d;
  }
  return EGN_OK;
}

egn_status egn_island_terms(egn_link* l, const egn_opts* o, int n_isl, const int* isl, int all_terms, double* out) {
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  if (n_isl < 0 || (n_isl > 0 && (!isl || !out))) return fail(EGN_E_INVALID_ARG, "bad island list");
  if (n_isl == 0) return EGN_OK;
  DeviceGuard g(l->device);
  s = ensure_tables(l, o);
  if (s != EGN_OK) return s;
  std::vector<uint64_t> keys(n_isl);
  std::vector<uint32_t> e_list, f_list;
  for (int i = 0; i < n_isl; ++i) {
    const int* q = isl + 4 * i;
    for (int a = 0; a < 4; ++a)
      if (q[a] < 0 || q[a] >= l->n_ch) return fail(EGN_E_INVALID_ARG, "island %d: channel index out of range", i);
    keys[i] = pack_key(q[0], q[1], q[2], q[3]);
    if (o->terms && flag_e(q[1], q[2], q[3])) e_list.push_back(i);
    if (o->terms && flag_f(q[1], q[2], q[3])) f_list.push_back(i);
  }
  size_t tsz = o->precision == EGN_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t b_keys = align256(n_isl * sizeof(uint64_t)), b_e = align256(e_list.size() * 4 + 4),
         b_f = align256(f_list.size() * 4 + 4), b_t = align256(5 * (size_t)n_isl * tsz);
  DevBuf tmp;
  cudaError_t e = tmp.ensure(b_keys + b_e + b_f + b_t);
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
  char* p = (char*)tmp.p;
  uint64_t* d_keys = (uint64_t*)p;
  uint32_t* d_e = (uint32_t*)(p + b_keys);
  uint32_t* d_f = (uint32_t*)(p + b_keys + b_e);
  void* d_t = p + b_keys + b_e + b_f;
  egn_status rs = EGN_OK;
  do {
    if ((e = h2d(d_keys, keys.data(), n_isl * sizeof(uint64_t))) != cudaSuccess) break;
    if (!e_list.empty() && (e = h2d(d_e, e_list.data(), e_list.size() * 4)) != cudaSuccess) break;
    if (!f_list.empty() && (e = h2d(d_f, f_list.data(), f_list.size() * 4)) != cudaSuccess) break;
    if ((e = cudaMemset(d_t, 0, 5 * (size_t)n_isl * tsz)) != cudaSuccess) break;
    if ((e = inject(kFaultLaunch, cudaErrorLaunchOutOfResources)) != cudaSuccess) break;
    LinkParams prm = link_params(l, o, all_terms ? 1 : 0);
    e = integrate(prm, o->precision, d_keys, n_isl, nullptr, n_isl, d_e, (long long)e_list.size(), d_f,
                  (long long)f_list.size(), d_t, 0, nullptr);
    if (e != cudaSuccess) break;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) break;
    std::vector<char> h(5 * (size_t)n_isl * tsz);
    if ((e = cudaMemcpy(h.data(), d_t, h.size(), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
    for (int i = 0; i < n_isl; ++i)
      for (int t = 0; t < 5; ++t)
        out[5 * i + t] = tsz == 8 ? ((double*)h.data())[(size_t)t * n_isl + i] : ((float*)h.data())[(size_t)t * n_isl + i];
  } while (0);
  tmp.release();
  if (e != cudaSuccess) rs = fail(EGN_E_CUDA, "island terms: %s", cudaGetErrorString(e));
  return rs;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Evaluation without any device allocation.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// owned entirely by another allocator (a framework's caching allocator, or a
// pool sized up front on a shared GPU), where one more allocation can fail or
// fragment it; a control loop that re-evaluates a link online and cannot accept
// the device synchronisation cudaMalloc/cudaFree imply; or a plugin host that
// forbids its plugins to allocate device memory.  egn_nli_eta_static serves them
// from a fixed scratch array compiled into this library.  Every GPU that loads
// the library holds the array until the process exits.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device.  In host code the name
// g_static_scratch is a host-side stand-in, not a device address: only the
// address from cudaGetSymbolAddress (taken with that device current) may be
// handed to kernels.  Threads that make their first call on a device at the
// same time serialise on the mutex; later calls read the cached address.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_static_ptr[kMaxDevices];
std::mutex g_static_mu;

egn_status static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(EGN_E_UNSUPPORTED, "device %d out of range for the static scratch", dev);
  void* p = g_static_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    p = g_static_ptr[dev].load(std::memory_order_relaxed);
    if (!p) {
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);  // the device is current here
      if (e != cudaSuccess) return fail(EGN_E_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
      g_static_ptr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return EGN_OK;
}

// Where the link tables of one evaluation sit in the scratch, and the span
// scalars they are formed from: passed by value, so that the tables are built on
// the device from kernel parameters and no host buffer is read after the call.
struct StaticTables {
  int nt;
  int K[kMaxTypes];
  double L[kMaxTypes], alpha[kMaxTypes], pcr[kMaxTypes];
  double btot;
  double* zeta[kMaxTypes];
  double* ck[kMaxTypes];
  float* zf[kMaxTypes];
  float* cf[kMaxTypes];
  int ord[4];
  double* gx[4];
  double* gw[4];
  float* gf[4][5];  // x head, x tail, x^2 head, x^2 tail, w (FP32)
};

// Segment tables of every span type (segment_entry, as ensure_tables forms them
// on the host) and the Gauss-Legendre tables of the three outer orders (gl_node,
// as gauss_legendre forms them), one entry per thread.
__global__ void static_tables_kernel(StaticTables t) {
  for (int ty = 0; ty < t.nt; ++ty)
    for (int k = threadIdx.x; k < t.K[ty]; k += blockDim.x) {
      double z, c;
      segment_entry(k, t.K[ty], t.L[ty], t.alpha[ty], t.pcr[ty], t.btot, &z, &c);
      t.zeta[ty][k] = z;
      t.ck[ty][k] = c;
      t.zf[ty][k] = (float)(z * 1.4426950408889634);  // log2(e)
      t.cf[ty][k] = (float)c;
    }
  for (int p = 1; p <= 3; ++p) {
    const int m = t.ord[p];
    for (int k = 1 + threadIdx.x; k <= (m + 1) / 2; k += blockDim.x) {
      double xk, wk;
      gl_node(m, k, &xk, &wk);
      const bool mid = (m % 2 == 1) && k == (m + 1) / 2;  // the middle node of an odd order is 0
      const int idx[2] = {m - k, k - 1};
      const double xv[2] = {mid ? 0.0 : xk, mid ? 0.0 : -xk};
      for (int a = 0; a < 2; ++a) {
        const int i = idx[a];
        const double x = xv[a];
        t.gx[p][i] = x;
        t.gw[p][i] = wk;
        const float xh = (float)x;
        t.gf[p][0][i] = xh;
        t.gf[p][1][i] = (float)(x - (double)xh);
        const double x2 = x * x;
        t.gf[p][2][i] = (float)x2;
        t.gf[p][3][i] = (float)(x2 - (double)(float)x2);
        t.gf[p][4][i] = (float)wk;
      }
    }
  }
}

}  // namespace

extern "C" egn_status egn_nli_eta_static(egn_link* l, const egn_opts* o, double* eta_dev, double* pnli_dev) {
  egn_status s = check_opts(l, o);
  if (s != EGN_OK) return s;
  if (!eta_dev || !pnli_dev) return fail(EGN_E_INVALID_ARG, "eta_dev and pnli_dev must be device arrays of n_ch doubles");
  if (l->rule != RULE_GL) return fail(EGN_E_UNSUPPORTED, "the static scratch path evaluates the Gauss-Legendre rule only");
  DeviceGuard guard(l->device);
  void* base = nullptr;
  s = static_scratch(l->device, &base);
  if (s != EGN_OK) return s;

  // layout of the link tables for these options inside the scratch
  const int nt = l->identical ? 1 : (int)l->type_si.size();
  if (nt > kMaxTypes)
    return fail(EGN_E_UNSUPPORTED, "the static scratch path takes at most %d span types (this link has %d)", kMaxTypes, nt);
  Span sps[kMaxTypes];
  int Ks[kMaxTypes];
  size_t o_zeta[kMaxTypes], o_ck[kMaxTypes], o_zf[kMaxTypes], o_cf[kMaxTypes];
  size_t off = 0;
  for (int t = 0; t < nt; ++t) {
    sps[t] = to_internal(l->type_si[t], l->fc_hz);
    Ks[t] = std::max(1, (int)std::ceil(sps[t].L / o->dz_km));
    o_zeta[t] = off; off += align256(Ks[t] * sizeof(double));
    o_ck[t] = off;   off += align256(Ks[t] * sizeof(double));
    o_zf[t] = off;   off += align256(Ks[t] * sizeof(float));
    o_cf[t] = off;   off += align256(Ks[t] * sizeof(float));
  }
  const Span& sp = sps[0];
  const int K = Ks[0];
  const int n = o->gl_order;
  const int ord[4] = {0, n, (n + 1) / 2, (n + 2) / 3};
  size_t o_gl[4][7] = {};
  for (int p = 1; p <= 3; ++p) {
    for (int a = 0; a < 2; ++a) { o_gl[p][a] = off; off += align256(ord[p] * sizeof(double)); }
    for (int a = 2; a < 7; ++a) { o_gl[p][a] = off; off += align256(ord[p] * sizeof(float)); }
  }
  const size_t ws_off = off;
  const size_t need = ws_off + workspace_bytes(l->n_ch, l->cnt, o->precision);
  if (need > kStaticScratchBytes)
    return fail(EGN_E_CAPACITY, "this evaluation needs %zu bytes of scratch; the static scratch holds %zu bytes "
                "(use egn_nli_eta_device with a caller workspace)", need, kStaticScratchBytes);

  cudaStream_t st = (cudaStream_t)o->stream;
  char* b = (char*)base;
  StaticTables tab{};
  tab.nt = nt;
  tab.btot = l->btot;
  for (int t = 0; t < nt; ++t) {
    tab.K[t] = Ks[t];
    tab.L[t] = sps[t].L;
    tab.alpha[t] = sps[t].alpha;
    tab.pcr[t] = l->ptot * sps[t].cr;
    tab.zeta[t] = (double*)(b + o_zeta[t]);
    tab.ck[t] = (double*)(b + o_ck[t]);
    tab.zf[t] = (float*)(b + o_zf[t]);
    tab.cf[t] = (float*)(b + o_cf[t]);
  }
  for (int p = 1; p <= 3; ++p) {
    tab.ord[p] = ord[p];
    tab.gx[p] = (double*)(b + o_gl[p][0]);
    tab.gw[p] = (double*)(b + o_gl[p][1]);
    for (int a = 0; a < 5; ++a) tab.gf[p][a] = (float*)(b + o_gl[p][2 + a]);
  }

  LinkParams p{};
  p.ch = channel_table(l);
  p.n_types = nt;
  for (int t = 0; t < nt; ++t) {
    SpanType& ty = p.types[t];
    ty.alpha = sps[t].alpha;
    ty.beta2 = sps[t].beta2;
    ty.beta3 = sps[t].beta3;
    ty.gamma = sps[t].gamma;
    ty.L = sps[t].L;
    ty.dz = sps[t].L / Ks[t];
    ty.r = std::exp(-sps[t].alpha * ty.dz);
    ty.pcr = l->ptot * sps[t].cr;
    ty.seg.K = Ks[t];
    ty.seg.zeta = tab.zeta[t];
    ty.seg.ck = tab.ck[t];
    ty.seg.zeta_f = tab.zf[t];
    ty.seg.ck_f = tab.cf[t];
  }
  for (int q = 0; q < (int)l->span_type.size() && q < kMaxSpans; ++q) p.span_type[q] = l->span_type[q];
  p.seg = p.types[0].seg;
  p.gl.n = n;
  p.gl.order[0] = 0;
  for (int q = 1; q <= 3; ++q) {
    p.gl.order[q] = ord[q];
    p.gl.x[q] = tab.gx[q];
    p.gl.w[q] = tab.gw[q];
    p.gl.xh[q] = tab.gf[q][0];
    p.gl.xl[q] = tab.gf[q][1];
    p.gl.x2h[q] = tab.gf[q][2];
    p.gl.x2l[q] = tab.gf[q][3];
    p.gl.wf[q] = tab.gf[q][4];
  }
  p.n_spans = (int)l->spans_si.size();
  p.alpha = sp.alpha;
  p.beta2 = sp.beta2;
  p.beta3 = sp.beta3;
  p.gamma = sp.gamma;
  p.L = sp.L;
  p.dz = sp.L / K;
  p.r = std::exp(-sp.alpha * p.dz);
  p.rolloff = l->rolloff;
  p.terms = o->terms;
  p.all_terms = 0;
  p.fp32c_kp = l->fp32c_kp;
  set_mu_params(p, l, o);

  // tables -> plan -> integrate -> assemble on the caller's stream, all in the scratch
  Workspace ws = carve_workspace(b + ws_off, l->n_ch, l->cnt, o->precision);
  ChannelTable ch = p.ch;
  EGN_LAUNCH_GATE();
  static_tables_kernel<<<1, 128, 0, st>>>(tab);
  EGN_CUDA(cudaGetLastError());
  EGN_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), st));  // the array keeps the last call's contents
  EGN_CUDA(launch_plan(ch, ws, st));
  EGN_CUDA(integrate(p, o->precision, ws.keys, l->cnt.n_isl, ws.d_idx, l->cnt.n_half, ws.e_idx, l->cnt.n_e, ws.f_idx,
                     l->cnt.n_f, ws.terms, st, nullptr));
  EGN_CUDA(launch_assemble(ch, half_offsets(ws, l->n_ch), ws.keys, ws.h_idx, l->cnt.n_isl, ws.terms, o->precision,
                           o->terms, eta_dev, pnli_dev, st));
  return EGN_OK;
}
