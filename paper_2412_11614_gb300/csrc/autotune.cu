// autotune.cu -- choice of the segment length and of the launch shape.
//
// The segment form trades accuracy for time through Delta z (Sec. III-D,
// Fig. 11): K = ceil(L / Delta z) segments per span, time roughly linear in K.
// egn_autotune evaluates the link once at a fine reference Delta z, then the
// candidates from the coarsest down, and keeps the coarsest whose worst channel
// deviates from the reference by at most the target (dB).  For the FP32C path
// it then times both launch shapes of the D/G/H pass at that Delta z and sets
// the faster one on the link.  Every evaluation goes through the same entry
// points as a user's call.
#include <algorithm>
#include <cmath>
#include <vector>

#include "link.h"

using namespace egn_host;

namespace {

// Device milliseconds of one egn_nli_eta_device call (after one untimed call),
// median of `reps`, on the link's own workspace and a private stream.
egn_status time_eval(egn_link* l, egn_opts o, int reps, double* ms) {
  size_t need = 0;
  egn_status s = egn_workspace_size(l, &o, &need);
  if (s != EGN_OK) return s;
  cudaError_t e = l->ws.ensure(need);
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "workspace cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
  cudaStream_t st;
  EGN_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  o.stream = st;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  std::vector<float> t;
  s = egn_nli_eta_device(l, &o, l->ws.p, l->ws.bytes, nullptr, nullptr);
  for (int r = 0; r < reps && s == EGN_OK; ++r) {
    cudaEventRecord(a, st);
    s = egn_nli_eta_device(l, &o, l->ws.p, l->ws.bytes, nullptr, nullptr);
    cudaEventRecord(b, st);
    if (s == EGN_OK) s = wait_event(b, o.timeout_ms);
    float x = 0.0f;
    if (s == EGN_OK && cudaEventElapsedTime(&x, a, b) == cudaSuccess) t.push_back(x);
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaStreamDestroy(st);
  if (s != EGN_OK) return s;
  if (t.empty()) return fail(EGN_E_CUDA, "no timing");
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return EGN_OK;
}

double max_db(const std::vector<double>& a, const std::vector<double>& b) {
  double m = 0.0;
  for (size_t i = 0; i < a.size(); ++i) m = std::max(m, std::fabs(10.0 * std::log10(a[i] / b[i])));
  return m;
}

}  // namespace

extern "C" egn_status egn_autotune(egn_link* l, const egn_opts* opts, double target_db, const double* dz_cand,
                                   int n_cand, double dz_ref_km, egn_tune_result* out) {
  if (!l || !opts || !out || !dz_cand || n_cand < 1) return fail(EGN_E_INVALID_ARG, "null argument or no candidates");
  if (!(target_db > 0.0) || !std::isfinite(target_db)) return fail(EGN_E_INVALID_ARG, "target_db must be positive");
  if (!finite_pos(dz_ref_km)) return fail(EGN_E_INVALID_ARG, "dz_ref_km must be positive");
  for (int i = 0; i < n_cand; ++i)
    if (!finite_pos(dz_cand[i])) return fail(EGN_E_INVALID_ARG, "candidate %d is not a positive length", i);
  if (opts->mu_form != EGN_MU_SEGMENT) return fail(EGN_E_INVALID_ARG, "Delta z applies to the segment form only");
  egn_opts o = *opts;
  o.stream = nullptr;
  const int n = l->n_ch;
  if (n <= 0) return fail(EGN_E_STATE, "egn_set_wdm has not been called");
  std::vector<double> ref(n), eta(n);
  o.dz_km = dz_ref_km;
  egn_status s = egn_nli_eta(l, &o, ref.data(), nullptr);
  if (s != EGN_OK) return s;
  std::vector<double> cand(dz_cand, dz_cand + n_cand);
  std::sort(cand.begin(), cand.end(), [](double a, double b) { return a > b; });  // coarsest first
  double best = dz_ref_km, err = 0.0;
  for (double dz : cand) {
    if (dz < dz_ref_km) break;  // no finer than the reference
    o.dz_km = dz;
    s = egn_nli_eta(l, &o, eta.data(), nullptr);
    if (s != EGN_OK) return s;
    const double e = max_db(eta, ref);
    if (e <= target_db) {
      best = dz;
      err = e;
      break;
    }
  }
  o.dz_km = best;
  int kp = l->fp32c_kp;
  double ms = 0.0;
  if (o.precision == EGN_PREC_FP32C) {
    double t4 = 0.0, t8 = 0.0;
    l->fp32c_kp = 4;
    s = time_eval(l, o, 5, &t4);
    if (s == EGN_OK) {
      l->fp32c_kp = 8;
      s = time_eval(l, o, 5, &t8);
    }
    if (s != EGN_OK) {
      l->fp32c_kp = kp;
      return s;
    }
    kp = t8 < t4 ? 8 : 4;
    ms = std::min(t4, t8);
    l->fp32c_kp = kp;
  } else {
    s = time_eval(l, o, 3, &ms);
    if (s != EGN_OK) return s;
  }
  out->dz_km = best;
  out->points_per_thread = kp;
  out->max_err_db = err;
  out->ms = ms;
  return EGN_OK;
}

// Choice of the node rule and its order (the quadrature error of Eq. 17-21's
// island integrals).  The ridge-resolving rule (FP32C where the options ask for
// it and the link has at most kMaxTypes span types, else FP64) is evaluated at 4, 8, 16,
// ... nodes per piece, doubling until the worst channel moves by less than a
// quarter of the target between two orders or max_nodes is reached; the last
// order stands for the converged value.  The smallest order within target_db
// of it is chosen and set on the link (egn_set_node_rule); the configured
// Gauss-Legendre rule of opts->gl_order is scored against the same value.
extern "C" egn_status egn_autotune_rule(egn_link* l, const egn_opts* opts, double target_db, int max_nodes,
                                        egn_rule_result* out) {
  if (!l || !opts || !out) return fail(EGN_E_INVALID_ARG, "null argument");
  if (!(target_db > 0.0) || !std::isfinite(target_db)) return fail(EGN_E_INVALID_ARG, "target_db must be positive");
  if (max_nodes < 4 || max_nodes > egn::kRidgeMaxN)
    return fail(EGN_E_INVALID_ARG, "max_nodes %d not in [4, %d]", max_nodes, egn::kRidgeMaxN);
  const int n = l->n_ch;
  if (n <= 0) return fail(EGN_E_STATE, "egn_set_wdm has not been called");
  const int rule0 = l->rule, nmin0 = l->ridge_n_min;
  egn_opts o = *opts;
  o.stream = nullptr;
  o.precision = (opts->precision == EGN_PREC_FP32C && (l->identical || (int)l->type_si.size() <= egn::kMaxTypes))
                    ? EGN_PREC_FP32C
                    : EGN_PREC_FP64;
  // the configured rule first
  std::vector<double> gl(n);
  l->rule = egn::RULE_GL;
  egn_status s = egn_nli_eta(l, &o, gl.data(), nullptr);
  if (s != EGN_OK) {
    l->rule = rule0;
    return s;
  }
  l->rule = egn::RULE_RIDGE;
  l->ridge_n_min = 4;
  std::vector<std::vector<double>> eta;
  std::vector<int> order;
  double change = -1.0;
  for (int q = 4; q <= max_nodes; q *= 2) {
    o.gl_order = q;
    std::vector<double> e(n);
    s = egn_nli_eta(l, &o, e.data(), nullptr);
    if (s != EGN_OK) {
      l->rule = rule0;
      l->ridge_n_min = nmin0;
      return s;
    }
    eta.push_back(e);
    order.push_back(q);
    if (eta.size() >= 2) {
      change = max_db(eta[eta.size() - 1], eta[eta.size() - 2]);
      if (change < 0.25 * target_db) break;
    }
  }
  const std::vector<double>& ref = eta.back();
  size_t pick = eta.size() - 1;
  for (size_t i = 0; i < eta.size(); ++i)
    if (max_db(eta[i], ref) <= target_db) {
      pick = i;
      break;
    }
  o.gl_order = order[pick];
  double ms = 0.0;
  s = time_eval(l, o, 3, &ms);
  if (s != EGN_OK) {
    l->rule = rule0;
    l->ridge_n_min = nmin0;
    return s;
  }
  out->rule = EGN_RULE_RIDGE;
  out->nodes = order[pick];
  out->max_err_db = max_db(eta[pick], ref);
  out->last_change_db = change;
  out->reference_nodes = order.back();
  out->configured_err_db = max_db(gl, ref);
  out->ms = ms;
  return EGN_OK;
}
