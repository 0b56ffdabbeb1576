// batch.cu -- many links evaluated by one CUDA graph.
//
// egn_batch_create snapshots every link (its channel, segment and
// Gauss-Legendre tables are copied into batch-owned device memory, so later
// egn_set_wdm calls or egn_link_destroy do not touch the batch), sizes one
// workspace per link in a single allocation, runs the whole evaluation once
// without capture (which validates it and completes every lazy launch set-up),
// then captures the same sequence into a CUDA graph.
//
// FP32C batches run one flat work list per pass: every link's island planner
// (concurrent branches on up to kStreams streams), then each integrator pass
// (D/G/H, E, F) as one launch per kernel family over the work lists of all the
// links of that family (the job tables of integrate_fp32c.cu: island batches
// numbered across links), then every link's assembly (concurrent branches).
// FP64 batches capture each link's chain -- status reset, planner, integrator
// passes, assembly -- in two phases: links too small to fill the GPU as
// concurrent branches, then the links that fill it on their own ("heavy":
// estimated point-segment work above kHeavyWork) one after the other, because
// heavy links sharing the GPU were measured to slow each other down.
// egn_batch_launch replays the graph with one call; outputs of all links are
// concatenated in link order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "link.h"

using namespace egn_host;
using egn::ChannelTable;
using egn::LinkParams;
using egn::PlanCounts;
using egn::Workspace;

namespace {

constexpr int kStreams = 8;             // capture streams: concurrent branches of the graph
constexpr double kHeavyWork = 2e10;     // point x segment steps of a link that fills the GPU (a few ms)
constexpr double kSpanSerialCost = 5.0; // relative cost of a step on the span-serial path (MUFU-bound)

// Snapshot of one link inside a batch.
struct BatchLink {
  int n_ch = 0;
  PlanCounts cnt{};
  LinkParams p{};       // pointers rebased into the batch's table copy
  ChannelTable ch{};    // = p.ch
  size_t tab_off = 0;   // offset of this link's table copy in d_tab
  size_t ws_off = 0;    // offset of its workspace in d_ws
  bool heavy = false;   // fills the GPU on its own: serial branch
};

// Estimated work of one evaluation: quadrature points of the half list times
// segment steps per point (every span's on the span-serial path).
double link_work(const egn_link* l, const egn_opts* o) {
  const double pts = (double)l->cnt.n_half * o->gl_order * o->gl_order;
  double steps = 0.0;
  const int nt = (int)l->type_si.size();
  if (nt > egn::kMaxTypes) {
    for (const egn_span& s : l->spans_si) steps += std::ceil(s.length_m * 1e-3 / o->dz_km);
    steps *= kSpanSerialCost;
  } else {
    for (const egn_span& s : l->type_si) steps += std::ceil(s.length_m * 1e-3 / o->dz_km);
  }
  return pts * steps;
}

// Move q from [old, old + bytes) to the same offset after nb.
template <class T>
void rebase(const T*& q, const void* old, size_t bytes, const void* nb) {
  const char* c = (const char*)q;
  if (q && c >= (const char*)old && c < (const char*)old + bytes) q = (const T*)((const char*)nb + (c - (const char*)old));
}

void rebase_params(LinkParams& p, const egn_link* l, char* ch_copy, char* seg_copy, char* gl_copy) {
  ChannelTable& c = p.ch;
  for (const double** q : {&c.nu, &c.R, &c.W, &c.P, &c.phi, &c.psi}) rebase(*q, l->d_ch.p, l->d_ch.bytes, ch_copy);
  for (const double** q : {&c.nu_coi}) rebase(*q, l->d_ch.p, l->d_ch.bytes, ch_copy);
  for (const float** q : {&c.nu_f, &c.hw_f, &c.nu_coi_f}) rebase(*q, l->d_ch.p, l->d_ch.bytes, ch_copy);
  auto seg = [&](egn::SegmentTables& t) {
    rebase(t.zeta, l->d_seg.p, l->d_seg.bytes, seg_copy);
    rebase(t.ck, l->d_seg.p, l->d_seg.bytes, seg_copy);
    rebase(t.zeta_f, l->d_seg.p, l->d_seg.bytes, seg_copy);
    rebase(t.ck_f, l->d_seg.p, l->d_seg.bytes, seg_copy);
  };
  seg(p.seg);
  for (int t = 0; t < egn::kMaxTypes; ++t) seg(p.types[t].seg);
  for (int f = 0; f < p.n_fib; ++f) {
    rebase(p.fib_ck[f], l->d_seg.p, l->d_seg.bytes, seg_copy);
    rebase(p.fib_zk[f], l->d_seg.p, l->d_seg.bytes, seg_copy);
  }
  rebase(p.glx_all, l->d_gl.p, l->d_gl.bytes, gl_copy);
  rebase(p.glw_all, l->d_gl.p, l->d_gl.bytes, gl_copy);
  rebase(p.glxh_all, l->d_gl.p, l->d_gl.bytes, gl_copy);
  rebase(p.glxl_all, l->d_gl.p, l->d_gl.bytes, gl_copy);
  rebase(p.glwf_all, l->d_gl.p, l->d_gl.bytes, gl_copy);
  for (int q = 0; q < 4; ++q) {
    rebase(p.gl.x[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.w[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.xh[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.xl[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.x2h[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.x2l[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
    rebase(p.gl.wf[q], l->d_gl.p, l->d_gl.bytes, gl_copy);
  }
}

}  // namespace

struct egn_batch {
  int device = -1;
  egn_opts opts{};
  bool flat = false;                     // FP32C: one launch per pass and kernel family
  std::vector<egn::MultiLaunch> multi;   // those launches, in pass order
  std::vector<size_t> multi_off;         // their job tables' offsets in d_jobs
  DevBuf d_jobs;
  std::vector<BatchLink> links;
  std::vector<long long> off;  // channel offsets, off[n] = all channels
  DevBuf d_tab, d_ws, d_out;   // table copies; workspaces; eta | pnli | status
  double* h_stage = nullptr;   // pinned: eta | pnli | status of every link
  cudaStream_t cap = nullptr;
  cudaStream_t st[kStreams] = {};
  cudaEvent_t fork = nullptr, join[kStreams] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long total() const { return off.back(); }
  double* eta() const { return (double*)d_out.p; }
  double* pnli() const { return (double*)d_out.p + total(); }
  int* status() const { return (int*)((double*)d_out.p + 2 * total()); }
  ~egn_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : join)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    for (auto& s : st)
      if (s) cudaStreamDestroy(s);
    if (cap) cudaStreamDestroy(cap);
    if (h_stage) cudaFreeHost(h_stage);
    d_tab.release();
    d_ws.release();
    d_out.release();
    d_jobs.release();
  }
};

namespace {

// One link's chain on stream s.
egn_status enqueue_link(egn_batch* b, size_t i, cudaStream_t s) {
  const BatchLink& L = b->links[i];
  Workspace ws = egn::carve_workspace((char*)b->d_ws.p + L.ws_off, L.n_ch, L.cnt, b->opts.precision);
  EGN_LAUNCH_GATE();
  EGN_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
  EGN_CUDA(egn::launch_plan(L.ch, ws, s));
  EGN_CUDA(integrate(L.p, b->opts.precision, ws.keys, L.cnt.n_isl, ws.d_idx, L.cnt.n_half, ws.e_idx, L.cnt.n_e,
                     ws.f_idx, L.cnt.n_f, ws.terms, s, nullptr));
  EGN_CUDA(egn::launch_assemble(L.ch, half_offsets(ws, L.n_ch), ws.keys, ws.h_idx, L.cnt.n_isl, ws.terms,
                                b->opts.precision, b->opts.terms, b->eta() + b->off[i], b->pnli() + b->off[i], s));
  EGN_CUDA(cudaMemcpyAsync(b->status() + i, ws.status, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return EGN_OK;
}

// Island planner of link i on stream s (status word reset first).
egn_status plan_link(egn_batch* b, size_t i, cudaStream_t s) {
  const BatchLink& L = b->links[i];
  Workspace ws = egn::carve_workspace((char*)b->d_ws.p + L.ws_off, L.n_ch, L.cnt, b->opts.precision);
  EGN_CUDA(cudaMemsetAsync(ws.status, 0, sizeof(int), s));
  EGN_CUDA(egn::launch_plan(L.ch, ws, s));
  return EGN_OK;
}

// Assembly of link i into the batch outputs and its status word, on stream s.
egn_status assemble_link(egn_batch* b, size_t i, cudaStream_t s) {
  const BatchLink& L = b->links[i];
  Workspace ws = egn::carve_workspace((char*)b->d_ws.p + L.ws_off, L.n_ch, L.cnt, b->opts.precision);
  EGN_CUDA(egn::launch_assemble(L.ch, half_offsets(ws, L.n_ch), ws.keys, ws.h_idx, L.cnt.n_isl, ws.terms,
                                b->opts.precision, b->opts.terms, b->eta() + b->off[i], b->pnli() + b->off[i], s));
  EGN_CUDA(cudaMemcpyAsync(b->status() + i, ws.status, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return EGN_OK;
}

// fn(i, stream) for every link as concurrent branches of `root` (up to kStreams), joined back.
template <class F>
egn_status branches(egn_batch* b, cudaStream_t root, F fn) {
  const int ns = std::min<int>(kStreams, (int)b->links.size());
  EGN_CUDA(cudaEventRecord(b->fork, root));
  for (int j = 0; j < ns; ++j) EGN_CUDA(cudaStreamWaitEvent(b->st[j], b->fork, 0));
  for (size_t i = 0; i < b->links.size(); ++i) {
    egn_status s = fn(i, b->st[i % ns]);
    if (s != EGN_OK) return s;
  }
  for (int j = 0; j < ns; ++j) {
    EGN_CUDA(cudaEventRecord(b->join[j], b->st[j]));
    EGN_CUDA(cudaStreamWaitEvent(root, b->join[j], 0));
  }
  return EGN_OK;
}

// FP32C: planners, one launch per pass and kernel family over every link, assemblies.
egn_status enqueue_flat(egn_batch* b, cudaStream_t root) {
  EGN_LAUNCH_GATE();
  egn_status s = branches(b, root, [&](size_t i, cudaStream_t st) { return plan_link(b, i, st); });
  if (s != EGN_OK) return s;
  for (size_t k = 0; k < b->multi.size(); ++k)
    EGN_CUDA(egn::launch_fp32c_multi(b->multi[k], (const char*)b->d_jobs.p + b->multi_off[k], root));
  return branches(b, root, [&](size_t i, cudaStream_t st) { return assemble_link(b, i, st); });
}

// The job tables of the flat passes (FP32C): per pass (D/G/H, E, F) and kernel
// family, every link's work list of that pass; copied to device memory once.
egn_status build_flat(egn_batch* b) {
  std::vector<egn::FlatPass> fp[3][3];
  const bool corr = b->opts.terms != 0;
  for (BatchLink& L : b->links) {
    Workspace ws = egn::carve_workspace((char*)b->d_ws.p + L.ws_off, L.n_ch, L.cnt, b->opts.precision);
    const int fam = egn::fp32c_family(L.p);
    float* terms = (float*)ws.terms;
    fp[0][fam].push_back({&L.p, ws.keys, ws.d_idx, L.cnt.n_half, terms, L.cnt.n_isl});
    if (corr && L.cnt.n_e) fp[1][fam].push_back({&L.p, ws.keys, ws.e_idx, L.cnt.n_e, terms, L.cnt.n_isl});
    if (corr && L.cnt.n_f) fp[2][fam].push_back({&L.p, ws.keys, ws.f_idx, L.cnt.n_f, terms, L.cnt.n_isl});
  }
  size_t total = 0;
  for (auto& ord : fp)
    for (auto& v : ord)
      if (!v.empty()) total += align256(egn::fp32c_multi_bytes((int)v.size()));
  std::vector<char> image(total, 0);
  size_t off = 0;
  for (int ord = 0; ord < 3; ++ord)
    for (int fam = 0; fam < 3; ++fam) {
      auto& v = fp[ord][fam];
      if (v.empty()) continue;
      egn::MultiLaunch m{};
      EGN_CUDA(egn::fp32c_multi_build(ord, fam, v.data(), (int)v.size(), image.data() + off, &m));
      b->multi.push_back(m);
      b->multi_off.push_back(off);
      off += align256(egn::fp32c_multi_bytes((int)v.size()));
    }
  if (total) {
    EGN_ALLOC(b->d_jobs.ensure(total));
    EGN_CUDA(h2d(b->d_jobs.p, image.data(), total));
  }
  return EGN_OK;
}

// The whole evaluation of the batch on `root`: first the light links as
// concurrent branches (round-robin over up to kStreams streams, joined back),
// then the heavy links one after the other, so heavy work never shares the GPU.
egn_status enqueue(egn_batch* b, cudaStream_t root) {
  if (b->flat) return enqueue_flat(b, root);
  int n_light = 0;
  for (const BatchLink& L : b->links) n_light += !L.heavy;
  if (n_light) {
    const int ns = std::min<int>(kStreams, n_light);
    EGN_CUDA(cudaEventRecord(b->fork, root));
    for (int j = 0; j < ns; ++j) EGN_CUDA(cudaStreamWaitEvent(b->st[j], b->fork, 0));
    int k = 0;
    for (size_t i = 0; i < b->links.size(); ++i)
      if (!b->links[i].heavy) {
        egn_status s = enqueue_link(b, i, b->st[(k++) % ns]);
        if (s != EGN_OK) return s;
      }
    for (int j = 0; j < ns; ++j) {
      EGN_CUDA(cudaEventRecord(b->join[j], b->st[j]));
      EGN_CUDA(cudaStreamWaitEvent(root, b->join[j], 0));
    }
  }
  for (size_t i = 0; i < b->links.size(); ++i)
    if (b->links[i].heavy) {
      egn_status s = enqueue_link(b, i, root);
      if (s != EGN_OK) return s;
    }
  return EGN_OK;
}

// Copy outputs and statuses to the pinned stage on `st` and wait (timeout).
egn_status stage_and_check(egn_batch* b, cudaStream_t st) {
  const long long n = b->total();
  const size_t bytes = (size_t)(2 * n) * sizeof(double) + b->links.size() * sizeof(int);
  EGN_CUDA(cudaMemcpyAsync(b->h_stage, b->d_out.p, bytes, cudaMemcpyDeviceToHost, st));
  cudaEvent_t ev;
  EGN_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t re = cudaEventRecord(ev, st);
  if (re != cudaSuccess) { cudaEventDestroy(ev); return fail(EGN_E_CUDA, "cudaEventRecord: %s", cudaGetErrorString(re)); }
  egn_status s = wait_event(ev, b->opts.timeout_ms);
  cudaEventDestroy(ev);
  if (s != EGN_OK) return s;
  const int* stat = (const int*)(b->h_stage + 2 * n);
  for (size_t i = 0; i < b->links.size(); ++i)
    if (stat[i]) return fail(EGN_E_CUDA, "device planner overflow in link %zu (status %d)", i, stat[i]);
  return EGN_OK;
}

egn_status create(egn_link* const* links, int n_links, const egn_opts* o, bool capture, egn_batch* b) {
  if (!links || n_links <= 0 || !o) return fail(EGN_E_INVALID_ARG, "need n_links >= 1 links and options");
  b->opts = *o;
  b->opts.stream = nullptr;
  b->device = links[0] ? links[0]->device : -1;
  size_t tab = 0, ws = 0;
  b->off.assign(1, 0);
  for (int i = 0; i < n_links; ++i) {
    egn_link* l = links[i];
    if (!l) return fail(EGN_E_INVALID_ARG, "link %d is null", i);
    egn_status s = check_opts(l, o);
    if (s != EGN_OK) return s;
    if (l->device != b->device) return fail(EGN_E_INVALID_ARG, "links of one batch must share a device");
    DeviceGuard g(l->device);
    s = ensure_tables(l, o);
    if (s != EGN_OK) return s;
    BatchLink L;
    L.n_ch = l->n_ch;
    L.cnt = l->cnt;
    L.tab_off = tab;
    tab += align256(l->d_ch.bytes) + align256(l->d_seg.bytes) + align256(l->d_gl.bytes) +
           align256(l->types.size() > (size_t)egn::kMaxTypes ? l->types.size() * sizeof(egn::SpanType) : 0);
    L.ws_off = ws;
    L.heavy = link_work(l, o) >= kHeavyWork;
    ws += align256(egn::workspace_bytes(l->n_ch, l->cnt, o->precision));
    b->links.push_back(L);
    b->off.push_back(b->off.back() + l->n_ch);
  }
  DeviceGuard g(b->device);
  EGN_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  for (auto& s : b->st) EGN_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  EGN_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  for (auto& e : b->join) EGN_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaError_t e = b->d_tab.ensure(tab);
  if (e == cudaSuccess) e = b->d_ws.ensure(ws);
  const size_t out_b = (size_t)(2 * b->total()) * sizeof(double) + (size_t)n_links * sizeof(int);
  if (e == cudaSuccess) e = b->d_out.ensure(out_b);
  if (e != cudaSuccess) return fail(EGN_E_NOMEM, "batch cudaMalloc: %s", cudaGetErrorString(e));
  EGN_ALLOC(pinned_alloc((void**)&b->h_stage, out_b));
  // table snapshot (device to device), launch parameters rebased onto it
  for (int i = 0; i < n_links; ++i) {
    egn_link* l = links[i];
    BatchLink& L = b->links[i];
    char* base = (char*)b->d_tab.p + L.tab_off;
    char* ch_c = base;
    char* seg_c = ch_c + align256(l->d_ch.bytes);
    char* gl_c = seg_c + align256(l->d_seg.bytes);
    EGN_CUDA(cudaMemcpyAsync(ch_c, l->d_ch.p, l->d_ch.bytes, cudaMemcpyDeviceToDevice, b->cap));
    EGN_CUDA(cudaMemcpyAsync(seg_c, l->d_seg.p, l->d_seg.bytes, cudaMemcpyDeviceToDevice, b->cap));
    EGN_CUDA(cudaMemcpyAsync(gl_c, l->d_gl.p, l->d_gl.bytes, cudaMemcpyDeviceToDevice, b->cap));
    L.p = link_params(l, o, 0);
    rebase_params(L.p, l, ch_c, seg_c, gl_c);
    if (L.p.n_types > egn::kMaxTypes) {  // the device array of span types, its tables rebased too
      std::vector<egn::SpanType> ty(l->types);
      for (auto& t : ty) {
        rebase(t.seg.zeta, l->d_seg.p, l->d_seg.bytes, seg_c);
        rebase(t.seg.ck, l->d_seg.p, l->d_seg.bytes, seg_c);
        rebase(t.seg.zeta_f, l->d_seg.p, l->d_seg.bytes, seg_c);
        rebase(t.seg.ck_f, l->d_seg.p, l->d_seg.bytes, seg_c);
      }
      char* ty_c = gl_c + align256(l->d_gl.bytes);
      EGN_CUDA(h2d_async(ty_c, ty.data(), ty.size() * sizeof(egn::SpanType), b->cap));
      EGN_CUDA(cudaStreamSynchronize(b->cap));  // ty is a host temporary
      L.p.types_dev = (const egn::SpanType*)ty_c;
    }
    L.ch = L.p.ch;
  }
  b->flat = o->precision == EGN_PREC_FP32C;
  for (int i = 0; i < n_links; ++i)
    if (links[i]->rule != egn::RULE_GL) b->flat = false;  // the flat passes run the configured rule's kernels
  if (b->flat) {
    egn_status fs = build_flat(b);
    if (fs != EGN_OK) return fs;
  }
  // one plain run: validates the batch and completes lazy launch set-up
  egn_status s = enqueue(b, b->cap);
  if (s != EGN_OK) return s;
  s = stage_and_check(b, b->cap);
  if (s != EGN_OK || !capture) return s;
  // capture
  EGN_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  s = enqueue(b, b->cap);
  cudaGraph_t gr = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->cap, &gr);
  if (s != EGN_OK) {
    if (gr) cudaGraphDestroy(gr);
    return s;
  }
  if (ce != cudaSuccess) return fail(EGN_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  b->graph = gr;
  EGN_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return EGN_OK;
}

}  // namespace

extern "C" {

egn_status egn_batch_create(egn_link* const* links, int n_links, const egn_opts* opts, egn_batch** out) {
  if (!out) return fail(EGN_E_INVALID_ARG, "out is null");
  *out = nullptr;
  egn_batch* b = new (std::nothrow) egn_batch();
  if (!b) return fail(EGN_E_NOMEM, "out of host memory");
  egn_status s = create(links, n_links, opts, true, b);
  if (s != EGN_OK) {
    delete b;
    return s;
  }
  *out = b;
  return EGN_OK;
}

egn_status egn_batch_launch(egn_batch* b, void* stream) {
  NvtxRange range("egn_batch_launch");
  if (!b || !b->exec) return fail(EGN_E_INVALID_ARG, "batch is null");
  DeviceGuard g(b->device);
  EGN_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return EGN_OK;
}

egn_status egn_batch_outputs(const egn_batch* b, const double** eta_dev, const double** pnli_dev,
                             const long long** offsets) {
  if (!b) return fail(EGN_E_INVALID_ARG, "batch is null");
  if (eta_dev) *eta_dev = b->eta();
  if (pnli_dev) *pnli_dev = b->pnli();
  if (offsets) *offsets = b->off.data();
  return EGN_OK;
}

egn_status egn_batch_read(egn_batch* b, void* stream, double* eta, double* pnli) {
  NvtxRange range("egn_batch_read");
  if (!b) return fail(EGN_E_INVALID_ARG, "batch is null");
  DeviceGuard g(b->device);
  egn_status s = stage_and_check(b, (cudaStream_t)stream);
  if (s != EGN_OK) return s;
  const long long n = b->total();
  if (eta) std::memcpy(eta, b->h_stage, n * sizeof(double));
  if (pnli) std::memcpy(pnli, b->h_stage + n, n * sizeof(double));
  return EGN_OK;
}

void egn_batch_destroy(egn_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  cudaStreamSynchronize(b->cap);
  delete b;
}

egn_status egn_nli_eta_batch(egn_link* const* links, int n, const egn_opts* opts, double* const* eta,
                             double* const* pnli) {
  egn_batch* b = new (std::nothrow) egn_batch();
  if (!b) return fail(EGN_E_NOMEM, "out of host memory");
  egn_status s = create(links, n, opts, false, b);  // one plain run, no graph
  if (s != EGN_OK) {
    delete b;
    return s;
  }
  const long long tot = b->total();
  for (int i = 0; i < n; ++i) {
    const long long o = b->off[i], m = b->off[i + 1] - o;
    if (eta && eta[i]) std::memcpy(eta[i], b->h_stage + o, m * sizeof(double));
    if (pnli && pnli[i]) std::memcpy(pnli[i], b->h_stage + tot + o, m * sizeof(double));
  }
  egn_batch_destroy(b);
  return EGN_OK;
}

}  // extern "C"
