// link.h -- the link object behind the C ABI and the host helpers shared by
// the single-link entry points (api.cu) and the batch of links (batch.cu).
#pragma once

#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/egn.h"
#include "egn_internal.h"

namespace egn_host {

// Record a thread-local message for egn_last_error and return s.
egn_status fail(egn_status s, const char* fmt, ...);

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host-side fault injection for the failure tests.  The environment variable
// EGN_FAULT holds a comma-separated subset of "alloc", "h2d" and "launch"; while
// it names a kind, every device or pinned allocation, every host-to-device copy
// or every launch sequence of an evaluation fails with the error the real
// failure returns (cudaErrorMemoryAllocation, cudaErrorInvalidValue,
// cudaErrorLaunchOutOfResources) before anything reaches the device, so the
// link or batch stays usable once the variable is cleared.  Read on every call.
enum : unsigned { kFaultAlloc = 1u, kFaultH2D = 2u, kFaultLaunch = 4u };
unsigned fault_mask();
inline cudaError_t inject(unsigned kind, cudaError_t as) { return (fault_mask() & kind) ? as : cudaSuccess; }

inline cudaError_t h2d(void* dst, const void* src, size_t n) {
  if (cudaError_t f = inject(kFaultH2D, cudaErrorInvalidValue)) return f;
  return cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
}
inline cudaError_t h2d_async(void* dst, const void* src, size_t n, cudaStream_t st) {
  if (cudaError_t f = inject(kFaultH2D, cudaErrorInvalidValue)) return f;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
}
// Device and pinned-host allocations the library has asked the runtime for in
// this process (egn_allocation_count).
extern std::atomic<long long> g_alloc_count;

inline cudaError_t pinned_alloc(void** p, size_t n) {
  if (cudaError_t f = inject(kFaultAlloc, cudaErrorMemoryAllocation)) return f;
  g_alloc_count.fetch_add(1, std::memory_order_relaxed);
  return cudaMallocHost(p, n);
}

// NVTX range over a scope (host side: the enqueue of a phase); a no-op unless a
// profiler is attached, and the ranges let ncu --nvtx filter the phases.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device buffer owned by a link or a batch.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t want) {
    if (want <= bytes && p) return cudaSuccess;
    if (cudaError_t f = inject(kFaultAlloc, cudaErrorMemoryAllocation)) return f;  // the old buffer stays
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    g_alloc_count.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// Make a device current for the lifetime of the guard (-1: leave as is).
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev); else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace egn_host

#define EGN_CUDA(call)                                                                                    \
  do {                                                                                                    \
    cudaError_t e_ = (call);                                                                              \
    if (e_ != cudaSuccess) return egn_host::fail(EGN_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// An allocation: failure is EGN_E_NOMEM.
#define EGN_ALLOC(call)                                                                                    \
  do {                                                                                                     \
    cudaError_t e_ = (call);                                                                               \
    if (e_ != cudaSuccess) return egn_host::fail(EGN_E_NOMEM, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// The start of every evaluation's launch sequence (plan -> integrate -> assemble).
#define EGN_LAUNCH_GATE() EGN_CUDA(egn_host::inject(egn_host::kFaultLaunch, cudaErrorLaunchOutOfResources))

struct egn_link {
  std::vector<egn_span> spans_si;
  bool identical = true;
  std::vector<egn_span> type_si;      // distinct span types, in order of first appearance
  std::vector<unsigned char> span_type;
  // comb (internal units)
  int n_ch = 0;
  double fc_hz = 0, btot = 0, ptot = 0, rolloff = 0;
  std::vector<double> nu, R, W, P, phi, psi;
  bool mixed_rates = false, any_corr = false;
  egn::PlanCounts cnt{};
  std::vector<long long> per_coi;
  int device = -1;
  egn_host::DevBuf d_ch;  // 6 arrays of n_ch doubles, then nu and W/2 as floats
  // cached tables for the last (dz, gl_order)
  double tab_dz = -1.0;
  int tab_gl = -1;
  int K = 0;
  egn::Span span{};
  std::vector<egn::SpanType> types;  // every span type's tables (device pointers)
  egn_host::DevBuf d_types;          // the same array in device memory (more than kMaxTypes types)
  egn_host::DevBuf d_seg, d_gl;
  egn::SegmentTables seg{};
  egn::GlTables gl{};
  const double* gl_all_x = nullptr;  // every order 1..n (the ridge rule's pieces), inside d_gl
  const double* gl_all_w = nullptr;
  const float* gl_all_xh = nullptr;  // FP32 head, tail and weight of the same nodes
  const float* gl_all_xl = nullptr;
  const float* gl_all_wf = nullptr;
  int fp32c_kp = 4;  // tuning: points per thread of the FP32C D/G/H pass
  int rule = egn::RULE_GL;  // node rule (egn_set_node_rule)
  int ridge_n_min = 4;
  // optional per-stage device timing of the last evaluation
  bool prof_on = false;
  bool prof_valid = false;
  cudaEvent_t prof_ev[6] = {};
  // library-owned workspace and pinned staging for the host API
  egn_host::DevBuf ws;
  double* h_stage = nullptr;  // [2 n_ch + 1]
  size_t h_stage_n = 0;       // its capacity in doubles
  egn_host::DevBuf d_stage;
  // COI evaluation frequencies of the f-integral (egn_nli_eta_3d): n_ch doubles,
  // then n_ch floats; used by channel_table while coi_shift is set
  egn_host::DevBuf d_coi;
  bool coi_shift = false;
  egn_host::DevBuf d_count;  // the planner's row counts of the island count (egn_set_wdm)
  ~egn_link() {
    d_count.release();
    d_coi.release();
    d_ch.release();
    d_seg.release();
    d_gl.release();
    d_types.release();
    ws.release();
    d_stage.release();
    if (h_stage) cudaFreeHost(h_stage);
    for (auto& e : prof_ev)
      if (e) cudaEventDestroy(e);
  }
};

namespace egn_host {

// Validate options against a link (status and message on failure).
egn_status check_opts(const egn_link* l, const egn_opts* o);
// (Re)build the link's segment and Gauss-Legendre tables for these options.
egn_status ensure_tables(egn_link* l, const egn_opts* o);
// Device channel table of a link.
egn::ChannelTable channel_table(const egn_link* l);
// Launch parameters of a link (all_terms: every term on every island).
egn::LinkParams link_params(const egn_link* l, const egn_opts* o, int all_terms);
// Offsets of the half list per (COI, n1) row inside a workspace.
const uint32_t* half_offsets(const egn::Workspace& ws, int n_ch);
// Integrator passes D/G/H, E and F of one evaluation (ev: optional stage events).
cudaError_t integrate(const egn::LinkParams& p, int precision, const uint64_t* keys, long long n_isl,
                      const uint32_t* h_idx, long long n_half, const uint32_t* e_idx, long long n_e,
                      const uint32_t* f_idx, long long n_f, void* terms, cudaStream_t st, cudaEvent_t* ev);
// Wait for an event with a host-side limit (0 = none).
egn_status wait_event(cudaEvent_t ev, int timeout_ms);
egn_status count_islands(egn_link* l, egn::PlanCounts* cnt, std::vector<long long>* per_coi);

}  // namespace egn_host
