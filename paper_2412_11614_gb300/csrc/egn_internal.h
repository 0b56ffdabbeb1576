// egn_internal.h -- library-internal types shared by the host API and the CUDA
// kernels of the GB300 ISRS EGN integrator (not part of the C ABI).
#pragma once

#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace egn {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kC = 299792458.0;  // m/s
constexpr int kMaxGl = 128;
constexpr int kMaxK = 896;     // FP64 row tables: 32 lanes x K doubles of shared memory
constexpr int kMaxKSum = 880;  // links with 2..kMaxTypes span types: segments of all types together

// Internal span: power attenuation [1/km], beta2 at the spectral centre
// [ps^2/km], beta3 [ps^3/km], gamma [1/W/km], Cr [1/W/km/THz], length [km].
struct Span {
  double alpha, beta2, beta3, gamma, cr, L;
};

// Island key: COI, n1, n2, n3 packed in 16-bit fields (COI in the low bits).
__host__ __device__ inline uint64_t pack_key(int coi, int n1, int n2, int n3) {
  return (uint64_t)(uint16_t)coi | ((uint64_t)(uint16_t)n1 << 16) | ((uint64_t)(uint16_t)n2 << 32) |
         ((uint64_t)(uint16_t)n3 << 48);
}
__host__ __device__ inline void unpack_key(uint64_t k, int& coi, int& n1, int& n2, int& n3) {
  coi = (int)(k & 0xffff);
  n1 = (int)((k >> 16) & 0xffff);
  n2 = (int)((k >> 32) & 0xffff);
  n3 = (int)((k >> 48) & 0xffff);
}

// Channel table on the device (structure of arrays, FP64).  nu is the centre
// relative to the spectral centre [THz], R the symbol rate [THz], W = R (1 +
// rolloff) the support width [THz], P the launch power [W].
struct ChannelTable {
  int n_ch;
  double wmax;  // widest support [THz]
  const double* nu;
  const double* R;
  const double* W;
  const double* P;
  const double* phi;
  const double* psi;
  // FP32 copies for the planner's candidate search and pre-test: centres and
  // half supports W/2, the widest half support and the bound on the FP32 error of
  // (W1 + W2 + W3) / 2 - |d| (outside +-plan_margin the FP32 sign is exact)
  const float* nu_f;
  const float* hw_f;
  float hwmax_f;
  float plan_margin;
  // the frequency f at which each channel is evaluated as COI (FP64 and FP32):
  // its centre (nu, nu_f) for the white-NLI reading, or centre + offset for a
  // node of the f-integral of Eq. 17-21
  const double* nu_coi;
  const float* nu_coi_f;
};

// Gauss-Legendre tables for the three outer orders ceil(n/p), p = 1, 2, 3
// (p = 1 is also the inner order n).  Nodes ascending on [-1, 1].
struct GlTables {
  int n;
  int order[4];         // order[p] = ceil(n / p), p = 1..3
  const double* x[4];   // FP64 nodes
  const double* w[4];   // FP64 weights
  const float* xh[4];   // FP32 head of the node
  const float* xl[4];   // FP32 tail: x - (double)xh
  const float* x2h[4];  // head of x^2
  const float* x2l[4];  // tail of x^2
  const float* wf[4];   // FP32 weights
};

// Per-span-type tables of the segment closed form (Eq. 8-10):
// zeta_k = P_tot Cr L_eff(z_k), C_k = B_tot zeta_k / (2 sinh(B_tot zeta_k / 2)).
struct SegmentTables {
  int K;
  const double* zeta;   // [K]
  const double* ck;     // [K]
  const float* zeta_f;  // [K] zeta_k * log2(e), FP32
  const float* ck_f;    // [K]
};

// Distinct span types of a heterogeneous link (Eq. 22 with different fibres or
// lengths): up to kMaxSpans spans, any number of types.  Up to kMaxTypes types
// travel in the launch parameters (the fast general path); links with more
// types pass all of them in device memory (LinkParams::types_dev).
constexpr int kMaxTypes = 4;
constexpr int kMaxFibres = 4;  // fibre groups tabulated by the span-by-span path
constexpr int kMaxSpans = 64;
struct SpanType {
  double alpha, beta2, beta3, gamma, L;
  double dz;   // L / K
  double r;    // e^{-alpha dz}
  double pcr;  // P_tot Cr [1/(THz km)], the ISRS slope of Eq. 4 and Eq. 25
  SegmentTables seg;
};

// Forms of the FWM efficiency mu (egn_opts.mu_form).
enum { MU_SEGMENT = 0, MU_MACLAURIN = 1, MU_INTEGRAL = 2 };
// Node rules (egn_set_node_rule): the configured panels of Gauss-Legendre nodes,
// or the ridge-resolving rule (FP64 path).
enum { RULE_GL = 0, RULE_RIDGE = 1 };
constexpr int kRidgeMaxN = 64;  // nodes per piece of the ridge rule
constexpr int kMuGl = 10;  // Gauss-Legendre order per quarter period of the integral form

// Everything an integrator launch needs, passed by value.  With n_types == 1
// (identical spans) the single-type fields below describe the span and the
// phased-array closed form of Eq. 22 applies; otherwise types[] and span_type[]
// give the explicit coherent sum over spans.
struct LinkParams {
  ChannelTable ch;
  GlTables gl;
  SegmentTables seg;
  int n_spans;       // identical spans N_s
  double alpha;      // [1/km]
  double beta2;      // [ps^2/km] at the spectral centre
  double beta3;      // [ps^3/km]
  double gamma;      // [1/W/km]
  double L;          // span length [km]
  double dz;         // L / K [km]
  double r;          // e^{-alpha dz}
  double rolloff;
  int terms;         // 0 GN, 1 EGN
  int all_terms;     // evaluate E..H on every island (parity checks)
  int fp32c_kp;      // points per thread of the FP32C D/G/H pass (4 or 8)
  int rule;          // RULE_GL or RULE_RIDGE (then gl.n is the node count per piece)
  int ridge_n_min;   // ridge rule: fewest nodes of a piece that does not end on a ridge
  const double* glx_all;  // Gauss-Legendre nodes of every order m = 1 .. gl.n, order m at offset m (m - 1) / 2
  const double* glw_all;  // and their weights
  const float* glxh_all;  // the same nodes as FP32 head + tail (x - head) and FP32 weights
  const float* glxl_all;
  const float* glwf_all;
  int mu_form;       // MU_SEGMENT, MU_MACLAURIN or MU_INTEGRAL (the last two: FP64 path)
  double btot;       // B_tot [THz] of Eq. 25
  double mgx[kMuGl], mgw[kMuGl];  // Gauss-Legendre rule of the integral form on [-1, 1]
  int n_types;                       // distinct span types (1 = identical spans)
  SpanType types[kMaxTypes];         // the first kMaxTypes of them
  const SpanType* types_dev;         // all n_types in device memory when n_types > kMaxTypes
  unsigned char span_type[kMaxSpans];  // type of span s, s = 0 .. n_spans - 1
  // Span types of one fibre (equal alpha, P_tot Cr and segment length dz) have
  // the same C_k and zeta_k for k < K_t: their c_k are prefixes of one series, so
  // the span-by-span path (more than kMaxTypes types) tabulates c_k per row once
  // per fibre.  n_fib = 0: more than kMaxFibres fibres, c_k formed on the fly.
  int n_fib;
  unsigned char type_fib[kMaxSpans];      // fibre of span type t
  const float* fib_ck[kMaxFibres];        // C_k and log2(e) zeta_k of the fibre's longest type
  const float* fib_zk[kMaxFibres];
  int fib_K[kMaxFibres];                  // its K
};

// Span type t of a launch (either array).
__host__ __device__ inline const SpanType& span_type_of(const LinkParams& p, int t) {
  return p.n_types > kMaxTypes ? p.types_dev[t] : p.types[t];
}

// Flags of an island (Kronecker deltas of Eq. 15).
__host__ __device__ inline bool flag_e(int n1, int n2, int n3) { (void)n2; return n1 == n3; }
__host__ __device__ inline bool flag_f(int n1, int n2, int n3) { (void)n1; return n2 == n3; }
__host__ __device__ inline bool flag_g(int n1, int n2, int n3) { (void)n3; return n1 == n2; }
__host__ __device__ inline bool flag_h(int n1, int n2, int n3) { return n1 == n2 && n2 == n3; }

// Island counts of a comb.  Every island (n1, n2, n3) has a mirror (n2, n1, n3)
// (f1 <-> f2) with the same D and a mirror-image node set, so the integrator
// evaluates the "half" list n1 <= n2 only; the E list is the islands with
// n1 = n3 and n1 <= n2, the F list those with n2 = n3 and n1 < n2 (each E/F
// mirror pair is evaluated once).
constexpr int kGroupBlocks = 256;  // tiles of the half list in the grouping of the D/G/H work list

struct PlanCounts {
  long long n_isl, n_half, n_e, n_f;
};

// Device workspace carve-up (byte offsets from the workspace base, 256-aligned).
// Row-count arrays hold four counters per (COI, n1) row: all islands, half
// list, E list, F list.
struct Workspace {
  uint64_t* keys;       // [n_isl] every island, (COI, n1, n2, n3) lexicographic
  uint32_t* h_idx;      // [n_half] island indices with n1 <= n2
  uint32_t* d_idx;      // [n_half] the same islands grouped by (n3, n1 + n2 - n - n3): the D/G/H work list
  uint32_t* grp_cnt;    // [4 n_ch][kGroupBlocks] group sizes per tile of the half list, then
                        // the tiles' offsets inside their group
  uint32_t* grp_off;    // [2][4 n_ch] group totals and group offsets in d_idx
  uint32_t* e_idx;      // [n_e]
  uint32_t* f_idx;      // [n_f]
  uint32_t* row_cnt;    // [4 * n_rows]
  uint32_t* row_off;    // [4 * (n_rows + 1)]
  unsigned long long* row_tot;  // [4] the four list lengths in 64 bits (overflow check)
  void* terms;          // [5 * n_isl] of double (FP64) or float (FP32C), term-major
  double* out_eta;      // [n_ch] scratch outputs when the caller passes none
  double* out_pnli;     // [n_ch]
  int* status;          // device error word
  long long cap_isl, cap_half, cap_e, cap_f;
};

size_t workspace_bytes(int n_ch, const PlanCounts& c, int precision);
Workspace carve_workspace(void* base, int n_ch, const PlanCounts& c, int precision);

// ---- launchers (defined in the .cu files) ----
// Island planner (A1): counts per (COI, n1) row, scans, emits keys and E/F lists.
cudaError_t launch_plan(const ChannelTable& ch, const Workspace& ws, cudaStream_t st);
// Counting only (used by egn_set_wdm to size the workspace).
cudaError_t launch_plan_count(const ChannelTable& ch, const Workspace& ws, cudaStream_t st);

// Integrator passes.  ord = 0: D, G, H over `list` (DW order); ord = 1: E;
// ord = 2: F.  list == nullptr means work item i is island i.
cudaError_t launch_fp64_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                             long long n_items, double* terms, long long n_isl, cudaStream_t st);
cudaError_t launch_fp32c_pass(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                              long long n_items, float* terms, long long n_isl, cudaStream_t st);
// The ridge-resolving rule in FP32C (links of identical spans; launch_fp32c_pass
// dispatches here when p.rule == RULE_RIDGE).
cudaError_t launch_ridge_fp32c(int ord, const LinkParams& p, const uint64_t* keys, const uint32_t* list,
                               long long n_items, float* terms, long long n_isl, cudaStream_t st);

// Multi-link FP32C passes (batches of links): one launch per pass and kernel
// family over the work lists of several links.  A link's family: 0 identical
// spans (phased-array closed form), 1 up to kMaxTypes span types, 2 more.
struct FlatPass {
  const LinkParams* p;   // the link's launch parameters (host copy; device pointers inside)
  const uint64_t* keys;  // its island keys (device)
  const uint32_t* list;  // the pass's work list (device; nullptr: every island)
  long long n_items;
  float* terms;          // its term slots (device)
  long long n_isl;
};
struct MultiLaunch {
  int ord, family, n_jobs;
  long long batches;  // island batches of every link of the pass
  size_t smem;        // dynamic shared memory of the launch
};
int fp32c_family(const LinkParams& p);
// Bytes of the job table of one pass over n links.
size_t fp32c_multi_bytes(int n_links);
// Host image of the job table of pass `ord` over n links of one family, and the
// launch's shape; copy the image to device memory of fp32c_multi_bytes(n) bytes.
cudaError_t fp32c_multi_build(int ord, int family, const FlatPass* links, int n, void* image, MultiLaunch* out);
cudaError_t launch_fp32c_multi(const MultiLaunch& m, const void* d_jobs, cudaStream_t st);

// Assembly (Eq. 11, 15): per-COI sums over the half list, each island weighted
// for itself and its mirror.  half_off: per-row offsets of the half list.
cudaError_t launch_assemble(const ChannelTable& ch, const uint32_t* half_off, const uint64_t* keys,
                            const uint32_t* h_idx, long long n_isl, const void* terms, int precision, int terms_mode,
                            double* eta, double* pnli, cudaStream_t st);

// The k-th largest Gauss-Legendre node of order n on [-1, 1] (k = 1 ..
// ceil(n/2)) and its weight, by Newton's method on P_n from Tricomi's asymptotic
// estimate.  Host and device (the allocation-free entry point builds its tables
// on the device) evaluate the same arithmetic.
__host__ __device__ inline void gl_node(int n, int k, double* xk_out, double* wk_out) {
  const double th = kPi * (4.0 * k - 1.0) / (4.0 * n + 2.0);
  double xk = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) * cos(th);
  double dpn = 1.0;
  for (int it = 0; it < 50; ++it) {
    double pm1 = 1.0, pn = xk;  // P_0, P_1
    for (int j = 1; j < n; ++j) {
      const double pp = ((2.0 * j + 1.0) * xk * pn - j * pm1) / (j + 1.0);
      pm1 = pn;
      pn = pp;
    }
    dpn = n * (pm1 - xk * pn) / (1.0 - xk * xk);
    const double step = pn / dpn;
    xk -= step;
    if (fabs(step) <= 1e-16) break;
  }
  {
    double pm1 = 1.0, pn = xk;
    for (int j = 1; j < n; ++j) {
      const double pp = ((2.0 * j + 1.0) * xk * pn - j * pm1) / (j + 1.0);
      pm1 = pn;
      pn = pp;
    }
    dpn = n * (pm1 - xk * pn) / (1.0 - xk * xk);
  }
  *xk_out = xk;
  *wk_out = 2.0 / ((1.0 - xk * xk) * dpn * dpn);
}

// Host Gauss-Legendre nodes on [-1, 1], ascending.
void gauss_legendre(int n, double* x, double* w);

// Opt a kernel in to `bytes` of dynamic shared memory on the current device,
// once per device: `done` holds one bit per device (ordinal mod 64), set
// atomically after the attribute is set; concurrent first calls both set it,
// which is harmless.
template <class F>
inline cudaError_t opt_in_smem(F* fn, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Entry k of a span type's segment tables (Eq. 8-10 with the ISRS profile of
// Eq. 14/25): z_k = (k + 1/2) L / K, zeta_k = P_tot Cr L_eff(z_k) with
// L_eff(z) = (1 - e^{-alpha z}) / alpha, and C_k = B_tot zeta_k / (2 sinh(B_tot
// zeta_k / 2)), whose limit at Cr = 0 is 1.  pcr = P_tot Cr.  Host and device
// evaluate the same arithmetic.
__host__ __device__ inline void segment_entry(int k, int K, double L, double alpha, double pcr, double btot,
                                              double* zeta, double* ck) {
  const double z = (k + 0.5) / K * L;
  const double leff = -expm1(-alpha * z) / alpha;
  *zeta = pcr * leff;
  const double x = btot * *zeta;
  *ck = (x == 0.0) ? 1.0 : x / (2.0 * sinh(0.5 * x));
}

}  // namespace egn
