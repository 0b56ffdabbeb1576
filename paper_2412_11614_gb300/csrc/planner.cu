// planner.cu -- island planner on the device (Eq. 15-16).
//
// For every COI n and every pair (n1, n2) the islands are the channels n3 whose
// support meets the f3 = f1 + f2 - f range with positive area, f the frequency at
// which COI n is evaluated (its centre, or a node of the f-integral).  In the island's
// local coordinates (u, v, w offsets of f1, f2, f3 from their channel centres,
// w = u + v + d with d = (nu_n1 - nu_n) + (nu_n2 - nu_n3)) the (outer w, inner u)
// region is non-empty iff
//     min(W3/2, d + (W1 + W2)/2) > max(-W3/2, d - (W1 + W2)/2).
// On a uniform grid this is the set T_kappa of Eq. 16 with n3 = n1 + n2 - n + l.
//
// Rows are (COI, n1) pairs (row = COI * n_ch + n1).  Count per row (one warp per
// row, lanes over n2), exclusive scans of the row counts (one CTA per list), and
// emit (one warp per row, warp-scan of the per-lane counts), so that the island
// list comes out in (COI, n1, n2, n3) lexicographic order together with three
// index lists: the half list (n1 <= n2), the E list (n1 == n3, n1 <= n2) and the
// F list (n2 == n3, n1 < n2).  Then the half list is grouped by
// (n3, n1 + n2 - n - n3) into the D/G/H work list (four more kernels, below).
#include "egn_internal.h"

namespace egn {
namespace {

constexpr int kPlanWarps = 8;  // warps per CTA in count/emit

__device__ __forceinline__ bool island_exists(const ChannelTable& ch, int n, int n1, int n2, int n3) {
  double d = (ch.nu[n1] - ch.nu_coi[n]) + (ch.nu[n2] - ch.nu[n3]);
  double hw = 0.5 * ch.W[n1] + 0.5 * ch.W[n2];
  double a = 0.5 * ch.W[n3];
  double lo = fmax(-a, d - hw);
  double hi = fmin(a, d + hw);
  return hi > lo;
}

// First channel index whose centre is >= x (centres non-decreasing).
__device__ __forceinline__ int lower_bound_f(const float* nu, int n, float x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (nu[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Visit the islands of (n, n1, n2) in ascending n3; f(n3) is called for each.
// The candidates n3 (centres within the reach of f1 + f2 - f) are found in FP32
// with the error bound added to the reach, so they include every island.  Each
// candidate is decided by g = (W1 + W2 + W3) / 2 - |d| in FP32 where |g| exceeds
// its error bound, else by the FP64 test: the same islands as the FP64 test
// alone, with a fraction of the FP64 work.
template <class F>
__device__ __forceinline__ void for_each_n3(const ChannelTable& ch, int n, int n1, int n2, F&& f) {
  const float t = (ch.nu_f[n1] - ch.nu_coi_f[n]) + ch.nu_f[n2];
  const float hw12 = ch.hw_f[n1] + ch.hw_f[n2];
  const float m = ch.plan_margin;
  const float reach = (hw12 + ch.hwmax_f) + 2.0f * m + 1e-6f;
  int i = lower_bound_f(ch.nu_f, ch.n_ch, t - reach);
  for (; i < ch.n_ch && ch.nu_f[i] <= t + reach; ++i) {
    const float g = (hw12 + ch.hw_f[i]) - fabsf(t - ch.nu_f[i]);
    if (g > m || (g >= -m && island_exists(ch, n, n1, n2, i))) f(i);
  }
}

struct Counts {
  uint32_t a, h, e, f;
};

__device__ __forceinline__ Counts count_pair(const ChannelTable& ch, int n, int n1, int n2) {
  Counts c = {0, 0, 0, 0};
  for_each_n3(ch, n, n1, n2, [&](int n3) {
    ++c.a;
    c.h += (n1 <= n2);
    c.e += (n3 == n1 && n1 <= n2);
    c.f += (n3 == n2 && n1 < n2);
  });
  return c;
}

__global__ void plan_count_kernel(ChannelTable a, uint32_t* row_cnt, int n_rows) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n_rows) return;
  int n = warp / a.n_ch, n1 = warp % a.n_ch;
  Counts c = {0, 0, 0, 0};
  for (int n2 = lane; n2 < a.n_ch; n2 += 32) {
    Counts t = count_pair(a, n, n1, n2);
    c.a += t.a; c.h += t.h; c.e += t.e; c.f += t.f;
  }
  for (int o = 16; o > 0; o >>= 1) {
    c.a += __shfl_down_sync(0xffffffffu, c.a, o);
    c.h += __shfl_down_sync(0xffffffffu, c.h, o);
    c.e += __shfl_down_sync(0xffffffffu, c.e, o);
    c.f += __shfl_down_sync(0xffffffffu, c.f, o);
  }
  if (lane == 0) {
    row_cnt[warp] = c.a;
    row_cnt[n_rows + warp] = c.h;
    row_cnt[2 * n_rows + warp] = c.e;
    row_cnt[3 * n_rows + warp] = c.f;
  }
}

// Exclusive scan of the four count arrays (one CTA of 1024 threads per array,
// each thread a contiguous chunk).  row_off[a * (n_rows + 1) + n_rows] is the
// total, and row_tot[a] the same total in 64 bits (the host refuses totals above
// 2^32 - 1).
__global__ void plan_scan_kernel(const uint32_t* row_cnt, uint32_t* row_off, unsigned long long* row_tot,
                                 int n_rows) {
  __shared__ uint32_t warp_sum[32];
  __shared__ unsigned long long warp_sum64[32];
  const int T = blockDim.x;
  int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int chunk = (n_rows + T - 1) / T;
  {
    const int arr = blockIdx.x;
    const uint32_t* in = row_cnt + (size_t)arr * n_rows;
    uint32_t* out = row_off + (size_t)arr * (n_rows + 1);
    int b = tid * chunk, e = min(b + chunk, n_rows);
    uint32_t s = 0;
    unsigned long long s64 = 0;
    for (int i = b; i < e; ++i) {
      s += in[i];
      s64 += in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
    if (lane == 0) warp_sum64[wid] = s64;
    // block exclusive scan of s
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t v = (lane < (T >> 5)) ? warp_sum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      warp_sum[lane] = v;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t base = (wid > 0 ? warp_sum[wid - 1] : 0) + x - s;
    for (int i = b; i < e; ++i) {
      out[i] = base;
      base += in[i];
    }
    if (tid == T - 1) out[n_rows] = warp_sum[(T >> 5) - 1];
    if (tid == 0) {
      unsigned long long t64 = 0;
      for (int w = 0; w < (T >> 5); ++w) t64 += warp_sum64[w];
      row_tot[arr] = t64;
    }
    __syncthreads();
  }
}

__global__ void plan_emit_kernel(ChannelTable a, const uint32_t* row_off, int n_rows, Workspace ws) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n_rows) return;
  const int nch = a.n_ch;
  int n = warp / nch, n1 = warp % nch;
  uint32_t base = row_off[warp];
  uint32_t base_h = row_off[(n_rows + 1) + warp];
  uint32_t base_e = row_off[2 * (n_rows + 1) + warp];
  uint32_t base_f = row_off[3 * (n_rows + 1) + warp];
  for (int n2b = 0; n2b < nch; n2b += 32) {
    int n2 = n2b + lane;
    Counts c = {0, 0, 0, 0};
    if (n2 < nch) c = count_pair(a, n, n1, n2);
    // warp inclusive scans
    Counts ic = c;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y0 = __shfl_up_sync(0xffffffffu, ic.a, o);
      uint32_t y1 = __shfl_up_sync(0xffffffffu, ic.h, o);
      uint32_t y2 = __shfl_up_sync(0xffffffffu, ic.e, o);
      uint32_t y3 = __shfl_up_sync(0xffffffffu, ic.f, o);
      if (lane >= o) { ic.a += y0; ic.h += y1; ic.e += y2; ic.f += y3; }
    }
    uint32_t pos = base + ic.a - c.a, ph = base_h + ic.h - c.h, pe = base_e + ic.e - c.e, pf = base_f + ic.f - c.f;
    if (n2 < nch)
      for_each_n3(a, n, n1, n2, [&](int n3) {
        if ((long long)pos < ws.cap_isl) ws.keys[pos] = pack_key(n, n1, n2, n3); else atomicOr(ws.status, 1);
        if (n1 <= n2) {
          if ((long long)ph < ws.cap_half) ws.h_idx[ph] = pos; else atomicOr(ws.status, 8);
          ++ph;
        }
        if (n3 == n1 && n1 <= n2) {
          if ((long long)pe < ws.cap_e) ws.e_idx[pe] = pos; else atomicOr(ws.status, 2);
          ++pe;
        }
        if (n3 == n2 && n1 < n2) {
          if ((long long)pf < ws.cap_f) ws.f_idx[pf] = pos; else atomicOr(ws.status, 4);
          ++pf;
        }
        ++pos;
      });
    base += __shfl_sync(0xffffffffu, ic.a, 31);
    base_h += __shfl_sync(0xffffffffu, ic.h, 31);
    base_e += __shfl_sync(0xffffffffu, ic.e, 31);
    base_f += __shfl_sync(0xffffffffu, ic.f, 31);
  }
}

// ---- the D/G/H work list: the half list grouped by (n3, n1 + n2 - n - n3),
// which on a uniform grid is (n3, -l): the islands of a group have the same
// outer nodes f3, so consecutive islands can share the c_k tables of their rows.
// A counting sort with atomic cursors: the order inside a group is arbitrary,
// which changes no result (every island is integrated on its own).
__device__ __forceinline__ int dw_group(uint64_t key) {
  int c, a, b, d;
  unpack_key(key, c, a, b, d);
  int t = a + b - c - d + 1;
  t = t < 0 ? 0 : (t > 3 ? 3 : t);
  return 4 * d + t;
}

// The grouping runs on kGroupBlocks tiles of the half list: per tile a shared-
// memory histogram of the groups, then one exclusive scan over (group, tile), then
// each tile scatters its islands from its own offsets (shared-memory cursors).
__global__ void group_count_kernel(const uint64_t* keys, const uint32_t* h_idx, long long n_half, int ng,
                                   uint32_t* blk_cnt) {
  extern __shared__ uint32_t hist[];
  const int nb = gridDim.x, b = blockIdx.x;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) hist[g] = 0;
  __syncthreads();
  const long long tile = (n_half + nb - 1) / nb;
  const long long i0 = (long long)b * tile, i1 = min(n_half, i0 + tile);
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) atomicAdd(&hist[dw_group(keys[h_idx[i]])], 1u);
  __syncthreads();
  for (int g = threadIdx.x; g < ng; g += blockDim.x) blk_cnt[(size_t)g * nb + b] = hist[g];
}

// Per group (one warp each): exclusive offsets of its tiles inside the group, in
// place over the tile counts, and the group's total.
__global__ void group_tile_scan_kernel(uint32_t* blk, int ng, int nb, uint32_t* gtot) {
  const int g = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (g >= ng) return;
  uint32_t* row = blk + (size_t)g * nb;
  const int per = (nb + 31) / 32, t0 = lane * per, t1 = min(t0 + per, nb);
  uint32_t s = 0;
  for (int t = t0; t < t1; ++t) s += row[t];
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  uint32_t base = x - s;
  for (int t = t0; t < t1; ++t) {
    const uint32_t c = row[t];
    row[t] = base;
    base += c;
  }
  if (lane == 31) gtot[g] = x;
}

// Exclusive scan of the group totals (one CTA, each thread a contiguous chunk).
__global__ void group_scan_kernel(const uint32_t* cnt, uint32_t* off, int n) {
  __shared__ uint32_t warp_sum[32];
  const int T = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int chunk = (n + T - 1) / T;
  const int b = tid * chunk, e = min(b + chunk, n);
  uint32_t s = 0;
  for (int i = b; i < e; ++i) s += cnt[i];
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = (lane < (T >> 5)) ? warp_sum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    warp_sum[lane] = v;
  }
  __syncthreads();
  uint32_t base = (wid > 0 ? warp_sum[wid - 1] : 0) + x - s;
  for (int i = b; i < e; ++i) {
    off[i] = base;
    base += cnt[i];
  }
}

__global__ void group_scatter_kernel(const uint64_t* keys, const uint32_t* h_idx, long long n_half, int ng,
                                     const uint32_t* blk_off, const uint32_t* gbase, uint32_t* d_idx, int* status) {
  extern __shared__ uint32_t cur[];
  const int nb = gridDim.x, b = blockIdx.x;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) cur[g] = gbase[g] + blk_off[(size_t)g * nb + b];
  __syncthreads();
  const long long tile = (n_half + nb - 1) / nb;
  const long long i0 = (long long)b * tile, i1 = min(n_half, i0 + tile);
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint32_t isl = h_idx[i];
    const long long at = atomicAdd(&cur[dw_group(keys[isl])], 1u);
    if (at < n_half) d_idx[at] = isl; else atomicOr(status, 16);
  }
}

}  // namespace

cudaError_t launch_plan_count(const ChannelTable& ch, const Workspace& ws, cudaStream_t st) {
  int n_rows = ch.n_ch * ch.n_ch;
  int threads = kPlanWarps * 32;
  int blocks = (n_rows + kPlanWarps - 1) / kPlanWarps;
  plan_count_kernel<<<blocks, threads, 0, st>>>(ch, ws.row_cnt, n_rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  plan_scan_kernel<<<4, 1024, 0, st>>>(ws.row_cnt, ws.row_off, ws.row_tot, n_rows);
  return cudaGetLastError();
}

cudaError_t launch_plan(const ChannelTable& ch, const Workspace& ws, cudaStream_t st) {
  cudaError_t e = launch_plan_count(ch, ws, st);
  if (e != cudaSuccess) return e;
  int n_rows = ch.n_ch * ch.n_ch;
  int threads = kPlanWarps * 32;
  int blocks = (n_rows + kPlanWarps - 1) / kPlanWarps;
  plan_emit_kernel<<<blocks, threads, 0, st>>>(ch, ws.row_off, n_rows, ws);
  e = cudaGetLastError();
  if (e != cudaSuccess || ws.cap_half <= 0) return e;
  const int ng = 4 * ch.n_ch;
  const size_t hist_b = (size_t)ng * sizeof(uint32_t);  // <= 64 KB (n_ch <= 4096)
  static std::atomic<unsigned long long> count_done{0}, scatter_done{0};  // opt in to more than 48 KB once per device
  if ((e = opt_in_smem(group_count_kernel, 16384 * 4, count_done)) != cudaSuccess) return e;
  if ((e = opt_in_smem(group_scatter_kernel, 16384 * 4, scatter_done)) != cudaSuccess) return e;
  group_count_kernel<<<kGroupBlocks, 256, hist_b, st>>>(ws.keys, ws.h_idx, ws.cap_half, ng, ws.grp_cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // tile offsets inside each group (in place), group totals, group offsets
  uint32_t* gtot = ws.grp_off;
  uint32_t* gbase = ws.grp_off + ng;
  group_tile_scan_kernel<<<(ng + 7) / 8, 256, 0, st>>>(ws.grp_cnt, ng, kGroupBlocks, gtot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  group_scan_kernel<<<1, 1024, 0, st>>>(gtot, gbase, ng);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  group_scatter_kernel<<<kGroupBlocks, 256, hist_b, st>>>(ws.keys, ws.h_idx, ws.cap_half, ng, ws.grp_cnt, gbase,
                                                          ws.d_idx, ws.status);
  return cudaGetLastError();
}

}  // namespace egn
