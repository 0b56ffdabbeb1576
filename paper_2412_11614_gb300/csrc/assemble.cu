// assemble.cu -- per-COI assembly of the island terms (Eq. 11, 15).
//
//   P_NLI,n = sum_islands P_n1 P_n2 P_n3 [D + Phi_n1 d13 E + Phi_n2 d23 F
//                                         + Phi_n1 d12 G + Psi_n1 d12 d23 H]
//   eta_n   = P_NLI,n / P_n^3
//
// The sum runs over the half list (n1 <= n2) and counts every island's mirror
// (n2, n1, n3), which has the same D and P_n1 P_n2 P_n3:
//   D x 2 when n1 < n2 (x 1 when n1 = n2);
//   an E island (n1 = n3 <= n2) stands for itself and the mirror F island
//   (n2, n1, n1), whose F is (32/81)/(16/27) = 2/3 of its E: Phi_n1 E x 5/3;
//   an F island (n2 = n3, n1 < n2) stands for itself and the mirror E island,
//   E = 3/2 F: Phi_n2 F x 5/2;
//   G (n1 = n2) and H (n1 = n2 = n3) islands are their own mirrors.
// One CTA per COI walks the COI's contiguous range of the half list.  Every
// thread accumulates a strided subset in a fixed order and the CTA combines the
// partial sums with a fixed tree, so results are bitwise reproducible.  FP64
// terms accumulate in FP64; FP32 terms accumulate in compensated FP32 (a
// double-float pair updated by an error-free two-sum).
#include "egn_internal.h"

namespace egn {
namespace {

constexpr int kAsmThreads = 256;

// Error-free transformation: a + b = s + e exactly (Knuth two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct Df {
  float hi, lo;
};

__device__ __forceinline__ Df df_add(Df x, float y) {
  float s, e;
  two_sum(x.hi, y, s, e);
  e += x.lo;
  float hi, lo;
  two_sum(s, e, hi, lo);
  return {hi, lo};
}

__device__ __forceinline__ Df df_add(Df x, Df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e += x.lo + y.lo;
  float hi, lo;
  two_sum(s, e, hi, lo);
  return {hi, lo};
}

template <class T>
__device__ __forceinline__ double island_contrib(const ChannelTable& ch, const T* terms, long long n_isl,
                                                 long long i, uint64_t key, int egn) {
  int coi, n1, n2, n3;
  unpack_key(key, coi, n1, n2, n3);
  double s = (double)terms[i] * (n1 < n2 ? 2.0 : 1.0);
  if (egn) {
    if (n1 == n3) s += (5.0 / 3.0) * ch.phi[n1] * (double)terms[1 * n_isl + i];
    if (n2 == n3 && n1 < n2) s += 2.5 * ch.phi[n2] * (double)terms[2 * n_isl + i];
    if (flag_g(n1, n2, n3)) s += ch.phi[n1] * (double)terms[3 * n_isl + i];
    if (flag_h(n1, n2, n3)) s += ch.psi[n1] * (double)terms[4 * n_isl + i];
  }
  return ch.P[n1] * ch.P[n2] * ch.P[n3] * s;
}

__global__ void __launch_bounds__(kAsmThreads) assemble_fp64_kernel(ChannelTable ch, const uint32_t* half_off,
                                                                    const uint64_t* keys, const uint32_t* h_idx,
                                                                    long long n_isl, const double* terms, int egn,
                                                                    double* eta, double* pnli) {
  __shared__ double red[kAsmThreads];
  int coi = blockIdx.x;
  long long b = half_off[(size_t)coi * ch.n_ch], e = half_off[(size_t)(coi + 1) * ch.n_ch];
  double acc = 0.0;
  for (long long j = b + threadIdx.x; j < e; j += kAsmThreads) {
    long long i = h_idx[j];
    acc += island_contrib(ch, terms, n_isl, i, keys[i], egn);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kAsmThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double p = ch.P[coi];
    if (pnli) pnli[coi] = red[0];
    if (eta) eta[coi] = red[0] / (p * p * p);
  }
}

// Compensated FP32 assembly: island contributions are formed in FP32 from the
// FP32 terms and FP32 copies of the powers, and summed as double-float pairs.
__global__ void __launch_bounds__(kAsmThreads) assemble_fp32c_kernel(ChannelTable ch, const uint32_t* half_off,
                                                                     const uint64_t* keys, const uint32_t* h_idx,
                                                                     long long n_isl, const float* terms, int egn,
                                                                     double* eta, double* pnli) {
  __shared__ Df red[kAsmThreads];
  int coi = blockIdx.x;
  long long b = half_off[(size_t)coi * ch.n_ch], e = half_off[(size_t)(coi + 1) * ch.n_ch];
  // Scale the sum by 1 / P_coi^3 up front so that the FP32 range is centred on eta.
  float inv_p3 = (float)(1.0 / (ch.P[coi] * ch.P[coi] * ch.P[coi]));
  Df acc = {0.0f, 0.0f};
  for (long long j = b + threadIdx.x; j < e; j += kAsmThreads) {
    long long i = h_idx[j];
    int c, n1, n2, n3;
    unpack_key(keys[i], c, n1, n2, n3);
    float s = terms[i] * (n1 < n2 ? 2.0f : 1.0f);
    if (egn) {
      if (n1 == n3) s = fmaf((5.0f / 3.0f) * (float)ch.phi[n1], terms[1 * n_isl + i], s);
      if (n2 == n3 && n1 < n2) s = fmaf(2.5f * (float)ch.phi[n2], terms[2 * n_isl + i], s);
      if (flag_g(n1, n2, n3)) s = fmaf((float)ch.phi[n1], terms[3 * n_isl + i], s);
      if (flag_h(n1, n2, n3)) s = fmaf((float)ch.psi[n1], terms[4 * n_isl + i], s);
    }
    float w = (float)ch.P[n1] * (float)ch.P[n2] * (float)ch.P[n3] * inv_p3;
    acc = df_add(acc, w * s);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kAsmThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = df_add(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double p = ch.P[coi];
    double et = (double)red[0].hi + (double)red[0].lo;
    if (eta) eta[coi] = et;
    if (pnli) pnli[coi] = et * (p * p * p);
  }
}

}  // namespace

cudaError_t launch_assemble(const ChannelTable& ch, const uint32_t* half_off, const uint64_t* keys,
                            const uint32_t* h_idx, long long n_isl, const void* terms, int precision, int terms_mode,
                            double* eta, double* pnli, cudaStream_t st) {
  if (precision == 0)
    assemble_fp64_kernel<<<ch.n_ch, kAsmThreads, 0, st>>>(ch, half_off, keys, h_idx, n_isl, (const double*)terms,
                                                          terms_mode, eta, pnli);
  else
    assemble_fp32c_kernel<<<ch.n_ch, kAsmThreads, 0, st>>>(ch, half_off, keys, h_idx, n_isl, (const float*)terms,
                                                           terms_mode, eta, pnli);
  return cudaGetLastError();
}

}  // namespace egn
