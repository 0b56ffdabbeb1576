// probe.cu -- throughput probes of the arithmetic pipes (include/egn_probe.h).
//
// One kernel per pipe.  Every thread runs `iters` rounds of eight independent
// dependency chains of one instruction, so that each SM sub-partition always has
// independent work for the pipe; the chain values go to a sink at the end.  The
// chain operands keep the values finite and away from denormals: FMA chains
// x <- x * a + b with |a| < 1 converge to b / (1 - a); sin(x) stays in [-1, 1];
// 2^-x maps (0, 1] into [1/2, 1); x <- 1/x + 1/2 stays in [1/2, 5/2].
#include "../../include/egn_probe.h"
#include "link.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__global__ void probe_ffma(int iters, float a, float b, double* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.001f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_ffma2(int iters, float a, float b, double* sink) {
  unsigned long long x[kChains];
  const unsigned long long a2 = f2_pack(a, a), b2 = f2_pack(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = f2_pack(0.001f * (float)(threadIdx.x + c), 0.002f * (float)c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    f2_unpack(x[c], lo, hi);
    s += lo + hi;
  }
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed and scalar FMA chains side by side: 8 of each per thread.
__global__ void probe_fma_mix(int iters, float a, float b, double* sink) {
  unsigned long long x[kChains];
  float y[kChains];
  const unsigned long long a2 = f2_pack(a, a), b2 = f2_pack(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = f2_pack(0.001f * (float)(threadIdx.x + c), 0.002f * (float)c);
    y[c] = 0.003f * (float)(threadIdx.x + c);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(a2), "l"(b2));
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(y[c]) : "f"(a), "f"(b));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    f2_unpack(x[c], lo, hi);
    s += lo + hi + y[c];
  }
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_dfma(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.001 * (double)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[c]) : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int KIND>
__global__ void probe_mufu(int iters, double* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 0.001f * (float)((threadIdx.x + c) & 255);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (KIND == EGN_PROBE_MUFU_SIN) asm volatile("sin.approx.f32 %0, %0;" : "+f"(x[c]));
      if (KIND == EGN_PROBE_MUFU_EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
      // 1/x alone is an involution the assembler may fold in pairs: x <- 1/x + 1/2
      // (the addition runs on the FMA pipe) converges to (1 + sqrt(17)) / 4
      if (KIND == EGN_PROBE_MUFU_RCP) asm volatile("rcp.approx.ftz.f32 %0, %0;\n\tadd.f32 %0, %0, 0f3F000000;" : "+f"(x[c]));
    }
    if (KIND == EGN_PROBE_MUFU_EX2) {  // 2^x grows: keep the argument in (0, 1] with one negation per round
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = -x[c];
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

bool valid(int kind, int blocks, int threads, int iters) {
  return kind >= EGN_PROBE_FFMA && kind <= EGN_PROBE_FMA_MIX && blocks >= 1 && threads >= 32 && threads <= 1024 &&
         threads % 32 == 0 && iters >= 1;
}

}  // namespace

extern "C" {

egn_status egn_probe_ops(int kind, int blocks, int threads, int iters, double* ops) {
  if (!ops || !valid(kind, blocks, threads, iters)) return egn_host::fail(EGN_E_INVALID_ARG, "bad probe arguments");
  const double lanes = (double)blocks * threads * kChains * iters;
  switch (kind) {
    case EGN_PROBE_FFMA: *ops = 2.0 * lanes; break;
    case EGN_PROBE_FFMA2: *ops = 4.0 * lanes; break;
    case EGN_PROBE_DFMA: *ops = 2.0 * lanes; break;
    case EGN_PROBE_FMA_MIX: *ops = 6.0 * lanes; break;
    default: *ops = lanes; break;
  }
  return EGN_OK;
}

egn_status egn_probe_launch(int kind, int blocks, int threads, int iters, void* sink, void* stream) {
  if (!sink || !valid(kind, blocks, threads, iters)) return egn_host::fail(EGN_E_INVALID_ARG, "bad probe arguments");
  cudaStream_t st = (cudaStream_t)stream;
  double* s = (double*)sink;
  switch (kind) {
    case EGN_PROBE_FFMA: probe_ffma<<<blocks, threads, 0, st>>>(iters, 0.5f, 0.25f, s); break;
    case EGN_PROBE_FFMA2: probe_ffma2<<<blocks, threads, 0, st>>>(iters, 0.5f, 0.25f, s); break;
    case EGN_PROBE_DFMA: probe_dfma<<<blocks, threads, 0, st>>>(iters, 0.5, 0.25, s); break;
    case EGN_PROBE_MUFU_SIN: probe_mufu<EGN_PROBE_MUFU_SIN><<<blocks, threads, 0, st>>>(iters, s); break;
    case EGN_PROBE_MUFU_EX2: probe_mufu<EGN_PROBE_MUFU_EX2><<<blocks, threads, 0, st>>>(iters, s); break;
    case EGN_PROBE_FMA_MIX: probe_fma_mix<<<blocks, threads, 0, st>>>(iters, 0.5f, 0.25f, s); break;
    default: probe_mufu<EGN_PROBE_MUFU_RCP><<<blocks, threads, 0, st>>>(iters, s); break;
  }
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

}  // extern "C"
