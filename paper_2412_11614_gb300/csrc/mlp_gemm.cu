// mlp_gemm.cu -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the
// MLP surrogate: D = A B^T, A [m][k] and B [n][k] row-major (k contiguous),
// FP32 accumulation in tensor memory (TMEM), fused epilogues.
//
// Persistent warp-specialised kernel, one CTA of 192 threads per SM, tiles of
// 128 x 256 of D taken round-robin in groups of 8 m-tiles by every n-tile:
//   warp 0, one lane : TMA producer, 64-wide k blocks of A (128 x 64) and B
//                      (256 x 64) into a 4-stage ring, 128-byte swizzle, running
//                      ahead across tiles;
//   warp 1, one lane : MMA issuer, 4 x tcgen05.mma (M 128, N 256, K 16) per k
//                      block into one of two TMEM accumulators (2 x 256 columns);
//                      tcgen05.commit releases each stage and marks a finished
//                      accumulator;
//   warps 2-5        : epilogue, warp w reads TMEM lanes 32 (w mod 4) .. + 31
//                      (rows) with tcgen05.ld, 32 columns at a time, then hands
//                      the accumulator back: the next tile's MMAs overlap it.
// The k range may be split (partial sums written to slab z, summed by
// egn_mlp_reduce_splits in a fixed order).  Every mbarrier wait is bounded
// (kWaitNs of wall time); a wait that runs out sets the error word and a shared
// abort flag that stops every role, the producer drains its own copies in
// flight, the MMA issuer waits for its MMAs, TMEM is freed and the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "../../include/egn_mlp.h"
#include "link.h"

using namespace egn_host;

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int kStageA = BM * BK * 2;  // 16 KB
constexpr int kStageB = BN * BK * 2;  // 32 KB
constexpr int kSmem = STAGES * (kStageA + kStageB) + 1024 /* alignment */ + 256 /* barriers */;
constexpr int kGemmThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kGroupM = 8;         // m-tiles per group of the tile order
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try_wait(b, parity)) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand with 128-byte swizzle: rows of
// 64 BF16 (128 bytes), 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused (1), descriptor version 1 (bits 46-47), layout
// SWIZZLE_128B (2 at bits 61-63).  The tile base is 1024-byte aligned.
__device__ __forceinline__ uint64_t sdesc_sw128(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a & 0x3FFFFull) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void umma_bf16(uint32_t taddr, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          taddr),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Epilogue of one accumulator row chunk: 32 columns n .. n + 31 of row `row`.
// GELU(z) = z Phi(z) with Phi the standard normal distribution function, and
// its derivative Phi(z) + z phi(z).
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * (0.39894228040143268f * __expf(-0.5f * z * z));
}

template <int EPI>
__device__ __forceinline__ void store_chunk(const float (&v)[32], int row, int n, int M, int N, int z,
                                            const float* __restrict__ bias, __nv_bfloat16* aux,
                                            void* __restrict__ out) {
  if (EPI == EGN_MLP_EPI_F32) {
    float* o = (float*)out + (size_t)z * (size_t)M * N + (size_t)row * N + n;
#pragma unroll
    for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
  } else {
    __nv_bfloat16* o = (__nv_bfloat16*)out + (size_t)row * N + n;
    __align__(16) __nv_bfloat16 h[32];
    if (EPI == EGN_MLP_EPI_BIAS_RELU) {
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16_rn(fmaxf(v[j] + bias[n + j], 0.0f));
    } else if (EPI == EGN_MLP_EPI_BIAS) {
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16_rn(v[j] + bias[n + j]);
    } else if (EPI == EGN_MLP_EPI_BIAS_GELU) {  // GELU of the pre-activation, which goes to aux
      __align__(16) __nv_bfloat16 za[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const __nv_bfloat16 zb = __float2bfloat16_rn(v[j] + bias[n + j]);
        za[j] = zb;
        h[j] = __float2bfloat16_rn(gelu_f(__bfloat162float(zb)));
      }
      __nv_bfloat16* zo = aux + (size_t)row * N + n;
#pragma unroll
      for (int j = 0; j < 32; j += 8) *reinterpret_cast<uint4*>(zo + j) = *reinterpret_cast<const uint4*>(za + j);
    } else if (EPI == EGN_MLP_EPI_GELU_GRAD) {  // times GELU' of the stored pre-activation
      const __nv_bfloat16* a = aux + (size_t)row * N + n;
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16_rn(v[j] * gelu_grad_f(__bfloat162float(a[j])));
    } else {  // EGN_MLP_EPI_RELU_GRAD: the gradient passes where the layer's output was positive
      const __nv_bfloat16* a = aux + (size_t)row * N + n;
#pragma unroll
      for (int j = 0; j < 32; ++j) h[j] = __float2bfloat16_rn(__bfloat162float(a[j]) > 0.0f ? v[j] : 0.0f);
    }
#pragma unroll
    for (int j = 0; j < 32; j += 8) *reinterpret_cast<uint4*>(o + j) = *reinterpret_cast<const uint4*>(h + j);
  }
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ... (grouped order, see decode).  Two TMEM accumulators (2 x 256 columns): the MMA issuer fills one
// while the epilogue warps drain the other.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
                     int kb_per_split, int kb_total, int splits, const float* __restrict__ bias,
                     __nv_bfloat16* aux, void* __restrict__ out, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * kStageA;
  uint64_t* full = (uint64_t*)(sB + STAGES * kStageB);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;  // [2] accumulator b holds a finished tile
  uint64_t* acce = accf + 2;        // [2] accumulator b has been read out
  uint64_t* drain = acce + 2;       // the MMA issuer's last commit
  uint32_t* tslot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const long long total = (long long)tm * tn * splits;
  // tile t -> (m, n, split): within a split, groups of kGroupM m-tiles by every
  // n-tile, m fastest inside a group, so one wave's A and B blocks fit in L2 together
  auto decode = [&](long long t, int& m0, int& n0, int& z, int& kb0, int& nk) {
    const long long per = (long long)tm * tn;
    z = (int)(t / per);
    const int r = (int)(t - (long long)z * per);
    const int g = r / (kGroupM * tn), first = g * kGroupM, gm = min(kGroupM, tm - first);
    const int l = r - g * kGroupM * tn;
    m0 = (first + l % gm) * BM;
    n0 = (l / gm) * BN;
    kb0 = z * kb_per_split;
    nk = min(kb_per_split, kb_total - kb0);
  };
  auto fail = [&](int code) {
    *abort_flag = 1;
    atomicExch(err, code);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], kGemmThreads / 32 - 2);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();  // the .sync.aligned tcgen05 instructions need the whole warp converged
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t taddr = *tslot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer: k blocks of every tile through the ring
      long long g = 0;
      for (long long t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x) {
        int m0, n0, z, kb0, nk;
        decode(t, m0, n0, z, kb0, nk);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (g >= STAGES && !mbar_wait(&empty[s], ph ^ 1)) { ok = false; break; }
          mbar_expect_tx(&full[s], kStageA + kStageB);
          tma_load_2d(sA + s * kStageA, &ta, &full[s], (kb0 + kb) * BK, m0);
          tma_load_2d(sB + s * kStageB, &tb, &full[s], (kb0 + kb) * BK, n0);
        }
        if (!ok) { fail(1); break; }
      }
      // every copy issued has landed before the CTA may exit
      for (long long gg = g > STAGES ? g - STAGES : 0; gg < g; ++gg) mbar_wait(&full[gg % STAGES], (gg / STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      long long g = 0;
      int i = 0;
      for (long long t = blockIdx.x; t < total && !*abort_flag; t += gridDim.x, ++i) {
        int m0, n0, z, kb0, nk;
        decode(t, m0, n0, z, kb0, nk);
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(&acce[b], ((i >> 1) & 1) ^ 1)) { fail(2); break; }
        fence_after();
        const uint32_t acc = taddr + (uint32_t)(b * BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (!mbar_wait(&full[s], ph)) { ok = false; break; }
          fence_after();
          const uint64_t ad = sdesc_sw128(sA + s * kStageA), bd = sdesc_sw128(sB + s * kStageB);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) umma_bf16(acc, ad + 2 * k, bd + 2 * k, (kb | k) != 0);  // +32 B per k step
          umma_commit(&empty[s]);
        }
        if (!ok) { fail(2); break; }
        umma_commit(&accf[b]);
      }
      umma_commit(drain);  // arrives when every MMA issued above has completed
      mbar_wait(drain, 0);
    }
  } else {  // epilogue warps 2..5: warp w reads TMEM lanes 32 (w mod 4) .. + 31
    const int grp = warp & 3;
    int i = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++i) {
      if (*abort_flag) break;
      int m0, n0, z, kb0, nk;
      decode(t, m0, n0, z, kb0, nk);
      const int b = i & 1;
      const bool ready = __all_sync(0xffffffffu, mbar_wait(&accf[b], (i >> 1) & 1));
      if (!ready) {
        if (lane == 0) fail(3);
        break;
      }
      fence_after();
      const int row = m0 + grp * 32 + lane;
      for (int c = 0; c < BN; c += 32) {
        float v[32];
        tmem_ld32(taddr + ((uint32_t)(grp * 32) << 16) + (uint32_t)(b * BN + c), v);
        if (row < M && n0 + c < N) store_chunk<EPI>(v, row, n0 + c, M, N, z, bias, aux, out);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
    }
  }
  fence_before();
  __syncthreads();
  __syncwarp();  // the producer lane rejoins its warp before the .sync.aligned dealloc
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * BN));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// Tensor map of a row-major [rows][cols] BF16 matrix, boxes of box_rows x 64
// with 128-byte swizzle (the shared-memory layout the MMA descriptors expect).
egn_status make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return fail(EGN_E_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(EGN_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return EGN_OK;
}

template <int EPI>
egn_status launch(const CUtensorMap& ta, const CUtensorMap& tb, int m, int n, int kb_per, int kb, int splits,
                  const float* bias, const void* aux, void* out, int* err, cudaStream_t st) {
  static std::atomic<unsigned long long> attr_done{0};  // per device
  EGN_CUDA(egn::opt_in_smem(gemm_bf16_kernel<EPI>, kSmem, attr_done));
  int dev = 0, sms = 0;
  EGN_CUDA(cudaGetDevice(&dev));
  EGN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long tiles = (long long)((m + BM - 1) / BM) * ((n + BN - 1) / BN) * splits;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);  // persistent: one CTA per SM
  gemm_bf16_kernel<EPI><<<grid, kGemmThreads, kSmem, st>>>(ta, tb, m, n, kb_per, kb, splits, bias,
                                                            (__nv_bfloat16*)const_cast<void*>(aux), out, err);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

}  // namespace

extern "C" egn_status egn_mlp_gemm(int m, int n, int k, int splits, const void* a, const void* b, int epilogue,
                                   const float* bias, const void* aux, void* out, int* err_dev, void* stream) {
  if (m < 1 || n < 1 || k < 1) return fail(EGN_E_INVALID_ARG, "m, n, k must be positive");
  if (k % BK) return fail(EGN_E_INVALID_ARG, "k = %d is not a multiple of %d", k, BK);
  if (n % 32) return fail(EGN_E_INVALID_ARG, "n = %d is not a multiple of 32", n);
  if (!a || !b || !out || !err_dev) return fail(EGN_E_INVALID_ARG, "null pointer");
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)out) & 15) return fail(EGN_E_INVALID_ARG, "A, B, out must be 16-byte aligned");
  const int kb = k / BK;
  if (splits < 1 || splits > kb) return fail(EGN_E_INVALID_ARG, "splits must be in [1, k/64]");
  if (splits > 1 && epilogue != EGN_MLP_EPI_F32) return fail(EGN_E_INVALID_ARG, "split k needs the FP32 epilogue");
  if ((epilogue == EGN_MLP_EPI_BIAS_RELU || epilogue == EGN_MLP_EPI_BIAS || epilogue == EGN_MLP_EPI_BIAS_GELU) && !bias)
    return fail(EGN_E_INVALID_ARG, "bias required");
  if ((epilogue == EGN_MLP_EPI_RELU_GRAD || epilogue == EGN_MLP_EPI_BIAS_GELU || epilogue == EGN_MLP_EPI_GELU_GRAD) &&
      (!aux || ((uintptr_t)aux & 15)))
    return fail(EGN_E_INVALID_ARG, "aux required (16-byte aligned)");
  const int kb_per = (kb + splits - 1) / splits;
  if ((long long)(splits - 1) * kb_per >= kb) return fail(EGN_E_INVALID_ARG, "splits leaves an empty k range");
  CUtensorMap ta, tb;
  egn_status s = make_map(&ta, a, (uint64_t)m, (uint64_t)k, BM);
  if (s == EGN_OK) s = make_map(&tb, b, (uint64_t)n, (uint64_t)k, BN);
  if (s != EGN_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  switch (epilogue) {
    case EGN_MLP_EPI_BIAS_RELU: return launch<EGN_MLP_EPI_BIAS_RELU>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    case EGN_MLP_EPI_BIAS: return launch<EGN_MLP_EPI_BIAS>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    case EGN_MLP_EPI_F32: return launch<EGN_MLP_EPI_F32>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    case EGN_MLP_EPI_RELU_GRAD: return launch<EGN_MLP_EPI_RELU_GRAD>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    case EGN_MLP_EPI_BIAS_GELU: return launch<EGN_MLP_EPI_BIAS_GELU>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    case EGN_MLP_EPI_GELU_GRAD: return launch<EGN_MLP_EPI_GELU_GRAD>(ta, tb, m, n, kb_per, kb, splits, bias, aux, out, err_dev, st);
    default: return fail(EGN_E_INVALID_ARG, "unknown epilogue %d", epilogue);
  }
}
