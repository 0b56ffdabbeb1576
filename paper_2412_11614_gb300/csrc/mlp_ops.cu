// mlp_ops.cu -- the FP32 / BF16 kernels around the surrogate's tensor-core
// GEMMs: split-k reduction, transpose, column sums, output layer with loss and
// gradients, Adam.  All sums are in a fixed order (results are reproducible).
#include <cuda_bf16.h>

#include "../../include/egn_mlp.h"
#include "link.h"

using namespace egn_host;

namespace {

__global__ void reduce_splits_kernel(const float* __restrict__ part, int splits, long long count, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * count + i];
    out[i] = s;
  }
}

// 32 x 32 tiles through shared memory (padded against bank conflicts).
__global__ void transpose_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols, int rows_pad,
                                 __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    t[i][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * cols + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows_pad) out[(size_t)c * rows_pad + r] = t[threadIdx.x][i];
  }
}

// One CTA per 32 columns; 8 warps stride over rows; fixed-order tree at the end.
__global__ void colsum_kernel(const __nv_bfloat16* __restrict__ in, int rows, int cols, float* __restrict__ out) {
  __shared__ float s[8][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float a = 0.0f;
  if (c < cols)
    for (int r = threadIdx.y; r < rows; r += 8) a += __bfloat162float(in[(size_t)r * cols + c]);
  s[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    float t = ((s[0][threadIdx.x] + s[1][threadIdx.x]) + (s[2][threadIdx.x] + s[3][threadIdx.x])) +
              ((s[4][threadIdx.x] + s[5][threadIdx.x]) + (s[6][threadIdx.x] + s[7][threadIdx.x]));
    out[c] = t;
  }
}

// Output layer: one warp per row.  y = h . w + b.
__global__ void head_fwd_kernel(const __nv_bfloat16* __restrict__ h, int rows, int hid, const float* __restrict__ w,
                                const float* __restrict__ b, float* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  float a = 0.0f;
  for (int j = lane; j < hid; j += 32) a = fmaf(__bfloat162float(h[(size_t)warp * hid + j]), w[j], a);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) y[warp] = a + b[0];
}

// Loss and dL/dy in one CTA (fixed order): g[r] = 2 mask[r] (y[r] - t[r]) / sum(mask).
__global__ void loss_kernel(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask,
                            int rows, float* __restrict__ g, float* __restrict__ loss) {
  __shared__ float s1[256], s2[256];
  float a = 0.0f, m = 0.0f;
  for (int r = threadIdx.x; r < rows; r += 256) {
    const float d = y[r] - t[r];
    a = fmaf(mask[r] * d, d, a);
    m += mask[r];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  const float msum = s2[0] > 0.0f ? s2[0] : 1.0f;
  if (threadIdx.x == 0) loss[0] = s1[0] / msum;
  for (int r = threadIdx.x; r < rows; r += 256) g[r] = 2.0f * mask[r] * (y[r] - t[r]) / msum;
}

// dh[r][j] = g[r] w[j] where h[r][j] > 0.
__global__ void head_bwd_kernel(const __nv_bfloat16* __restrict__ h, int rows, int hid, const float* __restrict__ w,
                                const float* __restrict__ g, __nv_bfloat16* __restrict__ dh) {
  const long long n = (long long)rows * hid;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / hid), j = (int)(i - (long long)r * hid);
    dh[i] = __float2bfloat16_rn(__bfloat162float(h[i]) > 0.0f ? g[r] * w[j] : 0.0f);
  }
}

// dw[j] = sum_r g[r] h[r][j] (one CTA per 32 columns, like colsum); db = sum_r g[r].
__global__ void head_wgrad_kernel(const __nv_bfloat16* __restrict__ h, int rows, int hid, const float* __restrict__ g,
                                  float* __restrict__ dw, float* __restrict__ db) {
  __shared__ float s[8][32];
  const int c = blockIdx.x * 32 + threadIdx.x;
  const bool bias_col = (blockIdx.x == gridDim.x - 1) && threadIdx.x == 31 && db;  // spare lane computes db
  float a = 0.0f, gb = 0.0f;
  for (int r = threadIdx.y; r < rows; r += 8) {
    if (c < hid) a = fmaf(g[r], __bfloat162float(h[(size_t)r * hid + c]), a);
    gb += g[r];
  }
  s[threadIdx.y][threadIdx.x] = c < hid ? a : gb;
  __syncthreads();
  if (threadIdx.y == 0) {
    const float t = ((s[0][threadIdx.x] + s[1][threadIdx.x]) + (s[2][threadIdx.x] + s[3][threadIdx.x])) +
                    ((s[4][threadIdx.x] + s[5][threadIdx.x]) + (s[6][threadIdx.x] + s[7][threadIdx.x]));
    if (c < hid) dw[c] = t;
    else if (bias_col) db[0] = t;
  }
}

// Multi-output layer: y[r][j] = acc[r][j] + b[j] for the n_out live columns.
__global__ void outputs_fwd_kernel(const float* __restrict__ acc, int rows, int n_out, int n_pad,
                                   const float* __restrict__ b, float* __restrict__ y) {
  const long long n = (long long)rows * n_out;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n_out), j = (int)(i - (long long)r * n_out);
    y[i] = acc[(size_t)r * n_pad + j] + b[j];
  }
}

// Loss, dL/dy (BF16, zero-padded to [rows_pad][n_pad]) and the bias gradient in
// one CTA of 1024 threads, every sum in a fixed order:
// L = sum_r mask[r] sum_j (y - t)^2 / (n_out sum_r mask[r]), dL/dy = 2 mask[r] (y - t) / (n_out sum mask).
__global__ void __launch_bounds__(1024) outputs_loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                            const float* __restrict__ mask, int rows, int rows_pad,
                                                            int n_out, int n_pad, float* __restrict__ loss,
                                                            __nv_bfloat16* __restrict__ g, float* __restrict__ db) {
  __shared__ float s1[1024], s2[1024];
  const int tid = threadIdx.x;
  float a = 0.0f, m = 0.0f;
  const long long n = (long long)rows * n_out;
  for (long long i = tid; i < n; i += 1024) {
    const int r = (int)(i / n_out);
    const float d = y[i] - t[i];
    a = fmaf(mask[r] * d, d, a);
  }
  for (int r = tid; r < rows; r += 1024) m += mask[r];
  s1[tid] = a;
  s2[tid] = m;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o) {
      s1[tid] += s1[tid + o];
      s2[tid] += s2[tid + o];
    }
    __syncthreads();
  }
  const float msum = s2[0] > 0.0f ? s2[0] : 1.0f;
  const float scale = 2.0f / ((float)n_out * msum);
  if (tid == 0) loss[0] = s1[0] / ((float)n_out * msum);
  const long long np = (long long)rows_pad * n_pad;
  for (long long i = tid; i < np; i += 1024) {
    const int r = (int)(i / n_pad), j = (int)(i - (long long)r * n_pad);
    float v = 0.0f;
    if (r < rows && j < n_out) {
      const size_t k = (size_t)r * n_out + j;
      v = scale * mask[r] * (y[k] - t[k]);
    }
    g[i] = __float2bfloat16_rn(v);
  }
  for (int j = tid; j < n_out; j += 1024) {  // column j over the rows in order
    float c = 0.0f;
    for (int r = 0; r < rows; ++r) {
      const size_t k = (size_t)r * n_out + j;
      c = fmaf(scale * mask[r], y[k] - t[k], c);
    }
    db[j] = c;
  }
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wt, int rows,
                            int cols) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    const __nv_bfloat16 q = __float2bfloat16_rn(wi);
    if (wb) wb[i] = q;
    if (wt) {
      const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
      wt[(size_t)c * rows + r] = q;
    }
  }
}

__global__ void cast_kernel(const float* __restrict__ in, long long n, __nv_bfloat16* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

unsigned grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

}  // namespace

extern "C" {

egn_status egn_mlp_reduce_splits(const float* part, int splits, long long count, float* out, void* stream) {
  if (!part || !out || splits < 1 || count < 0) return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (count == 0) return EGN_OK;
  reduce_splits_kernel<<<grid_for(count, 256), 256, 0, (cudaStream_t)stream>>>(part, splits, count, out);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_transpose(const void* in, int rows, int cols, int rows_pad, void* out, void* stream) {
  if (!in || !out || rows < 0 || cols < 1 || rows_pad < rows) return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (rows_pad == 0) return EGN_OK;
  dim3 grid((rows_pad + 31) / 32, (cols + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)in, rows, cols, rows_pad,
                                                                    (__nv_bfloat16*)out);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_colsum(const void* in, int rows, int cols, float* out, void* stream) {
  if (!in || !out || rows < 0 || cols < 1) return fail(EGN_E_INVALID_ARG, "bad arguments");
  colsum_kernel<<<(cols + 31) / 32, dim3(32, 8), 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)in, rows, cols, out);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_head(const void* h, int rows, int hid, const float* w, const float* b, float* y,
                        const float* target, const float* mask, float* loss, float* g, void* dh, float* dw, float* db,
                        void* stream) {
  if (!h || !w || !b || !y || rows < 1 || hid < 1 || hid % 32) return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (target && (!mask || !loss || !g || !dh || !dw || !db)) return fail(EGN_E_INVALID_ARG, "training needs every output");
  cudaStream_t st = (cudaStream_t)stream;
  const __nv_bfloat16* hb = (const __nv_bfloat16*)h;
  head_fwd_kernel<<<(rows * 32 + 255) / 256, 256, 0, st>>>(hb, rows, hid, w, b, y);
  EGN_CUDA(cudaGetLastError());
  if (!target) return EGN_OK;
  loss_kernel<<<1, 256, 0, st>>>(y, target, mask, rows, g, loss);
  EGN_CUDA(cudaGetLastError());
  head_bwd_kernel<<<grid_for((long long)rows * hid, 256), 256, 0, st>>>(hb, rows, hid, w, g, (__nv_bfloat16*)dh);
  EGN_CUDA(cudaGetLastError());
  head_wgrad_kernel<<<hid / 32 + 1, dim3(32, 8), 0, st>>>(hb, rows, hid, g, dw, db);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_outputs(const float* acc, int rows, int rows_pad, int n_out, int n_pad, const float* b, float* y,
                           const float* target, const float* mask, float* loss, void* g, float* db, void* stream) {
  if (!acc || !b || !y || rows < 1 || n_out < 1 || n_pad < n_out || rows_pad < rows)
    return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (target && (!mask || !loss || !g || !db)) return fail(EGN_E_INVALID_ARG, "training needs every output");
  cudaStream_t st = (cudaStream_t)stream;
  outputs_fwd_kernel<<<grid_for((long long)rows * n_out, 256), 256, 0, st>>>(acc, rows, n_out, n_pad, b, y);
  EGN_CUDA(cudaGetLastError());
  if (!target) return EGN_OK;
  outputs_loss_kernel<<<1, 1024, 0, st>>>(y, target, mask, rows, rows_pad, n_out, n_pad, loss, (__nv_bfloat16*)g, db);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float beta1, float beta2,
                        float eps, int t, void* w_bf16, void* wt_bf16, int rows, int cols, void* stream) {
  if (!w || !g || !m || !v || n < 1 || t < 1) return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (wt_bf16 && ((long long)rows * cols != n || rows < 1)) return fail(EGN_E_INVALID_ARG, "rows x cols != n");
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  adam_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                                                   (__nv_bfloat16*)w_bf16, (__nv_bfloat16*)wt_bf16,
                                                                   rows, cols);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

egn_status egn_mlp_cast(const float* in, long long n, void* out, void* stream) {
  if (!in || !out || n < 0) return fail(EGN_E_INVALID_ARG, "bad arguments");
  if (n == 0) return EGN_OK;
  cast_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(in, n, (__nv_bfloat16*)out);
  EGN_CUDA(cudaGetLastError());
  return EGN_OK;
}

}  // extern "C"
