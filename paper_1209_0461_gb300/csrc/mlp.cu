// Learned response surrogate: a 3-layer perceptron (n_in -> 128 -> 128 -> 1,
// tanh) with BF16 weight matrices, FP32 biases and FP32 accumulation, and its
// training kernels (mean-squared-error gradient by the chain rule, Adam).  It
// maps per-bin features of a kick to ln R_b (R_b = P_nu^{1/2} / P_cdm^{1/2} of
// Eq. P-final); the paper has no learned part.
//
// Layout of the flat parameter vector (FP32 master copy):
//   W1 [128][n_in], b1 [128], W2 [128][128], b2 [128], w3 [128], b3 [1]
//
// Kernels (one CTA of 128 threads per SM, persistent over tiles of 32
// samples; thread j owns hidden unit j of both layers):
//   k_mlp_forward   y = y_mu + y_sigma * out(x)                 (inference)
//   k_mlp_backward  per-CTA partial gradients and loss, fixed tile order
//   k_mlp_reduce    sum of the CTA partials in CTA order (deterministic)
//   k_mlp_adam      Adam on the master copy, then the BF16 weight copies
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "nupm_internal.h"

namespace nupm {
namespace {

constexpr int kW = 128;        // hidden width
constexpr int kMaxIn = 16;     // input features (<=)
constexpr int kTS = 32;        // samples per tile
constexpr int kHP = 36;        // padded row of the [unit][sample] tiles (16-byte rows)
constexpr int kWP = 129;       // padded row of the 128x128 shared matrices

// Shared-memory layout (floats) of the two kernels.
struct MlpSmem {
  static constexpr int W2 = 0;                        // W2s[k][j] = W2[j][k], rows of kWP
  static constexpr int DW2 = W2 + kW * kWP;            // dW2 partial, same layout
  static constexpr int H1 = DW2 + kW * kWP;            // h1T[k][s], rows of kHP
  static constexpr int DZ2 = H1 + kW * kHP;            // dz2T[j][s]
  static constexpr int XH = DZ2 + kW * kHP;            // xh[s][i], rows of kMaxIn
  static constexpr int OUT = XH + kTS * kMaxIn;        // out / dout per sample
  static constexpr int RED = OUT + kTS;                // [4 warps][kTS] reduction
  static constexpr int TOTAL = RED + 4 * kTS;
  static constexpr size_t BYTES = (size_t)TOTAL * sizeof(float);
};

struct MlpArgs {
  int n_in;
  int64_t n;                          // samples
  const float* X;                     // [n][n_in] raw features
  const float* Y;                     // [n] raw targets (ln R), backward only
  float* out;                         // [n] forward output (ln R)
  const __nv_bfloat16* W1;            // [128][n_in]
  const float* b1;
  const __nv_bfloat16* W2;            // [128][128]
  const float* b2;
  const __nv_bfloat16* w3;            // [128]
  const float* b3;
  const float* mu;                    // [n_in]
  const float* sig;                   // [n_in]
  float y_mu, y_sig;
  float* partial;                     // [gridDim][P + 1] (backward)
  int64_t P;                          // parameter count
};

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }

// Forward pass of one tile of kTS samples (rows s0 .. s0 + kTS - 1; rows past
// n are zero inputs whose results are ignored).  Leaves h1T, this thread's
// h2[s] (unit j) and out[s] (normalised) in shared memory / registers.
__device__ __forceinline__ void tile_forward(const MlpArgs& A, float* sm, int64_t s0, float (&h2)[kTS]) {
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  float* xh = sm + MlpSmem::XH;
  float* h1T = sm + MlpSmem::H1;
  const float* W2s = sm + MlpSmem::W2;
  float* outs = sm + MlpSmem::OUT;
  float* red = sm + MlpSmem::RED;
  for (int idx = j; idx < kTS * kMaxIn; idx += kW) {   // unused columns and rows past n: 0
    const int s = idx / kMaxIn, i = idx - s * kMaxIn;
    const int64_t row = s0 + s;
    xh[idx] = (i < A.n_in && row < A.n) ? (A.X[row * A.n_in + i] - A.mu[i]) / A.sig[i] : 0.0f;
  }
  __syncthreads();
  // layer 1: unit j for every sample of the tile
  {
    float w[kMaxIn];
#pragma unroll
    for (int i = 0; i < kMaxIn; ++i) w[i] = i < A.n_in ? bf(A.W1[j * A.n_in + i]) : 0.0f;
    const float b = A.b1[j];
#pragma unroll 4
    for (int s = 0; s < kTS; ++s) {
      float acc = b;
#pragma unroll
      for (int i = 0; i < kMaxIn; ++i) acc = fmaf(w[i], xh[s * kMaxIn + i], acc);
      h1T[j * kHP + s] = tanhf(acc);
    }
  }
  __syncthreads();
  // layer 2: h2[s] = tanh(b2[j] + sum_k W2[j][k] h1[s][k])
  {
    const float b = A.b2[j];
#pragma unroll
    for (int s = 0; s < kTS; ++s) h2[s] = b;
#pragma unroll 2
    for (int k = 0; k < kW; ++k) {
      const float w = W2s[k * kWP + j];
      const float4* hk = reinterpret_cast<const float4*>(h1T + k * kHP);
#pragma unroll
      for (int q = 0; q < kTS / 4; ++q) {
        const float4 hv = hk[q];
        h2[4 * q + 0] = fmaf(w, hv.x, h2[4 * q + 0]);
        h2[4 * q + 1] = fmaf(w, hv.y, h2[4 * q + 1]);
        h2[4 * q + 2] = fmaf(w, hv.z, h2[4 * q + 2]);
        h2[4 * q + 3] = fmaf(w, hv.w, h2[4 * q + 3]);
      }
    }
#pragma unroll
    for (int s = 0; s < kTS; ++s) h2[s] = tanhf(h2[s]);
  }
  // layer 3: out[s] = b3 + sum_j w3[j] h2[s][j], fixed reduction tree
  const float w3j = bf(A.w3[j]);
#pragma unroll
  for (int s = 0; s < kTS; ++s) {
    float v = w3j * h2[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp * kTS + s] = v;
  }
  __syncthreads();
  if (j < kTS) outs[j] = A.b3[0] + ((red[j] + red[kTS + j]) + (red[2 * kTS + j] + red[3 * kTS + j]));
  __syncthreads();
}

__device__ __forceinline__ void load_w2(const MlpArgs& A, float* sm) {
  float* W2s = sm + MlpSmem::W2;
  for (int idx = threadIdx.x; idx < kW * kW; idx += kW) {
    const int jj = idx / kW, k = idx - jj * kW;          // W2[jj][k]
    W2s[k * kWP + jj] = bf(A.W2[idx]);
  }
}

__global__ void __launch_bounds__(kW, 1) k_mlp_forward(MlpArgs A) {
  extern __shared__ __align__(16) float sm[];
  load_w2(A, sm);
  __syncthreads();
  float h2[kTS];
  const int64_t tiles = (A.n + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    tile_forward(A, sm, s0, h2);
    if (threadIdx.x < kTS && s0 + threadIdx.x < A.n)
      A.out[s0 + threadIdx.x] = A.y_mu + A.y_sig * sm[MlpSmem::OUT + threadIdx.x];
    __syncthreads();
  }
}

// Partial gradient of L = (1/n) sum (out - (Y - y_mu)/y_sig)^2 over the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... (in that order), written to
// partial[blockIdx.x][0..P) in the flat parameter layout, the partial loss
// at [P].
__global__ void __launch_bounds__(kW, 1) k_mlp_backward(MlpArgs A) {
  extern __shared__ __align__(16) float sm[];
  const int j = threadIdx.x;
  float* W2s = sm + MlpSmem::W2;
  float* dW2s = sm + MlpSmem::DW2;
  float* h1T = sm + MlpSmem::H1;
  float* dz2T = sm + MlpSmem::DZ2;
  float* xh = sm + MlpSmem::XH;
  float* outs = sm + MlpSmem::OUT;
  load_w2(A, sm);
  for (int idx = j; idx < kW * kWP; idx += kW) dW2s[idx] = 0.0f;
  float dW1[kMaxIn];
#pragma unroll
  for (int i = 0; i < kMaxIn; ++i) dW1[i] = 0.0f;
  float db1 = 0.0f, db2 = 0.0f, dw3 = 0.0f, db3 = 0.0f, loss = 0.0f;
  const float inv_n = 1.0f / (float)A.n;
  const float w3j = bf(A.w3[j]);
  __syncthreads();
  float h2[kTS];
  const int64_t tiles = (A.n + kTS - 1) / kTS;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t s0 = t * kTS;
    tile_forward(A, sm, s0, h2);
    // dL/dout per sample (zero past n)
    if (j < kTS) {
      const int64_t row = s0 + j;
      float d = 0.0f;
      if (row < A.n) {
        const float r = outs[j] - (A.Y[row] - A.y_mu) / A.y_sig;
        d = 2.0f * r * inv_n;
        outs[j] = r * r;       // squared residual (read by thread 0 below)
      } else {
        outs[j] = 0.0f;
      }
      sm[MlpSmem::RED + j] = d;
    }
    __syncthreads();
    if (j == 0)
      for (int s = 0; s < kTS; ++s) loss += outs[s];
    const float* dout = sm + MlpSmem::RED;
    // layer 3 and the pre-activation gradient of layer 2 (unit j)
    float dz2[kTS];
#pragma unroll
    for (int s = 0; s < kTS; ++s) {
      const float d = dout[s];
      dw3 = fmaf(d, h2[s], dw3);
      if (j == 0) db3 += d;
      dz2[s] = d * w3j * (1.0f - h2[s] * h2[s]);
      db2 += dz2[s];
      dz2T[j * kHP + s] = dz2[s];
    }
    // dW2[j][k] += sum_s dz2[s] h1[s][k]
#pragma unroll 2
    for (int k = 0; k < kW; ++k) {
      const float4* hk = reinterpret_cast<const float4*>(h1T + k * kHP);
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < kTS / 4; ++q) {
        const float4 hv = hk[q];
        acc = fmaf(dz2[4 * q + 0], hv.x, acc);
        acc = fmaf(dz2[4 * q + 1], hv.y, acc);
        acc = fmaf(dz2[4 * q + 2], hv.z, acc);
        acc = fmaf(dz2[4 * q + 3], hv.w, acc);
      }
      dW2s[k * kWP + j] += acc;
    }
    __syncthreads();
    // thread j now acts as layer-1 unit k = j: dh1[s] = sum_jj W2[jj][k] dz2[s][jj]
    {
      const int k = j;
      float dh[kTS];
#pragma unroll
      for (int s = 0; s < kTS; ++s) dh[s] = 0.0f;
#pragma unroll 2
      for (int jj = 0; jj < kW; ++jj) {
        const float w = W2s[k * kWP + jj];
        const float4* dz = reinterpret_cast<const float4*>(dz2T + jj * kHP);
#pragma unroll
        for (int q = 0; q < kTS / 4; ++q) {
          const float4 dv = dz[q];
          dh[4 * q + 0] = fmaf(w, dv.x, dh[4 * q + 0]);
          dh[4 * q + 1] = fmaf(w, dv.y, dh[4 * q + 1]);
          dh[4 * q + 2] = fmaf(w, dv.z, dh[4 * q + 2]);
          dh[4 * q + 3] = fmaf(w, dv.w, dh[4 * q + 3]);
        }
      }
#pragma unroll
      for (int s = 0; s < kTS; ++s) {
        const float h = h1T[k * kHP + s];
        const float dz1 = dh[s] * (1.0f - h * h);
        db1 += dz1;
#pragma unroll
        for (int i = 0; i < kMaxIn; ++i) dW1[i] = fmaf(dz1, xh[s * kMaxIn + i], dW1[i]);
      }
    }
    __syncthreads();   // h1T, dz2T, xh and outs are rewritten by the next tile
  }
  // write this CTA's partials in the flat layout
  float* out = A.partial + (int64_t)blockIdx.x * (A.P + 1);
  const int n_in = A.n_in;
  const int oW1 = 0, ob1 = kW * n_in, oW2 = ob1 + kW, ob2 = oW2 + kW * kW, ow3 = ob2 + kW, ob3 = ow3 + kW;
  for (int i = 0; i < n_in; ++i) out[oW1 + j * n_in + i] = dW1[i];
  out[ob1 + j] = db1;
  for (int idx = j; idx < kW * kW; idx += kW) {
    const int jj = idx / kW, k = idx - jj * kW;
    out[oW2 + idx] = dW2s[k * kWP + jj];
  }
  out[ob2 + j] = db2;
  out[ow3 + j] = dw3;
  if (j == 0) {
    out[ob3] = db3;
    out[A.P] = loss * inv_n;
  }
}

// grad[p] = sum over CTAs in order; loss = the same sum at index P.
__global__ void k_mlp_reduce(const float* __restrict__ partial, int nblk, int64_t P1, float* __restrict__ grad) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P1) return;
  float acc = 0.0f;
  for (int b = 0; b < nblk; ++b) acc += partial[(int64_t)b * P1 + p];
  grad[p] = acc;
}

// Adam (Kingma & Ba 2015) on the FP32 master copy, then the BF16 copies of
// the weight matrices.  bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int64_t P, float lr, float b1, float b2, float eps, float bc1,
                           float bc2, __nv_bfloat16* __restrict__ wbf, int n_in) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float th = theta[p] - lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
  theta[p] = th;
  const int64_t ob1 = (int64_t)kW * n_in, oW2 = ob1 + kW, ob2 = oW2 + (int64_t)kW * kW, ow3 = ob2 + kW;
  if (p < ob1) wbf[p] = __float2bfloat16_rn(th);                                // W1
  else if (p >= oW2 && p < ob2) wbf[ob1 + (p - oW2)] = __float2bfloat16_rn(th);   // W2
  else if (p >= ow3 && p < ow3 + kW) wbf[ob1 + kW * kW + (p - ow3)] = __float2bfloat16_rn(th);   // w3
}

// BF16 copies of the weight matrices from the master copy.
__global__ void k_mlp_to_bf16(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf, int n_in) {
  const int64_t ob1 = (int64_t)kW * n_in, oW2 = ob1 + kW, ob2 = oW2 + (int64_t)kW * kW, ow3 = ob2 + kW;
  const int64_t nb = ob1 + (int64_t)kW * kW + kW;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb) return;
  int64_t p;
  if (q < ob1) p = q;
  else if (q < ob1 + kW * kW) p = oW2 + (q - ob1);
  else p = ow3 + (q - ob1 - kW * kW);
  wbf[q] = __float2bfloat16_rn(theta[p]);
}

}  // namespace
}  // namespace nupm

using namespace nupm;

struct pm_mlp {
  int n_in = 0;
  int64_t P = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 152;
  float* theta = nullptr;          // [P] master
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;           // [P + 1] (loss at P)
  float* partial = nullptr;        // [nblk][P + 1]
  __nv_bfloat16* wbf = nullptr;    // W1 | W2 | w3
  float* norm = nullptr;           // mu [n_in] | sigma [n_in]
  float y_mu = 0.0f, y_sig = 1.0f;
  int64_t step = 0;
  int nblk = 0;
};

namespace {

int mlp_check(cudaError_t e) { return e == cudaSuccess ? PM_OK : PM_ERR_CUDA; }

MlpArgs mlp_args(const pm_mlp* m, const float* X, const float* Y, int64_t n, float* out) {
  MlpArgs A{};
  A.n_in = m->n_in;
  A.n = n;
  A.X = X;
  A.Y = Y;
  A.out = out;
  A.W1 = m->wbf;
  A.b1 = m->theta + (int64_t)kW * m->n_in;
  A.W2 = m->wbf + (int64_t)kW * m->n_in;
  A.b2 = m->theta + (int64_t)kW * m->n_in + kW + (int64_t)kW * kW;
  A.w3 = m->wbf + (int64_t)kW * m->n_in + (int64_t)kW * kW;
  A.b3 = m->theta + m->P - 1;
  A.mu = m->norm;
  A.sig = m->norm + m->n_in;
  A.y_mu = m->y_mu;
  A.y_sig = m->y_sig;
  A.partial = m->partial;
  A.P = m->P;
  return A;
}

int mlp_grad_launch(pm_mlp* m, const float* X, const float* Y, int64_t n) {
  MlpArgs A = mlp_args(m, X, Y, n, nullptr);
  const int64_t tiles = (n + kTS - 1) / kTS;
  const int grid = (int)(tiles < m->nblk ? tiles : m->nblk);
  k_mlp_backward<<<grid, kW, MlpSmem::BYTES, m->stream>>>(A);
  k_mlp_reduce<<<(unsigned)((m->P + 1 + 255) / 256), 256, 0, m->stream>>>(m->partial, grid, m->P + 1, m->grad);
  return mlp_check(cudaGetLastError());
}

}  // namespace

namespace nupm {

int mlp_inputs(const pm_mlp* m) { return m ? m->n_in : 0; }

int mlp_forward_on(pm_mlp* m, const float* X, int64_t n, float* y, cudaStream_t s) {
  if (!m || n < 0 || (n > 0 && (!X || !y))) return PM_ERR_INVALID;
  if (n == 0) return PM_OK;
  MlpArgs A = mlp_args(m, X, nullptr, n, y);
  const int64_t tiles = (n + kTS - 1) / kTS;
  const int grid = (int)(tiles < m->sm_count ? tiles : m->sm_count);
  k_mlp_forward<<<grid, kW, MlpSmem::BYTES, s>>>(A);
  return mlp_check(cudaGetLastError());
}

}  // namespace nupm

extern "C" {

int pm_mlp_create(int32_t n_in, int32_t width, void* cuda_stream, pm_mlp** out) {
  if (!out) return PM_ERR_INVALID;
  *out = nullptr;
  if (n_in < 1 || n_in > kMaxIn || width != kW) return PM_ERR_INVALID;
  pm_mlp* m = new (std::nothrow) pm_mlp;
  if (!m) return PM_ERR_ALLOC;
  m->n_in = n_in;
  m->P = (int64_t)kW * n_in + kW + (int64_t)kW * kW + kW + kW + 1;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
  m->nblk = m->sm_count;
  const size_t pb = (size_t)m->P * sizeof(float);
  bool ok = cudaMalloc(&m->theta, pb) == cudaSuccess && cudaMalloc(&m->m, pb) == cudaSuccess &&
            cudaMalloc(&m->v, pb) == cudaSuccess && cudaMalloc(&m->grad, pb + sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->partial, (size_t)m->nblk * (m->P + 1) * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->wbf, (size_t)((int64_t)kW * n_in + (int64_t)kW * kW + kW) * sizeof(__nv_bfloat16)) ==
                cudaSuccess &&
            cudaMalloc(&m->norm, 2 * (size_t)n_in * sizeof(float)) == cudaSuccess;
  if (ok) {
    ok = cudaMemsetAsync(m->theta, 0, pb, m->stream) == cudaSuccess &&
         cudaMemsetAsync(m->m, 0, pb, m->stream) == cudaSuccess &&
         cudaMemsetAsync(m->v, 0, pb, m->stream) == cudaSuccess;
    std::vector<float> nrm(2 * n_in, 0.0f);
    for (int i = 0; i < n_in; ++i) nrm[n_in + i] = 1.0f;
    ok = ok && cudaMemcpy(m->norm, nrm.data(), nrm.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)MlpSmem::BYTES) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)MlpSmem::BYTES) == cudaSuccess;
  }
  if (ok) {
    k_mlp_to_bf16<<<(unsigned)((kW * n_in + kW * kW + kW + 255) / 256), 256, 0, m->stream>>>(m->theta, m->wbf, n_in);
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (!ok) {
    pm_mlp_free(m);
    return PM_ERR_ALLOC;
  }
  *out = m;
  return PM_OK;
}

void pm_mlp_free(pm_mlp* m) {
  if (!m) return;
  void* ptrs[] = {m->theta, m->m, m->v, m->grad, m->partial, m->wbf, m->norm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

int64_t pm_mlp_param_count(const pm_mlp* m) { return m ? m->P : 0; }

int pm_mlp_set_params(pm_mlp* m, const float* host_params) {
  if (!m || !host_params) return PM_ERR_INVALID;
  const size_t pb = (size_t)m->P * sizeof(float);
  if (cudaMemcpyAsync(m->theta, host_params, pb, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
    return PM_ERR_CUDA;
  if (cudaMemsetAsync(m->m, 0, pb, m->stream) != cudaSuccess || cudaMemsetAsync(m->v, 0, pb, m->stream) != cudaSuccess)
    return PM_ERR_CUDA;
  m->step = 0;
  k_mlp_to_bf16<<<(unsigned)((kW * m->n_in + kW * kW + kW + 255) / 256), 256, 0, m->stream>>>(m->theta, m->wbf,
                                                                                              m->n_in);
  if (cudaGetLastError() != cudaSuccess) return PM_ERR_CUDA;
  return mlp_check(cudaStreamSynchronize(m->stream));
}

int pm_mlp_get_params(const pm_mlp* m, float* host_params) {
  if (!m || !host_params) return PM_ERR_INVALID;
  if (cudaMemcpyAsync(host_params, m->theta, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToHost, m->stream) !=
      cudaSuccess)
    return PM_ERR_CUDA;
  return mlp_check(cudaStreamSynchronize(m->stream));
}

int pm_mlp_set_norm(pm_mlp* m, const float* mu, const float* sigma, float y_mu, float y_sigma) {
  if (!m || !mu || !sigma) return PM_ERR_INVALID;
  for (int i = 0; i < m->n_in; ++i)
    if (!(sigma[i] > 0.0f)) return PM_ERR_INVALID;
  if (!(y_sigma > 0.0f)) return PM_ERR_INVALID;
  std::vector<float> nrm(2 * m->n_in);
  memcpy(nrm.data(), mu, m->n_in * sizeof(float));
  memcpy(nrm.data() + m->n_in, sigma, m->n_in * sizeof(float));
  if (cudaMemcpy(m->norm, nrm.data(), nrm.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return PM_ERR_CUDA;
  m->y_mu = y_mu;
  m->y_sig = y_sigma;
  return PM_OK;
}

int pm_mlp_forward(pm_mlp* m, const float* X, int64_t n, float* y) {
  return m ? mlp_forward_on(m, X, n, y, m->stream) : PM_ERR_INVALID;
}

int pm_mlp_grad(pm_mlp* m, const float* X, const float* y, int64_t n, float* grad, float* loss) {
  if (!m || n <= 0 || !X || !y) return PM_ERR_INVALID;
  int rc = mlp_grad_launch(m, X, y, n);
  if (rc != PM_OK) return rc;
  if (grad && cudaMemcpyAsync(grad, m->grad, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToDevice, m->stream) !=
                  cudaSuccess)
    return PM_ERR_CUDA;
  if (loss && cudaMemcpyAsync(loss, m->grad + m->P, sizeof(float), cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
    return PM_ERR_CUDA;
  return PM_OK;
}

int pm_mlp_train_step(pm_mlp* m, const float* X, const float* y, int64_t n, float lr, float* loss) {
  if (!m || n <= 0 || !X || !y || !(lr > 0.0f)) return PM_ERR_INVALID;
  int rc = mlp_grad_launch(m, X, y, n);
  if (rc != PM_OK) return rc;
  m->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - pow(b1, (double)m->step)), bc2 = (float)(1.0 - pow(b2, (double)m->step));
  k_mlp_adam<<<(unsigned)((m->P + 255) / 256), 256, 0, m->stream>>>(m->theta, m->grad, m->m, m->v, m->P, lr, (float)b1,
                                                                  (float)b2, 1e-8f, bc1, bc2, m->wbf, m->n_in);
  if (loss && cudaMemcpyAsync(loss, m->grad + m->P, sizeof(float), cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
    return PM_ERR_CUDA;
  return mlp_check(cudaGetLastError());
}

}  // extern "C"
