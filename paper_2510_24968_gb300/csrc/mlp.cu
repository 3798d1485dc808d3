// Small MLP for the learned initial density (three linear layers, SiLU, width
// 256): forward, backward and Adam, all in this file's kernels.
//
//   z1 = x W1 + b1, h1 = silu(z1), z2 = h1 W2 + b2, h2 = silu(z2), y = h2 W3 + b3
//   loss = sum(mask (y - t)^2) / sum(mask)
// Weights are kept in FP32 (master, Adam state) with BF16 copies; the GEMMs run
// on the fifth-generation tensor cores (tcgen05.mma, BF16 x BF16 -> FP32
// accumulation in tensor memory, tc_gemm.cuh).  A plain FP32 GEMM path (no
// BF16 rounding) serves the gradient check.
// silu(z) = z s(z), s = logistic; silu'(z) = s(z) (1 + z (1 - s(z))).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fsim_internal.h"
#include "tc_gemm.cuh"

struct fsim_mlp {
  int nin = 0, width = 0, nout = 0;
  size_t np = 0;
  float* p = nullptr;  // W1 [nin x w] | b1 [w] | W2 [w x w] | b2 [w] | W3 [w x nout] | b3 [nout]
  float* g = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* pb = nullptr;
  int maxb = 0;
  float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *y = nullptr;
  float *dy = nullptr, *d1 = nullptr, *d2 = nullptr;
  float* scal = nullptr;  // [0] loss numerator, [1] mask sum
  int* tc_err = nullptr;  // set by a tensor-core GEMM whose MMAs did not complete
  long step = 0;
};

namespace fsim {
namespace {

struct Off {
  size_t W1, b1, W2, b2, W3, b3, n;
};
Off offsets(int nin, int w, int nout) {
  Off o;
  o.W1 = 0;
  o.b1 = o.W1 + (size_t)nin * w;
  o.W2 = o.b1 + w;
  o.b2 = o.W2 + (size_t)w * w;
  o.W3 = o.b2 + w;
  o.b3 = o.W3 + (size_t)w * nout;
  o.n = o.b3 + nout;
  return o;
}

// C[M x N] = op(A) op(B) (+ bias[N]), op(A) M x K, op(B) K x N, all row-major
// FP32 in memory; tA: A stored K x M; tB: B stored N x K.  This kernel is the
// plain FP32 path (FMAs, no BF16 rounding) of the gradient check; BF16 GEMMs
// run on the tensor cores (tc_gemm_kernel).
constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ float ldA(const float* A, int M, int K, bool tA, int r, int k) {
  if (r >= M || k >= K) return 0.0f;
  return tA ? A[(size_t)k * M + r] : A[(size_t)r * K + k];
}
__device__ __forceinline__ float ldB(const float* B, int K, int N, bool tB, int k, int c) {
  if (k >= K || c >= N) return 0.0f;
  return tB ? B[(size_t)c * K + k] : B[(size_t)k * N + c];
}

__global__ void __launch_bounds__(128) gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                   float* __restrict__ C, const float* __restrict__ bias, int M,
                                                   int N, int K, int tA, int tB) {
  __shared__ float Af[TM][TK + 1];
  __shared__ float Bf[TK][TN + 1];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tid = threadIdx.x;
  // thread owns rows (tid / 4) * 2 .. +1 and columns (tid % 4) * 16 .. +15 of the tile (32 outputs)
  const int rr = (tid >> 2) * 2, cc = (tid & 3) * 16;
  float accf[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) accf[r] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int x = tid; x < TM * TK; x += 128) {
      const int r = x / TK, k = x % TK;
      Af[r][k] = ldA(A, M, K, tA, m0 + r, k0 + k);
    }
    for (int x = tid; x < TK * TN; x += 128) {
      const int k = x / TN, c = x % TN;
      Bf[k][c] = ldB(B, K, N, tB, k0 + k, n0 + c);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) accf[i * 16 + j] = fmaf(Af[rr + i][k], Bf[k][cc + j], accf[i * 16 + j]);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int r = m0 + rr + i, c = n0 + cc + j;
      if (r < M && c < N) C[(size_t)r * N + c] = accf[i * 16 + j] + (bias ? bias[c] : 0.0f);
    }
}

__device__ __forceinline__ float sig(float z) { return 1.0f / (1.0f + expf(-z)); }

__global__ void silu_kernel(const float* z, float* h, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    h[i] = z[i] * sig(z[i]);
}
// d <- d * silu'(z)
__global__ void silu_back_kernel(const float* z, float* d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float s = sig(z[i]);
    d[i] *= s * (1.0f + z[i] * (1.0f - s));
  }
}
// loss numerator / mask sum; dy = 2 mask (y - t) (scaled by 1/sum(mask) afterwards)
__global__ void loss_kernel(const float* y, const float* t, const float* mask, float* dy, float* scal, size_t n) {
  float a = 0.0f, s = 0.0f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    a += mask[i] * d * d;
    s += mask[i];
    dy[i] = 2.0f * mask[i] * d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(scal, a);
    atomicAdd(scal + 1, s);
  }
}
__global__ void scale_kernel(float* x, const float* scal, size_t n) {
  const float inv = 1.0f / fmaxf(scal[1], 1.0f);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] *= inv;
}
// column sums (bias gradients): out[c] = sum_r d[r, c]
__global__ void colsum_kernel(const float* d, float* out, int M, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.0f;
  for (int r = 0; r < M; ++r) s += d[(size_t)r * N + c];
  out[c] = s;
}
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, size_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.0f - b1) * gi;
    v[i] = b2 * v[i] + (1.0f - b2) * gi * gi;
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    pb[i] = __float2bfloat16(p[i]);
  }
}
__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* pb, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    pb[i] = __float2bfloat16(p[i]);
}

// BF16: operands rounded to BF16, tcgen05 MMAs (Bb, when given, is the BF16
// copy of B for tB == false); otherwise the FP32 kernel.  err: device flag.
cudaError_t gemm(const float* A, const float* B, const __nv_bfloat16* Bb, float* C, const float* bias, int M, int N,
                 int K, bool tA, bool tB, bool bf16, int* err, cudaStream_t s) {
  if (bf16) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((N + kTcN - 1) / kTcN, (M + kTcM - 1) / kTcM);
    tc_gemm_kernel<<<grid, kTcThreads, kTcSmemBytes, s>>>(A, B, tB ? nullptr : Bb, C, bias, M, N, K, tA, tB, err);
    return cudaGetLastError();
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_kernel<<<grid, 128, 0, s>>>(A, B, C, bias, M, N, K, tA, tB);
  return cudaGetLastError();
}

// FSIM_ECUDA when a tensor-core GEMM since the last check gave up waiting for
// its MMAs (the flag is cleared); synchronises the stream
int tc_status(fsim_mlp* n, cudaStream_t s) {
  int flag = 0;
  FSIM_CK(cudaMemcpyAsync(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FSIM_CK(cudaStreamSynchronize(s));
  if (flag) {
    FSIM_CK(cudaMemset(n->tc_err, 0, sizeof(int)));
    set_error("MLP GEMM: tensor-core MMAs did not complete");
    return FSIM_ECUDA;
  }
  return FSIM_OK;
}

int ensure_batch(fsim_mlp* n, int b) {
  if (b <= n->maxb) return FSIM_OK;
  float** bufs[] = {&n->z1, &n->h1, &n->z2, &n->h2, &n->d1, &n->d2};
  for (float** q : bufs) {
    dev_free(*q);
    FSIM_TRY(dev_alloc(q, (size_t)b * n->width));
  }
  dev_free(n->y);
  dev_free(n->dy);
  FSIM_TRY(dev_alloc(&n->y, (size_t)b * n->nout));
  FSIM_TRY(dev_alloc(&n->dy, (size_t)b * n->nout));
  n->maxb = b;
  return FSIM_OK;
}

int forward(fsim_mlp* n, const float* x, int b, bool bf16, cudaStream_t s) {
  const Off o = offsets(n->nin, n->width, n->nout);
  const int w = n->width;
  const size_t bw = (size_t)b * w;
  const int th = 256, bl = (int)std::min<size_t>((bw + th - 1) / th, 1024);
  FSIM_CK(gemm(x, n->p + o.W1, n->pb + o.W1, n->z1, n->p + o.b1, b, w, n->nin, false, false, bf16, n->tc_err, s));
  silu_kernel<<<bl, th, 0, s>>>(n->z1, n->h1, bw);
  FSIM_CK(gemm(n->h1, n->p + o.W2, n->pb + o.W2, n->z2, n->p + o.b2, b, w, w, false, false, bf16, n->tc_err, s));
  silu_kernel<<<bl, th, 0, s>>>(n->z2, n->h2, bw);
  FSIM_CK(gemm(n->h2, n->p + o.W3, n->pb + o.W3, n->y, n->p + o.b3, b, n->nout, w, false, false, bf16, n->tc_err, s));
  return FSIM_OK;
}

// loss and gradient (into n->g)
int backward(fsim_mlp* n, const float* x, const float* t, const float* mask, int b, bool bf16, cudaStream_t s) {
  const Off o = offsets(n->nin, n->width, n->nout);
  const int w = n->width;
  const size_t bw = (size_t)b * w, bo = (size_t)b * n->nout;
  const int th = 256;
  auto blocks = [&](size_t k) { return (int)std::min<size_t>((k + th - 1) / th, 1024); };
  FSIM_CK(cudaMemsetAsync(n->scal, 0, 2 * sizeof(float), s));
  loss_kernel<<<blocks(bo), th, 0, s>>>(n->y, t, mask, n->dy, n->scal, bo);
  scale_kernel<<<blocks(bo), th, 0, s>>>(n->dy, n->scal, bo);
  // layer 3
  FSIM_CK(gemm(n->h2, n->dy, nullptr, n->g + o.W3, nullptr, w, n->nout, b, true, false, bf16, n->tc_err, s));
  colsum_kernel<<<(n->nout + 127) / 128, 128, 0, s>>>(n->dy, n->g + o.b3, b, n->nout);
  FSIM_CK(gemm(n->dy, n->p + o.W3, nullptr, n->d2, nullptr, b, w, n->nout, false, true, bf16, n->tc_err, s));
  silu_back_kernel<<<blocks(bw), th, 0, s>>>(n->z2, n->d2, bw);
  // layer 2
  FSIM_CK(gemm(n->h1, n->d2, nullptr, n->g + o.W2, nullptr, w, w, b, true, false, bf16, n->tc_err, s));
  colsum_kernel<<<(w + 127) / 128, 128, 0, s>>>(n->d2, n->g + o.b2, b, w);
  FSIM_CK(gemm(n->d2, n->p + o.W2, nullptr, n->d1, nullptr, b, w, w, false, true, bf16, n->tc_err, s));
  silu_back_kernel<<<blocks(bw), th, 0, s>>>(n->z1, n->d1, bw);
  // layer 1
  FSIM_CK(gemm(x, n->d1, nullptr, n->g + o.W1, nullptr, n->nin, w, b, true, false, bf16, n->tc_err, s));
  colsum_kernel<<<(w + 127) / 128, 128, 0, s>>>(n->d1, n->g + o.b1, b, w);
  return FSIM_OK;
}

}  // namespace
}  // namespace fsim

void fsim::mlp_dims(const fsim_mlp* n, int* nin, int* width, int* nout) {
  *nin = n->nin;
  *width = n->width;
  *nout = n->nout;
}

using namespace fsim;

extern "C" {

int fsim_mlp_create(int nin, int width, int nout, const float* init_params, fsim_mlp** out) {
  if (!out || nin <= 0 || width <= 0 || nout <= 0 || !init_params) {
    set_error("fsim_mlp_create: bad arguments");
    return FSIM_EINVAL;
  }
  fsim_mlp* n = new fsim_mlp();
  n->nin = nin;
  n->width = width;
  n->nout = nout;
  n->np = offsets(nin, width, nout).n;
  int rc;
  auto fail = [&](int r) {
    fsim_mlp_destroy(n);
    return r;
  };
  float** bufs[] = {&n->p, &n->g, &n->m, &n->v};
  for (float** q : bufs)
    if ((rc = dev_alloc(q, n->np)) != FSIM_OK) return fail(rc);
  if ((rc = dev_alloc(&n->pb, n->np)) != FSIM_OK || (rc = dev_alloc(&n->scal, 2)) != FSIM_OK ||
      (rc = dev_alloc(&n->tc_err, 1)) != FSIM_OK)
    return fail(rc);
  if (cudaMemcpy(n->p, init_params, sizeof(float) * n->np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->tc_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * n->np) != cudaSuccess ||
      cudaMemset(n->v, 0, sizeof(float) * n->np) != cudaSuccess) {
    set_error("fsim_mlp_create: upload failed");
    return fail(FSIM_ECUDA);
  }
  to_bf16_kernel<<<256, 256>>>(n->p, n->pb, n->np);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(FSIM_ECUDA);
  *out = n;
  return FSIM_OK;
}

void fsim_mlp_destroy(fsim_mlp* n) {
  if (!n) return;
  float** bufs[] = {&n->p, &n->g, &n->m, &n->v, &n->z1, &n->h1, &n->z2, &n->h2, &n->y, &n->dy, &n->d1, &n->d2,
                    &n->scal};
  for (float** q : bufs) dev_free(*q);
  dev_free(n->pb);
  dev_free(n->tc_err);
  delete n;
}

long long fsim_mlp_nparams(const fsim_mlp* n) { return n ? (long long)n->np : -1; }

int fsim_mlp_params(fsim_mlp* n, float* host_out, const float* host_in) {
  if (!n) return FSIM_EINVAL;
  if (host_out) FSIM_CK(cudaMemcpy(host_out, n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  if (host_in) {
    FSIM_CK(cudaMemcpy(n->p, host_in, sizeof(float) * n->np, cudaMemcpyHostToDevice));
    to_bf16_kernel<<<256, 256>>>(n->p, n->pb, n->np);
    FSIM_CK(cudaDeviceSynchronize());
  }
  return FSIM_OK;
}

int fsim_mlp_save(fsim_mlp* n, const char* path) {
  if (!n || !path) {
    set_error("fsim_mlp_save: null pointer");
    return FSIM_EINVAL;
  }
  std::vector<float> p(n->np);
  FSIM_CK(cudaMemcpy(p.data(), n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error("fsim_mlp_save: cannot open %s", path);
    return FSIM_EINVAL;
  }
  const int32_t dims[3] = {n->nin, n->width, n->nout};
  const bool ok = std::fwrite("FSIMMLP1", 1, 8, f) == 8 && std::fwrite(dims, sizeof(int32_t), 3, f) == 3 &&
                  std::fwrite(p.data(), sizeof(float), n->np, f) == n->np;
  if (std::fclose(f) != 0 || !ok) {
    set_error("fsim_mlp_save: write to %s failed", path);
    return FSIM_EINVAL;
  }
  return FSIM_OK;
}

int fsim_mlp_load(const char* path, fsim_mlp** out) {
  if (!path || !out) {
    set_error("fsim_mlp_load: null pointer");
    return FSIM_EINVAL;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error("fsim_mlp_load: cannot open %s", path);
    return FSIM_EINVAL;
  }
  char magic[8];
  int32_t dims[3];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "FSIMMLP1", 8) == 0 &&
            std::fread(dims, sizeof(int32_t), 3, f) == 3 && dims[0] > 0 && dims[1] > 0 && dims[2] > 0 &&
            dims[0] <= 4096 && dims[1] <= 4096 && dims[2] <= 4096;
  std::vector<float> p;
  if (ok) {
    p.resize(offsets(dims[0], dims[1], dims[2]).n);
    ok = std::fread(p.data(), sizeof(float), p.size(), f) == p.size() && std::fgetc(f) == EOF;
  }
  std::fclose(f);
  if (!ok) {
    set_error("fsim_mlp_load: %s is not a weights file of fsim_mlp_save", path);
    return FSIM_EINVAL;
  }
  return fsim_mlp_create(dims[0], dims[1], dims[2], p.data(), out);
}

int fsim_mlp_forward(fsim_mlp* n, const float* x, float* y, int batch, int bf16, void* stream) {
  if (!n || !x || !y || batch <= 0) {
    set_error("fsim_mlp_forward: bad arguments");
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FSIM_TRY(ensure_batch(n, batch));
  FSIM_TRY(forward(n, x, batch, bf16 != 0, s));
  FSIM_CK(cudaMemcpyAsync(y, n->y, sizeof(float) * batch * n->nout, cudaMemcpyDeviceToDevice, s));
  return bf16 ? tc_status(n, s) : FSIM_OK;
}

int fsim_mlp_grad(fsim_mlp* n, const float* x, const float* t, const float* mask, int batch, int bf16, float* loss,
                  float* grad_host, void* stream) {
  if (!n || !x || !t || !mask || batch <= 0) {
    set_error("fsim_mlp_grad: bad arguments");
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FSIM_TRY(ensure_batch(n, batch));
  FSIM_TRY(forward(n, x, batch, bf16 != 0, s));
  FSIM_TRY(backward(n, x, t, mask, batch, bf16 != 0, s));
  float sc[2];
  FSIM_CK(cudaMemcpyAsync(sc, n->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
  if (grad_host) FSIM_CK(cudaMemcpyAsync(grad_host, n->g, sizeof(float) * n->np, cudaMemcpyDeviceToHost, s));
  FSIM_CK(cudaStreamSynchronize(s));
  if (loss) *loss = sc[0] / std::max(sc[1], 1.0f);
  return bf16 ? tc_status(n, s) : FSIM_OK;
}

int fsim_mlp_adam_step(fsim_mlp* n, const float* grad_host, float lr, void* stream) {
  if (!n || !grad_host || !(lr > 0.0f)) {
    set_error("fsim_mlp_adam_step: bad arguments");
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FSIM_CK(cudaMemcpyAsync(n->g, grad_host, sizeof(float) * n->np, cudaMemcpyHostToDevice, s));
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<256, 256, 0, s>>>(n->p, n->g, n->m, n->v, n->pb, n->np, lr, b1, b2, 1e-8f,
                                  1.0f - std::pow(b1, (float)n->step), 1.0f - std::pow(b2, (float)n->step));
  FSIM_CK(cudaGetLastError());
  FSIM_CK(cudaStreamSynchronize(s));
  return FSIM_OK;
}

int fsim_mlp_train_step(fsim_mlp* n, const float* x, const float* t, const float* mask, int batch, float lr,
                        float* loss, void* stream) {
  if (!n || !x || !t || !mask || batch <= 0 || !(lr > 0.0f)) {
    set_error("fsim_mlp_train_step: bad arguments");
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FSIM_TRY(ensure_batch(n, batch));
  FSIM_TRY(forward(n, x, batch, true, s));
  FSIM_TRY(backward(n, x, t, mask, batch, true, s));
  ++n->step;
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<256, 256, 0, s>>>(n->p, n->g, n->m, n->v, n->pb, n->np, lr, b1, b2, 1e-8f,
                                  1.0f - std::pow(b1, (float)n->step), 1.0f - std::pow(b2, (float)n->step));
  FSIM_CK(cudaGetLastError());
  if (loss) {
    float sc[2];
    FSIM_CK(cudaMemcpyAsync(sc, n->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    FSIM_CK(cudaStreamSynchronize(s));
    *loss = sc[0] / std::max(sc[1], 1.0f);
  }
  return tc_status(n, s);
}

}  // extern "C"
