// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores for the
// learned-guess network: C[M x N] = op(A)[M x K] op(B)[K x N] (+ bias[N]).
//
// One CTA of four warps per 128 x 128 tile of C.  The K dimension is walked in
// chunks of 64: all threads stage the chunk of A (128 rows) and of op(B)^T
// (128 columns of C) into shared memory as BF16, in the canonical no-swizzle
// K-major layout (core matrices of 8 rows x 16 bytes, 128 contiguous bytes
// each); one thread issues four tcgen05.mma (M 128, N 128, K 16 each) that
// accumulate in tensor memory (128 lanes x 128 FP32 columns) and commits them
// to an mbarrier, which every thread waits on (bounded) before the next chunk
// overwrites the operands.  The epilogue reads the accumulator back with
// tcgen05.ld (warp w: lanes, i.e. rows, 32w .. 32w + 31), adds the bias and
// stores FP32.  A wait that runs out sets *err and the CTA frees its tensor
// memory and returns.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace fsim {

constexpr int kTcM = 128, kTcN = 128, kTcK = 64;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcStage = (uint32_t)kTcM * kTcK * 2;  // bytes of one operand chunk
// dynamic shared memory per CTA: the two chunks (16 KB each), alignment slack
// and the barrier, rounded up so that at most three CTAs share an SM and their
// tensor-memory allocations (3 x 128 columns) fit the SM's 512 columns
constexpr int kTcSmemBytes = 60 * 1024;
static_assert(2 * kTcStage + 1024 + 64 <= (uint32_t)kTcSmemBytes, "tile does not fit");
static_assert(4 * kTcSmemBytes > 227 * 1024, "four CTAs per SM would oversubscribe tensor memory");

// byte offset of element (row, k) of a 128 x 64 BF16 chunk: core matrix
// (row / 8, k / 8) at ((row / 8) * 8 + k / 8) * 128, row % 8 at 16-byte steps,
// k % 8 at 2-byte steps.  K-adjacent core matrices are 128 B apart, row groups
// 1024 B apart.
__host__ __device__ __forceinline__ uint32_t tc_off(int row, int k) {
  return ((uint32_t)(((row >> 3) * (kTcK / 8) + (k >> 3)) << 7)) + ((uint32_t)(row & 7) << 4) +
         ((uint32_t)(k & 7) << 1);
}

constexpr uint32_t kTcLbo = 128, kTcSbo = 1024;  // K-adjacent core matrices, 8-row groups

// shared-memory matrix descriptor: start address, leading-dimension byte offset
// (between K-adjacent core matrices), stride-dimension byte offset (between
// 8-row groups), descriptor version 1, no swizzle
__host__ __device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

// bounded wait for the mbarrier phase of the given parity to complete
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (int i = 0; i < (1 << 22); ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// op(A) element (r, k): tA ? A[k M + r] : A[r K + k]; op(B) element (k, n):
// tB ? B[n K + k] : (Bb ? Bb[k N + n] : B[k N + n]).
__global__ void __launch_bounds__(kTcThreads) tc_gemm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                             const __nv_bfloat16* __restrict__ Bb,
                                                             float* __restrict__ C, const float* __restrict__ bias,
                                                             int M, int N, int K, int tA, int tB,
                                                             int* __restrict__ err) {
  extern __shared__ unsigned char tc_smem_raw[];
  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tc_smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  unsigned char* sA = tc_smem_raw + pad;
  unsigned char* sB = sA + kTcStage;
  const uint32_t aS = raw + pad, bS = aS + kTcStage, mS = bS + kTcStage, tS = mS + 8;
  const uint32_t* tslot = reinterpret_cast<const uint32_t*>(sB + kTcStage + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * kTcN;

  if (warp == 0) {  // whole warp: 128 columns of tensor memory, address written to tslot
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tS), "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mS));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;

  bool ok = true;
  int cfail = 0;
  const int nchunk = (K + kTcK - 1) / kTcK;
  for (int c = 0; c < nchunk; ++c) {
    const int k0 = c * kTcK;
    // stage the chunk (zero outside M, N, K); the previous chunk's MMAs are done
    for (int x = tid; x < kTcM * kTcK; x += kTcThreads) {
      const int r = tA ? x % kTcM : x / kTcK, k = tA ? x / kTcM : x % kTcK;
      const int gr = m0 + r, gk = k0 + k;
      float a = 0.0f;
      if (gr < M && gk < K) a = tA ? A[(size_t)gk * M + gr] : A[(size_t)gr * K + gk];
      *reinterpret_cast<__nv_bfloat16*>(sA + tc_off(r, k)) = __float2bfloat16(a);
    }
    for (int x = tid; x < kTcN * kTcK; x += kTcThreads) {
      const int n = tB ? x / kTcK : x % kTcN, k = tB ? x % kTcK : x / kTcN;
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (gn < N && gk < K)
        v = tB ? __float2bfloat16(B[(size_t)gn * K + gk])
               : (Bb ? Bb[(size_t)gk * N + gn] : __float2bfloat16(B[(size_t)gk * N + gn]));
      *reinterpret_cast<__nv_bfloat16*>(sB + tc_off(n, k)) = v;
    }
    // generic-proxy stores become visible to the tensor cores' (async proxy) reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        if (k0 + kk * 16 >= K) break;  // the zero padding past K needs no MMA (kk = 0 always runs)
        const uint64_t ad = tc_desc(aS + (uint32_t)kk * 256u, kTcLbo, kTcSbo);
        const uint64_t bd = tc_desc(bS + (uint32_t)kk * 256u, kTcLbo, kTcSbo);
        const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mS)
                   : "memory");
    }
    ok = tc_wait(mS, (uint32_t)(c & 1));
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (__syncthreads_or(!ok)) {
      ok = false;
      cfail = c;
      break;
    }
  }
  if (ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < kTcN; c0 += 8) {
      uint32_t v[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int r = m0 + warp * 32 + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        if (r < M && col < N) C[(size_t)r * N + col] = __uint_as_float(v[j]) + (bias ? bias[col] : 0.0f);
      }
    }
  } else {
    // a chunk's MMAs did not complete in time: give them one more bounded wait
    // before the tensor memory they write is released
    tc_wait(mS, (uint32_t)(cfail & 1));
    if (tid == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN));
}

}  // namespace fsim
