// Warp-cooperative shell-quartet kernel with runtime class (table driven).
//
// Same mathematics as eri_core.cuh (paper Sec. 2.3.4 Eq. twoe-final, Sec. 2.5
// Eq. eri-tensor-contracted), organised for classes whose per-quartet arrays
// are too large for one thread: one warp per shell quartet,
//   * R^0_{tuv} built cooperatively in a shared-memory cube R[t][u][v]
//     (edge S = L+1, so R[h + h'] = cube[base(h) + off(h')]), level by level
//     of Eq. R-recursion with a warp barrier between total orders;
//   * W[h][c] (ket transform) and out[a][c] (bra transform) distributed over
//     the lanes, W passed through shared memory between the two transforms.
// Loops run over runtime index tables, so one compiled kernel serves every
// class pair.  Used for explicit quartet lists (Schwarz diagonal, debug dumps)
// and as one of the autotuner's launch shapes for the J/K build.
#pragma once
#include "eri_core.cuh"

namespace fsim {

constexpr int kCoopWarps = 4;
constexpr int kCoopMaxW = 40;    // ceil(35 * 36 / 32)
constexpr int kCoopMaxOut = 41;  // ceil(36 * 36 / 32)
constexpr int kCoopCube = 729;   // 9^3
constexpr int kCoopWsize = 35 * 36;

// Runtime description of a pair class (component extents and E non-zeros).
struct ClsDesc {
  int la, lb, na, nb, nc, L, nh, nnz;
  short ext[36][3];    // Hermite extent per axis of each component
  short off[37];       // first non-zero of each component
};

__host__ __device__ inline void make_cls_desc(int cls, ClsDesc& d) {
  d.la = pair_cls_la(cls);
  d.lb = pair_cls_lb(cls);
  d.na = ncart(d.la);
  d.nb = ncart(d.lb);
  d.nc = d.na * d.nb;
  d.L = d.la + d.lb;
  d.nh = nherm(d.L);
  int s = 0;
  for (int a = 0; a < d.nc; ++a) {
    for (int x = 0; x < 3; ++x) d.ext[a][x] = cart_comp(d.la, a / d.nb, x) + cart_comp(d.lb, a % d.nb, x);
    d.off[a] = s;
    s += (d.ext[a][0] + 1) * (d.ext[a][1] + 1) * (d.ext[a][2] + 1);
  }
  d.off[d.nc] = s;
  d.nnz = s;
}

constexpr int kCoopDescBytes = (sizeof(ClsDesc) + 15) / 16 * 16;
template <typename Real>
constexpr size_t coop_smem_bytes() {
  return 2 * kCoopDescBytes + (size_t)kCoopWarps * (kCoopCube + kCoopWsize) * sizeof(Real);
}

template <typename Real>
struct CoopParams {
  PairView<Real> bra, ket;
  ClsDesc bd, kd;
  int same;
  // JK mode (items from tile prefix) or list mode (explicit items)
  int list_mode;
  const int* __restrict__ tile_prefix;
  const int* __restrict__ ket_count;
  int tq;  // kets per work item
  const int2* __restrict__ items;
  int nitems;
  double* out;  // list mode: block per item
  int N;
  const Real* __restrict__ D;
  double* J;
  double* K;
  const Real* __restrict__ boys;
  float boys64_T;  // FP32 path: Boys in FP64 at T >= this (infinity = never)
};

// Boys F_0..F_L for a runtime L <= 8 in the working precision.
template <typename Real, int L>
__device__ __forceinline__ void boys_to(Real T, Real* F, const Real* tab, float t64) {
  Real f[L + 1];
  Boys<Real>::template eval<L>(T, f, tab + L, kBoysCols, t64);
#pragma unroll
  for (int n = 0; n <= L; ++n) F[n] = f[n];
}

template <typename Real>
__device__ __forceinline__ void boys_rt(int L, Real T, Real* F, const Real* tab, float t64) {
  switch (L) {
    case 0: boys_to<Real, 0>(T, F, tab, t64); break;
    case 1: boys_to<Real, 1>(T, F, tab, t64); break;
    case 2: boys_to<Real, 2>(T, F, tab, t64); break;
    case 3: boys_to<Real, 3>(T, F, tab, t64); break;
    case 4: boys_to<Real, 4>(T, F, tab, t64); break;
    case 5: boys_to<Real, 5>(T, F, tab, t64); break;
    case 6: boys_to<Real, 6>(T, F, tab, t64); break;
    case 7: boys_to<Real, 7>(T, F, tab, t64); break;
    default: boys_to<Real, 8>(T, F, tab, t64); break;
  }
}

__device__ __forceinline__ void herm_of(int h, int& t, int& u, int& v) {
  // inverse of hidx by search over the (small) triangle
  int n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= h) ++n;
  int r = h - n * (n + 1) * (n + 2) / 6;
  int m = 0;
  while ((m + 1) * (m + 2) / 2 <= r) ++m;
  v = r - m * (m + 1) / 2;
  u = m - v;
  t = n - m;
}

template <typename Real>
__global__ void __launch_bounds__(kCoopWarps * 32) coop_kernel(CoopParams<Real> P) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  ClsDesc& sbd = *reinterpret_cast<ClsDesc*>(coop_smem);
  ClsDesc& skd = *reinterpret_cast<ClsDesc*>(coop_smem + kCoopDescBytes);
  Real* sRall = reinterpret_cast<Real*>(coop_smem + 2 * kCoopDescBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sbd = P.bd;
    skd = P.kd;
  }
  __syncthreads();
  const ClsDesc& bd = sbd;
  const ClsDesc& kd = skd;
  const int L = bd.L + kd.L;
  const int S = L + 1;
  Real* R = sRall + (size_t)warp * (kCoopCube + kCoopWsize);
  Real* Ws = R + kCoopCube;
  const int NW = bd.nh * kd.nc;   // W entries (h, c)
  const int NO = bd.nc * kd.nc;   // out entries (a, c)
  const size_t bst = (size_t)P.bra.ppmax * P.bra.n, kst = (size_t)P.ket.ppmax * P.ket.n;

  // quartet assignment
  int i = 0, j0 = 0, jn = 0;
  if (P.list_mode) {
    const int t = blockIdx.x * kCoopWarps + warp;
    if (t < P.nitems) {
      i = P.items[t].x;
      j0 = P.items[t].y;
      jn = 1;
    }
  } else {
    if (blockIdx.x < P.nitems) {
      i = find_bra(P.tile_prefix, P.bra.n, blockIdx.x);
      const int tile = blockIdx.x - P.tile_prefix[i];
      j0 = tile * P.tq;
      jn = min(P.tq, P.ket_count[i] - j0);
    }
  }
  const int4 bi = P.bra.idx[i];
  const int nppb = P.bra.npp[i];
  for (int qq = (P.list_mode ? 0 : warp); qq < jn; qq += (P.list_mode ? 1 : kCoopWarps)) {
    const int j = P.list_mode ? j0 : j0 + qq;
    const int4 ki = P.ket.idx[j];
    const int nppk = P.ket.npp[j];
    Real outv[kCoopMaxOut];
#pragma unroll
    for (int m = 0; m < kCoopMaxOut; ++m) outv[m] = Real(0);
    for (int b = 0; b < nppb; ++b) {
      const Real* bp = P.bra.pd + (size_t)b * P.bra.n + i;
      const auto b4 = P.bra.pq[(size_t)b * P.bra.n + i];
      const Real p = b4.x, Px = b4.y, Py = b4.z, Pz = b4.w;
      Real Wv[kCoopMaxW];
#pragma unroll
      for (int m = 0; m < kCoopMaxW; ++m) Wv[m] = Real(0);
      for (int k = 0; k < nppk; ++k) {
        const Real* kp = P.ket.pd + (size_t)k * P.ket.n + j;
        const auto k4 = P.ket.pq[(size_t)k * P.ket.n + j];
        const Real q = k4.x, X = Px - k4.y, Y = Py - k4.z, Z = Pz - k4.w;
        const Real s = p + q;
        const Real rs = rsqrt_r<Real>(s);
        const Real al = p * q * (rs * rs);
        Real F[kBoysMaxN + 1];
        boys_rt<Real>(L, al * (X * X + Y * Y + Z * Z), F, P.boys, P.boys64_T);
        // source terms (-2 al)^n F_n / sqrt(p+q)
        Real fac = rs;
        for (int n = 0; n <= L; ++n) {
          F[n] *= fac;
          fac *= Real(-2) * al;
        }
        // R cube, in place level by level (Eq. R-recursion)
        __syncwarp();
        if (lane == 0) R[0] = F[L];
        __syncwarp();
        for (int n = L - 1; n >= 0; --n) {
          for (int sord = L - n; sord >= 1; --sord) {
            const int cnt = (sord + 1) * (sord + 2) / 2;
            for (int e = lane; e < cnt; e += 32) {
              // e -> (t, u, v) with t + u + v = sord
              int m = 0;
              while ((m + 1) * (m + 2) / 2 <= e) ++m;
              const int v = e - m * (m + 1) / 2, u = m - v, t = sord - m;
              Real r;
              if (t > 0) r = X * R[((t - 1) * S + u) * S + v] + (t > 1 ? Real(t - 1) * R[((t - 2) * S + u) * S + v] : Real(0));
              else if (u > 0) r = Y * R[(t * S + u - 1) * S + v] + (u > 1 ? Real(u - 1) * R[(t * S + u - 2) * S + v] : Real(0));
              else r = Z * R[(t * S + u) * S + v - 1] + (v > 1 ? Real(v - 1) * R[(t * S + u) * S + v - 2] : Real(0));
              R[(t * S + u) * S + v] = r;
            }
            __syncwarp();
          }
          if (lane == 0) R[0] = F[n];
          __syncwarp();
        }
        // ket transform: lane owns W entries w = lane + 32 m, (h, c) = (w / nc_k, w % nc_k)
#pragma unroll
        for (int m = 0; m < kCoopMaxW; ++m) {
          const int w = lane + 32 * m;
          if (w < NW) {
            const int h = w / kd.nc, c = w % kd.nc;
            int t, u, v;
            herm_of(h, t, u, v);
            const int base = (t * S + u) * S + v;
            const int ex = kd.ext[c][0], ey = kd.ext[c][1], ez = kd.ext[c][2];
            const Real* ep = kp + (size_t)(4 + kd.off[c]) * kst;
            Real acc = Real(0);
            int z = 0;
            for (int ta = 0; ta <= ex; ++ta)
              for (int nu = 0; nu <= ey; ++nu)
                for (int ph = 0; ph <= ez; ++ph, ++z) {
                  const Real e = ep[(size_t)z * kst];
                  const Real r = R[base + (ta * S + nu) * S + ph];
                  acc = ((ta + nu + ph) & 1) ? fma(-e, r, acc) : fma(e, r, acc);
                }
            Wv[m] += acc;
          }
        }
      }
      // W -> shared, then bra transform: lane owns out entries o = lane + 32 m, (a, c)
      __syncwarp();
#pragma unroll
      for (int m = 0; m < kCoopMaxW; ++m) {
        const int w = lane + 32 * m;
        if (w < NW) Ws[w] = Wv[m];
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < kCoopMaxOut; ++m) {
        const int o = lane + 32 * m;
        if (o < NO) {
          const int a = o / kd.nc, c = o % kd.nc;
          const int ex = bd.ext[a][0], ey = bd.ext[a][1], ez = bd.ext[a][2];
          const Real* ep = bp + (size_t)(4 + bd.off[a]) * bst;
          Real acc = Real(0);
          int z = 0;
          for (int t = 0; t <= ex; ++t)
            for (int u = 0; u <= ey; ++u)
              for (int v = 0; v <= ez; ++v, ++z) acc = fma(ep[(size_t)z * bst], Ws[hidx(t, u, v) * kd.nc + c], acc);
          outv[m] += acc;
        }
      }
      __syncwarp();
    }
    // emit
    if (P.list_mode) {
      double* o = P.out + (size_t)(blockIdx.x * kCoopWarps + warp) * NO;
#pragma unroll
      for (int m = 0; m < kCoopMaxOut; ++m) {
        const int e = lane + 32 * m;
        if (e < NO) o[e] = (double)outv[m];
      }
    } else {
      const int N = P.N;
      const Real deg = Real((bi.z == bi.w ? 1 : 2) * (ki.z == ki.w ? 1 : 2) * ((P.same && i == j) ? 1 : 2));
#pragma unroll
      for (int m = 0; m < kCoopMaxOut; ++m) {
        const int e = lane + 32 * m;
        if (e < NO) {
          const int a = e / kd.nc, c = e % kd.nc;
          const int mu = bi.x + a / bd.nb, nu = bi.y + a % bd.nb;
          const int la = ki.x + c / kd.nb, si = ki.y + c % kd.nb;
          const Real v = deg * outv[m];
          atomicAdd(&P.J[(size_t)mu * N + nu], (double)(P.D[(size_t)la * N + si] * v));
          atomicAdd(&P.J[(size_t)la * N + si], (double)(P.D[(size_t)mu * N + nu] * v));
          atomicAdd(&P.K[(size_t)mu * N + la], (double)(P.D[(size_t)nu * N + si] * v));
          atomicAdd(&P.K[(size_t)nu * N + si], (double)(P.D[(size_t)mu * N + la] * v));
          atomicAdd(&P.K[(size_t)mu * N + si], (double)(P.D[(size_t)nu * N + la] * v));
          atomicAdd(&P.K[(size_t)nu * N + la], (double)(P.D[(size_t)mu * N + si] * v));
        }
      }
    }
  }
}

}  // namespace fsim

namespace fsim {
template <typename Real>
cudaError_t launch_coop(const CoopParams<Real>& p, int nblocks, cudaStream_t s) {
  const size_t smem = coop_smem_bytes<Real>();
  cudaError_t e = cudaFuncSetAttribute(coop_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nblocks == 0) return cudaSuccess;
  coop_kernel<Real><<<nblocks, kCoopWarps * 32, smem, s>>>(p);
  return cudaGetLastError();
}
}  // namespace fsim
