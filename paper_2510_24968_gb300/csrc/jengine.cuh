// Coulomb-only build in Hermite space ("J-engine"; paper Sec. 2.5, the
// intermediate that contracts the ket's Hermite coefficients with the density
// before the Hermite Coulomb integrals are touched).
//
// J_mu,nu = sum_{la,si} D_la,si (mu nu|la si) (Eq. fock) never needs a
// Cartesian quartet.  With Eq. twoe-final, for a bra pair (ab) and a ket pair
// (cd) of primitive pairs b and k,
//   J_ab[a] += sum_b sum_{h in nz(a)} E^{ab,b}_{a,h}
//              sum_{kets cd} sum_k sum_{h'} R^{bk}[h + h'] rho^{cd,k}[h']
// where the density-contracted ket vector
//   rho^{cd,k}[h'] = deg_cd (-1)^{tau+nu+phi} sum_{c in (cd)} D_c E^{cd,k}_{c,h'}
// (h' = (tau, nu, phi); deg_cd = 2 when the two ket shells differ, for the
// (dc) order) is made once per build for every pair.  Per primitive quartet
// this costs the R recursion and n_h(Lbra) n_h(Lket) multiply-adds instead of
// the Cartesian transforms of both sides.  Each ordered (bra, ket) pair of
// classes is its own launch and contributes only to its bra block, so no ket
// side accumulation is needed: the bra is shared by the whole CTA and its J
// block is reduced over the CTA before one FP64 atomic per element.
#pragma once
#include "eri_core.cuh"

namespace fsim {

template <typename Real>
struct JEngParams {
  PairView<Real> bra, ket;
  const Real* __restrict__ rho;       // ket class: [h'][pp][pair] density-contracted Hermite vectors
  const int* __restrict__ prefix;     // [nbra + 1] cumulative ket tiles per bra
  const int* __restrict__ ket_count;  // [nbra] screened kets of each bra (all orders, no triangle)
  int N;
  double* J;                          // accumulator, N x N: J_acc(A,B) of the stored pair order
  int nitems;
  int psplit;                         // bra primitive pairs split over this many threads
  int bra_ppmax;
  const Real* __restrict__ boys;
  float boys64_T;
};

// rho^{cd,k}[h'] for every pair j and primitive pair k of one class (one thread
// each): rho[(h' * ppmax + k) * n + j].
template <typename Real, int LC, int LD>
__global__ void jeng_rho_kernel(PairView<Real> ket, const Real* __restrict__ D, int N, Real* __restrict__ rho) {
  using KC = PairCls<LC, LD>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ket.n * ket.ppmax) return;
  const int j = t % ket.n, k = t / ket.n;
  Real acc[KC::NH];
#pragma unroll
  for (int h = 0; h < KC::NH; ++h) acc[h] = Real(0);
  const size_t kstride = (size_t)ket.ppmax * ket.n;
  if (k < ket.npp[j]) {
    const int4 ki = ket.idx[j];
    const Real* kp = ket.pd + (size_t)k * ket.n + j;
    static_for<KC::NC>([&](auto Cc) {
      constexpr int c = decltype(Cc)::value;
      const Real Dc = D[(size_t)(ki.x + c / KC::NB) * N + ki.y + c % KC::NB];
      static_for<KC::nnz(c)>([&](auto Kk) {
        constexpr int kk = decltype(Kk)::value;
        constexpr int tau = KC::nz_t(c, kk), nu = KC::nz_u(c, kk), phi = KC::nz_v(c, kk);
        const Real e = ldg_r(kp + (size_t)(4 + KC::off(c) + kk) * kstride);
        acc[hidx(tau, nu, phi)] = fma(((tau + nu + phi) & 1) ? -Dc : Dc, e, acc[hidx(tau, nu, phi)]);
      });
    });
    const Real deg = Real(ki.z == ki.w ? 1 : 2);
#pragma unroll
    for (int h = 0; h < KC::NH; ++h) acc[h] = deg * acc[h];
  }
#pragma unroll
  for (int h = 0; h < KC::NH; ++h) rho[((size_t)h * ket.ppmax + k) * ket.n + j] = acc[h];
}

template <typename Real, int LA, int LB>
__host__ __device__ constexpr size_t jeng_smem_bytes(int bra_ppmax) {
  using BC = PairCls<LA, LB>;
  return (jk_boys_smem<Real>() + 15) / 16 * 16 +
         ((size_t)BC::NC * kJKThreads + (kJKThreads / 32) * BC::NC + (size_t)bra_ppmax * (4 + BC::NNZ)) *
             sizeof(Real);
}

// One ordered class pair (bra class (LA,LB), ket class (LC,LD)), persistent:
// a work item is (bra pair, tile of its screened kets); thread = (ket of the
// tile, subset of the bra primitive pairs).  The bra's primitive data sit in
// shared memory; each thread keeps its share of the bra's J block in its
// shared-memory slots, added into once per bra primitive pair.
template <typename Real, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(kJKThreads) jeng_kernel(JEngParams<Real> P) {
  using BC = PairCls<LA, LB>;
  using KC = PairCls<LC, LD>;
  constexpr int L = LA + LB + LC + LD;
  constexpr int NH = nherm(L), NH1 = BC::NH, NH2 = KC::NH;
  constexpr int NFB = 4 + BC::NNZ;
  constexpr int BK = Boys<Real>::NCOL, BR = Boys<Real>::NROW;
  constexpr int NWARP = kJKThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sBoys = reinterpret_cast<Real*>(smem_raw);
  Real* sJ = reinterpret_cast<Real*>(smem_raw + (jk_boys_smem<Real>() + 15) / 16 * 16);  // [a][thread]
  Real* sJw = sJ + BC::NC * kJKThreads;                                                    // [warp][a]
  Real* sbra = sJw + NWARP * BC::NC;                                                       // [pp][field]
  for (int x = threadIdx.x; x < BR * BK; x += blockDim.x)
    sBoys[x] = P.boys[(x / BK) * kBoysCols + Boys<Real>::col(L, x % BK)];
  const int ps = P.psplit, tq = kJKThreads / ps;
  const int q = threadIdx.x / ps, bs = threadIdx.x % ps;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Real* jslot = sJ + threadIdx.x;
  const size_t kstride = (size_t)P.ket.ppmax * P.ket.n;
  for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
    const int i = find_bra(P.prefix, P.bra.n, item);
    const int tile = item - __ldg(P.prefix + i);
    const int nppb = P.bra.npp[i];
    __syncthreads();  // previous item done with the bra buffers (and the Boys table staged)
    for (int x = threadIdx.x; x < nppb * NFB; x += blockDim.x) {
      const int pp = x / NFB, f = x % NFB;
      sbra[x] = P.bra.pd[((size_t)f * P.bra.ppmax + pp) * P.bra.n + i];
    }
#pragma unroll
    for (int a = 0; a < BC::NC; ++a) jslot[a * kJKThreads] = Real(0);
    __syncthreads();
    const int j = tile * tq + q;
    if (q < tq && j < __ldg(P.ket_count + i)) {
      const int nppk = P.ket.npp[j];
      for (int b = bs; b < nppb; b += ps) {
        const Real* sb = sbra + b * NFB;
        const Real p = sb[0], Px = sb[1], Py = sb[2], Pz = sb[3];
        Real jt[NH1];
#pragma unroll
        for (int h = 0; h < NH1; ++h) jt[h] = Real(0);
        for (int k = 0; k < nppk; ++k) {
          const auto q4 = P.ket.pq[(size_t)k * P.ket.n + j];
          const Real qq = q4.x;
          const Real s = p + qq;
          const Real rs = rsqrt_r<Real>(s);
          const Real al = p * qq * (rs * rs);
          const Real X = Px - q4.y, Y = Py - q4.z, Z = Pz - q4.w;
          const Real T = al * (X * X + Y * Y + Z * Z);
          Real F[L + 1];
          Boys<Real>::template eval<L>(T, F, sBoys, BK, P.boys64_T);
          Real src[L + 1];
          Real fac = rs;
          const Real m2a = Real(-2) * al;
#pragma unroll
          for (int n = 0; n <= L; ++n) {
            src[n] = fac * F[n];
            fac *= m2a;
          }
          Real R[NH];
          hermite_R<Real, L>(R, src, X, Y, Z);
          const Real* rk = P.rho + (size_t)k * P.ket.n + j;
          static_for<NH2>([&](auto Hk) {
            constexpr int hk = decltype(Hk)::value;
            const Real r = ldg_r(rk + (size_t)hk * kstride);
            static_for<NH1>([&](auto Hb) {
              constexpr int hb = decltype(Hb)::value;
              constexpr int hr = hidx(herm_t(hb) + herm_t(hk), herm_u(hb) + herm_u(hk), herm_v(hb) + herm_v(hk));
              jt[hb] = fma(r, R[hr], jt[hb]);
            });
          });
        }
        // bra transform of this bra primitive pair into the thread's J slots
        static_for<BC::NC>([&](auto Aa) {
          constexpr int a = decltype(Aa)::value;
          Real acc = Real(0);
          static_for<BC::nnz(a)>([&](auto Kk) {
            constexpr int kk = decltype(Kk)::value;
            constexpr int h = hidx(BC::nz_t(a, kk), BC::nz_u(a, kk), BC::nz_v(a, kk));
            acc = fma(sb[4 + BC::off(a) + kk], jt[h], acc);
          });
          jslot[a * kJKThreads] += acc;
        });
      }
    }
    // the bra block summed over the CTA: warp reduction, per-warp partials,
    // one FP64 atomic per element and work item
#pragma unroll
    for (int a = 0; a < BC::NC; ++a) {
      Real v = jslot[a * kJKThreads];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += shfl_xor_r(v, o);
      if (lane == 0) sJw[warp * BC::NC + a] = v;
    }
    __syncthreads();
    const int4 bi = P.bra.idx[i];
    const double degb = bi.z == bi.w ? 1.0 : 2.0;
    for (int x = threadIdx.x; x < BC::NC; x += blockDim.x) {
      double v = 0.0;
      for (int w = 0; w < NWARP; ++w) v += (double)sJw[w * BC::NC + x];
      atomicAdd(&P.J[(size_t)(bi.x + x / BC::NB) * P.N + bi.y + x % BC::NB], degb * v);
    }
  }
}

}  // namespace fsim
