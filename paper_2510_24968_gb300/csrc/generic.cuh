// Shell-quartet kernel with runtime angular momenta, for every class pair that
// contains an f shell (paper Sec. 2.3.4 Eq. twoe-final, Sec. 2.5 Eq.
// eri-tensor-contracted; J/K digestion Eq. fock).  Same mathematics and
// conventions as eri_core.cuh (pair data with the contraction coefficients,
// Cartesian normalisation and sqrt(2) pi^{5/4}/p folded into E; degeneracy-
// weighted accumulators symmetrised by the caller), organised for quartets
// whose arrays are far too large for one thread ((ff|ff): R has 455 values, the
// block 10^4): one CTA per shell quartet,
//   * R^0_{tuv} in a shared-memory cube R[t][u][v] (edge L+1), built level by
//     level of Eq. R-recursion from R^L_000 down, two buffers, a barrier per level;
//   * W[h][c] = sum_k sum_{h' in nz(c)} (-1)^{|h'|} E^{cd,k}_{c,h'} R[h + h'] and
//     the block out[a][c] += sum_{h in nz(a)} E^{ab,b}_{a,h} W[h][c], both in
//     shared memory, their elements shared out over the threads;
//   * digestion: each thread adds its elements' six J/K terms with FP64 atomics.
// JK mode walks the class pair's flattened screened (bra, ket) list; list mode
// writes the blocks of explicit (bra, ket) items (Schwarz bounds, ERI dumps).
#pragma once
#include "eri_core.cuh"

namespace fsim {

constexpr int kGenThreads = 256;
constexpr int kGenMaxL = 12;     // (ff|ff)
constexpr int kGenMaxNC = 100;   // Cartesian components of an (f f) pair
constexpr int kGenMaxNH = 455;   // n_h(12)

template <typename Real>
struct GenParams {
  PairView<Real> bra, ket;
  int la, lb, lc, ld;
  int same;                          // bra class == ket class
  int list_mode;
  const int* __restrict__ prefix;    // JK mode: [nbra + 1] cumulative screened kets per bra
  const int2* __restrict__ items;    // list mode: (bra, ket) pair indices
  int nitems;                        // quartets (JK mode) or items (list mode)
  double* out;                       // list mode: block of item q at out + q * NA*NB * NC*ND
  int N;
  const Real* __restrict__ D;
  double* J;
  double* K;
  const Real* __restrict__ boys;     // full table, rows of kBoysCols
  float boys64_T;
};

// Dynamic shared memory of a class pair (Real values plus index tables).
template <typename Real>
__host__ __device__ constexpr size_t gen_smem_bytes(int la, int lb, int lc, int ld) {
  const int L = la + lb + lc + ld, S = L + 1;
  const int A = ncart(la) * ncart(lb), C = ncart(lc) * ncart(ld);
  const int NH1 = nherm(la + lb);
  return ((size_t)A * C + (size_t)NH1 * C + 2 * (size_t)S * S * S + 16) * sizeof(Real) +
         ((size_t)nherm(L) * 3 + (size_t)(A + C) * 3 + (A + 1) + (C + 1)) * sizeof(short) + 64;
}

template <typename Real, int L>
__device__ __forceinline__ void gen_boys_to(Real T, Real* F, const Real* tab, float t64) {
  Real f[L + 1];
  Boys<Real>::template eval<L>(T, f, tab + L, kBoysCols, t64);
#pragma unroll
  for (int n = 0; n <= L; ++n) F[n] = f[n];
}

template <typename Real>
__device__ void gen_boys(int L, Real T, Real* F, const Real* tab, float t64) {
  switch (L) {
    case 3: gen_boys_to<Real, 3>(T, F, tab, t64); break;
    case 4: gen_boys_to<Real, 4>(T, F, tab, t64); break;
    case 5: gen_boys_to<Real, 5>(T, F, tab, t64); break;
    case 6: gen_boys_to<Real, 6>(T, F, tab, t64); break;
    case 7: gen_boys_to<Real, 7>(T, F, tab, t64); break;
    case 8: gen_boys_to<Real, 8>(T, F, tab, t64); break;
    case 9: gen_boys_to<Real, 9>(T, F, tab, t64); break;
    case 10: gen_boys_to<Real, 10>(T, F, tab, t64); break;
    case 11: gen_boys_to<Real, 11>(T, F, tab, t64); break;
    default: gen_boys_to<Real, 12>(T, F, tab, t64); break;
  }
}

template <typename Real>
__global__ void __launch_bounds__(kGenThreads) gen_kernel(GenParams<Real> P) {
  extern __shared__ __align__(16) unsigned char gen_smem[];
  const int la = P.la, lb = P.lb, lc = P.lc, ld = P.ld;
  const int NA = ncart(la), NB = ncart(lb), NCc = ncart(lc), NDc = ncart(ld);
  const int A = NA * NB, C = NCc * NDc;
  const int Lb = la + lb, Lk = lc + ld, L = Lb + Lk, S = L + 1, S3 = S * S * S;
  const int NH = nherm(L), NH1 = nherm(Lb);
  Real* sOut = reinterpret_cast<Real*>(gen_smem);  // [a][c]
  Real* sW = sOut + (size_t)A * C;                   // [h][c]
  Real* sR0 = sW + (size_t)NH1 * C;                  // two cubes
  Real* sR1 = sR0 + S3;
  Real* sSrc = sR1 + S3;                             // R^n_000 sources, n = 0..L  (<= 13)
  Real* sGeo = sSrc + 13;                            // X, Y, Z of P - Q
  short* hT = reinterpret_cast<short*>(sGeo + 3);    // (t, u, v) of Hermite index h < NH
  short* extA = hT + 3 * NH;                         // Hermite extents of bra components
  short* extC = extA + 3 * A;
  short* offA = extC + 3 * C;                        // first non-zero of each component
  short* offC = offA + (A + 1);
  const int tid = threadIdx.x;
  // index tables of this class pair
  for (int h = tid; h < NH; h += blockDim.x) {
    int n = 0;
    while ((n + 1) * (n + 2) * (n + 3) / 6 <= h) ++n;
    int r = h - n * (n + 1) * (n + 2) / 6, m = 0;
    while ((m + 1) * (m + 2) / 2 <= r) ++m;
    const int v = r - m * (m + 1) / 2;
    hT[3 * h] = (short)(n - m);
    hT[3 * h + 1] = (short)(m - v);
    hT[3 * h + 2] = (short)v;
  }
  if (tid == 0) {
    int s = 0;
    for (int a = 0; a < A; ++a) {
      int e = 1;
      for (int x = 0; x < 3; ++x) {
        extA[3 * a + x] = (short)(cart_comp(la, a / NB, x) + cart_comp(lb, a % NB, x));
        e *= extA[3 * a + x] + 1;
      }
      offA[a] = (short)s;
      s += e;
    }
    offA[A] = (short)s;
    s = 0;
    for (int c = 0; c < C; ++c) {
      int e = 1;
      for (int x = 0; x < 3; ++x) {
        extC[3 * c + x] = (short)(cart_comp(lc, c / NDc, x) + cart_comp(ld, c % NDc, x));
        e *= extC[3 * c + x] + 1;
      }
      offC[c] = (short)s;
      s += e;
    }
    offC[C] = (short)s;
  }
  __syncthreads();
  const size_t bstride = (size_t)P.bra.ppmax * P.bra.n, kstride = (size_t)P.ket.ppmax * P.ket.n;
  for (int q = blockIdx.x; q < P.nitems; q += gridDim.x) {
    int i, j;
    if (P.list_mode) {
      const int2 it = P.items[q];
      i = it.x;
      j = it.y;
    } else {
      i = find_bra(P.prefix, P.bra.n, q);
      j = q - __ldg(P.prefix + i);
    }
    const int nppb = P.bra.npp[i], nppk = P.ket.npp[j];
    for (int x = tid; x < A * C; x += blockDim.x) sOut[x] = Real(0);
    for (int b = 0; b < nppb; ++b) {
      for (int x = tid; x < NH1 * C; x += blockDim.x) sW[x] = Real(0);
      for (int k = 0; k < nppk; ++k) {
        __syncthreads();  // previous primitive quartet done with the R cube and sources
        if (tid == 0) {
          const Real p = ldg_r(P.bra.pd + (size_t)b * P.bra.n + i);
          const Real Px = ldg_r(P.bra.pd + bstride + (size_t)b * P.bra.n + i);
          const Real Py = ldg_r(P.bra.pd + 2 * bstride + (size_t)b * P.bra.n + i);
          const Real Pz = ldg_r(P.bra.pd + 3 * bstride + (size_t)b * P.bra.n + i);
          const auto q4 = P.ket.pq[(size_t)k * P.ket.n + j];
          const Real qq = q4.x;
          const Real s = p + qq;
          const Real rs = rsqrt_r<Real>(s);
          const Real al = p * qq * (rs * rs);
          const Real X = Px - q4.y, Y = Py - q4.z, Z = Pz - q4.w;
          Real F[kGenMaxL + 1];
          gen_boys<Real>(L, al * (X * X + Y * Y + Z * Z), F, P.boys, P.boys64_T);
          Real fac = rs;
          for (int n = 0; n <= L; ++n) {
            sSrc[n] = fac * F[n];
            fac *= Real(-2) * al;
          }
          sGeo[0] = X;
          sGeo[1] = Y;
          sGeo[2] = Z;
        }
        __syncthreads();
        // R^n for n = L .. 0; level n holds t+u+v <= L-n and reads level n+1
        Real* cur = sR0;
        Real* nxt = sR1;
        if (tid == 0) cur[0] = sSrc[L];
        const Real X = sGeo[0], Y = sGeo[1], Z = sGeo[2];
        for (int n = L - 1; n >= 0; --n) {
          __syncthreads();
          const int nh = nherm(L - n);
          for (int h = tid; h < nh; h += blockDim.x) {
            const int t = hT[3 * h], u = hT[3 * h + 1], v = hT[3 * h + 2];
            Real r;
            if (h == 0) r = sSrc[n];
            else if (t > 0) r = X * cur[((t - 1) * S + u) * S + v] + (t > 1 ? Real(t - 1) * cur[((t - 2) * S + u) * S + v] : Real(0));
            else if (u > 0) r = Y * cur[(t * S + u - 1) * S + v] + (u > 1 ? Real(u - 1) * cur[(t * S + u - 2) * S + v] : Real(0));
            else r = Z * cur[(t * S + u) * S + v - 1] + (v > 1 ? Real(v - 1) * cur[(t * S + u) * S + v - 2] : Real(0));
            nxt[(t * S + u) * S + v] = r;
          }
          Real* tmp = cur;
          cur = nxt;
          nxt = tmp;
        }
        __syncthreads();
        // ket transform into W
        const Real* kp = P.ket.pd + (size_t)k * P.ket.n + j;
        for (int x = tid; x < NH1 * C; x += blockDim.x) {
          const int h = x / C, c = x % C;
          const int t = hT[3 * h], u = hT[3 * h + 1], v = hT[3 * h + 2];
          const int ex = extC[3 * c], ey = extC[3 * c + 1], ez = extC[3 * c + 2];
          int kk = offC[c];
          Real acc = Real(0);
          for (int ta = 0; ta <= ex; ++ta)
            for (int nu = 0; nu <= ey; ++nu)
              for (int ph = 0; ph <= ez; ++ph, ++kk) {
                const Real e = ldg_r(kp + (size_t)(4 + kk) * kstride);
                const Real r = cur[((t + ta) * S + u + nu) * S + v + ph];
                acc = fma(((ta + nu + ph) & 1) ? -e : e, r, acc);
              }
          sW[x] += acc;
        }
      }
      __syncthreads();
      // bra transform of this bra primitive pair into the block
      const Real* bp = P.bra.pd + (size_t)b * P.bra.n + i;
      for (int x = tid; x < A * C; x += blockDim.x) {
        const int a = x / C, c = x % C;
        const int ex = extA[3 * a], ey = extA[3 * a + 1], ez = extA[3 * a + 2];
        int kk = offA[a];
        Real acc = Real(0);
        for (int t = 0; t <= ex; ++t)
          for (int u = 0; u <= ey; ++u)
            for (int v = 0; v <= ez; ++v, ++kk)
              acc = fma(ldg_r(bp + (size_t)(4 + kk) * bstride), sW[hidx(t, u, v) * C + c], acc);
        sOut[x] += acc;
      }
      __syncthreads();
    }
    const int4 bi = P.bra.idx[i], ki = P.ket.idx[j];
    if (P.list_mode) {
      double* o = P.out + (size_t)q * A * C;
      for (int x = tid; x < A * C; x += blockDim.x) o[x] = (double)sOut[x];
    } else {
      const Real deg = Real((bi.z == bi.w ? 1 : 2) * (ki.z == ki.w ? 1 : 2) * ((P.same && i == j) ? 1 : 2));
      const int N = P.N;
      for (int x = tid; x < A * C; x += blockDim.x) {
        const int a = x / C, c = x % C;
        const int mu = bi.x + a / NB, nu = bi.y + a % NB, lam = ki.x + c / NDc, sig = ki.y + c % NDc;
        const Real v = deg * sOut[x];
        atomicAdd(&P.J[(size_t)lam * N + sig], (double)(P.D[(size_t)mu * N + nu] * v));
        atomicAdd(&P.J[(size_t)mu * N + nu], (double)(P.D[(size_t)lam * N + sig] * v));
        atomicAdd(&P.K[(size_t)mu * N + lam], (double)(P.D[(size_t)nu * N + sig] * v));
        atomicAdd(&P.K[(size_t)mu * N + sig], (double)(P.D[(size_t)nu * N + lam] * v));
        atomicAdd(&P.K[(size_t)nu * N + sig], (double)(P.D[(size_t)mu * N + lam] * v));
        atomicAdd(&P.K[(size_t)nu * N + lam], (double)(P.D[(size_t)mu * N + sig] * v));
      }
    }
    __syncthreads();  // block read before the next quartet clears it
  }
}

}  // namespace fsim
