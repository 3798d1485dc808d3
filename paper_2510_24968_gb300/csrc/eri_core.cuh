// Shell-quartet kernels of the McMurchie-Davidson ERI engine (paper Sec. 2.3.4,
// Eq. twoe-final; contracted form Eq. eri-tensor-contracted of Sec. 2.5),
// fused with Schwarz screening and J/K digestion (Eq. fock).
//
// For a quartet (ab|cd) of bra pair class (LA,LB) and ket pair class (LC,LD),
// each primitive quartet contributes
//   [ab|cd] = 2 pi^{5/2} / (p q sqrt(p+q))
//             sum_{tuv} sum_{tau nu phi} (-1)^{tau+nu+phi} E^{ab}_{tuv} E^{cd}_{tau nu phi}
//             R^0_{t+tau, u+nu, v+phi}(alpha = pq/(p+q), P - Q)
// with R^0 from the recursion of Eq. R-recursion seeded by the Boys function.
// Evaluation order (per thread = one shell quartet, or a share of its bra
// primitive pairs / ket chunks; ket components in chunks of CS so that R, W and
// the chunk's E non-zeros stay in registers; out lives in shared memory):
//   for each bra primitive pair b:
//     W[h][c] = sum_k sum_{h' in nz(c)} sign(h') E^{cd,k}_{h'} R^{bk}[h + h']   (ket transform)
//     out[a][c] += sum_{h in nz(a)} E^{ab,b}_h W[h][c]                            (bra transform)
// Pair data already folds the contraction coefficients, the Cartesian
// normalisation and sqrt(2) pi^{5/4} / p into E, so only 1/sqrt(p+q) remains
// per primitive quartet (folded into the Boys source terms).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

#include "boys.cuh"
#include "md_tables.cuh"

namespace fsim {

constexpr int kJKThreads = 128;

// One pair class on the device.  Pairs are sorted by Schwarz bound, descending.
// Primitive-pair data is SoA: value (field f, primitive pair k, pair j) at
// pd[(f * ppmax + k) * n + j]; fields: 0 = p, 1..3 = P, 4.. = E non-zeros.
template <typename Real>
struct Vec4;
template <>
struct Vec4<double> {
  using type = double4_32a;
};
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<dfloat> {
  using type = dfloat4;
};

template <typename Real>
struct PairView {
  int n;
  int ppmax;
  const int4* __restrict__ idx;                     // (ao_a, ao_b, shell_a, shell_b)
  const int* __restrict__ npp;                      // primitive pairs of each pair
  const Real* __restrict__ pd;                      // [field][pp][pair]
  const typename Vec4<Real>::type* __restrict__ pq;  // (p, Px, Py, Pz) at [pp][pair]
};

// Everything a work item needs about its molecule.
template <typename Real>
struct JKMol {
  PairView<Real> bra, ket;
  const int* __restrict__ prefix;       // [nbra + 1] cumulative work units per bra: ket tiles
                                        // (per-bra form) or screened quartets (flattened form)
  const int* __restrict__ ket_count;    // [nbra] screened ket prefix length per bra
  int N;
  const Real* __restrict__ D;           // density, N x N, in the working precision
  double* J;                            // accumulators (FP64), N x N
  double* K;
  const double* __restrict__ bq = nullptr;  // Schwarz bounds of the bra / ket class's pairs (same order);
  const double* __restrict__ kq = nullptr;  // read only when JKParams::tau_mol is set
};

template <typename Real>
struct JKParams {
  JKMol<Real> one;                      // single molecule (nmol == 0)
  const JKMol<Real>* __restrict__ mols; // batched: one entry per molecule
  const int* __restrict__ mol_prefix;   // batched: [nmol + 1] cumulative work items
  const int* __restrict__ active;       // batched, optional: molecules whose items run
  const int* __restrict__ mol_ids;      // batched: table entry -> index into active
  int nmol;
  int nitems;                           // total work items
  int same;                             // bra class == ket class
  int psplit;                           // primitive quartets of a quartet split over this many threads
                                        // (bra primitive pairs first, then ket primitive pairs)
  int csplit;                           // ket chunks shared out over this many thread groups (1, 2, 4)
  int bra_ppmax;                        // largest bra primitive-pair count (shared-memory size)
  const Real* __restrict__ boys;
  float boys64_T;                       // FP32 path: Boys in FP64 at T >= this (infinity = never)
  // batched, optional: per molecule (indexed like active) a density-weighted
  // threshold; a quartet with Q_ab Q_cd below it is skipped (0: none skipped)
  const float* __restrict__ tau_mol = nullptr;
};

// Hermite Coulomb integrals R^0_{tuv} for t+u+v <= L, in place (Eq. R-recursion):
// level n is derived from level n+1 processing total orders s = L-n .. 1
// (higher first) so that lower orders still hold level n+1 when read.
template <typename Real, int L>
__device__ __forceinline__ void hermite_R(Real (&R)[nherm(L)], const Real (&src)[L + 1], Real X, Real Y,
                                          Real Z) {
  R[0] = src[L];
  static_for<L>([&](auto I) {
    constexpr int n = L - 1 - decltype(I)::value;
    static_for<L - n>([&](auto S) {
      constexpr int s = L - n - decltype(S)::value;
      static_for<s + 1>([&](auto Tt) {
        constexpr int t = decltype(Tt)::value;
        static_for<s - t + 1>([&](auto Uu) {
          constexpr int u = decltype(Uu)::value;
          constexpr int v = s - t - u;
          if constexpr (t > 0) {
            if constexpr (t > 1)
              R[hidx(t, u, v)] = X * R[hidx(t - 1, u, v)] + Real(t - 1) * R[hidx(t - 2, u, v)];
            else
              R[hidx(t, u, v)] = X * R[hidx(t - 1, u, v)];
          } else if constexpr (u > 0) {
            if constexpr (u > 1)
              R[hidx(t, u, v)] = Y * R[hidx(t, u - 1, v)] + Real(u - 1) * R[hidx(t, u - 2, v)];
            else
              R[hidx(t, u, v)] = Y * R[hidx(t, u - 1, v)];
          } else {
            if constexpr (v > 1)
              R[hidx(t, u, v)] = Z * R[hidx(t, u, v - 1)] + Real(v - 1) * R[hidx(t, u, v - 2)];
            else
              R[hidx(t, u, v)] = Z * R[hidx(t, u, v - 1)];
          }
        });
      });
    });
    R[0] = src[n];
  });
}

template <typename Real>
__device__ __forceinline__ Real rsqrt_r(Real x);
template <>
__device__ __forceinline__ double rsqrt_r<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ dfloat rsqrt_r<dfloat>(dfloat x) { return rsqrt_dfloat(x); }

// Chunk bookkeeping for the ket side: chunks of CS consecutive components, the
// last one possibly shorter.
template <class KC, int CS>
struct KetChunks {
  static constexpr int NCH = (KC::NC + CS - 1) / CS;
  __host__ __device__ static constexpr int end(int ch) { return (ch + 1) * CS < KC::NC ? (ch + 1) * CS : KC::NC; }
  __host__ __device__ static constexpr int nnz_of(int ch) { return KC::off(end(ch)) - KC::off(ch * CS); }
  __host__ __device__ static constexpr int max_nnz() {
    int m = 0;
    for (int ch = 0; ch < NCH; ++ch) m = nnz_of(ch) > m ? nnz_of(ch) : m;
    return m;
  }
};

// Contracted quartet block for one ket chunk: out(a, cs) for all bra components
// a and ket components c = ch*CS + cs < NC, accumulated in this thread's
// shared-memory slots so[(a * CS + cs) * kJKThreads] (so the registers hold
// only R, the chunk's W and its E non-zeros).  Bra data: accessor bra(field, pp).
// The bstep threads of a quartet share its primitive quartets: with bstep <=
// nppb each takes whole bra primitive pairs (b0, b0 + bstep, ...) and every ket
// primitive pair; with more threads than bra primitive pairs the ket primitive
// pairs are split ks = ceil(bstep / nppb) ways as well, thread b0 taking the
// units u = b0, b0 + bstep, ... < nppb * ks, each unit one bra primitive pair
// (u % nppb) with every ks-th ket primitive pair from u / nppb.  The caller sums
// the bstep partial blocks.
// The chunk index is a runtime value (uniform across the warp), so the Boys
// function, the R recursion, the bra transform and the caller's digestion exist
// once in the code; only the ket transform (and its loads of the chunk's E
// non-zeros) is specialised per chunk behind a warp-uniform branch, which keeps
// the instruction footprint of a chunk small enough for the instruction cache.
template <typename Real, int LA, int LB, int LC, int LD, int CS, class BraAt>
__device__ __forceinline__ void quartet_chunk(Real* __restrict__ so, const BraAt& bra, int nppb, int b0, int bstep,
                                              const PairView<Real>& ket, int j, int nppk,
                                              const Real* __restrict__ boysL, int bstride, float t64, int ch) {
  using BC = PairCls<LA, LB>;
  using KC = PairCls<LC, LD>;
  using KCh = KetChunks<KC, CS>;
  constexpr int L = LA + LB + LC + LD;
  constexpr int NH = nherm(L);
  constexpr int NH1 = BC::NH;
  constexpr int NZM = KCh::max_nnz();
#pragma unroll
  for (int x = 0; x < BC::NC * CS; ++x) so[x * kJKThreads] = Real(0);
  const size_t kstride = (size_t)ket.ppmax * ket.n;
  const int ks = (bstep + nppb - 1) / nppb;
  for (int u = b0; u < nppb * ks; u += bstep) {
    const int b = u % nppb;
    const Real p = bra(0, b), Px = bra(1, b), Py = bra(2, b), Pz = bra(3, b);
    Real W[NH1][CS];
#pragma unroll
    for (int h = 0; h < NH1; ++h)
#pragma unroll
      for (int cs = 0; cs < CS; ++cs) W[h][cs] = Real(0);
    for (int k = u / nppb; k < nppk; k += ks) {
      const Real* kp = ket.pd + (size_t)k * ket.n + j;
      const auto q4 = ket.pq[(size_t)k * ket.n + j];
      const Real q = q4.x, Qx = q4.y, Qy = q4.z, Qz = q4.w;
      const Real s = p + q;
      const Real rs = rsqrt_r<Real>(s);
      const Real al = p * q * (rs * rs);
      const Real X = Px - Qx, Y = Py - Qy, Z = Pz - Qz;
      const Real T = al * (X * X + Y * Y + Z * Z);
      Real F[L + 1];
      Boys<Real>::template eval<L>(T, F, boysL, bstride, t64);
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
      Real Ek[NZM];
      static_for<KCh::NCH>([&](auto Ch) {
        constexpr int CH = decltype(Ch)::value;
        if (ch != CH) return;
        constexpr int c0 = CH * CS;
        constexpr int nzoff = KC::off(c0);
        constexpr int NZ = KCh::nnz_of(CH);
#pragma unroll
        for (int z = 0; z < NZ; ++z) Ek[z] = ldg_r(kp + (size_t)(4 + nzoff + z) * kstride);
        static_for<CS>([&](auto Cs) {
          constexpr int cs = decltype(Cs)::value;
          constexpr int c = c0 + cs;
          if constexpr (c < KC::NC) {
            constexpr int zb = KC::off(c) - nzoff;
            static_for<KC::nnz(c)>([&](auto Kk) {
              constexpr int kk = decltype(Kk)::value;
              constexpr int tau = KC::nz_t(c, kk), nu = KC::nz_u(c, kk), phi = KC::nz_v(c, kk);
              const Real e = ((tau + nu + phi) & 1) ? -Ek[zb + kk] : Ek[zb + kk];
              static_for<NH1>([&](auto Hh) {
                constexpr int h = decltype(Hh)::value;
                constexpr int hr = hidx(herm_t(h) + tau, herm_u(h) + nu, herm_v(h) + phi);
                W[h][cs] = fma(e, R[hr], W[h][cs]);
              });
            });
          }
        });
      });
    }
    static_for<BC::NC>([&](auto Aa) {
      constexpr int a = decltype(Aa)::value;
      Real acc[CS];
#pragma unroll
      for (int cs = 0; cs < CS; ++cs) acc[cs] = Real(0);
      static_for<BC::nnz(a)>([&](auto Kk) {
        constexpr int kk = decltype(Kk)::value;
        constexpr int h = hidx(BC::nz_t(a, kk), BC::nz_u(a, kk), BC::nz_v(a, kk));
        const Real e = bra(4 + BC::off(a) + kk, b);
#pragma unroll
        for (int cs = 0; cs < CS; ++cs) acc[cs] = fma(e, W[h][cs], acc[cs]);
      });
#pragma unroll
      for (int cs = 0; cs < CS; ++cs) so[(a * CS + cs) * kJKThreads] += acc[cs];
    });
  }
}

// Barrier over the warps of chunk group g (0..3) of nthreads threads (a
// multiple of 32): named barriers 1..4, id 0 being __syncthreads'.  The ids
// are immediates so that a kernel reserves only the barriers it uses.
__device__ __forceinline__ void group_barrier(int g, int nthreads) {
  switch (g) {
    case 0: asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory"); break;
    case 1: asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory"); break;
    case 2: asm volatile("bar.sync 3, %0;" ::"r"(nthreads) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(nthreads) : "memory"); break;
  }
}

// Binary search: largest i in [0, n) with prefix[i] <= item.
__device__ __forceinline__ int find_bra(const int* __restrict__ prefix, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Fused ERI + J/K kernel, persistent: each CTA walks work items with a grid
// stride; threads = (ket chunk group, quartet of the tile, bra-primitive
// subset).  Two work decompositions (compile-time, by precision):
//  * FP32 (kFlat false): a work item is (bra pair, tile of its screened kets).
//    The CTA stages the bra's primitive data and D block in shared memory,
//    where every thread reads them as broadcasts, and reduces J_bra over the
//    CTA (one FP64 add per element and item).
//  * FP64 and double-float (kFlat true: 8-byte values): a work item is a tile
//    of consecutive quartets of the class pair's flattened (bra, screened ket)
//    list, so tiles are full however few kets a bra has, and the loop has no
//    barriers.  Each thread reads its
//    bra data through the L1 cache and reduces J_bra over the warp when the
//    warp's quartets share one bra (else lane by lane).  At the FP64 rate the
//    extra loads are free and the full tiles and missing barriers win (5-26 %
//    per class on the 12-atom cloud); at the FP32 rate the per-bra staging is
//    faster (up to 1.9x on the 30-atom cloud).
// Shared memory: the Boys table columns L..L+K-1 (loaded once per CTA), the
// per-thread quartet-block and J_bra slots, and (per-bra form) the bra block.
// Accumulates J_acc, K_acc with the 8-fold degeneracy factor; the caller
// symmetrises J = (J_acc + J_acc^T)/4 and K = (K_acc + K_acc^T)/8.
template <typename Real>
__host__ __device__ constexpr size_t jk_boys_smem() {
  return (size_t)Boys<Real>::NROW * Boys<Real>::NCOL * sizeof(Real);
}

template <typename Real>
__host__ __device__ constexpr bool jk_flat() {
  return sizeof(Real) == 8;
}

// Dynamic shared memory of one CTA (bra_ppmax: largest bra primitive-pair count).
template <typename Real, int LA, int LB, int CS>
__host__ __device__ constexpr size_t jk_smem_bytes(int bra_ppmax) {
  using BC = PairCls<LA, LB>;
  return (jk_boys_smem<Real>() + 15) / 16 * 16 + (size_t)(CS + 1) * BC::NC * kJKThreads * sizeof(Real) +
         (jk_flat<Real>() ? 0
                          : ((1 + kJKThreads / 32) * BC::NC + (size_t)bra_ppmax * (4 + BC::NNZ)) * sizeof(Real));
}

template <typename Real, int LA, int LB, int LC, int LD, int CS>
__global__ void __launch_bounds__(kJKThreads) jk_kernel(JKParams<Real> P) {
  using BC = PairCls<LA, LB>;
  using KC = PairCls<LC, LD>;
  constexpr bool kFlat = jk_flat<Real>();
  constexpr int L = LA + LB + LC + LD;
  constexpr int NFB = 4 + BC::NNZ;
  constexpr int BK = Boys<Real>::NCOL, BR = Boys<Real>::NROW;
  constexpr int NWARP = kJKThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sBoys = reinterpret_cast<Real*>(smem_raw);                     // [BR][BK]
  Real* sOut = reinterpret_cast<Real*>(smem_raw + (jk_boys_smem<Real>() + 15) / 16 * 16);  // [a * CS + cs][thread]
  Real* sJb = sOut + BC::NC * CS * kJKThreads;  // per-thread part of J_acc for the bra block [a][thread]
  Real* sDab = sJb + BC::NC * kJKThreads;       // per-bra form: D bra block [a]
  Real* sJw = sDab + BC::NC;                    // per-bra form: per-warp J_bra partials [warp][a]
  Real* sbra = sJw + NWARP * BC::NC;            // per-bra form: bra primitive data [pp][field]

  for (int x = threadIdx.x; x < BR * BK; x += blockDim.x)
    sBoys[x] = P.boys[(x / BK) * kBoysCols + Boys<Real>::col(L, x % BK)];
  __syncthreads();
  // thread = (chunk group cg, quartet q of the tile, bra-primitive subset bs);
  // the chunk group is the slowest index, so it is uniform within each warp
  const int ps = P.psplit, ncg = P.csplit;
  const int gsz = blockDim.x / ncg;
  const int cg = threadIdx.x / gsz, t = threadIdx.x % gsz;
  const int tq = gsz / ps;
  const int q = t / ps, bs = t % ps;
  const int lane = threadIdx.x & 31;
  Real* so = sOut + threadIdx.x;
  Real* jb = sJb + threadIdx.x;  // this thread's part of J_acc for its bra block, jb[a * kJKThreads]

  for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
    int litem = item;
    int mol_id = 0;
    const JKMol<Real>* Mp = &P.one;
    if (P.nmol > 0) {
      const int m = find_bra(P.mol_prefix, P.nmol, item);
      mol_id = __ldg(P.mol_ids + m);
      if (P.active && !__ldg(P.active + mol_id)) continue;  // uniform per CTA: a converged molecule
      Mp = P.mols + m;
      litem = item - __ldg(P.mol_prefix + m);
    }
    const JKMol<Real> M = *Mp;
    const int N = M.N;
    // this thread's quartet (bra i, ket j), if any
    int i = -1, j = 0;
    bool valid;
    if constexpr (kFlat) {
      const int g = litem * tq + q;  // quartet index in the flattened list
      valid = q < tq && g < __ldg(M.prefix + M.bra.n);
      if (valid) {
        i = find_bra(M.prefix, M.bra.n, g);
        j = g - __ldg(M.prefix + i);
      }
    } else {
      i = find_bra(M.prefix, M.bra.n, litem);
      const int tile = litem - __ldg(M.prefix + i);
      const int nppb = M.bra.npp[i];
      const int4 bb = M.bra.idx[i];
      __syncthreads();  // previous item done with the bra buffers
      for (int x = threadIdx.x; x < nppb * NFB; x += blockDim.x) {
        const int pp = x / NFB, f = x % NFB;
        sbra[x] = M.bra.pd[((size_t)f * M.bra.ppmax + pp) * M.bra.n + i];
      }
      for (int x = threadIdx.x; x < BC::NC; x += blockDim.x)
        sDab[x] = M.D[(size_t)(bb.x + x / BC::NB) * N + bb.y + x % BC::NB];
      __syncthreads();
      j = tile * tq + q;
      valid = q < tq && j < __ldg(M.ket_count + i);
    }
    if (P.tau_mol != nullptr && valid) {
      // density-weighted screening of an incremental build: every term this
      // quartet adds is bounded by Q_ab Q_cd max|dD|, compared here with tau / max|dD|
      const float te = __ldg(P.tau_mol + mol_id);
      if (te > 0.0f && (float)(__ldg(M.bq + i) * __ldg(M.kq + j)) < te) valid = false;
    }
    const int4 bi = i >= 0 ? M.bra.idx[i] : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int a = 0; a < BC::NC; ++a) jb[a * kJKThreads] = Real(0);
    {
      const int4 ki = valid ? M.ket.idx[j] : make_int4(0, 0, 0, 0);
      const int nppb = valid ? M.bra.npp[i] : 0;
      const int nppk = valid ? M.ket.npp[j] : 0;
      const Real deg = Real((bi.z == bi.w ? 1 : 2) * (ki.z == ki.w ? 1 : 2) * ((P.same && i == j) ? 1 : 2));
      const size_t bstride = (size_t)M.bra.ppmax * M.bra.n;
      const Real* bpd = M.bra.pd + (i >= 0 ? i : 0);
      const Real* Dbra = M.D + (size_t)bi.x * N + bi.y;
      auto bra = [&](int f, int pp) -> Real {
        if constexpr (kFlat) return ldg_r(bpd + (size_t)f * bstride + (size_t)pp * M.bra.n);
        else return sbra[pp * NFB + f];
      };
      auto Dab = [&](int a) -> Real {
        if constexpr (kFlat) return ldg_r(Dbra + (size_t)(a / BC::NB) * N + a % BC::NB);
        else return sDab[a];
      };
      // Every thread of a chunk group runs the same chunk iterations (valid
      // quartet or not), so the group's named barrier below is always met.
#pragma unroll 1
      for (int ch = cg; ch < KetChunks<KC, CS>::NCH; ch += ncg) {
        if (valid)
          quartet_chunk<Real, LA, LB, LC, LD, CS>(so, bra, nppb, bs, ps, M.ket, j, nppk, sBoys, BK, P.boys64_T, ch);
        if (ps > 1) {
          // the ps threads of a quartet hold partial blocks over their bra
          // primitive pairs: sum them into the first thread's slots (each
          // element by one thread), which alone digests the chunk, so the
          // J/K atomics are issued once per quartet instead of ps times
          group_barrier(cg, gsz);
          if (valid) {
            Real* base = sOut + (threadIdx.x - bs);
            for (int x = bs; x < BC::NC * CS; x += ps) {
              Real acc = base[x * kJKThreads];
              for (int r = 1; r < ps; ++r) acc += base[x * kJKThreads + r];
              base[x * kJKThreads] = acc;
            }
          }
          group_barrier(cg, gsz);
        }
        if (!valid || bs != 0) continue;
        auto out = [&](int a, int cs) -> Real { return so[(a * CS + cs) * kJKThreads]; };
        // digestion (Eq. fock) of this chunk
#pragma unroll
        for (int cs = 0; cs < CS; ++cs) {
          const int c = ch * CS + cs;
          if (c >= KC::NC) break;
          const int lam = ki.x + c / KC::NB, sig = ki.y + c % KC::NB;
          // J_ket[la si] += sum_a D_ab v ; J_bra[a] += D_{la si} v
          const Real Dls = M.D[(size_t)lam * N + sig];
          Real jk = Real(0);
#pragma unroll
          for (int a = 0; a < BC::NC; ++a) {
            const Real v = deg * out(a, cs);
            jk = fma(Dab(a), v, jk);
            jb[a * kJKThreads] = fma(Dls, v, jb[a * kJKThreads]);
          }
          atomicAdd(&M.J[(size_t)lam * N + sig], (double)jk);
          // K: (mu la) += D_nu si v ; (nu si) += D_mu la v ; (mu si) += D_nu la v ; (nu la) += D_mu si v
#pragma unroll
          for (int ia = 0; ia < BC::NA; ++ia) {
            const int mu = bi.x + ia;
            Real k1 = Real(0), k3 = Real(0);
#pragma unroll
            for (int ib = 0; ib < BC::NB; ++ib) {
              const int nu = bi.y + ib;
              const Real v = deg * out(ia * BC::NB + ib, cs);
              k1 = fma(M.D[(size_t)nu * N + sig], v, k1);
              k3 = fma(M.D[(size_t)nu * N + lam], v, k3);
            }
            atomicAdd(&M.K[(size_t)mu * N + lam], (double)k1);
            atomicAdd(&M.K[(size_t)mu * N + sig], (double)k3);
          }
#pragma unroll
          for (int ib = 0; ib < BC::NB; ++ib) {
            const int nu = bi.y + ib;
            Real k2 = Real(0), k4 = Real(0);
#pragma unroll
            for (int ia = 0; ia < BC::NA; ++ia) {
              const int mu = bi.x + ia;
              const Real v = deg * out(ia * BC::NB + ib, cs);
              k2 = fma(M.D[(size_t)mu * N + lam], v, k2);
              k4 = fma(M.D[(size_t)mu * N + sig], v, k4);
            }
            atomicAdd(&M.K[(size_t)nu * N + sig], (double)k2);
            atomicAdd(&M.K[(size_t)nu * N + lam], (double)k4);
          }
        }
      }
    }
    if constexpr (kFlat) {
      // J_bra: when every active lane of the warp holds lane 0's bra, a warp
      // reduction and one FP64 add per element; otherwise each lane adds its own
      const int i0 = __shfl_sync(0xffffffffu, i, 0);
      if (__all_sync(0xffffffffu, i == i0 || i < 0)) {
        if (i0 >= 0) {
#pragma unroll
          for (int a = 0; a < BC::NC; ++a) {
            Real v = jb[a * kJKThreads];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += shfl_xor_r(v, o);
            if (lane == 0) atomicAdd(&M.J[(size_t)(bi.x + a / BC::NB) * N + bi.y + a % BC::NB], (double)v);
          }
        }
      } else if (i >= 0) {
#pragma unroll
        for (int a = 0; a < BC::NC; ++a)
          atomicAdd(&M.J[(size_t)(bi.x + a / BC::NB) * N + bi.y + a % BC::NB], (double)jb[a * kJKThreads]);
      }
    } else {
      // J_bra: warp reduction (every lane takes part, idle lanes hold zeros), one
      // shared-memory partial per warp and element, one FP64 global add per CTA
      // and element
      const int warp = threadIdx.x >> 5;
#pragma unroll
      for (int a = 0; a < BC::NC; ++a) {
        Real v = jb[a * kJKThreads];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += shfl_xor_r(v, o);
        if (lane == 0) sJw[warp * BC::NC + a] = v;
      }
      __syncthreads();
      for (int x = threadIdx.x; x < BC::NC; x += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < NWARP; ++w) v += (double)sJw[w * BC::NC + x];
        atomicAdd(&M.J[(size_t)(bi.x + x / BC::NB) * N + bi.y + x % BC::NB], v);
      }
    }
  }
}

}  // namespace fsim
