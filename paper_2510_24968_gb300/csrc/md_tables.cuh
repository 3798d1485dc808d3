// Compile-time index tables for the McMurchie-Davidson scheme (paper Sec. 2.1.3,
// 2.3.4, 2.5).  Everything here is constexpr so that, inside fully unrolled
// kernel loops, every Cartesian/Hermite index is a constant and the per-class
// arrays live in registers.
//
// Conventions
//  * Cartesian components of a shell of angular momentum l are ordered
//    lexicographically descending: p = x y z, d = xx xy xz yy yz zz.
//  * A shell pair (A, B) has la >= lb; its Cartesian block index is
//    a = ia * ncart(lb) + ib.
//  * Hermite triples (t, u, v) with t + u + v <= L are stored at
//    hidx(t,u,v) = n(n+1)(n+2)/6 + m(m+1)/2 + v, n = t+u+v, m = u+v.
//  * For a pair component a, the Hermite coefficient product
//      E^{ab}_{tuv} = E^{ix jx}_t E^{iy jy}_u E^{iz jz}_v            (Eq. E-tuv)
//    is non-zero only for t <= ix+jx, u <= iy+jy, v <= iz+jz; only these
//    "non-zeros" are stored, component after component, t-major.
#pragma once

namespace fsim {

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

__host__ __device__ constexpr int cart_comp(int l, int c, int axis) {
  int n = 0;
  for (int a = l; a >= 0; --a)
    for (int b = l - a; b >= 0; --b) {
      if (n == c) return axis == 0 ? a : (axis == 1 ? b : l - a - b);
      ++n;
    }
  return 0;
}

__host__ __device__ constexpr int hidx(int t, int u, int v) {
  int n = t + u + v, m = u + v;
  return n * (n + 1) * (n + 2) / 6 + m * (m + 1) / 2 + v;
}

// Pair class (LA >= LB).
template <int LA, int LB>
struct PairCls {
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = NA * NB;
  static constexpr int L = LA + LB, NH = nherm(LA + LB);
  // Hermite extent per axis of component a
  __host__ __device__ static constexpr int ext(int a, int axis) {
    return cart_comp(LA, a / NB, axis) + cart_comp(LB, a % NB, axis);
  }
  __host__ __device__ static constexpr int nnz(int a) {
    return (ext(a, 0) + 1) * (ext(a, 1) + 1) * (ext(a, 2) + 1);
  }
  __host__ __device__ static constexpr int off(int a) {
    int s = 0;
    for (int k = 0; k < a; ++k) s += nnz(k);
    return s;
  }
  static constexpr int NNZ = off(NC);
  // the k-th non-zero of component a: its (t, u, v)
  __host__ __device__ static constexpr int nz_t(int a, int k) {
    return k / ((ext(a, 1) + 1) * (ext(a, 2) + 1));
  }
  __host__ __device__ static constexpr int nz_u(int a, int k) {
    return (k / (ext(a, 2) + 1)) % (ext(a, 1) + 1);
  }
  __host__ __device__ static constexpr int nz_v(int a, int k) { return k % (ext(a, 2) + 1); }
};

// Pair classes: the six s/p/d classes ss, ps, pp, ds, dp, dd (indices 0..5,
// served by the compile-time kernels) and the four f classes fs, fp, fd, ff
// (6..9, served by the runtime-angular-momentum kernel of generic.cuh).
constexpr int kNumPairCls = 6;
constexpr int kNumPairClsAll = 10;
__host__ __device__ constexpr int pair_cls_index(int la, int lb) {
  return la == 3 ? 6 + lb
                 : (la == 0 ? 0 : (la == 1 ? (lb == 0 ? 1 : 2) : (lb == 0 ? 3 : (lb == 1 ? 4 : 5))));
}
__host__ __device__ constexpr int pair_cls_la(int c) { return c >= 6 ? 3 : (c == 0 ? 0 : (c <= 2 ? 1 : 2)); }
__host__ __device__ constexpr int pair_cls_lb(int c) {
  return c >= 6 ? c - 6 : (c == 0 ? 0 : (c == 1 ? 0 : (c == 2 ? 1 : (c == 3 ? 0 : (c == 4 ? 1 : 2)))));
}
// non-zero E^{ab}_{tuv} over the Cartesian components of a pair class
__host__ __device__ constexpr int pair_cls_nnz(int c) {
  const int la = pair_cls_la(c), lb = pair_cls_lb(c);
  int s = 0;
  for (int a = 0; a < ncart(la) * ncart(lb); ++a) {
    int e = 1;
    for (int x = 0; x < 3; ++x) e *= cart_comp(la, a / ncart(lb), x) + cart_comp(lb, a % ncart(lb), x) + 1;
    s += e;
  }
  return s;
}

}  // namespace fsim

#include <utility>

namespace fsim {

// inverse of hidx: (t, u, v) of the h-th Hermite triple
__host__ __device__ constexpr int herm_t(int h) {
  for (int n = 0; n < 32; ++n)
    for (int m = 0; m <= n; ++m)
      for (int v = 0; v <= m; ++v)
        if (hidx(n - m, m - v, v) == h) return n - m;
  return -1;
}
__host__ __device__ constexpr int herm_u(int h) {
  for (int n = 0; n < 32; ++n)
    for (int m = 0; m <= n; ++m)
      for (int v = 0; v <= m; ++v)
        if (hidx(n - m, m - v, v) == h) return m - v;
  return -1;
}
__host__ __device__ constexpr int herm_v(int h) {
  for (int n = 0; n < 32; ++n)
    for (int m = 0; m <= n; ++m)
      for (int v = 0; v <= m; ++v)
        if (hidx(n - m, m - v, v) == h) return v;
  return -1;
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1.
template <class F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (N > 0) static_for_impl(f, std::make_integer_sequence<int, N>{});
}

}  // namespace fsim
