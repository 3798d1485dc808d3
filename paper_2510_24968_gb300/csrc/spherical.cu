// Real solid-harmonic (spherical) basis (paper Sec. 2.1.1: the contracted
// functions are real solid harmonics times Gaussians) on top of the Cartesian
// integral engine.
//
// A spherical function is a fixed combination of the normalised Cartesian
// components of its shell, phi_i = sum_a T_ia chi_a, so for any density in the
// spherical basis the Fock-build matrices follow exactly from the Cartesian ones:
//   D_cart = T^T D T,  J = T J_cart[D_cart] T^T,  K = T K_cart[D_cart] T^T,
// and one-electron matrices M = T M_cart T^T.  s and p shells are unchanged
// (p in x, y, z order).  A d shell (Cartesian order xx xy xz yy yz zz, each
// component unit-normalised, so <xx|yy> = 1/3 within the shell) gives, for
// m = -2 .. 2:
//   xy;  yz;  zz - (xx + yy)/2;  xz;  (sqrt 3 / 2)(xx - yy),
// the polynomials xy, yz, (2z^2 - x^2 - y^2)/2, xz, (x^2 - y^2)/2 written on the
// unit-normalised components; each has unit norm and the five are orthogonal
// (the sixth Cartesian combination, xx + yy + zz, is the r^2 s-type function
// that the spherical basis drops).
#include <cmath>

#include "fsim_internal.h"

namespace fsim {

namespace {

// out_sph[i][j] = sum_{a,b} T[i][a] T[j][b] in_cart[a][b]; T rows as (index, coef) x 3
__global__ void sph_from_cart_kernel(const double* __restrict__ in, int nc, double* __restrict__ out, int ns,
                                     const int* __restrict__ ti, const double* __restrict__ tc) {
  const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double ca = tc[i * 3 + a];
    if (ca == 0.0) continue;
    const double* row = in + (size_t)ti[i * 3 + a] * nc;
#pragma unroll
    for (int b = 0; b < 3; ++b) s += ca * tc[j * 3 + b] * row[ti[j * 3 + b]];
  }
  out[(size_t)i * ns + j] = s;
}

// out_cart[a][b] = sum_{i,j} T[i][a] T[j][b] in_sph[i][j]; T columns as (index, coef) x 2
__global__ void cart_from_sph_kernel(const double* __restrict__ in, int ns, double* __restrict__ out, int nc,
                                     const int* __restrict__ ci, const double* __restrict__ cc) {
  const int a = blockIdx.y, b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nc) return;
  double s = 0.0;
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const double ca = cc[a * 2 + x];
    if (ca == 0.0) continue;
    const double* row = in + (size_t)ci[a * 2 + x] * ns;
#pragma unroll
    for (int y = 0; y < 2; ++y) s += ca * cc[b * 2 + y] * row[ci[b * 2 + y]];
  }
  out[(size_t)a * nc + b] = s;
}

}  // namespace

// An f shell (Cartesian order xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz) gives,
// for m = -3 .. 3, the real solid harmonics
//   y(3x^2 - y^2), xyz, y(4z^2 - x^2 - y^2), z(2z^2 - 3x^2 - 3y^2),
//   x(4z^2 - x^2 - y^2), z(x^2 - y^2), x(x^2 - 3y^2),
// written on the unit-normalised components (a monomial x^i y^j z^k is its
// component times sqrt((2i-1)!!(2j-1)!!(2k-1)!!), up to the shell's common
// radial factor) and scaled to unit norm with the components' overlap within
// the shell, <a|b> = prod_axes (i_a + i_b - 1)!! / sqrt(prod (2i_a - 1)!! (2i_b - 1)!!)
// (zero when an exponent sum is odd).
namespace {
double dfact_odd(int n) {  // n!! for odd n >= -1
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}
struct Mono {
  int i, j, k;
  double c;
};
void f_rows(std::vector<std::vector<std::pair<int, double>>>& rows) {
  const std::vector<std::vector<Mono>> poly = {
      {{2, 1, 0, 3.0}, {0, 3, 0, -1.0}},
      {{1, 1, 1, 1.0}},
      {{0, 1, 2, 4.0}, {2, 1, 0, -1.0}, {0, 3, 0, -1.0}},
      {{0, 0, 3, 2.0}, {2, 0, 1, -3.0}, {0, 2, 1, -3.0}},
      {{1, 0, 2, 4.0}, {3, 0, 0, -1.0}, {1, 2, 0, -1.0}},
      {{2, 0, 1, 1.0}, {0, 2, 1, -1.0}},
      {{3, 0, 0, 1.0}, {1, 2, 0, -3.0}}};
  auto comp = [](int i, int j) {  // component index of (i, j, 3 - i - j) in the shell's order
    int n = 0;
    for (int a = 3; a >= 0; --a)
      for (int b = 3 - a; b >= 0; --b) {
        if (a == i && b == j) return n;
        ++n;
      }
    return -1;
  };
  rows.clear();
  for (const auto& P : poly) {
    std::vector<Mono> t;
    for (const Mono& m : P)
      t.push_back(Mono{m.i, m.j, m.k, m.c * std::sqrt(dfact_odd(2 * m.i - 1) * dfact_odd(2 * m.j - 1) *
                                                     dfact_odd(2 * m.k - 1))});
    double n2 = 0.0;
    for (const Mono& x : t)
      for (const Mono& y : t) {
        if ((x.i + y.i) % 2 || (x.j + y.j) % 2 || (x.k + y.k) % 2) continue;
        const double ov = dfact_odd(x.i + y.i - 1) * dfact_odd(x.j + y.j - 1) * dfact_odd(x.k + y.k - 1) /
                          std::sqrt(dfact_odd(2 * x.i - 1) * dfact_odd(2 * x.j - 1) * dfact_odd(2 * x.k - 1) *
                                    dfact_odd(2 * y.i - 1) * dfact_odd(2 * y.j - 1) * dfact_odd(2 * y.k - 1));
        n2 += x.c * y.c * ov;
      }
    std::vector<std::pair<int, double>> row;
    for (const Mono& x : t) row.push_back({comp(x.i, x.j), x.c / std::sqrt(n2)});
    rows.push_back(row);
  }
}
}  // namespace

int sph_setup(fsim_basis* b) {
  std::vector<std::vector<std::pair<int, double>>> frows;
  f_rows(frows);
  const double h = 0.5, r3 = std::sqrt(3.0) / 2.0;
  std::vector<int> ti, ci((size_t)b->nbf * 2, 0);
  std::vector<double> tc, cc((size_t)b->nbf * 2, 0.0);
  std::vector<int> nci(b->nbf, 0);
  auto add = [&](int i, int a, double c) {  // T[i][a] = c
    int k = 0;
    while (tc[(size_t)i * 3 + k] != 0.0) ++k;
    ti[(size_t)i * 3 + k] = a;
    tc[(size_t)i * 3 + k] = c;
    const int m = nci[a]++;
    ci[(size_t)a * 2 + m] = i;
    cc[(size_t)a * 2 + m] = c;
  };
  int ns = 0;
  for (int s = 0; s < b->nshell; ++s) ns += 2 * b->sh_l[s] + 1;
  ti.assign((size_t)ns * 3, 0);
  tc.assign((size_t)ns * 3, 0.0);
  int i = 0;
  for (int s = 0; s < b->nshell; ++s) {
    const int c0 = b->sh_ao[s];
    if (b->sh_l[s] < 2) {
      for (int k = 0; k < ncart(b->sh_l[s]); ++k) add(i++, c0 + k, 1.0);
    } else if (b->sh_l[s] == 3) {
      for (const auto& row : frows) {
        for (const auto& e : row) add(i, c0 + e.first, e.second);
        ++i;
      }
    } else {  // xx 0, xy 1, xz 2, yy 3, yz 4, zz 5
      add(i, c0 + 1, 1.0);
      ++i;
      add(i, c0 + 4, 1.0);
      ++i;
      add(i, c0 + 5, 1.0);
      add(i, c0 + 0, -h);
      add(i, c0 + 3, -h);
      ++i;
      add(i, c0 + 2, 1.0);
      ++i;
      add(i, c0 + 0, r3);
      add(i, c0 + 3, -r3);
      ++i;
    }
  }
  b->nsph = ns;
  int rc;
  if ((rc = dev_alloc(&b->d_sti, ti.size())) != FSIM_OK) return rc;
  if ((rc = dev_alloc(&b->d_stc, tc.size())) != FSIM_OK) return rc;
  if ((rc = dev_alloc(&b->d_sci, ci.size())) != FSIM_OK) return rc;
  if ((rc = dev_alloc(&b->d_scc, cc.size())) != FSIM_OK) return rc;
  FSIM_CK(cudaMemcpy(b->d_sti, ti.data(), sizeof(int) * ti.size(), cudaMemcpyHostToDevice));
  FSIM_CK(cudaMemcpy(b->d_stc, tc.data(), sizeof(double) * tc.size(), cudaMemcpyHostToDevice));
  FSIM_CK(cudaMemcpy(b->d_sci, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice));
  FSIM_CK(cudaMemcpy(b->d_scc, cc.data(), sizeof(double) * cc.size(), cudaMemcpyHostToDevice));
  return FSIM_OK;
}

static int ensure_cart_scratch(fsim_basis* b) {
  const size_t n2 = (size_t)b->nbf * b->nbf;
  if (!b->d_cD) FSIM_TRY(dev_alloc(&b->d_cD, n2));
  if (!b->d_cJ) FSIM_TRY(dev_alloc(&b->d_cJ, n2));
  if (!b->d_cK) FSIM_TRY(dev_alloc(&b->d_cK, n2));
  return FSIM_OK;
}

static cudaError_t to_sph(const fsim_basis* b, const double* in, double* out, cudaStream_t s) {
  dim3 g((b->nsph + 127) / 128, b->nsph);
  sph_from_cart_kernel<<<g, 128, 0, s>>>(in, b->nbf, out, b->nsph, b->d_sti, b->d_stc);
  return cudaGetLastError();
}

int onee_ext_device(fsim_basis* b, int which, double* out, cudaStream_t s) {
  if (!b->spherical) return onee_device(b, which, out, s);
  FSIM_TRY(ensure_cart_scratch(b));
  FSIM_TRY(onee_device(b, which, b->d_cJ, s));
  FSIM_CK(to_sph(b, b->d_cJ, out, s));
  return FSIM_OK;
}

int fock_build_ext_device(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o) {
  if (!b->spherical) return fock_build_device(b, dD, dJ, dK, o);
  FSIM_TRY(ensure_cart_scratch(b));
  cudaStream_t s = (cudaStream_t)o.stream;
  dim3 g((b->nbf + 127) / 128, b->nbf);
  cart_from_sph_kernel<<<g, 128, 0, s>>>(dD, b->nsph, b->d_cD, b->nbf, b->d_sci, b->d_scc);
  FSIM_CK(cudaGetLastError());
  FSIM_TRY(fock_build_device(b, b->d_cD, b->d_cJ, b->d_cK, o));
  FSIM_CK(to_sph(b, b->d_cJ, dJ, s));
  FSIM_CK(to_sph(b, b->d_cK, dK, s));
  return FSIM_OK;
}

}  // namespace fsim
