// Basis creation, shell-pair data, Schwarz bounds and one-electron integrals.
//
//  * normalisation of contracted Cartesian Gaussians (paper Sec. 2.1.1)
//  * shell-pair data: Gaussian product theorem (Sec. 2.1.2) and Hermite
//    expansion coefficients E^{ij}_t (Sec. 2.1.3, Eqs. recurrence-A/B),
//    collapsed per Cartesian component pair (Sec. 2.5, Eq. E-tuv) and stored
//    as non-zeros only
//  * Schwarz bounds Q_ab = sqrt(max |(mu nu|mu nu)|) with the ERI kernels
//  * S, T, V (Sec. 2.3.1-2.3.3, Eqs. s-overall, Tab-final, Vab-final)
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <numeric>

#include "fsim_internal.h"
#include "pairdata.cuh"

namespace fsim {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error() { return g_last_error.c_str(); }

constexpr double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// Boys table F_m(T_i), m < kBoysCols: a high order by the convergent series in
// long double, then the downward recursion F_m = (2T F_{m+1} + e^{-T})/(2m+1).
// ---------------------------------------------------------------------------
static void boys_table(std::vector<double>& tab, int npts, double h) {
  const int Mtop = kBoysCols - 1 + 24;
  tab.assign((size_t)npts * kBoysCols, 0.0);
  std::vector<long double> F(Mtop + 1);
  for (int i = 0; i < npts; ++i) {
    long double T = (long double)i * h;
    long double term = 1.0L / (2 * Mtop + 1), sum = term;
    for (int k = 1; k < 4000; ++k) {
      term *= 2.0L * T / (2 * Mtop + 2 * k + 1);
      sum += term;
      if (term < 1e-24L * sum) break;
    }
    long double e = expl(-T);
    F[Mtop] = e * sum;
    for (int m = Mtop - 1; m >= 0; --m) F[m] = (2.0L * T * F[m + 1] + e) / (2 * m + 1);
    for (int m = 0; m < kBoysCols; ++m) tab[(size_t)i * kBoysCols + m] = (double)F[m];
  }
}

static cudaError_t launch_pair_data(int cls, int n, int ppmax, const int4* idx, const fsim_basis* b, double* pd64,
                                    float* pd32, double4_32a* pq64, float4* pq32) {
  const int total = n * ppmax, th = 128, bl = (total + th - 1) / th;
  if (total == 0) return cudaSuccess;
  switch (cls) {
    case 0: pair_data_kernel<0, 0><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 1: pair_data_kernel<1, 0><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 2: pair_data_kernel<1, 1><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 3: pair_data_kernel<2, 0><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 4: pair_data_kernel<2, 1><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    case 5: pair_data_kernel<2, 2><<<bl, th>>>(n, ppmax, idx, b->d_cen, b->d_alpha, b->d_coef, b->d_nprim, pd64, pd32, pq64, pq32); break;
    default: return launch_pair_data_f(cls, n, ppmax, idx, b, pd64, pd32, pq64, pq32);
  }
  return cudaGetLastError();
}

// (Re)build the device data of pair class `cls` in the given pair order.
int build_pair_data(fsim_basis* b, int cls, const std::vector<int4>& order) {
  DevClass& C = b->cls[cls];
  dev_free(C.idx); dev_free(C.npp); dev_free(C.pd64); dev_free(C.pd32); dev_free(C.pq64); dev_free(C.pq32);
  dev_free(C.pdx); dev_free(C.pqx);
  b->dfloat_ready = false;  // the double-float copies follow the pair order; remade on next use
  C.n = (int)order.size();
  C.nnz = pair_cls_nnz(cls);
  C.h_idx = order;
  C.h_npp.resize(C.n);
  C.ppmax = 1;
  for (int j = 0; j < C.n; ++j) {
    C.h_npp[j] = b->sh_nprim[order[j].z] * b->sh_nprim[order[j].w];
    C.ppmax = std::max(C.ppmax, C.h_npp[j]);
  }
  if (C.n == 0) return FSIM_OK;
  FSIM_TRY(dev_alloc(&C.idx, C.n));
  FSIM_TRY(dev_alloc(&C.npp, C.n));
  FSIM_TRY(dev_alloc(&C.pd64, (size_t)C.nfield() * C.ppmax * C.n));
  FSIM_TRY(dev_alloc(&C.pd32, (size_t)C.nfield() * C.ppmax * C.n));
  FSIM_TRY(dev_alloc(&C.pq64, (size_t)C.ppmax * C.n));
  FSIM_TRY(dev_alloc(&C.pq32, (size_t)C.ppmax * C.n));
  FSIM_CK(cudaMemcpy(C.idx, order.data(), sizeof(int4) * C.n, cudaMemcpyHostToDevice));
  FSIM_CK(cudaMemcpy(C.npp, C.h_npp.data(), sizeof(int) * C.n, cudaMemcpyHostToDevice));
  FSIM_CK(launch_pair_data(cls, C.n, C.ppmax, C.idx, b, C.pd64, C.pd32, C.pq64, C.pq32));
  return FSIM_OK;
}

// Double-float copies (nearest dfloat of each FP64 value) of the pair data, the
// Boys table and a density buffer, made once on the first FSIM_DFLOAT build.
__global__ void split_kernel(const double* __restrict__ in, dfloat* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = dsplit_rn(in[i]);
}

__global__ void split4_kernel(const double4_32a* __restrict__ in, dfloat4* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double4_32a v = in[i];
    out[i] = dfloat4{dsplit_rn(v.x), dsplit_rn(v.y), dsplit_rn(v.z), dsplit_rn(v.w)};
  }
}

// The double-float table keeps e^{-T_i} in its last column (an order no class
// reaches), read by the double-float Boys function.
__global__ void boys_exp_column_kernel(dfloat* __restrict__ tab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kBoysN64; i += gridDim.x * blockDim.x)
    tab[(size_t)i * kBoysCols + kBoysCols - 1] = dsplit_rn(exp(-i * kBoysH64));
}

void launch_split(const double* in, dfloat* out, size_t n, cudaStream_t s) {
  if (n) split_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 1024), 256, 0, s>>>(in, out, n);
}

int ensure_dfloat(fsim_basis* b) {
  if (b->dfloat_ready) return FSIM_OK;
  for (int X = 0; X < kNumPairCls; ++X) {
    DevClass& C = b->cls[X];
    if (C.n == 0) continue;
    const size_t nf = (size_t)C.nfield() * C.ppmax * C.n, nq = (size_t)C.ppmax * C.n;
    if (!C.pdx) FSIM_TRY(dev_alloc(&C.pdx, nf));
    if (!C.pqx) FSIM_TRY(dev_alloc(&C.pqx, nq));
    launch_split(C.pd64, C.pdx, nf, 0);
    split4_kernel<<<(unsigned)std::min<size_t>((nq + 255) / 256, 1024), 256>>>(C.pq64, C.pqx, nq);
  }
  const size_t nb = (size_t)kBoysN64 * kBoysCols;
  if (!b->d_boysx) {
    FSIM_TRY(dev_alloc(&b->d_boysx, nb));
    launch_split(b->d_boys64, b->d_boysx, nb, 0);
    boys_exp_column_kernel<<<(kBoysN64 + 127) / 128, 128>>>(b->d_boysx);
  }
  if (!b->d_Dx) FSIM_TRY(dev_alloc(&b->d_Dx, (size_t)b->nbf * b->nbf));
  FSIM_CK(cudaGetLastError());
  FSIM_CK(cudaDeviceSynchronize());
  b->dfloat_ready = true;
  return FSIM_OK;
}

// ---------------------------------------------------------------------------
// One-electron integrals: one block per ordered shell pair, one thread per
// Cartesian component pair.  Runtime loops (not on the hot path).
// ---------------------------------------------------------------------------
// E^{ij}_t of one axis for i <= la <= 3, j <= lb <= 5 (the kinetic term raises j by 2)
__device__ void herm_E_axis(double (&E)[4][6][9], int la, int lb, double a, double b, double XAB) {
  const double p = a + b, mu = a * b / p, XPA = -b * XAB / p, XPB = a * XAB / p, i2p = 0.5 / p;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 6; ++j)
      for (int t = 0; t < 9; ++t) E[i][j][t] = 0.0;
  E[0][0][0] = exp(-mu * XAB * XAB);
  for (int i = 1; i <= la; ++i)
    for (int t = 0; t <= i; ++t)
      E[i][0][t] = (t > 0 ? i2p * E[i - 1][0][t - 1] : 0.0) + (t <= i - 1 ? XPA * E[i - 1][0][t] : 0.0) +
                   (t + 1 <= i - 1 ? (t + 1) * E[i - 1][0][t + 1] : 0.0);
  for (int j = 1; j <= lb; ++j)
    for (int i = 0; i <= la; ++i)
      for (int t = 0; t <= i + j; ++t)
        E[i][j][t] = (t > 0 ? i2p * E[i][j - 1][t - 1] : 0.0) + (t <= i + j - 1 ? XPB * E[i][j - 1][t] : 0.0) +
                     (t + 1 <= i + j - 1 ? (t + 1) * E[i][j - 1][t + 1] : 0.0);
}

__global__ void onee_kernel(int which, int nshell, const int* __restrict__ lsh, const int* __restrict__ nprim,
                            const int* __restrict__ ao, const double* __restrict__ cen,
                            const double* __restrict__ alpha, const double* __restrict__ coef, int natom,
                            const double* __restrict__ axyz, const int* __restrict__ Zn,
                            const double* __restrict__ boys, int N, double* __restrict__ out) {
  const int sa = blockIdx.x / nshell, sb = blockIdx.x % nshell;
  const int la = lsh[sa], lb = lsh[sb], nb = ncart(lb);
  const int c = threadIdx.x;
  if (c >= ncart(la) * nb) return;
  const int ia = c / nb, ib = c % nb;
  int i3[3], j3[3];
  for (int x = 0; x < 3; ++x) {
    i3[x] = cart_comp(la, ia, x);
    j3[x] = cart_comp(lb, ib, x);
  }
  const double fn = comp_norm(la, ia) * comp_norm(lb, ib);
  double sum = 0.0;
  for (int ka = 0; ka < nprim[sa]; ++ka)
    for (int kb = 0; kb < nprim[sb]; ++kb) {
      const double a = alpha[sa * kMaxPrim + ka], b = alpha[sb * kMaxPrim + kb], p = a + b;
      double E[3][4][6][9];
      double P[3];
      for (int x = 0; x < 3; ++x) {
        herm_E_axis(E[x], la, lb + (which == 1 ? 2 : 0), a, b, cen[3 * sa + x] - cen[3 * sb + x]);
        P[x] = (a * cen[3 * sa + x] + b * cen[3 * sb + x]) / p;
      }
      double val = 0.0;
      if (which == 0) {
        val = E[0][i3[0]][j3[0]][0] * E[1][i3[1]][j3[1]][0] * E[2][i3[2]][j3[2]][0] * pow(kPi / p, 1.5);
      } else if (which == 1) {
        double S[3], T[3];
        for (int x = 0; x < 3; ++x) {
          const int i = i3[x], j = j3[x];
          S[x] = E[x][i][j][0];
          T[x] = -2.0 * b * b * E[x][i][j + 2][0] + b * (2 * j + 1) * E[x][i][j][0] -
                 (j >= 2 ? 0.5 * j * (j - 1) * E[x][i][j - 2][0] : 0.0);
        }
        val = (T[0] * S[1] * S[2] + S[0] * T[1] * S[2] + S[0] * S[1] * T[2]) * pow(kPi / p, 1.5);
      } else {
        const int L = la + lb;
        for (int nuc = 0; nuc < natom; ++nuc) {
          const double X = P[0] - axyz[3 * nuc], Y = P[1] - axyz[3 * nuc + 1], Z = P[2] - axyz[3 * nuc + 2];
          double F[7];
          boys_fp64<6>(p * (X * X + Y * Y + Z * Z), F, boys + 6, kBoysCols);
          // R^n_{tuv} for n + t + u + v <= L: level arrays, highest n first
          double R[7][84];
          for (int n = L; n >= 0; --n) {
            double fac = 1.0;
            for (int m = 0; m < n; ++m) fac *= -2.0 * p;
            R[n][0] = fac * F[n];
            for (int s = 1; s <= L - n; ++s)
              for (int t = 0; t <= s; ++t)
                for (int u = 0; u <= s - t; ++u) {
                  const int v = s - t - u;
                  double r;
                  if (t > 0) r = X * R[n + 1][hidx(t - 1, u, v)] + (t > 1 ? (t - 1) * R[n + 1][hidx(t - 2, u, v)] : 0.0);
                  else if (u > 0) r = Y * R[n + 1][hidx(t, u - 1, v)] + (u > 1 ? (u - 1) * R[n + 1][hidx(t, u - 2, v)] : 0.0);
                  else r = Z * R[n + 1][hidx(t, u, v - 1)] + (v > 1 ? (v - 1) * R[n + 1][hidx(t, u, v - 2)] : 0.0);
                  R[n][hidx(t, u, v)] = r;
                }
          }
          double s = 0.0;
          for (int t = 0; t <= i3[0] + j3[0]; ++t)
            for (int u = 0; u <= i3[1] + j3[1]; ++u)
              for (int v = 0; v <= i3[2] + j3[2]; ++v)
                s += E[0][i3[0]][j3[0]][t] * E[1][i3[1]][j3[1]][u] * E[2][i3[2]][j3[2]][v] * R[0][hidx(t, u, v)];
          val += -Zn[nuc] * (2.0 * kPi / p) * s;
        }
      }
      sum += coef[sa * kMaxPrim + ka] * coef[sb * kMaxPrim + kb] * val;
    }
  out[(size_t)(ao[sa] + ia) * N + ao[sb] + ib] = fn * sum;
}

int onee_device(fsim_basis* b, int which, double* d_out, cudaStream_t s) {
  if (which < 0 || which > 2) {
    set_error("fsim_onee: which must be 0 (S), 1 (T) or 2 (V)");
    return FSIM_EINVAL;
  }
  onee_kernel<<<b->nshell * b->nshell, 128, 0, s>>>(which, b->nshell, b->d_l, b->d_nprim, b->d_ao, b->d_cen,
                                                    b->d_alpha, b->d_coef, b->natom, b->d_axyz, b->d_Z, b->d_boys64,
                                                    b->nbf, d_out);
  FSIM_CK(cudaGetLastError());
  return FSIM_OK;
}

// ---------------------------------------------------------------------------
// Schwarz bounds: diagonal quartets (ab|ab) through the list kernels (FP64).
// ---------------------------------------------------------------------------
static int compute_schwarz(fsim_basis* b) {
  const int ns = b->nshell;
  b->Q.assign((size_t)ns * ns, 0.0);
  for (int X = 0; X < kNumPairClsAll; ++X) {
    DevClass& C = b->cls[X];
    if (C.n == 0) continue;
    const int nc = ncart(pair_cls_la(X)) * ncart(pair_cls_lb(X));
    std::vector<int2> items(C.n);
    for (int j = 0; j < C.n; ++j) items[j] = make_int2(j, j);
    double* d_out = nullptr;
    FSIM_TRY(dev_alloc(&d_out, (size_t)C.n * nc * nc));
    int rc = run_list(b, X, X, items, d_out, FSIM_FP64, 0);
    std::vector<double> h((size_t)C.n * nc * nc);
    if (rc == FSIM_OK && cudaMemcpy(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = FSIM_ECUDA;
    dev_free(d_out);
    if (rc != FSIM_OK) return rc;
    std::vector<double> q(C.n);
    for (int j = 0; j < C.n; ++j) {
      double m = 0.0;
      for (int a = 0; a < nc; ++a) m = std::max(m, std::fabs(h[(size_t)j * nc * nc + a * nc + a]));
      q[j] = std::sqrt(m);
      const int sa = C.h_idx[j].z, sb = C.h_idx[j].w;
      b->Q[(size_t)sa * ns + sb] = b->Q[(size_t)sb * ns + sa] = q[j];
    }
    // sort the class by Q descending (stable) and rebuild its device data in that order
    std::vector<int> perm(C.n);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return q[x] > q[y]; });
    std::vector<int4> order(C.n);
    C.h_Q.resize(C.n);
    for (int j = 0; j < C.n; ++j) {
      order[j] = C.h_idx[perm[j]];
      C.h_Q[j] = q[perm[j]];
    }
    FSIM_TRY(build_pair_data(b, X, order));
    if (!C.d_Q) FSIM_TRY(dev_alloc(&C.d_Q, std::max(C.n, 1)));
    if (C.n) FSIM_CK(cudaMemcpy(C.d_Q, C.h_Q.data(), sizeof(double) * C.n, cudaMemcpyHostToDevice));
  }
  FSIM_CK(cudaDeviceSynchronize());
  b->schwarz_done = true;
  return FSIM_OK;
}

int ensure_schwarz(fsim_basis* b) { return b->schwarz_done ? FSIM_OK : compute_schwarz(b); }

}  // namespace fsim

using namespace fsim;

extern "C" {

const char* fsim_last_error(void) { return fsim::last_error(); }

int fsim_basis_create(const fsim_atom* atoms, int natom, const fsim_shell_desc* shells, int nshell,
                      fsim_basis** out) {
  return fsim_basis_create_ex(atoms, natom, shells, nshell, 0, out);
}

int fsim_basis_create_ex(const fsim_atom* atoms, int natom, const fsim_shell_desc* shells, int nshell, int flags,
                         fsim_basis** out) {
  if (out) *out = nullptr;
  if (flags & ~FSIM_BASIS_SPHERICAL) {
    set_error("fsim_basis_create_ex: unknown flags %#x", flags);
    return FSIM_EINVAL;
  }
  if (!out || !atoms || !shells || natom <= 0 || nshell <= 0) {
    set_error("fsim_basis_create: null pointer or empty input");
    return FSIM_EINVAL;
  }
  *out = nullptr;
  for (int s = 0; s < nshell; ++s) {
    const fsim_shell_desc& d = shells[s];
    if (d.atom < 0 || d.atom >= natom || d.l < 0 || d.l > 3 || d.nprim < 1 || d.nprim > kMaxPrim || !d.alpha ||
        !d.coef) {
      set_error("fsim_basis_create: shell %d invalid (atom %d, l %d, nprim %d; need l<=3, 1<=nprim<=%d)", s, d.atom,
                d.l, d.nprim, kMaxPrim);
      return FSIM_EINVAL;
    }
    for (int k = 0; k < d.nprim; ++k)
      if (!(d.alpha[k] > 0.0)) {
        set_error("fsim_basis_create: shell %d has a non-positive exponent", s);
        return FSIM_EINVAL;
      }
  }
  fsim_basis* b = new fsim_basis();
  cudaGetDevice(&b->device);
  b->natom = natom;
  b->nshell = nshell;
  for (int a = 0; a < natom; ++a) {
    b->Z.push_back(atoms[a].Z);
    for (int x = 0; x < 3; ++x) b->axyz.push_back(atoms[a].xyz[x]);
  }
  b->sh_alpha.assign((size_t)nshell * kMaxPrim, 1.0);
  b->sh_coef.assign((size_t)nshell * kMaxPrim, 0.0);
  std::vector<double> cen(3 * nshell);
  int off = 0;
  for (int s = 0; s < nshell; ++s) {
    const fsim_shell_desc& d = shells[s];
    b->sh_atom.push_back(d.atom);
    b->sh_l.push_back(d.l);
    b->sh_nprim.push_back(d.nprim);
    b->sh_ao.push_back(off);
    off += ncart(d.l);
    for (int x = 0; x < 3; ++x) cen[3 * s + x] = atoms[d.atom].xyz[x];
    // primitive factor (2a/pi)^{3/4} (4a)^{l/2}; contraction renormalised with the
    // overlap of two normalised same-centre primitives (2 sqrt(ab)/(a+b))^{l+3/2}
    double S = 0.0;
    for (int k = 0; k < d.nprim; ++k)
      for (int m = 0; m < d.nprim; ++m)
        S += d.coef[k] * d.coef[m] *
             std::pow(2.0 * std::sqrt(d.alpha[k] * d.alpha[m]) / (d.alpha[k] + d.alpha[m]), d.l + 1.5);
    if (!(S > 0.0)) {
      delete b;
      set_error("fsim_basis_create: shell %d has zero norm", s);
      return FSIM_EINVAL;
    }
    for (int k = 0; k < d.nprim; ++k) {
      b->sh_alpha[s * kMaxPrim + k] = d.alpha[k];
      b->sh_coef[s * kMaxPrim + k] = d.coef[k] * std::pow(2.0 * d.alpha[k] / kPi, 0.75) *
                                     std::pow(4.0 * d.alpha[k], 0.5 * d.l) / std::sqrt(S);
    }
  }
  b->nbf = off;
  auto fail = [&](int rc) {
    fsim_basis_destroy(b);
    return rc;
  };
  int rc;
#define UP(dst, src, n)                                                                        \
  if ((rc = dev_alloc(&dst, n)) != FSIM_OK) return fail(rc);                                  \
  if (cudaMemcpy(dst, src, sizeof(*dst) * (n), cudaMemcpyHostToDevice) != cudaSuccess) {      \
    set_error("fsim_basis_create: upload failed");                                             \
    return fail(FSIM_ECUDA);                                                                   \
  }
  UP(b->d_cen, cen.data(), cen.size());
  UP(b->d_alpha, b->sh_alpha.data(), b->sh_alpha.size());
  UP(b->d_coef, b->sh_coef.data(), b->sh_coef.size());
  UP(b->d_nprim, b->sh_nprim.data(), b->sh_nprim.size());
  UP(b->d_l, b->sh_l.data(), b->sh_l.size());
  UP(b->d_ao, b->sh_ao.data(), b->sh_ao.size());
  UP(b->d_axyz, b->axyz.data(), b->axyz.size());
  UP(b->d_Z, b->Z.data(), b->Z.size());
  {
    std::vector<double> t64, t32d;
    boys_table(t64, kBoysN64, kBoysH64);
    boys_table(t32d, kBoysN32, (double)kBoysH32);
    std::vector<float> t32(t32d.begin(), t32d.end());
    UP(b->d_boys64, t64.data(), t64.size());
    UP(b->d_boys32, t32.data(), t32.size());
  }
#undef UP
  // canonical pairs per class: higher l first; equal l: higher shell index first
  std::vector<int4> order[kNumPairClsAll];
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb <= sa; ++sb) {
      int A = sa, B = sb;
      if (b->sh_l[B] > b->sh_l[A]) std::swap(A, B);
      const int X = pair_cls_index(b->sh_l[A], b->sh_l[B]);
      order[X].push_back(make_int4(b->sh_ao[A], b->sh_ao[B], A, B));
    }
  for (int X = 0; X < kNumPairClsAll; ++X)
    if ((rc = build_pair_data(b, X, order[X])) != FSIM_OK) return fail(rc);
  if (flags & FSIM_BASIS_SPHERICAL) {
    b->spherical = 1;
    if ((rc = sph_setup(b)) != FSIM_OK) return fail(rc);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error("fsim_basis_create: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(FSIM_ECUDA);
  }
  *out = b;
  return FSIM_OK;
}

void fsim_basis_destroy(fsim_basis* b) {
  if (!b) return;
  for (auto& C : b->cls) {
    dev_free(C.idx); dev_free(C.npp); dev_free(C.pd64); dev_free(C.pd32); dev_free(C.pq64); dev_free(C.pq32);
    dev_free(C.pdx); dev_free(C.pqx); dev_free(C.d_Q);
  }
  for (auto* p : b->plans) {
    for (auto& row : p->cp)
      for (auto& cp : row) {
        dev_free(cp.d_prefix);
        dev_free(cp.d_count);
      }
    delete p;
  }
  for (auto* p : b->jplans) {
    for (auto& row : p->cp)
      for (auto& cp : row) {
        dev_free(cp.d_prefix);
        dev_free(cp.d_count);
      }
    delete p;
  }
  for (int X = 0; X < kNumPairCls; ++X) {
    dev_free(b->d_rho32[X]);
    dev_free(b->d_rho64[X]);
  }
  dev_free(b->d_cen); dev_free(b->d_alpha); dev_free(b->d_coef); dev_free(b->d_nprim);
  dev_free(b->d_l); dev_free(b->d_ao); dev_free(b->d_axyz); dev_free(b->d_Z);
  dev_free(b->d_boys64); dev_free(b->d_boys32); dev_free(b->d_boysx); dev_free(b->d_Dx);
  dev_free(b->d_Jacc); dev_free(b->d_Kacc); dev_free(b->d_D); dev_free(b->d_J); dev_free(b->d_K);
  dev_free(b->d_D32);
  dev_free(b->d_sti); dev_free(b->d_stc); dev_free(b->d_sci); dev_free(b->d_scc);
  dev_free(b->d_cD); dev_free(b->d_cJ); dev_free(b->d_cK);
  if (b->ev_ok)
    for (auto& pr : b->ev)
      for (auto& e : pr) cudaEventDestroy(e);
  if (b->aux_ok) {
    for (int k = 0; k < fsim_basis::kAuxStreams; ++k) {
      cudaStreamDestroy(b->aux[k]);
      cudaEventDestroy(b->join_ev[k]);
    }
    cudaEventDestroy(b->fork_ev);
  }
  delete b;
}

int fsim_basis_nbf(const fsim_basis* b) { return b ? b->nbf_ext() : FSIM_EINVAL; }
int fsim_basis_nbf_cart(const fsim_basis* b) { return b ? b->nbf : FSIM_EINVAL; }
int fsim_basis_nshell(const fsim_basis* b) { return b ? b->nshell : FSIM_EINVAL; }

int fsim_basis_pair_counts(const fsim_basis* b, int counts[6]) {
  if (!b || !counts) return FSIM_EINVAL;
  for (int X = 0; X < kNumPairCls; ++X) counts[X] = b->cls[X].n;
  return FSIM_OK;
}

int fsim_enuc(const fsim_basis* b, double* e) {
  if (!b || !e) {
    set_error("fsim_enuc: null pointer");
    return FSIM_EINVAL;
  }
  double s = 0.0;
  for (int i = 0; i < b->natom; ++i)
    for (int j = 0; j < i; ++j) {
      double r2 = 0.0;
      for (int x = 0; x < 3; ++x) {
        const double d = b->axyz[3 * i + x] - b->axyz[3 * j + x];
        r2 += d * d;
      }
      s += b->Z[i] * b->Z[j] / std::sqrt(r2);
    }
  *e = s;
  return FSIM_OK;
}

int fsim_onee(fsim_basis* b, int which, double* out, int ptr_mode, void* stream) {
  if (!b || !out) {
    set_error("fsim_onee: null pointer");
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n2 = (size_t)b->nbf_ext() * b->nbf_ext();
  if (ptr_mode == FSIM_PTR_DEVICE) return onee_ext_device(b, which, out, s);
  double* d = nullptr;
  FSIM_TRY(dev_alloc(&d, n2));
  int rc = onee_ext_device(b, which, d, s);
  if (rc == FSIM_OK) {
    if (cudaMemcpyAsync(out, d, n2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("fsim_onee: copy back failed");
      rc = FSIM_ECUDA;
    }
  }
  dev_free(d);
  return rc;
}

int fsim_schwarz(fsim_basis* b, double* Q) {
  if (!b) {
    set_error("fsim_schwarz: null basis");
    return FSIM_EINVAL;
  }
  FSIM_TRY(ensure_schwarz(b));
  if (Q) std::memcpy(Q, b->Q.data(), sizeof(double) * b->Q.size());
  return FSIM_OK;
}

}  // extern "C"
