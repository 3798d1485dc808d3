// Restricted Hartree-Fock SCF (paper Sec. 3.2) with DIIS (Sec. 3.2.1).
//
// All matrices live on the device in FP64 (nbf x nbf, row-major; every matrix
// here is symmetric or used through symmetric products, so row/column-major
// only matters for X and C, handled explicitly).  Dense products use cuBLAS
// DGEMM, eigenpairs cuSOLVER DSYEVD; the small bordered DIIS system
// (Algorithm 1) is solved on the host by Gaussian elimination.
//
// Mixed precision (FSIM_MIXED): Fock builds with FP32 integrals and FP64
// accumulation.  With `incremental`, G(D_n) = G(D_{n-1}) + G(D_n - D_{n-1}),
// so the FP32 error scales with the density change; with `final_fp64`, once
// the mixed iteration has settled (|dE| < 1e-7) one full FP64-accurate build
// (FP64, or double-float with final_fp64 == 2) resets G and the iteration
// continues incrementally to the requested thresholds.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "fsim_internal.h"

namespace fsim {

namespace {

struct Dev {
  std::vector<void*> ptrs;
  ~Dev() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  int alloc(T** p, size_t n) {
    int rc = dev_alloc(p, n);
    if (rc == FSIM_OK) ptrs.push_back((void*)*p);
    return rc;
  }
};

__global__ void add_kernel(const double* A, const double* B, double alpha, double* C, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    C[i] = A[i] + alpha * B[i];
}

// e = M - M^T
__global__ void antisym_kernel(const double* M, double* e, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (c < N) e[(size_t)r * N + c] = M[(size_t)r * N + c] - M[(size_t)c * N + r];
}

// column scaling U[:, j] *= f(w[j]) in column-major storage (cuSOLVER output)
__global__ void scale_cols_kernel(double* U, const double* w, int N) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, c = blockIdx.y;
  if (r < N) U[(size_t)c * N + r] *= 1.0 / sqrt(w[c]);
}

// out[k] = sum_i f(a_k[i], b[i]), a_k = a0 + k * astride, f = a b (mode 0) or
// (a - b)^2 (mode 1).  Two passes with a fixed summation order (per-CTA tree,
// then the CTA partials in index order), so repeated runs give identical bits.
constexpr int kDotCTAs = 64;
__global__ void dots_partial_kernel(const double* a0, size_t astride, const double* b, size_t n, int mode,
                                    double* part) {
  __shared__ double sh[256];
  const double* a = a0 + blockIdx.y * astride;
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double d = mode == 0 ? a[i] * b[i] : (a[i] - b[i]) * (a[i] - b[i]);
    s += d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void dots_final_kernel(const double* part, int nparts, int cnt, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  double s = 0.0;
  for (int g = 0; g < nparts; ++g) s += part[k * nparts + g];
  out[k] = s;
}

struct Ctx {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
  cudaStream_t s = nullptr;
  ~Ctx() {
    if (blas) cublasDestroy(blas);
    if (sol) cusolverDnDestroy(sol);
  }
};

#define BLAS_CK(x)                                                           \
  do {                                                                       \
    cublasStatus_t st_ = (x);                                                \
    if (st_ != CUBLAS_STATUS_SUCCESS) {                                      \
      set_error("cuBLAS error %d in %s (%s:%d)", (int)st_, #x, __FILE__, __LINE__); \
      return FSIM_ECUDA;                                                     \
    }                                                                        \
  } while (0)
#define SOL_CK(x)                                                             \
  do {                                                                        \
    cusolverStatus_t st_ = (x);                                               \
    if (st_ != CUSOLVER_STATUS_SUCCESS) {                                     \
      set_error("cuSOLVER error %d in %s (%s:%d)", (int)st_, #x, __FILE__, __LINE__); \
      return FSIM_ECUDA;                                                      \
    }                                                                         \
  } while (0)

// C = op(A) op(B) for row-major N x N matrices.  Row-major A equals column-major
// A^T, so row-major C = A B is column-major C^T = B^T A^T: gemm(B, A).
int gemm_rm(Ctx& c, bool ta, bool tb, int M, int Nn, int K, const double* A, int lda, const double* B, int ldb,
            double* C, int ldc, double alpha = 1.0, double beta = 0.0) {
  BLAS_CK(cublasDgemm(c.blas, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, Nn, M, K, &alpha, B,
                      ldb, A, lda, &beta, C, ldc));
  return FSIM_OK;
}

struct Eig {
  double* w = nullptr;    // eigenvalues, ascending
  double* V = nullptr;    // column-major eigenvectors (== row-major V^T)
  double* work = nullptr;
  int lwork = 0;
  int* info = nullptr;
};

// Eigen-decomposition of the symmetric A (row-major == column-major for symmetric input).
int eigh(Ctx& c, Eig& e, const double* A, int N) {
  FSIM_CK(cudaMemcpyAsync(e.V, A, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, c.s));
  SOL_CK(cusolverDnDsyevd(c.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, e.V, N, e.w, e.work, e.lwork,
                          e.info));
  int info = 0;
  FSIM_CK(cudaMemcpyAsync(&info, e.info, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  FSIM_CK(cudaStreamSynchronize(c.s));
  if (info != 0) {
    set_error("cusolverDnDsyevd info = %d", info);
    return FSIM_ECUDA;
  }
  return FSIM_OK;
}

// cnt reductions (see dots_partial_kernel) copied to the host with one
// synchronisation.  scratch holds kDotCTAs * cnt + cnt doubles.
int host_dots(Ctx& c, double* scratch, const double* a0, size_t astride, const double* b, size_t n, int mode,
              int cnt, double* out) {
  dots_partial_kernel<<<dim3(kDotCTAs, cnt), 256, 0, c.s>>>(a0, astride, b, n, mode, scratch);
  dots_final_kernel<<<(cnt + 31) / 32, 32, 0, c.s>>>(scratch, kDotCTAs, cnt, scratch + (size_t)kDotCTAs * cnt);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(out, scratch + (size_t)kDotCTAs * cnt, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.s) !=
          cudaSuccess ||
      cudaStreamSynchronize(c.s) != cudaSuccess) {
    set_error("SCF reduction failed");
    return FSIM_ECUDA;
  }
  return FSIM_OK;
}

double host_dot(Ctx& c, double* scratch, const double* a, const double* b, size_t n, int mode, int* rc) {
  double v = 0.0;
  *rc = host_dots(c, scratch, a, 0, b, n, mode, 1, &v);
  return v;
}

// Solve the bordered DIIS system of Algorithm 1: [B -1; -1 0] x = [0; -1].
bool diis_solve(const std::vector<double>& B, int m, std::vector<double>& cvec) {
  const int n = m + 1;
  std::vector<double> A((size_t)n * n, 0.0), r(n, 0.0);
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) A[i * n + j] = B[i * m + j];
    A[i * n + m] = -1.0;
    A[m * n + i] = -1.0;
  }
  r[m] = -1.0;
  for (int k = 0; k < n; ++k) {  // partial pivoting
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[piv * n + k])) piv = i;
    if (std::fabs(A[piv * n + k]) < 1e-300) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
      std::swap(r[k], r[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      r[i] -= f * r[k];
    }
  }
  std::vector<double> x(n);
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  cvec.assign(x.begin(), x.begin() + m);
  for (double v : cvec)
    if (!std::isfinite(v)) return false;
  return true;
}

}  // namespace

}  // namespace fsim

using namespace fsim;

extern "C" {

void fsim_scf_opts_default(fsim_scf_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nelec = 0;
  o->max_iter = 100;
  o->conv_dE = 1e-10;
  o->conv_dD = 1e-7;
  o->diis_size = 8;
  o->guess = FSIM_GUESS_CORE;
  o->D0 = nullptr;
  fsim_fock_opts_default(&o->fock);
  o->final_fp64 = 2;  // resets as double-float builds: FP64-accurate, ~2x faster on GB300
  o->incremental = 1;
}

int fsim_scf(fsim_basis* b, const fsim_scf_opts* opts, fsim_scf_result* res) {
  if (!b || !opts || !res) {
    set_error("fsim_scf: null pointer");
    return FSIM_EINVAL;
  }
  const fsim_scf_opts& o = *opts;
  const int N = b->nbf_ext();
  if (o.nelec <= 0 || (o.nelec & 1) || o.nelec / 2 > N || o.max_iter < 1 || o.diis_size < 0 ||
      (o.guess == FSIM_GUESS_DENSITY && !o.D0) || (o.guess == FSIM_GUESS_LEARNED && !o.guess_model) ||
      (o.guess != FSIM_GUESS_CORE && o.guess != FSIM_GUESS_DENSITY && o.guess != FSIM_GUESS_LEARNED) ||
      o.final_fp64 < 0 || o.final_fp64 > 2) {
    set_error("fsim_scf: bad options (nelec %d must be even and <= 2 nbf, max_iter %d, final_fp64 %d in 0..2)",
              o.nelec, o.max_iter, o.final_fp64);
    return FSIM_EINVAL;
  }
  const auto t_start = std::chrono::steady_clock::now();
  auto elapsed = [&]() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  };
  const int nocc = o.nelec / 2;
  const size_t n2 = (size_t)N * N;
  Ctx c;
  c.s = (cudaStream_t)o.fock.stream;
  BLAS_CK(cublasCreate(&c.blas));
  BLAS_CK(cublasSetStream(c.blas, c.s));
  SOL_CK(cusolverDnCreate(&c.sol));
  SOL_CK(cusolverDnSetStream(c.sol, c.s));
  Dev mem;
  double *S, *H, *T, *X, *D, *Dn, *dD, *J, *K, *G, *F, *Fu, *tmp, *tmp2, *e, *scratch, *Dr;
  FSIM_TRY(mem.alloc(&S, n2)); FSIM_TRY(mem.alloc(&H, n2)); FSIM_TRY(mem.alloc(&T, n2));
  FSIM_TRY(mem.alloc(&X, n2)); FSIM_TRY(mem.alloc(&D, n2)); FSIM_TRY(mem.alloc(&Dn, n2));
  FSIM_TRY(mem.alloc(&dD, n2)); FSIM_TRY(mem.alloc(&J, n2)); FSIM_TRY(mem.alloc(&K, n2));
  FSIM_TRY(mem.alloc(&G, n2)); FSIM_TRY(mem.alloc(&F, n2)); FSIM_TRY(mem.alloc(&Fu, n2));
  FSIM_TRY(mem.alloc(&tmp, n2)); FSIM_TRY(mem.alloc(&tmp2, n2)); FSIM_TRY(mem.alloc(&e, n2));
  FSIM_TRY(mem.alloc(&scratch, (size_t)(kDotCTAs + 1) * std::max(o.diis_size, 1)));
  FSIM_TRY(mem.alloc(&Dr, n2));  // density of the last FP64 build (mixed path)
  const int m = o.diis_size;
  double *Fh = nullptr, *Eh = nullptr;
  if (m > 0) {
    FSIM_TRY(mem.alloc(&Fh, n2 * m));
    FSIM_TRY(mem.alloc(&Eh, n2 * m));
  }
  Eig eg;
  FSIM_TRY(mem.alloc(&eg.w, N));
  FSIM_TRY(mem.alloc(&eg.V, n2));
  FSIM_TRY(mem.alloc(&eg.info, 1));
  SOL_CK(cusolverDnDsyevd_bufferSize(c.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, eg.V, N, eg.w,
                                     &eg.lwork));
  FSIM_TRY(mem.alloc(&eg.work, eg.lwork));
  const int th = 256, bl = (int)std::min<size_t>((n2 + th - 1) / th, 1024);
  dim3 g2((N + 127) / 128, N);
  int rc = FSIM_OK;

  // one-electron matrices and H = T + V
  FSIM_TRY(onee_ext_device(b, 0, S, c.s));
  FSIM_TRY(onee_ext_device(b, 1, T, c.s));
  FSIM_TRY(onee_ext_device(b, 2, tmp, c.s));
  add_kernel<<<bl, th, 0, c.s>>>(T, tmp, 1.0, H, n2);
  FSIM_CK(cudaGetLastError());
  // X = U s^{-1/2} U^T
  FSIM_TRY(eigh(c, eg, S, N));
  double smin = 0.0;
  FSIM_CK(cudaMemcpy(&smin, eg.w, sizeof(double), cudaMemcpyDeviceToHost));
  res->min_s_eig = smin;
  res->mixed_fallback = 0;
  if (!(smin > 1e-10)) {
    set_error("fsim_scf: overlap matrix ill-conditioned (min eigenvalue %.3e)", smin);
    return FSIM_EILLCOND;
  }
  FSIM_CK(cudaMemcpyAsync(tmp, eg.V, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));
  scale_cols_kernel<<<dim3((N + 127) / 128, N), 128, 0, c.s>>>(tmp, eg.w, N);
  // column-major: X = (U s^-1/2) U^T ; symmetric so row-major identical
  {
    const double one = 1.0, zero = 0.0;
    BLAS_CK(cublasDgemm(c.blas, CUBLAS_OP_N, CUBLAS_OP_T, N, N, N, &one, tmp, N, eg.V, N, &zero, X, N));
  }
  // density from a Fock-like matrix M: F' = X^T M X, eig, C = X C', D = 2 C_occ C_occ^T
  auto density_from = [&](const double* M, double* Dout) -> int {
    FSIM_TRY(gemm_rm(c, true, false, N, N, N, X, N, M, N, tmp, N));    // X^T M
    FSIM_TRY(gemm_rm(c, false, false, N, N, N, tmp, N, X, N, tmp2, N));  // (X^T M) X
    FSIM_TRY(eigh(c, eg, tmp2, N));
    // eg.V column-major: C' columns.  C = X C' (column-major: X is symmetric)
    const double one = 1.0, zero = 0.0, two = 2.0;
    BLAS_CK(cublasDgemm(c.blas, CUBLAS_OP_N, CUBLAS_OP_N, N, nocc, N, &one, X, N, eg.V, N, &zero, tmp, N));
    // D = 2 C_occ C_occ^T (column-major C_occ: N x nocc in tmp); result symmetric
    BLAS_CK(cublasDgemm(c.blas, CUBLAS_OP_N, CUBLAS_OP_T, N, N, nocc, &two, tmp, N, tmp, N, &zero, Dout, N));
    return FSIM_OK;
  };
  res->guess_fallback = 0;
  const double t_guess0 = elapsed();
  if (o.guess == FSIM_GUESS_LEARNED) {
    // learned guess: pair features, the network's forward pass (BF16 weights,
    // FP32 accumulation) and the rotation/assembly of its local blocks into tmp
    if (b->spherical) {
      set_error("fsim_scf: the learned guess works on Cartesian bases only");
      return FSIM_EINVAL;
    }
    int npair = 0, nfeat = 0, nout = 0;
    FSIM_TRY(fsim_guess_layout(b, &npair, &nfeat, &nout));
    fsim_mlp* net = nullptr;
    FSIM_TRY(fsim_mlp_load(o.guess_model, &net));
    struct NetGuard {
      fsim_mlp* n;
      ~NetGuard() { fsim_mlp_destroy(n); }
    } guard{net};
    int nin = 0, width = 0, nout_net = 0;
    mlp_dims(net, &nin, &width, &nout_net);
    if (nin != nfeat || nout_net != nout) {
      set_error("fsim_scf: guess model %s does not map %d features to %d block values", o.guess_model, nfeat, nout);
      return FSIM_EINVAL;
    }
    std::vector<float> feat((size_t)npair * nfeat);
    FSIM_TRY(fsim_guess_features(b, feat.data()));
    float *xf, *yf;
    FSIM_TRY(mem.alloc(&xf, feat.size()));
    FSIM_TRY(mem.alloc(&yf, (size_t)npair * nout));
    FSIM_CK(cudaMemcpyAsync(xf, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, c.s));
    FSIM_TRY(fsim_mlp_forward(net, xf, yf, npair, 1, c.s));
    FSIM_TRY(fsim_guess_assemble(b, yf, tmp, c.s));
  } else if (o.guess == FSIM_GUESS_DENSITY) {
    FSIM_CK(cudaMemcpyAsync(tmp, o.D0, sizeof(double) * n2, cudaMemcpyHostToDevice, c.s));
  }
  if (o.guess == FSIM_GUESS_DENSITY || o.guess == FSIM_GUESS_LEARNED) {
    // supplied or learned guess in tmp: symmetrise, rescale to Tr(DS) = N_e,
    // and keep it only if |Tr(DS) - N_e| <= 0.5 before rescaling and
    // ||D S D - 2 D||_F / ||D||_F <= 0.2 after; otherwise fall back to core-H
    antisym_kernel<<<g2, 128, 0, c.s>>>(tmp, e, N);           // e = D0 - D0^T
    add_kernel<<<bl, th, 0, c.s>>>(tmp, e, -0.5, D, n2);       // D = (D0 + D0^T) / 2
    const double tr = host_dot(c, scratch, D, S, n2, 0, &rc);
    if (rc != FSIM_OK) return rc;
    bool ok = std::fabs(tr - o.nelec) <= 0.5 && tr > 0.0;
    if (ok) {
      const double f = o.nelec / tr;
      add_kernel<<<bl, th, 0, c.s>>>(D, D, f - 1.0, D, n2);
      FSIM_TRY(gemm_rm(c, false, false, N, N, N, D, N, S, N, tmp, N));    // D S
      FSIM_TRY(gemm_rm(c, false, false, N, N, N, tmp, N, D, N, tmp2, N));  // D S D
      add_kernel<<<bl, th, 0, c.s>>>(tmp2, D, -2.0, tmp2, n2);
      const double num = host_dot(c, scratch, tmp2, tmp2, n2, 0, &rc);
      if (rc != FSIM_OK) return rc;
      const double den = host_dot(c, scratch, D, D, n2, 0, &rc);
      if (rc != FSIM_OK) return rc;
      ok = std::sqrt(num / den) <= 0.2;
    }
    if (!ok) {
      res->guess_fallback = 1;
      FSIM_TRY(density_from(H, D));
    }
  } else {
    FSIM_TRY(density_from(H, D));
  }
  FSIM_CK(cudaStreamSynchronize(c.s));
  res->guess_s = elapsed() - t_guess0;
  res->e_nuc = 0.0;
  FSIM_TRY(fsim_enuc(b, &res->e_nuc));

  fsim_fock_opts fo = o.fock;
  fo.ptr_mode = FSIM_PTR_DEVICE;
  // mixed builds only in a basis whose overlap is well enough conditioned for
  // FP32 integrals (FSIM_MIXED_MIN_S_EIG); otherwise every build FP64-accurate
  const bool mixed_req = o.fock.precision == FSIM_MIXED;
  const bool mixed = mixed_req && smin >= FSIM_MIXED_MIN_S_EIG;
  res->mixed_fallback = mixed_req && !mixed;
  // precision of the FP64-accurate builds: the requested one; on the mixed path
  // the resets' (FP64, or double-float with final_fp64 == 2); FP64 for a mixed
  // request refused by the overlap bound, since a basis that near dependent
  // amplifies double-float's 2^-47 rounding of the integrals as well
  const int prec64 = !mixed_req ? o.fock.precision
                                : (mixed && o.final_fp64 == 2 ? FSIM_DFLOAT : FSIM_FP64);
  // phase 0: mixed settling; phase 2: final accuracy.  With final_fp64 each
  // FP64 build resets G; the iteration only stops once the density has not
  // moved (rms 1e-6) since the last reset, so the FP32 part of G is tiny.
  int phase = mixed ? 0 : 2;
  int nresets = 0;
  constexpr int kMaxResets = 6;
  bool have_G = false;
  int nstored = 0, head = 0;
  std::vector<double> Bring((size_t)std::max(m, 1) * std::max(m, 1), 0.0), row(std::max(m, 1));  // DIIS B by slot
  double E_old = 0.0, E = 0.0;
  bool have_old = false;
  res->converged = 0;
  res->quartets = 0;
  res->fp64_builds = 0;
  res->mixed_builds = 0;
  int it = 0;
  const double t_loop0 = elapsed();
  for (it = 1; it <= o.max_iter; ++it) {
    // ---- G(D), full or incremental
    const bool want64 = !mixed || (phase == 2 && o.final_fp64 && !have_G);
    fo.precision = want64 ? prec64 : FSIM_MIXED;
    if (o.incremental && have_G && !want64) {
      add_kernel<<<bl, th, 0, c.s>>>(D, Dn, -1.0, dD, n2);  // dD = D - D_prev (Dn holds D_prev)
      if (o.dw_screen && phase == 0) {
        // density-weighted screening while the mixed iteration settles:
        // threshold tau / max|dD|, rounded down to tau 2^k so that the cached
        // plans stay few.  The skipped terms are each below tau but add up in
        // the incrementally built G, so from the FP64-accurate reset on every
        // build keeps the plain threshold and the reset removes what was skipped
        int imax = 0;
        BLAS_CK(cublasIdamax(c.blas, (int)n2, dD, 1, &imax));
        double dmax = 0.0;
        FSIM_CK(cudaMemcpyAsync(&dmax, dD + (imax - 1), sizeof(double), cudaMemcpyDeviceToHost, c.s));
        FSIM_CK(cudaStreamSynchronize(c.s));
        dmax = std::fabs(dmax);
        double t_eff = o.fock.schwarz_tau;
        if (o.fock.schwarz_tau > 0.0 && dmax < 1.0)
          t_eff = dmax > 0.0 ? std::ldexp(o.fock.schwarz_tau, std::min(60, (int)std::floor(-std::log2(dmax))))
                             : std::ldexp(o.fock.schwarz_tau, 60);
        fo.schwarz_tau = t_eff;
      }
      FSIM_TRY(fock_build_ext_device(b, dD, J, K, fo));
      fo.schwarz_tau = o.fock.schwarz_tau;
      add_kernel<<<bl, th, 0, c.s>>>(G, J, 1.0, G, n2);
      add_kernel<<<bl, th, 0, c.s>>>(G, K, -0.5, G, n2);
    } else {
      FSIM_TRY(fock_build_ext_device(b, D, J, K, fo));
      add_kernel<<<bl, th, 0, c.s>>>(J, K, -0.5, G, n2);
      have_G = true;
      if (mixed && want64) {
        FSIM_CK(cudaMemcpyAsync(Dr, D, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));
        ++nresets;
      }
    }
    res->quartets += b->last_quartets;
    if (want64) ++res->fp64_builds; else ++res->mixed_builds;
    add_kernel<<<bl, th, 0, c.s>>>(H, G, 1.0, F, n2);
    FSIM_CK(cudaGetLastError());
    // ---- E_elec = 1/2 Tr[D (H + F)] (D, H, F symmetric)
    add_kernel<<<bl, th, 0, c.s>>>(H, F, 1.0, tmp, n2);
    E = 0.5 * host_dot(c, scratch, D, tmp, n2, 0, &rc);
    if (rc != FSIM_OK) return rc;
    if (res->e_hist && it <= o.max_iter) res->e_hist[it - 1] = E + res->e_nuc;
    if (res->t_hist && it <= o.max_iter) res->t_hist[it - 1] = elapsed() - t_loop0;
    // ---- DIIS (Algorithm 1): e = F D S - S D F
    const double* Fuse = F;
    if (m > 0) {
      FSIM_TRY(gemm_rm(c, false, false, N, N, N, F, N, D, N, tmp, N));
      FSIM_TRY(gemm_rm(c, false, false, N, N, N, tmp, N, S, N, tmp2, N));
      antisym_kernel<<<g2, 128, 0, c.s>>>(tmp2, e, N);
      FSIM_CK(cudaMemcpyAsync(Fh + (size_t)head * n2, F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));
      FSIM_CK(cudaMemcpyAsync(Eh + (size_t)head * n2, e, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));
      nstored = std::min(nstored + 1, m);
      // only the new error vector's row of B is new: <e_head, e_j> for the stored slots
      FSIM_TRY(host_dots(c, scratch, Eh, n2, Eh + (size_t)head * n2, n2, 0, nstored, row.data()));
      for (int j = 0; j < nstored; ++j) Bring[(size_t)head * m + j] = Bring[(size_t)j * m + head] = row[j];
      head = (head + 1) % m;
      if (nstored >= 2) {
        std::vector<double> B((size_t)nstored * nstored);
        for (int i = 0; i < nstored; ++i)
          for (int j = 0; j < nstored; ++j) B[i * nstored + j] = Bring[(size_t)i * m + j];
        std::vector<double> cv;
        if (diis_solve(B, nstored, cv)) {
          FSIM_CK(cudaMemsetAsync(Fu, 0, sizeof(double) * n2, c.s));
          for (int i = 0; i < nstored; ++i) add_kernel<<<bl, th, 0, c.s>>>(Fu, Fh + (size_t)i * n2, cv[i], Fu, n2);
          Fuse = Fu;
        }
      }
    }
    // ---- new density
    FSIM_CK(cudaMemcpyAsync(Dn, D, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));  // D_prev
    FSIM_TRY(density_from(Fuse, D));
    const double rmsD = std::sqrt(host_dot(c, scratch, D, Dn, n2, 1, &rc) / (double)n2);
    if (rc != FSIM_OK) return rc;
    const double dE = have_old ? std::fabs(E - E_old) : 1e300;
    E_old = E;
    have_old = true;
    if (phase == 0 && dE < 1e-7 && rmsD < 1e-4) {
      phase = 2;  // mixed iteration settled: reset G in FP64 next (final_fp64) and tighten
      if (o.final_fp64) {
        have_G = false;
        nstored = 0;
        head = 0;
        have_old = false;
      }
      continue;
    }
    if (phase == 2 && dE < o.conv_dE && rmsD < o.conv_dD) {
      if (mixed && o.final_fp64 && nresets < kMaxResets) {
        const double moved = std::sqrt(host_dot(c, scratch, Dn, Dr, n2, 1, &rc) / (double)n2);
        if (rc != FSIM_OK) return rc;
        if (moved > 1e-6) {  // another FP64 reset at the current density
          have_G = false;
          have_old = false;
          continue;
        }
      }
      res->converged = 1;
      // the density used for the reported energy is the one F was built from
      FSIM_CK(cudaMemcpyAsync(D, Dn, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c.s));
      break;
    }
  }
  if (it > o.max_iter) it = o.max_iter;
  res->iters = it;
  res->e_elec = E;
  res->e_total = E + res->e_nuc;
  res->time_s = elapsed() - t_loop0;
  if (res->D_out) {
    FSIM_CK(cudaMemcpyAsync(res->D_out, res->converged ? D : Dn, sizeof(double) * n2, cudaMemcpyDeviceToHost, c.s));
  }
  FSIM_CK(cudaStreamSynchronize(c.s));
  return res->converged ? FSIM_OK : FSIM_ENOCONV;
}

}  // extern "C"
