// Batched Fock builds and lockstep batched SCF for many molecules of uneven
// size (the paper's SCF of Sec. 3.2 for a set of molecules at once).
//
// fsim_batch: the per-molecule screened work plans of every class pair are
// concatenated into one table, so each class pair is ONE persistent launch
// over all molecules (a work item finds its molecule by binary search over the
// cumulative item counts); molecules switched off by a device-side flag skip
// their items.  The launch sequence of one build (clear accumulators, FP32
// density copies, the class-pair launches, symmetrisation) is captured once per
// precision into a CUDA graph and replayed.
//
// fsim_scf_batched: every iteration is one batched Fock build (graph replay,
// FP64 and/or mixed group) followed by the per-molecule FP64 linear algebra
// (cuBLAS / cuSOLVER on a few streams); converged molecules drop out through
// the active flags.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "fsim_internal.h"

namespace fsim {


namespace {

template <typename Real>
cudaError_t dispatch(int X, int Y, const JKParams<Real>& p, cudaStream_t s) {
  switch (X * 8 + Y) {
    case 0: return launch_jk<Real, 0, 0>(p, s);
    case 8: return launch_jk<Real, 1, 0>(p, s);
    case 9: return launch_jk<Real, 1, 1>(p, s);
    case 16: return launch_jk<Real, 2, 0>(p, s);
    case 17: return launch_jk<Real, 2, 1>(p, s);
    case 18: return launch_jk<Real, 2, 2>(p, s);
    case 24: return launch_jk<Real, 3, 0>(p, s);
    case 25: return launch_jk<Real, 3, 1>(p, s);
    case 26: return launch_jk<Real, 3, 2>(p, s);
    case 27: return launch_jk<Real, 3, 3>(p, s);
    case 32: return launch_jk<Real, 4, 0>(p, s);
    case 33: return launch_jk<Real, 4, 1>(p, s);
    case 34: return launch_jk<Real, 4, 2>(p, s);
    case 35: return launch_jk<Real, 4, 3>(p, s);
    case 36: return launch_jk<Real, 4, 4>(p, s);
    case 40: return launch_jk<Real, 5, 0>(p, s);
    case 41: return launch_jk<Real, 5, 1>(p, s);
    case 42: return launch_jk<Real, 5, 2>(p, s);
    case 43: return launch_jk<Real, 5, 3>(p, s);
    case 44: return launch_jk<Real, 5, 4>(p, s);
    case 45: return launch_jk<Real, 5, 5>(p, s);
  }
  return cudaErrorInvalidValue;
}

// Per-molecule pointer tables for the element-wise steps of a build.
struct MolPtrs {
  double* Jacc;
  double* Kacc;
  float* D32;
  const double* Din;
  double* J;
  double* K;
  int N;
};

__global__ void batch_prepare_kernel(const MolPtrs* __restrict__ m, const int* __restrict__ active, int mixed) {
  const int mol = blockIdx.y;
  if (!active[mol]) return;
  const MolPtrs M = m[mol];
  const size_t n2 = (size_t)M.N * M.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
    M.Jacc[i] = 0.0;
    M.Kacc[i] = 0.0;
    if (mixed) M.D32[i] = (float)M.Din[i];
  }
}

// Density-weighted threshold per molecule of an incremental build:
// tau / max|Din| (Din holds D_n - D_{n-1}); 0 for full builds (incr 0).
__global__ void batch_dw_kernel(const MolPtrs* __restrict__ m, const int* __restrict__ incr, float* __restrict__ tau_mol,
                                double tau) {
  const int mol = blockIdx.x;
  __shared__ double red[256];
  double mx = 0.0;
  if (incr[mol]) {
    const MolPtrs M = m[mol];
    const size_t n2 = (size_t)M.N * M.N;
    for (size_t i = threadIdx.x; i < n2; i += blockDim.x) mx = fmax(mx, fabs(M.Din[i]));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    float t = 0.0f;
    if (incr[mol] && tau > 0.0) t = red[0] > 0.0 ? (float)fmin(tau / red[0], 1e30) : 1e30f;
    tau_mol[mol] = t;
  }
}

__global__ void batch_symmetrize_kernel(const MolPtrs* __restrict__ m, const int* __restrict__ active) {
  const int mol = blockIdx.y;
  if (!active[mol]) return;
  const MolPtrs M = m[mol];
  const int N = M.N;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N * N; x += gridDim.x * blockDim.x) {
    const int r = x / N, c = x % N;
    M.J[x] = 0.25 * (M.Jacc[(size_t)r * N + c] + M.Jacc[(size_t)c * N + r]);
    M.K[x] = 0.125 * (M.Kacc[(size_t)r * N + c] + M.Kacc[(size_t)c * N + r]);
  }
}

}  // namespace

}  // namespace fsim

struct fsim_batch {
  std::vector<fsim_basis*> b;
  int nmol = 0;
  double tau = 0.0;
  cudaStream_t s = nullptr;
  struct CPB {
    int nitems = 0, bra_ppmax = 1, nin = 0;
    void* d_mols = nullptr;
    int* d_prefix = nullptr;
    int* d_ids = nullptr;
    std::vector<int> ids;
  };
  CPB cp[2][fsim::kNumPairCls][fsim::kNumPairCls];
  int* d_active = nullptr;
  float* d_tau = nullptr;  // per molecule density-weighted threshold (0: plain screening)
  int* d_incr = nullptr;   // per molecule: 1 when its next build is an increment G(D_n - D_{n-1})
  fsim::MolPtrs* d_ptrs = nullptr;
  std::vector<fsim::MolPtrs> h_ptrs;
  int maxN = 0;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraph_t graph[2] = {nullptr, nullptr};
};

namespace fsim {
namespace {

template <typename Real>
int build_tables(fsim_batch* bt, int prec) {
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      fsim_batch::CPB& C = bt->cp[prec][X][Y];
      std::vector<JKMol<Real>> mols;
      std::vector<int> prefix(1, 0);
      C.ids.clear();
      for (int m = 0; m < bt->nmol; ++m) {
        fsim_basis* b = bt->b[m];
        FockPlan* plan = nullptr;
        FSIM_TRY(get_plan(b, bt->tau, 0, 1, prec == 0 ? FSIM_FP64 : FSIM_MIXED, &plan, 1));
        const ClassPairPlan& cp = plan->cp[X][Y];
        if (cp.nitems == 0) continue;
        const Real* D = prec == 0 ? (const Real*)bt->h_ptrs[m].Din : (const Real*)bt->h_ptrs[m].D32;
        mols.push_back(JKMol<Real>{b->cls[X].view<Real>(), b->cls[Y].view<Real>(), cp.d_prefix, cp.d_count, b->nbf,
                                   D, b->d_Jacc, b->d_Kacc, b->cls[X].d_Q, b->cls[Y].d_Q});
        prefix.push_back(prefix.back() + cp.nitems);
        C.ids.push_back(m);
        C.bra_ppmax = std::max(C.bra_ppmax, b->cls[X].ppmax);
      }
      C.nin = (int)mols.size();
      C.nitems = prefix.back();
      if (C.nin == 0) continue;
      JKMol<Real>* dm = nullptr;
      FSIM_TRY(dev_alloc(&dm, mols.size()));
      C.d_mols = dm;
      FSIM_TRY(dev_alloc(&C.d_prefix, prefix.size()));
      FSIM_TRY(dev_alloc(&C.d_ids, C.ids.size()));
      FSIM_CK(cudaMemcpy(dm, mols.data(), sizeof(JKMol<Real>) * mols.size(), cudaMemcpyHostToDevice));
      FSIM_CK(cudaMemcpy(C.d_prefix, prefix.data(), sizeof(int) * prefix.size(), cudaMemcpyHostToDevice));
      FSIM_CK(cudaMemcpy(C.d_ids, C.ids.data(), sizeof(int) * C.ids.size(), cudaMemcpyHostToDevice));
    }
  return FSIM_OK;
}

// dry = true: no launch; every kernel of the sequence has its attributes set
// and its module loaded, so that the sequence can then be captured directly.
template <typename Real>
int launch_batch(fsim_batch* bt, int prec, cudaStream_t s, bool dry) {
  const int mixed = prec == 1;
  dim3 g(std::max(1, std::min(64, (bt->maxN * bt->maxN + 255) / 256)), bt->nmol);
  if (dry) {
    cudaFuncAttributes fa;
    FSIM_CK(cudaFuncGetAttributes(&fa, batch_prepare_kernel));
    FSIM_CK(cudaFuncGetAttributes(&fa, batch_symmetrize_kernel));
  } else {
    batch_prepare_kernel<<<g, 256, 0, s>>>(bt->d_ptrs, bt->d_active, mixed);
    FSIM_CK(cudaGetLastError());
  }
  for (int X = kNumPairCls - 1; X >= 0; --X)
    for (int Y = X; Y >= 0; --Y) {
      const fsim_batch::CPB& C = bt->cp[prec][X][Y];
      if (C.nin == 0) continue;
      cudaError_t e = cudaSuccess;
      {
        JKParams<Real> p{};
        p.mols = (const JKMol<Real>*)C.d_mols;
        p.mol_prefix = C.d_prefix;
        p.active = bt->d_active;
        p.tau_mol = bt->d_tau;
        p.mol_ids = C.d_ids;
        p.nmol = C.nin;
        p.nitems = dry ? 0 : C.nitems;
        p.same = X == Y ? 1 : 0;
        p.psplit = 1;
        p.csplit = 1;
        p.bra_ppmax = C.bra_ppmax;
        p.boys = std::is_same<Real, double>::value ? (const Real*)bt->b[0]->d_boys64 : (const Real*)bt->b[0]->d_boys32;
        p.boys64_T = INFINITY;
        e = dispatch<Real>(X, Y, p, s);
      }
      if (e != cudaSuccess) {
        set_error("batched J/K (%d|%d): %s", X, Y, cudaGetErrorString(e));
        return FSIM_ECUDA;
      }
    }
  if (dry) return FSIM_OK;
  dim3 g2(std::max(1, std::min(64, (bt->maxN * bt->maxN + 255) / 256)), bt->nmol);
  batch_symmetrize_kernel<<<g2, 256, 0, s>>>(bt->d_ptrs, bt->d_active);
  FSIM_CK(cudaGetLastError());
  return FSIM_OK;
}

int launch_prec(fsim_batch* bt, int prec, cudaStream_t s, bool dry = false) {
  return prec == 0 ? launch_batch<double>(bt, 0, s, dry) : launch_batch<float>(bt, 1, s, dry);
}

}  // namespace
}  // namespace fsim

using namespace fsim;

extern "C" {

int fsim_batch_create(fsim_basis* const* bases, int nmol, const fsim_fock_opts* opts, const double* const* D,
                      double* const* J, double* const* K, fsim_batch** out) {
  if (!bases || nmol <= 0 || !opts || !D || !J || !K || !out) {
    set_error("fsim_batch_create: bad arguments");
    return FSIM_EINVAL;
  }
  for (int m = 0; m < nmol; ++m)
    if (!bases[m] || bases[m]->spherical) {
      set_error("fsim_batch_create: molecule %d: null or spherical basis (batches are Cartesian)", m);
      return FSIM_EINVAL;
    }
  *out = nullptr;
  fsim_batch* bt = new fsim_batch();
  bt->nmol = nmol;
  bt->tau = opts->schwarz_tau;
  bt->s = (cudaStream_t)opts->stream;
  auto fail = [&](int rc) {
    fsim_batch_destroy(bt);
    return rc;
  };
  int rc;
  for (int m = 0; m < nmol; ++m) {
    fsim_basis* b = bases[m];
    if (!b || !D[m] || !J[m] || !K[m]) {
      set_error("fsim_batch_create: null entry for molecule %d", m);
      return fail(FSIM_EINVAL);
    }
    if (has_f(b)) {
      set_error("fsim_batch_create: molecule %d has f shells (batches serve s, p and d shells)", m);
      return fail(FSIM_EINVAL);
    }
    bt->b.push_back(b);
    if ((rc = ensure_schwarz(b)) != FSIM_OK || (rc = ensure_scratch(b)) != FSIM_OK) return fail(rc);
    bt->h_ptrs.push_back(MolPtrs{b->d_Jacc, b->d_Kacc, b->d_D32, D[m], J[m], K[m], b->nbf});
    bt->maxN = std::max(bt->maxN, b->nbf);
  }
  if ((rc = dev_alloc(&bt->d_ptrs, nmol)) != FSIM_OK || (rc = dev_alloc(&bt->d_active, nmol)) != FSIM_OK ||
      (rc = dev_alloc(&bt->d_tau, nmol)) != FSIM_OK || (rc = dev_alloc(&bt->d_incr, nmol)) != FSIM_OK)
    return fail(rc);
  std::vector<int> ones(nmol, 1);
  if (cudaMemcpy(bt->d_ptrs, bt->h_ptrs.data(), sizeof(MolPtrs) * nmol, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(bt->d_active, ones.data(), sizeof(int) * nmol, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(bt->d_tau, 0, sizeof(float) * nmol) != cudaSuccess) {
    set_error("fsim_batch_create: upload failed");
    return fail(FSIM_ECUDA);
  }
  if ((rc = build_tables<double>(bt, 0)) != FSIM_OK || (rc = build_tables<float>(bt, 1)) != FSIM_OK) return fail(rc);
  *out = bt;
  return FSIM_OK;
}

void fsim_batch_destroy(fsim_batch* bt) {
  if (!bt) return;
  for (int p = 0; p < 2; ++p) {
    if (bt->exec[p]) cudaGraphExecDestroy(bt->exec[p]);
    if (bt->graph[p]) cudaGraphDestroy(bt->graph[p]);
    for (auto& row : bt->cp[p])
      for (auto& C : row) {
        if (C.d_mols) cudaFree(C.d_mols);
        dev_free(C.d_prefix);
        dev_free(C.d_ids);
      }
  }
  dev_free(bt->d_active);
  dev_free(bt->d_tau);
  dev_free(bt->d_incr);
  dev_free(bt->d_ptrs);
  delete bt;
}

int fsim_batch_fock(fsim_batch* bt, int precision, const int* active, int use_graph) {
  if (!bt || (precision != FSIM_FP64 && precision != FSIM_MIXED)) {
    set_error("fsim_batch_fock: bad arguments");
    return FSIM_EINVAL;
  }
  const int prec = precision == FSIM_MIXED ? 1 : 0;
  cudaStream_t s = bt->s;
  if (active) FSIM_CK(cudaMemcpyAsync(bt->d_active, active, sizeof(int) * bt->nmol, cudaMemcpyHostToDevice, s));
  if (!use_graph) return launch_prec(bt, prec, s);
  if (!bt->exec[prec]) {
    // a dry pass sets the kernels' attributes (outside the capture), then the
    // sequence is captured once and replayed
    FSIM_TRY(launch_prec(bt, prec, s, true));
    cudaStream_t cs;
    FSIM_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    FSIM_CK(cudaStreamSynchronize(s));
    FSIM_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    int rc = launch_prec(bt, prec, cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != FSIM_OK) return rc;
    FSIM_CK(e);
    bt->graph[prec] = g;
    FSIM_CK(cudaGraphInstantiate(&bt->exec[prec], g, 0));
  }
  FSIM_CK(cudaGraphLaunch(bt->exec[prec], s));
  return FSIM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lockstep batched SCF
// ---------------------------------------------------------------------------
namespace fsim {
namespace {

__global__ void b_add(const double* A, const double* B, double alpha, double* C, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    C[i] = A[i] + alpha * B[i];
}
__global__ void b_antisym(const double* M, double* e, int N) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N * N; x += gridDim.x * blockDim.x) {
    const int r = x / N, c = x % N;
    e[x] = M[(size_t)r * N + c] - M[(size_t)c * N + r];
  }
}
__global__ void b_scale_cols(double* U, const double* w, int N) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N * N; x += gridDim.x * blockDim.x) U[x] *= 1.0 / sqrt(w[x / N]);
}
// out += sum(a*b) (mode 0) or sum((a-b)^2) (mode 1)
__global__ void b_dot(const double* a, const double* b, size_t n, double* out, int mode) {
  __shared__ double sh[256];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s += mode == 0 ? a[i] * b[i] : (a[i] - b[i]) * (a[i] - b[i]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, sh[0]);
}

constexpr int kNStreams = 8;
constexpr int kSlots = 24;  // per-molecule scalar slots: 0 E, 1 rmsD^2, 2 moved^2, 4.. DIIS dots

struct Lane {
  cudaStream_t s = nullptr;
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
  double* work = nullptr;
  int lwork = 0;
  int* info = nullptr;
  cudaEvent_t ev = nullptr;
};

struct Mol {
  fsim_basis* b;
  int N, nocc, lane;
  size_t n2;
  double *S, *H, *X, *D, *Dn, *Din, *J, *K, *G, *F, *Fu, *t1, *t2, *e, *Dr, *Fh, *Eh, *w, *V;
  int phase = 0, nresets = 0, nstored = 0, head = 0, iters = 0;
  bool have_G = false, have_old = false, conv = false, want64 = false, incr = false;
  double E = 0.0, E_old = 0.0, t_conv = 0.0, e_nuc = 0.0;
  std::vector<double> B;
  std::vector<double> cv;
  long long quartets = 0;
  int n64 = 0, nmx = 0;
  bool mixed = false;  // this molecule's builds are mixed (else FP64-accurate throughout)
  double smin = 0.0;   // smallest overlap eigenvalue
};

int gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
         const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  if (cublasDgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc) != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasDgemm failed");
    return FSIM_ECUDA;
  }
  return FSIM_OK;
}

// D = 2 C_occ C_occ^T from a Fock-like matrix M (all symmetric, so row/column major agree)
int density_from(Mol& m, Lane& ln, const double* M, double* Dout) {
  const int N = m.N;
  FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_N, N, N, N, 1.0, M, N, m.X, N, 0.0, m.t1, N));     // M X
  FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_N, N, N, N, 1.0, m.X, N, m.t1, N, 0.0, m.V, N));   // X M X
  if (cusolverDnDsyevd(ln.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, m.V, N, m.w, ln.work, ln.lwork,
                       ln.info) != CUSOLVER_STATUS_SUCCESS) {
    set_error("cusolverDnDsyevd failed");
    return FSIM_ECUDA;
  }
  FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_N, N, m.nocc, N, 1.0, m.X, N, m.V, N, 0.0, m.t1, N));  // C_occ
  FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_T, N, N, m.nocc, 2.0, m.t1, N, m.t1, N, 0.0, Dout, N));
  return FSIM_OK;
}

bool diis_coeffs(const std::vector<double>& B, int n, int m, std::vector<double>& c) {
  // B is m x m storage of which the first n rows/cols are used
  const int k = n + 1;
  std::vector<double> A((size_t)k * k, 0.0), r(k, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) A[i * k + j] = B[i * m + j];
    A[i * k + n] = A[n * k + i] = -1.0;
  }
  r[n] = -1.0;
  for (int p = 0; p < k; ++p) {
    int piv = p;
    for (int i = p + 1; i < k; ++i)
      if (std::fabs(A[i * k + p]) > std::fabs(A[piv * k + p])) piv = i;
    if (std::fabs(A[piv * k + p]) < 1e-300) return false;
    if (piv != p) {
      for (int j = 0; j < k; ++j) std::swap(A[p * k + j], A[piv * k + j]);
      std::swap(r[p], r[piv]);
    }
    for (int i = p + 1; i < k; ++i) {
      const double f = A[i * k + p] / A[p * k + p];
      for (int j = p; j < k; ++j) A[i * k + j] -= f * A[p * k + j];
      r[i] -= f * r[p];
    }
  }
  std::vector<double> x(k);
  for (int i = k - 1; i >= 0; --i) {
    double s = r[i];
    for (int j = i + 1; j < k; ++j) s -= A[i * k + j] * x[j];
    x[i] = s / A[i * k + i];
  }
  c.assign(x.begin(), x.begin() + n);
  for (double v : c)
    if (!std::isfinite(v)) return false;
  return true;
}

}  // namespace
}  // namespace fsim

extern "C" int fsim_scf_batched(fsim_basis* const* bases, int nmol, const fsim_scf_opts* opts,
                                fsim_scf_result* results) {
  using namespace fsim;
  if (!bases || nmol <= 0 || !opts || !results) {
    set_error("fsim_scf_batched: bad arguments");
    return FSIM_EINVAL;
  }
  const fsim_scf_opts& o = *opts;
  const bool mixed = o.fock.precision == FSIM_MIXED;
  const int md = o.diis_size;
  if (o.max_iter < 1 || md < 0 || md > 16 || o.guess != FSIM_GUESS_CORE ||
      (o.fock.precision != FSIM_FP64 && o.fock.precision != FSIM_MIXED)) {
    set_error("fsim_scf_batched: bad options (core guess only, diis_size <= 16, FSIM_FP64 or FSIM_MIXED)");
    return FSIM_EINVAL;
  }
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  cudaStream_t s0 = (cudaStream_t)o.fock.stream;
  std::vector<void*> allocs;
  auto A = [&](double** p, size_t n) {
    int rc = dev_alloc(p, n);
    if (rc == FSIM_OK) allocs.push_back(*p);
    return rc;
  };
  struct Cleanup {
    std::vector<void*>* a;
    Lane* lanes;
    fsim_batch** bt;
    ~Cleanup() {
      for (void* p : *a) cudaFree(p);
      for (int i = 0; i < kNStreams; ++i) {
        if (lanes[i].blas) cublasDestroy(lanes[i].blas);
        if (lanes[i].sol) cusolverDnDestroy(lanes[i].sol);
        if (lanes[i].ev) cudaEventDestroy(lanes[i].ev);
        if (lanes[i].s) cudaStreamDestroy(lanes[i].s);
        if (lanes[i].info) cudaFree(lanes[i].info);
        if (lanes[i].work) cudaFree(lanes[i].work);
      }
      if (*bt) fsim_batch_destroy(*bt);
    }
  };
  Lane lanes[kNStreams];
  fsim_batch* bt = nullptr;
  Cleanup cleanup{&allocs, lanes, &bt};
  std::vector<Mol> mols(nmol);
  int maxN = 0;
  for (int i = 0; i < nmol; ++i) {
    Mol& m = mols[i];
    m.b = bases[i];
    if (!m.b || m.b->spherical) {
      set_error("fsim_scf_batched: basis %d is null or spherical (batches are Cartesian)", i);
      return FSIM_EINVAL;
    }
    m.N = m.b->nbf;
    maxN = std::max(maxN, m.N);
    int ne = 0;
    for (int a = 0; a < m.b->natom; ++a) ne += m.b->Z[a];
    if (ne & 1) {
      set_error("fsim_scf_batched: molecule %d has an odd electron count", i);
      return FSIM_EINVAL;
    }
    m.nocc = ne / 2;
    m.n2 = (size_t)m.N * m.N;
    m.lane = i % kNStreams;
    double** bufs[] = {&m.S, &m.H, &m.X, &m.D, &m.Dn, &m.Din, &m.J, &m.K, &m.G, &m.F, &m.Fu, &m.t1, &m.t2, &m.e, &m.Dr, &m.V};
    for (double** p : bufs) FSIM_TRY(A(p, m.n2));
    FSIM_TRY(A(&m.w, m.N));
    if (md > 0) {
      FSIM_TRY(A(&m.Fh, m.n2 * md));
      FSIM_TRY(A(&m.Eh, m.n2 * md));
    }
    m.B.assign((size_t)std::max(md, 1) * std::max(md, 1), 0.0);
    FSIM_TRY(fsim_enuc(m.b, &m.e_nuc));
  }
  double* slots = nullptr;
  FSIM_TRY(A(&slots, (size_t)nmol * kSlots));
  double* d_smin = nullptr;  // smallest overlap eigenvalue per molecule
  FSIM_TRY(A(&d_smin, (size_t)nmol));
  std::vector<double> hs((size_t)nmol * kSlots);
  for (auto& ln : lanes) {
    FSIM_CK(cudaStreamCreateWithFlags(&ln.s, cudaStreamNonBlocking));
    if (cublasCreate(&ln.blas) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&ln.sol) != CUSOLVER_STATUS_SUCCESS) {
      set_error("fsim_scf_batched: handle creation failed");
      return FSIM_ECUDA;
    }
    cublasSetStream(ln.blas, ln.s);
    cusolverDnSetStream(ln.sol, ln.s);
    FSIM_CK(cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming));
    double* dummyV = nullptr;
    double* dummyW = nullptr;
    cusolverDnDsyevd_bufferSize(ln.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, maxN, dummyV, maxN, dummyW,
                                &ln.lwork);
    FSIM_TRY(dev_alloc(&ln.work, (size_t)ln.lwork));
    FSIM_TRY(dev_alloc(&ln.info, 1));
  }
  cudaEvent_t ev0;
  FSIM_CK(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
  auto fork = [&]() -> int {  // lanes wait for s0
    FSIM_CK(cudaEventRecord(ev0, s0));
    for (auto& ln : lanes) FSIM_CK(cudaStreamWaitEvent(ln.s, ev0, 0));
    return FSIM_OK;
  };
  auto join = [&]() -> int {  // s0 waits for the lanes
    for (auto& ln : lanes) {
      FSIM_CK(cudaEventRecord(ln.ev, ln.s));
      FSIM_CK(cudaStreamWaitEvent(s0, ln.ev, 0));
    }
    return FSIM_OK;
  };
  const int th = 256;
  auto blocks = [&](size_t n) { return (int)std::min<size_t>((n + th - 1) / th, 512); };
  // ---- set-up: S, H, X, core guess
  for (auto& m : mols) FSIM_TRY(onee_device(m.b, 0, m.S, s0));
  for (auto& m : mols) {
    FSIM_TRY(onee_device(m.b, 1, m.t1, s0));
    FSIM_TRY(onee_device(m.b, 2, m.t2, s0));
    b_add<<<blocks(m.n2), th, 0, s0>>>(m.t1, m.t2, 1.0, m.H, m.n2);
  }
  FSIM_TRY(fork());
  for (auto& m : mols) {
    Lane& ln = lanes[m.lane];
    FSIM_CK(cudaMemcpyAsync(m.V, m.S, sizeof(double) * m.n2, cudaMemcpyDeviceToDevice, ln.s));
    if (cusolverDnDsyevd(ln.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m.N, m.V, m.N, m.w, ln.work,
                         ln.lwork, ln.info) != CUSOLVER_STATUS_SUCCESS) {
      set_error("cusolverDnDsyevd failed (overlap)");
      return FSIM_ECUDA;
    }
    // eigenvalues ascending; m.w is reused for the orbital energies below
    FSIM_CK(cudaMemcpyAsync(d_smin + (&m - mols.data()), m.w, sizeof(double), cudaMemcpyDeviceToDevice, ln.s));
    FSIM_CK(cudaMemcpyAsync(m.t1, m.V, sizeof(double) * m.n2, cudaMemcpyDeviceToDevice, ln.s));
    b_scale_cols<<<blocks(m.n2), th, 0, ln.s>>>(m.t1, m.w, m.N);
    FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_T, m.N, m.N, m.N, 1.0, m.t1, m.N, m.V, m.N, 0.0, m.X, m.N));
    FSIM_TRY(density_from(m, ln, m.H, m.D));
  }
  FSIM_TRY(join());
  // per molecule: mixed builds only when the overlap is well enough conditioned
  FSIM_CK(cudaStreamSynchronize(s0));
  std::vector<double> smin_h(nmol);
  FSIM_CK(cudaMemcpy(smin_h.data(), d_smin, sizeof(double) * nmol, cudaMemcpyDeviceToHost));
  for (auto& m : mols) {
    m.smin = smin_h[&m - mols.data()];
    m.mixed = mixed && m.smin >= FSIM_MIXED_MIN_S_EIG;
    m.phase = m.mixed ? 0 : 2;  // without mixed builds there is no settling phase
  }
  // ---- the batch: Din -> J, K for every molecule
  {
    std::vector<const double*> Din(nmol);
    std::vector<double*> Jp(nmol), Kp(nmol);
    for (int i = 0; i < nmol; ++i) {
      Din[i] = mols[i].Din;
      Jp[i] = mols[i].J;
      Kp[i] = mols[i].K;
    }
    fsim_fock_opts fo = o.fock;
    fo.stream = s0;
    FSIM_TRY(fsim_batch_create(bases, nmol, &fo, Din.data(), Jp.data(), Kp.data(), &bt));
  }
  const double t_loop0 = elapsed();
  std::vector<int> act64(nmol), actmx(nmol), incr_h(nmol, 0);
  int nconv = 0, it = 0;
  for (it = 1; it <= o.max_iter && nconv < nmol; ++it) {
    bool any64 = false, anymx = false;
    for (int i = 0; i < nmol; ++i) {
      Mol& m = mols[i];
      act64[i] = actmx[i] = 0;
      if (m.conv) continue;
      m.want64 = !m.mixed || (m.phase == 2 && o.final_fp64 && !m.have_G);
      m.incr = o.incremental && m.have_G && !m.want64;
      if (m.incr)
        b_add<<<blocks(m.n2), th, 0, s0>>>(m.D, m.Dn, -1.0, m.Din, m.n2);
      else
        FSIM_CK(cudaMemcpyAsync(m.Din, m.D, sizeof(double) * m.n2, cudaMemcpyDeviceToDevice, s0));
      (m.want64 ? act64 : actmx)[i] = 1;
      (m.want64 ? any64 : anymx) = true;
    }
    if (o.dw_screen) {
      // density-weighted thresholds of this iteration's increments while each
      // molecule's mixed iteration settles (phase 0); 0 for full builds and from
      // the FP64 reset on (the skipped terms add up in the incremental G)
      for (int i = 0; i < nmol; ++i)
        incr_h[i] = !mols[i].conv && mols[i].incr && !mols[i].want64 && mols[i].phase == 0;
      FSIM_CK(cudaMemcpyAsync(bt->d_incr, incr_h.data(), sizeof(int) * nmol, cudaMemcpyHostToDevice, s0));
      batch_dw_kernel<<<nmol, 256, 0, s0>>>(bt->d_ptrs, bt->d_incr, bt->d_tau, o.fock.schwarz_tau);
      FSIM_CK(cudaGetLastError());
    }
    if (any64) FSIM_TRY(fsim_batch_fock(bt, FSIM_FP64, act64.data(), 1));
    if (anymx) FSIM_TRY(fsim_batch_fock(bt, FSIM_MIXED, actmx.data(), 1));
    FSIM_CK(cudaMemsetAsync(slots, 0, sizeof(double) * nmol * kSlots, s0));
    FSIM_TRY(fork());
    for (int i = 0; i < nmol; ++i) {
      Mol& m = mols[i];
      if (m.conv) continue;
      Lane& ln = lanes[m.lane];
      const size_t n2 = m.n2;
      if (m.incr) {
        b_add<<<blocks(n2), th, 0, ln.s>>>(m.G, m.J, 1.0, m.G, n2);
        b_add<<<blocks(n2), th, 0, ln.s>>>(m.G, m.K, -0.5, m.G, n2);
      } else {
        b_add<<<blocks(n2), th, 0, ln.s>>>(m.J, m.K, -0.5, m.G, n2);
        m.have_G = true;
        if (m.mixed && m.want64) {
          FSIM_CK(cudaMemcpyAsync(m.Dr, m.D, sizeof(double) * n2, cudaMemcpyDeviceToDevice, ln.s));
          ++m.nresets;
        }
      }
      (m.want64 ? m.n64 : m.nmx)++;
      b_add<<<blocks(n2), th, 0, ln.s>>>(m.H, m.G, 1.0, m.F, n2);
      b_add<<<blocks(n2), th, 0, ln.s>>>(m.H, m.F, 1.0, m.t1, n2);
      b_dot<<<64, 256, 0, ln.s>>>(m.D, m.t1, n2, slots + (size_t)i * kSlots + 0, 0);
      if (md > 0) {
        FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_N, m.N, m.N, m.N, 1.0, m.D, m.N, m.F, m.N, 0.0, m.t1, m.N));
        FSIM_TRY(gemm(ln.blas, CUBLAS_OP_N, CUBLAS_OP_N, m.N, m.N, m.N, 1.0, m.S, m.N, m.t1, m.N, 0.0, m.t2, m.N));
        // column-major products of symmetric matrices: t2 = (F D S)^T as row-major; e = t2 - t2^T up to sign,
        // and the DIIS metric is sign-free
        b_antisym<<<blocks(n2), th, 0, ln.s>>>(m.t2, m.e, m.N);
        FSIM_CK(cudaMemcpyAsync(m.Fh + (size_t)m.head * n2, m.F, sizeof(double) * n2, cudaMemcpyDeviceToDevice, ln.s));
        FSIM_CK(cudaMemcpyAsync(m.Eh + (size_t)m.head * n2, m.e, sizeof(double) * n2, cudaMemcpyDeviceToDevice, ln.s));
        const int nst = std::min(m.nstored + 1, md);
        for (int j = 0; j < nst; ++j)
          b_dot<<<64, 256, 0, ln.s>>>(m.Eh + (size_t)m.head * n2, m.Eh + (size_t)j * n2, n2,
                                      slots + (size_t)i * kSlots + 4 + j, 0);
      }
    }
    FSIM_TRY(join());
    FSIM_CK(cudaMemcpyAsync(hs.data(), slots, sizeof(double) * nmol * kSlots, cudaMemcpyDeviceToHost, s0));
    FSIM_CK(cudaStreamSynchronize(s0));
    for (int i = 0; i < nmol; ++i) {
      Mol& m = mols[i];
      if (m.conv) continue;
      m.E = 0.5 * hs[(size_t)i * kSlots + 0];
      m.quartets += 0;
      m.cv.clear();
      if (md > 0) {
        const int nst = std::min(m.nstored + 1, md);
        for (int j = 0; j < nst; ++j) m.B[m.head * md + j] = m.B[j * md + m.head] = hs[(size_t)i * kSlots + 4 + j];
        m.nstored = nst;
        m.head = (m.head + 1) % md;
        if (m.nstored >= 2 && !diis_coeffs(m.B, m.nstored, md, m.cv)) m.cv.clear();
      }
    }
    FSIM_CK(cudaMemsetAsync(slots, 0, sizeof(double) * nmol * kSlots, s0));
    FSIM_TRY(fork());
    for (int i = 0; i < nmol; ++i) {
      Mol& m = mols[i];
      if (m.conv) continue;
      Lane& ln = lanes[m.lane];
      const double* Fuse = m.F;
      if (!m.cv.empty()) {
        FSIM_CK(cudaMemsetAsync(m.Fu, 0, sizeof(double) * m.n2, ln.s));
        for (int j = 0; j < (int)m.cv.size(); ++j)
          b_add<<<blocks(m.n2), th, 0, ln.s>>>(m.Fu, m.Fh + (size_t)j * m.n2, m.cv[j], m.Fu, m.n2);
        Fuse = m.Fu;
      }
      FSIM_CK(cudaMemcpyAsync(m.Dn, m.D, sizeof(double) * m.n2, cudaMemcpyDeviceToDevice, ln.s));
      FSIM_TRY(density_from(m, ln, Fuse, m.D));
      b_dot<<<64, 256, 0, ln.s>>>(m.D, m.Dn, m.n2, slots + (size_t)i * kSlots + 1, 1);
      if (m.mixed && o.final_fp64) b_dot<<<64, 256, 0, ln.s>>>(m.Dn, m.Dr, m.n2, slots + (size_t)i * kSlots + 2, 1);
    }
    FSIM_TRY(join());
    FSIM_CK(cudaMemcpyAsync(hs.data(), slots, sizeof(double) * nmol * kSlots, cudaMemcpyDeviceToHost, s0));
    FSIM_CK(cudaStreamSynchronize(s0));
    const double now = elapsed() - t_loop0;
    for (int i = 0; i < nmol; ++i) {
      Mol& m = mols[i];
      if (m.conv) continue;
      if (results[i].e_hist && m.iters < o.max_iter) results[i].e_hist[m.iters] = m.E + m.e_nuc;
      if (results[i].t_hist && m.iters < o.max_iter) results[i].t_hist[m.iters] = now;
      ++m.iters;
      const double rmsD = std::sqrt(hs[(size_t)i * kSlots + 1] / (double)m.n2);
      const double dE = m.have_old ? std::fabs(m.E - m.E_old) : 1e300;
      m.E_old = m.E;
      m.have_old = true;
      if (m.phase == 0 && dE < 1e-7 && rmsD < 1e-4) {
        m.phase = 2;
        if (o.final_fp64) {
          m.have_G = false;
          m.nstored = 0;
          m.head = 0;
          m.have_old = false;
        }
        continue;
      }
      if (m.phase == 2 && dE < o.conv_dE && rmsD < o.conv_dD) {
        if (m.mixed && o.final_fp64 && m.nresets < 6 && std::sqrt(hs[(size_t)i * kSlots + 2] / (double)m.n2) > 1e-6) {
          m.have_G = false;
          m.have_old = false;
          continue;
        }
        m.conv = true;
        m.t_conv = now;
        ++nconv;
      }
    }
  }
  const double total = elapsed() - t_loop0;
  for (int i = 0; i < nmol; ++i) {
    Mol& m = mols[i];
    fsim_scf_result& r = results[i];
    r.e_elec = m.E;
    r.e_nuc = m.e_nuc;
    r.e_total = m.E + m.e_nuc;
    r.iters = m.iters;
    r.converged = m.conv ? 1 : 0;
    r.guess_fallback = 0;
    r.time_s = m.conv ? m.t_conv : total;
    r.min_s_eig = m.smin;
    r.mixed_fallback = mixed && !m.mixed;
    r.quartets = 0;
    r.fp64_builds = m.n64;
    r.mixed_builds = m.nmx;
    if (r.D_out) FSIM_CK(cudaMemcpy(r.D_out, m.conv ? m.Dn : m.D, sizeof(double) * m.n2, cudaMemcpyDeviceToHost));
  }
  cudaEventDestroy(ev0);
  return nconv == nmol ? FSIM_OK : FSIM_ENOCONV;
}
