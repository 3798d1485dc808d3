// Coulomb-only Fock build J <- D in Hermite space (fsim_j_build; paper Sec.
// 2.5, the density-contracted intermediate of the ket side; Sec. 2.2 Eq. fock
// for J).  Kernels in jengine.cuh.
//
// Work lists: every ordered pair of pair classes (X, Y) is one launch; the
// kets of bra pair i are the prefix of class Y (sorted by Schwarz bound) with
// Q_i Q_j >= tau, with no triangle cut, so each unique quartet of the fused
// J/K build appears in both orders and every quartet adds only to its bra
// block.  J = (J_acc + J_acc^T) / 2 with the bra factor 2 for pairs of two
// different shells applied in the kernel.
#include <algorithm>
#include <cmath>

#include "fsim_internal.h"
#include "jengine.cuh"

namespace fsim {

template <typename Real, int X, int Y>
cudaError_t launch_jeng(const JEngParams<Real>& p, cudaStream_t s);
template <typename Real, int Y>
cudaError_t launch_jeng_rho(const PairView<Real>& ket, const Real* D, int N, Real* rho, cudaStream_t s);

static __global__ void jeng_to_float_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

template <typename Real, int X>
static cudaError_t dispatch_y(int Y, const JEngParams<Real>& p, cudaStream_t s) {
  switch (Y) {
    case 0: return launch_jeng<Real, X, 0>(p, s);
    case 1: return launch_jeng<Real, X, 1>(p, s);
    case 2: return launch_jeng<Real, X, 2>(p, s);
    case 3: return launch_jeng<Real, X, 3>(p, s);
    case 4: return launch_jeng<Real, X, 4>(p, s);
    case 5: return launch_jeng<Real, X, 5>(p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename Real>
static cudaError_t dispatch_jeng(int X, int Y, const JEngParams<Real>& p, cudaStream_t s) {
  switch (X) {
    case 0: return dispatch_y<Real, 0>(Y, p, s);
    case 1: return dispatch_y<Real, 1>(Y, p, s);
    case 2: return dispatch_y<Real, 2>(Y, p, s);
    case 3: return dispatch_y<Real, 3>(Y, p, s);
    case 4: return dispatch_y<Real, 4>(Y, p, s);
    case 5: return dispatch_y<Real, 5>(Y, p, s);
  }
  return cudaErrorInvalidValue;
}

template <typename Real>
static cudaError_t dispatch_rho(int Y, const PairView<Real>& ket, const Real* D, int N, Real* rho, cudaStream_t s) {
  switch (Y) {
    case 0: return launch_jeng_rho<Real, 0>(ket, D, N, rho, s);
    case 1: return launch_jeng_rho<Real, 1>(ket, D, N, rho, s);
    case 2: return launch_jeng_rho<Real, 2>(ket, D, N, rho, s);
    case 3: return launch_jeng_rho<Real, 3>(ket, D, N, rho, s);
    case 4: return launch_jeng_rho<Real, 4>(ket, D, N, rho, s);
    case 5: return launch_jeng_rho<Real, 5>(ket, D, N, rho, s);
  }
  return cudaErrorInvalidValue;
}

// Screened kets of every bra of class X in class Y, both orders (no triangle).
static long long ordered_counts(const fsim_basis* b, int X, int Y, double tau, int shard, int nshards,
                                std::vector<int>& count) {
  const DevClass& CX = b->cls[X];
  const DevClass& CY = b->cls[Y];
  count.assign(CX.n, 0);
  long long nq = 0;
  for (int i = 0; i < CX.n; ++i) {
    int cnt = CY.n;
    if (tau > 0.0) {
      const double qi = CX.h_Q[i];
      int lo = 0, hi = CY.n;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (qi * CY.h_Q[mid] >= tau) lo = mid + 1; else hi = mid;
      }
      cnt = lo;
    }
    if (nshards > 1 && (i % nshards) != shard) cnt = 0;
    count[i] = cnt;
    nq += cnt;
  }
  return nq;
}

static int get_jplan(fsim_basis* b, double tau, int shard, int nshards, int precision, JPlan** out) {
  for (JPlan* p : b->jplans)
    if (p->tau == tau && p->shard == shard && p->nshards == nshards && p->precision == precision) {
      *out = p;
      return FSIM_OK;
    }
  JPlan* P = new JPlan();
  P->tau = tau;
  P->shard = shard;
  P->nshards = nshards;
  P->precision = precision;
  b->jplans.push_back(P);
  const long long target = (long long)device_sm_count() * 2 * kJKThreads;
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y < kNumPairCls; ++Y) {
      ClassPairPlan& cp = P->cp[X][Y];
      cp.nbra = b->cls[X].n;
      if (b->cls[X].n == 0 || b->cls[Y].n == 0) continue;
      std::vector<int> count;
      cp.nquartets = ordered_counts(b, X, Y, tau, shard, nshards, count);
      // few quartets: split the bra primitive pairs so one launch covers the device
      int ps = 1;
      for (int c : {3, 9})
        if (cp.nquartets * ps < target && c <= b->cls[X].ppmax) ps = c;
      FSIM_TRY(set_class_plan(b, X, Y, count, ps, 0, cp, 1, 0));
      P->nquartets += cp.nquartets;
    }
  *out = P;
  return FSIM_OK;
}

template <typename Real>
static Real*& rho_buf(fsim_basis* b, int Y);
template <>
float*& rho_buf<float>(fsim_basis* b, int Y) { return b->d_rho32[Y]; }
template <>
double*& rho_buf<double>(fsim_basis* b, int Y) { return b->d_rho64[Y]; }

// J = (J_acc + J_acc^T) / 2
static __global__ void jeng_symmetrize_kernel(const double* __restrict__ Ja, double* __restrict__ J, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (c >= N) return;
  J[(size_t)r * N + c] = 0.5 * (Ja[(size_t)r * N + c] + Ja[(size_t)c * N + r]);
}

template <typename Real>
static int jeng_launch_all(fsim_basis* b, JPlan* plan, const Real* Dr, float b64, cudaStream_t s) {
  // density-contracted ket vectors of every class
  for (int Y = 0; Y < kNumPairCls; ++Y) {
    const DevClass& C = b->cls[Y];
    if (C.n == 0) continue;
    Real*& rho = rho_buf<Real>(b, Y);
    if (!rho) FSIM_TRY(dev_alloc(&rho, (size_t)nherm(pair_cls_la(Y) + pair_cls_lb(Y)) * C.ppmax * C.n));
    const cudaError_t e = dispatch_rho<Real>(Y, C.view<Real>(), Dr, b->nbf, rho, s);
    if (e != cudaSuccess) {
      set_error("J-engine density vectors (%d): %s", Y, cudaGetErrorString(e));
      return FSIM_ECUDA;
    }
    ++b->last_launches;
  }
  // the 36 ordered class pairs over the caller's stream and the auxiliary
  // streams, longest first onto the least loaded stream
  FSIM_TRY(ensure_aux_streams(b));
  struct Job {
    int X, Y;
    double cost;
  };
  std::vector<Job> jobs;
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y < kNumPairCls; ++Y) {
      const ClassPairPlan& cp = plan->cp[X][Y];
      if (cp.nitems == 0) continue;
      const int L = pair_cls_la(X) + pair_cls_lb(X) + pair_cls_la(Y) + pair_cls_lb(Y);
      const double per = nherm(L) * 2.0 + nherm(pair_cls_la(X) + pair_cls_lb(X)) * nherm(pair_cls_la(Y) + pair_cls_lb(Y));
      jobs.push_back(Job{X, Y, (double)cp.nquartets * per});
    }
  std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& c) { return a.cost > c.cost; });
  constexpr int NS = fsim_basis::kAuxStreams + 1;
  cudaStream_t st[NS] = {s};
  for (int k = 0; k < fsim_basis::kAuxStreams; ++k) st[k + 1] = b->aux[k];
  const int nuse = std::min<int>(NS, (int)jobs.size());
  FSIM_CK(cudaEventRecord(b->fork_ev, s));
  for (int k = 1; k < nuse; ++k) FSIM_CK(cudaStreamWaitEvent(st[k], b->fork_ev, 0));
  double load[NS] = {};
  const Real* boys = std::is_same<Real, double>::value ? (const Real*)b->d_boys64 : (const Real*)b->d_boys32;
  for (const Job& jb : jobs) {
    int k = 0;
    for (int t = 1; t < nuse; ++t)
      if (load[t] < load[k]) k = t;
    load[k] += jb.cost;
    const ClassPairPlan& cp = plan->cp[jb.X][jb.Y];
    JEngParams<Real> p{};
    p.bra = b->cls[jb.X].view<Real>();
    p.ket = b->cls[jb.Y].view<Real>();
    p.rho = rho_buf<Real>(b, jb.Y);
    p.prefix = cp.d_prefix;
    p.ket_count = cp.d_count;
    p.N = b->nbf;
    p.J = b->d_Jacc;
    p.nitems = cp.nitems;
    p.psplit = cp.psplit;
    p.bra_ppmax = b->cls[jb.X].ppmax;
    p.boys = boys;
    p.boys64_T = b64;
    ++b->last_launches;
    const cudaError_t e = dispatch_jeng<Real>(jb.X, jb.Y, p, st[k]);
    if (e != cudaSuccess) {
      set_error("J-engine kernel (%d|%d): %s", jb.X, jb.Y, cudaGetErrorString(e));
      return FSIM_ECUDA;
    }
  }
  for (int k = 1; k < nuse; ++k) {
    FSIM_CK(cudaEventRecord(b->join_ev[k - 1], st[k]));
    FSIM_CK(cudaStreamWaitEvent(s, b->join_ev[k - 1], 0));
  }
  return FSIM_OK;
}

static int j_build_device(fsim_basis* b, const double* dD, double* dJ, const fsim_fock_opts& o) {
  if (o.precision != FSIM_FP64 && o.precision != FSIM_MIXED) {
    set_error("fsim_j_build: precision must be FSIM_FP64 or FSIM_MIXED");
    return FSIM_EINVAL;
  }
  if (o.nshards < 1 || o.shard < 0 || o.shard >= o.nshards || !(o.schwarz_tau >= 0.0)) {
    set_error("fsim_j_build: bad shard (%d of %d) or tau", o.shard, o.nshards);
    return FSIM_EINVAL;
  }
  if (!(o.boys_fp64_T == 0.0 || o.boys_fp64_T >= 30.0)) {
    set_error("fsim_j_build: boys_fp64_T must be 0 (never) or >= 30");
    return FSIM_EINVAL;
  }
  if (o.timing) {
    set_error("fsim_j_build: per-class timing is not recorded for the J-engine (timing must be 0)");
    return FSIM_EINVAL;
  }
  const float b64 = o.boys_fp64_T > 0.0 ? (float)o.boys_fp64_T : INFINITY;
  cudaStream_t s = (cudaStream_t)o.stream;
  FSIM_TRY(ensure_schwarz(b));
  FSIM_TRY(ensure_scratch(b));
  JPlan* plan = nullptr;
  FSIM_TRY(get_jplan(b, o.schwarz_tau, o.shard, o.nshards, o.precision, &plan));
  const int N = b->nbf;
  const size_t n2 = (size_t)N * N;
  b->last_timed = false;
  b->last_stream = s;
  b->last_launches = 0;
  for (auto& r : b->last_class_run) r = false;
  FSIM_CK(cudaMemsetAsync(b->d_Jacc, 0, n2 * sizeof(double), s));
  if (o.precision == FSIM_MIXED) {
    jeng_to_float_kernel<<<256, 256, 0, s>>>(dD, b->d_D32, n2);
    FSIM_CK(cudaGetLastError());
    ++b->last_launches;
    FSIM_TRY(jeng_launch_all<float>(b, plan, b->d_D32, b64, s));
  } else {
    FSIM_TRY(jeng_launch_all<double>(b, plan, dD, b64, s));
  }
  dim3 grid((N + 127) / 128, N);
  jeng_symmetrize_kernel<<<grid, 128, 0, s>>>(b->d_Jacc, dJ, N);
  FSIM_CK(cudaGetLastError());
  ++b->last_launches;
  b->last_quartets = plan->nquartets;
  return FSIM_OK;
}

}  // namespace fsim

using namespace fsim;

extern "C" int fsim_j_build(fsim_basis* b, const double* D, double* J, const fsim_fock_opts* opts) {
  if (!b || !D || !J) {
    set_error("fsim_j_build: null pointer");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    set_error("fsim_j_build: spherical bases are not supported (use fsim_fock_build)");
    return FSIM_EINVAL;
  }
  if (has_f(b)) {
    set_error("fsim_j_build: bases with f shells are not supported (use fsim_fock_build)");
    return FSIM_EINVAL;
  }
  fsim_fock_opts o;
  fsim_fock_opts_default(&o);
  if (opts) o = *opts;
  if (o.ptr_mode == FSIM_PTR_DEVICE) return j_build_device(b, D, J, o);
  if (o.ptr_mode != FSIM_PTR_HOST) {
    set_error("fsim_j_build: bad ptr_mode");
    return FSIM_EINVAL;
  }
  const size_t n2 = (size_t)b->nbf * b->nbf;
  cudaStream_t s = (cudaStream_t)o.stream;
  if (!b->d_D) FSIM_TRY(dev_alloc(&b->d_D, n2));
  if (!b->d_J) FSIM_TRY(dev_alloc(&b->d_J, n2));
  FSIM_CK(cudaMemcpyAsync(b->d_D, D, n2 * sizeof(double), cudaMemcpyHostToDevice, s));
  FSIM_TRY(j_build_device(b, b->d_D, b->d_J, o));
  FSIM_CK(cudaMemcpyAsync(J, b->d_J, n2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FSIM_CK(cudaStreamSynchronize(s));
  return FSIM_OK;
}
