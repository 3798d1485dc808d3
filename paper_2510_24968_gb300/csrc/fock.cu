// Fock build J, K from D (paper Sec. 2.2 Eq. fock; Sec. 3.2 step "Build the
// G-Matrix"), debug ERI access, and the screened work plans.
//
// Work decomposition: for each class pair (bra class X >= ket class Y) and
// each bra pair i (pairs of a class sorted by Schwarz bound Q, descending),
// the kets that survive Q_i Q_j >= tau form a prefix of class Y; with X == Y
// the prefix is cut at j <= i so each unique quartet appears once.  A work
// item is (bra, tile of consecutive kets), or for the FP64 kernels a tile of
// consecutive quartets of the flattened (bra, ket) list.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "coop.cuh"
#include "fsim_internal.h"
#include "generic.cuh"

namespace fsim {

extern template cudaError_t launch_coop<double>(const CoopParams<double>&, int, cudaStream_t);
extern template cudaError_t launch_coop<float>(const CoopParams<float>&, int, cudaStream_t);

int ensure_schwarz(fsim_basis* b);

int device_sm_count() {
  static int n = 0;
  if (n <= 0) {
    int d = 0;
    cudaGetDevice(&d);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename Real, int X, int Y>
static cudaError_t launch_if(const JKParams<Real>& p, cudaStream_t s) {
  if constexpr (std::is_same<Real, dfloat>::value && !dfloat_kernel(X, Y)) return cudaErrorInvalidValue;
  else return launch_jk<Real, X, Y>(p, s);
}

template <typename Real>
static cudaError_t dispatch_jk(int X, int Y, const JKParams<Real>& p, cudaStream_t s) {
  switch (X * 8 + Y) {
    case 0: return launch_if<Real, 0, 0>(p, s);
    case 8: return launch_if<Real, 1, 0>(p, s);
    case 9: return launch_if<Real, 1, 1>(p, s);
    case 16: return launch_if<Real, 2, 0>(p, s);
    case 17: return launch_if<Real, 2, 1>(p, s);
    case 18: return launch_if<Real, 2, 2>(p, s);
    case 24: return launch_if<Real, 3, 0>(p, s);
    case 25: return launch_if<Real, 3, 1>(p, s);
    case 26: return launch_if<Real, 3, 2>(p, s);
    case 27: return launch_if<Real, 3, 3>(p, s);
    case 32: return launch_if<Real, 4, 0>(p, s);
    case 33: return launch_if<Real, 4, 1>(p, s);
    case 34: return launch_if<Real, 4, 2>(p, s);
    case 35: return launch_if<Real, 4, 3>(p, s);
    case 36: return launch_if<Real, 4, 4>(p, s);
    case 40: return launch_if<Real, 5, 0>(p, s);
    case 41: return launch_if<Real, 5, 1>(p, s);
    case 42: return launch_if<Real, 5, 2>(p, s);
    case 43: return launch_if<Real, 5, 3>(p, s);
    case 44: return launch_if<Real, 5, 4>(p, s);
    case 45: return launch_if<Real, 5, 5>(p, s);
  }
  return cudaErrorInvalidValue;
}

int run_list(fsim_basis* b, int X, int Y, const std::vector<int2>& items, double* d_out, int precision,
             cudaStream_t s) {
  if (precision != FSIM_FP64) {
    set_error("explicit quartet lists are evaluated in FP64 only");
    return FSIM_EINVAL;
  }
  if (items.empty()) return FSIM_OK;
  int2* d_items = nullptr;
  FSIM_TRY(dev_alloc(&d_items, items.size()));
  cudaError_t e = cudaMemcpy(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && X >= kNumPairCls) {
    GenParams<double> p{};
    p.bra = b->cls[X].view<double>();
    p.ket = b->cls[Y].view<double>();
    p.la = pair_cls_la(X); p.lb = pair_cls_lb(X); p.lc = pair_cls_la(Y); p.ld = pair_cls_lb(Y);
    p.same = X == Y;
    p.list_mode = 1;
    p.items = d_items;
    p.nitems = (int)items.size();
    p.out = d_out;
    p.N = b->nbf;
    p.boys = b->d_boys64;
    p.boys64_T = INFINITY;
    e = launch_gen<double>(p, s);
  } else if (e == cudaSuccess) {
    CoopParams<double> p{};
    p.bra = b->cls[X].view<double>();
    p.ket = b->cls[Y].view<double>();
    make_cls_desc(X, p.bd);
    make_cls_desc(Y, p.kd);
    p.list_mode = 1;
    p.items = d_items;
    p.nitems = (int)items.size();
    p.out = d_out;
    p.boys = b->d_boys64;
    p.boys64_T = INFINITY;
    e = launch_coop<double>(p, (p.nitems + kCoopWarps - 1) / kCoopWarps, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(d_items);
  if (e != cudaSuccess) {
    set_error("ERI list kernel (%d,%d): %s", X, Y, cudaGetErrorString(e));
    return FSIM_ECUDA;
  }
  return FSIM_OK;
}

// Screened ket counts of class pair (X, Y): count[i] = kets of bra i with
// Q_i Q_j >= tau (class Y sorted by Q descending), cut at j <= i when X == Y.
static long long screened_counts(const fsim_basis* b, int X, int Y, double tau, int shard, int nshards,
                                 std::vector<int>& count) {
  const DevClass& CX = b->cls[X];
  const DevClass& CY = b->cls[Y];
  count.assign(CX.n, 0);
  long long nq = 0;
  for (int i = 0; i < CX.n; ++i) {
    int cnt;
    if (tau > 0.0) {
      const double qi = CX.h_Q[i];
      int lo = 0, hi = CY.n;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (qi * CY.h_Q[mid] >= tau) lo = mid + 1; else hi = mid;
      }
      cnt = lo;
    } else {
      cnt = CY.n;
    }
    if (X == Y) cnt = std::min(cnt, i + 1);
    if (nshards > 1 && (i % nshards) != shard) cnt = 0;
    count[i] = cnt;
    nq += cnt;
  }
  return nq;
}

// (Re)build the device work list of one class pair for a launch shape: on the
// unrolled kernel psplit threads per quartet share the bra primitive pairs and
// csplit thread groups share the ket chunks; or the cooperative kernel.
int set_class_plan(fsim_basis* b, int X, int Y, const std::vector<int>& count, int psplit, int coop,
                   ClassPairPlan& cp, int csplit, int flat) {
  const DevClass& CX = b->cls[X];
  if (!coop && !(psplit >= 1 && psplit <= kJKThreads / 4 && (csplit == 1 || csplit == 2 || csplit == 4))) {
    set_error("bad launch shape (%d|%d): psplit %d, csplit %d", X, Y, psplit, csplit);
    return FSIM_EINVAL;
  }
  cp.coop = coop;
  cp.psplit = coop ? 1 : psplit;
  cp.csplit = coop ? 1 : csplit;
  cp.tq = coop ? kCoopWarps : (kJKThreads / cp.csplit) / cp.psplit;
  // tiles per bra (prefix of tile counts: cooperative kernel, per-bra form of
  // the unrolled kernel) or tiles of the flattened (bra, ket) list (prefix of
  // quartet counts: flattened form)
  const bool fl = flat && !coop;
  std::vector<int> prefix(CX.n + 1, 0);
  long long acc = 0;
  for (int i = 0; i < CX.n; ++i) {
    acc += fl ? count[i] : (count[i] + cp.tq - 1) / cp.tq;
    if (acc > 2147483647LL - kJKThreads) {
      set_error("class pair (%d|%d): more than 2^31 screened quartets; shard the build", X, Y);
      return FSIM_EINVAL;
    }
    prefix[i + 1] = (int)acc;
  }
  cp.nitems = fl ? (prefix[CX.n] + cp.tq - 1) / cp.tq : prefix[CX.n];
  if (!cp.d_prefix) FSIM_TRY(dev_alloc(&cp.d_prefix, CX.n + 1));
  if (!cp.d_count) FSIM_TRY(dev_alloc(&cp.d_count, CX.n));
  FSIM_CK(cudaMemcpy(cp.d_prefix, prefix.data(), sizeof(int) * (CX.n + 1), cudaMemcpyHostToDevice));
  FSIM_CK(cudaMemcpy(cp.d_count, count.data(), sizeof(int) * CX.n, cudaMemcpyHostToDevice));
  return FSIM_OK;
}

// psplit 1, 3, 9 up to the bra class's primitive pairs; 27 (a ket-primitive
// split on top of nine bra threads) where the bra class has at least 9 and the
// ket class at least 3 primitive pairs.
static bool psplit_legal(const fsim_basis* b, int X, int Y, int ps) {
  if (ps == 27) return b->cls[X].ppmax >= 9 && b->cls[Y].ppmax >= 3;
  return (ps == 1 || ps == 3 || ps == 9) && ps <= b->cls[X].ppmax;
}

// Screened plan for (tau, shard, precision, psplit_force); cached on the basis.
// psplit_force = 0: class pairs with few quartets split the bra primitive pairs
// over several threads so that one launch still covers the device.
int get_plan(fsim_basis* b, double tau, int shard, int nshards, int precision, FockPlan** out, int psplit_force) {
  for (FockPlan* p : b->plans)
    if (p->tau == tau && p->shard == shard && p->nshards == nshards && p->precision == precision &&
        p->psplit_force == psplit_force) {
      *out = p;
      return FSIM_OK;
    }
  FockPlan* P = new FockPlan();
  P->tau = tau;
  P->shard = shard;
  P->nshards = nshards;
  P->precision = precision;
  P->psplit_force = psplit_force;
  b->plans.push_back(P);
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      ClassPairPlan& cp = P->cp[X][Y];
      const DevClass& CX = b->cls[X];
      cp.nbra = CX.n;
      if (CX.n == 0 || b->cls[Y].n == 0) continue;
      std::vector<int> count;
      cp.nquartets = screened_counts(b, X, Y, tau, shard, nshards, count);
      const int coop = 0;  // the cooperative kernel is an autotuner candidate only
      int ps = 1, cs = 1;
      {
        if (psplit_force > 0) {
          ps = std::min(psplit_force, CX.ppmax);
        } else {
          // few quartets: split the bra primitive pairs, then the ket chunks,
          // until one launch has about two CTAs' worth of threads per SM (the
          // ket-primitive split, psplit 27, is left to the autotuner: it
          // repeats the bra transform per ket group and lost on every class
          // pair timed but the smallest)
          const long long target = (long long)device_sm_count() * 2 * kJKThreads;
          for (int c : {3, 9})
            if (cp.nquartets * ps < target && psplit_legal(b, X, Y, c)) ps = c;
          const int nch = jk_chunks_precision(precision, X, Y);
          for (int c : {2, 4})
            if (cp.nquartets * ps * cs < target && c <= nch) cs = c;
        }
      }
      FSIM_TRY(set_class_plan(b, X, Y, count, ps, coop, cp, cs, jk_flat_precision(precision)));
      cp.fp64 = precision == FSIM_DFLOAT && !dfloat_default(X, Y);
      P->nquartets += cp.nquartets;
    }
  // class pairs with an f class: flattened screened (bra, ket) lists, one
  // quartet per CTA of the generic kernel (FP64 in double-float builds)
  for (int X = kNumPairCls; X < kNumPairClsAll; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      ClassPairPlan& cp = P->cp[X][Y];
      cp.nbra = b->cls[X].n;
      if (b->cls[X].n == 0 || b->cls[Y].n == 0) continue;
      std::vector<int> count;
      cp.nquartets = screened_counts(b, X, Y, tau, shard, nshards, count);
      FSIM_TRY(set_class_plan(b, X, Y, count, 1, 0, cp, 1, 1));
      cp.fp64 = precision == FSIM_DFLOAT;
      P->nquartets += cp.nquartets;
    }
  *out = P;
  return FSIM_OK;
}

// The class pairs with an f class, on stream s (their quartet counts are below
// 2^31 by set_class_plan's check).
template <typename Real>
static int launch_f_pairs(fsim_basis* b, FockPlan* plan, const Real* Dr, float boys64_T, double* Jacc,
                          double* Kacc, cudaStream_t s, const double* D64 = nullptr) {
  for (int X = kNumPairClsAll - 1; X >= kNumPairCls; --X)
    for (int Y = X; Y >= 0; --Y) {
      const ClassPairPlan& cp = plan->cp[X][Y];
      if (cp.nquartets == 0) continue;
      cudaError_t e = cudaSuccess;
      if constexpr (std::is_same<Real, dfloat>::value) {
        return launch_f_pairs<double>(b, plan, D64, boys64_T, Jacc, Kacc, s);
      } else {
        GenParams<Real> p{};
        p.bra = b->cls[X].view<Real>();
        p.ket = b->cls[Y].view<Real>();
        p.la = pair_cls_la(X); p.lb = pair_cls_lb(X); p.lc = pair_cls_la(Y); p.ld = pair_cls_lb(Y);
        p.same = X == Y;
        p.list_mode = 0;
        p.prefix = cp.d_prefix;
        p.nitems = (int)cp.nquartets;
        p.N = b->nbf;
        p.D = Dr;
        p.J = Jacc;
        p.K = Kacc;
        p.boys = std::is_same<Real, double>::value ? (const Real*)b->d_boys64 : (const Real*)b->d_boys32;
        p.boys64_T = boys64_T;
        e = launch_gen<Real>(p, s);
      }
      ++b->last_launches;
      if (e != cudaSuccess) {
        set_error("J/K kernel for f class pair (%d|%d): %s", X, Y, cudaGetErrorString(e));
        return FSIM_ECUDA;
      }
    }
  return FSIM_OK;
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// J = (Jacc + Jacc^T)/4, K = (Kacc + Kacc^T)/8 (degeneracy-weighted unique-quartet digestion)
__global__ void symmetrize_kernel(const double* __restrict__ Ja, const double* __restrict__ Ka, double* __restrict__ J,
                                  double* __restrict__ K, int N) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (c >= N) return;
  J[(size_t)r * N + c] = 0.25 * (Ja[(size_t)r * N + c] + Ja[(size_t)c * N + r]);
  K[(size_t)r * N + c] = 0.125 * (Ka[(size_t)r * N + c] + Ka[(size_t)c * N + r]);
}

int ensure_scratch(fsim_basis* b) {
  const size_t n2 = (size_t)b->nbf * b->nbf;
  if (!b->d_Jacc) {
    // set-up of this basis on its device: also make the non-allocating entry
    // point's fixed scratch resident here, so that its calls load nothing
    FSIM_TRY(noalloc_scratch_prepare());
    FSIM_TRY(dev_alloc(&b->d_Jacc, n2));
  }
  if (!b->d_Kacc) FSIM_TRY(dev_alloc(&b->d_Kacc, n2));
  if (!b->d_D32) FSIM_TRY(dev_alloc(&b->d_D32, n2));
  return FSIM_OK;
}

// One class pair's launch with the shape its plan entry holds; J/K
// accumulators passed in (the basis's own or caller-supplied scratch).
// D64: the FP64 density, which a double-float build passes for the class pairs
// it evaluates with the FP64 kernel.
template <typename Real>
static cudaError_t launch_cp(fsim_basis* b, int X, int Y, const ClassPairPlan& cp, const Real* Dr, double* Jacc,
                             double* Kacc, float boys64_T, cudaStream_t s, const double* D64 = nullptr) {
  if constexpr (std::is_same<Real, dfloat>::value) {
    if (!dfloat_kernel(X, Y) || cp.fp64) return launch_cp<double>(b, X, Y, cp, D64, Jacc, Kacc, boys64_T, s);
  }
  const Real* boys = std::is_same<Real, double>::value   ? (const Real*)b->d_boys64
                     : std::is_same<Real, float>::value  ? (const Real*)b->d_boys32
                                                         : (const Real*)b->d_boysx;
  if (cp.nitems == 0) return cudaSuccess;
  if constexpr (!std::is_same<Real, dfloat>::value) {  // the cooperative kernel exists in FP32 and FP64
    if (cp.coop) {
      CoopParams<Real> p{};
      p.bra = b->cls[X].view<Real>();
      p.ket = b->cls[Y].view<Real>();
      make_cls_desc(X, p.bd);
      make_cls_desc(Y, p.kd);
      p.same = X == Y ? 1 : 0;
      p.list_mode = 0;
      p.tile_prefix = cp.d_prefix;
      p.ket_count = cp.d_count;
      p.tq = cp.tq;
      p.nitems = cp.nitems;
      p.N = b->nbf;
      p.D = Dr;
      p.J = Jacc;
      p.K = Kacc;
      p.boys = boys;
      p.boys64_T = boys64_T;
      return launch_coop<Real>(p, cp.nitems, s);
    }
  }
  JKParams<Real> p{};
  p.one = JKMol<Real>{b->cls[X].view<Real>(), b->cls[Y].view<Real>(), cp.d_prefix, cp.d_count, b->nbf, Dr, Jacc, Kacc};
  p.nitems = cp.nitems;
  p.same = X == Y ? 1 : 0;
  p.psplit = cp.psplit;
  p.csplit = cp.csplit;
  p.bra_ppmax = b->cls[X].ppmax;
  p.boys = boys;
  p.boys64_T = boys64_T;
  return dispatch_jk<Real>(X, Y, p, s);
}

// Relative cost of one quartet of a class pair: the algorithmic flop count per
// primitive quartet (R recursion + the cheaper contraction order).
static double class_cost(int X, int Y) {
  const int la = pair_cls_la(X), lb = pair_cls_lb(X), lc = pair_cls_la(Y), ld = pair_cls_lb(Y);
  const double A = ncart(la) * ncart(lb), C = ncart(lc) * ncart(ld);
  const double H1 = nherm(la + lb), H2 = nherm(lc + ld);
  double r = 0.0;
  for (int n = 0; n <= la + lb + lc + ld; ++n) r += nherm(n);
  return 2.0 * r + 2.0 * std::min(A * H1 * H2 + A * C * H2, C * H1 * H2 + A * C * H1) + 16.0;
}

int ensure_aux_streams(fsim_basis* b) {
  if (b->aux_ok) return FSIM_OK;
  for (int k = 0; k < fsim_basis::kAuxStreams; ++k) {
    FSIM_CK(cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking));
    FSIM_CK(cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming));
  }
  FSIM_CK(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
  b->aux_ok = true;
  return FSIM_OK;
}

// The class-pair launches of one build.  Timed builds run them one after the
// other on s (per-class events); otherwise they are spread over s and the
// auxiliary streams, longest first onto the least loaded stream, between a
// fork and a join event on s, so that the short launches and the tails of the
// long ones overlap.  All launches add into the same accumulators (atomics).
template <typename Real>
static int launch_all(fsim_basis* b, FockPlan* plan, const Real* Dr, float boys64_T, bool timing, cudaStream_t s,
                      const double* D64 = nullptr) {
  if (!timing) {
    FSIM_TRY(ensure_aux_streams(b));
    struct Job {
      int X, Y;
      double cost;
    };
    std::vector<Job> jobs;
    for (int X = kNumPairCls - 1; X >= 0; --X)
      for (int Y = X; Y >= 0; --Y) {
        const ClassPairPlan& cp = plan->cp[X][Y];
        const int ci = X * kNumPairCls + Y;
        b->last_class_q[ci] = cp.nquartets;
        b->last_class_run[ci] = cp.nitems > 0;
        if (cp.nitems > 0) jobs.push_back(Job{X, Y, (double)cp.nquartets * class_cost(X, Y)});
      }
    std::stable_sort(jobs.begin(), jobs.end(), [](const Job& a, const Job& c) { return a.cost > c.cost; });
    constexpr int NS = fsim_basis::kAuxStreams + 1;
    cudaStream_t st[NS] = {s};
    for (int k = 0; k < fsim_basis::kAuxStreams; ++k) st[k + 1] = b->aux[k];
    const int nuse = std::min<int>(NS, (int)jobs.size());
    FSIM_CK(cudaEventRecord(b->fork_ev, s));
    for (int k = 1; k < nuse; ++k) FSIM_CK(cudaStreamWaitEvent(st[k], b->fork_ev, 0));
    double load[NS] = {};
    for (const Job& j : jobs) {
      int k = 0;
      for (int t = 1; t < nuse; ++t)
        if (load[t] < load[k]) k = t;
      load[k] += j.cost;
      ++b->last_launches;
      const cudaError_t e = launch_cp<Real>(b, j.X, j.Y, plan->cp[j.X][j.Y], Dr, b->d_Jacc, b->d_Kacc, boys64_T,
                                            st[k], D64);
      if (e != cudaSuccess) {
        set_error("J/K kernel (%d|%d): %s", j.X, j.Y, cudaGetErrorString(e));
        return FSIM_ECUDA;
      }
    }
    FSIM_TRY(launch_f_pairs<Real>(b, plan, Dr, boys64_T, b->d_Jacc, b->d_Kacc, s, D64));
    for (int k = 1; k < nuse; ++k) {
      FSIM_CK(cudaEventRecord(b->join_ev[k - 1], st[k]));
      FSIM_CK(cudaStreamWaitEvent(s, b->join_ev[k - 1], 0));
    }
    return FSIM_OK;
  }
  FSIM_TRY(launch_f_pairs<Real>(b, plan, Dr, boys64_T, b->d_Jacc, b->d_Kacc, s, D64));
  for (int X = kNumPairCls - 1; X >= 0; --X)
    for (int Y = X; Y >= 0; --Y) {
      const ClassPairPlan& cp = plan->cp[X][Y];
      const int ci = X * kNumPairCls + Y;
      b->last_class_q[ci] = cp.nquartets;
      b->last_class_run[ci] = cp.nitems > 0;
      if (cp.nitems == 0) continue;
      ++b->last_launches;
      if (timing) FSIM_CK(cudaEventRecord(b->ev[ci][0], s));
      const cudaError_t e = launch_cp<Real>(b, X, Y, cp, Dr, b->d_Jacc, b->d_Kacc, boys64_T, s, D64);
      if (e != cudaSuccess) {
        set_error("J/K kernel (%d|%d): %s", X, Y, cudaGetErrorString(e));
        return FSIM_ECUDA;
      }
      if (timing) FSIM_CK(cudaEventRecord(b->ev[ci][1], s));
    }
  return FSIM_OK;
}

int fock_build_device(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o) {
  if (o.precision != FSIM_FP64 && o.precision != FSIM_MIXED && o.precision != FSIM_DFLOAT) {
    set_error("fsim_fock_build: precision must be FSIM_FP64, FSIM_MIXED or FSIM_DFLOAT");
    return FSIM_EINVAL;
  }
  if (o.nshards < 1 || o.shard < 0 || o.shard >= o.nshards || !(o.schwarz_tau >= 0.0)) {
    set_error("fsim_fock_build: bad shard (%d of %d) or tau", o.shard, o.nshards);
    return FSIM_EINVAL;
  }
  if (!(o.boys_fp64_T == 0.0 || o.boys_fp64_T >= 30.0)) {
    set_error("fsim_fock_build: boys_fp64_T must be 0 (never) or >= 30 (the FP32 table covers T < 30)");
    return FSIM_EINVAL;
  }
  const float b64 = o.boys_fp64_T > 0.0 ? (float)o.boys_fp64_T : INFINITY;
  cudaStream_t s = (cudaStream_t)o.stream;
  FSIM_TRY(ensure_schwarz(b));
  FSIM_TRY(ensure_scratch(b));
  if (o.precision == FSIM_DFLOAT) FSIM_TRY(ensure_dfloat(b));
  FockPlan* plan = nullptr;
  FSIM_TRY(get_plan(b, o.schwarz_tau, o.shard, o.nshards, o.precision, &plan, 0));
  const int N = b->nbf;
  const size_t n2 = (size_t)N * N;
  if (o.timing && !b->ev_ok) {
    for (auto& pr : b->ev)
      for (auto& e : pr) FSIM_CK(cudaEventCreate(&e));
    b->ev_ok = true;
  }
  b->last_timed = o.timing != 0;
  b->last_stream = s;
  b->last_launches = 0;
  for (auto& r : b->last_class_run) r = false;
  FSIM_CK(cudaMemsetAsync(b->d_Jacc, 0, n2 * sizeof(double), s));
  FSIM_CK(cudaMemsetAsync(b->d_Kacc, 0, n2 * sizeof(double), s));
  if (o.precision == FSIM_MIXED) {
    to_float_kernel<<<256, 256, 0, s>>>(dD, b->d_D32, n2);
    FSIM_CK(cudaGetLastError());
    ++b->last_launches;
    FSIM_TRY(launch_all<float>(b, plan, b->d_D32, b64, o.timing != 0, s));
  } else if (o.precision == FSIM_DFLOAT) {
    launch_split(dD, b->d_Dx, n2, s);
    FSIM_CK(cudaGetLastError());
    ++b->last_launches;
    FSIM_TRY(launch_all<dfloat>(b, plan, b->d_Dx, b64, o.timing != 0, s, dD));
  } else {
    FSIM_TRY(launch_all<double>(b, plan, dD, b64, o.timing != 0, s));
  }
  dim3 grid((N + 127) / 128, N);
  symmetrize_kernel<<<grid, 128, 0, s>>>(b->d_Jacc, b->d_Kacc, dJ, dK, N);
  FSIM_CK(cudaGetLastError());
  ++b->last_launches;
  b->last_quartets = plan->nquartets;
  return FSIM_OK;
}

// Map a shell pair to (class, index in class, swapped) after Schwarz sorting.
struct PairLoc {
  int cls, idx, swapped;
};

static std::vector<PairLoc> pair_locations(const fsim_basis* b) {
  const int ns = b->nshell;
  std::vector<PairLoc> loc((size_t)ns * ns, PairLoc{-1, -1, 0});
  for (int X = 0; X < kNumPairClsAll; ++X)
    for (int j = 0; j < b->cls[X].n; ++j) {
      const int A = b->cls[X].h_idx[j].z, B = b->cls[X].h_idx[j].w;
      loc[(size_t)A * ns + B] = PairLoc{X, j, 0};
      loc[(size_t)B * ns + A] = PairLoc{X, j, 1};
    }
  return loc;
}

}  // namespace fsim

using namespace fsim;

extern "C" {

void fsim_fock_opts_default(fsim_fock_opts* o) {
  if (!o) return;
  o->schwarz_tau = 1e-10;
  o->precision = FSIM_FP64;
  o->boys_fp64_T = 0.0;
  o->ptr_mode = FSIM_PTR_HOST;
  o->stream = nullptr;
  o->shard = 0;
  o->nshards = 1;
  o->timing = 0;
}

int fsim_last_class_times(fsim_basis* b, float* ms, long long* quartets, int* nlaunch) {
  if (!b || !ms || !quartets || !nlaunch) {
    set_error("fsim_last_class_times: null pointer");
    return FSIM_EINVAL;
  }
  FSIM_CK(cudaStreamSynchronize(b->last_stream));
  for (int ci = 0; ci < kNumPairCls * kNumPairCls; ++ci) {
    ms[ci] = -1.0f;
    quartets[ci] = b->last_class_q[ci];
    if (b->last_timed && b->last_class_run[ci]) FSIM_CK(cudaEventElapsedTime(&ms[ci], b->ev[ci][0], b->ev[ci][1]));
  }
  *nlaunch = b->last_launches;
  return FSIM_OK;
}

int fsim_fock_build(fsim_basis* b, const double* D, double* J, double* K, const fsim_fock_opts* opts) {
  if (!b || !D || !J || !K) {
    set_error("fsim_fock_build: null pointer");
    return FSIM_EINVAL;
  }
  fsim_fock_opts o;
  fsim_fock_opts_default(&o);
  if (opts) o = *opts;
  if (o.ptr_mode == FSIM_PTR_DEVICE) return fock_build_ext_device(b, D, J, K, o);
  if (o.ptr_mode != FSIM_PTR_HOST) {
    set_error("fsim_fock_build: bad ptr_mode");
    return FSIM_EINVAL;
  }
  const size_t n2 = (size_t)b->nbf_ext() * b->nbf_ext();
  cudaStream_t s = (cudaStream_t)o.stream;
  if (!b->d_D) FSIM_TRY(dev_alloc(&b->d_D, (size_t)b->nbf * b->nbf));
  if (!b->d_J) FSIM_TRY(dev_alloc(&b->d_J, (size_t)b->nbf * b->nbf));
  if (!b->d_K) FSIM_TRY(dev_alloc(&b->d_K, (size_t)b->nbf * b->nbf));
  FSIM_CK(cudaMemcpyAsync(b->d_D, D, n2 * sizeof(double), cudaMemcpyHostToDevice, s));
  FSIM_TRY(fock_build_ext_device(b, b->d_D, b->d_J, b->d_K, o));
  FSIM_CK(cudaMemcpyAsync(J, b->d_J, n2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FSIM_CK(cudaMemcpyAsync(K, b->d_K, n2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FSIM_CK(cudaStreamSynchronize(s));
  return FSIM_OK;
}

long long fsim_last_quartet_count(const fsim_basis* b) { return b ? b->last_quartets : -1; }

int fsim_eri_quartets(fsim_basis* b, int n, const int* quartets, double* out, int precision) {
  if (!b || (n > 0 && (!quartets || !out)) || n < 0) {
    set_error("fsim_eri_quartets: bad arguments");
    return FSIM_EINVAL;
  }
  if (precision != FSIM_FP64) {
    set_error("fsim_eri_quartets: only FSIM_FP64 blocks are exposed");
    return FSIM_EINVAL;
  }
  FSIM_TRY(ensure_schwarz(b));
  const int ns = b->nshell;
  const std::vector<PairLoc> loc = pair_locations(b);
  struct Req {
    int q;         // request index
    int i, j;      // bra / ket pair indices in their classes
    int sw_bk;     // bra and ket swapped
    int sw1, sw2;  // stored pair order swapped (bra, ket as stored)
  };
  std::vector<Req> groups[kNumPairClsAll][kNumPairClsAll];
  std::vector<size_t> out_off(n + 1, 0);
  for (int q = 0; q < n; ++q) {
    const int* s4 = quartets + 4 * q;
    for (int k = 0; k < 4; ++k)
      if (s4[k] < 0 || s4[k] >= ns) {
        set_error("fsim_eri_quartets: shell index out of range in quartet %d", q);
        return FSIM_EINVAL;
      }
    size_t sz = 1;
    for (int k = 0; k < 4; ++k) sz *= ncart(b->sh_l[s4[k]]);
    out_off[q + 1] = out_off[q] + sz;
    PairLoc p1 = loc[(size_t)s4[0] * ns + s4[1]], p2 = loc[(size_t)s4[2] * ns + s4[3]];
    int sw = 0;
    if (p1.cls < p2.cls) {
      std::swap(p1, p2);
      sw = 1;
    }
    groups[p1.cls][p2.cls].push_back(Req{q, p1.idx, p2.idx, sw, p1.swapped, p2.swapped});
  }
  for (int X = 0; X < kNumPairClsAll; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      auto& G = groups[X][Y];
      if (G.empty()) continue;
      const int ncb = ncart(pair_cls_la(X)) * ncart(pair_cls_lb(X));
      const int nck = ncart(pair_cls_la(Y)) * ncart(pair_cls_lb(Y));
      std::vector<int2> items(G.size());
      for (size_t t = 0; t < G.size(); ++t) items[t] = make_int2(G[t].i, G[t].j);
      double* d_out = nullptr;
      FSIM_TRY(dev_alloc(&d_out, G.size() * ncb * nck));
      int rc = run_list(b, X, Y, items, d_out, FSIM_FP64, 0);
      std::vector<double> h(G.size() * ncb * nck);
      if (rc == FSIM_OK && cudaMemcpy(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = FSIM_ECUDA;
      dev_free(d_out);
      if (rc != FSIM_OK) return rc;
      const int nbA = ncart(pair_cls_lb(X)), nkB = ncart(pair_cls_lb(Y));
      const int naA = ncart(pair_cls_la(X)), nkA = ncart(pair_cls_la(Y));
      for (size_t t = 0; t < G.size(); ++t) {
        const Req& r = G[t];
        const int* s4 = quartets + 4 * r.q;
        const int n0 = ncart(b->sh_l[s4[0]]), n1 = ncart(b->sh_l[s4[1]]), n2c = ncart(b->sh_l[s4[2]]),
                  n3 = ncart(b->sh_l[s4[3]]);
        double* o = out + out_off[r.q];
        const double* blk = h.data() + t * ncb * nck;
        for (int x0 = 0; x0 < n0; ++x0)
          for (int x1 = 0; x1 < n1; ++x1)
            for (int x2 = 0; x2 < n2c; ++x2)
              for (int x3 = 0; x3 < n3; ++x3) {
                // user (ab|cd) -> stored bra pair (first,second) and ket pair
                int ub0 = x0, ub1 = x1, uk0 = x2, uk1 = x3;
                if (r.sw_bk) {
                  std::swap(ub0, uk0);
                  std::swap(ub1, uk1);
                }
                const int sb0 = r.sw1 ? ub1 : ub0, sb1 = r.sw1 ? ub0 : ub1;
                const int sk0 = r.sw2 ? uk1 : uk0, sk1 = r.sw2 ? uk0 : uk1;
                (void)naA; (void)nkA;
                o[((x0 * n1 + x1) * n2c + x2) * n3 + x3] = blk[(sb0 * nbA + sb1) * nck + sk0 * nkB + sk1];
              }
      }
    }
  return FSIM_OK;
}

int fsim_eri_dump(fsim_basis* b, double* g, int precision) {
  if (!b || !g) {
    set_error("fsim_eri_dump: null pointer");
    return FSIM_EINVAL;
  }
  if (b->nbf > 64) {
    set_error("fsim_eri_dump: nbf %d > 64", b->nbf);
    return FSIM_EINVAL;
  }
  const int ns = b->nshell, N = b->nbf;
  std::vector<int> qs;
  for (int a = 0; a < ns; ++a)
    for (int bb = 0; bb <= a; ++bb)
      for (int c = 0; c <= a; ++c)
        for (int d = 0; d <= (c == a ? bb : c); ++d) {
          qs.push_back(a); qs.push_back(bb); qs.push_back(c); qs.push_back(d);
        }
  const int nq = (int)qs.size() / 4;
  size_t tot = 0;
  std::vector<size_t> off(nq);
  for (int q = 0; q < nq; ++q) {
    off[q] = tot;
    size_t sz = 1;
    for (int k = 0; k < 4; ++k) sz *= ncart(b->sh_l[qs[4 * q + k]]);
    tot += sz;
  }
  std::vector<double> blocks(tot);
  FSIM_TRY(fsim_eri_quartets(b, nq, qs.data(), blocks.data(), precision));
  for (int q = 0; q < nq; ++q) {
    const int s[4] = {qs[4 * q], qs[4 * q + 1], qs[4 * q + 2], qs[4 * q + 3]};
    int nc[4];
    for (int k = 0; k < 4; ++k) nc[k] = ncart(b->sh_l[s[k]]);
    const double* blk = blocks.data() + off[q];
    for (int x0 = 0; x0 < nc[0]; ++x0)
      for (int x1 = 0; x1 < nc[1]; ++x1)
        for (int x2 = 0; x2 < nc[2]; ++x2)
          for (int x3 = 0; x3 < nc[3]; ++x3) {
            const double v = blk[((x0 * nc[1] + x1) * nc[2] + x2) * nc[3] + x3];
            const size_t m = b->sh_ao[s[0]] + x0, nn = b->sh_ao[s[1]] + x1, l = b->sh_ao[s[2]] + x2,
                         sg = b->sh_ao[s[3]] + x3;
            const size_t idx[8][4] = {{m, nn, l, sg}, {nn, m, l, sg}, {m, nn, sg, l}, {nn, m, sg, l},
                                      {l, sg, m, nn}, {sg, l, m, nn}, {l, sg, nn, m}, {sg, l, nn, m}};
            for (auto& t : idx) g[((t[0] * N + t[1]) * N + t[2]) * N + t[3]] = v;
          }
  }
  return FSIM_OK;
}

}  // extern "C"

namespace fsim {

// ---------------------------------------------------------------------------
// Fock build into caller-supplied scratch (used by fsim_fock_build_noalloc in
// noalloc.cu).  Same kernels and plan as fock_build_device, but the J/K
// accumulators and the FP32 density copy live in the memory passed in, and no
// step allocates: the Schwarz bounds and the screening plan for these options
// must already exist on the basis.
// ---------------------------------------------------------------------------
template <typename Real>
static int launch_all_into(fsim_basis* b, FockPlan* plan, const Real* Dr, float boys64_T, double* Jacc,
                           double* Kacc, cudaStream_t s) {
  for (int X = kNumPairCls - 1; X >= 0; --X)
    for (int Y = X; Y >= 0; --Y) {
      if (plan->cp[X][Y].nitems > 0) ++b->last_launches;
      const cudaError_t e = launch_cp<Real>(b, X, Y, plan->cp[X][Y], Dr, Jacc, Kacc, boys64_T, s);
      if (e != cudaSuccess) {
        set_error("J/K kernel (%d|%d): %s", X, Y, cudaGetErrorString(e));
        return FSIM_ECUDA;
      }
    }
  return launch_f_pairs<Real>(b, plan, Dr, boys64_T, Jacc, Kacc, s);
}

int fock_build_into(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o, double* Jacc,
                    double* Kacc, float* D32) {
  if (o.precision != FSIM_FP64 && o.precision != FSIM_MIXED) {
    set_error("precision must be FSIM_FP64 or FSIM_MIXED");
    return FSIM_EINVAL;
  }
  if (o.nshards < 1 || o.shard < 0 || o.shard >= o.nshards || !(o.schwarz_tau >= 0.0)) {
    set_error("bad shard (%d of %d) or tau", o.shard, o.nshards);
    return FSIM_EINVAL;
  }
  if (!(o.boys_fp64_T == 0.0 || o.boys_fp64_T >= 30.0)) {
    set_error("boys_fp64_T must be 0 (never) or >= 30");
    return FSIM_EINVAL;
  }
  if (!b->schwarz_done) {
    set_error("no Schwarz bounds yet: call fsim_schwarz (or fsim_fock_build) during set-up");
    return FSIM_EINVAL;
  }
  FockPlan* plan = nullptr;
  for (FockPlan* p : b->plans)
    if (p->tau == o.schwarz_tau && p->shard == o.shard && p->nshards == o.nshards && p->precision == o.precision &&
        p->psplit_force == 0)
      plan = p;
  if (!plan) {
    set_error("no screening plan for tau %g, shard %d/%d, precision %d: run fsim_fock_build once with the same "
              "options during set-up",
              o.schwarz_tau, o.shard, o.nshards, o.precision);
    return FSIM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)o.stream;
  const int N = b->nbf;
  const size_t n2 = (size_t)N * N;
  // what fsim_last_quartet_count / fsim_last_class_times report for this build
  b->last_timed = false;
  b->last_stream = s;
  b->last_launches = 0;
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y < kNumPairCls; ++Y) {
      const int ci = X * kNumPairCls + Y;
      b->last_class_run[ci] = Y <= X && plan->cp[X][Y].nitems > 0;
      b->last_class_q[ci] = Y <= X ? plan->cp[X][Y].nquartets : 0;
    }
  FSIM_CK(cudaMemsetAsync(Jacc, 0, n2 * sizeof(double), s));
  FSIM_CK(cudaMemsetAsync(Kacc, 0, n2 * sizeof(double), s));
  const float b64 = o.boys_fp64_T > 0.0 ? (float)o.boys_fp64_T : INFINITY;
  if (o.precision == FSIM_MIXED) {
    to_float_kernel<<<256, 256, 0, s>>>(dD, D32, n2);
    FSIM_CK(cudaGetLastError());
    ++b->last_launches;
    FSIM_TRY(launch_all_into<float>(b, plan, D32, b64, Jacc, Kacc, s));
  } else {
    FSIM_TRY(launch_all_into<double>(b, plan, dD, b64, Jacc, Kacc, s));
  }
  dim3 grid((N + 127) / 128, N);
  symmetrize_kernel<<<grid, 128, 0, s>>>(Jacc, Kacc, dJ, dK, N);
  FSIM_CK(cudaGetLastError());
  ++b->last_launches;
  b->last_quartets = plan->nquartets;
  return FSIM_OK;
}

}  // namespace fsim

namespace fsim {

template <typename Real>
static int autotune_impl(fsim_basis* b, FockPlan* plan, const Real* Dr, float b64, cudaStream_t s, int* choice,
                         float* best_ms, const double* D64 = nullptr) {
  cudaEvent_t e0, e1;
  FSIM_CK(cudaEventCreate(&e0));
  FSIM_CK(cudaEventCreate(&e1));
  int rc = FSIM_OK;
  for (int X = 0; X < kNumPairCls && rc == FSIM_OK; ++X)
    for (int Y = 0; Y <= X && rc == FSIM_OK; ++Y) {
      ClassPairPlan& cp = plan->cp[X][Y];
      const int ci = X * kNumPairCls + Y;
      if (cp.nquartets == 0) continue;
      std::vector<int> count;
      screened_counts(b, X, Y, plan->tau, plan->shard, plan->nshards, count);
      struct Cand {
        int psplit, coop, csplit, fp64;
      };
      std::vector<Cand> cands;
      const int nch = jk_chunks<Real>(X, Y);
      // the ket-primitive split (psplit 27) is tried only where nine threads
      // per quartet leave the device short of two CTAs per SM
      const long long fill = (long long)device_sm_count() * 2 * kJKThreads;
      constexpr bool kDf = std::is_same<Real, dfloat>::value;
      // double-float builds: each shape with the double-float and with the FP64 kernel
      const int f64_lo = kDf && !dfloat_kernel(X, Y) ? 1 : 0, f64_hi = kDf ? 1 : 0;
      for (int f64 = f64_lo; f64 <= f64_hi; ++f64)
        for (int ps : {1, 3, 9, 27})
          for (int cs : {1, 2, 4})
            if (psplit_legal(b, X, Y, ps) && cs <= nch && (ps < 27 || cp.nquartets * 9 < fill))
              cands.push_back({ps, 0, cs, f64});
      if (!kDf) cands.push_back({1, 1, 1, 0});
      float best = 1e30f;
      Cand win = cands[0];
      ClassPairPlan tmp;
      for (const Cand& c : cands) {
        if ((rc = set_class_plan(b, X, Y, count, c.psplit, c.coop, tmp, c.csplit, jk_flat<Real>())) != FSIM_OK)
          break;
        tmp.fp64 = c.fp64;
        float t[3];
        cudaError_t e = launch_cp<Real>(b, X, Y, tmp, Dr, b->d_Jacc, b->d_Kacc, b64, s, D64);  // warm-up
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
          cudaEventRecord(e0, s);
          e = launch_cp<Real>(b, X, Y, tmp, Dr, b->d_Jacc, b->d_Kacc, b64, s, D64);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&t[r], e0, e1);
        }
        if (e != cudaSuccess) {
          set_error("autotune launch (%d|%d): %s", X, Y, cudaGetErrorString(e));
          rc = FSIM_ECUDA;
          break;
        }
        std::sort(t, t + 3);
        if (t[1] < best) {
          best = t[1];
          win = c;
        }
      }
      dev_free(tmp.d_prefix);
      dev_free(tmp.d_count);
      if (rc != FSIM_OK) break;
      rc = set_class_plan(b, X, Y, count, win.psplit, win.coop, cp, win.csplit, jk_flat<Real>());
      cp.fp64 = win.fp64;
      if (choice) choice[ci] = win.coop ? -1 : 10 * win.psplit + win.csplit + 1000 * win.fp64;
      if (best_ms) best_ms[ci] = best;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FSIM_OK) plan->tuned = true;
  return rc;
}

}  // namespace fsim

extern "C" int fsim_set_launch(fsim_basis* b, const fsim_fock_opts* opts, const int* choice) {
  if (!b || !opts || !choice) {
    set_error("fsim_set_launch: null pointer");
    return FSIM_EINVAL;
  }
  const fsim_fock_opts& o = *opts;
  if (o.precision != FSIM_FP64 && o.precision != FSIM_MIXED && o.precision != FSIM_DFLOAT) {
    set_error("fsim_set_launch: bad precision");
    return FSIM_EINVAL;
  }
  FSIM_TRY(ensure_schwarz(b));
  FockPlan* plan = nullptr;
  FSIM_TRY(get_plan(b, o.schwarz_tau, o.shard, o.nshards, o.precision, &plan, 0));
  const bool df = o.precision == FSIM_DFLOAT;
  for (int X = 0; X < kNumPairCls; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const int c = choice[X * kNumPairCls + Y];
      ClassPairPlan& cp = plan->cp[X][Y];
      if (c == 0 || cp.nquartets == 0) continue;
      const int coop = c == -1 ? 1 : 0;
      const int f64 = c >= 1000 ? 1 : 0, ps = coop ? 1 : (c % 1000) / 10, cs = coop ? 1 : c % 10;
      const bool ok = c >= -1 && c < 2000 && (coop ? !df : (psplit_legal(b, X, Y, ps) &&
                                                          (cs == 1 || cs == 2 || cs == 4) &&
                                                          cs <= jk_chunks_precision(o.precision, X, Y))) &&
                      (!f64 || df) && (!df || f64 || dfloat_kernel(X, Y));
      if (!ok) {
        set_error("fsim_set_launch: choice %d not valid for class pair (%d|%d) in precision %d", c, X, Y, o.precision);
        return FSIM_EINVAL;
      }
      std::vector<int> count;
      screened_counts(b, X, Y, plan->tau, plan->shard, plan->nshards, count);
      FSIM_TRY(set_class_plan(b, X, Y, count, ps, coop, cp, cs, jk_flat_precision(o.precision)));
      cp.fp64 = df && (f64 || !dfloat_kernel(X, Y));
    }
  return FSIM_OK;
}

extern "C" int fsim_autotune(fsim_basis* b, const fsim_fock_opts* opts, int* choice, float* best_ms) {
  if (!b || !opts) {
    set_error("fsim_autotune: null pointer");
    return FSIM_EINVAL;
  }
  const fsim_fock_opts& o = *opts;
  if (o.precision != FSIM_FP64 && o.precision != FSIM_MIXED && o.precision != FSIM_DFLOAT) {
    set_error("fsim_autotune: bad precision");
    return FSIM_EINVAL;
  }
  if (choice)
    for (int i = 0; i < 36; ++i) choice[i] = 0;
  if (best_ms)
    for (int i = 0; i < 36; ++i) best_ms[i] = -1.0f;
  FSIM_TRY(ensure_schwarz(b));
  FSIM_TRY(ensure_scratch(b));
  if (o.precision == FSIM_DFLOAT) FSIM_TRY(ensure_dfloat(b));
  FockPlan* plan = nullptr;
  FSIM_TRY(get_plan(b, o.schwarz_tau, o.shard, o.nshards, o.precision, &plan, 0));
  cudaStream_t s = (cudaStream_t)o.stream;
  const size_t n2 = (size_t)b->nbf * b->nbf;
  const float b64 = o.boys_fp64_T > 0.0 ? (float)o.boys_fp64_T : INFINITY;
  if (o.precision == FSIM_MIXED) {
    FSIM_CK(cudaMemsetAsync(b->d_D32, 0, n2 * sizeof(float), s));
    return autotune_impl<float>(b, plan, b->d_D32, b64, s, choice, best_ms);
  }
  if (o.precision == FSIM_DFLOAT) {
    // zero bytes: also a zero FP64 density of the same size for the FP64-evaluated class pairs
    FSIM_CK(cudaMemsetAsync(b->d_Dx, 0, n2 * sizeof(dfloat), s));
    return autotune_impl<dfloat>(b, plan, b->d_Dx, b64, s, choice, best_ms, reinterpret_cast<const double*>(b->d_Dx));
  }
  double* Dz = nullptr;
  FSIM_TRY(dev_alloc(&Dz, n2));
  FSIM_CK(cudaMemsetAsync(Dz, 0, n2 * sizeof(double), s));
  int rc = autotune_impl<double>(b, plan, Dz, b64, s, choice, best_ms);
  cudaStreamSynchronize(s);
  dev_free(Dz);
  return rc;
}
