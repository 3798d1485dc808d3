// Internal state of a basis handle and helpers shared by the host-side
// translation units of libfsim.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/fsim.h"
#include "eri_core.cuh"

namespace fsim {

constexpr int kMaxPrim = 4;

void set_error(const char* fmt, ...);

#define FSIM_CK(x)                                                                              \
  do {                                                                                          \
    cudaError_t e_ = (x);                                                                       \
    if (e_ != cudaSuccess) {                                                                    \
      ::fsim::set_error("CUDA error '%s' in %s (%s:%d)", cudaGetErrorString(e_), #x, __FILE__, \
                        __LINE__);                                                              \
      return FSIM_ECUDA;                                                                        \
    }                                                                                           \
  } while (0)

#define FSIM_TRY(x)           \
  do {                        \
    int r_ = (x);             \
    if (r_ != FSIM_OK) return r_; \
  } while (0)

template <typename T>
int dev_alloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
    return FSIM_ENOMEM;
  }
  return FSIM_OK;
}

template <typename T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// One pair class (ss, ps, pp, ds, dp, dd) on the device.
struct DevClass {
  int n = 0;
  int ppmax = 1;
  int nnz = 0;
  int4* idx = nullptr;      // (ao_a, ao_b, shell_a, shell_b), sorted by Q descending
  int* npp = nullptr;
  double* pd64 = nullptr;   // [4 + nnz][ppmax][n]
  float* pd32 = nullptr;
  double4_32a* pq64 = nullptr;  // (p, P) at [ppmax][n]
  float4* pq32 = nullptr;
  dfloat* pdx = nullptr;    // double-float copies of pd64 / pq64 (made on first FSIM_DFLOAT use)
  dfloat4* pqx = nullptr;
  std::vector<int4> h_idx;  // host copy, same order
  std::vector<int> h_npp;
  std::vector<double> h_Q;  // Schwarz bound of each pair, same order
  double* d_Q = nullptr;    // device copy of h_Q
  int nfield() const { return 4 + nnz; }
  template <typename Real>
  PairView<Real> view() const;
};

template <>
inline PairView<double> DevClass::view<double>() const {
  return PairView<double>{n, ppmax, idx, npp, pd64, pq64};
}
template <>
inline PairView<float> DevClass::view<float>() const {
  return PairView<float>{n, ppmax, idx, npp, pd32, pq32};
}
template <>
inline PairView<dfloat> DevClass::view<dfloat>() const {
  return PairView<dfloat>{n, ppmax, idx, npp, pdx, pqx};
}

// Ket components per register chunk.  The per-thread registers of the unrolled
// kernel hold R (nherm(L)), the chunk's W (bra Hermite terms x CS) and the
// chunk's E non-zeros; the quartet block itself lives in shared memory.  The
// largest chunk whose estimate (in values, not registers) fits the budget is
// taken (the last chunk may be shorter; chunks are balanced), capped by the
// shared memory of the per-thread quartet blocks.  Every extra chunk repeats
// the Boys function and the Hermite recursion, so larger chunks win until
// spills or lost occupancy cost more: the budgets were set by timing every
// class pair on the 12- and 30-atom organic clouds at several budgets.
// FP64 classes with L <= 4 keep the whole quartet in one chunk: GB300 issues
// FP64 FMAs at a small fraction of the FP32 rate, so arrays that overflow into
// L1-resident local memory cost little next to repeated FP64 recursions.
#ifndef FSIM_CHUNK_REG_BUDGET
#define FSIM_CHUNK_REG_BUDGET 230
#endif
#ifndef FSIM_CHUNK_REG_BUDGET64
#define FSIM_CHUNK_REG_BUDGET64 350
#endif
constexpr int kChunkRegBudget = FSIM_CHUNK_REG_BUDGET;
// shared memory for the per-thread quartet blocks and J_bra partials of a CTA
constexpr size_t kJKBlockSmemMax = 160 * 1024;
constexpr int kChunkRegBudget64 = FSIM_CHUNK_REG_BUDGET64;

__host__ __device__ constexpr int pair_comp_nnz(int la, int lb, int c) {
  int p = 1;
  for (int ax = 0; ax < 3; ++ax) p *= cart_comp(la, c / ncart(lb), ax) + cart_comp(lb, c % ncart(lb), ax) + 1;
  return p;
}

__host__ __device__ constexpr int chunk_nnz_max(int lc, int ld, int cs) {
  const int C = ncart(lc) * ncart(ld);
  int m = 0;
  for (int c0 = 0; c0 < C; c0 += cs) {
    int z = 0;
    for (int c = c0; c < c0 + cs && c < C; ++c) z += pair_comp_nnz(lc, ld, c);
    m = z > m ? z : m;
  }
  return m;
}

template <typename Real>
__host__ __device__ constexpr int chunk_size(int X, int Y) {
  const int lc = pair_cls_la(Y), ld = pair_cls_lb(Y);
  const int C = ncart(lc) * ncart(ld);
  // measured exception: FP32 (dd|dd) runs faster with two-component chunks than
  // the budget rule's one (class times on the 12- and 30-atom organic clouds)
  if (sizeof(Real) == 4 && X == 5 && Y == 5) return 2;
  if (sizeof(Real) == 8 && pair_cls_la(X) + pair_cls_lb(X) + lc + ld <= 4) return C;
  const int budget = sizeof(Real) == 8 ? kChunkRegBudget64 : kChunkRegBudget;
  const int H1 = nherm(pair_cls_la(X) + pair_cls_lb(X));
  const int NH = nherm(pair_cls_la(X) + pair_cls_lb(X) + lc + ld);
  const int A = ncart(pair_cls_la(X)) * ncart(pair_cls_lb(X));
  for (int cs = C; cs > 1; --cs)
    if (NH + H1 * cs + chunk_nnz_max(lc, ld, cs) <= budget &&
        (size_t)(cs + 1) * A * kJKThreads * sizeof(Real) <= kJKBlockSmemMax) {
      const int nch = (C + cs - 1) / cs;
      return (C + nch - 1) / nch;  // same chunk count, balanced sizes
    }
  return 1;
}

// Class pairs that have a double-float kernel: all but (dd|dp) and (dd|dd),
// whose fully unrolled double-float code takes minutes to compile and spills
// far more than the FP64 kernel; FSIM_DFLOAT builds run those two in FP64.
__host__ __device__ constexpr bool dfloat_kernel(int X, int Y) { return !(X == 5 && Y >= 4); }
// Default kernel of a class pair in an FSIM_DFLOAT build (the autotuner times
// both): double-float up to total angular momentum 4, where the Boys function
// and the prologue weigh most (measured on (H2O)_8: 3-8x faster than FP64);
// FP64 from 5, where R and the chunk's W outgrow 255 registers at two per value
// and live in L1-backed local memory, which the double-float kernel, at 15 FP32
// instructions per multiply-add, cannot feed fast enough: the two run even.
__host__ __device__ constexpr bool dfloat_default(int X, int Y) {
  return dfloat_kernel(X, Y) && pair_cls_la(X) + pair_cls_lb(X) + pair_cls_la(Y) + pair_cls_lb(Y) <= 4;
}
static_assert(sizeof(dfloat) == sizeof(double), "double-float values share the FP64 layouts and chunk sizes");

// Ket chunks of the unrolled kernel for a class pair (host side of KetChunks).
template <typename Real>
__host__ __device__ constexpr int jk_chunks(int X, int Y) {
  return (ncart(pair_cls_la(Y)) * ncart(pair_cls_lb(Y)) + chunk_size<Real>(X, Y) - 1) / chunk_size<Real>(X, Y);
}

// Screened work list of one class pair (bra class X >= ket class Y).
struct ClassPairPlan {
  int nbra = 0;
  int nitems = 0;
  long long nquartets = 0;
  int psplit = 1;
  int csplit = 1;           // ket chunk groups per CTA (unrolled kernel)
  int coop = 0;             // 1: warp-cooperative table-driven kernel
  int fp64 = 0;             // FSIM_DFLOAT plans: 1 = this class pair runs the FP64 kernel
  int tq = kJKThreads;      // kets per work item
  int* d_prefix = nullptr;  // [nbra + 1]
  int* d_count = nullptr;   // [nbra]
};

// Screened work lists of a Coulomb-only (J-engine) build: every ordered
// (bra class X, ket class Y), kets j of bra i with Q_i Q_j >= tau.
struct JPlan {
  double tau = -1.0;
  int shard = 0, nshards = 1;
  int precision = 0;
  ClassPairPlan cp[kNumPairCls][kNumPairCls];
  long long nquartets = 0;
};

struct FockPlan {
  double tau = -1.0;
  int shard = 0, nshards = 1;
  int precision = 0;
  int psplit_force = 0;
  bool tuned = false;
  // s/p/d class pairs at [X][Y], X, Y < kNumPairCls; the class pairs with an f
  // class (X >= kNumPairCls) hold flattened quartet lists for the generic kernel
  ClassPairPlan cp[kNumPairClsAll][kNumPairClsAll];
  long long nquartets = 0;
};

template <typename Real>
struct GenParams;
template <typename Real>
cudaError_t launch_gen(const GenParams<Real>& p, cudaStream_t s);

// Kernel launchers (explicit instantiations in eri_inst_*.cu).
template <typename Real, int X, int Y>
cudaError_t launch_jk(const JKParams<Real>& p, cudaStream_t s);
template <typename Real>
struct CoopParams;
template <typename Real>
cudaError_t launch_coop(const CoopParams<Real>& p, int nblocks, cudaStream_t s);


}  // namespace fsim

struct fsim_basis {
  int device = 0;
  int natom = 0, nshell = 0, nbf = 0;  // nbf: Cartesian functions (the integral engine's basis)
  // spherical (real solid-harmonic) basis on top of the Cartesian engine: nsph
  // functions, T rows (index, coef) x 3 and T columns (index, coef) x 2
  int spherical = 0, nsph = 0;
  int* d_sti = nullptr;
  double* d_stc = nullptr;
  int* d_sci = nullptr;
  double* d_scc = nullptr;
  double* d_cD = nullptr;  // Cartesian D, J, K of a spherical build
  double* d_cJ = nullptr;
  double* d_cK = nullptr;
  int nbf_ext() const { return spherical ? nsph : nbf; }
  std::vector<int> Z;
  std::vector<double> axyz;
  std::vector<int> sh_atom, sh_l, sh_nprim, sh_ao;
  std::vector<double> sh_alpha;  // kMaxPrim per shell
  std::vector<double> sh_coef;   // d_k (2a/pi)^{3/4} (4a)^{l/2} N_contr, kMaxPrim per shell
  // device copies of the shell data
  double* d_cen = nullptr;
  double* d_alpha = nullptr;
  double* d_coef = nullptr;
  int* d_nprim = nullptr;
  int* d_l = nullptr;
  int* d_ao = nullptr;
  double* d_axyz = nullptr;
  int* d_Z = nullptr;
  fsim::DevClass cls[fsim::kNumPairClsAll];
  bool schwarz_done = false;
  std::vector<double> Q;  // nshell x nshell
  double* d_boys64 = nullptr;
  float* d_boys32 = nullptr;
  fsim::dfloat* d_boysx = nullptr;  // double-float copy of the FP64 table (first FSIM_DFLOAT use)
  bool dfloat_ready = false;
  std::vector<fsim::FockPlan*> plans;
  std::vector<fsim::JPlan*> jplans;
  // density-contracted ket Hermite vectors of a J-engine build, per pair class
  float* d_rho32[fsim::kNumPairCls] = {};
  double* d_rho64[fsim::kNumPairCls] = {};
  long long last_quartets = 0;
  // scratch
  double* d_Jacc = nullptr;
  double* d_Kacc = nullptr;
  double* d_D = nullptr;   // staging for host-pointer calls / outputs
  double* d_J = nullptr;
  double* d_K = nullptr;
  float* d_D32 = nullptr;
  fsim::dfloat* d_Dx = nullptr;  // double-float density copy
  // per class-pair timing of the last build
  cudaEvent_t ev[fsim::kNumPairCls * fsim::kNumPairCls][2] = {};
  bool ev_ok = false;
  bool last_timed = false;
  int last_launches = 0;
  long long last_class_q[fsim::kNumPairCls * fsim::kNumPairCls] = {};
  bool last_class_run[fsim::kNumPairCls * fsim::kNumPairCls] = {};
  cudaStream_t last_stream = nullptr;
  // auxiliary streams of the concurrent class-pair launches (created on first use)
  static constexpr int kAuxStreams = 3;
  cudaStream_t aux[kAuxStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kAuxStreams] = {};
  bool aux_ok = false;
};

namespace fsim {
int get_plan(fsim_basis* b, double tau, int shard, int nshards, int precision, FockPlan** out, int psplit_force);
int set_class_plan(fsim_basis* b, int X, int Y, const std::vector<int>& count, int psplit, int coop,
                   ClassPairPlan& cp, int csplit, int flat);
// the unrolled kernel's work decomposition of a precision (see jk_kernel)
inline int jk_flat_precision(int precision) {
  return precision == FSIM_MIXED ? (int)jk_flat<float>() : (int)jk_flat<double>();  // dfloat: as FP64
}
// ket chunks of a class pair in the precision's kernel
inline int jk_chunks_precision(int precision, int X, int Y) {
  return precision == FSIM_MIXED ? jk_chunks<float>(X, Y) : jk_chunks<double>(X, Y);  // dfloat: as FP64
}
// double-float pair data, Boys table and density buffer (allocated on first use)
int ensure_dfloat(fsim_basis* b);
// out[i] = nearest dfloat of in[i]
void launch_split(const double* in, dfloat* out, size_t n, cudaStream_t s);
int ensure_scratch(fsim_basis* b);
// Looks up, once per device (the current one), the device address of the fixed
// scratch array of fsim_fock_build_noalloc; loading that array's module is the
// only device memory this takes (noalloc.cu).
int noalloc_scratch_prepare();
int ensure_schwarz(fsim_basis* b);
int ensure_aux_streams(fsim_basis* b);
// true when the basis has f shells (class pairs served by the generic kernel)
inline bool has_f(const fsim_basis* b);
// input, hidden and output widths of a network handle (mlp.cu)
void mlp_dims(const fsim_mlp* net, int* nin, int* width, int* nout);
int device_sm_count();
int build_pair_data(fsim_basis* b, int cls, const std::vector<int4>& order);
int run_list(fsim_basis* b, int X, int Y, const std::vector<int2>& items, double* d_out, int precision,
             cudaStream_t s);
int fock_build_device(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o);
// the same in the basis the caller sees (spherical when the basis is)
int fock_build_ext_device(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o);
int onee_ext_device(fsim_basis* b, int which, double* out, cudaStream_t s);
int sph_setup(fsim_basis* b);
int onee_device(fsim_basis* b, int which, double* d_out, cudaStream_t s);
}  // namespace fsim

inline bool fsim::has_f(const fsim_basis* b) {
  for (int X = kNumPairCls; X < kNumPairClsAll; ++X)
    if (b->cls[X].n > 0) return true;
  return false;
}
