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
  std::vector<int4> h_idx;  // host copy, same order
  std::vector<int> h_npp;
  std::vector<double> h_Q;  // Schwarz bound of each pair, same order
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

// Screened work list of one class pair (bra class X >= ket class Y).
struct ClassPairPlan {
  int nbra = 0;
  int nitems = 0;
  long long nquartets = 0;
  int psplit = 1;
  int coop = 0;             // 1: warp-cooperative table-driven kernel
  int cw = 0;               // 1: chunk-warp variant of the unrolled kernel (FP32)
  int tq = kJKThreads;      // kets per work item
  int* d_prefix = nullptr;  // [nbra + 1]
  int* d_count = nullptr;   // [nbra]
};

struct FockPlan {
  double tau = -1.0;
  int shard = 0, nshards = 1;
  int precision = 0;
  int psplit_force = 0;
  bool tuned = false;
  ClassPairPlan cp[kNumPairCls][kNumPairCls];
  long long nquartets = 0;
};

// Kernel launchers (explicit instantiations in eri_inst_*.cu).
template <typename Real, int X, int Y>
cudaError_t launch_jk(const JKParams<Real>& p, cudaStream_t s);
template <typename Real, int X, int Y>
cudaError_t launch_jk_cw(const JKParams<Real>& p, cudaStream_t s);
template <typename Real>
struct CoopParams;
template <typename Real>
cudaError_t launch_coop(const CoopParams<Real>& p, int nblocks, cudaStream_t s);
// FP64 classes with L = la+lb+lc+ld >= this run on the cooperative kernel
constexpr int kCoopMinL64 = 5;

}  // namespace fsim

struct fsim_basis {
  int device = 0;
  int natom = 0, nshell = 0, nbf = 0;
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
  fsim::DevClass cls[fsim::kNumPairCls];
  bool schwarz_done = false;
  std::vector<double> Q;  // nshell x nshell
  double* d_boys64 = nullptr;
  float* d_boys32 = nullptr;
  std::vector<fsim::FockPlan*> plans;
  long long last_quartets = 0;
  // scratch
  double* d_Jacc = nullptr;
  double* d_Kacc = nullptr;
  double* d_D = nullptr;   // staging for host-pointer calls / outputs
  double* d_J = nullptr;
  double* d_K = nullptr;
  float* d_D32 = nullptr;
  // per class-pair timing of the last build
  cudaEvent_t ev[fsim::kNumPairCls * fsim::kNumPairCls][2] = {};
  bool ev_ok = false;
  bool last_timed = false;
  int last_launches = 0;
  long long last_class_q[fsim::kNumPairCls * fsim::kNumPairCls] = {};
  bool last_class_run[fsim::kNumPairCls * fsim::kNumPairCls] = {};
  cudaStream_t last_stream = nullptr;
};

namespace fsim {
int get_plan(fsim_basis* b, double tau, int shard, int nshards, int precision, FockPlan** out, int psplit_force);
int set_class_plan(fsim_basis* b, int X, int Y, const std::vector<int>& count, int psplit, int coop,
                   ClassPairPlan& cp, int cw = 0);
bool has_cw_variant(int X, int Y);
int ensure_scratch(fsim_basis* b);
int ensure_schwarz(fsim_basis* b);
int device_sm_count();
int build_pair_data(fsim_basis* b, int cls, const std::vector<int4>& order);
int run_list(fsim_basis* b, int X, int Y, const std::vector<int2>& items, double* d_out, int precision,
             cudaStream_t s);
int fock_build_device(fsim_basis* b, const double* dD, double* dJ, double* dK, const fsim_fock_opts& o);
int onee_device(fsim_basis* b, int which, double* d_out, cudaStream_t s);
}  // namespace fsim
