// Learned initial density: per-atom-pair features, pair-local frames, and the
// rotation/assembly of predicted density blocks.
//
// For an atom pair (A, B), A <= B, the density block D_AB (functions of A x
// functions of B) is represented in a frame attached to the pair: z along
// A -> B, x towards the atom C nearest to the pair's midpoint (its component
// perpendicular to z), y = z x x.  For A == B: z towards the nearest
// neighbour, x towards the second nearest.  If the molecule is rotated by R,
// basis functions transform as phi'(R s) = U phi(s) shell by shell (s: 1, p: R,
// Cartesian d: the map of degree-2 monomials under R, rescaled by the
// component normalisation), and a rotation-covariant density obeys
// D' = U^{-T} D U^{-1}.  With R = the frame's rotation, the local block
// L = U_A^{-T} D_AB U_B^{-1} depends only on the pair's internal geometry, which
// the network sees through invariant features; D_AB = U_A^T L U_B maps it back.
// Features (48 per pair): r_AB / 10; one-hot element of A and of B (H, C, N,
// O); 32 Gaussian radial basis values of r_AB (centres 0..10 bohr, width 0.4);
// distances / 10 of the frame atom(s) to A and B; one-hot element of the frame
// atom; a flag for A == B.
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "fsim_internal.h"

namespace fsim {
namespace {

constexpr int kFeat = 48;
constexpr int kMaxF = 15;  // functions per atom of the supported bases (3s 2p 1d)
constexpr int kOut = kMaxF * kMaxF;

int elem_slot(int Z) { return Z == 1 ? 0 : Z == 6 ? 1 : Z == 7 ? 2 : Z == 8 ? 3 : -1; }

struct AtomFns {
  int first = 0, n = 0;
  std::vector<int> shell_l;
};

int atom_layout(const fsim_basis* b, std::vector<AtomFns>& at) {
  at.assign(b->natom, AtomFns());
  std::vector<int> last(b->natom, -1);
  for (int s = 0; s < b->nshell; ++s) {
    const int a = b->sh_atom[s];
    if (at[a].n == 0) at[a].first = b->sh_ao[s];
    else if (b->sh_ao[s] != at[a].first + at[a].n) {
      set_error("learned guess: the shells of atom %d are not contiguous", a);
      return FSIM_EINVAL;
    }
    at[a].n += ncart(b->sh_l[s]);
    at[a].shell_l.push_back(b->sh_l[s]);
  }
  for (int a = 0; a < b->natom; ++a)
    if (at[a].n > kMaxF) {
      set_error("learned guess: atom %d has %d functions (at most %d supported)", a, at[a].n, kMaxF);
      return FSIM_EINVAL;
    }
  return FSIM_OK;
}

using M3 = std::array<std::array<double, 3>, 3>;

void vsub(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i) c[i] = a[i] - b[i];
}
double vnorm(const double* a) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

// rows: local x, y, z in global coordinates
M3 frame_from(const double* z_in, const double* xhint) {
  double z[3], x[3], y[3];
  const double nz = vnorm(z_in);
  for (int i = 0; i < 3; ++i) z[i] = z_in[i] / nz;
  double d = 0.0;
  for (int i = 0; i < 3; ++i) d += xhint[i] * z[i];
  for (int i = 0; i < 3; ++i) x[i] = xhint[i] - d * z[i];
  double nx = vnorm(x);
  if (!(nx > 1e-6)) {  // hint parallel to z: any perpendicular direction
    const double e[3] = {std::fabs(z[0]) < 0.9 ? 1.0 : 0.0, std::fabs(z[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    d = e[0] * z[0] + e[1] * z[1];
    for (int i = 0; i < 3; ++i) x[i] = e[i] - d * z[i];
    nx = vnorm(x);
  }
  for (int i = 0; i < 3; ++i) x[i] /= nx;
  y[0] = z[1] * x[2] - z[2] * x[1];
  y[1] = z[2] * x[0] - z[0] * x[2];
  y[2] = z[0] * x[1] - z[1] * x[0];
  M3 R;
  for (int i = 0; i < 3; ++i) {
    R[0][i] = x[i];
    R[1][i] = y[i];
    R[2][i] = z[i];
  }
  return R;
}

// U for one atom under rotation R: block diagonal over its shells.
void atom_U(const AtomFns& af, const M3& R, double* U /* n x n */) {
  const int n = af.n;
  for (int i = 0; i < n * n; ++i) U[i] = 0.0;
  int off = 0;
  for (int l : af.shell_l) {
    if (l == 0) {
      U[off * n + off] = 1.0;
    } else if (l == 1) {
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) U[(off + a) * n + off + c] = R[a][c];
    } else {
      // component c <-> (i, j) with monomial x_i x_j; m_a(R v) = sum_c T_ac m_c(v)
      int cidx[3][3];
      int pi[6], pj[6];
      for (int c = 0; c < 6; ++c) {
        int e[3] = {cart_comp(2, c, 0), cart_comp(2, c, 1), cart_comp(2, c, 2)};
        int q[2], k = 0;
        for (int ax = 0; ax < 3; ++ax)
          for (int r = 0; r < e[ax]; ++r) q[k++] = ax;
        pi[c] = q[0];
        pj[c] = q[1];
        cidx[q[0]][q[1]] = cidx[q[1]][q[0]] = c;
      }
      double T[6][6] = {};
      for (int a = 0; a < 6; ++a)
        for (int s = 0; s < 3; ++s)
          for (int t = 0; t < 3; ++t) T[a][cidx[s][t]] += R[pi[a]][s] * R[pj[a]][t];
      auto nrm = [&](int c) { return pi[c] == pj[c] ? 0.57735026918962576451 : 1.0; };
      for (int a = 0; a < 6; ++a)
        for (int c = 0; c < 6; ++c) U[(off + a) * n + off + c] = nrm(a) * T[a][c] / nrm(c);
    }
    off += ncart(l);
  }
}

bool invert(const double* A, double* Ai, int n) {
  std::vector<double> M((size_t)n * 2 * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(M[r * 2 * n + c]) > std::fabs(M[p * 2 * n + c])) p = r;
    if (std::fabs(M[p * 2 * n + c]) < 1e-14) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[c * 2 * n + j], M[p * 2 * n + j]);
    const double d = M[c * 2 * n + c];
    for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r)
      if (r != c) {
        const double f = M[r * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ai[i * n + j] = M[i * 2 * n + n + j];
  return true;
}

struct PairGeo {
  int A, B;
  M3 R;
  float feat[kFeat];
};

void pair_geometry(const fsim_basis* b, std::vector<PairGeo>& out) {
  const int na = b->natom;
  const double* X = b->axyz.data();
  out.clear();
  for (int A = 0; A < na; ++A)
    for (int B = A; B < na; ++B) {
      PairGeo g;
      g.A = A;
      g.B = B;
      for (float& f : g.feat) f = 0.0f;
      double zv[3], hint[3];
      int C = -1, C2 = -1;
      double rAB = 0.0;
      if (A != B) {
        vsub(X + 3 * B, X + 3 * A, zv);
        rAB = vnorm(zv);
        double mid[3];
        for (int i = 0; i < 3; ++i) mid[i] = 0.5 * (X[3 * A + i] + X[3 * B + i]);
        double best = 1e300;
        for (int c = 0; c < na; ++c) {
          if (c == A || c == B) continue;
          double d[3];
          vsub(X + 3 * c, mid, d);
          const double r = vnorm(d);
          if (r < best) {
            best = r;
            C = c;
          }
        }
        if (C >= 0) vsub(X + 3 * C, mid, hint);
        else hint[0] = hint[1] = hint[2] = 0.0;
      } else {
        double b1 = 1e300, b2 = 1e300;
        for (int c = 0; c < na; ++c) {
          if (c == A) continue;
          double d[3];
          vsub(X + 3 * c, X + 3 * A, d);
          const double r = vnorm(d);
          if (r < b1) {
            b2 = b1;
            C2 = C;
            b1 = r;
            C = c;
          } else if (r < b2) {
            b2 = r;
            C2 = c;
          }
        }
        if (C >= 0) vsub(X + 3 * C, X + 3 * A, zv);
        else zv[0] = zv[1] = 0.0, zv[2] = 1.0;
        if (C2 >= 0) vsub(X + 3 * C2, X + 3 * A, hint);
        else hint[0] = hint[1] = hint[2] = 0.0;
      }
      g.R = frame_from(zv, hint);
      float* f = g.feat;
      f[0] = (float)(0.1 * rAB);
      const int sa = elem_slot(b->Z[A]), sb = elem_slot(b->Z[B]);
      if (sa >= 0) f[1 + sa] = 1.0f;
      if (sb >= 0) f[5 + sb] = 1.0f;
      for (int k = 0; k < 32; ++k) {
        const double mu = 10.0 * k / 31.0, w = 0.4;
        f[9 + k] = (float)std::exp(-(rAB - mu) * (rAB - mu) / (2 * w * w));
      }
      auto dist = [&](int p, int q) {
        double d[3];
        vsub(X + 3 * p, X + 3 * q, d);
        return vnorm(d);
      };
      if (A != B) {
        if (C >= 0) {
          f[41] = (float)(0.1 * dist(C, A));
          f[42] = (float)(0.1 * dist(C, B));
          const int sc = elem_slot(b->Z[C]);
          if (sc >= 0) f[43 + sc] = 1.0f;
        }
      } else {
        if (C >= 0) {
          f[41] = (float)(0.1 * dist(C, A));
          const int sc = elem_slot(b->Z[C]);
          if (sc >= 0) f[43 + sc] = 1.0f;
        }
        if (C2 >= 0) f[42] = (float)(0.1 * dist(C2, A));
        f[47] = 1.0f;
      }
      out.push_back(g);
    }
}

// D_AB = U_A^T L U_B for one pair per block; writes D_AB and its transpose.
__global__ void assemble_kernel(const float* __restrict__ L, const double* __restrict__ UA,
                                const double* __restrict__ UB, const int4* __restrict__ geo, int N,
                                double* __restrict__ D) {
  __shared__ double T[kMaxF * kMaxF];
  const int pr = blockIdx.x;
  const int4 g = geo[pr];  // (first_A, nA, first_B, nB)
  const int nA = g.y, nB = g.w;
  const float* Lp = L + (size_t)pr * kOut;
  const double* ua = UA + (size_t)pr * kOut;
  const double* ub = UB + (size_t)pr * kOut;
  for (int x = threadIdx.x; x < nA * nB; x += blockDim.x) {  // T = L U_B
    const int r = x / nB, c = x % nB;
    double s = 0.0;
    for (int k = 0; k < nB; ++k) s += (double)Lp[r * kMaxF + k] * ub[k * nB + c];
    T[r * kMaxF + c] = s;
  }
  __syncthreads();
  const bool self = g.x == g.z;
  for (int x = threadIdx.x; x < nA * nB; x += blockDim.x) {  // U_A^T T
    const int r = x / nB, c = x % nB;
    double s = 0.0;
    for (int k = 0; k < nA; ++k) s += ua[k * nA + r] * T[k * kMaxF + c];
    if (self) {
      if (r <= c) {
        double s2 = 0.0;  // symmetrised: average with the (c, r) element
        for (int k = 0; k < nA; ++k) {
          double t2 = 0.0;
          for (int q = 0; q < nB; ++q) t2 += (double)Lp[k * kMaxF + q] * ub[q * nB + r];
          s2 += ua[k * nA + c] * t2;
        }
        const double v = 0.5 * (s + s2);
        D[(size_t)(g.x + r) * N + g.z + c] = v;
        D[(size_t)(g.z + c) * N + g.x + r] = v;
      }
    } else {
      D[(size_t)(g.x + r) * N + g.z + c] = s;
      D[(size_t)(g.z + c) * N + g.x + r] = s;
    }
  }
}

}  // namespace
}  // namespace fsim

using namespace fsim;

extern "C" {

int fsim_guess_layout(const fsim_basis* b, int* npairs, int* nfeat, int* nout) {
  if (!b || !npairs || !nfeat || !nout) {
    set_error("fsim_guess_layout: null pointer");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    set_error("fsim_guess_layout: the learned guess works on Cartesian bases only");
    return FSIM_EINVAL;
  }
  std::vector<AtomFns> at;
  FSIM_TRY(atom_layout(b, at));
  *npairs = b->natom * (b->natom + 1) / 2;
  *nfeat = kFeat;
  *nout = kOut;
  return FSIM_OK;
}

int fsim_guess_features(const fsim_basis* b, float* feat) {
  if (!b || !feat) {
    set_error("fsim_guess_features: null pointer");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    set_error("fsim_guess_features: the learned guess works on Cartesian bases only");
    return FSIM_EINVAL;
  }
  std::vector<AtomFns> at;
  FSIM_TRY(atom_layout(b, at));
  std::vector<PairGeo> pg;
  pair_geometry(b, pg);
  for (size_t p = 0; p < pg.size(); ++p) std::memcpy(feat + p * kFeat, pg[p].feat, sizeof(float) * kFeat);
  return FSIM_OK;
}

int fsim_guess_targets(const fsim_basis* b, const double* D, float* target, float* mask) {
  if (!b || !D || !target || !mask) {
    set_error("fsim_guess_targets: null pointer");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    set_error("fsim_guess_targets: the learned guess works on Cartesian bases only");
    return FSIM_EINVAL;
  }
  std::vector<AtomFns> at;
  FSIM_TRY(atom_layout(b, at));
  std::vector<PairGeo> pg;
  pair_geometry(b, pg);
  const int N = b->nbf;
  double UA[kOut], UB[kOut], UAi[kOut], UBi[kOut], T[kOut];
  for (size_t p = 0; p < pg.size(); ++p) {
    const AtomFns &fa = at[pg[p].A], &fb = at[pg[p].B];
    atom_U(fa, pg[p].R, UA);
    atom_U(fb, pg[p].R, UB);
    if (!invert(UA, UAi, fa.n) || !invert(UB, UBi, fb.n)) {
      set_error("fsim_guess_targets: singular frame transform");
      return FSIM_EINVAL;
    }
    float* t = target + p * kOut;
    float* m = mask + p * kOut;
    for (int i = 0; i < kOut; ++i) t[i] = m[i] = 0.0f;
    // L = UA^{-T} D_AB UB^{-1}
    for (int r = 0; r < fa.n; ++r)
      for (int c = 0; c < fb.n; ++c) {
        double s = 0.0;
        for (int k = 0; k < fb.n; ++k) s += D[(size_t)(fa.first + r) * N + fb.first + k] * UBi[k * fb.n + c];
        T[r * kMaxF + c] = s;
      }
    for (int r = 0; r < fa.n; ++r)
      for (int c = 0; c < fb.n; ++c) {
        double s = 0.0;
        for (int k = 0; k < fa.n; ++k) s += UAi[k * fa.n + r] * T[k * kMaxF + c];
        t[r * kMaxF + c] = (float)s;
        m[r * kMaxF + c] = 1.0f;
      }
  }
  return FSIM_OK;
}

int fsim_guess_assemble(fsim_basis* b, const float* blocks, double* D, void* stream) {
  if (!b || !blocks || !D) {
    set_error("fsim_guess_assemble: null pointer");
    return FSIM_EINVAL;
  }
  if (b->spherical) {
    set_error("fsim_guess_assemble: the learned guess works on Cartesian bases only");
    return FSIM_EINVAL;
  }
  std::vector<AtomFns> at;
  FSIM_TRY(atom_layout(b, at));
  std::vector<PairGeo> pg;
  pair_geometry(b, pg);
  const size_t np = pg.size();
  std::vector<double> UA(np * kOut, 0.0), UB(np * kOut, 0.0);
  std::vector<int4> geo(np);
  for (size_t p = 0; p < np; ++p) {
    const AtomFns &fa = at[pg[p].A], &fb = at[pg[p].B];
    atom_U(fa, pg[p].R, UA.data() + p * kOut);
    atom_U(fb, pg[p].R, UB.data() + p * kOut);
    geo[p] = make_int4(fa.first, fa.n, fb.first, fb.n);
  }
  double *dUA = nullptr, *dUB = nullptr;
  int4* dgeo = nullptr;
  FSIM_TRY(dev_alloc(&dUA, UA.size()));
  FSIM_TRY(dev_alloc(&dUB, UB.size()));
  FSIM_TRY(dev_alloc(&dgeo, np));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = FSIM_OK;
  if (cudaMemcpyAsync(dUA, UA.data(), sizeof(double) * UA.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dUB, UB.data(), sizeof(double) * UB.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dgeo, geo.data(), sizeof(int4) * np, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("fsim_guess_assemble: upload failed");
    rc = FSIM_ECUDA;
  }
  if (rc == FSIM_OK) {
    assemble_kernel<<<(unsigned)np, 128, 0, s>>>(blocks, dUA, dUB, dgeo, b->nbf, D);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("fsim_guess_assemble: kernel failed");
      rc = FSIM_ECUDA;
    }
  }
  dev_free(dUA);
  dev_free(dUB);
  dev_free(dgeo);
  return rc;
}

}  // extern "C"
