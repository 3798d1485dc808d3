/*
 * fsim.h -- C-ABI of libfsim, a GB300 (sm_103a) implementation of the
 * McMurchie-Davidson restricted Hartree-Fock hot path of arXiv 2510.24968
 * ("FSIM: A Pedagogical and Extensible HPC Framework for the Hartree-Fock
 * Method").  The calls follow the paper's statement of the problem: a molecule
 * and a basis go in (Sec. 3.1), the two-electron part of the Fock matrix
 * F[D] = H + J - K/2 is built from a density (Sec. 2.2, Eq. fock; Sec. 3.2),
 * and the SCF of Sec. 3.2 returns the total energy.
 *
 * Conventions (all calls):
 *  - Return FSIM_OK (0) on success, a negative FSIM_E* code otherwise; the
 *    message of the last failure on the calling thread is fsim_last_error().
 *  - Units: bohr, hartree.  Basis functions are contracted CARTESIAN Gaussians
 *    (s, p, d); inside a shell the components are ordered x, y, z (p) and
 *    xx, xy, xz, yy, yz, zz (d).  Matrices are nbf x nbf, row-major, FP64, with
 *    the basis functions in the order of the shells passed to
 *    fsim_basis_create.
 *  - The library copies every input it needs; arrays passed in stay owned by
 *    the caller and may be freed after the call returns.  Outputs are written
 *    into caller-owned arrays of the stated size.
 *  - Work runs on the CUDA device that is current when fsim_basis_create is
 *    called; the basis keeps device buffers until fsim_basis_destroy.
 *  - A basis handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef FSIM_H
#define FSIM_H

#ifdef __cplusplus
extern "C" {
#endif

#define FSIM_OK 0
#define FSIM_EINVAL (-1)          /* bad argument (null pointer, size, l > 3, ...) */
#define FSIM_ECUDA (-2)           /* a CUDA runtime / library call failed */
#define FSIM_ENOCONV (-3)         /* SCF hit max_iter; the result struct is still filled */
#define FSIM_EILLCOND (-4)        /* overlap matrix (near) singular: min eigenvalue < 1e-10 */
#define FSIM_EDEVICE_TIMEOUT (-5) /* a bounded device-side wait gave up */
#define FSIM_ENOMEM (-6)          /* device allocation failed */

#define FSIM_FP64 0   /* every step in FP64 */
#define FSIM_MIXED 1  /* FP32 Boys, Hermite integrals and contraction; FP64 J/K accumulation */
/* FP64-accurate integrals with the light class pairs in double-float
 * arithmetic: each value an unevaluated sum of two FP32 numbers (~2^-47
 * relative rounding, FP32 exponent range) on the FP32 pipe, FP64 J/K
 * accumulation.  By default class pairs of total angular momentum <= 4 run the
 * double-float kernel and the others the FP64 kernel (fsim_autotune times
 * both).  Exponent range: products (2 p q / (p + q))^n up to n = 8 must stay
 * below FP32's 3.4e38, as on the FSIM_MIXED path. */
#define FSIM_DFLOAT 2

#define FSIM_PTR_HOST 0
#define FSIM_PTR_DEVICE 1

#define FSIM_GUESS_CORE 0     /* diagonalise H_core in the orthogonal basis (Sec. 3.2, step 1) */
#define FSIM_GUESS_DENSITY 1  /* caller-supplied density fsim_scf_opts.D0 (checked; core-H fallback) */
#define FSIM_GUESS_LEARNED 2  /* density predicted by the network in fsim_scf_opts.guess_model (checked;
                                 core-H fallback) */

typedef struct fsim_basis fsim_basis; /* opaque, owned by the library */

typedef struct {
  int Z;          /* nuclear charge (electrons counted from it) */
  double xyz[3];  /* bohr */
} fsim_atom;

typedef struct {
  int atom;             /* index into the atom array */
  int l;                /* 0, 1 or 2 */
  int nprim;            /* 1 .. 4 primitives */
  const double* alpha;  /* nprim exponents, > 0 */
  const double* coef;   /* nprim raw contraction coefficients d_k */
} fsim_shell_desc;

/*
 * Build a contracted Cartesian basis (Sec. 2.1.1, 2.4).  Each primitive is
 * normalised per Cartesian component, N = (2a/pi)^{3/4} (4a)^{l/2} /
 * sqrt((2i-1)!!(2j-1)!!(2k-1)!!), and each contracted function is rescaled so
 * that S_mumu = 1.  Builds the shell-pair data (Gaussian product theorem,
 * Sec. 2.1.2; Hermite coefficients E^{ij}_t of Eqs. recurrence-A/B, collapsed
 * per Eq. E-tuv) on the device.  *out receives a new handle.
 * Errors: FSIM_EINVAL for bad sizes or l > 3 or nprim outside 1..4,
 * FSIM_ECUDA / FSIM_ENOMEM from the device.
 */
int fsim_basis_create(const fsim_atom* atoms, int natom, const fsim_shell_desc* shells, int nshell,
                      fsim_basis** out);

/*
 * The same with flags.  FSIM_BASIS_SPHERICAL: the basis the caller sees is the
 * real solid-harmonic one of Sec. 2.1.1 (2l+1 functions per shell: s; p in x, y,
 * z order; d as m = -2..2: xy, yz, z^2 - (x^2+y^2)/2, xz, (sqrt 3/2)(x^2 - y^2)
 * on the unit-normalised Cartesian components, each unit-normalised; f as
 * m = -3..3: y(3x^2 - y^2), xyz, y(4z^2 - x^2 - y^2), z(2z^2 - 3x^2 - 3y^2),
 * x(4z^2 - x^2 - y^2), z(x^2 - y^2), x(x^2 - 3y^2), each unit-normalised).
 * Shells up to f (l = 3) in every build path except fsim_j_build, batches and
 * the learned guess, which refuse bases with f shells (FSIM_EINVAL).  The
 * integrals are still evaluated over Cartesian shells; fsim_onee,
 * fsim_fock_build and fsim_scf take and return matrices in the spherical basis
 * (D_cart = T^T D T before the build, J = T J_cart T^T after).  fsim_eri_quartets
 * and fsim_eri_dump stay Cartesian; batches, the learned guess and
 * fsim_fock_build_noalloc reject spherical bases (FSIM_EINVAL).
 */
#define FSIM_BASIS_SPHERICAL 1
int fsim_basis_create_ex(const fsim_atom* atoms, int natom, const fsim_shell_desc* shells, int nshell, int flags,
                         fsim_basis** out);
void fsim_basis_destroy(fsim_basis* b);
/* Functions of the basis the caller sees (spherical count for spherical bases). */
int fsim_basis_nbf(const fsim_basis* b);
/* Cartesian functions of the integral engine (equal to fsim_basis_nbf for Cartesian bases). */
int fsim_basis_nbf_cart(const fsim_basis* b);
int fsim_basis_nshell(const fsim_basis* b);
/* Number of unique shell pairs in each of the six pair classes ss, ps, pp, ds, dp, dd. */
int fsim_basis_pair_counts(const fsim_basis* b, int counts[6]);

/*
 * Nuclear repulsion sum_{A<B} Z_A Z_B / R_AB (added to E_elec, Sec. 3.2).
 */
int fsim_enuc(const fsim_basis* b, double* e_nuc);

/*
 * One-electron matrices (Sec. 2.3.1 Eq. s-overall, Sec. 2.3.2 Eq. Tab-final,
 * Sec. 2.3.3 Eq. Vab-final); which = 0 overlap S, 1 kinetic T, 2 nuclear
 * attraction V.  out: nbf*nbf, host or device pointer per ptr_mode.  stream:
 * cudaStream_t or NULL.
 */
int fsim_onee(fsim_basis* b, int which, double* out, int ptr_mode, void* stream);

/*
 * Schwarz bounds (not defined in the paper; this library's reading):
 * Q_ab = sqrt(max_{mu in a, nu in b} |(mu nu|mu nu)|) for every shell pair,
 * evaluated in FP64 with the ERI kernels on the diagonal quartets.  Also sorts
 * each pair class by Q (descending), which the Fock build uses for screening.
 * Q: nshell*nshell host array (may be NULL to only prepare the screening).
 */
int fsim_schwarz(fsim_basis* b, double* Q);

typedef struct {
  double schwarz_tau;  /* skip unique quartets with Q_ab Q_cd < tau; 0 = no screening */
  int precision;       /* FSIM_FP64, FSIM_MIXED or FSIM_DFLOAT */
  double boys_fp64_T;  /* mixed path: Boys to FP64-level accuracy (double-float arithmetic on the FP32
                          pipe, relative error <= 1e-13) for T >= this; 0 = never; values in (0, 30)
                          are rejected */
  int ptr_mode;        /* FSIM_PTR_HOST or FSIM_PTR_DEVICE for D, J, K */
  void* stream;        /* cudaStream_t; NULL = legacy default stream */
  int shard;           /* this shard's index in [0, nshards): bra pairs i with i % nshards == shard */
  int nshards;         /* 1 = whole build */
  int timing;          /* 1: record CUDA events around each class-pair kernel (fsim_last_class_times) */
} fsim_fock_opts;

/* Fills the defaults: tau 1e-10, FP64, boys_fp64_T 0, host pointers, NULL stream, 1 shard. */
void fsim_fock_opts_default(fsim_fock_opts* o);

/*
 * Coulomb and exchange matrices of a symmetric density (Sec. 2.2, Eq. fock):
 *   J_mu,nu = sum_{la,si} D_la,si (mu nu|la si),  K_mu,nu = sum_{la,si} D_la,si (mu la|nu si),
 * so that G = J - K/2.  ERIs by the McMurchie-Davidson scheme (Eq. twoe-final)
 * over each shell quartet unique under the 8-fold permutational symmetry that
 * survives Schwarz screening, digested directly into J and K.  D, J, K:
 * nbf*nbf row-major FP64, host or device per opts->ptr_mode (J and K are
 * overwritten).  With nshards > 1 only this shard's bra pairs contribute (the
 * caller sums J and K over shards).  Calls fsim_schwarz first if it has not run.
 * Errors: FSIM_EINVAL (null pointers, bad options), FSIM_ECUDA.
 */
int fsim_fock_build(fsim_basis* b, const double* D, double* J, double* K, const fsim_fock_opts* opts);

/*
 * fsim_fock_build for callers that must not allocate device memory while they
 * run (a server whose memory pool owns the device budget, a loop that cannot
 * take the device-wide synchronisation of cudaMalloc/cudaFree, an allocator
 * that forbids raw cudaMalloc).  The paper has no counterpart; this is an
 * interface addition.  Same result as fsim_fock_build (same kernels), but the
 * J/K accumulators and the FP32 density copy live in one fixed file-scope
 * device array of 5 MiB that every GPU loading the library keeps until exit,
 * so the call allocates nothing.  Limits and rules:
 *  - nbf <= 512, else FSIM_EINVAL; D, J, K device pointers (ptr_mode
 *    FSIM_PTR_DEVICE); opts->timing must be 0; precision FSIM_FP64 or
 *    FSIM_MIXED only (FSIM_DFLOAT: FSIM_EINVAL, it needs per-basis
 *    double-float copies that are allocated); Cartesian bases only;
 *  - the basis must already hold its Schwarz bounds and the screening plan for
 *    these options: call fsim_fock_build once with the same opts during
 *    set-up (else FSIM_EINVAL, nothing launched);
 *  - that set-up build also looks up the array's device address on its device
 *    (loading the module that holds the array), so later calls load nothing;
 *    a first call on a device without that set-up does the look-up itself
 *    (with the basis' device current): make it before any stream capture;
 *  - all calls share the array; calls whose GPU work overlaps race on it;
 *  - afterwards fsim_last_quartet_count reports this build; per-class times
 *    (fsim_last_class_times) are not recorded (-1).
 */
int fsim_fock_build_noalloc(fsim_basis* b, const double* D, double* J, double* K, const fsim_fock_opts* opts);

/*
 * Coulomb matrix alone, J_mu,nu = sum_{la,si} D_la,si (mu nu|la si) (Sec. 2.2
 * Eq. fock), built in Hermite space without Cartesian quartets (Sec. 2.5: the
 * ket's Hermite coefficients are contracted with the density first, so each
 * primitive quartet costs the Hermite Coulomb recursion and
 * n_h(L_bra) x n_h(L_ket) multiply-adds).  Same screening rule as
 * fsim_fock_build (Q_ab Q_cd >= tau), evaluated over both orders of every
 * screened unique quartet; fsim_last_quartet_count then reports that ordered
 * count.  D, J: nbf*nbf row-major FP64, host or device per opts->ptr_mode (J
 * overwritten).  opts: schwarz_tau, precision FSIM_FP64 or FSIM_MIXED (FP32
 * integrals, FP64 accumulation), boys_fp64_T, ptr_mode, stream, shard/nshards
 * (bra pairs i with i % nshards == shard; the caller sums J over shards);
 * timing must be 0.  Cartesian bases only.  Errors: FSIM_EINVAL (null
 * pointers, bad options, FSIM_DFLOAT, spherical basis), FSIM_ECUDA,
 * FSIM_ENOMEM.
 */
int fsim_j_build(fsim_basis* b, const double* D, double* J, const fsim_fock_opts* opts);

/*
 * Autotuner for the Fock-build launches of this basis and these options
 * (screening, precision, shard): for every class pair it times each launch
 * shape on the device -- the unrolled per-class kernel with each quartet's
 * primitive quartets split over psplit = 1, 3, 9 or 27 threads (bra primitive
 * pairs first; 27 also splits the ket primitive pairs three ways, tried only
 * for class pairs with fewer than 2 x 128 x SMs / 9 quartets) and the
 * ket-component chunks shared out over csplit = 1, 2 or 4 warp groups (a CTA
 * of 128 threads takes floor(128 / csplit / psplit) kets), and the
 * warp-cooperative kernel (4 kets per CTA) -- and keeps the fastest in the
 * basis' cached plan, which later fsim_fock_build calls with the same options
 * use.  FSIM_DFLOAT: every shape with the double-float kernel and with the
 * FP64 kernel (both FP64-accurate), no cooperative kernel.  choice (36
 * entries, optional): 10 * psplit + csplit for the unrolled kernel (+ 1000
 * when a double-float build runs the class pair with the FP64 kernel), -1 for
 * the cooperative kernel, 0 for class pairs
 * without work; best_ms (36, optional): its median time.  Index X*6+Y as in
 * fsim_last_class_times.
 */
int fsim_autotune(fsim_basis* b, const fsim_fock_opts* opts, int* choice, float* best_ms);

/*
 * Sets launch shapes in the basis' cached plan for these options (screening,
 * precision, shard), e.g. choices saved from an earlier fsim_autotune.
 * choice: 36 host ints in fsim_autotune's encoding; 0 leaves a class pair as
 * it is.  Errors (FSIM_EINVAL, plan unchanged for that and later class pairs):
 * psplit not 1/3/9 or above the bra class's primitive pairs (27: bra class
 * below 9 or ket class below 3 primitive pairs), csplit not 1/2/4 or above its
 * ket chunks, the cooperative kernel with FSIM_DFLOAT, +1000 outside
 * FSIM_DFLOAT, or the double-float kernel for (dd|dp) and (dd|dd).
 */
int fsim_set_launch(fsim_basis* b, const fsim_fock_opts* opts, const int* choice);

/* Unique shell quartets the last fsim_fock_build evaluated (after screening). */
long long fsim_last_quartet_count(const fsim_basis* b);

/*
 * Per class pair (bra pair class X >= ket pair class Y, index X*6+Y; classes
 * ss ps pp ds dp dd) of the last fsim_fock_build: kernel time in ms from CUDA
 * events recorded on the build's stream (only when opts.timing was set; else
 * -1), and unique quartets evaluated.  ms, quartets: 36 entries each (host).
 * *nlaunch: kernels the build launched.  Synchronises the build's stream.
 */
int fsim_last_class_times(fsim_basis* b, float* ms, long long* quartets, int* nlaunch);

/*
 * Contracted ERI blocks (mu nu|la si) for explicit shell quartets (debug /
 * parity), by the FP64 warp-cooperative quartet kernel that also serves the
 * Schwarz diagonal.
 * quartets: 4*n shell indices (a,b,c,d); out: concatenated blocks, each
 * na*nb*nc*nd in (a,b,c,d) row-major order; host pointers; precision must be
 * FSIM_FP64.
 */
int fsim_eri_quartets(fsim_basis* b, int n, const int* quartets, double* out, int precision);

/*
 * All ERIs g[mu][nu][la][si] (nbf <= 64, nbf^4 host doubles).  Debug / parity.
 */
int fsim_eri_dump(fsim_basis* b, double* g, int precision);

typedef struct {
  int nelec;            /* electrons (even) */
  int max_iter;         /* e.g. 100 */
  double conv_dE;       /* |E_n - E_{n-1}| threshold, e.g. 1e-10 */
  double conv_dD;       /* rms(D_n - D_{n-1}) threshold, e.g. 1e-7 */
  int diis_size;        /* stored Fock/error pairs (Sec. 3.2.1: 6-8); 0 disables DIIS */
  int guess;            /* FSIM_GUESS_CORE or FSIM_GUESS_DENSITY */
  const double* D0;     /* host nbf*nbf initial density for FSIM_GUESS_DENSITY */
  fsim_fock_opts fock;  /* screening, precision and stream of the Fock builds */
  int final_fp64;       /* FSIM_MIXED: after mixed convergence, finish with FP64-accurate Fock builds:
                           0 never, 1 FSIM_FP64 builds, 2 FSIM_DFLOAT builds (fsim_scf_batched:
                           any non-zero value means FSIM_FP64 builds) */
  int incremental;      /* build G(D_n) as G(D_{n-1}) + G(D_n - D_{n-1}) */
  const char* guess_model; /* FSIM_GUESS_LEARNED: weights file written by fsim_mlp_save (its input and
                              output widths must match fsim_guess_layout) */
  int dw_screen;        /* 1: density-weighted screening of the incremental builds (Sec. 5, direct SCF)
                           of a FSIM_MIXED SCF while its mixed iteration settles: G(dD) skips quartets
                           with Q_ab Q_cd max|dD| < schwarz_tau (fsim_scf: the threshold tau / max|dD|,
                           rounded down to tau times a power of two, is the build's schwarz_tau;
                           fsim_scf_batched: per molecule on the device).  The skipped terms add up in
                           the incremental G, so the FP64-accurate resets and every build after the
                           first one keep schwarz_tau (final_fp64 != 0 is needed for FP64-level
                           energies).  0 (default): off */
} fsim_scf_opts;

/* Defaults: 100 iterations, |dE| 1e-10, rms(dD) 1e-7, DIIS 8, core-H guess, the Fock
 * defaults, final_fp64 2 (double-float resets), incremental builds. */
void fsim_scf_opts_default(fsim_scf_opts* o);

typedef struct {
  double e_total, e_elec, e_nuc;
  int iters;
  int converged;
  int guess_fallback;   /* 1 when a supplied guess failed its trace/idempotency check and core-H was used */
  double* D_out;        /* optional caller-owned nbf*nbf host array: final density */
  double* e_hist;       /* optional caller-owned max_iter array: total energy after each Fock build */
  double* t_hist;       /* optional caller-owned max_iter array: seconds from the start of the iteration
                           loop (after the set-up) to the end of each iteration */
  double time_s;        /* wall time of the SCF loop */
  double min_s_eig;     /* smallest eigenvalue of S */
  long long quartets;   /* unique quartets evaluated over all Fock builds (after any density weighting) */
  int fp64_builds;      /* FP64-accurate Fock builds (FSIM_FP64 or FSIM_DFLOAT) */
  int mixed_builds;     /* Fock builds done in mixed precision */
  double guess_s;       /* wall time of the initial density (prediction and check for a learned or
                           supplied guess, core-H diagonalisation otherwise), inside the set-up */
  int mixed_fallback;   /* 1: FSIM_MIXED was requested, but the overlap's smallest eigenvalue is below
                           FSIM_MIXED_MIN_S_EIG: in so nearly linearly dependent a basis the density has
                           large elements, and FP32 integral errors multiplied by them exceed the mixed
                           path's 1e-6 Eh bound, so every build ran in FSIM_FP64 */
} fsim_scf_result;

/* Smallest overlap eigenvalue for which fsim_scf / fsim_scf_batched run FSIM_MIXED builds. */
#define FSIM_MIXED_MIN_S_EIG 1e-4

/*
 * Restricted Hartree-Fock SCF (Sec. 3.2): core-Hamiltonian (or supplied)
 * guess, symmetric orthogonalisation X = U s^{-1/2} U^T, then per iteration
 * G(D) by fsim_fock_build, F = H + G, E_elec = 1/2 Tr[D (H + F)], DIIS
 * extrapolation (Sec. 3.2.1, Algorithm 1; error F D S - S D F), F' = X^T F X,
 * diagonalisation, C = X C', D = 2 C_occ C_occ^T.  Converged when
 * |dE| < conv_dE and rms(dD) < conv_dD.  All linear algebra in FP64 on the
 * device.  Returns FSIM_ENOCONV (result filled) at max_iter, FSIM_EILLCOND if
 * min eig(S) < 1e-10.
 */
int fsim_scf(fsim_basis* b, const fsim_scf_opts* opts, fsim_scf_result* res);

/*
 * Batched Fock builds for many molecules of uneven size (the paper's
 * J/K construction, Sec. 3.2, for a set of molecules at once).  A batch binds
 * nmol bases to fixed device buffers D[m] -> J[m], K[m] (each nbf_m^2 FP64,
 * owned by the caller, which must outlive the batch) and concatenates their
 * screened work so that every class pair is ONE persistent launch over all
 * molecules.  fsim_batch_fock runs one build of every molecule flagged in
 * `active` (host array of nmol ints, NULL = all); with use_graph the whole
 * launch sequence of a precision is captured into a CUDA graph on first use
 * and replayed afterwards.  Screening tau and the stream come from opts.
 * Schwarz bounds and plans are built at creation (allocates).
 */
typedef struct fsim_batch fsim_batch;
int fsim_batch_create(fsim_basis* const* bases, int nmol, const fsim_fock_opts* opts, const double* const* D,
                      double* const* J, double* const* K, fsim_batch** out);
int fsim_batch_fock(fsim_batch* batch, int precision, const int* active, int use_graph);
void fsim_batch_destroy(fsim_batch* batch);

/*
 * Restricted Hartree-Fock for nmol molecules in lockstep (Sec. 3.2, 3.2.1):
 * per iteration one batched Fock build (graph replay; FP64 and/or mixed
 * group as each molecule's state requires) and the per-molecule FP64 linear
 * algebra spread over several streams; converged molecules drop out.  Same
 * options and per-molecule semantics as fsim_scf (core-H guess only; FSIM_FP64
 * or FSIM_MIXED, the FP64-accurate fallback of FSIM_MIXED_MIN_S_EIG decided per molecule; each
 * molecule's electron count is its nuclear charge).  results: nmol entries;
 * time_s is the time from the start of the iteration loop (after the set-up:
 * one-electron matrices, orthogonaliser, guess, batch plans) at which that
 * molecule converged; t_hist counts from the same point.
 */
int fsim_scf_batched(fsim_basis* const* bases, int nmol, const fsim_scf_opts* opts, fsim_scf_result* results);

/*
 * Learned initial density (a network that predicts the SCF starting density
 * from geometry; the converged SCF is unchanged, only the number of iterations).
 * Per atom pair (A <= B, row-major over A then B; npairs = natom (natom+1)/2):
 * fsim_guess_features writes 48 rotation-invariant features (host, npairs x 48);
 * fsim_guess_targets turns a density D (host, nbf^2) into the pair blocks in
 * pair-local frames (host, npairs x 225, row-major 15 x 15, zero padded) and
 * their mask; fsim_guess_assemble rotates predicted local blocks (device,
 * npairs x 225 FP32) back and writes the full density (device, nbf^2 FP64).
 * Atoms must own contiguous shells with at most 15 functions.
 */
int fsim_guess_layout(const fsim_basis* b, int* npairs, int* nfeat, int* nout);
int fsim_guess_features(const fsim_basis* b, float* feat);
int fsim_guess_targets(const fsim_basis* b, const double* D, float* target, float* mask);
int fsim_guess_assemble(fsim_basis* b, const float* blocks, double* D, void* stream);

/*
 * The network: three linear layers with SiLU (nin -> width -> width -> nout),
 * FP32 master weights with BF16 copies; forward and backward GEMMs on the
 * fifth-generation tensor cores (tcgen05.mma: BF16 inputs, FP32 accumulation
 * in tensor memory), Adam (beta 0.9/0.999, eps 1e-8).  The BF16 calls
 * (fsim_mlp_forward with bf16 != 0, fsim_mlp_grad with bf16 != 0,
 * fsim_mlp_train_step) synchronise the stream before returning and return
 * FSIM_ECUDA if a GEMM's MMAs did not complete within its bounded wait.  init_params: host array of fsim_mlp_nparams() floats laid out
 * W1 [nin x width], b1, W2 [width x width], b2, W3 [width x nout], b3 (row-major).
 * x, y, t, mask: device FP32 arrays (batch x nin / batch x nout).  loss =
 * sum(mask (y - t)^2) / sum(mask).  fsim_mlp_grad returns that loss and its
 * gradient (host, nparams floats; bf16 = 0 computes every product in FP32, for
 * gradient checks); fsim_mlp_params copies parameters out (host_out) and/or in.
 */
typedef struct fsim_mlp fsim_mlp;
int fsim_mlp_create(int nin, int width, int nout, const float* init_params, fsim_mlp** out);
void fsim_mlp_destroy(fsim_mlp* net);
long long fsim_mlp_nparams(const fsim_mlp* net);
int fsim_mlp_params(fsim_mlp* net, float* host_out, const float* host_in);
/* Weights file of a network (the input of FSIM_GUESS_LEARNED): the 8 bytes
 * "FSIMMLP1", int32 nin, width, nout (little-endian), then the
 * fsim_mlp_nparams() FP32 master parameters in fsim_mlp_create's layout.
 * fsim_mlp_load creates a new network from such a file (caller destroys it).
 * Errors: FSIM_EINVAL (null pointers, unreadable or malformed file), FSIM_ECUDA. */
int fsim_mlp_save(fsim_mlp* net, const char* path);
/* One Adam step (the same update as fsim_mlp_train_step) from a gradient the
 * caller supplies (host, fsim_mlp_nparams() floats): for data-parallel
 * training, where each rank's fsim_mlp_grad of its share of a minibatch is
 * combined over the ranks (weighted by each share's mask sum, since the loss
 * is normalised per call) before every replica takes the same step. */
int fsim_mlp_adam_step(fsim_mlp* net, const float* grad_host, float lr, void* stream);
int fsim_mlp_load(const char* path, fsim_mlp** out);
int fsim_mlp_forward(fsim_mlp* net, const float* x, float* y, int batch, int bf16, void* stream);
int fsim_mlp_grad(fsim_mlp* net, const float* x, const float* t, const float* mask, int batch, int bf16, float* loss,
                  float* grad_host, void* stream);
int fsim_mlp_train_step(fsim_mlp* net, const float* x, const float* t, const float* mask, int batch, float lr,
                        float* loss, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* fsim_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSIM_H */
