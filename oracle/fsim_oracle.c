/*
 * fsim_oracle.c -- plain, slow, double-precision CPU oracle for the
 * McMurchie-Davidson restricted Hartree-Fock hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table
 * or constant generator with the CUDA library; both only read the same seeded
 * inputs.
 *
 * Every function below follows one passage of the paper (arXiv 2510.24968,
 * "FSIM"), written out as plainly as possible:
 *   - primitive normalisation and contraction renormalisation   (Sec. 2.1.1)
 *   - Gaussian product theorem                                   (Sec. 2.1.2)
 *   - Hermite expansion coefficients E^{ij}_t, Eqs. recurrence-A/B (Sec. 2.1.3)
 *   - overlap S_ab, Eq. s-overall                                (Sec. 2.3.1)
 *   - kinetic T_ab, Eqs. Tij-hermite / Tab-final                 (Sec. 2.3.2)
 *   - Boys function and Hermite Coulomb integrals R^n_tuv,
 *     Eqs. Rn-definition / R-recursion; nuclear attraction Eq. Vab-final
 *                                                                (Sec. 2.3.3)
 *   - primitive ERI, Eq. twoe-final, literal six-fold Hermite sum for each
 *     Cartesian component, then contraction over primitives     (Sec. 2.3.4)
 *   - J and K from G_mu,nu = sum D [(mu nu|la si) - 1/2 (mu la|nu si)],
 *     Eq. fock / Eq. eri                                         (Sec. 2.2)
 *   - symmetric orthogonalisation needs eigenpairs: cyclic Jacobi (textbook)
 * Schwarz screening is not defined in the paper; the oracle's reading is the
 * shell-level bound Q_ab = sqrt(max |(mu nu|mu nu)|), quartets skipped when
 * Q_ab Q_cd < tau.
 *
 * Parity pins for each function live in tests/ (closed forms, quadrature,
 * finite differences, symmetry, invariants).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_LMAX 3            /* s, p, d, f shells */
#define ORC_NCMAX 10          /* Cartesian components of an f shell */
#define ORC_KMAX 8            /* primitives per shell */
#define ORC_RMAX (4 * ORC_LMAX + 1)

/* ------------------------------------------------------------------ */
/* Cartesian components in lexicographic-descending order:            */
/* p: x y z ; d: xx xy xz yy yz zz ; f: xxx xxy xxz xyy xyz xzz yyy   */
/* yyz yzz zzz                                                        */
/* ------------------------------------------------------------------ */
static int orc_ncart(int l) { return (l + 1) * (l + 2) / 2; }

static void orc_cart(int l, int idx, int *ix, int *iy, int *iz) {
    int n = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (n == idx) { *ix = a; *iy = b; *iz = l - a - b; return; }
            ++n;
        }
}

static double orc_dfact(int n) { /* (n)!! with (-1)!! = 1 */
    double r = 1.0;
    for (int k = n; k > 1; k -= 2) r *= k;
    return r;
}

/* ------------------------------------------------------------------ */
/* Boys function F_n(T) = int_0^1 exp(-T t^2) t^{2n} dt  (Sec. 2.3.3)  */
/* T < 40: convergent series                                           */
/*   F_n(T) = e^{-T} sum_k (2T)^k / ((2n+1)(2n+3)...(2n+2k+1));        */
/* T >= 40: F_0 = (1/2) sqrt(pi/T) erf(sqrt T), then the upward        */
/*   recursion F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T).                 */
/* ------------------------------------------------------------------ */
double orc_boys(int n, double T) {
    if (T < 40.0) {
        double term = 1.0 / (2 * n + 1);
        double sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2 * n + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return exp(-T) * sum;
    }
    double F = 0.5 * sqrt(ORC_PI / T) * erf(sqrt(T));
    double e = exp(-T);
    for (int m = 0; m < n; ++m) F = ((2 * m + 1) * F - e) / (2.0 * T);
    return F;
}

/* ------------------------------------------------------------------ */
/* Hermite expansion coefficient E^{ij}_t for one Cartesian axis,      */
/* Eqs. recurrence-A/B with E^{00}_0 = exp(-mu X_AB^2) and zero         */
/* outside 0 <= t <= i+j (Sec. 2.1.3).  Xab = A_x - B_x.                */
/* ------------------------------------------------------------------ */
double orc_hermite_E(int i, int j, int t, double Xab, double a, double b) {
    double p = a + b;
    if (t < 0 || t > i + j) return 0.0;
    if (i == 0 && j == 0) return exp(-(a * b / p) * Xab * Xab);
    double XPA = -b * Xab / p; /* P_x - A_x */
    double XPB = a * Xab / p;  /* P_x - B_x */
    if (i > 0)
        return orc_hermite_E(i - 1, j, t - 1, Xab, a, b) / (2.0 * p)
             + XPA * orc_hermite_E(i - 1, j, t, Xab, a, b)
             + (t + 1) * orc_hermite_E(i - 1, j, t + 1, Xab, a, b);
    return orc_hermite_E(i, j - 1, t - 1, Xab, a, b) / (2.0 * p)
         + XPB * orc_hermite_E(i, j - 1, t, Xab, a, b)
         + (t + 1) * orc_hermite_E(i, j - 1, t + 1, Xab, a, b);
}

/* ------------------------------------------------------------------ */
/* Hermite Coulomb integrals R^n_tuv(a, X, Y, Z), Eq. R-recursion with  */
/* source R^n_000 = (-2a)^n F_n(a |R|^2).  Plain recursion; results    */
/* are memoised only to keep the oracle's run time finite.             */
/* ------------------------------------------------------------------ */
typedef struct {
    double a, X, Y, Z;
    int S; /* stride = L + 1 */
    double F[4 * ORC_RMAX];
    double *val;          /* S^4 memo entries */
    unsigned char *have;
} orc_rctx;

static orc_rctx *orc_rctx_new(int L) {
    orc_rctx *c = (orc_rctx *)malloc(sizeof(orc_rctx));
    size_t n = (size_t)(L + 1) * (L + 1) * (L + 1) * (L + 1);
    c->S = L + 1;
    c->val = (double *)malloc(sizeof(double) * n);
    c->have = (unsigned char *)malloc(n);
    return c;
}

static void orc_rctx_free(orc_rctx *c) {
    free(c->val);
    free(c->have);
    free(c);
}

static double orc_R(orc_rctx *c, int n, int t, int u, int v) {
    if (t < 0 || u < 0 || v < 0) return 0.0;
    int k = ((n * c->S + t) * c->S + u) * c->S + v;
    if (c->have[k]) return c->val[k];
    double r;
    if (t == 0 && u == 0 && v == 0) {
        r = pow(-2.0 * c->a, n) * c->F[n];
    } else if (t > 0) {
        r = (t - 1) * orc_R(c, n + 1, t - 2, u, v) + c->X * orc_R(c, n + 1, t - 1, u, v);
    } else if (u > 0) {
        r = (u - 1) * orc_R(c, n + 1, t, u - 2, v) + c->Y * orc_R(c, n + 1, t, u - 1, v);
    } else {
        r = (v - 1) * orc_R(c, n + 1, t, u, v - 2) + c->Z * orc_R(c, n + 1, t, u, v - 1);
    }
    c->val[k] = r;
    c->have[k] = 1;
    return r;
}

/* c must come from orc_rctx_new(L) with the same L. */
static void orc_rctx_init(orc_rctx *c, int L, double a, double X, double Y, double Z) {
    c->a = a; c->X = X; c->Y = Y; c->Z = Z;
    c->S = L + 1;
    double T = a * (X * X + Y * Y + Z * Z);
    for (int n = 0; n <= L; ++n) c->F[n] = orc_boys(n, T);
    memset(c->have, 0, (size_t)c->S * c->S * c->S * c->S);
}

/* Public single-value access (used by the pins). */
double orc_hermite_R(int n, int t, int u, int v, double a, double X, double Y, double Z) {
    orc_rctx *c = orc_rctx_new(n + t + u + v);
    orc_rctx_init(c, n + t + u + v, a, X, Y, Z);
    double r = orc_R(c, n, t, u, v);
    orc_rctx_free(c);
    return r;
}

/* ------------------------------------------------------------------ */
/* Basis: shells with centre, l, primitives; normalised coefficients.   */
/* ------------------------------------------------------------------ */
typedef struct {
    int nshell, nbf, natom;
    int *l, *nprim, *ao, *atom;
    double *cen;     /* 3 per shell */
    double *alpha;   /* ORC_KMAX per shell */
    double *cn;      /* normalised coefficient [shell][component][prim] */
    int *Z;          /* nuclear charges */
    double *axyz;    /* 3 per atom */
} orc_basis;

/* Unnormalised primitive overlap of one Cartesian component, Eq. s-overall */
static double orc_prim_overlap(const int *ia, const int *jb, double a, const double *A,
                               double b, const double *B) {
    double p = a + b, s = pow(ORC_PI / p, 1.5);
    for (int d = 0; d < 3; ++d) s *= orc_hermite_E(ia[d], jb[d], 0, A[d] - B[d], a, b);
    return s;
}

/*
 * Primitive normalisation N(a; i,j,k) = (2a/pi)^{3/4} (4a)^{l/2} /
 * sqrt((2i-1)!!(2j-1)!!(2k-1)!!) makes <G|G> = 1 for each Cartesian component;
 * then each contracted component is rescaled so that S_mumu = 1 (Sec. 2.1.1).
 */
void *orc_basis_create(int natom, const int *Z, const double *axyz, int nshell,
                       const int *shell_atom, const int *shell_l, const int *shell_nprim,
                       const double *alpha, const double *coef) {
    orc_basis *B = (orc_basis *)calloc(1, sizeof(orc_basis));
    B->nshell = nshell; B->natom = natom;
    B->l = (int *)malloc(sizeof(int) * nshell);
    B->nprim = (int *)malloc(sizeof(int) * nshell);
    B->ao = (int *)malloc(sizeof(int) * nshell);
    B->atom = (int *)malloc(sizeof(int) * nshell);
    B->cen = (double *)malloc(sizeof(double) * 3 * nshell);
    B->alpha = (double *)calloc((size_t)nshell * ORC_KMAX, sizeof(double));
    B->cn = (double *)calloc((size_t)nshell * ORC_NCMAX * ORC_KMAX, sizeof(double));
    B->Z = (int *)malloc(sizeof(int) * natom);
    B->axyz = (double *)malloc(sizeof(double) * 3 * natom);
    memcpy(B->Z, Z, sizeof(int) * natom);
    memcpy(B->axyz, axyz, sizeof(double) * 3 * natom);
    int off = 0, poff = 0;
    for (int s = 0; s < nshell; ++s) {
        int l = shell_l[s], K = shell_nprim[s];
        B->l[s] = l; B->nprim[s] = K; B->ao[s] = off; B->atom[s] = shell_atom[s];
        for (int d = 0; d < 3; ++d) B->cen[3 * s + d] = axyz[3 * shell_atom[s] + d];
        for (int k = 0; k < K; ++k) B->alpha[s * ORC_KMAX + k] = alpha[poff + k];
        for (int c = 0; c < orc_ncart(l); ++c) {
            int i3[3];
            orc_cart(l, c, &i3[0], &i3[1], &i3[2]);
            double *cc = &B->cn[((size_t)s * ORC_NCMAX + c) * ORC_KMAX];
            for (int k = 0; k < K; ++k) {
                double a = alpha[poff + k];
                double N = pow(2.0 * a / ORC_PI, 0.75) * pow(4.0 * a, 0.5 * l)
                         / sqrt(orc_dfact(2 * i3[0] - 1) * orc_dfact(2 * i3[1] - 1) * orc_dfact(2 * i3[2] - 1));
                cc[k] = coef[poff + k] * N;
            }
            double S = 0.0;
            for (int k = 0; k < K; ++k)
                for (int m = 0; m < K; ++m)
                    S += cc[k] * cc[m] * orc_prim_overlap(i3, i3, alpha[poff + k], &B->cen[3 * s],
                                                          alpha[poff + m], &B->cen[3 * s]);
            for (int k = 0; k < K; ++k) cc[k] /= sqrt(S);
        }
        off += orc_ncart(l);
        poff += K;
    }
    B->nbf = off;
    return B;
}

void orc_basis_destroy(void *vB) {
    orc_basis *B = (orc_basis *)vB;
    if (!B) return;
    free(B->l); free(B->nprim); free(B->ao); free(B->atom); free(B->cen);
    free(B->alpha); free(B->cn); free(B->Z); free(B->axyz); free(B);
}

int orc_basis_nbf(const void *vB) { return ((const orc_basis *)vB)->nbf; }

/* ------------------------------------------------------------------ */
/* One-electron integrals over contracted Cartesian functions           */
/* ------------------------------------------------------------------ */
/* Kinetic, one axis: Eq. Tij-hermite (without the sqrt(pi/p) factor). */
static double orc_kin_axis(int i, int j, double Xab, double a, double b) {
    double t = -2.0 * b * b * orc_hermite_E(i, j + 2, 0, Xab, a, b)
             + b * (2 * j + 1) * orc_hermite_E(i, j, 0, Xab, a, b);
    if (j >= 2) t -= 0.5 * j * (j - 1) * orc_hermite_E(i, j - 2, 0, Xab, a, b);
    return t;
}

/* which: 0 = overlap (Eq. s-overall), 1 = kinetic (Eq. Tab-final),
          2 = nuclear attraction summed over all nuclei (Eq. Vab-final). */
static double orc_onee_prim(int which, const int *i3, const int *j3, double a, const double *A,
                            double b, const double *B, const orc_basis *Bs) {
    double p = a + b;
    double X[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    if (which == 0) {
        double s = pow(ORC_PI / p, 1.5);
        for (int d = 0; d < 3; ++d) s *= orc_hermite_E(i3[d], j3[d], 0, X[d], a, b);
        return s;
    }
    if (which == 1) {
        double S[3], T[3];
        for (int d = 0; d < 3; ++d) {
            S[d] = orc_hermite_E(i3[d], j3[d], 0, X[d], a, b);
            T[d] = orc_kin_axis(i3[d], j3[d], X[d], a, b);
        }
        return (T[0] * S[1] * S[2] + S[0] * T[1] * S[2] + S[0] * S[1] * T[2]) * pow(ORC_PI / p, 1.5);
    }
    double P[3];
    for (int d = 0; d < 3; ++d) P[d] = (a * A[d] + b * B[d]) / p;
    int L = i3[0] + i3[1] + i3[2] + j3[0] + j3[1] + j3[2];
    double v = 0.0;
    orc_rctx *c = orc_rctx_new(L);
    for (int n = 0; n < Bs->natom; ++n) {
        const double *C = &Bs->axyz[3 * n];
        orc_rctx_init(c, L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2]);
        double s = 0.0;
        for (int t = 0; t <= i3[0] + j3[0]; ++t)
            for (int u = 0; u <= i3[1] + j3[1]; ++u)
                for (int w = 0; w <= i3[2] + j3[2]; ++w)
                    s += orc_hermite_E(i3[0], j3[0], t, X[0], a, b)
                       * orc_hermite_E(i3[1], j3[1], u, X[1], a, b)
                       * orc_hermite_E(i3[2], j3[2], w, X[2], a, b) * orc_R(c, 0, t, u, w);
        v += -Bs->Z[n] * (2.0 * ORC_PI / p) * s;
    }
    orc_rctx_free(c);
    return v;
}

/* out: nbf x nbf row-major; which as above. */
void orc_onee(const void *vB, int which, double *out) {
    const orc_basis *B = (const orc_basis *)vB;
    int N = B->nbf;
    for (int sa = 0; sa < B->nshell; ++sa)
        for (int sb = 0; sb < B->nshell; ++sb)
            for (int ca = 0; ca < orc_ncart(B->l[sa]); ++ca)
                for (int cb = 0; cb < orc_ncart(B->l[sb]); ++cb) {
                    int i3[3], j3[3];
                    orc_cart(B->l[sa], ca, &i3[0], &i3[1], &i3[2]);
                    orc_cart(B->l[sb], cb, &j3[0], &j3[1], &j3[2]);
                    double s = 0.0;
                    for (int k = 0; k < B->nprim[sa]; ++k)
                        for (int m = 0; m < B->nprim[sb]; ++m)
                            s += B->cn[((size_t)sa * ORC_NCMAX + ca) * ORC_KMAX + k]
                               * B->cn[((size_t)sb * ORC_NCMAX + cb) * ORC_KMAX + m]
                               * orc_onee_prim(which, i3, j3, B->alpha[sa * ORC_KMAX + k], &B->cen[3 * sa],
                                               B->alpha[sb * ORC_KMAX + m], &B->cen[3 * sb], B);
                    out[(size_t)(B->ao[sa] + ca) * N + B->ao[sb] + cb] = s;
                }
}

/* Nuclear repulsion sum_{A<B} Z_A Z_B / R_AB. */
double orc_enuc(const void *vB) {
    const orc_basis *B = (const orc_basis *)vB;
    double e = 0.0;
    for (int i = 0; i < B->natom; ++i)
        for (int j = 0; j < i; ++j) {
            double dx = B->axyz[3 * i] - B->axyz[3 * j], dy = B->axyz[3 * i + 1] - B->axyz[3 * j + 1],
                   dz = B->axyz[3 * i + 2] - B->axyz[3 * j + 2];
            e += B->Z[i] * B->Z[j] / sqrt(dx * dx + dy * dy + dz * dz);
        }
    return e;
}

/* ------------------------------------------------------------------ */
/* Two-electron integrals, Eq. twoe-final + primitive contraction      */
/* ------------------------------------------------------------------ */
/*
 * Contracted Cartesian block (ab|cd) for one shell quartet, written as
 * out[((ia*nb + ib)*nc + ic)*nd + id].  For every primitive quartet:
 * p = a+b, q = c+d, P, Q by the Gaussian product theorem, alpha = pq/(p+q),
 * prefactor 2 pi^{5/2} / (p q sqrt(p+q)), then for each Cartesian component
 * the literal six-fold sum over t,u,v (bra) and tau,nu,phi (ket) of
 * (-1)^{tau+nu+phi} E E E E E E R^0_{t+tau,u+nu,v+phi}(alpha, P-Q).
 */
void orc_eri_shell_quartet(const void *vB, int sa, int sb, int sc, int sd, double *out) {
    const orc_basis *B = (const orc_basis *)vB;
    int s4[4] = {sa, sb, sc, sd};
    int nc4[4], comp[4][ORC_NCMAX][3];
    for (int q = 0; q < 4; ++q) {
        nc4[q] = orc_ncart(B->l[s4[q]]);
        for (int c = 0; c < nc4[q]; ++c) orc_cart(B->l[s4[q]], c, &comp[q][c][0], &comp[q][c][1], &comp[q][c][2]);
    }
    int nblk = nc4[0] * nc4[1] * nc4[2] * nc4[3];
    for (int i = 0; i < nblk; ++i) out[i] = 0.0;
    int L = B->l[sa] + B->l[sb] + B->l[sc] + B->l[sd];
    const double *A = &B->cen[3 * sa], *Bc = &B->cen[3 * sb], *C = &B->cen[3 * sc], *D = &B->cen[3 * sd];
    orc_rctx *rc = orc_rctx_new(L);
    for (int ka = 0; ka < B->nprim[sa]; ++ka)
    for (int kb = 0; kb < B->nprim[sb]; ++kb) {
        double a = B->alpha[sa * ORC_KMAX + ka], b = B->alpha[sb * ORC_KMAX + kb];
        double p = a + b, P[3], Xab[3];
        for (int x = 0; x < 3; ++x) {
            P[x] = (a * A[x] + b * Bc[x]) / p;
            Xab[x] = A[x] - Bc[x];
        }
        /* tabulate E^{ij}_t per axis for this primitive pair (Eqs. recurrence-A/B) */
        double Eab[3][ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 1];
        for (int x = 0; x < 3; ++x)
            for (int i = 0; i <= B->l[sa]; ++i)
                for (int j = 0; j <= B->l[sb]; ++j)
                    for (int t = 0; t <= i + j; ++t) Eab[x][i][j][t] = orc_hermite_E(i, j, t, Xab[x], a, b);
    for (int kc = 0; kc < B->nprim[sc]; ++kc)
    for (int kd = 0; kd < B->nprim[sd]; ++kd) {
        double c = B->alpha[sc * ORC_KMAX + kc], d = B->alpha[sd * ORC_KMAX + kd];
        double q = c + d, al = p * q / (p + q);
        double Q[3], Xcd[3];
        for (int x = 0; x < 3; ++x) {
            Q[x] = (c * C[x] + d * D[x]) / q;
            Xcd[x] = C[x] - D[x];
        }
        orc_rctx_init(rc, L, al, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2]);
        double pref = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q));
        double Ecd[3][ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 1];
        for (int x = 0; x < 3; ++x)
            for (int i = 0; i <= B->l[sc]; ++i)
                for (int j = 0; j <= B->l[sd]; ++j)
                    for (int t = 0; t <= i + j; ++t) Ecd[x][i][j][t] = orc_hermite_E(i, j, t, Xcd[x], c, d);
        /* R^0_{tuv} for t+u+v <= L from the recursion */
        double R0[ORC_RMAX][ORC_RMAX][ORC_RMAX];
        for (int t = 0; t <= L; ++t)
            for (int u = 0; u <= L - t; ++u)
                for (int v = 0; v <= L - t - u; ++v) R0[t][u][v] = orc_R(rc, 0, t, u, v);
        int idx = 0;
        for (int ia = 0; ia < nc4[0]; ++ia)
        for (int ib = 0; ib < nc4[1]; ++ib)
        for (int ic = 0; ic < nc4[2]; ++ic)
        for (int id = 0; id < nc4[3]; ++id, ++idx) {
            const int *i3 = comp[0][ia], *j3 = comp[1][ib], *k3 = comp[2][ic], *l3 = comp[3][id];
            double s = 0.0;
            for (int t = 0; t <= i3[0] + j3[0]; ++t)
            for (int u = 0; u <= i3[1] + j3[1]; ++u)
            for (int v = 0; v <= i3[2] + j3[2]; ++v) {
                double Eb = Eab[0][i3[0]][j3[0]][t] * Eab[1][i3[1]][j3[1]][u] * Eab[2][i3[2]][j3[2]][v];
                for (int ta = 0; ta <= k3[0] + l3[0]; ++ta)
                for (int nu = 0; nu <= k3[1] + l3[1]; ++nu)
                for (int ph = 0; ph <= k3[2] + l3[2]; ++ph) {
                    double Ek = Ecd[0][k3[0]][l3[0]][ta] * Ecd[1][k3[1]][l3[1]][nu] * Ecd[2][k3[2]][l3[2]][ph];
                    double sign = ((ta + nu + ph) & 1) ? -1.0 : 1.0;
                    s += sign * Eb * Ek * R0[t + ta][u + nu][v + ph];
                }
            }
            out[idx] += B->cn[((size_t)sa * ORC_NCMAX + ia) * ORC_KMAX + ka]
                      * B->cn[((size_t)sb * ORC_NCMAX + ib) * ORC_KMAX + kb]
                      * B->cn[((size_t)sc * ORC_NCMAX + ic) * ORC_KMAX + kc]
                      * B->cn[((size_t)sd * ORC_NCMAX + id) * ORC_KMAX + kd] * pref * s;
        }
    }
    }
    orc_rctx_free(rc);
}

/* Full N^4 tensor g[mu][nu][la][si] (small N only). */
void orc_eri_full(const void *vB, double *g) {
    const orc_basis *B = (const orc_basis *)vB;
    int N = B->nbf;
    double blk[ORC_NCMAX * ORC_NCMAX * ORC_NCMAX * ORC_NCMAX];
    for (int sa = 0; sa < B->nshell; ++sa)
    for (int sb = 0; sb < B->nshell; ++sb)
    for (int sc = 0; sc < B->nshell; ++sc)
    for (int sd = 0; sd < B->nshell; ++sd) {
        orc_eri_shell_quartet(vB, sa, sb, sc, sd, blk);
        int na = orc_ncart(B->l[sa]), nb = orc_ncart(B->l[sb]), nc = orc_ncart(B->l[sc]), nd = orc_ncart(B->l[sd]);
        int idx = 0;
        for (int ia = 0; ia < na; ++ia)
        for (int ib = 0; ib < nb; ++ib)
        for (int ic = 0; ic < nc; ++ic)
        for (int id = 0; id < nd; ++id, ++idx)
            g[(((size_t)(B->ao[sa] + ia) * N + B->ao[sb] + ib) * N + B->ao[sc] + ic) * N + B->ao[sd] + id] = blk[idx];
    }
}

/* A list of nq shell quartets q[4*i .. 4*i+3]; block i is written at
 * out + off[i] in the layout of orc_eri_shell_quartet.  Each quartet is
 * independent, so the list is shared out over OpenMP threads. */
void orc_eri_quartet_list(const void *vB, int nq, const int *q, const long long *off, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < nq; ++i)
        orc_eri_shell_quartet(vB, q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3], out + off[i]);
}

/* Shell-level Schwarz bounds Q[a*nshell+b] = sqrt(max |(mu nu|mu nu)|). */
void orc_schwarz(const void *vB, double *Q) {
    const orc_basis *B = (const orc_basis *)vB;
    int ns = B->nshell;
#pragma omp parallel for schedule(dynamic, 1)
    for (int sa = 0; sa < ns; ++sa) {
        double blk[ORC_NCMAX * ORC_NCMAX * ORC_NCMAX * ORC_NCMAX];
        for (int sb = 0; sb <= sa; ++sb) {
            orc_eri_shell_quartet(vB, sa, sb, sa, sb, blk);
            int na = orc_ncart(B->l[sa]), nb = orc_ncart(B->l[sb]);
            double m = 0.0;
            for (int ia = 0; ia < na; ++ia)
                for (int ib = 0; ib < nb; ++ib) {
                    double v = fabs(blk[((ia * nb + ib) * na + ia) * nb + ib]);
                    if (v > m) m = v;
                }
            Q[sa * ns + sb] = Q[sb * ns + sa] = sqrt(m);
        }
    }
}

/*
 * J_mu,nu = sum_{la,si} D_la,si (mu nu|la si) and
 * K_mu,nu = sum_{la,si} D_la,si (mu la|nu si)                   (Eq. fock)
 * over each shell quartet that is unique under the 8-fold permutational
 * symmetry (a>=b, c>=d, (ab)>=(cd)); each unique block is scattered to every
 * DISTINCT ordered image of its shell quartet, so that every ordered index
 * quadruple of the full sums is visited exactly once.  Optional Schwarz skip
 * when Q_ab Q_cd < tau (tau <= 0: no screening).  OpenMP over bra pairs
 * with per-thread J/K, summed at the end.
 */
void orc_jk_shard(const void *vB, const double *D, double *J, double *K, double tau, int nthreads,
                  long long *n_quartets, int shard, int nshards);

void orc_jk(const void *vB, const double *D, double *J, double *K, double tau, int nthreads,
            long long *n_quartets) {
    orc_jk_shard(vB, D, J, K, tau, nthreads, n_quartets, 0, 1);
}

/* As orc_jk, restricted to the bra pairs ij with ij % bra_stride == 0: a
 * bounded sample of the same work, for timing the oracle on large cases. */
void orc_jk_sample(const void *vB, const double *D, double *J, double *K, double tau, int nthreads,
                   long long *n_quartets, int bra_stride) {
    orc_jk_shard(vB, D, J, K, tau, nthreads, n_quartets, 0, bra_stride);
}

/* The contribution of the bra pairs ij with ij % nshards == shard; the sum
 * over all shards is orc_jk. */
void orc_jk_shard(const void *vB, const double *D, double *J, double *K, double tau, int nthreads,
                  long long *n_quartets, int shard, int nshards) {
    const orc_basis *B = (const orc_basis *)vB;
    int N = B->nbf, ns = B->nshell;
    double *Q = NULL;
    if (tau > 0.0) {
        Q = (double *)malloc(sizeof(double) * ns * ns);
        orc_schwarz(vB, Q);
    }
    int npair = ns * (ns + 1) / 2;
    int *pa = (int *)malloc(sizeof(int) * npair), *pb = (int *)malloc(sizeof(int) * npair);
    for (int a = 0, k = 0; a < ns; ++a)
        for (int b = 0; b <= a; ++b, ++k) { pa[k] = a; pb[k] = b; }
    memset(J, 0, sizeof(double) * N * N);
    memset(K, 0, sizeof(double) * N * N);
    long long nq = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : nq)
    {
        double *Jt = (double *)calloc((size_t)N * N, sizeof(double));
        double *Kt = (double *)calloc((size_t)N * N, sizeof(double));
        double blk[ORC_NCMAX * ORC_NCMAX * ORC_NCMAX * ORC_NCMAX];
#pragma omp for schedule(dynamic, 1)
        for (int ij = 0; ij < npair; ++ij) {
            if (ij % nshards != shard) continue;
            for (int kl = 0; kl <= ij; ++kl) {
                int s[4] = {pa[ij], pb[ij], pa[kl], pb[kl]};
                if (Q && Q[s[0] * ns + s[1]] * Q[s[2] * ns + s[3]] < tau) continue;
                ++nq;
                orc_eri_shell_quartet(vB, s[0], s[1], s[2], s[3], blk);
                int n4[4];
                for (int q = 0; q < 4; ++q) n4[q] = orc_ncart(B->l[s[q]]);
                /* The 8 images as position permutations of (0,1,2,3). */
                static const int perm[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                                               {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};
                int seen[8][4], nseen = 0;
                for (int g = 0; g < 8; ++g) {
                    int img[4];
                    for (int q = 0; q < 4; ++q) img[q] = s[perm[g][q]];
                    int dup = 0;
                    for (int h = 0; h < nseen; ++h)
                        if (!memcmp(seen[h], img, sizeof(img))) { dup = 1; break; }
                    if (dup) continue;
                    memcpy(seen[nseen++], img, sizeof(img));
                    /* scatter every element of the block to this image */
                    int i4[4];
                    for (i4[0] = 0; i4[0] < n4[0]; ++i4[0])
                    for (i4[1] = 0; i4[1] < n4[1]; ++i4[1])
                    for (i4[2] = 0; i4[2] < n4[2]; ++i4[2])
                    for (i4[3] = 0; i4[3] < n4[3]; ++i4[3]) {
                        double v = blk[((i4[0] * n4[1] + i4[1]) * n4[2] + i4[2]) * n4[3] + i4[3]];
                        int f[4];
                        for (int q = 0; q < 4; ++q) f[q] = B->ao[s[perm[g][q]]] + i4[perm[g][q]];
                        /* image index order (f0 f1 | f2 f3) */
                        Jt[(size_t)f[0] * N + f[1]] += D[(size_t)f[2] * N + f[3]] * v;
                        Kt[(size_t)f[0] * N + f[2]] += D[(size_t)f[1] * N + f[3]] * v;
                    }
                }
            }
        }
#pragma omp critical
        {
            for (size_t i = 0; i < (size_t)N * N; ++i) { J[i] += Jt[i]; K[i] += Kt[i]; }
        }
        free(Jt); free(Kt);
    }
    if (n_quartets) *n_quartets = nq;
    free(pa); free(pb); free(Q);
}

/*
 * One block of J and K by definition, for the functions of shells (sa, sb):
 *   J_mu,nu = sum_{c,d} sum_{la in c, si in d} D_la,si (mu nu|la si)
 *   K_mu,nu = sum_{c,d} sum_{la in c, si in d} D_la,si (mu la|nu si)
 * over ALL ordered shell pairs (c, d); with tau > 0 a quartet is skipped when
 * its Schwarz product is below tau (Q passed in, nshell x nshell), the same
 * rule as the unique-quartet loop since Q_ab Q_cd is permutation invariant.
 * A ket pair (c, d) whose density block D_cd is entirely zero adds nothing to
 * either sum and is skipped.  Jb, Kb: na x nb row-major.  Used to check
 * sampled blocks of large cases.
 */
void orc_jk_block(const void *vB, const double *D, int sa, int sb, double *Jb, double *Kb,
                  double tau, const double *Q) {
    const orc_basis *B = (const orc_basis *)vB;
    int N = B->nbf, ns = B->nshell;
    int na = orc_ncart(B->l[sa]), nb = orc_ncart(B->l[sb]);
    for (int i = 0; i < na * nb; ++i) { Jb[i] = 0.0; Kb[i] = 0.0; }
#pragma omp parallel
    {
        double blk[ORC_NCMAX * ORC_NCMAX * ORC_NCMAX * ORC_NCMAX];
        double Jt[ORC_NCMAX * ORC_NCMAX], Kt[ORC_NCMAX * ORC_NCMAX];
        for (int i = 0; i < na * nb; ++i) { Jt[i] = 0.0; Kt[i] = 0.0; }
#pragma omp for schedule(dynamic, 1)
        for (int sc = 0; sc < ns; ++sc) {
            int nc = orc_ncart(B->l[sc]);
            for (int sd = 0; sd < ns; ++sd) {
                int nd = orc_ncart(B->l[sd]);
                int dz = 1;
                for (int ic = 0; ic < nc && dz; ++ic)
                    for (int id = 0; id < nd; ++id)
                        if (D[(size_t)(B->ao[sc] + ic) * N + B->ao[sd] + id] != 0.0) { dz = 0; break; }
                if (dz) continue;
                if (!(tau > 0.0) || Q[sa * ns + sb] * Q[sc * ns + sd] >= tau) {
                    orc_eri_shell_quartet(vB, sa, sb, sc, sd, blk); /* (ab|cd) */
                    for (int ia = 0; ia < na; ++ia)
                    for (int ib = 0; ib < nb; ++ib)
                    for (int ic = 0; ic < nc; ++ic)
                    for (int id = 0; id < nd; ++id)
                        Jt[ia * nb + ib] += D[(size_t)(B->ao[sc] + ic) * N + B->ao[sd] + id]
                                          * blk[((ia * nb + ib) * nc + ic) * nd + id];
                }
                if (!(tau > 0.0) || Q[sa * ns + sc] * Q[sb * ns + sd] >= tau) {
                    orc_eri_shell_quartet(vB, sa, sc, sb, sd, blk); /* (ac|bd) */
                    for (int ia = 0; ia < na; ++ia)
                    for (int ic = 0; ic < nc; ++ic)
                    for (int ib = 0; ib < nb; ++ib)
                    for (int id = 0; id < nd; ++id)
                        Kt[ia * nb + ib] += D[(size_t)(B->ao[sc] + ic) * N + B->ao[sd] + id]
                                          * blk[((ia * nc + ic) * nb + ib) * nd + id];
                }
            }
        }
#pragma omp critical
        for (int i = 0; i < na * nb; ++i) { Jb[i] += Jt[i]; Kb[i] += Kt[i]; }
    }
}

/* ------------------------------------------------------------------ */
/* Cyclic Jacobi eigensolver for a real symmetric matrix (textbook).   */
/* A (n x n, row-major) is destroyed; w ascending; V columns = vectors. */
/* ------------------------------------------------------------------ */
int orc_jacobi_eigh(int n, double *A, double *w, double *V) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (fabs(apq) < 1e-300) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* columns p, q */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* rows p, q */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    /* selection sort ascending, lower index first on ties */
    for (int i = 0; i < n - 1; ++i) {
        int m = i;
        for (int j = i + 1; j < n; ++j) if (w[j] < w[m]) m = j;
        if (m != i) {
            double t = w[i]; w[i] = w[m]; w[m] = t;
            for (int k = 0; k < n; ++k) { t = V[k * n + i]; V[k * n + i] = V[k * n + m]; V[k * n + m] = t; }
        }
    }
    return sweep;
}
