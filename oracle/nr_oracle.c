/*
 * nr_oracle.c -- CPU reference oracle for the FP64 BSSN hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see nr_oracle.h).  Written for a reader who
 * checks it against arXiv 2505.00097 by eye:
 *   - everything is evaluated in the coordinate basis of the curvilinear
 *     coordinates, exactly in the notation of Sec. 2.1 (Eqs.
 *     metric_RHS_orig_final .. Lambda_RHS_orig_final, the Ricci tensor, the
 *     gauge Eqs. gauge_eqns/damping_eta_final and Eq. Hconstraint);
 *   - gridfunctions are stored rescaled (Sec. 2.2, "Tensor rescaling"):
 *     eps_ij = h_ij S_i S_j, Abar_ij = a_ij S_i S_j, V^i = v^i / S_i, and
 *     only the rescaled gridfunctions are finite-differenced, with the
 *     singular scale factors S_i handled analytically by the chain rule;
 *   - every tensor contraction is a generic index loop (no sparsity or
 *     symmetry is exploited beyond storing symmetric tensors twice);
 *   - FP64 throughout, compiled with -fno-fast-math -ffp-contract=off.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   R-Lambda: Eq. Lambda_RHS_orig_final is read as
 *       -2 Abar^{ij}(d_j alpha - 6 alpha d_j phi) + 2 alpha Abar^{jk} Delta^i_jk
 *     (the printed form lacks the two factors of alpha; with alpha=beta=0
 *     the slice must not evolve, which only this reading satisfies).
 *   R-Lie: d_perp = d_t - L_beta, the Lie derivative written with partial
 *     derivatives; only the beta^k d_k(.) parts use upwinded stencils.
 *   R-betalow: in 2 Dhat_(i beta_j) the index of beta is lowered with
 *     gammahat (the only choice consistent with d_t gammabar of the
 *     covariant BSSN system).
 *   R-Delta: Delta^k_ij = 1/2 gammabar^{kl}(Dhat_i eps_jl + Dhat_j eps_il
 *     - Dhat_l eps_ij), never Gammabar - Gammahat evaluated separately.
 *   R-gauge: d_t beta^i and d_t B^i use coordinate partial derivatives of the
 *     unrescaled components; the d_t Lambdabar^i substituted into d_t B^i is
 *     the right-hand side of Eq. Lambda as printed, i.e. d_perp Lambdabar^i
 *     (the Lie derivative is not added back), without Kreiss-Oliger
 *     dissipation.
 *   R-KO: rhs_g += sum_d sigma/(64 S_d dxx_d) delta^6_d g on the rescaled g:
 *     the strength refers to the physical spacing S_d dxx_d.  With the
 *     logical spacing dxx_d alone, the damping rate sigma/dxx_d of the Nyquist
 *     mode exceeds the RK4 stability bound (2.785/dt) on the stretched sinh
 *     grids of Sec. 4.1 at the CFL factor 0.5, since dt is set by the physical
 *     spacing.
 *   R-Sommerfeld: at pure-outer ghosts d_t f = -v [ (x^j/r) d_j f + (f - f_inf)/r ]
 *     on each rescaled gridfunction; one-sided 4th-order stencils where the
 *     centred one does not fit.
 */
#include "nr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NGF 24
enum { G_HDD = 0, G_ADD = 6, G_CF = 12, G_TRK = 13, G_LAM = 14, G_VET = 17, G_BET = 20, G_ALPHA = 23 };

static const int SYM_I[6] = {0, 0, 0, 1, 1, 2};
static const int SYM_J[6] = {0, 1, 2, 1, 2, 2};

/* tensor type of a gridfunction: 0 scalar, 1+i vector component i, 4+s DD component s */
static int gf_type(int gf)
{
    if (gf < 6) return 4 + gf;
    if (gf < 12) return 4 + (gf - 6);
    if (gf == G_CF || gf == G_TRK || gf == G_ALPHA) return 0;
    if (gf >= G_LAM && gf < G_LAM + 3) return 1 + (gf - G_LAM);
    if (gf >= G_VET && gf < G_VET + 3) return 1 + (gf - G_VET);
    return 1 + (gf - G_BET);
}

/* Loop parallelism of the point-wise loops below (every iteration writes its own
 * points only; no expression depends on the thread count): p->nthreads threads,
 * or the runtime default when it is <= 0. */
static int team_of(const orc_params* p)
{
#ifdef _OPENMP
    return p->nthreads > 0 ? p->nthreads : omp_get_max_threads();
#else
    (void)p;
    return 1;
#endif
}
#ifdef _OPENMP
#define ORC_PARALLEL_FOR _Pragma("omp parallel for schedule(static) num_threads(nt)")
#else
#define ORC_PARALLEL_FOR
#endif

/* ------------------------------------------------------------------ grid */

/* Logical domain of each coordinate system (Sec. 3: cell-centred, logically
 * rectangular grid; sinh radial map of Sec. 4.1). */
static void domain(const orc_params* p, double lo[3], double hi[3])
{
    if (p->coords == ORC_SINH_CYLINDRICAL) {
        lo[0] = 0.0;   hi[0] = 1.0;   /* rho via sinh map   */
        lo[1] = -M_PI; hi[1] = M_PI;  /* phi                */
        lo[2] = -1.0;  hi[2] = 1.0;   /* z via sinh map     */
    } else {
        lo[0] = 0.0;   hi[0] = 1.0;   /* r via sinh (or linear) map */
        lo[1] = 0.0;   hi[1] = M_PI;  /* theta */
        lo[2] = -M_PI; hi[2] = M_PI;  /* phi   */
    }
}

long orc_sizes(const orc_params* p, int n_out[3])
{
    long T = 1;
    for (int d = 0; d < 3; d++) {
        int n = p->N[d] + 2 * p->NG;
        if (n_out) n_out[d] = n;
        T *= n;
    }
    return T;
}

static double dxx_of(const orc_params* p, int d)
{
    double lo[3], hi[3];
    domain(p, lo, hi);
    return (hi[d] - lo[d]) / p->N[d];
}

/* cell centres: xx_min + (i - NG + 1/2) dxx  (Sec. 3) */
double orc_xx(const orc_params* p, int d, int i)
{
    double lo[3], hi[3];
    domain(p, lo, hi);
    return lo[d] + ((double)(i - p->NG) + 0.5) * dxx_of(p, d);
}

static void unflatten(const int n[3], long idx, int ii[3])
{
    ii[0] = (int)(idx % n[0]);
    ii[1] = (int)((idx / n[0]) % n[1]);
    ii[2] = (int)(idx / ((long)n[0] * n[1]));
}

/* x'(x) = A sinh(x/w)/sinh(1/w) and its first three derivatives (Sec. 4.1);
 * linear map r = A x when sinh_kind == 0. */
static void radial_map(double A, double w, int sinh_kind, double x, double f[4])
{
    if (sinh_kind) {
        double s = sinh(1.0 / w), sh = sinh(x / w), ch = cosh(x / w);
        f[0] = A * sh / s;
        f[1] = A * ch / (w * s);
        f[2] = A * sh / (w * w * s);
        f[3] = A * ch / (w * w * w * s);
    } else {
        f[0] = A * x;
        f[1] = A;
        f[2] = 0.0;
        f[3] = 0.0;
    }
}

/* Reference-metric scale factors S_i = sqrt(gammahat_ii) (Sec. 2.2), their
 * derivatives, the Cartesian position and the Jacobian dx^a/dxx^d, all
 * analytically continued (signed S) so that ghost points outside the
 * coordinate range are described too. */
typedef struct {
    double S[3], dS[3][3], ddS[3][3][3]; /* dS[i][k] = d_k S_i */
    double cart[3];
    double J[3][3];                      /* J[a][d] = d x^a / d xx^d */
} rfm_pt;

static void rfm_eval(const orc_params* p, const double xx[3], rfm_pt* o)
{
    memset(o, 0, sizeof *o);
    if (p->coords == ORC_SINH_CYLINDRICAL) {
        double rho[4], z[4];
        radial_map(p->ampl[0], p->sinhw[0], 1, xx[0], rho);
        radial_map(p->ampl[2], p->sinhw[2], 1, xx[2], z);
        double c = cos(xx[1]), s = sin(xx[1]);
        o->S[0] = rho[1];
        o->S[1] = rho[0];
        o->S[2] = z[1];
        o->dS[0][0] = rho[2];
        o->dS[1][0] = rho[1];
        o->dS[2][2] = z[2];
        o->ddS[0][0][0] = rho[3];
        o->ddS[1][0][0] = rho[2];
        o->ddS[2][2][2] = z[3];
        o->cart[0] = rho[0] * c;
        o->cart[1] = rho[0] * s;
        o->cart[2] = z[0];
        o->J[0][0] = rho[1] * c;  o->J[0][1] = -rho[0] * s; o->J[0][2] = 0.0;
        o->J[1][0] = rho[1] * s;  o->J[1][1] = rho[0] * c;  o->J[1][2] = 0.0;
        o->J[2][0] = 0.0;         o->J[2][1] = 0.0;         o->J[2][2] = z[1];
    } else {
        double r[4];
        radial_map(p->ampl[0], p->sinhw[0], p->coords == ORC_SINH_SPHERICAL, xx[0], r);
        double st = sin(xx[1]), ct = cos(xx[1]), sp = sin(xx[2]), cp = cos(xx[2]);
        o->S[0] = r[1];
        o->S[1] = r[0];
        o->S[2] = r[0] * st;
        o->dS[0][0] = r[2];
        o->dS[1][0] = r[1];
        o->dS[2][0] = r[1] * st;
        o->dS[2][1] = r[0] * ct;
        o->ddS[0][0][0] = r[3];
        o->ddS[1][0][0] = r[2];
        o->ddS[2][0][0] = r[2] * st;
        o->ddS[2][0][1] = r[1] * ct;
        o->ddS[2][1][0] = r[1] * ct;
        o->ddS[2][1][1] = -r[0] * st;
        o->cart[0] = r[0] * st * cp;
        o->cart[1] = r[0] * st * sp;
        o->cart[2] = r[0] * ct;
        o->J[0][0] = r[1] * st * cp; o->J[0][1] = r[0] * ct * cp; o->J[0][2] = -r[0] * st * sp;
        o->J[1][0] = r[1] * st * sp; o->J[1][1] = r[0] * ct * sp; o->J[1][2] = r[0] * st * cp;
        o->J[2][0] = r[1] * ct;      o->J[2][1] = -r[0] * st;     o->J[2][2] = 0.0;
    }
}

static void xx_of_idx(const orc_params* p, const int n[3], long idx, double xx[3], int ii[3])
{
    unflatten(n, idx, ii);
    for (int d = 0; d < 3; d++) xx[d] = orc_xx(p, d, ii[d]);
}

void orc_cart(const orc_params* p, long idx, double out[3])
{
    int n[3], ii[3];
    double xx[3];
    rfm_pt R;
    orc_sizes(p, n);
    xx_of_idx(p, n, idx, xx, ii);
    rfm_eval(p, xx, &R);
    for (int a = 0; a < 3; a++) out[a] = R.cart[a];
}

void orc_cart_all(const orc_params* p, double* out)
{
    int n[3];
    long T = orc_sizes(p, n);
    for (long idx = 0; idx < T; idx++) {
        int ii[3];
        double xx[3];
        rfm_pt R;
        xx_of_idx(p, n, idx, xx, ii);
        rfm_eval(p, xx, &R);
        for (int a = 0; a < 3; a++) out[3 * idx + a] = R.cart[a];
    }
}

/* generic 3x3 inverse by cofactors; returns the determinant */
static double det3(const double m[3][3])
{
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* Levi-Civita symbol [ijk] */
static int levi(int i, int j, int k)
{
    if (i == j || j == k || i == k) return 0;
    return ((i == 0 && j == 1) || (i == 1 && j == 2) || (i == 2 && j == 0)) ? 1 : -1;
}

static double inv3(const double m[3][3], double inv[3][3])
{
    double c00 = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    double c01 = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    double c02 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    double det = m[0][0] * c00 + m[0][1] * c01 + m[0][2] * c02;
    double id = 1.0 / det;
    inv[0][0] = c00 * id;
    inv[1][0] = c01 * id;
    inv[2][0] = c02 * id;
    inv[0][1] = (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id;
    inv[1][1] = (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id;
    inv[2][1] = (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id;
    inv[0][2] = (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id;
    inv[1][2] = (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id;
    inv[2][2] = (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id;
    return det;
}

/* ----------------------------------------------------- reference metric */

typedef struct {
    double g[3][3], dg[3][3][3], ddg[3][3][3][3]; /* gammahat_ij, d_k, d_k d_l */
    double ginv[3][3], dginv[3][3][3];
    double Gam[3][3][3];                          /* Gammahat^k_ij = Gam[k][i][j] */
    double dGam[3][3][3][3];                      /* d_m Gammahat^k_ij = dGam[k][i][j][m] */
} refmet;

/* gammahat_ij = diag(S_i^2) (Sec. 2.2) and its Christoffel symbols by the
 * textbook formula with generic index loops. */
static void refmet_from(const rfm_pt* R, refmet* M)
{
    memset(M, 0, sizeof *M);
    for (int i = 0; i < 3; i++) {
        M->g[i][i] = R->S[i] * R->S[i];
        for (int k = 0; k < 3; k++) {
            M->dg[i][i][k] = 2.0 * R->S[i] * R->dS[i][k];
            for (int l = 0; l < 3; l++)
                M->ddg[i][i][k][l] = 2.0 * (R->dS[i][k] * R->dS[i][l] + R->S[i] * R->ddS[i][k][l]);
        }
    }
    inv3(M->g, M->ginv);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int k = 0; k < 3; k++) {
                double s = 0.0;
                for (int c = 0; c < 3; c++)
                    for (int d = 0; d < 3; d++) s += M->ginv[a][c] * M->dg[c][d][k] * M->ginv[d][b];
                M->dginv[a][b][k] = -s;
            }
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0.0;
                for (int l = 0; l < 3; l++)
                    s += M->ginv[k][l] * (M->dg[j][l][i] + M->dg[i][l][j] - M->dg[i][j][l]);
                M->Gam[k][i][j] = 0.5 * s;
                for (int m = 0; m < 3; m++) {
                    double t = 0.0;
                    for (int l = 0; l < 3; l++)
                        t += M->dginv[k][l][m] * (M->dg[j][l][i] + M->dg[i][l][j] - M->dg[i][j][l]) +
                             M->ginv[k][l] * (M->ddg[j][l][i][m] + M->ddg[i][l][j][m] - M->ddg[i][j][l][m]);
                    M->dGam[k][i][j][m] = 0.5 * t;
                }
            }
}

void orc_refmetric(const orc_params* p, const double xx[3], double* S3, double* ghat, double* dghat,
                   double* ddghat, double* Gam, double* dGam)
{
    rfm_pt R;
    refmet M;
    rfm_eval(p, xx, &R);
    refmet_from(&R, &M);
    if (S3) memcpy(S3, R.S, sizeof R.S);
    if (ghat) memcpy(ghat, M.g, sizeof M.g);
    if (dghat) memcpy(dghat, M.dg, sizeof M.dg);
    if (ddghat) memcpy(ddghat, M.ddg, sizeof M.ddg);
    if (Gam) memcpy(Gam, M.Gam, sizeof M.Gam);
    if (dGam) memcpy(dGam, M.dGam, sizeof M.dGam);
}

/* ------------------------------------------------------------- stencils */
/* 4th-order finite differences (Sec. 3 "Spatial derivatives"). */

double orc_d1(const double* f, long st, double h)
{
    return (f[-2 * st] - 8.0 * f[-st] + 8.0 * f[st] - f[2 * st]) / (12.0 * h);
}

double orc_d2(const double* f, long st, double h)
{
    return (-f[-2 * st] + 16.0 * f[-st] - 30.0 * f[0] + 16.0 * f[st] - f[2 * st]) / (12.0 * h * h);
}

/* mixed second derivative: product of the two first-derivative stencils */
double orc_d11(const double* f, long sa, long sb, double ha, double hb)
{
    static const double w[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
    double s = 0.0;
    for (int b = -2; b <= 2; b++) {
        double inner = 0.0;
        for (int a = -2; a <= 2; a++) inner += w[a + 2] * f[a * sa + b * sb];
        s += w[b + 2] * inner;
    }
    return s / (144.0 * ha * hb);
}

/* Finite differences of order N_FD = 2 (NG - 1) for NG other than 3 (the
 * production scheme of Sec. 4.1 uses N_FD = 8, NG = 5).  The weights come from
 * Fornberg's recursion (B. Fornberg, Math. Comp. 51 (1988) 699-706) on the
 * offsets each stencil uses:
 *   centred first and second derivatives: -m..m (m = N_FD/2);
 *   upwind first derivative: -(m-1)..m+1 for vet > 0, the mirror otherwise
 *     (the centred window shifted one point upwind; N_G = m+1, Sec. 3);
 *   one-sided first derivatives at outer ghosts: the 2m+1 window a..a+2m with
 *     a = clamp(-m, -i, n-1-i-2m) (the centred one where it fits);
 *   Kreiss-Oliger: the difference of order 2r = N_FD + 2 (binomial weights). */
static void fd_weights(double x0, const double* x, int n, int mord, double* c)
{
    memset(c, 0, sizeof(double) * (size_t)(mord + 1) * n);
    double c1 = 1.0, c4 = x[0] - x0;
    c[0] = 1.0;
    for (int i = 1; i < n; i++) {
        int mn = i < mord ? i : mord;
        double c2 = 1.0, c5 = c4;
        c4 = x[i] - x0;
        for (int j = 0; j < i; j++) {
            double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                for (int k = mn; k >= 1; k--) c[k * n + i] = c1 * (k * c[(k - 1) * n + i - 1] - c5 * c[k * n + i - 1]) / c2;
                c[i] = -c1 * c5 * c[i - 1] / c2;
            }
            for (int k = mn; k >= 1; k--) c[k * n + j] = (c4 * c[k * n + j] - k * c[(k - 1) * n + j]) / c3;
            c[j] = c4 * c[j] / c3;
        }
        c1 = c2;
    }
}

/* The weights are rational; each set is kept as integers over the smallest
 * common denominator found from the recursion's doubles, so that the stencils
 * of a constant are exactly zero (a flat metric stays exactly flat). */
#define FD_MAXW 17
typedef struct {
    int m;                    /* N_FD / 2 */
    double d1[FD_MAXW];       /* offsets -m..m: integer weights over den1, times h */
    double d2[FD_MAXW];       /* offsets -m..m, over den2, times h^2 */
    double up[FD_MAXW];       /* offsets -(m-1)..m+1, over denu, times h */
    double ko[FD_MAXW + 2];   /* offsets -(m+1)..m+1 (integers) */
    double os[FD_MAXW][FD_MAXW]; /* os[-a]: offsets a..a+2m, over deno[-a], times h */
    double den1, den2, denu, deno[FD_MAXW];
} fdw;

/* smallest D <= 10^7 with every w D within 1e-7 of an integer; w <- round(w D) */
static double integerise(double* w, int n)
{
    for (long D = 1; D <= 10000000; D++) {
        int ok = 1;
        for (int i = 0; i < n && ok; i++) ok = fabs(w[i] * D - nearbyint(w[i] * D)) < 1e-7;
        if (ok) {
            for (int i = 0; i < n; i++) w[i] = nearbyint(w[i] * D);
            return (double)D;
        }
    }
    return 0.0;
}

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

static void fdw_make(int NG, fdw* W)
{
    int m = NG - 1, n = 2 * m + 1;
    double x[FD_MAXW], c[3 * FD_MAXW];
    memset(W, 0, sizeof *W);
    W->m = m;
    for (int i = 0; i < n; i++) x[i] = i - m;
    fd_weights(0.0, x, n, 2, c);
    for (int i = 0; i < n; i++) { W->d1[i] = c[n + i]; W->d2[i] = c[2 * n + i]; }
    W->den1 = integerise(W->d1, n);
    W->den2 = integerise(W->d2, n);
    for (int i = 0; i < n; i++) x[i] = i - (m - 1);
    fd_weights(0.0, x, n, 1, c);
    for (int i = 0; i < n; i++) W->up[i] = c[n + i];
    W->denu = integerise(W->up, n);
    for (int a = 0; a <= 2 * m; a++) {
        for (int i = 0; i < n; i++) x[i] = i - a;
        fd_weights(0.0, x, n, 1, c);
        for (int i = 0; i < n; i++) W->os[a][i] = c[n + i];
        W->deno[a] = integerise(W->os[a], n);
    }
    int r = m + 1;
    /* (E^(1/2) - E^(-1/2))^(2r): (-1)^(r+k) C(2r, r+k) at offset k */
    for (int k = -r; k <= r; k++) W->ko[k + r] = (((k + r) % 2) ? -1.0 : 1.0) * binom(2 * r, k + r);
}

/* weights of the order-(2(NG-1)) stencils, for the pins: which 0 centred first
 * derivative, 1 centred second, 2 upwind (forward), 3 Kreiss-Oliger difference,
 * 4 one-sided with window start a; returns the number of weights */
int orc_fd_weights(int NG, int which, int a, double* w)
{
    fdw W;
    if (NG < 2 || 2 * (NG - 1) + 3 > FD_MAXW) return 0;
    fdw_make(NG, &W);
    int n = 2 * W.m + 1;
    if (which == 4 && (a > 0 || a < -2 * W.m)) return 0;
    const double* src = which == 0 ? W.d1 : which == 1 ? W.d2 : which == 2 ? W.up : which == 3 ? W.ko : W.os[-a];
    const double den = which == 0 ? W.den1 : which == 1 ? W.den2 : which == 2 ? W.denu : which == 3 ? 1.0 : W.deno[-a];
    if (which == 3) n += 2;
    for (int i = 0; i < n; i++) w[i] = src[i] / den;
    return n;
}

static double sten(const double* f, long st, const double* w, int lo, int hi)
{
    double s = 0.0;
    for (int k = lo; k <= hi; k++) s += w[k - lo] * f[k * st];
    return s;
}

/* upwind-biased first derivative: offsets -1..+3 (forward) or -3..+1 */
double orc_dup(const double* f, long st, double h, int forward)
{
    if (forward)
        return (-3.0 * f[-st] - 10.0 * f[0] + 18.0 * f[st] - 6.0 * f[2 * st] + f[3 * st]) / (12.0 * h);
    return (-f[-3 * st] + 6.0 * f[-2 * st] - 18.0 * f[-st] + 10.0 * f[0] + 3.0 * f[st]) / (12.0 * h);
}

/* sixth difference used by Kreiss-Oliger dissipation */
double orc_ko6(const double* f, long st)
{
    return f[-3 * st] - 6.0 * f[-2 * st] + 15.0 * f[-st] - 20.0 * f[0] + 15.0 * f[st] - 6.0 * f[2 * st] +
           f[3 * st];
}

/* first derivative with the one-sided variants used at outer ghosts:
 * kind 0 centred, 1 offsets -3..+1, 2 offsets -4..0, 3 offsets -1..+3, 4 offsets 0..+4 */
double orc_d1_onesided(const double* f, long st, double h, int kind)
{
    switch (kind) {
    case 0: return orc_d1(f, st, h);
    case 1: return (-f[-3 * st] + 6.0 * f[-2 * st] - 18.0 * f[-st] + 10.0 * f[0] + 3.0 * f[st]) / (12.0 * h);
    case 2: return (3.0 * f[-4 * st] - 16.0 * f[-3 * st] + 36.0 * f[-2 * st] - 48.0 * f[-st] + 25.0 * f[0]) / (12.0 * h);
    case 3: return (-3.0 * f[-st] - 10.0 * f[0] + 18.0 * f[st] - 6.0 * f[2 * st] + f[3 * st]) / (12.0 * h);
    default: return (-25.0 * f[0] + 48.0 * f[st] - 36.0 * f[2 * st] + 16.0 * f[3 * st] - 3.0 * f[4 * st]) / (12.0 * h);
    }
}

static int onesided_kind(int i, int n)
{
    if (i - 2 >= 0 && i + 2 < n) return 0;
    if (i + 2 >= n) return (i + 1 < n && i - 3 >= 0) ? 1 : 2;
    return (i - 1 >= 0) ? 3 : 4;
}

/* ------------------------------------------------------------ boundaries */

static int is_canonical(const orc_params* p, const int ii[3])
{
    int NG = p->NG;
    if (ii[0] < NG) return 0; /* r<0 or rho<0 */
    if (p->coords == ORC_SINH_CYLINDRICAL) return ii[1] >= NG && ii[1] < NG + p->N[1];
    return ii[1] >= NG && ii[1] < NG + p->N[1] && ii[2] >= NG && ii[2] < NG + p->N[2];
}

static int is_interior(const orc_params* p, const int ii[3])
{
    for (int d = 0; d < 3; d++)
        if (ii[d] < p->NG || ii[d] >= p->NG + p->N[d]) return 0;
    return 1;
}

/* unit frame vectors e_d = (dx/dxx^d)/S_d with signed, analytically
 * continued S (the rescaled basis of Sec. 2.2) */
static void frame_vectors(const rfm_pt* R, double e[3][3])
{
    for (int d = 0; d < 3; d++)
        for (int a = 0; a < 3; a++) e[d][a] = R->J[a][d] / R->S[d];
}

/* Parity signs p_d = e_d(ghost) . e_d(source); the frames must be related by
 * a diagonal +-1 matrix. */
static int parity_from_frames(const rfm_pt* Rg, const rfm_pt* Rs, int8_t par[10])
{
    double eg[3][3], es[3][3];
    int pd[3];
    frame_vectors(Rg, eg);
    frame_vectors(Rs, es);
    for (int d = 0; d < 3; d++) {
        for (int d2 = 0; d2 < 3; d2++) {
            double dot = eg[d][0] * es[d2][0] + eg[d][1] * es[d2][1] + eg[d][2] * es[d2][2];
            if (d2 == d) {
                if (fabs(fabs(dot) - 1.0) > 1e-10) return 1;
                pd[d] = dot > 0 ? 1 : -1;
            } else if (fabs(dot) > 1e-10) {
                return 1;
            }
        }
    }
    par[0] = 1;
    for (int d = 0; d < 3; d++) par[1 + d] = (int8_t)pd[d];
    for (int s = 0; s < 6; s++) par[4 + s] = (int8_t)(pd[SYM_I[s]] * pd[SYM_J[s]]);
    return 0;
}

/* Inverse coordinate map: Cartesian point -> canonical logical coordinates. */
static void cart_to_xx(const orc_params* p, const double x[3], double xx[3])
{
    if (p->coords == ORC_SINH_CYLINDRICAL) {
        double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
        xx[0] = p->sinhw[0] * asinh(rho * sinh(1.0 / p->sinhw[0]) / p->ampl[0]);
        xx[1] = atan2(x[1], x[0]);
        xx[2] = p->sinhw[2] * asinh(x[2] * sinh(1.0 / p->sinhw[2]) / p->ampl[2]);
    } else {
        double rxy = sqrt(x[0] * x[0] + x[1] * x[1]);
        double r = sqrt(rxy * rxy + x[2] * x[2]);
        if (p->coords == ORC_SINH_SPHERICAL)
            xx[0] = p->sinhw[0] * asinh(r * sinh(1.0 / p->sinhw[0]) / p->ampl[0]);
        else
            xx[0] = r / p->ampl[0];
        xx[1] = atan2(rxy, x[2]);
        xx[2] = atan2(x[1], x[0]);
    }
}

/* Map builder: each point's Cartesian position is inverted to canonical
 * coordinates and rounded to the nearest cell centre (Sec. 3: inner
 * boundary points map to interior or outer-boundary points elsewhere on the
 * grid, with parity transformations). */
int orc_build_map(const orc_params* p, int32_t* src, int8_t* parity, int32_t* cls)
{
    int n[3];
    long T = orc_sizes(p, n);
    double lo[3], hi[3];
    domain(p, lo, hi);
    int bad = 0;
    const int nt = team_of(p);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
#endif
    for (long idx = 0; idx < T; idx++) {
        int ii[3], jj[3];
        double xx[3], sx[3];
        rfm_pt Rg, Rs;
        xx_of_idx(p, n, idx, xx, ii);
        rfm_eval(p, xx, &Rg);
        if (is_canonical(p, ii)) {
            src[idx] = (int32_t)idx;
            cls[idx] = is_interior(p, ii) ? 0 : 1;
            for (int t = 0; t < 10; t++) parity[10 * idx + t] = 1;
            continue;
        }
        cart_to_xx(p, Rg.cart, sx);
        long sidx = 0;
        for (int d = 2; d >= 0; d--) {
            double f = (sx[d] - lo[d]) / dxx_of(p, d) + p->NG - 0.5;
            double fr = floor(f + 0.5);
            if (fabs(f - fr) > 1e-6 || fr < 0 || fr >= n[d]) { bad = 1; fr = 0; }
            jj[d] = (int)fr;
            sidx = sidx * n[d] + jj[d];
        }
        if (!bad && !is_canonical(p, jj)) bad = 1;
        double sxx[3];
        for (int d = 0; d < 3; d++) sxx[d] = orc_xx(p, d, jj[d]);
        rfm_eval(p, sxx, &Rs);
        src[idx] = (int32_t)sidx;
        cls[idx] = 2;
        if (parity_from_frames(&Rg, &Rs, &parity[10 * idx])) bad = 1;
    }
    return bad;
}

/* Same map by brute-force nearest Cartesian search over all canonical points
 * (O(T^2); for tiny grids, to pin orc_build_map). */
int orc_build_map_bruteforce(const orc_params* p, int32_t* src, int8_t* parity, int32_t* cls)
{
    int n[3];
    long T = orc_sizes(p, n);
    double* cart = (double*)malloc(sizeof(double) * 3 * T);
    char* canon = (char*)malloc(T);
    for (long idx = 0; idx < T; idx++) {
        int ii[3];
        double xx[3];
        rfm_pt R;
        xx_of_idx(p, n, idx, xx, ii);
        rfm_eval(p, xx, &R);
        memcpy(&cart[3 * idx], R.cart, sizeof R.cart);
        canon[idx] = (char)is_canonical(p, ii);
    }
    int bad = 0;
    for (long idx = 0; idx < T; idx++) {
        long best = -1;
        double bd = 1e300;
        for (long c = 0; c < T; c++) {
            if (!canon[c]) continue;
            double dx = cart[3 * c] - cart[3 * idx], dy = cart[3 * c + 1] - cart[3 * idx + 1],
                   dz = cart[3 * c + 2] - cart[3 * idx + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < bd) { bd = d2; best = c; }
        }
        double scale = 1.0 + fabs(cart[3 * idx]) + fabs(cart[3 * idx + 1]) + fabs(cart[3 * idx + 2]);
        if (best < 0 || sqrt(bd) > 1e-9 * scale) { bad = 1; best = idx; }
        int ii[3];
        double xx[3], sxx[3];
        rfm_pt Rg, Rs;
        xx_of_idx(p, n, idx, xx, ii);
        xx_of_idx(p, n, best, sxx, ii);
        rfm_eval(p, xx, &Rg);
        rfm_eval(p, sxx, &Rs);
        src[idx] = (int32_t)best;
        if (best == idx) {
            xx_of_idx(p, n, idx, xx, ii);
            cls[idx] = is_interior(p, ii) ? 0 : 1;
            for (int t = 0; t < 10; t++) parity[10 * idx + t] = 1;
        } else {
            cls[idx] = 2;
            if (parity_from_frames(&Rg, &Rs, &parity[10 * idx])) bad = 1;
        }
    }
    free(cart);
    free(canon);
    return bad;
}

typedef struct {
    long T;
    int32_t* src;
    int8_t* par;
    int32_t* cls;
} bmap;

static int bmap_make(const orc_params* p, bmap* m)
{
    int n[3];
    m->T = orc_sizes(p, n);
    m->src = (int32_t*)malloc(sizeof(int32_t) * m->T);
    m->cls = (int32_t*)malloc(sizeof(int32_t) * m->T);
    m->par = (int8_t*)malloc(10 * m->T);
    return orc_build_map(p, m->src, m->par, m->cls);
}

static void bmap_free(bmap* m)
{
    free(m->src);
    free(m->cls);
    free(m->par);
}

static void inner_bc_with(const bmap* m, double* gfs, int nt)
{
    /* sources are interior or pure-outer points, never written here */
    ORC_PARALLEL_FOR
    for (long idx = 0; idx < m->T; idx++) {
        if (m->cls[idx] != 2) continue;
        for (int gf = 0; gf < NGF; gf++)
            gfs[gf * m->T + idx] = (double)m->par[10 * idx + gf_type(gf)] * gfs[gf * m->T + m->src[idx]];
    }
}

int orc_inner_bc(const orc_params* p, double* gfs)
{
    bmap m;
    int bad = bmap_make(p, &m);
    inner_bc_with(&m, gfs, team_of(p));
    bmap_free(&m);
    return bad;
}

/* Sommerfeld radiation condition at pure-outer ghost points (Sec. 3, outer
 * boundary points; form R-Sommerfeld in the header comment). */
static void outer_bc_with(const orc_params* p, const bmap* m, const double* gfs, double* rhs)
{
    int n[3];
    long T = orc_sizes(p, n);
    long st[3] = {1, n[0], (long)n[0] * n[1]};
    double h[3] = {dxx_of(p, 0), dxx_of(p, 1), dxx_of(p, 2)};
    fdw Wd;
    fdw_make(p->NG, &Wd);
    const int nt = team_of(p);
    ORC_PARALLEL_FOR
    for (long idx = 0; idx < T; idx++) {
        if (m->cls[idx] != 1) continue;
        int ii[3];
        double xx[3], Jinv[3][3];
        rfm_pt R;
        xx_of_idx(p, n, idx, xx, ii);
        rfm_eval(p, xx, &R);
        inv3(R.J, Jinv); /* Jinv[d][a] = d xx^d / d x^a */
        double r = sqrt(R.cart[0] * R.cart[0] + R.cart[1] * R.cart[1] + R.cart[2] * R.cart[2]);
        int kind[3];
        for (int d = 0; d < 3; d++) kind[d] = onesided_kind(ii[d], n[d]);
        for (int gf = 0; gf < NGF; gf++) {
            const double* f = &gfs[gf * T + idx];
            double dl[3], radial = 0.0;
            for (int d = 0; d < 3; d++) {
                if (p->NG == 3) {
                    dl[d] = orc_d1_onesided(f, st[d], h[d], kind[d]);
                } else {
                    int mm = Wd.m, a = -mm;
                    if (a < -ii[d]) a = -ii[d];
                    if (a > n[d] - 1 - ii[d] - 2 * mm) a = n[d] - 1 - ii[d] - 2 * mm;
                    dl[d] = sten(f, st[d], Wd.os[-a], a, a + 2 * mm) / (Wd.deno[-a] * h[d]);
                }
            }
            for (int a = 0; a < 3; a++) {
                double dfa = 0.0;
                for (int d = 0; d < 3; d++) dfa += Jinv[d][a] * dl[d];
                radial += (R.cart[a] / r) * dfa;
            }
            rhs[gf * T + idx] = -p->wavespeed[gf] * (radial + (f[0] - p->f_inf[gf]) / r);
        }
    }
}

void orc_outer_bc(const orc_params* p, const double* gfs, double* rhs)
{
    bmap m;
    bmap_make(p, &m);
    outer_bc_with(p, &m, gfs, rhs);
    bmap_free(&m);
}

/* ------------------------------------------------------- point evaluation */

/* Unrescaled coordinate-basis fields at one interior point. */
typedef struct {
    double eps[3][3], deps[3][3][3], ddeps[3][3][3][3], adv_eps[3][3];
    double A[3][3], dA[3][3][3], adv_A[3][3];   /* dA[i][j][k] = d_k Abar_ij */
    double W, dW[3], ddW[3][3], adv_W;
    double K, dK[3], adv_K;
    double Lam[3], dLam[3][3], adv_Lam[3];   /* dLam[i][k] = d_k Lambda^i */
    double beta[3], dbeta[3][3], ddbeta[3][3][3], adv_beta[3];
    double B[3], adv_B[3];
    double alpha, dalpha[3], ddalpha[3][3], adv_alpha;
} pt_fields;

/* rescaling factor X = Rv * x of a gridfunction of the given tensor type,
 * with its first and second coordinate derivatives */
static void rescale_factor(const rfm_pt* R, int type, double* Rv, double Rd[3], double Rdd[3][3])
{
    if (type == 0) {
        *Rv = 1.0;
        for (int k = 0; k < 3; k++) {
            Rd[k] = 0.0;
            for (int l = 0; l < 3; l++) Rdd[k][l] = 0.0;
        }
    } else if (type < 4) { /* contravariant vector: V^i = v^i / S_i */
        int i = type - 1;
        double S = R->S[i];
        *Rv = 1.0 / S;
        for (int k = 0; k < 3; k++) {
            Rd[k] = -R->dS[i][k] / (S * S);
            for (int l = 0; l < 3; l++)
                Rdd[k][l] = -R->ddS[i][k][l] / (S * S) + 2.0 * R->dS[i][k] * R->dS[i][l] / (S * S * S);
        }
    } else { /* covariant 2-tensor: T_ij = t_ij S_i S_j */
        int i = SYM_I[type - 4], j = SYM_J[type - 4];
        *Rv = R->S[i] * R->S[j];
        for (int k = 0; k < 3; k++) {
            Rd[k] = R->dS[i][k] * R->S[j] + R->S[i] * R->dS[j][k];
            for (int l = 0; l < 3; l++)
                Rdd[k][l] = R->ddS[i][k][l] * R->S[j] + R->dS[i][k] * R->dS[j][l] + R->dS[i][l] * R->dS[j][k] +
                            R->S[i] * R->ddS[j][k][l];
        }
    }
}

static void load_point(const orc_params* p, const int n[3], long T, const double* gfs, long idx,
                       const rfm_pt* R, pt_fields* F, const fdw* Wd)
{
    long st[3] = {1, n[0], (long)n[0] * n[1]};
    double h[3] = {dxx_of(p, 0), dxx_of(p, 1), dxx_of(p, 2)};
    double X[NGF], dX[NGF][3], ddX[NGF][3][3], adv[NGF];
    int fwd[3];
    double beta[3];
    for (int k = 0; k < 3; k++) {
        double vet = gfs[(G_VET + k) * T + idx];
        fwd[k] = vet > 0.0;
        beta[k] = vet / R->S[k];
    }
    for (int gf = 0; gf < NGF; gf++) {
        const double* f = &gfs[gf * T + idx];
        double v = f[0], d1[3], d2[3][3], up[3];
        for (int k = 0; k < 3; k++) {
            if (p->NG == 3) {
                d1[k] = orc_d1(f, st[k], h[k]);
                up[k] = orc_dup(f, st[k], h[k], fwd[k]);
                for (int l = 0; l < 3; l++)
                    d2[k][l] = (k == l) ? orc_d2(f, st[k], h[k]) : orc_d11(f, st[k], st[l], h[k], h[l]);
                continue;
            }
            int m = Wd->m;
            d1[k] = sten(f, st[k], Wd->d1, -m, m) / (Wd->den1 * h[k]);
            /* the backward stencil is the mirror image: weight -w(-o) at offset o */
            up[k] = (fwd[k] ? sten(f, st[k], Wd->up, -(m - 1), m + 1) : -sten(f, -st[k], Wd->up, -(m - 1), m + 1)) /
                    (Wd->denu * h[k]);
            for (int l = 0; l < 3; l++) {
                if (k == l) {
                    d2[k][l] = sten(f, st[k], Wd->d2, -m, m) / (Wd->den2 * h[k] * h[k]);
                } else {
                    double s2 = 0.0;
                    for (int b = -m; b <= m; b++) s2 += Wd->d1[b + m] * sten(f + b * st[l], st[k], Wd->d1, -m, m);
                    d2[k][l] = s2 / (Wd->den1 * Wd->den1 * h[k] * h[l]);
                }
            }
        }
        double Rv, Rd[3], Rdd[3][3];
        rescale_factor(R, gf_type(gf), &Rv, Rd, Rdd);
        X[gf] = Rv * v;
        adv[gf] = 0.0;
        for (int k = 0; k < 3; k++) {
            dX[gf][k] = Rd[k] * v + Rv * d1[k];
            for (int l = 0; l < 3; l++)
                ddX[gf][k][l] = Rdd[k][l] * v + Rd[k] * d1[l] + Rd[l] * d1[k] + Rv * d2[k][l];
            adv[gf] += beta[k] * (Rd[k] * v + Rv * up[k]);
        }
    }
    memset(F, 0, sizeof *F);
    for (int s = 0; s < 6; s++) {
        int i = SYM_I[s], j = SYM_J[s];
        for (int sym = 0; sym < 2; sym++) {
            int a = sym ? j : i, b = sym ? i : j;
            F->eps[a][b] = X[G_HDD + s];
            F->adv_eps[a][b] = adv[G_HDD + s];
            F->A[a][b] = X[G_ADD + s];
            F->adv_A[a][b] = adv[G_ADD + s];
            for (int k = 0; k < 3; k++) {
                F->dA[a][b][k] = dX[G_ADD + s][k];
                F->deps[a][b][k] = dX[G_HDD + s][k];
                for (int l = 0; l < 3; l++) F->ddeps[a][b][k][l] = ddX[G_HDD + s][k][l];
            }
        }
    }
    F->W = X[G_CF];
    F->adv_W = adv[G_CF];
    F->K = X[G_TRK];
    F->adv_K = adv[G_TRK];
    F->alpha = X[G_ALPHA];
    F->adv_alpha = adv[G_ALPHA];
    for (int k = 0; k < 3; k++) {
        F->dW[k] = dX[G_CF][k];
        F->dK[k] = dX[G_TRK][k];
        F->dalpha[k] = dX[G_ALPHA][k];
        for (int l = 0; l < 3; l++) {
            F->ddW[k][l] = ddX[G_CF][k][l];
            F->ddalpha[k][l] = ddX[G_ALPHA][k][l];
        }
    }
    for (int i = 0; i < 3; i++) {
        F->Lam[i] = X[G_LAM + i];
        F->adv_Lam[i] = adv[G_LAM + i];
        F->beta[i] = X[G_VET + i];
        F->adv_beta[i] = adv[G_VET + i];
        F->B[i] = X[G_BET + i];
        F->adv_B[i] = adv[G_BET + i];
        for (int k = 0; k < 3; k++) {
            F->dLam[i][k] = dX[G_LAM + i][k];
            F->dbeta[i][k] = dX[G_VET + i][k];
            for (int l = 0; l < 3; l++) F->ddbeta[i][k][l] = ddX[G_VET + i][k][l];
        }
    }
}

/* Geometric quantities shared by the RHS and the Hamiltonian constraint. */
typedef struct {
    double gb[3][3], gbinv[3][3];
    double Deps[3][3][3];      /* Dhat_k eps_ij = Deps[i][j][k] */
    double dDeps[3][3][3][3];  /* d_l (Dhat_k eps_ij) = dDeps[i][j][k][l] */
    double Dl[3][3][3];        /* Delta_lij (first index lowered with gammabar) */
    double Dup[3][3][3];       /* Delta^k_ij = Dup[k][i][j] */
    double Dvec[3];            /* Delta^k */
    double Gb[3][3][3];        /* Gammabar^k_ij */
    double Ric[3][3];          /* Rbar_ij */
    double dphi[3], DDphi[3][3];
    double Aud[3][3], Auu[3][3], trA, AA;
} geom_pt;

static void geometry(const refmet* M, const pt_fields* F, geom_pt* G)
{
    memset(G, 0, sizeof *G);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) G->gb[i][j] = M->g[i][j] + F->eps[i][j];
    inv3(G->gb, G->gbinv);
    /* Dhat_k eps_ij and its partial derivative */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) {
                double s = F->deps[i][j][k];
                for (int m = 0; m < 3; m++) s -= M->Gam[m][k][i] * F->eps[m][j] + M->Gam[m][k][j] * F->eps[i][m];
                G->Deps[i][j][k] = s;
                for (int l = 0; l < 3; l++) {
                    double t = F->ddeps[i][j][k][l];
                    for (int m = 0; m < 3; m++)
                        t -= M->dGam[m][k][i][l] * F->eps[m][j] + M->Gam[m][k][i] * F->deps[m][j][l] +
                             M->dGam[m][k][j][l] * F->eps[i][m] + M->Gam[m][k][j] * F->deps[i][m][l];
                    G->dDeps[i][j][k][l] = t;
                }
            }
    /* Delta_lij = 1/2 (Dhat_i eps_jl + Dhat_j eps_il - Dhat_l eps_ij), Delta^k_ij, Delta^k */
    for (int l = 0; l < 3; l++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                G->Dl[l][i][j] = 0.5 * (G->Deps[j][l][i] + G->Deps[i][l][j] - G->Deps[i][j][l]);
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double s = 0.0;
                for (int l = 0; l < 3; l++) s += G->gbinv[k][l] * G->Dl[l][i][j];
                G->Dup[k][i][j] = s;
                G->Gb[k][i][j] = M->Gam[k][i][j] + s;
            }
    for (int k = 0; k < 3; k++) {
        double s = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) s += G->gbinv[i][j] * G->Dup[k][i][j];
        G->Dvec[k] = s;
    }
    /* Ricci tensor: Dhat_l Dhat_k eps_ij, then the four groups of terms */
    double DDeps[3][3][3][3], DLam[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double s = G->dDeps[i][j][k][l];
                    for (int m = 0; m < 3; m++)
                        s -= M->Gam[m][l][k] * G->Deps[i][j][m] + M->Gam[m][l][i] * G->Deps[m][j][k] +
                             M->Gam[m][l][j] * G->Deps[i][m][k];
                    DDeps[i][j][k][l] = s;
                }
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++) {
            double s = F->dLam[k][j];
            for (int m = 0; m < 3; m++) s += M->Gam[k][j][m] * F->Lam[m];
            DLam[k][j] = s; /* Dhat_j Lambda^k */
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double r1 = 0.0, r2 = 0.0, r3 = 0.0, r4 = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) r1 += G->gbinv[k][l] * DDeps[i][j][k][l];
            for (int k = 0; k < 3; k++) r2 += G->gb[k][i] * DLam[k][j] + G->gb[k][j] * DLam[k][i];
            for (int k = 0; k < 3; k++) r3 += G->Dvec[k] * 0.5 * (G->Dl[i][j][k] + G->Dl[j][i][k]);
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) {
                    double s = 0.0;
                    for (int m = 0; m < 3; m++)
                        s += G->Dup[m][k][i] * G->Dl[j][m][l] + G->Dup[m][k][j] * G->Dl[i][m][l] +
                             G->Dup[m][i][k] * G->Dl[m][j][l];
                    r4 += G->gbinv[k][l] * s;
                }
            G->Ric[i][j] = -0.5 * r1 + 0.5 * r2 + r3 + r4;
        }
    /* conformal factor: W = exp(-2 phi) */
    for (int i = 0; i < 3; i++) G->dphi[i] = -F->dW[i] / (2.0 * F->W);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double ddphi = -F->ddW[i][j] / (2.0 * F->W) + F->dW[i] * F->dW[j] / (2.0 * F->W * F->W);
            double s = ddphi;
            for (int k = 0; k < 3; k++) s -= G->Gb[k][i][j] * G->dphi[k];
            G->DDphi[i][j] = s;
        }
    /* Abar with raised indices */
    for (int k = 0; k < 3; k++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int l = 0; l < 3; l++) s += G->gbinv[k][l] * F->A[l][j];
            G->Aud[k][j] = s;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) s += G->gbinv[i][k] * G->gbinv[j][l] * F->A[k][l];
            G->Auu[i][j] = s;
        }
    G->trA = 0.0;
    G->AA = 0.0;
    for (int k = 0; k < 3; k++) G->trA += G->Aud[k][k];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) G->AA += F->A[i][j] * G->Auu[i][j];
}

/* BSSN right-hand sides in the coordinate basis (Sec. 2.1), then rescaled. */
static void rhs_at_point(const orc_params* p, const rfm_pt* R, const refmet* M, const pt_fields* F,
                         double out[NGF])
{
    geom_pt G;
    geometry(M, F, &G);
    const double al = F->alpha, W = F->W, K = F->K;
    const double W2 = W * W; /* exp(-4 phi) */

    /* shift: Dhat_k beta^i, d_l Dhat_k beta^i, Dhat_l Dhat_k beta^i */
    double Db[3][3], dDb[3][3][3], DDb[3][3][3];
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) {
            double s = F->dbeta[i][k];
            for (int m = 0; m < 3; m++) s += M->Gam[i][k][m] * F->beta[m];
            Db[i][k] = s;
            for (int l = 0; l < 3; l++) {
                double t = F->ddbeta[i][k][l];
                for (int m = 0; m < 3; m++) t += M->dGam[i][k][m][l] * F->beta[m] + M->Gam[i][k][m] * F->dbeta[m][l];
                dDb[i][k][l] = t;
            }
        }
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++)
            for (int l = 0; l < 3; l++) {
                double s = dDb[i][k][l];
                for (int m = 0; m < 3; m++) s += M->Gam[i][l][m] * Db[m][k] - M->Gam[m][l][k] * Db[i][m];
                DDb[i][k][l] = s;
            }
    /* Dbar_k beta^k = Dhat_k beta^k + Delta^k_km beta^m, with
     * Delta^k_km = 1/2 gammabar^{ab} Dhat_m eps_ab, and its gradient */
    double dgb[3][3][3], dgbinv[3][3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) dgb[i][j][k] = M->dg[i][j][k] + F->deps[i][j][k];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int k = 0; k < 3; k++) {
                double s = 0.0;
                for (int c = 0; c < 3; c++)
                    for (int d = 0; d < 3; d++) s += G.gbinv[a][c] * dgb[c][d][k] * G.gbinv[d][b];
                dgbinv[a][b][k] = -s;
            }
    double Dtr[3], dDtr[3][3];
    for (int m = 0; m < 3; m++) {
        double s = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s += G.gbinv[a][b] * G.Deps[a][b][m];
        Dtr[m] = 0.5 * s;
        for (int l = 0; l < 3; l++) {
            double t = 0.0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) t += dgbinv[a][b][l] * G.Deps[a][b][m] + G.gbinv[a][b] * G.dDeps[a][b][m][l];
            dDtr[m][l] = 0.5 * t;
        }
    }
    double divbar = 0.0, d_divbar[3];
    for (int k = 0; k < 3; k++) divbar += Db[k][k];
    for (int m = 0; m < 3; m++) divbar += Dtr[m] * F->beta[m];
    for (int l = 0; l < 3; l++) {
        double s = 0.0;
        for (int k = 0; k < 3; k++) s += dDb[k][k][l];
        for (int m = 0; m < 3; m++) s += dDtr[m][l] * F->beta[m] + Dtr[m] * F->dbeta[m][l];
        d_divbar[l] = s;
    }
    double DDal[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = F->ddalpha[i][j];
            for (int k = 0; k < 3; k++) s -= G.Gb[k][i][j] * F->dalpha[k];
            DDal[i][j] = s;
        }

    double r_eps[3][3], r_A[3][3], r_Lam[3], r_beta[3], r_B[3];
    /* Eq. metric_RHS_orig_final + L_beta eps_ij */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = F->adv_eps[i][j];
            for (int k = 0; k < 3; k++) t += F->eps[k][j] * F->dbeta[k][i] + F->eps[i][k] * F->dbeta[k][j];
            t += (2.0 / 3.0) * G.gb[i][j] * (al * G.trA - divbar);
            for (int k = 0; k < 3; k++) t += M->g[j][k] * Db[k][i] + M->g[i][k] * Db[k][j];
            t -= 2.0 * al * F->A[i][j];
            r_eps[i][j] = t;
        }
    /* Eq. Abar_RHS_orig_final + L_beta Abar_ij */
    double X[3][3], trX = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            X[i][j] = -2.0 * al * G.DDphi[i][j] + 4.0 * al * G.dphi[i] * G.dphi[j] +
                      2.0 * (F->dalpha[i] * G.dphi[j] + F->dalpha[j] * G.dphi[i]) - DDal[i][j] + al * G.Ric[i][j];
    for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++) trX += G.gbinv[k][l] * X[k][l];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = F->adv_A[i][j];
            for (int k = 0; k < 3; k++) t += F->A[k][j] * F->dbeta[k][i] + F->A[i][k] * F->dbeta[k][j];
            t -= (2.0 / 3.0) * F->A[i][j] * divbar;
            double AA_ij = 0.0;
            for (int k = 0; k < 3; k++) AA_ij += F->A[i][k] * G.Aud[k][j];
            t -= 2.0 * al * AA_ij;
            t += al * F->A[i][j] * K;
            t += W2 * (X[i][j] - (1.0 / 3.0) * G.gb[i][j] * trX);
            r_A[i][j] = t;
        }
    /* Eq. W_RHS_orig_final + beta^k d_k W */
    double r_W = F->adv_W - (1.0 / 3.0) * W * (divbar - al * K);
    /* Eq. K_RHS_orig_final + beta^k d_k K */
    double lapl_al = 0.0, grad_ap = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            lapl_al += G.gbinv[i][j] * DDal[i][j];
            grad_ap += G.gbinv[i][j] * F->dalpha[i] * G.dphi[j];
        }
    double r_K = F->adv_K + (1.0 / 3.0) * al * K * K + al * G.AA - W2 * (lapl_al + 2.0 * grad_ap);
    /* Eq. Lambda_RHS_orig_final (reading R-Lambda): d_perp Lambda^i, then + L_beta Lambda^i */
    double r_Lam_perp[3];
    for (int i = 0; i < 3; i++) {
        double t = 0.0;
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) t += G.gbinv[j][k] * DDb[i][j][k];
        t += (2.0 / 3.0) * G.Dvec[i] * divbar;
        for (int k = 0; k < 3; k++) t += (1.0 / 3.0) * G.gbinv[i][k] * d_divbar[k];
        for (int j = 0; j < 3; j++) t -= 2.0 * G.Auu[i][j] * (F->dalpha[j] - 6.0 * al * G.dphi[j]);
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < 3; k++) t += 2.0 * al * G.Auu[j][k] * G.Dup[i][j][k];
        for (int j = 0; j < 3; j++) t -= (4.0 / 3.0) * al * G.gbinv[i][j] * F->dK[j];
        r_Lam_perp[i] = t;
        double lie = F->adv_Lam[i];
        for (int j = 0; j < 3; j++) lie -= F->Lam[j] * F->dbeta[i][j];
        r_Lam[i] = lie + t;
    }
    /* Eqs. gauge_eqns, damping_eta_final */
    double r_al = -2.0 * al * K + F->adv_alpha;
    for (int i = 0; i < 3; i++) {
        r_beta[i] = F->B[i] + F->adv_beta[i];
        r_B[i] = 0.75 * r_Lam_perp[i] - p->eta * F->B[i] + F->adv_B[i];
    }
    /* back to rescaled gridfunctions (S is time independent) */
    for (int s = 0; s < 6; s++) {
        int i = SYM_I[s], j = SYM_J[s];
        out[G_HDD + s] = r_eps[i][j] / (R->S[i] * R->S[j]);
        out[G_ADD + s] = r_A[i][j] / (R->S[i] * R->S[j]);
    }
    out[G_CF] = r_W;
    out[G_TRK] = r_K;
    for (int i = 0; i < 3; i++) {
        out[G_LAM + i] = R->S[i] * r_Lam[i];
        out[G_VET + i] = R->S[i] * r_beta[i];
        out[G_BET + i] = R->S[i] * r_B[i];
    }
    out[G_ALPHA] = r_al;
}

/* ----------------------------------------------------------------- RHS */

void orc_rhs(const orc_params* p, const double* gfs, double* rhs, int k_lo, int k_hi)
{
    int n[3];
    long T = orc_sizes(p, n);
    int NG = p->NG;
    long st[3] = {1, n[0], (long)n[0] * n[1]};
    double h[3] = {dxx_of(p, 0), dxx_of(p, 1), dxx_of(p, 2)};
    if (k_lo < 0) k_lo = 0;
    if (k_hi > p->N[2]) k_hi = p->N[2];
    fdw Wd;
    fdw_make(p->NG, &Wd);
    int nt = p->nthreads;
#ifdef _OPENMP
    if (nt <= 0) nt = omp_get_max_threads();
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
#endif
    for (int k = k_lo; k < k_hi; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                int ii[3] = {i + NG, j + NG, k + NG};
                long idx = ii[0] + (long)n[0] * (ii[1] + (long)n[1] * ii[2]);
                double xx[3] = {orc_xx(p, 0, ii[0]), orc_xx(p, 1, ii[1]), orc_xx(p, 2, ii[2])};
                rfm_pt R;
                refmet M;
                pt_fields F;
                double out[NGF];
                rfm_eval(p, xx, &R);
                refmet_from(&R, &M);
                load_point(p, n, T, gfs, idx, &R, &F, &Wd);
                rhs_at_point(p, &R, &M, &F, out);
                /* Kreiss-Oliger dissipation (reading R-KO): sigma / (2^(2r) S_d dxx_d) times the
                 * difference of order 2r = N_FD + 2 along each axis, physical spacing S_d dxx_d */
                for (int gf = 0; gf < NGF; gf++) {
                    double ko = 0.0;
                    for (int d = 0; d < 3; d++) {
                        const double* f = &gfs[gf * T + idx];
                        if (p->NG == 3) {
                            ko += p->ko_sigma[gf] / (64.0 * h[d] * R.S[d]) * orc_ko6(f, st[d]);
                        } else {
                            int r = Wd.m + 1;
                            ko += p->ko_sigma[gf] / (ldexp(1.0, 2 * r) * h[d] * R.S[d]) * sten(f, st[d], Wd.ko, -r, r);
                        }
                    }
                    rhs[gf * T + idx] = out[gf] + ko;
                }
            }
    (void)nt;
}

static int full_rhs_with(const orc_params* p, const bmap* m, const double* gfs, double* rhs)
{
    orc_rhs(p, gfs, rhs, 0, p->N[2]);
    outer_bc_with(p, m, gfs, rhs); /* 1. outer boundary (Sec. 3 ordering) */
    inner_bc_with(m, rhs, team_of(p)); /* 2. inner boundary, sources may be outer ghosts */
    return 0;
}

int orc_full_rhs(const orc_params* p, const double* gfs, double* rhs)
{
    bmap m;
    int bad = bmap_make(p, &m);
    full_rhs_with(p, &m, gfs, rhs);
    bmap_free(&m);
    return bad;
}

/* det(gammabar_ij)/det(gammahat_ij) = det(delta_ij + h_ij) := 1 (the
 * Lagrangian choice of Sec. 2.1), by rescaling gammabar_ij = delta_ij + h_ij
 * with det^(-1/3).  Written in terms of the deviation h so that small h keeps
 * its relative precision: det(I + h) - 1 = e1 + e2 + e3 with the invariants
 * e1 = tr h, e2 = ((tr h)^2 - tr(h^2))/2, e3 = det h, the factor minus one is
 * f1 = expm1(-log1p(det - 1)/3), and h_ij <- h_ij + f1 (delta_ij + h_ij). */
void orc_enforce_detgb(const orc_params* p, double* gfs)
{
    long T = orc_sizes(p, NULL);
    const int nt = team_of(p);
    ORC_PARALLEL_FOR
    for (long idx = 0; idx < T; idx++) {
        double h[3][3], inv[3][3];
        for (int s = 0; s < 6; s++) {
            double v = gfs[(G_HDD + s) * T + idx];
            h[SYM_I[s]][SYM_J[s]] = v;
            h[SYM_J[s]][SYM_I[s]] = v;
        }
        double e1 = 0.0, trh2 = 0.0;
        for (int i = 0; i < 3; i++) {
            e1 += h[i][i];
            for (int j = 0; j < 3; j++) trh2 += h[i][j] * h[j][i];
        }
        double e2 = 0.5 * (e1 * e1 - trh2);
        double e3 = inv3(h, inv);
        double f1 = expm1(-log1p(e1 + e2 + e3) / 3.0);
        for (int s = 0; s < 6; s++) {
            double delta = SYM_I[s] == SYM_J[s] ? 1.0 : 0.0;
            double v = gfs[(G_HDD + s) * T + idx];
            gfs[(G_HDD + s) * T + idx] = v + f1 * (delta + v);
        }
    }
}

/* ------------------------------------------------------------------ RK4 */

/* classic RK4 (Sec. 4.2.1 footnote: the performance runs use RK4) */
/* SSPRK3 (Gottlieb, Shu & Tadmor 2001; named in Sec. 3 and Sec. 4.1):
 *   y1 = y + dt f(y),  y2 = 3/4 y + 1/4 (y1 + dt f(y1)),  y' = 1/3 y + 2/3 (y2 + dt f(y2)),
 * boundary conditions on each right-hand side, det(gammabar) enforced after each
 * substage update. */
int orc_ssprk3_step(const orc_params* p, double* gfs, double dt, int nsteps)
{
    bmap m;
    int bad = bmap_make(p, &m);
    const int nt = team_of(p);
    long n = (long)NGF * m.T;
    double* k = (double*)malloc(sizeof(double) * n);
    double* y1 = (double*)malloc(sizeof(double) * n);
    double* y2 = (double*)malloc(sizeof(double) * n);
    for (int step = 0; step < nsteps; step++) {
        full_rhs_with(p, &m, gfs, k);
        ORC_PARALLEL_FOR
        for (long i = 0; i < n; i++) y1[i] = gfs[i] + dt * k[i];
        if (p->enforce_detgb) orc_enforce_detgb(p, y1);
        full_rhs_with(p, &m, y1, k);
        ORC_PARALLEL_FOR
        for (long i = 0; i < n; i++) y2[i] = 0.75 * gfs[i] + 0.25 * (y1[i] + dt * k[i]);
        if (p->enforce_detgb) orc_enforce_detgb(p, y2);
        full_rhs_with(p, &m, y2, k);
        ORC_PARALLEL_FOR
        for (long i = 0; i < n; i++) gfs[i] = (1.0 / 3.0) * gfs[i] + (2.0 / 3.0) * (y2[i] + dt * k[i]);
        if (p->enforce_detgb) orc_enforce_detgb(p, gfs);
    }
    free(k);
    free(y1);
    free(y2);
    bmap_free(&m);
    return bad;
}

void orc_ssprk3_generic(long n, double* y, double dt, orc_rhs_fn f, void* ctx)
{
    double* k = (double*)malloc(sizeof(double) * n);
    double* y1 = (double*)malloc(sizeof(double) * n);
    double* y2 = (double*)malloc(sizeof(double) * n);
    f(ctx, y, k);
    for (long i = 0; i < n; i++) y1[i] = y[i] + dt * k[i];
    f(ctx, y1, k);
    for (long i = 0; i < n; i++) y2[i] = 0.75 * y[i] + 0.25 * (y1[i] + dt * k[i]);
    f(ctx, y2, k);
    for (long i = 0; i < n; i++) y[i] = (1.0 / 3.0) * y[i] + (2.0 / 3.0) * (y2[i] + dt * k[i]);
    free(k);
    free(y1);
    free(y2);
}

void orc_rk4_generic(long n, double* y, double dt, orc_rhs_fn f, void* ctx)
{
    double* k1 = (double*)malloc(sizeof(double) * n);
    double* k2 = (double*)malloc(sizeof(double) * n);
    double* k3 = (double*)malloc(sizeof(double) * n);
    double* k4 = (double*)malloc(sizeof(double) * n);
    double* yt = (double*)malloc(sizeof(double) * n);
    f(ctx, y, k1);
    for (long i = 0; i < n; i++) yt[i] = y[i] + 0.5 * dt * k1[i];
    f(ctx, yt, k2);
    for (long i = 0; i < n; i++) yt[i] = y[i] + 0.5 * dt * k2[i];
    f(ctx, yt, k3);
    for (long i = 0; i < n; i++) yt[i] = y[i] + dt * k3[i];
    f(ctx, yt, k4);
    for (long i = 0; i < n; i++) y[i] = y[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    free(k1);
    free(k2);
    free(k3);
    free(k4);
    free(yt);
}

int orc_rk4_step(const orc_params* p, double* gfs, double dt, int nsteps)
{
    bmap m;
    int bad = bmap_make(p, &m);
    const int nt = team_of(p);
    long n = (long)NGF * m.T;
    double* k[4];
    double* yt = (double*)malloc(sizeof(double) * n);
    for (int s = 0; s < 4; s++) k[s] = (double*)malloc(sizeof(double) * n);
    static const double c[3] = {0.5, 0.5, 1.0};
    for (int step = 0; step < nsteps; step++) {
        const double* yin = gfs;
        for (int s = 0; s < 4; s++) {
            full_rhs_with(p, &m, yin, k[s]);
            if (s < 3) {
                ORC_PARALLEL_FOR
                for (long i = 0; i < n; i++) yt[i] = gfs[i] + c[s] * dt * k[s][i];
                if (p->enforce_detgb) orc_enforce_detgb(p, yt);
                yin = yt;
            }
        }
        ORC_PARALLEL_FOR
        for (long i = 0; i < n; i++) gfs[i] = gfs[i] + (dt / 6.0) * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
        if (p->enforce_detgb) orc_enforce_detgb(p, gfs);
    }
    for (int s = 0; s < 4; s++) free(k[s]);
    free(yt);
    bmap_free(&m);
    return bad;
}

/* ---------------------------------------------------------- Hamiltonian */

/* Eq. Hconstraint with Rbar = gammabar^{ij} Rbar_ij,
 * Dbar^i phi Dbar_i phi = gammabar^{ij} d_i phi d_j phi,
 * Dbar^2 phi = gammabar^{ij} (d_i d_j phi - Gammabar^k_ij d_k phi). */
void orc_hamiltonian(const orc_params* p, const double* gfs, double* H, double rmin, double rmax, double* l2,
                     double* linf, long* count)
{
    int n[3];
    long T = orc_sizes(p, n);
    int NG = p->NG;
    for (long idx = 0; idx < T; idx++) H[idx] = 0.0;
    fdw Wd;
    fdw_make(p->NG, &Wd);
    int nt = p->nthreads;
#ifdef _OPENMP
    if (nt <= 0) nt = omp_get_max_threads();
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
#endif
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                int ii[3] = {i + NG, j + NG, k + NG};
                long idx = ii[0] + (long)n[0] * (ii[1] + (long)n[1] * ii[2]);
                double xx[3] = {orc_xx(p, 0, ii[0]), orc_xx(p, 1, ii[1]), orc_xx(p, 2, ii[2])};
                rfm_pt R;
                refmet M;
                pt_fields F;
                geom_pt G;
                rfm_eval(p, xx, &R);
                refmet_from(&R, &M);
                load_point(p, n, T, gfs, idx, &R, &F, &Wd);
                geometry(&M, &F, &G);
                double Rs = 0.0, gp = 0.0, lp = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        Rs += G.gbinv[a][b] * G.Ric[a][b];
                        gp += G.gbinv[a][b] * G.dphi[a] * G.dphi[b];
                        lp += G.gbinv[a][b] * G.DDphi[a][b];
                    }
                H[idx] = (2.0 / 3.0) * F.K * F.K - G.AA + F.W * F.W * (Rs - 8.0 * gp - 8.0 * lp);
            }
    (void)nt;
    double s2 = 0.0, mx = 0.0;
    long cnt = 0;
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                long idx = (i + NG) + (long)n[0] * ((j + NG) + (long)n[1] * (k + NG));
                double x[3];
                orc_cart(p, idx, x);
                double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                if (r < rmin || r > rmax) continue;
                s2 += H[idx] * H[idx];
                if (fabs(H[idx]) > mx) mx = fabs(H[idx]);
                cnt++;
            }
    if (l2) *l2 = cnt ? sqrt(s2 / cnt) : 0.0;
    if (linf) *linf = mx;
    if (count) *count = cnt;
}

/* Eq. Mconstraint:
 *   M^i = e^{-4 phi} (Dhat_j Abar^{ij} + 2 Abar^{k(i} Delta^{j)}_{jk} + 6 Abar^{ij} d_j phi
 *                     - 2/3 gammabar^{ij} d_j K),
 * the symmetrisation taken over the free index i and the upper index j of
 * Delta^j_{jk} before the contraction: 2 Abar^{k(i} Delta^{j)}_{jk} =
 * Abar^{ki} Delta^j_{jk} + Abar^{kj} Delta^i_{jk}.  Dhat_j Abar^{ij} =
 * d_j Abar^{ij} + Gammahat^i_{jm} Abar^{mj} + Gammahat^j_{jm} Abar^{im}, with
 * d_j Abar^{ij} from the product rule on gammabar^{ik} gammabar^{jl} Abar_kl
 * and d gammabar^{-1} = -gammabar^{-1} (d gammabar) gammabar^{-1}.
 * Outputs (any may be NULL): M (3*T) the rescaled components S_i M^i at
 * interior points (ghosts 0), Mnorm (T) |M| = sqrt(gamma_ij M^i M^j) with the
 * physical metric gamma_ij = e^{4 phi} gammabar_ij, and the L2 / Linf norms of
 * |M| over interior points with Cartesian radius in [rmin, rmax]. */
void orc_momentum(const orc_params* p, const double* gfs, double* Mout, double* Mnorm, double rmin, double rmax,
                  double* l2, double* linf, long* count)
{
    int n[3];
    long T = orc_sizes(p, n);
    int NG = p->NG;
    double* mag = (double*)calloc((size_t)T, sizeof(double));
    if (Mout)
        for (long q = 0; q < 3 * T; q++) Mout[q] = 0.0;
    fdw Wd;
    fdw_make(p->NG, &Wd);
    int nt = p->nthreads;
#ifdef _OPENMP
    if (nt <= 0) nt = omp_get_max_threads();
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
#endif
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                int ii[3] = {i + NG, j + NG, k + NG};
                long idx = ii[0] + (long)n[0] * (ii[1] + (long)n[1] * ii[2]);
                double xx[3] = {orc_xx(p, 0, ii[0]), orc_xx(p, 1, ii[1]), orc_xx(p, 2, ii[2])};
                rfm_pt R;
                refmet M;
                pt_fields F;
                geom_pt G;
                rfm_eval(p, xx, &R);
                refmet_from(&R, &M);
                load_point(p, n, T, gfs, idx, &R, &F, &Wd);
                geometry(&M, &F, &G);
                /* d_m gammabar^{ab} */
                double dgi[3][3][3];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        for (int m = 0; m < 3; m++) {
                            double t = 0.0;
                            for (int c = 0; c < 3; c++)
                                for (int d = 0; d < 3; d++)
                                    t += G.gbinv[a][c] * (M.dg[c][d][m] + F.deps[c][d][m]) * G.gbinv[d][b];
                            dgi[a][b][m] = -t;
                        }
                double Mv[3];
                for (int a = 0; a < 3; a++) {
                    /* Dhat_j Abar^{aj} */
                    double div = 0.0;
                    for (int b = 0; b < 3; b++) {
                        double dAuu = 0.0; /* d_b Abar^{ab} */
                        for (int c = 0; c < 3; c++)
                            for (int d = 0; d < 3; d++)
                                dAuu += dgi[a][c][b] * G.gbinv[b][d] * F.A[c][d] +
                                        G.gbinv[a][c] * dgi[b][d][b] * F.A[c][d] +
                                        G.gbinv[a][c] * G.gbinv[b][d] * F.dA[c][d][b];
                        div += dAuu;
                        for (int m = 0; m < 3; m++)
                            div += M.Gam[a][b][m] * G.Auu[m][b] + M.Gam[b][b][m] * G.Auu[a][m];
                    }
                    /* Abar^{ka} Delta^j_{jk} + Abar^{kj} Delta^a_{jk} */
                    double dterm = 0.0;
                    for (int b = 0; b < 3; b++)
                        for (int c = 0; c < 3; c++)
                            dterm += G.Auu[c][a] * G.Dup[b][b][c] + G.Auu[c][b] * G.Dup[a][b][c];
                    double ph = 0.0, kk = 0.0;
                    for (int b = 0; b < 3; b++) {
                        ph += G.Auu[a][b] * G.dphi[b];
                        kk += G.gbinv[a][b] * F.dK[b];
                    }
                    Mv[a] = F.W * F.W * (div + dterm + 6.0 * ph - (2.0 / 3.0) * kk);
                }
                double q = 0.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) q += G.gb[a][b] * Mv[a] * Mv[b];
                mag[idx] = sqrt(q) / F.W;
                if (Mout)
                    for (int a = 0; a < 3; a++) Mout[a * T + idx] = Mv[a] * R.S[a];
            }
    (void)nt;
    double s2 = 0.0, mx = 0.0;
    long cnt = 0;
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                long idx = (i + NG) + (long)n[0] * ((j + NG) + (long)n[1] * (k + NG));
                double x[3];
                orc_cart(p, idx, x);
                double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                if (r < rmin || r > rmax) continue;
                s2 += mag[idx] * mag[idx];
                if (mag[idx] > mx) mx = mag[idx];
                cnt++;
            }
    if (Mnorm)
        for (long q = 0; q < T; q++) Mnorm[q] = mag[q];
    free(mag);
    if (l2) *l2 = cnt ? sqrt(s2 / cnt) : 0.0;
    if (linf) *linf = mx;
    if (count) *count = cnt;
}

/* ---------------------------------------------------------- Weyl scalar psi4 */
/* The paper decomposes the Weyl scalar psi4 into spin-weight -2 harmonics
 * (Sec. 4.1) without printing its definition; the oracle takes the textbook
 * 3+1 form (vacuum):
 *   E_ij = R_ij - K_ik K^k_j + K K_ij,   B_ij = eps_(i|^kl D_k K_l|j),
 *   psi4 = -(E_ij - i B_ij) mbar^i mbar^j,
 * with R_ij = Rbar_ij + R^phi_ij (Rbar_ij of the evolution equations),
 * R^phi_ij = -2 Dbar_i Dbar_j phi - 2 gammabar_ij Dbar^2 phi + 4 d_i phi d_j phi
 *            - 4 gammabar_ij |d phi|^2,
 * K_ij = e^{4 phi} (Abar_ij + gammabar_ij K / 3), eps^{mkl} = [mkl] / sqrt(det gamma)
 * in the (positively oriented) coordinate basis, and m = (u_theta + i u_phi)/sqrt 2
 * from Gram-Schmidt, in the physical metric, of the radial, theta and phi
 * directions of the point's Cartesian position.  For a linearised outgoing wave
 * this gives psi4 = d_t^2 h_+ - i d_t^2 h_x, h_+ = (h_thth - h_phph)/2, h_x = h_thph. */
static void weyl_point(const orc_params* p, const rfm_pt* R, const refmet* M, const pt_fields* F, double Et[3][3],
                       double Bt[3][3])
{
    geom_pt G;
    geometry(M, F, &G);
    const double W = F->W, iW2 = 1.0 / (W * W);
    double gam[3][3], gami[3][3], dgam[3][3][3], Kd[3][3], dK[3][3][3], Ric[3][3];
    double lap = 0.0, gp = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            lap += G.gbinv[a][b] * G.DDphi[a][b];
            gp += G.gbinv[a][b] * G.dphi[a] * G.dphi[b];
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            gam[i][j] = G.gb[i][j] * iW2;
            gami[i][j] = G.gbinv[i][j] * W * W;
            Kd[i][j] = (F->A[i][j] + G.gb[i][j] * F->K / 3.0) * iW2;
            Ric[i][j] = G.Ric[i][j] - 2.0 * G.DDphi[i][j] - 2.0 * G.gb[i][j] * lap + 4.0 * G.dphi[i] * G.dphi[j] -
                        4.0 * G.gb[i][j] * gp;
            for (int k = 0; k < 3; k++) {
                const double dgb = M->dg[i][j][k] + F->deps[i][j][k];
                dgam[i][j][k] = dgb * iW2 - 2.0 * G.gb[i][j] * iW2 / W * F->dW[k];
                dK[i][j][k] = (F->dA[i][j][k] + dgb * F->K / 3.0 + G.gb[i][j] * F->dK[k] / 3.0) * iW2 -
                              2.0 * (F->A[i][j] + G.gb[i][j] * F->K / 3.0) * iW2 / W * F->dW[k];
            }
        }
    (void)p;
    /* physical Christoffel symbols Gam[k][i][j] */
    double Gp[3][3][3];
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double t = 0.0;
                for (int l = 0; l < 3; l++) t += gami[k][l] * (dgam[j][l][i] + dgam[i][l][j] - dgam[i][j][l]);
                Gp[k][i][j] = 0.5 * t;
            }
    double DK[3][3][3]; /* DK[k][i][j] = D_k K_ij */
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double t = dK[i][j][k];
                for (int m = 0; m < 3; m++) t -= Gp[m][k][i] * Kd[m][j] + Gp[m][k][j] * Kd[i][m];
                DK[k][i][j] = t;
            }
    double E[3][3], Bm[3][3];
    const double sq = sqrt(det3(gam));
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double kk = 0.0;
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) kk += Kd[i][k] * gami[k][l] * Kd[l][j];
            E[i][j] = Ric[i][j] - kk + F->K * Kd[i][j];
            /* eps_i^{kl} D_k K_lj = gamma_im [mkl] / sqrt(gamma) D_k K_lj */
            double b = 0.0;
            for (int m = 0; m < 3; m++)
                for (int k = 0; k < 3; k++)
                    for (int l = 0; l < 3; l++) {
                        const int e = levi(m, k, l);
                        if (e) b += gam[i][m] * e * DK[k][l][j];
                    }
            Bm[i][j] = b / sq;
        }
    /* tetrad: Gram-Schmidt of the radial, theta, phi directions of the Cartesian position */
    double Jinv[3][3];
    inv3(R->J, Jinv);
    const double x = R->cart[0], y = R->cart[1], z = R->cart[2];
    const double rr = sqrt(x * x + y * y + z * z), th = acos(z / rr), ph = atan2(y, x);
    const double vc[3][3] = {{x / rr, y / rr, z / rr},
                             {cos(th) * cos(ph), cos(th) * sin(ph), -sin(th)},
                             {-sin(ph), cos(ph), 0.0}};
    double u[3][3];
    for (int a = 0; a < 3; a++) {
        for (int d = 0; d < 3; d++) {
            double t = 0.0;
            for (int c = 0; c < 3; c++) t += Jinv[d][c] * vc[a][c];
            u[a][d] = t;
        }
        for (int b = 0; b < a; b++) {
            double dot = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) dot += gam[i][j] * u[a][i] * u[b][j];
            for (int d = 0; d < 3; d++) u[a][d] -= dot * u[b][d];
        }
        double nn = 0.0;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) nn += gam[i][j] * u[a][i] * u[a][j];
        for (int d = 0; d < 3; d++) u[a][d] /= sqrt(nn);
    }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double e = 0.0, bb = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    e += E[i][j] * u[a][i] * u[b][j];
                    bb += 0.5 * (Bm[i][j] + Bm[j][i]) * u[a][i] * u[b][j];
                }
            Et[a][b] = e;
            Bt[a][b] = bb;
        }
}

/* E and B in the tetrad (u_r, u_theta, u_phi) at interior points: Eout, Bout
 * (6*T each, symmetric pairs rr, rt, rp, tt, tp, pp; either may be NULL), and
 * psi4 (2*T: real, imaginary; may be NULL).  Ghost points are set to 0. */
void orc_psi4(const orc_params* p, const double* gfs, double* psi4, double* Eout, double* Bout)
{
    int n[3];
    long T = orc_sizes(p, n);
    int NG = p->NG;
    if (psi4)
        for (long q = 0; q < 2 * T; q++) psi4[q] = 0.0;
    if (Eout)
        for (long q = 0; q < 6 * T; q++) Eout[q] = 0.0;
    if (Bout)
        for (long q = 0; q < 6 * T; q++) Bout[q] = 0.0;
    fdw Wd;
    fdw_make(p->NG, &Wd);
    int nt = p->nthreads;
#ifdef _OPENMP
    if (nt <= 0) nt = omp_get_max_threads();
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
#endif
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                int ii[3] = {i + NG, j + NG, k + NG};
                long idx = ii[0] + (long)n[0] * (ii[1] + (long)n[1] * ii[2]);
                double xx[3] = {orc_xx(p, 0, ii[0]), orc_xx(p, 1, ii[1]), orc_xx(p, 2, ii[2])};
                rfm_pt R;
                refmet M;
                pt_fields F;
                rfm_eval(p, xx, &R);
                refmet_from(&R, &M);
                load_point(p, n, T, gfs, idx, &R, &F, &Wd);
                double Et[3][3], Bt[3][3];
                weyl_point(p, &R, &M, &F, Et, Bt);
                if (psi4) {
                    psi4[idx] = -0.5 * (Et[1][1] - Et[2][2]) + Bt[1][2];
                    psi4[T + idx] = Et[1][2] + 0.5 * (Bt[1][1] - Bt[2][2]);
                }
                for (int s = 0; s < 6; s++) {
                    if (Eout) Eout[s * T + idx] = Et[SYM_I[s]][SYM_J[s]];
                    if (Bout) Bout[s * T + idx] = Bt[SYM_I[s]][SYM_J[s]];
                }
            }
    (void)nt;
}

/* spin-weighted spherical harmonic sY_lm (Goldberg et al. 1967 closed form):
 * (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)] sin^{2l}(th/2)
 *   sum_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} e^{i m ph} cot^{2r+s-m}(th/2) */
static double fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; i++) r *= i;
    return r;
}
void orc_sylm(int s, int l, int m, double th, double ph, double* re, double* im)
{
    double pre = ((m % 2) ? -1.0 : 1.0) *
                 sqrt(fact(l + m) * fact(l - m) * (2 * l + 1) / (4.0 * M_PI * fact(l + s) * fact(l - s)));
    double sh = sin(0.5 * th), ch = cos(0.5 * th), sum = 0.0;
    for (int r = 0; r <= l - s; r++) {
        int k2 = r + s - m;
        if (k2 < 0 || k2 > l + s) continue;
        int pw = 2 * r + s - m; /* power of cot(th/2) = ch/sh; combined with sh^{2l}: ch^pw sh^{2l-pw} */
        double term = binom(l - s, r) * binom(l + s, k2) * (((l - r - s) % 2) ? -1.0 : 1.0);
        term *= pow(ch, pw) * pow(sh, 2 * l - pw);
        sum += term;
    }
    *re = pre * sum * cos(m * ph);
    *im = pre * sum * sin(m * ph);
}

/* Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n) */
static void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; i++) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Modes C_lm = integral of psi4 conj(-2Y_lm) over the sphere of radius Rext,
 * l = 2..lmax, m = -l..l in that order (2 doubles each: re, im).  psi4 (2*T)
 * holds the field at interior points; inner ghosts are filled here by the
 * parity map (psi4 is a scalar: the same physical point); the sphere must keep
 * two cells from the outer boundary.  Quadrature: ntheta Gauss-Legendre nodes
 * in cos(theta) times nphi uniform nodes in phi; psi4 at each node by cubic
 * Lagrange interpolation in the logical coordinates. */
int orc_psi4_modes(const orc_params* p, const double* psi4, double Rext, int ntheta, int nphi, int lmax, double* out)
{
    int n[3];
    long T = orc_sizes(p, n);
    bmap m;
    int bad = bmap_make(p, &m);
    double* f = (double*)malloc(sizeof(double) * 2 * T);
    memcpy(f, psi4, sizeof(double) * 2 * T);
    for (long idx = 0; idx < T; idx++)
        if (m.cls[idx] == 2) {
            f[idx] = f[m.src[idx]];
            f[T + idx] = f[T + m.src[idx]];
        }
    double lo[3], hi[3];
    domain(p, lo, hi);
    double* x = (double*)malloc(sizeof(double) * ntheta);
    double* w = (double*)malloc(sizeof(double) * ntheta);
    gauss_legendre(ntheta, x, w);
    int nm = 0;
    for (int l = 2; l <= lmax; l++) nm += 2 * l + 1;
    for (int q = 0; q < 2 * nm; q++) out[q] = 0.0;
    for (int it = 0; it < ntheta; it++)
        for (int jp = 0; jp < nphi; jp++) {
            const double th = acos(x[it]), ph = -M_PI + 2.0 * M_PI * (jp + 0.5) / nphi;
            const double c[3] = {Rext * sin(th) * cos(ph), Rext * sin(th) * sin(ph), Rext * cos(th)};
            double xx[3];
            cart_to_xx(p, c, xx);
            int base[3];
            double L[3][4];
            for (int d = 0; d < 3; d++) {
                double fi = (xx[d] - lo[d]) / dxx_of(p, d) + p->NG - 0.5;
                int i0 = (int)floor(fi);
                double t = fi - i0;
                base[d] = i0 - 1;
                L[d][0] = -t * (t - 1.0) * (t - 2.0) / 6.0;
                L[d][1] = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
                L[d][2] = -(t + 1.0) * t * (t - 2.0) / 2.0;
                L[d][3] = (t + 1.0) * t * (t - 1.0) / 6.0;
                if (base[d] < 0 || base[d] + 3 >= n[d]) bad = 1;
            }
            if (bad) continue;
            double vr = 0.0, vi = 0.0;
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++)
                    for (int cc = 0; cc < 4; cc++) {
                        long idx = (base[0] + a) + (long)n[0] * ((base[1] + b) + (long)n[1] * (base[2] + cc));
                        double wt = L[0][a] * L[1][b] * L[2][cc];
                        vr += wt * f[idx];
                        vi += wt * f[T + idx];
                    }
            const double dw = w[it] * 2.0 * M_PI / nphi;
            int q = 0;
            for (int l = 2; l <= lmax; l++)
                for (int mm = -l; mm <= l; mm++, q++) {
                    double yr, yi;
                    orc_sylm(-2, l, mm, th, ph, &yr, &yi);
                    /* psi4 conj(Y) */
                    out[2 * q] += dw * (vr * yr + vi * yi);
                    out[2 * q + 1] += dw * (vi * yr - vr * yi);
                }
        }
    free(x);
    free(w);
    free(f);
    bmap_free(&m);
    return bad;
}

/* -------------------------------------------------------- initial data */

/* SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based hash: the
 * first output of a generator seeded with (seed ^ ctr). */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_splitmix_uniform(uint64_t seed, uint64_t ctr)
{
    uint64_t u = splitmix64(seed ^ ctr);
    return 2.0 * ((double)(u >> 11) * 0x1.0p-53) - 1.0;
}

/* Brill-Lindquist: psi = 1 + sum_n m_n / (2 |x - x_n|); gamma_ij = psi^4 delta_ij,
 * K_ij = 0, so gammabar = gammahat, W = psi^-2; lapse alpha = psi^-2, zero shift. */
int orc_brill_lindquist(const orc_params* p, int npunct, const double* mass, const double* xyz,
                        double perturb_amp, uint64_t seed, double* gfs)
{
    bmap m;
    int bad = bmap_make(p, &m);
    long T = m.T;
    memset(gfs, 0, sizeof(double) * NGF * T);
    for (long idx = 0; idx < T; idx++) {
        if (m.cls[idx] == 2) continue;
        double x[3];
        orc_cart(p, idx, x);
        double psi = 1.0;
        for (int q = 0; q < npunct; q++) {
            double dx = x[0] - xyz[3 * q], dy = x[1] - xyz[3 * q + 1], dz = x[2] - xyz[3 * q + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d < 1e-12) bad = 2;
            psi += mass[q] / (2.0 * d);
        }
        gfs[G_CF * T + idx] = 1.0 / (psi * psi);
        gfs[G_ALPHA * T + idx] = 1.0 / (psi * psi);
        if (perturb_amp != 0.0)
            for (int s = 0; s < 6; s++)
                gfs[(G_HDD + s) * T + idx] =
                    perturb_amp * orc_splitmix_uniform(seed, ((uint64_t)(G_HDD + s) << 40) | (uint64_t)idx);
    }
    inner_bc_with(&m, gfs, team_of(p));
    bmap_free(&m);
    return bad;
}

/* CFL: dt = cfl * min_{interior, d} |S_d| dxx_d */
double orc_dt(const orc_params* p)
{
    double mn = 1e300;
    int NG = p->NG;
    for (int k = 0; k < p->N[2]; k++)
        for (int j = 0; j < p->N[1]; j++)
            for (int i = 0; i < p->N[0]; i++) {
                double xx[3] = {orc_xx(p, 0, i + NG), orc_xx(p, 1, j + NG), orc_xx(p, 2, k + NG)};
                rfm_pt R;
                rfm_eval(p, xx, &R);
                for (int d = 0; d < 3; d++) {
                    double ds = fabs(R.S[d]) * dxx_of(p, d);
                    if (ds < mn) mn = ds;
                }
            }
    return p->cfl * mn;
}
