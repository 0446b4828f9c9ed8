/*
 * nr_oracle.h -- CPU reference oracle for the FP64 BSSN hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct C
 * implementation of the covariant BSSN system in the reference-metric
 * formalism (arXiv 2505.00097, Sec. 2.1 "Evolution equations", Eqs.
 * metric/Abar/W/K/Lambda RHS, Ricci tensor, gauge Eqs., Hamiltonian
 * constraint Eq. Hconstraint; Sec. 2.2 "Tensor rescaling"; Sec. 3 grid,
 * stencils and boundary classes; Sec. 4.2.1 RK4).  Only tests/, the
 * package smoke check and bench.py's CPU baseline may load it.  It shares
 * no code, header, table or helper with the CUDA library; the product path
 * never calls it.
 *
 * Layout of every 24-gridfunction set: gfs[gf*T + idx] with
 * idx = i0 + n0*(i1 + n1*i2), n_d = N_d + 2*NG, i0 fastest.
 * Gridfunction order: hDD00,hDD01,hDD02,hDD11,hDD12,hDD22,
 * aDD00..aDD22, cf(W), trK, lambdaU0..2, vetU0..2, betU0..2, alpha.
 */
#ifndef NR_ORACLE_H
#define NR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SINH_SPHERICAL = 0, ORC_SINH_CYLINDRICAL = 1, ORC_SPHERICAL = 2 };
enum { ORC_NGF = 24 };

typedef struct {
    int coords;          /* ORC_* */
    int N[3];            /* interior cells per axis */
    int NG;              /* ghost layers (3 for 4th-order FD + upwinding) */
    int enforce_detgb;   /* 1: rescale h so det(delta+h)=1 after every RK substage */
    double ampl[3];      /* sinh/plain map amplitude per axis (r_max, rho_max, -, z_max) */
    double sinhw[3];     /* sinh width per axis */
    double ko_sigma[24]; /* Kreiss-Oliger strength per gridfunction */
    double eta;          /* Gamma-driver damping */
    double cfl;          /* CFL factor */
    double wavespeed[24];/* Sommerfeld wave speed per gridfunction */
    double f_inf[24];    /* Sommerfeld asymptotic value per gridfunction */
    int nthreads;        /* OpenMP threads (<=0: runtime default) */
} orc_params;

/* sizes: padded n[3], total points; returns T */
long orc_sizes(const orc_params* p, int n_out[3]);
/* logical coordinate of padded index i along axis d */
double orc_xx(const orc_params* p, int d, int i);
/* Cartesian position of padded point idx (analytically continued coordinates) */
void orc_cart(const orc_params* p, long idx, double out[3]);
void orc_cart_all(const orc_params* p, double* out /* 3*T */);
/* Reference-metric data at logical point xx: ghat[3][3], dghat[3][3][3]
 * (dghat[i][j][k] = d_k ghat_ij), Gammahat[k][i][j], dGammahat[k][i][j][m]
 * (= d_m Gammahat^k_ij).  Any pointer may be NULL. */
void orc_refmetric(const orc_params* p, const double xx[3], double* S3, double* ghat,
                   double* dghat, double* ddghat, double* Gam, double* dGam);

/* Boundary maps.  cls: 0 interior, 1 pure outer ghost, 2 inner ghost.
 * src: flat source index (self for cls 0/1).  parity[10*idx+t]: sign for
 * tensor type t (0 scalar, 1..3 vector U0..U2, 4..9 DD00,01,02,11,12,22).
 * Return 0 on success, nonzero if some ghost has no source on the grid. */
int orc_build_map(const orc_params* p, int32_t* src, int8_t* parity, int32_t* cls);
int orc_build_map_bruteforce(const orc_params* p, int32_t* src, int8_t* parity, int32_t* cls);

/* CFL time step: cfl * min over interior points and axes of |S_d| dxx_d */
double orc_dt(const orc_params* p);

/* Brill-Lindquist data (+ seeded SplitMix64 perturbation of hDD), then inner BCs.
 * Returns nonzero if a canonical point lies within 1e-12 of a puncture. */
int orc_brill_lindquist(const orc_params* p, int npunct, const double* mass, const double* xyz,
                        double perturb_amp, uint64_t seed, double* gfs);

/* Interior RHS (+KO) for interior planes i2 in [k_lo, k_hi) (interior-relative).
 * Ghost points of rhs are not touched. */
void orc_rhs(const orc_params* p, const double* gfs, double* rhs, int k_lo, int k_hi);
/* Sommerfeld radiation RHS at pure-outer ghosts */
void orc_outer_bc(const orc_params* p, const double* gfs, double* rhs);
/* inner parity copies on any 24-gf set */
int orc_inner_bc(const orc_params* p, double* gfs);
/* full RHS: interior + outer + inner */
int orc_full_rhs(const orc_params* p, const double* gfs, double* rhs);
/* det(gammabar)=det(gammahat) enforcement at all points */
void orc_enforce_detgb(const orc_params* p, double* gfs);
/* nsteps of classic RK4 on the 24-gf state (all T points) */
int orc_rk4_step(const orc_params* p, double* gfs, double dt, int nsteps);
/* Hamiltonian constraint at interior points (ghosts set to 0); L2 (rms) and
 * Linf over interior points with Cartesian radius in [rmin, rmax]. */
void orc_hamiltonian(const orc_params* p, const double* gfs, double* H, double rmin, double rmax,
                     double* l2, double* linf, long* count);
/* Momentum constraint, Eq. Mconstraint (see nr_oracle.c): rescaled S_i M^i
 * (3*T, interior points; may be NULL), |M| with the physical metric (T; may be
 * NULL) and its L2 / Linf norms over the radius band [rmin, rmax]. */
void orc_momentum(const orc_params* p, const double* gfs, double* M, double* Mnorm, double rmin, double rmax,
                  double* l2, double* linf, long* count);
/* Weyl scalar psi4 (see nr_oracle.c) at interior points: psi4 (2*T: re, im),
 * E and B in the tetrad (6*T each: rr rt rp tt tp pp); any may be NULL */
void orc_psi4(const orc_params* p, const double* gfs, double* psi4, double* E, double* B);
/* spin-weighted spherical harmonic sY_lm(theta, phi) */
void orc_sylm(int s, int l, int m, double th, double ph, double* re, double* im);
/* modes of psi4 (2*T) on the sphere of radius Rext, l = 2..lmax, m = -l..l:
 * out[2q], out[2q+1] = re, im; nonzero return: a stencil left the grid */
int orc_psi4_modes(const orc_params* p, const double* psi4, double Rext, int ntheta, int nphi, int lmax, double* out);

/* Generic classic RK4 (used by orc_rk4_step; exported for its pin). */
typedef void (*orc_rhs_fn)(void* ctx, const double* y, double* k);
void orc_rk4_generic(long n, double* y, double dt, orc_rhs_fn f, void* ctx);
/* SSPRK3 (Gottlieb-Shu-Tadmor) on the 24 gridfunctions, as orc_rk4_step; and on a
 * plain vector for the pins */
int orc_ssprk3_step(const orc_params* p, double* gfs, double dt, int nsteps);
void orc_ssprk3_generic(long n, double* y, double dt, orc_rhs_fn f, void* ctx);
/* weights of the order-2(NG-1) stencils (NG != 3 paths): which 0 centred first
 * derivative, 1 centred second, 2 upwind forward (offsets -(NG-2)..NG), 3 the
 * Kreiss-Oliger difference of order 2 NG, 4 one-sided with window start a;
 * returns their number */
int orc_fd_weights(int NG, int which, int a, double* w);

/* Stencil helpers on a strided line (exported for their pins).  f points at
 * the centre value. */
double orc_d1(const double* f, long st, double h);
double orc_d2(const double* f, long st, double h);
double orc_d11(const double* f, long sa, long sb, double ha, double hb);
double orc_dup(const double* f, long st, double h, int forward);
double orc_ko6(const double* f, long st);
double orc_d1_onesided(const double* f, long st, double h, int kind);

/* SplitMix64 counter draw in [-1,1) used by the perturbation */
double orc_splitmix_uniform(uint64_t seed, uint64_t ctr);

#ifdef __cplusplus
}
#endif
#endif
