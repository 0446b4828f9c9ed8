/*
 * nr.h -- C ABI of the GB300 FP64 BSSN library (libnrgpu.so).
 *
 * The library evolves the BSSN equations in the reference-metric formalism
 * on one structured SinhSpherical, Spherical or SinhCylindrical grid per
 * nr_grid, as stated in arXiv 2505.00097:
 *   - Sec. 2.1: evolution equations (Eqs. metric_RHS_orig_final,
 *     Abar_RHS_orig_final, W_RHS_orig_final, K_RHS_orig_final,
 *     Lambda_RHS_orig_final), the conformal Ricci tensor, 1+log slicing and
 *     the Gamma-driver shift (Eqs. gauge_eqns, damping_eta_final), the
 *     Hamiltonian and momentum constraints (Eqs. Hconstraint, Mconstraint);
 *   - Sec. 2.2: tensor rescaling by the scale factors S_i;
 *   - Sec. 3: cell-centred logically rectangular grids, centred finite
 *     differences of order N_FD with upwinded shift advection and
 *     N_G = N_FD/2 + 1 ghost layers (N_FD = 4: N_G = 3; N_FD = 8: N_G = 5),
 *     outer (radiation) and inner (parity) boundary points, and the boundary
 *     order outer -> inner after every time-integrator substage;
 *   - Sec. 4.1: the sinh coordinate map x'(x) = x_max sinh(x/w)/sinh(1/w),
 *     Kreiss-Oliger dissipation, the CFL factor, the production scheme
 *     (8th order, SSPRK3) and the psi4 waveforms;
 *   - Sec. 4.2.1: method-of-lines RK4.
 *
 * Conventions (all entry points):
 *   - Return an nr_status; on failure nr_last_error() gives a thread-local
 *     message.  No entry point aborts the process.
 *   - A 24-gridfunction set is T*24 doubles laid out gfs[gf*T + idx],
 *     idx = i0 + n0*(i1 + n1*i2), n_d = N_d + 2*NG, i0 fastest.  Gridfunction
 *     order (rescaled components): hDD00,hDD01,hDD02,hDD11,hDD12,hDD22,
 *     aDD00..aDD22, cf (W), trK, lambdaU0..2, vetU0..2, betU0..2, alpha.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller (for
 *     example torch tensors); the library never frees them.  Buffers created
 *     by nr_grid_create are owned by the library and released by
 *     nr_grid_destroy.
 *   - Device work is issued on params.stream (a cudaStream_t, NULL for the
 *     legacy default stream) and is stream-ordered: an entry point returns
 *     after enqueueing, except where it says it synchronises.
 */
#ifndef NR_H
#define NR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NR_OK = 0,
    NR_EINVAL = 1,      /* bad argument (sizes, coordinates, null pointer, puncture on a grid point) */
    NR_ENOMEM = 2,      /* device allocation failed */
    NR_ECUDA = 3,       /* a CUDA runtime call failed */
    NR_ETIMEOUT = 4,    /* a bounded device wait gave up */
    NR_ENONFINITE = 5,  /* a NaN/Inf was found in the evolved state */
    NR_EMAP = 6         /* a ghost point has no source on the grid (e.g. odd N_phi) */
} nr_status;

typedef enum { NR_SINH_SPHERICAL = 0, NR_SINH_CYLINDRICAL = 1, NR_SPHERICAL = 2 } nr_coords;

enum { NR_NGF = 24 };

/* Grid and physics parameters.
 *   ampl/sinhw: per-axis map amplitude and sinh width (Sec. 4.1).
 *     SinhSpherical: r = ampl[0] sinh(xx0/sinhw[0])/sinh(1/sinhw[0]), xx0 in [0,1],
 *                    theta = xx1 in [0,pi], phi = xx2 in [-pi,pi].
 *     Spherical:     r = ampl[0] xx0.
 *     SinhCylindrical: rho from xx0 in [0,1] with ampl[0], sinhw[0];
 *                    phi = xx1 in [-pi,pi]; z from xx2 in [-1,1] with ampl[2], sinhw[2].
 *   ko_sigma: Kreiss-Oliger strength per gridfunction (Sec. 4.1); it must take
 *     one value on the 17 metric gridfunctions 0-16 (hDD, aDD, cf, trK,
 *     lambdaU) and one on the 7 gauge gridfunctions 17-23 (vetU, betU, alpha),
 *     as in the paper's runs (0.3 metric / 0.99 gauge); NR_EINVAL otherwise.
 *   eta: Gamma-driver damping; cfl: CFL factor.
 *   wavespeed, f_inf: radiation condition d_t f = -v [(x^j/r) d_j f + (f - f_inf)/r].
 *   h_rmin, h_rmax: radius band of the Hamiltonian-constraint norms.
 *   NG: ghost layers, N_G = N_FD/2 + 1 (Sec. 3): 3 selects the 4th-order
 *     scheme (6th-difference dissipation over 64 S dxx), 5 the 8th-order
 *     production scheme of Sec. 4.1 (10th-difference dissipation over
 *     1024 S dxx, 8th-order one-sided derivatives in the radiation condition);
 *     any other value is NR_EINVAL.
 *   enforce_detgb: rescale h so det(gammabar)=det(gammahat) after every RK
 *     substage (the Lagrangian choice of Sec. 2.1).
 *   integrator: the time integrator of a served request, NR_RK4 or NR_SSPRK3
 *     (NR_EINVAL otherwise); the single-grid and batch calls name theirs.
 *   stream: cudaStream_t used for all device work of the grid (NULL: legacy stream). */
typedef struct {
    double ampl[3];
    double sinhw[3];
    double ko_sigma[24];
    double eta;
    double cfl;
    double wavespeed[24];
    double f_inf[24];
    double h_rmin;
    double h_rmax;
    int NG;
    int enforce_detgb;
    int device;
    int integrator;
    void* stream;
} nr_params;

enum { NR_RK4 = 0, NR_SSPRK3 = 1 };

typedef struct nr_grid nr_grid;

typedef struct {
    int N[3];          /* interior cells */
    int n[3];          /* padded dimensions N + 2 NG */
    int64_t T;         /* points per gridfunction (padded) */
    int64_t interior;  /* N0 N1 N2 */
    int64_t n_outer;   /* pure outer ghost points (radiation condition) */
    int64_t n_inner;   /* inner ghost points (parity copies) */
    double dt_cfl;     /* cfl * min over interior points and axes of |S_d| dxx_d */
    size_t device_bytes; /* device memory held by the grid */
    int64_t n_inner_stencil; /* inner ghosts every RK stage copies (all, unless the azimuth holds
                                two points: then its ghosts are refreshed on demand, see nr_rk4_step) */
    int launches_per_step;   /* kernel launches of one nr_rk4_step (the on-demand ghost refresh
                                described at nr_rk4_step is one more, outside the step) */
    int launches_per_ssprk3_step; /* kernel launches of one nr_ssprk3_step */
    int64_t n_state_points;  /* interior + pure outer ghost points: the points of a compact state */
} nr_grid_info;

/* Defaults: ko_sigma 0.3, eta 2, cfl 0.5, wavespeed 1, f_inf 1 for W and alpha
 * (0 otherwise), NG 3, enforce_detgb 1, h band [0, inf), stream NULL, and
 * ampl/sinhw of 10/0.2 (spherical) or 300/0.2 (cylindrical). */
int nr_params_default(int coords, nr_params* out);

/* Create a grid: builds the per-axis reference-metric arrays, the boundary
 * maps and the CFL step on the host, uploads them and allocates the state
 * (y_n) and RK4 work sets (three more 24-gf sets) on params->device.
 * Nxx: interior cells per axis; N_phi must be even.  *out owned by the caller,
 * release with nr_grid_destroy.  Errors: NR_EINVAL, NR_EMAP, NR_ENOMEM, NR_ECUDA. */
int nr_grid_create(int coords, const int Nxx[3], const nr_params* params, nr_grid** out);
void nr_grid_destroy(nr_grid* grid);
int nr_query(const nr_grid* grid, nr_grid_info* info);

/* Brill-Lindquist puncture data on the grid-owned state (textbook closed form,
 * psi = 1 + sum_n m_n/(2|x - x_n|), gammabar = gammahat, W = alpha = psi^-2,
 * K = Abar = Lambdabar = beta = B = 0) at interior and outer points, an
 * optional SplitMix64 perturbation perturb_amp * U[-1,1) of the six hDD at
 * those points (counter (gf << 40) | idx, seed), then inner parity copies.
 * xyz: 3*npunct Cartesian positions (host).  NR_EINVAL if a grid point lies
 * within 1e-12 of a puncture (checked on the host). */
int nr_set_brill_lindquist(nr_grid* grid, int npunct, const double* mass, const double* xyz, double perturb_amp,
                           uint64_t seed);

/* Right-hand side of all 24 gridfunctions (Sec. 2.1 equations, upwinded
 * advection, Kreiss-Oliger dissipation) at interior points, from the
 * 24-gf set y_dev.  Its ghost points must be valid: outer ghosts set, inner
 * ghosts holding the parity copies (nr_apply_inner_bcs), as in every state
 * the RK4 driver produces.  Where the azimuth holds two points, its stencils
 * read the other azimuthal slice in place of the ghost copies of it.  Ghost points of rhs_dev
 * are not written.  y_dev and rhs_dev: caller-owned device buffers of 24*T
 * doubles, distinct. */
int nr_rhs(nr_grid* grid, const double* y_dev, double* rhs_dev);

/* Boundary conditions on a right-hand side (Sec. 3, outer then inner):
 * radiation condition at pure-outer ghosts computed from y_dev, then parity
 * copies rhs[ghost] = p * rhs[source] at inner ghosts. */
int nr_apply_bcs(nr_grid* grid, const double* y_dev, double* rhs_dev);

/* Inner parity copies on any caller-owned 24-gf device set (in place). */
int nr_apply_inner_bcs(nr_grid* grid, double* gfs_dev);

/* Advance the grid-owned state by nsteps classic RK4 steps of size dt (Sec.
 * 4.2.1): per substage, the interior RHS with the RK update fused into its
 * epilogue, the radiation condition at outer ghosts, parity copies at inner
 * ghosts, and (enforce_detgb) det(gammabar) enforcement.  The launches of
 * one step (nr_grid_info.launches_per_step) are captured once in a CUDA graph
 * (re-captured when dt changes) and replayed.  dt > 0, nsteps >= 0.
 * With a two-point azimuth the steps copy only the inner ghosts the stencils
 * read; the azimuthal ghost copies of the state are refreshed (one launch, on
 * params.stream) by the next call that returns or reads them: nr_get_state,
 * nr_check_finite, and nr_hamiltonian, nr_momentum, nr_psi4 and nr_psi4_modes
 * on the grid-owned state.  Results are the same as if every step had copied
 * them. */
int nr_rk4_step(nr_grid* grid, double dt, int nsteps);

/* nsteps steps of SSPRK3 (Gottlieb-Shu-Tadmor; the integrator of the paper's
 * production runs, Sec. 4.1) on the grid-owned state:
 *   y1 = y + dt k(y),  y2 = 3/4 y + 1/4 (y1 + dt k(y1)),
 *   y_{n+1} = 1/3 y + 2/3 (y2 + dt k(y2)),
 * each k with the boundary conditions of Sec. 3 and each stage followed by
 * det(gammabar) enforcement when enforce_detgb is set.  Three RHS evaluations
 * per step, captured in a CUDA graph like nr_rk4_step, with the same
 * on-demand refresh of azimuthal ghosts.  dt > 0, nsteps >= 0. */
int nr_ssprk3_step(nr_grid* grid, double dt, int nsteps);

/* Hamiltonian constraint (Eq. Hconstraint) at interior points of y_dev (NULL:
 * the grid-owned state).  H_dev (NULL allowed): caller-owned T doubles, ghost
 * points set to 0.  l2_out = sqrt(mean H^2), linf_out = max |H| over interior
 * points with Cartesian radius in [h_rmin, h_rmax]; either may be NULL.  The
 * norms are reduced on the device in a fixed order and copied to the host:
 * this call synchronises params.stream when l2_out or linf_out is given. */
int nr_hamiltonian(nr_grid* grid, const double* y_dev, double* H_dev, double* l2_out, double* linf_out);

/* Momentum constraint (Eq. Mconstraint) at interior points of y_dev (NULL:
 * the grid-owned state),
 *   M^i = e^{-4 phi} (Dhat_j Abar^ij + 2 Abar^k(i Delta^j)_jk + 6 Abar^ij d_j phi
 *                     - 2/3 gammabar^ij d_j K).
 * M_dev (NULL allowed): caller-owned 3*T doubles, the rescaled components
 * (S_i M^i, the layout of lambdaU) at interior points, ghost points set to 0.
 * l2_out / linf_out: sqrt(mean |M|^2) and max |M| over interior points with
 * Cartesian radius in [h_rmin, h_rmax], |M| = sqrt(gamma_ij M^i M^j) with the
 * physical metric gamma_ij = e^{4 phi} gammabar_ij; either may be NULL.
 * Reduced on the device in a fixed order; synchronises params.stream when a
 * norm is asked for. */
int nr_momentum(nr_grid* grid, const double* y_dev, double* M_dev, double* l2_out, double* linf_out);

/* Weyl scalar psi4 (the waveform of Sec. 4.1; the paper prints no formula):
 *   psi4 = -(E_ij - i B_ij) mbar^i mbar^j,  E_ij = R_ij - K_ik K^k_j + K K_ij,
 *   B_ij = eps_(i|^kl D_k K_l|j),  R_ij = Rbar_ij (as in the evolution) + R^phi_ij,
 * m = (u_theta + i u_phi)/sqrt 2, u from Gram-Schmidt in the physical metric of
 * the spherical directions of the point's Cartesian position; a linearised
 * outgoing wave gives psi4 = d_t^2 h_+ - i d_t^2 h_x.  At interior points of
 * y_dev (NULL: the grid-owned state) into psi4_dev (caller-owned 2*T doubles:
 * real part, imaginary part); inner ghosts take the value of the point they map
 * to (psi4 is a scalar), outer ghosts are 0.  Stream-ordered, no sync. */
int nr_psi4(nr_grid* grid, const double* y_dev, double* psi4_dev);

/* Spin-weight -2 modes C_lm = integral over the sphere of radius Rext of
 * psi4 conj(-2Y_lm), l = 2..lmax (lmax <= 16), m = -l..l in that order,
 * written to modes_out (host, 2 doubles per mode: re, im).  psi4 of y_dev (NULL:
 * the grid-owned state) is sampled at ntheta Gauss-Legendre nodes in cos(theta)
 * times nphi uniform nodes in phi by cubic Lagrange interpolation in the logical
 * coordinates.  NR_EINVAL if a node's stencil reaches the outer boundary or if
 * modes x nodes ((lmax+1)^2 - 4 times ntheta*nphi) exceeds 2^26.
 * Allocates its scratch and synchronises params.stream. */
int nr_psi4_modes(nr_grid* grid, const double* y_dev, double Rext, int ntheta, int nphi, int lmax, double* modes_out);

/* Copy the grid-owned state (24*T doubles) to / from dst / src.  to_host /
 * from_host = 1: dst/src is host memory (pinned or pageable) and the call
 * synchronises; 0: device memory, stream-ordered. */
int nr_get_state(nr_grid* grid, double* dst, int to_host);
int nr_set_state(nr_grid* grid, const double* src, int from_host);

/* Compact state: the 24 gridfunctions at the n_state_points canonical points only
 * (interior and pure outer ghosts, flat-index order; layout [gf][t], 24 *
 * n_state_points doubles).  Inner ghost points hold parity copies of canonical
 * points (Sec. 3), so the compact state determines the full one:
 * nr_set_state_compact scatters it and then applies the inner boundary
 * condition (its azimuthal copies on demand, as after nr_rk4_step), which
 * leaves the same state, bit for bit, as nr_set_state of the full array it
 * came from.  to_host / from_host = 1: host memory (pinned or
 * pageable), staged through a grid-owned device buffer allocated on first use
 * (NR_ENOMEM / NR_ECUDA if that fails); the call synchronises.  0: device
 * memory, stream-ordered. */
int nr_get_state_compact(nr_grid* grid, double* dst, int to_host);
int nr_set_state_compact(nr_grid* grid, const double* src, int from_host);

/* Host-resident stepping: nr_set_state_compact(host_in) (skipped if NULL), then
 * nsteps >= 1 steps of integrator (NR_RK4 or NR_SSPRK3) at dt, then the new
 * compact state into host_out (skipped if NULL); returns when host_out is
 * written.  Same results, bit for bit, as those calls one after another.
 * When host_out is pinned (page-locked, hence mapped) host memory, the last
 * stage of the last step stores each point's new values there itself, over the
 * host link while the stage computes, so the read-back costs no separate copy;
 * other host memory takes the gather-and-copy path.  The upload of host_in is
 * not waited for on its own: the steps follow it on the grid's stream, and the
 * call returns after that stream has drained, on an error too, so host_in may
 * be reused on return.  The first such call allocates a rank table of T ints
 * on the device.  Errors: NR_EINVAL, NR_ENOMEM, NR_ECUDA. */
int nr_step_io(nr_grid* grid, int integrator, double dt, int nsteps, const double* host_in, double* host_out);

/* 64-bit digest of a 24-gridfunction set (y_dev, or the grid-owned state if NULL) at
 * the canonical points -- interior and pure outer ghosts, which determine the whole
 * state since inner ghosts are parity copies (Sec. 3):
 *   sum modulo 2^64 over gridfunctions g and canonical flat indices idx of
 *   splitmix64(bits(y[g*T + idx]) XOR splitmix64((g << 40) | idx)),
 * splitmix64(x) being the first output of the SplitMix64 generator (Steele, Lea &
 * Flood 2014) with state x, bits() the IEEE-754 bit pattern.  The paper has no
 * counterpart: it is a service for bitwise comparisons of results (batched or
 * served runs against runs alone) without copying states to the host.  Each term
 * is a bijective mix of one value, so states that differ in one value always get
 * different digests, and states that differ in several collide with probability
 * about 2^-64.  Independent of the device and launch shape.  Synchronises
 * params.stream.  Errors: NR_EINVAL, NR_ECUDA. */
int nr_state_digest(nr_grid* grid, const double* y_dev, uint64_t* out);

/* Wait for all work of the grid's stream. */
int nr_sync(nr_grid* grid);

/* NaN/Inf guard: NR_ENONFINITE if alpha or W of the grid-owned state holds a
 * non-finite value (synchronises). */
int nr_check_finite(nr_grid* grid);

/* Host-only helpers (no GPU needed).
 * nr_build_maps: boundary maps of a grid, closed-form integer mirrors:
 *   cls[T]: 0 interior, 1 pure outer ghost, 2 inner ghost; src[T]: source flat
 *   index (self for cls 0/1); parity[10*T]: sign per tensor type (scalar,
 *   U0..U2, DD00,DD01,DD02,DD11,DD12,DD22).  Caller-owned host arrays.
 * nr_dt_cfl: the CFL step of a grid. */
int nr_build_maps(int coords, const int Nxx[3], int NG, int32_t* src, int8_t* parity, int32_t* cls);
int nr_dt_cfl(int coords, const int Nxx[3], const nr_params* params, double* dt_out);

/* Batched mode (the uneven-grid workload of the paper's single-node and
 * scaling tests run many times over): many grids of uneven sizes, all of one
 * coordinate family (spherical-like or cylindrical-like), one azimuth kind
 * (two points, or more: the right-hand-side kernel is specialised for a
 * two-point azimuth), one finite-difference order (NG), one device and one
 * stream, advanced together.  Each RK4 or SSPRK3 substage is one launch over
 * the work items of all grids -- a tile of one grid's interior points or a
 * chunk of its pure-outer ghost points, one thread block each -- followed by
 * one parity-copy launch for all grids; one step is captured in a CUDA graph
 * (re-captured when the step sizes, the integrator or the tile shape change)
 * and replayed.  Every point runs the same arithmetic as nr_rk4_step /
 * nr_ssprk3_step, so each grid's state is bitwise what those would give, for
 * any tile shape and any batch composition (azimuthal ghost copies are
 * refreshed on demand, as described at nr_rk4_step).
 *   nr_batch_create: grids stay owned by the caller and must outlive the
 *     batch; their library-owned states are advanced in place.  Work is issued
 *     on the grids' stream.  Errors: NR_EINVAL (mixed families, orders,
 *     devices, streams or azimuth kinds, duplicates), NR_ENOMEM, NR_ECUDA.
 *   nr_batch_set_tile: tile shape tile_x x tile_y of interior points per work
 *     item, one of 32x4, 64x2, 128x1, 16x8, 32x2, 64x1, 32x1 (default 16x8).
 *   nr_batch_autotune: times one substage launch of each compiled tile shape
 *     on the batch (it writes only the RK work buffers, not the states), keeps
 *     the fastest and returns it (synchronises).
 *   nr_batch_rk4_step, nr_batch_ssprk3_step: dts[ngrids] per-grid step sizes
 *     (host), nsteps steps of RK4 or SSPRK3. */
typedef struct nr_batch nr_batch;
int nr_batch_create(nr_grid* const* grids, int ngrids, nr_batch** out);
void nr_batch_destroy(nr_batch* batch);
int nr_batch_set_tile(nr_batch* batch, int tile_x, int tile_y);
int nr_batch_autotune(nr_batch* batch, const double* dts, int* tile_x, int* tile_y, double* best_ms);
int nr_batch_rk4_step(nr_batch* batch, const double* dts, int nsteps);
int nr_batch_ssprk3_step(nr_batch* batch, const double* dts, int nsteps);

/* Served mode: continuous batching of evolution requests on one device.
 * A request is one grid (coords, Nxx, params) with Brill-Lindquist data
 * (npunct masses at xyz) evolved at its own CFL step until t_final by
 * params->integrator (RK4 or SSPRK3), with the scheme params->NG selects.
 *   nr_server_create: hbm_budget_bytes caps the summed device bytes of the
 *     running requests; max_slots caps their number; work is issued on stream.
 *   nr_server_submit: queues a request and returns its id (no device work;
 *     NR_EINVAL if its grid has no valid CFL step).
 *     keep_state bit 0 (1) keeps the final 24-gf state on the host for
 *     nr_server_fetch_state; bit 1 (2) keeps its digest (nr_state_digest) for
 *     nr_server_fetch_digest.
 *   nr_server_advance: makes queued requests resident (running) in policy
 *     order while the budget and the slots allow, then advances the selected
 *     running requests together -- one nr_batch per kind of request (coordinate
 *     family x azimuth kind x order x integrator), one launch per substage
 *     for each -- by up to nsteps steps.  Membership changes only at step boundaries:
 *     a request reaching t_final is retired (Hamiltonian-constraint norms
 *     recorded, state kept if asked, device memory released) and queued
 *     requests are admitted into the freed budget.  A request that
 *     cannot fit even alone is marked failed.  Synchronises at retirements;
 *     after enqueuing a chunk of steps it waits for the chunk before it, so
 *     at most one chunk is queued behind the one the GPU runs and the policy
 *     acts on new arrivals within about a chunk of GPU time.
 *   nr_server_poll: status 0 queued, 1 running, 2 done, 3 failed; steps done
 *     and total; the final L2/Linf Hamiltonian-constraint norms when done (NaN
 *     for a request the guard retired).
 *   nr_server_set_starvation_cap: SRPT with a bound on starvation: a request
 *     submitted more than `seconds` ago (wall clock) goes ahead of every request
 *     submitted since, in arrival order, both for admission and for the chunks
 *     (0 = off, the default; NR_EINVAL for a negative or NaN value).
 *   nr_server_set_prefetch: depth 0 (default): a request's host-side set-up
 *     (coordinates, per-axis arrays, boundary maps) runs when it is admitted.
 *     depth k > 0: a worker thread computes the set-ups of the next k queued
 *     requests in admission order while the GPU works, and while other
 *     requests run, a queued request is admitted only once its set-up is ready
 *     (the admission then only allocates, uploads and sets initial data);
 *     with nothing running it is admitted at once.  NR_EINVAL for depth < 0.
 *   nr_server_set_guard: every every_steps steps of a request (default 100;
 *     0 = off) the server checks alpha and W of the requests it advanced for
 *     NaN/Inf on the device (one flag per request, read back behind the next
 *     chunk, so without a synchronisation of its own).  A request found
 *     non-finite is retired as failed with NR_ENONFINITE (its device memory
 *     released, nothing kept) while the others continue, bitwise unaffected.
 *     A request that finishes is also checked at retirement.
 *   nr_server_stats: host-side accounting since creation, out[9] = chunks
 *     enqueued, batch rebuilds, admissions, retirements, then wall seconds spent
 *     admitting (grid set-up, upload, initial data), retiring (constraint norms,
 *     kept state or digest, release), rebuilding batches (and capturing their
 *     graphs), waiting at chunk fences (the GPU busy with the chunk before) and
 *     enqueueing chunks.
 *   nr_server_request_error: the status that ended a failed request
 *     (NR_ENONFINITE, NR_ENOMEM when it cannot fit the budget even alone, or
 *     the set-up's error); NR_OK for the others.
 *   nr_server_fetch_digest: the kept digest of a finished request.
 *   nr_server_set_tile: fixed tile shape for the batches (default: autotune at
 *     every membership change).
 *   nr_server_set_policy: the order in which queued requests become resident
 *     and running requests are advanced.  NR_SERVE_FIFO (default): arrival
 *     order.  NR_SERVE_SRPT: least remaining work first (remaining steps x
 *     substeps per step x interior points; for a queued request the steps
 *     follow from its CFL step), preemptive at chunk boundaries: a running request that is not
 *     selected keeps its state in HBM and resumes later, with a result that is
 *     still bitwise the one it gets alone.  Each chunk advances the longest
 *     prefix of that order whose interior points sum to at most
 *     max_batch_points (at least one request; 0 = no cap, so every running
 *     request advances).  NR_EINVAL for an unknown policy or a negative cap.
 * Each request's result is bitwise what running it alone with nr_rk4_step
 * or nr_ssprk3_step gives, whichever requests shared the GPU with it. */
typedef struct nr_server nr_server;
enum { NR_SERVE_FIFO = 0, NR_SERVE_SRPT = 1 };
int nr_server_create(size_t hbm_budget_bytes, int max_slots, int device, void* stream, nr_server** out);
void nr_server_destroy(nr_server* server);
int nr_server_set_tile(nr_server* server, int tile_x, int tile_y);
int nr_server_set_policy(nr_server* server, int policy, int64_t max_batch_points);
int nr_server_submit(nr_server* server, int coords, const int Nxx[3], const nr_params* params, int npunct,
                     const double* mass, const double* xyz, double t_final, int keep_state, int64_t* id_out);
int nr_server_advance(nr_server* server, int nsteps, int* n_running, int* n_queued);
int nr_server_poll(nr_server* server, int64_t id, int* status, int64_t* steps_done, int64_t* steps_total,
                   double* l2, double* linf);
int nr_server_fetch_state(nr_server* server, int64_t id, double* host_state, size_t capacity_doubles);
int nr_server_set_guard(nr_server* server, int every_steps);
int nr_server_set_starvation_cap(nr_server* server, double seconds);
int nr_server_set_prefetch(nr_server* server, int depth);
int nr_server_stats(const nr_server* server, double out[9]);
int nr_server_request_error(nr_server* server, int64_t id, int* code);
int nr_server_fetch_digest(nr_server* server, int64_t id, uint64_t* digest);

/* Partitioned grid: one grid cut into partitions, the chare decomposition of
 * Sec. 3 ("Charm++ parallelization": the grid divided into chares of
 * prod_i N_i / N_chare^i points, each larger than N_G; face-sequential halo
 * exchange E-W, N-S, T-B; per-chare send lists, built at set-up, for inner
 * boundary points whose source lies on another chare).
 *   parts[3]: partitions per axis.  The interior along axis d is cut into
 *     parts[d] slabs of N_d / parts[d] points (rounded down at the cut k:
 *     N_G + floor(k N_d / parts[d])), each at least N_G thick (NR_EINVAL
 *     otherwise; so a two-point azimuth is never cut); at most 4096 partitions.
 *     Partition q = q0 + parts[0] (q1 + parts[1] q2) owns its interior box and,
 *     at the grid's edges, the ghost layers beyond it, and stores that box
 *     widened by N_G on every side: T_q = prod_d (N_d,q + 2 N_G) points per
 *     gridfunction, its own four 24-gridfunction sets.
 *   Each substage of nr_part_rk4_step / nr_part_ssprk3_step computes, on every
 *     partition, the right-hand side and the update of the points it owns, then
 *     fills the inner boundary points -- from sources on the same partition by
 *     parity copies, from sources on other partitions by messages -- and then
 *     the halos, one axis after the other.  A message is gathered into a send
 *     buffer on its source partition, copied to a receive buffer of its
 *     destination (cudaMemcpyAsync), and scattered there with its parity signs.
 *     All partitions live on params->device.  Every point runs the arithmetic of
 *     nr_rk4_step / nr_ssprk3_step on the same values, so the evolution is
 *     bitwise that of the whole grid.  A step is captured in a CUDA graph
 *     (re-captured when dt or the integrator changes).
 *   nr_part_set_brill_lindquist: as nr_set_brill_lindquist (the perturbation
 *     counter is the whole grid's flat index), then the boundary fills.
 *   nr_part_set_state / nr_part_get_state: the whole grid's 24-gridfunction set
 *     (24*T doubles, the layout of nr_get_state) to every partition's box /
 *     from the points each partition owns; from_host / to_host = 1: host memory,
 *     staged through a device buffer of the whole set allocated on first use
 *     (the call synchronises); 0: device memory, stream-ordered.  The state set
 *     must hold the inner ghosts' parity copies, as every state of the method.
 *   nr_part_digest: nr_state_digest of the whole grid's state, summed over the
 *     partitions (the same value as for the unsplit grid); synchronises.
 *   nr_part_hamiltonian: the L2 and Linf norms of the Hamiltonian constraint over
 *     the interior points in the radius band [h_rmin, h_rmax], as nr_hamiltonian:
 *     each partition's points into block partials, one fixed-order reduction over
 *     all of them (the norms agree with the whole grid's to rounding; the summation
 *     order differs); either output may be NULL, not both; synchronises.
 *   nr_part_query: partitions, messages per phase (0: inner boundary across
 *     partitions; 1..3: halos along axes 0..2), CFL step, device bytes.
 *   nr_part_plan_info / nr_part_plan_boxes / nr_part_plan_records (host only, no
 *   GPU): the plan of the grid (coords, Nxx, NG) cut by parts.  Boxes: 15 ints
 *     per partition, interior lo[3], hi[3], owned lo[3], hi[3] (global padded
 *     indices, hi exclusive) and the local origin[3] (lo - NG); local index of
 *     global (g0,g1,g2): (g0-o0) + m0 ((g1-o1) + m1 (g2-o2)), m_d = hi_d - lo_d
 *     + 2 NG.  Records of phase 0..3: 5 ints each, source partition, source
 *     local index, destination partition, destination local index, parity mask
 *     (bit t: sign -1 for tensor type t, as in nr_build_maps; phase 0 lists every
 *     inner boundary fill, within a partition too, phases 1..3 the halo copies
 *     along axes 0..2 in the order they are applied).  records[4] of plan_info:
 *     the counts per phase; capacity: the records rec can hold (NR_EINVAL if
 *     too small).
 * Errors: NR_EINVAL, NR_EMAP, NR_ENOMEM, NR_ECUDA. */
typedef struct nr_part nr_part;
int nr_part_create(int coords, const int Nxx[3], const nr_params* params, const int parts[3], nr_part** out);
void nr_part_destroy(nr_part* part);
int nr_part_query(const nr_part* part, int64_t* nparts, int64_t messages[4], double* dt_cfl, size_t* device_bytes);
int nr_part_set_brill_lindquist(nr_part* part, int npunct, const double* mass, const double* xyz, double perturb_amp,
                                uint64_t seed);
int nr_part_set_state(nr_part* part, const double* src, int from_host);
int nr_part_get_state(nr_part* part, double* dst, int to_host);
int nr_part_rk4_step(nr_part* part, double dt, int nsteps);
int nr_part_ssprk3_step(nr_part* part, double dt, int nsteps);
int nr_part_digest(nr_part* part, uint64_t* out);
int nr_part_hamiltonian(nr_part* part, double* l2_out, double* linf_out);
int nr_part_sync(nr_part* part);
int nr_part_plan_info(int coords, const int Nxx[3], int NG, const int parts[3], int64_t* nparts, int64_t records[4]);
int nr_part_plan_boxes(int coords, const int Nxx[3], int NG, const int parts[3], int32_t* boxes);
int nr_part_plan_records(int coords, const int Nxx[3], int NG, const int parts[3], int phase, int32_t* rec,
                         int64_t capacity);

/* Hamiltonian constraint that allocates nothing.  The paper has no
 * counterpart: this is a library service for callers that cannot call
 * cudaMalloc -- a host framework that owns all device memory through its own
 * pool or HBM budget, a caller that holds no nr_grid (creating one allocates
 * four 24-gridfunction sets) and only wants to check a state it already has
 * on the device, or a latency-critical loop that cannot take cudaMalloc's
 * implicit device synchronisation.  It computes what nr_hamiltonian computes
 * (H at interior points of y_dev, the L2/Linf norms over the radius band
 * [params->h_rmin, params->h_rmax]) for the grid described by coords, Nxx and
 * *params, on params->device and params->stream.  Its scratch memory (per-axis
 * reference-metric arrays, per-block partial norms, the reduced norms) is one
 * file-scope device array of 512 KiB that every GPU loading the library holds
 * until the process exits; nothing is allocated per call (no cudaMalloc,
 * cudaFree or allocating library routine).
 *   Limit: the per-axis arrays must fit 59,360 doubles, i.e.
 *   4 n0 + 4 n1 + 2 n2 (SinhSpherical, Spherical) or 4 n0 + 2 n1 + 3 n2
 *   (SinhCylindrical) with n_d = N_d + 2 NG; larger grids get NR_EINVAL.
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.  The
 *   address is kept for the life of the process: do not call this entry point
 *   on a device after its primary context has been reset (cudaDeviceReset).
 *   All calls share the one array and every call overwrites it: calls that
 *   overlap on the GPU (different streams, threads or processes' streams on
 *   the same device) race.  Each call writes every scratch value it reads.
 *   y_dev: caller-owned 24*T doubles; H_dev: caller-owned T doubles or NULL
 *   (ghost points set to 0); l2_out/linf_out: host doubles or NULL (given:
 *   the call synchronises params->stream).  Errors: NR_EINVAL, NR_ECUDA. */
int nr_hamiltonian_noalloc(int coords, const int Nxx[3], const nr_params* params, const double* y_dev,
                           double* H_dev, double* l2_out, double* linf_out);

/* Measured FP64 FMA throughput of a device (FLOP/s, FMA = 2 FLOP): a fixed-size
 * kernel of independent FMA chains, best of five timed launches with CUDA events.
 * The roofline denominator of the FP64-bound kernels.  Synchronises. */
int nr_fp64_peak(int device, double* flops_out);

/* Thread-local message of the last error (empty string if none). */
const char* nr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
