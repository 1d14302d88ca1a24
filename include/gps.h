/*
 * gps.h -- C ABI of the GB300 generalized Poisson / Poisson-Boltzmann solver.
 *
 * Method: arXiv:1509.00680 (Fisicaro, Genovese, Andreussi, Marzari, Goedecker),
 * "A generalized Poisson and Poisson-Boltzmann solver for electrostatic
 * environments".  The solver computes phi with
 *     div eps grad phi = -4 pi (rho + rho_ions[phi])        (Eqs. GPe, PBe)
 * by the preconditioned conjugate gradient of Algorithm 2, whose
 * preconditioner is one vacuum Poisson solve (Eq. PCGdef) and whose operator
 * is applied through the identity of Eq. (corr) / (corrPB); the nonlinear
 * Poisson-Boltzmann case adds the ionic-charge outer loop of Algorithm 4.
 *
 * Conventions
 *   Atomic units (bohr, Hartree, e = 1), Gaussian 4 pi as in the paper.
 *   Fields are contiguous IEEE double arrays of nx*ny*nz points with x
 *   fastest: index i + nx*(j + ny*k), point (origin + i hx, j hy, k hz).
 *   "_dev" pointers are CUDA device pointers on the context's device; the
 *   caller owns them, the library never frees or retains them after a call.
 *   "_host" entry points take host pointers and copy through library-owned
 *   device buffers.  Calls are ordered on the given CUDA stream (NULL = the
 *   legacy default stream) and return after the result is complete on the
 *   host side (the reports carry host-read scalars).
 *   A context is not thread safe: one host thread per context.
 *   Every entry point returns a gps_status; nothing is thrown across the ABI.
 */
#ifndef GPS_H
#define GPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPS_OK = 0,
  GPS_ERR_INVALID = 1,        /* bad argument: sizes, pointer, eps <= 0, unsupported size */
  GPS_ERR_NOMEM = 2,          /* device allocation failed or the HBM budget is exceeded */
  GPS_ERR_NOT_CONVERGED = 3,  /* max_iter / max_outer reached; phi holds the last iterate */
  GPS_ERR_BREAKDOWN = 4,      /* (p, A p) >= 0 or not finite: the operator is not negative definite */
  GPS_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
  GPS_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  GPS_PENDING = 7             /* asynchronous request not finished yet */
} gps_status;

typedef enum {
  GPS_BC_FREE = 0,       /* isolated system: truncated-Coulomb vacuum kernel on a 2x padded grid */
  GPS_BC_PERIODIC = 1,   /* periodic cell: spectral 4 pi / k^2 kernel */
  GPS_BC_SURFACE = 2,    /* periodic in x and y, free in z (2x padded in z) */
  GPS_BC_WIRE = 3        /* periodic in z, free in x and y (2x padded in x and y): the Coulomb
                            kernel truncated at transverse radius sqrt((nx hx)^2 + (ny hy)^2) */
} gps_bc;

/* Arithmetic of the spectrum passes (the vacuum solve inside the
 * preconditioner); every vector, dot product, alpha/beta and the ionic term
 * are FP64 in all modes.
 *   GPS_FP64        FP64 spectrum.
 *   GPS_MIXED       FP64 spectrum until ||r|| <= mixed_switch ||r_0||, then FP32.
 *                   For nonlinear PB r_0 is the residual of the first outer
 *                   step (4 pi F_0): an inner solve that starts below the
 *                   switch runs in FP32 throughout.
 *   GPS_DF64        double-float spectrum: each value the unevaluated sum of
 *                   two floats (about 48 significant bits), computed on the
 *                   FP32 pipe, which on GB300 issues 64x the FP64 rate.
 *   GPS_MIXED_DF64  double-float spectrum until the switch, then FP32. */
typedef enum { GPS_FP64 = 0, GPS_MIXED = 1, GPS_DF64 = 2, GPS_MIXED_DF64 = 3 } gps_precision;
typedef enum { GPS_GPE = 0, GPS_LPB = 1, GPS_NLPB = 2, GPS_MPB = 3 } gps_problem;
typedef enum { GPS_OUTER_NEWTON = 0, GPS_OUTER_PRINTED = 1 } gps_outer_mode;
typedef enum { GPS_FORCING_EW2 = 0, GPS_FORCING_RATIO = 1 } gps_forcing_rule;

/* Solver of the generalized Poisson equation (gps_opts.method; accepted by
 * gps_gpe_solve and gps_gpe_solve_host only, with precision GPS_FP64 and
 * warm_start 0; other methods than GPS_PCG return GPS_ERR_INVALID elsewhere).
 *   GPS_PCG  Algorithm 2 with the preconditioner of Eq. (PCGdef) (default).
 *   GPS_SC   Algorithm 1, the self-consistent iteration (Eqs. remap, rhoiter):
 *            phi_k = S(rho/eps + rho_iter_k), rho~ = grad ln eps . grad phi_k / 4 pi,
 *            rho_iter_(k+1) = eta rho~ + (1 - eta) rho_iter_k (opts.eta).
 *   GPS_PSD  Algorithm 2 with beta = 0 and the preconditioner of Eq. (PrePSD),
 *            eps lap v = r; step opts.alpha, or (alpha = 0) the steepest-
 *            descent step (v, r) / (v, A v); with opts.diis = m >= 2, Pulay's
 *            DIIS over the last m iterates before every step.
 * Both comparison solvers take grad ln eps by the order-16 central first
 * derivative (Sec. "Numerical results") and the Laplacian that the vacuum
 * solve inverts: A phi = eps (lap_S phi + grad ln eps . grad phi), a
 * discretization of Eq. (GPe) that differs from Algorithm 2's at the level of
 * the discretization error.  They stop on ||r||_2 <= max(tol_abs, tol_rel
 * ||r_0||_2) with r = -4 pi rho - A phi (SC: r_k = -4 pi eps (rho~ - rho_iter_k),
 * the residual of phi_k), for periodic BC measured modulo its component along
 * eps; rep->iters counts vacuum solves.  Periodic axes need at least 8
 * points.  One vacuum solve and one order-16 stencil pass per iteration. */
typedef enum { GPS_PCG = 0, GPS_SC = 1, GPS_PSD = 2 } gps_method;
#define GPS_MAX_DIIS 8

/* Uniform orthorhombic grid.  nx, ny, nz >= 4; each padded FFT length
 * (2n on free axes, n on periodic axes) must factor into 2, 3 and 5, be even
 * and be at most 4096.  Free and wire BC also need 4 n_d h_d >= n_d h_d + R on
 * every free axis d, R the truncation radius (the box diagonal; for wire the
 * diagonal of the x-y cross-section), for the 4x oversampled kernel.
 * Sec. "Numerical results" (orthorhombic grid of uniform spacing). */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  int bc;                /* gps_bc */
} gps_grid;

/* Mobile ions (Eqs. rhoions, ionsconcPB).  Species i has valence z[i] and
 * bulk concentration c_molar[i] (mol/L).  The ion-exclusion function is the
 * cavity function gamma = (eps - 1)/(eps0 - 1), so ions live in the solvent
 * only.  The linear PB term of Eq. (corrPB) is lambda(r) = gamma(r) * 4 pi
 * sum_i z_i^2 n_i / kT with n_i the number densities in bohr^-3. */
#define GPS_MAX_SPECIES 8
typedef struct {
  int nspecies;
  int z[GPS_MAX_SPECIES];
  double c_molar[GPS_MAX_SPECIES];
  double temperature;    /* K */
  double eps0;           /* bulk dielectric constant of the solvent (for gamma) */
  /* Steric (modified PB, GPS_MPB) parameters, Eqs. (ionsconcMPB, maxconc):
   * effective ion radii R_i and packing coefficient p give the maximum
   * concentration c_i^max = p / ((4/3) pi R_i^3 N_A) and
   * c_i = c_i^inf e_i / (1 + sum_j (c_j^inf / c_j^max)(e_j - 1)),
   * e_i = exp(-Z_i phi / kT) (the paper prints "+ 1" in the bracket; read as
   * "- 1", the form that gives c_i^inf where phi = 0).  Unused (zero) for the
   * other problems. */
  double radius_angstrom[GPS_MAX_SPECIES];
  double packing;
  /* Ion-exclusion function gamma(r) >= 0 of Eq. (rhoions), nx*ny*nz values, or
   * NULL for the cavity function gamma = (eps - 1)/(eps0 - 1).  A device array
   * for gps_pb_solve and gps_ionic_charge, a host array for gps_pb_solve_host;
   * must be NULL in batched and served requests.  A solve with it takes no
   * warm start. */
  const double* exclusion;
} gps_electrolyte;

/* Solver options.  Convergence of Algorithm 2 is tested on the Euclidean norm
 * of the residual r (Sec. "Preconditioned conjugate gradient"):
 * ||r||_2 <= max(tol_abs, tol_rel * ||r_0||_2), r_0 = -4 pi rho.
 * For GPS_NLPB the outer loop stops when the Euclidean norm of the ionic
 * charge residual falls below tol_outer. */
typedef struct {
  double tol_abs;        /* absolute residual tolerance (e.g. 1e-10) */
  double tol_rel;        /* relative residual tolerance (0 = off) */
  int max_iter;          /* PCG iterations per solve (inner solves for NLPB) */
  int max_outer;         /* NLPB outer steps */
  double tol_outer;      /* NLPB outer tolerance on the ionic-charge residual */
  double eta;            /* mixing: NLPB printed Algorithm 4; GPS_SC rho_iter (Algorithm 1) */
  int outer_mode;        /* gps_outer_mode */
  double forcing;        /* NLPB Newton: cap of the inner solve's relative tolerance eta_k
                            (see forcing_rule); in (0, 1) */
  int precision;         /* gps_precision */
  double mixed_switch;   /* GPS_MIXED(_DF64): high-precision preconditioner until
                            ||r|| <= mixed_switch*||r_0|| (nonlinear PB: r_0 of the first outer step) */
  int certify;           /* 1: compute rep->fixed_point_res (always done for GPS_MIXED) */
  int warm_start;        /* GPe / LPB through the single-solve entry points: 1 = when the
                            previous solve of the same kind on this context and grid had the
                            same eps (compared value by value on the device) and, for LPB, the
                            same electrolyte, start from its potential, phi_0 = phi_prev, with
                            r_0 = b - (b_prev - r_prev), b = -4 pi rho: the previous solve's
                            final residual stands in for A phi_prev, so no operator is applied
                            (a warm start of Algorithm 2).  Every solve with warm_start set
                            keeps eps, phi and b - r on the device for the next one (three
                            more grid-sized arrays in the context).  Batched and served
                            requests (gps_batch_solve, gps_server_submit): the same, from the
                            last warm-start request of the same kind and electrolyte (compared
                            by value) that completed in the pool of its grid, if that one was
                            done when the request was admitted; the pool then keeps three
                            more grid-sized arrays.  Otherwise a cold start (rep->warm 0). */
  int method;            /* gps_method (GPS_PCG) */
  double alpha;          /* GPS_PSD: fixed step length; 0 = steepest-descent step */
  int diis;              /* GPS_PSD: DIIS history length 0..GPS_MAX_DIIS (0 and 1: plain PSD) */
  int forcing_rule;      /* NLPB Newton, inner tolerance eta_k relative to the inner solve's
                            initial residual (F_k the outer residual of step k):
                            GPS_FORCING_EW2 (default) Eisenstat & Walker's choice 2: eta_0 =
                            forcing, eta_k = 0.9 (F_k/F_(k-1))^2, raised to 0.9 eta_(k-1)^2 when
                            that exceeds 0.1, capped at forcing;
                            GPS_FORCING_RATIO: eta_k = min(forcing, F_k/F_0).
                            Both reach the same solution; they differ in how far each inner
                            solve is taken. */
} gps_opts;

typedef struct {
  int status;            /* gps_status of the solve */
  int iters;             /* PCG iterations (summed over inner solves for NLPB) */
  int outer_iters;       /* NLPB outer steps */
  int fp64_iters;        /* iterations that used the FP64 preconditioner */
  double res0;           /* ||r_0||_2 of the (last) PCG */
  double res;            /* ||r||_2 at exit of the (last) PCG */
  double outer_res;      /* NLPB: final ionic-charge residual */
  double background;     /* periodic GPe: mean of rho removed to neutralize the cell */
  double fixed_point_res; /* ||g|| / ||phi||, g = M(rho [+ rho_ions] - (q + lambda) phi / 4pi)
                             [+ <sqrt(eps) phi> s, periodic] - phi with an FP64 vacuum solve:
                             zero for the exact discrete solution (certificate of the result);
                             -1 when not computed */
  double time_ms;        /* wall time of the call (host clock, synchronized) */
  int warm;              /* 1: the solve started from the previous one (opts.warm_start) */
} gps_report;

typedef struct gps_ctx gps_ctx;

/* Fill *opts with defaults: tol_abs 1e-10, tol_rel 0, max_iter 500,
 * max_outer 100, tol_outer 1e-10, eta 0.6, Newton outer mode, forcing 0.3,
 * FP64, mixed_switch 1e-2, certify 0, warm_start 0, method GPS_PCG (alpha 0,
 * diis 0). */
void gps_default_opts(gps_opts* opts);

/* Human-readable name of a status code (static storage). */
const char* gps_status_string(int status);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context keeps in cached plans (0 = no cap).  Returns
 * GPS_ERR_INVALID for a NULL out pointer or bad device, GPS_ERR_CUDA if the
 * device cannot be selected. */
int gps_create(gps_ctx** out, int device, size_t hbm_budget_bytes);

/* Release every plan and buffer of the context (NULL is a no-op). */
void gps_destroy(gps_ctx* ctx);

/* Device bytes held by the context's cached plans. */
size_t gps_bytes_in_use(const gps_ctx* ctx);

/* Generalized Poisson equation, Eq. (GPe), by Algorithm 2 from phi_0 = 0.
 * rho_dev, eps_dev: inputs (eps > 0 everywhere, else GPS_ERR_INVALID);
 * phi_dev: output.  Periodic BC: the mean of rho is removed (reported in
 * rep->background) and phi satisfies sum sqrt(eps) phi = 0.  rep may be NULL. */
int gps_gpe_solve(gps_ctx* ctx, const gps_grid* grid, const double* rho_dev,
                  const double* eps_dev, double* phi_dev, const gps_opts* opts,
                  gps_report* rep, void* cuda_stream);

/* Poisson-Boltzmann.  kind = GPS_LPB: linear PB, Eq. (corrPB), by Algorithm 2.
 * kind = GPS_NLPB: nonlinear PB, Eqs. (PBe, rhoions, ionsconcPB), by the
 * outer loop of Algorithm 4 (opts->outer_mode selects the printed linear
 * mixing or the Newton-linearized inner operator), each inner solve by
 * Algorithm 2.  kind = GPS_MPB: modified (steric) PB, Eqs. (PBe, rhoions,
 * ionsconcMPB, maxconc), by the same outer loop; needs packing > 0 and
 * radius_angstrom > 0 for every species (else GPS_ERR_INVALID).
 * kind = GPS_GPE ignores the electrolyte. */
int gps_pb_solve(gps_ctx* ctx, const gps_grid* grid, const double* rho_dev,
                 const double* eps_dev, const gps_electrolyte* el, int kind,
                 double* phi_dev, const gps_opts* opts, gps_report* rep,
                 void* cuda_stream);

/* Same as gps_gpe_solve / gps_pb_solve with host arrays: rho and eps are
 * copied to library-owned device buffers, phi is copied back. */
int gps_gpe_solve_host(gps_ctx* ctx, const gps_grid* grid, const double* rho_host,
                       const double* eps_host, double* phi_host, const gps_opts* opts,
                       gps_report* rep, void* cuda_stream);
int gps_pb_solve_host(gps_ctx* ctx, const gps_grid* grid, const double* rho_host,
                      const double* eps_host, const gps_electrolyte* el, int kind,
                      double* phi_host, const gps_opts* opts, gps_report* rep,
                      void* cuda_stream);

/* Step S1 (Eq. corr): s = eps^-1/2 and q = sqrt(eps) lap sqrt(eps) -- the
 * order-16 finite-difference Laplacian (Sec. "Numerical results") for free
 * and surface BC, the spectral Laplacian that the vacuum solve inverts for
 * periodic BC.  s_dev, q_dev: outputs of nx*ny*nz doubles. */
int gps_setup_fields(gps_ctx* ctx, const gps_grid* grid, const double* eps_dev,
                     double* s_dev, double* q_dev, void* cuda_stream);

/* Vacuum Poisson solve w = S(sigma), lap w = -4 pi sigma (Eq. SPe) under the
 * grid's BC.  Periodic BC drops the mean of sigma. */
int gps_vacuum_solve(gps_ctx* ctx, const gps_grid* grid, const double* sigma_dev,
                     double* w_dev, void* cuda_stream);

/* Step S3, the preconditioner of Eq. (PCGdef): v = s S(s r) for a given
 * s = eps^-1/2.  precision: GPS_FP64, GPS_MIXED (FFT passes in FP32) or
 * GPS_DF64 (FFT passes in double-float). */
int gps_precondition(gps_ctx* ctx, const gps_grid* grid, const double* s_dev,
                     const double* r_dev, double* v_dev, int precision,
                     void* cuda_stream);

/* Ionic charge of Eqs. (rhoions, ionsconcPB) with the cavity exclusion
 * function: out = gamma sum_i z_i n_i exp(-z_i phi / kT), exponent capped at
 * +40; with el->packing > 0 the steric distribution of Eq. (ionsconcMPB)
 * (see gps_electrolyte).  Inputs phi_dev, eps_dev; output out_dev. */
int gps_ionic_charge(gps_ctx* ctx, const gps_grid* grid, const double* phi_dev,
                     const double* eps_dev, const gps_electrolyte* el,
                     double* out_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Quantities a DFT code takes from the solve (Sec. "Charge-dependent
 * cavity").  Gradients by the order-16 central differences (periodic axes
 * wrap and need at least 8 points; free faces continue the field by its face
 * value).  All arrays are nx*ny*nz doubles on the current device unless
 * stated; the calls are asynchronous on the stream except
 * gps_electrostatic_energy, which returns after synchronizing it. */

/* Charge-dependent (sccs) dielectric, Eq. (sccs): eps = 1 where rho_elec >=
 * rho_max, eps0 where rho_elec <= rho_min, and eps0^w(rho) in between, w =
 * (z - sin z) / (2 pi), z = 2 pi ln(rho_max / rho) / ln(rho_max / rho_min).
 * (The printed middle branch eps0 exp(w) is 1 at neither threshold; eps0^w
 * is continuous with both.)  deps_dev (may be NULL) receives d eps / d rho_elec
 * (0 outside the transition).  n values; rho_max > rho_min > 0, eps0 > 1.
 * The paper uses rho_max = 5e-3, rho_min = 1e-4. */
int gps_sccs_eps(gps_ctx* ctx, size_t n, const double* rho_elec_dev, double rho_max, double rho_min,
                 double eps0, double* eps_dev, double* deps_dev, void* cuda_stream);

/* Polarization charge, Eqs. (remap, rhopol): rho_pol = grad ln eps . grad phi
 * / 4 pi - ((eps - 1) / eps) rho (the sign Eq. remap requires; the paper
 * prints "+").  eps > 0. */
int gps_polarization_charge(gps_ctx* ctx, const gps_grid* grid, const double* rho_dev,
                            const double* eps_dev, const double* phi_dev, double* rho_pol_dev,
                            void* cuda_stream);

/* Kohn-Sham correction of a charge-dependent cavity, Eq. (veps):
 * v_eps = -(1/8 pi) (d eps / d rho_elec) |grad phi|^2. */
int gps_v_eps(gps_ctx* ctx, const gps_grid* grid, const double* deps_dev, const double* phi_dev,
              double* v_eps_dev, void* cuda_stream);

/* Electrostatic energy in its two forms (Sec. "Charge-dependent cavity"):
 * e_rho_phi = (1/2) sum rho phi h^3 and e_eps_grad = (1/8 pi) sum eps
 * |grad phi|^2 h^3.  They are equal up to discretization error for a converged
 * phi whose field is contained in the box; for a charged solute with free BC
 * the second misses the field energy outside the box.  Either output pointer
 * may be NULL. */
int gps_electrostatic_energy(gps_ctx* ctx, const gps_grid* grid, const double* rho_dev,
                             const double* eps_dev, const double* phi_dev, double* e_rho_phi,
                             double* e_eps_grad, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched and served solves.  A request carries its own grid, problem,
 * electrolyte and options and host arrays (rho and eps are read when the
 * request is admitted; phi is written when it completes; all three must stay
 * valid until then).  Requests with the same grid (shape, spacing, BC) share
 * a pool of slots: one launch sequence advances every slot of a pool by a
 * few PCG iterations (Algorithm 2), each slot at its own stage (setup,
 * iterations, the outer steps of Algorithm 4, certificate).  A request is
 * admitted into a free slot as soon as one frees up and device memory
 * allows, while the other slots keep iterating (continuous batching); pools
 * of different grids run on their own streams and overlap on the device.
 * Every slot reduces in a fixed order, so a result does not depend on which
 * other requests shared its launches.
 */
typedef struct {
  gps_grid grid;
  int kind;                 /* gps_problem */
  gps_electrolyte el;       /* ignored for GPS_GPE */
  gps_opts opts;
  const double* rho_host;
  const double* eps_host;
  double* phi_host;
} gps_request;

/* Solve `count` requests on the context's device with continuous batching,
 * returning when all are done; reps[i] receives request i's report (its
 * time_ms is the latency from the call to that request's completion).
 * Returns GPS_OK if every request succeeded, else the first failing status. */
int gps_batch_solve(gps_ctx* ctx, int count, const gps_request* reqs, gps_report* reps);

/* Asynchronous serving loop: a host thread admits submitted requests
 * against the HBM budget (hbm_budget_bytes, 0 = no cap) into pools of at
 * most max_slots slots (0 = automatic by grid size) and drives them.
 * gps_server_submit returns a ticket; gps_server_poll returns GPS_PENDING
 * until the request is done, then its final status (and report, whose
 * time_ms is the submit-to-completion latency); gps_server_wait blocks.
 * A ticket can be polled or waited on until it has returned a final status
 * once. */
typedef struct gps_server gps_server;
int gps_server_create(gps_server** out, int device, size_t hbm_budget_bytes, int max_slots);
int gps_server_submit(gps_server* srv, const gps_request* req, unsigned long long* ticket);
int gps_server_poll(gps_server* srv, unsigned long long ticket, gps_report* rep);
int gps_server_wait(gps_server* srv, unsigned long long ticket, gps_report* rep);
/* Device bytes held by the server's pools and the largest number of
 * requests that were in slots at the same time. */
int gps_server_stats(gps_server* srv, size_t* bytes_in_use, int* max_concurrent);
void gps_server_destroy(gps_server* srv);

/* Vacuum Poisson solve w = S(sigma) (as gps_vacuum_solve) for callers that
 * cannot allocate device memory -- for example a plugin whose host
 * application owns the device-memory budget, a process whose framework has
 * already reserved nearly all of HBM in its own pool, or a latency-critical
 * loop that cannot afford the implicit device synchronization of
 * cudaMalloc/cudaFree.  The paper has no counterpart: it is an interface
 * variant of the vacuum solve.  No context is needed and no device memory
 * is allocated: the twiddle tables, the Green's-function table and the
 * spectrum live in one file-scope device array of 8 MiB that every GPU
 * loading this library holds until the process exits.
 * Supported: GPS_BC_PERIODIC and GPS_BC_SURFACE grids whose padded FFT
 * lengths (nx, ny, and nz periodic or 2 nz surface) are even, at most 4096
 * and factor into 2, 3 and 5, and for which
 *     16 (nx + ny + Pz) + 8 (nx/2+1)(ny/2+1)(Pz/2+1) + 16 Hp ny nz
 * bytes, Hp = nx/2+1 rounded up to even (twiddles, Green's-function octant
 * table, spectrum with an even row pitch; each of the first four parts
 * rounded up to 256 bytes) fit in the 8 MiB (8,388,608 byte) array.  The
 * largest cubic periodic grid is 96^3 (8,318,720 bytes); 96 x 96 x 100 and
 * 100^3 are over the limit.  Anything else returns
 * GPS_ERR_INVALID.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not use
 * this entry point after cudaDeviceReset.  Every call uses the same array
 * and keeps the previous call's contents (each call rebuilds its tables, and
 * every spectrum value it reads it has written): calls that overlap on the
 * GPU (other streams, other host threads) race with each other and must be
 * serialized by the caller.
 * sigma_dev, w_dev: nx*ny*nz doubles on the current device.  The call
 * returns after synchronizing the stream. */
int gps_vacuum_solve_noalloc(const gps_grid* grid, const double* sigma_dev, double* w_dev,
                             void* cuda_stream);

/* Instrumentation.  gps_set_profiling(ctx, mask): every kernel of a kind
 * whose bit is set in `mask` that the solve entry points launch is
 * bracketed by CUDA events on the call's stream, and the elapsed times are
 * collected when the call returns (mask 0 turns profiling off, 0xFFFFF times
 * every kind).  Kernel kinds: 0 x_fwd, 1 y_fwd, 2 z (forward, Green's
 * multiply, inverse), 3 y_inv, 4 x_inv -- the spectrum passes of the FP64
 * spectrum; 10-14 the same passes of the double-float spectrum and 15-19 of
 * the FP32 spectrum; 5 update_p, 6 update_r, 7 setup, 8 stencil (the
 * order-16 passes of GPS_SC / GPS_PSD), 9 sc_vector (their vector updates
 * and DIIS).
 * Launches that return at once because the PCG had already converged are
 * not counted.  gps_get_profile writes per kind the launch count and the
 * total milliseconds accumulated since the last reset (arrays of
 * GPS_PROFILE_KINDS entries). */
#define GPS_PROFILE_KINDS 20
int gps_set_profiling(gps_ctx* ctx, int mask);
int gps_get_profile(gps_ctx* ctx, long long* launches, double* total_ms, int reset);

/* Radix order of the shared-memory FFT passes.  -1 (the default): the tuner
 * times, per grid and spectrum precision, the orders 0 (radix-8 stages first),
 * 1 (radix-8 stages last), 2 (radix 4) and, for the FP64 spectrum, 3 (radix
 * 16 first) and keeps the fastest; 0..3: plans made from now on use that
 * order where it applies to the length (else order 0), for reproducible
 * plans and for tests of each order.  Clears the process-wide tuning cache;
 * shapes already planned in a context keep their plans (use a new context). */
int gps_set_radix_order(int order);

/* Kernels of the x passes of the FP32 spectrum, for reproducible plans and
 * for tests of both: -1 (the default) the tuner times the shared-memory
 * Stockham kernels against the register-resident ones (padded lengths 64 ..
 * 1024) and keeps the faster; 0 always the shared-memory kernels; 1 the
 * register-resident ones where the length allows.  Clears the process-wide
 * tuning cache like gps_set_radix_order. */
int gps_set_x_kernel(int kind);

/* Kernel of the z pass of the FP32 and double-float spectra, for
 * reproducible plans and for tests of both: -1 (the default) the tuner times
 * the register-resident column kernel against its TMA-staged form (column
 * tiles moved to shared memory by tensor copies, double-buffered in a
 * persistent CTA; padded lengths 64 .. 1024) and keeps the faster; 0 always
 * the plain kernel; 1 the TMA-staged one where it applies.  A bounded wait
 * of the TMA-staged kernel that gives up makes the call return
 * GPS_ERR_TIMEOUT.  Clears the process-wide tuning cache. */
int gps_set_z_kernel(int kind);

/* Scheduling of the batching engine (gps_batch_solve and servers created
 * afterwards), for measurements: 1 (the default) every pool of the engine
 * advances on its own -- a pool whose round of PCG iterations has finished
 * is collected, takes queued requests into its free slots and starts its
 * next round while the other pools' rounds run, with more iterations per
 * round for small pools; 0 lockstep -- one round of four iterations on
 * every busy pool, then all pools are synchronized and collected. */
int gps_set_engine_mode(int async);

/* Number of CUDA kernels this library has launched in the process so far. */
unsigned long long gps_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* GPS_H */
