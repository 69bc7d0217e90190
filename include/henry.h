/*
 * henry.h - C ABI of libhenry: batched GB300 (sm_103a) scenario solves of the
 * Henry saltwater-intrusion problem and multilevel Monte Carlo accumulation,
 * after arXiv 2302.07804 ("Uncertainty quantification in coastal aquifers
 * using the multilevel Monte Carlo method").
 *
 * The problem (Sec. 2.1): fluid mass and salt mass balances, Eqs. (e_cont_eq)
 * and (e_tran_eq), with Darcy's law (e_Darcy_vel), rho(c) = rho0 + (rho1 -
 * rho0) c (e_lin_density), D = phi Dm I (e_mol_diff), on [0, Lx] x [0, Ly]
 * with the seaside (x = Lx) at brine hydrostatic pressure and c = 1, fresh
 * water flowing in at x = 0 with c = 0, no flux through top and bottom, and
 * c = 0 at t = 0 with fresh-water hydrostatic pressure.  Discretisation
 * (Sec. 2.3): cell-centred finite volumes with upwind advection on a uniform
 * grid of square cells (nx0 2^l x ny0 2^l cells at MLMC level l), implicit
 * Euler with r_l = steps0 2^l steps over [0, T], Newton's method per step,
 * each Newton system solved by BiCGStab preconditioned by one geometric
 * multigrid V-cycle (red-black 2x2-block Gauss-Seidel smoothing, coarse
 * operators rediscretised on the 2x coarser grids (or Galerkin products), a
 * dense solve on the 2 x 1 coarsest grid).  Random inputs (Sec. 4, three iid
 * U[-1, 1] factors): phi = phi_mean (1 + phi_amp xi1), K = K_mean exp(logK_amp
 * xi2), q_in = qin_mean (1 + qin_amp xi3).
 *
 * Conventions for every call below:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; they
 *    must stay valid until the work queued on `stream` has finished.  Pointers
 *    named *_host are host pointers.  `stream` is a cudaStream_t (NULL = the
 *    legacy default stream).
 *  - Arrays are dense, C order, FP64 unless stated.  A "state" array is
 *    [n][ny][nx][2] with (p [Pa], c [-]) per cell, cell (ix, iy) centred at
 *    ((ix + 1/2) h, (iy + 1/2) h), y pointing up.
 *  - Return value: HENRY_OK or an error code; on error henry_last_error()
 *    gives a message (per calling thread).  No call throws or aborts.
 *  - Calls are asynchronous with respect to the host except where stated
 *    ("synchronises"): the batch solve synchronises `stream` between Newton
 *    and Krylov iterations to test convergence.
 *  - The handle owns all device workspace; it grows on demand and is freed by
 *    henry_destroy.  A handle is not thread-safe: one host thread at a time.
 */
#ifndef HENRY_H
#define HENRY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
  HENRY_OK = 0,
  HENRY_EINVAL = 1,  /* invalid argument (NULL pointer, n <= 0, level out of range, ...) */
  HENRY_ECUDA = 2,   /* a CUDA runtime call failed */
  HENRY_ENOMEM = 3,  /* device allocation failed */
  HENRY_ENOCONV = 4, /* at least one sample did not converge; see status_dev */
  HENRY_ELIMIT = 5   /* an iteration cap of the driver was reached */
};

/* Per-sample status codes written to status_dev. */
enum {
  HENRY_SAMPLE_OK = 0,
  HENRY_SAMPLE_NEWTON = 1,   /* Newton did not converge within newton_maxit in some step */
  HENRY_SAMPLE_LINEAR = 2,   /* henry_adjoint: an adjoint system J^T lam = rhs did not converge within
                                adj_maxit (a forward BiCGStab that stops early leaves Newton's residual
                                test to decide, so forward solves report 1 or 3 instead) */
  HENRY_SAMPLE_NONFINITE = 3 /* a residual or coefficient was NaN or infinite */
};

/* Arithmetic of the linear solves (the Newton residual, update, QoIs and
 * MLMC sums are FP64 in both). */
enum { HENRY_FP64 = 0, HENRY_MIXED = 1 /* FP32 Jacobian, BiCGStab and V-cycle */ };

/* Coefficient models (the random inputs per sample and their meaning):
 *  UNIFORM3 (default): xi[3] uniform on [-1, 1]; phi = phi_mean (1 + phi_amp xi1),
 *    K = K_mean exp(logK_amp xi2), q_in = qin_mean (1 + qin_amp xi3), all constant in space.
 *  KL: xi[2 kl_terms + 1] = (theta_K[kl_terms], theta_phi[kl_terms], xi3): Gaussian random
 *    fields log K = log K_mean + kl_sigma_logK sum_t sqrt(lam_t) theta_K,t psi_t(x, y) and
 *    phi = clip(phi_mean + kl_sigma_phi sum_t sqrt(lam_t) theta_phi,t psi_t, phi_lo, phi_hi),
 *    the kl_terms leading Karhunen-Loeve terms of the covariance exp(-r^2 / (2 kl_corr_len^2))
 *    on [0, Lx] x [0, Ly] (Nystrom on 256 Gauss-Legendre nodes per direction; theta iid N(0, 1)
 *    supplied by the caller); q_in as above.
 *  TWO_LAYER: xi[3] uniform; the paper's two-layer porosity, Eq. (poro_2levels), with the
 *    Kozeny-Carman permeability, Eq. (e_perm_Kozeny_Carman), K = kappa phi^3 / (1 - phi^2),
 *    kappa such that K(phi_mean) = K_mean; q_in = qin_mean (1 + qin_amp xi3).
 * The field models use harmonic means of K and phi Dm on faces. */
enum { HENRY_MODEL_UNIFORM3 = 0, HENRY_MODEL_KL = 1, HENRY_MODEL_TWO_LAYER = 2 };

/* QoI sets (henry_config.qoi_set); henry_n_qoi gives the count per sample.
 * STANDARD (2): [0] salt mass sum phi rho(c) c h^2 at T (kg per metre of
 *   depth), [1] c at (1.5, 0.25), the mean of the four cells at that vertex.
 * PAPER (15): those two, [2] the freshwater integral Q_FW of Eq.
 *   (integral_fw), the area of the cells with c <= 0.012178, and [3..14] c at
 *   the 12 points of Eq. (12points) in the paper's order (its y in [-1, 0] is
 *   y - Ly here) by bilinear interpolation of the surrounding cell centres.
 * PAPER_FIELD (15 + nx0 ny0): those 15 and the c field averaged over the cells
 *   of the level-0 grid, row-major; its MLMC mean and variance (mlmc_accumulate)
 *   are the paper's mean and variance fields (Sec. 4).
 * PAPER_SERIES (15 + steps0): the 15 of PAPER and Q_FW after every level-0 time
 *   step (every 2^level fine steps, so the same instants at every level), the
 *   paper's Q_FW(t) curves and crossing times (Sec. 4); the last one is [2]. */
enum { HENRY_QOI_STANDARD = 0, HENRY_QOI_PAPER = 1, HENRY_QOI_PAPER_FIELD = 2, HENRY_QOI_PAPER_SERIES = 3 };

/* Discretisations (henry_config.scheme).
 * CELL (default): cell-centred finite volumes with upwind advection, the
 *   configuration's scheme (states [n][ny][nx][2] in the per-step calls).
 * VERTEX: the paper's own vertex-centred finite volumes (Sec. 2.3): (p, c)
 *   at the (ny + 1) x (nx + 1) grid vertices, n_l = 2 (nx + 1)(ny + 1)
 *   unknowns as in Table tab:adaptiveTS_times, a "consistent velocity" and
 *   partial upwinding (the readings are stated in henry_vc.cuh); Newton with
 *   BiCGStab preconditioned by a V-cycle on vertex-nested grids (four-colour
 *   2x2-block Gauss-Seidel, full-weighting restriction, bilinear
 *   prolongation, rediscretised coarse operators, a dense solve on the 2 x 1
 *   element grid).  QoIs: the lumped salt mass and c at the vertex (1.5,
 *   0.25).  Three-parameter model and the standard QoIs only; per-step
 *   states are [n][ny + 1][nx + 1][2], henry_assemble's blocks
 *   [n][ny + 1][nx + 1][9][2][2] (neighbour (dj, di) at (dj + 1) 3 + di + 1).
 *   Not available in henry_adjoint and henry_level_batch_solve_static. */
enum { HENRY_SCHEME_CELL = 0, HENRY_SCHEME_VERTEX = 1 };

/* Coarse-grid operators of the multigrid hierarchy. */
enum { HENRY_COARSE_REDISCRETISE = 0, HENRY_COARSE_GALERKIN = 1 };

/* Number of QoIs per sample: [0] total salt mass sum phi rho c h^2 [kg per m
 * of depth] at T, [1] c at (1.5 m, 0.25 m) at T (mean of the 4 cells meeting
 * at that vertex). */
#define HENRY_N_QOI 2
/* Number of random inputs per sample (xi1, xi2, xi3). */
#define HENRY_N_XI 3

typedef struct henry_handle henry_handle;

/* Physics, discretisation and solver settings, SI units.  Paper values
 * (Table tab:HenryParam): E[phi] 0.35, D 18.8571e-6, K 1.020408e-9, g 9.8,
 * rho0 1000, rho1 1024.99, mu 1e-3; henry_default_config() fills the
 * configuration solved here (g 9.81, rho1 1025, Dm 1.886e-5, T 7200 s,
 * 32 x 16 cells and 20 steps at level 0). */
typedef struct {
  double Lx, Ly, T, rho0, rho1, mu, g, Dm;
  double phi_mean, K_mean, qin_mean; /* qin_mean: inflow velocity [m/s] into the domain at x = 0 */
  double phi_amp, logK_amp, qin_amp;
  int32_t nx0, ny0, steps0, max_level; /* nx0 even, ny0 divisible by 4, nx0 / ny0 = Lx / Ly */
  int32_t precision;                   /* HENRY_FP64 or HENRY_MIXED */
  int32_t coarse_op;                   /* HENRY_COARSE_REDISCRETISE or HENRY_COARSE_GALERKIN */
  double newton_atol;  /* stop when max |R| / (rho0 h^2 / tau) <= newton_atol ... */
  double newton_dxtol; /* ... or right after an update with max(|dp| / (rho0 g Ly), |dc|) <= newton_dxtol */
  double lin_rtol;     /* BiCGStab: ||r||_2 <= lin_rtol ||b||_2 per sample (default 1e-3: inexact Newton) */
  int32_t newton_maxit, lin_maxit, nu1, nu2; /* caps; pre/post smoothing sweeps of the V-cycle */
  double workspace_bytes;                    /* device workspace budget per batch (chunking) */
  double newton_predictor; /* weight w in [0, 1] of the time predictor of Newton's first iterate of step
                              n+1 (0: x^n; default 1: the full extrapolation of newton_predictor_order) */
  double newton_dc_limit;  /* Newton steps with max |dc| > limit are scaled down to it (default 1; 0: off) */
  int32_t fused_small_grids; /* grids of <= 512 cells solved by one CTA per sample with the whole hierarchy in
                                shared memory: 1 (default) in HENRY_MIXED only, 2 also in HENRY_FP64,
                                0 never (always the multi-kernel path); not used by the field models */
  int32_t coef_model;        /* HENRY_MODEL_* */
  int32_t kl_terms;          /* KL terms per field (default 32) */
  double kl_corr_len, kl_sigma_logK, kl_sigma_phi, phi_lo, phi_hi; /* 0.3 m, 0.5, 0.1, 0.05, 0.65 */
  int32_t lin_retry; /* field models: 1 (default) re-solves a failed Newton system with a V-cycle on the
                        Jacobian without density derivatives; 0 keeps the failed iterate */
  int32_t finalize_nct; /* BiCGStab dot products of samples with >= this many 256-cell blocks are reduced
                           once per sample by a separate kernel (default 512; 0: never); same values */
  double adj_rtol;   /* henry_adjoint: relative residual of each adjoint solve J^T lam = rhs (default 1e-10) */
  int32_t adj_maxit; /* henry_adjoint: BiCGStab iteration cap of each adjoint solve (default 200) */
  int32_t cuda_graphs; /* 1 (default): each BiCGStab iteration's body (two V-cycles, two matvecs, vector
                          updates) is captured once per workspace and batch size into a CUDA graph and
                          replayed; 0: plain launches.  Same values either way; off while profiling */
  int32_t qoi_set;     /* HENRY_QOI_* (default STANDARD); sets other than STANDARD use the multi-kernel path */
  int32_t tile_assembly; /* 1 (default): face-once assembly in tiles of 256 cells (whole rows up to 256 cells
                            wide, else 128 x 2 blocks), every face inside a tile evaluated once; 0: every
                            cell evaluates its four faces.  Same values up to rounding */
  int32_t newton_residual_first; /* Newton iterations with this index (0 = the step's first residual) or later
                                    evaluate the fine residual alone first and assemble the Jacobian only for
                                    the samples that do not pass the residual test (default 2: after two
                                    updates, when most samples have converged); < 0: always residual and
                                    Jacobian together.  Same values either way */
  int32_t mg_tail_cells; /* the V-cycle's coarse levels from the first one with at most this many cells per
                            sample down to the coarsest run as one kernel, one CTA per sample with those
                            levels' vectors in shared memory, and their operators too where they fit beside
                            them (the finest tail levels' operators are otherwise read from global memory at
                            each use); -1 (default): 2048 cells (64 x 32) with FP32 linear algebra on fine grids
                            of 128 x 64 cells or more, else 128 (16 x 8), the faster choice measured on the
                            MLMC levels' batches; 0: every level as separate kernels.  Same values either
                            way */
  int32_t mg_tail_batch_cells; /* ... only while the batch times that level's cells per sample is at most this
                                  (default 2^20; 0: no limit): large batches of small grids run those levels
                                  as separate, large launches */
  int32_t scheme; /* HENRY_SCHEME_CELL (default) or HENRY_SCHEME_VERTEX */
  int32_t newton_jacobian_every; /* Newton assembles the Jacobian and the coarse operators at
                                    iterations 0, k, 2k, ... of a time step and reuses them in between (chord
                                    Newton; k = 1, the default: every iteration).  The FP64 residual test
                                    decides convergence either way, so the converged states agree to it */
  int32_t level_priority; /* henry_batch_solve_mixed: 1 (default) runs finer levels on higher-priority
                             streams (their solves are the pass's critical path); 0: equal priorities.
                             Fixed when a level's stream is first created.  Same values either way */
  int32_t assembly_tile_w; /* face-once assembly tiles: 0 (default) whole rows up to 256 cells wide, else
                              128 x 2; 32, 64, 128 or 256: tiles of that many cells x 256 / width rows on
                              every grid whose width and height they divide (the default elsewhere).
                              Every shape evaluates each face with the same source arithmetic: F is
                              bit-identical, Jacobian entries may differ in the last bit (the compiler
                              contracts multiply-adds per call site, and tile-edge faces are evaluated
                              at another call site) */
  int32_t mg_threads; /* threads per CTA of the multigrid smoother, restriction and prolongation kernels of
                         the cell-centred scheme: 64, 128, 256 or 512 (0, the default: 256).  Identical
                         values for every size */
  int32_t newton_predictor_order; /* Newton's first iterate of step n+1 (with weight newton_predictor): 1
                                     linear extrapolation from x^n and x^{n-1}; 2 (default) quadratic, x^n +
                                     w (2 (x^n - x^{n-1}) - (x^{n-1} - x^{n-2})), from step 2 on (linear at
                                     step 1).  Every solve path and henry_adjoint (whose checkpoints then hold
                                     three states) follow it.  The FP64 residual test decides convergence
                                     either way */
} henry_config;

/* Iteration statistics of one henry_level_batch_solve call (host struct). */
typedef struct {
  int64_t newton_iters; /* Newton iterations summed over samples and steps (fine + coarse) */
  int64_t linear_iters; /* BiCGStab iterations summed over samples and Newton iterations */
  int64_t newton_solves; /* Newton solves (samples x steps) */
  int64_t failed_samples;
  double cell_steps; /* sum over solved scenarios of cells x steps (coarse partners included) */
} henry_stats;

/* Fill *cfg with the defaults described above.  Never fails. */
void henry_default_config(henry_config* cfg);

/* The defaults changed to the paper's variant of the problem (Table
 * tab:HenryParam and Sec. 4): g = 9.8, rho1 = 1024.99, Dm = 18.8571e-6, K_mean
 * = 1.020408e-9, T = 6016 s in steps0 = 188 steps (tau = 32 s at level 0),
 * the two-layer porosity with Kozeny-Carman K, recharge amplitude 0.5 and the
 * paper's QoIs (HENRY_QOI_PAPER).  Never fails. */
void henry_paper_config(henry_config* cfg);

/* Project autotuner.  Solver settings that change only how fast a solve
 * converges, never where (the FP64 Newton test decides): the Krylov tolerance,
 * the V-cycle's smoothing counts and, where the level's grid allows it, the
 * fused one-CTA-per-sample solver; then, one at a time from the best so far,
 * the fused multigrid tail (mg_tail_cells in {0, 32, 128, 512, 2048}), the
 * residual-first Newton test (newton_residual_first in {-1, 2, 3, 4}), chord
 * Newton (newton_jacobian_every in {1, 2, 3}), the assembly tile
 * (assembly_tile_w in {0, 32, 64, 128, 256} where it divides the grid), the
 * multigrid kernels' CTA size (mg_threads in {64, 128, 256, 512}) and the
 * order of Newton's time predictor (newton_predictor_order in {1, 2}).
 * henry_autotune times every candidate - first lin_rtol in {1e-4, 1e-3,
 * 1e-2} x (nu1, nu2) in {(2,2), (1,2), (2,1)} x (fused small-grid solver on /
 * off where eligible), then the later stages - on n_trial samples
 * xi_dev[n_trial][n_xi] of `level` (with their coarse partners if
 * with_coarse), after one untimed warm-up, with CUDA events on `stream`, and
 * keeps the fastest candidate that solves every sample for that level of
 * this handle: henry_level_batch_solve and henry_batch_solve_mixed use it from
 * then on (henry_adjoint keeps the configuration's settings).  QoIs move only
 * within the Newton tolerance.  Allocates its trial outputs; synchronises
 * `stream`.  best_out (nullable) receives the choice with its measured rate.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOCONV (no candidate solved every sample);
 * after an error the level keeps the settings it had before the call. */
typedef struct {
  double lin_rtol;
  int32_t nu1, nu2, fused_small_grids;
  double cell_steps_per_s; /* measured on the trial batch (0 for the configuration's own settings) */
  int32_t mg_tail_cells, newton_residual_first, newton_jacobian_every; /* as in henry_config */
  int32_t assembly_tile_w, mg_threads;                                 /* as in henry_config */
  int32_t newton_predictor_order; /* as in henry_config (0: the configuration's) */
} henry_tuning;
int henry_autotune(henry_handle* h, int level, int with_coarse, const double* xi_dev, int n_trial,
                   henry_tuning* best_out, void* stream);
/* The settings a level's solves use: henry_autotune's choice, else the configuration's. */
int henry_get_tuning(henry_handle* h, int level, henry_tuning* out);
/* Give a level these settings (for example another handle's henry_autotune
 * choice); NULL returns the level to the configuration's.  EINVAL on bad values. */
int henry_set_tuning(henry_handle* h, int level, const henry_tuning* t);

/* The KL basis of HENRY_MODEL_KL for cfg (kl_terms, kl_corr_len, Lx, Ly): the
 * square roots of the eigenvalues, sqrt_lam[kl_terms], and, if modes is not
 * NULL, the modes psi_t at the cell centres of `level`, modes[kl_terms][ny][nx]
 * (row-major), so that log K = log K_mean + sigma_K sum_t sqrt_lam[t] theta_K[t]
 * psi_t (and likewise phi before its clip).  Use it to turn henry_adjoint's
 * dQ/dtheta into fields.  The same host computation as the solves' (Nystrom
 * on 256 Gauss-Legendre nodes, cyclic Jacobi).  Host only, no GPU; EINVAL on
 * NULL or bad settings. */
int henry_kl_basis(const henry_config* cfg, int level, double* sqrt_lam, double* modes);

/* QoIs per sample for cfg's qoi_set (2, 15, 15 + nx0 ny0 or 15 + steps0); -HENRY_EINVAL for a
 * NULL pointer or an unknown set. */
int henry_n_qoi(const henry_config* cfg);

/* Create a handle for `cfg` (copied).  Allocates no device memory yet.
 * Errors: EINVAL on a NULL pointer, inconsistent grid sizes (nx0 = 2 ny0 with
 * ny0 a power of two >= 4, Lx = 2 Ly, max_level in [0, 8]), a finest level
 * past 2^30 cells per sample or 2^30 time steps, an unknown enum value, a
 * floating-point setting that is NaN or infinite, a non-positive physical
 * constant (Lx, Ly, T, rho0, rho1, mu, g, Dm, K_mean; 0 < phi_mean < 1) or
 * non-positive solver settings. */
int henry_create(const henry_config* cfg, henry_handle** out);

/* Free the handle and its device workspace (synchronises the device).
 * NULL is ignored. */
void henry_destroy(henry_handle* h);

/* Message of the last error on this thread ("" if none). */
const char* henry_last_error(void);

/* a1. Sample xi[n][3] (the UNIFORM3 and TWO_LAYER inputs) for samples first_sample .. first_sample + n - 1 of
 * MLMC level `level` with Philox4x32-10 (Salmon et al., SC'11) keyed by the
 * two 32-bit halves of `seed`; sample s uses counters (level, lo32(s),
 * hi32(s), 0) -> xi1 from words (0,1), xi2 from words (2,3) and (level,
 * lo32(s), hi32(s), 1) -> xi3 from words (0,1); two words (w0, w1) map
 * exactly to (2 u + 1 - 2^52) 2^-52 with u = (w0 << 20) | (w1 >> 12), a value
 * in (-1, 1).  The paper draws xi iid uniform on [-1, 1] (Sec. 4). */
int henry_sample_xi(uint64_t seed, int level, uint64_t first_sample, int n, double* xi_dev, void* stream);

/* a2-a11. Solve n scenarios at MLMC level `level` (0 <= level <= max_level)
 * for inputs xi_dev[n][n_xi] (n_xi = 3, or 2 kl_terms + 1 for HENRY_MODEL_KL) and write the QoIs at T to qoi_fine_dev[n][n_qoi] (n_qoi = henry_n_qoi).
 * If with_coarse != 0 (level >= 1) also solve the same xi on level - 1 (the
 * coarse partner of the telescoping difference, Eq. (A): same xi, grid and
 * time step of the coarser level) into qoi_coarse_dev[n][n_qoi].
 * status_dev[n] (int32) receives HENRY_SAMPLE_* (worst over fine and coarse).
 * stats_host may be NULL.  Synchronises `stream`.  Returns HENRY_ENOCONV if
 * any sample failed (its QoIs are then unspecified). */
int henry_level_batch_solve(henry_handle* h, int level, int with_coarse, const double* xi_dev, int n,
                            double* qoi_fine_dev, double* qoi_coarse_dev, int32_t* status_dev,
                            henry_stats* stats_host, void* stream);

/* a2-a11 over an uneven batch (samples at several MLMC levels in one call,
 * the situation of an MLMC pass, Sec. 3: each level l needs m_l samples of
 * Y_l, Eq. (A)).  Sample i is solved at level levels_host[i] (host array,
 * 0 <= level <= max_level, any order) with inputs xi_dev[i][n_xi]; its QoIs go
 * to qoi_fine_dev[i][n_qoi] and, when with_coarse != 0, those of its coarse partner
 * (level - 1, same xi) to qoi_coarse_dev[i][n_qoi] (zeros for level-0 samples).
 * status_dev[i] as in henry_level_batch_solve.  The levels run concurrently:
 * each on its own child handle (created on first use, same configuration,
 * its own workspace), CUDA stream and host thread, forked from `stream` by an
 * event; samples not already in level order are gathered into level order
 * and their results scattered back.  Results are bit-identical to
 * henry_level_batch_solve on the same samples.  stats_host (nullable) sums
 * over levels.  Synchronises `stream`.  Errors: EINVAL (NULL pointer, n <= 0,
 * a level out of range), ENOMEM, ECUDA, ENOCONV as in henry_level_batch_solve
 * (the first failing level's message for the others). */
int henry_batch_solve_mixed(henry_handle* h, const int32_t* levels_host, int n, int with_coarse,
                            const double* xi_dev, double* qoi_fine_dev, double* qoi_coarse_dev, int32_t* status_dev,
                            henry_stats* stats_host, void* stream);

/* Discrete adjoint (dQ/dtheta of the implicit-Euler solve of Sec. 2.3; the
 * gradients the paper's future work on parameter identification needs,
 * Sec. 5).  For each of the n samples, inputs xi_dev[n][n_xi] as in
 * henry_level_batch_solve and weights qoi_weights_dev[n][2], Q = w0 salt mass +
 * w1 c(1.5, 0.25) at T; writes grad_dev[n][n_xi] = dQ/dxi (three-parameter
 * and two-layer models: d/d(xi1, xi2, xi3); KL: d/d(theta_K[terms],
 * theta_phi[terms], xi3)), qoi_dev[n][n_qoi] (the forward QoIs; the weights act on the first two, the standard QoIs; the same values as
 * henry_level_batch_solve) and status_dev[n] (HENRY_SAMPLE_*; 2: an adjoint
 * solve did not converge).  Always computed in FP64, whatever `precision`.
 * The forward keeps the state pair every checkpoint_every steps (>= 1; values
 * above the step count keep every state) and recomputes each segment's states
 * in the backward sweep; each step's adjoint system J_m^T lam_m = rhs is solved
 * by BiCGStab preconditioned by the V-cycle of the transposed hierarchy, to
 * adj_rtol.  Device workspace: the level's FP64 group plus (2 ceil(steps /
 * checkpoint_every) + checkpoint_every + 1) x 16 B + 64 B per cell and sample,
 * within workspace_bytes (larger batches are chunked).  Synchronises `stream`.
 * Errors: EINVAL (NULL pointer, n <= 0, level out of range, checkpoint_every <=
 * 0), ENOMEM, ECUDA, ENOCONV (>= 1 sample failed; see status_dev). */
int henry_adjoint(henry_handle* h, int level, const double* xi_dev, int n, const double* qoi_weights_dev,
                  double* grad_dev, double* qoi_dev, int checkpoint_every, int32_t* status_dev, void* stream);

/* a12. Merge one batch of level-`level` samples into running MLMC sums.
 * Y = qoi_fine - qoi_coarse (qoi_coarse_dev NULL: Y = qoi_fine, level 0), the
 * level term of the telescoping sum Eq. (EgL) / Def. (Yell).  Samples with
 * status_dev[i] != 0 are skipped (status_dev may be NULL: all used).
 * sums_dev[2][n_qoi][3] holds (count, mean, M2) with M2 the centred sum of
 * squares; [0] for Y and [1] for qoi_fine itself; it is read and updated in
 * place (zero it before the first batch).  The batch's moments are formed in
 * one block on the device and merged with Chan's pairwise update.  `level` is
 * only checked (>= 0).  Asynchronous on `stream`. */
int mlmc_accumulate(int level, int n, int n_qoi, const double* qoi_fine_dev, const double* qoi_coarse_dev,
                    const int32_t* status_dev, double* sums_dev, void* stream);

/* a13. Eq. (M_ell): m_l = ceil(var_budget^-1 sqrt(V_l / s_l) sum_i sqrt(V_i s_i))
 * for l = 0 .. n_levels - 1 (host arrays; V_l >= 0, s_l > 0, var_budget > 0).
 * Levels with V_l = 0 get m_l = 0.  Host only, synchronous. */
int mlmc_allocate(int n_levels, const double* V_host, const double* s_host, double var_budget, int64_t* m_out_host);

/* Rates of Theorem (costMLMC), estimated from per-level statistics as the
 * paper does from its preliminary runs (Sec. 3; the slopes of Fig.
 * weak_strong): least-squares slopes over levels first_level .. n_levels - 1
 * of log2 |mean_Y_l| (alpha = -slope, weak rate of Eq. weak_error_model),
 * log2 V_l (beta = -slope, Eq. strong_error_model) and log2 s_l (gamma_d =
 * d gamma = +slope, cost growth).  Host arrays indexed by level; any output
 * pointer may be NULL (that rate is skipped, its input may then be NULL).
 * Errors: EINVAL with fewer than two levels, or a zero / non-finite value
 * (negative V_l or s_l).  Host only, synchronous. */
int mlmc_rates(int n_levels, int first_level, const double* mean_Y_host, const double* V_host,
               const double* s_host, double* alpha, double* beta, double* gamma_d);

/* Bias test for adding levels (Eq. MSE asks (E[g_L - g])^2 <= eps^2 / 2):
 * with the weak error model |E[g_l - g]| ~ c 2^-alpha l the remaining bias is
 * the geometric tail E[Y_L] / (2^alpha - 1), so *bias_est = |mean_Y[L]| /
 * (2^alpha - 1), L = n_levels - 1, and *converged = (bias_est <= eps /
 * sqrt 2).  Either output may be NULL.  Errors: EINVAL (n_levels < 2, alpha
 * or eps <= 0, non-finite mean).  Host only, synchronous. */
int mlmc_bias_test(int n_levels, const double* mean_Y_host, double alpha, double eps, double* bias_est,
                   int32_t* converged);

/* The same bias test with E[Y_L] from the fitted weak error model rather
 * than the level-L sample mean alone (on the finest levels that mean rests
 * on a handful of samples and its noise decides the test): log2 |mean_Y_l|
 * = a - alpha l fitted by least squares over l = first_level .. L (L =
 * n_levels - 1); alpha = max(fitted slope, alpha_min) (*alpha_out), a
 * refitted for that alpha; *bias_est = 2^(a - alpha L) / (2^alpha - 1);
 * *converged = (bias_est <= eps / sqrt 2).  Outputs may be NULL.  Errors:
 * EINVAL (fewer than two levels from first_level, a zero or non-finite
 * mean, alpha_min or eps <= 0).  Host only, synchronous. */
int mlmc_bias_test_fit(int n_levels, int first_level, const double* mean_Y_host, double alpha_min, double eps,
                       double* alpha_out, double* bias_est, int32_t* converged);

/* ---- Per-step entry points: one step of the solve on given states, for
 * checking each step on its own.  Each evaluates the coefficients of
 * xi_dev[n][3] at `level` and takes the current and previous-time-step states
 * state_dev, state_old_dev ([n][ny][nx][2]).  Residuals and Jacobians are
 * scaled by 1 / (rho0 h^2 / tau) of that level.  Asynchronous on `stream`. */

/* a4. F_dev[n][ny][nx][2] = scaled residual (fluid mass, salt mass) and, if
 * J_dev is not NULL, J_dev[n][ny][nx][5][2][2] = scaled Jacobian blocks
 * (J_dev NULL: the residual alone, by the residual-only kernel of the Newton
 * test, bit-identical to the residual assembled with the Jacobian)
 * coupling each cell to (self, west, east, south, north) neighbour; block
 * [eq][var], eq 0 = fluid mass, 1 = salt; var 0 = p, 1 = c; zero across the
 * domain boundary.  In HENRY_MIXED the blocks are the FP32 copy the solver
 * uses, widened to FP64. */
int henry_assemble(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                   const double* state_old_dev, double* F_dev, double* J_dev, void* stream);

/* a8. y_dev = J x_dev with J the scaled Jacobian at the given states; x, y
 * are [n][ny][nx][2]. */
int henry_apply_jacobian(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                         const double* state_old_dev, const double* x_dev, double* y_dev, void* stream);

/* a5 + a7. z_dev = one V(nu1, nu2) cycle applied to b_dev from a zero
 * initial guess, on the hierarchy built at the given states; b, z are
 * [n][ny][nx][2]. */
int henry_precondition(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                       const double* state_old_dev, const double* b_dev, double* z_dev, void* stream);

/* a6. x_dev = BiCGStab solution of J x = b_dev to lin_rtol (right-
 * preconditioned by the V-cycle, from x = 0); iters_dev[n] (int32, may be
 * NULL) receives the iteration counts (-1: not converged within lin_maxit).
 * Synchronises `stream`. */
int henry_linear_solve(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                       const double* state_old_dev, const double* b_dev, double* x_dev, int32_t* iters_dev,
                       void* stream);

/* a4 of the paper's own vertex-centred scheme (Sec. 2.3: two unknowns per
 * grid vertex, n_l = 2 (nx+1)(ny+1) as in Table tab:adaptiveTS_times, a
 * "consistent velocity" and partial upwinding; the readings are stated in
 * henry_vc.cuh).  Three-parameter model only (EINVAL otherwise).
 * state_dev, state_old_dev: [n][ny+1][nx+1][2] (p, c) at the vertices of
 * `level` (nx = nx0 2^level, ny = ny0 2^level), natural order.
 * R_dev[n][ny+1][nx+1][2] receives the unscaled residuals (fluid, salt), with
 * the Dirichlet vertices' equations (x = Lx: p and c; x = 0: c) replaced by
 * (value - boundary value) x rho0 h^2 / tau (p in units of rho0 g Ly).
 * J_dev (may be NULL) receives [n][ny+1][nx+1][3][3][2][2]: for each vertex
 * the 2x2 blocks d(R^m, R^s)/d(p, c) of the vertices (j+dj, i+di),
 * dj, di in {-1, 0, 1} (zero outside the grid).  The coefficients are
 * checked first: a sample whose xi gives phi outside (0, 1) or a non-finite
 * K or q_in makes the call return HENRY_EINVAL, naming the first such sample,
 * with nothing assembled.  Synchronises `stream` for that check (a
 * stream-ordered scratch of n x 36 + 4 bytes). */
int henry_vc_assemble(henry_handle* h, int level, const double* xi_dev, int n, const double* state_dev,
                      const double* state_old_dev, double* R_dev, double* J_dev, void* stream);

/* ---- Allocation-free variant of henry_level_batch_solve (the paper has no
 * counterpart: this is a deployment aid).  For callers that cannot call
 * cudaMalloc at run time - processes whose device memory is owned by another
 * allocator or pool, plug-ins that must not grow their footprint after load -
 * it solves the same batch with the same kernels but takes its whole
 * workspace from one device array of HENRY_STATIC_SCRATCH_BYTES compiled into
 * the library (held by every GPU that loads it until the process exits); it
 * makes no device or pinned allocation and needs no handle (cfg is read, as
 * in henry_create).  The caller passes inputs and outputs as for
 * henry_level_batch_solve (without stats).  The workspace of n samples at
 * `level` (plus that of the coarse partners) must fit in the array - with the
 * default configuration up to 64 level-0 samples in FP64 - otherwise
 * HENRY_EINVAL with a message giving the sizes.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress with that
 * device current), a set-up step: make that first call before any stream
 * capture begins.  All
 * calls share the array and host counter words; calls that overlap on the GPU
 * or across host threads race.  Only the three-parameter model and the two
 * standard QoIs (qoi_set 0) are accepted (HENRY_EINVAL otherwise).
 * Synchronises `stream`. */
#define HENRY_STATIC_SCRATCH_BYTES (16u << 20)
int henry_level_batch_solve_static(const henry_config* cfg, int level, int with_coarse, const double* xi_dev, int n,
                                   double* qoi_fine_dev, double* qoi_coarse_dev, int32_t* status_dev, void* stream);

/* ---- Kernel timing.  Classes of kernels whose launches the timer brackets
 * with CUDA events on the launching stream. */
enum {
  HENRY_K_ASSEMBLE = 0,          /* a4: fine-grid residual + Jacobian */
  HENRY_K_COARSE_OPS = 1,        /* a5: coarse operators (rediscretised or Galerkin) + coarsest inverse */
  HENRY_K_STATE_RESTRICT = 2,    /* a5: 2x2 averages of the state for rediscretisation */
  HENRY_K_SMOOTH = 3,            /* a7: red-black block Gauss-Seidel half-sweeps on the solve's fine grid */
  HENRY_K_RESIDUAL_RESTRICT = 4, /* a7: residual + restriction (and x += P x_c without post-smoothing) */
  HENRY_K_COARSE_SOLVE = 5,      /* a7: 4x4 solve on the 2 x 1 grid */
  HENRY_K_SPMV = 6,              /* a8: y = J x with dot products */
  HENRY_K_KRYLOV = 7,            /* a6: BiCGStab vector updates and reductions */
  HENRY_K_NEWTON = 8,            /* a9, a10: Newton update, tests, step start */
  HENRY_K_QOI = 9,               /* a2, a3, a11: coefficients, initial state, QoIs */
  HENRY_K_FUSED = 10,            /* a3-a11 for a small grid: the one-CTA-per-sample solver */
  HENRY_K_SMOOTH_COARSE = 11,    /* a7: the same half-sweeps on the coarser multigrid levels */
  HENRY_K_RESIDUAL = 12,         /* a4: fine-grid residual alone (the Newton test before a Jacobian is needed) */
  HENRY_K_MG_TAIL = 13,          /* a7: the fused V-cycle below mg_tail_cells (sweeps, restrictions, coarsest
                                    solve of those levels in one kernel) */
  HENRY_K_COUNT = 14
};

/* Start (enable != 0: counters reset) or stop timing on this handle.  While
 * on, each launch of the solver's kernels is bracketed by two CUDA events
 * (which adds host overhead; time the workload with it off).  Host only. */
int henry_profile(henry_handle* h, int enable);

/* Per class since the last reset: summed event time [ms], launches, the
 * algorithmic (compulsory) DRAM bytes of those launches - every array a kernel
 * touches counted once per launch, for the samples still iterating - and the
 * algorithmic floating-point operations (FMA = 2) of the block-stencil
 * classes (smooth, residual_restrict, spmv; 0 for the others).  Synchronises
 * the device if events are pending.  Any output may be NULL. */
int henry_profile_read(henry_handle* h, int kclass, double* total_ms, int64_t* launches, double* alg_bytes,
                       double* alg_flops);

#ifdef __cplusplus
}
#endif

#endif /* HENRY_H */
