/*
 * qpfrg.h -- C ABI of the GB300 (sm_103a) quasi-particle fRG flow library.
 *
 * Method: D. Rohe and C. Honerkamp, "Quasi-particle functional
 * Renormalisation Group calculations in the two-dimensional half-filled
 * Hubbard model at finite temperatures", arXiv:2005.00827.
 *
 *   model        H of Eq. (model_definition), xi_k of Eq. (free_dispersion_xi)
 *   vertex flow  one-loop dV = sum V G S V, App. A.1 Eq. (vertex_flow_general),
 *                static SU(2) coupling V(k1,k2,k3) (App. A, "static
 *                components"), quasi-particle lines of Eq. (both_propagators_Z)
 *                and Eq. (vertex_flow_feedback_Z)
 *   self-energy  real-frequency two-loop term (Sec. 2.2, App. A.2/A.3), Z from
 *                Eq. (definition_Z) with the slope taken "from outside" over
 *                +-2T (Sec. 3.1.1, Fig. 2 caption), projected on the Fermi
 *                surface patch (Sec. A.3)
 *   flow         integrated until the largest coupling passes a bound
 *                (Sec. 3.2, scale U*(T) / T*(U))
 *
 * Conventions shared by every call:
 *   - Patches j = 0..N-1.  Wedge mode: angular wedges about the origin with
 *     centres at theta_j = 2 pi j / N (N a multiple of 4); patch
 *     representative k_F(j) on the Fermi surface along theta_j; a fine loop
 *     grid of n_theta x n_r points per wedge (n_r even: half inside, half
 *     outside the Fermi surface).  Lattice mode: all L x L momenta
 *     2 pi (m1, m2)/L are patches (N = L*L, one loop point each, index
 *     m1*L + m2): the exact finite-lattice one-loop flow, for tests.
 *   - The coupling V is FP64, row-major V[k1][k2][k3], N^3 entries; k1 -> k3
 *     carries spin s, k2 -> k4 = k1 + k2 - k3 carries spin s'.
 *   - Z is FP64, one weight per patch.  Sigma is FP64, row-major [j][m]
 *     over the real-frequency grid omega_m = linspace(omega_min, omega_max,
 *     n_omega) (inclusive).
 *   - Pointers named d_* are DEVICE pointers owned by the caller; they must
 *     stay valid until the work enqueued by the call has completed.  h_*
 *     pointers are host memory owned by the caller.  All device work is
 *     enqueued on the CUDA stream given to qpfrg_create.
 *   - Every call returns a qpfrg_status.  The text of the last error of a
 *     context is available from qpfrg_last_error.  There is no host fallback:
 *     without a CUDA device every compute call fails with QPFRG_ERR_CUDA.
 *   - A context is not thread-safe; calls on one context must be serialised.
 */
#ifndef QPFRG_H
#define QPFRG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qpfrg_ctx *qpfrg_t;      /* opaque; created and owned by the library */

typedef enum {
    QPFRG_OK = 0,
    QPFRG_ERR_INVALID = -1,      /* bad argument; nothing was enqueued          */
    QPFRG_ERR_CUDA = -2,         /* a CUDA call failed (no device, launch error) */
    QPFRG_ERR_OOM = -3,          /* device or host allocation failed            */
    QPFRG_ERR_UNSUPPORTED = -4,  /* valid request this build does not implement */
    QPFRG_ERR_TIMEOUT = -5,      /* a bounded wait or wall-clock budget ran out  */
    QPFRG_ERR_NONFINITE = -6     /* NaN/Inf met in an input or in the state      */
} qpfrg_status;

typedef enum {
    QPFRG_REG_TEMPERATURE = 0,   /* Lambda = T: dV/dT with T-derivative loop kernels   */
    QPFRG_REG_INTERACTION = 1    /* Lambda = g: G = g Z G0, S = Z^2 G0 at fixed T (App. A) */
} qpfrg_regulator;

typedef enum {
    QPFRG_FP64 = 0,              /* every step in FP64                                */
    QPFRG_MIXED = 1,             /* FP32 loop kernels and contraction, FP64 ODE state  */
    QPFRG_MIXED_TC = 2           /* as MIXED, contraction on tcgen05 tensor cores with
                                    BF16 hi/lo split products (hi*hi + hi*lo + lo*hi) and
                                    FP32 accumulation; needs n_p^2 % 8 == 0                */
} qpfrg_precision;

typedef enum {
    QPFRG_PROP_PAPER = 0,        /* G = Z/(iw - xi): Z a prefactor, Eq. (both_propagators_Z) */
    QPFRG_PROP_QP = 1            /* G = Z/(iw - Z xi): Z also renormalises the pole          */
} qpfrg_propagator;

enum { QPFRG_CH_PP = 1, QPFRG_CH_CR = 2, QPFRG_CH_D = 4, QPFRG_CH_ALL = 7 };

/* Patch geometry (Sec. 3.2 gives only patch counts):
 *   WEDGE   -- n_p angular wedges about the origin, representatives on the Fermi
 *              surface along the wedge centres, polar fine grid per wedge;
 *   LATTICE -- the n_p = L*L momenta of an L x L lattice (exact finite-lattice sums);
 *   SHELL   -- (angle, energy) patches, Sec. 3.2's "7 shells in the energy direction
 *              and 32 angular sections": n_p / n_shell wedges (a multiple of 4),
 *              each cut into n_shell (odd) energy shells of width shell_width centred
 *              on the Fermi surface (outer shells reach the band edges), patch
 *              j = wedge * n_shell + shell; representatives on the wedge's centre ray
 *              at the shell's middle energy (k_F for the Fermi shell; the ray's zone-
 *              edge point where the band ends below that energy); n_shell = 1 is WEDGE. */
typedef enum { QPFRG_GRID_WEDGE = 0, QPFRG_GRID_LATTICE = 1, QPFRG_GRID_SHELL = 2 } qpfrg_grid_mode;

typedef enum {
    QPFRG_FLOW_RUNNING = 0,      /* neither bound nor end reached yet            */
    QPFRG_FLOW_REACHED_END = 1,  /* Lambda reached lambda_end                    */
    QPFRG_FLOW_DIVERGED = 2,     /* max|V| passed stop_abs_v (strong coupling)   */
    QPFRG_FLOW_NONFINITE = 3,    /* NaN/Inf in V or Z                            */
    QPFRG_FLOW_Z_OUT_OF_RANGE = 4,/* Z left (0, z_max]                           */
    QPFRG_FLOW_MAX_STEPS = 5,    /* max_steps completed                          */
    QPFRG_FLOW_TIMEOUT = 6       /* wall-clock budget of qpfrg_flow ran out      */
} qpfrg_flow_status;

typedef struct { double t, tp, mu; } qpfrg_lattice;   /* Eq. (free_dispersion_xi) */

typedef struct {
    int n_theta;                 /* angular fine points per wedge (>= 1)               */
    int n_r;                     /* radial fine points per wedge (even, >= 2)          */
    int mode;                    /* qpfrg_grid_mode                                    */
    int n_shell;                 /* SHELL: energy shells per wedge (odd >= 1; else ignored) */
    double shell_width;          /* SHELL: energy width of a shell; <= 0: the band width
                                    2 max|xi| over n_shell                               */
} qpfrg_fine_grid;

typedef struct {
    unsigned channel_mask;       /* OR of QPFRG_CH_*; pp off = particle-hole-only flow (Sec. 3.2) */
    int z_feedback;              /* recompute Z from Sigma once per flow step          */
    int propagator;              /* qpfrg_propagator                                   */
    int precision;               /* qpfrg_precision                                    */
    double eta;                  /* Lorentzian broadening of the retarded Sigma        */
    int n_omega;                 /* real-frequency grid of qpfrg_selfenergy (0: none)  */
    double omega_min, omega_max;
    double stop_abs_v;           /* divergence bound on max|V| (default 20 t)          */
    double step;                 /* T-flow: d ln T per step (<0); g-flow: dg (>0)      */
    double lambda_end;           /* end of the flow: T_end or g_end                    */
    double z_max;                /* Z outside (0, z_max] stops the flow                */
    int max_steps;               /* bound on flow steps per qpfrg_flow call            */
    double T_fixed;              /* temperature of the interaction flow                */
    double timeout_s;            /* wall-clock budget of one qpfrg_flow call (<=0: none) */
    int autotune;                /* qpfrg_flow_batch: nonzero tunes the launch shapes of
                                    each patch-count group (qpfrg_autotune) before stepping */
    int no_loop_symmetry;        /* 0: C4v reductions on (wedge and shell modes): one
                                    loop-kernel row per orbit of (transfer, patch), and
                                    with QPFRG_MIXED_TC and a C4v-symmetric V and Z one
                                    contraction row per orbit of transfers, expanded;
                                    2: the loop-kernel orbits only; other nonzero: every
                                    loop-kernel row and every contraction row evaluated */
    /* interaction flow only: the self-energy ODE of App. A.2-A.5 (state V,
       Sigma, Sigma'; see qpfrg_read_sigma_flow) */
    int sigma_ode;               /* nonzero: carry Sigma, Sigma' and feed Z (z_feedback) */
    int katanin;                 /* nonzero: Katanin factor K on the S lines (App. A.5)  */
    int a_mode;                  /* 0: patch average of A, 1: its minimum, 2: its maximum
                                    (the bracket flows of App. B), 3: one-loop term dropped */
    int sigma_table;             /* >= 0: the FP32 wedge self-energy of a C4v-symmetric state
                                    reads the patch of r = k + p - q from a table built on
                                    first use (N_irr M^2 bytes: 126 GB at N_p = 96, 32 x 32),
                                    when it fits in 60 % of the free device memory; < 0: it
                                    decides every patch per pair.  Same sums either way. */
} qpfrg_options;

typedef struct {
    int status;                  /* qpfrg_flow_status                                  */
    int steps;                   /* RK4 steps completed since creation / set_state      */
    double lambda;               /* flow parameter now (T or g)                         */
    double lambda_c;             /* interpolated crossing of stop_abs_v (DIVERGED only) */
    double max_abs_v;            /* max|V| of the current state                         */
} qpfrg_flow_result;

/* Fill *o with the defaults: all channels, no Z feedback, PAPER propagators,
 * FP64, eta 0.02, no omega grid (range [-4, 4]), stop_abs_v 20, step ln 0.98,
 * lambda_end 0.05, z_max 2, max_steps 100000, T_fixed 0.1, no timeout. */
void qpfrg_default_options(qpfrg_options *o);

/* Create a context: builds the patch geometry (FP64, on the host), uploads
 * the fine-point tables, computes the partner-patch maps proj(Q - p) and
 * proj(p + Q) for every transfer Q = k_F(x) +- k_F(y) and fine point p on the
 * device (FP64), and sets the flow state to V = U, Z = 1 at Lambda = lambda0
 * (Sec. 3.2: the flow starts from the bare Hubbard coupling).
 * n_p: number of patches (wedge: multiple of 4, <= 256; lattice: L*L <= 256).
 * cuda_stream: cudaStream_t (NULL = legacy default stream).
 * Errors: QPFRG_ERR_INVALID for bad parameters, QPFRG_ERR_OOM, QPFRG_ERR_CUDA,
 * QPFRG_ERR_UNSUPPORTED (e.g. more than 2048 fine points per wedge).
 * On error *out is NULL. */
qpfrg_status qpfrg_create(const qpfrg_lattice *lattice, int n_p, const qpfrg_fine_grid *grid,
                          double U, double lambda0, qpfrg_regulator regulator,
                          const qpfrg_options *options, void *cuda_stream, qpfrg_t *out);

/* One evaluation of the one-loop right-hand side dV/dLambda (App. A.1,
 * Eq. (vertex_flow_general); Eq. (vertex_flow_feedback_Z) with Z):
 *   pp : Q = k1+k2, dV -= sum_p L'_pp(p,Q-p) V(k1,k2,p) V(p,Q-p,k3)
 *   cr : Q = k3-k2, dV -= sum_p L'_ph(p,p+Q) V(k1,p,p+Q) V(p+Q,k2,k3)
 *   d  : Q = k1-k3, dV += sum_p L'_ph(p,p+Q) [2V(k1,p,k3)V(p+Q,k2,p)
 *                          - V(p,k1,k3)V(p+Q,k2,p) - V(k1,p,k3)V(k2,p+Q,p)]
 * p runs over the fine points, vertex arguments are patches.  L' is Z_a Z_b
 * dL/dT (T-flow) or g Z_a Z_b (Z_a + Z_b) L (g-flow).
 * d_V: N^3 FP64 input, d_Z: N FP64 input (NULL = all ones), d_dV: N^3 FP64
 * output (may not alias d_V).  lambda = T (T-flow, > 0) or g (g-flow).
 * Uses the context's precision.  The context's flow state is not changed.
 * With QPFRG_MIXED_TC and the contraction's row orbits available (see
 * qpfrg_rhs_work) the call first tests V and Z for C4v symmetry on the device
 * (1e-12 of max|V|, max|Z|) and waits for that test on the context's stream:
 * a symmetric input contracts one row per orbit of transfer pairs, any other
 * every row.  Otherwise the work is only enqueued. */
qpfrg_status qpfrg_rhs(qpfrg_t ctx, double lambda, const double *d_V, const double *d_Z,
                       double *d_dV);

/* Real-frequency two-loop self-energy at the patch representatives for the
 * vertex d_V and weights d_Z at temperature T (T-flow: T = lambda):
 *   Sigma(k_j, w) = sum_{p,q} w_p w_q Z_a Z_b Z_c W F / (w + i eta - E),
 *   r = k_j + p - q, E = xi_q + xi_r - xi_p,
 *   F = f_p(1-f_q)(1-f_r) + (1-f_p) f_q f_r,
 *   W = 2 V(k_j,p,q)^2 - V(k_j,p,q) V(k_j,p,r),
 * and Z_j = 1/(1 - [Re Sigma(xi_j+2T) - Re Sigma(xi_j-2T)]/(4T)).
 * d_sigma_re/d_sigma_im: N x n_omega FP64 outputs (may be NULL when
 * n_omega == 0; the frequency grid is binned, see the design notes);
 * d_Z_out: N FP64 output (may be NULL).  Regulator must be TEMPERATURE
 * (QPFRG_ERR_UNSUPPORTED otherwise). */
qpfrg_status qpfrg_selfenergy(qpfrg_t ctx, double lambda, const double *d_V, const double *d_Z,
                              double *d_sigma_re, double *d_sigma_im, double *d_Z_out);

/* Single-particle spectral function on the patch representatives k_j from a
 * real-frequency self-energy on the context's frequency grid (as written by
 * qpfrg_selfenergy), the observable of Sec. 3.1.1 and Figs. 3 and 7:
 *   A(k_j, w_m) = -(1/pi) Im [w_m - xi_j - Sigma(k_j, w_m)]^-1,
 * and its Fermi-liquid (Gaussian) approximation of Fig. 3: a Gaussian of
 * weight Z_j centred on xi_j with the value of A there (A interpolated
 * linearly on the grid; 0 when xi_j lies outside it):
 *   A_FL(k_j, w) = A0 exp(-pi A0^2 (w - xi_j)^2 / Z_j^2).
 * d_sigma_re, d_sigma_im: N x n_omega FP64 inputs ([j][m]); d_Z: N FP64
 * (NULL = ones); d_A: N x n_omega FP64 output; d_A_fl: N x n_omega FP64
 * output (may be NULL).  Where Sigma vanishes exactly at w = xi_j the grid
 * holds no value of the delta peak and A is written as 0.  Needs n_omega > 0
 * (QPFRG_ERR_INVALID otherwise). */
qpfrg_status qpfrg_spectral(qpfrg_t ctx, const double *d_sigma_re, const double *d_sigma_im, const double *d_Z,
                            double *d_A, double *d_A_fl);

/* Advance the context's flow state by at most n_steps RK4 steps (T-flow:
 * uniform in ln T, last step clamped onto lambda_end; g-flow: uniform in g),
 * stopping early at divergence, end of flow, non-finite state or Z out of
 * range.  With z_feedback, Z is recomputed from Sigma[V, Z] at the start of
 * every step and held over its four stages.  *out (may be NULL) receives the
 * state summary.  Blocks the host once per step to read max|V|. */
qpfrg_status qpfrg_step(qpfrg_t ctx, int n_steps, qpfrg_flow_result *out);

/* Run qpfrg_step until the flow stops (any status other than RUNNING) or
 * max_steps / timeout_s is reached. */
qpfrg_status qpfrg_flow(qpfrg_t ctx, qpfrg_flow_result *out);

/* One flow of a batch: patch count, bare coupling U, start and end of the
 * flow parameter (T-flow: T0 > T_end > 0). */
typedef struct {
    int n_p;
    double U;
    double lambda0;
    double lambda_end;
} qpfrg_flow_spec;

/* Run n_flows independent flows in one call -- a sweep of the strong-coupling
 * scale U*(T) / T*(U) over (U, T, patching) as in Sec. 3.2 and Fig. 4 -- each
 * stopping at its own bound (max|V| > stop_abs_v), end of flow or failure.
 * Flows with the same n_p share one geometry (partner-patch maps) and one set
 * of per-evaluation scratch tables and queue on one internal stream; groups of
 * different n_p run concurrently.  Every running flow advances one RK4 step
 * per round, with one host synchronisation per round for the whole batch.
 * options applies to every flow (its lambda_end is replaced by each spec's).
 * results[i] receives flow i's outcome.  The call waits for the work already
 * on cuda_stream before it starts and returns with the device idle for the
 * batch.  Errors: as qpfrg_create for invalid specs or allocation failures;
 * QPFRG_ERR_TIMEOUT when a tensor-core wait expired. */
qpfrg_status qpfrg_flow_batch(const qpfrg_lattice *lattice, const qpfrg_fine_grid *grid,
                              qpfrg_regulator regulator, const qpfrg_options *options, int n_flows,
                              const qpfrg_flow_spec *specs, void *cuda_stream, qpfrg_flow_result *results);

/* Checkpoint: size in bytes of the state image (64-byte header, then V as
 * N^3 FP64, then Z as N FP64, then -- with the self-energy ODE -- its state
 * [s1, s2, Re S, Im S, Re S', Im S'] (2N + 4 N n_omega FP64), little endian). */
qpfrg_status qpfrg_state_size(qpfrg_t ctx, size_t *bytes);
/* Copy the flow state into h_buf (host, at least qpfrg_state_size bytes;
 * page-locked memory makes the copy a direct DMA).  Synchronises the
 * context's stream. */
qpfrg_status qpfrg_get_state(qpfrg_t ctx, void *h_buf, size_t bytes);
/* Replace the flow state by h_buf (as written by qpfrg_get_state; host,
 * page-locked memory preferred).  The image is uploaded into scratch space and
 * checked on the device (finiteness, max|V|, C4v symmetry of the state, which
 * selects the self-energy's irreducible targets); synchronises the context's
 * stream.  Returns QPFRG_ERR_INVALID on a wrong header or size,
 * QPFRG_ERR_NONFINITE (state unchanged) when V or Z holds NaN/Inf.  Between
 * steps only (it reuses the RK scratch buffers). */
qpfrg_status qpfrg_set_state(qpfrg_t ctx, const void *h_buf, size_t bytes);
/* Copy V (N^3 FP64) and Z (N FP64) of the flow state into device buffers
 * (either may be NULL); enqueued on the context's stream. */
qpfrg_status qpfrg_read_state(qpfrg_t ctx, double *d_V, double *d_Z);

/* Interaction flow with the self-energy ODE (options.sigma_ode, regulator
 * QPFRG_REG_INTERACTION, QPFRG_PROP_PAPER lines): App. A.2-A.5, Eq.
 * (nutshell_2).  The flow state is (V, Sigma, Sigma') at fixed T = T_fixed,
 * from g = lambda0 with Sigma = Sigma' = 0:
 *   d/dg Sigma  = Sigma',
 *   d/dg Sigma' = Abar Sigma' + 6 g T2(w),
 *   d/dg V      = the one-loop RHS with G = g Z G0, S = K Z^2 G0,
 * with per patch j, s1 and s2 the chord slopes of Re Sigma and Re Sigma' over
 * w = xi_j +- 2T: Z = (1 - g s1)^-1 (Eq. (definition_Z) for g Sigma_g),
 * K = 1 + g^2 s2 with the Katanin correction (Eq. (K_definition), else 1),
 * A = 2 Z (s1 + g s2) (Eq. (single_scale_propagator_extended_2)), and Abar the
 * patch average of A (or its minimum / maximum / 0 by options.a_mode).  Without
 * z_feedback, Z = K = 1 and A = 0 (App. A.3 Step 1).  T2 is the two-loop term
 * of qpfrg_selfenergy with the lines of a G, an S and an inner K S line
 * averaged over their assignments, Z_a Z_b Z_c (1/6)[K_a Z_a (Z_b + Z_c) +
 * K_b Z_b (Z_a + Z_c) + K_c Z_c (Z_a + Z_b)]; 6 g makes g Sigma_g at g = 1 the
 * second-order self-energy for a frozen vertex and Z = 1 (App. A.3).
 * Copies the current state into device buffers (each may be NULL):
 *   d_slopes: 2N FP64, s1 then s2;
 *   d_sigma:  4 x N x n_omega FP64, Re Sigma, Im Sigma, Re Sigma', Im Sigma'
 *             on the frequency grid (n_omega > 0);
 *   d_zka:    3N + 1 FP64, Z, K, A of the state and Abar.
 * QPFRG_ERR_INVALID for a context without the self-energy ODE. */
qpfrg_status qpfrg_read_sigma_flow(qpfrg_t ctx, double *d_slopes, double *d_sigma, double *d_zka);

/* Geometry of the context as built on the host: N, the number of fine
 * points M, k_F (N x 2 FP64) and the fine points (M x 4 FP64: kx, ky,
 * weight, patch).  Any output pointer may be NULL. */
qpfrg_status qpfrg_geometry(qpfrg_t ctx, int *n_p, int *n_fine, double *h_kf, double *h_fine);

/* Kernel timing with CUDA events on the context's stream (off by default).
 * qpfrg_profile_get returns the accumulated device milliseconds and launch
 * count of kernel id (0 <= id < qpfrg_profile_count()); names via
 * qpfrg_profile_name.  qpfrg_profile_reset clears the counters. */
qpfrg_status qpfrg_set_profiling(qpfrg_t ctx, int on);
qpfrg_status qpfrg_profile_reset(qpfrg_t ctx);
int          qpfrg_profile_count(void);
const char  *qpfrg_profile_name(int id);
qpfrg_status qpfrg_profile_get(qpfrg_t ctx, int id, double *ms, long long *launches);

/* Work of one right-hand-side evaluation.  In wedge and shell modes the loop kernels
 * evaluate one row per orbit of (transfer Q, patch a) under the point group
 * C4v and write it to every image row with its columns permuted: the
 * dispersion and the fine grid are C4v invariant, so B[gQ][ga][gb] =
 * B[Q][a][b] wherever the patch projection is covariant, which the context
 * checks byte by byte on its partner maps at creation (rows that differ are
 * evaluated by themselves; C4v moves the wedge of a patch and keeps its
 * energy shell).  With quasi-particle lines (QPFRG_PROP_QP) the
 * reduction needs a C4v-symmetric Z.  With QPFRG_MIXED_TC, every row
 * covariant and a C4v-symmetric V and Z (the flow's state, or a qpfrg_rhs
 * input that passes a device test at 1e-12 relative), each channel's output
 * is C4v invariant too: then only one output row per orbit of transfer pairs
 * Q = (x, y) is tabled (all its patches a) and contracted, and every other
 * row is its representative's with the columns permuted (row orbits).
 *   loop_evals: loop-kernel evaluations of the context's last RHS;
 *   loop_evals_full: 2 N^2 M, the evaluations of the unreduced RHS;
 *   rows_unreduced: rows evaluated by themselves because the covariance check
 *     failed for them;
 *   contraction_rows: rows of each channel GEMM in the last RHS (N^2, or the
 *     number of row orbits).
 * All outputs may be NULL; loop_evals equals loop_evals_full when the
 * reduction is off (lattice mode, no_loop_symmetry). */
qpfrg_status qpfrg_rhs_work(qpfrg_t ctx, long long *loop_evals, long long *loop_evals_full,
                            long long *rows_unreduced, long long *contraction_rows);

/* The patch-of-r table of the flow's self-energy (options.sigma_table),
 * for verification: *bytes = its size (0 while not built: it is built by the
 * first Z evaluation of a C4v-symmetric state in the FP32 wedge path, when it
 * fits), and, when h_out is not NULL, count bytes from offset copied into
 * h_out (host memory; blocks until done).  Byte (jidx, a, iq, i), at
 * (((jidx N + a) P/8 + i/8) M + iq) 8 + i mod 8, is the patch of r = k_j + p - q for the
 * irreducible target j = jidx (patches 0 .. N/8), p = a P + i (fine points in
 * their storage order) and q the fine point iq of the kernel's angular-minor
 * order: iq = b P + t' with q = b P + (t' mod n_theta) n_r + t' / n_theta.
 * A byte N denotes patch 0 (the kernel's slot for the wedge past the last
 * ray between wedges N-1 and 0).
 * Errors: QPFRG_ERR_INVALID for a range outside the table. */
qpfrg_status qpfrg_sigma_table(qpfrg_t ctx, size_t *bytes, long long offset, long long count,
                               unsigned char *h_out);

/* Launch shapes of the hot kernels; 0 in a field selects the built-in
 * heuristic.  The paper has no counterpart: these are GPU schedule choices.
 *   bubble_qchunk:  transfers per loop-kernel CTA (a CTA's eight warps take
 *                   them two at a time);
 *   sigma_qblocks:  blocks of 512 loop points q per self-energy CTA (the CTA
 *                   stages its tables once for all of them), at most 64;
 *   tc_splits[3]:   split-K factors of the pp, cr and d tensor-core
 *                   contractions, clipped to the number of 64-wide k blocks;
 *   ms_bubble, ms_sigma, ms_contract: fastest times found by qpfrg_autotune
 *                   (outputs; ignored by qpfrg_set_tuning);
 *   bubble_transfers: transfers a warp of the FP32 loop kernels carries per
 *                   pass over the patch's points, 2 or 4 (0: 2). */
typedef struct {
    int bubble_qchunk;
    int sigma_qblocks;
    int tc_splits[3];
    double ms_bubble, ms_sigma, ms_contract;
    int bubble_transfers;
} qpfrg_tuning;

/* Project-written autotuner: times candidate launch shapes on the context's
 * own state at Lambda = lambda -- the loop kernels (transfers per CTA and per
 * warp pass), the
 * tensor-core contraction of each channel (split-K; QPFRG_MIXED_TC), the FP32
 * self-energy of the wedge grid (q blocks per CTA) -- one untimed and one
 * timed launch each with CUDA events on the context's stream, keeps the
 * fastest in the context and reports them in *out (may be NULL).  The call
 * waits for its work.  It writes only scratch buffers (the loop-kernel table,
 * the tensor-core B operands, the RK stage buffer, the Z work buffer) and, on
 * its first self-energy launch, may build the patch-of-r table (a function of
 * the geometry only, options.sigma_table); never the flow state, and the
 * profiler does not count its launches.  QPFRG_ERR_INVALID for a bad lambda
 * (as qpfrg_rhs). */
qpfrg_status qpfrg_autotune(qpfrg_t ctx, double lambda, qpfrg_tuning *out);

/* Apply launch shapes (e.g. those qpfrg_autotune found on another context of
 * the same size).  QPFRG_ERR_INVALID for a negative field, sigma_qblocks > 64
 * or bubble_transfers other than 0, 2, 4. */
qpfrg_status qpfrg_set_tuning(qpfrg_t ctx, const qpfrg_tuning *t);

/* ---------------------------------------------------------------------------
 * Allocation-free Z evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run
 * -- code living inside another runtime's memory pool, a driver that may only
 * use memory it was handed, a process that must not grow its footprint after
 * start-up.  It computes the same Z_j as qpfrg_selfenergy (FP64, every
 * patch) without a context and without calling cudaMalloc, cudaFree or any
 * allocating routine.  Its only scratch is one FP64 accumulator per patch in
 * a static device array of QPFRG_STATIC_MAX_PATCHES entries, which every GPU
 * that loads this library holds until the process exits.
 *   lattice, n_p, grid_mode, propagator: as for qpfrg_create (n_p <= the
 *     static limit, else QPFRG_ERR_INVALID);
 *   d_fine: n_fine x 4 FP64 device array (kx, ky, weight, patch) exactly as
 *     qpfrg_geometry returns it: patch-major, n_fine / n_p points per patch
 *     (at most 2048, the limit of qpfrg_create; else QPFRG_ERR_UNSUPPORTED).
 *     The patch of point q is taken as q / (n_fine / n_p); the patch column is
 *     not read, so an array in another order gives wrong Z without an error;
 *   d_kf: n_p x 2 FP64 patch representatives; d_V: n_p^3 FP64; d_Z: n_p FP64
 *     line weights (NULL = ones); T > 0; eta > 0; d_Z_out: n_p FP64 output.
 * The first call on a device looks up the device address of the scratch
 * array (with that device current) and caches it: make that first call
 * before any stream capture.  The cached address lives as long as the
 * process: after cudaDeviceReset (or any teardown of the device's primary
 * context) the entry point must not be called again in that process.  A
 * CUDA error already pending when the call starts is returned as
 * QPFRG_ERR_CUDA without launching anything (and is left pending).  All calls share the scratch array, which keeps
 * the last call's values; each call clears the entries it uses first.  Calls
 * that overlap on the GPU (other streams, other host threads) race. */
#define QPFRG_STATIC_MAX_PATCHES 256
qpfrg_status qpfrg_zfactor_static(const qpfrg_lattice *lattice, int n_p, int n_fine, int grid_mode,
                                  int propagator, const double *d_fine, const double *d_kf,
                                  const double *d_V, const double *d_Z, double T, double eta,
                                  void *cuda_stream, double *d_Z_out);

/* Measured ALU rates of the current device, for the rooflines of the
 * ALU-bound kernels (no counterpart in the paper): results per SM per clock of
 * ex2.approx.f32, rcp.approx.f32 and FP32 FMA, each from one launch of eight
 * independent dependency chains per thread, 8 CTAs of 256 threads per SM,
 * timed in SM clocks (clock64, the longest CTA), after one warm-up launch.
 * Synchronous on the legacy default stream; allocates and frees two small
 * device buffers.  Outputs may be NULL.  QPFRG_ERR_CUDA without a device,
 * QPFRG_ERR_OOM when the buffers cannot be allocated. */
qpfrg_status qpfrg_alu_rates(double *ex2_per_sm_clk, double *rcp_per_sm_clk, double *ffma_per_sm_clk);

const char  *qpfrg_last_error(qpfrg_t ctx);   /* never NULL; ctx may be NULL */
const char  *qpfrg_version(void);
void         qpfrg_destroy(qpfrg_t ctx);      /* frees device memory; NULL is a no-op */

#ifdef __cplusplus
}
#endif
#endif
