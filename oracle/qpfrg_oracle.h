/*
 * qpfrg_oracle.h -- plain FP64 CPU oracle of the quasi-particle fRG hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py (its cpu_baseline leg and
 * its reference arm) load the compiled oracle.  It shares no code, header,
 * table or constant with the CUDA library under paper_2005_00827_gb300/csrc.
 *
 * Every function restates the method of Rohe & Honerkamp, "Quasi-particle
 * functional Renormalisation Group calculations in the two-dimensional
 * half-filled Hubbard model at finite temperatures" (arXiv:2005.00827):
 *   - dispersion: Sec. 2.1, Eq. (free_dispersion_xi);
 *   - one-loop vertex flow: App. A.1 Eq. (vertex_flow_general), with the
 *     quasi-particle weights of Eq. (vertex_flow_feedback_Z);
 *   - propagators G = gZ G0, S = Z^2 G0: Eq. (both_propagators_Z);
 *   - real-frequency two-loop self-energy: Sec. 2.2, Eq. (sigma_flow_simple)
 *     and the Z-weighted two-loop term after Eq. (Z_prime_of_sigma);
 *   - Z from the real part of Sigma: Eq. (definition_Z) with the chord slope
 *     "from outside" at a margin of 2T (Sec. 3.1.1, Fig. 2 caption);
 *   - flow to strong coupling: Sec. 3.2 (largest coupling grows past a bound).
 * Where the paper is silent (patch geometry, loop kernels, T-flow) the oracle
 * follows the readings listed in the repository's design notes; each function
 * names the reading it takes.
 */
#ifndef QPFRG_ORACLE_H
#define QPFRG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MODE_WEDGE = 0, ORC_MODE_LATTICE = 1, ORC_MODE_SHELL = 2 };
enum { ORC_REG_TEMPERATURE = 0, ORC_REG_INTERACTION = 1 };
enum { ORC_PROP_PAPER = 0, ORC_PROP_QP = 1 };
enum { ORC_CH_PP = 1, ORC_CH_CR = 2, ORC_CH_D = 4 };
enum { ORC_END = 0, ORC_DIVERGED = 1, ORC_NONFINITE = 2, ORC_Z_RANGE = 3, ORC_MAX_STEPS = 4 };

typedef struct orc_params {
    double t, tp, mu;      /* hoppings t, t' and chemical potential (Sec. 2.1)        */
    int mode;              /* ORC_MODE_WEDGE, ORC_MODE_LATTICE or ORC_MODE_SHELL       */
    int N;                 /* number of patches (lattice: L*L; shell: wedges x shells) */
    int n_theta, n_r;      /* fine loop grid per wedge: angular x radial points        */
    int regulator;         /* ORC_REG_TEMPERATURE (Lambda = T) or _INTERACTION (g)     */
    int prop_mode;         /* ORC_PROP_PAPER: G = Z/(iw - xi); _QP: G = Z/(iw - Z xi)   */
    unsigned channels;     /* OR of ORC_CH_*                                           */
    double T_fixed;        /* temperature of the interaction flow                      */
    double eta;            /* Lorentzian broadening of the retarded self-energy        */
    int n_shell;           /* shell mode: energy shells per angular wedge (odd)        */
    double shell_width;    /* shell mode: energy width of a shell (<= 0: band / n_shell) */
} orc_params;

typedef struct orc_geom {
    orc_params P;
    int M;                 /* number of fine loop points                               */
    double *kf;            /* N x 2 patch representatives k_F(j)                       */
    double *fk;            /* M x 2 fine point momenta                                 */
    double *fw;            /* M quadrature weights, sum ~ 1 = int d^2k/(2pi)^2         */
    int    *fpatch;        /* M patch index of each fine point                         */
} orc_geom;

typedef struct orc_flow_opts {
    double lambda0;        /* start of the flow: T0 (T-flow) or g0 (g-flow)            */
    double lambda_end;     /* end: T_end or g_end                                      */
    double step;           /* T-flow: d ln T per step (negative); g-flow: dg (>0)      */
    double stop_abs_v;     /* divergence bound on max |V|                              */
    double z_max;          /* Z outside (0, z_max] stops the flow                      */
    int z_feedback;        /* recompute Z from Sigma once per step                     */
    int max_steps;
} orc_flow_opts;

typedef struct orc_flow_result {
    int status;            /* ORC_END, ORC_DIVERGED, ...                               */
    int steps;             /* completed RK4 steps                                      */
    double lambda;         /* flow parameter after the last completed step             */
    double lambda_c;       /* interpolated crossing of stop_abs_v (DIVERGED only)      */
    double max_abs_v;      /* max |V| after the last completed step                    */
} orc_flow_result;

/* geometry ------------------------------------------------------------------ */
int    orc_geom_create(const orc_params *P, orc_geom **out);
void   orc_geom_free(orc_geom *g);
int    orc_geom_M(const orc_geom *g);
void   orc_geom_export(const orc_geom *g, double *kf, double *fk, double *fw, int *fpatch);
int    orc_proj(const orc_geom *g, double kx, double ky);
double orc_xi(const orc_params *P, double kx, double ky);
double orc_shell_width(const orc_params *P);   /* shell mode: the energy width of a shell */

/* Fermi functions and bubbles ------------------------------------------------- */
double orc_fermi(double x, double T);
double orc_dfermi_dT(double x, double T);
double orc_D(double a, double b, double T);
double orc_dD_dT(double a, double b, double T);
double orc_Lph(double a, double b, double T);
double orc_Lpp(double a, double b, double T);
double orc_dLph_dT(double a, double b, double T);
double orc_dLpp_dT(double a, double b, double T);

/* one-loop right-hand side -------------------------------------------------- */
void orc_rhs_triple(const orc_geom *g, double lambda, const double *V, const double *Z,
                    int i, int j, int l, double out[3]);
void orc_rhs(const orc_geom *g, double lambda, const double *V, const double *Z,
             double *dV, int nthreads);

/* self-energy and Z ---------------------------------------------------------- */
void orc_sigma(const orc_geom *g, double T, const double *V, const double *Z, int j,
               int n_omega, const double *omega, double *re, double *im, int nthreads);
int  orc_zfactor(const orc_geom *g, double T, const double *V, const double *Zin,
                 double *Zout, int nthreads);
int  orc_zfactor_targets(const orc_geom *g, double T, const double *V, const double *Zin,
                         int n, const int *js, double *Zout, int nthreads);

/* interaction flow with the self-energy ODE (App. A.2-A.5) ------------------- */
enum { ORC_A_AVG = 0, ORC_A_MIN = 1, ORC_A_MAX = 2, ORC_A_DROP = 3 };

typedef struct orc_gflow_opts {
    double g0, g_end, dg;  /* flow parameter: start, end, RK4 step                     */
    double stop_abs_v;     /* divergence bound on max |V|                               */
    int z_feedback;        /* Z, K, A from the self-energy; 0: Z = K = 1, A = 0          */
    int katanin;           /* Katanin factor K on the S lines (App. A.5)                */
    int a_mode;            /* ORC_A_AVG / _MIN / _MAX / _DROP (App. B, App. A.4)         */
    int freeze_vertex;     /* dV/dg = 0 (the self-energy ODE at the bare vertex)        */
    int max_steps;
    int n_omega;           /* frequency grid of Sigma besides xi_j +- 2T                */
    const double *omega;
} orc_gflow_opts;

void orc_sigma_gflow(const orc_geom *g, double T, const double *V, const double *Z, const double *K, int j,
                     int n_omega, const double *omega, double *re, double *im, int nthreads);
void orc_gflow_zka(const orc_geom *g, const orc_gflow_opts *o, double gv, const double *Sre, const double *Dre,
                   double *Z, double *K, double *A, double *Abar);
void orc_gflow_rhs(const orc_geom *g, const orc_gflow_opts *o, double gv, const double *V, const double *Sre,
                   const double *Sim, const double *Dre, const double *Dim, double *dV, double *dSre,
                   double *dSim, double *dDre, double *dDim, int nthreads);
int  orc_gflow(const orc_geom *g, const orc_gflow_opts *o, double *V, double *Sre, double *Sim, double *Dre,
               double *Dim, orc_flow_result *res, int nthreads);

/* spectral function and its Fermi-liquid (Gaussian) approximation ------------- */
void orc_spectral(const orc_geom *g, int j, int n_omega, const double *omega, const double *re,
                  const double *im, double Zj, double *A, double *Afl);

/* ODE ------------------------------------------------------------------------ */
void orc_rk4_step(const orc_geom *g, double lambda, double h, double *V, const double *Z,
                  int nthreads);
int  orc_flow(const orc_geom *g, const orc_flow_opts *o, double *V, double *Z,
              orc_flow_result *res, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
