/*
 * qpfrg_oracle.c -- plain, slow, FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline/reference
 * arm may load this code.  It shares nothing with the CUDA library.  Every sum
 * is written out in the order the method defines it: no Q-grouping, no
 * blocking, no tabulation.  See qpfrg_oracle.h for the paper passages.
 */
#include "qpfrg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI (2.0 * M_PI)

/* ------------------------------------------------------------------------- */
/* Dispersion, Sec. 2.1, Eq. (free_dispersion_xi):                           */
/*   xi_k = -2t (cos kx + cos ky) - 4t' cos kx cos ky - mu                   */
/* ------------------------------------------------------------------------- */
double orc_xi(const orc_params *P, double kx, double ky)
{
    double cx = cos(kx), cy = cos(ky);
    return -2.0 * P->t * (cx + cy) - 4.0 * P->tp * cx * cy - P->mu;
}

/* ------------------------------------------------------------------------- */
/* Patch geometry (the paper states only patch counts, Sec. 3.2 and Fig. 4   */
/* caption; the reading taken here):                                         */
/*  wedge mode  -- N angular wedges about the origin, centres theta_j =      */
/*                 2 pi j / N, so (pi,0) is a centre; k_F(j) is the Fermi     */
/*                 surface point on the ray theta_j.  Fine grid per wedge:    */
/*                 n_theta angular midpoints x n_r radial midpoint cells,     */
/*                 n_r/2 uniform cells in (0, r_F(theta)) and n_r/2 in        */
/*                 (r_F(theta), r_BZ(theta)); weight = cell area / (2 pi)^2.  */
/*  lattice mode -- all L*L momenta 2 pi (m1, m2)/L are patches; each patch   */
/*                 holds one loop point of weight 1/L^2; projection = nearest */
/*                 lattice momentum.  This is the exact finite-lattice sum.   */
/*  shell mode  -- (angle, energy) patches (Sec. 3.2: 32 angular sections x  */
/*                 7 shells in the energy direction = 224).  N_a = N/n_s      */
/*                 wedges as above, each cut into n_s (odd) energy shells of  */
/*                 width D centred on the Fermi surface: shell s holds        */
/*                 xi in [(s - n_s/2) D, (s + 1 - n_s/2) D), the outer shells */
/*                 extended to the band edges; D defaults to the band width   */
/*                 2 max|xi| over n_s.  Patch j = w n_s + s.  Representative:  */
/*                 the point of the wedge's centre ray at the shell's middle  */
/*                 energy (s - (n_s-1)/2) D (k_F for the Fermi shell), the    */
/*                 zone edge of the ray when the ray ends below that energy.  */
/*                 Fine grid: per angular midpoint ray, the shell's radial    */
/*                 segment between the radii where xi crosses its two edges  */
/*                 (xi increases along every ray: checked) in n_r midpoint    */
/*                 cells, the Fermi shell's n_r/2 below and n_r/2 above       */
/*                 r_F(theta), so n_s = 1 is wedge mode.  Projection: wedge   */
/*                 by angle, shell by xi of the folded momentum.              */
/* ------------------------------------------------------------------------- */
static double r_bz(double th)
{
    /* distance from the origin to the edge of [-pi, pi]^2 along theta */
    return M_PI / fmax(fabs(cos(th)), fabs(sin(th)));
}

static double ray_radius(const orc_params *P, double th, double eps)
{
    /* first crossing of xi = eps along the ray, by bisection; the zone edge */
    /* when xi stays below eps, 0 when the origin is already at or above it  */
    double lo = 0.0, hi = r_bz(th);
    if (orc_xi(P, hi * cos(th), hi * sin(th)) < eps) return hi;
    if (orc_xi(P, 0.0, 0.0) >= eps) return 0.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_xi(P, mid * cos(th), mid * sin(th)) < eps) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double r_fermi(const orc_params *P, double th) { return ray_radius(P, th, 0.0); }

double orc_shell_width(const orc_params *P)
{
    if (P->shell_width > 0.0) return P->shell_width;
    /* band extremes at (0,0), (pi,pi) and (pi,0) for |t'| <= t/2 */
    double w = fabs(orc_xi(P, 0.0, 0.0));
    w = fmax(w, fabs(orc_xi(P, M_PI, M_PI)));
    w = fmax(w, fabs(orc_xi(P, M_PI, 0.0)));
    return 2.0 * w / P->n_shell;
}

/* shell of an energy: floor(xi / D + n_s / 2), clamped to the outer shells */
static int shell_of(const orc_params *P, double D, double xi)
{
    long s = (long)floor(xi / D + 0.5 * P->n_shell);
    if (s < 0) s = 0;
    if (s > P->n_shell - 1) s = P->n_shell - 1;
    return (int)s;
}

/* xi non-decreasing along the ray (checked on 512 points) */
static int ray_monotone(const orc_params *P, double th)
{
    const double rb = r_bz(th);
    double prev = orc_xi(P, 0.0, 0.0);
    for (int i = 1; i <= 512; ++i) {
        const double r = rb * i / 512.0;
        const double x = orc_xi(P, r * cos(th), r * sin(th));
        if (x < prev - 1e-12) return 0;
        prev = x;
    }
    return 1;
}

static double fold_bz(double x)
{
    /* map a momentum component into [-pi, pi] (ties to even) */
    return x - TWO_PI * nearbyint(x / TWO_PI);
}

static int lattice_L(int N)
{
    int L = (int)llround(sqrt((double)N));
    return (L * L == N) ? L : -1;
}

int orc_proj(const orc_geom *g, double kx, double ky)
{
    const int N = g->P.N;
    if (g->P.mode == ORC_MODE_LATTICE) {
        int L = lattice_L(N);
        long m1 = (long)nearbyint(kx * L / TWO_PI) % L;
        long m2 = (long)nearbyint(ky * L / TWO_PI) % L;
        if (m1 < 0) m1 += L;
        if (m2 < 0) m2 += L;
        return (int)(m1 * L + m2);
    }
    const int ns = g->P.mode == ORC_MODE_SHELL ? g->P.n_shell : 1;
    const int Na = N / ns;
    double x = fold_bz(kx), y = fold_bz(ky);
    double th = atan2(y, x);
    double dth = TWO_PI / Na;
    long j = (long)floor(th / dth + 0.5);
    j %= Na;
    if (j < 0) j += Na;
    if (ns == 1) return (int)j;
    return (int)(j * ns + shell_of(&g->P, orc_shell_width(&g->P), orc_xi(&g->P, x, y)));
}

int orc_geom_create(const orc_params *P, orc_geom **out)
{
    *out = NULL;
    const int N = P->N;
    if (N < 1) return -1;
    orc_geom *g = (orc_geom *)calloc(1, sizeof(orc_geom));
    if (!g) return -2;
    g->P = *P;
    if (P->mode == ORC_MODE_LATTICE) {
        int L = lattice_L(N);
        if (L < 1) { free(g); return -1; }
        g->M = N;
    } else {
        const int ns = P->mode == ORC_MODE_SHELL ? P->n_shell : 1;
        if (ns < 1 || ns % 2 == 0 || N % ns != 0 || (N / ns) % 4 != 0 || P->n_theta < 1 || P->n_r < 2 ||
            (P->n_r % 2) != 0) {
            free(g);
            return -1;
        }
        g->M = N * P->n_theta * P->n_r;
    }
    const int M = g->M;
    g->kf = (double *)malloc(sizeof(double) * 2 * N);
    g->fk = (double *)malloc(sizeof(double) * 2 * M);
    g->fw = (double *)malloc(sizeof(double) * M);
    g->fpatch = (int *)malloc(sizeof(int) * M);
    if (!g->kf || !g->fk || !g->fw || !g->fpatch) { orc_geom_free(g); return -2; }

    if (P->mode == ORC_MODE_LATTICE) {
        int L = lattice_L(N);
        for (int m1 = 0; m1 < L; ++m1)
            for (int m2 = 0; m2 < L; ++m2) {
                int j = m1 * L + m2;
                g->kf[2 * j + 0] = TWO_PI * m1 / L;
                g->kf[2 * j + 1] = TWO_PI * m2 / L;
                g->fk[2 * j + 0] = g->kf[2 * j + 0];
                g->fk[2 * j + 1] = g->kf[2 * j + 1];
                g->fw[j] = 1.0 / N;
                g->fpatch[j] = j;
            }
        *out = g;
        return 0;
    }

    if (P->mode == ORC_MODE_SHELL) {
        const int ns = P->n_shell, Na = N / ns, nt = P->n_theta, nr = P->n_r, half = P->n_r / 2;
        const int sF = ns / 2;
        const double dth = TWO_PI / Na, D = orc_shell_width(P);
        for (int w = 0; w < Na; ++w) {
            const double thw = dth * w;
            if (!ray_monotone(P, thw)) { orc_geom_free(g); return -1; }
            for (int t = 0; t < nt; ++t)
                if (!ray_monotone(P, thw + ((t + 0.5) / nt - 0.5) * dth)) { orc_geom_free(g); return -1; }
            for (int sh = 0; sh < ns; ++sh) {
                const int j = w * ns + sh;
                const double rj = sh == sF ? r_fermi(P, thw) : ray_radius(P, thw, (sh - sF) * D);
                g->kf[2 * j + 0] = rj * cos(thw);
                g->kf[2 * j + 1] = rj * sin(thw);
                for (int t = 0; t < nt; ++t) {
                    const double th = thw + ((t + 0.5) / nt - 0.5) * dth;
                    const double r0 = sh == 0 ? 0.0 : ray_radius(P, th, (sh - 0.5 * ns) * D);
                    const double r1 = sh == ns - 1 ? r_bz(th) : ray_radius(P, th, (sh + 1 - 0.5 * ns) * D);
                    const double rF = r_fermi(P, th);
                    for (int i = 0; i < nr; ++i) {
                        double rlo, rhi;
                        if (sh != sF) {
                            rlo = r0 + (r1 - r0) * i / nr;
                            rhi = r0 + (r1 - r0) * (i + 1) / nr;
                        } else if (i < half) {
                            rlo = r0 + (rF - r0) * i / half;
                            rhi = r0 + (rF - r0) * (i + 1) / half;
                        } else {
                            rlo = rF + (r1 - rF) * (i - half) / half;
                            rhi = rF + (r1 - rF) * (i - half + 1) / half;
                        }
                        const double r = 0.5 * (rlo + rhi);
                        const int p = (j * nt + t) * nr + i;
                        g->fk[2 * p + 0] = r * cos(th);
                        g->fk[2 * p + 1] = r * sin(th);
                        g->fw[p] = 0.5 * (rhi * rhi - rlo * rlo) * (dth / nt) / (TWO_PI * TWO_PI);
                        g->fpatch[p] = j;
                    }
                }
            }
        }
        *out = g;
        return 0;
    }

    const double dth = TWO_PI / N;
    const int nt = P->n_theta, nr = P->n_r, half = P->n_r / 2;
    for (int j = 0; j < N; ++j) {
        double thj = dth * j;
        double rf = r_fermi(P, thj);
        g->kf[2 * j + 0] = rf * cos(thj);
        g->kf[2 * j + 1] = rf * sin(thj);
        for (int t = 0; t < nt; ++t) {
            double th = thj + ((t + 0.5) / nt - 0.5) * dth;
            double rF = r_fermi(P, th), rB = r_bz(th);
            for (int s = 0; s < nr; ++s) {
                double rlo, rhi;
                if (s < half) {
                    rlo = rF * s / half;
                    rhi = rF * (s + 1) / half;
                } else {
                    rlo = rF + (rB - rF) * (s - half) / half;
                    rhi = rF + (rB - rF) * (s - half + 1) / half;
                }
                double r = 0.5 * (rlo + rhi);
                int p = (j * nt + t) * nr + s;
                g->fk[2 * p + 0] = r * cos(th);
                g->fk[2 * p + 1] = r * sin(th);
                g->fw[p] = 0.5 * (rhi * rhi - rlo * rlo) * (dth / nt) / (TWO_PI * TWO_PI);
                g->fpatch[p] = j;
            }
        }
    }
    *out = g;
    return 0;
}

void orc_geom_free(orc_geom *g)
{
    if (!g) return;
    free(g->kf); free(g->fk); free(g->fw); free(g->fpatch);
    free(g);
}

int orc_geom_M(const orc_geom *g) { return g->M; }

void orc_geom_export(const orc_geom *g, double *kf, double *fk, double *fw, int *fpatch)
{
    memcpy(kf, g->kf, sizeof(double) * 2 * g->P.N);
    memcpy(fk, g->fk, sizeof(double) * 2 * g->M);
    memcpy(fw, g->fw, sizeof(double) * g->M);
    memcpy(fpatch, g->fpatch, sizeof(int) * g->M);
}

/* ------------------------------------------------------------------------- */
/* Fermi function and the closed-form Matsubara sums of the bubbles.        */
/* With G0 = 1/(iw - xi) (Sec. A.3, Eq. (both_propagators_Z) at Z = 1):      */
/*   L_ph(a,b) = T sum_n G0_a(iw) G0_b(iw)   = (f(a) - f(b)) / (a - b) = D   */
/*   L_pp(a,b) = T sum_n G0_a(iw) G0_b(-iw)  = (1 - f(a) - f(b)) / (a + b)   */
/*             = -D(a, -b)                                                   */
/* The limit a -> b of D is f'(a).  Below |a-b| < 1e-5 T the oracle uses the */
/* midpoint derivative, whose error there is O((a-b)^2/T^2) < 1e-10.         */
/* ------------------------------------------------------------------------- */
double orc_fermi(double x, double T)
{
    double y = x / T;
    if (y > 0.0) { double e = exp(-y); return e / (1.0 + e); }
    return 1.0 / (1.0 + exp(y));
}

/* f(1 - f), computed without cancellation */
static double fermi_ff(double x, double T)
{
    double e = exp(-fabs(x) / T);
    return e / ((1.0 + e) * (1.0 + e));
}

static double dfermi_dx(double x, double T) { return -fermi_ff(x, T) / T; }

double orc_dfermi_dT(double x, double T) { return x / (T * T) * fermi_ff(x, T); }

/* d/dx d/dT f = f'(x) (-1/T + x (1 - 2 f) / T^2) */
static double d2fermi_dxdT(double x, double T)
{
    double one_m_2f = orc_fermi(-x, T) - orc_fermi(x, T);
    return dfermi_dx(x, T) * (-1.0 / T + x * one_m_2f / (T * T));
}

static int near_degenerate(double a, double b, double T) { return fabs(a - b) < 1e-5 * T; }

double orc_D(double a, double b, double T)
{
    if (near_degenerate(a, b, T)) return dfermi_dx(0.5 * (a + b), T);
    double num;
    if (a < 0.0 && b < 0.0)          /* both occupied: difference of 1 - f */
        num = orc_fermi(-b, T) - orc_fermi(-a, T);
    else
        num = orc_fermi(a, T) - orc_fermi(b, T);
    return num / (a - b);
}

double orc_dD_dT(double a, double b, double T)
{
    if (near_degenerate(a, b, T)) return d2fermi_dxdT(0.5 * (a + b), T);
    return (orc_dfermi_dT(a, T) - orc_dfermi_dT(b, T)) / (a - b);
}

double orc_Lph(double a, double b, double T) { return orc_D(a, b, T); }
double orc_Lpp(double a, double b, double T) { return -orc_D(a, -b, T); }
double orc_dLph_dT(double a, double b, double T) { return orc_dD_dT(a, b, T); }
double orc_dLpp_dT(double a, double b, double T) { return -orc_dD_dT(a, -b, T); }

/* ------------------------------------------------------------------------- */
/* Loop weight of one internal line pair (p in patch a, partner in patch b). */
/*  T-flow (Lambda = T, the flow of the configurations): the scale derivative */
/*    of the Z-weighted bubble, Z_a Z_b dL/dT, Z held fixed over a step.      */
/*  g-flow (Lambda = g, Sec. A.1/A.3, Eq. (vertex_flow_feedback_Z)): G S + S G */
/*    with G = g Z G0 and S = Z^2 G0, symmetrised over the two lines:         */
/*    g Z_a Z_b (Z_a + Z_b) L at fixed T  (= 2 g L at Z = 1, Eq.               */
/*    (vertex_flow_simple)).                                                 */
/*  prop_mode QP puts Z into the pole, G = Z/(iw - Z xi).                     */
/* ------------------------------------------------------------------------- */
static double line_xi(const orc_geom *g, const double *Z, double xi, int patch)
{
    return g->P.prop_mode == ORC_PROP_QP ? Z[patch] * xi : xi;
}

/* K (may be NULL = ones): the Katanin factor of App. A.5 on the S line of   */
/* the g-flow, Eq. (vertex_flow_feedback_Z_with_Katanin): G S + S G with      */
/* G = g Z G0, S = K Z^2 G0 gives g Z_a Z_b (K_a Z_a + K_b Z_b) L.             */
static double loop_weight(const orc_geom *g, double lambda, const double *Z, const double *K, int pp,
                          double xi_p, int a, double xi_q, int b)
{
    double xa = line_xi(g, Z, xi_p, a), xb = line_xi(g, Z, xi_q, b);
    if (g->P.regulator == ORC_REG_TEMPERATURE) {
        double T = lambda;
        double dl = pp ? orc_dLpp_dT(xa, xb, T) : orc_dLph_dT(xa, xb, T);
        return Z[a] * Z[b] * dl;
    }
    double T = g->P.T_fixed, gg = lambda;
    double l = pp ? orc_Lpp(xa, xb, T) : orc_Lph(xa, xb, T);
    double ka = K ? K[a] : 1.0, kb = K ? K[b] : 1.0;
    return gg * Z[a] * Z[b] * (ka * Z[a] + kb * Z[b]) * l;
}

/* ------------------------------------------------------------------------- */
/* One-loop SU(2) flow of the static coupling V(k1,k2,k3), App. A.1 Eq.      */
/* (vertex_flow_general) with the propagators of Eq. (both_propagators_Z).   */
/* k1 -> k3 carries spin s, k2 -> k4 carries s', k4 = k1 + k2 - k3.  The      */
/* loop momentum p runs over the fine points; every vertex argument is the   */
/* patch of its momentum.                                                    */
/*   pp : Q = k1 + k2,  dV -= L'_pp(p, Q-p) V(k1,k2,p) V(p,Q-p,k3)           */
/*   cr : Q = k3 - k2,  dV -= L'_ph(p, p+Q) V(k1,p,p+Q) V(p+Q,k2,k3)         */
/*   d  : Q = k1 - k3,  dV += L'_ph(p, p+Q) [2 V(k1,p,k3) V(p+Q,k2,p)         */
/*                           - V(p,k1,k3) V(p+Q,k2,p) - V(k1,p,k3) V(k2,p+Q,p)] */
/* out[0..2] = pp, cr, d contributions; the RHS is their sum.                */
/* ------------------------------------------------------------------------- */
#define VV(a, b, c) V[((size_t)(a) * N + (b)) * N + (c)]

static void rhs_triple_k(const orc_geom *g, double lambda, const double *V, const double *Z,
                         const double *K, int i, int j, int l, double out[3]);

void orc_rhs_triple(const orc_geom *g, double lambda, const double *V, const double *Z,
                    int i, int j, int l, double out[3])
{
    rhs_triple_k(g, lambda, V, Z, NULL, i, j, l, out);
}

static void rhs_triple_k(const orc_geom *g, double lambda, const double *V, const double *Z,
                         const double *K, int i, int j, int l, double out[3])
{
    const int N = g->P.N, M = g->M;
    const orc_params *P = &g->P;
    const double *kf = g->kf;
    double s_pp = 0.0, s_cr = 0.0, s_d = 0.0;

    for (int p = 0; p < M; ++p) {
        const int a = g->fpatch[p];
        const double px = g->fk[2 * p], py = g->fk[2 * p + 1], w = g->fw[p];
        const double xi_p = orc_xi(P, px, py);

        if (P->channels & ORC_CH_PP) {
            double Qx = kf[2 * i] + kf[2 * j], Qy = kf[2 * i + 1] + kf[2 * j + 1];
            double qx = Qx - px, qy = Qy - py;
            int b = orc_proj(g, qx, qy);
            double L = loop_weight(g, lambda, Z, K, 1, xi_p, a, orc_xi(P, qx, qy), b);
            s_pp -= w * L * VV(i, j, a) * VV(a, b, l);
        }
        if (P->channels & ORC_CH_CR) {
            double Qx = kf[2 * l] - kf[2 * j], Qy = kf[2 * l + 1] - kf[2 * j + 1];
            double qx = px + Qx, qy = py + Qy;
            int b = orc_proj(g, qx, qy);
            double L = loop_weight(g, lambda, Z, K, 0, xi_p, a, orc_xi(P, qx, qy), b);
            s_cr -= w * L * VV(i, a, b) * VV(b, j, l);
        }
        if (P->channels & ORC_CH_D) {
            double Qx = kf[2 * i] - kf[2 * l], Qy = kf[2 * i + 1] - kf[2 * l + 1];
            double qx = px + Qx, qy = py + Qy;
            int b = orc_proj(g, qx, qy);
            double L = loop_weight(g, lambda, Z, K, 0, xi_p, a, orc_xi(P, qx, qy), b);
            s_d += w * L * (2.0 * VV(i, a, l) * VV(b, j, a)
                            - VV(a, i, l) * VV(b, j, a)
                            - VV(i, a, l) * VV(j, b, a));
        }
    }
    out[0] = s_pp;
    out[1] = s_cr;
    out[2] = s_d;
}

static void rhs_k(const orc_geom *g, double lambda, const double *V, const double *Z, const double *K,
                  double *dV, int nthreads)
{
    const int N = g->P.N;
    const long n3 = (long)N * N * N;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long idx = 0; idx < n3; ++idx) {
        int i = (int)(idx / ((long)N * N)), j = (int)((idx / N) % N), l = (int)(idx % N);
        double o[3];
        rhs_triple_k(g, lambda, V, Z, K, i, j, l, o);
        dV[idx] = o[0] + o[1] + o[2];
    }
    (void)nthreads;
}

void orc_rhs(const orc_geom *g, double lambda, const double *V, const double *Z,
             double *dV, int nthreads)
{
    rhs_k(g, lambda, V, Z, NULL, dV, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Two-loop retarded self-energy with the static vertex (Sec. A.2-A.3: the   */
/* frequency dependence comes from the two-loop term, Eq. (sigma_flow_simple) */
/* and the Z-weighted line product after Eq. (Z_prime_of_sigma)), evaluated  */
/* at fixed vertex on the real axis, omega + i eta:                          */
/*   Sigma(k_j, w) = sum_{p,q} w_p w_q Z_a Z_b Z_c W F / (w + i eta - E),     */
/*   r = k_j + p - q,  E = xi_q + xi_r - xi_p,                                */
/*   F = f_p (1-f_q)(1-f_r) + (1-f_p) f_q f_r,                                */
/*   W = 2 V(k,p,q)^2 - V(k,p,q) V(k,p,r)   (spin sum of the SU(2) vertex,    */
/*       exchange and time-reversal symmetric; = U^2 for V = U, i.e. SOPT,   */
/*       Sec. 3.1),                                                          */
/* with a, b, c the patches of p, q, r.                                      */
/* ------------------------------------------------------------------------- */
void orc_sigma(const orc_geom *g, double T, const double *V, const double *Z, int j,
               int n_omega, const double *omega, double *re, double *im, int nthreads)
{
    const int N = g->P.N, M = g->M;
    const orc_params *P = &g->P;
    const double kx = g->kf[2 * j], ky = g->kf[2 * j + 1], eta = P->eta;
    for (int m = 0; m < n_omega; ++m) { re[m] = 0.0; im[m] = 0.0; }

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *lre = (double *)calloc((size_t)n_omega, sizeof(double));
        double *lim = (double *)calloc((size_t)n_omega, sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int p = 0; p < M; ++p) {
            const int a = g->fpatch[p];
            const double px = g->fk[2 * p], py = g->fk[2 * p + 1];
            const double xp = line_xi(g, Z, orc_xi(P, px, py), a);
            const double fp = orc_fermi(xp, T), fpc = orc_fermi(-xp, T);
            for (int q = 0; q < M; ++q) {
                const int b = g->fpatch[q];
                /* W = V(k,p,q) (2 V(k,p,q) - V(k,p,r)) vanishes with V(k,p,q): such a
                   pair adds exactly zero, so it is not evaluated */
                if (VV(j, a, b) == 0.0) continue;
                const double qx = g->fk[2 * q], qy = g->fk[2 * q + 1];
                const double rx = kx + px - qx, ry = ky + py - qy;
                const int c = orc_proj(g, rx, ry);
                const double xq = line_xi(g, Z, orc_xi(P, qx, qy), b);
                const double xr = line_xi(g, Z, orc_xi(P, rx, ry), c);
                const double F = fp * orc_fermi(-xq, T) * orc_fermi(-xr, T)
                               + fpc * orc_fermi(xq, T) * orc_fermi(xr, T);
                const double vab = VV(j, a, b), vac = VV(j, a, c);
                const double W = Z[a] * Z[b] * Z[c] * (2.0 * vab * vab - vab * vac);
                const double amp = g->fw[p] * g->fw[q] * W * F;
                const double E = xq + xr - xp;
                for (int m = 0; m < n_omega; ++m) {
                    double d = omega[m] - E, den = d * d + eta * eta;
                    lre[m] += amp * d / den;
                    lim[m] -= amp * eta / den;
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int m = 0; m < n_omega; ++m) { re[m] += lre[m]; im[m] += lim[m]; }
        free(lre);
        free(lim);
    }
    (void)nthreads;
}

/* Z_j = (1 - dRe Sigma/dw)^-1, Eq. (definition_Z): the derivative at       */
/* w = xi_j, taken as the chord over w = xi_j +- 2T ("from outside" with a    */
/* margin of 2T, Sec. 3.1.1), for the n targets js[0..n-1]; Zout[m] belongs  */
/* to js[m].  Returns 0 or ORC_NONFINITE when a value is not finite.          */
int orc_zfactor_targets(const orc_geom *g, double T, const double *V, const double *Zin,
                        int n, const int *js, double *Zout, int nthreads)
{
    int st = 0;
    for (int m = 0; m < n; ++m) {
        const int j = js[m];
        double xij = orc_xi(&g->P, g->kf[2 * j], g->kf[2 * j + 1]);
        double w[2] = {xij + 2.0 * T, xij - 2.0 * T}, re[2], im[2];
        orc_sigma(g, T, V, Zin, j, 2, w, re, im, nthreads);
        double slope = (re[0] - re[1]) / (4.0 * T);
        Zout[m] = 1.0 / (1.0 - slope);
        if (!isfinite(Zout[m])) st = ORC_NONFINITE;
    }
    return st;
}

/* Z of every patch (the flow's Z update) */
int orc_zfactor(const orc_geom *g, double T, const double *V, const double *Zin,
                double *Zout, int nthreads)
{
    const int N = g->P.N;
    int *js = (int *)malloc(sizeof(int) * N);
    if (!js) return ORC_NONFINITE;
    for (int j = 0; j < N; ++j) js[j] = j;
    int st = orc_zfactor_targets(g, T, V, Zin, N, js, Zout, nthreads);
    free(js);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Single-particle spectral function on the Fermi-surface patch k_j from the  */
/* real-frequency self-energy (Sec. 3.1.1, Figs. 2-3: A(k, w) of SOPT):        */
/*   A(w) = -(1/pi) Im [w - xi_j - Sigma(k_j, w)]^-1,                          */
/* and its Fermi-liquid (Gaussian) approximation of Fig. 3: a Gaussian of      */
/* weight Z_j centred on xi_j whose value there equals the full A, taken by   */
/* linear interpolation of A on the grid w_0 < ... < w_{n-1}:                 */
/*   A_FL(w) = A(xi_j) exp(-pi A(xi_j)^2 (w - xi_j)^2 / Z_j^2).                */
/* Inputs: Sigma on the grid (re, im), Z_j; outputs A and A_FL on the grid.   */
/* ------------------------------------------------------------------------- */
void orc_spectral(const orc_geom *g, int j, int n_omega, const double *omega, const double *re,
                  const double *im, double Zj, double *A, double *Afl)
{
    const double xij = orc_xi(&g->P, g->kf[2 * j], g->kf[2 * j + 1]);
    for (int m = 0; m < n_omega; ++m) {
        /* G = 1 / (x - i y), x = w - xi - Re Sigma, y = Im Sigma: Im G = y / (x^2 + y^2) */
        const double x = omega[m] - xij - re[m], y = im[m];
        const double d = x * x + y * y;
        A[m] = d > 0.0 ? -(1.0 / M_PI) * y / d : 0.0;   /* Sigma = 0 at w = xi: delta peak, no grid value */
    }
    double A0 = 0.0;
    for (int m = 0; m + 1 < n_omega; ++m)
        if (omega[m] <= xij && xij <= omega[m + 1]) {
            const double u = (xij - omega[m]) / (omega[m + 1] - omega[m]);
            A0 = (1.0 - u) * A[m] + u * A[m + 1];
            break;
        }
    for (int m = 0; m < n_omega; ++m) {
        const double d = omega[m] - xij;
        Afl[m] = A0 * exp(-M_PI * A0 * A0 * d * d / (Zj * Zj));
    }
}

/* ------------------------------------------------------------------------- */
/* Classical RK4.  T-flow: in l = ln T, dV/dl = T dV/dT.  g-flow: in g.      */
/* ------------------------------------------------------------------------- */
static void flow_rhs(const orc_geom *g, double x, const double *V, const double *Z,
                     double *k, int nthreads)
{
    const long n3 = (long)g->P.N * g->P.N * g->P.N;
    if (g->P.regulator == ORC_REG_TEMPERATURE) {
        double T = exp(x);
        orc_rhs(g, T, V, Z, k, nthreads);
        for (long n = 0; n < n3; ++n) k[n] *= T;
    } else {
        orc_rhs(g, x, V, Z, k, nthreads);
    }
}

void orc_rk4_step(const orc_geom *g, double x, double h, double *V, const double *Z,
                  int nthreads)
{
    const long n3 = (long)g->P.N * g->P.N * g->P.N;
    double *k1 = (double *)malloc(sizeof(double) * n3), *k2 = (double *)malloc(sizeof(double) * n3);
    double *k3 = (double *)malloc(sizeof(double) * n3), *k4 = (double *)malloc(sizeof(double) * n3);
    double *Vs = (double *)malloc(sizeof(double) * n3);
    flow_rhs(g, x, V, Z, k1, nthreads);
    for (long n = 0; n < n3; ++n) Vs[n] = V[n] + 0.5 * h * k1[n];
    flow_rhs(g, x + 0.5 * h, Vs, Z, k2, nthreads);
    for (long n = 0; n < n3; ++n) Vs[n] = V[n] + 0.5 * h * k2[n];
    flow_rhs(g, x + 0.5 * h, Vs, Z, k3, nthreads);
    for (long n = 0; n < n3; ++n) Vs[n] = V[n] + h * k3[n];
    flow_rhs(g, x + h, Vs, Z, k4, nthreads);
    for (long n = 0; n < n3; ++n) V[n] += h / 6.0 * (k1[n] + 2.0 * k2[n] + 2.0 * k3[n] + k4[n]);
    free(k1); free(k2); free(k3); free(k4); free(Vs);
}

static double max_abs(const double *V, long n, int *finite)
{
    double m = 0.0;
    *finite = 1;
    for (long i = 0; i < n; ++i) {
        if (!isfinite(V[i])) *finite = 0;
        double a = fabs(V[i]);
        if (a > m) m = a;
    }
    return m;
}

/* Flow to strong coupling (Sec. 3.2): integrate until the largest |V|       */
/* exceeds stop_abs_v or the end of the flow is reached.  T-flow steps are   */
/* uniform in ln T (the last one clamped onto T_end); Lambda_c interpolates  */
/* ln max|V| linearly in the step variable between the bracketing steps.     */
/* With z_feedback, Z is recomputed from Sigma[V, Z_prev] at the start of    */
/* every step and held over its four stages.                                 */
int orc_flow(const orc_geom *g, const orc_flow_opts *o, double *V, double *Z,
             orc_flow_result *res, int nthreads)
{
    const int N = g->P.N;
    const long n3 = (long)N * N * N;
    const int tflow = g->P.regulator == ORC_REG_TEMPERATURE;
    double x = tflow ? log(o->lambda0) : o->lambda0;
    const double x_end = tflow ? log(o->lambda_end) : o->lambda_end;
    int finite;
    double m = max_abs(V, n3, &finite);
    memset(res, 0, sizeof(*res));
    res->lambda = o->lambda0;
    res->max_abs_v = m;
    double *Znew = (double *)malloc(sizeof(double) * N);

    for (int step = 0;; ++step) {
        double remaining = x_end - x;                  /* negative in the T-flow */
        if ((tflow && remaining > -1e-12) || (!tflow && remaining < 1e-12)) { res->status = ORC_END; break; }
        if (step >= o->max_steps) { res->status = ORC_MAX_STEPS; break; }
        double h = o->step;
        if ((tflow && x + h < x_end) || (!tflow && x + h > x_end)) h = x_end - x;

        if (o->z_feedback) {
            double T = tflow ? exp(x) : g->P.T_fixed;
            int st = orc_zfactor(g, T, V, Z, Znew, nthreads);
            int bad = st != 0;
            for (int j = 0; j < N; ++j)
                if (!(Znew[j] > 0.0 && Znew[j] <= o->z_max)) bad = 1;
            if (bad) { res->status = st ? ORC_NONFINITE : ORC_Z_RANGE; break; }
            memcpy(Z, Znew, sizeof(double) * N);
        }

        orc_rk4_step(g, x, h, V, Z, nthreads);
        double m_new = max_abs(V, n3, &finite);
        double x_new = x + h;
        res->steps = step + 1;
        res->lambda = tflow ? exp(x_new) : x_new;
        res->max_abs_v = m_new;
        if (!finite) { res->status = ORC_NONFINITE; break; }
        if (m_new > o->stop_abs_v) {
            double s = (log(o->stop_abs_v) - log(m)) / (log(m_new) - log(m));
            double xc = x + s * h;
            res->lambda_c = tflow ? exp(xc) : xc;
            res->status = ORC_DIVERGED;
            break;
        }
        x = x_new;
        m = m_new;
    }
    free(Znew);
    return res->status;
}

/* ------------------------------------------------------------------------- */
/* Interaction flow with the self-energy ODE, App. A.2-A.5, Eq. (nutshell_2):  */
/*   d/dg Sigma   = Sigma'                                                     */
/*   d/dg Sigma'  = Abar Sigma' + 6 g T2[V, Z, K](w)                           */
/*   d/dg V       = one-loop RHS with G = g Z G0, S = K Z^2 G0                 */
/* at fixed T (T_fixed), from g0 with V = U, Sigma = Sigma' = 0 (App. B).      */
/* Per patch j, from the chord slopes "from outside" (margin 2T, Sec. 3.1.1)  */
/* of the state at w = xi_j +- 2T, s1 = slope Re Sigma, s2 = slope Re Sigma':  */
/*   Z = (1 - g s1)^-1           Eq. (definition_Z) applied to g Sigma_g       */
/*   K = 1 + g^2 s2              Eq. (K_definition) (1 without Katanin)        */
/*   A = 2 Z (s1 + g s2)         Eq. (single_scale_propagator_extended_2)      */
/*                               (= 2 (dZ/dg)/Z = -(2/g)(1 - Z K), Eq. (A_g_simple)) */
/* and Abar is the mean of A over the Fermi-surface patches (Eq.              */
/* (second_derivative_sigma_approximation)), or its minimum / maximum (the    */
/* bracket flows of App. B), or 0 (the one-loop term dropped, App. A.4).      */
/* T2 is the two-loop term at the static vertex, Sigma of orc_sigma with the  */
/* line weights of a G, an S and an inner K S line averaged over their six    */
/* assignments to the lines a, b, c:                                          */
/*   Z_a Z_b Z_c (1/6) [K_a Z_a (Z_b + Z_c) + K_b Z_b (Z_a + Z_c) + K_c Z_c (Z_a + Z_b)] */
/* (= Z_a Z_b Z_c (Z_a Z_b + Z_b Z_c + Z_a Z_c)/3 at K = 1); the factor 6g     */
/* makes g Sigma_g at g = 1 the second-order self-energy of U for a frozen    */
/* vertex and Z = 1 (Eq. (sigma_flow_simple): g Sigma_g is the self-energy    */
/* of the bare coupling g^2 U, App. A.3).                                     */
/* ------------------------------------------------------------------------- */
void orc_sigma_gflow(const orc_geom *g, double T, const double *V, const double *Z, const double *K, int j,
                     int n_omega, const double *omega, double *re, double *im, int nthreads)
{
    const int N = g->P.N, M = g->M;
    const orc_params *P = &g->P;
    const double kx = g->kf[2 * j], ky = g->kf[2 * j + 1], eta = P->eta;
    for (int m = 0; m < n_omega; ++m) { re[m] = 0.0; im[m] = 0.0; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *lre = (double *)calloc((size_t)n_omega, sizeof(double));
        double *lim = (double *)calloc((size_t)n_omega, sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int p = 0; p < M; ++p) {
            const int a = g->fpatch[p];
            const double px = g->fk[2 * p], py = g->fk[2 * p + 1];
            const double xp = orc_xi(P, px, py);
            const double fp = orc_fermi(xp, T), fpc = orc_fermi(-xp, T);
            for (int q = 0; q < M; ++q) {
                const int b = g->fpatch[q];
                const double qx = g->fk[2 * q], qy = g->fk[2 * q + 1];
                const double rx = kx + px - qx, ry = ky + py - qy;
                const int c = orc_proj(g, rx, ry);
                const double xq = orc_xi(P, qx, qy), xr = orc_xi(P, rx, ry);
                const double F = fp * orc_fermi(-xq, T) * orc_fermi(-xr, T)
                               + fpc * orc_fermi(xq, T) * orc_fermi(xr, T);
                const double vab = VV(j, a, b), vac = VV(j, a, c);
                const double lines = Z[a] * Z[b] * Z[c]
                    * (K[a] * Z[a] * (Z[b] + Z[c]) + K[b] * Z[b] * (Z[a] + Z[c]) + K[c] * Z[c] * (Z[a] + Z[b])) / 6.0;
                const double amp = g->fw[p] * g->fw[q] * lines * (2.0 * vab * vab - vab * vac) * F;
                const double E = xq + xr - xp;
                for (int m = 0; m < n_omega; ++m) {
                    double d = omega[m] - E, den = d * d + eta * eta;
                    lre[m] += amp * d / den;
                    lim[m] -= amp * eta / den;
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int m = 0; m < n_omega; ++m) { re[m] += lre[m]; im[m] += lim[m]; }
        free(lre);
        free(lim);
    }
    (void)nthreads;
}

/* frequencies of patch j: xi_j + 2T, xi_j - 2T, then the grid */
static void gflow_freqs(const orc_geom *g, const orc_gflow_opts *o, int j, double *w)
{
    const double T = g->P.T_fixed, xij = orc_xi(&g->P, g->kf[2 * j], g->kf[2 * j + 1]);
    w[0] = xij + 2.0 * T;
    w[1] = xij - 2.0 * T;
    for (int m = 0; m < o->n_omega; ++m) w[2 + m] = o->omega[m];
}

void orc_gflow_zka(const orc_geom *g, const orc_gflow_opts *o, double gv, const double *Sre, const double *Dre,
                   double *Z, double *K, double *A, double *Abar)
{
    const int N = g->P.N, nw = 2 + o->n_omega;
    const double T = g->P.T_fixed;
    /* A-bar runs over the Fermi surface (App. B): every patch of the angular  */
    /* modes, the Fermi shell s = n_s / 2 of every wedge in shell mode        */
    const int ns = g->P.mode == ORC_MODE_SHELL ? g->P.n_shell : 1;
    double sum = 0.0, amin = 0.0, amax = 0.0;
    int nfs = 0;
    for (int j = 0; j < N; ++j) {
        const double s1 = (Sre[j * nw] - Sre[j * nw + 1]) / (4.0 * T);
        const double s2 = (Dre[j * nw] - Dre[j * nw + 1]) / (4.0 * T);
        if (o->z_feedback) {
            Z[j] = 1.0 / (1.0 - gv * s1);
            K[j] = o->katanin ? 1.0 + gv * gv * s2 : 1.0;
            A[j] = 2.0 * Z[j] * (s1 + gv * s2);
        } else {
            Z[j] = 1.0;
            K[j] = 1.0;
            A[j] = 0.0;
        }
        if (j % ns != ns / 2) continue;
        sum += A[j];
        if (nfs == 0 || A[j] < amin) amin = A[j];
        if (nfs == 0 || A[j] > amax) amax = A[j];
        ++nfs;
    }
    switch (o->a_mode) {
    case ORC_A_MIN: *Abar = amin; break;
    case ORC_A_MAX: *Abar = amax; break;
    case ORC_A_DROP: *Abar = 0.0; break;
    default: *Abar = sum / nfs; break;
    }
}

/* right-hand side of the whole state at g = gv */
void orc_gflow_rhs(const orc_geom *g, const orc_gflow_opts *o, double gv, const double *V, const double *Sre,
                   const double *Sim, const double *Dre, const double *Dim, double *dV, double *dSre,
                   double *dSim, double *dDre, double *dDim, int nthreads)
{
    const int N = g->P.N, nw = 2 + o->n_omega;
    const long n3 = (long)N * N * N;
    double *Z = (double *)malloc(sizeof(double) * N), *K = (double *)malloc(sizeof(double) * N);
    double *A = (double *)malloc(sizeof(double) * N), *w = (double *)malloc(sizeof(double) * nw);
    double *tr = (double *)malloc(sizeof(double) * nw), *ti = (double *)malloc(sizeof(double) * nw);
    double Abar;
    orc_gflow_zka(g, o, gv, Sre, Dre, Z, K, A, &Abar);
    if (o->freeze_vertex) memset(dV, 0, sizeof(double) * n3);
    else rhs_k(g, gv, V, Z, K, dV, nthreads);
    for (int j = 0; j < N; ++j) {
        gflow_freqs(g, o, j, w);
        orc_sigma_gflow(g, g->P.T_fixed, V, Z, K, j, nw, w, tr, ti, nthreads);
        for (int m = 0; m < nw; ++m) {
            const int i = j * nw + m;
            dSre[i] = Dre[i];
            dSim[i] = Dim[i];
            dDre[i] = Abar * Dre[i] + 6.0 * gv * tr[m];
            dDim[i] = Abar * Dim[i] + 6.0 * gv * ti[m];
        }
    }
    free(Z); free(K); free(A); free(w); free(tr); free(ti);
}

/* RK4 in g over (V, Sigma, Sigma'); stops like orc_flow (divergence of max|V|
   with g_c interpolated in ln max|V|, end of the flow, non-finite state) */
int orc_gflow(const orc_geom *g, const orc_gflow_opts *o, double *V, double *Sre, double *Sim, double *Dre,
              double *Dim, orc_flow_result *res, int nthreads)
{
    const int N = g->P.N, nw = 2 + o->n_omega;
    const long n3 = (long)N * N * N, ns = (long)N * nw;
    const long tot = n3 + 4 * ns;
    memset(res, 0, sizeof(*res));
    if (g->P.regulator != ORC_REG_INTERACTION) { res->status = ORC_NONFINITE; return res->status; }
    double *y = (double *)malloc(sizeof(double) * tot), *ys = (double *)malloc(sizeof(double) * tot);
    double *k[4], *acc = (double *)malloc(sizeof(double) * tot);
    for (int s = 0; s < 4; ++s) k[s] = (double *)malloc(sizeof(double) * tot);
#define PACK(dst) do { memcpy(dst, V, sizeof(double) * n3); memcpy(dst + n3, Sre, sizeof(double) * ns); \
        memcpy(dst + n3 + ns, Sim, sizeof(double) * ns); memcpy(dst + n3 + 2 * ns, Dre, sizeof(double) * ns); \
        memcpy(dst + n3 + 3 * ns, Dim, sizeof(double) * ns); } while (0)
#define RHS(src, gv, out) orc_gflow_rhs(g, o, gv, src, src + n3, src + n3 + ns, src + n3 + 2 * ns, src + n3 + 3 * ns, \
        out, out + n3, out + n3 + ns, out + n3 + 2 * ns, out + n3 + 3 * ns, nthreads)
    PACK(y);
    double x = o->g0;
    int finite;
    double m = max_abs(y, n3, &finite);
    res->lambda = x;
    res->max_abs_v = m;
    for (int step = 0;; ++step) {
        if (o->g_end - x < 1e-12) { res->status = ORC_END; break; }
        if (step >= o->max_steps) { res->status = ORC_MAX_STEPS; break; }
        double h = o->dg;
        if (x + h > o->g_end) h = o->g_end - x;
        RHS(y, x, k[0]);
        for (long i = 0; i < tot; ++i) ys[i] = y[i] + 0.5 * h * k[0][i];
        RHS(ys, x + 0.5 * h, k[1]);
        for (long i = 0; i < tot; ++i) ys[i] = y[i] + 0.5 * h * k[1][i];
        RHS(ys, x + 0.5 * h, k[2]);
        for (long i = 0; i < tot; ++i) ys[i] = y[i] + h * k[2][i];
        RHS(ys, x + h, k[3]);
        for (long i = 0; i < tot; ++i) y[i] += h / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
        const double m_new = max_abs(y, n3, &finite);
        int fin_s = 1;
        max_abs(y + n3, 4 * ns, &fin_s);
        res->steps = step + 1;
        res->lambda = x + h;
        res->max_abs_v = m_new;
        if (!finite || !fin_s) { res->status = ORC_NONFINITE; x += h; break; }
        if (m_new > o->stop_abs_v) {
            const double sfrac = (log(o->stop_abs_v) - log(m)) / (log(m_new) - log(m));
            res->lambda_c = x + sfrac * h;
            res->status = ORC_DIVERGED;
            x += h;
            break;
        }
        x += h;
        m = m_new;
    }
#undef RHS
    memcpy(V, y, sizeof(double) * n3);
    memcpy(Sre, y + n3, sizeof(double) * ns);
    memcpy(Sim, y + n3 + ns, sizeof(double) * ns);
    memcpy(Dre, y + n3 + 2 * ns, sizeof(double) * ns);
    memcpy(Dim, y + n3 + 3 * ns, sizeof(double) * ns);
#undef PACK
    free(y); free(ys); free(acc);
    for (int s = 0; s < 4; ++s) free(k[s]);
    return res->status;
}

