// Real-frequency two-loop self-energy and the quasi-particle weight Z.
//
// Sigma(k_j, w) = sum_{p,q} w_p w_q Z_a Z_b Z_c W F / (w + i eta - E)
//   r = k_j + p - q,  E = x_q + x_r - x_p,
//   F = f_p (1-f_q)(1-f_r) + (1-f_p) f_q f_r,
//   W = 2 V(k_j,p,q)^2 - V(k_j,p,q) V(k_j,p,r),
// a, b, c the patches of p, q, r (the two-loop term of Sec. A.2/A.3 with the
// static vertex and Z-weighted lines).  Z_j = (1 - slope)^-1, Eq.
// (definition_Z), with the slope the chord of Re Sigma over xi_j +- 2T
// ("from outside", Sec. 3.1.1).
//
// sigma_kernel<R,false> evaluates Re Sigma exactly at the two chord frequencies.
// Launch shape: grid (q blocks, patch a of p, target j), 256 threads, one q
// per thread; the CTA stages patch a's points (k_j + p, cos/sin, Fermi
// factors) and the vertex row V[j][a][:] in shared memory and loops over
// them.  In the flow only the C4v-irreducible patches 0..N/8 are evaluated
// (the vertex and Z keep the lattice symmetry) and Z is copied to their
// images.  sigma_kernel<R,true> bins W F by pole energy E with moments 0..4 for
// the frequency grid; sigma_grid_kernel resums the moments on the grid.
#include <algorithm>

#include "atan_poly.h"
#include "qpfrg_internal.h"

namespace qpfrg {

__device__ __forceinline__ float sexp(float x) { return __expf(x); }
__device__ __forceinline__ double sexp(double x) { return exp(x); }
// typed absolute value: plain sabs() on a float would promote to FP64
__device__ __forceinline__ float sabs(float x) { return fabsf(x); }
__device__ __forceinline__ double sabs(double x) { return fabs(x); }
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float srint(float x) { return rintf(x); }
__device__ __forceinline__ double srint(double x) { return rint(x); }
__device__ __forceinline__ float satan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double satan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float sfloor(float x) { return floorf(x); }
__device__ __forceinline__ double sfloor(double x) { return floor(x); }

// f(x) and 1 - f(x) without cancellation: with e = exp(-|x|/T) they are
// e/(1+e) and 1/(1+e), one reciprocal.
template <typename R>
__device__ __forceinline__ void sfermi(R x, R invT, R &f, R &fc)
{
    const R e = sexp(-sabs(x) * invT);
    const R hi = sdiv(R(1), R(1) + e), lo = e * hi;
    f = x > R(0) ? lo : hi;
    fc = x > R(0) ? hi : lo;
}

// atan2 in FP32 from the odd polynomial t P(t^2), t = min/max on [0, 1], a
// Remez minimax fit of atan(t) (degree 11; coefficients and the error bound
// kAtanErr = 1.75e-6 rad of the FP32 evaluation generated by atan_fit.py into
// atan_poly.h), then octant reflections.  Caller guarantees (x, y) != (0, 0).
__device__ __forceinline__ float atan2_poly(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float t = __fdividef(fminf(ax, ay), fmaxf(ax, ay));
    const float s = t * t;
    float p = fmaf(s, kAtanC5, kAtanC4);
    p = fmaf(s, p, kAtanC3);
    p = fmaf(s, p, kAtanC2);
    p = fmaf(s, p, kAtanC1);
    p = fmaf(s, p, kAtanC0);
    float a = t * p;
    if (ay > ax) a = 1.57079633f - a;
    if (x < 0.f) a = 3.14159265f - a;
    return copysignf(a, y);
}

// Round to nearest even without a conversion instruction (|x| < 2^22): the
// float sum with 1.5 * 2^23 keeps rint(x) in its low mantissa bits.
__device__ __forceinline__ float rint_add(float x, int &as_int)
{
    const float s = x + 12582912.f;
    as_int = __float_as_int(s) - 0x4B400000;
    return s - 12582912.f;
}

// FP32 wedge projection with a guard band: the FP32 momentum carries an
// absolute error below 1.4e-6 per component (FP32 rounding of k+p, q, their
// difference and the fold) and atan2_poly below 2.3e-6 rad (kAtanErr, the
// approximate quotient t and the rounding of the octant reflections), so the angle is
// trusted only when it lies more than 8e-6 + 8e-6/|r| rad from a wedge
// boundary and the point is more than 4e-6 from the zone edge.  Returns -1
// near a wedge boundary, -2 near the zone edge or the origin; jc gets the
// nearest-centre estimate.
__device__ __forceinline__ void fold32(float rx, float ry, float &x, float &y)
{
    const float tp = 6.28318531f;
    int ix;
    x = rx - tp * rint_add(rx * 0.159154943f, ix);
    y = ry - tp * rint_add(ry * 0.159154943f, ix);
}

// (x, y) already folded.
__device__ __forceinline__ int project32_guarded(float x, float y, int N, float inv_dth, float dth, int &jc)
{
    const float r2 = x * x + y * y;
    const float u = atan2_poly(y, x) * inv_dth;      // angle in units of the wedge width
    int j;
    const float fj = rint_add(u, j);                 // nearest centre
    jc = j;
    if (fabsf(x) > 3.14159265f - 4e-6f || fabsf(y) > 3.14159265f - 4e-6f || r2 < 1e-8f) return -2;
    const float m = (0.5f - fabsf(u - fj)) * dth;    // distance to the nearest boundary, rad
    if (m < 8e-6f || m * m * r2 < 6.4e-11f) return -1;
    if (j < 0) j += N;
    if (j >= N) j -= N;
    return j;
}

// Error-free transformations on the FP32 pipes (float-float arithmetic).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// sign of cross(b, x) = b_c x_y - b_s x_x with b and x as float-float pairs;
// accurate to ~1e-14 of |b||x|
__device__ __forceinline__ float cross_ff(float4 b, float xh, float xl, float yh, float yl)
{
    const float p1 = b.x * yh, e1 = fmaf(b.x, yh, -p1);
    const float p2 = b.z * xh, e2 = fmaf(b.z, xh, -p2);
    float s, es;
    two_sum(p1, -p2, s, es);
    const float t = es + e1 - e2 + b.x * yl + b.y * yh - b.z * xl - b.w * xh;
    return s + t;
}

// Guarded cases away from the zone edge: r = (k+p) - q in float-float, folded
// (|r| < 3 pi; the fold decision is safe away from the zone edge), then the
// point is tested against the boundary rays of the estimated wedge and its
// neighbours.  bnd[m] = (cos hi, cos lo, sin hi, sin lo) of the ray between
// wedges m-1 and m, at angle (m - 1/2) 2 pi / N.
__device__ __forceinline__ int project_ff(float kph, float kpl, float kqh, float kql, float qxh, float qxl,
                                          float qyh, float qyl, int jc, int N, const float4 *bnd)
{
    const float C1 = 6.28318548f, C2 = -1.7484555e-7f;   // 2 pi = C1 + C2 (float-float)
    float xh, xl, yh, yl, e;
    two_sum(kph, -qxh, xh, e);
    xl = e + (kpl - qxl);
    two_sum(kqh, -qyh, yh, e);
    yl = e + (kql - qyl);
    const float kx_ = xh > 3.14159265f ? 1.f : (xh < -3.14159265f ? -1.f : 0.f);
    const float ky_ = yh > 3.14159265f ? 1.f : (yh < -3.14159265f ? -1.f : 0.f);
    two_sum(xh, -kx_ * C1, xh, e);
    xl = xl + e - kx_ * C2;
    two_sum(yh, -ky_ * C1, yh, e);
    yl = yl + e - ky_ * C2;
    int j = jc;
    for (int it = 0; it < 3; ++it) {
        const int jj = j < 0 ? j + N : (j >= N ? j - N : j);
        const int jn = jj + 1 == N ? 0 : jj + 1;
        const bool ccw_lo = cross_ff(bnd[jj], xh, xl, yh, yl) >= 0.f;   // on or after the lower ray
        const bool cw_hi = cross_ff(bnd[jn], xh, xl, yh, yl) < 0.f;     // before the upper ray
        if (ccw_lo && cw_hi) return jj;
        j = ccw_lo ? jj + 1 : jj - 1;
    }
    return j < 0 ? j + N : (j >= N ? j - N : j);
}

// Per target and loop point, once per self-energy call: k_j + p as FP32
// hi/lo pairs (from the FP64 sum, the same sum as the FP64 path) and, per
// target, cos/sin of k_j's components.
__global__ void kp_table_kernel(const double *kf, const int *jlist, int nj, const double *kx64, const double *ky64,
                                int M, float4 *kp, float4 *kcs)
{
    const long total = (long)nj * M;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int ji = (int)(idx / M), p = (int)(idx - (long)ji * M);
        const int j = jlist ? jlist[ji] : ji;
        const double x = kf[2 * j] + kx64[p], y = kf[2 * j + 1] + ky64[p];
        const float xh = (float)x, yh = (float)y;
        kp[idx] = make_float4(xh, (float)(x - xh), yh, (float)(y - yh));
        if (p == 0) {
            double sx, cx, sy, cy;
            sincos(kf[2 * j], &sx, &cx);
            sincos(kf[2 * j + 1], &sy, &cy);
            kcs[ji] = make_float4((float)cx, (float)sx, (float)cy, (float)sy);
        }
    }
}

template <typename R>
struct SigmaArgs {
    Problem pb;
    FineTable<R> fine;
    const double *kf;    // N x 2
    const double *V;     // N^3 FP64
    const double *Z;     // N
    // interaction flow with the self-energy ODE: Katanin factors per patch
    // (NULL otherwise); the lines then carry the weights of a G, an S and an
    // inner K S line averaged over their assignments (see gflow.cu)
    const double *K;
    double *sig;         // [target]: chord slope of Re Sigma over xi_j +- 2T
    double T;
    int nj;
    const int *jlist;    // targets (may be NULL: j = blockIdx.z)
    const double *kx64, *ky64;  // FP64 fine momenta (guarded FP32 projection)
    const double *xij;          // xi(k_F(j)), FP64
    const float4 *bnd;          // boundary rays of the wedges, float-float (FP32 projection fallback)
    const float4 *kp;           // [target][p]: k_j + p as (x hi, x lo, y hi, y lo)
    const float4 *kcs;          // [target]: cos, sin of k_j's components
    const float *qxl, *qyl;     // FP32 residuals of the fine momenta
    // scalars of the inner loop in R (a double scalar re-read inside the loop
    // would cost a conversion on the FP64 pipe per use)
    R t_r, tp_r, mu_r, eta_r, invT_r, twoT_r;
    const R *xij_r;             // xi(k_F(j)) in R
    // frequency-grid histogram (sigma_hist_kernel)
    double *hist;        // [j][moment 0..4][bin]
    double e_min, inv_h;
    int nbins;
};

// Shared-memory record of one loop point p of patch a, for target k_j:
// k+p (x, y), cos/sin of its components, line energy x_p, f_p, 1-f_p, w_p.
constexpr int REC = 12;

__device__ __forceinline__ void load_rec(const float *base, int i, float (&r)[REC])
{
    const float4 *p = reinterpret_cast<const float4 *>(base + REC * i);
    const float4 a = p[0], b = p[1], c = p[2];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
    r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
}

__device__ __forceinline__ void load_rec(const double *base, int i, double (&r)[REC])
{
    const double2 *p = reinterpret_cast<const double2 *>(base + REC * i);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double2 v = p[k];
        r[2 * k] = v.x;
        r[2 * k + 1] = v.y;
    }
    r[10] = r[11] = 0.0;
}

template <typename R, bool HIST>
__global__ void __launch_bounds__(256) sigma_kernel(SigmaArgs<R> A)
{
    const int N = A.pb.N, P = A.pb.P, M = A.pb.M;
    const int a = blockIdx.y;
    const int jidx = blockIdx.z;
    const int j = A.jlist ? A.jlist[jidx] : jidx;
    const int tid = threadIdx.x;
    const bool qp = A.pb.propagator == QPFRG_PROP_QP;
    // wedge and shell modes: the FP32 path decides the wedge by guarded ray
    // tests (and the shell by the FP32 line energy, guarded)
    const bool angular = A.pb.mode == QPFRG_GRID_WEDGE || A.pb.mode == QPFRG_GRID_SHELL;
    const int ns = A.pb.n_shell, Na = N / ns;
    const R invT = A.invT_r, eta = A.eta_r;
    const R t = A.t_r, tp = A.tp_r, mu = A.mu_r;
    constexpr bool f32 = sizeof(R) == 4;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *s_rec = reinterpret_cast<R *>(smem_raw);          // P x REC
    R *s_VZ = s_rec + (size_t)REC * P;                   // N x {V[j][a][c], Z_c}
    float4 *s_bnd = reinterpret_cast<float4 *>(s_VZ + 2 * N + (2 * N * sizeof(R)) % 16 / sizeof(R));
    R *s_K = reinterpret_cast<R *>(s_bnd + N);           // N Katanin factors (interaction-flow lines)

    const double kx = A.kf[2 * j], ky = A.kf[2 * j + 1];
    for (int i = tid; i < N; i += blockDim.x) {
        s_VZ[2 * i] = (R)A.V[((long)j * N + a) * N + i];
        s_VZ[2 * i + 1] = A.Z ? (R)A.Z[i] : R(1);
        if (f32 && angular) s_bnd[i] = A.bnd[i];
        if (A.K) s_K[i] = (R)A.K[i];
    }
    __shared__ R s_k[4];
    if (tid == 0) {
        if (f32) {
            const float4 k4 = A.kcs[jidx];
            s_k[0] = (R)k4.x; s_k[1] = (R)k4.y; s_k[2] = (R)k4.z; s_k[3] = (R)k4.w;
        } else {
            double sx, cx, sy, cy;
            sincos(kx, &sx, &cx);
            sincos(ky, &sy, &cy);
            s_k[0] = (R)cx; s_k[1] = (R)sx; s_k[2] = (R)cy; s_k[3] = (R)sy;
        }
    }
    __syncthreads();
    const R Za = s_VZ[2 * a + 1];
    const R ckx = s_k[0], skx = s_k[1], cky = s_k[2], sky = s_k[3];
    // records in angular-minor order: storage index s * n_theta + t for the
    // point (t, s), so consecutive records are angular neighbours
    const int nt = A.pb.n_theta, nr = A.pb.n_r;
    for (int i = tid; i < P; i += blockDim.x) {
        const int p = a * P + (i % nt) * nr + i / nt;
        R *rec = s_rec + (size_t)REC * i;
        if (f32) {
            // k_j + p as FP32 hi/lo pairs from the per-call table
            const float4 k4 = A.kp[(long)jidx * M + p];
            rec[0] = (R)k4.x;
            rec[10] = (R)k4.y;
            rec[1] = (R)k4.z;
            rec[11] = (R)k4.w;
        } else {
            rec[0] = (R)(kx + A.kx64[p]);
            rec[1] = (R)(ky + A.ky64[p]);
            rec[10] = rec[11] = R(0);
        }
        const R cpx = A.fine.cx[p], spx = A.fine.sx[p], cpy = A.fine.cy[p], spy = A.fine.sy[p];
        rec[2] = ckx * cpx - skx * spx;
        rec[3] = skx * cpx + ckx * spx;
        rec[4] = cky * cpy - sky * spy;
        rec[5] = sky * cpy + cky * spy;
        const R xp = qp ? Za * A.fine.xi[p] : A.fine.xi[p];
        rec[6] = xp;
        R f, fc;
        sfermi(xp, invT, f, fc);
        rec[7] = f;
        rec[8] = fc;
        rec[9] = A.fine.w[p];
    }
    __syncthreads();

    const int q = blockIdx.x * blockDim.x + tid;
    R acc = R(0);
    if (q < M) {
        const int b = q / P;
        const R qx = A.fine.kx[q], qy = A.fine.ky[q];
        const double qxd = A.kx64[q], qyd = A.ky64[q];
        const float qxl = f32 ? A.qxl[q] : 0.f, qyl = f32 ? A.qyl[q] : 0.f;
        const R cqx = A.fine.cx[q], sqx = A.fine.sx[q], cqy = A.fine.cy[q], sqy = A.fine.sy[q];
        const R Zb = s_VZ[2 * b + 1];
        const R xq = qp ? Zb * A.fine.xi[q] : A.fine.xi[q];
        R fq, fcq;
        sfermi(xq, invT, fq, fcq);
        const R vab = s_VZ[2 * b];
        const R pref = Za * Zb * A.fine.w[q];
        const bool glines = A.K != nullptr;
        const R uab = glines ? s_K[a] * Za * Zb + s_K[b] * Zb * Za : R(0);   // K_a Z_a Z_b + K_b Z_b Z_a
        const R kza = glines ? s_K[a] * Za : R(0), kzb = glines ? s_K[b] * Zb : R(0);
        const R d0shift = A.xij_r[j], twoT = A.twoT_r;
        const R eta2 = eta * eta;
        const float inv_dth = (float)(Na / kTwoPi), dth = (float)(kTwoPi / Na);
        const float invD = ns > 1 ? (float)(1.0 / A.pb.shell_D) : 0.f, half_ns = 0.5f * ns;
        // guard band of the shell decision in units of the shell width: ten
        // times the error bound of the FP32 line energy (products of FP32-rounded
        // cosines: 1.2e-6 per unit of 2|t| + 4|t'|, 1.2e-7 |mu|) plus the
        // rounding of u itself
        const float gu = 10.f * (1.2e-6f * (2.f * fabsf((float)A.pb.t) + 4.f * fabsf((float)A.pb.tp)) +
                                 1.2e-7f * fabsf((float)A.pb.mu)) * invD + 1e-6f;
        // wedge of the previous pair and its two boundary rays (FP32)
        int cprev = -1;
        float blx = 0.f, bly = 0.f, bhx = 0.f, bhy = 0.f;
        for (int i = 0; i < P; ++i) {
            R r[REC];
            load_rec(s_rec, i, r);
            // cos(k+p-q) by angle addition, and the bare line energy of r
            const R crx = r[2] * cqx + r[3] * sqx;
            const R cry = r[4] * cqy + r[5] * sqy;
            R xr = R(-2) * t * (crx + cry) - R(4) * tp * crx * cry - mu;
            int c = -1;
            if (f32 && angular) {
                float x, y;
                fold32((float)(r[0] - qx), (float)(r[1] - qy), x, y);
                // inside the previous pair's wedge by more than the FP32 error
                // of (x, y) (2.1e-6) plus that of the rays: same wedge
                const bool edge = fabsf(x) > 3.14159265f - 4e-6f || fabsf(y) > 3.14159265f - 4e-6f;
                int cw;
                if (!edge && cprev >= 0 && blx * y - bly * x >= 4e-6f && bhx * y - bhy * x <= -4e-6f) {
                    cw = cprev;
                } else {
                    int jc;
                    cw = project32_guarded(x, y, Na, inv_dth, dth, jc);
                    if (cw == -1) {
                        // near a wedge boundary: float-float decision on the FP32 pipes
                        cw = project_ff((float)r[0], (float)r[10], (float)r[1], (float)r[11], (float)qx, qxl,
                                        (float)qy, qyl, jc, Na, s_bnd);
                    } else if (cw == -2) {
                        // zone edge or origin: the exact FP64 projection
                        const int p = a * P + (i % nt) * nr + i / nt;
                        c = project_fp64((kx + A.kx64[p]) - qxd, (ky + A.ky64[p]) - qyd, A.pb);
                        cw = c / ns;
                    }
                    cprev = cw;
                    const float4 lo = s_bnd[cw], hi = s_bnd[cw + 1 == Na ? 0 : cw + 1];
                    blx = lo.x; bly = lo.z; bhx = hi.x; bhy = hi.z;
                }
                if (c < 0) {
                    if (ns == 1) {
                        c = cw;
                    } else {
                        // shell of the FP32 line energy; within the guard band of
                        // a shell edge the exact FP64 projection decides
                        const float u = (float)xr * invD + half_ns;
                        const float ur = rintf(u);
                        if (fabsf(u - ur) < gu && ur >= 1.f && ur <= (float)(ns - 1)) {
                            const int p = a * P + (i % nt) * nr + i / nt;
                            c = project_fp64((kx + A.kx64[p]) - qxd, (ky + A.ky64[p]) - qyd, A.pb);
                        } else {
                            int sh = (int)floorf(u);
                            sh = sh < 0 ? 0 : (sh > ns - 1 ? ns - 1 : sh);
                            c = cw * ns + sh;
                        }
                    }
                }
            } else {
                const int p = a * P + (i % nt) * nr + i / nt;
                c = project_fp64((kx + A.kx64[p]) - qxd, (ky + A.ky64[p]) - qyd, A.pb);
            }
            const R vac = s_VZ[2 * c], Zc = s_VZ[2 * c + 1];
            if (qp) xr *= Zc;
            R fr, fcr;
            sfermi(xr, invT, fr, fcr);
            const R F = r[7] * fcq * fcr + r[8] * fq * fr;
            R amp = r[9] * pref * Zc * (R(2) * vab * vab - vab * vac) * F;
            if (glines)   // (1/6)[K_a Z_a (Z_b + Z_c) + K_b Z_b (Z_a + Z_c) + K_c Z_c (Z_a + Z_b)]
                amp *= (uab + Zc * (kza + kzb) + s_K[c] * Zc * (Za + Zb)) * R(1.0 / 6.0);
            const R E = xq + xr - r[6];
            if (HIST) {
                const double eb = ((double)E - A.e_min) * A.inv_h;
                int bin = (int)floor(eb);
                bin = bin < 0 ? 0 : (bin >= A.nbins ? A.nbins - 1 : bin);
                const double d = (double)E - (A.e_min + (bin + 0.5) / A.inv_h);
                double *h = A.hist + ((long)jidx * 5) * A.nbins + bin;
                double m = (double)amp;
#pragma unroll
                for (int mo = 0; mo < 5; ++mo) {
                    atomicAdd(h + (long)mo * A.nbins, m);
                    m *= d;
                }
            } else {
                // chord slope of Re 1/(w - E + i eta) over w = xi_j +- 2T:
                // [d+/(d+^2+eta^2) - d-/(d-^2+eta^2)] / 4T
                //   = (eta^2 - d+ d-) / ((d+^2 + eta^2)(d-^2 + eta^2))
                const R d0 = d0shift - E;
                const R dp = d0 + twoT, dm = d0 - twoT;
                acc += amp * sdiv(eta2 - dp * dm, (dp * dp + eta2) * (dm * dm + eta2));
            }
        }
    }
    if (HIST) return;
    // block reduction of the partial slopes
    __shared__ double red[32];
    double v = (double)acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(&A.sig[jidx], v);
    }
}

// ---------------------------------------------------------------------------
// FP32 chord-slope kernel of the wedge grid (the flow's self-energy).
//
// Same sum as sigma_kernel<float,false>, arranged for instruction count:
// * momenta are fixed-point turns (angle_fx), so r = k_j + p - q folds by
//   integer wrap-around; the patch c of r comes from a shared-memory cell
//   table over the folded zone indexed by the top bytes (one byte per cell:
//   the lower of the at most two wedges the cell touches) and one FP32 test
//   against the ray between them; cells near the origin, points within 4e-6
//   of a ray and points within 4e-6 of the zone edge take the guarded paths
//   of sigma_kernel (float-float rays, exact FP64 projection), so every patch
//   decision equals the FP64 one;
// * f_r enters only through F = A + f_r (B - A) with A = w_p f_p (1 - f_q),
//   B = w_p (1 - f_p) f_q (times Z_a Z_b w_q), so one exp2 and one
//   reciprocal give it;
// * per patch c the table cz holds (Z_c, Z_c V[j][a][c], -2t l_c, -mu l_c)
//   times (1, 1, log2(e)/T, log2(e)/T), l_c = Z_c for quasi-particle lines
//   (else 1), so the line energy of r (Z-scaled, in units of T/log2(e)) is one
//   FMA from cos(r_x) + cos(r_y) and feeds exp2 directly;
// * with d0 = xi_j - E the chord term is -u / (u^2 + 4 eta^2 d0^2),
//   u = d0^2 - 4T^2 - eta^2 (the product of the two Lorentzian denominators
//   written out);
// * each thread owns SF_QPT = 2 loop points q, so a record of p read from
//   shared memory serves two pairs, whose arithmetic runs as the two lanes of
//   packed FP32x2 instructions (Fermi factor, weight, chord term, sum), and
//   cos r_x, cos r_y of one pair form one packed FMA pair; the lanes of a warp own angular neighbours at
//   one radius (angular-minor order), so their r lie on a short arc and their
//   table cells, rays and patch slots mostly coincide (few bank conflicts,
//   rare divergence into the guarded paths).
// Launch: grid (ceil(M / (256 SF_QPT qb)), N patches a, targets), 256 threads,
// two CTAs per SM.
constexpr int SF_QPT = 2;
constexpr int SF_QB = 4;        // default blocks of 256 SF_QPT loop points q per CTA
constexpr int SF_PCH = 1024;    // loop points p staged per pass
constexpr int SF_SLOTS = 257;   // per-patch slots: c in 0..N (c = N is patch 0 again), padded to 257

struct SigmaFastArgs {
    Problem pb;
    FineTable<float> fine;
    const double *V, *Z, *kx64, *ky64, *kf;
    const float *xij_f, *qxl, *qyl;
    const float4 *kp, *kcs, *bnd;
    const uint8_t *ptab;
    const uint8_t *rtab;    // patch of r per (target, p, q) (RT launches; rtab_build_kernel)
    const int *jlist;
    double *sig;
    float t, tp, mu, eta2, invT, cT, twoT, fourT;   // cT = log2(e) / T
    float tln2, kchord, eta2x4;                     // T ln 2, 4 T^2 + eta^2, 4 eta^2
    float inv_dth, dth;                             // N / 2 pi, 2 pi / N
    int mirror;     // n_theta even and symmetric targets: 1 halves every mirror-line target,
                    // 2 all but the zone-edge ones (j a multiple of N/4)
    int qb;         // blocks of 256 SF_QPT loop points q per CTA
    // grid mode: pole energies E binned from e_min in bins of h, moments 0..4
    // of the offset from the bin centre, hist[target][moment][bin] (FP64)
    double *hist;
    float e_min, inv_h, h;
    int nbins;
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Table patch of r = (k+p) - q from fixed-point components: the lower wedge e
// of the cell and the side of the ray between e and e + 1 (c = e or e + 1).
// slow: within the guard band of that ray, of the zone edge, or in a cell of
// three or more wedges (e = 255 reads the zero ray 256, cr = 0).  tabc points
// at the cell of the origin; x, y come back in fixed-point units.
__device__ __forceinline__ int fx_patch(int kpx, int kpy, int qx, int qy, const unsigned char *tabc,
                                        const float2 *ray, float &x, float &y, bool &slow)
{
    const int X = (int)((unsigned)kpx - (unsigned)qx);
    const int Y = (int)((unsigned)kpy - (unsigned)qy);
    x = __int2float_rn(X);
    y = __int2float_rn(Y);
    const int e = tabc[(Y >> 24) * kProjStride + (X >> 24)];
    const float2 rr = ray[e + 1];
    const float cr = rr.x * y - rr.y * x;
    slow = fmaxf(fabsf(x), fabsf(y)) > kFxEdge || fabsf(cr) < kFxGuard;
    return e + (cr >= 0.f ? 1 : 0);
}

struct SfSmem {
    size_t rA, rB, cz, ray, cd, rC, tab, hist, total;
};

// nbins > 0: a histogram of nbins x 5 FP32 moments follows the table (grid mode)
__host__ __device__ inline SfSmem sf_smem_layout(int pch, int nbins = 0)
{
    SfSmem L;
    L.rA = 0;                                  // pch + 1 records: room for a pad record
    L.rB = L.rA + (size_t)16 * (pch + 1);
    L.cz = L.rB + (size_t)16 * (pch + 1);
    L.ray = L.cz + (size_t)16 * SF_SLOTS;
    L.cd = L.ray + (size_t)8 * SF_SLOTS;
    L.rC = (L.cd + (size_t)4 * SF_SLOTS + 15) / 16 * 16;
    L.tab = (L.rC + (size_t)4 * (pch + 1) + 15) / 16 * 16;
    L.hist = L.tab + ((size_t)kProjW * kProjStride + 15) / 16 * 16;
    L.total = L.hist + (size_t)5 * 4 * nbins;
    return L;
}

// Patch of r for a lane that left the table path: near a ray or the origin
// (float-float ray tests) or near the zone edge (FP64 projection).
__device__ __noinline__ int sf_slow_patch(const SigmaFastArgs &A, int jidx, int j, int p, int q, float x, float y,
                                          bool edge, const float4 *bnd)
{
    const int N = A.pb.N;
    int c = -2;
    if (!edge) {
        int jc;
        c = project32_guarded(x, y, N, A.inv_dth, A.dth, jc);
        if (c == -1) {
            const float4 k4 = A.kp[(long)jidx * A.pb.M + p];
            c = project_ff(k4.x, k4.y, k4.z, k4.w, A.fine.kx[q], A.qxl[q], A.fine.ky[q], A.qyl[q], jc, N, bnd);
        }
    }
    if (c < 0)
        c = project_fp64((A.kf[2 * j] + A.kx64[p]) - A.kx64[q], (A.kf[2 * j + 1] + A.ky64[p]) - A.ky64[q], A.pb);
    return c;
}

// The patch of r = k_j + p - q for every target of the list (position jidx),
// every loop point p = a P + i and every loop point q (angular-minor index iq,
// the order in which sigma_fast_kernel walks them), one byte each at
// rtab[(((jidx N + a) P/8 + i/8) M + iq) 8 + i % 8]: a thread reads the bytes
// of eight records as one 8-byte word, and the words of a warp's 32 loop
// points q are contiguous (256 B): the same decisions as the kernel's table
// path and its guarded slow path, so a launch that reads them gives the same
// sums.  They depend on the geometry only (targets, fine grid), so one build
// serves every later call.  Grid (ceil(M / 256), N, targets), 256 threads.
constexpr size_t kRtabTabBytes = ((size_t)kProjW * kProjStride + 15) / 16 * 16;
constexpr size_t kRtabSmem = kRtabTabBytes + (size_t)SF_SLOTS * sizeof(float2);   // + P int2 records

__global__ void __launch_bounds__(256) rtab_build_kernel(SigmaFastArgs A, uint8_t *__restrict__ rtab)
{
    const int N = A.pb.N, M = A.pb.M, PP = A.pb.P;
    const int a = blockIdx.y, jidx = blockIdx.z;
    const int j = A.jlist ? A.jlist[jidx] : jidx;
    const int tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *tab = smem_raw;                                      // the cell table
    float2 *ray = reinterpret_cast<float2 *>(smem_raw + kRtabTabBytes); // rays between wedges
    int2 *rec = reinterpret_cast<int2 *>(ray + SF_SLOTS);               // k_j + p of the patch (fixed point)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(A.ptab);
        uint4 *dst = reinterpret_cast<uint4 *>(tab);
        const int n16 = (kProjW * kProjStride + 15) / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
        for (int i = tid; i < SF_SLOTS; i += blockDim.x) {
            const float4 bd = A.bnd[i == N ? 0 : (i < N ? i : 0)];
            ray[i] = i <= N ? make_float2(bd.x, bd.z) : make_float2(0.f, 0.f);
        }
        for (int i = tid; i < PP; i += blockDim.x) {
            const float4 k4 = A.kp[(long)jidx * M + a * PP + i];
            rec[i] = make_int2(angle_fx((double)k4.x + (double)k4.y), angle_fx((double)k4.z + (double)k4.w));
        }
    }
    __syncthreads();
    const unsigned char *tabc = tab + (kProjW / 2) * (kProjStride + 1);   // the cell of the origin
    const int iq = blockIdx.x * 256 + tid;
    if (iq >= M) return;
    const int b = iq / PP, rem = iq - b * PP;
    const int qq = b * PP + (rem % A.pb.n_theta) * A.pb.n_r + rem / A.pb.n_theta;
    const int qx = angle_fx(A.kx64[qq]), qy = angle_fx(A.ky64[qq]);
    // the thread's P bytes, as P/8 words of eight records (P a multiple of 16)
    uint2 *out = reinterpret_cast<uint2 *>(rtab) + ((long)jidx * N + a) * (long)(PP / 8) * M + iq;
    for (int i0 = 0; i0 < PP; i0 += 8) {
        unsigned w[2] = {0u, 0u};
        for (int i = i0; i < i0 + 8; ++i) {
            const int p = a * PP + i;
            const int2 kr = rec[i];
            float x, y;
            bool slow;
            int c = fx_patch(kr.x, kr.y, qx, qy, tabc, ray, x, y, slow);
            if (slow) {
                const bool edge = fmaxf(fabsf(x), fabsf(y)) > kFxEdge;
                c = sf_slow_patch(A, jidx, j, p, qq, x * kRadPerFx, y * kRadPerFx, edge, A.bnd);
            }
            w[(i - i0) >> 2] |= (unsigned)c << (8 * ((i - i0) & 3));
        }
        out[(long)(i0 >> 3) * M] = make_uint2(w[0], w[1]);
    }
}

// UNIB: every block of 256 SF_QPT loop points q lies in one patch b (P a
// multiple of 256 SF_QPT), so the vertex weight is a per-patch table:
// cz[c] = (Z_c (2 V_jab^2 - V_jab V_jac), -, -2t l_c, -mu l_c); otherwise
// cz[c] = (Z_c, Z_c V_jac, -2t l_c, -mu l_c) and the weight is formed per pair.
template <bool TP0, bool UNIB, bool RT>
__global__ void __launch_bounds__(256, 2) sigma_fast_kernel(SigmaFastArgs A)
{
    const int N = A.pb.N, M = A.pb.M;
    const int a = blockIdx.y, jidx = blockIdx.z;
    const int j = A.jlist ? A.jlist[jidx] : jidx;
    const int tid = threadIdx.x;
    const bool qp = A.pb.propagator == QPFRG_PROP_QP;
    // A target on a mirror line of the zone (theta_j = 0 or pi/4) has a sum
    // symmetric under that mirror: keep the patches a on one side of it with
    // weight 2 and half of each patch the mirror maps onto itself.
    int fac = 1, P = A.pb.P;
    if (A.mirror) {
        int ma = -1;
        if (j == 0) ma = (N - a) % N;
        else if (8 * j == N) ma = ((N / 4 - a) % N + N) % N;
        if (ma == a) {
            fac = 2;
            P = A.pb.P / 2;     // angular index t < n_theta / 2
        } else if (ma >= 0) {
            const int rel = j == 0 ? a : ((a - N / 8) % N + N) % N;
            fac = (rel > 0 && 2 * rel < N) ? 2 : 0;
        }
    }
    if (fac == 0) return;       // the mirror patch carries this one (uniform over the CTA)
    const int PP = A.pb.P;      // points per patch (record and loop-point indexing)
    const int pch = P < SF_PCH ? P : SF_PCH;
    const SfSmem L = sf_smem_layout(pch);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *rA = reinterpret_cast<float4 *>(smem_raw + L.rA);   // (k+p)_x, (k+p)_y (fixed point), cos of both
    float4 *rB = reinterpret_cast<float4 *>(smem_raw + L.rB);   // sin of both, w_p f_p, w_p (1 - f_p)
    float4 *cz = reinterpret_cast<float4 *>(smem_raw + L.cz);
    float2 *ray = reinterpret_cast<float2 *>(smem_raw + L.ray);
    float *cd = reinterpret_cast<float *>(smem_raw + L.cd);     // -4 t' l_c
    float *rC = reinterpret_cast<float *>(smem_raw + L.rC);     // x_j + x_p + 2T
    unsigned char *tab = smem_raw + L.tab;

    if (!RT) {
        const uint4 *src = reinterpret_cast<const uint4 *>(A.ptab);
        uint4 *dst = reinterpret_cast<uint4 *>(tab);
        const int n16 = (kProjW * kProjStride + 15) / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    const double *Vja = A.V + ((long)j * N + a) * N;
    // per-patch slots; with UNIB the weight column is filled per q block (b)
    auto fill_slots = [&](int b) {
        const float vb = UNIB ? (float)Vja[b] : 0.f;
        for (int i = tid; i < SF_SLOTS; i += blockDim.x) {
            if (i <= N) {
                const int cc = i == N ? 0 : i;
                const float Zc = A.Z ? (float)A.Z[cc] : 1.f;
                const float lz = qp ? Zc : 1.f;
                const float vc = (float)Vja[cc];
                const float lzc = lz * A.cT;     // energies of r in units of T / log2(e)
                cz[i] = UNIB ? make_float4(Zc * (2.f * vb * vb - vb * vc), 0.f, -2.f * A.t * lzc, -A.mu * lzc)
                             : make_float4(Zc, Zc * vc, -2.f * A.t * lzc, -A.mu * lzc);
                cd[i] = -4.f * A.tp * lzc;
                const float4 bd = A.bnd[cc];
                ray[i] = make_float2(bd.x, bd.z);
            } else {
                cz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                cd[i] = 0.f;
                ray[i] = make_float2(0.f, 0.f);
            }
        }
    };
    int b_slots = UNIB ? (blockIdx.x * A.qb * 256 * SF_QPT) / PP : 0;
    fill_slots(b_slots);
    const float Za = A.Z ? (float)A.Z[a] : 1.f;
    const float lza = qp ? Za : 1.f;
    const float4 kcs = A.kcs[jidx];
    const float xj = A.xij_f[j];

    const unsigned char *tabc = tab + (kProjW / 2) * (kProjStride + 1);   // the cell of the origin
    // records of the loop points p0 .. p0 + cnt - 1 of patch a
    auto stage = [&](int p0, int cnt) {
        for (int i = tid; i < cnt; i += blockDim.x) {
            const int p = a * PP + p0 + i;
            const float4 k4 = A.kp[(long)jidx * M + p];
            const float cpx = A.fine.cx[p], spx = A.fine.sx[p], cpy = A.fine.cy[p], spy = A.fine.sy[p];
            const float xp = lza * A.fine.xi[p];
            float fp, fcp;
            sfermi(xp, A.invT, fp, fcp);
            const float wp = A.fine.w[p];
            const int kx = angle_fx((double)k4.x + (double)k4.y), ky = angle_fx((double)k4.z + (double)k4.w);
            rA[i] = make_float4(__int_as_float(kx), __int_as_float(ky), kcs.x * cpx - kcs.y * spx,
                                kcs.z * cpy - kcs.w * spy);
            rB[i] = make_float4(kcs.y * cpx + kcs.x * spx, kcs.w * cpy + kcs.z * spy, wp * fp, wp * fcp);
            rC[i] = xj + xp;
            if (i == cnt - 1 && (cnt & 1)) {   // pad: the same point with weight 0
                rA[i + 1] = rA[i];
                rB[i + 1] = make_float4(rB[i].x, rB[i].y, 0.f, 0.f);
                rC[i + 1] = rC[i];
            }
        }
    };
    const bool one_pass = P <= pch;
    if (one_pass) stage(0, P);
    __syncthreads();   // tables (and the records of a single pass) written

    static_assert(SF_QPT == 2, "the loop points of a thread are the two lanes of the packed arithmetic");
    const float2 one2 = make_float2(1.f, 1.f), ntln2 = make_float2(-A.tln2, -A.tln2);
    const float2 nkchord = make_float2(-A.kchord, -A.kchord), eta2x4 = make_float2(A.eta2x4, A.eta2x4);
    double vsum = 0.0;
    // A.qb blocks of 256 SF_QPT loop points q per CTA reuse the staged tables
    for (int qb = 0; qb < A.qb; ++qb) {
        const int blk = blockIdx.x * A.qb + qb;
        if (blk * (256 * SF_QPT) >= M) break;   // uniform over the CTA
        if (UNIB && blk * (256 * SF_QPT) / PP != b_slots) {
            b_slots = blk * (256 * SF_QPT) / PP;
            __syncthreads();   // every warp is done with the previous weights
            fill_slots(b_slots);
            __syncthreads();
        }
        // the SF_QPT loop points q of this thread (an index past M gets weight 0)
        // (cos, sin) of (q_x, q_y) as pairs: cos r_x and cos r_y in one packed FMA
        float2 cq[SF_QPT], sq[SF_QPT];
        float fqp[SF_QPT], fcqp[SF_QPT], v2[SF_QPT], vab[SF_QPT], mxq[SF_QPT];
        float2 acc = make_float2(0.f, 0.f);     // the SF_QPT = 2 loop points as the two lanes
        int qi[SF_QPT], qx[SF_QPT], qy[SF_QPT];
        const uint8_t *rq[SF_QPT];   // RT: the patch-of-r rows of this thread's loop points q
#pragma unroll
        for (int k = 0; k < SF_QPT; ++k) {
            const int iq = blk * (256 * SF_QPT) + k * 256 + tid;   // angular-minor index
            const bool valid = iq < M;
            const int ii = valid ? iq : M - 1;
            rq[k] = RT ? A.rtab + (((long)jidx * N + a) * (long)(PP / 8) * M + ii) * 8 : nullptr;
            const int b = ii / PP, rem = ii - b * PP;
            const int qq = b * PP + (rem % A.pb.n_theta) * A.pb.n_r + rem / A.pb.n_theta;
            qi[k] = qq;
            const float Zb = A.Z ? (float)A.Z[b] : 1.f;
            qx[k] = angle_fx(A.kx64[qq]);
            qy[k] = angle_fx(A.ky64[qq]);
            cq[k] = make_float2(A.fine.cx[qq], A.fine.cy[qq]);
            sq[k] = make_float2(A.fine.sx[qq], A.fine.sy[qq]);
            const float xq = (qp ? Zb : 1.f) * A.fine.xi[qq];
            float fq, fcq;
            sfermi(xq, A.invT, fq, fcq);
            const float pref = valid ? Za * Zb * A.fine.w[qq] : 0.f;
            fqp[k] = fq * pref;
            fcqp[k] = fcq * pref;
            vab[k] = (float)Vja[b];
            v2[k] = 2.f * vab[k] * vab[k];
            mxq[k] = -xq;
        }

        for (int p0 = 0; p0 < P; p0 += pch) {
            const int cnt = P - p0 < pch ? P - p0 : pch;
            if (!one_pass) {
                __syncthreads();   // previous pass done with the records
                stage(p0, cnt);
                __syncthreads();
            }
            // the arithmetic of two records (ra, rb, upp) and their 2 x SF_QPT
            // patches c: the two loop points q of a record as the lanes of
            // packed FP32x2 operations where the operands pair up
            auto pair_math = [&](const float4 (&ra)[2], const float4 (&rb)[2], const float (&upp)[2],
                                 const int (&c)[2][SF_QPT]) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float2 xr, amp, sum;
                    float2 fr, aq, dq;
#pragma unroll
                    for (int k = 0; k < SF_QPT; ++k) {
                        const float4 z = cz[c[r][k]];
                        // (cos r_x, cos r_y) by angle addition
                        const float2 cr2 = __ffma2_rn(make_float2(ra[r].z, ra[r].w), cq[k],
                                                      __fmul2_rn(make_float2(rb[r].x, rb[r].y), sq[k]));
                        float x = fmaf(cr2.x + cr2.y, z.z, z.w);       // Z-scaled line energy of r / (T ln 2)
                        if (!TP0) x = fmaf(cr2.x * cr2.y, cd[c[r][k]], x);
                        const float ex = ex2_approx(x);
                        const float a = rb[r].z * fcqp[k];
                        const float d = fmaf(rb[r].w, fqp[k], -a);
                        const float w = UNIB ? z.x : fmaf(-vab[k], z.y, z.x * v2[k]);
                        const float sm = upp[r] + mxq[k];
                        if (k == 0) { xr.x = x; fr.x = ex; aq.x = a; dq.x = d; amp.x = w; sum.x = sm; }
                        else        { xr.y = x; fr.y = ex; aq.y = a; dq.y = d; amp.y = w; sum.y = sm; }
                    }
                    const float2 g = __fadd2_rn(fr, one2);
                    fr = make_float2(rcp_approx(g.x), rcp_approx(g.y));
                    const float2 F = __ffma2_rn(fr, dq, aq);           // A + f_r (B - A)
                    amp = __fmul2_rn(amp, F);
                    // d0 = xi_j - E, E = x_q + x_r - x_p
                    const float2 d0 = __ffma2_rn(xr, ntln2, sum);
                    const float2 u = __ffma2_rn(d0, d0, nkchord);
                    const float2 den = __ffma2_rn(__fmul2_rn(eta2x4, d0), d0, __fmul2_rn(u, u));
                    acc = __ffma2_rn(__fmul2_rn(amp, u), make_float2(rcp_approx(den.x), rcp_approx(den.y)), acc);
                }
            };
            if (RT) {
                // eight records per trip: their patches for each loop point q
                // are one 8-byte word of the table, loaded one trip ahead
                // (word of records i .. i+7 at rq + i M)
                uint2 wn[SF_QPT];
#pragma unroll
                for (int k = 0; k < SF_QPT; ++k) wn[k] = __ldcs(reinterpret_cast<const uint2 *>(rq[k] + (long)p0 * M));
                for (int i = 0; i < cnt; i += 8) {
                    uint2 w[SF_QPT];
#pragma unroll
                    for (int k = 0; k < SF_QPT; ++k) {
                        w[k] = wn[k];
                        if (i + 8 < cnt) wn[k] = __ldcs(reinterpret_cast<const uint2 *>(rq[k] + (long)(p0 + i + 8) * M));
                    }
#pragma unroll 2
                    for (int s2 = 0; s2 < 4; ++s2) {
                        float4 ra[2], rb[2];
                        float upp[2];
                        int c[2][SF_QPT];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            ra[r] = rA[i + 2 * s2 + r];
                            rb[r] = rB[i + 2 * s2 + r];
                            upp[r] = rC[i + 2 * s2 + r];
#pragma unroll
                            for (int k = 0; k < SF_QPT; ++k) {
                                const int byte = 2 * s2 + r;
                                const unsigned word = byte < 4 ? w[k].x : w[k].y;
                                c[r][k] = (int)((word >> (8 * (byte & 3))) & 255u);
                            }
                        }
                        pair_math(ra, rb, upp, c);
                    }
                }
            } else {
            // two records per iteration: the patches of all 2 x SF_QPT pairs
            // first, one rarely taken branch for the guarded ones, then the
            // arithmetic of all of them (one large block for the scheduler);
            // an odd count reads the zero-weight pad record after the last one;
            // the loop is unrolled four times (eight records per trip, 122
            // registers: the loop overhead amortised, more independent work)
#pragma unroll 4
            for (int i = 0; i < cnt; i += 2) {
                float4 ra[2], rb[2];
                float upp[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    ra[r] = rA[i + r];
                    rb[r] = rB[i + r];
                    upp[r] = rC[i + r];
                }
                int c[2][SF_QPT];
                bool slow_any = false;
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int k = 0; k < SF_QPT; ++k) {
                        float x, y;
                        bool slow;
                        c[r][k] = fx_patch(__float_as_int(ra[r].x), __float_as_int(ra[r].y), qx[k], qy[k], tabc, ray,
                                           x, y, slow);
                        slow_any |= slow;
                    }
                if (slow_any) {
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int k = 0; k < SF_QPT; ++k) {
                            float x, y;
                            bool slow;
                            fx_patch(__float_as_int(ra[r].x), __float_as_int(ra[r].y), qx[k], qy[k], tabc, ray, x, y,
                                     slow);
                            // the pad record (weight 0) keeps its table patch
                            if (slow && i + r < cnt) {
                                const bool edge = fmaxf(fabsf(x), fabsf(y)) > kFxEdge;
                                c[r][k] = sf_slow_patch(A, jidx, j, a * PP + p0 + i + r, qi[k], x * kRadPerFx,
                                                        y * kRadPerFx, edge, A.bnd);
                            }
                        }
                }
                pair_math(ra, rb, upp, c);
            }
            }
        }
        vsum -= (double)acc.x + (double)acc.y;   // the chord term is -u / den
    }
    vsum *= fac;
    __shared__ double red[32];
    double v = vsum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) atomicAdd(&A.sig[jidx], v);
    }
}

// Frequency-grid variant of sigma_fast_kernel:
// instead of the chord slope, bin W F by pole energy E = x_q + x_r - x_p
// (moments 0..4 of E - E_bin) in a shared-memory histogram per CTA, flushed to
// the FP64 histogram once at the end (then sigma_grid_kernel).  A separate
// kernel, so that the chord kernel of the flow keeps its own code generation.
template <bool TP0, bool UNIB>
__global__ void __launch_bounds__(256, 1) sigma_grid_fast_kernel(SigmaFastArgs A)
{
    const int N = A.pb.N, M = A.pb.M;
    const int a = blockIdx.y, jidx = blockIdx.z;
    const int j = A.jlist ? A.jlist[jidx] : jidx;
    const int tid = threadIdx.x;
    const bool qp = A.pb.propagator == QPFRG_PROP_QP;
    // A target on a mirror line of the zone (theta_j = 0 or pi/4) has a sum
    // symmetric under that mirror: keep the patches a on one side of it with
    // weight 2 and half of each patch the mirror maps onto itself.
    // The mirror line through k_j (j a multiple of N/8) reflects patch a to 2j - a.
    int fac = 1, P = A.pb.P;
    if (A.mirror && (8 * j) % N == 0 && !(A.mirror == 2 && (4 * j) % N == 0)) {
        const int ma = ((2 * j - a) % N + N) % N;
        if (ma == a) {
            fac = 2;
            P = A.pb.P / 2;     // angular index t < n_theta / 2
        } else {
            const int rel = ((a - j) % N + N) % N;
            fac = (rel > 0 && 2 * rel < N) ? 2 : 0;
        }
    }
    if (fac == 0) return;       // the mirror patch carries this one (uniform over the CTA)
    const int PP = A.pb.P;      // points per patch (record and loop-point indexing)
    const int cap = SF_PCH / 2;     // room for the histogram
    const int pch = P < cap ? P : cap;
    const SfSmem L = sf_smem_layout(pch, A.nbins);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *rA = reinterpret_cast<float4 *>(smem_raw + L.rA);   // (k+p)_x, (k+p)_y, cos, sin of (k+p)_x
    float4 *rB = reinterpret_cast<float4 *>(smem_raw + L.rB);   // cos, sin of (k+p)_y, w_p f_p, w_p (1 - f_p)
    float4 *cz = reinterpret_cast<float4 *>(smem_raw + L.cz);
    float2 *ray = reinterpret_cast<float2 *>(smem_raw + L.ray);
    float *cd = reinterpret_cast<float *>(smem_raw + L.cd);     // -4 t' l_c
    float *rC = reinterpret_cast<float *>(smem_raw + L.rC);     // x_j + x_p + 2T
    unsigned char *tab = smem_raw + L.tab;
    float *hs = reinterpret_cast<float *>(smem_raw + L.hist);   // [moment][bin] (grid mode)
    for (int i = tid; i < 5 * A.nbins; i += blockDim.x) hs[i] = 0.f;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(A.ptab);
        uint4 *dst = reinterpret_cast<uint4 *>(tab);
        const int n16 = (kProjW * kProjStride + 15) / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    const double *Vja = A.V + ((long)j * N + a) * N;
    // per-patch slots; with UNIB the weight column is filled per q block (b)
    auto fill_slots = [&](int b) {
        const float vb = UNIB ? (float)Vja[b] : 0.f;
        for (int i = tid; i < SF_SLOTS; i += blockDim.x) {
            if (i <= N) {
                const int cc = i == N ? 0 : i;
                const float Zc = A.Z ? (float)A.Z[cc] : 1.f;
                const float lz = qp ? Zc : 1.f;
                const float vc = (float)Vja[cc];
                cz[i] = UNIB ? make_float4(Zc * (2.f * vb * vb - vb * vc), 0.f, -2.f * A.t * lz, -A.mu * lz)
                             : make_float4(Zc, Zc * vc, -2.f * A.t * lz, -A.mu * lz);
                cd[i] = -4.f * A.tp * lz;
                const float4 bd = A.bnd[cc];
                ray[i] = make_float2(bd.x, bd.z);
            } else {
                cz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                cd[i] = 0.f;
                ray[i] = make_float2(0.f, 0.f);
            }
        }
    };
    int b_slots = UNIB ? (blockIdx.x * A.qb * 256 * SF_QPT) / PP : 0;
    fill_slots(b_slots);
    const float Za = A.Z ? (float)A.Z[a] : 1.f;
    const float lza = qp ? Za : 1.f;
    const float4 kcs = A.kcs[jidx];

    const unsigned char *tabc = tab + (kProjW / 2) * (kProjStride + 1);   // the cell of the origin
    // records of the loop points p0 .. p0 + cnt - 1 of patch a
    auto stage = [&](int p0, int cnt) {
        for (int i = tid; i < cnt; i += blockDim.x) {
            const int p = a * PP + p0 + i;
            const float4 k4 = A.kp[(long)jidx * M + p];
            const float cpx = A.fine.cx[p], spx = A.fine.sx[p], cpy = A.fine.cy[p], spy = A.fine.sy[p];
            const float xp = lza * A.fine.xi[p];
            float fp, fcp;
            sfermi(xp, A.invT, fp, fcp);
            const float wp = A.fine.w[p];
            const int kx = angle_fx((double)k4.x + (double)k4.y), ky = angle_fx((double)k4.z + (double)k4.w);
            rA[i] = make_float4(__int_as_float(kx), __int_as_float(ky), kcs.x * cpx - kcs.y * spx,
                                kcs.y * cpx + kcs.x * spx);
            rB[i] = make_float4(kcs.z * cpy - kcs.w * spy, kcs.w * cpy + kcs.z * spy, wp * fp, wp * fcp);
            rC[i] = xp;
        }
    };
    const bool one_pass = P <= pch;
    if (one_pass) stage(0, P);
    __syncthreads();   // tables (and the records of a single pass) written

    // A.qb blocks of 256 SF_QPT loop points q per CTA reuse the staged tables
    for (int qb = 0; qb < A.qb; ++qb) {
        const int blk = blockIdx.x * A.qb + qb;
        if (blk * (256 * SF_QPT) >= M) break;   // uniform over the CTA
        if (UNIB && blk * (256 * SF_QPT) / PP != b_slots) {
            b_slots = blk * (256 * SF_QPT) / PP;
            __syncthreads();   // every warp is done with the previous weights
            fill_slots(b_slots);
            __syncthreads();
        }
        // the SF_QPT loop points q of this thread (an index past M gets weight 0)
        float cqx[SF_QPT], sqx[SF_QPT], cqy[SF_QPT], sqy[SF_QPT];
        float fqp[SF_QPT], fcqp[SF_QPT], v2[SF_QPT], vab[SF_QPT], mxq[SF_QPT];
        int qi[SF_QPT], qx[SF_QPT], qy[SF_QPT];
#pragma unroll
        for (int k = 0; k < SF_QPT; ++k) {
            const int iq = blk * (256 * SF_QPT) + k * 256 + tid;   // angular-minor index
            const bool valid = iq < M;
            const int ii = valid ? iq : M - 1;
            const int b = ii / PP, rem = ii - b * PP;
            const int qq = b * PP + (rem % A.pb.n_theta) * A.pb.n_r + rem / A.pb.n_theta;
            qi[k] = qq;
            const float Zb = A.Z ? (float)A.Z[b] : 1.f;
            qx[k] = angle_fx(A.kx64[qq]);
            qy[k] = angle_fx(A.ky64[qq]);
            cqx[k] = A.fine.cx[qq];
            sqx[k] = A.fine.sx[qq];
            cqy[k] = A.fine.cy[qq];
            sqy[k] = A.fine.sy[qq];
            const float xq = (qp ? Zb : 1.f) * A.fine.xi[qq];
            float fq, fcq;
            sfermi(xq, A.invT, fq, fcq);
            const float pref = valid ? Za * Zb * A.fine.w[qq] : 0.f;
            fqp[k] = fq * pref;
            fcqp[k] = fcq * pref;
            vab[k] = (float)Vja[b];
            v2[k] = 2.f * vab[k] * vab[k];
            mxq[k] = -xq;
        }

        for (int p0 = 0; p0 < P; p0 += pch) {
            const int cnt = P - p0 < pch ? P - p0 : pch;
            if (!one_pass) {
                __syncthreads();   // previous pass done with the records
                stage(p0, cnt);
                __syncthreads();
            }
#pragma unroll 2
            for (int i = 0; i < cnt; ++i) {
                const float4 ra = rA[i], rb = rB[i];
                const float upp = rC[i];   // x_p
                int c[SF_QPT];
                float x[SF_QPT], y[SF_QPT];
                bool slow_any = false;
                unsigned slow_mask = 0;
#pragma unroll
                for (int k = 0; k < SF_QPT; ++k) {
                    bool slow;
                    c[k] = fx_patch(__float_as_int(ra.x), __float_as_int(ra.y), qx[k], qy[k], tabc, ray, x[k], y[k],
                                    slow);
                    slow_mask |= slow ? 1u << k : 0u;
                    slow_any = slow_any || slow;
                }
                if (slow_any) {
#pragma unroll
                    for (int k = 0; k < SF_QPT; ++k)
                        if (slow_mask & (1u << k)) {
                            const bool edge = fmaxf(fabsf(x[k]), fabsf(y[k])) > kFxEdge;
                            c[k] = sf_slow_patch(A, jidx, j, a * PP + p0 + i, qi[k], x[k] * kRadPerFx,
                                                 y[k] * kRadPerFx, edge, A.bnd);
                        }
                }
#pragma unroll
                for (int k = 0; k < SF_QPT; ++k) {
                    const float4 z = cz[c[k]];
                    const float crx = ra.z * cqx[k] + ra.w * sqx[k];
                    const float cry = rb.x * cqy[k] + rb.y * sqy[k];
                    float xr = fmaf(crx + cry, z.z, z.w);           // Z-scaled line energy of r
                    if (!TP0) xr = fmaf(crx * cry, cd[c[k]], xr);
                    const float fr = rcp_approx(1.f + ex2_approx(xr * A.cT));
                    const float Aq = rb.z * fcqp[k], Bq = rb.w * fqp[k];
                    const float F = fmaf(fr, Bq - Aq, Aq);
                    const float amp = UNIB ? z.x * F : fmaf(-vab[k], z.y, z.x * v2[k]) * F;
                    // pole energy E = x_q + x_r - x_p (upp holds x_p here)
                    const float E = (xr - mxq[k]) - upp;
                    int bin = (int)floorf((E - A.e_min) * A.inv_h);
                    bin = bin < 0 ? 0 : (bin >= A.nbins ? A.nbins - 1 : bin);
                    const float d = E - (A.e_min + ((float)bin + 0.5f) * A.h);
                    float mm[5];
                    mm[0] = amp;
#pragma unroll
                    for (int mo = 1; mo < 5; ++mo) mm[mo] = mm[mo - 1] * d;
                    // neighbouring lanes often share a bin: sum runs of equal
                    // bins with shuffles (each lane adds the lanes up to the
                    // end of its run), then one atomic per run and moment
                    const int lane = tid & 31;
                    const int bup = __shfl_up_sync(0xffffffffu, bin, 1);
                    const bool head = lane == 0 || bup != bin;
                    const unsigned heads = __ballot_sync(0xffffffffu, head);
                    if (heads != 0xffffffffu) {
                        const unsigned above = lane == 31 ? 0u : heads >> (lane + 1);
                        const int end = above ? lane + __ffs(above) - 1 : 31;
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
                            for (int mo = 0; mo < 5; ++mo) {
                                const float o = __shfl_down_sync(0xffffffffu, mm[mo], off);
                                if (lane + off <= end) mm[mo] += o;
                            }
                        }
                    }
                    if (head) {
#pragma unroll
                        for (int mo = 0; mo < 5; ++mo) atomicAdd(&hs[mo * A.nbins + bin], mm[mo]);
                    }
                }
            }
        }
    }
    __syncthreads();
    double *H = A.hist + (long)jidx * 5 * A.nbins;
    for (int i = tid; i < 5 * A.nbins; i += blockDim.x) {
        const float v = hs[i];
        if (v != 0.f) atomicAdd(&H[i], (double)v * fac);
    }
}

// Z_j = 1/(1 - slope) with the chord slope accumulated per target.  rep[j]
// (may be NULL) is the slot of j's C4v representative among the targets.
__global__ void z_update_kernel(const double *slope, const int *rep, double *Zout, int N)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    Zout[j] = 1.0 / (1.0 - slope[rep ? rep[j] : j]);
}

// Sigma on the grid from the binned moments: sum_b sum_n H_n[b] / (z - E_b)^(n+1),
// z = w_m + i eta (Taylor expansion of 1/(z - E_b - d) in the offset d).
// rep (may be NULL): the histogram slot of patch j's C4v representative.
__global__ void sigma_grid_kernel(const double *hist, int nbins, double e_min, double h, int n_omega,
                                  double w0, double dw, double eta, double *re, double *im, int N,
                                  const int *rep)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (m >= n_omega) return;
    const double w = w0 + dw * m;
    const double *H = hist + (long)(rep ? rep[j] : j) * 5 * nbins;
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < nbins; ++b) {
        const double Eb = e_min + (b + 0.5) * h;
        // u = 1/(z - Eb) = (dx - i eta)/(dx^2 + eta^2)
        const double dx = w - Eb, den = dx * dx + eta * eta;
        const double ur = dx / den, ui = -eta / den;
        double pr = ur, pi = ui;                 // u^(n+1)
        for (int mo = 0; mo < 5; ++mo) {
            const double hv = H[(long)mo * nbins + b];
            sr += hv * pr;
            si += hv * pi;
            const double nr = pr * ur - pi * ui, ni = pr * ui + pi * ur;
            pr = nr;
            pi = ni;
        }
    }
    re[(long)j * n_omega + m] = sr;
    im[(long)j * n_omega + m] = si;
}

static qpfrg_status launch_kp_table(qpfrg_ctx *c, const int *jlist, int nj)
{
    const long total = (long)nj * c->pb.M;
    prof_begin(c);
    kp_table_kernel<<<(int)std::min<long>((total + 255) / 256, 152L * 8), 256, 0, c->stream>>>(
        c->d_kf, jlist, nj, c->f64.kx, c->f64.ky, c->pb.M, c->d_kp, c->d_kcs);
    prof_end(c, K_KP_TABLE);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "kp_table_kernel");
}

template <typename R>
static qpfrg_status launch_sigma(qpfrg_ctx *c, bool hist, SigmaArgs<R> &A, int kid)
{
    const int P = c->pb.P, N = c->pb.N;
    const size_t smem = (size_t)(REC * P + 2 * N) * sizeof(R) + 16 + (size_t)N * sizeof(float4) + (size_t)N * sizeof(R);
    if (sizeof(R) == 4) {
        const qpfrg_status s = launch_kp_table(c, A.jlist, A.nj);
        if (s != QPFRG_OK) return s;
    }
    auto kern = hist ? sigma_kernel<R, true> : sigma_kernel<R, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "sigma smem attribute");
    dim3 grid(div_up(c->pb.M, 256), N, A.nj);
    prof_begin(c);
    kern<<<grid, 256, smem, c->stream>>>(A);
    prof_end(c, kid);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "sigma_kernel");
}

// Shared memory of the fast kernel (grid mode with nbins > 0)
static size_t sigma_fast_smem(const qpfrg_ctx *c, int nbins)
{
    const int cap = nbins > 0 ? SF_PCH / 2 : SF_PCH;
    const int pch = c->pb.P < cap ? c->pb.P : cap;
    return sf_smem_layout(pch, nbins).total;
}

// nbins == 0: chord slopes into d_sig (the flow's Z); nbins > 0: the binned
// pole density into hist (frequency grid)
static qpfrg_status launch_sigma_fast(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z,
                                      const int *jlist, int nj, double *hist = nullptr, double e_min = 0.0,
                                      double h = 1.0, int nbins = 0)
{
    qpfrg_status s = launch_kp_table(c, jlist, nj);
    if (s != QPFRG_OK) return s;
    SigmaFastArgs A;
    A.pb = c->pb;
    A.fine = c->f32;
    A.V = d_V;
    A.Z = d_Z;
    A.kx64 = c->f64.kx;
    A.ky64 = c->f64.ky;
    A.kf = c->d_kf;
    A.xij_f = c->d_xij_f;
    A.qxl = c->d_qxl;
    A.qyl = c->d_qyl;
    A.kp = c->d_kp;
    A.kcs = c->d_kcs;
    A.bnd = c->d_bnd;
    A.ptab = c->d_ptab;
    A.jlist = jlist;
    A.sig = c->d_sig;
    A.t = (float)c->pb.t;
    A.tp = (float)c->pb.tp;
    A.mu = (float)c->pb.mu;
    A.eta2 = (float)(c->pb.eta * c->pb.eta);
    A.invT = (float)(1.0 / T);
    A.cT = (float)(1.4426950408889634 / T);
    A.twoT = (float)(2.0 * T);
    A.fourT = (float)(4.0 * T);
    A.tln2 = (float)(0.6931471805599453 * T);
    A.kchord = (float)(4.0 * T * T + c->pb.eta * c->pb.eta);
    A.eta2x4 = (float)(4.0 * c->pb.eta * c->pb.eta);
    A.inv_dth = (float)(c->pb.N / kTwoPi);
    A.dth = (float)(kTwoPi / c->pb.N);
    A.hist = hist;
    A.e_min = (float)e_min;
    A.h = (float)h;
    A.inv_h = (float)(1.0 / h);
    A.nbins = nbins;
    const bool grid_mode = nbins > 0;
    const size_t smem = sigma_fast_smem(c, nbins);
    // The zone-edge targets' sums are mirror symmetric only up to the pairs
    // whose momentum r lands on |r_x| or |r_y| = pi (their wedge is decided by
    // rounding): halving them is kept for the chord slope (a relative error
    // below 1e-4, shrinking with N) and left out on the frequency grid.
    A.mirror = (jlist != nullptr && c->pb.n_theta % 2 == 0) ? (grid_mode ? 2 : 1) : 0;
    const bool unib = c->pb.P % (256 * SF_QPT) == 0;
    // The flow's Z on the C4v-irreducible targets reads the patches of r from
    // a table built on first use (one byte per target, p and q: N_irr M^2
    // bytes, 126 GB at np96_n32), when it fits in 60 % of the free device
    // memory and options.sigma_table >= 0; otherwise it decides them per pair.
    // (record passes of a multiple of 8 records: P a multiple of 16, mirror halves included)
    const bool rt_list = !grid_mode && jlist != nullptr && jlist == c->d_jirr && nj == c->n_irr &&
                         c->pb.P % 16 == 0 && c->pb.P <= SF_PCH;
    if (rt_list && !c->rtab_tried && c->opt.sigma_table >= 0) {
        c->rtab_tried = true;
        const size_t bytes = (size_t)nj * c->pb.N * (size_t)c->pb.P * (size_t)c->pb.M;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes <= fr / 10 * 6) {
            if (cudaMalloc((void **)&c->d_rtab, bytes) == cudaSuccess) {
                const size_t smem_b = kRtabSmem + (size_t)c->pb.P * sizeof(int2);
                cudaError_t e = cudaFuncSetAttribute(rtab_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem_b);
                if (e != cudaSuccess) return cuda_fail(c, e, "rtab smem attribute");
                prof_begin(c);
                rtab_build_kernel<<<dim3(div_up(c->pb.M, 256), c->pb.N, nj), 256, smem_b, c->stream>>>(A,
                                                                                                      c->d_rtab);
                prof_end(c, K_RTAB);
                if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "rtab_build_kernel");
            } else {
                c->d_rtab = nullptr;
                cudaGetLastError();   // not enough memory: decide per pair
            }
        }
    }
    const bool rt = rt_list && c->d_rtab != nullptr;
    A.rtab = rt ? c->d_rtab : nullptr;
    using Kern = void (*)(SigmaFastArgs);
    Kern kern;
    if (grid_mode)
        kern = c->pb.tp == 0.0
                   ? (unib ? sigma_grid_fast_kernel<true, true> : sigma_grid_fast_kernel<true, false>)
                   : (unib ? sigma_grid_fast_kernel<false, true> : sigma_grid_fast_kernel<false, false>);
    else if (rt)
        kern = c->pb.tp == 0.0 ? (unib ? sigma_fast_kernel<true, true, true> : sigma_fast_kernel<true, false, true>)
                               : (unib ? sigma_fast_kernel<false, true, true> : sigma_fast_kernel<false, false, true>);
    else
        kern = c->pb.tp == 0.0 ? (unib ? sigma_fast_kernel<true, true, false> : sigma_fast_kernel<true, false, false>)
                               : (unib ? sigma_fast_kernel<false, true, false> : sigma_fast_kernel<false, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "sigma_fast smem attribute");
    // grid mode: one CTA per (patch a, target) takes every q block, so that the
    // per-CTA histogram reaches the FP64 one with few atomics per bin
    const int nqb = div_up(c->pb.M, 256 * SF_QPT);
    A.qb = grid_mode ? nqb : (c->tune.sigma_qblocks > 0 ? c->tune.sigma_qblocks : SF_QB);
    dim3 grid(div_up(nqb, A.qb), c->pb.N, nj);
    prof_begin(c);
    kern<<<grid, 256, smem, c->stream>>>(A);
    prof_end(c, grid_mode ? K_SIGMA_HIST : K_SIGMA_Z);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "sigma_fast_kernel");
}

template <typename R>
static void fill_args(qpfrg_ctx *c, SigmaArgs<R> &A, const FineTable<R> &fine, double T, const double *d_V,
                      const double *d_Z)
{
    A.pb = c->pb;
    A.fine = fine;
    A.kf = c->d_kf;
    A.V = d_V;
    A.Z = d_Z;
    A.K = nullptr;
    A.sig = c->d_sig;
    A.T = T;
    A.nj = c->pb.N;
    A.jlist = nullptr;
    A.kx64 = c->f64.kx;
    A.ky64 = c->f64.ky;
    A.xij = c->d_xij;
    A.t_r = (R)c->pb.t;
    A.tp_r = (R)c->pb.tp;
    A.mu_r = (R)c->pb.mu;
    A.eta_r = (R)c->pb.eta;
    A.invT_r = (R)(1.0 / T);
    A.twoT_r = (R)(2.0 * T);
    A.xij_r = sizeof(R) == 4 ? reinterpret_cast<const R *>(c->d_xij_f) : reinterpret_cast<const R *>(c->d_xij);
    A.bnd = c->d_bnd;
    A.kp = c->d_kp;
    A.kcs = c->d_kcs;
    A.qxl = c->d_qxl;
    A.qyl = c->d_qyl;
    A.hist = c->d_hist;
    A.e_min = 0.0;
    A.inv_h = 1.0;
    A.nbins = 0;
}

qpfrg_status launch_sigma_z(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z, double *d_Zout,
                            bool use_symmetry)
{
    const int N = c->pb.N;
    // The zone edge breaks the C4v covariance of the angular projection at
    // the rounding level (mirror pairs land on |k_x| = pi exactly), which
    // moves Z on symmetric patches by ~1e-6: reduce in mixed precision only.
    const bool sym = use_symmetry && c->d_jirr != nullptr && c->opt.precision != QPFRG_FP64;
    const int nj = sym ? c->n_irr : N;
    cudaError_t e = cudaMemsetAsync(c->d_sig, 0, 2 * (size_t)N * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset sigma");
    qpfrg_status s;
    if (c->opt.precision == QPFRG_FP64) {
        SigmaArgs<double> A;
        fill_args(c, A, c->f64, T, d_V, d_Z);
        A.nj = nj;
        A.jlist = sym ? c->d_jirr : nullptr;
        s = launch_sigma(c, false, A, K_SIGMA_Z);
    } else if (c->d_ptab) {
        s = launch_sigma_fast(c, T, d_V, d_Z, sym ? c->d_jirr : nullptr, nj);
    } else {
        SigmaArgs<float> A;
        fill_args(c, A, c->f32, T, d_V, d_Z);
        A.nj = nj;
        A.jlist = sym ? c->d_jirr : nullptr;
        s = launch_sigma(c, false, A, K_SIGMA_Z);
    }
    if (s != QPFRG_OK) return s;
    prof_begin(c);
    z_update_kernel<<<div_up(N, 128), 128, 0, c->stream>>>(c->d_sig, sym ? c->d_rep : nullptr, d_Zout, N);
    prof_end(c, K_Z_UPDATE);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "z_update_kernel");
}

// Whether (V, Z) keep the C4v symmetry of the angular patches: flag set when
// an image V(g k1, g k2, g k3) or Z(g k) differs from the original by more
// than tol (1 + |v|), g running over the rotations w -> w + m N_a/4 and the
// reflections w -> -w + m N_a/4 of the wedge w of patch j = w ns + s.
__global__ void c4v_check_kernel(const double *V, const double *Z, int N, int ns, double tol,
                                 unsigned long long *flag)
{
    const long NN = (long)N * N, n3 = NN * N;
    const int Na = N / ns, q = Na / 4;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n3; idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / NN), j = (int)((idx / N) % N), l = (int)(idx % N);
        const double v = V[idx];
        bool bad = false;
        for (int g = 1; g < 8; ++g) {
            const int m = g & 3, sg = g < 4 ? 1 : -1;
            auto img = [&](int x) { return ((sg * (x / ns) + m * q) % Na + Na) % Na * ns + x % ns; };
            const double w = V[((long)img(i) * N + img(j)) * N + img(l)];
            bad = bad || fabs(w - v) > tol * (1.0 + fabs(v));
            if (idx < N && Z) bad = bad || fabs(Z[img((int)idx)] - Z[idx]) > tol * (1.0 + fabs(Z[idx]));
        }
        if (bad) atomicOr(flag, 1ull);
    }
}

static qpfrg_status c4v_check(qpfrg_ctx *c, const double *d_V, const double *d_Z, bool &sym)
{
    sym = false;
    const int N = c->pb.N, ns = c->pb.n_shell;
    if ((N / ns) % 4 != 0) return QPFRG_OK;
    cudaError_t e = cudaMemsetAsync(c->d_red, 0, sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset symmetry flag");
    const long n3 = (long)N * N * N;
    c4v_check_kernel<<<(int)std::min<long>((n3 + 255) / 256, 152L * 8), 256, 0, c->stream>>>(d_V, d_Z, N, ns, 1e-5,
                                                                                            c->d_red);
    unsigned long long flag = 1;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&flag, c->d_red, sizeof(flag), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "symmetry check");
    sym = flag == 0;
    return QPFRG_OK;
}

// Bin count of the frequency-grid histogram: with h = eta/4 the offset of a
// pole from its bin centre is at most |z - E_b|/8, so the moment expansion
// truncated after moment 4 is accurate to 8^-5 = 3e-5 relative per pole.
static int grid_bins(const qpfrg_ctx *c, double e_min, double e_max)
{
    const double h_target = 0.25 * c->opt.eta;
    int nb = (int)std::ceil((e_max - e_min) / h_target);
    if (nb < 64) nb = 64;
    if (nb > 1 << 16) nb = 1 << 16;
    return nb;
}

// Chord slopes of the two-loop term with the interaction flow's line weights
// (Katanin factors d_K, ones without the correction) for every patch, into
// c->d_sig: the generic kernel, exact projection.
qpfrg_status launch_sigma_lines(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z, const double *d_K)
{
    cudaError_t e = cudaMemsetAsync(c->d_sig, 0, 2 * (size_t)c->pb.N * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset sigma");
    if (c->opt.precision == QPFRG_FP64) {
        SigmaArgs<double> A;
        fill_args(c, A, c->f64, T, d_V, d_Z);
        A.K = d_K;
        return launch_sigma(c, false, A, K_SIGMA_Z);
    }
    SigmaArgs<float> A;
    fill_args(c, A, c->f32, T, d_V, d_Z);
    A.K = d_K;
    return launch_sigma(c, false, A, K_SIGMA_Z);
}

qpfrg_status launch_sigma_grid(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z, double *d_re,
                               double *d_im, const double *d_K)
{
    const int N = c->pb.N, n_omega = c->opt.n_omega;
    // pole energies E = x_q + x_r - x_p lie in [2 min x - max x, 2 max x - min x]
    double xmin = 1e300, xmax = -1e300;
    for (int p = 0; p < c->pb.M; ++p) {
        const double kx = c->fk[2 * p], ky = c->fk[2 * p + 1];
        const double x = -2.0 * c->pb.t * (std::cos(kx) + std::cos(ky)) -
                         4.0 * c->pb.tp * std::cos(kx) * std::cos(ky) - c->pb.mu;
        xmin = x < xmin ? x : xmin;
        xmax = x > xmax ? x : xmax;
    }
    // r = k + p - q is not a fine point: bound its dispersion by the band
    const double band_lo = -4.0 * std::fabs(c->pb.t) - 4.0 * std::fabs(c->pb.tp) - c->pb.mu;
    const double band_hi = 4.0 * std::fabs(c->pb.t) + 4.0 * std::fabs(c->pb.tp) - c->pb.mu;
    xmin = std::fmin(xmin, band_lo);
    xmax = std::fmax(xmax, band_hi);
    if (c->pb.propagator == QPFRG_PROP_QP) {   // Z in (0, z_max] rescales the poles
        xmin *= c->opt.z_max;
        xmax *= c->opt.z_max;
    }
    const double e_min = 2.0 * xmin - xmax - 1e-9, e_max = 2.0 * xmax - xmin + 1e-9;
    const int nbins = grid_bins(c, e_min, e_max);
    const size_t need = (size_t)N * 5 * nbins;
    if (need > c->hist_elems) {
        if (c->d_hist) cudaFree(c->d_hist);
        c->d_hist = nullptr;
        cudaError_t e = cudaMalloc((void **)&c->d_hist, need * sizeof(double));
        if (e != cudaSuccess) {
            c->hist_elems = 0;
            return cuda_fail(c, e, "cudaMalloc(sigma histogram)");
        }
        c->hist_elems = need;
    }
    cudaError_t e = cudaMemsetAsync(c->d_hist, 0, need * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset histogram");
    const double h = (e_max - e_min) / nbins;
    qpfrg_status s;
    bool sym = false;
    if (!d_K && c->opt.precision != QPFRG_FP64 && c->d_ptab && sigma_fast_smem(c, nbins) <= 226 * 1024) {
        // FP32 wedge grid: table projection, histogram in shared memory; a
        // C4v-symmetric (V, Z) needs only the irreducible targets
        if (c->d_jgrid) {
            if ((s = c4v_check(c, d_V, d_Z, sym)) != QPFRG_OK) return s;
        }
        s = launch_sigma_fast(c, T, d_V, d_Z, sym ? c->d_jgrid : nullptr, sym ? c->n_grid : N, c->d_hist, e_min,
                              h, nbins);
    } else if (c->opt.precision == QPFRG_FP64) {
        SigmaArgs<double> A;
        fill_args(c, A, c->f64, T, d_V, d_Z);
        A.K = d_K;
        A.e_min = e_min;
        A.inv_h = 1.0 / h;
        A.nbins = nbins;
        s = launch_sigma(c, true, A, K_SIGMA_HIST);
    } else {
        SigmaArgs<float> A;
        fill_args(c, A, c->f32, T, d_V, d_Z);
        A.K = d_K;
        A.e_min = e_min;
        A.inv_h = 1.0 / h;
        A.nbins = nbins;
        s = launch_sigma(c, true, A, K_SIGMA_HIST);
    }
    if (s != QPFRG_OK) return s;
    const double w0 = c->opt.omega_min;
    const double dw = n_omega > 1 ? (c->opt.omega_max - c->opt.omega_min) / (n_omega - 1) : 0.0;
    dim3 grid(div_up(n_omega, 128), N);
    prof_begin(c);
    sigma_grid_kernel<<<grid, 128, 0, c->stream>>>(c->d_hist, nbins, e_min, h, n_omega, w0, dw, c->pb.eta,
                                                   d_re, d_im, N, sym ? c->d_repgrid : nullptr);
    prof_end(c, K_SIGMA_GRID);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "sigma_grid_kernel");
}

}  // namespace qpfrg

namespace qpfrg {

// Spectral function of patch j on the frequency grid, A = -(1/pi) Im G with
// G = 1/(w - xi_j - Sigma), and its Fermi-liquid (Gaussian) approximation: a
// Gaussian of weight Z_j centred on xi_j, equal to A there (linear
// interpolation on the grid): A_FL = A0 exp(-pi A0^2 (w - xi_j)^2 / Z_j^2).
// One CTA per patch; A at the grid points, then A0 and A_FL.
__global__ void spectral_kernel(const double *re, const double *im, const double *Z, const double *xij, int n_omega,
                                double w0, double dw, double *A, double *Afl)
{
    const int j = blockIdx.x;
    const double x0 = xij[j];
    const double *sr = re + (long)j * n_omega, *si = im + (long)j * n_omega;
    double *a = A + (long)j * n_omega;
    for (int m = threadIdx.x; m < n_omega; m += blockDim.x) {
        const double x = w0 + dw * m - x0 - sr[m], y = si[m];
        const double d = x * x + y * y;
        a[m] = d > 0.0 ? -y / (kPi * d) : 0.0;    // Sigma = 0 exactly at w = xi: no grid value
    }
    __syncthreads();
    __shared__ double A0;
    if (threadIdx.x == 0) {
        double v = 0.0;
        if (n_omega > 1 && dw > 0.0) {
            const double t = (x0 - w0) / dw;
            long m0 = (long)floor(t);
            if (m0 == n_omega - 1 && t == (double)m0) m0 -= 1;   // xi on the last grid point
            if (m0 >= 0 && m0 + 1 < n_omega) {
                const double u = t - (double)m0;
                v = (1.0 - u) * a[m0] + u * a[m0 + 1];
            }
        }
        A0 = v;
    }
    __syncthreads();
    if (!Afl) return;
    const double zj = Z ? Z[j] : 1.0;
    const double k = kPi * A0 * A0 / (zj * zj);
    for (int m = threadIdx.x; m < n_omega; m += blockDim.x) {
        const double d = w0 + dw * m - x0;
        Afl[(long)j * n_omega + m] = A0 * exp(-k * d * d);
    }
}

}  // namespace qpfrg

extern "C" qpfrg_status qpfrg_spectral(qpfrg_t c, const double *d_sigma_re, const double *d_sigma_im, const double *d_Z,
                                       double *d_A, double *d_A_fl)
{
    using namespace qpfrg;
    if (!c) return QPFRG_ERR_INVALID;
    if (c->opt.n_omega < 1 || !d_sigma_re || !d_sigma_im || !d_A) {
        c->err = "qpfrg_spectral needs the frequency grid (n_omega > 0), Sigma and an output";
        return QPFRG_ERR_INVALID;
    }
    const int n = c->opt.n_omega;
    const double w0 = c->opt.omega_min, dw = n > 1 ? (c->opt.omega_max - c->opt.omega_min) / (n - 1) : 0.0;
    spectral_kernel<<<c->pb.N, 256, 0, c->stream>>>(d_sigma_re, d_sigma_im, d_Z, c->d_xij, n, w0, dw, d_A, d_A_fl);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "spectral_kernel");
}
