// Patch geometry and partner-patch maps.
//
// The paper fixes only patch counts (Sec. 3.2: 32 angular x 7 energy, 48
// angular, 728 total; Fig. 4 caption: 1 and 4 patches between antinode and
// node).  This library takes angular wedges about the origin with centres at
// theta_j = 2 pi j / N ((pi,0) is a centre), representatives k_F(j) on the
// Fermi surface xi = 0 (Eq. (free_dispersion_xi)) along theta_j, and a polar
// fine grid per wedge: n_theta angular midpoints x n_r radial midpoint cells,
// n_r/2 uniform in (0, r_F(theta)) and n_r/2 in (r_F(theta), r_BZ(theta)),
// weight = cell area / (2 pi)^2 so that sum_p w_p ~ int d^2p/(2 pi)^2 = 1.
// Lattice mode instead takes every momentum of an L x L lattice as a patch.
#include <cmath>
#include <cstring>
#include <vector>

#include "qpfrg_internal.h"

namespace qpfrg {

// Cell table of the FP32 wedge projection (sigma.cu).  The kernels hold a
// folded momentum as fixed-point turns X = x 2^32 / 2 pi in [-2^31, 2^31), so
// the cell of a component is its top byte: K = (X >> 24) + W/2, K in 0..W-1,
// covering [-pi + K h, -pi + (K + 1) h), h = 2 pi / W (W = 256).  The entry is
// the lower of the at most two wedges that the cell, widened by 2e-5 on every
// side, touches (the ray between them is then tested in the kernel), or 255
// when it touches three or more wedges or contains the origin.  The margin
// exceeds the 2e-7 rad position error of the fixed-point momenta and of their
// FP32 conversion.  Rows (K_y) are kProjStride bytes apart.
static std::vector<uint8_t> build_proj_table(int N)
{
    const int W = kProjW;
    const double h = kTwoPi / W, m = 2e-5, dth = kTwoPi / N;
    std::vector<uint8_t> tab((size_t)W * kProjStride, 255);
    for (int ky = 0; ky < W; ++ky)
        for (int kx = 0; kx < W; ++kx) {
            const double x0 = -kPi + kx * h - m, x1 = -kPi + (kx + 1) * h + m;
            const double y0 = -kPi + ky * h - m, y1 = -kPi + (ky + 1) * h + m;
            if (x0 <= 0.0 && x1 >= 0.0 && y0 <= 0.0 && y1 >= 0.0) continue;
            // the angular extent of a rectangle clear of the origin is spanned
            // by its corners; unwrap them about the first corner
            const double cx[4] = {x0, x1, x0, x1}, cy[4] = {y0, y0, y1, y1};
            const double a0 = std::atan2(cy[0], cx[0]);
            double lo = 0.0, hi = 0.0;
            for (int k = 1; k < 4; ++k) {
                const double d = std::remainder(std::atan2(cy[k], cx[k]) - a0, kTwoPi);
                lo = std::fmin(lo, d);
                hi = std::fmax(hi, d);
            }
            const long jl = (long)std::floor((a0 + lo) / dth + 0.5);
            const long jh = (long)std::floor((a0 + hi) / dth + 0.5);
            if (jh - jl <= 1) tab[(size_t)ky * kProjStride + kx] = (uint8_t)(((jl % N) + N) % N);
        }
    return tab;
}

static double host_xi(const Problem &pb, double kx, double ky)
{
    const double ckx = std::cos(kx), cky = std::cos(ky);
    return -2.0 * pb.t * (ckx + cky) - 4.0 * pb.tp * ckx * cky - pb.mu;
}

// Distance from the origin to the boundary of [-pi, pi]^2 along angle th.
static double bz_radius(double th)
{
    return kPi / std::fmax(std::fabs(std::cos(th)), std::fabs(std::sin(th)));
}

// First crossing of xi = eps along the ray at angle th (bisection on
// xi < eps); the BZ edge when xi stays below eps, 0 when the origin is
// already at or above it.
static double level_radius(const Problem &pb, double th, double eps)
{
    const double c = std::cos(th), s = std::sin(th);
    double hi = bz_radius(th);
    if (host_xi(pb, hi * c, hi * s) < eps) return hi;
    if (host_xi(pb, 0.0, 0.0) >= eps) return 0.0;
    double lo = 0.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (host_xi(pb, mid * c, mid * s) < eps)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

// The Fermi surface along the ray: the level xi = 0.
static double fermi_radius(const Problem &pb, double th) { return level_radius(pb, th, 0.0); }

// Shell width of shell mode: the given width, else the band width 2 max|xi|
// (band extremes at (0,0), (pi,pi), (pi,0) for |t'| <= t/2) over the shells.
double shell_width(const Problem &pb, double given)
{
    if (given > 0.0) return given;
    const double w = std::fmax(std::fabs(host_xi(pb, 0.0, 0.0)),
                               std::fmax(std::fabs(host_xi(pb, kPi, kPi)), std::fabs(host_xi(pb, kPi, 0.0))));
    return 2.0 * w / pb.n_shell;
}

// Whether xi does not decrease along the ray (512 samples): the shells then
// cut every ray in one segment each.
static bool ray_monotone(const Problem &pb, double th)
{
    const double rb = bz_radius(th), c = std::cos(th), s = std::sin(th);
    double prev = host_xi(pb, 0.0, 0.0);
    for (int i = 1; i <= 512; ++i) {
        const double r = rb * i / 512.0;
        const double x = host_xi(pb, r * c, r * s);
        if (x < prev - 1e-12) return false;
        prev = x;
    }
    return true;
}

// Shell mode: N_a = N / n_s wedges, each cut at the shell edges
// e_b = (b - n_s/2) D; patch j = w n_s + s.  Per angular midpoint ray the
// shell's segment [r(e_s), r(e_{s+1})] (0 and the zone edge for the outer
// shells) is split into n_r midpoint cells, the Fermi shell's at r_F(theta)
// into n_r/2 + n_r/2, so that one shell reproduces the wedge grid.
static qpfrg_status build_shell_geometry(qpfrg_ctx *c)
{
    const Problem &pb = c->pb;
    const int ns = pb.n_shell, Na = pb.N / ns, sF = ns / 2;
    const int nt = c->n_theta, nr = c->n_r, nh = c->n_r / 2;
    const double dth = kTwoPi / Na, D = pb.shell_D;
    for (int w = 0; w < Na; ++w) {
        const double thw = dth * w;
        bool mono = ray_monotone(pb, thw);
        for (int a = 0; a < nt && mono; ++a) mono = ray_monotone(pb, thw + ((a + 0.5) / nt - 0.5) * dth);
        if (!mono) {
            c->err = "shell mode needs xi increasing along every ray from the origin to the zone edge";
            return QPFRG_ERR_UNSUPPORTED;
        }
        for (int sh = 0; sh < ns; ++sh) {
            const int j = w * ns + sh;
            const double rj = sh == sF ? fermi_radius(pb, thw) : level_radius(pb, thw, (sh - sF) * D);
            c->kf[2 * j] = rj * std::cos(thw);
            c->kf[2 * j + 1] = rj * std::sin(thw);
            for (int a = 0; a < nt; ++a) {
                const double th = thw + ((a + 0.5) / nt - 0.5) * dth;
                const double r0 = sh == 0 ? 0.0 : level_radius(pb, th, (sh - 0.5 * ns) * D);
                const double r1 = sh == ns - 1 ? bz_radius(th) : level_radius(pb, th, (sh + 1 - 0.5 * ns) * D);
                const double rf = fermi_radius(pb, th);
                for (int i = 0; i < nr; ++i) {
                    double q0, q1;
                    if (sh != sF) {
                        q0 = r0 + (r1 - r0) * i / nr;
                        q1 = r0 + (r1 - r0) * (i + 1) / nr;
                    } else if (i < nh) {
                        q0 = r0 + (rf - r0) * i / nh;
                        q1 = r0 + (rf - r0) * (i + 1) / nh;
                    } else {
                        q0 = rf + (r1 - rf) * (i - nh) / nh;
                        q1 = rf + (r1 - rf) * (i - nh + 1) / nh;
                    }
                    const double r = 0.5 * (q0 + q1);
                    const size_t p = ((size_t)j * nt + a) * nr + i;
                    c->fk[2 * p] = r * std::cos(th);
                    c->fk[2 * p + 1] = r * std::sin(th);
                    c->fw[p] = 0.5 * (q1 * q1 - q0 * q0) * (dth / nt) / (kTwoPi * kTwoPi);
                    c->fpatch[p] = j;
                }
            }
        }
    }
    c->fw_max = 0.0;
    for (double w : c->fw) c->fw_max = std::fmax(c->fw_max, w);
    return QPFRG_OK;
}

qpfrg_status build_host_geometry(qpfrg_ctx *c)
{
    const Problem &pb = c->pb;
    const int N = pb.N, M = pb.M;
    c->kf.assign(2 * (size_t)N, 0.0);
    c->fk.assign(2 * (size_t)M, 0.0);
    c->fw.assign((size_t)M, 0.0);
    c->fpatch.assign((size_t)M, 0);

    if (pb.mode == QPFRG_GRID_LATTICE) {
        const int L = pb.L;
        for (int m1 = 0; m1 < L; ++m1)
            for (int m2 = 0; m2 < L; ++m2) {
                const int j = m1 * L + m2;
                const double kx = kTwoPi * m1 / L, ky = kTwoPi * m2 / L;
                c->kf[2 * j] = kx;
                c->kf[2 * j + 1] = ky;
                c->fk[2 * j] = kx;
                c->fk[2 * j + 1] = ky;
                c->fw[j] = 1.0 / N;
                c->fpatch[j] = j;
            }
        c->fw_max = 1.0 / N;
        return QPFRG_OK;
    }
    if (pb.mode == QPFRG_GRID_SHELL) return build_shell_geometry(c);

    const double dth = kTwoPi / N;
    const int nt = c->n_theta, nr = c->n_r, nh = c->n_r / 2;
    for (int j = 0; j < N; ++j) {
        const double thj = dth * j;
        const double rfj = fermi_radius(pb, thj);
        c->kf[2 * j] = rfj * std::cos(thj);
        c->kf[2 * j + 1] = rfj * std::sin(thj);
        for (int a = 0; a < nt; ++a) {
            const double th = thj + ((a + 0.5) / nt - 0.5) * dth;
            const double rf = fermi_radius(pb, th), rb = bz_radius(th);
            for (int s = 0; s < nr; ++s) {
                double r0, r1;
                if (s < nh) {
                    r0 = rf * s / nh;
                    r1 = rf * (s + 1) / nh;
                } else {
                    r0 = rf + (rb - rf) * (s - nh) / nh;
                    r1 = rf + (rb - rf) * (s - nh + 1) / nh;
                }
                const double r = 0.5 * (r0 + r1);
                const size_t p = ((size_t)j * nt + a) * nr + s;
                c->fk[2 * p] = r * std::cos(th);
                c->fk[2 * p + 1] = r * std::sin(th);
                c->fw[p] = 0.5 * (r1 * r1 - r0 * r0) * (dth / nt) / (kTwoPi * kTwoPi);
                c->fpatch[p] = j;
            }
        }
    }
    c->fw_max = 0.0;
    for (double w : c->fw) c->fw_max = std::fmax(c->fw_max, w);
    return QPFRG_OK;
}

// part[f][Q][a P + part_byte(t, s)] = patch of (Q - p) for f = 0 (pp) and of
// (p + Q) for f = 1 (ph), p = a P + t n_r + s the fine point (t angular, s
// radial); part_byte orders a patch's bytes for the loop kernels' reads.
__global__ void partner_map_kernel(const double *__restrict__ Qpp, const double *__restrict__ Qph,
                                   const double *__restrict__ fkx, const double *__restrict__ fky,
                                   uint8_t *__restrict__ part, Problem pb)
{
    const int N = pb.N, M = pb.M, P = pb.P, nt = pb.n_theta, nr = pb.n_r;
    const int Q = blockIdx.x, f = blockIdx.z;
    const long NN = (long)N * N;
    const double *Qt = f == 0 ? Qpp : Qph;
    const double Qx = Qt[2 * Q], Qy = Qt[2 * Q + 1];
    uint8_t *row = part + ((long)f * NN + Q) * (long)M;
    for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < M; p += gridDim.y * blockDim.x) {
        const double px = fkx[p], py = fky[p];
        const double qx = f == 0 ? Qx - px : px + Qx;
        const double qy = f == 0 ? Qy - py : py + Qy;
        const int a = p / P, li = p - a * P, t = li / nr, s = li - t * nr;
        row[a * P + part_byte(t, s, nt, nr)] = (uint8_t)project_fp64(qx, qy, pb);
    }
}

// Wedge-mode partner maps from fixed-point momenta (angle_fx): the cell table
// and one FP32 test against the ray between its two wedges decide, as in the
// self-energy kernels; points within the guard bands of a ray or of the zone
// edge, or in a cell of three or more wedges, take project_patch, so every
// byte equals the FP64 projection.  Qfx[f][Q], pfx[p]: fixed-point momenta.
__global__ void partner_map_fx_kernel(const int2 *__restrict__ Qfx, const double *__restrict__ Qpp,
                                      const double *__restrict__ Qph, const int2 *__restrict__ pfx,
                                      const double *__restrict__ fkx, const double *__restrict__ fky,
                                      const uint8_t *__restrict__ ptab, const float4 *__restrict__ bnd,
                                      uint8_t *__restrict__ part, Problem pb)
{
    const int N = pb.N, M = pb.M, P = pb.P, nt = pb.n_theta, nr = pb.n_r;
    const int Q = blockIdx.x, f = blockIdx.z;
    const long NN = (long)N * N;
    const int2 qf = Qfx[f * NN + Q];
    const double *Qt = f == 0 ? Qpp : Qph;
    uint8_t *row = part + ((long)f * NN + Q) * (long)M;
    const uint8_t *tabc = ptab + (kProjW / 2) * (kProjStride + 1);   // the cell of the origin
    for (int p = blockIdx.y * blockDim.x + threadIdx.x; p < M; p += gridDim.y * blockDim.x) {
        const int2 pf = pfx[p];
        // pp: Q - p, ph: p + Q, folded by the wrap of 32-bit arithmetic
        const int X = (int)(f == 0 ? (unsigned)qf.x - (unsigned)pf.x : (unsigned)pf.x + (unsigned)qf.x);
        const int Y = (int)(f == 0 ? (unsigned)qf.y - (unsigned)pf.y : (unsigned)pf.y + (unsigned)qf.y);
        const float x = __int2float_rn(X), y = __int2float_rn(Y);
        const int e = __ldg(tabc + (Y >> 24) * kProjStride + (X >> 24));
        float rx = 0.f, ry = 0.f;   // ray between wedges e and e + 1 (none for e = 255)
        if (e + 1 <= N) {
            const float4 b = __ldg(bnd + (e + 1 == N ? 0 : e + 1));
            rx = b.x;
            ry = b.z;
        }
        const float cr = rx * y - ry * x;
        int c;
        if (fmaxf(fabsf(x), fabsf(y)) > kFxEdge || fabsf(cr) < kFxGuard) {
            const double px = fkx[p], py = fky[p], Qx = Qt[2 * Q], Qy = Qt[2 * Q + 1];
            c = project_fp64(f == 0 ? Qx - px : px + Qx, f == 0 ? Qy - py : py + Qy, pb);
        } else {
            c = e + (cr >= 0.f ? 1 : 0);
            if (c == N) c = 0;
        }
        const int a = p / P, li = p - a * P, t = li / nr, s = li - t * nr;
        row[a * P + part_byte(t, s, nt, nr)] = (uint8_t)c;
    }
}

template <typename R>
static qpfrg_status alloc_fine(qpfrg_ctx *c, FineTable<R> &t)
{
    const size_t M = c->pb.M;
    R **fields[] = {&t.kx, &t.ky, &t.cx, &t.sx, &t.cy, &t.sy, &t.xi, &t.w};
    for (R **f : fields) {
        cudaError_t e = cudaMalloc((void **)f, M * sizeof(R));
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(fine table)");
    }
    std::vector<R> h(M);
    auto put = [&](R *dst, auto fn) -> qpfrg_status {
        for (size_t p = 0; p < M; ++p) h[p] = (R)fn(p);
        cudaError_t e = cudaMemcpy(dst, h.data(), M * sizeof(R), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "upload fine table");
    };
    const std::vector<double> &fk = c->fk;
    qpfrg_status s;
    if ((s = put(t.kx, [&](size_t p) { return fk[2 * p]; })) != QPFRG_OK) return s;
    if ((s = put(t.ky, [&](size_t p) { return fk[2 * p + 1]; })) != QPFRG_OK) return s;
    if ((s = put(t.cx, [&](size_t p) { return std::cos(fk[2 * p]); })) != QPFRG_OK) return s;
    if ((s = put(t.sx, [&](size_t p) { return std::sin(fk[2 * p]); })) != QPFRG_OK) return s;
    if ((s = put(t.cy, [&](size_t p) { return std::cos(fk[2 * p + 1]); })) != QPFRG_OK) return s;
    if ((s = put(t.sy, [&](size_t p) { return std::sin(fk[2 * p + 1]); })) != QPFRG_OK) return s;
    if ((s = put(t.xi, [&](size_t p) { return host_xi(c->pb, fk[2 * p], fk[2 * p + 1]); })) != QPFRG_OK)
        return s;
    if ((s = put(t.w, [&](size_t p) { return c->fw[p]; })) != QPFRG_OK) return s;
    return QPFRG_OK;
}

template <typename R>
static qpfrg_status alloc_transfer(qpfrg_ctx *c, TransferTable<R> &t, const std::vector<double> &Q)
{
    const size_t NN = (size_t)c->pb.N * c->pb.N;
    R **fields[] = {&t.cx, &t.sx, &t.cy, &t.sy};
    for (R **f : fields) {
        cudaError_t e = cudaMalloc((void **)f, NN * sizeof(R));
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(transfer table)");
    }
    std::vector<R> h(NN);
    for (int comp = 0; comp < 4; ++comp) {
        for (size_t q = 0; q < NN; ++q) {
            const double v = Q[2 * q + (comp >= 2 ? 1 : 0)];
            h[q] = (R)((comp % 2 == 0) ? std::cos(v) : std::sin(v));
        }
        cudaError_t e = cudaMemcpy(*fields[comp], h.data(), NN * sizeof(R), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "upload transfer table");
    }
    return QPFRG_OK;
}

qpfrg_status upload_geometry(qpfrg_ctx *c)
{
    const int N = c->pb.N;
    const size_t NN = (size_t)N * N;
    std::vector<double> Qpp(2 * NN), Qph(2 * NN);
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
            const size_t q = (size_t)x * N + y;
            Qpp[2 * q] = c->kf[2 * x] + c->kf[2 * y];
            Qpp[2 * q + 1] = c->kf[2 * x + 1] + c->kf[2 * y + 1];
            Qph[2 * q] = c->kf[2 * x] - c->kf[2 * y];
            Qph[2 * q + 1] = c->kf[2 * x + 1] - c->kf[2 * y + 1];
        }
    qpfrg_status s;
    if ((s = alloc_fine(c, c->f64)) != QPFRG_OK) return s;
    if ((s = alloc_fine(c, c->f32)) != QPFRG_OK) return s;
    if ((s = alloc_transfer(c, c->qpp64, Qpp)) != QPFRG_OK) return s;
    if ((s = alloc_transfer(c, c->qph64, Qph)) != QPFRG_OK) return s;
    if ((s = alloc_transfer(c, c->qpp32, Qpp)) != QPFRG_OK) return s;
    if ((s = alloc_transfer(c, c->qph32, Qph)) != QPFRG_OK) return s;

    cudaError_t e;
    if ((e = cudaMalloc((void **)&c->d_kf, 2 * N * sizeof(double))) != cudaSuccess)
        return cuda_fail(c, e, "cudaMalloc(kf)");
    if ((e = cudaMemcpy(c->d_kf, c->kf.data(), 2 * N * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "upload kf");
    {
        std::vector<double> xij(N);
        std::vector<float4> bnd(N);
        for (int j = 0; j < N; ++j) {
            xij[j] = host_xi(c->pb, c->kf[2 * j], c->kf[2 * j + 1]);
            // ray between wedges w - 1 and w (entries past the N_a wedges repeat them)
            const int Na = N / c->pb.n_shell;
            const double th = (j % Na - 0.5) * kTwoPi / Na, cs = std::cos(th), sn = std::sin(th);
            const float ch = (float)cs, sh = (float)sn;
            bnd[j] = make_float4(ch, (float)(cs - ch), sh, (float)(sn - sh));
        }
        const size_t M = c->pb.M;
        std::vector<float> xl(M), yl(M);
        for (size_t p = 0; p < M; ++p) {
            xl[p] = (float)(c->fk[2 * p] - (double)(float)c->fk[2 * p]);
            yl[p] = (float)(c->fk[2 * p + 1] - (double)(float)c->fk[2 * p + 1]);
        }
        std::vector<float> xijf(xij.begin(), xij.end());
        if ((e = cudaMalloc((void **)&c->d_xij_f, N * sizeof(float))) != cudaSuccess)
            return cuda_fail(c, e, "cudaMalloc(xi_j fp32)");
        cudaMemcpy(c->d_xij_f, xijf.data(), N * sizeof(float), cudaMemcpyHostToDevice);
        if ((e = cudaMalloc((void **)&c->d_xij, N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_bnd, N * sizeof(float4))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_qxl, M * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_qyl, M * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_kp, (size_t)N * M * sizeof(float4))) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_kcs, N * sizeof(float4))) != cudaSuccess)
            return cuda_fail(c, e, "cudaMalloc(xi_j, rays, residuals, k+p)");
        cudaMemcpy(c->d_xij, xij.data(), N * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_bnd, bnd.data(), N * sizeof(float4), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_qxl, xl.data(), M * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_qyl, yl.data(), M * sizeof(float), cudaMemcpyHostToDevice);
        if (c->pb.mode == QPFRG_GRID_WEDGE && N <= 254) {
            std::vector<uint8_t> tab = build_proj_table(N);
            const size_t bytes = (tab.size() + 15) / 16 * 16;
            tab.resize(bytes, 255);
            if ((e = cudaMalloc((void **)&c->d_ptab, bytes)) != cudaSuccess)
                return cuda_fail(c, e, "cudaMalloc(projection table)");
            cudaMemcpy(c->d_ptab, tab.data(), bytes, cudaMemcpyHostToDevice);
        }
    }
    if ((e = cudaMalloc((void **)&c->d_Qpp, 2 * NN * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_Qph, 2 * NN * sizeof(double))) != cudaSuccess)
        return cuda_fail(c, e, "cudaMalloc(Q)");
    cudaMemcpy(c->d_Qpp, Qpp.data(), 2 * NN * sizeof(double), cudaMemcpyHostToDevice);
    if ((e = cudaMemcpy(c->d_Qph, Qph.data(), 2 * NN * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(c, e, "upload Q");

    const size_t part_bytes = 2 * NN * (size_t)c->pb.M;
    if ((e = cudaMalloc((void **)&c->d_part, part_bytes)) != cudaSuccess)
        return cuda_fail(c, e, "cudaMalloc(partner maps)");
    const int pblocks = div_up(c->pb.M, 256 * 4);
    dim3 grid((unsigned)NN, pblocks < 1 ? 1 : (pblocks > 65535 ? 65535 : pblocks), 2);
    if (c->d_ptab) {
        // wedge mode: fixed-point decisions, FP64 only in the guard bands
        const size_t M = c->pb.M;
        std::vector<int2> qfx(2 * NN), pfx(M);
        for (size_t q = 0; q < NN; ++q) {
            qfx[q] = make_int2(angle_fx(Qpp[2 * q]), angle_fx(Qpp[2 * q + 1]));
            qfx[NN + q] = make_int2(angle_fx(Qph[2 * q]), angle_fx(Qph[2 * q + 1]));
        }
        for (size_t p = 0; p < M; ++p) pfx[p] = make_int2(angle_fx(c->fk[2 * p]), angle_fx(c->fk[2 * p + 1]));
        int2 *d_qfx = nullptr, *d_pfx = nullptr;
        if ((e = cudaMalloc((void **)&d_qfx, 2 * NN * sizeof(int2))) != cudaSuccess ||
            (e = cudaMalloc((void **)&d_pfx, M * sizeof(int2))) != cudaSuccess) {
            cudaFree(d_qfx);
            return cuda_fail(c, e, "cudaMalloc(fixed-point momenta)");
        }
        cudaMemcpy(d_qfx, qfx.data(), 2 * NN * sizeof(int2), cudaMemcpyHostToDevice);
        cudaMemcpy(d_pfx, pfx.data(), M * sizeof(int2), cudaMemcpyHostToDevice);
        prof_begin(c);
        partner_map_fx_kernel<<<grid, 256, 0, c->stream>>>(d_qfx, c->d_Qpp, c->d_Qph, d_pfx, c->f64.kx, c->f64.ky,
                                                           c->d_ptab, c->d_bnd, c->d_part, c->pb);
        prof_end(c, K_PARTNER_MAP);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // before the momenta are released
        cudaFree(d_qfx);
        cudaFree(d_pfx);
        if (e != cudaSuccess) return cuda_fail(c, e, "partner_map_fx_kernel");
        return QPFRG_OK;
    }
    prof_begin(c);
    partner_map_kernel<<<grid, 256, 0, c->stream>>>(c->d_Qpp, c->d_Qph, c->f64.kx, c->f64.ky, c->d_part, c->pb);
    prof_end(c, K_PARTNER_MAP);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "partner_map_kernel");
    return QPFRG_OK;
}

}  // namespace qpfrg
