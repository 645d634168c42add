// Interaction flow with the self-energy ODE (App. A.2-A.5, Eq. (nutshell_2)):
// the state (V, Sigma, Sigma') advances in g at fixed T by RK4,
//   d/dg Sigma  = Sigma'
//   d/dg Sigma' = Abar Sigma' + 6 g T2[V, Z, K](w)
//   d/dg V      = one-loop RHS with G = g Z G0, S = K Z^2 G0
// where, per patch j, with s1 and s2 the chord slopes of Re Sigma and Re Sigma'
// over w = xi_j +- 2T (the margin of Sec. 3.1.1),
//   Z = (1 - g s1)^-1   (Eq. (definition_Z) for g Sigma_g)
//   K = 1 + g^2 s2      (Eq. (K_definition); 1 without the Katanin correction)
//   A = 2 Z (s1 + g s2) (Eq. (single_scale_propagator_extended_2) = Eq. (A_g_simple))
// and Abar is the average of A over the Fermi surface -- every patch of the
// angular patchings, the Fermi shell of shell mode (Eq.
// (second_derivative_sigma_approximation)),
// its minimum or maximum (the bracket flows of App. B) or 0 (the one-loop term
// dropped, App. A.4).  T2 is the two-loop term at the static vertex with the
// lines of a G, an S and an inner K S line averaged over their assignments;
// the factor 6 g makes g Sigma_g(g = 1) the second-order self-energy of U for
// a frozen vertex and Z = 1 (g Sigma_g is the self-energy of the bare coupling
// g^2 U, App. A.3).
//
// Z, K and A need only the chord slopes, so the state carries s1 and s2 per
// patch (their ODE is the chord of the one above) and, when the context has a
// frequency grid, Sigma and Sigma' on it (binned two-loop term, as
// qpfrg_selfenergy).  Small state y = [s1 (N), s2 (N), Re S, Im S, Re S',
// Im S' (N x n_omega each)], integrated by the same RK4 steps as V.
#include <cmath>

#include "qpfrg_internal.h"

namespace qpfrg {

// Z, K, A of every patch and Abar from the small state at g (one block)
__global__ void gflow_zka_kernel(const double *y, int N, int ns, double g, int z_feedback, int katanin, int a_mode,
                                 double *Z, double *K, double *A, double *Abar)
{
    __shared__ double sh_sum[256], sh_min[256], sh_max[256];
    double sum = 0.0, mn = 1e300, mx = -1e300;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double s1 = y[j], s2 = y[N + j];
        double z = 1.0, k = 1.0, a = 0.0;
        if (z_feedback) {
            z = 1.0 / (1.0 - g * s1);
            k = katanin ? 1.0 + g * g * s2 : 1.0;
            a = 2.0 * z * (s1 + g * s2);
        }
        Z[j] = z;
        K[j] = k;
        A[j] = a;
        if (j % ns != ns / 2) continue;     // Abar over the Fermi surface: the Fermi shell
        sum += a;
        mn = fmin(mn, a);
        mx = fmax(mx, a);
    }
    sh_sum[threadIdx.x] = sum;
    sh_min[threadIdx.x] = mn;
    sh_max[threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, lo = 1e300, hi = -1e300;
        for (int t = 0; t < (int)blockDim.x; ++t) {   // in thread order: deterministic
            s += sh_sum[t];
            lo = fmin(lo, sh_min[t]);
            hi = fmax(hi, sh_max[t]);
        }
        *Abar = a_mode == 1 ? lo : (a_mode == 2 ? hi : (a_mode == 3 ? 0.0 : s / (N / ns)));
    }
}

// derivative of the small state at g: d s1 = s2, d s2 = Abar s2 + 6 g chord(T2),
// on the grid d S = S', d S' = Abar S' + 6 g T2(w)
__global__ void gflow_deriv_kernel(const double *y, const double *chord, const double *t2re, const double *t2im,
                                   const double *Abar, double g, int N, int nom, double *dy)
{
    const double ab = *Abar, six_g = 6.0 * g;
    const long ng = (long)N * nom;
    const long L = 2L * N + 4 * ng;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x) {
        double d;
        if (i < N) {
            d = y[N + i];
        } else if (i < 2L * N) {
            const long j = i - N;
            d = ab * y[i] + six_g * chord[j];
        } else {
            const long r = i - 2L * N, part = r / ng, m = r - part * ng;
            const long base = 2L * N;
            if (part == 0) d = y[base + 2 * ng + m];                       // Re S' -> d Re S
            else if (part == 1) d = y[base + 3 * ng + m];                  // Im S' -> d Im S
            else if (part == 2) d = ab * y[i] + six_g * t2re[m];           // d Re S'
            else d = ab * y[i] + six_g * t2im[m];                           // d Im S'
        }
        dy[i] = d;
    }
}

// RK4 bookkeeping of the small state, the same stages as rk_stage/rk_final:
// stage 1..3: acc (+)= w k, ys = y + c_next k; stage 4: y += h/6 (acc + k)
__global__ void gflow_rk_kernel(int stage, double h, double *y, const double *k, double *acc, double *ys, long L)
{
    const double c_next = stage == 3 ? h : 0.5 * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < L; i += (long)gridDim.x * blockDim.x) {
        const double ki = k[i];
        if (stage < 4) {
            acc[i] = stage == 1 ? ki : acc[i] + 2.0 * ki;
            ys[i] = y[i] + c_next * ki;
        } else {
            y[i] += h / 6.0 * (acc[i] + ki);
        }
    }
}

long gflow_small_len(const qpfrg_ctx *c) { return 2L * c->pb.N + 4L * c->pb.N * c->opt.n_omega; }

qpfrg_status gflow_alloc(qpfrg_ctx *c)
{
    const long L = gflow_small_len(c), N = c->pb.N, ng = N * (long)c->opt.n_omega;
    double **bufs[] = {&c->d_gy, &c->d_gys, &c->d_gk, &c->d_gacc};
    for (double **b : bufs) {
        cudaError_t e = cudaMalloc((void **)b, L * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(*b, 0, L * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(self-energy ODE state)");
    }
    cudaError_t e = cudaMalloc((void **)&c->d_gzka, (3 * N + 1) * sizeof(double));
    if (e == cudaSuccess && ng > 0) e = cudaMalloc((void **)&c->d_gt2, 2 * ng * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc(self-energy ODE work)");
    return QPFRG_OK;
}

static qpfrg_status zka(qpfrg_ctx *c, const double *y, double g)
{
    const int N = c->pb.N;
    double *Z = c->d_gzka, *K = Z + N, *A = K + N, *Ab = A + N;
    gflow_zka_kernel<<<1, 256, 0, c->stream>>>(y, N, c->pb.n_shell, g, c->opt.z_feedback, c->opt.katanin, c->opt.a_mode, Z, K, A,
                                               Ab);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "gflow_zka_kernel");
}

// Enqueue one RK4 step of (V, Sigma, Sigma') from g = x with step h; the
// vertex part uses the context's RK buffers and kernels, max|V| and the
// finiteness flag land in d_red as for the other flows.
qpfrg_status gflow_enqueue_stages(qpfrg_ctx *c, double x, double h)
{
    const int N = c->pb.N, nom = c->opt.n_omega;
    const long n3 = (long)N * N * N, L = gflow_small_len(c), ng = (long)N * nom;
    const bool mixed = c->opt.precision != QPFRG_FP64;
    const double T = c->pb.T_fixed;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    const double *Zs = c->d_gzka, *Ks = Zs + N, *Ab = Ks + 2 * N;
    qpfrg_status s;
    cudaError_t e;
    if (mixed && (s = launch_convert_f32(c, c->d_V, c->d_Vf, n3)) != QPFRG_OK) return s;
    const double *Vst = c->d_V;                  // FP64 vertex of the stage (two-loop term)
    const void *Vin = mixed ? (const void *)c->d_Vf : (const void *)c->d_V;
    const double *yst = c->d_gy;
    for (int st = 0; st < 4; ++st) {
        const double gs = x + cst[st] * h;
        if ((s = zka(c, yst, gs)) != QPFRG_OK) return s;
        // vertex: loop kernels with Z and K on the lines, contraction
        if ((s = launch_bubbles(c, gs, Zs, true, c->opt.katanin ? Ks : nullptr, c->c4v_state)) != QPFRG_OK) return s;
        if ((e = cudaMemsetAsync(c->d_k, 0, n3 * sizeof(double), c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "memset k");
        if ((s = launch_contractions(c, Vin, 1.0, c->d_k)) != QPFRG_OK) return s;
        // two-loop term: chord slopes at xi_j +- 2T, and the frequency grid
        if ((s = launch_sigma_lines(c, T, Vst, Zs, c->opt.katanin ? Ks : c->d_ones)) != QPFRG_OK) return s;
        const double *t2re = nullptr, *t2im = nullptr;
        if (nom > 0) {
            if ((s = launch_sigma_grid(c, T, Vst, Zs, c->d_gt2, c->d_gt2 + ng, c->opt.katanin ? Ks : c->d_ones)) !=
                QPFRG_OK)
                return s;
            t2re = c->d_gt2;
            t2im = c->d_gt2 + ng;
        }
        gflow_deriv_kernel<<<(int)std::min<long>((L + 255) / 256, 1216), 256, 0, c->stream>>>(
            yst, c->d_sig, t2re, t2im, Ab, gs, N, nom, c->d_gk);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "gflow_deriv_kernel");
        // RK stages of both parts
        const int blocks = (int)std::min<long>((L + 255) / 256, 1216);
        gflow_rk_kernel<<<blocks, 256, 0, c->stream>>>(st + 1, h, c->d_gy, c->d_gk, c->d_gacc, c->d_gys, L);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "gflow_rk_kernel");
        if (st < 3) {
            if ((s = launch_rk_stage(c, st + 1, h, c->d_V, c->d_k, c->d_acc, c->d_Vs, mixed ? c->d_Vf : nullptr)) !=
                QPFRG_OK)
                return s;
            Vst = c->d_Vs;
            Vin = mixed ? (const void *)c->d_Vf : (const void *)c->d_Vs;
            yst = c->d_gys;
        } else if ((s = launch_rk_final(c, h, c->d_V, c->d_acc, c->d_k)) != QPFRG_OK) {
            return s;
        }
    }
    // Z, K, A of the new state (Z also becomes the context's Z)
    if ((s = zka(c, c->d_gy, x + h)) != QPFRG_OK) return s;
    e = cudaMemcpyAsync(c->d_Z, c->d_gzka, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "copy Z");
}

}  // namespace qpfrg

extern "C" qpfrg_status qpfrg_read_sigma_flow(qpfrg_t c, double *d_slopes, double *d_sigma, double *d_zka)
{
    using namespace qpfrg;
    if (!c) return QPFRG_ERR_INVALID;
    if (!c->d_gy) {
        c->err = "the context has no self-energy ODE (options.sigma_ode)";
        return QPFRG_ERR_INVALID;
    }
    const long N = c->pb.N, ng = N * (long)c->opt.n_omega;
    cudaError_t e = cudaSuccess;
    if (d_slopes) e = cudaMemcpyAsync(d_slopes, c->d_gy, 2 * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && d_sigma && ng > 0)
        e = cudaMemcpyAsync(d_sigma, c->d_gy + 2 * N, 4 * ng * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && d_zka)
        e = cudaMemcpyAsync(d_zka, c->d_gzka, (3 * N + 1) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "read_sigma_flow");
}
