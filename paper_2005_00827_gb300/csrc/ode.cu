// Classical RK4 on the FP64 flow state (Sec. 3.2: the flow is integrated
// until the largest coupling passes a bound).  The stage kernels combine the
// stage derivative k into the weighted sum and form the next stage input
// (FP64, plus the FP32 copy the mixed-precision right-hand side reads); the
// final kernel advances V and reduces max|V| and a non-finite flag.
#include "qpfrg_internal.h"

namespace qpfrg {

__global__ void convert_f32_kernel(const double *__restrict__ in, float *__restrict__ out, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// stage 1: acc = k;    Vs = V + h/2 k
// stage 2: acc += 2k;  Vs = V + h/2 k
// stage 3: acc += 2k;  Vs = V + h k
__global__ void rk_stage_kernel(int stage, double h, const double *__restrict__ V, const double *__restrict__ k,
                                double *__restrict__ acc, double *__restrict__ Vs, float *__restrict__ Vf, long n)
{
    const double c_next = stage == 3 ? h : 0.5 * h;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double ki = k[i];
        acc[i] = stage == 1 ? ki : acc[i] + 2.0 * ki;
        const double v = V[i] + c_next * ki;
        if (Vs) Vs[i] = v;
        if (Vf) Vf[i] = (float)v;
    }
}

__device__ __forceinline__ void reduce_max_flag(double m, unsigned nonfinite, unsigned long long *red)
{
    // |V| >= 0: the IEEE bit pattern orders like an unsigned integer
    unsigned long long bits = __double_as_longlong(m);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, bits, off);
        bits = o > bits ? o : bits;
        nonfinite |= __shfl_down_sync(0xffffffffu, nonfinite, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&red[0], bits);
        if (nonfinite) atomicOr(&red[1], 1ull);
    }
}

// V += h/6 (acc + k); red[0] = max|V| bits, red[1] = non-finite flag
__global__ void rk_final_kernel(double h, double *__restrict__ V, const double *__restrict__ acc,
                                const double *__restrict__ k, long n, unsigned long long *red)
{
    double m = 0.0;
    unsigned bad = 0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double v = V[i] + h / 6.0 * (acc[i] + k[i]);
        V[i] = v;
        if (!isfinite(v)) bad = 1;
        else m = fmax(m, fabs(v));
    }
    reduce_max_flag(m, bad, red);
}

__global__ void check_finite_kernel(const double *__restrict__ x, long n, unsigned long long *red)
{
    double m = 0.0;
    unsigned bad = 0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double v = x[i];
        if (!isfinite(v)) bad = 1;
        else m = fmax(m, fabs(v));
    }
    reduce_max_flag(m, bad, red);
}

// C4v test of a state image: red[4] is set when an element's image under one
// of the 7 non-trivial group elements (wedge w -> +-w + m N_a/4 of patch
// j = w ns + s, the shell s kept; N_a = N / ns a multiple of 4) differs from
// it by more than tol max|V| (tol max|Z| for Z); red[0] and red[2] hold max|V|
// and max|Z| (bits) from check_finite_kernel.
__global__ void state_c4v_kernel(const double *__restrict__ V, const double *__restrict__ Z, int N, int ns,
                                 double tol, unsigned long long *red)
{
    const double tv = tol * __longlong_as_double(red[0]), tz = tol * __longlong_as_double(red[2]);
    const long NN = (long)N * N, n3 = NN * N;
    const int Na = N / ns, q = Na / 4;
    unsigned bad = 0;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n3; idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / NN), j = (int)((idx / N) % N), l = (int)(idx % N);
        const double v = V[idx];
        for (int g = 1; g < 8; ++g) {
            const int m = g & 3, sg = g < 4 ? 1 : -1;
            auto img = [&](int x) { return ((sg * (x / ns) + m * q) % Na + Na) % Na * ns + x % ns; };
            if (fabs(V[((long)img(i) * N + img(j)) * N + img(l)] - v) > tv) bad = 1;
            if (idx < N && fabs(Z[img((int)idx)] - Z[idx]) > tz) bad = 1;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&red[4], 1ull);
}

static int grid_for(long n)
{
    long b = (n + 255) / 256;
    if (b > 152L * 16) b = 152L * 16;
    return (int)(b < 1 ? 1 : b);
}

qpfrg_status launch_convert_f32(qpfrg_ctx *c, const double *d_in, float *d_out, long n)
{
    prof_begin(c);
    convert_f32_kernel<<<grid_for(n), 256, 0, c->stream>>>(d_in, d_out, n);
    prof_end(c, K_CONVERT);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "convert_f32_kernel");
}

qpfrg_status launch_rk_stage(qpfrg_ctx *c, int stage, double h, const double *d_V, const double *d_k,
                             double *d_acc, double *d_Vs, float *d_Vf)
{
    const long n = (long)c->pb.N * c->pb.N * c->pb.N;
    prof_begin(c);
    rk_stage_kernel<<<grid_for(n), 256, 0, c->stream>>>(stage, h, d_V, d_k, d_acc, d_Vs, d_Vf, n);
    prof_end(c, K_RK_STAGE);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "rk_stage_kernel");
}

// Checks of a state image staged on the device: red[0], red[1] = max|V| bits and
// non-finite flag of V; red[2], red[3] the same for Z; red[4] = C4v asymmetry
// (only when c4v_test, with relative tolerance tol).
qpfrg_status launch_state_check(qpfrg_ctx *c, const double *d_V, const double *d_Z, bool c4v_test, double tol)
{
    const long n = (long)c->pb.N * c->pb.N * c->pb.N;
    cudaError_t e = cudaMemsetAsync(c->d_red, 0, 5 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset state check");
    check_finite_kernel<<<grid_for(n), 256, 0, c->stream>>>(d_V, n, c->d_red);
    check_finite_kernel<<<1, 256, 0, c->stream>>>(d_Z, c->pb.N, c->d_red + 2);
    if (c4v_test)
        state_c4v_kernel<<<grid_for(n), 256, 0, c->stream>>>(d_V, d_Z, c->pb.N, c->pb.n_shell, tol, c->d_red);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "state check kernels");
}

qpfrg_status launch_rk_final(qpfrg_ctx *c, double h, double *d_V, const double *d_acc, const double *d_k)
{
    const long n = (long)c->pb.N * c->pb.N * c->pb.N;
    cudaError_t e = cudaMemsetAsync(c->d_red, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset reduction");
    prof_begin(c);
    rk_final_kernel<<<grid_for(n), 256, 0, c->stream>>>(h, d_V, d_acc, d_k, n, c->d_red);
    prof_end(c, K_RK_FINAL);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "rk_final_kernel");
}

qpfrg_status launch_check_finite(qpfrg_ctx *c, const double *d_x, long n)
{
    cudaError_t e = cudaMemsetAsync(c->d_red, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset reduction");
    check_finite_kernel<<<grid_for(n), 256, 0, c->stream>>>(d_x, n, c->d_red);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "check_finite_kernel");
}

}  // namespace qpfrg
