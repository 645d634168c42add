// Quasi-particle weights Z_j without any device allocation.
//
// Some callers cannot allocate device memory while they run: code that
// executes inside another runtime's memory pool, a driver that may only use
// memory it was handed, or a process that must not grow its footprint once it
// has started.  qpfrg_zfactor_static serves them: the caller passes every
// input and output buffer, and the only scratch -- one FP64 accumulator per
// patch for the chord slope of Re Sigma -- lives in a file-scope device array
// of QPFRG_STATIC_MAX_PATCHES entries that every GPU loading this library
// holds until the process exits.
//
// The arithmetic is the FP64 two-loop self-energy of sigma.cu, with the
// point tables (cos/sin, dispersion, Fermi factors) built on the fly from
// the caller's fine-point array instead of a context.
#include <mutex>

#include "qpfrg_internal.h"

namespace qpfrg {
namespace zstatic {

// Shared scratch: the chord slope per patch.  All calls share it, so calls
// that overlap on the GPU (different streams, or different host threads on
// one device) race; each call zeroes the entries it uses before summing.
static __device__ __align__(256) double g_slope[QPFRG_STATIC_MAX_PATCHES];

struct Args {
    int N, P, M, mode, L;
    double t, tp, mu, T, eta;
    int qp;
    const double *fine;   // M x 4: kx, ky, w, patch
    const double *kf;     // N x 2
    const double *V;      // N^3
    const double *Z;      // N (may be NULL)
};

__device__ __forceinline__ double xi_of(const Args &A, double cx, double cy)
{
    return -2.0 * A.t * (cx + cy) - 4.0 * A.tp * cx * cy - A.mu;
}

__device__ __forceinline__ void fermi2(double x, double invT, double &f, double &fc)
{
    const double e = exp(-fabs(x) * invT);
    const double hi = 1.0 / (1.0 + e), lo = e * hi;
    f = x > 0.0 ? lo : hi;
    fc = x > 0.0 ? hi : lo;
}

__device__ __forceinline__ int proj(const Args &A, double kx, double ky)
{
    if (A.mode == QPFRG_GRID_LATTICE) {
        long m1 = (long)rint(kx * A.L / kTwoPi) % A.L;
        long m2 = (long)rint(ky * A.L / kTwoPi) % A.L;
        if (m1 < 0) m1 += A.L;
        if (m2 < 0) m2 += A.L;
        return (int)(m1 * A.L + m2);
    }
    const double x = kx - kTwoPi * rint(kx / kTwoPi);
    const double y = ky - kTwoPi * rint(ky / kTwoPi);
    long j = (long)floor(atan2(y, x) / (kTwoPi / A.N) + 0.5);
    j %= A.N;
    if (j < 0) j += A.N;
    return (int)j;
}

__global__ void zero_kernel(double *slope, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) slope[i] = 0.0;
}

// grid (q blocks, patch a of p, target j); one q per thread, patch a's points
// staged in shared memory: kx+p, ky+p, cos/sin of k+p, x_p, f_p, 1-f_p, w_p.
__global__ void __launch_bounds__(256) pair_kernel(Args A, double *slope)
{
    const int a = blockIdx.y, j = blockIdx.z, tid = threadIdx.x;
    const int N = A.N, P = A.P;
    extern __shared__ double sp[];   // 10 P
    const double invT = 1.0 / A.T, eta2 = A.eta * A.eta;
    const double kx = A.kf[2 * j], ky = A.kf[2 * j + 1];
    const double za = A.Z ? A.Z[a] : 1.0;
    for (int i = tid; i < P; i += blockDim.x) {
        const double *f = A.fine + 4 * (size_t)(a * P + i);
        const double px = f[0], py = f[1];
        const double kpx = kx + px, kpy = ky + py;
        double *rec = sp + 10 * i;
        rec[0] = kpx;
        rec[1] = kpy;
        sincos(kpx, &rec[3], &rec[2]);
        sincos(kpy, &rec[5], &rec[4]);
        const double x = (A.qp ? za : 1.0) * xi_of(A, cos(px), cos(py));
        rec[6] = x;
        fermi2(x, invT, rec[7], rec[8]);
        rec[9] = f[2];
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + tid;
    double acc = 0.0;
    if (q < A.M) {
        const double *fq = A.fine + 4 * (size_t)q;
        const double qx = fq[0], qy = fq[1], wq = fq[2];
        const int b = q / P;
        double sqx, cqx, sqy, cqy;
        sincos(qx, &sqx, &cqx);
        sincos(qy, &sqy, &cqy);
        const double zb = A.Z ? A.Z[b] : 1.0;
        const double xq = (A.qp ? zb : 1.0) * xi_of(A, cqx, cqy);
        double fqv, fcq;
        fermi2(xq, invT, fqv, fcq);
        const double vab = A.V[((size_t)j * N + a) * N + b];
        const double xij = xi_of(A, cos(kx), cos(ky));
        for (int i = 0; i < P; ++i) {
            const double *r = sp + 10 * i;
            const int c = proj(A, r[0] - qx, r[1] - qy);
            const double zc = A.Z ? A.Z[c] : 1.0;
            const double crx = r[2] * cqx + r[3] * sqx, cry = r[4] * cqy + r[5] * sqy;
            const double xr = (A.qp ? zc : 1.0) * xi_of(A, crx, cry);
            double fr, fcr;
            fermi2(xr, invT, fr, fcr);
            const double F = r[7] * fcq * fcr + r[8] * fqv * fr;
            const double W = za * zb * zc * (2.0 * vab * vab - vab * A.V[((size_t)j * N + a) * N + c]);
            const double E = xq + xr - r[6];
            const double d0 = xij - E, dp = d0 + 2.0 * A.T, dm = d0 - 2.0 * A.T;
            acc += r[9] * wq * W * F * (eta2 - dp * dm) / ((dp * dp + eta2) * (dm * dm + eta2));
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((tid & 31) == 0) atomicAdd(&slope[j], acc);
}

__global__ void finish_kernel(const double *slope, double *Zout, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) Zout[j] = 1.0 / (1.0 - slope[j]);
}

// Device address of g_slope, looked up once per device (with that device
// current) and cached; 0 when the lookup failed.
std::mutex g_mu;
double *g_addr[64];
bool g_done[64];

double *scratch_for_current_device(cudaError_t *err)
{
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_done[dev]) {
        void *p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_slope);
        if (*err != cudaSuccess) return nullptr;
        g_addr[dev] = static_cast<double *>(p);
        g_done[dev] = true;
    }
    return g_addr[dev];
}

}  // namespace zstatic
}  // namespace qpfrg

extern "C" qpfrg_status qpfrg_zfactor_static(const qpfrg_lattice *lattice, int n_p, int n_fine, int grid_mode,
                                             int propagator, const double *d_fine, const double *d_kf,
                                             const double *d_V, const double *d_Z, double T, double eta,
                                             void *cuda_stream, double *d_Z_out)
{
    using namespace qpfrg;
    if (!lattice || !d_fine || !d_kf || !d_V || !d_Z_out) return QPFRG_ERR_INVALID;
    if (n_p < 1 || n_p > QPFRG_STATIC_MAX_PATCHES) return QPFRG_ERR_INVALID;   // static scratch limit
    if (n_fine < n_p || n_fine % n_p != 0 || !(T > 0.0) || !(eta > 0.0)) return QPFRG_ERR_INVALID;
    if (propagator != QPFRG_PROP_PAPER && propagator != QPFRG_PROP_QP) return QPFRG_ERR_INVALID;
    zstatic::Args A{};
    A.N = n_p;
    A.M = n_fine;
    A.P = n_fine / n_p;
    A.mode = grid_mode;
    if (grid_mode == QPFRG_GRID_LATTICE) {
        const int L = (int)std::llround(std::sqrt((double)n_p));
        if (L * L != n_p || A.P != 1) return QPFRG_ERR_INVALID;
        A.L = L;
    } else if (grid_mode != QPFRG_GRID_WEDGE || n_p % 4 != 0) {
        return QPFRG_ERR_INVALID;
    }
    // the fine-grid limit of qpfrg_create: more points per patch is unsupported
    if (A.P > 2048) return QPFRG_ERR_UNSUPPORTED;
    const size_t smem = 10 * (size_t)A.P * sizeof(double);
    A.t = lattice->t;
    A.tp = lattice->tp;
    A.mu = lattice->mu;
    A.T = T;
    A.eta = eta;
    A.qp = propagator == QPFRG_PROP_QP;
    A.fine = d_fine;
    A.kf = d_kf;
    A.V = d_V;
    A.Z = d_Z;
    // an error left pending by earlier, unrelated work is not this call's:
    // report it without launching and without clearing it
    if (cudaPeekAtLastError() != cudaSuccess) return QPFRG_ERR_CUDA;
    cudaError_t e;
    double *slope = zstatic::scratch_for_current_device(&e);
    if (!slope) return QPFRG_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    e = cudaFuncSetAttribute(zstatic::pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return QPFRG_ERR_CUDA;
    zstatic::zero_kernel<<<1, 256, 0, st>>>(slope, n_p);
    if (cudaGetLastError() != cudaSuccess) return QPFRG_ERR_CUDA;
    dim3 grid(div_up(n_fine, 256), n_p, n_p);
    zstatic::pair_kernel<<<grid, 256, smem, st>>>(A, slope);
    if (cudaGetLastError() != cudaSuccess) return QPFRG_ERR_CUDA;
    zstatic::finish_kernel<<<div_up(n_p, 128), 128, 0, st>>>(slope, d_Z_out, n_p);
    return cudaGetLastError() == cudaSuccess ? QPFRG_OK : QPFRG_ERR_CUDA;
}
