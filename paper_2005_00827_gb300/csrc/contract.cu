// Contraction of the bubble tables with two vertices, all output triples.
//
// With B_f[Q][a][b] from bubble.cu (a = patch of the loop point p, b = patch of
// its partner), the three channels of the one-loop flow (App. A.1,
// Eq. (vertex_flow_general)) become, for k = (a, b) in N^2:
//   pp (Q = k1+k2 = (i,j)):  dV[i,j,l] -= sum_k B_pp[i,j][k] V[i,j,a] * V[a,b,l]
//   cr (Q = k3-k2 = (l,j)):  dV[i,j,l] -= sum_k B_ph[l,j][k] V[b,j,l] * V[i,a,b]
//   d  (Q = k1-k3 = (i,l)):  dV[i,j,l] += sum_k B_ph[i,l][k] {(2V[i,a,l] - V[a,i,l]) V[b,j,a]
//                                                          - V[i,a,l] V[j,b,a]}
// Each channel is a GEMM with N^2 rows r, K = N^2 (2N^2 for d) and N
// columns n, whose A operand is a row of a bubble table times a vertex
// factor (formed while staging into shared memory) and whose B operand is a
// permuted view of V:
//   pp: r = (i,j), n = l;  cr: r = (j,l), n = i;  d: r = (i,l), n = j.
// Output: out[index(r,n)] += scale * sign * sum.
#include <algorithm>

#include "qpfrg_internal.h"

namespace qpfrg {

constexpr int BM = 64, BN = 32, BK = 16, TM = 4, TN = 2;

template <typename R, typename VR, int CH>
struct ChannelOps {
    const R *B;      // bubble table family (pp or ph), [Q][a][b]
    const VR *V;     // vertex (FP64 or FP32)
    int N;
    long NN;

    // A operand: row r, reduction index k (k >= NN: second product of d)
    __device__ __forceinline__ R a_elem(int r, long k) const
    {
        if (CH == 0) {                         // pp: r = i*N + j
            const int a = (int)(k / N);
            return B[(long)r * NN + k] * (R)V[(long)r * N + a];
        } else if (CH == 1) {                  // cr: r = j*N + l, table row Q = (l, j)
            const int j = r / N, l = r % N;
            const int a = (int)(k / N), b = (int)(k % N);
            (void)a;
            return B[((long)l * N + j) * NN + k] * (R)V[((long)b * N + j) * N + l];
        } else {                               // d: r = i*N + l
            const int i = r / N, l = r % N;
            const bool second = k >= NN;
            const long kk = second ? k - NN : k;
            const int a = (int)(kk / N);
            const R bt = B[(long)r * NN + kk];
            const R v_ial = (R)V[((long)i * N + a) * N + l];
            if (!second) return bt * (R(2) * v_ial - (R)V[((long)a * N + i) * N + l]);
            return -bt * v_ial;
        }
    }
    // B operand: reduction index k, column n
    __device__ __forceinline__ R b_elem(long k, int n) const
    {
        if (CH == 0) return (R)V[k * N + n];                  // V[a,b,l]
        if (CH == 1) return (R)V[(long)n * NN + k];           // V[i,a,b]
        const bool second = k >= NN;
        const long kk = second ? k - NN : k;
        const int a = (int)(kk / N), b = (int)(kk % N);
        if (!second) return (R)V[((long)b * N + n) * N + a];  // V[b,j,a]
        return (R)V[((long)n * N + b) * N + a];               // V[j,b,a]
    }
    __device__ __forceinline__ long out_index(int r, int n) const
    {
        if (CH == 0) return (long)r * N + n;                  // (i,j,l) = (r, n)
        if (CH == 1) return (long)n * NN + r;                 // i = n, (j,l) = r
        const int i = r / N, l = r % N;
        return ((long)i * N + n) * N + l;                     // j = n
    }
};

template <typename R, typename VR, int CH>
__global__ void __launch_bounds__(256) contract_kernel(ChannelOps<R, VR, CH> ops, double *out,
                                                       double scale, double sign)
{
    const int N = ops.N;
    const long NN = ops.NN;
    const long K = CH == 2 ? 2 * NN : NN;
    const int r0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x;
    const int tr = tid / (BN / TN), tn = tid % (BN / TN);   // 16 x 16 thread grid

    __shared__ R As[BK][BM + 1];
    __shared__ R Bs[BK][BN + 1];
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = R(0);

    for (long k0 = 0; k0 < K; k0 += BK) {
        // stage A: BM x BK, 4 elements per thread
#pragma unroll
        for (int e = 0; e < (BM * BK) / 256; ++e) {
            const int idx = tid + e * 256;
            const int rr = idx / BK, kk = idx % BK;
            const int r = r0 + rr;
            const long k = k0 + kk;
            As[kk][rr] = (r < NN && k < K) ? ops.a_elem(r, k) : R(0);
        }
        // stage B: BK x BN, 2 elements per thread
#pragma unroll
        for (int e = 0; e < (BK * BN) / 256; ++e) {
            const int idx = tid + e * 256;
            const int kk = idx / BN, nn = idx % BN;
            const int n = n0 + nn;
            const long k = k0 + kk;
            Bs[kk][nn] = (n < N && k < K) ? ops.b_elem(k, n) : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            R av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][tr * TM + i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tn * TN + j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
    const double s = scale * sign;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = r0 + tr * TM + i;
        if (r >= NN) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tn * TN + j;
            if (n >= N) continue;
            const long o = ops.out_index(r, n);
            out[o] += s * (double)acc[i][j];
        }
    }
}

template <typename R, typename VR, int CH>
static qpfrg_status launch_channel(qpfrg_ctx *c, const R *B, const VR *V, double scale, double sign,
                                   double *out, int kid)
{
    ChannelOps<R, VR, CH> ops;
    ops.B = B;
    ops.V = V;
    ops.N = c->pb.N;
    ops.NN = (long)c->pb.N * c->pb.N;
    dim3 grid(div_up(ops.NN, BM), div_up(c->pb.N, BN));
    prof_begin(c);
    contract_kernel<R, VR, CH><<<grid, 256, 0, c->stream>>>(ops, out, scale, sign);
    prof_end(c, kid);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "contract_kernel");
}

template <typename R, typename VR>
static qpfrg_status launch_all(qpfrg_ctx *c, const VR *V, double scale, double *out)
{
    const R *B = reinterpret_cast<const R *>(c->d_B);
    const long table = (long)c->pb.N * c->pb.N * c->pb.N * c->pb.N;
    const R *Bpp = B, *Bph = B + table;
    const unsigned ch = c->pb.channels;
    qpfrg_status s = QPFRG_OK;
    if ((ch & QPFRG_CH_PP) && (s = launch_channel<R, VR, 0>(c, Bpp, V, scale, -1.0, out, K_CONTRACT_PP)))
        return s;
    if ((ch & QPFRG_CH_CR) && (s = launch_channel<R, VR, 1>(c, Bph, V, scale, -1.0, out, K_CONTRACT_CR)))
        return s;
    if ((ch & QPFRG_CH_D) && (s = launch_channel<R, VR, 2>(c, Bph, V, scale, 1.0, out, K_CONTRACT_D)))
        return s;
    return QPFRG_OK;
}

// C4v element g on patch j (wedge part, ns shells per wedge, Na wedges)
__device__ __forceinline__ int c4v_patch(int g, int j, int ns, int Na)
{
    const int w = ns == 1 ? j : j / ns, sh = j - w * ns;
    const int off = (g & 3) * (Na >> 2);
    int r = (g & 4) ? off - w : w + off;      // in (-Na, 2 Na)
    r = r >= Na ? r - Na : (r < 0 ? r + Na : r);
    return r * ns + sh;
}

// Expansion of the representative rows (row orbits, symmetry.cu): with a
// C4v-symmetric state each channel's output is invariant, out(g t) = out(t),
// so row Q = g rep of a channel at column n is the representative's row at
// column g^-1 n.  One thread per output triple (k1, k2, k3) adds the three
// channels' values: pp row (k1, k2) column k3, cr row (k3, k2) column k1,
// d row (k1, k3) column k2 (the row/column roles of the channel GEMMs above).
// Row (k1, k2) of out, threads over k3.
__device__ __forceinline__ void expand_row(const double *__restrict__ outc, const int *__restrict__ rowmap, int nr,
                                           int N, int ns, unsigned channels, double *__restrict__ out, int k1, int k2)
{
    const int Na = N / ns;
    const long ch_stride = (long)nr * N;
    double *row = out + ((long)k1 * N + k2) * N;
    const int e_pp = __ldg(rowmap + k1 * N + k2);
    for (int k3 = threadIdx.x; k3 < N; k3 += blockDim.x) {
        double v = 0.0;
        auto take = [&](int ch, int e, int n) {
            const int m = e & 0xffffff, gi = c4v_inverse(e >> 24);
            v += __ldg(outc + ch * ch_stride + (long)m * N + c4v_patch(gi, n, ns, Na));
        };
        if (channels & QPFRG_CH_PP) take(0, e_pp, k3);
        if (channels & QPFRG_CH_CR) take(1, __ldg(rowmap + k3 * N + k2), k1);
        if (channels & QPFRG_CH_D) take(2, __ldg(rowmap + k1 * N + k3), k2);
        row[k3] += v;
    }
}

// Block (k2, k1), thread k3.
__global__ void rows_expand_kernel(const double *__restrict__ outc, const int *__restrict__ rowmap, int nr, int N,
                                   int ns, unsigned channels, double *__restrict__ out)
{
    expand_row(outc, rowmap, nr, N, ns, channels, out, blockIdx.y, blockIdx.x);
}

// Batched flows: grid.z = flow; flows that are not running or have no step
// at this row of the schedule return at once.
__global__ void rows_expand_batch_kernel(TcBatch bt, const int *__restrict__ rowmap, int nr, int N, int ns,
                                         unsigned channels)
{
    const int f = blockIdx.z;
    if (bt.status[f] != QPFRG_FLOW_RUNNING || bt.h_tab[(long)bt.step * bt.nflows + f] == 0.0) return;
    expand_row(bt.outc[f], rowmap, nr, N, ns, channels, bt.out[f], blockIdx.y, blockIdx.x);
}

qpfrg_status launch_rows_expand_batch(qpfrg_ctx *c, const TcBatch &bt)
{
    const int N = c->pb.N, thr = std::min(256, (N + 31) / 32 * 32);
    prof_begin(c);
    rows_expand_batch_kernel<<<dim3(N, N, bt.nflows), thr, 0, c->stream>>>(bt, c->d_rowmap, c->n_rrep, N,
                                                                           c->pb.n_shell, c->pb.channels);
    prof_end(c, K_ROWS_EXPAND);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "rows_expand_batch_kernel");
}

qpfrg_status launch_contractions(qpfrg_ctx *c, const void *d_Vin, double scale, double *d_out)
{
    if (c->opt.precision == QPFRG_MIXED_TC) {
        // the weighted tables of this stage, formed into A tiles inside the contraction
        const unsigned ch = c->pb.channels;
        qpfrg_status s = QPFRG_OK;
        // representative rows only (row orbits): into the compact rows, then expanded
        double *dst[3] = {d_out, d_out, d_out};
        if (c->rows_compact) {
            const long per = (long)c->n_rrep * c->pb.N;
            cudaError_t e = cudaMemsetAsync(c->d_outc, 0, 3 * per * sizeof(double), c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "memset representative rows");
            for (int k = 0; k < 3; ++k) dst[k] = c->d_outc + k * per;
        }
        if ((ch & QPFRG_CH_PP) && (s = launch_tc_fused(c, 0, -scale, dst[0], K_TC_PP))) return s;
        if ((ch & QPFRG_CH_CR) && (s = launch_tc_fused(c, 1, -scale, dst[1], K_TC_CR))) return s;
        if ((ch & QPFRG_CH_D) && (s = launch_tc_fused(c, 2, scale, dst[2], K_TC_D))) return s;
        if (c->rows_compact) {
            const int N = c->pb.N, thr = std::min(256, (N + 31) / 32 * 32);
            prof_begin(c);
            rows_expand_kernel<<<dim3(N, N), thr, 0, c->stream>>>(c->d_outc, c->d_rowmap, c->n_rrep, N,
                                                                  c->pb.n_shell, ch, d_out);
            prof_end(c, K_ROWS_EXPAND);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(c, e, "rows_expand_kernel");
        }
        return QPFRG_OK;
    }
    if (c->opt.precision == QPFRG_FP64)
        return launch_all<double, double>(c, reinterpret_cast<const double *>(d_Vin), scale, d_out);
    return launch_all<float, float>(c, reinterpret_cast<const float *>(d_Vin), scale, d_out);
}

}  // namespace qpfrg
