// Per-stage vertex operands of the tensor-core contraction (QPFRG_MIXED_TC):
// the B operands of the three channel GEMMs (permuted views of the FP32 stage
// vertex, split into BF16 hi/lo and stored in tensor-core tiles that the
// contraction loads with TMA) and V^T for the crossed channel's row factors;
// plus the TMA maps of those tiles (encoded once per context).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "qpfrg_internal.h"

namespace qpfrg {

// Per-stage B operands of the three channel GEMMs from the FP32 stage vertex,
// rows n (n >= N zero) by reduction index k = (a, b) = a N + b, split into
// BF16 hi/lo and stored in tiles (tile_index, Npad rows per tile):
// pp: V[a,b,n];  cr: V[n,a,b];  d: V[b,n,a] at k and V[n,b,a] at Kp + k, so
// that each half of the d reduction starts on a 64-wide block;  pads (n >= N,
// k >= N^2 within a half) are written as zeros;  plus the row-factor tables
// of the A operands, rows in transfer order: VT[0][Q = (l,j)][b] = V[b,j,l]
// (cr), VT[1][Q = (i,l)][a] = 2 V[i,a,l] - V[a,i,l] and VT[2][Q][a] =
// -V[i,a,l] (the two halves of d).
struct TcPrepArgs {
    const float *V;
    int N, Npad;
    long Kp, Kpd;
    __nv_bfloat16 *Bpp[2], *Bcr[2], *Bd[2];
    float *VT;
};

// Job blockIdx.y: 0, 1, 2 the pp, cr, d operands, one thread per row n and
// 8 consecutive k (one 16-byte chunk of hi and of lo in the tile layout;
// neighbouring threads take neighbouring rows, so the pp reads are coalesced);
// 3, 4, 5 the three factor tables, one element per thread.  32-bit indices:
// N <= 256 keeps N^3 and Npad K_pd below 2^31.
__device__ __forceinline__ void tc_prep_body(const TcPrepArgs &t)
{
    const int N = t.N, Npad = t.Npad, job = blockIdx.y;
    const int NN = N * N, Kp = (int)t.Kp;
    const float *V = t.V;
    const int stride = gridDim.x * blockDim.x;
    const int g0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (job < 3) {
        const int K = job == 2 ? 2 * Kp : Kp;
        const int total = Npad * (K / 8);
        __nv_bfloat16 *const dhi = job == 0 ? t.Bpp[0] : (job == 1 ? t.Bcr[0] : t.Bd[0]);
        __nv_bfloat16 *const dlo = job == 0 ? t.Bpp[1] : (job == 1 ? t.Bcr[1] : t.Bd[1]);
        for (int g = g0; g < total; g += stride) {
            const int n = g % Npad, k0 = (g / Npad) * 8;
            const bool second = k0 >= Kp;
            const int kk0 = second ? k0 - Kp : k0;
            int a = kk0 / N, b = kk0 - a * N;
            uint4 hi, lo;
            uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                float x[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    float v = 0.f;
                    if (n < N && kk0 + e + u < NN) {
                        if (job == 0) v = V[(kk0 + e + u) * N + n];
                        else if (job == 1) v = V[n * NN + kk0 + e + u];
                        else if (!second) v = V[(b * N + n) * N + a];
                        else v = V[(n * N + b) * N + a];
                    }
                    x[u] = v;
                    if (++b == N) {
                        b = 0;
                        ++a;
                    }
                }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[0], x[1]);
                const __nv_bfloat162 l2 = __floats2bfloat162_rn(x[0] - __low2float(h2), x[1] - __high2float(h2));
                hp[e / 2] = *reinterpret_cast<const uint32_t *>(&h2);
                lp[e / 2] = *reinterpret_cast<const uint32_t *>(&l2);
            }
            // k0 % 8 == 0: the chunk's 8 elements are contiguous in the tile (16-byte aligned)
            const long o = tile_index(n, k0, Npad, K);
            *reinterpret_cast<uint4 *>(dhi + o) = hi;
            *reinterpret_cast<uint4 *>(dlo + o) = lo;
        }
    } else {
        const int part = job - 3, n3 = NN * N;
        float *VT = t.VT + (long)part * n3;
        for (int o = g0; o < n3; o += stride) {
            const int x = o % N, Q = o / N, q1 = Q / N, q2 = Q - q1 * N;
            float v;
            if (part == 0) v = V[(x * N + q2) * N + q1];                                  // Q = (l,j): V[b,j,l]
            else if (part == 1) v = 2.f * V[(q1 * N + x) * N + q2] - V[(x * N + q1) * N + q2];
            else v = -V[(q1 * N + x) * N + q2];                                         // Q = (i,l): -V[i,a,l]
            VT[o] = v;
        }
    }
}

__global__ void tc_prep_kernel(TcPrepArgs t) { tc_prep_body(t); }

// Batched flows: grid.y = flow; flows that are not running or have no step at
// this row of the schedule return at once.
__global__ void tc_prep_batch_kernel(TcPrepArgs t, const TcPrepFlow *flows, const int *status, const double *h_tab,
                                     int step, int nflows)
{
    const int f = blockIdx.z;
    if (status[f] != QPFRG_FLOW_RUNNING || h_tab[(long)step * nflows + f] == 0.0) return;
    const TcPrepFlow &p = flows[f];
    t.V = p.Vf;
    t.VT = p.VT;
    for (int h = 0; h < 2; ++h) {
        t.Bpp[h] = p.B[0][h];
        t.Bcr[h] = p.B[1][h];
        t.Bd[h] = p.B[2][h];
    }
    tc_prep_body(t);
}

qpfrg_status launch_tc_prep_batch(qpfrg_ctx *c, const TcPrepFlow *d_flows, const int *d_status, const double *d_h_tab,
                                  int step, int nflows)
{
    const int N = c->pb.N;
    const long NN = (long)N * N;
    const long total = std::max((long)c->tc.Npad * c->tc.Kp / 4, NN * N);   // the largest job
    const int blocks = (int)std::min<long>((total + 255) / 256, 152L);
    TcPrepArgs t{};
    t.N = N;
    t.Npad = c->tc.Npad;
    t.Kp = c->tc.Kp;
    t.Kpd = c->tc.Kpd;
    prof_begin(c);
    tc_prep_batch_kernel<<<dim3(blocks, 6, nflows), 256, 0, c->stream>>>(t, d_flows, d_status, d_h_tab, step, nflows);
    prof_end(c, K_TC_PREP);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_prep_batch_kernel");
}

qpfrg_status launch_tc_prep(qpfrg_ctx *c)
{
    const int N = c->pb.N;
    const long NN = (long)N * N;
    const long total = std::max((long)c->tc.Npad * c->tc.Kp / 4, NN * N);   // the largest job
    const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 4);
    TcPrepArgs t;
    t.V = c->d_Vf;
    t.N = N;
    t.Npad = c->tc.Npad;
    t.Kp = c->tc.Kp;
    t.Kpd = c->tc.Kpd;
    for (int h = 0; h < 2; ++h) {
        t.Bpp[h] = c->tc.Bpp[h];
        t.Bcr[h] = c->tc.Bcr[h];
        t.Bd[h] = c->tc.Bd[h];
    }
    t.VT = c->tc.VT;
    prof_begin(c);
    tc_prep_kernel<<<dim3(blocks, 6), 256, 0, c->stream>>>(t);
    prof_end(c, K_TC_PREP);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_prep_kernel");
}

// 2-D TMA map over a tiled BF16 buffer of `elems` elements viewed as rows of
// 128 elements (256 B): boxes of 128 x box_rows elements are whole tiles.
// The driver's tensor-map encoder, looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 map_encoder(qpfrg_ctx *c)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            c->err = "cuTensorMapEncodeTiled is not available";
            return nullptr;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}

qpfrg_status make_table_map(qpfrg_ctx *c, CUtensorMap *map, const float *table)
{
    const auto encode = map_encoder(c);
    if (!encode) return QPFRG_ERR_CUDA;
    // the tiled table as rows of 32 floats: 2 families x RT x KB x 2 halves x 128
    const cuuint64_t rows = 2ull * (cuuint64_t)c->tc.RT * (cuuint64_t)c->tc.KB * 256ull;
    const cuuint64_t dims[2] = {32, rows};
    const cuuint64_t strides[1] = {32 * sizeof(float)};
    const cuuint32_t box[2] = {32, 128};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(table), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->err = "cuTensorMapEncodeTiled failed for the loop-kernel table";
        return QPFRG_ERR_CUDA;
    }
    return QPFRG_OK;
}

qpfrg_status make_tile_map(qpfrg_ctx *c, CUtensorMap *map, const void *base, long elems, int box_rows)
{
    const auto encode = map_encoder(c);
    if (!encode) return QPFRG_ERR_CUDA;
    const cuuint64_t dims[2] = {128, (cuuint64_t)(elems / 128)};
    const cuuint64_t strides[1] = {256};
    const cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->err = "cuTensorMapEncodeTiled failed for a tensor-core operand";
        return QPFRG_ERR_CUDA;
    }
    return QPFRG_OK;
}

qpfrg_status tc_make_maps(qpfrg_ctx *c)
{
    TcBuffers &t = c->tc;
    const long nb = (long)t.Npad * t.Kp, nbd = (long)t.Npad * t.Kpd;
    qpfrg_status s = QPFRG_OK;
    for (int h = 0; h < 2 && s == QPFRG_OK; ++h) {
        if ((s = make_tile_map(c, &t.tmB[0][h], t.Bpp[h], nb, t.Npad / 2)) ||
            (s = make_tile_map(c, &t.tmB[1][h], t.Bcr[h], nb, t.Npad / 2)))
            break;
        s = make_tile_map(c, &t.tmB[2][h], t.Bd[h], nbd, t.Npad / 2);
    }
    if (s == QPFRG_OK) s = make_table_map(c, &t.tmTab, reinterpret_cast<const float *>(c->d_B));
    return s;
}

}  // namespace qpfrg
