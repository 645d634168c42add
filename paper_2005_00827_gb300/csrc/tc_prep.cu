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

__device__ __forceinline__ void tc_prep_body(const TcPrepArgs &t)
{
    const int N = t.N, Npad = t.Npad;
    const long NN = (long)N * N, n3 = NN * N, Kp = t.Kp;
    const long s_pp = (long)Npad * Kp, s_d = 2 * s_pp;
    const long total = 2 * s_pp + s_d + 3 * n3;
    const float *V = t.V;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        if (idx < 2 * s_pp + s_d) {
            int which;
            long loc;
            if (idx < s_pp) { which = 0; loc = idx; }
            else if (idx < 2 * s_pp) { which = 1; loc = idx - s_pp; }
            else { which = 2; loc = idx - 2 * s_pp; }
            const long K = which == 2 ? 2 * Kp : Kp;
            const int n = (int)(loc / K);
            const long k = loc - (long)n * K;
            const bool second = k >= Kp;
            const long kk = second ? k - Kp : k;
            float v = 0.f;
            if (n < N && kk < NN) {
                const int a = (int)(kk / N), b = (int)(kk - (long)a * N);
                if (which == 0) v = V[kk * N + n];
                else if (which == 1) v = V[(long)n * NN + kk];
                else if (!second) v = V[((long)b * N + n) * N + a];
                else v = V[((long)n * N + b) * N + a];
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            __nv_bfloat16 *const *dst = which == 0 ? t.Bpp : (which == 1 ? t.Bcr : t.Bd);
            const long o = tile_index(n, k, Npad, which == 2 ? t.Kpd : t.Kp);
            dst[0][o] = hi;
            dst[1][o] = lo;
        } else {
            const long o = idx - (2 * s_pp + s_d);
            const int part = (int)(o / n3);
            const long r = o - part * n3;             // Q N + x
            const int x = (int)(r % N), Q = (int)(r / N), q1 = Q / N, q2 = Q - q1 * N;
            float v;
            if (part == 0) v = V[((long)x * N + q2) * N + q1];                         // Q = (l,j): V[b,j,l]
            else if (part == 1) v = 2.f * V[((long)q1 * N + x) * N + q2] - V[((long)x * N + q1) * N + q2];
            else v = -V[((long)q1 * N + x) * N + q2];                                 // Q = (i,l): -V[i,a,l]
            t.VT[o] = v;
        }
    }
}

__global__ void tc_prep_kernel(TcPrepArgs t) { tc_prep_body(t); }

// Batched flows: grid.y = flow; flows that are not running or have no step at
// this row of the schedule return at once.
__global__ void tc_prep_batch_kernel(TcPrepArgs t, const TcPrepFlow *flows, const int *status, const double *h_tab,
                                     int step, int nflows)
{
    const int f = blockIdx.y;
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
    const long total = 4 * (long)c->tc.Npad * c->tc.Kp + 3 * NN * N;
    const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 4);
    TcPrepArgs t{};
    t.N = N;
    t.Npad = c->tc.Npad;
    t.Kp = c->tc.Kp;
    t.Kpd = c->tc.Kpd;
    prof_begin(c);
    tc_prep_batch_kernel<<<dim3(blocks, nflows), 256, 0, c->stream>>>(t, d_flows, d_status, d_h_tab, step, nflows);
    prof_end(c, K_TC_PREP);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_prep_batch_kernel");
}

qpfrg_status launch_tc_prep(qpfrg_ctx *c)
{
    const int N = c->pb.N;
    const long NN = (long)N * N;
    const long total = 4 * (long)c->tc.Npad * c->tc.Kp + 3 * NN * N;
    int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
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
    tc_prep_kernel<<<blocks, 256, 0, c->stream>>>(t);
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
