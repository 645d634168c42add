// Tensor-core contraction (5th-generation tensor cores, tcgen05) for the
// mixed-precision path QPFRG_MIXED_TC.
//
//   D[m][n] = sum_k A[m][k] B[n][k],   A = A_hi + A_lo,  B = B_hi + B_lo  (BF16)
//   computed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in
//   tensor memory; the dropped A_lo B_lo term is 2^-16 relative.
//
// A is a formed bubble table (the loop kernels of one channel times the vertex
// factor that depends on the row and the first loop patch), B a permuted view
// of the vertex; see contract.cu for the channel algebra.  One CTA computes
// a 128-row tile for all N columns over a slice of K (split-K, partial sums
// added to the FP64 output with atomics).
//
// Data path per 64-wide k-block: the operands are stored in tensor-core tiles
// (tile_index: 128 x 64 for A, Npad x 64 for B, each in the canonical K-major
// no-swizzle order of the descriptors), so one thread loads a stage with four
// TMA tile copies (cp.async.bulk.tensor, 2-D maps over the tiled buffers)
// signalled on the stage's "full" mbarrier (expect-tx bytes), issues 4 K16
// slices x 3 products of tcgen05.mma (M = 128, N = Npad) and commits them to
// the stage's "empty" mbarrier; the stage of k-block i-1 is refilled with
// k-block i-1+S behind the MMAs of k-block i, a ring of S stages.  Waits are
// bounded: on expiry the CTA raises an error flag, waits (bounded) for the
// copies and MMAs it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "qpfrg_internal.h"

namespace qpfrg {

namespace tc {

constexpr int BM = 128, BK = 64, NTHR = 128;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz: bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading (K-direction core
// matrix) and stride (8-row group) byte offsets, version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;      // descriptor version
    return d;                     // layout type 0 (no swizzle), base offset 0
}

// Instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mbar_init(uint32_t addr, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(addr), "r"(count));
}

// true when the phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(addr, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// 2-D TMA tile copy global -> shared, completion counted on mbar in bytes;
// the inner coordinate x is 0 (16-byte aligned by construction)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc

struct TcGemmArgs {
    int M, Ncol, Npad;                // valid rows, valid columns, padded columns
    int nkb_total, kb_per_split;      // 64-wide k blocks of the (padded) reduction; per CTA along grid.y
    int map_mode, N;                  // output index map: 0 pp, 1 cr, 2 d
    double *out;
    double scale;
    unsigned *err;
};

template <int S>
__global__ void __launch_bounds__(tc::NTHR, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                   const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcGemmArgs A)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full[S], empty[S];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int mt = blockIdx.x, m0 = mt * BM;
    const int kb0 = blockIdx.y * A.kb_per_split;
    const int kb1 = min(A.nkb_total, kb0 + A.kb_per_split);
    const int nkb = kb1 - kb0;
    const int Npad = A.Npad;
    const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)Npad * BK * 2;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t tmem_cols = Npad <= 32 ? 32 : (Npad <= 64 ? 64 : (Npad <= 128 ? 128 : 256));

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(smem_u32(&full[s]), 1);
            tc::mbar_init(smem_u32(&empty[s]), 1);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (tid == 0 && nkb > 0) {
        // k block kb (global index) into stage s: A tile (mt, kb) = 64 rows of
        // the 128-wide 2-D view from row (mt nkb_total + kb) 64; B tile kb =
        // Npad/2 rows from row kb Npad/2
        auto issue = [&](int kb, int s) {
            const uint32_t sb = base + (uint32_t)s * stage_bytes, fb = smem_u32(&full[s]);
            tc::mbar_expect_tx(fb, stage_bytes);
            const int ya = (mt * A.nkb_total + kb) * 64, yb = kb * (Npad / 2);
            tc::tma_load_2d(sb, &mAhi, 0, ya, fb);
            tc::tma_load_2d(sb + a_bytes, &mAlo, 0, ya, fb);
            tc::tma_load_2d(sb + 2 * a_bytes, &mBhi, 0, yb, fb);
            tc::tma_load_2d(sb + 2 * a_bytes + b_bytes, &mBlo, 0, yb, fb);
        };
        const uint32_t idesc = tc::make_idesc(BM, Npad);
        int issued = 0, consumed = 0;   // k blocks copied / multiplied
        for (; issued < S && issued < nkb; ++issued) issue(kb0 + issued, issued);
        bool ok = true;
        for (int i = 0; i < nkb && ok; ++i) {
            const int s = i % S;
            if (!tc::mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((i / S) & 1))) {
                ok = false;
                break;
            }
            const uint32_t sb = base + (uint32_t)s * stage_bytes;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                // K16 slice: core matrices 2ks, 2ks+1 along K
                const uint32_t a_off = (uint32_t)(2 * ks * (BM / 8) * 128);
                const uint32_t b_off = (uint32_t)(2 * ks * (Npad / 8) * 128);
                const uint64_t ahi = tc::make_desc(sb + a_off, (BM / 8) * 128, 128);
                const uint64_t alo = tc::make_desc(sb + a_bytes + a_off, (BM / 8) * 128, 128);
                const uint64_t bhi = tc::make_desc(sb + 2 * a_bytes + b_off, (Npad / 8) * 128, 128);
                const uint64_t blo = tc::make_desc(sb + 2 * a_bytes + b_bytes + b_off, (Npad / 8) * 128, 128);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                tc::mma_bf16(tmem, ahi, bhi, idesc, acc);
                tc::mma_bf16(tmem, ahi, blo, idesc, 1u);
                tc::mma_bf16(tmem, alo, bhi, idesc, 1u);
            }
            tc::mma_commit(smem_u32(&empty[s]));
            consumed = i + 1;
            // refill the stage of k block i-1 once its products are done (the
            // products of k block i are already queued behind them)
            if (i >= 1 && issued < nkb) {
                const int j = i - 1;
                if (!tc::mbar_wait_bounded(smem_u32(&empty[j % S]), (uint32_t)((j / S) & 1))) {
                    ok = false;
                    break;
                }
                issue(kb0 + issued, issued % S);
                ++issued;
            }
        }
        if (ok) {
            // all products done before the accumulators are read
            const int last = nkb - 1;
            ok = tc::mbar_wait_bounded(smem_u32(&empty[last % S]), (uint32_t)((last / S) & 1));
        } else {
            // drain: every copy issued lands and every product committed ends
            // (bounded waits) before the CTA frees its memory
            for (int j = consumed; j < issued; ++j)
                tc::mbar_wait_bounded(smem_u32(&full[j % S]), (uint32_t)((j / S) & 1));
            if (consumed > 0)
                tc::mbar_wait_bounded(smem_u32(&empty[(consumed - 1) % S]), (uint32_t)(((consumed - 1) / S) & 1));
        }
        if (!ok) abort_flag = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_flag) {
        if (tid == 0) atomicOr(A.err, 1u);
    } else if (nkb > 0) {
        // epilogue: warp w owns accumulator rows 32w .. 32w+31 (TMEM lanes).
        // The lanes of a pp store add to outputs N apart: spread over many L2
        // slices, which the FP64 atomics need more than contiguity (a
        // transposed, contiguous pp epilogue measured slower)
        const int r = warp * 32 + (tid & 31);
        const int m = m0 + r;
        const int N = A.N;
        const long NN = (long)N * N;
        for (int c0 = 0; c0 < Npad; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (m < A.M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c0 + q;
                    if (n >= A.Ncol) continue;
                    long o;
                    if (A.map_mode == 0) o = (long)m * N + n;
                    else if (A.map_mode == 1) o = (long)n * NN + m;
                    else o = ((long)(m / N) * N + n) * N + (m % N);
                    atomicAdd(&A.out[o], A.scale * (double)v[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
}

// Per-stage B operands of the three channel GEMMs from the FP32 stage vertex,
// rows n (n >= N zero) by reduction index k = (a, b) = a N + b, split into
// BF16 hi/lo and stored in tiles (tile_index, Npad rows per tile):
// pp: V[a,b,n];  cr: V[n,a,b];  d: V[b,n,a] (k < N^2) and V[n,b,a]
// (k >= N^2);  plus VT[j][l][b] = V[b][j][l] for the cr factor.
struct TcPrepArgs {
    const float *V;
    int N, Npad;
    long Kp, Kpd;
    __nv_bfloat16 *Bpp[2], *Bcr[2], *Bd[2];
    float *VT;
};

__global__ void tc_prep_kernel(TcPrepArgs t)
{
    const int N = t.N, Npad = t.Npad;
    const long NN = (long)N * N, n3 = NN * N;
    const long s_pp = (long)Npad * NN, s_d = 2 * s_pp;
    const long total = 2 * s_pp + s_d + n3;
    const float *V = t.V;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        if (idx < 2 * s_pp + s_d) {
            int which;
            long loc;
            if (idx < s_pp) { which = 0; loc = idx; }
            else if (idx < 2 * s_pp) { which = 1; loc = idx - s_pp; }
            else { which = 2; loc = idx - 2 * s_pp; }
            const long K = which == 2 ? 2 * NN : NN;
            const int n = (int)(loc / K);
            const long k = loc - (long)n * K;
            float v = 0.f;
            if (n < N) {
                const long kk = k >= NN ? k - NN : k;
                const int a = (int)(kk / N), b = (int)(kk - (long)a * N);
                if (which == 0) v = V[kk * N + n];
                else if (which == 1) v = V[(long)n * NN + kk];
                else if (k < NN) v = V[((long)b * N + n) * N + a];
                else v = V[((long)n * N + b) * N + a];
            }
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
            __nv_bfloat16 *const *dst = which == 0 ? t.Bpp : (which == 1 ? t.Bcr : t.Bd);
            const long o = tile_index(n, k, Npad, which == 2 ? t.Kpd : t.Kp);
            dst[0][o] = hi;
            dst[1][o] = lo;
        } else {
            const long o = idx - (2 * s_pp + s_d);     // o = (j N + l) N + b
            const int b = (int)(o % N), jl = (int)(o / N);
            t.VT[o] = V[(long)b * NN + jl];
        }
    }
}

qpfrg_status launch_tc_prep(qpfrg_ctx *c)
{
    const int N = c->pb.N;
    const long NN = (long)N * N;
    const long total = 4 * (long)c->tc.Npad * NN + NN * N;
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
static qpfrg_status make_tile_map(qpfrg_ctx *c, CUtensorMap *map, const void *base, long elems, int box_rows)
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
            return QPFRG_ERR_CUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
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
    const long na = t.Mp * t.Kp, nad = t.Mp * t.Kpd, nb = (long)t.Npad * t.Kp, nbd = (long)t.Npad * t.Kpd;
    qpfrg_status s = QPFRG_OK;
    for (int h = 0; h < 2 && s == QPFRG_OK; ++h) {
        if ((s = make_tile_map(c, &t.tmA[0][h], t.App[h], na, 64)) ||
            (s = make_tile_map(c, &t.tmA[1][h], t.Acr[h], na, 64)) ||
            (s = make_tile_map(c, &t.tmA[2][h], t.Ad[h], nad, 64)) ||
            (s = make_tile_map(c, &t.tmB[0][h], t.Bpp[h], nb, t.Npad / 2)) ||
            (s = make_tile_map(c, &t.tmB[1][h], t.Bcr[h], nb, t.Npad / 2)))
            break;
        s = make_tile_map(c, &t.tmB[2][h], t.Bd[h], nbd, t.Npad / 2);
    }
    return s;
}

// Host launcher of channel ch (0 pp, 1 cr, 2 d): D += scale * A B^T over the
// tiled operands, M valid rows, K valid reduction length.
qpfrg_status launch_tc_gemm(qpfrg_ctx *c, int ch, int M, double scale, double *out, int kid)
{
    const TcBuffers &t = c->tc;
    const int Npad = t.Npad;
    const long Kp = ch == 2 ? t.Kpd : t.Kp;
    // stage ring: as many stages of A and B tiles as fit (at most 4)
    const size_t stage_bytes = 2 * (size_t)tc::BM * tc::BK * 2 + 2 * (size_t)Npad * tc::BK * 2;
    const size_t smem_max = 226 * 1024;       // leaves room for the static barriers (1 KB aligned)
    int S = (int)std::min<size_t>(4, smem_max / stage_bytes);
    if (Npad % 16 != 0 || Npad > 256 || S < 2) {
        c->err = "tensor-core contraction: unsupported shape";
        return QPFRG_ERR_UNSUPPORTED;
    }
    const size_t smem = S * stage_bytes;
    auto kern = S == 4 ? tc_gemm_kernel<4> : (S == 3 ? tc_gemm_kernel<3> : tc_gemm_kernel<2>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_gemm smem attribute");
    const int mtiles = div_up(M, tc::BM);
    const int nkb = (int)(Kp / tc::BK);
    // split K so that the grid fills whole waves of the 152 SMs (one CTA per
    // SM): the split count whose waves are fullest, at least 4 k-blocks each
    int splits = 1;
    double best = -1.0;
    for (int sp = 1; sp <= std::max(1, nkb / 4) && sp <= 16; ++sp) {
        const int ctas = mtiles * sp;
        const double waves = (double)ctas / 152.0, fill = waves / std::ceil(waves);
        const double score = fill - 0.02 * std::ceil(waves);   // prefer fewer waves at equal fill
        if (score > best + 1e-9) {
            best = score;
            splits = sp;
        }
    }
    if (c->tune.tc_splits[ch] > 0) splits = std::min(c->tune.tc_splits[ch], nkb);
    const int kb_per = div_up(nkb, splits);
    splits = div_up(nkb, kb_per);
    TcGemmArgs A{M, c->pb.N, Npad, nkb, kb_per, ch, c->pb.N, out, scale, c->d_tc_err};
    prof_begin(c);
    kern<<<dim3(mtiles, splits), tc::NTHR, smem, c->stream>>>(t.tmA[ch][0], t.tmA[ch][1], t.tmB[ch][0],
                                                            t.tmB[ch][1], A);
    prof_end(c, kid);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_gemm_kernel");
}

}  // namespace qpfrg
