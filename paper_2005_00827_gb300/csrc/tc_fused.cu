// Tensor-core contraction with the A operand formed in shared memory
// (QPFRG_MIXED_TC).
//
//   D[m][n] = sum_k A[m][k] B[n][k],  A = A_hi + A_lo,  B = B_hi + B_lo (BF16),
//   computed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in
//   tensor memory (the dropped A_lo B_lo term is 2^-16 relative).
//
// A row m of channel ch is a row of the weighted loop-kernel table (bubble.cu:
// the loop kernels binned by partner patch, times the line weights) times the
// vertex factor of (row, first loop patch) -- the channel algebra of
// contract.cu:
//   pp: m = (i,j), Q = (i,j), A[m][(a,b)] = B_pp[Q][a][b] V[i,j,a]
//   cr: m = (j,l), Q = (l,j), A[m][(a,b)] = B_ph[Q][a][b] V[b,j,l]
//   d : m = (i,l), Q = (i,l), A[m][(a,b)] = B_ph[Q][a][b] (2V[i,a,l] - V[a,i,l]),
//                             A[m][N^2 + (a,b)] = -B_ph[Q][a][b] V[i,a,l]
// so a row of A is a contiguous slice of the table (k = a N + b, taken
// modulo N^2 in the d channel) scaled elementwise.
//
// Warp roles (160 threads): warps 0-3 are producers -- they form each 128 x 64
// A block (coalesced reads of the table, BF16 hi/lo split) straight into the
// shared-memory stage in the canonical K-major no-swizzle order,
// makes its writes visible to the tensor cores (fence.proxy.async) and
// arrives on the stage's "full" mbarrier -- and afterwards read the
// accumulators back (tcgen05.ld) and add them to the FP64 output; warp 4 loads
// the B blocks (pre-formed per stage by tc_prep_kernel) with TMA and one of its
// threads issues the MMAs, committing each block to the stage's "empty"
// mbarrier.  A ring of S stages; every wait is bounded by a clock budget and
// aborts the CTA (error flag, bounded drain, tensor memory freed).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>

#include "qpfrg_internal.h"
#include "tc_ptx.h"

namespace qpfrg {

namespace {

constexpr int kProducers = 128;                 // threads forming A (one row each)
constexpr int kFusedThreads = kProducers + 32;  // + the TMA / MMA warp

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// bounded wait that also gives up once another thread of the CTA aborted
__device__ __forceinline__ bool mbar_wait_abortable(uint32_t addr, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(addr, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > tc::kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float x0, float x1)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace

struct TcFusedArgs {
    int M, Ncol, Npad, N;             // valid rows, valid columns, padded columns, patches
    int nkb_total, kb_per_split;      // 64-wide k blocks of the padded reduction; per CTA along grid.y
    int ch;                           // 0 pp, 1 cr, 2 d
    const float *table;               // weighted loop-kernel table [f][Q][a][b] (FP32)
    const float *Vf, *VT;             // stage vertex [k1][k2][k3] and VT[j][l][b] = V[b][j][l]
    double *out;
    double scale;
    unsigned *err;
    TcBatch batch;
    // test of the bounded waits (QPFRG_TEST_TC_WAIT): the MMA thread first
    // waits on a barrier nothing arrives on, with a budget of test_wait cycles
    long long test_wait;
};

template <int S>
__global__ void __launch_bounds__(kFusedThreads, 1)
    tc_fused_kernel(const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, TcFusedArgs A)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t full[S], empty[S], never;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    // the flow of this CTA (batched launch) or the context's single flow
    const float *tab_base = A.table, *Vf = A.Vf, *VT = A.VT;
    double *out = A.out;
    double scale = A.scale;
    const CUtensorMap *mhi = &mBhi, *mlo = &mBlo;
    if (A.batch.nflows) {
        const TcBatch &Bt = A.batch;
        const int f = blockIdx.z;
        const long sf = (long)Bt.step * Bt.nflows + f;
        const double h = Bt.h_tab[sf];
        if (Bt.status[f] != QPFRG_FLOW_RUNNING || h == 0.0) return;   // uniform, before any barrier
        tab_base = Bt.rows[Bt.slot_tab[sf]];
        Vf = Bt.Vf[f];
        VT = Bt.VT[f];
        out = Bt.out[f];
        scale *= exp(Bt.x[f] + Bt.cst * h);      // dV/d ln T = T dV/dT at the stage temperature
        mhi = Bt.maps + 6L * f + 2 * A.ch;
        mlo = mhi + 1;
    }
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * BM;
    const int kb0 = blockIdx.y * A.kb_per_split;
    const int kb1 = min(A.nkb_total, kb0 + A.kb_per_split);
    const int nkb = kb1 - kb0;
    const int Npad = A.Npad, N = A.N;
    const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)Npad * BK * 2;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    const uint32_t base = smem_u32(smem_raw);
    const uint32_t tmem_cols = Npad <= 32 ? 32 : (Npad <= 64 ? 64 : (Npad <= 128 ? 128 : 256));

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), kProducers + 1);   // producers + the B copy's expect-tx arrival
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&never), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    volatile int *abort_v = &abort_flag;

    if (warp < 4) {
        // ---- producers: each warp forms rows 32 w .. 32 w + 31 of every A
        // block in eight rounds of four rows; lane (rg, kc) = (lane / 8, lane % 8)
        // takes row 4 q + rg of round q and the 8-wide k chunk kc.  A row of the
        // channel is a contiguous slice of the weighted table (pp: B_pp[Q]; cr,
        // d: B_ph[Q], k taken modulo N^2), so the eight lanes of a row read 256
        // contiguous bytes as two aligned 16-byte loads each, then scale by the
        // vertex factor and write one 16-byte chunk of hi and of lo.
        const long NN = (long)N * N;
        const int lane = tid & 31, rg = lane >> 3, kc = lane & 7;
        const int ch = A.ch, fam = ch == 0 ? 0 : 1;
        const long Kvalid = ch == 2 ? 2 * NN : NN;
        const bool n8 = (N & 7) == 0;                // a chunk of 8 lies within one a
        bool ok = true;
        for (int it = 0; it < nkb && ok; ++it) {
            const int s = it % S;
            if (it >= S && !mbar_wait_abortable(smem_u32(&empty[s]), (uint32_t)(((it / S) - 1) & 1), abort_v)) {
                ok = false;
                break;
            }
            const long k0 = (long)(kb0 + it) * BK + kc * 8;     // first k of this lane's chunk
            unsigned char *st = smem_raw + (size_t)s * stage_bytes;
#pragma unroll 2
            for (int q = 0; q < 8; ++q) {
                const int rr = warp * 32 + 4 * q + rg;          // row within the block
                const int r = m0 + rr;
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
                if (r < A.M && k0 < Kvalid) {                    // N^2 % 8 == 0: a chunk never crosses Kvalid
                    int Qr, ri = 0, rl = 0;
                    if (ch == 0) {
                        Qr = r;
                    } else if (ch == 1) {
                        const int j = r / N, l = r - j * N;
                        Qr = l * N + j;
                    } else {
                        ri = r / N;
                        rl = r - ri * N;
                        Qr = r;
                    }
                    const bool second = ch == 2 && k0 >= NN;
                    const int kk = (int)(second ? k0 - NN : k0);
                    const float4 *src = reinterpret_cast<const float4 *>(tab_base + ((long)fam * NN + Qr) * NN + kk);
                    const float4 t0 = __ldg(src), t1 = __ldg(src + 1);
                    const float t[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
                    int a = kk / N, b = kk - a * N;
                    if (n8) {
                        if (ch == 1) {
                            // V[b][j][l] = VT[(j N + l) N + b] for b .. b+7 (aligned)
                            const float4 *vt = reinterpret_cast<const float4 *>(VT + (long)r * N + b);
                            const float4 c0 = __ldg(vt), c1 = __ldg(vt + 1);
                            const float c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[e] = t[e] * c[e];
                        } else {
                            float fac;
                            if (ch == 0) {
                                fac = __ldg(Vf + (long)Qr * N + a);
                            } else {
                                const float v_ial = __ldg(Vf + ((long)ri * N + a) * N + rl);
                                fac = second ? -v_ial : 2.f * v_ial - __ldg(Vf + ((long)a * N + ri) * N + rl);
                            }
#pragma unroll
                            for (int e = 0; e < 8; ++e) v[e] = t[e] * fac;
                        }
                    } else {
                        // N not a multiple of 8: the chunk may cross to the next a
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            float fac;
                            if (ch == 0) {
                                fac = __ldg(Vf + (long)Qr * N + a);
                            } else if (ch == 1) {
                                fac = __ldg(VT + (long)r * N + b);
                            } else {
                                const float v_ial = __ldg(Vf + ((long)ri * N + a) * N + rl);
                                fac = second ? -v_ial : 2.f * v_ial - __ldg(Vf + ((long)a * N + ri) * N + rl);
                            }
                            v[e] = t[e] * fac;
                            if (++b == N) {
                                b = 0;
                                ++a;
                            }
                        }
                    }
                }
                uint4 hi, lo;
                uint32_t *h = &hi.x, *l = &lo.x;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * qq], v[2 * qq + 1]);
                    h[qq] = *reinterpret_cast<const uint32_t *>(&hh);
                    l[qq] = pack_bf16x2(v[2 * qq] - __low2float(hh), v[2 * qq + 1] - __high2float(hh));
                }
                // core matrix (kc, row group) at ((kc (BM/8) + rr/8) 128) + (rr%8) 16 bytes
                const uint32_t o = (uint32_t)kc * (BM / 8) * 128 + (uint32_t)((rr >> 3) * 128 + (rr & 7) * 16);
                *reinterpret_cast<uint4 *>(st + o) = hi;
                *reinterpret_cast<uint4 *>(st + a_bytes + o) = lo;
            }
            fence_async_shared();
            mbar_arrive(smem_u32(&full[s]));
        }
        if (!ok) abort_flag = 1;
        // all products of the CTA done before the accumulators are read
        if (ok && nkb > 0) {
            const int last = nkb - 1;
            if (!mbar_wait_abortable(smem_u32(&empty[last % S]), (uint32_t)((last / S) & 1), abort_v)) abort_flag = 1;
        }
    } else if (tid == 128 && nkb > 0) {
        // ---- B copies and MMAs ----
        auto issue_b = [&](int kb, int s) {
            const uint32_t sb = base + (uint32_t)s * stage_bytes, fb = smem_u32(&full[s]);
            mbar_expect_tx(fb, 2 * b_bytes);
            const int yb = kb * (Npad / 2);
            tma_load_2d(sb + 2 * a_bytes, mhi, 0, yb, fb);
            tma_load_2d(sb + 2 * a_bytes + b_bytes, mlo, 0, yb, fb);
        };
        const uint32_t idesc = make_idesc(BM, Npad);
        int issued = 0, consumed = 0;
        bool ok = true;
        if (A.test_wait > 0) {
            // a wait that runs out: nothing ever arrives on `never`
            const long long t0 = clock64();
            while (!mbar_try_wait(smem_u32(&never), 0u))
                if (clock64() - t0 > A.test_wait) {
                    ok = false;
                    break;
                }
        }
        for (; ok && issued < S && issued < nkb; ++issued) issue_b(kb0 + issued, issued);
        for (int i = 0; i < nkb && ok; ++i) {
            const int s = i % S;
            if (!mbar_wait_abortable(smem_u32(&full[s]), (uint32_t)((i / S) & 1), abort_v)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sb = base + (uint32_t)s * stage_bytes;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t a_off = (uint32_t)(2 * ks * (BM / 8) * 128);
                const uint32_t b_off = (uint32_t)(2 * ks * (Npad / 8) * 128);
                const uint64_t ahi = make_desc(sb + a_off, (BM / 8) * 128, 128);
                const uint64_t alo = make_desc(sb + a_bytes + a_off, (BM / 8) * 128, 128);
                const uint64_t bhi = make_desc(sb + 2 * a_bytes + b_off, (Npad / 8) * 128, 128);
                const uint64_t blo = make_desc(sb + 2 * a_bytes + b_bytes + b_off, (Npad / 8) * 128, 128);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                mma_bf16(tmem, ahi, bhi, idesc, acc);
                mma_bf16(tmem, ahi, blo, idesc, 1u);
                mma_bf16(tmem, alo, bhi, idesc, 1u);
            }
            mma_commit(smem_u32(&empty[s]));
            consumed = i + 1;
            // refill the B half of the stage of block i-1 once its products are done
            if (i >= 1 && issued < nkb) {
                const int j = i - 1;
                if (!mbar_wait_abortable(smem_u32(&empty[j % S]), (uint32_t)((j / S) & 1), abort_v)) {
                    ok = false;
                    break;
                }
                issue_b(kb0 + issued, issued % S);
                ++issued;
            }
        }
        if (!ok) {
            abort_flag = 1;
            // drain (bounded): the B copies issued land and the products committed end
            for (int j = consumed; j < issued; ++j)
                mbar_wait_bounded(smem_u32(&full[j % S]), (uint32_t)((j / S) & 1));
            if (consumed > 0)
                mbar_wait_bounded(smem_u32(&empty[(consumed - 1) % S]), (uint32_t)(((consumed - 1) / S) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_flag) {
        if (tid == 0) atomicOr(A.err, 1u);
    } else if (nkb > 0 && warp < 4) {
        // epilogue: warp w reads accumulator rows 32w .. 32w+31 (its TMEM lanes)
        const int r = m0 + tid;
        const long NN = (long)N * N;
        for (int c0 = 0; c0 < Npad; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (r < A.M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c0 + q;
                    if (n >= A.Ncol) continue;
                    long o;
                    if (A.ch == 0) o = (long)r * N + n;
                    else if (A.ch == 1) o = (long)n * NN + r;
                    else o = ((long)(r / N) * N + n) * N + (r % N);
                    atomicAdd(&out[o], scale * (double)v[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
}

// Shape of the launch of channel ch: stage count, split-K, grid; fills A's
// shape fields.  nz = flows along grid.z (1 for a single flow).
static qpfrg_status launch_fused(qpfrg_ctx *c, int ch, TcFusedArgs &A, int nz, int kid)
{
    const TcBuffers &t = c->tc;
    const int N = c->pb.N, Npad = t.Npad;
    const long NN = (long)N * N;
    const long Kp = ch == 2 ? t.Kpd : t.Kp;
    const size_t stage_bytes = 2 * (size_t)tc::BM * tc::BK * 2 + 2 * (size_t)Npad * tc::BK * 2;
    // as many stages as fit beside the kernel's static shared memory (barriers,
    // Z and K tables) within the 227 KB a block may opt into
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, tc_fused_kernel<4>);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_fused attributes");
    const size_t smem_max = 227 * 1024 - fa.sharedSizeBytes;
    int S = (int)std::min<size_t>(4, smem_max / stage_bytes);
    if (Npad % 16 != 0 || Npad > 256 || N > 256 || S < 2) {
        c->err = "tensor-core contraction: unsupported shape";
        return QPFRG_ERR_UNSUPPORTED;
    }
    const size_t smem = S * stage_bytes;
    auto kern = S == 4 ? tc_fused_kernel<4> : (S == 3 ? tc_fused_kernel<3> : tc_fused_kernel<2>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_fused smem attribute");
    const int M = (int)NN;
    const int mtiles = div_up(M, tc::BM);
    const int nkb = (int)(Kp / tc::BK);
    // split K so that the grid fills whole waves of the 152 SMs (one CTA per SM)
    int splits = 1;
    double best = -1.0;
    for (int sp = 1; sp <= std::max(1, nkb / 4) && sp <= 16; ++sp) {
        const int ctas = mtiles * sp * nz;
        const double waves = (double)ctas / 152.0, fill = waves / std::ceil(waves);
        const double score = fill - 0.02 * std::ceil(waves);
        if (score > best + 1e-9) {
            best = score;
            splits = sp;
        }
    }
    if (c->tune.tc_splits[ch] > 0) splits = std::min(c->tune.tc_splits[ch], nkb);
    const int kb_per = div_up(nkb, splits);
    splits = div_up(nkb, kb_per);
    A.M = M;
    A.Ncol = N;
    A.Npad = Npad;
    A.N = N;
    A.nkb_total = nkb;
    A.kb_per_split = kb_per;
    A.ch = ch;
    A.err = c->d_tc_err;
    A.test_wait = std::getenv("QPFRG_TEST_TC_WAIT") ? 10000000LL : 0;   // ~5 ms
    prof_begin(c);
    kern<<<dim3(mtiles, splits, nz), kFusedThreads, smem, c->stream>>>(t.tmB[ch][0], t.tmB[ch][1], A);
    prof_end(c, kid);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_fused_kernel");
}

// Host launcher of channel ch (0 pp, 1 cr, 2 d): out += scale * A B^T with A
// formed from the weighted loop-kernel table of the context.
qpfrg_status launch_tc_fused(qpfrg_ctx *c, int ch, double scale, double *out, int kid)
{
    TcFusedArgs A{};
    A.table = reinterpret_cast<const float *>(c->d_B);
    A.Vf = c->d_Vf;
    A.VT = c->tc.VT;
    A.out = out;
    A.scale = scale;
    return launch_fused(c, ch, A, 1, kid);
}

// Batched launch over the flows of a group (temperature flow, Z = 1):
// out_f += sign T_stage(f) A_f B_f^T for every running flow f with a step.
qpfrg_status launch_tc_fused_batch(qpfrg_ctx *c, int ch, const TcBatch &bt, double sign)
{
    TcFusedArgs A{};
    A.scale = sign;
    A.batch = bt;
    return launch_fused(c, ch, A, bt.nflows, K_TC_PP + ch);
}

}  // namespace qpfrg
