// Tensor-core contraction with the A operand formed in shared memory
// (QPFRG_MIXED_TC).
//
//   D[m][n] = sum_k A[m][k] B[n][k],  A = A_hi + A_lo,  B = B_hi + B_lo (BF16),
//   computed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in
//   tensor memory (the dropped A_lo B_lo term is 2^-16 relative).
//
// Row Q of A in channel ch is row Q of the weighted loop-kernel table
// (bubble.cu: the loop kernels binned by partner patch, times the line
// weights) times the vertex factor of (row, first loop patch a) -- the
// channel algebra of contract.cu, with the rows taken in transfer order so
// that a block of A rows is a block of table rows:
//   pp: Q = (i,j), out row (i,j),  A[Q][(a,b)] = B_pp[Q][a][b] V[i,j,a]
//   cr: Q = (l,j), out row (j,l),  A[Q][(a,b)] = B_ph[Q][a][b] V[b,j,l]
//   d : Q = (i,l), out row (i,l),  A[Q][(a,b)] = B_ph[Q][a][b] (2V[i,a,l] - V[a,i,l]),
//                                  A[Q][Kp + (a,b)] = -B_ph[Q][a][b] V[i,a,l]
//
// The table of the tensor-core path is stored in tiles (tc_table_index:
// [f][row tile][k block][half][128 rows][32 floats]), so a 128 x 64 block is
// two contiguous 16 KB boxes.  Per 64-wide k block and stage, one thread of the
// copy warp (warp 9) loads the raw FP32 block (two TMA boxes, 128-byte
// swizzle) and the B blocks (pre-formed per stage by tc_prep_kernel), refilling
// a stage as soon as the products of its previous block have committed.  The
// producer warps 0-7 (two threads per A row, one per 32-column half) read
// their half rows, scale them by the vertex factors (staged once per CTA in
// shared memory where they fit) and overwrite them, in place, with BF16 hi and
// lo in the K-major 128-byte-swizzle layout of the MMA descriptors (both
// operands): a row of 64 BF16 is 128 bytes, so row r of A_hi occupies exactly
// the bytes of raw row r of columns 0-31 and row r of A_lo those of columns
// 32-63 -- the two threads of a row read both halves before either writes.
// One thread of warp 8 issues the MMAs and commits each block to the stage's
// "empty" mbarrier.  Every wait is bounded by a clock budget and aborts the CTA
// (error flag, bounded drain, tensor memory freed).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>

#include "qpfrg_internal.h"
#include "tc_ptx.h"

namespace qpfrg {

namespace {

constexpr int kProducers = 256;                 // threads forming A (two per row)
constexpr int kMmaWarp = kProducers / 32;       // the MMA warp (one issuing thread)
constexpr int kCopyWarp = kMmaWarp + 1;         // the TMA copy warp (one issuing thread)
constexpr int kFusedThreads = kProducers + 64;
constexpr uint32_t kRawBytes = tc::BM * tc::BK * 4;   // FP32 table block = hi + lo of A

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
    int nkb_half;                     // k blocks per half of the d reduction (Kp / 64)
    long RT, KB;                      // row tiles and k blocks per family of the tiled table
    int ch;                           // 0 pp, 1 cr, 2 d
    // row orbits: A row m is the transfer pair rows[m] (table row m of the
    // compact table), output row m of out[m][n]; nullptr: row m is Q = m,
    // written to the channel's place in the N^3 output
    const int *rows;
    const float *Vf, *VT;             // stage vertex [k1][k2][k3]; factor tables of cr and d (tc_prep)
    int fw;                           // row stride of the staged factor rows (odd), 0: not staged
    double *out;
    double scale;
    unsigned *err;
    TcBatch batch;
    // test of the bounded waits (QPFRG_TEST_TC_WAIT): the MMA thread first
    // waits on a barrier nothing arrives on, with a budget of test_wait cycles
    long long test_wait;
};

// The vertex factor of A row Q at column k = (a, b) is a row of a factor
// table F[Q][x] (tc_prep_kernel): x = a for pp (F = V itself, Q = (i,j)) and d
// (F1 = 2V[i,a,l] - V[a,i,l] for the first half of the reduction, F2 =
// -V[i,a,l] for the second, Q = (i,l)), x = b for cr (V[b,j,l], Q = (l,j)).
// Each CTA needs the x range its k blocks touch, per half: seg_lo[h] and
// seg_n[h] (seg_n = 0 when the CTA has no block in half h).
__host__ __device__ inline void factor_segments(int ch, int N, int kb0, int kb1, int nkb_half, int (&lo)[2],
                                                int (&n)[2])
{
    const int NN = N * N;
    for (int h = 0; h < 2; ++h) {
        const int s0 = h == 0 ? kb0 : (kb0 > nkb_half ? kb0 : nkb_half) - nkb_half;
        const int s1 = h == 0 ? (ch == 2 ? (kb1 < nkb_half ? kb1 : nkb_half) : kb1) : (ch == 2 ? kb1 - nkb_half : 0);
        lo[h] = 0;
        n[h] = 0;
        if (s1 <= s0) continue;
        if (ch == 1) {
            n[h] = N;    // every b
            continue;
        }
        const int k_first = s0 * 64, k_last = (s1 * 64 < NN ? s1 * 64 : NN) - 1;
        lo[h] = k_first / N;
        n[h] = k_last / N - lo[h] + 1;
    }
}

template <int S, bool N8, bool STG>
__global__ void __launch_bounds__(kFusedThreads, 1)
    tc_fused_kernel(const __grid_constant__ CUtensorMap mTab, const __grid_constant__ CUtensorMap mBhi,
                    const __grid_constant__ CUtensorMap mBlo, TcFusedArgs A)
{
    using namespace tc;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t rfull[S], full[S], empty[S], never;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    // the flow of this CTA (batched launch) or the context's single flow
    const float *Vf = A.Vf, *VT = A.VT;
    double *out = A.out;
    double scale = A.scale;
    const CUtensorMap *mtab = &mTab, *mhi = &mBhi, *mlo = &mBlo;
    if (A.batch.nflows) {
        const TcBatch &Bt = A.batch;
        const int f = blockIdx.z;
        const long sf = (long)Bt.step * Bt.nflows + f;
        const double h = Bt.h_tab[sf];
        if (Bt.status[f] != QPFRG_FLOW_RUNNING || h == 0.0) return;   // uniform, before any barrier
        mtab = Bt.tab_maps + Bt.slot_tab[sf];
        Vf = Bt.Vf[f];
        VT = Bt.VT[f];
        out = Bt.outc ? Bt.outc[f] + (long)A.ch * A.M * A.N : Bt.out[f];
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
    const int NN = N * N;
    const int fam = A.ch == 0 ? 0 : 1;
    const uint32_t b_bytes = (uint32_t)Npad * BK * 2;
    const uint32_t stage_bytes = kRawBytes + 2 * b_bytes;
    // stages on 1024-byte boundaries (the 128-byte swizzle repeats every 1024 B)
    const uint32_t raw_base = smem_u32(smem_raw);
    const uint32_t base = (raw_base + 1023u) & ~1023u;
    unsigned char *const sbase = smem_raw + (base - raw_base);
    const uint32_t tmem_cols = Npad <= 32 ? 32 : (Npad <= 64 ? 64 : (Npad <= 128 ? 128 : 256));

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&rfull[s]), 1);            // the copies' expect-tx arrival (table and B)
            mbar_init(smem_u32(&full[s]), kProducers);    // the producers' A rows
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&never), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kMmaWarp) {
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

    if (warp < kMmaWarp) {
        // ---- producers: warp w owns rows 16 w .. 16 w + 15 of every block,
        // lanes l and l + 16 the two halves (columns 0-31, 32-63) of row 16 w + l ----
        const int lane = tid & 31;
        const int rr = (warp << 4) | (lane & 15), hh = lane >> 4;
        const bool valid = m0 + rr < A.M;
        const int Q = !valid ? 0 : (A.rows ? A.rows[m0 + rr] : m0 + rr);   // transfer pair of the row
        // raw row rr of the half h (columns 32 h .. 32 h + 31), 16-byte chunk c:
        // h 16 KB + rr 128 + (c ^ (rr % 8)) 16 (128-byte swizzle); A_hi row rr,
        // 8-wide k chunk kc: rr 128 + (kc ^ (rr % 8)) 16, A_lo the same + 16 KB
        // (the 128-byte-swizzled K-major layout of the MMA): the thread's
        // converted row occupies exactly its own raw row's bytes
        const uint32_t raw_row = (uint32_t)rr * 128, sw = (uint32_t)(rr & 7);
        // this row's factor rows (per half of the reduction) and the x ranges
        // the CTA's k blocks touch
        const long n3 = (long)NN * N;
        const float *frow0 = (A.ch == 0 ? Vf : (A.ch == 1 ? VT : VT + n3)) + (long)Q * N;
        const float *frow1 = VT + 2 * n3 + (long)Q * N;
        int seg_lo[2], seg_n[2];
        factor_segments(A.ch, N, kb0, kb1, A.nkb_half, seg_lo, seg_n);
        // staged: the row's two threads copy its factor row segments into
        // shared memory once (row stride fw, odd: the rows hit distinct banks);
        // only they read them, after the warp's barrier
        float *fs = reinterpret_cast<float *>(sbase + (size_t)S * stage_bytes) + (size_t)rr * (STG ? A.fw : 0);
        if (STG) {
            // 24 loads in flight per thread (a dependent one-by-one copy cost
            // a DRAM round trip per value; the cr rows are N values long)
            for (int g = 0; g < 2; ++g) {
                const float *src = (g ? frow1 + seg_lo[1] : frow0 + seg_lo[0]);
                float *dst = fs + (g ? seg_n[0] : 0);
                const int n = seg_n[g];
                for (int t0 = hh; t0 < n; t0 += 48) {
                    float tmp[24];
#pragma unroll
                    for (int u = 0; u < 24; ++u) {
                        const int t = t0 + 2 * u;
                        tmp[u] = (valid && t < n) ? __ldg(src + t) : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 24; ++u)
                        if (t0 + 2 * u < n) dst[t0 + 2 * u] = tmp[u];
                }
            }
            __syncwarp();
        }
        // factor of table column x (a or b) in half h
        auto factor = [&](int h, int x) -> float {
            if (STG) return fs[(h ? seg_n[0] - seg_lo[1] : -seg_lo[0]) + x];
            return valid ? __ldg((h ? frow1 : frow0) + x) : 0.f;
        };
        bool ok = true;
        for (int it = 0; it < nkb && ok; ++it) {
            const int s = it % S;
            const int kb = kb0 + it;
            const bool second = A.ch == 2 && kb >= A.nkb_half;
            const int h = second ? 1 : 0;
            const int kk0 = (kb - (second ? A.nkb_half : 0)) * BK;
            const bool got = mbar_wait_abortable(smem_u32(&rfull[s]), (uint32_t)((it / S) & 1), abort_v);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            unsigned char *st = sbase + (size_t)s * stage_bytes;
            // this thread's half row: columns 32 hh .. 32 hh + 31
            float v[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float4 x = *reinterpret_cast<const float4 *>(st + hh * (kRawBytes / 2) + raw_row +
                                                                   ((c ^ sw) << 4));
                v[4 * c + 0] = x.x;
                v[4 * c + 1] = x.y;
                v[4 * c + 2] = x.z;
                v[4 * c + 3] = x.w;
            }
            // both halves of every row of the warp read before any is overwritten
            // (the row's lo chunks 0-3 lie in the other half's bytes)
            __syncwarp();
            // (a, b) of the thread's first column; N8: a chunk of 8 columns
            // lies in one a and never passes N^2
            const int kt0 = kk0 + 32 * hh;
            int a = kt0 / N, b = kt0 - a * N;
#pragma unroll
            for (int kcl = 0; kcl < 4; ++kcl) {
                const int kc = 4 * hh + kcl;
                float f[8];
                if (N8) {
                    if (A.ch == 1 && !STG) {
                        // 8 consecutive b (b % 8 == 0, N % 8 == 0): two aligned 16-byte loads
                        float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
                        if (valid) {
                            c0 = __ldg(reinterpret_cast<const float4 *>(frow0 + b));
                            c1 = __ldg(reinterpret_cast<const float4 *>(frow0 + b) + 1);
                        }
                        f[0] = c0.x; f[1] = c0.y; f[2] = c0.z; f[3] = c0.w;
                        f[4] = c1.x; f[5] = c1.y; f[6] = c1.z; f[7] = c1.w;
                    } else if (A.ch == 1) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = factor(h, b + e);
                    } else {
                        const float fa = factor(h, a);
#pragma unroll
                        for (int e = 0; e < 8; ++e) f[e] = fa;
                    }
                    b += 8;
                    if (b >= N) {
                        b -= N;
                        ++a;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        f[e] = kt0 + 8 * kcl + e < NN ? factor(h, A.ch == 1 ? b : a) : 0.f;
                        if (++b == N) {
                            b = 0;
                            ++a;
                        }
                    }
                }
                uint4 hi, lo;
                uint32_t *hp = &hi.x, *lp = &lo.x;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x0 = v[8 * kcl + 2 * q] * f[2 * q];
                    const float x1 = v[8 * kcl + 2 * q + 1] * f[2 * q + 1];
                    const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
                    hp[q] = *reinterpret_cast<const uint32_t *>(&hh);
                    lp[q] = pack_bf16x2(x0 - __low2float(hh), x1 - __high2float(hh));
                }
                *reinterpret_cast<uint4 *>(st + raw_row + ((kc ^ sw) << 4)) = hi;
                *reinterpret_cast<uint4 *>(st + kRawBytes / 2 + raw_row + ((kc ^ sw) << 4)) = lo;
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
    } else if (tid == kCopyWarp * 32 && nkb > 0) {
        // ---- table and B copies: stage s is refilled as soon as the products
        // of its previous block are done ----
        const long tile0 = ((long)fam * A.RT + blockIdx.x) * A.KB;   // first k block of this row tile
        int issued = 0;
        for (; issued < nkb; ++issued) {
            const int s = issued % S;
            if (issued >= S &&
                !mbar_wait_abortable(smem_u32(&empty[s]), (uint32_t)(((issued / S) - 1) & 1), abort_v))
                break;
            const int kb = kb0 + issued;
            const uint32_t sb = base + (uint32_t)s * stage_bytes;
            const bool second = A.ch == 2 && kb >= A.nkb_half;
            const int kbl = kb - (second ? A.nkb_half : 0);           // k block within the table row
            const int y = (int)((tile0 + kbl) * 256);                 // two halves of 128 rows of 32 floats
            const uint32_t rb = smem_u32(&rfull[s]);
            mbar_expect_tx(rb, kRawBytes + 2 * b_bytes);
            tma_load_2d(sb, mtab, 0, y, rb);
            tma_load_2d(sb + kRawBytes / 2, mtab, 0, y + 128, rb);
            const int yb = kb * (Npad / 2);
            tma_load_2d(sb + kRawBytes, mhi, 0, yb, rb);
            tma_load_2d(sb + kRawBytes + b_bytes, mlo, 0, yb, rb);
        }
        if (issued < nkb) {
            abort_flag = 1;
            // drain (bounded): the copies in flight land
            for (int j = issued > S ? issued - S : 0; j < issued; ++j)
                mbar_wait_bounded(smem_u32(&rfull[j % S]), (uint32_t)((j / S) & 1));
        }
    } else if (tid == kMmaWarp * 32 && nkb > 0) {
        // ---- MMAs ----
        const uint32_t idesc = make_idesc(BM, Npad);
        int consumed = 0;
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
        for (int i = 0; i < nkb && ok; ++i) {
            const int s = i % S;
            // the A rows formed, and (already complete by then) the B copies
            if (!mbar_wait_abortable(smem_u32(&full[s]), (uint32_t)((i / S) & 1), abort_v) ||
                !mbar_wait_abortable(smem_u32(&rfull[s]), (uint32_t)((i / S) & 1), abort_v)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sb = base + (uint32_t)s * stage_bytes;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint32_t k_off = (uint32_t)(ks * 32);                   // 16 BF16 along the swizzled row
                const uint64_t ahi = make_desc_sw128(sb + k_off, 1024);
                const uint64_t alo = make_desc_sw128(sb + kRawBytes / 2 + k_off, 1024);
                const uint64_t bhi = make_desc_sw128(sb + kRawBytes + k_off, 1024);
                const uint64_t blo = make_desc_sw128(sb + kRawBytes + b_bytes + k_off, 1024);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                mma_bf16(tmem, ahi, bhi, idesc, acc);
                mma_bf16(tmem, ahi, blo, idesc, 1u);
                mma_bf16(tmem, alo, bhi, idesc, 1u);
            }
            mma_commit(smem_u32(&empty[s]));
            consumed = i + 1;
        }
        if (!ok) {
            abort_flag = 1;
            // drain (bounded): the products committed end
            if (consumed > 0)
                mbar_wait_bounded(smem_u32(&empty[(consumed - 1) % S]), (uint32_t)(((consumed - 1) / S) & 1));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (abort_flag) {
        if (tid == 0) atomicOr(A.err, 1u);
    } else if (nkb > 0 && warp < kMmaWarp) {
        // epilogue: warp w reads accumulator rows 32 (w % 4) .. +31 (the TMEM
        // lanes of its rank in the warpgroup); warps 0-3 take the even
        // 16-column chunks, warps 4-7 the odd ones
        const int lane = tid & 31, wq = warp & 3;
        const int Q = m0 + 32 * wq + lane;          // row (compact index with row orbits)
        const int qa = Q / N, qb = Q - qa * N;
        for (int c0 = 16 * (warp >> 2); c0 < Npad; c0 += 32) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, v);
            if (Q < A.M) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c0 + q;
                    if (n >= A.Ncol) continue;
                    long o;
                    if (A.ch == 0 || A.rows) o = (long)Q * N + n;                // (i, j, n); compact rows [m][n]
                    else if (A.ch == 1) o = (long)n * NN + (long)qb * N + qa;     // (n, j, l)
                    else o = ((long)qa * N + n) * N + qb;                         // (i, n, l)
                    atomicAdd(&out[o], scale * (double)v[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols));
}

// Shape of the launch of channel ch: stage count, split-K, grid; fills A's
// shape fields.  nz = flows along grid.z (1 for a single flow).
static qpfrg_status launch_fused(qpfrg_ctx *c, int ch, TcFusedArgs &A, int nz, int kid)
{
    const TcBuffers &t = c->tc;
    const int N = c->pb.N, Npad = t.Npad;
    const long NN = (long)N * N;
    const long Kp = ch == 2 ? t.Kpd : t.Kp;
    if (Npad % 16 != 0 || Npad > 256 || N > 256 || (N & 1)) {
        c->err = "tensor-core contraction: unsupported shape";
        return QPFRG_ERR_UNSUPPORTED;
    }
    const int M = A.rows ? c->n_rrep : (int)NN;
    const int mtiles = div_up(M, tc::BM);
    const int nkb = (int)(Kp / tc::BK);
    const int nkb_half = (int)(t.Kp / tc::BK);
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
    // the factor rows the widest split touches, staged in shared memory when
    // they fit beside at least two stages (row stride odd)
    int wmax = 1;
    for (int y = 0; y < splits; ++y) {
        int lo[2], n[2];
        factor_segments(ch, N, y * kb_per, std::min(nkb, (y + 1) * kb_per), nkb_half, lo, n);
        wmax = std::max(wmax, n[0] + n[1]);
    }
    const int fw = wmax | 1;
    const size_t stage_bytes = kRawBytes + 2 * (size_t)Npad * tc::BK * 2;
    const size_t fbytes = (size_t)tc::BM * fw * sizeof(float);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, tc_fused_kernel<4, true, true>);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_fused attributes");
    // 227 KB a block may opt into, less the static barriers and 1 KB of alignment slack
    const size_t avail = 227 * 1024 - 1024 - fa.sharedSizeBytes;
    int S = avail > fbytes ? (int)std::min<size_t>(4, (avail - fbytes) / stage_bytes) : 0;
    const bool stg = S >= 2;
    if (!stg) S = (int)std::min<size_t>(4, avail / stage_bytes);
    if (S < 2) {
        c->err = "tensor-core contraction: unsupported shape";
        return QPFRG_ERR_UNSUPPORTED;
    }
    const size_t smem = S * stage_bytes + 1024 + (stg ? fbytes : 0);
    using KernT = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, TcFusedArgs);
    static const KernT table[3][2][2] = {
        {{tc_fused_kernel<2, false, false>, tc_fused_kernel<2, false, true>},
         {tc_fused_kernel<2, true, false>, tc_fused_kernel<2, true, true>}},
        {{tc_fused_kernel<3, false, false>, tc_fused_kernel<3, false, true>},
         {tc_fused_kernel<3, true, false>, tc_fused_kernel<3, true, true>}},
        {{tc_fused_kernel<4, false, false>, tc_fused_kernel<4, false, true>},
         {tc_fused_kernel<4, true, false>, tc_fused_kernel<4, true, true>}}};
    const KernT kern = table[S - 2][(N & 7) == 0 ? 1 : 0][stg ? 1 : 0];
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "tc_fused smem attribute");
    A.M = M;
    A.Ncol = N;
    A.Npad = Npad;
    A.N = N;
    A.nkb_total = nkb;
    A.kb_per_split = kb_per;
    A.nkb_half = (int)(t.Kp / tc::BK);
    A.RT = t.RT;
    A.KB = t.KB;
    A.ch = ch;
    A.fw = stg ? fw : 0;
    A.err = c->d_tc_err;
    A.test_wait = std::getenv("QPFRG_TEST_TC_WAIT") ? 10000000LL : 0;   // ~5 ms
    prof_begin(c);
    kern<<<dim3(mtiles, splits, nz), kFusedThreads, smem, c->stream>>>(t.tmTab, t.tmB[ch][0], t.tmB[ch][1], A);
    prof_end(c, kid);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "tc_fused_kernel");
}

// Host launcher of channel ch (0 pp, 1 cr, 2 d): out += scale * A B^T with A
// formed from the weighted loop-kernel table of the context.
qpfrg_status launch_tc_fused(qpfrg_ctx *c, int ch, double scale, double *out, int kid)
{
    TcFusedArgs A{};
    A.Vf = c->d_Vf;
    A.VT = c->tc.VT;
    A.out = out;
    A.scale = scale;
    A.rows = c->rows_compact ? c->d_rrep : nullptr;
    return launch_fused(c, ch, A, 1, kid);
}

// Batched launch over the flows of a group (temperature flow, Z = 1):
// out_f += sign T_stage(f) A_f B_f^T for every running flow f with a step.
qpfrg_status launch_tc_fused_batch(qpfrg_ctx *c, int ch, const TcBatch &bt, double sign)
{
    TcFusedArgs A{};
    A.scale = sign;
    A.batch = bt;
    A.rows = bt.outc ? c->d_rrep : nullptr;
    return launch_fused(c, ch, A, bt.nflows, K_TC_PP + ch);
}

}  // namespace qpfrg
