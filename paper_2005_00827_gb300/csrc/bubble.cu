// Loop kernels of the one-loop vertex flow, grouped by transfer momentum.
//
// For every transfer Q of the particle-particle family (Q = k_F(x) + k_F(y),
// partner Q - p) and of the particle-hole family (Q = k_F(x) - k_F(y),
// partner p + Q) this kernel bins the Z-weighted loop kernel of each fine
// point p into the bubble table
//     B_f[Q][a][b] = s(a,b) * sum_{p in a, proj(partner) = b} w_p L'_f(x_p, x_partner)
// with L'_ph = dD/dT, L'_pp = -dD(x_p, -x_q)/dT in the temperature flow and
// L'_ph = D, L'_pp = -D(x_p, -x_q) in the interaction flow, where
// D(a,b) = (f(a) - f(b))/(a - b) is the closed-form Matsubara sum of G0 G0.
// s(a,b) = Z_a Z_b (T-flow) or g Z_a Z_b (Z_a + Z_b) (g-flow), the line
// weights of Eq. (both_propagators_Z) / Eq. (vertex_flow_feedback_Z).
//
// Launch shape: one CTA of 8 warps per (patch a, chunk of Q, family) -- or,
// in wedge mode, per task of the C4v-reduced launch (symmetry.cu: one row per
// orbit of (Q, a) under the point group, written to every image row with its
// columns permuted; or, for the tensor-core contraction of a C4v-symmetric
// state, the representative transfer pairs of the row orbits with every patch
// a, each row written once to the compact table).  The CTA stages its wedge's
// fine points in shared
// memory; each warp takes one transfer at a time, streams its partner-patch
// bytes (coalesced) and bins the loop kernels into a private row of N
// accumulators.  Output: the weighted tables B_f[Q][a][b] (FP64, or FP32 for
// the SIMT and the tensor-core contractions), every image row written with
// coalesced stores.
#include <algorithm>

#include "qpfrg_internal.h"

namespace qpfrg {

template <typename R>
struct BubbleArgs {
    Problem pb;
    FineTable<R> fine;
    TransferTable<R> qpp, qph;
    const uint8_t *part;
    const double *Z;
    const double *K;      // Katanin factors of the interaction flow's S line (NULL = 1)
    R *B;
    R T, invT, g, thr;
    // FP32 rows accumulate as 32-bit fixed point: bin = int / fscale (finv = 1/fscale)
    float fscale, finv;
    R t, tp, mu;          // hoppings and chemical potential, already in R (no per-use conversion)
    int qchunk;
    // C4v-reduced launch (symmetry.cu; tasks == nullptr: every row evaluated):
    // CTA task (family, patch, first representative, count); per
    // representative its transfer and its image rows (Q', a' | g << 16); img
    // == nullptr with tasks: the contraction's representative rows, each
    // written once to row kq of the compact table
    const int4 *tasks;
    const int *repQ;
    const int *nimg;
    const int2 *img;
    // batched flows: a device flag read by every CTA; 0 = nothing to do
    const int *active;
    // tensor-core path: the table in tiles (tc_table_index; tRT = 0: row-major)
    long tRT, tKB;
};

// ---- scalar helpers ---------------------------------------------------------
__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
// exp(-|x|/T) from k = log2(e)/T (FP32: one multiply and ex2.approx) or k = 1/T (FP64)
__device__ __forceinline__ float exp_mT(float x, float k)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-fabsf(x) * k));
    return y;
}
__device__ __forceinline__ double exp_mT(double x, double k) { return exp(-fabs(x) * k); }
// a / b with one reciprocal (FP32: rcp.approx; FP64: the division)
__device__ __forceinline__ float qdiv(float a, float b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return a * r;
}
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
// typed absolute value: plain fabs() on a float would promote to FP64
__device__ __forceinline__ float qabs(float x) { return fabsf(x); }
__device__ __forceinline__ double qabs(double x) { return fabs(x); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// f(x) and 1 - f(x) without cancellation: e = exp(-|x|/T)
template <typename R>
__device__ __forceinline__ void fermi_pair(R x, R invT, R &f, R &fc)
{
    const R e = fexp(-qabs(x) * invT);
    const R lo = fdiv(e, R(1) + e), hi = fdiv(R(1), R(1) + e);
    f = x > R(0) ? lo : hi;
    fc = x > R(0) ? hi : lo;
}

// f(1-f) = e/(1+e)^2
template <typename R>
__device__ __forceinline__ R fermi_ff(R x, R invT)
{
    const R e = fexp(-qabs(x) * invT);
    const R d = R(1) + e;
    return fdiv(e, d * d);
}

// d/dT f(x) = x/T^2 f(1-f)
template <typename R>
__device__ __forceinline__ R fermi_dT(R x, R invT)
{
    return x * invT * invT * fermi_ff(x, invT);
}

// d/dx d/dT f = f'(x) (-1/T + x tanh(x/2T)/T^2), f' = -f(1-f)/T
template <typename R>
__device__ __forceinline__ R fermi_dxdT(R x, R invT)
{
    const R e = fexp(-qabs(x) * invT);
    const R d = R(1) + e;
    const R ff = fdiv(e, d * d);
    R th = fdiv(R(1) - e, d);
    th = x > R(0) ? th : -th;
    return -ff * invT * (-invT + x * th * invT * invT);
}

// Loop kernel of one line pair (x_p, x_q), temperature flow.
//   ph: dD(x_p, x_q)/dT = (g_p - g_q)/(x_p - x_q),   g = df/dT
//   pp: -dD(x_p, -x_q)/dT = -(g_p + g_q)/(x_p + x_q)   (g odd in x)
// Below |difference| < thr*T the analytic derivative at the midpoint is used.
template <typename R>
__device__ __forceinline__ R loop_T(bool pp, R xp, R gp, R xq, R invT, R invT2, R kexp, R thrT)
{
    const R den = pp ? xp + xq : xp - xq;
    if (qabs(den) < thrT) {
        const R m = R(0.5) * (pp ? xp - xq : xp + xq);
        const R v = fermi_dxdT(m, invT);
        return pp ? -v : v;
    }
    const R e = exp_mT(xq, kexp);
    const R d = R(1) + e, d2 = d * d;
    const R gq_num = xq * invT2 * e;                 // g_q * d2
    const R num = pp ? gp * d2 + gq_num : gp * d2 - gq_num;
    const R v = qdiv(num, d2 * den);
    return pp ? -v : v;
}

// Two loop_T values of one fine point (x_p, g_p) against two partners, as
// packed FP32x2 arithmetic, times the point's weight w; a lane whose difference
// is near-degenerate is replaced by loop_T's midpoint derivative.
__device__ __forceinline__ float2 loop_T2(bool pp, float xp, float gp, float w, float2 xq, float invT,
                                          float invT2, float kexp, float thrT)
{
    const float sd = pp ? 1.f : -1.f;
    const float2 den = __ffma2_rn(xq, make_float2(sd, sd), make_float2(xp, xp));
    const float2 e = make_float2(exp_mT(xq.x, kexp), exp_mT(xq.y, kexp));
    const float2 d = __fadd2_rn(e, make_float2(1.f, 1.f));
    const float2 d2 = __fmul2_rn(d, d);
    const float sg = pp ? invT2 : -invT2;        // +- g_q (1 + e)^2 = +- x_q e / T^2
    const float2 num = __ffma2_rn(make_float2(gp, gp), d2, __fmul2_rn(__fmul2_rn(xq, make_float2(sg, sg)), e));
    const float2 dd = __fmul2_rn(d2, den);
    const float2 v = __fmul2_rn(num, make_float2(qdiv(1.f, dd.x), qdiv(1.f, dd.y)));
    const float ws = pp ? -w : w;
    float2 r = __fmul2_rn(v, make_float2(ws, ws));
    // a near-degenerate lane takes the midpoint derivative instead (one rarely
    // taken branch for both lanes)
    const bool m0 = fabsf(den.x) < thrT, m1 = fabsf(den.y) < thrT;
    if (m0 || m1) {
        if (m0) r.x = w * loop_T(pp, xp, gp, xq.x, invT, invT2, kexp, thrT);
        if (m1) r.y = w * loop_T(pp, xp, gp, xq.y, invT, invT2, kexp, thrT);
    }
    return r;
}

// Loop kernel of one line pair, interaction flow at fixed T.
//   ph: D(x_p, x_q),  pp: -D(x_p, -x_q) = (1 - f_p - f_q)/(x_p + x_q)
template <typename R>
__device__ __forceinline__ R loop_g(bool pp, R xp, R fp, R fcp, R xq, R invT, R thrT)
{
    const R den = pp ? xp + xq : xp - xq;
    if (qabs(den) < thrT) {
        const R m = R(0.5) * (pp ? xp - xq : xp + xq);
        const R v = -fermi_ff(m, invT) * invT;       // f'(m)
        return pp ? -v : v;
    }
    R fq, fcq;
    fermi_pair(xq, invT, fq, fcq);
    // numerator f(a) - f(b) with b = x_q (ph) or -x_q (pp); f(-x_q) = fc_q
    R fa = fp, fb = pp ? fcq : fq, ca = fcp, cb = pp ? fq : fcq;
    const R xb = pp ? -xq : xq;
    const R num = (xp < R(0) && xb < R(0)) ? cb - ca : fa - fb;
    const R v = fdiv(num, den);
    return pp ? -v : v;
}

// Lane layout of a patch's fine points (local index t n_r + s, t angular,
// s radial): a warp row holds 32 points, lanes along the radius.  With
// n_r >= 32 a row is 32 radii of one angle (radial chunks of 32, all angles of
// a chunk before the next chunk); with n_r < 32 the warp splits into 32 / lr
// groups of lr lanes (lr = n_r rounded up to a power of two), group g taking
// the g-th contiguous block of per_chunk angles.  Either way consecutive rows
// of a lane are adjacent angles at one radius, whose partners mostly share a
// patch (runs are long, flushes rare).
struct LaneMap {
    int lr, apr, nchunk, per_chunk;   // lanes per angle, angles per row, radial chunks, rows per chunk
    __host__ __device__ LaneMap(int nt, int nr)
    {
        if (nr >= 32) {
            lr = 32;
            apr = 1;
            nchunk = (nr + 31) / 32;
        } else {
            lr = 1;
            while (lr < nr) lr <<= 1;
            apr = 32 / lr;
            nchunk = 1;
        }
        per_chunk = (nt + apr - 1) / apr;
    }
};

template <typename R>
struct alignas(4 * sizeof(R)) Quad {
    R x, y, z, w;
};

// Row accumulators.  FP32: 32-bit fixed point in units of 1/fscale, so that a
// run's flush is one native integer shared-memory add (a float add on shared
// memory is a compare-and-swap loop, which diverges the warp); the host picks
// fscale from the bound |bin| <= P w_max max|L| (max|dD/dT| = 1/(4T^2),
// max|D| = 1/(4T)) with a factor 2 to spare, so no bin leaves +-2^29.  FP64:
// double adds.
__device__ __forceinline__ void row_add(float *slot, float v, float fscale)
{
    atomicAdd(reinterpret_cast<int *>(slot), __float2int_rn(v * fscale));
}
__device__ __forceinline__ void row_add(double *slot, double v, float) { atomicAdd(slot, v); }
// the run's flush when the partner patch b differs from the run's patch rb:
// the FP32 path issues it as one shared reduction predicated on that test (no
// branch around it), the FP64 path branches
__device__ __forceinline__ void row_add_if(float *slot, float v, float fscale, int b, int rb)
{
    const int iv = __float2int_rn(v * fscale);
    const unsigned addr = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %2, %3;\n\t@q red.shared.add.s32 [%0], %1;\n\t}" ::"r"(addr),
        "r"(iv), "r"(b), "r"(rb)
        : "memory");
}
__device__ __forceinline__ void row_add_if(double *slot, double v, float, int b, int rb)
{
    if (b != rb) atomicAdd(slot, v);
}
__device__ __forceinline__ float row_get(const float *slot, float finv)
{
    return (float)*reinterpret_cast<const int *>(slot) * finv;
}
__device__ __forceinline__ double row_get(const double *slot, float) { return *slot; }

// Column b of the image row under g (g = m | reflection << 2 acting on the
// wedge w of b = w ns + s: w -> +-w + m N_a/4, the shell s kept) holds the
// representative's bin g^-1(b).
__device__ __forceinline__ int img_src(int b, int off, bool refl, int N, int ns)
{
    if (ns == 1) {
        const int r = refl ? off - b : b - off;
        return r < 0 ? r + N : r;
    }
    const int w = b / ns, sh = b - w * ns, Na = N / ns;
    const int r = refl ? off - w : w - off;
    return (r < 0 ? r + Na : r) * ns + sh;
}

// Write-out of one row to the bubble table B[fam][Qi][ai][:] of the image row
// under g, with the line weights s(ai, b) (interaction flow: g Z_a Z_b
// (K_a Z_a + K_b Z_b)).  The row is read, not cleared.
template <typename R, bool TFLOW>
__device__ __forceinline__ void table_row(const BubbleArgs<R> &A, const R *row, const R *Zs, const R *Ks, int fam,
                                          int Qi, int ai, int g, int lane)
{
    const int N = A.pb.N, ns = A.pb.n_shell;
    const long NN = (long)N * N;
    const int off = (g & 3) * (N / ns / 4);
    const bool refl = (g & 4) != 0;
    const R Za = Zs[ai], KZa = Ks[ai] * Za;
    // column b goes to k = ai N + b of row Qi: row-major at base + k, tiled
    // (tc_table_index) at base + (k / 32) 4096 + k % 32
    const int k0 = ai * N;
    R *dst = A.B + (A.tRT ? ((long)fam * A.tRT + (Qi >> 7)) * A.tKB * 8192 + (Qi & 127) * 32
                          : ((long)fam * NN + Qi) * NN);
    for (int b = lane; b < N; b += 32) {
        const R v = row_get(row + img_src(b, off, refl, N, ns), A.finv);
        const R Zb = Zs[b];
        const R sw = TFLOW ? Za * Zb : A.g * Za * Zb * (KZa + Ks[b] * Zb);
        const int k = k0 + b;
        dst[A.tRT ? ((long)(k >> 5) << 12) + (k & 31) : (long)k] = v * sw;
    }
}

// Kernel body for one transfer family (PP: particle-particle, else
// particle-hole) and one regulator (TFLOW: temperature flow, else
// interaction flow), both fixed at compile time.
//
// One warp per transfer Q: it walks the patch's points row by row, keeps a
// run (partner patch, partial sum) per lane, adds a run to its private
// shared-memory row of N accumulators when the lane's partner patch changes
// (lanes on one radius change on different wedge boundaries, so these atomic
// adds rarely collide), flushes the last runs through a segmented warp
// reduction (one atomic per run of equal partners among the lanes) and writes
// the row out.  No block barrier inside the transfer loop.
//
// Rows k in [q0, q1): the transfer Q = k (unreduced launch) or the
// representative k of the C4v-reduced launch, Q = repQ[k], written to each of
// its image rows.  A warp carries H transfers at once (H = 2 or 4): one
// shared-memory read of a point serves all of them.
template <typename R, bool PP, bool TFLOW, bool TP0, int H, bool FULL>
__device__ __forceinline__ void bubble_body(const BubbleArgs<R> &A, unsigned char *smem_raw, int a, int q0, int q1)
{
    const int N = A.pb.N, P = A.pb.P, M = A.pb.M;
    const long NN = (long)N * N;
    const int fam = PP ? 0 : 1;
    constexpr bool pp = PP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    constexpr bool tflow = TFLOW;
    const bool qp = A.pb.propagator == QPFRG_PROP_QP;
    const int nr = A.pb.n_r, nt = A.pb.n_theta;

    Quad<R> *pc = reinterpret_cast<Quad<R> *>(smem_raw);   // cos p_x, cos p_y, sin p_x, sin p_y
    Quad<R> *pe = pc + P;                                   // x_p, f-terms, weight
    R *Zs = reinterpret_cast<R *>(pe + P);                  // N
    // H nwarp rows (H transfers per warp) of N accumulators and a sink (slot
    // N) for lanes without points, so that a change of partner is one add of
    // the finished run; the row stride N + 2 is even, keeping every row 8-byte
    // aligned (an odd stride once misaligned 8-byte reads of these rows)
    const int RS = N + 2;
    R *rows = Zs + N;
    R *Ks = rows + H * nwarp * RS;                          // N Katanin factors
    for (int i = tid; i < N; i += blockDim.x) {
        Zs[i] = A.Z ? (R)A.Z[i] : R(1);
        Ks[i] = A.K ? (R)A.K[i] : R(1);
    }
    for (int i = tid; i < H * nwarp * RS; i += blockDim.x) rows[i] = R(0);
    __syncthreads();
    const R Za = Zs[a];
    const R invT = A.invT, thrT = A.thr * A.T, invT2 = invT * invT;
    const R kexp = sizeof(R) == 4 ? invT * R(1.4426950408889634) : invT;
    const R t = A.t, tp = A.tp, mu = A.mu;
    for (int i = tid; i < P; i += blockDim.x) {
        const int p = a * P + i;
        Quad<R> c4, e4;
        c4.x = A.fine.cx[p];
        c4.y = A.fine.cy[p];
        c4.z = A.fine.sx[p];
        c4.w = A.fine.sy[p];
        const R x = qp ? Za * A.fine.xi[p] : A.fine.xi[p];
        e4.x = x;
        if (tflow) {
            e4.y = fermi_dT(x, invT);
            e4.z = R(0);
        } else {
            fermi_pair(x, invT, e4.y, e4.z);
        }
        e4.w = A.fine.w[p];
        pc[i] = c4;
        pe[i] = e4;
    }
    __syncthreads();

    const LaneMap lm(nt, nr);
    const TransferTable<R> &Qt = pp ? A.qpp : A.qph;
    const int dt = lane / lm.lr, sl = lane & (lm.lr - 1);
    const int stride = nr;                             // local index step between a lane's rows
    const bool vec4 = nt % 4 == 0 && lm.per_chunk % 4 == 0;
    // Each warp carries H transfers at once (independent chains for the
    // schedulers; one shared-memory read of a point serves all of them).
    for (int Q0 = q0 + warp; Q0 < q1; Q0 += H * nwarp) {
        const int nq = min(H, (q1 - Q0 + nwarp - 1) / nwarp);   // warp-uniform, >= 1
        R cQx[H], sQx[H], cQy[H], sQy[H];
        float2 CQ[H], SQ[H];    // FP32: (cos Q_x, cos Q_y), +-(sin Q_x, sin Q_y) (+ pp, - ph)
        const uint8_t *prow[H];
        int run_b[H];
        R run_v[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int kq = h < nq ? Q0 + h * nwarp : Q0;
            const int Q = A.repQ ? A.repQ[kq] : kq;
            cQx[h] = Qt.cx[Q];
            sQx[h] = Qt.sx[Q];
            cQy[h] = Qt.cy[Q];
            sQy[h] = Qt.sy[Q];
            CQ[h] = make_float2((float)cQx[h], (float)cQy[h]);
            SQ[h] = pp ? make_float2((float)sQx[h], (float)sQy[h]) : make_float2(-(float)sQx[h], -(float)sQy[h]);
            prow[h] = A.part + ((long)fam * NN + Q) * (long)M + (long)a * P;
            run_b[h] = N;
            run_v[h] = R(0);
        }
        for (int ch = 0; ch < lm.nchunk; ++ch) {
            const int s = ch * 32 + sl;
            // rows of this lane in the chunk: t = dt per_chunk + r < n_theta
            const int t0 = dt * lm.per_chunk;
            // FULL: every lane has per_chunk rows (a multiple of 4), read as words
            const int nrow = FULL ? lm.per_chunk : ((s < nr && t0 < nt) ? min(lm.per_chunk, nt - t0) : 0);
            const int li0 = t0 * nr + s;     // staged point of the lane's first row
            // partner bytes of the rows rr .. rr+3 of transfer h as one word
            // (one aligned 4-byte load, coalesced over the warp's radii, where
            // n_theta and the row blocks are multiples of 4), loaded one group ahead
            auto part_word = [&](int h, int rr) -> unsigned {
                if (rr >= nrow || h >= nq) return 0u;
                if (FULL || vec4)
                    return __ldg(reinterpret_cast<const unsigned *>(prow[h] + part_byte(t0 + rr, s, nt, nr)));
                unsigned w = 0u;
                for (int k = 0; k < 4; ++k)
                    if (rr + k < nrow) w |= (unsigned)__ldg(prow[h] + part_byte(t0 + rr + k, s, nt, nr)) << (8 * k);
                return w;
            };
            unsigned wb[H], wn[H];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                wb[h] = part_word(h, 0);
                // a lane's first run starts on its first partner patch: no flush
                // of an empty run (all lanes flushing into one slot at once would
                // serialise the compare-and-swap of the shared float add)
                if (ch == 0 && nrow > 0) run_b[h] = (int)(wb[h] & 255u);
            }
            for (int r = 0; r < lm.per_chunk; r += 4) {
                const int li = li0 + r * stride;
#pragma unroll
                for (int h = 0; h < H; ++h) wn[h] = part_word(h, r + 4);
                int bb[H][4];
#pragma unroll
                for (int h = 0; h < H; ++h)
#pragma unroll
                    for (int k = 0; k < 4; ++k) bb[h][k] = (int)__byte_perm(wb[h], 0u, 0x4440u | k);
                // two rows at a time: the loop kernels of 2 rows x H transfers
                // first (a block of independent arithmetic), then the runs in
                // row order
#pragma unroll
                for (int k0 = 0; k0 < 4; k0 += 2) {
                    R vv[2][H];
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int k = k0 + kk;
                        const bool ok = FULL || r + k < nrow;
                        const int lk = ok ? li + k * stride : 0;
                        const Quad<R> c4 = pc[lk], e4 = pe[lk];
                        if constexpr (sizeof(R) == 4 && TFLOW) {
                            // FP32 temperature flow: transfers h and h + 1 are the two
                            // lanes of packed FP32x2 arithmetic
                            const float2 cp = make_float2(c4.x, c4.y), sp = make_float2(c4.z, c4.w);
#pragma unroll
                            for (int h2 = 0; h2 < H; h2 += 2) {
                                float2 xq2;
#pragma unroll
                                for (int h = h2; h < h2 + 2; ++h) {
                                    // (cos q_x, cos q_y) of the partner by angle addition:
                                    // pp: cos(Q - p) = cQ cp + sQ sp;  ph: cos(p + Q) = cp cQ - sp sQ
                                    const float2 cq = __ffma2_rn(cp, CQ[h], __fmul2_rn(sp, SQ[h]));
                                    float xq = TP0 ? -2.f * t * (cq.x + cq.y) - mu
                                                   : -2.f * t * (cq.x + cq.y) - 4.f * tp * cq.x * cq.y - mu;
                                    if (qp) xq *= Zs[bb[h][k]];
                                    if (h == h2) xq2.x = xq;
                                    else xq2.y = xq;
                                }
                                const float2 v = loop_T2(pp, e4.x, e4.y, e4.w, xq2, invT, invT2, kexp, thrT);
                                vv[kk][h2] = v.x;
                                vv[kk][h2 + 1] = v.y;
                            }
                        } else {
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                const R cqx = pp ? cQx[h] * c4.x + sQx[h] * c4.z : c4.x * cQx[h] - c4.z * sQx[h];
                                const R cqy = pp ? cQy[h] * c4.y + sQy[h] * c4.w : c4.y * cQy[h] - c4.w * sQy[h];
                                // t' = 0 (the nested lattice): the product term drops at compile time
                                R xq = TP0 ? R(-2) * t * (cqx + cqy) - mu
                                           : R(-2) * t * (cqx + cqy) - R(4) * tp * cqx * cqy - mu;
                                if (qp) xq *= Zs[bb[h][k]];
                                vv[kk][h] = e4.w * (tflow ? loop_T(pp, e4.x, e4.y, xq, invT, invT2, kexp, thrT)
                                                          : loop_g(pp, e4.x, e4.y, e4.z, xq, invT, thrT));
                            }
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int k = k0 + kk;
                        if (!FULL && r + k >= nrow) continue;
                        // every transfer slot of the warp updates its run: a slot
                        // past nq (the warp's last pass only) repeats transfer 0
                        // into its own row, which is never written out and is
                        // cleared when the CTA starts
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            const int b = bb[h][k];
                            const bool change = b != run_b[h];
                            row_add_if(&rows[(H * warp + h) * RS + run_b[h]], run_v[h], A.fscale, b, run_b[h]);
                            run_v[h] = (change ? R(0) : run_v[h]) + vv[kk][h];
                            run_b[h] = b;
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < H; ++h) wb[h] = wn[h];
            }
        }
        for (int h = 0; h < nq; ++h) {
            R *row = rows + (H * warp + h) * RS;
            // last runs: segmented sum over lanes with equal partner patch, one
            // atomic per segment head
            const int key = run_b[h];
            const int kup = __shfl_up_sync(0xffffffffu, key, 1);
            const bool head = lane == 0 || kup != key;
            const unsigned heads = __ballot_sync(0xffffffffu, head);
            const unsigned above = lane == 31 ? 0u : heads >> (lane + 1);
            const int end = above ? lane + __ffs(above) - 1 : 31;   // last lane of this segment
            R v = run_v[h];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const R o = __shfl_down_sync(0xffffffffu, v, off);
                if (lane + off <= end) v += o;
            }
            if (head) row_add(&row[key], v, A.fscale);
            __syncwarp();
            const int kq = Q0 + h * nwarp;
            // the row's image rows: (Q', a', g) of the representative, or the
            // row itself (unreduced launch: row Q; representative rows of the
            // contraction's row orbits: row kq of the compact table)
            const int nimg = A.img ? A.nimg[kq] : 1;
            for (int im = 0; im < nimg; ++im) {
                int Qi = kq, ai = a, g = 0;
                if (A.img) {
                    const int2 e = A.img[8 * (long)kq + im];
                    Qi = e.x;
                    ai = e.y & 0xffff;
                    g = e.y >> 16;
                }
                table_row<R, TFLOW>(A, row, Zs, Ks, fam, Qi, ai, g, lane);
            }
            __syncwarp();
            for (int b = lane; b < N; b += 32) row[b] = R(0);
            __syncwarp();
        }
    }
}

template <typename R, bool TP0, int H, bool FULL>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? (H == 2 ? 3 : 2) : 1) bubble_kernel(BubbleArgs<R> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (A.active && *A.active == 0) return;      // uniform over the grid
    const bool tflow = A.pb.regulator == QPFRG_REG_TEMPERATURE;
    int fam, a, q0, q1;
    if (A.tasks) {
        const int4 t = A.tasks[blockIdx.x];
        fam = t.x;
        a = t.y;
        q0 = t.z;
        q1 = t.z + t.w;
    } else {
        const long NN = (long)A.pb.N * A.pb.N;
        fam = blockIdx.z;
        a = blockIdx.x;
        q0 = blockIdx.y * A.qchunk;
        q1 = (int)min((long)q0 + A.qchunk, NN);
    }
    if (fam == 0) {
        if (tflow) bubble_body<R, true, true, TP0, H, FULL>(A, smem_raw, a, q0, q1);
        else bubble_body<R, true, false, TP0, H, FULL>(A, smem_raw, a, q0, q1);
    } else {
        if (tflow) bubble_body<R, false, true, TP0, H, FULL>(A, smem_raw, a, q0, q1);
        else bubble_body<R, false, false, TP0, H, FULL>(A, smem_raw, a, q0, q1);
    }
}

template <typename R>
static qpfrg_status launch_r(qpfrg_ctx *c, double lambda, const double *d_Z, const double *d_K, bool z_symmetric,
                             const FineTable<R> &fine, const TransferTable<R> &qpp, const TransferTable<R> &qph,
                             R thr, bool compact = false)
{
    const Problem &pb = c->pb;
    BubbleArgs<R> A{};
    A.pb = pb;
    A.fine = fine;
    A.qpp = qpp;
    A.qph = qph;
    A.part = c->d_part;
    A.Z = d_Z;
    A.K = d_K;
    A.B = reinterpret_cast<R *>(c->loop_out ? c->loop_out : c->d_B);
    A.active = c->loop_active;
    if (c->opt.precision == QPFRG_MIXED_TC) {
        A.tRT = c->tc.RT;
        A.tKB = c->tc.KB;
    }
    const bool tflow = pb.regulator == QPFRG_REG_TEMPERATURE;
    const double T = tflow ? lambda : pb.T_fixed;
    A.T = (R)T;
    A.invT = (R)(1.0 / T);
    A.g = (R)(tflow ? 1.0 : lambda);
    A.thr = thr;
    // fixed-point scale of the FP32 row accumulators (see row_add)
    const double lmax = tflow ? 0.25 / (T * T) : 0.25 / T;
    const double bin_max = 2.0 * pb.P * c->fw_max * lmax;
    A.fscale = bin_max > 0.0 ? (float)(1073741824.0 / bin_max) : 1.f;
    A.finv = 1.f / A.fscale;
    A.t = (R)pb.t;
    A.tp = (R)pb.tp;
    A.mu = (R)pb.mu;
    const long NN = (long)pb.N * pb.N;
    // transfers per CTA: 8 per warp where the grid still fills the GPU
    A.qchunk = c->tune.bubble_qchunk > 0 ? (int)std::min<long>(c->tune.bubble_qchunk, NN)
                                         : (int)std::max(8L, std::min(64L, NN / 16));
    const int qchunks = div_up(NN, A.qchunk);
    // C4v-reduced launch: one row per orbit (the Z-free loop kernels of
    // quasi-particle lines depend on Z, which must then be symmetric)
    const bool red = c->loop_red && (pb.propagator == QPFRG_PROP_PAPER || z_symmetric);
    int ntask = 0;
    if (compact) {
        // representative rows of the contraction's row orbits, all patches a
        A.qchunk = std::max(8, A.qchunk);
        qpfrg_status st = row_tasks(c, A.qchunk, &ntask);
        if (st != QPFRG_OK) return st;
        A.tasks = c->d_rtask;
        A.repQ = c->d_rrep;
    } else if (red) {
        qpfrg_status st = loop_tasks(c, A.qchunk, &ntask);
        if (st != QPFRG_OK) return st;
        A.tasks = c->d_ltask;
        A.repQ = c->d_lrepQ;
        A.nimg = c->d_lnimg;
        A.img = c->d_limg;
    }
    // transfers per warp pass: 4 only in FP32 (the packed pairs of the
    // temperature flow), 2 otherwise or when tuned so
    const int H = (sizeof(R) == 4 && c->tune.bubble_transfers == 4) ? 4 : 2;
    const int nthr = 256;
    const size_t smem = 2 * (size_t)pb.P * sizeof(Quad<R>) +
                        (2 * (size_t)pb.N + (size_t)H * (nthr / 32) * (size_t)(pb.N + 2)) * sizeof(R);
    if (smem > 200 * 1024) {
        c->err = "fine grid too large for the loop-kernel launch";
        return QPFRG_ERR_UNSUPPORTED;
    }
    // every lane with the same whole number of 4-row groups: no per-row bounds tests
    const LaneMap lm(pb.n_theta, pb.n_r);
    const bool full = pb.n_theta % 4 == 0 && lm.per_chunk % 4 == 0 &&
                      (pb.n_r >= 32 ? pb.n_r % 32 == 0 : (lm.lr == pb.n_r && pb.n_theta % lm.apr == 0));
    void (*kern)(BubbleArgs<R>) = pb.tp == 0.0 ? bubble_kernel<R, true, 2, false> : bubble_kernel<R, false, 2, false>;
    if (full) kern = pb.tp == 0.0 ? bubble_kernel<R, true, 2, true> : bubble_kernel<R, false, 2, true>;
    if constexpr (sizeof(R) == 4)
        if (H == 4) kern = pb.tp == 0.0 ? bubble_kernel<R, true, 4, false> : bubble_kernel<R, false, 4, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(c, e, "bubble smem attribute");
    const dim3 grid = (compact || red) ? dim3(ntask) : dim3(pb.N, qchunks, 2);
    prof_begin(c);
    kern<<<grid, nthr, smem, c->stream>>>(A);
    prof_end(c, K_BUBBLE);
    e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "bubble_kernel");
}

// Width of the near-degenerate window |x_p -+ x_q| < thr T (midpoint
// derivative instead of the difference quotient).  The quotient loses about
// eps / thr of relative accuracy to cancellation, the midpoint derivative is
// off by about thr^2 / 24 (times the loop kernel's third derivative in units
// of T); the two balance near thr = eps^(1/3): 1e-5 in FP64, 6e-3 in FP32
// (eps of the FP32 loop kernel ~3e-7 with ex2.approx).
constexpr double kThrF64 = 1e-5;
constexpr float kThrF32 = 6e-3f;

qpfrg_status launch_bubbles(qpfrg_ctx *c, double lambda, const double *d_Z, bool z_symmetric, const double *d_K,
                            bool state_symmetric)
{
    c->rows_compact = false;
    if (c->opt.precision == QPFRG_FP64)
        return launch_r<double>(c, lambda, d_Z, d_K, z_symmetric, c->f64, c->qpp64, c->qph64, kThrF64);
    if (c->opt.precision == QPFRG_MIXED_TC) {
        qpfrg_status s = launch_tc_prep(c);       // B operands and V^T of this stage
        if (s != QPFRG_OK) return s;
    }
    const bool compact = c->rows_ok && state_symmetric && c->opt.precision == QPFRG_MIXED_TC;
    const qpfrg_status s =
        launch_r<float>(c, lambda, d_Z, d_K, z_symmetric, c->f32, c->qpp32, c->qph32, kThrF32, compact);
    c->rows_compact = compact && s == QPFRG_OK;
    return s;
}

// The loop kernel alone into an explicit buffer (batched flows): the table
// B[f][Q][a][b] at Lambda with Z = 1 (compact: the representative rows of the
// row orbits); every CTA returns at once when *active == 0.  No vertex
// operands are prepared.
qpfrg_status launch_loop_rows(qpfrg_ctx *c, double lambda, float *rows, const int *active, bool compact)
{
    c->loop_out = rows;
    c->loop_active = active;
    const qpfrg_status s =
        launch_r<float>(c, lambda, c->d_ones, nullptr, true, c->f32, c->qpp32, c->qph32, kThrF32, compact && c->rows_ok);
    c->loop_out = nullptr;
    c->loop_active = nullptr;
    return s;
}

}  // namespace qpfrg
