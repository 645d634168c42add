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
// Launch shape: one CTA per (patch a, chunk of Q, family).  The CTA keeps its
// wedge's fine points in registers (PPT consecutive radial points per
// thread), streams the partner-patch bytes of each Q (coalesced), merges
// equal consecutive partners in registers and adds runs into shared-memory
// rows of N accumulators, G transfers per barrier, double-buffered.
#include <cuda_bf16.h>

#include <algorithm>

#include "qpfrg_internal.h"

namespace qpfrg {

constexpr int G = 2;   // transfers per barrier

template <typename R>
struct BubbleArgs {
    Problem pb;
    FineTable<R> fine;
    TransferTable<R> qpp, qph;
    const uint8_t *part;
    const double *Z;
    R *B;
    R T, invT, g, thr;
    R t, tp, mu;          // hoppings and chemical potential, already in R (no per-use conversion)
    int qchunk;
    // formed operands of the tensor-core contraction (QPFRG_MIXED_TC)
    const float *Vf;            // stage vertex, FP32 [k1][k2][k3]
    const float *VT;            // VT[j][l][b] = V[b][j][l]
    __nv_bfloat16 *App[2];      // [N^2][N^2]   hi, lo: B_pp[Q][a][b] V[Q][a]
    __nv_bfloat16 *Acr[2];      // [N^2][N^2]   row (j,l) of Q = (l,j): B_ph[Q][a][b] V[b][j][l]
    __nv_bfloat16 *Ad[2];       // [N^2][2N^2]  B_ph[Q][a][b] (2V[i,a,l] - V[a,i,l]) | -B_ph V[i,a,l]
};

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// ---- scalar helpers ---------------------------------------------------------
__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
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
__device__ __forceinline__ R loop_T(bool pp, R xp, R gp, R xq, R invT, R thrT)
{
    const R den = pp ? xp + xq : xp - xq;
    if (qabs(den) < thrT) {
        const R m = R(0.5) * (pp ? xp - xq : xp + xq);
        const R v = fermi_dxdT(m, invT);
        return pp ? -v : v;
    }
    const R e = fexp(-qabs(xq) * invT);
    const R d = R(1) + e, d2 = d * d;
    const R gq_num = xq * invT * invT * e;           // g_q * d2
    const R num = pp ? gp * d2 + gq_num : gp * d2 - gq_num;
    const R v = fdiv(num, d2 * den);
    return pp ? -v : v;
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

// Kernel body for one transfer family (PP: particle-particle, else
// particle-hole) and one regulator (TFLOW: temperature flow, else
// interaction flow), both fixed at compile time.
template <typename R, int PPT, bool FORM, bool PP, bool TFLOW>
__device__ __forceinline__ void bubble_body(const BubbleArgs<R> &A, unsigned char *smem_raw)
{
    const int N = A.pb.N, P = A.pb.P, M = A.pb.M;
    const long NN = (long)N * N;
    const int a = blockIdx.x;
    const int fam = PP ? 0 : 1;
    constexpr bool pp = PP;
    const int q0 = blockIdx.y * A.qchunk;
    const int q1 = min((long)q0 + A.qchunk, NN);
    const int tid = threadIdx.x, nthr = blockDim.x;
    constexpr bool tflow = TFLOW;
    const bool qp = A.pb.propagator == QPFRG_PROP_QP;

    R *acc = reinterpret_cast<R *>(smem_raw);  // 2 x G x N
    R *Zs = acc + 2 * G * N;                   // N
    for (int i = tid; i < 2 * G * N; i += nthr) acc[i] = R(0);
    for (int i = tid; i < N; i += nthr) Zs[i] = A.Z ? (R)A.Z[i] : R(1);
    __syncthreads();
    const R Za = Zs[a];
    const R invT = A.invT, thrT = A.thr * A.T;
    const R t = A.t, tp = A.tp, mu = A.mu;

    // This thread's fine points: PPT consecutive angular points at one radius,
    // local index (t0 + u) n_r + s with s = tid % n_r, t0 = (tid / n_r) PPT.
    // Partners of angular neighbours are ~0.004 rad apart and mostly share a
    // patch, so runs are long (few shared-memory atomics, which are CAS loops
    // for floats), and the lanes of a warp sit at different radii (few
    // conflicts).  Partner bytes of one u are contiguous across the lanes.
    const int nr = A.pb.n_r, nt = A.pb.n_theta;
    const int s_r = tid % nr, t0 = (tid / nr) * PPT;
    R pcx[PPT], psx[PPT], pcy[PPT], psy[PPT], px[PPT], pw[PPT], pa[PPT], pb2[PPT];
    bool valid[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        const int loc = (t0 + u) * nr + s_r;
        valid[u] = t0 + u < nt;
        const int p = a * P + (valid[u] ? loc : 0);
        pcx[u] = A.fine.cx[p];
        psx[u] = A.fine.sx[p];
        pcy[u] = A.fine.cy[p];
        psy[u] = A.fine.sy[p];
        pw[u] = valid[u] ? A.fine.w[p] : R(0);
        px[u] = qp ? Za * A.fine.xi[p] : A.fine.xi[p];
        if (tflow) {
            pa[u] = fermi_dT(px[u], invT);
            pb2[u] = R(0);
        } else {
            fermi_pair(px[u], invT, pa[u], pb2[u]);
        }
    }
    const bool any_valid = t0 < nt;
    const TransferTable<R> &Qt = pp ? A.qpp : A.qph;

    // Q's are processed in groups of G: the G x PPT partner loads are issued
    // together, runs are added into G shared rows, one barrier per group.
    for (int Qb = q0; Qb < q1; Qb += G) {
        R *accb = acc + (((Qb - q0) / G) & 1) * (G * N);
        if (any_valid) {
            int bq[G][PPT];
            R cQx[G], sQx[G], cQy[G], sQy[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int Q = min(Qb + g, q1 - 1);
                const uint8_t *row = A.part + ((long)fam * NN + Q) * (long)M + (long)a * P + s_r;
#pragma unroll
                for (int u = 0; u < PPT; ++u) bq[g][u] = valid[u] ? row[(t0 + u) * nr] : 0;
                cQx[g] = Qt.cx[Q];
                sQx[g] = Qt.sx[Q];
                cQy[g] = Qt.cy[Q];
                sQy[g] = Qt.sy[Q];
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (Qb + g >= q1) break;
                R *row = accb + g * N;
                int run_b = -1;
                R run_v = R(0);
#pragma unroll
                for (int u = 0; u < PPT; ++u) {
                    if (!valid[u]) continue;
                    // cos of the partner momentum components by angle addition:
                    // pp: cos(Q - p) = cQ cp + sQ sp;  ph: cos(p + Q) = cp cQ - sp sQ
                    const R cqx = pp ? cQx[g] * pcx[u] + sQx[g] * psx[u] : pcx[u] * cQx[g] - psx[u] * sQx[g];
                    const R cqy = pp ? cQy[g] * pcy[u] + sQy[g] * psy[u] : pcy[u] * cQy[g] - psy[u] * sQy[g];
                    R xq = R(-2) * t * (cqx + cqy) - R(4) * tp * cqx * cqy - mu;
                    const int b = bq[g][u];
                    if (qp) xq *= Zs[b];
                    const R v = pw[u] * (tflow ? loop_T(pp, px[u], pa[u], xq, invT, thrT)
                                               : loop_g(pp, px[u], pa[u], pb2[u], xq, invT, thrT));
                    if (b == run_b) {
                        run_v += v;
                    } else {
                        if (run_b >= 0) atomicAdd(&row[run_b], run_v);
                        run_b = b;
                        run_v = v;
                    }
                }
                if (run_b >= 0) atomicAdd(&row[run_b], run_v);
            }
        }
        __syncthreads();
#pragma unroll
        for (int g = 0; g < G; ++g)
        for (int b = tid; b < N; b += nthr) {
            const int idx = g * N + b;
            const int Q = Qb + g;
            const R v = accb[idx];
            accb[idx] = R(0);
            if (Q < q1) {
                const R Zb = Zs[b];
                const R s = tflow ? Za * Zb : A.g * Za * Zb * (Za + Zb);
                if constexpr (!FORM) {
                    A.B[(((long)fam * NN + Q) * N + a) * (long)N + b] = v * s;
                } else {
                    const float bt = (float)(v * s);
                    const long col = (long)a * N + b;
                    __nv_bfloat16 h, l;
                    if (pp) {
                        split_bf16(bt * A.Vf[(long)Q * N + a], h, l);
                        A.App[0][(long)Q * NN + col] = h;
                        A.App[1][(long)Q * NN + col] = l;
                    } else {
                        const int x = Q / N, y = Q - (Q / N) * N;          // Q = k_F(x) - k_F(y)
                        const long rcr = (long)y * N + x;                 // cr row (j,l) = (y,x)
                        split_bf16(bt * A.VT[rcr * N + b], h, l);
                        A.Acr[0][rcr * NN + col] = h;
                        A.Acr[1][rcr * NN + col] = l;
                        const float v_ial = A.Vf[((long)x * N + a) * N + y];
                        const float v_ail = A.Vf[((long)a * N + x) * N + y];
                        split_bf16(bt * (2.f * v_ial - v_ail), h, l);
                        A.Ad[0][(long)Q * 2 * NN + col] = h;
                        A.Ad[1][(long)Q * 2 * NN + col] = l;
                        split_bf16(-bt * v_ial, h, l);
                        A.Ad[0][(long)Q * 2 * NN + NN + col] = h;
                        A.Ad[1][(long)Q * 2 * NN + NN + col] = l;
                    }
                }
            }
        }
    }
}

// FP32 variants with up to 4 points per thread fit 3 CTAs of 256 threads per SM
template <typename R, int PPT>
struct BubbleMinBlocks {
    static constexpr int value = (sizeof(R) == 4 && PPT <= 4) ? 3 : 1;
};

template <typename R, int PPT, bool FORM>
__global__ void __launch_bounds__(256, BubbleMinBlocks<R, PPT>::value) bubble_kernel(BubbleArgs<R> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool tflow = A.pb.regulator == QPFRG_REG_TEMPERATURE;
    if (blockIdx.z == 0) {
        if (tflow) bubble_body<R, PPT, FORM, true, true>(A, smem_raw);
        else bubble_body<R, PPT, FORM, true, false>(A, smem_raw);
    } else {
        if (tflow) bubble_body<R, PPT, FORM, false, true>(A, smem_raw);
        else bubble_body<R, PPT, FORM, false, false>(A, smem_raw);
    }
}

template <typename R, int PPT, bool FORM>
static void launch_t(qpfrg_ctx *c, const BubbleArgs<R> &A, int nthr, int qchunks)
{
    const int N = c->pb.N;
    dim3 grid(N, qchunks, 2);
    const size_t smem = (2 * G + 1) * (size_t)N * sizeof(R);
    bubble_kernel<R, PPT, FORM><<<grid, nthr, smem, c->stream>>>(A);
}

template <typename R, bool FORM>
static qpfrg_status launch_r(qpfrg_ctx *c, double lambda, const double *d_Z, const FineTable<R> &fine,
                             const TransferTable<R> &qpp, const TransferTable<R> &qph, R thr)
{
    const Problem &pb = c->pb;
    BubbleArgs<R> A{};
    A.pb = pb;
    A.fine = fine;
    A.qpp = qpp;
    A.qph = qph;
    A.part = c->d_part;
    A.Z = d_Z;
    A.B = reinterpret_cast<R *>(c->d_B);
    A.Vf = c->d_Vf;
    A.VT = c->tc.VT;
    for (int h = 0; h < 2; ++h) {
        A.App[h] = c->tc.App[h];
        A.Acr[h] = c->tc.Acr[h];
        A.Ad[h] = c->tc.Ad[h];
    }
    const bool tflow = pb.regulator == QPFRG_REG_TEMPERATURE;
    const double T = tflow ? lambda : pb.T_fixed;
    A.T = (R)T;
    A.invT = (R)(1.0 / T);
    A.g = (R)(tflow ? 1.0 : lambda);
    A.thr = thr;
    A.t = (R)pb.t;
    A.tp = (R)pb.tp;
    A.mu = (R)pb.mu;
    const long NN = (long)pb.N * pb.N;
    A.qchunk = (int)std::max(1L, std::min(64L, NN / 16));
    const int qchunks = div_up(NN, A.qchunk);

    const int P = pb.P;
    int ppt = (P + 255) / 256;
    if (ppt > 8) {
        c->err = "more than 2048 fine points per patch are not supported";
        return QPFRG_ERR_UNSUPPORTED;
    }
    ppt = ppt <= 1 ? 1 : (ppt <= 2 ? 2 : (ppt <= 4 ? 4 : 8));
    // threads: n_r radii x ceil(n_theta / PPT) angular chunks
    int nthr = pb.n_r * ((pb.n_theta + ppt - 1) / ppt);
    nthr = std::max(32, ((nthr + 31) / 32) * 32);
    if (nthr > 256) {
        c->err = "fine grid too large for the loop-kernel launch";
        return QPFRG_ERR_UNSUPPORTED;
    }
    prof_begin(c);
    switch (ppt) {
    case 1: launch_t<R, 1, FORM>(c, A, nthr, qchunks); break;
    case 2: launch_t<R, 2, FORM>(c, A, nthr, qchunks); break;
    case 4: launch_t<R, 4, FORM>(c, A, nthr, qchunks); break;
    default: launch_t<R, 8, FORM>(c, A, nthr, qchunks); break;
    }
    prof_end(c, K_BUBBLE);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "bubble_kernel");
}

qpfrg_status launch_bubbles(qpfrg_ctx *c, double lambda, const double *d_Z)
{
    if (c->opt.precision == QPFRG_FP64)
        return launch_r<double, false>(c, lambda, d_Z, c->f64, c->qpp64, c->qph64, 1e-5);
    if (c->opt.precision == QPFRG_MIXED_TC) {
        qpfrg_status s = launch_tc_prep(c);       // B operands and V^T of this stage
        if (s != QPFRG_OK) return s;
        return launch_r<float, true>(c, lambda, d_Z, c->f32, c->qpp32, c->qph32, 2e-2f);
    }
    return launch_r<float, false>(c, lambda, d_Z, c->f32, c->qpp32, c->qph32, 2e-2f);
}

}  // namespace qpfrg
