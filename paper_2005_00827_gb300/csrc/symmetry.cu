// C4v orbits of the loop-kernel rows (wedge and shell modes).
//
// The point group C4v of the square lattice acts on the wedges as
// g = (m, s): w -> s w + m N_a/4 (mod N_a), s = +-1, and leaves the energy
// shells in place (patch j = w n_s + s -> (g w) n_s + s), on the transfers
// Q = (x, y) (Q = k_F(x) +- k_F(y)) as (x, y) -> (g x, g y), and on the fine
// points of a patch as (a, t, r) -> (g a, t, r) for the rotations and
// (g a, n_theta - 1 - t, r) for the reflections.  The dispersion (Eq.
// (free_dispersion_xi)) and the quadrature weights are invariant, and where
// the patch projection is covariant, proj(g k) = g proj(k), the Z-free binned
// loop kernels satisfy
//     B_f[g Q][g a][g b] = B_f[Q][a][b].
// So one row per orbit of (Q, a) is evaluated and written to every image,
// its columns permuted by g (the Z weights and vertex factors are applied per
// image).  Covariance is not assumed: check_covariance_kernel compares every
// image row of the partner maps with its representative's row, byte by byte,
// and a row that differs anywhere is evaluated by itself.
//
// When every row is covariant and V and Z are C4v symmetric, each channel's
// output is invariant as well, dV_ch(g k1, g k2, g k3) = dV_ch(k1, k2, k3), so
// the tensor-core contraction needs one output row per orbit of transfer pairs
// Q only (build_row_orbits: representatives, and per pair Q its
// representative and the g with Q = g rep); contract.cu expands the rows.
#include <algorithm>
#include <cstring>
#include <vector>

#include "qpfrg_internal.h"

namespace qpfrg {

// flag[f][Q N + a] = 1 where the partner-map row (f, Q, a) is not the image
// of its representative's row under g.  rep[Q N + a] = representative's Q N + a,
// gof[Q N + a] = g with (Q, a) = g (representative).
__global__ void check_covariance_kernel(const uint8_t *__restrict__ part, const int *__restrict__ rep,
                                        const uint8_t *__restrict__ gof, uint8_t *__restrict__ flag, int N, int M,
                                        int P, int nt, int nr, int ns)
{
    const int Q = blockIdx.x, f = blockIdx.y;
    const long NN = (long)N * N;
    __shared__ int bad;
    for (int a = 0; a < N; ++a) {
        const long row = (long)Q * N + a;
        const int r = rep[row];
        if (r == row) continue;                    // uniform over the block
        const int g = gof[row];
        const int Qr = r / N, ar = r - Qr * N;
        const uint8_t *src = part + ((long)f * NN + Qr) * (long)M + (long)ar * P;
        const uint8_t *dst = part + ((long)f * NN + Q) * (long)M + (long)a * P;
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        int mine = 0;
        for (int li = threadIdx.x; li < P; li += blockDim.x) {
            const int t = li / nr, s = li - t * nr;
            const int ts = (g & 4) ? nt - 1 - t : t;   // the representative's point mapped onto (t, s)
            const int want = c4v_apply(g, src[part_byte(ts, s, nt, nr)], N, ns);
            if (dst[part_byte(t, s, nt, nr)] != want) mine = 1;
        }
        if (mine) bad = 1;
        __syncthreads();
        if (threadIdx.x == 0) flag[(long)f * NN * N + row] = (uint8_t)bad;
        __syncthreads();
    }
}

// Row orbits of the tensor-core contraction: the representative of the
// transfer pair Q = (x, y) is its image g Q = (g x, g y) with the smallest
// index; rowmap[Q] = (representative index | g << 24) with Q = g rep.  Only
// built when every loop-kernel row passed the covariance check, so that the
// table rows of the images are exactly the representative's, permuted.
static qpfrg_status build_row_orbits(qpfrg_ctx *c)
{
    const int N = c->pb.N, ns = c->pb.n_shell;
    const long NN = (long)N * N;
    std::vector<int> repidx(NN, -1), reps, rowmap(NN);
    // in increasing Q the representative (the orbit's smallest index, <= Q)
    // is always met first
    for (long Q = 0; Q < NN; ++Q) {
        const int x = (int)(Q / N), y = (int)(Q - (long)x * N);
        long best = -1;
        int bg = 0;
        for (int g = 0; g < 8; ++g) {
            const long gQ = (long)c4v_apply(g, x, N, ns) * N + c4v_apply(g, y, N, ns);
            if (best < 0 || gQ < best) {
                best = gQ;
                bg = g;
            }
        }
        if (best == Q) {
            repidx[Q] = (int)reps.size();
            reps.push_back((int)Q);
        }
        // bg maps Q onto its representative: Q = bg^-1 rep
        rowmap[Q] = repidx[best] | (c4v_inverse(bg) << 24);
    }
    const int nr = (int)reps.size();
    cudaError_t e;
    if ((e = cudaMalloc((void **)&c->d_rrep, nr * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_rowmap, NN * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_rtask, (2L * N * ((nr + 7) / 8) + 8) * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_outc, 3L * nr * N * sizeof(double))) != cudaSuccess)
        return cuda_fail(c, e, "cudaMalloc(row orbits)");
    e = cudaMemcpy(c->d_rrep, reps.data(), nr * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_rowmap, rowmap.data(), NN * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload row orbits");
    c->n_rrep = nr;
    c->rtask_qchunk = 0;
    c->loop_evals_rows = 2LL * nr * c->pb.M;
    c->rows_ok = true;
    return QPFRG_OK;
}

qpfrg_status build_loop_orbits(qpfrg_ctx *c)
{
    c->loop_red = false;
    if ((c->pb.mode != QPFRG_GRID_WEDGE && c->pb.mode != QPFRG_GRID_SHELL) ||
        (c->opt.no_loop_symmetry != 0 && c->opt.no_loop_symmetry != 2))
        return QPFRG_OK;
    const int N = c->pb.N, ns = c->pb.n_shell;
    if ((N / ns) % 4 != 0) return QPFRG_OK;
    const long NN = (long)N * N, rows = NN * N;
    // canonical representative of every (Q, a): the image with the smallest
    // (a, Q); its patch lies in the fundamental domain 0..N/8
    std::vector<int> rep(rows);
    std::vector<uint8_t> gof(rows);
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
            for (int a = 0; a < N; ++a) {
                long best = -1;
                int bg = 0;
                for (int g = 0; g < 8; ++g) {
                    const long ga = c4v_apply(g, a, N, ns);
                    const long gQ = (long)c4v_apply(g, x, N, ns) * N + c4v_apply(g, y, N, ns);
                    const long key = ga * NN + gQ;
                    if (best < 0 || key < best) {
                        best = key;
                        bg = g;
                    }
                }
                const long ra = best / NN, rQ = best - ra * NN;
                const long row = ((long)x * N + y) * N + a;
                rep[row] = (int)(rQ * N + ra);
                gof[row] = (uint8_t)c4v_inverse(bg);    // (Q, a) = g^-1 applied to the representative
            }
    int *d_rep = nullptr;
    uint8_t *d_g = nullptr, *d_flag = nullptr;
    auto release = [&]() {
        cudaFree(d_rep);
        cudaFree(d_g);
        cudaFree(d_flag);
    };
    cudaError_t e;
    if ((e = cudaMalloc((void **)&d_rep, rows * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&d_g, rows)) != cudaSuccess || (e = cudaMalloc((void **)&d_flag, 2 * rows)) != cudaSuccess) {
        release();
        return cuda_fail(c, e, "cudaMalloc(loop orbits)");
    }
    std::vector<uint8_t> flag(2 * rows);
    e = cudaMemcpyAsync(d_rep, rep.data(), rows * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_g, gof.data(), rows, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flag, 0, 2 * rows, c->stream);
    if (e == cudaSuccess) {
        check_covariance_kernel<<<dim3((unsigned)NN, 2), 256, 0, c->stream>>>(c->d_part, d_rep, d_g, d_flag, N, c->pb.M,
                                                                          c->pb.P, c->pb.n_theta, c->pb.n_r, ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), d_flag, 2 * rows, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    release();
    if (e != cudaSuccess) return cuda_fail(c, e, "partner-map covariance check");

    // representatives per family grouped by patch, each with its images;
    // rows whose partner bytes broke covariance are representatives of themselves
    struct Rep {
        int a, Q, n;
        int2 img[8];
    };
    std::vector<Rep> reps[2];
    long mism = 0;
    for (int f = 0; f < 2; ++f) {
        const uint8_t *fl = flag.data() + (long)f * rows;
        for (long row = 0; row < rows; ++row) {
            const int Q = (int)(row / N), a = (int)(row - (long)Q * N);
            if (fl[row]) {
                ++mism;
                Rep r{a, Q, 1, {}};
                r.img[0] = make_int2(Q, a);
                reps[f].push_back(r);
                continue;
            }
            if (rep[row] != row) continue;
            Rep r{a, Q, 0, {}};
            const int x = Q / N, y = Q - x * N;
            for (int g = 0; g < 8; ++g) {
                const int Qi = c4v_apply(g, x, N, ns) * N + c4v_apply(g, y, N, ns), ai = c4v_apply(g, a, N, ns);
                const long irow = (long)Qi * N + ai;
                if (fl[irow]) continue;                // evaluated by itself
                bool dup = false;
                for (int k = 0; k < r.n; ++k) dup |= r.img[k].x == Qi && (r.img[k].y & 0xffff) == ai;
                if (!dup) r.img[r.n++] = make_int2(Qi, ai | (g << 16));
            }
            reps[f].push_back(r);
        }
        std::stable_sort(reps[f].begin(), reps[f].end(), [](const Rep &u, const Rep &v) { return u.a < v.a; });
    }
    const long nrep = (long)reps[0].size() + (long)reps[1].size();
    std::vector<int> hQ(nrep), hn(nrep);
    std::vector<int2> himg(8 * nrep, make_int2(0, 0));
    c->lgroups.clear();
    long k = 0, evals = 0;
    for (int f = 0; f < 2; ++f) {
        long start = k;
        for (size_t i = 0; i < reps[f].size(); ++i, ++k) {
            const Rep &r = reps[f][i];
            hQ[k] = r.Q;
            hn[k] = r.n;
            for (int m = 0; m < r.n; ++m) himg[8 * k + m] = r.img[m];
            evals += c->pb.P;
            const bool last = i + 1 == reps[f].size() || reps[f][i + 1].a != r.a;
            if (last) {
                c->lgroups.push_back({f, r.a, (int)start, (int)(k + 1 - start)});
                start = k + 1;
            }
        }
    }
    if ((e = cudaMalloc((void **)&c->d_lrepQ, nrep * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_lnimg, nrep * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_limg, 8 * nrep * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc((void **)&c->d_ltask, (nrep + 2 * (long)N + 8) * sizeof(int4))) != cudaSuccess)
        return cuda_fail(c, e, "cudaMalloc(loop representatives)");
    e = cudaMemcpy(c->d_lrepQ, hQ.data(), nrep * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_lnimg, hn.data(), nrep * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_limg, himg.data(), 8 * nrep * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload loop representatives");
    c->n_lrep = nrep;
    c->ltask_qchunk = 0;
    c->loop_evals_red = evals;
    c->loop_mismatch_rows = mism;
    c->loop_red = true;
    if (mism == 0 && c->opt.precision == QPFRG_MIXED_TC && c->opt.no_loop_symmetry == 0)
        return build_row_orbits(c);
    return QPFRG_OK;
}

// Tasks of the reduced loop-kernel launch for a chunk size: (family, patch,
// first representative, count) per CTA; rebuilt when the chunk size changes.
qpfrg_status loop_tasks(qpfrg_ctx *c, int qchunk, int *ntask)
{
    if (c->ltask_qchunk == qchunk) {
        *ntask = c->n_ltask;
        return QPFRG_OK;
    }
    std::vector<int4> t;
    for (const LoopGroup &g : c->lgroups)
        for (int s = 0; s < g.count; s += qchunk) t.push_back(make_int4(g.fam, g.a, g.start + s, std::min(qchunk, g.count - s)));
    if ((long)t.size() > c->n_lrep + 2L * c->pb.N + 8) {
        c->err = "loop-kernel task list overflow";
        return QPFRG_ERR_INVALID;
    }
    cudaError_t e = cudaMemcpyAsync(c->d_ltask, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload loop tasks");
    c->ltask_qchunk = qchunk;
    c->n_ltask = (int)t.size();
    *ntask = c->n_ltask;
    return QPFRG_OK;
}

// Tasks of the loop-kernel launch on representative rows: (family, patch,
// first representative, count) per CTA, chunks of qchunk rows (qchunk >= 8).
qpfrg_status row_tasks(qpfrg_ctx *c, int qchunk, int *ntask)
{
    if (c->rtask_qchunk == qchunk) {
        *ntask = c->n_rtask;
        return QPFRG_OK;
    }
    if (qchunk < 8) {
        c->err = "row tasks: chunk below 8 rows";
        return QPFRG_ERR_INVALID;
    }
    std::vector<int4> t;
    for (int f = 0; f < 2; ++f)
        for (int a = 0; a < c->pb.N; ++a)
            for (int s0 = 0; s0 < c->n_rrep; s0 += qchunk) t.push_back(make_int4(f, a, s0, std::min(qchunk, c->n_rrep - s0)));
    cudaError_t e = cudaMemcpyAsync(c->d_rtask, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "upload row tasks");
    c->rtask_qchunk = qchunk;
    c->n_rtask = (int)t.size();
    *ntask = c->n_rtask;
    return QPFRG_OK;
}

}  // namespace qpfrg

extern "C" qpfrg_status qpfrg_sigma_table(qpfrg_t c, size_t *bytes, long long offset, long long count,
                                          unsigned char *h_out)
{
    if (!c) return QPFRG_ERR_INVALID;
    const size_t size = c->d_rtab ? (size_t)c->n_irr * c->pb.N * (size_t)c->pb.M * (size_t)c->pb.P : 0;
    if (bytes) *bytes = size;
    if (!h_out) return QPFRG_OK;
    if (offset < 0 || count < 0 || (size_t)offset + (size_t)count > size) {
        c->err = "qpfrg_sigma_table: range outside the table";
        return QPFRG_ERR_INVALID;
    }
    cudaError_t e = cudaMemcpyAsync(h_out, c->d_rtab + offset, (size_t)count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? QPFRG_OK : qpfrg::cuda_fail(c, e, "qpfrg_sigma_table");
}

extern "C" qpfrg_status qpfrg_rhs_work(qpfrg_t c, long long *loop_evals, long long *loop_evals_full,
                                       long long *rows_unreduced, long long *contraction_rows)
{
    if (!c) return QPFRG_ERR_INVALID;
    const long long full = 2LL * c->pb.N * c->pb.N * c->pb.M;
    if (loop_evals) *loop_evals = c->rows_compact ? c->loop_evals_rows : (c->loop_red ? c->loop_evals_red : full);
    if (loop_evals_full) *loop_evals_full = full;
    if (rows_unreduced) *rows_unreduced = c->loop_red ? c->loop_mismatch_rows : 0;
    if (contraction_rows) *contraction_rows = c->rows_compact ? c->n_rrep : (long long)c->pb.N * c->pb.N;
    return QPFRG_OK;
}
