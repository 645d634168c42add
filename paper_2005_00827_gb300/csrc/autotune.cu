// Launch-shape autotuner (qpfrg_autotune, qpfrg_set_tuning).
//
// The hot kernels have schedule parameters that do not change results beyond
// the order of floating-point sums: transfers per loop-kernel CTA, q blocks
// per self-energy CTA, split-K of the tensor-core contraction.  Their best
// values depend on N_p, the fine grid and the part, so they are measured:
// each candidate runs once untimed and once between CUDA events on the
// context's stream, on the context's own state, and the fastest is kept.
#include <cmath>

#include "qpfrg_internal.h"

using namespace qpfrg;

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    EventPair()
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// ms of the second of two runs of `launch`; negative (and st set) on failure
template <typename F>
double time_launch(qpfrg_ctx *c, EventPair &ev, F &&launch, qpfrg_status &st)
{
    if ((st = launch()) != QPFRG_OK) return -1.0;
    cudaEventRecord(ev.a, c->stream);
    if ((st = launch()) != QPFRG_OK) return -1.0;
    cudaEventRecord(ev.b, c->stream);
    cudaError_t e = cudaEventSynchronize(ev.b);
    if (e != cudaSuccess) {
        st = cuda_fail(c, e, "autotune timing");
        return -1.0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    return ms;
}

}  // namespace

extern "C" qpfrg_status qpfrg_autotune(qpfrg_t c, double lambda, qpfrg_tuning *out)
{
    if (!c) return QPFRG_ERR_INVALID;
    const bool tflow = c->pb.regulator == QPFRG_REG_TEMPERATURE;
    if (!std::isfinite(lambda) || (tflow && !(lambda > 0.0))) {
        c->err = "lambda must be finite (and T > 0)";
        return QPFRG_ERR_INVALID;
    }
    const bool prof = c->prof;
    c->prof = false;    // tuning launches are not part of any profile
    EventPair ev;
    qpfrg_status st = QPFRG_OK;
    const long N = c->pb.N, NN = N * N, n3 = NN * N;
    const bool mixed = c->opt.precision != QPFRG_FP64;
    const void *Vin = c->d_V;
    double best_b = 0.0, best_s = 0.0, best_c = 0.0;
    do {
        if (mixed) {
            if ((st = launch_convert_f32(c, c->d_V, c->d_Vf, n3)) != QPFRG_OK) break;
            Vin = c->d_Vf;
        }
        // loop kernels: transfers per CTA and per warp pass (4 only in FP32)
        {
            const int cand[] = {8, 16, 32, 64, 128, 256};
            int pick = 0, pick_h = 2;
            double best = 1e300;
            for (int hw = 2; hw <= (mixed ? 4 : 2) && st == QPFRG_OK; hw += 2)
                for (int q : cand) {
                    if (q > NN && q != cand[0]) break;
                    c->tune.bubble_qchunk = q;
                    c->tune.bubble_transfers = hw;
                    const double ms = time_launch(
                        c, ev,
                        [&] { return launch_bubbles(c, lambda, c->d_Z, c->c4v_state, nullptr, c->c4v_state); }, st);
                    if (ms < 0.0) break;
                    if (ms < best) {
                        best = ms;
                        pick = q;
                        pick_h = hw;
                    }
                }
            if (st != QPFRG_OK) break;
            c->tune.bubble_qchunk = pick;
            c->tune.bubble_transfers = pick_h;
            best_b = best;
            // leave the loop-kernel rows of the fastest shape for the contraction below
            if ((st = launch_bubbles(c, lambda, c->d_Z, c->c4v_state, nullptr, c->c4v_state)) != QPFRG_OK) break;
        }
        // tensor-core contraction: split-K per channel (0 = the wave-filling heuristic)
        if (c->opt.precision == QPFRG_MIXED_TC) {
            const int cand[] = {0, 1, 2, 3, 4, 6, 8, 12, 16};
            double best = 0.0;
            for (int ch = 0; ch < 3 && st == QPFRG_OK; ++ch) {
                int pick = 0;
                best = 1e300;
                for (int sp : cand) {
                    c->tune.tc_splits[ch] = sp;
                    const double ms = time_launch(
                        c, ev, [&] { return launch_contractions(c, Vin, 1.0, c->d_k); }, st);
                    if (ms < 0.0) break;
                    if (ms < best) {
                        best = ms;
                        pick = sp;
                    }
                }
                c->tune.tc_splits[ch] = pick;
            }
            if (st != QPFRG_OK) break;
            best_c = best;      // all three channels with their chosen splits
        }
        // FP32 self-energy of the wedge grid: q blocks per CTA
        if (mixed && c->d_ptab) {
            const double T = tflow ? lambda : c->pb.T_fixed;
            const int cand[] = {1, 2, 4, 8};
            int pick = 0;
            double best = 1e300;
            for (int qb : cand) {
                c->tune.sigma_qblocks = qb;
                const double ms = time_launch(
                    c, ev, [&] { return launch_sigma_z(c, T, c->d_V, c->d_Z, c->d_Zwork, c->c4v_state); }, st);
                if (ms < 0.0) break;
                if (ms < best) {
                    best = ms;
                    pick = qb;
                }
            }
            if (st != QPFRG_OK) break;
            c->tune.sigma_qblocks = pick;
            best_s = best;
        }
    } while (false);
    c->prof = prof;
    if (st != QPFRG_OK) return st;
    if (out) {
        out->bubble_qchunk = c->tune.bubble_qchunk;
        out->bubble_transfers = c->tune.bubble_transfers;
        out->sigma_qblocks = c->tune.sigma_qblocks;
        for (int i = 0; i < 3; ++i) out->tc_splits[i] = c->tune.tc_splits[i];
        out->ms_bubble = best_b;
        out->ms_sigma = best_s;
        out->ms_contract = best_c;
    }
    return QPFRG_OK;
}

extern "C" qpfrg_status qpfrg_set_tuning(qpfrg_t c, const qpfrg_tuning *t)
{
    if (!c || !t) return QPFRG_ERR_INVALID;
    if (t->bubble_qchunk < 0 || t->sigma_qblocks < 0 || t->sigma_qblocks > 64 || t->tc_splits[0] < 0 ||
        t->tc_splits[1] < 0 || t->tc_splits[2] < 0 ||
        (t->bubble_transfers != 0 && t->bubble_transfers != 2 && t->bubble_transfers != 4)) {
        c->err = "invalid launch shape";
        return QPFRG_ERR_INVALID;
    }
    c->tune.bubble_qchunk = t->bubble_qchunk;
    c->tune.bubble_transfers = t->bubble_transfers;
    c->tune.sigma_qblocks = t->sigma_qblocks;
    for (int i = 0; i < 3; ++i) c->tune.tc_splits[i] = t->tc_splits[i];
    return QPFRG_OK;
}
