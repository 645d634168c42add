// Batched temperature flows of one call (qpfrg_flow_batch): the sweep of the
// strong-coupling scale over (U, T_end, N_p) of Sec. 3.2 / Fig. 4, each flow
// stopping at its own bound.
//
// With Z = 1 the loop-kernel tables of a stage depend on the patching and on T
// alone, and every flow of one patch count that starts at the same T steps in
// lockstep (d ln T fixed) until its last step, which is clamped onto its
// T_end.  So each patch-count group evaluates the loop-kernel rows once per
// stage and distinct (ln T, h) -- a "slot": the regular step, plus one per
// flow that clamps at this step -- and every running flow contracts the table
// of its slot with its own vertex on the tensor cores:
//   per stage: loop table per active slot | operands of every flow |
//              3 batched contractions    | batched RK update
//   per step:  a finalize kernel: max|V| and finiteness -> status, Lambda_c,
//              and the slots still in use at the next step.
// The schedule (per step and flow: h, slot) is fixed on the host from the
// specs; divergence is decided on the device, and every batched kernel skips
// a flow that stopped (the loop launch of a slot without running flows does
// nothing).  The launches of a chunk of steps are captured into one CUDA
// graph per group and the groups run concurrently on their own streams; the
// host waits once per chunk (time budget).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "qpfrg_internal.h"

namespace qpfrg {

namespace {

// device state of the flows of a group, one array per field
struct FlowArrays {
    int *status, *steps;
    double *x, *m_old, *lambda_c, *max_v;
};

// RK4 bookkeeping of every running flow with a step, grid.y = flow; k (and
// the representative rows outc of the row orbits, nc values per flow) are
// cleared after use (the contractions add into them); the final stage also
// refreshes the FP32 copy for the next step and reduces max|V| and finiteness.
__global__ void rk_batch_kernel(int stage, const TcPrepFlow *pf, double *const *V, double *const *k,
                                double *const *acc, double *const *outc, long nc, const double *h_tab,
                                const int *status, int step, int nflows, unsigned long long *red, long n)
{
    const int f = blockIdx.y;
    const double h = h_tab[(long)step * nflows + f];
    if (status[f] != QPFRG_FLOW_RUNNING || h == 0.0) return;
    double *Vf64 = V[f], *kf = k[f], *af = acc[f];
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nc; i += (long)gridDim.x * blockDim.x)
        outc[f][i] = 0.0;
    float *Vf = const_cast<float *>(pf[f].Vf);
    const double c_next = stage == 3 ? h : 0.5 * h;
    double m = 0.0;
    bool bad = false;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double ki = kf[i];
        kf[i] = 0.0;
        if (stage < 4) {
            af[i] = stage == 1 ? ki : af[i] + 2.0 * ki;
            Vf[i] = (float)(Vf64[i] + c_next * ki);
        } else {
            const double v = Vf64[i] + h / 6.0 * (af[i] + ki);
            Vf64[i] = v;
            Vf[i] = (float)v;
            bad = bad || !isfinite(v);
            m = fmax(m, fabs(v));
        }
    }
    if (stage == 4) {
        for (int off = 16; off > 0; off >>= 1) {
            m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
            bad = bad || __shfl_down_sync(0xffffffffu, (int)bad, off);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&red[2 * f], (unsigned long long)__double_as_longlong(m));
            if (bad) atomicOr(&red[2 * f + 1], 1ull);
        }
    }
}

// After a step: per flow with a step, max|V| and finiteness decide the status
// (the rule of the single flows: divergence with Lambda_c interpolated in
// ln max|V|, end of the flow); then the slots in use at the next step.
__global__ void finalize_kernel(FlowArrays st, const double *h_tab, const signed char *slot_tab, const double *x_end,
                                unsigned long long *red, int *act, int step, int nsteps, int nflows, int nslots,
                                double stop)
{
    for (int f = threadIdx.x; f < nflows; f += blockDim.x) {
        const double h = h_tab[(long)step * nflows + f];
        if (st.status[f] != QPFRG_FLOW_RUNNING || h == 0.0) continue;
        const double m_new = __longlong_as_double((long long)red[2 * f]);
        const bool bad = red[2 * f + 1] != 0;
        red[2 * f] = 0;
        red[2 * f + 1] = 0;
        const double x = st.x[f], m_old = st.m_old[f], x_new = x + h;
        st.steps[f] += 1;
        st.max_v[f] = m_new;
        if (bad) {
            st.status[f] = QPFRG_FLOW_NONFINITE;
        } else if (m_new > stop) {
            const double fr = (log(stop) - log(m_old)) / (log(m_new) - log(m_old));
            st.lambda_c[f] = exp(x + fr * h);
            st.status[f] = QPFRG_FLOW_DIVERGED;
        } else if (x_new - x_end[f] <= 1e-12) {
            st.status[f] = QPFRG_FLOW_REACHED_END;
        }
        st.x[f] = x_new;
        st.m_old[f] = m_new;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) act[i] = 0;
    __syncthreads();
    if (step + 1 < nsteps)
        for (int f = threadIdx.x; f < nflows; f += blockDim.x)
            if (st.status[f] == QPFRG_FLOW_RUNNING && h_tab[(long)(step + 1) * nflows + f] != 0.0)
                atomicOr(&act[slot_tab[(long)(step + 1) * nflows + f]], 1);
}

template <typename T>
qpfrg_status dalloc(qpfrg_ctx *c, T **p, size_t n, const char *what)
{
    const cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(c, e, what);
    }
    return QPFRG_OK;
}

// One patch-count group of the batch.
struct Group {
    qpfrg_ctx *geo = nullptr;          // geometry, orbits, loop-kernel tasks, tensor-core shapes
    cudaStream_t stream = nullptr;
    std::vector<int> members;          // indices into the specs
    int F = 0, nsteps = 0, nslots = 0;
    // schedule: h and slot per (step, flow); per (step, slot) ln T and h of the slot
    std::vector<double> h_tab;
    std::vector<signed char> slot_tab;
    std::vector<std::vector<std::pair<double, double>>> slot_xh;
    // device
    std::vector<void *> allocs;
    double *d_h = nullptr, *d_xend = nullptr;
    signed char *d_slot = nullptr;
    FlowArrays st{};
    unsigned long long *d_red = nullptr;
    int *d_act = nullptr;
    std::vector<float *> rows;         // per slot
    float **d_rows = nullptr;
    TcPrepFlow *d_pf = nullptr;
    double **d_V = nullptr, **d_k = nullptr, **d_acc = nullptr;
    bool compact = false;              // row orbits: representative rows, expanded per flow
    double **d_outc = nullptr;         // per flow: [ch][representative][n]
    long nc = 0;                       // values per flow of d_outc
    const float **d_Vf = nullptr, **d_VT = nullptr;
    CUtensorMap *d_maps = nullptr;
    CUtensorMap *d_tmaps = nullptr;    // table map per slot

    Group() = default;
    Group(const Group &) = delete;
    Group &operator=(const Group &) = delete;
    ~Group()
    {
        for (void *p : allocs) cudaFree(p);
        for (float *r : rows) cudaFree(r);
        if (geo) qpfrg_destroy(geo);
        if (stream) cudaStreamDestroy(stream);
    }
};

template <typename T>
qpfrg_status galloc(Group &g, T **p, size_t n, const char *what)
{
    qpfrg_status s = dalloc(g.geo, p, n, what);
    if (s == QPFRG_OK) g.allocs.push_back(*p);
    return s;
}

// Host schedule of the group: the steps of each flow from ln T0 with the
// regular step, the last one clamped onto ln T_end (as the single flows), and
// the slots of distinct (ln T, h) at each step.
void make_schedule(Group &g, const qpfrg_flow_spec *specs, double step, int max_steps)
{
    const int F = g.F;
    std::vector<std::vector<std::pair<double, double>>> xh(F);   // per flow: (x, h) of each step
    int nst = 0;
    for (int i = 0; i < F; ++i) {
        const qpfrg_flow_spec &sp = specs[g.members[i]];
        double x = std::log(sp.lambda0);
        const double x_end = std::log(sp.lambda_end);
        for (int k = 0; k < max_steps; ++k) {
            if (x - x_end <= 1e-12) break;
            double h = step;
            if (x + h < x_end) h = x_end - x;
            xh[i].push_back({x, h});
            x = x + h;
        }
        nst = std::max(nst, (int)xh[i].size());
    }
    g.nsteps = nst;
    g.h_tab.assign((size_t)nst * F, 0.0);
    g.slot_tab.assign((size_t)nst * F, 0);
    g.slot_xh.assign(nst, {});
    g.nslots = 1;
    for (int k = 0; k < nst; ++k) {
        std::map<std::pair<double, double>, int> slots;
        for (int i = 0; i < F; ++i) {
            if (k >= (int)xh[i].size()) continue;
            const auto key = xh[i][k];
            auto it = slots.find(key);
            int sl;
            if (it == slots.end()) {
                sl = (int)slots.size();
                slots[key] = sl;
                g.slot_xh[k].push_back(key);
            } else {
                sl = it->second;
            }
            g.h_tab[(size_t)k * F + i] = key.second;
            g.slot_tab[(size_t)k * F + i] = (signed char)sl;
        }
        g.nslots = std::max(g.nslots, (int)slots.size());
    }
}

qpfrg_status setup_group(Group &g, const qpfrg_lattice *lattice, const qpfrg_fine_grid *grid, qpfrg_options opt,
                         const qpfrg_flow_spec *specs, cudaEvent_t start)
{
    qpfrg_status s;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking)) != cudaSuccess) return QPFRG_ERR_CUDA;
    cudaStreamWaitEvent(g.stream, start, 0);
    const qpfrg_flow_spec &first = specs[g.members[0]];
    if ((s = qpfrg_create(lattice, first.n_p, grid, first.U, first.lambda0, QPFRG_REG_TEMPERATURE, &opt, g.stream,
                          &g.geo)) != QPFRG_OK)
        return s;
    qpfrg_ctx *c = g.geo;
    if (opt.autotune && (s = qpfrg_autotune(c, first.lambda0, nullptr)) != QPFRG_OK) return s;
    make_schedule(g, specs, opt.step, opt.max_steps);
    if (g.nslots > 127) {
        c->err = "batched flows: more than 127 distinct step sizes in one step of a group";
        return QPFRG_ERR_UNSUPPORTED;
    }
    const int F = g.F, N = c->pb.N;
    const long n3 = (long)N * N * N;
    const TcBuffers &t = c->tc;
    const size_t nb = (size_t)t.Npad * t.Kp, nbd = (size_t)t.Npad * t.Kpd;
    // per-flow state and operands, one allocation per kind
    double *V, *k, *acc;
    float *Vf, *VT;
    __nv_bfloat16 *B;
    const size_t bper = 2 * (2 * nb + nbd);
    if ((s = galloc(g, &V, F * n3, "batch V")) || (s = galloc(g, &k, F * n3, "batch k")) ||
        (s = galloc(g, &acc, F * n3, "batch acc")) || (s = galloc(g, &Vf, F * n3, "batch V fp32")) ||
        (s = galloc(g, &VT, F * 3 * n3, "batch row-factor tables")) || (s = galloc(g, &B, F * bper, "batch operands")))
        return s;
    if ((e = cudaMemsetAsync(k, 0, F * n3 * sizeof(double), g.stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(B, 0, F * bper * sizeof(__nv_bfloat16), g.stream)) != cudaSuccess)
        return cuda_fail(c, e, "clear batch buffers");
    // every flow starts at V = U with Z = 1, C4v symmetric, and stays so:
    // the row orbits apply to the whole batch when the context built them
    g.compact = c->rows_ok;
    double *outc = nullptr;
    std::vector<double *> poutc(F, nullptr);
    if (g.compact) {
        g.nc = 3L * c->n_rrep * N;
        if ((s = galloc(g, &outc, F * g.nc, "batch representative rows")) ||
            (s = galloc(g, &g.d_outc, F, "batch representative row ptrs")))
            return s;
        if ((e = cudaMemsetAsync(outc, 0, F * g.nc * sizeof(double), g.stream)) != cudaSuccess)
            return cuda_fail(c, e, "clear batch representative rows");
        for (int i = 0; i < F; ++i) poutc[i] = outc + i * g.nc;
    }
    std::vector<double> hv(n3);
    std::vector<float> hf(n3);
    std::vector<TcPrepFlow> pf(F);
    std::vector<double *> pV(F), pk(F), pacc(F);
    std::vector<const float *> pVf(F), pVT(F);
    std::vector<CUtensorMap> maps(6 * (size_t)F);
    std::vector<int> h_status(F), h_steps(F, 0);
    std::vector<double> h_x(F), h_m(F), h_lc(F, 0.0), xend(F);
    for (int i = 0; i < F; ++i) {
        const qpfrg_flow_spec &sp = specs[g.members[i]];
        std::fill(hv.begin(), hv.end(), sp.U);
        std::fill(hf.begin(), hf.end(), (float)sp.U);
        if ((e = cudaMemcpy(V + i * n3, hv.data(), n3 * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(Vf + i * n3, hf.data(), n3 * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(c, e, "batch initial state");
        pV[i] = V + i * n3;
        pk[i] = k + i * n3;
        pacc[i] = acc + i * n3;
        pVf[i] = Vf + i * n3;
        pVT[i] = VT + i * 3 * n3;
        __nv_bfloat16 *bb = B + i * bper;
        pf[i].Vf = Vf + i * n3;
        pf[i].VT = VT + i * 3 * n3;
        pf[i].B[0][0] = bb;
        pf[i].B[0][1] = bb + nb;
        pf[i].B[1][0] = bb + 2 * nb;
        pf[i].B[1][1] = bb + 3 * nb;
        pf[i].B[2][0] = bb + 4 * nb;
        pf[i].B[2][1] = bb + 4 * nb + nbd;
        for (int ch = 0; ch < 3; ++ch)
            for (int h = 0; h < 2; ++h)
                if ((s = make_tile_map(c, &maps[6 * i + 2 * ch + h], pf[i].B[ch][h], ch == 2 ? (long)nbd : (long)nb,
                                       t.Npad / 2)) != QPFRG_OK)
                    return s;
        h_x[i] = std::log(sp.lambda0);
        h_m[i] = std::fabs(sp.U);
        h_status[i] = g.nsteps > 0 ? QPFRG_FLOW_RUNNING : QPFRG_FLOW_REACHED_END;
        xend[i] = std::log(sp.lambda_end);
    }
    if ((s = galloc(g, &g.d_pf, F, "batch flows")) || (s = galloc(g, &g.d_V, F, "batch V ptrs")) ||
        (s = galloc(g, &g.d_k, F, "batch k ptrs")) || (s = galloc(g, &g.d_acc, F, "batch acc ptrs")) ||
        (s = galloc(g, &g.d_Vf, F, "batch Vf ptrs")) || (s = galloc(g, &g.d_VT, F, "batch VT ptrs")) ||
        (s = galloc(g, &g.d_maps, 6 * (size_t)F, "batch maps")) || (s = galloc(g, &g.st.status, F, "batch status")) ||
        (s = galloc(g, &g.st.steps, F, "batch steps")) || (s = galloc(g, &g.st.x, F, "batch ln T")) ||
        (s = galloc(g, &g.st.m_old, F, "batch max|V|")) || (s = galloc(g, &g.st.lambda_c, F, "batch scales")) ||
        (s = galloc(g, &g.st.max_v, F, "batch max|V| now")) ||
        (s = galloc(g, &g.d_xend, F, "batch ends")) || (s = galloc(g, &g.d_red, 2 * (size_t)F, "batch reductions")) ||
        (s = galloc(g, &g.d_act, g.nslots, "batch slots")) ||
        (s = galloc(g, &g.d_h, std::max<size_t>(1, g.h_tab.size()), "batch schedule")) ||
        (s = galloc(g, &g.d_slot, std::max<size_t>(1, g.slot_tab.size()), "batch slots table")) ||
        (s = galloc(g, &g.d_rows, g.nslots, "batch rows ptrs")) ||
        (s = galloc(g, &g.d_tmaps, g.nslots, "batch table maps")))
        return s;
    g.rows.assign(g.nslots, nullptr);
    std::vector<CUtensorMap> tmaps(g.nslots);
    for (int sl = 0; sl < g.nslots; ++sl) {
        if ((e = cudaMalloc((void **)&g.rows[sl], c->B_bytes)) != cudaSuccess ||
            (e = cudaMemset(g.rows[sl], 0, c->B_bytes)) != cudaSuccess)
            return cuda_fail(c, e, "batch rows");
        if ((s = make_table_map(c, &tmaps[sl], g.rows[sl])) != QPFRG_OK) return s;
    }
    std::vector<int> act(g.nslots, 0);
    if (g.nsteps > 0)
        for (int i = 0; i < F; ++i) act[g.slot_tab[i]] = 1;
    struct Up {
        void *dst;
        const void *src;
        size_t bytes;
    } ups[] = {{g.d_pf, pf.data(), F * sizeof(TcPrepFlow)},
               {g.d_V, pV.data(), F * sizeof(double *)},
               {g.d_k, pk.data(), F * sizeof(double *)},
               {g.d_acc, pacc.data(), F * sizeof(double *)},
               {g.d_Vf, pVf.data(), F * sizeof(float *)},
               {g.d_VT, pVT.data(), F * sizeof(float *)},
               {g.d_maps, maps.data(), maps.size() * sizeof(CUtensorMap)},
               {g.st.status, h_status.data(), F * sizeof(int)},
               {g.st.steps, h_steps.data(), F * sizeof(int)},
               {g.st.x, h_x.data(), F * sizeof(double)},
               {g.st.m_old, h_m.data(), F * sizeof(double)},
               {g.st.lambda_c, h_lc.data(), F * sizeof(double)},
               {g.st.max_v, h_m.data(), F * sizeof(double)},
               {g.d_xend, xend.data(), F * sizeof(double)},
               {g.d_act, act.data(), g.nslots * sizeof(int)},
               {g.d_h, g.h_tab.data(), g.h_tab.size() * sizeof(double)},
               {g.d_slot, g.slot_tab.data(), g.slot_tab.size()},
               {g.d_rows, g.rows.data(), g.nslots * sizeof(float *)},
               {g.d_tmaps, tmaps.data(), g.nslots * sizeof(CUtensorMap)},
               {g.d_outc, poutc.data(), g.compact ? F * sizeof(double *) : 0}};
    for (const Up &u : ups)
        if (u.bytes && (e = cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(c, e, "batch upload");
    if ((e = cudaMemset(g.d_red, 0, 2 * (size_t)F * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(c, e, "batch reductions");
    // loop-kernel tasks of the chosen chunk before any capture (the upload synchronises)
    const int qchunk = c->tune.bubble_qchunk > 0 ? (int)std::min<long>(c->tune.bubble_qchunk, (long)N * N)
                                                 : (int)std::max(8L, std::min(64L, (long)N * N / 16));
    int ntask = 0;
    return g.compact ? row_tasks(c, std::max(8, qchunk), &ntask) : loop_tasks(c, qchunk, &ntask);
}

// Enqueue step k of the group on its stream.
qpfrg_status enqueue_group_step(Group &g, int k, double stop)
{
    qpfrg_ctx *c = g.geo;
    const long n3 = (long)c->pb.N * c->pb.N * c->pb.N;
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    qpfrg_status s;
    for (int st = 0; st < 4; ++st) {
        const auto &sx = g.slot_xh[k];
        for (int sl = 0; sl < (int)sx.size(); ++sl) {
            const double T = std::exp(sx[sl].first + cst[st] * sx[sl].second);
            if ((s = launch_loop_rows(c, T, g.rows[sl], g.d_act + sl, g.compact)) != QPFRG_OK) return s;
        }
        if ((s = launch_tc_prep_batch(c, g.d_pf, g.st.status, g.d_h, k, g.F)) != QPFRG_OK) return s;
        TcBatch bt{};
        bt.nflows = g.F;
        bt.step = k;
        bt.cst = cst[st];
        bt.status = g.st.status;
        bt.h_tab = g.d_h;
        bt.slot_tab = g.d_slot;
        bt.x = g.st.x;
        bt.rows = g.d_rows;
        bt.Vf = g.d_Vf;
        bt.VT = g.d_VT;
        bt.out = g.d_k;
        bt.outc = g.compact ? g.d_outc : nullptr;
        bt.maps = g.d_maps;
        bt.tab_maps = g.d_tmaps;
        const unsigned ch = c->pb.channels;
        if ((ch & QPFRG_CH_PP) && (s = launch_tc_fused_batch(c, 0, bt, -1.0))) return s;
        if ((ch & QPFRG_CH_CR) && (s = launch_tc_fused_batch(c, 1, bt, -1.0))) return s;
        if ((ch & QPFRG_CH_D) && (s = launch_tc_fused_batch(c, 2, bt, 1.0))) return s;
        if (g.compact && (s = launch_rows_expand_batch(c, bt)) != QPFRG_OK) return s;
        const int blocks = (int)std::min<long>((n3 + 255) / 256, 152L * 4 / std::max(1, g.F / 8 + 1) + 1);
        prof_begin(c);
        rk_batch_kernel<<<dim3(blocks, g.F), 256, 0, g.stream>>>(st + 1, g.d_pf, g.d_V, g.d_k, g.d_acc, g.d_outc,
                                                                 g.compact ? g.nc : 0, g.d_h, g.st.status, k, g.F,
                                                                 g.d_red, n3);
        prof_end(c, st < 3 ? K_RK_STAGE : K_RK_FINAL);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "rk_batch_kernel");
    }
    finalize_kernel<<<1, 256, 0, g.stream>>>(g.st, g.d_h, g.d_slot, g.d_xend, g.d_red, g.d_act, k, g.nsteps, g.F,
                                             g.nslots, stop);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "finalize_kernel");
}

}  // namespace

// Whether qpfrg_flow_batch takes the batched device path: tensor-core
// precision, wedge patches with the C4v-reduced loop kernels, temperature
// flow with Z = 1 (no feedback), all flows starting at the same T.
bool batch_device_path(const qpfrg_fine_grid *grid, qpfrg_regulator regulator, const qpfrg_options &opt, int n,
                       const qpfrg_flow_spec *specs)
{
    if (opt.precision != QPFRG_MIXED_TC || grid->mode != QPFRG_GRID_WEDGE || regulator != QPFRG_REG_TEMPERATURE ||
        opt.z_feedback || opt.sigma_ode || opt.no_loop_symmetry)
        return false;
    for (int i = 1; i < n; ++i)
        if (specs[i].lambda0 != specs[0].lambda0) return false;
    return true;
}

qpfrg_status flow_batch_device(const qpfrg_lattice *lattice, const qpfrg_fine_grid *grid, const qpfrg_options &opt,
                               int n, const qpfrg_flow_spec *specs, cudaStream_t caller, qpfrg_flow_result *results,
                               std::string &err)
{
    std::vector<int> sizes;
    for (int i = 0; i < n; ++i)
        if (std::find(sizes.begin(), sizes.end(), specs[i].n_p) == sizes.end()) sizes.push_back(specs[i].n_p);
    std::vector<Group> groups(sizes.size());
    cudaEvent_t start = nullptr;
    cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    cudaEventRecord(start, caller);
    qpfrg_status s = QPFRG_OK;
    for (size_t gi = 0; gi < sizes.size() && s == QPFRG_OK; ++gi) {
        Group &g = groups[gi];
        for (int i = 0; i < n; ++i)
            if (specs[i].n_p == sizes[gi]) g.members.push_back(i);
        g.F = (int)g.members.size();
        s = setup_group(g, lattice, grid, opt, specs, start);
        if (s != QPFRG_OK && g.geo) err = g.geo->err;
    }
    cudaEventDestroy(start);
    if (s != QPFRG_OK) return s;
    // chunks of steps: one CUDA graph per group and chunk, groups concurrent
    const int chunk = 16;
    int maxsteps = 0;
    for (const Group &g : groups) maxsteps = std::max(maxsteps, g.nsteps);
    const auto t0 = std::chrono::steady_clock::now();
    bool timed_out = false;
    for (int k0 = 0; k0 < maxsteps && s == QPFRG_OK; k0 += chunk) {
        for (Group &g : groups) {
            const int k1 = std::min(g.nsteps, k0 + chunk);
            if (k0 >= k1) continue;
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            cudaError_t e = cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeRelaxed);
            for (int k = k0; k < k1 && s == QPFRG_OK && e == cudaSuccess; ++k) s = enqueue_group_step(g, k, opt.stop_abs_v);
            const cudaError_t e2 = cudaStreamEndCapture(g.stream, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess && s == QPFRG_OK) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess && s == QPFRG_OK) e = cudaGraphLaunch(exec, g.stream);
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            if (s == QPFRG_OK && e != cudaSuccess) {
                err = std::string("batched flows: ") + cudaGetErrorString(e);
                s = QPFRG_ERR_CUDA;
            }
            if (s != QPFRG_OK) break;
        }
        for (Group &g : groups)
            if (cudaStreamSynchronize(g.stream) != cudaSuccess && s == QPFRG_OK) {
                err = "batched flows: stream failed";
                s = QPFRG_ERR_CUDA;
            }
        if (opt.timeout_s > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > opt.timeout_s) {
            timed_out = true;
            break;
        }
    }
    // tensor-core waits that expired
    for (Group &g : groups) {
        unsigned flag = 0;
        if (g.geo->d_tc_err) cudaMemcpy(&flag, g.geo->d_tc_err, sizeof(flag), cudaMemcpyDeviceToHost);
        if (flag && s == QPFRG_OK) {
            err = "a tensor-core contraction wait expired";
            s = QPFRG_ERR_TIMEOUT;
        }
    }
    for (Group &g : groups) {
        const int F = g.F;
        std::vector<int> status(F), steps(F);
        std::vector<double> x(F), lc(F), mv(F);
        cudaMemcpy(status.data(), g.st.status, F * sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemcpy(steps.data(), g.st.steps, F * sizeof(int), cudaMemcpyDeviceToHost);
        cudaMemcpy(x.data(), g.st.x, F * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(lc.data(), g.st.lambda_c, F * sizeof(double), cudaMemcpyDeviceToHost);
        cudaMemcpy(mv.data(), g.st.max_v, F * sizeof(double), cudaMemcpyDeviceToHost);
        for (int i = 0; i < F; ++i) {
            qpfrg_flow_result &r = results[g.members[i]];
            int st = status[i];
            if (st == QPFRG_FLOW_RUNNING) st = timed_out ? QPFRG_FLOW_TIMEOUT : QPFRG_FLOW_MAX_STEPS;
            r.status = st;
            r.steps = steps[i];
            r.lambda = std::exp(x[i]);
            r.lambda_c = lc[i];
            r.max_abs_v = mv[i];
        }
    }
    return s;
}

}  // namespace qpfrg
