// C ABI of the qpfrg library: context management, right-hand side,
// self-energy/Z, the RK4 flow driver, checkpoints and the kernel profiler.
// The declarations and their contracts are in include/qpfrg.h.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "qpfrg_internal.h"

using namespace qpfrg;

namespace {

const char *const kKernelNames[K_COUNT] = {
    "partner_map", "bubble", "contract_pp", "contract_cr", "contract_d", "sigma_z",
    "sigma_hist", "sigma_grid", "z_update", "rk_stage", "rk_final", "convert_f32",
    "tc_prep", "tc_fused_pp", "tc_fused_cr", "tc_fused_d", "kp_table", "rtab_build", "rows_expand",
};

struct PendingEvent {
    int id;
    cudaEvent_t a, b;
};

struct Profiler {
    std::vector<PendingEvent> pending;
    std::vector<cudaEvent_t> spare;
};

Profiler *prof_of(qpfrg_ctx *c) { return reinterpret_cast<Profiler *>(c->profiler); }

constexpr uint32_t kStateMagic = 0x52465051u;  // "QPFR"
constexpr uint32_t kStateVersion = 1u;

struct StateHeader {
    uint32_t magic;
    uint32_t version;
    int32_t N;
    int32_t status;
    int64_t steps;
    double lambda;
    double max_abs_v;
    double lambda_c;
    double reserved[2];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

qpfrg_status set_err(qpfrg_ctx *c, qpfrg_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

cudaEvent_t take_event(Profiler *p)
{
    if (!p->spare.empty()) {
        cudaEvent_t e = p->spare.back();
        p->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void flush_profile(qpfrg_ctx *c)
{
    Profiler *p = prof_of(c);
    if (!p || p->pending.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (const PendingEvent &pe : p->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            c->slots[pe.id].ms += ms;
            c->slots[pe.id].launches += 1;
        }
        p->spare.push_back(pe.a);
        p->spare.push_back(pe.b);
    }
    p->pending.clear();
}

template <typename T>
qpfrg_status dev_alloc(qpfrg_ctx *c, T **p, size_t count, const char *what)
{
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        c->err = std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? QPFRG_ERR_OOM : QPFRG_ERR_CUDA;
    }
    return QPFRG_OK;
}

long n3_of(const qpfrg_ctx *c) { return (long)c->pb.N * c->pb.N * c->pb.N; }

}  // namespace

namespace qpfrg {

qpfrg_status cuda_fail(qpfrg_ctx *c, cudaError_t e, const char *what)
{
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QPFRG_ERR_OOM : QPFRG_ERR_CUDA;
}

void prof_begin(qpfrg_ctx *c)
{
    if (!c->prof) return;
    Profiler *p = prof_of(c);
    if (p->pending.size() >= 8192) flush_profile(c);
    PendingEvent pe{-1, take_event(p), take_event(p)};
    cudaEventRecord(pe.a, c->stream);
    p->pending.push_back(pe);
}

void prof_end(qpfrg_ctx *c, int id)
{
    if (!c->prof) return;
    Profiler *p = prof_of(c);
    PendingEvent &pe = p->pending.back();
    pe.id = id;
    cudaEventRecord(pe.b, c->stream);
}

}  // namespace qpfrg

// ---------------------------------------------------------------------------
// public API
// ---------------------------------------------------------------------------
extern "C" {

void qpfrg_default_options(qpfrg_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->channel_mask = QPFRG_CH_ALL;
    o->z_feedback = 0;
    o->propagator = QPFRG_PROP_PAPER;
    o->precision = QPFRG_FP64;
    o->eta = 0.02;
    o->n_omega = 0;
    o->omega_min = -4.0;
    o->omega_max = 4.0;
    o->stop_abs_v = 20.0;
    o->step = std::log(0.98);
    o->lambda_end = 0.05;
    o->z_max = 2.0;
    o->max_steps = 100000;
    o->T_fixed = 0.1;
    o->timeout_s = 0.0;
}

const char *qpfrg_version(void) { return "qpfrg 0.1 (sm_103a)"; }

const char *qpfrg_last_error(qpfrg_t ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

void qpfrg_destroy(qpfrg_t c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    // per-flow state: always owned
    void *own[] = {c->d_V, c->d_Z, c->d_Vs, c->d_k, c->d_acc, c->d_Vf, c->d_Zwork, c->d_red,
                   c->d_gy, c->d_gys, c->d_gk, c->d_gacc, c->d_gzka, c->d_gt2};
    for (void *p : own)
        if (p) cudaFree(p);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (!c->shares_geometry) {
        void *ptrs[] = {c->f64.kx, c->f64.ky, c->f64.cx, c->f64.sx, c->f64.cy, c->f64.sy, c->f64.xi, c->f64.w,
                        c->f32.kx, c->f32.ky, c->f32.cx, c->f32.sx, c->f32.cy, c->f32.sy, c->f32.xi, c->f32.w,
                        c->qpp64.cx, c->qpp64.sx, c->qpp64.cy, c->qpp64.sy, c->qph64.cx, c->qph64.sx,
                        c->qph64.cy, c->qph64.sy, c->qpp32.cx, c->qpp32.sx, c->qpp32.cy, c->qpp32.sy,
                        c->qph32.cx, c->qph32.sx, c->qph32.cy, c->qph32.sy, c->d_kf, c->d_Qpp, c->d_Qph,
                        c->d_part, c->d_B, c->d_ones, c->d_sig, c->d_hist, c->d_jirr, c->d_rep,
                        c->tc.Bpp[0], c->tc.Bpp[1], c->tc.Bcr[0], c->tc.Bcr[1], c->tc.Bd[0], c->tc.Bd[1],
                        c->tc.VT, c->d_tc_err, c->d_xij, c->d_bnd, c->d_qxl, c->d_qyl, c->d_kp, c->d_kcs, c->d_xij_f,
                        c->d_ptab, c->d_jgrid, c->d_repgrid, c->d_lrepQ, c->d_lnimg, c->d_limg, c->d_ltask,
                        c->d_rtab, c->d_rrep, c->d_rowmap, c->d_rtask, c->d_outc};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    Profiler *p = prof_of(c);
    if (p) {
        for (auto &pe : p->pending) {
            cudaEventDestroy(pe.a);
            cudaEventDestroy(pe.b);
        }
        for (auto e : p->spare) cudaEventDestroy(e);
        delete p;
    }
    delete c;
}

qpfrg_status qpfrg_create(const qpfrg_lattice *lattice, int n_p, const qpfrg_fine_grid *grid, double U,
                          double lambda0, qpfrg_regulator regulator, const qpfrg_options *options,
                          void *cuda_stream, qpfrg_t *out)
{
    if (!out) return QPFRG_ERR_INVALID;
    *out = nullptr;
    if (!lattice || !grid) return QPFRG_ERR_INVALID;
    qpfrg_ctx *c = new (std::nothrow) qpfrg_ctx();
    if (!c) return QPFRG_ERR_OOM;
    c->profiler = new (std::nothrow) Profiler();
    if (!c->profiler) {
        delete c;
        return QPFRG_ERR_OOM;
    }
    auto fail = [&](qpfrg_status s) {
        fprintf(stderr, "qpfrg_create: %s\n", c->err.c_str());
        qpfrg_destroy(c);
        return s;
    };
    if (options)
        c->opt = *options;
    else
        qpfrg_default_options(&c->opt);

    // ---- validation -------------------------------------------------------
    Problem &pb = c->pb;
    pb.t = lattice->t;
    pb.tp = lattice->tp;
    pb.mu = lattice->mu;
    pb.mode = grid->mode;
    pb.N = n_p;
    pb.n_shell = 1;
    pb.regulator = regulator;
    pb.propagator = c->opt.propagator;
    pb.channels = c->opt.channel_mask & QPFRG_CH_ALL;
    pb.T_fixed = c->opt.T_fixed;
    pb.eta = c->opt.eta;
    c->U = U;
    c->lambda0 = lambda0;
    const bool tflow = regulator == QPFRG_REG_TEMPERATURE;
    if (!std::isfinite(pb.t) || !std::isfinite(pb.tp) || !std::isfinite(pb.mu) || !std::isfinite(U) ||
        !std::isfinite(lambda0))
        return fail(set_err(c, QPFRG_ERR_INVALID, "non-finite lattice, U or lambda0"));
    if (regulator != QPFRG_REG_TEMPERATURE && regulator != QPFRG_REG_INTERACTION)
        return fail(set_err(c, QPFRG_ERR_INVALID, "unknown regulator"));
    if (tflow ? !(lambda0 > 0.0) : !(lambda0 >= 0.0))
        return fail(set_err(c, QPFRG_ERR_INVALID, "lambda0 must be T > 0 (T-flow) or g >= 0 (g-flow)"));
    if (!tflow && !(pb.T_fixed > 0.0))
        return fail(set_err(c, QPFRG_ERR_INVALID, "interaction flow needs T_fixed > 0"));
    if (c->opt.precision != QPFRG_FP64 && c->opt.precision != QPFRG_MIXED && c->opt.precision != QPFRG_MIXED_TC)
        return fail(set_err(c, QPFRG_ERR_INVALID, "unknown precision"));
    if (pb.propagator != QPFRG_PROP_PAPER && pb.propagator != QPFRG_PROP_QP)
        return fail(set_err(c, QPFRG_ERR_INVALID, "unknown propagator mode"));
    if (c->opt.sigma_ode && (tflow || pb.propagator != QPFRG_PROP_PAPER))
        return fail(set_err(c, QPFRG_ERR_UNSUPPORTED,
                            "the self-energy ODE is implemented for the interaction flow with QPFRG_PROP_PAPER lines"));
    if (c->opt.a_mode < 0 || c->opt.a_mode > 3) return fail(set_err(c, QPFRG_ERR_INVALID, "unknown a_mode"));
    if (c->opt.z_feedback && !tflow && !c->opt.sigma_ode)
        return fail(set_err(c, QPFRG_ERR_UNSUPPORTED,
                            "Z feedback of the interaction flow needs the self-energy ODE (sigma_ode)"));
    if (!(pb.eta > 0.0)) return fail(set_err(c, QPFRG_ERR_INVALID, "eta must be > 0"));
    if (c->opt.n_omega < 0 || (c->opt.n_omega > 0 && !(c->opt.omega_max >= c->opt.omega_min)))
        return fail(set_err(c, QPFRG_ERR_INVALID, "bad frequency grid"));
    if (!(c->opt.stop_abs_v > 0.0) || !(c->opt.z_max > 0.0) || c->opt.max_steps < 0)
        return fail(set_err(c, QPFRG_ERR_INVALID, "bad stop_abs_v, z_max or max_steps"));
    if (tflow ? !(c->opt.step < 0.0 && c->opt.lambda_end > 0.0) : !(c->opt.step > 0.0))
        return fail(set_err(c, QPFRG_ERR_INVALID, "T-flow needs step < 0 and lambda_end > 0; g-flow step > 0"));
    if (pb.mode == QPFRG_GRID_LATTICE) {
        int L = (int)std::llround(std::sqrt((double)n_p));
        if (L < 1 || L * L != n_p || n_p > 256)
            return fail(set_err(c, QPFRG_ERR_INVALID, "lattice mode needs n_p = L*L <= 256"));
        pb.L = L;
        pb.P = 1;
        c->n_theta = c->n_r = 1;
        pb.n_theta = pb.n_r = 1;
    } else if (pb.mode == QPFRG_GRID_WEDGE || pb.mode == QPFRG_GRID_SHELL) {
        if (pb.mode == QPFRG_GRID_SHELL) {
            const int ns = grid->n_shell;
            if (ns < 1 || ns % 2 == 0 || n_p % ns != 0 || (n_p / ns) % 4 != 0 || n_p > 256 ||
                !std::isfinite(grid->shell_width))
                return fail(set_err(c, QPFRG_ERR_INVALID,
                                    "shell mode needs an odd n_shell and n_p / n_shell a multiple of 4, n_p <= 256"));
            pb.n_shell = ns;
            pb.shell_D = shell_width(pb, grid->shell_width);
        }
        if (n_p < 4 || n_p % 4 != 0 || n_p > 256)
            return fail(set_err(c, QPFRG_ERR_INVALID, "wedge mode needs n_p a multiple of 4, 4 <= n_p <= 256"));
        if (grid->n_theta < 1 || grid->n_r < 2 || grid->n_r % 2 != 0)
            return fail(set_err(c, QPFRG_ERR_INVALID, "fine grid needs n_theta >= 1 and even n_r >= 2"));
        c->n_theta = grid->n_theta;
        c->n_r = grid->n_r;
        pb.n_theta = grid->n_theta;
        pb.n_r = grid->n_r;
        pb.P = grid->n_theta * grid->n_r;
        pb.L = 0;
        if (pb.P > 2048)
            return fail(set_err(c, QPFRG_ERR_UNSUPPORTED, "more than 2048 fine points per patch"));
    } else {
        return fail(set_err(c, QPFRG_ERR_INVALID, "unknown fine-grid mode"));
    }
    pb.M = pb.N * pb.P;
    if (c->opt.precision == QPFRG_MIXED_TC && ((long)n_p * n_p) % 8 != 0)
        return fail(set_err(c, QPFRG_ERR_UNSUPPORTED, "tensor-core contraction needs n_p^2 % 8 == 0"));

    // ---- device ------------------------------------------------------------
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(set_err(c, QPFRG_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)));
    }
    cudaGetDevice(&c->device);
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);

    qpfrg_status s;
    if ((s = build_host_geometry(c)) != QPFRG_OK) return fail(s);
    if ((s = upload_geometry(c)) != QPFRG_OK) return fail(s);
    if ((s = build_loop_orbits(c)) != QPFRG_OK) return fail(s);

    const size_t N = pb.N, n3 = N * N * N, n4 = n3 * N;
    const size_t rsz = c->opt.precision == QPFRG_FP64 ? sizeof(double) : sizeof(float);
    const bool tcmode = c->opt.precision == QPFRG_MIXED_TC;
    c->B_bytes = 2 * n4 * rsz;
    if (tcmode) {
        // tiled table of the tensor-core path (tc_table_index): padded to
        // whole 128-row tiles and 64-wide k blocks
        const size_t NN = N * N, RT = (NN + 127) / 128, KB = (NN + 63) / 64;
        c->tc.RT = (long)RT;
        c->tc.KB = (long)KB;
        c->B_bytes = 2 * RT * KB * 128 * 64 * sizeof(float);
    }
    if (std::getenv("QPFRG_TEST_FAIL_ALLOC")) {   // host-side fault injection for tests
        c->err = "allocation failure injected by QPFRG_TEST_FAIL_ALLOC";
        return fail(QPFRG_ERR_OOM);
    }
    if ((s = dev_alloc(c, (unsigned char **)&c->d_B, c->B_bytes, "bubble tables")) != QPFRG_OK) return fail(s);
    if (tcmode) {
        TcBuffers &t = c->tc;
        t.Npad = (int)((N + 15) / 16 * 16);
        const size_t NN = N * N, Np = t.Npad;
        t.Kp = (long)((NN + 63) / 64 * 64);
        t.Kpd = 2 * t.Kp;
        const size_t nb = Np * (size_t)t.Kp, nbd = Np * (size_t)t.Kpd;
        for (int h = 0; h < 2; ++h)
            if ((s = dev_alloc(c, &t.Bpp[h], nb, "pp operand")) || (s = dev_alloc(c, &t.Bcr[h], nb, "cr operand")) ||
                (s = dev_alloc(c, &t.Bd[h], nbd, "d operand")))
                return fail(s);
        if ((s = dev_alloc(c, &t.VT, 3 * n3, "row-factor tables")) || (s = dev_alloc(c, &c->d_tc_err, 1, "tc error flag")))
            return fail(s);
        // tile pads (rows past N, k past the reduction length) stay zero
        for (int h = 0; h < 2 && e == cudaSuccess; ++h) {
            if ((e = cudaMemset(t.Bpp[h], 0, nb * 2)) != cudaSuccess || (e = cudaMemset(t.Bcr[h], 0, nb * 2)) != cudaSuccess)
                break;
            e = cudaMemset(t.Bd[h], 0, nbd * 2);
        }
        if (e == cudaSuccess) e = cudaMemset(c->d_tc_err, 0, sizeof(unsigned));
        // the table's pads (rows past N^2, columns past N^2 in the last block) stay zero
        if (e == cudaSuccess) e = cudaMemset(c->d_B, 0, c->B_bytes);
        if (e != cudaSuccess) return fail(cuda_fail(c, e, "clear tensor-core operands"));
        if ((s = tc_make_maps(c)) != QPFRG_OK) return fail(s);
    }
    if ((s = dev_alloc(c, &c->d_V, n3, "V")) || (s = dev_alloc(c, &c->d_Vs, n3, "V stage")) ||
        (s = dev_alloc(c, &c->d_k, n3, "k")) || (s = dev_alloc(c, &c->d_acc, n3, "acc")) ||
        (s = dev_alloc(c, &c->d_Vf, n3, "V fp32")) || (s = dev_alloc(c, &c->d_Z, N, "Z")) ||
        (s = dev_alloc(c, &c->d_Zwork, N, "Z work")) || (s = dev_alloc(c, &c->d_ones, N, "ones")) ||
        (s = dev_alloc(c, &c->d_sig, 2 * N, "sigma chord")) || (s = dev_alloc(c, &c->d_red, 5, "reduction")))
        return fail(s);
    e = cudaMallocHost((void **)&c->h_red, 5 * sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "cudaMallocHost"));
    if (c->opt.sigma_ode && (s = gflow_alloc(c)) != QPFRG_OK) return fail(s);

    // C4v-irreducible patches (wedges 0..floor(N_a/8), every shell) and each
    // patch's representative (its index in the irreducible list)
    if (pb.mode == QPFRG_GRID_WEDGE || pb.mode == QPFRG_GRID_SHELL) {
        const int ns = pb.n_shell, Na = (int)N / ns, q = Na / 4;
        std::vector<int> jirr, rep(N);
        for (int w = 0; 8 * w <= Na; ++w)
            for (int sh = 0; sh < ns; ++sh) jirr.push_back(w * ns + sh);
        for (int j = 0; j < (int)N; ++j) {
            int r = (j / ns) % q;
            if (2 * r > q) r = q - r;
            rep[j] = r * ns + j % ns;
        }
        c->n_irr = (int)jirr.size();
        if ((s = dev_alloc(c, &c->d_jirr, jirr.size(), "irreducible patches")) ||
            (s = dev_alloc(c, &c->d_rep, N, "representatives")))
            return fail(s);
        cudaMemcpy(c->d_jirr, jirr.data(), jirr.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(c->d_rep, rep.data(), N * sizeof(int), cudaMemcpyHostToDevice);
        if (pb.mode == QPFRG_GRID_WEDGE) {
            // frequency grid of the wedge kernels: zone-edge patches j = m N/4
            // get slots of their own
            std::vector<int> jgrid(jirr), repgrid(rep);
            for (int m = 1; m < 4; ++m) {
                repgrid[m * q] = (int)jgrid.size();
                jgrid.push_back(m * q);
            }
            c->n_grid = (int)jgrid.size();
            if ((s = dev_alloc(c, &c->d_jgrid, jgrid.size(), "grid targets")) ||
                (s = dev_alloc(c, &c->d_repgrid, N, "grid representatives")))
                return fail(s);
            cudaMemcpy(c->d_jgrid, jgrid.data(), jgrid.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(c->d_repgrid, repgrid.data(), N * sizeof(int), cudaMemcpyHostToDevice);
        }
    }

    // state: V = U, Z = 1 at lambda0
    std::vector<double> h(n3, U);
    e = cudaMemcpy(c->d_V, h.data(), n3 * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "init V"));
    h.assign(N, 1.0);
    cudaMemcpy(c->d_Z, h.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    e = cudaMemcpy(c->d_ones, h.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "init Z"));
    c->lambda = lambda0;
    c->lambda_end = c->opt.lambda_end;
    c->c4v_state = pb.mode == QPFRG_GRID_WEDGE || pb.mode == QPFRG_GRID_SHELL;
    c->steps = 0;
    c->status = QPFRG_FLOW_RUNNING;
    c->max_abs_v = std::fabs(U);
    c->lambda_c = 0.0;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(c, e, "create"));
    *out = c;
    return QPFRG_OK;
}

qpfrg_status qpfrg_rhs(qpfrg_t c, double lambda, const double *d_V, const double *d_Z, double *d_dV)
{
    if (!c) return QPFRG_ERR_INVALID;
    if (!d_V || !d_dV || d_V == d_dV) return set_err(c, QPFRG_ERR_INVALID, "bad V / dV pointers");
    const bool tflow = c->pb.regulator == QPFRG_REG_TEMPERATURE;
    if (!std::isfinite(lambda) || (tflow && !(lambda > 0.0)))
        return set_err(c, QPFRG_ERR_INVALID, "lambda must be finite (and T > 0)");
    const long n3 = n3_of(c);
    const void *Vin = d_V;
    qpfrg_status s;
    if (c->opt.precision != QPFRG_FP64) {
        if ((s = launch_convert_f32(c, d_V, c->d_Vf, n3)) != QPFRG_OK) return s;
        Vin = c->d_Vf;
    }
    // row orbits of the tensor-core contraction need a C4v-symmetric V and Z:
    // tested on the device (relative 1e-12 of max|V|, max|Z|) and read back
    bool sym = false;
    if (c->rows_ok) {
        if ((s = launch_state_check(c, d_V, d_Z ? d_Z : c->d_ones, true, 1e-12)) != QPFRG_OK) return s;
        cudaError_t e = cudaMemcpyAsync(&c->h_red[4], &c->d_red[4], sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "C4v test of the RHS input");
        sym = c->h_red[4] == 0;
    }
    if ((s = launch_bubbles(c, lambda, d_Z ? d_Z : c->d_ones, d_Z == nullptr, nullptr, sym)) != QPFRG_OK) return s;
    cudaError_t e = cudaMemsetAsync(d_dV, 0, n3 * sizeof(double), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "memset dV");
    return launch_contractions(c, Vin, 1.0, d_dV);
}

qpfrg_status qpfrg_selfenergy(qpfrg_t c, double lambda, const double *d_V, const double *d_Z,
                              double *d_sigma_re, double *d_sigma_im, double *d_Z_out)
{
    if (!c) return QPFRG_ERR_INVALID;
    if (c->pb.regulator != QPFRG_REG_TEMPERATURE)
        return set_err(c, QPFRG_ERR_UNSUPPORTED, "self-energy is implemented for the temperature flow");
    if (!d_V || !(lambda > 0.0) || !std::isfinite(lambda)) return set_err(c, QPFRG_ERR_INVALID, "bad V or T");
    const double *Z = d_Z ? d_Z : c->d_ones;
    qpfrg_status s;
    if (d_Z_out && (s = launch_sigma_z(c, lambda, d_V, Z, d_Z_out, false)) != QPFRG_OK) return s;
    if (c->opt.n_omega > 0 && d_sigma_re && d_sigma_im)
        return launch_sigma_grid(c, lambda, d_V, Z, d_sigma_re, d_sigma_im);
    return QPFRG_OK;
}

static void fill_result(const qpfrg_ctx *c, qpfrg_flow_result *out)
{
    if (!out) return;
    out->status = c->status;
    out->steps = c->steps;
    out->lambda = c->lambda;
    out->lambda_c = c->lambda_c;
    out->max_abs_v = c->max_abs_v;
}

// Enqueue one RK4 step of the flow state (see qpfrg.h) on the context's
// stream; finish_step completes it once the stream has reached the end.
// With Z feedback the new Z is read back (and range-checked) before the
// stages are enqueued, so that a flow whose Z left its range does not step.
static qpfrg_status enqueue_step(qpfrg_ctx *c)
{
    c->pending = false;
    const bool tflow = c->pb.regulator == QPFRG_REG_TEMPERATURE;
    const double x = tflow ? std::log(c->lambda) : c->lambda;
    const double x_end = tflow ? std::log(c->lambda_end) : c->lambda_end;
    if ((tflow && x - x_end <= 1e-12) || (!tflow && x_end - x <= 1e-12)) {
        c->status = QPFRG_FLOW_REACHED_END;
        return QPFRG_OK;
    }
    double h = c->opt.step;
    if ((tflow && x + h < x_end) || (!tflow && x + h > x_end)) h = x_end - x;
    const long n3 = n3_of(c);
    const int N = c->pb.N;
    const bool mixed = c->opt.precision != QPFRG_FP64;
    qpfrg_status s;
    cudaError_t e;

    if (c->opt.sigma_ode) {
        // interaction flow of (V, Sigma, Sigma'): Z, K, A from the state at every stage
        if ((s = gflow_enqueue_stages(c, x, h)) != QPFRG_OK) return s;
    } else {
    if (c->opt.z_feedback) {
        const double T = tflow ? c->lambda : c->pb.T_fixed;
        if ((s = launch_sigma_z(c, T, c->d_V, c->d_Z, c->d_Zwork, c->c4v_state)) != QPFRG_OK) return s;
        std::vector<double> hz(N);
        e = cudaMemcpyAsync(hz.data(), c->d_Zwork, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "read Z");
        for (int j = 0; j < N; ++j) {
            if (!std::isfinite(hz[j])) {
                c->status = QPFRG_FLOW_NONFINITE;
                return QPFRG_OK;
            }
            if (!(hz[j] > 0.0 && hz[j] <= c->opt.z_max)) {
                c->status = QPFRG_FLOW_Z_OUT_OF_RANGE;
                return QPFRG_OK;
            }
        }
        e = cudaMemcpyAsync(c->d_Z, c->d_Zwork, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy Z");
    }

    const void *Vin = c->d_V;
    if (mixed) {
        if ((s = launch_convert_f32(c, c->d_V, c->d_Vf, n3)) != QPFRG_OK) return s;
        Vin = c->d_Vf;
    }
    const double cst[4] = {0.0, 0.5, 0.5, 1.0};
    for (int st = 0; st < 4; ++st) {
        const double xs = x + cst[st] * h;
        const double lam = tflow ? std::exp(xs) : xs;
        const double scale = tflow ? lam : 1.0;   // dV/d ln T = T dV/dT
        if ((s = launch_bubbles(c, lam, c->d_Z, c->c4v_state, nullptr, c->c4v_state)) != QPFRG_OK) return s;
        if ((e = cudaMemsetAsync(c->d_k, 0, n3 * sizeof(double), c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "memset k");
        if ((s = launch_contractions(c, Vin, scale, c->d_k)) != QPFRG_OK) return s;
        if (st < 3) {
            s = launch_rk_stage(c, st + 1, h, c->d_V, c->d_k, c->d_acc, mixed ? nullptr : c->d_Vs,
                                mixed ? c->d_Vf : nullptr);
            if (s != QPFRG_OK) return s;
            Vin = mixed ? (const void *)c->d_Vf : (const void *)c->d_Vs;
        } else if ((s = launch_rk_final(c, h, c->d_V, c->d_acc, c->d_k)) != QPFRG_OK) {
            return s;
        }
    }
    }
    c->h_red[2] = 0;
    e = cudaMemcpyAsync(c->h_red, c->d_red, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && c->d_tc_err)
        e = cudaMemcpyAsync(&c->h_red[2], c->d_tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "flow step");
    c->pending = true;
    c->pend_x = x;
    c->pend_h = h;
    c->pend_m = c->max_abs_v;
    return QPFRG_OK;
}

// Complete the step enqueued by enqueue_step; the stream must have drained.
static qpfrg_status finish_step(qpfrg_ctx *c)
{
    if (!c->pending) return QPFRG_OK;
    c->pending = false;
    const bool tflow = c->pb.regulator == QPFRG_REG_TEMPERATURE;
    const double x = c->pend_x, h = c->pend_h, m_old = c->pend_m;
    const double x_end = tflow ? std::log(c->lambda_end) : c->lambda_end;
    if (c->h_red[2])
        return set_err(c, QPFRG_ERR_TIMEOUT, "a tensor-core contraction wait expired");
    double m_new;
    std::memcpy(&m_new, &c->h_red[0], sizeof(double));
    const double x_new = x + h;
    c->steps += 1;
    c->lambda = tflow ? std::exp(x_new) : x_new;
    c->max_abs_v = m_new;
    if (c->h_red[1]) {
        c->status = QPFRG_FLOW_NONFINITE;
        return QPFRG_OK;
    }
    if (m_new > c->opt.stop_abs_v) {
        const double sfrac = (std::log(c->opt.stop_abs_v) - std::log(m_old)) / (std::log(m_new) - std::log(m_old));
        const double xc = x + sfrac * h;
        c->lambda_c = tflow ? std::exp(xc) : xc;
        c->status = QPFRG_FLOW_DIVERGED;
        return QPFRG_OK;
    }
    if ((tflow && x_new - x_end <= 1e-12) || (!tflow && x_end - x_new <= 1e-12)) c->status = QPFRG_FLOW_REACHED_END;
    return QPFRG_OK;
}

static qpfrg_status do_step(qpfrg_ctx *c)
{
    qpfrg_status s = enqueue_step(c);
    if (s != QPFRG_OK || !c->pending) return s;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->pending = false;
        return cuda_fail(c, e, "flow step");
    }
    return finish_step(c);
}

qpfrg_status qpfrg_step(qpfrg_t c, int n_steps, qpfrg_flow_result *out)
{
    if (!c || n_steps < 0) return QPFRG_ERR_INVALID;
    for (int i = 0; i < n_steps && c->status == QPFRG_FLOW_RUNNING; ++i) {
        qpfrg_status s = do_step(c);
        if (s != QPFRG_OK) {
            fill_result(c, out);
            return s;
        }
    }
    fill_result(c, out);
    return QPFRG_OK;
}

qpfrg_status qpfrg_flow(qpfrg_t c, qpfrg_flow_result *out)
{
    if (!c) return QPFRG_ERR_INVALID;
    const auto t0 = std::chrono::steady_clock::now();
    int done = 0;
    while (c->status == QPFRG_FLOW_RUNNING) {
        if (done >= c->opt.max_steps) {
            c->status = QPFRG_FLOW_MAX_STEPS;
            break;
        }
        if (c->opt.timeout_s > 0.0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > c->opt.timeout_s) {
                c->status = QPFRG_FLOW_TIMEOUT;
                break;
            }
        }
        qpfrg_status s = do_step(c);
        if (s != QPFRG_OK) {
            fill_result(c, out);
            return s;
        }
        ++done;
    }
    fill_result(c, out);
    return QPFRG_OK;
}

// A flow that shares the geometry tables and the per-evaluation scratch of
// `parent` and owns its FP64 state: V = U, Z = 1 at lambda0.  Flows sharing a
// parent must run on the parent's stream (the scratch is reused in order).
static qpfrg_status make_child(qpfrg_ctx *parent, double U, double lambda0, double lambda_end, qpfrg_ctx **out)
{
    *out = nullptr;
    qpfrg_ctx *c = new (std::nothrow) qpfrg_ctx(*parent);
    if (!c) return QPFRG_ERR_OOM;
    c->shares_geometry = true;
    c->rtab_tried = true;   // a child reads the parent's table (if built) and never builds its own
    c->rows_ok = c->rows_compact = false;   // batched flows contract every row
    c->profiler = new (std::nothrow) Profiler();
    c->prof = false;
    for (auto &sl : c->slots) sl = ProfileSlot();
    c->d_V = c->d_Z = c->d_Vs = c->d_k = c->d_acc = c->d_Zwork = nullptr;
    c->d_Vf = nullptr;
    c->d_red = nullptr;
    c->h_red = nullptr;
    c->d_gy = c->d_gys = c->d_gk = c->d_gacc = c->d_gzka = c->d_gt2 = nullptr;
    c->err.clear();
    const size_t N = c->pb.N, n3 = N * N * N;
    qpfrg_status s = QPFRG_ERR_OOM;
    if (!c->profiler || (s = dev_alloc(c, &c->d_V, n3, "V")) || (s = dev_alloc(c, &c->d_Vs, n3, "V stage")) ||
        (s = dev_alloc(c, &c->d_k, n3, "k")) || (s = dev_alloc(c, &c->d_acc, n3, "acc")) ||
        (s = dev_alloc(c, &c->d_Vf, n3, "V fp32")) || (s = dev_alloc(c, &c->d_Z, N, "Z")) ||
        (s = dev_alloc(c, &c->d_Zwork, N, "Z work")) || (s = dev_alloc(c, &c->d_red, 5, "reduction"))) {
        qpfrg_destroy(c);
        return s;
    }
    if (cudaMallocHost((void **)&c->h_red, 5 * sizeof(unsigned long long)) != cudaSuccess) {
        qpfrg_destroy(c);
        return QPFRG_ERR_OOM;
    }
    if (c->opt.sigma_ode && (s = gflow_alloc(c)) != QPFRG_OK) {
        qpfrg_destroy(c);
        return s;
    }
    std::vector<double> h(n3, U);
    cudaError_t e = cudaMemcpy(c->d_V, h.data(), n3 * sizeof(double), cudaMemcpyHostToDevice);
    h.assign(N, 1.0);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_Z, h.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        qpfrg_destroy(c);
        return QPFRG_ERR_CUDA;
    }
    c->lambda = lambda0;
    c->lambda_end = lambda_end;
    c->steps = 0;
    c->status = QPFRG_FLOW_RUNNING;
    c->max_abs_v = std::fabs(U);
    c->lambda_c = 0.0;
    c->pending = false;
    c->c4v_state = c->pb.mode == QPFRG_GRID_WEDGE || c->pb.mode == QPFRG_GRID_SHELL;
    *out = c;
    return QPFRG_OK;
}

qpfrg_status qpfrg_flow_batch(const qpfrg_lattice *lattice, const qpfrg_fine_grid *grid, qpfrg_regulator regulator,
                              const qpfrg_options *options, int n_flows, const qpfrg_flow_spec *specs,
                              void *cuda_stream, qpfrg_flow_result *results)
{
    if (!lattice || !grid || !specs || !results || n_flows < 1) return QPFRG_ERR_INVALID;
    qpfrg_options opt;
    if (options)
        opt = *options;
    else
        qpfrg_default_options(&opt);
    const bool tflow = regulator == QPFRG_REG_TEMPERATURE;
    for (int i = 0; i < n_flows; ++i) {
        const qpfrg_flow_spec &f = specs[i];
        if (!std::isfinite(f.U) || !std::isfinite(f.lambda0) || !std::isfinite(f.lambda_end)) return QPFRG_ERR_INVALID;
        if (tflow && !(f.lambda0 > 0.0 && f.lambda_end > 0.0)) return QPFRG_ERR_INVALID;
    }
    // the batched device path: every group's steps on the device, flows
    // stopping there, captured as CUDA graphs (batch.cu)
    if (batch_device_path(grid, regulator, opt, n_flows, specs)) {
        std::string err;
        const qpfrg_status st = flow_batch_device(lattice, grid, opt, n_flows, specs,
                                                  reinterpret_cast<cudaStream_t>(cuda_stream), results, err);
        if (st != QPFRG_OK) fprintf(stderr, "qpfrg_flow_batch: %s\n", err.c_str());
        return st;
    }
    // flows grouped by patch count: one geometry, one scratch set and one stream per group
    std::vector<int> sizes;
    for (int i = 0; i < n_flows; ++i)
        if (std::find(sizes.begin(), sizes.end(), specs[i].n_p) == sizes.end()) sizes.push_back(specs[i].n_p);
    const int G = (int)sizes.size();
    std::vector<cudaStream_t> streams(G, nullptr);
    std::vector<qpfrg_ctx *> parents(G, nullptr), flows(n_flows, nullptr);
    std::vector<int> group_of(n_flows, 0);
    qpfrg_status st = QPFRG_OK;
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t ev = nullptr;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, caller);
    auto cleanup = [&]() {
        for (auto *c : flows) qpfrg_destroy(c);
        for (auto *c : parents) qpfrg_destroy(c);
        for (auto s2 : streams)
            if (s2) cudaStreamDestroy(s2);
        if (ev) cudaEventDestroy(ev);
    };
    for (int g = 0; g < G && st == QPFRG_OK; ++g) {
        if (cudaStreamCreateWithFlags(&streams[g], cudaStreamNonBlocking) != cudaSuccess) {
            st = QPFRG_ERR_CUDA;
            break;
        }
        cudaStreamWaitEvent(streams[g], ev, 0);
        int first = 0;
        while (specs[first].n_p != sizes[g]) ++first;
        st = qpfrg_create(lattice, sizes[g], grid, specs[first].U, specs[first].lambda0, regulator, &opt,
                          streams[g], &parents[g]);
        // launch shapes of the group, measured on its first flow's initial state
        if (st == QPFRG_OK && opt.autotune) st = qpfrg_autotune(parents[g], specs[first].lambda0, nullptr);
    }
    for (int i = 0; i < n_flows && st == QPFRG_OK; ++i) {
        group_of[i] = (int)(std::find(sizes.begin(), sizes.end(), specs[i].n_p) - sizes.begin());
        st = make_child(parents[group_of[i]], specs[i].U, specs[i].lambda0, specs[i].lambda_end, &flows[i]);
    }
    if (st != QPFRG_OK) {
        cleanup();
        return st;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int> done_steps(n_flows, 0);
    for (;;) {
        bool any = false;
        // one step for every running flow; flows of a group queue on its stream
        for (int i = 0; i < n_flows && st == QPFRG_OK; ++i) {
            qpfrg_ctx *c = flows[i];
            if (c->status != QPFRG_FLOW_RUNNING) continue;
            if (done_steps[i] >= opt.max_steps) {
                c->status = QPFRG_FLOW_MAX_STEPS;
                continue;
            }
            st = enqueue_step(c);
            any = any || c->pending;
        }
        for (int g = 0; g < G; ++g)
            if (cudaStreamSynchronize(streams[g]) != cudaSuccess && st == QPFRG_OK) st = QPFRG_ERR_CUDA;
        for (int i = 0; i < n_flows; ++i) {
            if (!flows[i]->pending) continue;
            const qpfrg_status s2 = finish_step(flows[i]);
            ++done_steps[i];
            if (s2 != QPFRG_OK && st == QPFRG_OK) st = s2;
        }
        if (st != QPFRG_OK || !any) break;
        if (opt.timeout_s > 0.0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > opt.timeout_s) {
            for (auto *c : flows)
                if (c->status == QPFRG_FLOW_RUNNING) c->status = QPFRG_FLOW_TIMEOUT;
            break;
        }
    }
    for (int i = 0; i < n_flows; ++i) fill_result(flows[i], &results[i]);
    cleanup();
    return st;
}

qpfrg_status qpfrg_state_size(qpfrg_t c, size_t *bytes)
{
    if (!c || !bytes) return QPFRG_ERR_INVALID;
    *bytes = sizeof(StateHeader) + (n3_of(c) + c->pb.N + (c->d_gy ? gflow_small_len(c) : 0)) * sizeof(double);
    return QPFRG_OK;
}

qpfrg_status qpfrg_get_state(qpfrg_t c, void *h_buf, size_t bytes)
{
    size_t need = 0;
    if (qpfrg_state_size(c, &need) != QPFRG_OK || !h_buf) return QPFRG_ERR_INVALID;
    if (bytes < need) return set_err(c, QPFRG_ERR_INVALID, "state buffer too small");
    StateHeader hd{};
    hd.magic = kStateMagic;
    hd.version = kStateVersion;
    hd.N = c->pb.N;
    hd.status = c->status;
    hd.steps = c->steps;
    hd.lambda = c->lambda;
    hd.max_abs_v = c->max_abs_v;
    hd.lambda_c = c->lambda_c;
    std::memcpy(h_buf, &hd, sizeof(hd));
    unsigned char *p = static_cast<unsigned char *>(h_buf) + sizeof(hd);
    cudaError_t e = cudaMemcpyAsync(p, c->d_V, n3_of(c) * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p + n3_of(c) * sizeof(double), c->d_Z, c->pb.N * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && c->d_gy)
        e = cudaMemcpyAsync(p + (n3_of(c) + c->pb.N) * sizeof(double), c->d_gy, gflow_small_len(c) * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "get_state");
}

qpfrg_status qpfrg_set_state(qpfrg_t c, const void *h_buf, size_t bytes)
{
    size_t need = 0;
    if (qpfrg_state_size(c, &need) != QPFRG_OK || !h_buf) return QPFRG_ERR_INVALID;
    if (bytes != need) return set_err(c, QPFRG_ERR_INVALID, "state image has the wrong size");
    StateHeader hd;
    std::memcpy(&hd, h_buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != kStateVersion || hd.N != c->pb.N)
        return set_err(c, QPFRG_ERR_INVALID, "state image header does not match this context");
    if (hd.status < QPFRG_FLOW_RUNNING || hd.status > QPFRG_FLOW_TIMEOUT || hd.steps < 0)
        return set_err(c, QPFRG_ERR_INVALID, "state image has a bad status or step count");
    const double *V = reinterpret_cast<const double *>(static_cast<const unsigned char *>(h_buf) + sizeof(hd));
    const double *Z = V + n3_of(c);
    if (!std::isfinite(hd.lambda)) return set_err(c, QPFRG_ERR_NONFINITE, "state image holds NaN or Inf");
    // The image is staged in the RK scratch buffers (free between steps) and
    // checked there on the device: finiteness, max|V|, and the C4v symmetry of
    // V and Z to the rounding level of the precision that produced them (a
    // mixed-precision flow keeps it only to FP32 rounding).  A rejected image
    // leaves the state untouched.
    const bool wedge = c->pb.mode == QPFRG_GRID_WEDGE || c->pb.mode == QPFRG_GRID_SHELL;
    const double tol = c->opt.precision == QPFRG_FP64 ? 1e-12 : 1e-5;
    cudaError_t e = cudaMemcpyAsync(c->d_k, V, n3_of(c) * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_acc, Z, c->pb.N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_state upload");
    qpfrg_status st = launch_state_check(c, c->d_k, c->d_acc, wedge, tol);
    if (st != QPFRG_OK) return st;
    if ((e = cudaMemcpyAsync(c->h_red, c->d_red, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "set_state check");
    if (c->h_red[1] || c->h_red[3]) return set_err(c, QPFRG_ERR_NONFINITE, "state image holds NaN or Inf");
    double m = 0.0;
    std::memcpy(&m, &c->h_red[0], sizeof(double));
    if ((e = cudaMemcpyAsync(c->d_V, c->d_k, n3_of(c) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(c->d_Z, c->d_acc, c->pb.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess)
        return cuda_fail(c, e, "set_state");
    if (c->d_gy &&
        (e = cudaMemcpyAsync(c->d_gy, Z + c->pb.N, gflow_small_len(c) * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "set_state (self-energy ODE)");
    c->c4v_state = wedge && c->h_red[4] == 0;
    c->status = hd.status;
    c->steps = (int)hd.steps;
    c->lambda = hd.lambda;
    c->lambda_c = hd.lambda_c;
    c->max_abs_v = m;
    return QPFRG_OK;
}

qpfrg_status qpfrg_read_state(qpfrg_t c, double *d_V, double *d_Z)
{
    if (!c) return QPFRG_ERR_INVALID;
    cudaError_t e = cudaSuccess;
    if (d_V) e = cudaMemcpyAsync(d_V, c->d_V, n3_of(c) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && d_Z)
        e = cudaMemcpyAsync(d_Z, c->d_Z, c->pb.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? QPFRG_OK : cuda_fail(c, e, "read_state");
}

qpfrg_status qpfrg_geometry(qpfrg_t c, int *n_p, int *n_fine, double *h_kf, double *h_fine)
{
    if (!c) return QPFRG_ERR_INVALID;
    if (n_p) *n_p = c->pb.N;
    if (n_fine) *n_fine = c->pb.M;
    if (h_kf) std::memcpy(h_kf, c->kf.data(), c->kf.size() * sizeof(double));
    if (h_fine)
        for (int p = 0; p < c->pb.M; ++p) {
            h_fine[4 * p] = c->fk[2 * p];
            h_fine[4 * p + 1] = c->fk[2 * p + 1];
            h_fine[4 * p + 2] = c->fw[p];
            h_fine[4 * p + 3] = c->fpatch[p];
        }
    return QPFRG_OK;
}

qpfrg_status qpfrg_set_profiling(qpfrg_t c, int on)
{
    if (!c) return QPFRG_ERR_INVALID;
    if (!on) flush_profile(c);
    c->prof = on != 0;
    return QPFRG_OK;
}

qpfrg_status qpfrg_profile_reset(qpfrg_t c)
{
    if (!c) return QPFRG_ERR_INVALID;
    flush_profile(c);
    for (auto &s : c->slots) s = ProfileSlot();
    return QPFRG_OK;
}

int qpfrg_profile_count(void) { return K_COUNT; }

const char *qpfrg_profile_name(int id) { return (id >= 0 && id < K_COUNT) ? kKernelNames[id] : ""; }

qpfrg_status qpfrg_profile_get(qpfrg_t c, int id, double *ms, long long *launches)
{
    if (!c || id < 0 || id >= K_COUNT) return QPFRG_ERR_INVALID;
    flush_profile(c);
    if (ms) *ms = c->slots[id].ms;
    if (launches) *launches = c->slots[id].launches;
    return QPFRG_OK;
}

}  // extern "C"
