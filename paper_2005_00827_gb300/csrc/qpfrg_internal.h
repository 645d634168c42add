// Internal declarations of the qpfrg CUDA library (sm_103a).  Not part of
// the public ABI (include/qpfrg.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qpfrg.h"

namespace qpfrg {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * kPi;
// cells per 2 pi of the FP32 wedge-projection table (rows = columns = kProjW;
// 256: the cell index of a fixed-point coordinate is its top byte)
constexpr int kProjW = 256;
// row stride of that table in bytes: 65 words, so adjacent rows start in adjacent banks
constexpr int kProjStride = 260;

// Fixed-point angles: a momentum component as turns x 2^32 in an int32, so
// that the difference of two wraps into [-pi, pi) by itself (the zone fold,
// ties at -pi) and the projection table's cell is the top byte.  The FP32
// value of such a difference is off by at most 64 units (9.4e-8 rad).
constexpr double kFxPerRad = 4294967296.0 / kTwoPi;
constexpr float kRadPerFx = (float)(kTwoPi / 4294967296.0);
// guard bands of the FP32 decisions in fixed-point units: 4e-6 rad from a ray
// and from the zone edge
constexpr float kFxGuard = (float)(4e-6 * kFxPerRad);
constexpr float kFxEdge = (float)((kPi - 4e-6) * kFxPerRad);

// angle (rad, FP64) -> fixed point; the same on host and device (round to
// nearest even of the same FP64 product)
__host__ __device__ inline int angle_fx(double r)
{
    const double t = r * (1.0 / kTwoPi);
    return (int)(unsigned)(long long)llrint((t - rint(t)) * 4294967296.0);
}

// Byte of fine point (t, s) (t angular, s radial) of a patch in the partner
// maps.  With n_theta a multiple of 4 the bytes come in blocks of four angles,
// radius-major inside a block: one lane of the loop kernels reads the partner
// patches of four consecutive angles at its radius as one aligned word, and the
// 32 lanes of a warp (32 radii) read 128 contiguous bytes.  Otherwise angle-major.
__host__ __device__ inline int part_byte(int t, int s, int nt, int nr)
{
    return nt % 4 == 0 ? (((t >> 2) * nr + s) << 2) + (t & 3) : t * nr + s;
}

// Kernel ids of the built-in profiler (order = qpfrg_profile_name).
enum KernelId {
    K_PARTNER_MAP = 0,
    K_BUBBLE,
    K_CONTRACT_PP,
    K_CONTRACT_CR,
    K_CONTRACT_D,
    K_SIGMA_Z,
    K_SIGMA_HIST,
    K_SIGMA_GRID,
    K_Z_UPDATE,
    K_RK_STAGE,
    K_RK_FINAL,
    K_CONVERT,
    K_TC_PREP,
    K_TC_PP,
    K_TC_CR,
    K_TC_D,
    K_KP_TABLE,
    K_RTAB,
    K_ROWS_EXPAND,
    K_COUNT
};

// Launch shapes chosen by qpfrg_autotune (0 = built-in heuristic).
struct Tuning {
    int bubble_qchunk = 0;      // transfers per loop-kernel CTA
    int bubble_transfers = 0;   // transfers per warp pass of the FP32 loop kernels (2 or 4; 0: 2)
    int sigma_qblocks = 0;      // blocks of 512 loop points q per self-energy CTA
    int tc_splits[3] = {0, 0, 0};   // split-K factors of the pp, cr, d contractions
};

// Problem constants that every kernel needs, passed by value.
struct Problem {
    int N;           // patches
    int M;           // fine points
    int P;           // fine points per patch (wedge: n_theta*n_r; lattice: 1)
    int n_theta, n_r;  // fine grid per patch (lattice: 1 x 1)
    int mode;        // qpfrg_grid_mode
    int L;           // lattice mode: side length
    int n_shell;     // energy shells per wedge (1 outside shell mode)
    double shell_D;  // shell mode: energy width of a shell
    double t, tp, mu;
    int regulator;   // qpfrg_regulator
    int propagator;  // qpfrg_propagator
    unsigned channels;
    double T_fixed;
    double eta;
};

// Device tables, FP64 and FP32 copies.  Fine points are stored patch-major:
// point p = a*P + local, local = t*n_r + s (angle-major, radius-minor).
template <typename R>
struct FineTable {
    R *kx, *ky;          // momenta
    R *cx, *sx, *cy, *sy;// cos/sin of the momentum components
    R *xi;               // bare dispersion
    R *w;                // quadrature weight
};

template <typename R>
struct TransferTable {   // for Q index x*N + y (pp: k_F(x)+k_F(y); ph: k_F(x)-k_F(y))
    R *cx, *sx, *cy, *sy;
};

// Buffers of the tensor-core contraction (QPFRG_MIXED_TC), index 0 = hi, 1 = lo:
// the vertex (B) operands in tensor-core tiles (tile_index, Npad-row x 64-wide
// tiles, reduction length padded to Kp / Kpd with zeros) and their TMA maps.
// The A operands are formed in shared memory by the contraction itself.
struct TcBuffers {
    __nv_bfloat16 *Bpp[2] = {nullptr, nullptr};   // [Npad][Kp]
    __nv_bfloat16 *Bcr[2] = {nullptr, nullptr};   // [Npad][Kp]
    __nv_bfloat16 *Bd[2] = {nullptr, nullptr};    // [Npad][Kpd]
    float *VT = nullptr;                          // row-factor tables [3][N^2][N] (tc_prep)
    int Npad = 0;
    long Kp = 0, Kpd = 0;                         // N^2 up to 64 and 2 Kp (d: halves at 0 and Kp)
    long RT = 0, KB = 0;                          // row tiles (N^2 / 128) and k blocks (Kp / 64) of the table
    CUtensorMap tmB[3][2];                        // TMA maps of the tiles: [pp, cr, d][hi, lo]
    CUtensorMap tmTab;                            // TMA map of the FP32 weighted loop-kernel table
};

// Element offset of (row r, reduction index k) in the tile layout of a BF16
// operand with `rows` rows per tile (Npad for B) and reduction length Kp (a
// multiple of 64): tiles ordered (row tile, k tile), each tile in the K-major
// 128-byte-swizzle order of the tcgen05 descriptors: row rr's 64 elements
// (128 B) at rr * 64, its 8-element chunk c stored at chunk c ^ (rr % 8).
__host__ __device__ inline long tile_index(long r, long k, int rows, long Kp)
{
    const long rt = r / rows, rr = r - rt * rows;
    const long kt = k >> 6, kk = k & 63;
    return (rt * (Kp >> 6) + kt) * (long)rows * 64 + rr * 64 + ((((kk >> 3) ^ (rr & 7)) << 3) | (kk & 7));
}

// FP64 projection of a momentum onto its patch.  Lattice: nearest lattice
// momentum.  Wedge and shell: fold each component into [-pi, pi] (ties to
// even), wedge of the angle (nearest centre 2 pi w / N_a, half-open), and in
// shell mode the shell floor(xi / D + n_s / 2) of the folded momentum's
// energy, clamped to the outer shells (the products of xi rounded one by one,
// as written, without fused multiply-adds).
__device__ __forceinline__ int project_fp64(double kx, double ky, const Problem &pb)
{
    if (pb.mode == QPFRG_GRID_LATTICE) {
        const int L = pb.L;
        long m1 = (long)rint(kx * L / kTwoPi) % L;
        long m2 = (long)rint(ky * L / kTwoPi) % L;
        if (m1 < 0) m1 += L;
        if (m2 < 0) m2 += L;
        return (int)(m1 * L + m2);
    }
    const double x = __dsub_rn(kx, __dmul_rn(kTwoPi, rint(kx / kTwoPi)));
    const double y = __dsub_rn(ky, __dmul_rn(kTwoPi, rint(ky / kTwoPi)));
    const int ns = pb.n_shell, Na = pb.N / ns;
    long w = (long)floor(atan2(y, x) / (kTwoPi / Na) + 0.5);
    w %= Na;
    if (w < 0) w += Na;
    if (ns == 1) return (int)w;
    const double cx = cos(x), cy = cos(y);
    const double xi = __dsub_rn(__dsub_rn(__dmul_rn(-2.0 * pb.t, __dadd_rn(cx, cy)),
                                          __dmul_rn(__dmul_rn(4.0 * pb.tp, cx), cy)),
                                pb.mu);
    long sh = (long)floor(__dadd_rn(xi / pb.shell_D, 0.5 * ns));
    sh = sh < 0 ? 0 : (sh > ns - 1 ? ns - 1 : sh);
    return (int)(w * ns + sh);
}

// Element offset of (family f, row Q, column k) in the tiled loop-kernel
// table of the tensor-core path, [f][Q / 128][k / 64][(k % 64) / 32][Q % 128][k % 32]
// with RT = ceil(N^2 / 128) row tiles and KB = ceil(N^2 / 64) k blocks per
// family: one 128 x 32 box of the contraction is 16 KB of contiguous memory.
__host__ __device__ inline long tc_table_index(int f, long Q, long k, long RT, long KB)
{
    return ((((f * RT + (Q >> 7)) * KB + (k >> 6)) * 2 + ((k >> 5) & 1)) * 128 + (Q & 127)) * 32 + (k & 31);
}

struct ProfileSlot {
    double ms = 0.0;
    long long launches = 0;
};

// Representatives of one (family, patch) of the C4v-reduced loop kernels:
// d_lrepQ[start .. start + count) (symmetry.cu).
struct LoopGroup {
    int fam, a, start, count;
};

// C4v element g = m | (reflection << 2) acting on patch j (ns energy shells
// per wedge, N_a = N / ns wedges): wedge w -> +-w + m N_a / 4 (mod N_a), the
// shell kept.
__host__ __device__ inline int c4v_apply(int g, int j, int N, int ns)
{
    const int Na = N / ns, w = j / ns, sh = j - w * ns;
    const int off = (g & 3) * (Na / 4);
    int r = (g & 4) ? off - w : w + off;
    r %= Na;
    return (r < 0 ? r + Na : r) * ns + sh;
}

// inverse element: rotations by m -> by 4 - m; every reflection is an involution
__host__ __device__ inline int c4v_inverse(int g) { return (g & 4) ? g : ((4 - (g & 3)) & 3); }

}  // namespace qpfrg

struct qpfrg_ctx {
    qpfrg::Problem pb{};
    qpfrg_options opt{};
    int n_theta = 0, n_r = 0;
    double U = 0.0, lambda0 = 0.0;
    cudaStream_t stream = nullptr;
    int device = 0;

    // host geometry (FP64)
    std::vector<double> kf;      // N x 2
    std::vector<double> fk;      // M x 2
    std::vector<double> fw;      // M
    double fw_max = 0.0;         // max of fw
    std::vector<int> fpatch;     // M

    // device geometry
    qpfrg::FineTable<double> f64{};
    qpfrg::FineTable<float> f32{};
    qpfrg::TransferTable<double> qpp64{}, qph64{};
    qpfrg::TransferTable<float> qpp32{}, qph32{};
    double *d_kf = nullptr;      // N x 2
    double *d_xij = nullptr;     // N: xi(k_F(j))
    float *d_xij_f = nullptr;    // N: xi(k_F(j)) in FP32
    float4 *d_bnd = nullptr;     // N: (cos hi, cos lo, sin hi, sin lo) of the ray between wedges j-1 and j
    float *d_qxl = nullptr, *d_qyl = nullptr;   // M: FP32 residuals kx - (float)kx, ky - (float)ky
    float4 *d_kp = nullptr;      // [target][p]: k_j + p as FP32 hi/lo pairs (self-energy scratch)
    float4 *d_kcs = nullptr;     // [target]: cos/sin of k_j (self-energy scratch)
    uint8_t *d_rtab = nullptr;   // patch of r per (irreducible target, p, q) of the flow's Z (sigma.cu)
    bool rtab_tried = false;     // built, or found not to fit, once per context
    uint8_t *d_ptab = nullptr;   // W rows x kProjStride bytes: cell table of the FP32 wedge projection (wedge mode, N <= 254)
    double *d_Qpp = nullptr, *d_Qph = nullptr;  // N^2 x 2 transfer momenta (FP64)
    uint8_t *d_part = nullptr;   // 2 x N^2 x M partner patches (pp family, then ph)

    // C4v-reduced loop kernels (symmetry.cu): one row per orbit of (Q, a),
    // written to its images; rows whose partner maps break covariance are
    // evaluated by themselves
    bool loop_red = false;
    std::vector<qpfrg::LoopGroup> lgroups;
    int *d_lrepQ = nullptr;      // transfer Q of each representative row (families concatenated)
    int *d_lnimg = nullptr;      // number of image rows of each representative
    int2 *d_limg = nullptr;      // 8 slots per representative: (Q', a' | g << 16)
    int4 *d_ltask = nullptr;     // (family, patch, first representative, count) per CTA
    long n_lrep = 0;
    int ltask_qchunk = 0, n_ltask = 0;
    long long loop_evals_red = 0;   // loop-kernel evaluations of one reduced RHS
    long loop_mismatch_rows = 0;    // rows evaluated by themselves (covariance broken)

    // C4v row orbits of the tensor-core contraction (symmetry.cu): with a
    // C4v-symmetric state (V, Z) every channel's output row Q = (x, y) at
    // column n equals its representative's row at column g^-1 n, Q = g rep, so
    // only representative rows are tabled and contracted and the result is
    // expanded (contract.cu).  Built when every loop-kernel row is covariant.
    bool rows_ok = false;
    bool rows_compact = false;   // the table of the current RHS holds representative rows only
    int n_rrep = 0;
    int *d_rrep = nullptr;       // Q of each representative row
    int *d_rowmap = nullptr;     // per Q: representative index | g << 24, Q = g rep
    int4 *d_rtask = nullptr;     // (family, patch, first representative, count) per loop-kernel CTA
    int rtask_qchunk = 0, n_rtask = 0;
    double *d_outc = nullptr;    // [channel][representative][n] contraction rows
    long long loop_evals_rows = 0;  // loop-kernel evaluations of one RHS on representative rows

    // bubble tables B[f][Q][a][b] (FP32 or FP64 according to precision)
    void *d_B = nullptr;
    size_t B_bytes = 0;
    void *loop_out = nullptr;           // set only inside launch_loop_rows
    const int *loop_active = nullptr;   // set only inside launch_loop_rows

    qpfrg::TcBuffers tc;
    unsigned *d_tc_err = nullptr;   // set by a tensor-core CTA whose bounded wait expired

    // flow state and work buffers
    double *d_V = nullptr, *d_Z = nullptr;
    double *d_Vs = nullptr, *d_k = nullptr, *d_acc = nullptr, *d_ones = nullptr;
    float *d_Vf = nullptr;       // FP32 copy of the RHS input (MIXED)
    double *d_Zwork = nullptr;   // Z computed at the start of a step
    // interaction flow with the self-energy ODE (gflow.cu): small state
    // [s1, s2, Re S, Im S, Re S', Im S'], its RK4 stage, derivative and sum;
    // Z, K, A (N each) and Abar; the binned two-loop term on the grid
    double *d_gy = nullptr, *d_gys = nullptr, *d_gk = nullptr, *d_gacc = nullptr;
    double *d_gzka = nullptr, *d_gt2 = nullptr;
    double *d_sig = nullptr;     // N x 2 Re Sigma at xi_j +- 2T
    int *d_jirr = nullptr;       // C4v-irreducible patches 0..N/8 (wedge mode)
    int *d_rep = nullptr;        // slot of each patch's representative in d_jirr
    int n_irr = 0;
    // targets of the frequency-grid self-energy of a C4v-symmetric state: the
    // irreducible patches plus the zone-edge patches N/4, N/2, 3N/4, whose sums
    // differ from patch 0's where a momentum lands on |k_x| or |k_y| = pi
    int *d_jgrid = nullptr;
    int *d_repgrid = nullptr;    // slot of each patch's representative in d_jgrid
    int n_grid = 0;
    bool c4v_state = false;      // flow state V, Z is C4v symmetric
    double *d_hist = nullptr;    // Sigma frequency-grid histogram (lazily sized)
    size_t hist_elems = 0;
    unsigned long long *d_red = nullptr;  // [0] max|V| bits, [1] nonfinite flag; [2..4] state-image checks
    unsigned long long *h_red = nullptr;  // pinned mirror
    double lambda = 0.0;
    double lambda_end = 0.0;     // end of this flow (batched flows differ)
    bool shares_geometry = false;  // tables and scratch belong to another context
    // step in flight (enqueued, not yet finished): x, h, max|V| before it
    bool pending = false;
    double pend_x = 0.0, pend_h = 0.0, pend_m = 0.0;
    int steps = 0;
    int status = QPFRG_FLOW_RUNNING;
    double max_abs_v = 0.0;
    double lambda_c = 0.0;

    // profiling
    bool prof = false;
    qpfrg::Tuning tune;          // launch shapes (qpfrg_autotune / qpfrg_set_tuning)
    qpfrg::ProfileSlot slots[qpfrg::K_COUNT];
    void *profiler = nullptr;    // pending CUDA-event pairs (qpfrg_api.cu)

    std::string err;
};

namespace qpfrg {

// geometry.cu
qpfrg_status build_host_geometry(qpfrg_ctx *c);
double shell_width(const Problem &pb, double given);   // shell mode: the width of a shell
qpfrg_status upload_geometry(qpfrg_ctx *c);

// bubble.cu: fill the bubble tables for the given Lambda and Z (device ptr).
// z_symmetric: Z is C4v symmetric (needed by the reduced launch with
// quasi-particle lines, whose loop kernels depend on Z).
// d_K: Katanin factors of the interaction flow's S line (nullptr = 1).
// state_symmetric: V and Z are C4v symmetric, so that (tensor-core precision,
// row orbits built) only representative rows are tabled; sets c->rows_compact
// for the contraction of the same RHS.
qpfrg_status launch_bubbles(qpfrg_ctx *c, double lambda, const double *d_Z, bool z_symmetric,
                            const double *d_K = nullptr, bool state_symmetric = false);

qpfrg_status launch_loop_rows(qpfrg_ctx *c, double lambda, float *rows, const int *active, bool compact = false);

// symmetry.cu: C4v orbits of the loop-kernel rows and the reduced launch's tasks
qpfrg_status build_loop_orbits(qpfrg_ctx *c);
qpfrg_status loop_tasks(qpfrg_ctx *c, int qchunk, int *ntask);
qpfrg_status row_tasks(qpfrg_ctx *c, int qchunk, int *ntask);

// contract.cu: d_out (N^3 FP64) += scale * contraction of the bubble tables.
// V input is FP64 (precision FP64) or FP32 (MIXED).
qpfrg_status launch_contractions(qpfrg_ctx *c, const void *d_Vin, double scale, double *d_out);

// sigma.cu
qpfrg_status launch_sigma_z(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z,
                            double *d_Zout, bool use_symmetry);
// d_K: the interaction flow's line weights with these Katanin factors (the
// generic kernel); nullptr: the temperature flow's Z_a Z_b Z_c
qpfrg_status launch_sigma_grid(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z,
                               double *d_re, double *d_im, const double *d_K = nullptr);
qpfrg_status launch_sigma_lines(qpfrg_ctx *c, double T, const double *d_V, const double *d_Z, const double *d_K);

// gflow.cu: interaction flow with the self-energy ODE
long gflow_small_len(const qpfrg_ctx *c);
qpfrg_status gflow_alloc(qpfrg_ctx *c);
qpfrg_status gflow_enqueue_stages(qpfrg_ctx *c, double x, double h);

// Per-flow vertex operands of the batched tensor-core contraction (batch.cu)
struct TcPrepFlow {
    const float *Vf;             // stage vertex (FP32)
    float *VT;                   // row-factor tables of cr and d, [3][N^2][N]
    __nv_bfloat16 *B[3][2];      // B operands of pp, cr, d: hi, lo (tiles)
};
qpfrg_status launch_tc_prep_batch(qpfrg_ctx *c, const TcPrepFlow *d_flows, const int *d_status, const double *d_h_tab,
                                  int step, int nflows);
qpfrg_status make_tile_map(qpfrg_ctx *c, CUtensorMap *map, const void *base, long elems, int box_rows);
// TMA map of a tiled weighted loop-kernel table (tc_table_index, FP32):
// rows of 32 floats, boxes of 128 rows, 128-byte swizzle
qpfrg_status make_table_map(qpfrg_ctx *c, CUtensorMap *map, const float *table);
// Batched flows (batch.cu): grid.z runs over the flows of a patch-count group;
// each flow brings its table slot, stage vertex, output and B tensor maps,
// and is skipped (uniformly, before any barrier) when it is not running or
// has no step at this row of the schedule.
struct TcBatch {
    int nflows;                       // 0: a single flow (the fields below unused)
    int step;                         // schedule row
    double cst;                       // stage offset of h (0, 1/2, 1/2, 1)
    const int *status;                // per flow, QPFRG_FLOW_RUNNING runs
    const double *h_tab;              // [step][flow] step in ln T (0: no step)
    const signed char *slot_tab;      // [step][flow] table slot
    const double *x;                  // per flow: ln T at the start of the step
    float *const *rows;               // table per slot
    const float *const *Vf, *const *VT;
    double *const *out;
    double *const *outc;              // per flow: [ch][representative][n] rows (row orbits), nullptr: every row
    const CUtensorMap *maps;          // [flow][ch][hi, lo]
    const CUtensorMap *tab_maps;      // table map per slot
};

qpfrg_status launch_tc_fused_batch(qpfrg_ctx *c, int ch, const TcBatch &bt, double sign);
// contract.cu: out_f += the expansion of the representative rows outc_f of
// every running flow f with a step at this row of the schedule
qpfrg_status launch_rows_expand_batch(qpfrg_ctx *c, const TcBatch &bt);

// batch.cu: batched temperature flows (qpfrg_flow_batch)
bool batch_device_path(const qpfrg_fine_grid *grid, qpfrg_regulator regulator, const qpfrg_options &opt, int n,
                       const qpfrg_flow_spec *specs);
qpfrg_status flow_batch_device(const qpfrg_lattice *lattice, const qpfrg_fine_grid *grid, const qpfrg_options &opt,
                               int n, const qpfrg_flow_spec *specs, cudaStream_t caller, qpfrg_flow_result *results,
                               std::string &err);

// tc_prep.cu / tc_fused.cu: tensor-core contraction
qpfrg_status launch_tc_prep(qpfrg_ctx *c);
qpfrg_status tc_make_maps(qpfrg_ctx *c);   // TMA maps of the tensor-core operand tiles
qpfrg_status launch_tc_fused(qpfrg_ctx *c, int ch, double scale, double *out, int kid);

// ode.cu
qpfrg_status launch_convert_f32(qpfrg_ctx *c, const double *d_in, float *d_out, long n);
qpfrg_status launch_rk_stage(qpfrg_ctx *c, int stage, double h, const double *d_V,
                             const double *d_k, double *d_acc, double *d_Vs, float *d_Vf);
qpfrg_status launch_state_check(qpfrg_ctx *c, const double *d_V, const double *d_Z, bool c4v_test, double tol);
qpfrg_status launch_rk_final(qpfrg_ctx *c, double h, double *d_V, const double *d_acc,
                             const double *d_k);
qpfrg_status launch_check_finite(qpfrg_ctx *c, const double *d_x, long n);

// profiling helpers (qpfrg_api.cu)
void prof_begin(qpfrg_ctx *c);
void prof_end(qpfrg_ctx *c, int id);
qpfrg_status cuda_fail(qpfrg_ctx *c, cudaError_t e, const char *what);

inline int div_up(long a, long b) { return (int)((a + b - 1) / b); }

}  // namespace qpfrg
