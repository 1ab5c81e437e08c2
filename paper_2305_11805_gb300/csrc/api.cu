// C ABI of libpanna_gb300: context, workspace and the sequencing of the stages of the
// energy / force / weight-gradient path.  Every step of the path runs in the kernels of
// this library; there is no host or CPU fallback.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "common.cuh"
#include "mlp.cuh"

using namespace panna;

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

static panna_status fail(panna_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void panna::set_last_error_message(const char* msg) { g_last_error = msg; }

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(PANNA_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
    } while (0)

#define ST(call)                                  \
    do {                                          \
        panna_status s_ = (call);                 \
        if (s_ != PANNA_OK) return s_;            \
    } while (0)

// ------------------------------------------------------------------ workspace arena

namespace {

struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    bool sizing = true;
    template <class T>
    T* take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = sizing ? nullptr : reinterpret_cast<T*>(base + off);
        off += (n ? n : 1) * sizeof(T);
        return p;
    }
};

constexpr int kNumVariants = 6;   // most variants of one descriptor-family kernel
// variants per kernel: descriptor and JVP 0..4, adjoint 0..5
constexpr int kKindVariants[3] = {5, 6, 5};
const char* kStages[] = {"neighbors", "descriptor", "mlp", "adjoint", "forces", "jvp", "mlp_grad", "loss"};
constexpr int kNumStages = 8;

}  // namespace

struct panna_ctx {
    int device = 0;
    DescDev d{};
    MlpPlan plan{};
    int32_t cap = 64;
    int32_t cap_c = 0;                // dynamics: candidate slots per atom (cutoff rc + skin)
    int async = 0;
    int profiling = 0;
    int ang_mode = 0;
    int autotune = 1;
    int force_variant[3] = {-1, -1, -1};   // descriptor, adjoint, jvp: -1 = tuned
    int fp32_tc = TF32_TAN | TF32_WGRAD;   // FP32 networks: first-layer products on the tensor cores
    int64_t norm_C = 0, norm_N = 0;   // loss normalisers (0 = the batch's own counts)
    LossOpts loss_opts{0, 0, 0, 0.0, 0.0};
    bool frozen[kMaxSpecies][kMaxLayers] = {};
    int last_launches = 0;
    int last_variant[3] = {-1, -1, -1};   // descriptor, adjoint, JVP variants of the last call
    DescGrid64 g64{};                 // FP64 descriptor parameters (stored Jacobians)
    QeqDev qeq{};                     // charge-equilibration constants (3-output networks)
    bool qeq_set = false;
    // autotuner: kernel variant per problem signature, measured on the first call
    // per problem signature (atoms, configurations, capacity, precision, extended angular terms)
    struct Tuned { int64_t N, C; int cap, prec, ext; int variant[3]; };   // -1 = not measured yet
    Tuned tuned[16];
    int n_tuned = 0;
    cudaEvent_t tev[3] = {};
    // captured graph
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    int graph_launches = 0;
    Arena ws;
    DevStatus* h_status = nullptr;   // pinned
    cudaEvent_t ev[kNumStages + 1] = {};
    float stage_ms[kNumStages] = {};
    bool stage_seen[kNumStages] = {};
    int stage_order[kNumStages + 1] = {};   // stages in the order they were marked
    int n_marked = 0;
};

// ------------------------------------------------------------------ workspace layout

namespace {

struct Layout {
    Work w;
    MlpBuffers mb;
    float* G = nullptr;
    float* g = nullptr;
    float* E_rows = nullptr;
    float* vir_atom = nullptr;
    double* cfg_part = nullptr;
    float* F_int = nullptr;
    float* F_tune = nullptr;
    double* E_cfg_int = nullptr;
    // training
    float* u = nullptr;
    double* alpha_cfg = nullptr;
    float* alpha_rows = nullptr;
    float* wdot = nullptr;
    double* loss_part = nullptr;
    void* tc_ws = nullptr;   // BF16 tensor-core network buffers
    void* tf_ws = nullptr;   // FP32 networks: TF32 first-layer buffers
    // dynamics: candidates of the last neighbour build (cutoff rc + skin), its positions
    int32_t* cand_count = nullptr;
    float4* cand_vec = nullptr;
    int2* cand_idx = nullptr;
    double* pos_ref = nullptr;
    double* qbuf = nullptr;   // charge equilibration: the charges of the forward pass
};

constexpr int kSplits = 16;

// TF32_* products of the first layer that run on the tensor cores in this evaluation
int tf32_mask(const panna_ctx* c, bool bf16, bool train)
{
    if (bf16 || !tf32_first_layer_ok(c->plan)) return 0;
    return c->fp32_tc & (train ? (TF32_FWD | TF32_TAN | TF32_WGRAD) : TF32_FWD);
}

void carve(panna_ctx* c, Arena& a, int64_t N, int64_t C, bool train, bool bf16, Layout& L, int cap_c = 0)
{
    const int S = c->d.S, D = c->d.D, cap = c->cap;
    const MlpPlan& p = c->plan;
    Work& w = L.w;
    w.N = N; w.C = C; w.cap = cap;
    w.cap_cells = 2 * N + C + 1;
    w.status = a.take<DevStatus>(1);
    w.geom = a.take<CfgGeom>(C);
    w.cell_count = a.take<int64_t>(w.cap_cells + 1);
    w.cell_start = a.take<int64_t>(w.cap_cells + 1);
    w.cell_fill = a.take<int32_t>(w.cap_cells);
    w.cell_atoms = a.take<int32_t>(N);
    w.atom_cell = a.take<int32_t>(N);
    w.atom_cfg = a.take<int32_t>(N);
    w.pos_hi = a.take<float4>(N);
    w.pos_lo = a.take<float4>(N);
    w.pos_hi_s = a.take<float4>(N);
    w.pos_lo_s = a.take<float4>(N);
    w.wrap = a.take<int32_t>(3 * N);
    int64_t mx = w.cap_cells + 1 > N + 1 ? w.cap_cells + 1 : N + 1;
    w.scan_tmp = a.take<int64_t>(scan_scratch_elems(mx));
    w.nb_count = a.take<int32_t>(N);
    w.nb_vec = a.take<float4>((size_t)N * cap);
    w.nb_idx = a.take<int2>((size_t)N * cap);
    // low parts of the neighbour vectors, for the float-pair angular terms of FP32 networks
    w.nb_vlo = bf16 ? nullptr : a.take<float4>((size_t)N * cap);
    w.row_of_atom = a.take<int32_t>(N);
    w.atom_of_row = a.take<int32_t>(N);
    w.seg_off = a.take<int32_t>(S + 1);
    w.blk_counts = a.take<int32_t>(((N + 1023) / 1024 + 1) * S);
    w.split_part = nullptr;
    w.split_rows = 0;
    if (N > 0 && N < kSplitAtoms) {
        w.split_rows = N * kMaxSplits;
        w.split_part = a.take<float>((size_t)w.split_rows * D);
    }
    L.G = a.take<float>((size_t)N * D);
    L.g = a.take<float>((size_t)N * D);
    L.E_rows = a.take<float>(N);
    L.vir_atom = a.take<float>(9 * (size_t)N);
    L.cfg_part = a.take<double>((size_t)C * cfg_chunks(N, C) * 10);
    L.F_int = a.take<float>(3 * (size_t)N);
    L.F_tune = a.take<float>(3 * (size_t)N);
    L.E_cfg_int = a.take<double>(C);
    L.qbuf = a.take<double>(N);
    MlpBuffers& b = L.mb;
    b.G = L.G;
    for (int l = 1; l <= p.L; ++l) {
        b.Z[l] = a.take<float>((size_t)N * p.ld[l]);
        b.A[l] = a.take<float>((size_t)N * p.ld[l]);
    }
    b.Ab = a.take<float>((size_t)N * p.max_hidden);
    b.Ab2 = a.take<float>((size_t)N * p.max_hidden);
    b.seg_off = w.seg_off;
    b.tile_start = a.take<int32_t>(S + 1);
    b.splits = kSplits;
    if (bf16) L.tc_ws = a.take<char>(tc_workspace_bytes(p, N, true));
    if (const int m = tf32_mask(c, bf16, train)) L.tf_ws = a.take<char>(tf32_workspace_bytes(p, N, m));
    if (cap_c > 0) {
        L.cand_count = a.take<int32_t>(N);
        L.cand_vec = a.take<float4>((size_t)N * cap_c);
        L.cand_idx = a.take<int2>((size_t)N * cap_c);
        L.pos_ref = a.take<double>(3 * (size_t)N);
    }
    if (train) {
        for (int l = 1; l <= p.L; ++l) {
            b.Zd[l] = a.take<float>((size_t)N * p.ld[l]);
            b.Ad[l] = a.take<float>((size_t)N * p.ld[l]);
        }
        b.Adb = a.take<float>((size_t)N * p.max_hidden);
        b.Zb = a.take<float>((size_t)N * p.max_hidden);
        b.Zdb = a.take<float>((size_t)N * p.max_hidden);
        b.part = a.take<float>((size_t)kSplits * p.P);
        L.u = a.take<float>(3 * (size_t)N);
        L.alpha_cfg = a.take<double>(C);
        L.alpha_rows = a.take<float>(N);
        L.wdot = a.take<float>((size_t)N * D);
        L.loss_part = a.take<double>(kLossParts);
    }
}

panna_status prepare(panna_ctx* c, const panna_system* sys, bool train, bool bf16, Layout& L, cudaStream_t s,
                     int cap_c = 0)
{
    const int64_t N = sys->n_atoms, C = sys->n_cfg;
    Arena sz;
    sz.sizing = true;
    carve(c, sz, N, C, train, bf16, L, cap_c);
    if (sz.off > c->ws.cap) {
        if (c->ws.base) {
            CU(cudaStreamSynchronize(s));
            CU(cudaFree(c->ws.base));
            c->ws.base = nullptr;
            c->ws.cap = 0;
        }
        size_t want = sz.off + sz.off / 8;
        cudaError_t e = cudaMalloc((void**)&c->ws.base, want);
        if (e != cudaSuccess) {
            c->ws.base = nullptr;
            return fail(PANNA_ERR_NO_MEMORY, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        c->ws.cap = want;
    }
    Arena real = c->ws;
    real.sizing = false;
    real.off = 0;
    carve(c, real, N, C, train, bf16, L, cap_c);
    L.w.sys = sys;
    return PANNA_OK;
}

// geometry = false: a batch evaluated from stored descriptors (only the counts and atom_off)
panna_status check_system(const panna_ctx* c, const panna_system* sys, bool geometry = true)
{
    if (!c || !sys) return fail(PANNA_ERR_INVALID_ARG, "null context or system");
    if (sys->n_cfg < 1 || sys->n_atoms < 0) return fail(PANNA_ERR_INVALID_ARG, "n_cfg must be >= 1, n_atoms >= 0");
    if (sys->n_atoms > ((int64_t)1 << 31) - 1) return fail(PANNA_ERR_UNSUPPORTED, "more than 2^31-1 atoms");
    if (!sys->atom_off) return fail(PANNA_ERR_INVALID_ARG, "null atom_off");
    if (geometry && (!sys->cell || !sys->pbc || (sys->n_atoms > 0 && (!sys->pos || !sys->species))))
        return fail(PANNA_ERR_INVALID_ARG, "null system array");
    return PANNA_OK;
}

void stage_mark(panna_ctx* c, int k, cudaStream_t s)
{
    if (c->profiling) {
        cudaEventRecord(c->ev[k], s);
        c->stage_seen[k] = true;
        if (c->n_marked <= kNumStages) c->stage_order[c->n_marked++] = k;
    }
}

// Reads the status word (synchronising); returns it and the overflow requirement.
panna_status collect(panna_ctx* c, const Layout& L, cudaStream_t s, int* need)
{
    CU(cudaMemcpyAsync(c->h_status, L.w.status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *need = c->h_status->need_cap;
    if (c->h_status->code == 0) return PANNA_OK;
    if (c->h_status->code == PANNA_ERR_NEIGHBOR_OVERFLOW)
        return fail(PANNA_ERR_NEIGHBOR_OVERFLOW, "atom %d has %d neighbours, capacity %d", c->h_status->bad_index,
                    c->h_status->need_cap, c->cap);
    if (c->h_status->code == PANNA_ERR_BAD_INPUT)
        return fail(PANNA_ERR_BAD_INPUT, "invalid input at index %d (species out of range, non-finite or coincident"
                    " positions, or singular cell)", c->h_status->bad_index);
    return fail((panna_status)c->h_status->code, "device error %d at index %d", c->h_status->code,
                c->h_status->bad_index);
}

// each stage lasts from its mark to the next mark in time (the last one to the end event)
void finish_profile(panna_ctx* c)
{
    if (!c->profiling) return;
    cudaEventSynchronize(c->ev[kNumStages]);
    for (int q = 0; q < c->n_marked; ++q) {
        const int k = c->stage_order[q];
        const int nxt = q + 1 < c->n_marked ? c->stage_order[q + 1] : kNumStages;
        cudaEventElapsedTime(&c->stage_ms[k], c->ev[k], c->ev[nxt]);
    }
}

// The core sequence; flags select what is computed.
struct Request {
    const float* theta = nullptr;
    int prec = PANNA_MLP_FP32;
    double* E_cfg = nullptr;
    float* E_atom = nullptr;
    float* F = nullptr;
    double* virial = nullptr;
    float* G_out = nullptr;     // descriptors only
    bool forces = false;
    bool energy = false;
    // parameter gradient
    bool train = false;         // loss from E_ref/F_ref
    bool vjp = false;           // upstream dE/dF given
    const double* E_ref = nullptr;
    const float* F_ref = nullptr;
    double w_force = 0.0;
    double* loss = nullptr;
    const double* dE = nullptr;
    const float* dF = nullptr;
    float* dtheta = nullptr;
    const Work* cand = nullptr;  // dynamics: refresh these candidates instead of a neighbour search
    const StoreView* store = nullptr;   // stored descriptors and Jacobians instead of geometry
};

// parameter ranges of the weights (biases excluded) of every layer of every species
ParamRanges weight_ranges(const MlpPlan& p)
{
    ParamRanges r{};
    for (int s = 0; s < p.S; ++s)
        for (int l = 0; l < p.L; ++l) {
            r.off[r.n] = p.w_off[s][l];
            r.len[r.n] = (int64_t)p.widths[s][l + 1] * p.widths[s][l];
            ++r.n;
        }
    return r;
}

// parameter ranges (weights and biases) of the frozen layers
ParamRanges frozen_ranges(const panna_ctx* c)
{
    ParamRanges r{};
    const MlpPlan& p = c->plan;
    for (int s = 0; s < p.S; ++s)
        for (int l = 0; l < p.L; ++l)
            if (c->frozen[s][l]) {
                r.off[r.n] = p.w_off[s][l];
                r.len[r.n] = (int64_t)p.widths[s][l + 1] * (p.widths[s][l] + 1);
                ++r.n;
            }
    return r;
}

// Kernel variants of the descriptor-family kernels for this problem signature (0 blocked,
// 1 flattened, 2 / 3 / 4 compensated with 32 / 16 / 8 lanes per unit; the adjoint's 4 is the
// flattened compensated walk and its 5 the diagonal-order walk without shared-memory atomics):
// measured once per kernel
// (each variant launched once to warm up, then timed over three launches with CUDA events on
// the caller's stream),
// then cached.  Asynchronous calls never measure (they may be under stream capture) and use
// the cached or default choice.
enum { KV_DESC = 0, KV_ADJ = 1, KV_JVP = 2 };

template <class Launch>
int tuned_variant_(panna_ctx* c, const panna_system* sys, int prec, int kind, cudaStream_t s, Launch launch, bool ext);

// ext (descriptor with FP32 networks, force tolerance 1e-5 of RMS): only the kernels that carry
// the angular terms as float pairs (variants 0 and 1) are candidates.  The compensated FP32
// kernels keep the angle in single floats, whose rounding (about 6e-8 rad) the zeta-th power
// turns into ~1e-6 relative per term; on the 1024 molecules that put one atom's force at
// 0.95-1.16e-5 of RMS against 4.3e-6 with the float pairs.
template <class Launch>
int tuned_variant(panna_ctx* c, const panna_system* sys, int prec, int kind, cudaStream_t s, Launch launch,
                  bool ext = false)
{
    const int v = tuned_variant_(c, sys, prec, kind, s, launch, ext && kind == KV_DESC);
    c->last_variant[kind] = v;
    return v;
}

template <class Launch>
int tuned_variant_(panna_ctx* c, const panna_system* sys, int prec, int kind, cudaStream_t s, Launch launch, bool ext)
{
    if (c->force_variant[kind] >= 0) return c->force_variant[kind];
    panna_ctx::Tuned* t = nullptr;
    for (int k = 0; k < c->n_tuned; ++k) {
        panna_ctx::Tuned& q = c->tuned[k];
        if (q.N == sys->n_atoms && q.C == sys->n_cfg && q.cap == c->cap && q.prec == prec && q.ext == (int)ext)
            t = &q;
    }
    if (t && t->variant[kind] >= 0) return t->variant[kind];
    const int fallback = (sys->n_atoms < kSplitAtoms || ext) ? 0 : (kind == KV_ADJ ? 5 : 2);
    if (!c->autotune || c->async || sys->n_atoms == 0) return fallback;
    float ms[kNumVariants] = {};
    const int nv = ext ? 2 : kKindVariants[kind];
    for (int v = 0; v < nv; ++v) launch(v);   // first launches load and configure the kernels
    int best = 0;
    // three back-to-back launches per variant: the host's launch work then overlaps the kernels
    // instead of showing up as idle device time in a single short measurement
    for (int v = 0; v < nv; ++v) {
        cudaEventRecord(c->tev[0], s);
        for (int r = 0; r < 3; ++r) launch(v);
        cudaEventRecord(c->tev[1], s);
        cudaEventSynchronize(c->tev[1]);
        cudaEventElapsedTime(&ms[v], c->tev[0], c->tev[1]);
        if (ms[v] < ms[best]) best = v;
    }
    if (!t) {
        t = &c->tuned[c->n_tuned < 16 ? c->n_tuned++ : 15];
        *t = panna_ctx::Tuned{sys->n_atoms, sys->n_cfg, c->cap, prec, (int)ext, {-1, -1, -1}};
    }
    t->variant[kind] = best;
    return best;
}

panna_status run_once(panna_ctx* c, const panna_system* sys, const Request& rq, Layout& L, cudaStream_t s)
{
    int& nl = c->last_launches;
    const int64_t N = sys->n_atoms;
    const bool grad = rq.train || rq.vjp;
    // FP32 networks get the extended-precision angular terms (force tolerance 1e-5 of RMS);
    // BF16 networks (tolerance 1e-2) the plain FP32 form
    const bool acc = c->ang_mode == 1 || (c->ang_mode == 0 && rq.prec == PANNA_MLP_FP32);
    if (!acc) L.w.nb_vlo = nullptr;   // the plain and compensated kernels read no low parts
    for (int k = 0; k < kNumStages; ++k) c->stage_seen[k] = false;
    c->n_marked = 0;
    CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
    const StoreView* sv = rq.store;
    bool g16_ready = false;   // BF16 networks: the descriptor kernel wrote their operand rows
    if (sv) {
        // stored descriptors: rows, maps and configuration indices come from the store
        L.w.row_of_atom = sv->row_of_atom;
        L.w.atom_of_row = sv->atom_of_row;
        L.w.seg_off = sv->seg_off;
        L.w.atom_cfg = sv->atom_cfg;
        L.G = sv->G;
        L.mb.G = sv->G;
        L.mb.seg_off = sv->seg_off;
        CU(mlp_tiles(c->plan, L.w.seg_off, L.mb.tile_start, s, &nl));
    } else {
        stage_mark(c, 0, s);
        if (rq.cand) CU(refresh_neighbors(*rq.cand, L.w, c->d, s, &nl));
        else CU(build_neighbors(L.w, c->d, s, &nl));
        if (rq.G_out) {
            stage_mark(c, 1, s);
            const int fv = c->force_variant[KV_DESC];
            CU(launch_descriptor(L.w, c->d, rq.G_out, nullptr, c->ang_mode != 2, s, &nl,
                                 fv >= 0 ? fv : (sys->n_atoms < kSplitAtoms ? 0 : 2)));
            if (c->profiling) cudaEventRecord(c->ev[kNumStages], s);
            return PANNA_OK;
        }
        CU(species_order(L.w, c->d.S, s, &nl));
        CU(mlp_tiles(c->plan, L.w.seg_off, L.mb.tile_start, s, &nl));
        stage_mark(c, 1, s);
        int dummy = 0;
        const int v = tuned_variant(c, sys, rq.prec, KV_DESC, s, [&](int vv) {
            launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &dummy, vv);
        }, acc);
        const bool tcp = rq.prec == PANNA_MLP_BF16 || rq.prec == PANNA_MLP_BF16_FAST;
        __nv_bfloat16 *gh = nullptr, *gl = nullptr;
        if (tcp) tc_g16(c->plan, N, rq.prec == PANNA_MLP_BF16, L.tc_ws, &gh, &gl);
        cudaError_t eb = gh ? launch_descriptor_bf16(L.w, c->d, gh, gl, L.w.row_of_atom, v, s, &nl, !acc)
                            : cudaErrorNotSupported;
        if (eb == cudaErrorNotSupported) {
            CU(launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &nl, v));
        } else {
            CU(eb);
            g16_ready = true;
        }
    }
    stage_mark(c, 2, s);
    float* F = rq.F ? rq.F : L.F_int;
    double* E_cfg = rq.E_cfg ? rq.E_cfg : L.E_cfg_int;
    const bool need_forces = rq.forces || rq.train;
    const bool tc = rq.prec == PANNA_MLP_BF16 || rq.prec == PANNA_MLP_BF16_FAST;
    const int tfm = tf32_mask(c, tc, grad);
    const bool tf = tfm != 0;
    if (tc) {
        // BF16 operands on the tensor cores: energies and dE/dG together
        CU(mlp_bf16_energy_grad(c->plan, L.mb, rq.theta, N, L.tc_ws, rq.prec == PANNA_MLP_BF16, L.E_rows, L.g,
                                L.w.status, s, &nl, g16_ready));
    } else if (tf) {
        // FP32 networks: first-layer products on the tensor cores (TF32 parts), the rest on CUDA cores
        CU(tf32_prepare(c->plan, L.mb, rq.theta, N, L.tf_ws, tfm, s, &nl));
        if (tfm & TF32_FWD) CU(tf32_forward1(c->plan, L.mb, N, L.tf_ws, tfm, L.w.status, s, &nl));
        CU(mlp_forward(c->plan, L.mb, rq.theta, N, s, &nl, (tfm & TF32_FWD) ? 1 : 0));
        CU(mlp_energy_rows(c->plan, L.mb, N, L.E_rows, s, &nl));
    } else {
        CU(mlp_forward(c->plan, L.mb, rq.theta, N, s, &nl));
        CU(mlp_energy_rows(c->plan, L.mb, N, L.E_rows, s, &nl));
    }
    if (need_forces) {
        if (!tc) {
            CU(mlp_input_grad(c->plan, L.mb, rq.theta, N, L.g, s, &nl));
        }
        stage_mark(c, 3, s);
        if (sv) {
            CU(cudaMemsetAsync(F, 0, sizeof(float) * 3 * N, s));
            CU(launch_store_adjoint(*sv, c->d, L.g, F, rq.virial ? L.vir_atom : nullptr, s, &nl));
        } else {
            int dummy = 0;
            const int variant = tuned_variant(c, sys, rq.prec, KV_ADJ, s, [&](int vv) {
                launch_adjoint(L.w, c->d, L.g, L.F_tune, nullptr, acc, vv, s, &dummy);
            });
            CU(cudaMemsetAsync(F, 0, sizeof(float) * 3 * N, s));
            CU(launch_adjoint(L.w, c->d, L.g, F, rq.virial ? L.vir_atom : nullptr, acc, variant, s, &nl));
        }
    }
    stage_mark(c, 4, s);
    CU(launch_cfg_reduce(L.w, L.E_rows, (rq.virial && need_forces) ? L.vir_atom : nullptr, E_cfg, rq.virial,
                         rq.E_atom, L.cfg_part, s, &nl));
    if (grad) {
        const float* u = nullptr;
        const double* alpha = nullptr;
        if (rq.train) {
            stage_mark(c, 7, s);
            CU(launch_loss(L.w, c->norm_C, c->norm_N, c->loss_opts, weight_ranges(c->plan), rq.theta, E_cfg,
                           rq.E_ref, F, rq.F_ref, rq.w_force, rq.loss,
                           L.alpha_cfg, L.u, L.loss_part, s, &nl));
            u = L.u;
            alpha = L.alpha_cfg;
        } else {
            u = rq.dF;
            alpha = rq.dE;
        }
        CU(launch_row_scale(L.w, alpha, L.alpha_rows, s, &nl));
        stage_mark(c, 5, s);
        if (u && sv) {
            CU(launch_store_tangent(*sv, c->d, u, L.wdot, s, &nl));
        } else if (u) {
            // the tangent enters only the weight gradient (tolerance 1e-4 against 1e-5 for
            // forces): the plain FP32 angular form unless extended precision is forced
            const bool acc_jvp = c->ang_mode == 1;
            int dummy = 0;
            const int v = tuned_variant(c, sys, rq.prec, KV_JVP, s, [&](int vv) {
                launch_jvp(L.w, c->d, u, L.wdot, acc_jvp, s, &dummy, vv);
            });
            CU(launch_jvp(L.w, c->d, u, L.wdot, acc_jvp, s, &nl, v));
        } else {
            CU(cudaMemsetAsync(L.wdot, 0, sizeof(float) * (size_t)N * c->d.D, s));
        }
        stage_mark(c, 6, s);
        const bool tan_tc = tf && (tfm & TF32_TAN);
        const WgradTc wtc{(tf && (tfm & TF32_WGRAD)) ? L.tf_ws : nullptr, tfm, L.w.status};
        if (tan_tc) CU(tf32_tangent1(c->plan, L.mb, N, L.tf_ws, tfm, L.wdot, L.w.status, s, &nl));
        CU(mlp_param_grad(c->plan, L.mb, rq.theta, N, L.wdot, L.alpha_rows, rq.dtheta, s, &nl, tan_tc, &wtc));
        if (rq.train) CU(launch_penalty_grad(c->loss_opts, weight_ranges(c->plan), rq.theta, rq.dtheta, s, &nl));
    }
    if (c->profiling) cudaEventRecord(c->ev[kNumStages], s);
    return PANNA_OK;
}

panna_status run(panna_ctx* c, const panna_system* sys, const Request& rq, cudaStream_t s)
{
    ST(check_system(c, sys, rq.store == nullptr));
    if (c->plan.n_out != 1 && !rq.G_out)
        return fail(PANNA_ERR_UNSUPPORTED, "networks with 3 outputs serve panna_qeq_energy_forces only");
    CU(cudaSetDevice(c->device));
    const bool train = rq.train || rq.vjp;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Layout L;
        ST(prepare(c, sys, train, rq.prec != PANNA_MLP_FP32, L, s));
        c->last_launches = 0;
        ST(run_once(c, sys, rq, L, s));
        CU(cudaGetLastError());
        if (c->async) return PANNA_OK;
        int need = 0;
        panna_status st = collect(c, L, s, &need);
        finish_profile(c);
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt == 0) {
            c->cap = need + need / 4 + 8;
            continue;
        }
        return st;
    }
    return PANNA_OK;
}

// ------------------------------------------------------------------ dynamics

constexpr double kMdAcc = 9.648533212e-3;   // (eV/A)/amu in A/fs^2
constexpr double kMdKb = 8.617333262e-5;    // eV/K

// candidates of a neighbour search with cutoff rc + skin into L.cand_*, positions recorded
panna_status md_build(panna_ctx* c, const panna_system* sys, Layout& L, Work& wc, double skin, cudaStream_t s)
{
    wc = L.w;
    wc.nb_count = L.cand_count;
    wc.nb_vec = L.cand_vec;
    wc.nb_idx = L.cand_idx;
    wc.nb_vlo = nullptr;   // candidates keep no low parts (the refresh forms them at each step)
    wc.cap = c->cap_c;
    DescDev dc = c->d;
    dc.rc_d = c->d.rc_d + skin;
    dc.rc = (float)dc.rc_d;
    int nl = 0;
    CU(build_neighbors(wc, dc, s, &nl));
    CU(cudaMemcpyAsync(L.pos_ref, sys->pos, sizeof(double) * 3 * (size_t)sys->n_atoms, cudaMemcpyDeviceToDevice, s));
    return PANNA_OK;
}

// reads the status word (one copy, one synchronisation)
panna_status md_status(panna_ctx* c, const Layout& L, cudaStream_t s, bool* stale, int* need)
{
    CU(cudaMemcpyAsync(c->h_status, L.w.status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *stale = c->h_status->stale != 0;
    *need = c->h_status->need_cap;
    return (panna_status)c->h_status->code;
}

}  // namespace

// ------------------------------------------------------------------ public API

extern "C" {

const char* panna_version(void) { return "panna_gb300 0.1 (sm_103a)"; }

const char* panna_last_error(void) { return g_last_error.c_str(); }

static int64_t desc_size(const panna_desc_params* p)
{
    if (!p) return -1;
    if (p->n_species < 1 || p->n_species > kMaxSpecies) return -1;
    if (p->n_rad < 1 || p->n_ang_r < 1 || p->n_theta < 1) return -1;
    const int64_t S = p->n_species;
    return S * p->n_rad + S * (S + 1) / 2 * p->n_theta * p->n_ang_r;
}

int64_t panna_descriptor_size(const panna_desc_params* p) { return desc_size(p); }

panna_status panna_create(const panna_desc_params* p, int32_t n_archs, const panna_mlp_arch* archs, panna_ctx** out)
{
    if (!out) return fail(PANNA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    const int64_t D = desc_size(p);
    if (D < 0) return fail(PANNA_ERR_INVALID_ARG, "invalid descriptor sizes or species count (1..%d)", kMaxSpecies);
    bool unsupported = false;
    if (const char* why = desc_params_check(p, &unsupported))
        return fail(unsupported ? PANNA_ERR_UNSUPPORTED : PANNA_ERR_INVALID_ARG, "%s", why);
    if (n_archs != p->n_species || !archs) return fail(PANNA_ERR_INVALID_ARG, "one network per species required");
    panna_ctx* c = new panna_ctx();
    cudaGetDevice(&c->device);
    DescDev& d = c->d;
    desc_dev_from_params(p, d);
    DescGrid64& g64 = c->g64;
    g64.rc = p->rc; g64.eta_rad = p->eta_rad;
    for (int k = 0; k < p->n_rad; ++k) g64.rs_rad[k] = p->rs_rad[k];
    if (d.ang_kind == 0) {   // the stored Jacobians take the modified angular term
        g64.eta_ang = p->eta_ang; g64.zeta = p->zeta;
        g64.eps_theta = p->eps_theta; g64.pref = pow(2.0, 1.0 - p->zeta); g64.zeta_int = d.zeta_int;
        for (int k = 0; k < p->n_ang_r; ++k) g64.rs_ang[k] = p->rs_ang[k];
        for (int k = 0; k < p->n_theta; ++k) {
            g64.cos_t[k] = cos(p->theta_s[k]);
            g64.sin_t[k] = sin(p->theta_s[k]);
        }
    }
    MlpPlan& pl = c->plan;
    pl.S = d.S;
    pl.L = archs[0].n_layers;
    int64_t off = 0;
    for (int s = 0; s < d.S; ++s) {
        const panna_mlp_arch& a = archs[s];
        if (a.n_layers != pl.L || a.n_layers < 1 || a.n_layers > kMaxLayers) {
            delete c;
            return fail(PANNA_ERR_UNSUPPORTED, "every species needs the same number of layers (1..%d)", kMaxLayers);
        }
        const int n_out = archs[0].widths[archs[0].n_layers];
        if (a.widths[0] != D || (n_out != 1 && n_out != 3) || a.widths[a.n_layers] != n_out) {
            delete c;
            return fail(PANNA_ERR_INVALID_ARG, "species %d: input width must be D=%lld and every species' output "
                        "width 1 (energy) or 3 (charge equilibration)", s, (long long)D);
        }
        for (int l = 0; l < a.n_layers; ++l) {
            if (a.widths[l + 1] < 1 || a.widths[l + 1] > 1024 || a.act[l] < 0 || a.act[l] > 3) {
                delete c;
                return fail(PANNA_ERR_UNSUPPORTED, "species %d layer %d: width 1..1024 and activation 0..3", s, l + 1);
            }
            pl.widths[s][l] = a.widths[l];
            pl.acts[s][l] = a.act[l];
            pl.w_off[s][l] = off;
            off += (int64_t)a.widths[l + 1] * a.widths[l];
            pl.b_off[s][l] = off;
            off += a.widths[l + 1];
        }
        pl.widths[s][a.n_layers] = a.widths[a.n_layers];
    }
    pl.P = off;
    pl.n_out = archs[0].widths[archs[0].n_layers];
    pl.max_hidden = 1;
    for (int l = 0; l <= pl.L; ++l) {
        int m = 0;
        for (int s = 0; s < d.S; ++s) m = pl.widths[s][l] > m ? pl.widths[s][l] : m;
        pl.ld[l] = m;
        if (l >= 1 && m > pl.max_hidden) pl.max_hidden = m;
    }
    if (cudaMallocHost((void**)&c->h_status, sizeof(DevStatus)) != cudaSuccess) {
        delete c;
        return fail(PANNA_ERR_CUDA, "pinned status allocation failed");
    }
    for (int k = 0; k <= kNumStages; ++k) cudaEventCreate(&c->ev[k]);
    for (int k = 0; k < 3; ++k) cudaEventCreate(&c->tev[k]);
    *out = c;
    return PANNA_OK;
}

void panna_destroy(panna_ctx* c)
{
    if (!c) return;
    if (c->ws.base) cudaFree(c->ws.base);
    if (c->h_status) cudaFreeHost(c->h_status);
    for (int k = 0; k <= kNumStages; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    for (int k = 0; k < 3; ++k)
        if (c->tev[k]) cudaEventDestroy(c->tev[k]);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

int64_t panna_param_count(const panna_ctx* c) { return c ? c->plan.P : -1; }

panna_status panna_set_neighbor_capacity(panna_ctx* c, int32_t cap)
{
    if (!c || cap < 1 || cap > 4096) return fail(PANNA_ERR_INVALID_ARG, "capacity must be 1..4096");
    c->cap = cap;
    return PANNA_OK;
}

int32_t panna_neighbor_capacity(const panna_ctx* c) { return c ? c->cap : -1; }

panna_status panna_set_async(panna_ctx* c, int32_t async)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    c->async = async ? 1 : 0;
    return PANNA_OK;
}

panna_status panna_set_angular_precision(panna_ctx* c, int32_t mode)
{
    if (!c || mode < 0 || mode > 2) return fail(PANNA_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
    c->ang_mode = mode;
    return PANNA_OK;
}

int32_t panna_tuning_choice(const panna_ctx* c, const char* knob)
{
    if (!c || !knob) return -1;
    const char* kinds[3] = {"descriptor", "adjoint", "jvp"};
    for (int k = 0; k < 3; ++k)
        if (strcmp(knob, kinds[k]) == 0) return c->last_variant[k];
    return -1;
}

panna_status panna_set_tuning(panna_ctx* c, const char* knob, int32_t value)
{
    if (!c || !knob) return fail(PANNA_ERR_INVALID_ARG, "null argument");
    if (strcmp(knob, "autotune") == 0 && (value == 0 || value == 1)) {
        c->autotune = value;
        c->n_tuned = 0;
        return PANNA_OK;
    }
    const char* kinds[3] = {"descriptor", "adjoint", "jvp"};
    for (int k = 0; k < 3; ++k)
        if (strcmp(knob, kinds[k]) == 0 && value >= -1 && value < kKindVariants[k]) {
            c->force_variant[k] = value;
            return PANNA_OK;
        }
    if (strcmp(knob, "mlp_fp32") == 0 && value >= 0 && value <= 15 && !(value & 2)) {
        c->fp32_tc = value;
        return PANNA_OK;
    }
    return fail(PANNA_ERR_INVALID_ARG, "unknown tuning knob or value: %s=%d", knob, value);
}

panna_status panna_md_run(panna_ctx* c, const panna_system* sys, double* vel, const float* theta, int32_t prec,
                          const panna_md_params* p, int64_t n_steps, float* F, int32_t forces_valid, double* E_cfg,
                          double* E_traj, int64_t* n_builds, panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (!vel || !theta || !p || !F || !E_cfg || !p->mass || n_steps < 0)
        return fail(PANNA_ERR_INVALID_ARG, "vel, theta, params (with masses), F and E_cfg are required");
    if (!(p->dt > 0.0) || !(p->temperature >= 0.0) || !(p->friction >= 0.0) || !(p->skin >= 0.0))
        return fail(PANNA_ERR_INVALID_ARG, "dt must be > 0; temperature, friction and skin >= 0");
    if (prec < PANNA_MLP_FP32 || prec > PANNA_MLP_BF16_FAST) return fail(PANNA_ERR_INVALID_ARG, "unknown precision");
    if (sys->ghost) return fail(PANNA_ERR_UNSUPPORTED, "dynamics of a batch with ghost atoms");
    if (c->plan.n_out != 1) return fail(PANNA_ERR_UNSUPPORTED, "dynamics with 3-output networks");
    MdSpecies ms{};
    for (int sp = 0; sp < c->d.S; ++sp) {
        if (!(p->mass[sp] > 0.0)) return fail(PANNA_ERR_INVALID_ARG, "mass of species %d must be > 0", sp);
        ms.acc[sp] = kMdAcc / p->mass[sp];
        ms.sigma[sp] = sqrt(kMdKb * p->temperature * ms.acc[sp]);
    }
    CU(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = sys->n_atoms;
    double* pos = const_cast<double*>(sys->pos);     // the dynamics moves the caller's positions
    const double c1 = exp(-p->friction * p->dt), c2 = sqrt(fmax(0.0, 1.0 - c1 * c1));
    const int thermostat = (p->friction > 0.0 || p->temperature > 0.0) ? 1 : 0;
    const double lim2 = 0.25 * p->skin * p->skin;
    const bool bf16 = prec != PANNA_MLP_FP32;
    const double grow = (c->d.rc_d + p->skin) / c->d.rc_d;
    c->cap_c = std::max<int32_t>(c->cap_c, (int32_t)(c->cap * grow * grow * grow) + 8);
    Request rq;
    rq.theta = theta; rq.prec = prec; rq.E_cfg = E_cfg; rq.F = F; rq.forces = true; rq.energy = true;
    Layout L;
    Work wc{};
    bool stale = false;
    int need = 0;
    int64_t builds = 0;
    // first neighbour build, and the forces at the starting positions; capacities grow here
    for (int attempt = 0;; ++attempt) {
        ST(prepare(c, sys, false, bf16, L, s, c->cap_c));
        CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
        ST(md_build(c, sys, L, wc, p->skin, s));
        panna_status st = md_status(c, L, s, &stale, &need);
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt < 3) { c->cap_c = need + need / 4 + 8; continue; }
        if (st != PANNA_OK) return collect(c, L, s, &need);
        rq.cand = &wc;
        c->last_launches = 0;
        if (!forces_valid || attempt > 0) {
            ST(run_once(c, sys, rq, L, s));
            st = md_status(c, L, s, &stale, &need);
            if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt < 3) { c->cap = need + need / 4 + 8; continue; }
            if (st != PANNA_OK) return collect(c, L, s, &need);
        }
        ++builds;
        break;
    }
    for (int64_t t = 0; t < n_steps; ++t) {
        CU(launch_md_baoa(N, sys->species, ms, pos, vel, F, p->dt, c1, c2, thermostat, p->seed, p->step0 + t,
                          L.pos_ref, lim2, &L.w.status->stale, s));
        const panna_status st = md_status(c, L, s, &stale, &need);
        if (st != PANNA_OK) {
            collect(c, L, s, &need);
            return fail(st, "step %lld: %s (raise the neighbour capacity and restart)", (long long)t,
                        panna_last_error());
        }
        if (stale || p->skin == 0.0) {
            ST(md_build(c, sys, L, wc, p->skin, s));
            ++builds;
        }
        ST(run_once(c, sys, rq, L, s));
        CU(launch_md_b(N, sys->species, ms, vel, F, p->dt, s));
        if (E_traj)
            CU(cudaMemcpyAsync(E_traj + t * sys->n_cfg, E_cfg, sizeof(double) * (size_t)sys->n_cfg,
                               cudaMemcpyDeviceToDevice, s));
    }
    if (n_builds) *n_builds = builds;
    return collect(c, L, s, &need);
}

panna_status panna_set_loss_options(panna_ctx* c, const panna_loss_options* o)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    if (!o) { c->loss_opts = LossOpts{0, 0, 0, 0.0, 0.0}; return PANNA_OK; }
    if (o->energy_loss < 0 || o->energy_loss > 1 || o->force_loss < 0 || o->force_loss > 1 ||
        !(o->l1 >= 0.0) || !(o->l2 >= 0.0))
        return fail(PANNA_ERR_INVALID_ARG, "loss kinds must be 0 or 1, penalties >= 0");
    c->loss_opts = LossOpts{o->energy_loss, o->force_loss, o->energy_per_atom ? 1 : 0, o->l1, o->l2};
    return PANNA_OK;
}

panna_status panna_set_frozen(panna_ctx* c, int32_t species, int32_t layer, int32_t frozen)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    if (species < 0 || species >= c->plan.S || layer < 0 || layer >= c->plan.L)
        return fail(PANNA_ERR_INVALID_ARG, "species %d / layer %d out of range", species, layer);
    c->frozen[species][layer] = frozen != 0;
    return PANNA_OK;
}

panna_status panna_adam_step(panna_ctx* c, float* theta, const float* grad, float* m, float* v, int64_t t,
                             const panna_adam_params* a, panna_stream_t stream)
{
    if (!c || !theta || !grad || !m || !v || !a) return fail(PANNA_ERR_INVALID_ARG, "null argument");
    if (t < 1 || !(a->lr > 0.0) || !(a->beta1 >= 0.0 && a->beta1 < 1.0) || !(a->beta2 >= 0.0 && a->beta2 < 1.0) ||
        !(a->eps >= 0.0) || !(a->decay_steps >= 0.0) || !(a->decay_rate > 0.0))
        return fail(PANNA_ERR_INVALID_ARG, "Adam needs t >= 1, lr > 0, betas in [0, 1), eps >= 0, decay rate > 0");
    CU(cudaSetDevice(c->device));
    const double lr = a->decay_steps > 0.0 ? a->lr * pow(a->decay_rate, (double)t / a->decay_steps) : a->lr;
    const double c1 = 1.0 - pow(a->beta1, (double)t), c2 = 1.0 - pow(a->beta2, (double)t);
    int nl = 0;
    CU(launch_adam(c->plan.P, theta, grad, m, v, lr, a->beta1, a->beta2, c1, c2, a->eps, frozen_ranges(c),
                   (cudaStream_t)stream, &nl));
    c->last_launches = nl;
    return PANNA_OK;
}

panna_status panna_set_loss_normalization(panna_ctx* c, int64_t n_cfg_total, int64_t n_atoms_total)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    const bool reset = n_cfg_total == 0 && n_atoms_total == 0;
    if (!reset && (n_cfg_total <= 0 || n_atoms_total <= 0))
        return fail(PANNA_ERR_INVALID_ARG, "loss normalisers must both be positive, or both 0");
    c->norm_C = n_cfg_total;
    c->norm_N = n_atoms_total;
    return PANNA_OK;
}

panna_status panna_check(panna_ctx* c, panna_stream_t stream)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    if (!c->ws.base) return PANNA_OK;
    CU(cudaMemcpyAsync(c->h_status, c->ws.base, sizeof(DevStatus), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    DevStatus st = *c->h_status;
    CU(cudaMemsetAsync(c->ws.base, 0, sizeof(DevStatus), (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    if (st.code == PANNA_ERR_NEIGHBOR_OVERFLOW) {
        c->cap = st.need_cap + st.need_cap / 4 + 8;
        return fail(PANNA_ERR_NEIGHBOR_OVERFLOW, "neighbour capacity exceeded (needed %d); capacity raised to %d",
                    st.need_cap, c->cap);
    }
    if (st.code) return fail((panna_status)st.code, "device error %d at index %d", st.code, st.bad_index);
    return PANNA_OK;
}

panna_status panna_neighbors(panna_ctx* c, const panna_system* sys, int64_t cap_total, int64_t* nbr_off,
                             int64_t* nbr_j, int32_t* nbr_shift, int64_t* n_total, panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (!nbr_off || !n_total) return fail(PANNA_ERR_INVALID_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(c->device));
    for (int attempt = 0; attempt < 2; ++attempt) {
        Layout L;
        ST(prepare(c, sys, false, false, L, s));
        L.w.nb_vlo = nullptr;   // the export needs no low parts
        c->last_launches = 0;
        CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
        CU(build_neighbors(L.w, c->d, s, &c->last_launches));
        int need = 0;
        panna_status st = collect(c, L, s, &need);
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt == 0) {
            c->cap = need + need / 4 + 8;
            continue;
        }
        if (st != PANNA_OK) return st;
        CU(export_neighbors(L.w, nbr_off, nbr_j, nbr_shift, cap_total, s, &c->last_launches));
        CU(cudaMemcpyAsync(n_total, nbr_off + sys->n_atoms, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (*n_total > cap_total)
            return fail(PANNA_ERR_INVALID_ARG, "%lld entries, output holds %lld", (long long)*n_total,
                        (long long)cap_total);
        return PANNA_OK;
    }
    return PANNA_OK;
}

panna_status panna_descriptors(panna_ctx* c, const panna_system* sys, float* G, panna_stream_t stream)
{
    if (!G) return fail(PANNA_ERR_INVALID_ARG, "null G");
    Request rq;
    rq.G_out = G;
    return run(c, sys, rq, (cudaStream_t)stream);
}

panna_status panna_energy_forces(panna_ctx* c, const panna_system* sys, const float* theta, int32_t prec,
                                 double* E_cfg, float* E_atom, float* F, double* virial, panna_stream_t stream)
{
    if (!theta || !E_cfg || !F) return fail(PANNA_ERR_INVALID_ARG, "theta, E_cfg and F are required");
    if (prec != PANNA_MLP_FP32 && prec != PANNA_MLP_BF16 && prec != PANNA_MLP_BF16_FAST)
        return fail(PANNA_ERR_INVALID_ARG, "bad precision");
    if (prec != PANNA_MLP_FP32 && c && c->plan.L < 2)
        return fail(PANNA_ERR_UNSUPPORTED, "BF16 networks need at least one hidden layer");
    if (prec != PANNA_MLP_FP32 && c && (c->d.D % 8 != 0))
        return fail(PANNA_ERR_UNSUPPORTED, "BF16 networks need a descriptor size that is a multiple of 8");
    Request rq;
    rq.theta = theta; rq.prec = prec; rq.E_cfg = E_cfg; rq.E_atom = E_atom; rq.F = F; rq.virial = virial;
    rq.forces = true; rq.energy = true;
    return run(c, sys, rq, (cudaStream_t)stream);
}

panna_status panna_param_vjp(panna_ctx* c, const panna_system* sys, const float* theta, const double* dE,
                             const float* dF, float* dtheta, panna_stream_t stream)
{
    if (!theta || !dtheta) return fail(PANNA_ERR_INVALID_ARG, "theta and dtheta are required");
    Request rq;
    rq.theta = theta; rq.vjp = true; rq.dE = dE; rq.dF = dF; rq.dtheta = dtheta; rq.energy = true;
    return run(c, sys, rq, (cudaStream_t)stream);
}

panna_status panna_loss_grad(panna_ctx* c, const panna_system* sys, const float* theta, const double* E_ref,
                             const float* F_ref, double w_force, double* loss, float* dtheta, double* E_cfg, float* F,
                             panna_stream_t stream)
{
    if (!theta || !E_ref || !F_ref || !loss || !dtheta)
        return fail(PANNA_ERR_INVALID_ARG, "theta, E_ref, F_ref, loss and dtheta are required");
    if (sys && sys->ghost)
        return fail(PANNA_ERR_UNSUPPORTED, "the training loss needs complete forces: no ghost atoms");
    Request rq;
    rq.theta = theta; rq.train = true; rq.E_ref = E_ref; rq.F_ref = F_ref; rq.w_force = w_force; rq.loss = loss;
    rq.dtheta = dtheta; rq.E_cfg = E_cfg; rq.F = F; rq.forces = true; rq.energy = true;
    return run(c, sys, rq, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ charge equilibration

panna_status panna_set_qeq(panna_ctx* c, const panna_qeq_params* p)
{
    if (!c || !p || !p->sigma || !p->chi0 || !p->hard0) return fail(PANNA_ERR_INVALID_ARG, "null argument");
    if (c->plan.n_out != 3) return fail(PANNA_ERR_INVALID_ARG, "charge equilibration needs networks with 3 outputs");
    if (!(p->k_coulomb >= 0.0)) return fail(PANNA_ERR_INVALID_ARG, "k_coulomb must be >= 0");
    QeqDev q{};
    for (int s = 0; s < c->d.S; ++s) {
        if (!(p->sigma[s] > 0.0) || !std::isfinite(p->chi0[s]) || !std::isfinite(p->hard0[s]))
            return fail(PANNA_ERR_INVALID_ARG, "species %d: sigma must be > 0, chi0 and hard0 finite", s);
        q.sigma[s] = p->sigma[s];
        q.chi0[s] = p->chi0[s];
        q.hard0[s] = p->hard0[s];
    }
    q.ke = p->k_coulomb > 0.0 ? p->k_coulomb : 14.399645478425668;
    c->qeq = q;
    c->qeq_set = true;
    return PANNA_OK;
}

panna_status panna_qeq_energy_forces(panna_ctx* c, const panna_system* sys, const float* theta,
                                     const double* total_charge, double* E_cfg, float* E_atom, double* charges,
                                     float* F, panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (!theta || !E_cfg || !F) return fail(PANNA_ERR_INVALID_ARG, "theta, E_cfg and F are required");
    if (c->plan.n_out != 3 || !c->qeq_set)
        return fail(PANNA_ERR_INVALID_ARG, "needs 3-output networks and panna_set_qeq");
    if (sys->ghost) return fail(PANNA_ERR_UNSUPPORTED, "charge equilibration of a batch with ghost atoms");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(c->device));
    const int64_t N = sys->n_atoms;
    const bool acc = c->ang_mode != 2;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Layout L;
        ST(prepare(c, sys, false, false, L, s));
        if (!acc) L.w.nb_vlo = nullptr;
        int& nl = c->last_launches;
        nl = 0;
        for (int k = 0; k < kNumStages; ++k) c->stage_seen[k] = false;
        c->n_marked = 0;
        CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
        stage_mark(c, 0, s);
        CU(build_neighbors(L.w, c->d, s, &nl));
        CU(species_order(L.w, c->d.S, s, &nl));
        CU(mlp_tiles(c->plan, L.w.seg_off, L.mb.tile_start, s, &nl));
        stage_mark(c, 1, s);
        int dummy = 0;
        const int vd = tuned_variant(c, sys, PANNA_MLP_FP32, KV_DESC, s, [&](int vv) {
            launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &dummy, vv);
        }, acc);
        CU(launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &nl, vd));
        stage_mark(c, 2, s);
        CU(mlp_forward(c->plan, L.mb, theta, N, s, &nl));
        // the charge-equilibration solve ("forces" stage): charges, energies, pair forces, seeds
        stage_mark(c, 4, s);
        const int ldL = c->plan.ld[c->plan.L];
        CU(cudaMemsetAsync(F, 0, sizeof(float) * 3 * N, s));
        CU(launch_qeq(c->qeq, L.w, L.mb.A[c->plan.L], ldL, total_charge, L.E_rows, charges, F, L.mb.Ab, ldL, s,
                      &nl));
        stage_mark(c, 3, s);
        CU(mlp_input_grad(c->plan, L.mb, theta, N, L.g, s, &nl, nullptr, true));
        const int va = tuned_variant(c, sys, PANNA_MLP_FP32, KV_ADJ, s, [&](int vv) {
            launch_adjoint(L.w, c->d, L.g, L.F_tune, nullptr, acc, vv, s, &dummy);
        });
        CU(launch_adjoint(L.w, c->d, L.g, F, nullptr, acc, va, s, &nl));
        stage_mark(c, 7, s);
        CU(launch_cfg_reduce(L.w, L.E_rows, nullptr, E_cfg, nullptr, E_atom, L.cfg_part, s, &nl));
        if (c->profiling) cudaEventRecord(c->ev[kNumStages], s);
        CU(cudaGetLastError());
        if (c->async) return PANNA_OK;
        int need = 0;
        panna_status st = collect(c, L, s, &need);
        finish_profile(c);
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt == 0) {
            c->cap = need + need / 4 + 8;
            continue;
        }
        if (st == PANNA_ERR_UNSUPPORTED)
            return fail(PANNA_ERR_UNSUPPORTED, "configuration %d: charge equilibration takes non-periodic "
                        "configurations of at most %d atoms", c->h_status->bad_index, kQeqMax);
        if (st == PANNA_ERR_BAD_INPUT && c->h_status->code == PANNA_ERR_BAD_INPUT)
            return fail(PANNA_ERR_BAD_INPUT, "configuration or atom %d: invalid input or singular "
                        "charge-equilibration system", c->h_status->bad_index);
        return st;
    }
    return PANNA_OK;
}

panna_status panna_qeq_loss_grad(panna_ctx* c, const panna_system* sys, const float* theta,
                                 const double* total_charge, const double* E_ref, const float* F_ref, double w_force,
                                 const double* q_ref, double w_charge, double* loss, float* dtheta, double* E_cfg,
                                 double* charges, float* F, panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (!theta || !E_ref || !F_ref || !loss || !dtheta)
        return fail(PANNA_ERR_INVALID_ARG, "theta, E_ref, F_ref, loss and dtheta are required");
    if (c->plan.n_out != 3 || !c->qeq_set)
        return fail(PANNA_ERR_INVALID_ARG, "needs 3-output networks and panna_set_qeq");
    if (!(w_charge >= 0.0) || !(w_force >= 0.0)) return fail(PANNA_ERR_INVALID_ARG, "weights must be >= 0");
    if (sys->ghost) return fail(PANNA_ERR_UNSUPPORTED, "charge equilibration of a batch with ghost atoms");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(c->device));
    const int64_t N = sys->n_atoms;
    const bool acc = c->ang_mode != 2;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Layout L;
        ST(prepare(c, sys, true, false, L, s));
        if (!acc) L.w.nb_vlo = nullptr;
        int& nl = c->last_launches;
        nl = 0;
        for (int k = 0; k < kNumStages; ++k) c->stage_seen[k] = false;
        c->n_marked = 0;
        float* Fo = F ? F : L.F_int;
        double* Eo = E_cfg ? E_cfg : L.E_cfg_int;
        CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
        stage_mark(c, 0, s);
        CU(build_neighbors(L.w, c->d, s, &nl));
        CU(species_order(L.w, c->d.S, s, &nl));
        CU(mlp_tiles(c->plan, L.w.seg_off, L.mb.tile_start, s, &nl));
        stage_mark(c, 1, s);
        int dummy = 0;
        const int vd = tuned_variant(c, sys, PANNA_MLP_FP32, KV_DESC, s, [&](int vv) {
            launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &dummy, vv);
        }, acc);
        CU(launch_descriptor(L.w, c->d, L.G, L.w.row_of_atom, acc, s, &nl, vd));
        stage_mark(c, 2, s);
        CU(mlp_forward(c->plan, L.mb, theta, N, s, &nl));
        stage_mark(c, 4, s);
        const int ldL = c->plan.ld[c->plan.L];
        CU(cudaMemsetAsync(Fo, 0, sizeof(float) * 3 * N, s));
        CU(launch_qeq(c->qeq, L.w, L.mb.A[c->plan.L], ldL, total_charge, L.E_rows, L.qbuf, Fo, L.mb.Ab, ldL, s,
                      &nl));
        stage_mark(c, 3, s);
        CU(mlp_input_grad(c->plan, L.mb, theta, N, L.g, s, &nl, nullptr, true));
        const int va = tuned_variant(c, sys, PANNA_MLP_FP32, KV_ADJ, s, [&](int vv) {
            launch_adjoint(L.w, c->d, L.g, L.F_tune, nullptr, acc, vv, s, &dummy);
        });
        CU(launch_adjoint(L.w, c->d, L.g, Fo, nullptr, acc, va, s, &nl));
        CU(launch_cfg_reduce(L.w, L.E_rows, nullptr, Eo, nullptr, nullptr, L.cfg_part, s, &nl));
        stage_mark(c, 7, s);
        CU(launch_loss(L.w, c->norm_C, c->norm_N, c->loss_opts, weight_ranges(c->plan), theta, Eo, E_ref, Fo, F_ref,
                       w_force, loss, L.alpha_cfg, L.u, L.loss_part, s, &nl));
        stage_mark(c, 5, s);
        const bool acc_jvp = c->ang_mode == 1;
        const int vj = tuned_variant(c, sys, PANNA_MLP_FP32, KV_JVP, s, [&](int vv) {
            launch_jvp(L.w, c->d, L.u, L.wdot, acc_jvp, s, &dummy, vv);
        });
        CU(launch_jvp(L.w, c->d, L.u, L.wdot, acc_jvp, s, &nl, vj));
        stage_mark(c, 6, s);
        CU(mlp_param_grad(c->plan, L.mb, theta, N, L.wdot, nullptr, dtheta, s, &nl, false, nullptr,
                          MLP_GRAD_TANGENT));
        QeqTrain tr{L.qbuf, L.u, L.mb.Ad[c->plan.L], L.alpha_cfg, q_ref, w_charge, L.mb.Adb, loss};
        CU(launch_qeq_response(c->qeq, L.w, L.mb.A[c->plan.L], ldL, tr, L.mb.Ab, ldL, s, &nl));
        CU(mlp_param_grad(c->plan, L.mb, theta, N, L.wdot, nullptr, dtheta, s, &nl, false, nullptr,
                          MLP_GRAD_REVERSE_SEEDED));
        CU(launch_penalty_grad(c->loss_opts, weight_ranges(c->plan), theta, dtheta, s, &nl));
        if (charges) CU(cudaMemcpyAsync(charges, L.qbuf, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        if (c->profiling) cudaEventRecord(c->ev[kNumStages], s);
        CU(cudaGetLastError());
        if (c->async) return PANNA_OK;
        int need = 0;
        panna_status st = collect(c, L, s, &need);
        finish_profile(c);
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt == 0) {
            c->cap = need + need / 4 + 8;
            continue;
        }
        if (st == PANNA_ERR_UNSUPPORTED)
            return fail(PANNA_ERR_UNSUPPORTED, "configuration %d: charge equilibration takes non-periodic "
                        "configurations of at most %d atoms", c->h_status->bad_index, kQeqMax);
        return st;
    }
    return PANNA_OK;
}

// ------------------------------------------------------------------ stored descriptors

static panna_status store_view(const panna_ctx* c, const panna_system* sys, const panna_store_info* info,
                               const void* store, StoreView& v)
{
    if (!info || !store) return fail(PANNA_ERR_INVALID_ARG, "null store info or buffer");
    if ((uintptr_t)store % 256 != 0) return fail(PANNA_ERR_INVALID_ARG, "the store buffer must be 256-byte aligned");
    if (info->n_atoms != sys->n_atoms || info->n_cfg != sys->n_cfg)
        return fail(PANNA_ERR_INVALID_ARG, "store of another batch (%lld atoms, %lld configurations)",
                    (long long)info->n_atoms, (long long)info->n_cfg);
    v = StoreView{};
    v.N = info->n_atoms;
    v.C = info->n_cfg;
    v.P = info->n_entries;
    store_dims(c->d, v);
    if (info->D != v.D || info->width != v.W || v.P < 0)
        return fail(PANNA_ERR_INVALID_ARG, "store of another descriptor (D %d, width %d)", info->D, info->width);
    if (store_carve(v, reinterpret_cast<char*>(const_cast<void*>(store)), nullptr) != info->bytes)
        return fail(PANNA_ERR_INVALID_ARG, "store size does not match its entry count");
    return PANNA_OK;
}

// neighbour search of a batch for a store; *total (host) = number of entries (synchronous)
static panna_status store_search(panna_ctx* c, const panna_system* sys, Layout& L, int64_t* total, cudaStream_t s)
{
    for (int attempt = 0; attempt < 2; ++attempt) {
        ST(prepare(c, sys, false, false, L, s));
        c->last_launches = 0;
        CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
        CU(build_neighbors(L.w, c->d, s, &c->last_launches));
        CU(launch_store_offsets(L.w, L.w.cell_start, s, &c->last_launches));
        CU(cudaMemcpyAsync(total, L.w.cell_start + sys->n_atoms, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        int need = 0;
        panna_status st = collect(c, L, s, &need);   // synchronises the stream
        if (st == PANNA_ERR_NEIGHBOR_OVERFLOW && attempt == 0) {
            c->cap = need + need / 4 + 8;
            continue;
        }
        if (st != PANNA_OK) return st;
        if (c->cap > kStoreMaxCap)
            return fail(PANNA_ERR_UNSUPPORTED, "stored Jacobians take at most %d neighbours per atom", kStoreMaxCap);
        return PANNA_OK;
    }
    return PANNA_OK;
}

panna_status panna_store_plan(panna_ctx* c, const panna_system* sys, panna_store_info* info, panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (!info) return fail(PANNA_ERR_INVALID_ARG, "null info");
    if (sys->ghost) return fail(PANNA_ERR_UNSUPPORTED, "stored descriptors of a batch with ghost atoms");
    if (c->d.D > kStoreMaxD) return fail(PANNA_ERR_UNSUPPORTED, "stored descriptors take D <= %d", kStoreMaxD);
    if (c->d.ang_kind != 0) return fail(PANNA_ERR_UNSUPPORTED, "stored Jacobians take the modified angular term");
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(c->device));
    Layout L;
    int64_t n_entries = 0;
    ST(store_search(c, sys, L, &n_entries, s));
    StoreView v{};
    v.N = sys->n_atoms;
    v.C = sys->n_cfg;
    v.P = n_entries;
    store_dims(c->d, v);
    info->n_atoms = v.N;
    info->n_cfg = v.C;
    info->n_entries = v.P;
    info->D = v.D;
    info->width = v.W;
    info->bytes = store_carve(v, nullptr, nullptr);
    return PANNA_OK;
}

panna_status panna_store_sections(const panna_ctx* c, const panna_store_info* info, int64_t* offsets)
{
    if (!c || !info || !offsets) return fail(PANNA_ERR_INVALID_ARG, "null argument");
    StoreView v{};
    v.N = info->n_atoms;
    v.C = info->n_cfg;
    v.P = info->n_entries;
    store_dims(c->d, v);
    store_carve(v, nullptr, offsets);
    return PANNA_OK;
}

panna_status panna_store_build(panna_ctx* c, const panna_system* sys, const panna_store_info* info, void* store,
                               panna_stream_t stream)
{
    ST(check_system(c, sys));
    if (sys->ghost) return fail(PANNA_ERR_UNSUPPORTED, "stored descriptors of a batch with ghost atoms");
    StoreView v;
    ST(store_view(c, sys, info, store, v));
    cudaStream_t s = (cudaStream_t)stream;
    CU(cudaSetDevice(c->device));
    Layout L;
    int64_t total = 0;
    ST(store_search(c, sys, L, &total, s));
    if (total != v.P)
        return fail(PANNA_ERR_INVALID_ARG, "the batch has %lld neighbour entries, the store was planned for %lld",
                    (long long)total, (long long)v.P);
    int& nl = c->last_launches;
    CU(cudaMemsetAsync(L.w.status, 0, sizeof(DevStatus), s));
    CU(species_order(L.w, c->d.S, s, &nl));
    CU(launch_store_offsets(L.w, v.ent_off, s, &nl));
    const bool acc = c->ang_mode != 2;
    int dummy = 0;
    const int variant = tuned_variant(c, sys, PANNA_MLP_FP32, KV_DESC, s, [&](int vv) {
        launch_descriptor(L.w, c->d, v.G, L.w.row_of_atom, acc, s, &dummy, vv);
    }, acc);
    CU(launch_descriptor(L.w, c->d, v.G, L.w.row_of_atom, acc, s, &nl, variant));
    const int64_t N = sys->n_atoms;
    CU(cudaMemcpyAsync(v.row_of_atom, L.w.row_of_atom, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(v.atom_of_row, L.w.atom_of_row, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(v.seg_off, L.w.seg_off, sizeof(int32_t) * (c->d.S + 1), cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(v.atom_cfg, L.w.atom_cfg, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    CU(launch_store_entries(L.w, v, s, &nl));
    CU(launch_store_jacobian(L.w, c->d, c->g64, v, s, &nl));
    CU(cudaGetLastError());
    int need = 0;
    return collect(c, L, s, &need);
}

panna_status panna_store_energy_forces(panna_ctx* c, const panna_system* sys, const panna_store_info* info,
                                       const void* store, const float* theta, int32_t prec, double* E_cfg,
                                       float* E_atom, float* F, double* virial, panna_stream_t stream)
{
    ST(check_system(c, sys, false));
    if (!theta || !E_cfg || !F) return fail(PANNA_ERR_INVALID_ARG, "theta, E_cfg and F are required");
    if (prec != PANNA_MLP_FP32 && prec != PANNA_MLP_BF16 && prec != PANNA_MLP_BF16_FAST)
        return fail(PANNA_ERR_INVALID_ARG, "bad precision");
    if (prec != PANNA_MLP_FP32 && (c->plan.L < 2 || c->d.D % 8 != 0))
        return fail(PANNA_ERR_UNSUPPORTED, "BF16 networks need a hidden layer and D a multiple of 8");
    StoreView v;
    ST(store_view(c, sys, info, store, v));
    Request rq;
    rq.theta = theta; rq.prec = prec; rq.E_cfg = E_cfg; rq.E_atom = E_atom; rq.F = F; rq.virial = virial;
    rq.forces = true; rq.energy = true; rq.store = &v;
    return run(c, sys, rq, (cudaStream_t)stream);
}

panna_status panna_store_loss_grad(panna_ctx* c, const panna_system* sys, const panna_store_info* info,
                                   const void* store, const float* theta, const double* E_ref, const float* F_ref,
                                   double w_force, double* loss, float* dtheta, double* E_cfg, float* F,
                                   panna_stream_t stream)
{
    ST(check_system(c, sys, false));
    if (!theta || !E_ref || !F_ref || !loss || !dtheta)
        return fail(PANNA_ERR_INVALID_ARG, "theta, E_ref, F_ref, loss and dtheta are required");
    StoreView v;
    ST(store_view(c, sys, info, store, v));
    Request rq;
    rq.theta = theta; rq.train = true; rq.E_ref = E_ref; rq.F_ref = F_ref; rq.w_force = w_force; rq.loss = loss;
    rq.dtheta = dtheta; rq.E_cfg = E_cfg; rq.F = F; rq.forces = true; rq.energy = true; rq.store = &v;
    return run(c, sys, rq, (cudaStream_t)stream);
}

panna_status panna_capture(panna_ctx* c, const panna_system* sys, const float* theta, int32_t prec, double* E_cfg,
                           float* E_atom, float* F, double* virial, panna_stream_t stream)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    // 1. one synchronous call: workspace sized, variants tuned, inputs validated
    ST(panna_energy_forces(c, sys, theta, prec, E_cfg, E_atom, F, virial, stream));
    // 2. record the same launches
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {
        if (!c->capture_stream) CU(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
        s = c->capture_stream;
    }
    if (c->graph_exec) {
        CU(cudaGraphExecDestroy(c->graph_exec));
        c->graph_exec = nullptr;
    }
    Request rq;
    rq.theta = theta; rq.prec = prec; rq.E_cfg = E_cfg; rq.E_atom = E_atom; rq.F = F; rq.virial = virial;
    rq.forces = true; rq.energy = true;
    const int old_async = c->async, old_prof = c->profiling;
    c->async = 1;
    c->profiling = 0;
    Layout L;
    panna_status st = prepare(c, sys, false, prec != PANNA_MLP_FP32, L, s);
    cudaGraph_t g = nullptr;
    if (st == PANNA_OK) {
        CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        c->last_launches = 0;
        st = run_once(c, sys, rq, L, s);
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st == PANNA_OK && e != cudaSuccess)
            st = fail(PANNA_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    }
    c->async = old_async;
    c->profiling = old_prof;
    if (st != PANNA_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    cudaError_t e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(PANNA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->graph_launches = c->last_launches;
    return PANNA_OK;
}

panna_status panna_replay(panna_ctx* c, panna_stream_t stream)
{
    if (!c || !c->graph_exec) return fail(PANNA_ERR_INVALID_ARG, "no captured graph");
    CU(cudaGraphLaunch(c->graph_exec, (cudaStream_t)stream));
    c->last_launches = c->graph_launches;
    return PANNA_OK;
}

int32_t panna_last_launch_count(const panna_ctx* c) { return c ? c->last_launches : -1; }

panna_status panna_set_profiling(panna_ctx* c, int32_t on)
{
    if (!c) return fail(PANNA_ERR_INVALID_ARG, "null context");
    c->profiling = on ? 1 : 0;
    return PANNA_OK;
}

float panna_stage_ms(const panna_ctx* c, const char* stage)
{
    if (!c || !stage || !c->profiling) return -1.f;
    for (int k = 0; k < kNumStages; ++k)
        if (strcmp(stage, kStages[k]) == 0) return c->stage_seen[k] ? c->stage_ms[k] : -1.f;
    return -1.f;
}

}  // extern "C"
