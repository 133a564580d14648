// cd_api.cu -- host runtime behind the C ABI of include/cd_api.h: the system
// object, the workspace layout, parameter validation and the order of the
// kernel launches for detection, colouring, solve and time step.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cd_internal.cuh"

struct cd_system {
    cd_params p;
    int64_t n;
    double* pos;
    double* vel;
    double* omega;
    double* theta;
    const double* radius;
    const double* inv_m;
    const double* inv_I;
    const double* f_ext;
    cudaStream_t stream;
    int device;
    int num_sms;
    int pw;
    int sweep_blocks;
    int sweep_threads;
    int colour_blocks;
    int has_contacts;
    size_t ws_bytes;
    void* ws;
    CdGeom g;
    CdWork w;
    int launches;                      // kernels launched since the call began
    std::vector<CdPack> pk_host;       // packing table (one entry for a plain system)
    std::vector<int> pack_of_host;     // packing of each particle (batched systems)
    std::vector<double> pk_wall0;      // initial wall planes, 6 per packing
    cudaGraphExec_t step_graph;        // params.use_graph: one captured time step
    int graph_launches;                // kernels in the captured step
    int tape_head;                     // next tape slot a step records into
    int tape_count;                    // recorded steps not yet consumed by cd_adjoint_step
    int adj_blocks;                    // cooperative grid of the adjoint kernel
    // params.merge_last_colour 4: sweeps + 1 of the last solve as last read
    // back (0: none yet), valid while no solve has been launched since; lets
    // a direct launch skip the merge passes the device would skip anyway
    int mg_hint = 0;
    bool mg_hint_valid = false;
    bool capturing = false;            // inside capture_step: every launch goes into the graph
    std::vector<cudaEvent_t> events;   // phase events (params.timing)
    size_t ev_used;
    std::string err;
};

static thread_local std::string g_create_err;

// Sets the message cd_last_error(NULL) returns (used by entry points that
// have no system object).
__attribute__((visibility("hidden"))) void cd_set_global_error(const char* msg)
{
    g_create_err = msg ? msg : "";
}

static cd_status fail(cd_system* s, cd_status st, const std::string& msg)
{
    if (s) s->err = msg; else g_create_err = msg;
    return st;
}

static cd_status cuda_fail(cd_system* s, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(s, CD_ERR_CUDA, m);
}

#define CD_CUDA(s, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Workspace layout: every array 256-byte aligned, in one caller buffer.
// ---------------------------------------------------------------------------
struct Layout {
    size_t off = 0;
    template <typename T>
    T* take(char* base, size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};

static size_t layout(cd_system* s, char* base, CdWork* w)
{
    Layout L;
    const size_t n = (size_t)s->n;
    const size_t cap = (size_t)s->p.max_contacts;
    const size_t ncell = (size_t)s->g.ncell_total;
    const size_t real = (s->p.precision == CD_FP64) ? 8 : 4;
    const size_t vrec = (s->p.dim == 2 ? 4 : 8) * real;   // velocity record bytes
    const size_t nchunk = (cap + CD_CHUNK - 1) / CD_CHUNK;
    const size_t G = (size_t)(s->sweep_blocks > s->colour_blocks ? s->sweep_blocks : s->colour_blocks) + 1;
    size_t scan_max = ncell + 1;
    if (n + 7 > scan_max) scan_max = n + 7;
    if (CD_KMAX * nchunk > scan_max) scan_max = CD_KMAX * nchunk;
    if (cap + 1 > scan_max) scan_max = cap + 1;   // the colour repair's scan over the contacts
    CdWork t;
    t.ctrl = L.take<CdCtrl>(base, 1);
    // records n .. n + 5 belong to force-controlled walls, then the domain views
    const size_t vcap = (s->g.ndom_total > 1) ? 2 * cap : 0;
    t.V = L.take<char>(base, (n + 6 + vcap) * vrec);
    t.S = L.take<char>(base, (n + 6) * 4 * real);
    t.cell_of = L.take<int>(base, n);
    t.cell_cnt = L.take<int>(base, ncell + 1);
    t.cell_start = L.take<int>(base, ncell + 1);
    t.cell_fill = L.take<int>(base, ncell);
    t.cell_pid = L.take<int>(base, n);
    t.pcnt = L.take<int>(base, n + 1);
    t.poff = L.take<int>(base, n + 1);
    t.poff_prev = L.take<int>(base, n + 1);
    t.cand = L.take<int>(base, n * CD_CAND);
    t.wmask = L.take<unsigned char>(base, n);
    t.pf = L.take<float4>(base, n);
    t.scan_tmp = L.take<int>(base, cd_scan_tmp_ints((int)scan_max) + 32);
    t.pairs = L.take<int2>(base, cap);
    t.pairs_nx = L.take<int2>(base, cap);
    t.Pk = L.take<double>(base, cap * s->pw);
    t.Pk_nx = L.take<double>(base, cap * s->pw);
    t.nrm = L.take<double>(base, cap * 3);
    t.gap = L.take<double>(base, cap);
    t.mn = L.take<double>(base, cap);
    t.mt = L.take<double>(base, cap);
    t.colour = L.take<int>(base, cap);
    t.p2c_cnt = L.take<int>(base, n + 7);
    t.p2c_off = L.take<int>(base, n + 7);
    t.p2c_fill = L.take<int>(base, n + 6);
    t.p2c = L.take<int>(base, 2 * cap);
    t.prio = L.take<unsigned long long>(base, cap);
    t.round_cnt = L.take<int>(base, 4);
    t.chunk_cnt = L.take<int>(base, CD_KMAX * nchunk + 1);
    t.colour_off = L.take<int>(base, CD_KMAX + 1);
    t.perm = L.take<int>(base, cap);
    t.c_ab = L.take<int2>(base, cap);
    t.c_geo = L.take<char>(base, cap * 4 * real);
    t.c_m = L.take<char>(base, cap * (s->p.dim == 2 ? 1 : 2) * real);
    t.c_P = L.take<char>(base, cap * (s->p.dim == 2 ? 2 : 4) * real);
    t.partials = L.take<double>(base, 2 * 3 * G);
    t.wpart = L.take<double>(base, 6 * G);
    const size_t npk = (size_t)s->g.npk;
    t.pk = L.take<CdPack>(base, npk);
    t.pack_of = L.take<int>(base, npk > 1 ? n : 1);
    t.pk_wall_pos = L.take<double>(base, 6 * npk);
    if (npk == 1 && base) t.pk_wall_pos = t.ctrl->wall_pos;   // the plain system's walls live in the control block
    t.pk_coff = L.take<int>(base, npk + 1);
    t.pk_done = L.take<int>(base, npk);
    t.pk_stats = L.take<double>(base, CD_PKSTATS * npk);
    t.c_abs = L.take<double>(base, cap);
    t.c_flag = L.take<int>(base, cap);
    t.act_cnt = L.take<int>(base, 8);
    {
        const size_t cb = (npk > 1) ? cap : 1;
        t.c_ab2 = L.take<int2>(base, cb);
        t.c_geo2 = L.take<char>(base, cb * 4 * real);
        t.c_m2 = L.take<char>(base, cb * (s->p.dim == 2 ? 1 : 2) * real);
        t.c_P2 = L.take<char>(base, cb * (s->p.dim == 2 ? 2 : 4) * real);
        t.perm2 = L.take<int>(base, cb);
        t.cmp_blk = L.take<int>(base, G);
        t.cmp_off = L.take<int>(base, CD_KMAX + 1);
    }
    t.c_dpar = L.take<double>(base, s->g.par_p > 0.0 ? cap * s->pw : 1);
    {
        const bool dom = s->g.ndom_total > 1;
        t.dom_key = L.take<int>(base, dom ? cap : 1);
        t.dom_home = L.take<int>(base, dom ? n : 1);
        t.view_cnt = L.take<int>(base, dom ? n + 1 : 1);
        t.view_off = L.take<int>(base, dom ? n + 1 : 1);
        t.view_owner = L.take<int>(base, dom ? vcap : 1);
        t.V0 = L.take<char>(base, (dom ? vcap : 1) * vrec);
        t.c_vab = L.take<int2>(base, dom ? cap : 1);
    }
    {
        const bool mg = s->g.merge_last != 0;
        const size_t nbk = CD_MG_MAXC * (size_t)s->g.merge_blocks + 1;
        t.mg_slot = L.take<int>(base, mg ? CD_MG_MAXC * n : 1);
        t.mg_label = L.take<int>(base, mg ? cap : 1);
        t.mg_size = L.take<int>(base, mg ? cap + 1 : 1);
        t.mg_w = L.take<int>(base, mg ? cap + 1 : 1);
        t.mg_start = L.take<int>(base, mg ? cap + 1 : 1);
        t.mg_bucket = L.take<int>(base, mg ? cap : 1);
        t.mg_list = L.take<int>(base, mg ? cap : 1);
        t.mg_bcnt = L.take<int>(base, mg ? nbk : 1);
        t.mg_boff = L.take<int>(base, mg ? nbk : 1);
        t.mg_bmin = L.take<int>(base, mg ? nbk : 1);
        t.mg_bmax = L.take<int>(base, mg ? nbk : 1);
    }
    t.rep_top = L.take<int>(base, npk);
    t.rep_dmax = L.take<int>(base, npk);
    t.rep_flag = L.take<int>(base, cap + 1);
    t.rep_pos = L.take<int>(base, cap + 1);
    t.rep_list = L.take<int>(base, cap);
    t.rep_path = L.take<int>(base, cap);
    t.obs = L.take<double>(base, CD_OBS_MAX);
    const size_t T = (size_t)s->p.tape_steps;
    t.tape = L.take<char>(base, T ? T * cd_tape_slot_bytes((int64_t)n, (int64_t)cap) : 1);
    t.adj_Y = L.take<double2>(base, T ? cap : 1);
    t.adj_B = L.take<double4_16a>(base, T ? 2 * n : 1);
    t.adj_lam = L.take<double4_16a>(base, T ? n : 1);
    t.adj_gx = L.take<double2>(base, T ? n : 1);
    t.adj_mark = L.take<int>(base, T ? n : 1);
    if (w) *w = t;
    return (L.off + 255) & ~(size_t)255;
}

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------
__global__ void k_begin_call(CdCtrl* ctrl, int reset_accum)
{
    ctrl->skip = 0;
    ctrl->overflow = 0;
    ctrl->error = CDE_NONE;
    if (reset_accum) {
        ctrl->steps_done = 0;
        ctrl->total_sweeps = 0;
        ctrl->total_updates = 0;
        ctrl->max_sweeps_step = 0;
        ctrl->n_not_conv = 0;
    }
}

__global__ void k_error_gate(CdCtrl* ctrl)
{
    if (ctrl->error != CDE_NONE) ctrl->skip = 1;
}

// Records the next phase event on the system's stream (params.timing).
static cd_status mark(cd_system* s)
{
    if (!s->p.timing) return CD_OK;
    if (s->ev_used == s->events.size()) {
        cudaEvent_t e;
        CD_CUDA(s, cudaEventCreate(&e));
        s->events.push_back(e);
    }
    CD_CUDA(s, cudaEventRecord(s->events[s->ev_used++], s->stream));
    return CD_OK;
}

// Sums the recorded phase intervals (5 events per step: before detection,
// after detection, after colouring + ordering + free flight, after the
// persistent sweep kernel, after integration).
static cd_status collect_phases(cd_system* s, double* phase_ms)
{
    for (int k = 0; k < 4; ++k) phase_ms[k] = 0.0;
    if (!s->p.timing) return CD_OK;
    for (size_t b = 0; b + 5 <= s->ev_used; b += 5) {
        for (int k = 0; k < 4; ++k) {
            float ms = 0.0f;
            CD_CUDA(s, cudaEventElapsedTime(&ms, s->events[b + k], s->events[b + k + 1]));
            phase_ms[k] += (double)ms;
        }
    }
    s->ev_used = 0;
    return CD_OK;
}

static cd_status read_ctrl(cd_system* s, CdCtrl* h)
{
    CD_CUDA(s, cudaMemcpyAsync(h, s->w.ctrl, sizeof(CdCtrl), cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    s->mg_hint = h->mg_prev;
    s->mg_hint_valid = true;
    return CD_OK;
}

static cd_status ctrl_status(cd_system* s, const CdCtrl& h)
{
    if (h.overflow) {
        char buf[160];
        snprintf(buf, sizeof buf, "contact capacity %lld exceeded: %d contacts needed",
                 (long long)s->p.max_contacts, h.nc_needed);
        return fail(s, CD_ERR_CAPACITY, buf);
    }
    if (h.error == CDE_TIMEOUT) return fail(s, CD_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (h.error == CDE_COLOURS) return fail(s, CD_ERR_CAPACITY, "the contact graph needs more than 64 colours");
    if (h.error == CDE_PER_PARTICLE) return fail(s, CD_ERR_CAPACITY, "a particle has more than 64 contact candidates");
    if (h.error == CDE_TAPE) return fail(s, CD_ERR_STATE, "the recorded step had failed (contact overflow or timeout)");
    return CD_OK;
}

static void fill_solve_stats(const cd_system* s, const CdCtrl& h, cd_solve_stats* o)
{
    o->sweeps = h.sweeps;
    o->converged = h.converged;
    o->residual = h.residual;
    o->r_avg = h.r_avg;
    o->n_contacts = h.nc;
    o->n_colours = h.ncolours;
    for (int k = 0; k < 6; ++k) o->wall_force[k] = h.wall_force[k];
    o->n_phases = h.ncolours - ((s->g.merge_last && h.merge >= 2) ? h.merge - 1 : 0);
}

static cd_status need_ready(cd_system* s)
{
    if (!s) return CD_ERR_INVALID_ARG;
    if (!s->ws) return fail(s, CD_ERR_OOM, "no workspace set (cd_workspace_size / cd_set_workspace)");
    CD_CUDA(s, cudaSetDevice(s->device));
    return CD_OK;
}

static cd_status launch_detect_chain(cd_system* s, int timed)
{
    cd_status st;
    CD_CUDA(s, cd_launch_detect(s->g, s->w, s->pos, s->radius, s->inv_m, s->inv_I, (int)s->p.warm_start, s->pw,
                                s->stream, &s->launches));
    if (s->g.npk > 1) CD_CUDA(s, cd_launch_pk_ranges(s->g, s->w, s->stream, &s->launches));
    if (timed && (st = mark(s)) != CD_OK) return st;
    CD_CUDA(s, cd_launch_colour(s->g, s->w, s->colour_blocks, (int)s->p.precision, s->pw, s->stream, &s->launches,
                                s->pos));
    k_error_gate<<<1, 1, 0, s->stream>>>(s->w.ctrl);
    ++s->launches;
    CD_CUDA(s, cudaGetLastError());
    if (s->g.ndom_total > 1)
        CD_CUDA(s, cd_launch_domains(s->g, s->w, s->pos, s->radius, s->stream, &s->launches));
    if (s->g.merge_last) {
        if (s->g.merge_auto && !s->capturing && s->mg_hint_valid && s->mg_hint > 0 &&
            s->mg_hint - 1 < CD_MG_MIN_SWEEPS) {
            // the previous solve was short (known on the host): no merge passes;
            // merge = -1 tells the sweep that this step is not merged
            CD_CUDA(s, cudaMemsetAsync(&s->w.ctrl->merge, 0xFF, sizeof(int), s->stream));
        } else {
            CD_CUDA(s, cd_launch_merge(s->g, s->w, s->colour_blocks, s->stream, &s->launches));
        }
    }
    return CD_OK;
}

static cd_status launch_solve(cd_system* s, int free_flight, int timed)
{
    cd_status st;
    s->mg_hint_valid = false;   // this solve's sweeps are unknown to the host until read back
    CD_CUDA(s, cd_launch_pack(s->g, s->w, s->vel, s->omega, s->radius, s->inv_m, s->inv_I, s->f_ext, free_flight,
                              (int)s->p.precision, s->stream, &s->launches));
    if (timed && (st = mark(s)) != CD_OK) return st;
    CD_CUDA(s, cd_launch_sweep(s->g, s->w, s->sweep_blocks, s->sweep_threads, (int)s->p.precision,
                               (int)s->p.criterion, s->p.alpha,
                               (int)s->p.max_sweeps, s->pw, s->stream, &s->launches));
    return CD_OK;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
static cd_status check_packing(const cd_params& p, int dim)
{
    if (!(p.mu >= 0.0) || !std::isfinite(p.mu)) return fail(nullptr, CD_ERR_INVALID_ARG, "mu must be >= 0");
    for (int k = 0; k < dim; ++k) {
        if (!(p.box_hi[k] > p.box_lo[k]) || !std::isfinite(p.box_hi[k] - p.box_lo[k]))
            return fail(nullptr, CD_ERR_INVALID_ARG, "box_hi must exceed box_lo on every axis");
    }
    for (int q = 0; q < 3; ++q)
        if (!std::isfinite(p.gravity[q])) return fail(nullptr, CD_ERR_INVALID_ARG, "gravity not finite");
    for (int k = 0; k < 6; ++k) {
        if (!((p.wall_mask >> k) & 1)) continue;
        if ((k >> 1) >= dim) return fail(nullptr, CD_ERR_INVALID_ARG, "wall on an axis the dimension lacks");
        if (p.periodic[k >> 1]) return fail(nullptr, CD_ERR_INVALID_ARG, "wall on a periodic axis");
        if (!std::isfinite(p.wall_pos[k])) return fail(nullptr, CD_ERR_INVALID_ARG, "wall position not finite");
    }
    if (((p.wall_mask & 3) == 3 && !(p.wall_pos[1] > p.wall_pos[0])) ||
        ((p.wall_mask & 12) == 12 && !(p.wall_pos[3] > p.wall_pos[2])) ||
        ((p.wall_mask & 48) == 48 && !(p.wall_pos[5] > p.wall_pos[4])))
        return fail(nullptr, CD_ERR_INVALID_ARG, "opposite walls overlap");
    return CD_OK;
}

// Shared by cd_create_system (one packing) and cd_create_batch.
static cd_status create_impl(const cd_params* params, int64_t npk, const int64_t* offsets, int64_t n, double* pos,
                             double* vel, double* omega, double* theta, const double* radius,
                             const double* inv_mass, const double* inv_inertia, const double* f_ext,
                             void* cuda_stream, cd_system** out)
{
    if (!out) return fail(nullptr, CD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!params) return fail(nullptr, CD_ERR_INVALID_ARG, "params is NULL");
    const cd_params& p = params[0];
    if (p.dim != 2 && p.dim != 3) return fail(nullptr, CD_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (p.precision != CD_FP64 && p.precision != CD_FP32) return fail(nullptr, CD_ERR_INVALID_ARG, "bad precision");
    if (n <= 0 || n + 6 * npk >= (int64_t)0x7fffffff) return fail(nullptr, CD_ERR_INVALID_ARG, "particle count out of range");
    if (!(p.dt > 0.0) || !std::isfinite(p.dt)) return fail(nullptr, CD_ERR_INVALID_ARG, "dt must be positive");
    if (!(p.delta >= 0.0) || !std::isfinite(p.delta)) return fail(nullptr, CD_ERR_INVALID_ARG, "delta must be >= 0");
    if (!(p.alpha >= 0.0)) return fail(nullptr, CD_ERR_INVALID_ARG, "alpha must be >= 0");
    if (p.max_sweeps < 0) return fail(nullptr, CD_ERR_INVALID_ARG, "max_sweeps must be >= 0");
    if (p.criterion < CD_CONV_NONE || p.criterion > CD_CONV_LOCAL) return fail(nullptr, CD_ERR_INVALID_ARG, "bad criterion");
    if (p.max_contacts <= 0 || p.max_contacts > (int64_t)0x3fffffff)
        return fail(nullptr, CD_ERR_INVALID_ARG, "max_contacts out of range");
    if (!pos || !vel || !omega || !radius || !inv_mass || !inv_inertia)
        return fail(nullptr, CD_ERR_INVALID_ARG, "a required state array is NULL");
    if (npk < 1 || npk > (1 << 20)) return fail(nullptr, CD_ERR_INVALID_ARG, "packing count out of range");
    if (offsets[0] != 0 || offsets[npk] != n) return fail(nullptr, CD_ERR_INVALID_ARG, "offsets must run from 0 to n");
    for (int64_t b = 0; b < npk; ++b) {
        if (offsets[b + 1] < offsets[b]) return fail(nullptr, CD_ERR_INVALID_ARG, "offsets must not decrease");
        cd_status st = check_packing(params[b], (int)p.dim);
        if (st != CD_OK) return st;
    }

    cd_system* s = new cd_system();
    s->p = p;
    s->n = n;
    s->pos = pos; s->vel = vel; s->omega = omega; s->theta = theta;
    s->radius = radius; s->inv_m = inv_mass; s->inv_I = inv_inertia; s->f_ext = f_ext;
    s->stream = (cudaStream_t)cuda_stream;
    s->pw = (p.dim == 2) ? 2 : 4;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
    if (e != cudaSuccess) { cuda_fail(nullptr, e, "device query"); delete s; return CD_ERR_CUDA; }
    if (!coop) { delete s; return fail(nullptr, CD_ERR_CUDA, "device lacks cooperative launch"); }

    // radii, inverse masses, positions and velocities: validated on the host once
    std::vector<double> hr((size_t)n), hm((size_t)n), hx((size_t)(n * p.dim)), hv((size_t)(n * p.dim));
    e = cudaMemcpy(hr.data(), radius, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hm.data(), inv_mass, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hx.data(), pos, sizeof(double) * hx.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hv.data(), vel, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { cuda_fail(nullptr, e, "reading the particle state"); delete s; return CD_ERR_CUDA; }
    for (size_t i = 0; i < hx.size(); ++i) {
        if (!std::isfinite(hx[i]) || !std::isfinite(hv[i])) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG, "positions and velocities must be finite");
        }
    }
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(hr[(size_t)i] > 0.0) || !std::isfinite(hr[(size_t)i])) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG, "radius must be positive and finite");
        }
        if (!(hm[(size_t)i] >= 0.0) || !std::isfinite(hm[(size_t)i])) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG, "inv_mass must be >= 0 and finite");
        }
        if (hr[(size_t)i] > rmax) rmax = hr[(size_t)i];
    }

    CdGeom& g = s->g;
    memset(&g, 0, sizeof g);
    g.dim = (int)p.dim;
    g.n = (int)n;
    g.cap = (int)p.max_contacts;
    g.wall_mask = (int)p.wall_mask;
    g.delta = p.delta;
    g.dt = p.dt;
    g.mu = p.mu;
    g.rotations = (int)p.rotations;
    g.seed = p.seed;
    g.npk = (int)npk;
    for (int k = 0; k < 18; ++k) g.wall_vel[k] = p.wall_vel[k];
    // Sec. 3.1: cell side l = 2 r_max + delta, here longer by a relative 1e-9:
    // rounding may file a particle within a few ulps of a cell face in the
    // neighbouring cell, and a side longer than any contact distance by more
    // than that keeps every contact within the cells next to its particles'
    // (for grids of up to 1e6 cells per axis)
    const double ell = (2.0 * rmax + p.delta) * (1.0 + 1e-9);
    double ncell_total = 0.0;
    s->pk_host.resize((size_t)npk);
    s->pk_wall0.resize((size_t)(6 * npk));
    for (int64_t b = 0; b < npk; ++b) {
        const cd_params& q = params[b];
        CdPack& pk = s->pk_host[(size_t)b];
        memset(&pk, 0, sizeof pk);
        double cells = 1.0;
        for (int k = 0; k < 3; ++k) {
            pk.periodic[k] = (k < p.dim) ? (int)q.periodic[k] : 0;
            pk.gravity[k] = q.gravity[k];
            if (k < p.dim) {
                pk.lo[k] = q.box_lo[k];
                pk.hi[k] = q.box_hi[k];
                pk.L[k] = q.box_hi[k] - q.box_lo[k];
                double m = std::floor(pk.L[k] / ell);
                if (m < 1.0) m = 1.0;
                if (m > 1.0e6) m = 1.0e6;
                pk.ncell[k] = (int)m;
                pk.cs[k] = pk.L[k] / m;
                pk.inv_cs[k] = 1.0 / pk.cs[k];
                if (pk.periodic[k] && pk.ncell[k] < 3) {
                    delete s;
                    return fail(nullptr, CD_ERR_INVALID_ARG, "a periodic axis needs at least 3 cells (box >= 3 l)");
                }
            } else {
                pk.lo[k] = 0.0; pk.hi[k] = 1.0; pk.L[k] = 1.0; pk.ncell[k] = 1; pk.cs[k] = 1.0; pk.inv_cs[k] = 1.0;
            }
            cells *= pk.ncell[k];
        }
        pk.cell_base = (int)ncell_total;
        ncell_total += cells;
        pk.wall_mask = (int)q.wall_mask;
        pk.mu = q.mu;
        for (int k = 0; k < 18; ++k) pk.wall_vel[k] = q.wall_vel[k];
        for (int k = 0; k < 6; ++k) s->pk_wall0[(size_t)(6 * b + k)] = q.wall_pos[k];
        pk.first = (int)offsets[b];
        pk.count = (int)(offsets[b + 1] - offsets[b]);
        pk.seed = q.seed;
    }
    if (ncell_total > 2.0e8) { delete s; return fail(nullptr, CD_ERR_INVALID_ARG, "cell grid too large for the box"); }
    g.ncell_total = (int)ncell_total;
    {
        const CdPack& p0 = s->pk_host[0];
        for (int k = 0; k < 3; ++k) {
            g.gravity[k] = p.gravity[k];
            g.periodic[k] = p0.periodic[k];
            g.lo[k] = p0.lo[k]; g.hi[k] = p0.hi[k]; g.L[k] = p0.L[k];
            g.ncell[k] = p0.ncell[k]; g.cs[k] = p0.cs[k]; g.inv_cs[k] = p0.inv_cs[k];
        }
    }
    if (npk > 1) {
        s->pack_of_host.resize((size_t)n);
        for (int64_t b = 0; b < npk; ++b)
            for (int64_t i = offsets[b]; i < offsets[b + 1]; ++i) s->pack_of_host[(size_t)i] = (int)b;
    }
    if (!(p.parallel_p >= 0.0 && p.parallel_p <= 1.0)) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "parallel_p must be in [0, 1]");
    }
    if (p.parallel_p > 0.0 && npk > 1) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "parallel_p needs a plain system with the colour-barrier schedule");
    }
    g.par_p = p.parallel_p;
    if (p.parallel_redraw != 0 && p.parallel_redraw != 1) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "parallel_redraw must be 0 or 1");
    }
    g.par_redraw = (int)p.parallel_redraw;
    {
        // force-controlled walls
        int dyn = 0;
        for (int k = 0; k < 6; ++k) {
            if (!std::isfinite(p.wall_push[k]) || !(p.wall_mass[k] >= 0.0) || !std::isfinite(p.wall_mass[k])) {
                delete s;
                return fail(nullptr, CD_ERR_INVALID_ARG, "wall_push must be finite and wall_mass >= 0");
            }
            if (p.wall_mass[k] > 0.0) {
                if (!((p.wall_mask >> k) & 1) || (k >> 1) >= p.dim) {
                    delete s;
                    return fail(nullptr, CD_ERR_INVALID_ARG, "a force-controlled wall must be present");
                }
                dyn |= 1 << k;
                g.wall_im[k] = 1.0 / p.wall_mass[k];
                g.wall_push[k] = p.wall_push[k];
            }
        }
        for (int64_t b = 1; b < npk; ++b)
            for (int k = 0; k < 6; ++k)
                if (params[b].wall_mass[k] > 0.0) dyn |= 1 << 8;
        if (dyn && (npk > 1 || p.parallel_p > 0.0 || p.tape_steps > 0)) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG,
                        "force-controlled walls need a plain system with no mixed update and no tape");
        }
        g.dyn_walls = dyn;
    }
    {
        // domain-wise update (Sec. 3.1)
        long long total = 1;
        for (int k = 0; k < 3; ++k) {
            if (p.domains[k] < 0 || p.domains[k] > 65536) {
                delete s;
                return fail(nullptr, CD_ERR_INVALID_ARG, "domains must be in [0, 65536] per axis");
            }
            g.ndom[k] = (k < p.dim && p.domains[k] > 1) ? (int)p.domains[k] : 1;
            total *= g.ndom[k];
        }
        for (int64_t b = 1; b < npk; ++b)
            for (int k = 0; k < 3; ++k)
                if (params[b].domains[k] > 1) total = total > 1 ? total : 2;
        if (total > (1LL << 24)) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG, "at most 2^24 domains");
        }
        if (total > 1 && (npk > 1 || p.parallel_p > 0.0 || g.dyn_walls ||
                          p.tape_steps > 0)) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG,
                        "domains need a plain system with kinematic walls, no mixed update and no tape");
        }
        g.ndom_total = (int)total;
    }
    if (p.use_graph && p.timing) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "use_graph needs timing 0 (a replayed step records no phase events)");
    }
    if (!(p.adjoint_compliance >= 0.0) || !std::isfinite(p.adjoint_compliance)) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "adjoint_compliance must be >= 0");
    }
    if (p.tape_steps < 0 || p.tape_steps > 100000) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "tape_steps must be in [0, 100000]");
    }
    if (p.tape_steps > 0 && (p.dim != 2 || p.precision != CD_FP64 || npk > 1)) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG,
                    "tape_steps (the adjoint) needs a plain 2D FP64 system");
    }
    s->adj_blocks = (p.tape_steps > 0 && cd_adjoint_blocks_per_sm() >= 1) ? s->num_sms : 0;
    if (p.tape_steps > 0 && s->adj_blocks == 0) {
        delete s;
        return fail(nullptr, CD_ERR_CUDA, "the adjoint kernel does not fit on this device");
    }
    s->sweep_blocks = cd_sweep_max_blocks((int)p.precision, (int)p.dim, s->num_sms);
    s->colour_blocks = cd_colour_max_blocks(s->num_sms);
    if (s->sweep_blocks <= 0 || s->colour_blocks <= 0) {
        delete s;
        return fail(nullptr, CD_ERR_CUDA, "cooperative kernels do not fit on this device");
    }
    {
        // block shape of the persistent sweep grid (params.sweep_threads / sweep_blocks_per_sm)
        const int th = p.sweep_threads ? (int)p.sweep_threads : CD_SWEEP_THREADS;
        const int per = p.sweep_blocks_per_sm ? (int)p.sweep_blocks_per_sm : 1;
        if ((th != 128 && th != 256 && th != 512) || (per != 1 && per != 2 && per != 4) || th * per > 1024) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG,
                        "sweep_threads must be 128, 256 or 512 and sweep_blocks_per_sm 1, 2 or 4 (at most 1024 "
                        "threads per SM)");
        }
        if (!cd_sweep_fits(g, (int)p.precision, th, per)) {
            delete s;
            return fail(nullptr, CD_ERR_INVALID_ARG, "that many sweep blocks do not fit on one SM");
        }
        s->sweep_threads = th;
        s->sweep_blocks = s->num_sms * per;
    }
    // merging of the last colours: plain systems with the colour-barrier
    // schedule (ignored otherwise)
    if (p.merge_last_colour < 0 || p.merge_last_colour > 4) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "merge_last_colour must be 0, 1, 2, 3 or 4");
    }
    g.merge_auto = (p.merge_last_colour == 4) ? 1 : 0;
    g.merge_last = (p.merge_last_colour && npk == 1 && g.par_p == 0.0 &&
                    g.ndom_total == 1 && !g.dyn_walls && p.tape_steps == 0 && cd_merge_label_blocks_per_sm() >= 1)
                       ? (p.merge_last_colour == 2 ? 2 : 3) : 0;
    g.merge_blocks = s->sweep_blocks;
    if (g.merge_last && !cd_sweep_fits(g, (int)p.precision, s->sweep_threads, s->sweep_blocks / s->num_sms)) {
        delete s;
        return fail(nullptr, CD_ERR_INVALID_ARG, "that many sweep blocks do not fit on one SM");
    }
    *out = s;
    return CD_OK;
}

extern "C" cd_status cd_create_system(const cd_params* params, int64_t n, double* pos, double* vel, double* omega,
                                      double* theta, const double* radius, const double* inv_mass,
                                      const double* inv_inertia, const double* f_ext, void* cuda_stream,
                                      cd_system** out)
{
    const int64_t offsets[2] = {0, n};
    return create_impl(params, 1, offsets, n, pos, vel, omega, theta, radius, inv_mass, inv_inertia, f_ext,
                       cuda_stream, out);
}

extern "C" cd_status cd_create_batch(const cd_params* params, int64_t n_packings, const int64_t* offsets_host,
                                     double* pos, double* vel, double* omega, double* theta, const double* radius,
                                     const double* inv_mass, const double* inv_inertia, const double* f_ext,
                                     void* cuda_stream, cd_system** out)
{
    if (!offsets_host || n_packings < 1) return fail(nullptr, CD_ERR_INVALID_ARG, "offsets or packing count missing");
    return create_impl(params, n_packings, offsets_host, offsets_host[n_packings], pos, vel, omega, theta, radius,
                       inv_mass, inv_inertia, f_ext, cuda_stream, out);
}

extern "C" cd_status cd_workspace_size(const cd_system* sys, size_t* bytes)
{
    if (!sys || !bytes) return CD_ERR_INVALID_ARG;
    *bytes = layout(const_cast<cd_system*>(sys), nullptr, nullptr);
    return CD_OK;
}

extern "C" cd_status cd_set_workspace(cd_system* s, void* dev_ptr, size_t bytes)
{
    if (!s) return CD_ERR_INVALID_ARG;
    size_t need = layout(s, nullptr, nullptr);
    if (!dev_ptr || bytes < need) return fail(s, CD_ERR_OOM, "workspace missing or smaller than cd_workspace_size()");
    if (((uintptr_t)dev_ptr & 255) != 0) return fail(s, CD_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    CD_CUDA(s, cudaSetDevice(s->device));
    s->ws = dev_ptr;
    s->ws_bytes = bytes;
    layout(s, (char*)dev_ptr, &s->w);
    CdCtrl h;
    memset(&h, 0, sizeof h);
    for (int k = 0; k < 6; ++k) h.wall_pos[k] = s->pk_wall0[(size_t)k];
    CD_CUDA(s, cudaMemcpyAsync(s->w.ctrl, &h, sizeof h, cudaMemcpyHostToDevice, s->stream));
    CD_CUDA(s, cudaMemcpyAsync(s->w.pk, s->pk_host.data(), sizeof(CdPack) * s->pk_host.size(), cudaMemcpyHostToDevice,
                               s->stream));
    if (s->g.npk > 1) {
        CD_CUDA(s, cudaMemcpyAsync(s->w.pack_of, s->pack_of_host.data(), sizeof(int) * s->pack_of_host.size(),
                                   cudaMemcpyHostToDevice, s->stream));
        CD_CUDA(s, cudaMemcpyAsync(s->w.pk_wall_pos, s->pk_wall0.data(), sizeof(double) * s->pk_wall0.size(),
                                   cudaMemcpyHostToDevice, s->stream));
    }
    CD_CUDA(s, cd_launch_static(s->g, s->w, s->radius, s->inv_m, s->inv_I, (int)s->p.precision, s->stream,
                                &s->launches));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    s->has_contacts = 0;
    s->tape_head = 0;
    s->tape_count = 0;
    if (s->step_graph) {
        cudaGraphExecDestroy(s->step_graph);
        s->step_graph = nullptr;
    }
    return CD_OK;
}

extern "C" cd_status cd_detect_contacts(cd_system* s, int64_t* n_contacts)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    k_begin_call<<<1, 1, 0, s->stream>>>(s->w.ctrl, 0);
    if ((st = launch_detect_chain(s, 0)) != CD_OK) return st;
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    if (n_contacts) *n_contacts = h.overflow ? h.nc_needed : h.nc;
    st = ctrl_status(s, h);
    if (st == CD_OK) s->has_contacts = 1;
    return st;
}

extern "C" cd_status cd_set_contacts(cd_system* s, int64_t nc, const int32_t* pairs, const double* impulses)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (nc < 0 || nc > s->p.max_contacts) return fail(s, CD_ERR_CAPACITY, "contact list larger than max_contacts");
    if (nc > 0 && !pairs) return fail(s, CD_ERR_INVALID_ARG, "pairs is NULL");
    k_begin_call<<<1, 1, 0, s->stream>>>(s->w.ctrl, 0);
    CD_CUDA(s, cd_launch_set_contacts(s->g, s->w, s->pos, s->radius, s->inv_m, s->inv_I, (int)nc, pairs, impulses,
                                      s->pw, s->stream, &s->launches));
    if (s->g.npk > 1) CD_CUDA(s, cd_launch_pk_ranges(s->g, s->w, s->stream, &s->launches));
    CD_CUDA(s, cd_launch_colour(s->g, s->w, s->colour_blocks, (int)s->p.precision, s->pw, s->stream, &s->launches,
                                s->pos));
    k_error_gate<<<1, 1, 0, s->stream>>>(s->w.ctrl);
    if (s->g.ndom_total > 1)
        CD_CUDA(s, cd_launch_domains(s->g, s->w, s->pos, s->radius, s->stream, &s->launches));
    if (s->g.merge_last) CD_CUDA(s, cd_launch_merge(s->g, s->w, s->colour_blocks, s->stream, &s->launches));
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    st = ctrl_status(s, h);
    if (st == CD_OK) s->has_contacts = 1;
    return st;
}

extern "C" cd_status cd_solve_contacts(cd_system* s, cd_solve_stats* out)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (!s->has_contacts) return fail(s, CD_ERR_STATE, "no contact set: call cd_detect_contacts or cd_set_contacts");
    k_begin_call<<<1, 1, 0, s->stream>>>(s->w.ctrl, 1);
    if ((st = launch_solve(s, 0, 0)) != CD_OK) return st;
    CD_CUDA(s, cd_launch_unpack(s->g, s->w, s->pos, s->vel, s->omega, s->theta, 0, (int)s->p.precision, s->stream,
                                &s->launches));
    if (!out) return CD_OK;
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    if ((st = ctrl_status(s, h)) != CD_OK) return st;
    fill_solve_stats(s, h, out);
    return h.converged ? CD_OK : CD_ERR_NOT_CONVERGED;
}

// The launches of one time step (Fig. 3): detection, colouring and order,
// free flight, the solve, the Euler update and, with a tape, its record.
static cd_status launch_step(cd_system* s, int timed)
{
    cd_status st;
    if (timed && (st = mark(s)) != CD_OK) return st;
    if ((st = launch_detect_chain(s, timed)) != CD_OK) return st;
    if ((st = launch_solve(s, 1, timed)) != CD_OK) return st;
    if (timed && (st = mark(s)) != CD_OK) return st;
    CD_CUDA(s, cd_launch_unpack(s->g, s->w, s->pos, s->vel, s->omega, s->theta, 1, (int)s->p.precision, s->stream,
                                &s->launches));
    if (timed && (st = mark(s)) != CD_OK) return st;
    if (s->p.tape_steps > 0)
        CD_CUDA(s, cd_launch_tape_record(s->g, s->w, s->p.max_contacts, (int)s->p.tape_steps, s->stream,
                                         &s->launches));
    return CD_OK;
}

// Captures launch_step into a CUDA graph on the system's stream.
static cd_status capture_step(cd_system* s)
{
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamBeginCapture (use_graph needs a non-default stream)");
    const int l0 = s->launches;
    s->capturing = true;
    cd_status st = launch_step(s, 0);
    s->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s->stream, &graph);
    if (st != CD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
    s->graph_launches = s->launches - l0;
    s->launches = l0;
    e = cudaGraphInstantiate(&s->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        s->step_graph = nullptr;
        return cuda_fail(s, e, "cudaGraphInstantiate");
    }
    return CD_OK;
}

extern "C" cd_status cd_step(cd_system* s, int64_t n_steps, cd_step_stats* out)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (n_steps < 0) return fail(s, CD_ERR_INVALID_ARG, "n_steps must be >= 0");
    s->launches = 0;
    k_begin_call<<<1, 1, 0, s->stream>>>(s->w.ctrl, 1);
    ++s->launches;
    const bool graph = s->p.use_graph != 0;
    if (graph && n_steps > 0 && !s->step_graph && (st = capture_step(s)) != CD_OK) return st;
    for (int64_t i = 0; i < n_steps; ++i) {
        if (graph) {
            CD_CUDA(s, cudaGraphLaunch(s->step_graph, s->stream));
            s->launches += s->graph_launches;
        } else if ((st = launch_step(s, 1)) != CD_OK) {
            return st;
        }
        if (s->p.tape_steps > 0) {
            const int T = (int)s->p.tape_steps;
            s->tape_head = (s->tape_head + 1) % T;
            if (s->tape_count < T) ++s->tape_count;
        }
    }
    if (n_steps > 0) s->has_contacts = 1;
    if (!out) return CD_OK;
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    out->steps_done = h.steps_done;
    out->total_sweeps = h.total_sweeps;
    out->total_contact_updates = h.total_updates;
    out->max_sweeps_in_step = h.max_sweeps_step;
    out->n_not_converged = h.n_not_conv;
    out->kernel_launches = s->launches;
    if ((st = collect_phases(s, out->phase_ms)) != CD_OK) return st;
    fill_solve_stats(s, h, &out->last);
    if ((st = ctrl_status(s, h)) != CD_OK) return st;
    return h.n_not_conv ? CD_ERR_NOT_CONVERGED : CD_OK;
}

extern "C" cd_status cd_get_contacts(cd_system* s, int64_t* n_contacts, int32_t* pairs, double* normal, double* gap,
                                     double* impulse, int32_t* colour)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    size_t nc = (size_t)h.nc;
    if (n_contacts) *n_contacts = (int64_t)nc;
    if (nc == 0) return CD_OK;
    cudaStream_t q = s->stream;
    if (pairs) CD_CUDA(s, cudaMemcpyAsync(pairs, s->w.pairs, nc * sizeof(int2), cudaMemcpyDeviceToDevice, q));
    if (normal) CD_CUDA(s, cudaMemcpyAsync(normal, s->w.nrm, nc * 3 * sizeof(double), cudaMemcpyDeviceToDevice, q));
    if (gap) CD_CUDA(s, cudaMemcpyAsync(gap, s->w.gap, nc * sizeof(double), cudaMemcpyDeviceToDevice, q));
    if (impulse)
        CD_CUDA(s, cudaMemcpyAsync(impulse, s->w.Pk, nc * s->pw * sizeof(double), cudaMemcpyDeviceToDevice, q));
    if (colour) CD_CUDA(s, cudaMemcpyAsync(colour, s->w.colour, nc * sizeof(int), cudaMemcpyDeviceToDevice, q));
    CD_CUDA(s, cudaStreamSynchronize(q));
    return CD_OK;
}

extern "C" cd_status cd_get_walls(cd_system* s, double* wall_pos_host)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (!wall_pos_host) return fail(s, CD_ERR_INVALID_ARG, "wall_pos_host is NULL");
    CD_CUDA(s, cudaMemcpyAsync(wall_pos_host, s->w.pk_wall_pos, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    return CD_OK;
}

extern "C" cd_status cd_upload_state(cd_system* s, const double* pos_host, const double* vel_host,
                                     const double* omega_host)
{
    if (!s) return CD_ERR_INVALID_ARG;
    CD_CUDA(s, cudaSetDevice(s->device));
    size_t nd = (size_t)s->n * (size_t)s->p.dim * sizeof(double);
    size_t nw = (size_t)s->n * (s->p.dim == 2 ? 1 : 3) * sizeof(double);
    if (pos_host) CD_CUDA(s, cudaMemcpyAsync(s->pos, pos_host, nd, cudaMemcpyHostToDevice, s->stream));
    if (vel_host) CD_CUDA(s, cudaMemcpyAsync(s->vel, vel_host, nd, cudaMemcpyHostToDevice, s->stream));
    if (omega_host) CD_CUDA(s, cudaMemcpyAsync(s->omega, omega_host, nw, cudaMemcpyHostToDevice, s->stream));
    return CD_OK;
}

extern "C" cd_status cd_download_state(cd_system* s, double* pos_host, double* vel_host, double* omega_host)
{
    if (!s) return CD_ERR_INVALID_ARG;
    CD_CUDA(s, cudaSetDevice(s->device));
    size_t nd = (size_t)s->n * (size_t)s->p.dim * sizeof(double);
    size_t nw = (size_t)s->n * (s->p.dim == 2 ? 1 : 3) * sizeof(double);
    if (pos_host) CD_CUDA(s, cudaMemcpyAsync(pos_host, s->pos, nd, cudaMemcpyDeviceToHost, s->stream));
    if (vel_host) CD_CUDA(s, cudaMemcpyAsync(vel_host, s->vel, nd, cudaMemcpyDeviceToHost, s->stream));
    if (omega_host) CD_CUDA(s, cudaMemcpyAsync(omega_host, s->omega, nw, cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    return CD_OK;
}

extern "C" cd_status cd_get_packing_stats(cd_system* s, int64_t first, int64_t count, cd_packing_stats* out_host)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (!out_host || first < 0 || count < 0 || first + count > s->g.npk)
        return fail(s, CD_ERR_INVALID_ARG, "packing range out of bounds");
    if (count == 0) return CD_OK;
    std::vector<double> hs((size_t)(CD_PKSTATS * count)), hw((size_t)(6 * count));
    std::vector<int> hc((size_t)count + 1);
    CD_CUDA(s, cudaMemcpyAsync(hs.data(), s->w.pk_stats + CD_PKSTATS * first, sizeof(double) * hs.size(),
                               cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaMemcpyAsync(hw.data(), s->w.pk_wall_pos + 6 * first, sizeof(double) * hw.size(),
                               cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaMemcpyAsync(hc.data(), s->w.pk_coff + first, sizeof(int) * hc.size(), cudaMemcpyDeviceToHost,
                               s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < count; ++i) {
        const double* q = hs.data() + CD_PKSTATS * i;
        cd_packing_stats& o = out_host[i];
        o.sweeps = (int64_t)q[PKS_SWEEPS];
        o.converged = (int64_t)q[PKS_CONV];
        o.residual = q[PKS_RESID];
        o.r_avg = q[PKS_RAVG];
        o.n_contacts = (s->g.npk > 1) ? (int64_t)(hc[(size_t)i + 1] - hc[(size_t)i]) : (int64_t)q[PKS_NC];
        for (int k = 0; k < 6; ++k) {
            o.wall_force[k] = q[PKS_WF0 + k];
            o.wall_pos[k] = hw[(size_t)(6 * i + k)];
        }
    }
    return CD_OK;
}

extern "C" cd_status cd_force_orientation(cd_system* s, int64_t nbins, int64_t* counts_host)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (s->p.dim != 2) return fail(s, CD_ERR_INVALID_ARG, "the force-orientation distribution is defined in 2D");
    if (nbins < 1 || nbins > CD_OBS_MAX || !counts_host) return fail(s, CD_ERR_INVALID_ARG, "bad nbins or output");
    if (!s->has_contacts) return fail(s, CD_ERR_STATE, "no contact set");
    unsigned long long* d = reinterpret_cast<unsigned long long*>(s->w.obs);
    CD_CUDA(s, cd_launch_orient(s->g, s->w, (int)nbins, d, s->stream, &s->launches));
    std::vector<unsigned long long> h((size_t)nbins);
    CD_CUDA(s, cudaMemcpyAsync(h.data(), d, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    for (int64_t i = 0; i < nbins; ++i) counts_host[i] = (int64_t)h[(size_t)i];
    return CD_OK;
}

extern "C" cd_status cd_stress_profile(cd_system* s, int64_t axis, double lo, double width, int64_t nstripes,
                                       double* sigma_host)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (axis < 0 || axis >= s->p.dim) return fail(s, CD_ERR_INVALID_ARG, "axis out of range");
    if (!(width > 0.0) || nstripes < 1 || nstripes > CD_OBS_MAX || !sigma_host)
        return fail(s, CD_ERR_INVALID_ARG, "bad stripes or output");
    if (s->g.npk > 1) return fail(s, CD_ERR_INVALID_ARG, "stress profiles are per system (use a plain system)");
    if (!s->has_contacts) return fail(s, CD_ERR_STATE, "no contact set");
    CD_CUDA(s, cd_launch_stress(s->g, s->w, s->pos, s->radius, (int)axis, lo, width, (int)nstripes, s->w.obs,
                                s->stream, &s->launches));
    CD_CUDA(s, cudaMemcpyAsync(sigma_host, s->w.obs, sizeof(double) * (size_t)nstripes, cudaMemcpyDeviceToHost,
                               s->stream));
    CD_CUDA(s, cudaStreamSynchronize(s->stream));
    double area = width;
    for (int k = 0; k < s->p.dim; ++k)
        if (k != axis) area *= s->g.L[k];
    for (int64_t i = 0; i < nstripes; ++i) sigma_host[i] /= area;
    return CD_OK;
}

// ---------------------------------------------------------------------------
// Adjoint and checkpoints
// ---------------------------------------------------------------------------
extern "C" cd_status cd_adjoint_step(cd_system* s, const double* dL_dpos, const double* dL_dvel,
                                     const double* dL_domega, const double* dL_dwall_force_host,
                                     double* dL_dpos_prev, double* dL_dvel_prev, double* dL_domega_prev, double alpha,
                                     int64_t max_sweeps, cd_adjoint_stats* out_host)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    if (s->p.tape_steps <= 0) return fail(s, CD_ERR_STATE, "no tape: create the system with tape_steps > 0");
    if (s->tape_count <= 0) return fail(s, CD_ERR_STATE, "no recorded step left on the tape");
    if (!dL_dpos || !dL_dvel || !dL_domega || !dL_dpos_prev || !dL_dvel_prev || !dL_domega_prev)
        return fail(s, CD_ERR_INVALID_ARG, "a gradient array is NULL");
    if (!(alpha >= 0.0) || max_sweeps < 1 || max_sweeps > (int64_t)0x7fffffff)
        return fail(s, CD_ERR_INVALID_ARG, "alpha must be >= 0 and max_sweeps >= 1");
    const int T = (int)s->p.tape_steps;
    const int slot = (s->tape_head + T - 1) % T;
    s->launches = 0;
    k_begin_call<<<1, 1, 0, s->stream>>>(s->w.ctrl, 0);
    ++s->launches;
    CD_CUDA(s, cudaGetLastError());
    CdAdjIO io;
    io.dLx = dL_dpos; io.dLv = dL_dvel; io.dLw = dL_domega;
    io.ox = dL_dpos_prev; io.ov = dL_dvel_prev; io.ow = dL_domega_prev;
    io.inv_I = s->inv_I;
    io.eps = s->p.adjoint_compliance;
    for (int k = 0; k < 6; ++k) {
        const double f = dL_dwall_force_host ? dL_dwall_force_host[k] : 0.0;
        if (!std::isfinite(f)) return fail(s, CD_ERR_INVALID_ARG, "dL_dwall_force not finite");
        io.wq[k] = f / s->p.dt;
    }
    CD_CUDA(s, cd_launch_adjoint(s->g, s->w, cd_tape_slot(s->w.tape, s->n, s->p.max_contacts, slot), io, alpha,
                                 (int)max_sweeps, s->adj_blocks, s->stream, &s->launches));
    CdCtrl h;
    if ((st = read_ctrl(s, &h)) != CD_OK) return st;
    if ((st = ctrl_status(s, h)) != CD_OK) return st;
    s->tape_head = slot;
    --s->tape_count;
    CD_CUDA(s, cd_launch_set_tape_slot(s->w, slot, s->stream, &s->launches));
    if (out_host) {
        out_host->sweeps = h.adj_sweeps;
        out_host->converged = h.adj_converged;
        out_host->residual = h.adj_residual;
        out_host->n_contacts = h.adj_nc;
        out_host->n_stick = h.adj_nstick;
        out_host->n_slide = h.adj_nslide;
        out_host->n_open = h.adj_nc - h.adj_nstick - h.adj_nslide;
        out_host->dL_dmu = h.adj_dmu;
        out_host->kernel_launches = s->launches;
        out_host->n_rows = 2 * h.adj_nstick + h.adj_nslide;
        out_host->n_dof = h.adj_nbodies * (s->p.rotations ? 3 : 2);
        out_host->diverged = h.adj_diverged;
    }
    return h.adj_converged ? CD_OK : CD_ERR_NOT_CONVERGED;
}

// Checkpoint sections, each 256-byte aligned: pos, vel, omega, theta (if
// any), wall planes (6 per packing), contact count, contact keys and
// impulses of the current set (the warm start of the next step).
struct CkptLayout {
    size_t pos, vel, omega, theta, walls, pk, nc, pairs, P, total;
};

static CkptLayout ckpt_layout(const cd_system* s)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t n = (size_t)s->n, D = (size_t)s->p.dim, cap = (size_t)s->p.max_contacts;
    const size_t rot = (D == 2) ? 1 : 3;
    CkptLayout L;
    size_t o = 0;
    L.pos = o; o += al(n * D * 8);
    L.vel = o; o += al(n * D * 8);
    L.omega = o; o += al(n * rot * 8);
    L.theta = o; o += s->theta ? al(n * 8) : 0;
    L.walls = o; o += al((size_t)s->g.npk * 6 * 8);
    L.pk = o; o += al((size_t)s->g.npk * sizeof(CdPack));   // wall velocities of force-controlled walls
    L.nc = o; o += 256;
    L.pairs = o; o += al(cap * sizeof(int2));
    L.P = o; o += al(cap * (size_t)s->pw * 8);
    L.total = o;
    return L;
}

extern "C" cd_status cd_checkpoint_size(const cd_system* s, size_t* bytes)
{
    if (!s || !bytes) return CD_ERR_INVALID_ARG;
    *bytes = ckpt_layout(s).total;
    return CD_OK;
}

static cd_status ckpt_copy(cd_system* s, void* buf, size_t bytes, bool save)
{
    cd_status st = need_ready(s);
    if (st != CD_OK) return st;
    const CkptLayout L = ckpt_layout(s);
    if (!buf || bytes < L.total) return fail(s, CD_ERR_INVALID_ARG, "checkpoint buffer missing or smaller than cd_checkpoint_size()");
    if (((uintptr_t)buf & 255) != 0) return fail(s, CD_ERR_INVALID_ARG, "checkpoint buffer must be 256-byte aligned");
    char* b = (char*)buf;
    const size_t n = (size_t)s->n, D = (size_t)s->p.dim, cap = (size_t)s->p.max_contacts;
    const size_t rot = (D == 2) ? 1 : 3;
    struct Sec { void* dev; size_t off, len; } sec[] = {
        {s->pos, L.pos, n * D * 8},
        {s->vel, L.vel, n * D * 8},
        {s->omega, L.omega, n * rot * 8},
        {s->theta, L.theta, s->theta ? n * 8 : 0},
        {s->w.pk_wall_pos, L.walls, (size_t)s->g.npk * 6 * 8},
        {s->w.pk, L.pk, (size_t)s->g.npk * sizeof(CdPack)},
        {&s->w.ctrl->nc, L.nc, sizeof(int)},
        {s->w.pairs, L.pairs, cap * sizeof(int2)},
        {s->w.Pk, L.P, cap * (size_t)s->pw * 8},
    };
    for (const Sec& q : sec) {
        if (q.len == 0) continue;
        if (save) CD_CUDA(s, cudaMemcpyAsync(b + q.off, q.dev, q.len, cudaMemcpyDeviceToDevice, s->stream));
        else CD_CUDA(s, cudaMemcpyAsync(q.dev, b + q.off, q.len, cudaMemcpyDeviceToDevice, s->stream));
    }
    if (!save) {
        // the loaded set's per-particle offsets are not kept: the next warm
        // start searches the whole set
        CD_CUDA(s, cudaMemsetAsync(&s->w.ctrl->prev_offsets, 0, sizeof(int), s->stream));
        s->has_contacts = 1;
        s->tape_head = 0;
        s->tape_count = 0;
        if (s->p.tape_steps > 0) CD_CUDA(s, cd_launch_set_tape_slot(s->w, 0, s->stream, &s->launches));
    }
    return CD_OK;
}

extern "C" cd_status cd_save_checkpoint(cd_system* s, void* dev_buf, size_t bytes)
{
    return ckpt_copy(s, dev_buf, bytes, true);
}

extern "C" cd_status cd_load_checkpoint(cd_system* s, const void* dev_buf, size_t bytes)
{
    return ckpt_copy(s, const_cast<void*>(dev_buf), bytes, false);
}

// ---------------------------------------------------------------------------
// Self-check of the bounded waits
// ---------------------------------------------------------------------------
__global__ void k_barrier_withheld(CdCtrl* ctrl, int withheld)
{
    if ((int)blockIdx.x == withheld) return;   // this block never arrives
    unsigned long long epoch = 0;
    cd_grid_sync(ctrl, gridDim.x, epoch);
}

extern "C" cd_status cd_selfcheck_wait_bound(void* dev_scratch, size_t bytes, void* cuda_stream,
                                             double* elapsed_ms_host)
{
    static_assert(sizeof(CdCtrl) <= 1024, "control block larger than the self-check scratch");
    if (!dev_scratch || bytes < 1024) return fail(nullptr, CD_ERR_INVALID_ARG, "dev_scratch must hold at least 1024 bytes");
    if (((uintptr_t)dev_scratch & 255) != 0) return fail(nullptr, CD_ERR_INVALID_ARG, "dev_scratch must be 256-byte aligned");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
    if (!coop) return fail(nullptr, CD_ERR_CUDA, "device lacks cooperative launch");
    CdCtrl* ctrl = (CdCtrl*)dev_scratch;
    if ((e = cudaMemsetAsync(ctrl, 0, sizeof(CdCtrl), st)) != cudaSuccess) return cuda_fail(nullptr, e, "memset");
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaEventCreate");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(nullptr, e, "cudaEventCreate"); }
    int withheld = sms - 1;
    void* args[] = {&ctrl, &withheld};
    cudaEventRecord(e0, st);
    e = cudaLaunchCooperativeKernel((const void*)k_barrier_withheld, dim3(sms), dim3(32), args, 0, st);
    cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "withheld barrier");
    int err = 0;
    if ((e = cudaMemcpy(&err, &ctrl->error, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(nullptr, e, "reading the flag");
    if (elapsed_ms_host) *elapsed_ms_host = (double)ms;
    if (err != CDE_TIMEOUT) return fail(nullptr, CD_ERR_STATE, "the withheld barrier did not report a timeout");
    return CD_OK;
}

extern "C" void cd_destroy_system(cd_system* s)
{
    if (!s) return;
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
    delete s;
}

extern "C" const char* cd_last_error(const cd_system* s)
{
    return s ? s->err.c_str() : g_create_err.c_str();
}
