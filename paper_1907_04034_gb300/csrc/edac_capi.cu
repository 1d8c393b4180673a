// C ABI of the EDAC SPH library (declared in include/edac.h): parameter validation,
// workspace layout, step orchestration (eager or one CUDA graph per step, replayed),
// uploads and canonical (ascending-id) read-back.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "edac.h"
#include "edac_internal.cuh"

static_assert(edac::T_DIR == EDAC_TANGENT_DIRECTIONS, "tangent directions of header and kernels");
static_assert(edac::IN_MODES == EDAC_INLET_MODES && edac::IN_PULSE == EDAC_INLET_PULSE &&
                  edac::IN_RAMP == EDAC_INLET_RAMP && edac::IN_VORTEX == EDAC_INLET_VORTEX &&
                  edac::PROBE_MAX == EDAC_MAX_PROBES,
              "inlet kinds and probe limit of the header and the kernels agree");
static_assert(edac::OUT_HYBRID == EDAC_OUTLET_HYBRID && edac::OUT_DONOTHING == EDAC_OUTLET_DONOTHING &&
                  edac::OUT_MOD_DONOTHING == EDAC_OUTLET_MOD_DONOTHING &&
                  edac::OUT_CHARACTERISTIC == EDAC_OUTLET_CHARACTERISTIC &&
                  edac::OUT_MIRROR == EDAC_OUTLET_MIRROR,
              "outlet kinds of the header and the kernels agree");
static_assert(edac::EV_DELETE == EDAC_EVENT_DELETE && edac::EV_TO_OUTLET == EDAC_EVENT_TO_OUTLET &&
                  edac::EV_SPAWN == EDAC_EVENT_SPAWN,
              "event kinds of the header and the kernels agree");
static_assert((int)edac::FLUID == (int)EDAC_FLUID && (int)edac::INLET == (int)EDAC_INLET &&
                  (int)edac::OUTLET == (int)EDAC_OUTLET && (int)edac::WALL == (int)EDAC_WALL &&
                  (int)edac::SLIPWALL == (int)EDAC_SLIPWALL,
              "particle tags of the header and the kernels agree");

using namespace edac;

struct EventPair {
    cudaEvent_t a, b;
};

struct edac_ctx {
    edac_params P;
    Dev d;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int mixed = 0;
    bool loaded = false;   // particles uploaded
    bool failed = false;   // device error seen
    bool graph_ok = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_step = 0;
    long long launches = 0;
    bool prof_on[EDAC_NUM_KERNELS] = {};
    std::vector<EventPair> prof_ev[EDAC_NUM_KERNELS];
    size_t prof_used[EDAC_NUM_KERNELS] = {};
    double prof_ms[EDAC_NUM_KERNELS] = {};
    long long prof_launches[EDAC_NUM_KERNELS] = {};
    std::string err;
    void *tws = nullptr;        // tangent workspace (edac_tangent_enable)
    size_t tws_bytes = 0;
    long long tangent_steps = 0;
};

namespace {

// Last error of calls made without a context (parameter checks), per host thread.
thread_local std::string g_err = "NULL context";

edac_status fail(edac_ctx *c, edac_status st, const std::string &msg)
{
    if (c) c->err = msg;
    else g_err = msg;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, EDAC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool is_fin(double v) { return std::isfinite(v); }

// ---------------------------------------------------------------- parameters -> device
edac_status make_geo(const edac_params &P, Geo &g, std::string &why)
{
    const double h = P.hdx * P.dx;
    const double rc = 3.0 * (P.hdx * P.dx);
    g.x_min = P.x_min; g.x_max = P.x_max; g.y_min = P.y_min; g.y_max = P.y_max;
    g.Lx = P.x_max - P.x_min;
    g.Ly = P.y_max - P.y_min;
    g.hLx = 0.5 * g.Lx;
    g.hLy = 0.5 * g.Ly;
    g.px = P.periodic_x ? 1 : 0;
    g.py = P.periodic_y ? 1 : 0;
    // cells a little wider than 3h: rounding of the cell index can then never put two
    // particles closer than 3h more than one cell apart
    const double s_min = rc * (1.0 + 1e-9);
    double nxd = std::floor(g.Lx / s_min), nyd = std::floor(g.Ly / s_min);
    if (nxd < 1) nxd = 1;
    if (nyd < 1) nyd = 1;
    if (nxd * nyd > 2.0e8) { why = "cell grid too large (> 2e8 cells)"; return EDAC_E_INVALID; }
    g.nx = (int)nxd;
    g.ny = (int)nyd;
    if ((g.px && g.nx < 3) || (g.py && g.ny < 3)) {
        why = "a periodic axis needs a box at least 3 support radii (9h) long";
        return EDAC_E_INVALID;
    }
    g.ncells = g.nx * g.ny;
    g.sx = g.Lx / g.nx;
    g.sy = g.Ly / g.ny;
    g.inv_sx = 1.0 / g.sx;
    g.inv_sy = 1.0 / g.sy;
    g.sxf = (float)g.sx;
    g.syf = (float)g.sy;
    g.rc2 = rc * rc;
    g.rc2_lo = (float)(g.rc2 * (1.0 - 4e-5));
    g.rc2_hi = (float)(g.rc2 * (1.0 + 4e-5));
    (void)h;
    return EDAC_OK;
}

void make_phys(const edac_params &P, Phys &ph)
{
    const double h = P.hdx * P.dx;
    ph.h = h;
    ph.inv_h = 1.0 / h;
    ph.a2 = 7.0 / (478.0 * M_PI * h * h);
    ph.a2h = ph.a2 / h;
    ph.rho0 = P.rho0;
    ph.cs = P.cs;
    ph.c2 = P.cs * P.cs;
    ph.nu = P.nu;
    ph.nu_e = P.alpha * h * P.cs / 8.0;  // Eq. (edac-nu)
    ph.eh2 = P.eta_reg * h * h;
    ph.pb = P.pb;
    ph.gx = P.gx;
    ph.gy = P.gy;
    ph.dt = P.dt;
    ph.U = P.U;
    ph.inv_2rc = 1.0 / (2.0 * P.rho0 * P.cs);
    ph.inv_navg = 1.0 / 6.0;
    ph.inv_hf = (float)ph.inv_h;
    ph.a2f = (float)ph.a2;
    ph.a2hf = (float)ph.a2h;
    ph.c2f = (float)ph.c2;
    ph.nuf = (float)ph.nu;
    ph.nuef = (float)ph.nu_e;
    ph.eh2f = (float)ph.eh2;
    ph.w0f = (float)(ph.a2 * 66.0);  // W(0) = alpha_2 w(0), w(0) = 3^5 - 6 2^5 + 15
    ph.gxf = (float)P.gx;
    ph.gyf = (float)P.gy;
    ph.pbf = (float)P.pb;
    ph.inv_2rcf = (float)ph.inv_2rc;
    ph.use_pavg = P.use_pavg ? 1 : 0;
    ph.has_inlet = 0;
    ph.n_modes = 0;
    ph.x_in = 0; ph.L_in = 0; ph.in_y0 = 0; ph.in_H = 1;
    for (int k = 0; k < MAX_MODES; ++k) ph.modes[k] = 0.0;
    ph.has_outlet = 0;
    ph.outlet_kind = OUT_HYBRID;
    ph.moc_u_ref = P.U;
    ph.moc_p_ref = 0.0;
    ph.in_kind = IN_MODES;
    for (int k = 0; k < 4; ++k) ph.in_prm[k] = 0.0;
    ph.n_avg = 6;
    ph.x_out = 0; ph.L_out = 0;
    const double q = 0.5 * P.rho0 * P.U * P.U;
    ph.I_thr = q * q / (2.0 * P.rho0 * P.cs);  // Eq. (acouinten)
    ph.wall_slip[0] = 0; ph.wall_slip[1] = 1;
    ph.wall_drag[0] = 1; ph.wall_drag[1] = 0;
    ph.wall_u[0] = ph.wall_u[1] = ph.wall_v[0] = ph.wall_v[1] = 0.0;
}

edac_status check_params(const edac_params *P, std::string &why)
{
    if (!P) { why = "params is NULL"; return EDAC_E_INVALID; }
    const double vals[] = {P->x_min, P->x_max, P->y_min, P->y_max, P->dx, P->hdx, P->rho0, P->U,
                           P->nu, P->cs, P->alpha, P->pb, P->eta_reg, P->gx, P->gy, P->dt};
    for (double v : vals)
        if (!is_fin(v)) { why = "non-finite parameter"; return EDAC_E_INVALID; }
    if (!(P->x_max > P->x_min && P->y_max > P->y_min)) { why = "empty domain box"; return EDAC_E_INVALID; }
    if (!(P->dx > 0 && P->hdx > 0 && P->rho0 > 0 && P->cs > 0 && P->dt > 0 && P->eta_reg > 0)) {
        why = "dx, hdx, rho0, cs, dt and eta_reg must be > 0";
        return EDAC_E_INVALID;
    }
    if (P->nu < 0 || P->alpha < 0) { why = "nu and alpha must be >= 0"; return EDAC_E_INVALID; }
    if (P->precision != EDAC_FP64 && P->precision != EDAC_MIXED) {
        why = "precision must be EDAC_FP64 or EDAC_MIXED";
        return EDAC_E_INVALID;
    }
    if (P->capacity < 1 || P->capacity >= (1 << 28)) { why = "capacity out of range [1, 2^28)"; return EDAC_E_INVALID; }
    if (P->max_history < 1 || P->max_history > (1 << 26)) { why = "max_history out of range"; return EDAC_E_INVALID; }
    return EDAC_OK;
}

// Carve the workspace (base may be null: size computation only).
size_t layout(Dev &d, const Geo &g, int cap, int max_history, int mixed, char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? (void *)(base + off) : nullptr;
        off += bytes;
        return p;
    };
    const size_t C = (size_t)cap;
#define DARR(field, T, count) d.field = (T *)take(sizeof(T) * (count))
    DARR(cnt, Counters, 1);
    DARR(x, double, C); DARR(y, double, C); DARR(u, double, C); DARR(v, double, C);
    DARR(ut, double, C); DARR(vt, double, C); DARR(p, double, C); DARR(m, double, C);
    DARR(x0, double, C); DARR(y0, double, C); DARR(u0, double, C); DARR(v0, double, C);
    DARR(p0, double, C);
    DARR(au, double, C); DARR(av, double, C); DARR(ap, double, C); DARR(abu, double, C);
    DARR(abv, double, C); DARR(fx, double, C); DARR(fy, double, C); DARR(rho, double, C);
    DARR(vol, double, C);
    DARR(nnb, int, C);
    DARR(tag, uint8_t, C);
    DARR(id, unsigned long long, C);
    DARR(ring, double, C * NAVG_MAX * 3);
    DARR(rpos, uint8_t, C);
    DARR(ubar, double, C); DARR(vbar, double, C); DARR(pbar, double, C); DARR(J2, double, C);
    DARR(J2p, double, C); DARR(advp, double, C);
    DARR(redp, uint8_t, C);
    DARR(org_x, double, (size_t)g.nx);
    DARR(org_y, double, (size_t)g.ny);
    DARR(cell_count, int, (size_t)g.ncells);
    DARR(cell_start, int, (size_t)g.ncells + 1);
    DARR(slot_cell, int, C);
    DARR(within, int, C);
    DARR(order, int, C);
    DARR(order_raw, int, C);
    DARR(scan_part, int, (size_t)(g.ncells + 4095) / 4096 + 1);
    DARR(cellk, int, C);
    DARR(stag, uint8_t, C);
    DARR(P, float4, C);
    DARR(XY, double2, C);
    DARR(AUX, double2, C);
    DARR(snnb, int, C);
    if (mixed) {
        DARR(Bf, float4, C);
        DARR(Qf, float4, C);
        DARR(nbm, uint4, 2 * C);
        d.UV = d.DUV = d.PV = d.RM = nullptr;
        d.Ms = nullptr;
        d.GS = nullptr;
    } else {
        DARR(UV, double2, C); DARR(DUV, double2, C); DARR(PV, double2, C); DARR(RM, double2, C);
        DARR(GS, double, 3 * C);
        DARR(Ms, double, C);
        d.Bf = d.Qf = nullptr;
        d.nbm = nullptr;
    }
    DARR(bnd, int, C);
    DARR(free_stack, int, C);
    DARR(ev_spawn_key, unsigned long long, LIST_MAX); DARR(ev_spawn_slot, int, LIST_MAX);
    DARR(ev_del_key, unsigned long long, LIST_MAX); DARR(ev_del_slot, int, LIST_MAX);
    DARR(ev_out_key, unsigned long long, LIST_MAX); DARR(ev_out_m, double, LIST_MAX);
    DARR(drag_slots, int, C);
    DARR(spawn_map, int2, LIST_MAX);
    DARR(scratch_m, double, LIST_MAX);
    DARR(hist, double, (size_t)max_history * 8);
    DARR(probe_part, double, (size_t)PROBE_BLK * PROBE_MAX * 8);
    DARR(probe_out, double, (size_t)PROBE_MAX * 4);
#undef DARR
    return (off + 255) & ~(size_t)255;
}

// ------------------------------------------------------------------ step orchestration
struct Group {
    edac_ctx *c;
    int k;
    bool on;
    size_t idx;
    Group(edac_ctx *ctx, int kernel) : c(ctx), k(kernel), on(ctx->prof_on[kernel]), idx(0)
    {
        if (!on) return;
        auto &v = c->prof_ev[k];
        idx = c->prof_used[k]++;
        if (idx >= v.size()) {
            EventPair e;
            cudaEventCreate(&e.a);
            cudaEventCreate(&e.b);
            v.push_back(e);
        }
        cudaEventRecord(v[idx].a, c->stream);
    }
    ~Group()
    {
        if (on) cudaEventRecord(c->prof_ev[k][idx].b, c->stream);
    }
};

int issue_eval(edac_ctx *c, int end_of_step, int counted = 0)
{
    int n = 0;
    { Group g(c, EDAC_K_REBUILD); n += launch_rebuild(c->d, c->stream, c->mixed, counted); }
    { Group g(c, EDAC_K_PASS_A); n += launch_pass_a(c->d, c->stream, c->mixed); }
    { Group g(c, EDAC_K_BOUNDARY); n += launch_boundary(c->d, c->stream, c->mixed, end_of_step); }
    { Group g(c, EDAC_K_PASS_B); n += launch_pass_b(c->d, c->stream, c->mixed); }
    return n;
}

int issue_step(edac_ctx *c)
{
    int n = 0;
    // each stage also counts the particles into the cells of the evaluation that follows it
    { Group g(c, EDAC_K_STAGE); n += launch_stage(c->d, c->stream, c->mixed, 0, 1); }
    n += issue_eval(c, 0, 1);
    { Group g(c, EDAC_K_STAGE); n += launch_stage(c->d, c->stream, c->mixed, 1, 1); }
    n += issue_eval(c, 1, 1);
    { Group g(c, EDAC_K_RECYCLE); n += launch_recycle(c->d, c->stream); }
    return n;
}

bool any_profiling(const edac_ctx *c)
{
    for (int k = 0; k < EDAC_NUM_KERNELS; ++k)
        if (c->prof_on[k]) return true;
    return false;
}

void drop_graph(edac_ctx *c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->graph_ok = false;
}

// Sticky device error word -> status.
edac_status check_device(edac_ctx *ctx)
{
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h.err) {
        ctx->failed = true;
        if (h.err & ERR_NONFINITE) return fail(ctx, EDAC_E_NONFINITE, "non-finite value in the particle fields");
        if (h.err & ERR_DOMAIN) {
            char buf[192];
            snprintf(buf, sizeof buf, "a particle left the domain box (id %llu, tag %d, at x = %.9g, "
                     "y = %.9g, in step %d)", h.err_id, h.err_tag, h.err_x, h.err_y, h.step + 1);
            return fail(ctx, EDAC_E_DOMAIN, buf);
        }
        if (h.err & (ERR_CAPACITY | ERR_LIST)) return fail(ctx, EDAC_E_CAPACITY, "particle capacity or event list exceeded");
        if (h.err & ERR_TIMEOUT) return fail(ctx, EDAC_E_TIMEOUT, "a device wait timed out");
        return fail(ctx, EDAC_E_STATE, "device error");
    }
    return EDAC_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

edac_status edac_workspace_bytes(const edac_params *params, size_t *bytes)
{
    std::string why;
    edac_status st = check_params(params, why);
    if (st) return fail(nullptr, st, why);
    if (!bytes) return fail(nullptr, EDAC_E_INVALID, "bytes is NULL");
    Geo g;
    st = make_geo(*params, g, why);
    if (st) return fail(nullptr, st, why);
    Dev d;
    *bytes = layout(d, g, params->capacity, params->max_history, params->precision == EDAC_MIXED, nullptr);
    return EDAC_OK;
}

edac_status edac_create(const edac_params *params, void *d_workspace, size_t bytes, edac_ctx **out)
{
    if (!out) return fail(nullptr, EDAC_E_INVALID, "out is NULL");
    *out = nullptr;
    std::string why;
    edac_status st = check_params(params, why);
    if (st) return fail(nullptr, st, why);
    Geo g;
    st = make_geo(*params, g, why);
    if (st) return fail(nullptr, st, why);
    Dev probe;
    const size_t need = layout(probe, g, params->capacity, params->max_history,
                               params->precision == EDAC_MIXED, nullptr);
    if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255u))
        return fail(nullptr, EDAC_E_INVALID, "workspace missing, too small or not 256-byte aligned");
    edac_ctx *c = new edac_ctx();
    c->P = *params;
    c->mixed = params->precision == EDAC_MIXED;
    c->stream = (cudaStream_t)params->cuda_stream;
    c->ws = (char *)d_workspace;
    c->ws_bytes = bytes;
    c->d.g = g;
    make_phys(*params, c->d.ph);
    c->d.cap = params->capacity;
    c->d.mixed = c->mixed;
    c->d.max_history = params->max_history;
    c->d.tile_tx = 11;
    c->d.tile_tpb = 160;
    layout(c->d, g, params->capacity, params->max_history, c->mixed, c->ws);
    *out = c;
    return EDAC_OK;
}

edac_status edac_set_inlet(edac_ctx *ctx, double x_in, int n_layers, int n_modes,
                           const double *h_modes, double y0, double H)
{
    if (!ctx) return EDAC_E_INVALID;
    if (!is_fin(x_in) || n_layers < 1 || n_modes < 0 || n_modes > MAX_MODES || !is_fin(y0) ||
        !(H > 0) || (n_modes > 0 && !h_modes))
        return fail(ctx, EDAC_E_INVALID, "bad inlet arguments");
    Phys &ph = ctx->d.ph;
    ph.has_inlet = 1;
    ph.x_in = x_in;
    ph.L_in = (double)n_layers * ctx->P.dx;
    ph.n_modes = n_modes;
    for (int k = 0; k < MAX_MODES; ++k) ph.modes[k] = k < n_modes ? h_modes[k] : 0.0;
    for (int k = 0; k < n_modes; ++k)
        if (!is_fin(ph.modes[k])) return fail(ctx, EDAC_E_INVALID, "non-finite inlet mode");
    ph.in_y0 = y0;
    ph.in_H = H;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_set_outlet(edac_ctx *ctx, double x_out, int n_layers, int kind, int n_avg,
                            double i_thresh)
{
    if (!ctx) return EDAC_E_INVALID;
    if (!is_fin(x_out) || n_layers < 1 || kind < EDAC_OUTLET_HYBRID || kind > EDAC_OUTLET_MIRROR ||
        n_avg < 1 || n_avg > NAVG_MAX ||
        !is_fin(i_thresh))
        return fail(ctx, EDAC_E_INVALID, "bad outlet arguments");
    Phys &ph = ctx->d.ph;
    ph.has_outlet = 1;
    ph.outlet_kind = kind;
    ph.x_out = x_out;
    ph.L_out = (double)n_layers * ctx->P.dx;
    ph.n_avg = n_avg;
    ph.inv_navg = 1.0 / (double)n_avg;
    if (i_thresh >= 0) ph.I_thr = i_thresh;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_set_inlet_transient(edac_ctx *ctx, int kind, int nprm, const double *prm)
{
    if (!ctx) return EDAC_E_INVALID;
    static const int need[4] = {0, 4, 1, 4};
    if (kind < EDAC_INLET_MODES || kind > EDAC_INLET_VORTEX || nprm != need[kind] || (nprm > 0 && !prm))
        return fail(ctx, EDAC_E_INVALID, "bad inlet kind or parameter count");
    for (int k = 0; k < nprm; ++k)
        if (!is_fin(prm[k])) return fail(ctx, EDAC_E_INVALID, "non-finite inlet parameter");
    if ((kind == EDAC_INLET_PULSE && !(prm[3] > 0 && prm[2] > prm[1])) ||
        (kind == EDAC_INLET_RAMP && !(prm[0] > 0)) || (kind == EDAC_INLET_VORTEX && !(prm[1] > 0)))
        return fail(ctx, EDAC_E_INVALID, "inlet parameters out of range");
    Phys &ph = ctx->d.ph;
    ph.in_kind = kind;
    for (int k = 0; k < 4; ++k) ph.in_prm[k] = k < nprm ? prm[k] : 0.0;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_set_outlet_reference(edac_ctx *ctx, double u_ref, double p_ref)
{
    if (!ctx) return EDAC_E_INVALID;
    if (!is_fin(u_ref) || !is_fin(p_ref)) return fail(ctx, EDAC_E_INVALID, "non-finite reference");
    ctx->d.ph.moc_u_ref = u_ref;
    ctx->d.ph.moc_p_ref = p_ref;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_probe(edac_ctx *ctx, int n, const double *h_x, const double *h_y, double *h_out)
{
    if (!ctx) return EDAC_E_INVALID;
    if (n < 1 || n > EDAC_MAX_PROBES || !h_x || !h_y || !h_out)
        return fail(ctx, EDAC_E_INVALID, "1 <= n <= EDAC_MAX_PROBES points and non-NULL arrays");
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    edac_status st = check_device(ctx);
    if (st) return st;
    ProbePts q;
    q.n = n;
    for (int i = 0; i < PROBE_MAX; ++i) {
        q.x[i] = i < n ? h_x[i] : 0.0;
        q.y[i] = i < n ? h_y[i] : 0.0;
        if (i < n && (!is_fin(q.x[i]) || !is_fin(q.y[i]))) return fail(ctx, EDAC_E_INVALID, "non-finite probe point");
    }
    ctx->launches += launch_probe(ctx->d, ctx->stream, q);
    CK(cudaMemcpyAsync(h_out, ctx->d.probe_out, sizeof(double) * 4 * (size_t)n, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaGetLastError());
    return EDAC_OK;
}

edac_status edac_set_wall(edac_ctx *ctx, int tag, int slip, double uw, double vw, int count_in_drag)
{
    if (!ctx) return EDAC_E_INVALID;
    if ((tag != EDAC_WALL && tag != EDAC_SLIPWALL) || !is_fin(uw) || !is_fin(vw) ||
        count_in_drag < 0 || count_in_drag > 2)
        return fail(ctx, EDAC_E_INVALID, "bad wall arguments");
    if (ctx->loaded) return fail(ctx, EDAC_E_STATE, "set walls before edac_set_particles");
    const int w = tag == EDAC_WALL ? 0 : 1;
    Phys &ph = ctx->d.ph;
    ph.wall_slip[w] = slip ? 1 : 0;
    ph.wall_u[w] = uw;
    ph.wall_v[w] = vw;
    ph.wall_drag[w] = count_in_drag;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_set_particles(edac_ctx *ctx, int n, const double *h_x, const double *h_y,
                               const double *h_u, const double *h_v, const double *h_p,
                               const double *h_m, const uint8_t *h_tag, const uint64_t *h_id)
{
    if (!ctx) return EDAC_E_INVALID;
    const int cap = ctx->d.cap;
    if (n < 0 || n > cap) return fail(ctx, EDAC_E_INVALID, "n out of range [0, capacity]");
    if (n > 0 && (!h_x || !h_y || !h_u || !h_v || !h_p || !h_m || !h_tag || !h_id))
        return fail(ctx, EDAC_E_INVALID, "NULL input array");
    const Geo &g = ctx->d.g;
    Dev &d = ctx->d;
    // Validation, in chunks on host threads (the inputs are ~50 bytes a particle); the first
    // failing particle in input order decides the error, as a sequential scan would.  Each
    // chunk also lists its particles counted in the drag (ascending).
    const int nthreads = n < (1 << 16) ? 1 : 16;
    const int chunk = (n + nthreads - 1) / nthreads;
    std::vector<int> bad_at(nthreads, -1);
    std::vector<edac_status> bad_st(nthreads, EDAC_OK);
    std::vector<const char *> bad_msg(nthreads, nullptr);
    std::vector<std::vector<int>> drag_part(nthreads);
    auto validate = [&](int c) {
        const int i0 = c * chunk, i1 = std::min(n, i0 + chunk);
        for (int i = i0; i < i1; ++i) {
            const char *why = nullptr;
            edac_status st = EDAC_E_INVALID;
            if (h_tag[i] > EDAC_SLIPWALL) why = "tag out of range";
            else if (!(is_fin(h_x[i]) && is_fin(h_y[i]) && is_fin(h_u[i]) && is_fin(h_v[i]) &&
                       is_fin(h_p[i]) && is_fin(h_m[i])))
                why = "non-finite input value";
            else if (!(h_m[i] > 0)) why = "masses must be > 0";
            else if (!(h_x[i] >= g.x_min && h_x[i] < g.x_max && h_y[i] >= g.y_min && h_y[i] < g.y_max)) {
                why = "particle outside the domain box";
                st = EDAC_E_DOMAIN;
            } else if (h_tag[i] == EDAC_INLET && !d.ph.has_inlet)
                why = "inlet particles without edac_set_inlet";
            else if (h_tag[i] == EDAC_OUTLET && !d.ph.has_outlet)
                why = "outlet particles without edac_set_outlet";
            if (why) {
                bad_at[c] = i;
                bad_st[c] = st;
                bad_msg[c] = why;
                return;
            }
            const int t = h_tag[i];
            if (drag_mode(d.ph, t))
                drag_part[c].push_back(i);
        }
    };
    {
        std::vector<std::thread> th;
        for (int c = 1; c < nthreads; ++c) {
            try {
                th.emplace_back(validate, c);
            } catch (...) {  // no thread to be had: this thread does the chunk
                validate(c);
            }
        }
        validate(0);
        for (auto &t : th) t.join();
    }
    for (int c = 0; c < nthreads; ++c)
        if (bad_at[c] >= 0) return fail(ctx, bad_st[c], bad_msg[c]);
    // duplicate ids: a strictly increasing sequence (the usual input, and what edac_read_state
    // returns) has none; anything else is sorted and scanned
    bool increasing = true;
    uint64_t max_id = n ? h_id[0] : 0;
    for (int i = 1; i < n; ++i) {
        increasing = increasing && h_id[i - 1] < h_id[i];
        max_id = h_id[i] > max_id ? h_id[i] : max_id;
    }
    if (!increasing) {
        std::vector<uint64_t> ids(h_id, h_id + n);
        std::sort(ids.begin(), ids.end());
        if (std::adjacent_find(ids.begin(), ids.end()) != ids.end())
            return fail(ctx, EDAC_E_INVALID, "duplicate particle ids");
    }
    cudaStream_t s = ctx->stream;
    CK(cudaMemsetAsync(ctx->ws, 0, ctx->ws_bytes, s));
    ctx->launches += launch_origins(ctx->d, s);
    std::vector<int> drag;
    for (auto &p : drag_part) drag.insert(drag.end(), p.begin(), p.end());
    Counters hc;
    std::memset(&hc, 0, sizeof(hc));
    hc.n_alive = n;
    hc.free_top = cap - n;
    hc.n_drag = (int)drag.size();
    hc.next_id = n ? (unsigned long long)max_id + 1ull : 0ull;
    if (n > 0) {
        CK(cudaMemcpyAsync(d.x, h_x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.y, h_y, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.u, h_u, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.v, h_v, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.p, h_p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.m, h_m, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d.id, h_id, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s));
    }
    if (n > 0) CK(cudaMemcpyAsync(d.tag, h_tag, n, cudaMemcpyHostToDevice, s));
    if (cap - n > 0) {
        CK(cudaMemsetAsync(d.tag + n, TAG_DEAD, cap - n, s));
        ctx->launches += launch_free_stack(d, s, n);
    }
    if (!drag.empty())
        CK(cudaMemcpyAsync(d.drag_slots, drag.data(), sizeof(int) * drag.size(),
                           cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d.cnt, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    ctx->launches += launch_init(d, s);
    ctx->launches += issue_eval(ctx, 0);
    CK(cudaGetLastError());
    // the host vectors above must outlive the asynchronous copies
    CK(cudaStreamSynchronize(s));
    ctx->loaded = true;
    ctx->failed = false;
    return check_device(ctx);
}

edac_status edac_step(edac_ctx *ctx, int nsteps)
{
    if (!ctx) return EDAC_E_INVALID;
    if (nsteps < 0) return fail(ctx, EDAC_E_INVALID, "nsteps < 0");
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles: call edac_set_particles first");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error: re-initialise with edac_set_particles");
    if (nsteps == 0) return EDAC_OK;
    const bool graphs = ctx->P.use_graphs && ctx->stream != nullptr && !any_profiling(ctx);
    if (graphs) {
        if (!ctx->graph_ok) {
            drop_graph(ctx);
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            const int k = issue_step(ctx);
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
            if (e != cudaSuccess) return fail(ctx, EDAC_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            ctx->graph = gr;
            CK(cudaGraphInstantiate(&ctx->exec, gr, 0));
            ctx->kernels_per_step = k;
            ctx->graph_ok = true;
        }
        for (int i = 0; i < nsteps; ++i) CK(cudaGraphLaunch(ctx->exec, ctx->stream));
        ctx->launches += (long long)ctx->kernels_per_step * nsteps;
    } else {
        for (int i = 0; i < nsteps; ++i) ctx->launches += issue_step(ctx);
    }
    CK(cudaGetLastError());
    return EDAC_OK;
}

edac_status edac_evaluate(edac_ctx *ctx)
{
    if (!ctx) return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    ctx->launches += issue_eval(ctx, 0);
    CK(cudaGetLastError());
    return EDAC_OK;
}

edac_status edac_get_count(edac_ctx *ctx, int *n_active)
{
    if (!ctx || !n_active) return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *n_active = h.n_alive;
    return check_device(ctx);
}

edac_status edac_read_state(edac_ctx *ctx, int cap, uint64_t *h_id, uint8_t *h_tag, int nfields,
                            const int *field_ids, double *const *h_out, int *n)
{
    if (!ctx || !n || nfields < 0 || (nfields > 0 && (!field_ids || !h_out)))
        return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    for (int f = 0; f < nfields; ++f)
        if (field_ids[f] < 0 || field_ids[f] >= EDAC_NUM_FIELDS || !h_out[f])
            return fail(ctx, EDAC_E_INVALID, "bad field id or output pointer");
    edac_status st = check_device(ctx);
    if (st) return st;
    const Dev &d = ctx->d;
    const int C = d.cap;
    cudaStream_t s = ctx->stream;
    // field id -> device column and its type (0 double, 1 int, 2 byte)
    std::vector<const void *> src(nfields);
    std::vector<int> kind(nfields, 0);
    for (int f = 0; f < nfields; ++f) {
        switch (field_ids[f]) {
            case EDAC_F_X: src[f] = d.x; break;
            case EDAC_F_Y: src[f] = d.y; break;
            case EDAC_F_U: src[f] = d.u; break;
            case EDAC_F_V: src[f] = d.v; break;
            case EDAC_F_UT: src[f] = d.ut; break;
            case EDAC_F_VT: src[f] = d.vt; break;
            case EDAC_F_P: src[f] = d.p; break;
            case EDAC_F_M: src[f] = d.m; break;
            case EDAC_F_RHO: src[f] = d.rho; break;
            case EDAC_F_VOL: src[f] = d.vol; break;
            case EDAC_F_AU: src[f] = d.au; kind[f] = d.mixed ? 3 : 0; break;
            case EDAC_F_AV: src[f] = d.av; kind[f] = d.mixed ? 3 : 0; break;
            case EDAC_F_AP: src[f] = d.ap; kind[f] = d.mixed ? 3 : 0; break;
            case EDAC_F_ABU: src[f] = d.abu; kind[f] = d.mixed ? 3 : 0; break;
            case EDAC_F_ABV: src[f] = d.abv; kind[f] = d.mixed ? 3 : 0; break;
            case EDAC_F_FX: src[f] = d.fx; break;
            case EDAC_F_FY: src[f] = d.fy; break;
            case EDAC_F_UBAR: src[f] = d.ubar; break;
            case EDAC_F_VBAR: src[f] = d.vbar; break;
            case EDAC_F_PBAR: src[f] = d.pbar; break;
            case EDAC_F_J2: src[f] = d.J2; break;
            case EDAC_F_J2P: src[f] = d.J2p; break;
            case EDAC_F_ADVP: src[f] = d.advp; break;
            case EDAC_F_NNB: src[f] = d.nnb; kind[f] = 1; break;
            case EDAC_F_REDP: src[f] = d.redp; kind[f] = 2; break;
            default: src[f] = d.rpos; kind[f] = 2; break;  // EDAC_F_RPOS
        }
    }
    std::vector<uint8_t> tag(C);
    std::vector<unsigned long long> id(C);
    CK(cudaMemcpyAsync(tag.data(), d.tag, C, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(id.data(), d.id, sizeof(unsigned long long) * C, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // live slots in ascending id order.  Slots keep their ids and a recycled slot takes a new,
    // larger id, so the slot order is mostly id order: the slots that continue the increasing
    // run are kept in place, the others (recycled slots) are sorted apart and merged in.
    std::vector<int> run, side;
    run.reserve(C);
    unsigned long long last = 0;
    bool any = false;
    for (int i = 0; i < C; ++i) {
        if (tag[i] == TAG_DEAD) continue;
        if (!any || id[i] > last) {
            run.push_back(i);
            last = id[i];
            any = true;
        } else {
            side.push_back(i);
        }
    }
    auto by_id = [&](int a, int b) { return id[a] < id[b]; };
    std::sort(side.begin(), side.end(), by_id);
    std::vector<int> live(run.size() + side.size());
    std::merge(run.begin(), run.end(), side.begin(), side.end(), live.begin(), by_id);
    const int nl = (int)live.size();
    *n = nl;
    if (nl > cap) return fail(ctx, EDAC_E_INVALID, "output arrays too short");
    if (nl == 0) return EDAC_OK;
    // The columns are permuted on the device and copied straight into the caller's arrays.
    // Scratch: the predictor's base-state arrays, which are dead between steps (every step's
    // predictor writes them before its corrector reads them): y0 holds the order, x0 each
    // permuted column, u0 the permuted tags.
    int *d_live = reinterpret_cast<int *>(d.y0);
    double *d_col = d.x0;
    CK(cudaMemcpyAsync(d_live, live.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
    for (int f = 0; f < nfields; ++f) {
        ctx->launches += launch_permute(s, src[f], kind[f], d_live, nl, d_col);
        CK(cudaMemcpyAsync(h_out[f], d_col, sizeof(double) * nl, cudaMemcpyDeviceToHost, s));
    }
    if (h_id || h_tag) {
        unsigned long long *d_id = reinterpret_cast<unsigned long long *>(d.x0);
        uint8_t *d_tag = reinterpret_cast<uint8_t *>(d.u0);
        ctx->launches += launch_permute_id_tag(d, s, d_live, nl, d_id, d_tag);
        if (h_id) CK(cudaMemcpyAsync(h_id, d_id, sizeof(uint64_t) * nl, cudaMemcpyDeviceToHost, s));
        if (h_tag) CK(cudaMemcpyAsync(h_tag, d_tag, nl, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));  // live must outlive its copy
    return EDAC_OK;
}

edac_status edac_read_history(edac_ctx *ctx, int max_steps, double *h_fx, double *h_fy,
                              double *h_mass_flux, int *h_n_active, int *h_n_spawn,
                              int *h_n_delete, int *h_n_to_outlet, int *nsteps)
{
    if (!ctx || !nsteps || max_steps < 0) return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    edac_status st = check_device(ctx);
    if (st) return st;
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    const int H = ctx->d.max_history;
    std::vector<double> hist((size_t)H * 8);
    CK(cudaMemcpyAsync(hist.data(), ctx->d.hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int avail = std::min(h.hist_len, H);
    const int k = std::min(avail, max_steps);
    for (int r = 0; r < k; ++r) {
        const int stepi = h.step - k + r;
        const double *rec = hist.data() + (size_t)(stepi % H) * 8;
        if (h_fx) h_fx[r] = rec[0];
        if (h_fy) h_fy[r] = rec[1];
        if (h_mass_flux) h_mass_flux[r] = rec[2];
        if (h_n_active) h_n_active[r] = (int)rec[3];
        if (h_n_spawn) h_n_spawn[r] = (int)rec[4];
        if (h_n_delete) h_n_delete[r] = (int)rec[5];
        if (h_n_to_outlet) h_n_to_outlet[r] = (int)rec[6];
    }
    *nsteps = k;
    return EDAC_OK;
}

edac_status edac_events_bytes(int max_events, size_t *bytes)
{
    if (!bytes || max_events < 0) return EDAC_E_INVALID;
    *bytes = sizeof(EventRec) * (size_t)max_events;
    return EDAC_OK;
}

edac_status edac_events_enable(edac_ctx *ctx, void *d_log, size_t bytes)
{
    if (!ctx) return EDAC_E_INVALID;
    if (d_log && (((uintptr_t)d_log & 255u) || bytes < sizeof(EventRec)))
        return fail(ctx, EDAC_E_INVALID, "event log not 256-byte aligned or smaller than one record");
    // kernels already issued keep the previous log: let them finish before it is released
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->d.evlog = static_cast<EventRec *>(d_log);
    ctx->d.ev_cap = d_log ? (int)std::min<size_t>(bytes / sizeof(EventRec), (size_t)INT_MAX) : 0;
    CK(cudaMemsetAsync(&ctx->d.cnt->ev_len, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(&ctx->d.cnt->ev_dropped, 0, sizeof(unsigned long long), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_read_events(edac_ctx *ctx, int cap, int *h_step, int *h_kind, uint64_t *h_id,
                             uint64_t *h_other, int *n, int64_t *n_dropped)
{
    if (!ctx || !n || cap < 0) return EDAC_E_INVALID;
    if (!ctx->d.evlog) return fail(ctx, EDAC_E_STATE, "no event log: call edac_events_enable first");
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *n = h.ev_len;
    if (h.ev_len > cap) return fail(ctx, EDAC_E_INVALID, "cap is below the number of logged events");
    std::vector<EventRec> rec((size_t)std::max(h.ev_len, 1));
    if (h.ev_len > 0)
        CK(cudaMemcpyAsync(rec.data(), ctx->d.evlog, sizeof(EventRec) * (size_t)h.ev_len,
                           cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemsetAsync(&ctx->d.cnt->ev_len, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(&ctx->d.cnt->ev_dropped, 0, sizeof(unsigned long long), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < h.ev_len; ++i) {
        if (h_step) h_step[i] = rec[i].step;
        if (h_kind) h_kind[i] = rec[i].kind;
        if (h_id) h_id[i] = rec[i].id;
        if (h_other) h_other[i] = rec[i].other;
    }
    if (n_dropped) *n_dropped = (int64_t)h.ev_dropped;
    return EDAC_OK;
}

edac_status edac_neighbor_scratch_bytes(edac_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    ctx->launches += launch_rebuild(ctx->d, ctx->stream, ctx->mixed);
    ctx->launches += launch_pass_a(ctx->d, ctx->stream, ctx->mixed);
    CK(cudaGetLastError());
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<int> cntv(std::max(h.n_alive, 1));
    if (h.n_alive > 0)
        CK(cudaMemcpy(cntv.data(), ctx->d.snnb, sizeof(int) * h.n_alive, cudaMemcpyDeviceToHost));
    long long tot = 0;
    for (int k = 0; k < h.n_alive; ++k) tot += cntv[k];
    *bytes = sizeof(long long) * ((size_t)h.n_alive + 1) + sizeof(unsigned long long) * (size_t)tot + 256;
    return EDAC_OK;
}

edac_status edac_read_neighbors(edac_ctx *ctx, void *d_scratch, size_t scratch_bytes, int cap_n,
                                int64_t *h_start, int64_t cap_ids, uint64_t *h_nbr_ids, int *n,
                                int64_t *total)
{
    if (!ctx || !n || !total || !d_scratch || !h_start || (cap_ids > 0 && !h_nbr_ids))
        return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    cudaStream_t s = ctx->stream;
    const Dev &d = ctx->d;
    ctx->launches += launch_rebuild(d, s, ctx->mixed);
    ctx->launches += launch_pass_a(d, s, ctx->mixed);
    CK(cudaGetLastError());
    Counters h;
    CK(cudaMemcpyAsync(&h, d.cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int na = h.n_alive;
    std::vector<int> cntv(std::max(na, 1)), order(std::max(na, 1));
    std::vector<unsigned long long> id(d.cap);
    if (na > 0) {
        CK(cudaMemcpy(cntv.data(), d.snnb, sizeof(int) * na, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(order.data(), d.order, sizeof(int) * na, cudaMemcpyDeviceToHost));
    }
    CK(cudaMemcpy(id.data(), d.id, sizeof(unsigned long long) * d.cap, cudaMemcpyDeviceToHost));
    std::vector<long long> start(na + 1, 0);
    for (int k = 0; k < na; ++k) start[k + 1] = start[k] + cntv[k];
    const long long tot = start[na];
    const size_t need = sizeof(long long) * ((size_t)na + 1) + sizeof(unsigned long long) * (size_t)tot + 256;
    if (scratch_bytes < need) return fail(ctx, EDAC_E_INVALID, "neighbour scratch too small");
    if (cap_n < na || cap_ids < tot) return fail(ctx, EDAC_E_INVALID, "output arrays too short");
    long long *d_start = (long long *)d_scratch;
    unsigned long long *d_ids =
        (unsigned long long *)(((uintptr_t)(d_start + na + 1) + 255) & ~(uintptr_t)255);
    CK(cudaMemcpyAsync(d_start, start.data(), sizeof(long long) * (na + 1), cudaMemcpyHostToDevice, s));
    ctx->launches += launch_neighbor_dump(d, s, ctx->mixed, d_start, d_ids);
    CK(cudaGetLastError());
    std::vector<unsigned long long> ids(std::max<long long>(tot, 1));
    if (tot > 0)
        CK(cudaMemcpyAsync(ids.data(), d_ids, sizeof(unsigned long long) * tot, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // canonical order: particles by ascending id, each list ascending
    std::vector<int> ks(na);
    std::iota(ks.begin(), ks.end(), 0);
    std::sort(ks.begin(), ks.end(), [&](int a, int b) { return id[order[a]] < id[order[b]]; });
    long long pos = 0;
    h_start[0] = 0;
    for (int r = 0; r < na; ++r) {
        const int k = ks[r];
        std::vector<unsigned long long> lst(ids.begin() + start[k], ids.begin() + start[k + 1]);
        std::sort(lst.begin(), lst.end());
        for (auto v : lst) h_nbr_ids[pos++] = v;
        h_start[r + 1] = pos;
    }
    *n = na;
    *total = tot;
    return check_device(ctx);
}

edac_status edac_profile(edac_ctx *ctx, int kernel, int enable)
{
    if (!ctx || kernel < 0 || kernel >= EDAC_NUM_KERNELS) return EDAC_E_INVALID;
    ctx->prof_on[kernel] = enable != 0;
    return EDAC_OK;
}

edac_status edac_read_profile(edac_ctx *ctx, int kernel, double *ms, int64_t *launches, int reset)
{
    if (!ctx || kernel < 0 || kernel >= EDAC_NUM_KERNELS) return EDAC_E_INVALID;
    CK(cudaStreamSynchronize(ctx->stream));
    auto &v = ctx->prof_ev[kernel];
    for (size_t i = 0; i < ctx->prof_used[kernel]; ++i) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, v[i].a, v[i].b));
        ctx->prof_ms[kernel] += t;
        ctx->prof_launches[kernel] += 1;
    }
    ctx->prof_used[kernel] = 0;
    if (ms) *ms = ctx->prof_ms[kernel];
    if (launches) *launches = ctx->prof_launches[kernel];
    if (reset) {
        ctx->prof_ms[kernel] = 0.0;
        ctx->prof_launches[kernel] = 0;
    }
    return EDAC_OK;
}

edac_status edac_launch_count(edac_ctx *ctx, int64_t *count)
{
    if (!ctx || !count) return EDAC_E_INVALID;
    *count = ctx->launches;
    return EDAC_OK;
}

const char *edac_last_error(edac_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

// ------------------------------------------------------------ tangent-linear model
edac_status edac_tangent_workspace_bytes(edac_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return EDAC_E_INVALID;
    *bytes = tangent_bytes(ctx->d);
    return EDAC_OK;
}

namespace {

// One evaluation with its tangents (value kernel, then the tangent kernel of the same part).
int tangent_eval(edac_ctx *c, int end_of_step)
{
    const Dev &d = c->d;
    cudaStream_t s = c->stream;
    int n = 0;
    n += launch_rebuild(d, s, 0);
    n += launch_pass_a(d, s, 0);
    n += launch_tangent(d, c->tws, s, TG_PASS_A, 0.0);
    n += launch_boundary(d, s, 0, end_of_step);
    n += launch_tangent(d, c->tws, s, TG_BOUNDARY, 0.0);
    n += launch_pass_b(d, s, 0);
    n += launch_tangent(d, c->tws, s, TG_PASS_B, 0.0);
    // the outlet update of this evaluation: its values went to the slot arrays only, after the
    // rates of this evaluation were fixed on the step's outlet values; so are its tangents
    if (end_of_step && d.ph.has_outlet) n += launch_tangent(d, c->tws, s, TG_OUTLET, 0.0);
    return n;
}

}  // namespace

edac_status edac_tangent_enable(edac_ctx *ctx, void *d_workspace, size_t bytes)
{
    if (!ctx) return EDAC_E_INVALID;
    if (ctx->mixed) return fail(ctx, EDAC_E_STATE, "the tangent model is built on the fp64 path");
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    const Phys &ph = ctx->d.ph;
    if (ph.in_kind != IN_MODES || (ph.has_outlet && ph.outlet_kind != OUT_HYBRID))
        return fail(ctx, EDAC_E_STATE, "the tangent model needs the steady inlet modes and the hybrid outlet");
    if (ph.wall_drag[0] == 2 || ph.wall_drag[1] == 2)
        return fail(ctx, EDAC_E_STATE, "the tangent model takes the solid force over fluid neighbours (count_in_drag 1)");
    if (!d_workspace || bytes < tangent_bytes(ctx->d) || ((uintptr_t)d_workspace & 255u))
        return fail(ctx, EDAC_E_INVALID, "tangent workspace missing, too small or not 256-byte aligned");
    ctx->tws = d_workspace;
    ctx->tws_bytes = bytes;
    ctx->tangent_steps = 0;
    CK(cudaMemsetAsync(d_workspace, 0, bytes, ctx->stream));
    ctx->launches += launch_tangent(ctx->d, ctx->tws, ctx->stream, TG_INIT, 0.0);
    // the rates of the current state, with their tangents
    ctx->launches += tangent_eval(ctx, 0);
    CK(cudaGetLastError());
    return check_device(ctx);
}

edac_status edac_step_tangent(edac_ctx *ctx, int nsteps)
{
    if (!ctx) return EDAC_E_INVALID;
    if (nsteps < 0) return fail(ctx, EDAC_E_INVALID, "nsteps < 0");
    if (!ctx->tws) return fail(ctx, EDAC_E_STATE, "call edac_tangent_enable first");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    const Dev &d = ctx->d;
    cudaStream_t s = ctx->stream;
    for (int k = 0; k < nsteps; ++k) {
        int n = 0;
        n += launch_stage(d, s, 0, 0);
        n += launch_tangent(d, ctx->tws, s, TG_STAGE_PRED, 0.5 * d.ph.dt);
        n += tangent_eval(ctx, 0);
        n += launch_stage(d, s, 0, 1);
        n += launch_tangent(d, ctx->tws, s, TG_STAGE_CORR, d.ph.dt);
        n += tangent_eval(ctx, 1);
        n += launch_tangent(d, ctx->tws, s, TG_RECYCLE_PRE, 0.0);
        n += launch_recycle(d, s);
        n += launch_tangent(d, ctx->tws, s, TG_RECYCLE_POST, 0.0);
        ctx->launches += n;
    }
    ctx->tangent_steps += nsteps;
    CK(cudaGetLastError());
    return EDAC_OK;
}

// ------------------------------------------------------------ reverse-mode adjoint
namespace {

// one fp64 evaluation of the values (the sequence the tangent model interleaves with)
int value_eval(edac_ctx *c, int end_of_step)
{
    const Dev &d = c->d;
    cudaStream_t s = c->stream;
    int n = 0;
    n += launch_rebuild(d, s, 0);
    n += launch_pass_a(d, s, 0);
    n += launch_boundary(d, s, 0, end_of_step);
    n += launch_pass_b(d, s, 0);
    return n;
}

// One step of values, eager.  With aws: the decisions its adjoint holds fixed are recorded
// in record rec (the ring write index before the corrector, the gate after it, the tags
// before recycling), and the workspace after the first evaluation is copied to mid.
int value_step(edac_ctx *c, void *aws = nullptr, int nsteps_ws = 0, int nrec = 0, int rec = 0,
               void *mid = nullptr)
{
    const Dev &d = c->d;
    cudaStream_t s = c->stream;
    int n = 0;
    n += launch_stage(d, s, 0, 0);
    n += value_eval(c, 0);
    if (mid) cudaMemcpyAsync(mid, c->ws, c->ws_bytes, cudaMemcpyDeviceToDevice, s);
    if (aws) n += launch_adjoint(d, aws, nsteps_ws, nrec, rec, s, AJ_REC_RPOS);
    n += launch_stage(d, s, 0, 1);
    if (aws) n += launch_adjoint(d, aws, nsteps_ws, nrec, rec, s, AJ_REC_GATE);
    n += value_eval(c, 1);
    if (aws) n += launch_adjoint(d, aws, nsteps_ws, nrec, rec, s, AJ_REC_TAG);
    n += launch_recycle(d, s);
    return n;
}

// workspace copies: the checkpoints, the final state, a segment's states before each step and
// after the last (K + 1) and after each step's first evaluation (K)
size_t adjoint_snapshots(int nsteps, int K) { return (size_t)((nsteps + K - 1) / K) + 1 + 2 * (size_t)K + 1; }

}  // namespace

edac_status edac_adjoint_workspace_bytes(edac_ctx *ctx, int nsteps, int checkpoint_every,
                                         size_t *bytes)
{
    if (!ctx) return EDAC_E_INVALID;
    if (!bytes || nsteps < 1 || checkpoint_every < 1)
        return fail(ctx, EDAC_E_INVALID, "adjoint: nsteps >= 1, checkpoint_every >= 1, bytes not NULL");
    const size_t wsb = (ctx->ws_bytes + 255) & ~(size_t)255;
    const size_t ab = (adjoint_bytes(ctx->d, nsteps, checkpoint_every) + 255) & ~(size_t)255;
    *bytes = ab + adjoint_snapshots(nsteps, checkpoint_every) * wsb;
    return EDAC_OK;
}

edac_status edac_adjoint_run(edac_ctx *ctx, void *d_workspace, size_t bytes, int nsteps,
                             int checkpoint_every, const double *h_w_fx, const double *h_w_fy,
                             const double *h_w_pe, double pe_x0, double pe_x1, double *h_loss,
                             double *h_grad)
{
    if (!ctx) return EDAC_E_INVALID;
    if (ctx->mixed) return fail(ctx, EDAC_E_STATE, "the adjoint is built on the fp64 path");
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    const Phys &ph = ctx->d.ph;
    if (ph.in_kind != IN_MODES || (ph.has_outlet && ph.outlet_kind != OUT_HYBRID))
        return fail(ctx, EDAC_E_STATE, "the adjoint covers the steady inlet modes and the hybrid outlet");
    if (ph.wall_drag[0] == 2 || ph.wall_drag[1] == 2)
        return fail(ctx, EDAC_E_STATE, "the adjoint takes the solid force over fluid neighbours (count_in_drag 1)");
    if (nsteps < 1 || checkpoint_every < 1 || !h_grad)
        return fail(ctx, EDAC_E_INVALID, "adjoint: nsteps >= 1, checkpoint_every >= 1, h_grad not NULL");
    if (nsteps > ctx->d.max_history)
        return fail(ctx, EDAC_E_INVALID, "adjoint: nsteps exceeds the context's history (max_history)");
    if (h_w_pe && !(pe_x1 > pe_x0))
        return fail(ctx, EDAC_E_INVALID, "adjoint: the pressure-energy window needs pe_x1 > pe_x0");
    if (any_profiling(ctx)) return fail(ctx, EDAC_E_STATE, "kernel profiling is on");
    size_t need = 0;
    edac_status st = edac_adjoint_workspace_bytes(ctx, nsteps, checkpoint_every, &need);
    if (st) return st;
    if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255u))
        return fail(ctx, EDAC_E_INVALID, "adjoint workspace missing, too small or not 256-byte aligned");
    Counters h0;
    CK(cudaMemcpyAsync(&h0, ctx->d.cnt, sizeof(h0), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h0.err) {
        ctx->failed = true;
        return fail(ctx, EDAC_E_STATE, "context in error");
    }
    if (h0.step != 0) return fail(ctx, EDAC_E_STATE, "run the adjoint from a freshly uploaded state (no steps taken)");
    const Dev &d = ctx->d;
    cudaStream_t s = ctx->stream;
    const int N = nsteps, K = checkpoint_every, nseg = (N + K - 1) / K;
    char *aws = static_cast<char *>(d_workspace);
    const size_t ab = (adjoint_bytes(d, N, K) + 255) & ~(size_t)255;
    const size_t wsb = (ctx->ws_bytes + 255) & ~(size_t)255;
    char *snaps = aws + ab;
    auto ckpt = [&](int i) { return snaps + (size_t)i * wsb; };
    char *fin = snaps + (size_t)nseg * wsb;
    auto state = [&](int j) { return snaps + (size_t)(nseg + 1 + j) * wsb; };      // j = 0..K
    auto mid = [&](int j) { return snaps + (size_t)(nseg + 2 + K + j) * wsb; };    // j = 0..K-1
    auto copy = [&](void *dst, const void *src) {
        return cudaMemcpyAsync(dst, src, ctx->ws_bytes, cudaMemcpyDeviceToDevice, s);
    };
    auto w_at = [](const double *w, int n) { return w ? w[n] : 0.0; };
    auto adj = [&](int rec, int what, double p0 = 0.0, double p1 = 0.0, double p2 = 0.0) {
        return launch_adjoint(d, aws, N, K, rec, s, what, p0, p1, p2);
    };
    long long launches = 0;
    launches += adj(0, AJ_ZERO);
    // forward: checkpoints every K steps, the pressure energy of every step
    for (int n = 0; n < N; ++n) {
        if (n % K == 0) CK(copy(ckpt(n / K), ctx->ws));
        launches += value_step(ctx);
        if (h_w_pe) launches += adj(0, AJ_PE_VALUE, (double)n, pe_x0, pe_x1);
    }
    CK(copy(fin, ctx->ws));
    CK(cudaGetLastError());
    // the loss from the forward history
    Counters h;
    CK(cudaMemcpyAsync(&h, d.cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    std::vector<double> hist((size_t)d.max_history * 8), pe((size_t)N, 0.0);
    CK(cudaMemcpyAsync(hist.data(), d.hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost, s));
    if (h_w_pe)
        CK(cudaMemcpyAsync(pe.data(), adjoint_pe(d, aws, N, K), sizeof(double) * (size_t)N,
                           cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h.err) {
        CK(copy(ctx->ws, fin));
        ctx->failed = true;
        return fail(ctx, EDAC_E_STATE, "the forward run of the adjoint set the device error word");
    }
    double L = 0.0;
    for (int n = 0; n < N; ++n) {
        const double *rec = hist.data() + (size_t)(n % d.max_history) * 8;
        L += w_at(h_w_fx, n) * rec[0] + w_at(h_w_fy, n) * rec[1] + w_at(h_w_pe, n) * pe[(size_t)n];
    }
    // reverse: each segment recomputed once from its checkpoint, keeping the workspace after
    // the first evaluation and at the end of every step and the step's decisions; then its
    // steps reversed from those copies
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int n0 = sg * K, len = std::min(K, N - n0);
        CK(copy(ctx->ws, ckpt(sg)));
        for (int j = 0; j < len; ++j) {
            launches += value_step(ctx, aws, N, K, j, mid(j));
            CK(copy(state(j + 1), ctx->ws));
        }
        for (int j = len - 1; j >= 0; --j) {
            const int n = n0 + j;
            CK(copy(ctx->ws, state(j + 1)));
            if (w_at(h_w_pe, n) != 0.0) launches += adj(j, AJ_PE_SEED, w_at(h_w_pe, n), pe_x0, pe_x1);
            launches += adj(j, AJ_RECYCLE);
            launches += adj(j, AJ_EVAL, 1.0, w_at(h_w_fx, n), w_at(h_w_fy, n));
            launches += adj(j, AJ_STAGE_CORR, d.ph.dt);
            CK(copy(ctx->ws, mid(j)));
            launches += adj(j, AJ_EVAL, 0.0);
            launches += adj(j, AJ_STAGE_PRED, 0.5 * d.ph.dt);
        }
        CK(cudaGetLastError());
    }
    // the evaluation and set-up of the upload
    CK(copy(ctx->ws, ckpt(0)));
    launches += adj(0, AJ_EVAL, 0.0);
    launches += adj(0, AJ_INIT);
    launches += adj(0, AJ_REDUCE);
    double g[T_DIR];
    CK(cudaMemcpyAsync(g, adjoint_grad(d, aws, N, K), sizeof(g), cudaMemcpyDeviceToHost, s));
    CK(copy(ctx->ws, fin));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    ctx->launches += launches;
    for (int c = 0; c < T_DIR; ++c) h_grad[c] = g[c];
    if (h_loss) *h_loss = L;
    return EDAC_OK;
}

edac_status edac_read_tangent_history(edac_ctx *ctx, int max_steps, double *h_dfx, double *h_dfy,
                                      int *nsteps)
{
    if (!ctx || !nsteps || max_steps < 0) return EDAC_E_INVALID;
    if (!ctx->tws) return fail(ctx, EDAC_E_STATE, "call edac_tangent_enable first");
    edac_status st = check_device(ctx);
    if (st) return st;
    Counters h;
    CK(cudaMemcpyAsync(&h, ctx->d.cnt, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    const int H = ctx->d.max_history;
    std::vector<double> hist((size_t)H * 2 * T_DIR);
    const double *dev_hist = tangent_hist(ctx->d, ctx->tws);
    CK(cudaMemcpyAsync(hist.data(), dev_hist, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const long long avail = std::min<long long>(std::min(h.hist_len, H), ctx->tangent_steps);
    const int k = (int)std::min<long long>(avail, max_steps);
    for (int r = 0; r < k; ++r) {
        const int stepi = h.step - k + r;
        const double *rec = hist.data() + (size_t)(stepi % H) * 2 * T_DIR;
        for (int c = 0; c < T_DIR; ++c) {
            if (h_dfx) h_dfx[(size_t)r * T_DIR + c] = rec[c];
            if (h_dfy) h_dfy[(size_t)r * T_DIR + c] = rec[T_DIR + c];
        }
    }
    *nsteps = k;
    return EDAC_OK;
}

edac_status edac_set_tiling(edac_ctx *ctx, int tile_cells, int threads)
{
    if (!ctx) return EDAC_E_INVALID;
    if (tile_cells < 1 || tile_cells > EDAC_TILE_MAX_CELLS || threads < 64 ||
        threads > EDAC_TILE_MAX_THREADS || threads % 32 != 0)
        return fail(ctx, EDAC_E_INVALID, "tiling: 1 <= tile_cells <= 16, threads a multiple of 32 in [64, 256]");
    ctx->d.tile_tx = tile_cells;
    ctx->d.tile_tpb = threads;
    drop_graph(ctx);
    return EDAC_OK;
}

edac_status edac_autotune(edac_ctx *ctx, int trials, int *tile_cells, int *threads, double *ms)
{
    if (!ctx || trials < 1) return EDAC_E_INVALID;
    if (!ctx->loaded) return fail(ctx, EDAC_E_STATE, "no particles");
    if (ctx->failed) return fail(ctx, EDAC_E_STATE, "context in error");
    if (any_profiling(ctx)) return fail(ctx, EDAC_E_STATE, "autotune with kernel profiling on");
    // candidate tilings of the mixed pair passes; the fp64 path has none to choose
    static const int cand[][2] = {{11, 160}, {16, 256}, {8, 128}, {6, 128},
                                  {4, 64},   {6, 64},   {3, 64},  {2, 64}};
    const int ncand = ctx->mixed ? (int)(sizeof(cand) / sizeof(cand[0])) : 1;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, EDAC_E_CUDA, "event create");
    }
    const int tx0 = ctx->d.tile_tx, tpb0 = ctx->d.tile_tpb;
    int best = -1;
    float best_ms = 0.0f;
    edac_status st = EDAC_OK;
    for (int c = 0; c < ncand && st == EDAC_OK; ++c) {
        if (ctx->mixed) {
            ctx->d.tile_tx = cand[c][0];
            ctx->d.tile_tpb = cand[c][1];
        }
        // an evaluation is idempotent (it recomputes the rates of the current state), so
        // the trials leave the state as they found it
        issue_eval(ctx, 0);  // warm-up of this tiling
        cudaEventRecord(e0, ctx->stream);
        for (int t = 0; t < trials; ++t) ctx->launches += issue_eval(ctx, 0);
        cudaEventRecord(e1, ctx->stream);
        float t_ms = 0.0f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess)
            st = fail(ctx, EDAC_E_CUDA, "autotune timing");
        else if (best < 0 || t_ms < best_ms) {
            best = c;
            best_ms = t_ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != EDAC_OK) {
        ctx->d.tile_tx = tx0;
        ctx->d.tile_tpb = tpb0;
        return st;
    }
    if (ctx->mixed) {
        ctx->d.tile_tx = cand[best][0];
        ctx->d.tile_tpb = cand[best][1];
    }
    ctx->launches += issue_eval(ctx, 0);  // the rates of the state under the chosen tiling
    drop_graph(ctx);
    if (tile_cells) *tile_cells = ctx->d.tile_tx;
    if (threads) *threads = ctx->d.tile_tpb;
    if (ms) *ms = (double)best_ms / (double)trials;
    CK(cudaGetLastError());
    return check_device(ctx);
}

}  // extern "C"

// ------------------------------------------------------------------------ batches
struct edac_batch {
    std::vector<edac_ctx *> ctx;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;  // [0] fork, [1..n] joins, [n+1] done
    std::vector<int> kper;        // kernels per step of each member
    int kernels = 0;
    bool fused = false;           // one launch per kernel over all members (edac_batch_create_fused)
    BatchPlan plan{};
};

namespace {

// One step of every member of a fused batch: the single-system launch sequence (stages with
// the cell count fused in, cell builds, pass A, boundary, pass B, recycling), each kernel
// launched once over the blocks of all members.
int issue_step_batch(const BatchPlan &p, cudaStream_t s)
{
    int n = 0;
    n += launch_stage_batch(p, s, 0);
    n += launch_rebuild_batch(p, s);
    n += launch_pass_a_batch(p, s);
    n += launch_boundary_batch(p, s, 0);
    n += launch_pass_b_batch(p, s);
    n += launch_stage_batch(p, s, 1);
    n += launch_rebuild_batch(p, s);
    n += launch_pass_a_batch(p, s);
    n += launch_boundary_batch(p, s, 1);
    n += launch_pass_b_batch(p, s);
    n += launch_recycle_batch(p, s);
    return n;
}

// Layout of a fused batch's device workspace: the members' Dev, then one block-offset table
// ([n + 1] ints) per kernel shape.
size_t batch_layout(int n, size_t *off_tables)
{
    size_t off = ((size_t)n * sizeof(Dev) + 255) & ~(size_t)255;
    for (int k = 0; k < BK_NUM; ++k) {
        if (off_tables) off_tables[k] = off;
        off += (((size_t)n + 1) * sizeof(int) + 255) & ~(size_t)255;
    }
    return off;
}

void batch_free(edac_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

}  // namespace

extern "C" {

edac_status edac_batch_create(edac_ctx *const *ctxs, int n, void *cuda_stream, edac_batch **out)
{
    if (!out) return fail(nullptr, EDAC_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return fail(nullptr, EDAC_E_INVALID, "no contexts");
    cudaStream_t ms = (cudaStream_t)cuda_stream;
    if (!ms) return fail(nullptr, EDAC_E_INVALID, "a batch needs a non-default stream");
    for (int i = 0; i < n; ++i) {
        edac_ctx *c = ctxs[i];
        if (!c) return fail(nullptr, EDAC_E_INVALID, "NULL context in the batch");
        if (!c->loaded || c->failed) return fail(nullptr, EDAC_E_STATE, "batch member without particles or in error");
        if (!c->stream || c->stream == ms) return fail(nullptr, EDAC_E_INVALID, "each member needs a non-default stream other than the batch's");
        if (any_profiling(c)) return fail(nullptr, EDAC_E_STATE, "batch member with kernel profiling on");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(nullptr, EDAC_E_INVALID, "batch members must be distinct");
    }
    edac_batch *b = new edac_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = ms;
    b->ev.assign((size_t)n + 2, nullptr);
    for (auto &e : b->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            batch_free(b);
            return fail(nullptr, EDAC_E_CUDA, "event create");
        }
    // one step of every member, each on its own stream, forked from and joined back to the
    // batch stream inside one capture: the members' kernels form independent graph branches
    cudaError_t e = cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[0], ms);
    int k = 0;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        edac_ctx *c = b->ctx[i];
        e = cudaStreamWaitEvent(c->stream, b->ev[0], 0);
        if (e != cudaSuccess) break;
        const int ki = issue_step(c);
        b->kper.push_back(ki);
        k += ki;
        e = cudaEventRecord(b->ev[1 + i], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ms, b->ev[1 + i], 0);
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ms, &gr);
    if (e == cudaSuccess) e = e2;
    b->graph = gr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, gr, 0);
    if (e != cudaSuccess) {
        batch_free(b);
        return fail(nullptr, EDAC_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    b->kernels = k;
    *out = b;
    return EDAC_OK;
}

edac_status edac_batch_workspace_bytes(int n, size_t *bytes)
{
    if (!bytes || n < 1) return fail(nullptr, EDAC_E_INVALID, "bad batch workspace arguments");
    *bytes = batch_layout(n, nullptr);
    return EDAC_OK;
}

edac_status edac_batch_create_fused(edac_ctx *const *ctxs, int n, void *cuda_stream,
                                    void *d_workspace, size_t bytes, edac_batch **out)
{
    if (!out) return fail(nullptr, EDAC_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return fail(nullptr, EDAC_E_INVALID, "no contexts");
    cudaStream_t ms = (cudaStream_t)cuda_stream;
    if (!ms) return fail(nullptr, EDAC_E_INVALID, "a batch needs a non-default stream");
    size_t tab[BK_NUM];
    const size_t need = batch_layout(n, tab);
    if (!d_workspace || bytes < need || ((uintptr_t)d_workspace & 255u))
        return fail(nullptr, EDAC_E_INVALID, "batch workspace missing, too small or not 256-byte aligned");
    for (int i = 0; i < n; ++i) {
        edac_ctx *c = ctxs[i];
        if (!c) return fail(nullptr, EDAC_E_INVALID, "NULL context in the batch");
        if (!c->loaded || c->failed) return fail(nullptr, EDAC_E_STATE, "batch member without particles or in error");
        if (!c->stream || c->stream == ms) return fail(nullptr, EDAC_E_INVALID, "each member needs a non-default stream other than the batch's");
        if (any_profiling(c)) return fail(nullptr, EDAC_E_STATE, "batch member with kernel profiling on");
        if (c->mixed != ctxs[0]->mixed) return fail(nullptr, EDAC_E_INVALID, "fused batch members must share the precision");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(nullptr, EDAC_E_INVALID, "batch members must be distinct");
    }
    edac_batch *b = new edac_batch();
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = ms;
    b->fused = true;
    b->ev.assign((size_t)n + 2, nullptr);
    for (auto &e : b->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            batch_free(b);
            return fail(nullptr, EDAC_E_CUDA, "event create");
        }
    // member table and block offsets, copied into the caller's workspace
    char *ws = static_cast<char *>(d_workspace);
    std::vector<Dev> devs((size_t)n);
    std::vector<int> offs((size_t)BK_NUM * (n + 1), 0);
    BatchPlan &p = b->plan;
    p.n = n;
    p.mixed = ctxs[0]->mixed;
    p.pair_tpb = 64;
    p.any_mirror = false;
    for (int i = 0; i < n; ++i) {
        const edac_ctx *c = ctxs[i];
        devs[i] = c->d;
        p.pair_tpb = std::max(p.pair_tpb, c->d.tile_tpb);
        p.any_mirror = p.any_mirror || (c->d.ph.has_outlet && c->d.ph.outlet_kind == OUT_MIRROR);
        for (int k = 0; k < BK_NUM; ++k) {
            long long nb = batch_blocks(c->d, k);
            long long tot = (long long)offs[(size_t)k * (n + 1) + i] + nb;
            if (nb < 0 || tot > (1LL << 30)) {
                batch_free(b);
                return fail(nullptr, EDAC_E_INVALID, "fused batch grid too large");
            }
            offs[(size_t)k * (n + 1) + i + 1] = (int)tot;
        }
    }
    p.devs = reinterpret_cast<const Dev *>(ws);
    for (int k = 0; k < BK_NUM; ++k) {
        p.off[k] = reinterpret_cast<const int *>(ws + tab[k]);
        p.total[k] = offs[(size_t)k * (n + 1) + n];
    }
    cudaError_t e = cudaMemcpyAsync(ws, devs.data(), sizeof(Dev) * (size_t)n, cudaMemcpyHostToDevice, ms);
    for (int k = 0; k < BK_NUM && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(ws + tab[k], offs.data() + (size_t)k * (n + 1), sizeof(int) * (size_t)(n + 1),
                            cudaMemcpyHostToDevice, ms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ms);
    // one step of all members: one launch per kernel, captured once
    int k = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        k = issue_step_batch(p, ms);
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(ms, &gr);
        b->graph = gr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, gr, 0);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return fail(nullptr, EDAC_E_CUDA, std::string("fused batch: ") + cudaGetErrorString(e));
    }
    b->kernels = k;
    b->kper.assign((size_t)n, k);
    *out = b;
    return EDAC_OK;
}

edac_status edac_batch_step(edac_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return fail(nullptr, EDAC_E_INVALID, "bad batch step arguments");
    for (edac_ctx *c : b->ctx)
        if (c->failed) return fail(c, EDAC_E_STATE, "batch member in error");
    if (nsteps == 0) return EDAC_OK;
    const int n = (int)b->ctx.size();
    cudaError_t e = cudaSuccess;
    // the batch stream waits for work queued on the members' streams (uploads, reads) ...
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventRecord(b->ev[1 + i], b->ctx[i]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[1 + i], 0);
    }
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = cudaGraphLaunch(b->exec, b->stream);
    // ... and the members' later calls wait for the batch
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[n + 1], b->stream);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->ctx[i]->stream, b->ev[n + 1], 0);
    if (e != cudaSuccess) return fail(nullptr, EDAC_E_CUDA, std::string("batch step: ") + cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) b->ctx[i]->launches += (long long)b->kper[i] * nsteps;
    return EDAC_OK;
}

edac_status edac_batch_launch_count(edac_batch *b, int64_t *kernels_per_step)
{
    if (!b || !kernels_per_step) return EDAC_E_INVALID;
    *kernels_per_step = b->kernels;
    return EDAC_OK;
}

void edac_batch_destroy(edac_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

void edac_destroy(edac_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->loaded) cudaStreamSynchronize(ctx->stream);
    drop_graph(ctx);
    for (int k = 0; k < EDAC_NUM_KERNELS; ++k)
        for (auto &e : ctx->prof_ev[k]) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
    delete ctx;
}

}  // extern "C"
