// Internal declarations of the EDAC SPH library: device-side parameter and
// pointer bundles, the quintic-kernel and neighbour-walk device helpers shared
// by the pair kernels, and the host launchers.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace edac {

constexpr int NAVG_MAX = 8;       // longest time-average window of the hybrid outlet
constexpr int MAX_MODES = 16;     // inlet profile modes
constexpr int LIST_MAX = 16384;   // recycling events per step (per kind)
constexpr uint8_t TAG_DEAD = 255; // free slot
constexpr uint8_t TAG_REDP = 0x80; // sorted-tag flag: outlet particle red in the previous step

enum : uint8_t { FLUID = 0, INLET = 1, OUTLET = 2, WALL = 3, SLIPWALL = 4 };

// sticky device error bits
enum : unsigned { ERR_CAPACITY = 1u, ERR_NONFINITE = 2u, ERR_DOMAIN = 4u, ERR_LIST = 8u,
                  ERR_TIMEOUT = 16u };
// inlet velocity in time: steady modes, and the 2D pulse, ramp and passing vortex of the
// outlet test problems (Secs. 4.2-4.4)
enum : int { IN_MODES = 0, IN_PULSE = 1, IN_RAMP = 2, IN_VORTEX = 3 };
// outlet treatments (Sec. 3): hybrid (3.4), do-nothing (3.1), modified do-nothing (3.1.1),
// method of characteristics (3.3), mirroring (3.2)
enum : int { OUT_HYBRID = 0, OUT_DONOTHING = 1, OUT_MOD_DONOTHING = 2, OUT_CHARACTERISTIC = 3,
             OUT_MIRROR = 4 };

// Geometry of the cell grid and the support radius.
struct Geo {
    double x_min, x_max, y_min, y_max;
    double Lx, Ly, hLx, hLy;  // box lengths and halves (minimum image)
    int px, py;               // periodic axes
    int nx, ny, ncells;
    double sx, sy, inv_sx, inv_sy;
    float sxf, syf;
    double rc2;               // (3h)^2, the membership bound
    float rc2_lo, rc2_hi;     // fp32 pre-test band around rc2
};

// Physical and zone parameters.
struct Phys {
    double h, inv_h, a2, a2h;        // alpha_2 = 7/(478 pi h^2), alpha_2 / h
    double rho0, cs, c2, nu, nu_e, eh2, pb, gx, gy, dt, U;
    double inv_2rc, inv_navg;        // 1/(2 rho0 c_s), 1/n_avg
    float inv_hf, a2f, a2hf, c2f, nuf, nuef, eh2f, w0f, gxf, gyf, pbf, inv_2rcf;
    int use_pavg;
    int has_inlet, n_modes;
    double x_in, L_in, in_y0, in_H;
    double modes[MAX_MODES];
    int has_outlet, n_avg;
    int outlet_kind;                 // EDAC_OUTLET_* (hybrid unless set)
    double moc_u_ref, moc_p_ref;     // reference state of the characteristic outlet
    int in_kind;                     // IN_*: inlet velocity in time
    double in_prm[4];                // its parameters
    double x_out, L_out, I_thr;
    int wall_slip[2], wall_drag[2];  // wall_drag: 0 off, 1 fluid neighbours, 2 every neighbour
    double wall_u[2], wall_v[2];
};

// How a particle of tag t enters the drag: 0 not at all, 1 its force over its fluid
// neighbours with the interpolated pressure, 2 Eq. tvf-momentum_solid over every neighbour.
__host__ __device__ __forceinline__ int drag_mode(const Phys &ph, int t)
{
    return t == WALL ? ph.wall_drag[0] : t == SLIPWALL ? ph.wall_drag[1] : 0;
}

// Device counters (one struct in the workspace).
struct Counters {
    int n_alive;     // live particles
    int n_bnd;       // boundary particles in the sorted order (rebuilt each gather)
    int free_top;    // free-slot stack height
    int n_spawn, n_del, n_out;  // recycling events of the current step
    unsigned err;    // sticky error word
    int step;        // completed steps
    int n_drag;      // solid particles in the drag sum (static)
    int hist_len;    // history records written (saturates at max_history)
    unsigned long long next_id;
    int last_spawn;  // inlet particles spawned by the last k_end_step (spawn_map entries)
    // the first particle found outside the domain box (error context for the host)
    int err_rec, err_tag;
    unsigned long long err_id;
    double err_x, err_y;
    // recycling event log: records written since the last read, events not logged
    int ev_len;
    unsigned long long ev_dropped;
};

// One recycling event of the log (EDAC_EVENT_*): the particle id, a second id (a spawn's
// parent), the step counter after the step and the kind.
struct EventRec {
    unsigned long long id, other;
    int step, kind;
};
enum : int { EV_DELETE = 0, EV_TO_OUTLET = 1, EV_SPAWN = 2 };

// Everything a kernel may touch.
struct Dev {
    Geo g;
    Phys ph;
    int cap;
    int max_history;
    int mixed;         // 1: mixed-precision path (fp32 ring samples, fp32 pair terms)
    Counters *cnt;
    // master particle state, slot-indexed [cap]
    double *x, *y, *u, *v, *ut, *vt, *p, *m;
    double *x0, *y0, *u0, *v0, *p0;
    // rates: fp64 on the fp64 path; on the mixed path (fp32 pair sums) au, av, ap, abu, abv
    // hold fp32 values in the first half of each array (rate_f), half the bytes per step
    double *au, *av, *ap, *abu, *abv, *fx, *fy, *rho, *vol;
    int *nnb;
    uint8_t *tag;
    unsigned long long *id;
    double *ring;   // [cap][NAVG_MAX][3] (fp64 path) or float [cap][NAVG_MAX][3] (mixed path)
    uint8_t *rpos;
    double *ubar, *vbar, *pbar, *J2, *J2p, *advp;
    uint8_t *redp;
    // cell list
    double *org_x, *org_y;  // [nx], [ny]: x_min + cx sx, y_min + cy sy (cell origins)
    int *cell_count;   // [ncells]
    int *cell_start;   // [ncells + 1]
    int *slot_cell;    // [cap]
    int *within;       // [cap]
    // sorted (cell-ordered) copies, index k < n_alive
    int *order;        // slot of k
    int *order_raw;    // slots scattered by cell in atomic order (input of the per-cell sort)
    int *scan_part;    // per-block partial sums of the cell-count scan
    int *cellk;        // cell of k
    uint8_t *stag;     // tag of k (| TAG_REDP)
    float4 *P;         // (x - cell x0, y - cell y0, m, p (mixed path) | 0) fp32, both paths
    double2 *XY;       // fp64 position
    double2 *AUX;      // (J2 of fluid | J2 of outlet previous step, outlet advection velocity)
    int *snnb;         // neighbour count N_k
    // fp64 path
    double2 *UV, *DUV; // (u, v), (u~ - u, v~ - v)
    double2 *PV;       // (p, V)
    double2 *RM;       // (rho, m / rho)
    double *Ms;        // m
    double *GS;        // [3 per k] pass B's sums G_x, G_y, sum (p_j - p_i) (the adjoint reads them)
    // mixed path
    float4 *Bf;        // (u, v, u~ - u, v~ - v)
    float4 *Qf;        // (p, V, rho, m / rho)
    uint4 *nbm;        // [2 per k] neighbour mask over the candidate windows (pass A -> pass B)
    int tile_tx, tile_tpb;  // tiling of the mixed pair passes: cells per tile, threads per block
    int *bnd;          // boundary particles (sorted index), n_bnd of them
    // recycling
    int *free_stack;   // [cap]
    unsigned long long *ev_spawn_key; int *ev_spawn_slot;   // [LIST_MAX]
    unsigned long long *ev_del_key;   int *ev_del_slot;     // [LIST_MAX]
    unsigned long long *ev_out_key;   double *ev_out_m;     // [LIST_MAX]
    EventRec *evlog;   // caller-owned event log (nullptr: not logged), ev_cap records
    int ev_cap;
    int *drag_slots;   // [n_drag], ascending slot
    int2 *spawn_map;   // [LIST_MAX] (parent slot, new slot) of the last step's spawns
    double *scratch_m; // [LIST_MAX]
    double *hist;      // [max_history][8]
    double *probe_part;  // [PROBE_BLK][PROBE_MAX][8] per-block probe sums
    double *probe_out;   // [PROBE_MAX][4] probe values
};

// The mixed path's fp32 view of a rate array (au, av, ap, abu, abv).
__host__ __device__ __forceinline__ float *rate_f(double *a) { return reinterpret_cast<float *>(a); }

// Probe points (by value into the probe kernels).
constexpr int PROBE_MAX = 8;
constexpr int PROBE_BLK = 304;
struct ProbePts {
    int n;
    double x[PROBE_MAX], y[PROBE_MAX];
};

// -------------------------------------------------------------------------------------------
// fp32 <-> fp64 conversions on the integer pipe.  On GB300 the hardware conversions between
// fp32 and fp64 issue to the fp64 pipe (about 0.6 T conversions/s, the DFMA rate), which makes
// them the largest fp64 cost of the gather, the stage, the pair-pass epilogues and the
// mirror sums.  These are the IEEE 754 conversions written out on the bit fields: widening a
// normal float moves the sign, re-biases the exponent (127 -> 1023) and appends 29 zero
// mantissa bits; narrowing a double whose result is a normal float (or overflows to
// infinity by rounding) keeps the top 23 of the 52 mantissa bits and rounds the 29 dropped
// bits to nearest, ties to even (a carry out of the mantissa steps the exponent, as the
// format intends).  Zeros are handled on the fast path; subnormals, infinities and NaNs (none
// of which the solver's fields hold) take the hardware conversion.  The results equal the
// hardware conversion bit for bit (edac_conversion_check: every float, and sampled doubles).
// -------------------------------------------------------------------------------------------
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned mag = b & 0x7fffffffu;
    if ((mag >> 23) - 1u < 254u) {  // normal: exponent field 1..254
        const unsigned hi = (b & 0x80000000u) | ((mag >> 3) + 0x38000000u);
        return __hiloint2double((int)hi, (int)(b << 29));
    }
    if (mag == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)f;
}

__device__ __forceinline__ float d2f(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned mag = hi & 0x7fffffffu;
    if ((mag >> 20) - 897u < 254u) {  // float exponent 1..254 before rounding
        const unsigned base = __funnelshift_l(lo, mag - 0x38000000u, 3);  // exponent | top 23 bits
        const unsigned inc = ((lo & 0x1fffffffu) + (base & 1u) + 0x0fffffffu) >> 29;  // RNE
        return __uint_as_float((hi & 0x80000000u) | (base + inc));
    }
    if ((mag | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rn(x);
}

// the same for code templated on the storage type R (float or double)
__device__ __forceinline__ double widen(float x) { return f2d(x); }
__device__ __forceinline__ double widen(double x) { return x; }
template <class R> __device__ __forceinline__ R narrow(double x);
template <> __device__ __forceinline__ float narrow<float>(double x) { return d2f(x); }
template <> __device__ __forceinline__ double narrow<double>(double x) { return x; }

// -------------------------------------------------------------------------------------------
// Quintic spline (Eq. quintic-spline) in the branch-free form: with t_k = max(0, k - q),
//   w(q) = t3^5 - 6 t2^5 + 15 t1^5,   dw/dq = -5 (t3^4 - 6 t2^4 + 15 t1^4),
// which equals the paper's piecewise definition on every branch (t_k vanishes where the
// corresponding term is absent).  W = alpha_2 w(q), dW/dr = (alpha_2 / h) dw/dq.
// -------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T quintic_w(T q)
{
    T t3 = q < T(3) ? T(3) - q : T(0);
    T t2 = q < T(2) ? T(2) - q : T(0);
    T t1 = q < T(1) ? T(1) - q : T(0);
    T a = t3 * t3, b = t2 * t2, c = t1 * t1;
    return t3 * a * a - T(6) * (t2 * b * b) + T(15) * (t1 * c * c);
}

template <class T>
__device__ __forceinline__ T quintic_dw(T q)
{
    T t3 = q < T(3) ? T(3) - q : T(0);
    T t2 = q < T(2) ? T(2) - q : T(0);
    T t1 = q < T(1) ? T(1) - q : T(0);
    T a = t3 * t3, b = t2 * t2, c = t1 * t1;
    return T(-5) * (a * a - T(6) * (b * b) + T(15) * (c * c));
}

// w(q) and dw/dq together (the branch terms t_k and their squares are shared).
template <class T>
__device__ __forceinline__ void quintic_w_dw(T q, T &w, T &dw)
{
    const T t3 = q < T(3) ? T(3) - q : T(0);
    const T t2 = q < T(2) ? T(2) - q : T(0);
    const T t1 = q < T(1) ? T(1) - q : T(0);
    const T a = t3 * t3, b = t2 * t2, c = t1 * t1;
    const T a4 = a * a, b4 = b * b, c4 = c * c;
    w = t3 * a4 - T(6) * (t2 * b4) + T(15) * (t1 * c4);
    dw = T(-5) * (a4 - T(6) * b4 + T(15) * c4);
}

// Canonical fp64 separation r_i - r_j with the minimum image on periodic axes and
// r^2 = dx*dx + dy*dy evaluated without fused multiply-add: the membership test
// r^2 < (3h)^2 is decided by exactly this operation sequence.
__device__ __forceinline__ double exact_r2(const Geo &g, double xi, double yi, double xj,
                                          double yj, double &dx, double &dy)
{
    dx = xi - xj;
    if (g.px) {
        if (dx > g.hLx) dx = dx - g.Lx;
        else if (dx < -g.hLx) dx = dx + g.Lx;
    }
    dy = yi - yj;
    if (g.py) {
        if (dy > g.hLy) dy = dy - g.Ly;
        else if (dy < -g.hLy) dy = dy + g.Ly;
    }
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__device__ __forceinline__ int cell_coord(double v, double lo, double inv_s, int n)
{
    const int c = __double2int_rd((v - lo) * inv_s);  // floor, in one conversion
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// The membership test of every pair kernel.  rxo, ryo: the query's fp32 position relative to
// the origin of j's cell; pj: j's fp32 cell-relative position.  The fp32 pre-test rejects
// pairs with r^2 >= rc^2 (1 + 4e-5) and accepts pairs with r^2 <= rc^2 (1 - 4e-5); inside that
// band the fp64 test exact_r2 < rc^2 decides.  The fp32 error of r^2 on cell-relative (or
// tile-relative, at most ~10 cells from the origin) coordinates stays below 1e-5 rc^2, so the
// result always equals the fp64 test.
__device__ __forceinline__ bool is_member(const Dev &d, float rxo, float ryo, const float4 &pj,
                                          int j, double qx, double qy, float &dxf, float &dyf,
                                          float &r2f)
{
    dxf = rxo - pj.x;
    dyf = ryo - pj.y;
    r2f = dxf * dxf + dyf * dyf;
    if (r2f >= d.g.rc2_hi) return false;
    if (r2f > d.g.rc2_lo) {
        const double2 xy = d.XY[j];
        double ex, ey;
        return exact_r2(d.g, qx, qy, xy.x, xy.y, ex, ey) < d.g.rc2;
    }
    return true;
}

// Visit the 3x3 block of cells around (cx, cy): f(ox, oy, j0, j1) for each existing cell,
// with [j0, j1) its range in the cell order (periodic axes wrap).
template <class F>
__device__ __forceinline__ void for_block(const Dev &d, int cx, int cy, F &&f)
{
    const Geo &g = d.g;
#pragma unroll 1
    for (int oy = -1; oy <= 1; ++oy) {
        int by = cy + oy;
        if (g.py) by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
        else if (by < 0 || by >= g.ny) continue;
#pragma unroll 1
        for (int ox = -1; ox <= 1; ++ox) {
            int bx = cx + ox;
            if (g.px) bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
            else if (bx < 0 || bx >= g.nx) continue;
            const int c = by * g.nx + bx;
            f(ox, oy, __ldg(d.cell_start + c), __ldg(d.cell_start + c + 1));
        }
    }
}

// Error-free transformation a + b = s + e (Knuth two-sum), used to fold per-cell partial
// sums into compensated accumulators in the fp32 pair passes.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    float s = hi + b;
    float z = s - hi;
    float e = (hi - (s - z)) + (b - z);
    hi = s;
    lo += e;
}

__device__ __forceinline__ void set_err(const Dev &d, unsigned bits)
{
    atomicOr(&d.cnt->err, bits);
}

// Inlet velocity (u, v) at height y and time t:
//   modes:  u = U + sum_k a_k sin(k pi (y - y0) / H), v = 0;
//   pulse:  u = U + A cos(pi (y - y0) / 12) exp(-(t - t0)^2 / delta) for t0 < t < t1 (Eq.
//           velfunc2 with a decaying exponent), prm = (A, t0, t1, delta);
//   ramp:   u = U min(t / T, 1), prm = (T);
//   vortex: x_r = U (d0 - t), y_r = y - y_c, r^2 = x_r^2 + y_r^2: u = U + G y_r / (r^2 + c),
//           v = -G x_r / (r^2 + c) (Eqs. vortex, vortexx), prm = (G, c, d0, y_c).
__device__ __forceinline__ void inlet_uv(const Phys &ph, double y, double t, double &u, double &v)
{
    const double *q = ph.in_prm;
    v = 0.0;
    if (ph.in_kind == IN_PULSE) {
        u = ph.U;
        if (t > q[1] && t < q[2]) u += q[0] * cos(3.141592653589793 * (y - ph.in_y0) / 12.0) *
                                       exp(-(t - q[1]) * (t - q[1]) / q[3]);
    } else if (ph.in_kind == IN_RAMP) {
        u = ph.U * (t < q[0] ? t / q[0] : 1.0);
    } else if (ph.in_kind == IN_VORTEX) {
        const double xr = ph.U * (q[2] - t), yr = y - q[3];
        const double den = xr * xr + yr * yr + q[1];
        u = ph.U + q[0] * yr / den;
        v = -q[0] * xr / den;
    } else {
        u = ph.U;
        for (int k = 0; k < ph.n_modes; ++k)
            u += ph.modes[k] * sin((double)(k + 1) * 3.141592653589793 * (y - ph.in_y0) / ph.in_H);
    }
}

// ------------------------------------------------------------- batches in one launch
// A batched launch runs one kernel over the blocks of every member of a batch of systems:
// member m owns blocks [off[m], off[m + 1]) of the grid (members with no blocks are skipped).
// Each block finds its member, copies the member's Dev into shared memory and runs the
// single-system body with its block index and block count within the member's range, so
// that a member's results do not depend on the batch it runs in.
struct BatchGrid {
    const Dev *devs;  // [n] device copies of the members' Dev
    const int *off;   // [n + 1] block offsets of this kernel
    int n;
};

// the member that owns grid block b: the largest m with off[m] <= b
__device__ __forceinline__ int batch_member(const int *off, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class Body>
__device__ __forceinline__ void run_member(const BatchGrid &bg, Body &&body)
{
    constexpr int W = (int)(sizeof(Dev) / sizeof(int2));
    static_assert(sizeof(Dev) % sizeof(int2) == 0, "Dev copied in 8-byte words");
    __shared__ int2 sdev[W];
    __shared__ int sinfo[3];
    if (threadIdx.x == 0) {
        const int m = batch_member(bg.off, bg.n, (int)blockIdx.x);
        sinfo[0] = m;
        sinfo[1] = __ldg(bg.off + m);
        sinfo[2] = __ldg(bg.off + m + 1);
    }
    __syncthreads();
    const int2 *src = reinterpret_cast<const int2 *>(bg.devs + sinfo[0]);
    for (int i = threadIdx.x; i < W; i += blockDim.x) sdev[i] = __ldg(src + i);
    __syncthreads();
    body(*reinterpret_cast<const Dev *>(sdev), (int)blockIdx.x - sinfo[1], sinfo[2] - sinfo[1]);
}

// Grids of a batched step, one block-offset table per kernel shape.
enum : int {
    BK_CAP,      // grid-stride over the slots, 256 threads (stage, scatter, gather, recycling)
    BK_SCAN,     // one 1024-thread block per 4096 cells (scan partials)
    BK_ONE,      // one 1024-thread block (scan top, end of step)
    BK_TILES,    // one block per cell tile (mixed pair passes)
    BK_CAP128,   // grid-stride over the particles, 128 threads (fp64 pair passes)
    BK_BND,      // boundary kernel, 256 threads
    BK_MIRROR,   // mirrored outlet, 256 threads (members with that outlet only)
    BK_NUM
};
struct BatchPlan {
    int n, mixed;
    int pair_tpb;               // threads of the mixed pair passes' blocks
    const Dev *devs;            // device
    const int *off[BK_NUM];     // device, [n + 1] each
    int total[BK_NUM];          // blocks of each kernel shape over all members
    bool any_mirror;
    BatchGrid grid(int k) const { return BatchGrid{devs, off[k], n}; }
};
// blocks of one member for a kernel shape
int batch_blocks(const Dev &d, int kind);
// one step of every member of the batch (the launch sequence of a single step), on s
int launch_stage_batch(const BatchPlan &p, cudaStream_t s, int corrector);
int launch_rebuild_batch(const BatchPlan &p, cudaStream_t s);
int launch_pass_a_batch(const BatchPlan &p, cudaStream_t s);
int launch_boundary_batch(const BatchPlan &p, cudaStream_t s, int end_of_step);
int launch_pass_b_batch(const BatchPlan &p, cudaStream_t s);
int launch_recycle_batch(const BatchPlan &p, cudaStream_t s);

// ------------------------------------------------------------------- host-side launchers
// Every launcher issues its kernels on `s` and returns the number of launches issued.
// counted: the cell count was fused into the preceding stage (launch_stage with count)
int launch_rebuild(const Dev &d, cudaStream_t s, int mixed, int counted = 0);
// cell-origin tables of the gather (after the workspace is cleared)
int launch_origins(const Dev &d, cudaStream_t s);
int launch_free_stack(const Dev &d, cudaStream_t s, int n);
int launch_permute(cudaStream_t s, const void *src, int kind, const int *live, int n, double *out);
int launch_permute_id_tag(const Dev &d, cudaStream_t s, const int *live, int n,
                          unsigned long long *id, uint8_t *tag);
// probe values (p, u, v, fluid count) into d.probe_out
int launch_probe(const Dev &d, cudaStream_t s, const ProbePts &q);

// Tangent-linear model of the fp64 step (edac_tangent.cu): slot-indexed tangent fields,
// T_DIR directions (inlet modes) each, in a workspace of their own.
constexpr int T_DIR = 8;
enum : int {
    T_X, T_Y, T_U, T_V, T_UT, T_VT, T_P, T_X0, T_Y0, T_U0, T_V0, T_P0, T_RHO, T_VOL,
    T_AU, T_AV, T_AP, T_ABU, T_ABV, T_FX, T_FY, T_UBAR, T_VBAR, T_PBAR, T_J2, T_J2P, T_ADVP,
    T_J2P_OLD, T_ADVP_OLD, T_RING, T_NF = T_RING + 3 * NAVG_MAX
};
enum : int { TG_INIT, TG_PASS_A, TG_BOUNDARY, TG_PASS_B, TG_OUTLET, TG_STAGE_PRED, TG_STAGE_CORR,
             TG_RECYCLE_PRE, TG_RECYCLE_POST };
size_t tangent_bytes(const Dev &d);
// Reverse-mode adjoint of the fp64 step (edac_adjoint.cu): slot-indexed lambdas of every
// field, per-evaluation temporaries and the recorded decisions of a recomputed step, in a
// workspace of their own; one operation's adjoint kernels per launch_adjoint call.
enum : int { AJ_ZERO, AJ_PE_VALUE, AJ_PE_SEED, AJ_REC_RPOS, AJ_REC_GATE, AJ_REC_TAG, AJ_RECYCLE,
             AJ_EVAL, AJ_STAGE_CORR, AJ_STAGE_PRED, AJ_INIT, AJ_REDUCE };
// nrec: steps whose decisions are recorded at a time (a segment), rec: the one in use
size_t adjoint_bytes(const Dev &d, int nsteps, int nrec);
int launch_adjoint(const Dev &d, void *ws, int nsteps, int nrec, int rec, cudaStream_t s, int what,
                   double p0 = 0.0, double p1 = 0.0, double p2 = 0.0);
const double *adjoint_grad(const Dev &d, const void *ws, int nsteps, int nrec);
const double *adjoint_pe(const Dev &d, const void *ws, int nsteps, int nrec);
const double *tangent_hist(const Dev &d, const void *ws);
int launch_tangent(const Dev &d, void *ws, cudaStream_t s, int what, double tau);
int launch_pass_a(const Dev &d, cudaStream_t s, int mixed);
int launch_boundary(const Dev &d, cudaStream_t s, int mixed, int end_of_step);
int launch_pass_b(const Dev &d, cudaStream_t s, int mixed);
// count: the stage also takes the first step of the next cell build
int launch_stage(const Dev &d, cudaStream_t s, int mixed, int corrector, int count = 0);
int launch_recycle(const Dev &d, cudaStream_t s);
int launch_init(const Dev &d, cudaStream_t s);
int launch_neighbor_dump(const Dev &d, cudaStream_t s, int mixed, const long long *start,
                         unsigned long long *ids);

}  // namespace edac
