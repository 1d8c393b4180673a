// Pair kernels of the EDAC SPH library (sm_103a): pass A (summation density and
// number-density volume), the boundary kernel (solid-wall projection, mirrored inlet
// pressure, hybrid-outlet update) and pass B (EDAC-TVF momentum, EDAC pressure rate,
// background-pressure acceleration, solid force).
//
// Pass A and pass B run one thread per particle in cell order, in two phases: the thread
// first walks the 3x3 block of cells around its particle with the cheap membership test and
// writes the accepted neighbours (index and cell offset, 4 bytes each) to its column of a
// shared-memory list; it then evaluates the pair terms over that list only.  A warp thus
// executes the expensive pair body about max(N_i) times over its lanes instead of once per
// candidate of any lane, which is what a single fused loop costs under divergence.
// MIXED = 1 evaluates the pair terms in fp32 on cell-relative coordinates with blocked
// two-sum compensated accumulation; MIXED = 0 evaluates them in fp64 on the canonical fp64
// separations.  The boundary kernel gives each boundary particle one warp.
#include "edac.h"
#include "edac_internal.cuh"

namespace edac {

namespace {

constexpr int TPB = 128;   // threads per block of the pair passes
constexpr int LMAX = 64;   // shared-memory list entries per thread (flushed when full)

__device__ __forceinline__ void cell_of(const Dev &d, int k, int &cx, int &cy)
{
    const int c = d.cellk[k];
    cx = c % d.g.nx;
    cy = c / d.g.nx;
}

__device__ __forceinline__ unsigned enc(int j, int ox, int oy)
{
    return ((unsigned)j << 4) | ((unsigned)(ox + 1) << 2) | (unsigned)(oy + 1);
}

// Phase 1 over the 3x3 block: list the exact neighbours of particle k (itself excluded),
// calling body(entry) on the list whenever it fills and once at the end.
template <class Body>
__device__ __forceinline__ void listed_neighbors(const Dev &d, int k, double qx, double qy, int cx,
                                                 int cy, float rx, float ry, unsigned *lst, Body &body)
{
    int cnt = 0;
    for_block(d, cx, cy, [&](int ox, int oy, int j0, int j1) {
        const float rxo = rx - (float)ox * d.g.sxf, ryo = ry - (float)oy * d.g.syf;
#pragma unroll 1
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            if (j == k || !is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f)) continue;
            lst[cnt * TPB] = enc(j, ox, oy);
            if (++cnt == LMAX) {
#pragma unroll 1
                for (int c = 0; c < LMAX; ++c) body(lst[c * TPB]);
                cnt = 0;
            }
        }
    });
#pragma unroll 1
    for (int c = 0; c < cnt; ++c) body(lst[c * TPB]);
}

// ------------------------------------------------------------------ fp64 path: pass A
// S_i = sum_j W_ij, V_i = 1/S_i (number-density volume, Sec. 2), rho_i = sum_j m_j W_ij
// (Eq. summation-density), N_i = number of neighbours (self included).
struct BodyA64 {
    const Dev &d;
    double qx, qy, a2, inv_h;
    double s = 0.0, r = 0.0;
    int n = 0;
    __device__ BodyA64(const Dev &dd, double x, double y)
        : d(dd), qx(x), qy(y), a2(dd.ph.a2), inv_h(dd.ph.inv_h) {}
    __device__ void operator()(unsigned e)
    {
        const int j = (int)(e >> 4);
        const double2 xy = d.XY[j];
        double dx, dy;
        const double r2 = exact_r2(d.g, qx, qy, xy.x, xy.y, dx, dy);
        const double w = a2 * quintic_w(sqrt(r2) * inv_h);
        s += w;
        r += d.Ms[j] * w;
        ++n;
    }
};

__device__ __forceinline__ void pass_a64(const Dev &d, int bid, int nblk)
{
    __shared__ unsigned lst_all[LMAX * TPB];
    unsigned *lst = lst_all + threadIdx.x;
    const int n = d.cnt->n_alive;
    for (int k = bid * blockDim.x + threadIdx.x; k < n; k += nblk * blockDim.x) {
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pi = d.P[k];
        const double2 xy = d.XY[k];
        const int s = d.order[k];
        BodyA64 f(d, xy.x, xy.y);
        const double mk = d.Ms[k];
        const double w0 = d.ph.a2 * quintic_w(0.0);
        listed_neighbors(d, k, xy.x, xy.y, cx, cy, pi.x, pi.y, lst, f);
        const double S = f.s + w0, R = f.r + mk * w0;
        const double V = 1.0 / S;
        d.PV[k].y = V;
        d.RM[k] = make_double2(R, mk / R);
        d.snnb[k] = f.n + 1;
        d.rho[s] = R;
        d.vol[s] = V;
        d.nnb[s] = f.n + 1;
    }
}

__global__ void __launch_bounds__(TPB) k_pass_a64(Dev d) { pass_a64(d, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(TPB) k_pass_a64_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) { pass_a64(d, b, nb); });
}

// ------------------------------------------------------------------ fp64 path: pass B
// Fluid and inlet particles (rates used by the integrator):
//   a_i   = (1/m_i) sum_j c_ij [ -p~_ij gW + (A_i + A_j).gW / 2
//                                + eta~_ij u_ij (gW . r_ij) / (r_ij^2 + eta h^2) ] + g
//   dp_i  = sum_j rho_i (m_j/rho_j) c^2 u_ij . gW + (c_ij/m_i) eta~e_ij p_ij (gW.r_ij)/(r^2+eta h^2)
//   abg_i = -(p_b / m_i) sum_j c_ij gW
// (Eqs. tvf-momentum, pavg, tvf-p-ij-basa, p-edac, transport-vel), c_ij = V_i^2 + V_j^2,
// A = rho u (x) (u~ - u), eta~_ij = 2 eta_i eta_j/(eta_i + eta_j) with eta = rho nu (rho nu_edac
// for the pressure diffusion).  p~_ij is split as (pbar_ij - p_i) + (p_i - p_avg,i) with
// pbar_ij - p_i = rho_i (p_j - p_i)/(rho_i + rho_j) and p_i - p_avg,i = -sum_j (p_j - p_i)/N_i,
// so that one pass over the neighbours suffices; the second part multiplies
// G_i = sum_j c_ij gW, which is also the background-pressure sum.  The self pair contributes
// exact zeros (gW = 0, p_j - p_i = 0).
// Solid particles counted in the drag: F_i = sum_{j fluid} c_ij [ -p~_ij gW + eta~_ij
// u_ij (gW . r_ij)/(r^2 + eta h^2) ] with u_ij = u_g,i - u_j (Eq. tvf-momentum_solid), or
// with all_nb (the equation as printed) the same sum over every neighbour.
struct BodyB64 {
    const Dev &d;
    double qx, qy;
    double pi, Vi, rhoi, ui, vi, dui, dvi, mi_inv;
    bool solid, all_nb;
    double ax = 0, ay = 0, apd = 0, gxs = 0, gys = 0, sdp = 0;
    __device__ BodyB64(const Dev &dd, double x, double y) : d(dd), qx(x), qy(y) {}
    __device__ void operator()(unsigned e)
    {
        const Phys &ph = d.ph;
        const int j = (int)(e >> 4);
        const double2 pv = d.PV[j];  // (p, V)
        const double dp = pv.x - pi;
        sdp += dp;
        if (solid && !all_nb && (d.stag[j] & 0x7f) != FLUID) return;
        const double2 xy = d.XY[j];
        double dx, dy;
        const double r2 = exact_r2(d.g, qx, qy, xy.x, xy.y, dx, dy);
        const double2 rm = d.RM[j];  // (rho, m/rho)
        const double2 uv = d.UV[j];
        const double r = sqrt(r2);
        const double dwq = quintic_dw(r * ph.inv_h);
        const double F = r > 0.0 ? ph.a2h * dwq / r : 0.0;
        const double gx = F * dx, gy = F * dy, gdotr = F * r2;
        const double cij = Vi * Vi + pv.y * pv.y;
        const double inv_rs = 1.0 / (rhoi + rm.x);
        const double e_ = rhoi * dp * inv_rs;
        const double hf = rhoi * rm.x * inv_rs * gdotr / (r2 + ph.eh2);
        const double vis = 2.0 * ph.nu * hf;
        const double uij = ui - uv.x, vij = vi - uv.y;
        const double cgx = cij * gx, cgy = cij * gy;
        gxs += cgx;
        gys += cgy;
        if (solid) {
            ax += cij * (vis * uij) - e_ * cgx;
            ay += cij * (vis * vij) - e_ * cgy;
            return;
        }
        const double2 duv = d.DUV[j];
        const double Ai = rhoi * (dui * gx + dvi * gy);
        const double Aj = rm.x * (duv.x * gx + duv.y * gy);
        ax += cij * (0.5 * (ui * Ai + uv.x * Aj) + vis * uij) - e_ * cgx;
        ay += cij * (0.5 * (vi * Ai + uv.y * Aj) + vis * vij) - e_ * cgy;
        apd += rhoi * ph.c2 * rm.y * (uij * gx + vij * gy) - cij * mi_inv * 2.0 * ph.nu_e * hf * dp;
    }
};

__device__ __forceinline__ void pass_b64(const Dev &d, int bid, int nblk)
{
    __shared__ unsigned lst_all[LMAX * TPB];
    unsigned *lst = lst_all + threadIdx.x;
    const Phys &ph = d.ph;
    const int n = d.cnt->n_alive;
    for (int k = bid * blockDim.x + threadIdx.x; k < n; k += nblk * blockDim.x) {
        const int t = d.stag[k] & 0x7f;
        const bool fl = (t == FLUID || t == INLET);
        const int dm = drag_mode(ph, t);
        const bool solid = dm != 0;
        if (!fl && !solid) continue;
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pk = d.P[k];
        const double2 xy = d.XY[k];
        const int s = d.order[k];
        const int N = d.snnb[k];
        const double mi = d.m[s];
        BodyB64 f(d, xy.x, xy.y);
        const double2 pv = d.PV[k], rm = d.RM[k], uv = d.UV[k], duv = d.DUV[k];
        f.pi = pv.x; f.Vi = pv.y; f.rhoi = rm.x; f.ui = uv.x; f.vi = uv.y;
        f.dui = duv.x; f.dvi = duv.y;
        f.mi_inv = 1.0 / d.Ms[k];
        f.solid = solid;
        f.all_nb = dm == 2;
        listed_neighbors(d, k, xy.x, xy.y, cx, cy, pk.x, pk.y, lst, f);
        // -sum c p~ gW = -sum c (pbar - p_i) gW + (p_avg - p_i) G   (with p_avg) or - p_i G;
        // the solid force over its fluid neighbours takes pbar_ij itself (no p_avg shift on
        // that one-sided sum)
        const double corr = (ph.use_pavg && dm != 1) ? f.sdp / (double)N : -pv.x;
        // the sums the epilogue multiplies, kept for the reverse-mode adjoint
        d.GS[3 * (size_t)k] = f.gxs;
        d.GS[3 * (size_t)k + 1] = f.gys;
        d.GS[3 * (size_t)k + 2] = f.sdp;
        if (solid) {
            d.fx[s] = f.ax + corr * f.gxs;
            d.fy[s] = f.ay + corr * f.gys;
        } else {
            d.au[s] = (f.ax + corr * f.gxs) / mi + ph.gx;
            d.av[s] = (f.ay + corr * f.gys) / mi + ph.gy;
            d.ap[s] = f.apd;
            d.abu[s] = -ph.pb / mi * f.gxs;
            d.abv[s] = -ph.pb / mi * f.gys;
        }
    }
}

__global__ void __launch_bounds__(TPB) k_pass_b64(Dev d) { pass_b64(d, blockIdx.x, gridDim.x); }
__global__ void __launch_bounds__(TPB) k_pass_b64_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) { pass_b64(d, b, nb); });
}

// ------------------------------------------------------------------ mixed-path pair bodies
// fp32 arithmetic on the (x, y) pairs uses Blackwell's paired instructions (FADD2, FMUL2,
// FFMA2); reciprocals, square roots and inverse square roots use the single-instruction
// approximations (relative error ~2^-23).  Sums are accumulated over a few neighbours in
// fp32 and folded into two-sum compensated (hi, lo) accumulators (see for_wmask; once per
// cell row in the other walks).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(0) = 0 exactly, so pass A's self term needs no guard (measured: pass A 0.162 -> 0.156 ms
// per launch at 1.51M particles against r^2 times the guarded inverse square root)
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }

__device__ __forceinline__ void two_sum_acc2(float2 &hi, float2 &lo, float2 b)
{
    const float2 s = __fadd2_rn(hi, b);
    const float2 z = __fadd2_rn(s, f2(-hi.x, -hi.y));
    const float2 e = __fadd2_rn(__fadd2_rn(hi, f2(-(s.x - z.x), -(s.y - z.y))),
                                __fadd2_rn(b, f2(-z.x, -z.y)));
    hi = s;
    lo = __fadd2_rn(lo, e);
}

// r >= 0 from r^2, guarded so that coincident particles (r^2 = 0) give q ~ 0 where the kernel
// derivative vanishes exactly: r^2 is raised to 1e-30 before the inverse square root.
__device__ __forceinline__ float inv_r_of(float r2) { return rsqrt_approx(fmaxf(r2, 1e-30f)); }

// w(q) and dw/dq of the quintic spline with t_k = max(k - q, 0) (see quintic_w/quintic_dw)
__device__ __forceinline__ float w_fast(float q)
{
    const float t3 = fmaxf(3.f - q, 0.f), t2 = fmaxf(2.f - q, 0.f), t1 = fmaxf(1.f - q, 0.f);
    const float2 s32 = __fmul2_rn(f2(t3, t2), f2(t3, t2));
    const float2 q32 = __fmul2_rn(s32, s32);
    const float2 p32 = __fmul2_rn(q32, f2(t3, t2));
    const float s1 = t1 * t1;
    return fmaf(15.f, s1 * s1 * t1, fmaf(-6.f, p32.y, p32.x));
}

__device__ __forceinline__ float dw_fast(float q)
{
    const float t3 = fmaxf(3.f - q, 0.f), t2 = fmaxf(2.f - q, 0.f), t1 = fmaxf(1.f - q, 0.f);
    const float2 s32 = __fmul2_rn(f2(t3, t2), f2(t3, t2));
    const float2 q32 = __fmul2_rn(s32, s32);
    const float s1 = t1 * t1;
    return -5.f * fmaf(15.f, s1 * s1, fmaf(-6.f, q32.y, q32.x));
}

// Pass A: sum of w(q_ij) and of m_j w(q_ij) over the neighbours (self included); alpha_2 is
// applied once at the end.
struct MixA {
    float inv_h;
    float s = 0.f, r = 0.f;
    float2 hi = f2(0.f, 0.f), lo = f2(0.f, 0.f);  // (sum w, sum m w)
    int n = 0;
    __device__ __forceinline__ void add(float2 dd, float mj)
    {
        const float r2 = fmaf(dd.x, dd.x, dd.y * dd.y);
        const float w = w_fast(sqrt_approx(r2) * inv_h);
        s += w;
        r = fmaf(mj, w, r);
        ++n;
    }
    __device__ __forceinline__ void fold()
    {
        two_sum_acc2(hi, lo, f2(s, r));
        s = r = 0.f;
    }
};

// Pass B body for a fluid / inlet particle i (SOLID = false) or a solid particle counted in
// the drag (SOLID = true: fluid neighbours only unless all_nb, no A-term, no pressure rate).
template <bool SOLID>
struct MixB {
    bool all_nb = false;
    // i-side constants
    float2 ui;       // (u_i, v_i)
    float2 rdi;      // rho_i (u~_i - u_i, v~_i - v_i)
    float pi, Vi2, rhoi, rhoic2, dif;  // dif = 2 nu_edac / m_i
    float a2h, inv_h, nu2, eh2;
    // per-row partial sums and compensated totals
    float2 am = f2(0.f, 0.f), gg = f2(0.f, 0.f);
    float ap = 0.f, sdp = 0.f;
    float2 am_h = f2(0.f, 0.f), am_l = f2(0.f, 0.f), gg_h = f2(0.f, 0.f), gg_l = f2(0.f, 0.f);
    float2 ap_hl = f2(0.f, 0.f);
    // dd = r_i - r_j; q = (p, V, rho, m/rho); b = (u, v, u~-u, v~-v) of j
    __device__ __forceinline__ void add(float2 dd, const float4 &q, const float4 &b, uint8_t tagj)
    {
        const float dp = q.x - pi;
        sdp += dp;
        if (SOLID && !all_nb && (tagj & 0x7f) != FLUID) return;
        const float r2 = fmaf(dd.x, dd.x, dd.y * dd.y);
        const float ir = inv_r_of(r2);
        const float F = a2h * dw_fast(r2 * ir * inv_h) * ir;   // gW = F r_ij
        const float2 g = __fmul2_rn(f2s(F), dd);
        const float gdotr = F * r2;
        const float cij = fmaf(q.y, q.y, Vi2);
        const float wi = rhoi * rcp_approx(rhoi + q.z);        // rho_i / (rho_i + rho_j)
        const float e = wi * dp;                                // pbar_ij - p_i
        const float hf = wi * q.z * gdotr * rcp_approx(r2 + eh2);
        const float2 uij = __fadd2_rn(ui, f2(-b.x, -b.y));
        const float2 cg = __fmul2_rn(f2s(cij), g);
        gg = __fadd2_rn(gg, cg);
        float2 mom = __fmul2_rn(f2s(nu2 * hf), uij);            // viscous term
        if (!SOLID) {
            const float Ai = fmaf(rdi.x, g.x, rdi.y * g.y);      // A_i . gW / u_i
            const float Aj = q.z * fmaf(b.z, g.x, b.w * g.y);    // A_j . gW / u_j
            const float2 A = __ffma2_rn(f2(b.x, b.y), f2s(Aj), __fmul2_rn(ui, f2s(Ai)));
            mom = __ffma2_rn(f2s(0.5f), A, mom);
            const float div = fmaf(uij.x, g.x, uij.y * g.y);
            ap = fmaf(rhoic2 * q.w, div, ap);
            ap = fmaf(-cij * dif * hf, dp, ap);
        }
        am = __ffma2_rn(f2s(cij), mom, am);
        am = __ffma2_rn(f2s(-e), cg, am);
    }
    __device__ __forceinline__ void fold()
    {
        two_sum_acc2(am_h, am_l, am);
        two_sum_acc2(gg_h, gg_l, gg);
        float s = ap_hl.x + ap, z = s - ap_hl.x;
        ap_hl.y += (ap_hl.x - (s - z)) + (ap - z);
        ap_hl.x = s;
        am = gg = f2(0.f, 0.f);
        ap = 0.f;
    }
};

// ------------------------------------------------------------ cell-tiled mixed passes
// A block owns a row segment of d.tile_tx (at most CT_TX) cells; its d.tile_tpb threads (at
// most CT_TPB; both set by edac_set_tiling or the autotuner).  It stages the particles of the
// 3 x (cells + 2) cells around the segment into shared memory once (positions relative to the
// tile origin, fields of the pass), then each thread takes one particle of the segment.
// Every staged row is x-sorted, so a particle's candidates in a row are a window of x (two
// binary searches).  Pass A tests the windows' candidates, sums its pair terms in the same
// loop and records the neighbours as a 64-bit mask per row window; pass B iterates the set
// bits of those masks instead of repeating the membership test.  Compensated sums are
// folded once per row window in pass A and as for_wmask says in pass B.  A tile whose halo
// exceeds CT_HMAX particles is processed from global
// memory instead (same membership test, same pair arithmetic), and a particle with a window
// of more than 64 candidates repeats the test in pass B.
constexpr int CT_TX = 16;         // most cells of a tile (default 11: ~143 particles at 13 a cell)
constexpr int CT_NV = CT_TX + 2;  // cells per staged row (halo included)
constexpr int CT_TPB = 256;       // most threads of a tile block
constexpr int CT_HMAX = 768;      // staged particles (11 cells: ~3 x 13 x 13 = 507)
static_assert(CT_TX == EDAC_TILE_MAX_CELLS && CT_TPB == EDAC_TILE_MAX_THREADS,
              "tiling limits of header and kernels");

struct TileHdr {
    int cstart[3][CT_NV + 1];  // shared index of each staged cell's first particle
    int gstart[3][CT_NV];      // global index of that particle (-1: no such cell)
    int H, i0, ni;
    uint8_t cell[CT_HMAX];     // staged cell (r CT_NV + v) of each staged particle
};

// Global index of staged particle t (tiles that fit).
__device__ __forceinline__ int staged_j(const TileHdr &th, int t)
{
    const int c = th.cell[t], r = c / CT_NV, v = c - r * CT_NV;
    return th.gstart[r][v] + (t - th.cstart[r][v]);
}

// Warp 0 builds the header: lane l takes staged cells l and l + 32 (cell index r CT_NV + v),
// and a warp scan of the cell counts gives the shared-memory offsets.
__device__ __forceinline__ void tile_cell(const Dev &d, int cx0, int cy, int txe, int cell, int &a,
                                          int &cnt)
{
    const Geo &g = d.g;
    const int r = cell / CT_NV, v = cell - r * CT_NV;
    bool ok = cell < 3 * CT_NV && v <= txe + 1;
    int by = cy + r - 1, bx = cx0 + v - 1;
    if (g.py) by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
    else ok = ok && by >= 0 && by < g.ny;
    if (g.px) bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
    else ok = ok && bx >= 0 && bx < g.nx;
    a = -1;
    cnt = 0;
    if (ok) {
        const int c = by * g.nx + bx;
        a = d.cell_start[c];
        cnt = d.cell_start[c + 1] - a;
    }
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

__device__ __forceinline__ void tile_setup(const Dev &d, int cx0, int cy, TileHdr &th)
{
    static_assert(3 * CT_NV <= 64, "tile header: at most two cells per lane");
    const int lane = threadIdx.x & 31;
    const int txe = min(d.tile_tx, d.g.nx - cx0);  // cells of this segment
    int a0, n0, a1, n1;
    tile_cell(d, cx0, cy, txe, lane, a0, n0);
    tile_cell(d, cx0, cy, txe, lane + 32, a1, n1);
    const int i0s = warp_incl_scan(n0, lane);
    const int tot0 = __shfl_sync(0xffffffffu, i0s, 31);
    const int i1s = warp_incl_scan(n1, lane) + tot0;
    const int cells[2] = {lane, lane + 32};
    const int incl[2] = {i0s, i1s}, cnt[2] = {n0, n1}, aa[2] = {a0, a1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int cell = cells[h];
        if (cell < 3 * CT_NV) {
            const int r = cell / CT_NV, v = cell - r * CT_NV;
            th.cstart[r][v] = incl[h] - cnt[h];
            th.gstart[r][v] = aa[h];
            if (v == CT_NV - 1) th.cstart[r][CT_NV] = incl[h];
        }
    }
    // the segment's own cells are row 1, v = 1..txe
    const int lo_cell = CT_NV + 1, hi_cell = CT_NV + txe;
    const int own_lo = lo_cell < 32 ? __shfl_sync(0xffffffffu, i0s - n0, lo_cell)
                                    : __shfl_sync(0xffffffffu, i1s - n1, lo_cell - 32);
    const int own_hi = __shfl_sync(0xffffffffu, hi_cell < 32 ? i0s : i1s, hi_cell & 31);
    const int i0 = lo_cell < 32 ? __shfl_sync(0xffffffffu, a0, lo_cell)
                                : __shfl_sync(0xffffffffu, a1, lo_cell - 32);
    const int last = 3 * CT_NV - 1;
    const int H = __shfl_sync(0xffffffffu, last < 32 ? i0s : i1s, last & 31);
    if (H <= CT_HMAX) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (cells[h] < 3 * CT_NV)
                for (int t = incl[h] - cnt[h]; t < incl[h]; ++t) th.cell[t] = (uint8_t)cells[h];
    }
    if (lane == 0) {
        th.H = H;
        th.i0 = i0;
        th.ni = own_hi - own_lo;
    }
}

// Stage positions relative to the tile origin (lower-left corner of cell (cx0, cy)):
// x = (x - cell x0) + (v - 1) sx, y likewise.  The H staged particles are taken flat (staged
// index t -> its cell from the header's table, then its global index), SB of them per thread
// at a time with all their loads issued before the first store: a warp keeps SB x (loads
// per particle) requests in flight with every lane busy, where one warp per cell kept ~13
// lanes and one cell's loads.
// load(j) fetches the pass's fields of particle j, store(t, fields, P_j, v) writes them (v:
// the staged cell's column, 0 .. CT_NV - 1).
template <int SB, class Load, class Store>
__device__ __forceinline__ void tile_stage(const Dev &d, const TileHdr &th, float2 *spos,
                                           Load &&load, Store &&store)
{
    using T = decltype(load(0));
    const int H = th.H;
    for (int base = threadIdx.x; base < H; base += SB * blockDim.x) {
        int jj[SB], vv[SB];
        float2 oo[SB];
        float4 pp[SB];
        T ff[SB];
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int t = base + u * blockDim.x;
            jj[u] = -1;
            if (t < H) {
                const int cell = th.cell[t], r = cell / CT_NV, v = cell - r * CT_NV;
                const int j = th.gstart[r][v] + (t - th.cstart[r][v]);
                jj[u] = j;
                vv[u] = v;
                oo[u] = make_float2((float)(v - 1) * d.g.sxf, (float)(r - 1) * d.g.syf);
                pp[u] = d.P[j];
                ff[u] = load(j);
            }
        }
#pragma unroll
        for (int u = 0; u < SB; ++u) {
            const int t = base + u * blockDim.x;
            if (jj[u] >= 0) {
                spos[t] = make_float2(pp[u].x + oo[u].x, pp[u].y + oo[u].y);
                store(t, ff[u], pp[u], vv[u]);
            }
        }
    }
}

// Candidate windows of a staged particle in virtual cell vi.  Every staged row is x-sorted
// (its cells in x order, a cell's particles by x), so the candidates of row r (0: the row
// below, 1: the particle's own, 2: the row above) that can lie within 3h of the particle form
// the window of staged x within the row's reach of the particle's x: 3h in its own row,
// sqrt((3h)^2 - dy^2) in the others, dy the distance to that row's nearer edge.  A margin of
// 1e-4 of 3h on every bound keeps the windows supersets of the neighbour sets (the staged
// fp32 coordinates are within ~1e-7 of the exact ones, and a row's x can step back by one
// ulp across a cell boundary).  The exact membership test runs on the windows only: about
// 67 candidates instead of the 3 x 3 block's 117.
constexpr int WMAX = 64;  // candidates of a row window held in one 64-bit mask word

struct Win {
    int lo[3], n[3];  // first shared index and length of each row's window
};

// first t in [a, b) with spos[t].x > xv
__device__ __forceinline__ int first_above(const float2 *spos, int a, int b, float xv)
{
    while (a < b) {
        const int m = (a + b) >> 1;
        if (spos[m].x > xv) b = m;
        else a = m + 1;
    }
    return a;
}

__device__ __forceinline__ Win windows(const Dev &d, const TileHdr &th, const float2 *spos, int vi,
                                       float2 pi)
{
    const float rc2 = d.g.rc2_hi;
    // square roots by the approximate inverse square root (relative error ~2^-22, far inside
    // the margin of 1e-4 of 3h that keeps the windows supersets)
    const float mrg = 1e-4f * rc2 * rsqrt_approx(rc2);
    const float sy = d.g.syf;
    Win w;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int a = th.cstart[r][vi - 1], b = th.cstart[r][vi + 2];
        const float dy0 = r == 1 ? 0.0f : (r == 0 ? pi.y : sy - pi.y);
        const float dy = fmaxf(dy0 - mrg, 0.0f);
        const float reach2 = rc2 - dy * dy;
        if (!(reach2 > 0.0f)) {
            w.lo[r] = a;
            w.n[r] = 0;
            continue;
        }
        const float reach = reach2 * rsqrt_approx(reach2) + mrg;
        // the window starts in cell vi - 1 or vi (or at the start of vi + 1 when those hold
        // nothing within reach) and ends after cell vi - 1: the cells are at least 3h wide
        const int lo = first_above(spos, a, th.cstart[r][vi + 1], pi.x - reach);
        const int hi = first_above(spos, max(lo, th.cstart[r][vi]), b, pi.x + reach);
        w.lo[r] = lo;
        w.n[r] = hi - lo;
    }
    return w;
}

// The neighbour mask of a particle over its windows, kept from pass A for pass B: a 64-bit
// word per row window and the windows' first shared indices; over: some window held more
// than WMAX candidates, and both passes test the windows' candidates directly.
struct WMask {
    unsigned long long m[3];
    int lo[3];
    bool over;
};

__device__ __forceinline__ void store_wmask(uint4 *nbm, int k, const WMask &w)
{
    nbm[2 * (size_t)k] = make_uint4((unsigned)w.m[0], (unsigned)(w.m[0] >> 32), (unsigned)w.m[1],
                                    (unsigned)(w.m[1] >> 32));
    nbm[2 * (size_t)k + 1] = make_uint4((unsigned)w.m[2], (unsigned)(w.m[2] >> 32),
                                        (unsigned)w.lo[0] | ((unsigned)w.lo[1] << 16),
                                        (unsigned)w.lo[2] | ((unsigned)w.over << 16));
}

__device__ __forceinline__ WMask load_wmask(const uint4 *nbm, int k)
{
    const uint4 a = nbm[2 * (size_t)k], b = nbm[2 * (size_t)k + 1];
    WMask w;
    w.m[0] = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
    w.m[1] = (unsigned long long)a.z | ((unsigned long long)a.w << 32);
    w.m[2] = (unsigned long long)b.x | ((unsigned long long)b.y << 32);
    w.lo[0] = (int)(b.z & 0xffffu);
    w.lo[1] = (int)(b.z >> 16);
    w.lo[2] = (int)(b.w & 0xffffu);
    w.over = (b.w >> 16) != 0u;
    return w;
}

__device__ __forceinline__ int tile_of_block(const Dev &d, int bid, int &cx0, int &cy)
{
    const int tpr = (d.g.nx + d.tile_tx - 1) / d.tile_tx;
    cy = bid / tpr;
    cx0 = (bid - cy * tpr) * d.tile_tx;
    return cy < d.g.ny;
}

// Global-memory walk for tiles whose halo does not fit: f(dd, j) over the neighbours of k
// (itself included), folding after each row of cells.
template <class F, class Fold>
__device__ __forceinline__ void global_neighbors(const Dev &d, int k, const float4 &pk, double qx,
                                                 double qy, F &&f, Fold &&fold)
{
    const int c = d.cellk[k];
    const int cx = c % d.g.nx, cy = c / d.g.nx;
    for_block(d, cx, cy, [&](int ox, int oy, int j0, int j1) {
        const float rxo = pk.x - (float)ox * d.g.sxf, ryo = pk.y - (float)oy * d.g.syf;
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            const float4 pj = __ldg(d.P + j);
            if (!is_member(d, rxo, ryo, pj, j, qx, qy, dxf, dyf, r2f)) continue;
            f(make_float2(dxf, dyf), j, pj);
        }
        if (ox == 1) fold();
    });
    fold();
}

// Pass A over the windows in one loop: for every window candidate the mask bits (a tentative
// bit: r^2 below the upper band edge, the sign of r^2 - hi2; a band bit: above the lower
// edge, the sign of lo2 - r^2; shifted in with one funnel shift each) and w(q), m w(q) added
// to the sums.  The branch-free quintic is exactly zero for q >= 3, so a candidate outside
// the support adds nothing, and one inside the fp32 band but outside the exact support adds
// w(q) with 3 - q < 1e-4, below 1e-20 of w(0), which the fp32 sums cannot hold: the sums
// equal those over the neighbours, and the loop's trip count does not depend on membership.
// The fp64 test settles the band candidates after the loop (kept out of it, so that it is
// not compiled to predicated fp64 work on every candidate).  The sums are folded into the
// compensated accumulators once per row.
__device__ __forceinline__ WMask pass_a_windows(const Dev &d, int k, const float2 *spos,
                                                const float *smass, const TileHdr &th, const Win &wn,
                                                float2 pi, MixA &f)
{
    const float hi2 = d.g.rc2_hi, lo2 = d.g.rc2_lo, inv_h = f.inv_h;
    WMask wm;
    wm.over = false;
    unsigned long long band[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        wm.lo[r] = wn.lo[r];
        unsigned word[2], bword[2];
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            const int c0 = 32 * hf, cnt = min(32, wn.n[r] - c0);
            unsigned cur = 0u, bcur = 0u;
            const int t0 = wn.lo[r] + c0;
#pragma unroll 4  // measured: 1 0.175, 2 0.166, 4 0.162, 6 0.168, 8 0.171 ms at D/100
            for (int c = 0; c < cnt; ++c) {
                const int t = t0 + c;
                const float2 pj = spos[t];
                const float2 dd = __fadd2_rn(pi, f2(-pj.x, -pj.y));
                const float r2 = fmaf(dd.x, dd.x, dd.y * dd.y);
                cur = __funnelshift_l(__float_as_uint(r2 - hi2), cur, 1);
                bcur = __funnelshift_l(__float_as_uint(lo2 - r2), bcur, 1);
                const float w = w_fast(sqrt_approx(r2) * inv_h);
                f.s += w;
                f.r = fmaf(smass[t], w, f.r);
            }
            word[hf] = cnt > 0 ? __brev(cur) >> (32 - cnt) : 0u;
            bword[hf] = cnt > 0 ? __brev(bcur) >> (32 - cnt) : 0u;
        }
        f.fold();
        wm.m[r] = (unsigned long long)word[0] | ((unsigned long long)word[1] << 32);
        band[r] = wm.m[r] & ((unsigned long long)bword[0] | ((unsigned long long)bword[1] << 32));
    }
    if (band[0] | band[1] | band[2]) {
        const double2 q = d.XY[k];  // the particle's fp64 position, for the band candidates only
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            unsigned long long bw = band[r];
#pragma unroll 1
            while (bw) {
                const int b = __ffsll((long long)bw) - 1;
                bw &= bw - 1ull;
                const double2 xy = d.XY[staged_j(th, wn.lo[r] + b)];
                double ex, ey;
                if (!(exact_r2(d.g, q.x, q.y, xy.x, xy.y, ex, ey) < d.g.rc2)) wm.m[r] &= ~(1ull << b);
            }
        }
    }
    f.n = __popcll(wm.m[0]) + __popcll(wm.m[1]) + __popcll(wm.m[2]);
    return wm;
}

// The candidates of the windows with the membership test (windows over WMAX candidates):
// body(t) over the neighbours, fold() after each row.
template <class Body, class Fold>
__device__ __forceinline__ void windows_tested(const Dev &d, const float2 *spos, const TileHdr &th,
                                               const Win &wn, float2 pi, double qx, double qy,
                                               Body &&body, Fold &&fold)
{
#pragma unroll 1
    for (int r = 0; r < 3; ++r) {
#pragma unroll 1
        for (int t = wn.lo[r]; t < wn.lo[r] + wn.n[r]; ++t) {
            const float2 pj = spos[t];
            const float2 dd = __fadd2_rn(pi, f2(-pj.x, -pj.y));
            const float r2 = fmaf(dd.x, dd.x, dd.y * dd.y);
            if (r2 >= d.g.rc2_hi) continue;
            if (r2 > d.g.rc2_lo) {
                const double2 xj = d.XY[staged_j(th, t)];
                double ex, ey;
                if (!(exact_r2(d.g, qx, qy, xj.x, xj.y, ex, ey) < d.g.rc2)) continue;
            }
            body(t);
        }
        fold();
    }
}

// Run body(t) over the set bits of a window mask (shared indices t), with one leading-zero
// count and one exclusive-or per neighbour on 32-bit words, highest bit first.  The particle's
// own row first, its two halves one after the other, then a fold; then the rows below and
// above in one walk, the next word taken when one runs out, with a fold every 16 terms and at
// the end (where the warp's lanes have reconverged).  The own row's neighbour count varies
// little between the lanes of a warp; the rows below and above vary with the particle's
// height in its cell, in opposite directions, so their sum varies little too: walking those
// two rows separately left 30% of the lanes idle.  (Pass B at D/100: 0.252 -> 0.221 ms.)
template <class Body, class Fold>
__device__ __forceinline__ void for_wmask(const WMask &m, Body &&body, Fold &&fold)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned w = (unsigned)(m.m[1] >> (32 * h));
        const int base = m.lo[1] + 32 * h;
#pragma unroll 2
        while (w) {
            const int b = 31 - __clz(w);
            w ^= 1u << b;
            body(base + b);
        }
    }
    fold();
    unsigned w0 = (unsigned)m.m[0], w1 = (unsigned)(m.m[0] >> 32), w2 = (unsigned)m.m[2],
             w3 = (unsigned)(m.m[2] >> 32);
    int b0 = m.lo[0], b1 = m.lo[0] + 32, b2 = m.lo[2], b3 = m.lo[2] + 32;
    const int n = __popcll(m.m[0]) + __popcll(m.m[2]);
#pragma unroll 2
    for (int it = 0; it < n; ++it) {
        while (w0 == 0u) {
            w0 = w1; w1 = w2; w2 = w3; w3 = 0u;
            b0 = b1; b1 = b2; b2 = b3;
        }
        const int b = 31 - __clz(w0);
        w0 ^= 1u << b;
        body(b0 + b);
        if ((it & 15) == 15) fold();
    }
    fold();
}

__device__ __forceinline__ void pass_a_tiled(const Dev &d, int bid)
{
    __shared__ TileHdr th;
    __shared__ float2 spos[CT_HMAX];
    __shared__ float smass[CT_HMAX];
    int cx0, cy;
    if (!tile_of_block(d, bid, cx0, cy)) return;
    if (threadIdx.x < 32) tile_setup(d, cx0, cy, th);
    __syncthreads();
    const bool fits = th.H <= CT_HMAX;
    if (fits)
        tile_stage<4>(d, th, spos, [](int) { return 0; },
                      [&](int t, int, const float4 &pj, int) { smass[t] = pj.z; });
    __syncthreads();
    const float a2 = d.ph.a2f;
    for (int ii = threadIdx.x; ii < th.ni; ii += blockDim.x) {
        const int k = th.i0 + ii;
        // the epilogue's loads first: their latency passes during the pair loop
        const int s = d.order[k];
        const float pk_p = d.P[k].w;
        float mk;
        MixA f;
        f.inv_h = d.ph.inv_hf;
        if (fits) {
            const int ti = th.cstart[1][1] + ii;
            mk = smass[ti];
            const int vi = th.cell[ti] - CT_NV;  // the own row's cells are row 1
            const float2 pi = spos[ti];
            const Win wn = windows(d, th, spos, vi, pi);
            if (wn.n[0] <= WMAX && wn.n[1] <= WMAX && wn.n[2] <= WMAX) {
                // the neighbour mask over the windows (also pass B's input) and the sums
                store_wmask(d.nbm, k, pass_a_windows(d, k, spos, smass, th, wn, pi, f));
            } else {
                const double2 xy = d.XY[k];
                windows_tested(d, spos, th, wn, pi, xy.x, xy.y,
                               [&](int t) {
                                   const float2 pj = spos[t];
                                   f.add(__fadd2_rn(pi, f2(-pj.x, -pj.y)), smass[t]);
                               },
                               [&]() { f.fold(); });
                WMask wm;
                wm.m[0] = wm.m[1] = wm.m[2] = 0ull;
                wm.lo[0] = wm.lo[1] = wm.lo[2] = 0;
                wm.over = true;
                store_wmask(d.nbm, k, wm);
            }
        } else {
            const float4 pk = d.P[k];
            const double2 xy = d.XY[k];
            mk = pk.z;
            global_neighbors(d, k, pk, xy.x, xy.y,
                             [&](float2 dd, int, const float4 &pj) { f.add(dd, pj.z); },
                             [&]() { f.fold(); });
        }
        const float S = a2 * (f.hi.x + f.lo.x), R = a2 * (f.hi.y + f.lo.y);
        const float V = 1.0f / S;
        d.Qf[k] = make_float4(pk_p, V, R, mk / R);
        d.snnb[k] = f.n;
        d.rho[s] = f2d(R);
        d.vol[s] = f2d(V);
        d.nnb[s] = f.n;
    }
}

__global__ void __launch_bounds__(CT_TPB) k_pass_a_tiled(Dev d) { pass_a_tiled(d, blockIdx.x); }
__global__ void __launch_bounds__(CT_TPB) k_pass_a_tiled_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int) { pass_a_tiled(d, b); });
}

template <bool SOLID>
__device__ __forceinline__ void pass_b_particle(const Dev &d, const TileHdr &th, bool fits, int cy,
                                                int cx0, int ii, const float2 *spos, const float4 *sq,
                                                const float4 *sb, const uint8_t *stg)
{
    const Phys &ph = d.ph;
    const int k = th.i0 + ii;
    const int ti = th.cstart[1][1] + ii;
    // global loads first (the epilogue's included), so that their latency passes together;
    // the particle's own fields come from the staged copy when the tile fits
    const float mk = d.P[k].z;
    const int N = d.snnb[k];
    const int s = d.order[k];
    const float4 q = fits ? sq[ti] : d.Qf[k];
    const float4 b = fits ? sb[ti] : d.Bf[k];
    MixB<SOLID> f;
    if (SOLID) f.all_nb = drag_mode(ph, d.stag[k] & 0x7f) == 2;
    f.ui = f2(b.x, b.y);
    f.rdi = f2(q.z * b.z, q.z * b.w);
    f.pi = q.x; f.Vi2 = q.y * q.y; f.rhoi = q.z; f.rhoic2 = q.z * ph.c2f;
    f.dif = 2.0f * ph.nuef / mk;
    f.a2h = ph.a2hf; f.inv_h = ph.inv_hf; f.nu2 = 2.0f * ph.nuf; f.eh2 = ph.eh2f;
    if (fits) {
        const float2 pi = spos[ti];
        auto body = [&](int tj) {
            const float2 pj = spos[tj];
            f.add(__fadd2_rn(pi, f2(-pj.x, -pj.y)), sq[tj], sb[tj], stg[tj]);
        };
        WMask wm = load_wmask(d.nbm, k);
        if (!wm.over) {
            // the neighbours pass A found, as set bits of the windows, less the particle
            // itself (its pair terms are exact zeros: gW = 0, p_j - p_i = 0)
            const int cs = ti - wm.lo[1];
            if (cs >= 0 && cs < WMAX) wm.m[1] &= ~(1ull << cs);
            for_wmask(wm, body, [&]() { f.fold(); });
        } else {
            const double2 xy = d.XY[k];
            const int vi = d.cellk[k] - cy * d.g.nx - cx0 + 1;
            const Win wn = windows(d, th, spos, vi, pi);
            windows_tested(d, spos, th, wn, pi, xy.x, xy.y,
                           [&](int tj) {
                               if (tj != ti) body(tj);
                           },
                           [&]() { f.fold(); });
        }
    } else {
        const float4 pk = d.P[k];
        const double2 xy = d.XY[k];
        global_neighbors(d, k, pk, xy.x, xy.y,
                         [&](float2 dd, int j, const float4 &) {
                             f.add(dd, __ldg(d.Qf + j), __ldg(d.Bf + j), d.stag[j]);
                         },
                         [&]() { f.fold(); });
    }
    // fp32 epilogue (the fp64 pipe of this part is a small fraction of the fp32 one): only the
    // stores of the fp64 rate arrays convert
    const float sx = f.am_h.x + f.am_l.x, sy = f.am_h.y + f.am_l.y;
    const float G0 = f.gg_h.x + f.gg_l.x, G1 = f.gg_h.y + f.gg_l.y;
    // -sum c p~ gW = -sum c (pbar - p_i) gW + (p_avg - p_i) G   (with p_avg) or - p_i G;
    // the solid force over its fluid neighbours takes pbar_ij itself (no p_avg shift on
    // that one-sided sum)
    const float corr = (ph.use_pavg && (!SOLID || f.all_nb)) ? f.sdp / (float)N : -q.x;
    if (SOLID) {
        d.fx[s] = f2d(fmaf(corr, G0, sx));
        d.fy[s] = f2d(fmaf(corr, G1, sy));
    } else {
        const float mi_inv = 1.0f / mk;
        rate_f(d.au)[s] = fmaf(fmaf(corr, G0, sx), mi_inv, ph.gxf);
        rate_f(d.av)[s] = fmaf(fmaf(corr, G1, sy), mi_inv, ph.gyf);
        rate_f(d.ap)[s] = f.ap_hl.x + f.ap_hl.y;
        const float pbm = -ph.pbf * mi_inv;
        rate_f(d.abu)[s] = pbm * G0;
        rate_f(d.abv)[s] = pbm * G1;
    }
}

constexpr int PB_SB = 2;  // staged particles per thread per round in pass B (registers)

__device__ __forceinline__ void pass_b_tiled(const Dev &d, int bid)
{
    __shared__ TileHdr th;
    __shared__ float2 spos[CT_HMAX];
    __shared__ float4 sq[CT_HMAX];
    __shared__ float4 sb[CT_HMAX];
    __shared__ uint8_t stg[CT_HMAX];
    const Phys &ph = d.ph;
    int cx0, cy;
    if (!tile_of_block(d, bid, cx0, cy)) return;
    if (threadIdx.x < 32) tile_setup(d, cx0, cy, th);
    __syncthreads();
    const bool fits = th.H <= CT_HMAX;
    struct Fields {
        float4 q, b;
        uint8_t tag;
    };
    if (fits)
        tile_stage<PB_SB>(
            d, th, spos, [&](int j) { return Fields{d.Qf[j], d.Bf[j], d.stag[j]}; },
            [&](int t, const Fields &f, const float4 &, int) {
                sq[t] = f.q;
                sb[t] = f.b;
                stg[t] = f.tag;
            });
    __syncthreads();
    for (int ii = threadIdx.x; ii < th.ni; ii += blockDim.x) {
        const int t = (fits ? stg[th.cstart[1][1] + ii] : d.stag[th.i0 + ii]) & 0x7f;
        if (t == FLUID || t == INLET)
            pass_b_particle<false>(d, th, fits, cy, cx0, ii, spos, sq, sb, stg);
        else if (drag_mode(ph, t))
            pass_b_particle<true>(d, th, fits, cy, cx0, ii, spos, sq, sb, stg);
    }
}

__global__ void __launch_bounds__(CT_TPB, 4) k_pass_b_tiled(Dev d) { pass_b_tiled(d, blockIdx.x); }
__global__ void __launch_bounds__(CT_TPB) k_pass_b_tiled_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int) { pass_b_tiled(d, b); });
}

// --------------------------------------------------------------------- boundary kernel
// One warp per boundary particle: the lanes share the candidates of the 3x3 block, each
// keeps partial sums, and a butterfly reduction combines them.
template <class T, int NA>
__device__ __forceinline__ void warp_sum(T (&a)[NA])
{
#pragma unroll
    for (int i = 0; i < NA; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
    }
}

// Reduce-scatter of NA <= 16 fp64 values (zero-padded to 16) over the warp: in each round a
// lane sends half of its values to lane ^ o and adds the half it receives, the last round
// (o = 1) being a plain exchange.  On return lane L holds the warp total of value L >> 1.
// The totals equal warp_sum's bit for bit (the same pairs are added in the same tree, and
// fp addition is commutative), at 16 additions per lane instead of 5 NA: on GB300 the fp64
// pipe runs at 1/64 of the fp32 rate, which makes the fp64 butterfly of the mirror's sums its
// largest cost.
template <int N>
__device__ __forceinline__ void rs_round(double (&v)[16], int o, bool up)
{
    constexpr int M = N / 2;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const double send = up ? v[j] : v[j + M];
        const double keep = up ? v[j + M] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

template <int NA>
__device__ __forceinline__ double warp_reduce_scatter16(const double (&a)[NA], int lane)
{
    static_assert(NA <= 16, "at most 16 values");
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < NA ? a[i] : 0.0;
    rs_round<16>(v, 16, lane & 16);
    rs_round<8>(v, 8, lane & 8);
    rs_round<4>(v, 4, lane & 4);
    rs_round<2>(v, 2, lane & 2);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Lane-strided walk of the neighbours of a query point: f(j, dx, dy, r2) with the pair
// geometry in T (fp32 cell-relative for the mixed path, canonical fp64 otherwise).
template <int MIXED, class F>
__device__ __forceinline__ void lane_neighbors(const Dev &d, int lane, double qx, double qy, int cx,
                                               int cy, float rx, float ry, F &&f)
{
    // lanes 0..8 look up the 9 cells of the block; a warp scan concatenates their ranges so
    // that the 32 lanes share the candidates evenly instead of walking cell after cell
    const Geo &g = d.g;
    int a = 0, cnt = 0;
    if (lane < 9) {
        const int oy = lane / 3 - 1, ox = lane % 3 - 1;
        int by = cy + oy, bx = cx + ox;
        bool ok = true;
        if (g.py) by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
        else ok = by >= 0 && by < g.ny;
        if (g.px) bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
        else ok = ok && bx >= 0 && bx < g.nx;
        if (ok) {
            const int c = by * g.nx + bx;
            a = __ldg(d.cell_start + c);
            cnt = __ldg(d.cell_start + c + 1) - a;
        }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    int ex[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ex[q] = __shfl_sync(0xffffffffu, incl, q);  // end of cell q
    const int total = __shfl_sync(0xffffffffu, incl, 8);
    const int excl = incl - cnt;
    const int trips = (total + 31) >> 5;  // uniform, so that the shuffles see the whole warp
#pragma unroll 1
    for (int it = 0; it < trips; ++it) {
        const int t = it * 32 + lane;
        int q = 0;
#pragma unroll
        for (int z = 0; z < 8; ++z) q += (t >= ex[z]);
        const int j = __shfl_sync(0xffffffffu, a, q) + (t - __shfl_sync(0xffffffffu, excl, q));
        if (t >= total) continue;
        const int oy = q / 3 - 1, ox = q % 3 - 1;
        const float rxo = rx - (float)ox * g.sxf, ryo = ry - (float)oy * g.syf;
        float dxf, dyf, r2f;
        if (!is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f)) continue;
        if (MIXED) {
            f(j, dxf, dyf, r2f);
        } else {
            const double2 xy = d.XY[j];
            double dx, dy;
            const double r2 = exact_r2(g, qx, qy, xy.x, xy.y, dx, dy);
            f(j, dx, dy, r2);
        }
    }
}

// Lane-strided walk that lists the *fluid* neighbours of a query point in a per-warp shared
// buffer (ballot compaction, CMP_CAP entries) and then runs body(j) over the list with all
// lanes busy, so that fp64 pair work does not idle the lanes of rejected candidates.
constexpr int CMP_CAP = 128;

template <class F>
__device__ __forceinline__ void lane_fluid_compact(const Dev &d, int lane, int *buf, double qx,
                                                   double qy, int cx, int cy, float rx, float ry,
                                                   F &&body)
{
    const Geo &g = d.g;
    int a = 0, cnt = 0;
    if (lane < 9) {
        const int oy = lane / 3 - 1, ox = lane % 3 - 1;
        int by = cy + oy, bx = cx + ox;
        bool ok = true;
        if (g.py) by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
        else ok = by >= 0 && by < g.ny;
        if (g.px) bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
        else ok = ok && bx >= 0 && bx < g.nx;
        if (ok) {
            const int c = by * g.nx + bx;
            a = __ldg(d.cell_start + c);
            cnt = __ldg(d.cell_start + c + 1) - a;
        }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    int ex[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ex[q] = __shfl_sync(0xffffffffu, incl, q);
    const int total = __shfl_sync(0xffffffffu, incl, 8);
    const int excl = incl - cnt;
    const int trips = (total + 31) >> 5;
    const unsigned below = (1u << lane) - 1u;
    int nacc = 0;
#pragma unroll 1
    for (int it = 0; it < trips; ++it) {
        const int t = it * 32 + lane;
        int q = 0;
#pragma unroll
        for (int z = 0; z < 8; ++z) q += (t >= ex[z]);
        const int j = __shfl_sync(0xffffffffu, a, q) + (t - __shfl_sync(0xffffffffu, excl, q));
        bool want = false;
        if (t < total) {
            const int oy = q / 3 - 1, ox = q % 3 - 1;
            const float rxo = rx - (float)ox * g.sxf, ryo = ry - (float)oy * g.syf;
            float dxf, dyf, r2f;
            want = is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f) &&
                   (d.stag[j] & 0x7f) == FLUID;
        }
        const unsigned m = __ballot_sync(0xffffffffu, want);
        if (want) buf[nacc + __popc(m & below)] = j;
        nacc += __popc(m);
        if (nacc > CMP_CAP - 32) {
            __syncwarp();
            for (int e = lane; e < nacc; e += 32) body(buf[e]);
            __syncwarp();
            nacc = 0;
        }
    }
    __syncwarp();
    for (int e = lane; e < nacc; e += 32) body(buf[e]);
    __syncwarp();
}

// (p, u, v, m/rho) of particle j in the path's own precision
template <int MIXED, class T>
__device__ __forceinline__ void fluid_fields(const Dev &d, int j, T &p, T &u, T &v, T &mrho)
{
    if (MIXED) {
        const float4 q = d.Qf[j];
        const float4 b = d.Bf[j];
        p = (T)q.x; u = (T)b.x; v = (T)b.y; mrho = (T)q.w;
    } else {
        const double2 pv = d.PV[j], uv = d.UV[j];
        p = (T)pv.x; u = (T)uv.x; v = (T)uv.y; mrho = (T)d.RM[j].y;
    }
}

template <class T>
__device__ __forceinline__ T sqrt_t(T x);
template <>
__device__ __forceinline__ float sqrt_t<float>(float x) { return x * rsqrt_approx(fmaxf(x, 1e-30f)); }
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }

// Gaussian elimination with partial pivoting on a 3x3 system, kept in registers (row
// exchanges by selects).  Returns false on a zero pivot.
__device__ __forceinline__ void swap_rows(bool c, double &a0, double &a1, double &a2, double &ab,
                                          double &b0, double &b1, double &b2, double &bb)
{
    double t;
    t = c ? b0 : a0; b0 = c ? a0 : b0; a0 = t;
    t = c ? b1 : a1; b1 = c ? a1 : b1; a1 = t;
    t = c ? b2 : a2; b2 = c ? a2 : b2; a2 = t;
    t = c ? bb : ab; bb = c ? ab : bb; ab = t;
}

__device__ bool solve3(const double (&M)[3][3], const double (&b)[3], double (&x)[3])
{
    double a00 = M[0][0], a01 = M[0][1], a02 = M[0][2], b0 = b[0];
    double a10 = M[1][0], a11 = M[1][1], a12 = M[1][2], b1 = b[1];
    double a20 = M[2][0], a21 = M[2][1], a22 = M[2][2], b2 = b[2];
    // column 0: the largest |a_r0| to the top (first maximum wins, as in a row scan)
    swap_rows(fabs(a10) > fabs(a00) && fabs(a10) >= fabs(a20), a00, a01, a02, b0, a10, a11, a12, b1);
    swap_rows(fabs(a20) > fabs(a00), a00, a01, a02, b0, a20, a21, a22, b2);
    if (a00 == 0.0) return false;
    double f = a10 / a00;
    a11 -= f * a01; a12 -= f * a02; b1 -= f * b0;
    f = a20 / a00;
    a21 -= f * a01; a22 -= f * a02; b2 -= f * b0;
    // column 1
    swap_rows(fabs(a21) > fabs(a11), a10, a11, a12, b1, a20, a21, a22, b2);
    if (a11 == 0.0) return false;
    f = a21 / a11;
    a22 -= f * a12; b2 -= f * b1;
    if (a22 == 0.0) return false;
    x[2] = b2 / a22;
    x[1] = (b1 - a12 * x[2]) / a11;
    x[0] = (b0 - a01 * x[1] - a02 * x[2]) / a00;
    return true;
}

// Mirrored Taylor extrapolation (Sec. 3.2): the first-order system of Eq. matform at the
// mirror point k over its fluid neighbours l (r_lk = r_l - r_k, V_l = m_l/rho_l), solved with
// partial pivoting for NF fluid fields (p, u, v in that order, one matrix), then
// f_o = f_k - (r_o - r_k).grad f_k (Eq. taylor2).  No fluid in reach: f_o = 0; singular
// system (|det| <= 1e-9 |M00 M11 M22|): the Shepard value sum f W V / sum W V; all weights
// zero (every fluid neighbour at the support edge): the plain mean of f.  fp64 on both paths:
// with disordered particles the system can be ill-conditioned and fp32 moment sums would
// lose the solution.
//
// mirror_sums: this lane's share of the sums a[mirror_na(NF)] (whole warp; the lanes split the
// fluid neighbours); mirror_solve: f_o from the warp totals of those sums (one lane).
__host__ __device__ constexpr int mirror_na(int nf) { return 9 + 3 * nf + 1 + nf; }

template <int MIXED, int NF>
__device__ __forceinline__ void mirror_sums(const Dev &d, int lane, int *wbuf, double xk, double yk,
                                            double (&a)[mirror_na(NF)])
{
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int cx = cell_coord(xk, g.x_min, g.inv_sx, g.nx);
    const int cy = cell_coord(yk, g.y_min, g.inv_sy, g.ny);
    const float rx = d2f(xk - (g.x_min + (double)cx * g.sx));
    const float ry = d2f(yk - (g.y_min + (double)cy * g.sy));
    // [M (9) | right-hand sides (3 per field) | count | plain sums (1 per field)]
    constexpr int NA = mirror_na(NF);
#pragma unroll
    for (int i = 0; i < NA; ++i) a[i] = 0.0;
    lane_fluid_compact(d, lane, wbuf, xk, yk, cx, cy, rx, ry, [&](int l) {
        const double2 xyl = d.XY[l];
        double xlk, ylk;  // r_lk = r_l - r_k, the canonical fp64 separation
        const double r2 = exact_r2(g, xyl.x, xyl.y, xk, yk, xlk, ylk);
        double fv[3], row[3];
        if (MIXED) {
            // mixed path: the kernel terms W V, W_x V, W_y V in fp32 (relative error ~1e-7
            // each, on the fp32 pipe); the moment sums, where the cancellation is, stay fp64
            const float4 q = d.Qf[l];
            const float4 b = d.Bf[l];
            fv[0] = f2d(q.x); fv[1] = f2d(b.x); fv[2] = f2d(b.y);
            const float Vl = q.w, r2f = d2f(r2);
            float w, wx = 0.0f, wy = 0.0f;
            if (r2f > 1e-30f) {
                const float ir = rsqrt_approx(r2f);
                float wq, dwq;
                quintic_w_dw(r2f * ir * ph.inv_hf, wq, dwq);
                w = ph.a2f * wq;
                const float dwr = ph.a2hf * dwq * ir;
                wx = dwr * d2f(xlk);
                wy = dwr * d2f(ylk);
            } else {
                w = ph.a2f * quintic_w(0.0f);
            }
            row[0] = f2d(w * Vl);
            row[1] = f2d(wx * Vl);
            row[2] = f2d(wy * Vl);
        } else {
            // fp64 path: IEEE square root and division (the oracle's arithmetic)
            double Vl;
            fluid_fields<MIXED>(d, l, fv[0], fv[1], fv[2], Vl);
            double w, wx = 0, wy = 0;
            if (r2 > 1e-30) {
                const double r = sqrt(r2), ir = 1.0 / r;
                double wq, dwq;
                quintic_w_dw(r * ph.inv_h, wq, dwq);
                w = ph.a2 * wq;
                const double dwr = ph.a2h * dwq * ir;
                wx = dwr * xlk;
                wy = dwr * ylk;
            } else {
                w = ph.a2 * quintic_w(0.0);
            }
            row[0] = w * Vl;
            row[1] = wx * Vl;
            row[2] = wy * Vl;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            a[3 * q + 0] += row[q];
            a[3 * q + 1] += xlk * row[q];
            a[3 * q + 2] += ylk * row[q];
#pragma unroll
            for (int f = 0; f < NF; ++f) a[9 + 3 * f + q] += fv[f] * row[q];
        }
        a[9 + 3 * NF] += 1.0;
#pragma unroll
        for (int f = 0; f < NF; ++f) a[10 + 3 * NF + f] += fv[f];
    });
}

template <int NF>
__device__ __forceinline__ void mirror_solve(const double (&a)[mirror_na(NF)], double xo, double yo,
                                             double xk, double yk, double (&fo)[NF])
{
    double M[3][3];
    for (int q = 0; q < 3; ++q)
        for (int c = 0; c < 3; ++c) M[q][c] = a[3 * q + c];
    const double cnt = a[9 + 3 * NF];
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    const bool singular = fabs(det) <= 1e-9 * fabs(M[0][0] * M[1][1] * M[2][2]);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const double bb[3] = {a[9 + 3 * f], a[10 + 3 * f], a[11 + 3 * f]};
        double pk = 0.0, gxp = 0.0, gyp = 0.0;
        if (cnt > 0.0 && !(M[0][0] > 0.0)) {
            pk = a[10 + 3 * NF + f] / cnt;
        } else if (cnt > 0.0) {
            pk = bb[0] / M[0][0];
            if (!singular) {
                double sol[3] = {0.0, 0.0, 0.0};
                if (solve3(M, bb, sol)) { pk = sol[0]; gxp = sol[1]; gyp = sol[2]; }
            }
        }
        fo[f] = pk - ((xo - xk) * gxp + (yo - yk) * gyp);
    }
}


// The whole extrapolation on one warp: lane 0 receives fo.
template <int MIXED, int NF>
__device__ __forceinline__ void mirror_extrapolate(const Dev &d, int lane, int *wbuf, double xo,
                                                   double yo, double xk, double yk,
                                                   double (&fo)[NF])
{
    double a[mirror_na(NF)];
    mirror_sums<MIXED, NF>(d, lane, wbuf, xk, yk, a);
    warp_sum(a);
    if (lane == 0) mirror_solve<NF>(a, xo, yo, xk, yk, fo);
}

// A warp takes the boundary particles in chunks of BND_CHUNK.  Walls and outlet particles are
// finished one by one (lane 0); an inlet particle's mirror sums are reduce-scattered into a
// per-warp stash, and the chunk's inlet particles are solved together at its end, lane i for
// the chunk's particle i, so that the fp64 3x3 solve runs once per warp-instruction for up
// to BND_CHUNK particles instead of once per particle.  Nothing in the kernel reads the
// inlet's values, so finishing them at the chunk end changes no result.
constexpr int BND_CHUNK = 8;
constexpr int BND_STASH = 17;  // stash row stride (doubles): odd, against bank conflicts

template <int MIXED>
__device__ __forceinline__ void boundary(const Dev &d, int end_of_step, int bid, int nblk)
{
    typedef typename std::conditional<MIXED, float, double>::type T;
    constexpr int NAI = mirror_na(1);
    static_assert(NAI <= 16 && NAI <= BND_STASH, "inlet mirror sums");
    __shared__ int wbuf[8][CMP_CAP];  // per-warp list of the mirror's fluid neighbours
    __shared__ double stash[8][BND_CHUNK][BND_STASH];  // per-warp inlet mirror sums
    const Phys &ph = d.ph;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = d.cnt->n_bnd;
    const int nwarps = (nblk * blockDim.x) >> 5;
    const T a2 = narrow<T>(ph.a2), a2h = narrow<T>(ph.a2h), inv_h = narrow<T>(ph.inv_h);
    for (int base = ((bid * blockDim.x + threadIdx.x) >> 5) * BND_CHUNK; base < nb;
         base += nwarps * BND_CHUNK) {
    const int nchunk = min(BND_CHUNK, nb - base);
    bool inlet_mine = false;  // lane i: chunk particle i is an inlet particle to solve
    for (int i = 0; i < nchunk; ++i) {
        const int b = base + i;
        const int k = d.bnd[b];
        const int t = d.stag[k] & 0x7f;
        const int s = d.order[k];
        const double2 xy = d.XY[k];
        if (t == WALL || t == SLIPWALL) {
            // Solid wall (Adami et al. 2012, cited in Sec. 2): Shepard pressure of the
            // fluid; ghost velocity 2 u_w - <u> (no-slip) or (<u>, -<v>) (slip, normal y).
            int cx, cy;
            cell_of(d, k, cx, cy);
            const float4 pk = d.P[k];
            // [sum W, sum W p, sum W u, sum W v, count, sum p, sum u, sum v] over fluid j
            T a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            lane_neighbors<MIXED>(d, lane, xy.x, xy.y, cx, cy, pk.x, pk.y, [&](int j, T, T, T r2) {
                if ((d.stag[j] & 0x7f) != FLUID) return;
                const T w = a2 * quintic_w(sqrt_t<T>(r2) * inv_h);
                T p, u, v, mr;
                fluid_fields<MIXED>(d, j, p, u, v, mr);
                a[0] += w; a[1] += w * p; a[2] += w * u; a[3] += w * v;
                a[4] += (T)1; a[5] += p; a[6] += u; a[7] += v;
            });
            warp_sum(a);
            if (lane == 0) {
                const int wi = (t == WALL) ? 0 : 1;
                T pw, ug, vg;
                const T sw = a[0];
                if (a[4] > (T)0) {
                    // Shepard average; all weights zero (every fluid neighbour at the support
                    // edge, where W rounds to 0): the plain mean over those neighbours
                    const bool wz = !(sw > (T)0);
                    const T isw = wz ? (T)1 / a[4] : (T)1 / sw;
                    pw = (wz ? a[5] : a[1]) * isw;
                    const T uf = (wz ? a[6] : a[2]) * isw, vf = (wz ? a[7] : a[3]) * isw;
                    if (ph.wall_slip[wi]) { ug = uf; vg = -vf; }
                    else { ug = narrow<T>(2.0 * ph.wall_u[wi]) - uf; vg = narrow<T>(2.0 * ph.wall_v[wi]) - vf; }
                } else {
                    pw = (T)0; ug = narrow<T>(ph.wall_u[wi]); vg = narrow<T>(ph.wall_v[wi]);
                }
                if (MIXED) {
                    float4 q = d.Qf[k];
                    q.x = (float)pw;
                    d.Qf[k] = q;
                    d.Bf[k] = make_float4((float)ug, (float)vg, 0.0f, 0.0f);
                } else {
                    d.PV[k].x = pw;
                    d.UV[k] = make_double2(ug, vg);
                    d.DUV[k] = make_double2(0.0, 0.0);
                }
                const double pwd = widen(pw), ugd = widen(ug), vgd = widen(vg);
                d.p[s] = pwd; d.u[s] = ugd; d.v[s] = vgd; d.ut[s] = ugd; d.vt[s] = vgd;
            }
        } else if (t == INLET && ph.has_inlet) {
            // Mirrored inlet pressure (Sec. 3.2) about k = (2 x_in - x_o, y_o): the sums now,
            // the solve at the end of the chunk
            double a[NAI];
            mirror_sums<MIXED, 1>(d, lane, wbuf[w], 2.0 * ph.x_in - xy.x, xy.y, a);
            const double v = warp_reduce_scatter16(a, lane);
            if (!(lane & 1) && (lane >> 1) < NAI) stash[w][i][lane >> 1] = v;
            inlet_mine = inlet_mine || lane == i;
        } else if (t == OUTLET && end_of_step && ph.has_outlet &&
                   (ph.outlet_kind == OUT_HYBRID || ph.outlet_kind == OUT_CHARACTERISTIC ||
                    ph.outlet_kind == OUT_MOD_DONOTHING)) {
            // Outlet update (Sec. 3), once per step; red particles have fluid in reach.
            //   hybrid (Sec. 3.4): red take the Shepard J2 of the fluid, blue the mean
            //     previous-step J2 of their red outlet neighbours; J3 = 0 gives p' = J2/2,
            //     u' = J2/(2 rho0 c); value = frozen average + acoustic part (Eq. acou);
            //   characteristic (Sec. 3.3): the same J2 against a fixed reference state
            //     (u_ref, p_ref), v stays frozen;
            //   modified do-nothing (Sec. 3.1.1): values stay frozen, red advect with the
            //     Shepard u of the fluid (Eq. shepard0), blue with the mean previous-step
            //     advection velocity of their red neighbours.
            // Do-nothing (Sec. 3.1) needs no update; mirroring runs in k_outlet_mirror.
            // Written to the slot arrays only: the rates of this evaluation still see the
            // outlet values of the step.
            const int kind = ph.outlet_kind;
            int cx, cy;
            cell_of(d, k, cx, cy);
            const float4 pk = d.P[k];
            // [sum W, sum W f, fluid count, sum J2p, sum adv of red, red count, sum f] with
            // f = J2 of the fluid (u for the modified do-nothing)
            T a[7] = {0, 0, 0, 0, 0, 0, 0};
            lane_neighbors<MIXED>(d, lane, xy.x, xy.y, cx, cy, pk.x, pk.y, [&](int j, T, T, T r2) {
                const uint8_t tj = d.stag[j];
                if ((tj & 0x7f) == FLUID) {
                    const T w = a2 * quintic_w(sqrt_t<T>(r2) * inv_h);
                    T fj;
                    if (kind == OUT_MOD_DONOTHING) {
                        T p, u, v, mr;
                        fluid_fields<MIXED>(d, j, p, u, v, mr);
                        fj = u;
                    } else {
                        fj = narrow<T>(d.AUX[j].x);  // J2 of the fluid particle
                    }
                    a[0] += w;
                    a[1] += w * fj;
                    a[2] += (T)1;
                    a[6] += fj;
                } else if (tj == (OUTLET | TAG_REDP)) {
                    const double2 x2 = d.AUX[j];
                    a[3] += narrow<T>(x2.x);
                    a[4] += narrow<T>(x2.y);
                    a[5] += (T)1;
                }
            });
            warp_sum(a);
            if (lane == 0) {
                const bool red = a[2] > (T)0;
                const T mr = a[5];
                // Shepard average; all weights zero (fluid at the support edge): plain mean
                const T shep = red ? (a[0] > (T)0 ? a[1] / a[0] : a[6] / a[2]) : (T)0;
                const double blue_adv = mr > (T)0 ? widen(a[4] / mr) : 0.0;
                if (kind == OUT_MOD_DONOTHING) {
                    d.J2p[s] = 0.0;
                    d.advp[s] = red ? widen(shep) : (mr > (T)0 ? blue_adv : d.ubar[s]);
                    d.redp[s] = red ? 1 : 0;
                } else {
                    const bool ch = kind == OUT_CHARACTERISTIC;
                    const T J2 = red ? shep : (mr > (T)0 ? a[3] / mr : (T)0);
                    const double ub = ch ? ph.moc_u_ref : d.ubar[s];
                    const double pb = ch ? ph.moc_p_ref : d.pbar[s];
                    const double un = ub + widen(J2 * (MIXED ? (T)ph.inv_2rcf : narrow<T>(ph.inv_2rc)));
                    const double adv = red ? un : (mr > (T)0 ? blue_adv : (ch ? un : ub));
                    d.u[s] = un;
                    d.v[s] = d.vbar[s];
                    d.p[s] = pb + widen((T)0.5 * J2);
                    d.ut[s] = un;
                    d.vt[s] = d.vbar[s];
                    d.J2p[s] = widen(J2);
                    d.advp[s] = adv;
                    d.redp[s] = red ? 1 : 0;
                }
            }
        }
    }
    __syncwarp();
    if (inlet_mine) {
        const int k = d.bnd[base + lane];
        const int s = d.order[k];
        const double2 xy = d.XY[k];
        double a[NAI], fo[1];
#pragma unroll
        for (int q = 0; q < NAI; ++q) a[q] = stash[w][lane][q];
        mirror_solve<1>(a, xy.x, xy.y, 2.0 * ph.x_in - xy.x, xy.y, fo);
        const double po = fo[0];
        if (MIXED) {
            float4 q = d.Qf[k];
            q.x = d2f(po);
            d.Qf[k] = q;
        } else {
            d.PV[k].x = po;
        }
        d.p[s] = po;
    }
    __syncwarp();  // the stash is refilled by the next chunk
    }
}

template <int MIXED>
__global__ void __launch_bounds__(256) k_boundary(Dev d, int end_of_step)
{
    boundary<MIXED>(d, end_of_step, blockIdx.x, gridDim.x);
}
template <int MIXED>
__global__ void __launch_bounds__(256) k_boundary_b(BatchGrid bg, int end_of_step)
{
    run_member(bg, [&](const Dev &d, int b, int nb) { boundary<MIXED>(d, end_of_step, b, nb); });
}

// Mirrored outlet (Sec. 3.2 at the outlet), once per step: p, u, v of every outlet particle
// by the Taylor extrapolation about k = (2 x_out - x_o, y_o); the particle advects with that
// u.  One warp per boundary particle, outlet particles only.
template <int MIXED>
__device__ __forceinline__ void outlet_mirror(const Dev &d, int bid, int nblk)
{
    __shared__ int wbuf[8][CMP_CAP];
    const Phys &ph = d.ph;
    const int lane = threadIdx.x & 31;
    const int nb = d.cnt->n_bnd;
    const int nwarps = (nblk * blockDim.x) >> 5;
    for (int b = (bid * blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
        const int k = d.bnd[b];
        if ((d.stag[k] & 0x7f) != OUTLET) continue;
        const int s = d.order[k];
        const double2 xy = d.XY[k];
        double fo[3];
        mirror_extrapolate<MIXED, 3>(d, lane, wbuf[threadIdx.x >> 5], xy.x, xy.y,
                                     2.0 * ph.x_out - xy.x, xy.y, fo);
        if (lane == 0) {
            d.p[s] = fo[0];
            d.u[s] = fo[1];
            d.v[s] = fo[2];
            d.ut[s] = fo[1];
            d.vt[s] = fo[2];
            d.advp[s] = fo[1];
            d.J2p[s] = 0.0;
            d.redp[s] = 0;
        }
    }
}

template <int MIXED>
__global__ void __launch_bounds__(256) k_outlet_mirror(Dev d) { outlet_mirror<MIXED>(d, blockIdx.x, gridDim.x); }
template <int MIXED>
__global__ void __launch_bounds__(256) k_outlet_mirror_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) { outlet_mirror<MIXED>(d, b, nb); });
}

// Debug: exact neighbour ids of every particle, with the membership test of the passes.
__global__ void k_dump(Dev d, const long long *start, unsigned long long *ids)
{
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pk = d.P[k];
        const double2 xy = d.XY[k];
        long long pos = start[k];
        const long long end = start[k + 1];
        for_block(d, cx, cy, [&](int ox, int oy, int j0, int j1) {
            const float rxo = pk.x - (float)ox * d.g.sxf, ryo = pk.y - (float)oy * d.g.syf;
            for (int j = j0; j < j1; ++j) {
                float dxf, dyf, r2f;
                if (!is_member(d, rxo, ryo, __ldg(d.P + j), j, xy.x, xy.y, dxf, dyf, r2f)) continue;
                if (pos < end) ids[pos] = d.id[d.order[j]];
                ++pos;
            }
        });
    }
}

int grid_for(int n, int tpb)
{
    int b = (n + tpb - 1) / tpb;
    return b < 1 ? 1 : b;
}

}  // namespace

int tiles(const Dev &d) { return d.g.ny * ((d.g.nx + d.tile_tx - 1) / d.tile_tx); }

int launch_pass_a(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_a_tiled<<<tiles(d), d.tile_tpb, 0, s>>>(d);
    else k_pass_a64<<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    return 1;
}

int launch_boundary(const Dev &d, cudaStream_t s, int mixed, int end_of_step)
{
    // one warp per chunk of BND_CHUNK boundary particles (grid-stride over the chunks; boundary
    // particles are O(sqrt(N))); at most three resident blocks per SM
    const int bblocks = min(grid_for(d.cap, 64 * BND_CHUNK), 152 * 3);
    if (mixed) k_boundary<1><<<bblocks, 256, 0, s>>>(d, end_of_step);
    else k_boundary<0><<<bblocks, 256, 0, s>>>(d, end_of_step);
    const int blocks = min(grid_for(d.cap, 64), 152 * 16);
    if (end_of_step && d.ph.has_outlet && d.ph.outlet_kind == OUT_MIRROR) {
        if (mixed) k_outlet_mirror<1><<<blocks, 256, 0, s>>>(d);
        else k_outlet_mirror<0><<<blocks, 256, 0, s>>>(d);
        return 2;
    }
    return 1;
}

int launch_pass_b(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_b_tiled<<<tiles(d), d.tile_tpb, 0, s>>>(d);
    else k_pass_b64<<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    return 1;
}

// ---------------------------------------------------------------- batched launches
int launch_pass_a_batch(const BatchPlan &p, cudaStream_t s)
{
    if (p.mixed) k_pass_a_tiled_b<<<p.total[BK_TILES], p.pair_tpb, 0, s>>>(p.grid(BK_TILES));
    else k_pass_a64_b<<<p.total[BK_CAP128], TPB, 0, s>>>(p.grid(BK_CAP128));
    return 1;
}

int launch_boundary_batch(const BatchPlan &p, cudaStream_t s, int end_of_step)
{
    if (p.mixed) k_boundary_b<1><<<p.total[BK_BND], 256, 0, s>>>(p.grid(BK_BND), end_of_step);
    else k_boundary_b<0><<<p.total[BK_BND], 256, 0, s>>>(p.grid(BK_BND), end_of_step);
    if (end_of_step && p.any_mirror) {
        if (p.mixed) k_outlet_mirror_b<1><<<p.total[BK_MIRROR], 256, 0, s>>>(p.grid(BK_MIRROR));
        else k_outlet_mirror_b<0><<<p.total[BK_MIRROR], 256, 0, s>>>(p.grid(BK_MIRROR));
        return 2;
    }
    return 1;
}

int launch_pass_b_batch(const BatchPlan &p, cudaStream_t s)
{
    if (p.mixed) k_pass_b_tiled_b<<<p.total[BK_TILES], p.pair_tpb, 0, s>>>(p.grid(BK_TILES));
    else k_pass_b64_b<<<p.total[BK_CAP128], TPB, 0, s>>>(p.grid(BK_CAP128));
    return 1;
}

int cells_batch_blocks(const Dev &d, int kind);

// Blocks of one member for each kernel shape: the grids of the single-system launches.
int batch_blocks(const Dev &d, int kind)
{
    switch (kind) {
    case BK_TILES: return tiles(d);
    case BK_CAP128: return grid_for(d.cap, TPB);
    case BK_BND: return min(grid_for(d.cap, 64 * BND_CHUNK), 152 * 3);
    case BK_MIRROR:
        return (d.ph.has_outlet && d.ph.outlet_kind == OUT_MIRROR) ? min(grid_for(d.cap, 64), 152 * 16)
                                                                  : 0;
    default: return cells_batch_blocks(d, kind);
    }
}

int launch_neighbor_dump(const Dev &d, cudaStream_t s, int mixed, const long long *start,
                         unsigned long long *ids)
{
    (void)mixed;
    k_dump<<<grid_for(d.cap, TPB), TPB, 0, s>>>(d, start, ids);
    return 1;
}

}  // namespace edac
