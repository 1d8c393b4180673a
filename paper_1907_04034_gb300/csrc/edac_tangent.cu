// Tangent-linear model of the fp64 step: the derivatives of every particle field with respect
// to the inlet-profile modes a_k of u(y) = U + sum_k a_k sin(k pi (y - y0) / H), carried
// forward step by step next to the values (forward-mode differentiation of the discrete step,
// with the neighbour sets, the acoustic-gate decisions, the red/blue outlet classes and the
// recycling events those values produce held fixed).
//
// Each tangent kernel follows the value kernel it differentiates (same formulas, same
// neighbour walk, same branch decisions, taken on the values) in dual numbers = value + one
// derivative; blockIdx.y is the direction (mode) k.  The pair passes, which dominate, use
// fp32 duals with four derivatives (FG: one neighbour walk and one value evaluation for four
// directions, blockIdx.y a group of four) on the fp32 pipe; the boundary parts (walls, the
// mirrored inlet's 3x3 solve, the outlet) fp64 duals (D1).  Tangents are slot-indexed,
// [field][direction][capacity] fp32, in a workspace of their own.  The value kernels run unchanged; the tangent
// kernels are interleaved after them (see edac_step_tangent).
#include "edac_internal.cuh"

namespace edac {
namespace {

// ------------------------------------------------------------------------ dual numbers
struct D1 {
    double v, d;
    __device__ D1() : v(0.0), d(0.0) {}
    __device__ D1(double a) : v(a), d(0.0) {}
    __device__ D1(double a, double b) : v(a), d(b) {}
};
__device__ __forceinline__ D1 operator+(D1 a, D1 b) { return D1(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ D1 operator*(D1 a, D1 b) { return D1(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ D1 operator/(D1 a, D1 b)
{
    const double r = 1.0 / b.v;
    const double q = a.v * r;
    return D1(q, (a.d - q * b.d) * r);
}
__device__ __forceinline__ D1 &operator+=(D1 &a, D1 b) { a = a + b; return a; }
__device__ __forceinline__ D1 dsqrt(D1 a)
{
    const double s = sqrt(a.v);
    return D1(s, s > 0.0 ? (0.5 * a.d) * (1.0 / s) : 0.0);
}

// quintic spline w(q), w'(q) with their derivatives along q (w'' for the derivative of w')
__device__ __forceinline__ void quintic_dual(D1 q, D1 &w, D1 &dw)
{
    const double t3 = q.v < 3.0 ? 3.0 - q.v : 0.0;
    const double t2 = q.v < 2.0 ? 2.0 - q.v : 0.0;
    const double t1 = q.v < 1.0 ? 1.0 - q.v : 0.0;
    const double a = t3 * t3, b = t2 * t2, c = t1 * t1;
    const double wv = t3 * a * a - 6.0 * (t2 * b * b) + 15.0 * (t1 * c * c);
    const double w1 = -5.0 * (a * a - 6.0 * b * b + 15.0 * c * c);
    const double w2 = 20.0 * (t3 * a - 6.0 * (t2 * b) + 15.0 * (t1 * c));
    w = D1(wv, w1 * q.d);
    dw = D1(w1, w2 * q.d);
}

// ------------------------------------------------------------------ tangent storage
struct TDev {
    float *f[T_NF];   // [direction][capacity] per field (fp32: derivatives carry ~1e-7
                      // relative rounding, far below the accuracy asked of the gradient)
    double *hist;     // [max_history][2][T_DIR]: d(F_x), d(F_y)
    float4 *vf;       // [capacity] fp32 copies (p, V, rho, m/rho) by sorted index
    float4 *vg;       // [capacity] fp32 copies (u, v, u~ - u, v~ - v) by sorted index
    int ndir;         // directions in use (modes)
};

__device__ __forceinline__ float &tg(const TDev &t, const Dev &d, int f, int c, int s)
{
    return t.f[f][(size_t)c * d.cap + s];
}

__device__ __forceinline__ D1 dual(const TDev &t, const Dev &d, double v, int f, int c, int s)
{
    return D1(v, f2d(t.f[f][(size_t)c * d.cap + s]));
}

// sin(k pi (y - y0)/H): the derivative of the inlet velocity with respect to mode k
__device__ __forceinline__ double mode_shape(const Phys &ph, int c, double y)
{
    return sin((double)(c + 1) * 3.141592653589793 * (y - ph.in_y0) / ph.in_H);
}

// Walk the neighbours of the point (qx, qy) in cell (cx, cy): the membership test of the
// value kernels (fp32 pre-test on cell-relative coordinates, the fp64 test in the band), so
// the tangent kernels visit exactly the neighbours the value kernels did.
template <class F>
__device__ __forceinline__ void t_walk(const Dev &d, double qx, double qy, int cx, int cy, F &&f)
{
    const Geo &g = d.g;
    const float rx = d2f(qx - (g.x_min + (double)cx * g.sx));
    const float ry = d2f(qy - (g.y_min + (double)cy * g.sy));
    for_block(d, cx, cy, [&](int ox, int oy, int j0, int j1) {
        const float rxo = rx - (float)ox * g.sxf, ryo = ry - (float)oy * g.syf;
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            if (is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f)) f(j);
        }
    });
}

// ------------------------------------------------------------- walls and inlet mirror
// fp64 duals with TGW derivatives: the wall and inlet tangents carry TGW directions per
// thread, so that the neighbour walk and the fp64 values (the Shepard sums, the mirror's
// moment sums and pivots) are evaluated once for all of them.
constexpr int TGW = 2;
static_assert(T_DIR % TGW == 0, "directions per thread");
struct DG {
    double v, d[TGW];
    __device__ DG() : v(0.0)
    {
#pragma unroll
        for (int g = 0; g < TGW; ++g) d[g] = 0.0;
    }
    __device__ explicit DG(double a) : v(a)
    {
#pragma unroll
        for (int g = 0; g < TGW; ++g) d[g] = 0.0;
    }
};
__device__ __forceinline__ DG operator+(const DG &a, const DG &b)
{
    DG r;
    r.v = a.v + b.v;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = a.d[g] + b.d[g];
    return r;
}
__device__ __forceinline__ DG operator-(const DG &a, const DG &b)
{
    DG r;
    r.v = a.v - b.v;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = a.d[g] - b.d[g];
    return r;
}
__device__ __forceinline__ DG operator-(const DG &a)
{
    DG r;
    r.v = -a.v;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = -a.d[g];
    return r;
}
__device__ __forceinline__ DG operator*(const DG &a, const DG &b)
{
    DG r;
    r.v = a.v * b.v;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = a.d[g] * b.v + a.v * b.d[g];
    return r;
}
__device__ __forceinline__ DG operator*(double s, const DG &a)  // a constant times a dual
{
    DG r;
    r.v = s * a.v;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = s * a.d[g];
    return r;
}
__device__ __forceinline__ DG operator/(const DG &a, const DG &b)
{
    const double rb = 1.0 / b.v;
    DG r;
    r.v = a.v * rb;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = (a.d[g] - r.v * b.d[g]) * rb;
    return r;
}
__device__ __forceinline__ DG &operator+=(DG &a, const DG &b) { a = a + b; return a; }
__device__ __forceinline__ DG &operator-=(DG &a, const DG &b) { a = a - b; return a; }
__device__ __forceinline__ DG dsqrt(const DG &a)
{
    DG r;
    r.v = sqrt(a.v);
    const double h = r.v > 0.0 ? 1.0 / r.v : 0.0;
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = r.v > 0.0 ? (0.5 * a.d[g]) * h : 0.0;
    return r;
}
__device__ __forceinline__ void quintic_dual(const DG &q, DG &w, DG &dw)
{
    const double t3 = q.v < 3.0 ? 3.0 - q.v : 0.0;
    const double t2 = q.v < 2.0 ? 2.0 - q.v : 0.0;
    const double t1 = q.v < 1.0 ? 1.0 - q.v : 0.0;
    const double a = t3 * t3, b = t2 * t2, c = t1 * t1;
    w.v = t3 * a * a - 6.0 * (t2 * b * b) + 15.0 * (t1 * c * c);
    dw.v = -5.0 * (a * a - 6.0 * b * b + 15.0 * c * c);
    const double w2 = 20.0 * (t3 * a - 6.0 * (t2 * b) + 15.0 * (t1 * c));
#pragma unroll
    for (int g = 0; g < TGW; ++g) {
        w.d[g] = dw.v * q.d[g];
        dw.d[g] = w2 * q.d[g];
    }
}

__device__ __forceinline__ DG dual_g(const TDev &t, const Dev &d, double v, int f, int c0, int s)
{
    DG r(v);
#pragma unroll
    for (int g = 0; g < TGW; ++g) r.d[g] = f2d(t.f[f][(size_t)(c0 + g) * d.cap + s]);
    return r;
}

// 3x3 solve with partial pivoting (pivots chosen on the values)
__device__ bool solve3_dual(DG (&M)[3][3], DG (&b)[3], DG (&x)[3])
{
    int piv[3] = {0, 1, 2};
    for (int col = 0; col < 3; ++col) {
        int p = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(M[piv[r]][col].v) > fabs(M[piv[p]][col].v)) p = r;
        const int tmp = piv[col];
        piv[col] = piv[p];
        piv[p] = tmp;
        const int pr = piv[col];
        if (M[pr][col].v == 0.0) return false;
        for (int r = col + 1; r < 3; ++r) {
            const int rr = piv[r];
            const DG f = M[rr][col] / M[pr][col];
            for (int cc = col; cc < 3; ++cc) M[rr][cc] -= f * M[pr][cc];
            b[rr] -= f * b[pr];
        }
    }
    for (int col = 2; col >= 0; --col) {
        const int pr = piv[col];
        DG s = b[pr];
        for (int cc = col + 1; cc < 3; ++cc) s -= M[pr][cc] * x[cc];
        x[col] = s / M[pr][col];
    }
    return true;
}

__global__ void t_walls_inlet(Dev d, TDev t)
{
    const int c0 = blockIdx.y * TGW;
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int nb = d.cnt->n_bnd;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int k = d.bnd[b];
        const int tag = d.stag[k] & 0x7f;
        const int s = d.order[k];
        const double2 xy = d.XY[k];
        const DG Xi = dual_g(t, d, xy.x, T_X, c0, s), Yi = dual_g(t, d, xy.y, T_Y, c0, s);
        if (tag == WALL || tag == SLIPWALL) {
            const int cc = d.cellk[k];
            DG sw, sp, su, sv, mp, mu, mv;
            int nf = 0;
            t_walk(d, xy.x, xy.y, cc % g.nx, cc / g.nx, [&](int j) {
                if ((d.stag[j] & 0x7f) != FLUID) return;
                const int sj = d.order[j];
                const double2 xj = d.XY[j];
                double ex, ey;
                exact_r2(g, xy.x, xy.y, xj.x, xj.y, ex, ey);
                DG dx(ex), dy(ey);
#pragma unroll
                for (int q = 0; q < TGW; ++q) {
                    dx.d[q] = Xi.d[q] - tg(t, d, T_X, c0 + q, sj);
                    dy.d[q] = Yi.d[q] - tg(t, d, T_Y, c0 + q, sj);
                }
                const DG r = dsqrt(dx * dx + dy * dy);
                DG w, dw;
                quintic_dual(ph.inv_h * r, w, dw);
                const DG W = ph.a2 * w;
                const double2 pv = d.PV[j], uv = d.UV[j];
                const DG fp = dual_g(t, d, pv.x, T_P, c0, sj);
                const DG fu = dual_g(t, d, uv.x, T_U, c0, sj);
                const DG fv = dual_g(t, d, uv.y, T_V, c0, sj);
                sw += W; sp += W * fp; su += W * fu; sv += W * fv;
                mp += fp; mu += fu; mv += fv;
                ++nf;
            });
            const int wi = tag == WALL ? 0 : 1;
            DG pw, ug(ph.wall_u[wi]), vg(ph.wall_v[wi]);
            if (nf > 0) {
                DG uf, vf;
                if (sw.v > 0.0) { pw = sp / sw; uf = su / sw; vf = sv / sw; }
                else {
                    const DG n_(static_cast<double>(nf));
                    pw = mp / n_; uf = mu / n_; vf = mv / n_;
                }
                if (ph.wall_slip[wi]) { ug = uf; vg = -vf; }
                else { ug = DG(2.0 * ph.wall_u[wi]) - uf; vg = DG(2.0 * ph.wall_v[wi]) - vf; }
            }
#pragma unroll
            for (int q = 0; q < TGW; ++q) {
                const int c = c0 + q;
                tg(t, d, T_P, c, s) = d2f(pw.d[q]);
                tg(t, d, T_U, c, s) = d2f(ug.d[q]);
                tg(t, d, T_V, c, s) = d2f(vg.d[q]);
                tg(t, d, T_UT, c, s) = d2f(ug.d[q]);
                tg(t, d, T_VT, c, s) = d2f(vg.d[q]);
            }
        } else if (tag == INLET && ph.has_inlet) {
            // mirrored inlet pressure (Eqs. matform, taylor2) about k = (2 x_in - x_o, y_o)
            const DG xk = DG(2.0 * ph.x_in) - Xi, yk = Yi;
            const int cx = cell_coord(xk.v, g.x_min, g.inv_sx, g.nx);
            const int cy = cell_coord(yk.v, g.y_min, g.inv_sy, g.ny);
            DG M[3][3], bb[3], mean;
            int nl = 0;
            t_walk(d, xk.v, yk.v, cx, cy, [&](int l) {
                if ((d.stag[l] & 0x7f) != FLUID) return;
                const int sl = d.order[l];
                const double2 xl = d.XY[l];
                double ex, ey;
                exact_r2(g, xl.x, xl.y, xk.v, yk.v, ex, ey);
                DG xlk(ex), ylk(ey);
#pragma unroll
                for (int q = 0; q < TGW; ++q) {
                    xlk.d[q] = f2d(tg(t, d, T_X, c0 + q, sl)) - xk.d[q];
                    ylk.d[q] = f2d(tg(t, d, T_Y, c0 + q, sl)) - yk.d[q];
                }
                const double2 pv = d.PV[l], rm = d.RM[l];
                const DG fp = dual_g(t, d, pv.x, T_P, c0, sl);
                const DG frho = dual_g(t, d, rm.x, T_RHO, c0, sl);
                const DG fmrho = DG(d.Ms[l]) / frho;
                const DG r2 = xlk * xlk + ylk * ylk;
                DG w, wx, wy;
                if (r2.v > 1e-30) {
                    const DG r = dsqrt(r2);
                    DG wq, dwq;
                    quintic_dual(ph.inv_h * r, wq, dwq);
                    w = ph.a2 * wq;
                    const DG dwr = (ph.a2h * dwq) / r;
                    wx = dwr * xlk;
                    wy = dwr * ylk;
                } else {
                    w = DG(ph.a2 * quintic_w(0.0));
                }
                const DG row[3] = {w * fmrho, wx * fmrho, wy * fmrho};
                for (int q = 0; q < 3; ++q) {
                    M[q][0] += row[q];
                    M[q][1] += xlk * row[q];
                    M[q][2] += ylk * row[q];
                    bb[q] += fp * row[q];
                }
                mean += fp;
                ++nl;
            });
            DG pk, gx, gy;
            if (nl > 0 && !(M[0][0].v > 0.0)) {
                pk = mean / DG(static_cast<double>(nl));
            } else if (nl > 0) {
                const double det = M[0][0].v * (M[1][1].v * M[2][2].v - M[1][2].v * M[2][1].v) -
                                   M[0][1].v * (M[1][0].v * M[2][2].v - M[1][2].v * M[2][0].v) +
                                   M[0][2].v * (M[1][0].v * M[2][1].v - M[1][1].v * M[2][0].v);
                pk = bb[0] / M[0][0];
                if (!(fabs(det) <= 1e-9 * fabs(M[0][0].v * M[1][1].v * M[2][2].v))) {
                    DG sol[3];
                    if (solve3_dual(M, bb, sol)) { pk = sol[0]; gx = sol[1]; gy = sol[2]; }
                }
            }
            const DG po = pk - ((Xi - xk) * gx + (Yi - yk) * gy);
#pragma unroll
            for (int q = 0; q < TGW; ++q) tg(t, d, T_P, c0 + q, s) = d2f(po.d[q]);
        }
    }
}

// --------------------------------------------------------------- hybrid outlet update
// Runs after the tangent pass B of the end-of-step evaluation (the rates of that evaluation
// see the outlet values of the step), reading the neighbours' previous J2p / advection
// tangents from a snapshot.
__global__ void t_snapshot(Dev d, TDev t)
{
    const int c = blockIdx.y;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        tg(t, d, T_J2P_OLD, c, s) = tg(t, d, T_J2P, c, s);
        tg(t, d, T_ADVP_OLD, c, s) = tg(t, d, T_ADVP, c, s);
    }
}

__global__ void t_outlet(Dev d, TDev t)
{
    const int c = blockIdx.y;
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int nb = d.cnt->n_bnd;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int k = d.bnd[b];
        if ((d.stag[k] & 0x7f) != OUTLET) continue;
        const int s = d.order[k];
        const double2 xy = d.XY[k];
        const int cc = d.cellk[k];
        D1 sw(0.0), sj(0.0), sjm(0.0), sjp(0.0), sadv(0.0);
        int nf = 0, mr = 0;
        const D1 Xo = dual(t, d, xy.x, T_X, c, s), Yo = dual(t, d, xy.y, T_Y, c, s);
        t_walk(d, xy.x, xy.y, cc % g.nx, cc / g.nx, [&](int j) {
            const uint8_t tj = d.stag[j];
            const int sjl = d.order[j];
            if ((tj & 0x7f) == FLUID) {
                const double2 xj = d.XY[j];
                double ex, ey;
                exact_r2(g, xy.x, xy.y, xj.x, xj.y, ex, ey);
                const D1 dx(ex, Xo.d - tg(t, d, T_X, c, sjl)), dy(ey, Yo.d - tg(t, d, T_Y, c, sjl));
                const D1 r = dsqrt(dx * dx + dy * dy);
                D1 w, dw;
                quintic_dual(r * D1(ph.inv_h), w, dw);
                const D1 W = D1(ph.a2) * w;
                const D1 J2j = dual(t, d, d.AUX[j].x, T_J2, c, sjl);
                sw += W; sj += W * J2j; sjm += J2j; ++nf;
            } else if (tj == (OUTLET | TAG_REDP)) {
                const double2 x2 = d.AUX[j];
                sjp += dual(t, d, x2.x, T_J2P_OLD, c, sjl);
                sadv += dual(t, d, x2.y, T_ADVP_OLD, c, sjl);
                ++mr;
            }
        });
        const bool red = nf > 0;
        D1 J2(0.0);
        if (red) J2 = sw.v > 0.0 ? sj / sw : sjm / D1((double)nf);
        else if (mr > 0) J2 = sjp / D1((double)mr);
        const D1 ub = dual(t, d, d.ubar[s], T_UBAR, c, s);
        const D1 un = ub + J2 * D1(ph.inv_2rc);
        const D1 adv = red ? un : (mr > 0 ? sadv / D1((double)mr) : ub);
        tg(t, d, T_U, c, s) = d2f(un.d);
        tg(t, d, T_V, c, s) = tg(t, d, T_VBAR, c, s);
        tg(t, d, T_P, c, s) = tg(t, d, T_PBAR, c, s) + 0.5 * J2.d;
        tg(t, d, T_UT, c, s) = d2f(un.d);
        tg(t, d, T_VT, c, s) = tg(t, d, T_VBAR, c, s);
        tg(t, d, T_J2P, c, s) = d2f(J2.d);
        tg(t, d, T_ADVP, c, s) = d2f(adv.d);
    }
}

// ------------------------------------------------------------------------------ stage
template <bool CORR>
__global__ void t_stage(Dev d, TDev t, double tau)
{
    const int c = blockIdx.y;
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        const uint8_t tag = d.tag[s];
        if (tag == FLUID) {
            if (!CORR) {
                tg(t, d, T_X0, c, s) = tg(t, d, T_X, c, s);
                tg(t, d, T_Y0, c, s) = tg(t, d, T_Y, c, s);
                tg(t, d, T_U0, c, s) = tg(t, d, T_U, c, s);
                tg(t, d, T_V0, c, s) = tg(t, d, T_V, c, s);
                tg(t, d, T_P0, c, s) = tg(t, d, T_P, c, s);
            }
            const double un = f2d(tg(t, d, T_U0, c, s)) + tau * f2d(tg(t, d, T_AU, c, s));
            const double vn = f2d(tg(t, d, T_V0, c, s)) + tau * f2d(tg(t, d, T_AV, c, s));
            const double utn = un + tau * f2d(tg(t, d, T_ABU, c, s));
            const double vtn = vn + tau * f2d(tg(t, d, T_ABV, c, s));
            const double pn = f2d(tg(t, d, T_P0, c, s)) + tau * f2d(tg(t, d, T_AP, c, s));
            tg(t, d, T_U, c, s) = d2f(un);
            tg(t, d, T_V, c, s) = d2f(vn);
            tg(t, d, T_UT, c, s) = d2f(utn);
            tg(t, d, T_VT, c, s) = d2f(vtn);
            tg(t, d, T_X, c, s) = d2f(f2d(tg(t, d, T_X0, c, s)) + tau * utn);
            tg(t, d, T_Y, c, s) = d2f(f2d(tg(t, d, T_Y0, c, s)) + tau * vtn);
            tg(t, d, T_P, c, s) = d2f(pn);
            if (CORR && ph.has_outlet && ph.outlet_kind == OUT_HYBRID) {
                // the value kernel sampled the ring iff the gate passed on the new pressure;
                // its write position has then moved on by one
                const double pv = d.p[s];
                if (pv * pv * ph.inv_2rc <= ph.I_thr) {
                    const int kk = (d.rpos[s] + ph.n_avg - 1) % ph.n_avg;
                    tg(t, d, T_RING + 3 * kk + 0, c, s) = d2f(un);
                    tg(t, d, T_RING + 3 * kk + 1, c, s) = d2f(vn);
                    tg(t, d, T_RING + 3 * kk + 2, c, s) = d2f(pn);
                }
                double su = 0, sv = 0, sp = 0;
                for (int q = 0; q < ph.n_avg; ++q) {
                    su += f2d(tg(t, d, T_RING + 3 * q + 0, c, s));
                    sv += f2d(tg(t, d, T_RING + 3 * q + 1, c, s));
                    sp += f2d(tg(t, d, T_RING + 3 * q + 2, c, s));
                }
                const double ub = su * ph.inv_navg, vb = sv * ph.inv_navg, pb = sp * ph.inv_navg;
                tg(t, d, T_UBAR, c, s) = d2f(ub);
                tg(t, d, T_VBAR, c, s) = d2f(vb);
                tg(t, d, T_PBAR, c, s) = d2f(pb);
                tg(t, d, T_J2, c, s) = d2f(ph.rho0 * ph.cs * (un - ub) + (pn - pb));
            }
        } else if (tag == INLET) {
            if (!CORR) tg(t, d, T_X0, c, s) = tg(t, d, T_X, c, s);
            const double du = c < ph.n_modes ? mode_shape(ph, c, d.y[s]) : 0.0;
            tg(t, d, T_U, c, s) = d2f(du);
            tg(t, d, T_V, c, s) = 0.0f;
            tg(t, d, T_UT, c, s) = d2f(du);
            tg(t, d, T_VT, c, s) = 0.0f;
            tg(t, d, T_X, c, s) = d2f(f2d(tg(t, d, T_X0, c, s)) + tau * du);
        } else if (tag == OUTLET) {
            if (!CORR) tg(t, d, T_X0, c, s) = tg(t, d, T_X, c, s);
            tg(t, d, T_X, c, s) = d2f(f2d(tg(t, d, T_X0, c, s)) + tau * f2d(tg(t, d, T_ADVP, c, s)));
        }
    }
}

// -------------------------------------------------------------------------- recycling
// Before the value kernel: the same transitions (decided on the values) applied to the
// tangents: fluid -> outlet keeps its time averages (hybrid) or freezes its values; inlet ->
// fluid fills its ring with its values.
__global__ void t_recycle_pre(Dev d, TDev t)
{
    const int c = blockIdx.y;
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        const uint8_t tag = d.tag[s];
        if (tag == FLUID && ph.has_outlet && d.x[s] >= ph.x_out) {
            if (ph.outlet_kind == OUT_HYBRID) {
                tg(t, d, T_U, c, s) = tg(t, d, T_UBAR, c, s);
                tg(t, d, T_V, c, s) = tg(t, d, T_VBAR, c, s);
                tg(t, d, T_P, c, s) = tg(t, d, T_PBAR, c, s);
            } else {
                tg(t, d, T_UBAR, c, s) = tg(t, d, T_U, c, s);
                tg(t, d, T_VBAR, c, s) = tg(t, d, T_V, c, s);
                tg(t, d, T_PBAR, c, s) = tg(t, d, T_P, c, s);
            }
            tg(t, d, T_UT, c, s) = tg(t, d, T_UBAR, c, s);
            tg(t, d, T_VT, c, s) = tg(t, d, T_VBAR, c, s);
            tg(t, d, T_J2P, c, s) = 0.0;
            tg(t, d, T_ADVP, c, s) = tg(t, d, T_UBAR, c, s);
        } else if (tag == INLET && ph.has_inlet && d.x[s] >= ph.x_in) {
            const double du = tg(t, d, T_U, c, s), dv = tg(t, d, T_V, c, s), dp = tg(t, d, T_P, c, s);
            for (int q = 0; q < ph.n_avg; ++q) {
                tg(t, d, T_RING + 3 * q + 0, c, s) = du;
                tg(t, d, T_RING + 3 * q + 1, c, s) = dv;
                tg(t, d, T_RING + 3 * q + 2, c, s) = dp;
            }
            tg(t, d, T_UBAR, c, s) = du;
            tg(t, d, T_VBAR, c, s) = dv;
            tg(t, d, T_PBAR, c, s) = dp;
            tg(t, d, T_J2, c, s) = 0.0;
        }
    }
}

// After the value kernel: the new inlet particles (parent p -> slot s, recorded by
// k_end_step) take x - L_in and p of the parent and the inlet profile's mode shapes; every
// other tangent of the slot starts at zero.  Then the drag tangents of the step.
__global__ void __launch_bounds__(1024) t_recycle_post(Dev d, TDev t)
{
    __shared__ double sh[2][1024];
    const int c = blockIdx.y;
    const Phys &ph = d.ph;
    const Counters *C = d.cnt;
    const int ns = C->last_spawn;
    for (int r = threadIdx.x; r < ns; r += blockDim.x) {
        const int2 m = d.spawn_map[r];
        const int ps = m.x, s = m.y;
        for (int f = 0; f < T_NF; ++f) tg(t, d, f, c, s) = 0.0;
        tg(t, d, T_X, c, s) = tg(t, d, T_X, c, ps);
        tg(t, d, T_Y, c, s) = tg(t, d, T_Y, c, ps);
        tg(t, d, T_P, c, s) = tg(t, d, T_P, c, ps);
        const double du = c < ph.n_modes ? mode_shape(ph, c, d.y[s]) : 0.0;
        tg(t, d, T_U, c, s) = du;
        tg(t, d, T_UT, c, s) = du;
    }
    double fx = 0.0, fy = 0.0;
    for (int i = threadIdx.x; i < C->n_drag; i += blockDim.x) {
        const int s = d.drag_slots[i];
        fx += tg(t, d, T_FX, c, s);
        fy += tg(t, d, T_FY, c, s);
    }
    sh[0][threadIdx.x] = fx;
    sh[1][threadIdx.x] = fy;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int slot = (C->step - 1 + d.max_history) % d.max_history;
        t.hist[((size_t)slot * 2 + 0) * T_DIR + c] = sh[0][0];
        t.hist[((size_t)slot * 2 + 1) * T_DIR + c] = sh[1][0];
    }
}

// Set-up: every tangent zero but the inlet particles' velocity (the mode shapes).
__global__ void t_init(Dev d, TDev t)
{
    const int c = blockIdx.y;
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        for (int f = 0; f < T_NF; ++f) tg(t, d, f, c, s) = 0.0;
        if (d.tag[s] == INLET) {
            const double du = c < ph.n_modes ? mode_shape(ph, c, d.y[s]) : 0.0;
            tg(t, d, T_U, c, s) = du;
            tg(t, d, T_UT, c, s) = du;
        }
    }
}

// ------------------------------------------------- fp32 pair tangents (passes A and B)
// The pair passes dominate the tangent step; their derivative arithmetic runs in fp32 duals
// on the fp32 pipe (GB300's fp64 pipe is 1/76 of it).  Values come from fp32 copies of the
// fp64 fields (t_prep), separations from the cell-relative fp32 coordinates of the membership
// test, and the differences that cancel (p_j - p_i, u_i - u_j, v_i - v_j) from the fp64
// values, rounded once.

// Neighbours of sorted particle k with the membership test of the value kernels; f(j, dx, dy,
// r2) with the fp32 separation r_k - r_j.
template <class F>
__device__ __forceinline__ void t_walk_f(const Dev &d, int k, double qx, double qy, F &&f)
{
    const Geo &g = d.g;
    const int cc = d.cellk[k];
    const float4 pk = d.P[k];
    for_block(d, cc % g.nx, cc / g.nx, [&](int ox, int oy, int j0, int j1) {
        const float rxo = pk.x - (float)ox * g.sxf, ryo = pk.y - (float)oy * g.syf;
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            if (is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f)) f(j, dxf, dyf, r2f);
        }
    });
}

// fp32 dual numbers with TG derivatives: the pair kernels carry TG directions per thread, so
// that the neighbour walk and the values are evaluated once for all of them (the value parts
// of every operation are shared; only the derivative parts repeat per direction).
constexpr int TG = 4;
static_assert(T_DIR % TG == 0, "directions per thread");
struct FG {
    float v, d[TG];
    __device__ FG() : v(0.0f)
    {
#pragma unroll
        for (int g = 0; g < TG; ++g) d[g] = 0.0f;
    }
    __device__ explicit FG(float a) : v(a)
    {
#pragma unroll
        for (int g = 0; g < TG; ++g) d[g] = 0.0f;
    }
};
__device__ __forceinline__ FG operator+(const FG &a, const FG &b)
{
    FG r;
    r.v = a.v + b.v;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = a.d[g] + b.d[g];
    return r;
}
__device__ __forceinline__ FG operator-(const FG &a, const FG &b)
{
    FG r;
    r.v = a.v - b.v;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = a.d[g] - b.d[g];
    return r;
}
__device__ __forceinline__ FG operator-(const FG &a)
{
    FG r;
    r.v = -a.v;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = -a.d[g];
    return r;
}
__device__ __forceinline__ FG operator*(const FG &a, const FG &b)
{
    FG r;
    r.v = a.v * b.v;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = fmaf(a.d[g], b.v, a.v * b.d[g]);
    return r;
}
__device__ __forceinline__ FG operator*(float s, const FG &a)  // a constant times a dual
{
    FG r;
    r.v = s * a.v;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = s * a.d[g];
    return r;
}
__device__ __forceinline__ FG operator/(const FG &a, const FG &b)
{
    const float rb = 1.0f / b.v;
    FG r;
    r.v = a.v * rb;
#pragma unroll
    for (int g = 0; g < TG; ++g) r.d[g] = (a.d[g] - r.v * b.d[g]) * rb;
    return r;
}
__device__ __forceinline__ FG &operator+=(FG &a, const FG &b) { a = a + b; return a; }

// fp32 copies of the fields the pair tangents read, by sorted index (after the value boundary
// kernel, so that wall and inlet pressures are the ones pass B uses)
__global__ void t_prep(Dev d, TDev t)
{
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double2 pv = d.PV[k], rm = d.RM[k], uv = d.UV[k], duv = d.DUV[k];
        t.vf[k] = make_float4(d2f(pv.x), d2f(pv.y), d2f(rm.x), d2f(rm.y));
        t.vg[k] = make_float4(d2f(uv.x), d2f(uv.y), d2f(duv.x), d2f(duv.y));
    }
}

// Directions c0 .. c0 + TG - 1 (blockIdx.y TG) of pass A's tangents: dW = W'(r) dr with
// dr = (r_ij . dr_ij) / r, summed to d(sum W) and d(sum m W).
__global__ void t_pass_a_f(Dev d, TDev t)
{
    const int c0 = blockIdx.y * TG;
    const int n = d.cnt->n_alive;
    const Phys &ph = d.ph;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int i = d.order[k];
        const double2 xi = d.XY[k];
        float tx[TG], ty[TG], dS[TG], dR[TG];
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            tx[g] = tg(t, d, T_X, c0 + g, i);
            ty[g] = tg(t, d, T_Y, c0 + g, i);
            dS[g] = dR[g] = 0.0f;
        }
        t_walk_f(d, k, xi.x, xi.y, [&](int j, float dx, float dy, float r2) {
            if (!(r2 > 0.0f)) return;  // self: W(0), no derivative
            const int sj = d.order[j];
            const float r = sqrtf(r2);
            const float dwq = quintic_dw(r * ph.inv_hf);
            const float base = ph.a2hf * dwq / r;  // dW = base (r_ij . dr_ij)
            const float mj = __ldg(d.P + j).z;
#pragma unroll
            for (int g = 0; g < TG; ++g) {
                const float ddx = tx[g] - tg(t, d, T_X, c0 + g, sj);
                const float ddy = ty[g] - tg(t, d, T_Y, c0 + g, sj);
                const float dW = base * fmaf(dx, ddx, dy * ddy);
                dS[g] += dW;
                dR[g] = fmaf(mj, dW, dR[g]);
            }
        });
        const double V = d.PV[k].y;
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            tg(t, d, T_RHO, c0 + g, i) = dR[g];
            tg(t, d, T_VOL, c0 + g, i) = d2f(-f2d(dS[g]) * V * V);
        }
    }
}

struct FluidG {
    FG p, u, v, rho, V, mrho, dut, dvt;
};
__device__ __forceinline__ FluidG fluid_g(const Dev &d, const TDev &t, int c0, int j)
{
    const int s = d.order[j];
    const float4 a = t.vf[j], b = t.vg[j];
    FluidG f;
    f.p.v = a.x; f.V.v = a.y; f.rho.v = a.z; f.mrho.v = a.w;
    f.u.v = b.x; f.v.v = b.y; f.dut.v = b.z; f.dvt.v = b.w;
    const float mr_rho = -a.w / a.z;  // d(m/rho) = -(m/rho) drho / rho
#pragma unroll
    for (int g = 0; g < TG; ++g) {
        const int c = c0 + g;
        f.p.d[g] = tg(t, d, T_P, c, s);
        f.V.d[g] = tg(t, d, T_VOL, c, s);
        f.rho.d[g] = tg(t, d, T_RHO, c, s);
        f.mrho.d[g] = mr_rho * f.rho.d[g];
        const float tu = tg(t, d, T_U, c, s), tv = tg(t, d, T_V, c, s);
        f.u.d[g] = tu;
        f.v.d[g] = tv;
        f.dut.d[g] = tg(t, d, T_UT, c, s) - tu;
        f.dvt.d[g] = tg(t, d, T_VT, c, s) - tv;
    }
    return f;
}

// Pass B's tangents for directions c0 .. c0 + TG - 1: the value kernel's pair terms in dual
// numbers, with the differences that cancel (p_j - p_i, u_i - u_j) taken in fp64 and rounded
// once.
__global__ void t_pass_b_f(Dev d, TDev t)
{
    const int c0 = blockIdx.y * TG;
    const Phys &ph = d.ph;
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int tag = d.stag[k] & 0x7f;
        const bool fl = (tag == FLUID || tag == INLET);
        const bool solid = drag_mode(ph, tag) != 0;
        if (!fl && !solid) continue;
        const int i = d.order[k];
        const double2 xy = d.XY[k];
        const double2 pvi = d.PV[k], uvi = d.UV[k];
        float tx[TG], ty[TG];
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            tx[g] = tg(t, d, T_X, c0 + g, i);
            ty[g] = tg(t, d, T_Y, c0 + g, i);
        }
        const FluidG fi = fluid_g(d, t, c0, k);
        const float mi_inv = 1.0f / d2f(d.Ms[k]);
        const int N = d.snnb[k];
        FG ax, ay, apd, gxs, gys, sdp;
        t_walk_f(d, k, xy.x, xy.y, [&](int j, float dxf, float dyf, float r2f) {
            const FluidG fj = fluid_g(d, t, c0, j);
            const double2 pvj = d.PV[j];
            FG dp = fj.p - fi.p;
            dp.v = d2f(pvj.x - pvi.x);
            sdp += dp;
            if (solid && (d.stag[j] & 0x7f) != FLUID) return;
            const int sj = d.order[j];
            FG dx, dy, r2;
            dx.v = dxf;
            dy.v = dyf;
            r2.v = r2f;
#pragma unroll
            for (int g = 0; g < TG; ++g) {
                dx.d[g] = tx[g] - tg(t, d, T_X, c0 + g, sj);
                dy.d[g] = ty[g] - tg(t, d, T_Y, c0 + g, sj);
                r2.d[g] = 2.0f * fmaf(dxf, dx.d[g], dyf * dy.d[g]);
            }
            FG F;
            if (r2f > 0.0f) {
                const float r = sqrtf(r2f);
                FG rr;
                rr.v = r;
                const float h2r = 0.5f / r;
#pragma unroll
                for (int g = 0; g < TG; ++g) rr.d[g] = r2.d[g] * h2r;
                // w'(q) and w''(q) at q = r / h: F = alpha_2/h w'(q) / r as a dual
                const float q = r * ph.inv_hf;
                const float t3 = q < 3.0f ? 3.0f - q : 0.0f;
                const float t2 = q < 2.0f ? 2.0f - q : 0.0f;
                const float t1 = q < 1.0f ? 1.0f - q : 0.0f;
                const float a = t3 * t3, b = t2 * t2, c = t1 * t1;
                const float w1 = -5.0f * (a * a - 6.0f * b * b + 15.0f * c * c);
                const float w2 = 20.0f * (t3 * a - 6.0f * (t2 * b) + 15.0f * (t1 * c));
                FG dwq;
                dwq.v = w1;
#pragma unroll
                for (int g = 0; g < TG; ++g) dwq.d[g] = w2 * (rr.d[g] * ph.inv_hf);
                F = (ph.a2hf * dwq) / rr;
            }
            const FG gx = F * dx, gy = F * dy, gdotr = F * r2;
            const FG cij = fi.V * fi.V + fj.V * fj.V;
            const FG inv_rs = FG(1.0f) / (fi.rho + fj.rho);
            const FG e_ = fi.rho * dp * inv_rs;
            FG r2e = r2;
            r2e.v += ph.eh2f;
            const FG hf = fi.rho * fj.rho * inv_rs * gdotr / r2e;
            const FG vis = (2.0f * ph.nuf) * hf;
            const double2 uvj = d.UV[j];
            FG uij = fi.u - fj.u, vij = fi.v - fj.v;
            uij.v = d2f(uvi.x - uvj.x);
            vij.v = d2f(uvi.y - uvj.y);
            const FG cgx = cij * gx, cgy = cij * gy;
            gxs += cgx;
            gys += cgy;
            if (solid) {
                ax += cij * (vis * uij) - e_ * cgx;
                ay += cij * (vis * vij) - e_ * cgy;
                return;
            }
            const FG Ai = fi.rho * (fi.dut * gx + fi.dvt * gy);
            const FG Aj = fj.rho * (fj.dut * gx + fj.dvt * gy);
            ax += cij * (0.5f * (fi.u * Ai + fj.u * Aj) + vis * uij) - e_ * cgx;
            ay += cij * (0.5f * (fi.v * Ai + fj.v * Aj) + vis * vij) - e_ * cgy;
            apd += (ph.c2f * fi.rho) * fj.mrho * (uij * gx + vij * gy) -
                   (mi_inv * 2.0f * ph.nuef) * (cij * hf * dp);
        });
        FG corr;
        if (ph.use_pavg && !solid) {
            corr = sdp / FG((float)N);
        } else {
            corr = -fi.p;
            corr.v = -d2f(pvi.x);
        }
        const FG fxv = ax + corr * gxs, fyv = ay + corr * gys;
#pragma unroll
        for (int g = 0; g < TG; ++g) {
            const int c = c0 + g;
            if (solid) {
                tg(t, d, T_FX, c, i) = fxv.d[g];
                tg(t, d, T_FY, c, i) = fyv.d[g];
            } else {
                tg(t, d, T_AU, c, i) = fxv.d[g] * mi_inv;
                tg(t, d, T_AV, c, i) = fyv.d[g] * mi_inv;
                tg(t, d, T_AP, c, i) = apd.d[g];
                tg(t, d, T_ABU, c, i) = -ph.pbf * mi_inv * gxs.d[g];
                tg(t, d, T_ABV, c, i) = -ph.pbf * mi_inv * gys.d[g];
            }
        }
    }
}

TDev tdev_of(const Dev &d, void *ws)
{
    TDev t;
    float *p = (float *)ws;
    for (int f = 0; f < T_NF; ++f) {
        t.f[f] = p;
        p += (size_t)T_DIR * d.cap;
    }
    t.hist = (double *)p;  // T_DIR * cap floats per field: a multiple of 8 bytes
    t.vf = (float4 *)(((uintptr_t)(t.hist + (size_t)d.max_history * 2 * T_DIR) + 15) & ~(uintptr_t)15);
    t.vg = t.vf + d.cap;
    t.ndir = T_DIR;
    return t;
}

dim3 tgrid(int n)
{
    int b = (n + 127) / 128;
    b = b < 1 ? 1 : (b > 4096 ? 4096 : b);
    return dim3((unsigned)b, T_DIR);
}

// the pair kernels: TG directions per thread
dim3 tgrid_pair(int n)
{
    const dim3 g = tgrid(n);
    return dim3(g.x, T_DIR / TG);
}

}  // namespace

size_t tangent_bytes(const Dev &d)
{
    return sizeof(float) * (size_t)T_NF * T_DIR * d.cap + sizeof(double) * (size_t)d.max_history * 2 * T_DIR +
           16 + 2 * sizeof(float4) * (size_t)d.cap;
}

const double *tangent_hist(const Dev &d, const void *ws)
{
    return tdev_of(d, const_cast<void *>(ws)).hist;
}

int launch_tangent(const Dev &d, void *ws, cudaStream_t s, int what, double tau)
{
    const TDev t = tdev_of(d, ws);
    switch (what) {
    case TG_INIT: t_init<<<tgrid(d.cap), 128, 0, s>>>(d, t); return 1;
    case TG_PASS_A: t_pass_a_f<<<tgrid_pair(d.cap), 128, 0, s>>>(d, t); return 1;
    case TG_BOUNDARY: {
        const dim3 gb = tgrid(d.cap / 8 + 1);
        t_walls_inlet<<<dim3(gb.x, T_DIR / TGW), 128, 0, s>>>(d, t);
        return 1;
    }
    case TG_PASS_B:
        t_prep<<<tgrid(d.cap).x, 128, 0, s>>>(d, t);
        t_pass_b_f<<<tgrid_pair(d.cap), 128, 0, s>>>(d, t);
        return 2;
    case TG_OUTLET:
        t_snapshot<<<tgrid(d.cap), 128, 0, s>>>(d, t);
        t_outlet<<<tgrid(d.cap / 8 + 1), 128, 0, s>>>(d, t);
        return 2;
    case TG_STAGE_PRED: t_stage<false><<<tgrid(d.cap), 128, 0, s>>>(d, t, tau); return 1;
    case TG_STAGE_CORR: t_stage<true><<<tgrid(d.cap), 128, 0, s>>>(d, t, tau); return 1;
    case TG_RECYCLE_PRE: t_recycle_pre<<<tgrid(d.cap), 128, 0, s>>>(d, t); return 1;
    case TG_RECYCLE_POST: t_recycle_post<<<dim3(1, T_DIR), 1024, 0, s>>>(d, t); return 1;
    default: return 0;
    }
}

}  // namespace edac
