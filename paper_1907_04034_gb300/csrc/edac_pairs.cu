// Pair kernels of the EDAC SPH library (sm_103a): pass A (summation density and
// number-density volume), the boundary kernel (solid-wall projection, mirrored inlet
// pressure, hybrid-outlet update) and pass B (EDAC-TVF momentum, EDAC pressure rate,
// background-pressure acceleration, solid force).
//
// One thread per particle in cell order; the 3x3 block of cells around the particle's
// cell is walked with an fp32 pre-test on cell-relative coordinates (for_neighbors).
// MIXED = 1 evaluates the pair terms in fp32 on cell-relative coordinates with per-cell
// partial sums folded into two-sum compensated accumulators; MIXED = 0 evaluates them in
// fp64 on the canonical fp64 separations.
#include "edac_internal.cuh"

namespace edac {

namespace {

constexpr int TPB = 128;

__device__ __forceinline__ void cell_of(const Dev &d, int k, int &cx, int &cy)
{
    const int c = d.cellk[k];
    cx = c % d.g.nx;
    cy = c / d.g.nx;
}

// ---------------------------------------------------------------------------- pass A
// S_i = sum_j W_ij, V_i = 1/S_i (number-density volume, Sec. 2), rho_i = sum_j m_j W_ij
// (Eq. summation-density), N_i = number of neighbours (self included).
struct PassA32 {
    const Dev &d;
    float a2, inv_h;
    float s_hi = 0.f, s_lo = 0.f, r_hi = 0.f, r_lo = 0.f, cs = 0.f, cr = 0.f;
    int n = 0;
    __device__ PassA32(const Dev &dd) : d(dd), a2(dd.ph.a2f), inv_h(dd.ph.inv_hf) {}
    __device__ void begin_cell() { cs = 0.f; cr = 0.f; }
    __device__ void end_cell() { two_sum_acc(s_hi, s_lo, cs); two_sum_acc(r_hi, r_lo, cr); }
    __device__ void operator()(int j, float, float, float r2f, double, double, double, bool,
                               const float4 &pj)
    {
        const float w = a2 * quintic_w(sqrtf(r2f) * inv_h);
        cs += w;
        cr += pj.z * w;
        ++n;
    }
};

struct PassA64 {
    const Dev &d;
    double a2, inv_h;
    double s = 0.0, r = 0.0;
    int n = 0;
    __device__ PassA64(const Dev &dd) : d(dd), a2(dd.ph.a2), inv_h(dd.ph.inv_h) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int j, float, float, float, double, double, double er2, bool,
                               const float4 &)
    {
        const double w = a2 * quintic_w(sqrt(er2) * inv_h);
        s += w;
        r += d.Ms[j] * w;
        ++n;
    }
};

template <int MIXED>
__global__ void __launch_bounds__(TPB) k_pass_a(Dev d)
{
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pi = d.P[k];
        const double2 xy = d.XY[k];
        const int s = d.order[k];
        if (MIXED) {
            PassA32 f(d);
            for_neighbors<false>(d, xy.x, xy.y, cx, cy, pi.x, pi.y, f);
            const float S = f.s_hi + f.s_lo, R = f.r_hi + f.r_lo;
            const float V = 1.0f / S;
            const float4 q = d.Qf[k];
            d.Qf[k] = make_float4(q.x, V, R, pi.z / R);
            d.snnb[k] = f.n;
            d.rho[s] = (double)R;
            d.vol[s] = (double)V;
            d.nnb[s] = f.n;
        } else {
            PassA64 f(d);
            for_neighbors<true>(d, xy.x, xy.y, cx, cy, pi.x, pi.y, f);
            const double V = 1.0 / f.s;
            const double mk = d.Ms[k];
            d.PV[k].y = V;
            d.RM[k] = make_double2(f.r, mk / f.r);
            d.snnb[k] = f.n;
            d.rho[s] = f.r;
            d.vol[s] = V;
            d.nnb[s] = f.n;
        }
    }
}

// --------------------------------------------------------------------- boundary kernel
template <int MIXED>
__device__ __forceinline__ void fluid_fields(const Dev &d, int j, double &p, double &u, double &v,
                                             double &mrho)
{
    if (MIXED) {
        const float4 q = d.Qf[j];
        const float4 b = d.Bf[j];
        p = q.x; u = b.x; v = b.y; mrho = q.w;
    } else {
        const double2 pv = d.PV[j], uv = d.UV[j];
        p = pv.x; u = uv.x; v = uv.y; mrho = d.RM[j].y;
    }
}

// Shepard sums of fluid neighbours of a wall particle.
template <int MIXED>
struct WallSums {
    const Dev &d;
    double sw = 0, sp = 0, su = 0, sv = 0;
    __device__ WallSums(const Dev &dd) : d(dd) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int j, float, float, float, double, double, double er2, bool,
                               const float4 &)
    {
        if ((d.stag[j] & 0x7f) != FLUID) return;
        const double w = d.ph.a2 * quintic_w(sqrt(er2) * d.ph.inv_h);
        double p, u, v, mr;
        fluid_fields<MIXED>(d, j, p, u, v, mr);
        sw += w; sp += w * p; su += w * u; sv += w * v;
    }
};

// Moment sums of the mirror system, Eq. (matform), around mirror point k over fluid l:
// rows (W, W_x, W_y) V_l, columns (1, x_lk, y_lk), right-hand side p_l.
template <int MIXED>
struct MirrorSums {
    const Dev &d;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
    int nl = 0;
    __device__ MirrorSums(const Dev &dd) : d(dd) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int l, float, float, float, double edx, double edy, double er2,
                               bool, const float4 &)
    {
        if ((d.stag[l] & 0x7f) != FLUID) return;
        // for_neighbors gives r_k - r_l; the system is written in r_lk = r_l - r_k
        const double xlk = -edx, ylk = -edy;
        const double r = sqrt(er2);
        double p, u, v, Vl;
        fluid_fields<MIXED>(d, l, p, u, v, Vl);
        const double w = d.ph.a2 * quintic_w(r * d.ph.inv_h);
        double wx = 0.0, wy = 0.0;
        if (r > 0.0) {
            const double dw = d.ph.a2h * quintic_dw(r * d.ph.inv_h);
            wx = dw * xlk / r;
            wy = dw * ylk / r;
        }
        const double row[3] = {w * Vl, wx * Vl, wy * Vl};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            M[a][0] += row[a];
            M[a][1] += xlk * row[a];
            M[a][2] += ylk * row[a];
            b[a] += p * row[a];
        }
        ++nl;
    }
};

// Gaussian elimination with partial pivoting on a 3x3 system.
__device__ bool solve3(double A[3][3], double b[3], double x[3])
{
    int piv[3] = {0, 1, 2};
    for (int c = 0; c < 3; ++c) {
        int best = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[piv[r]][c]) > fabs(A[piv[best]][c])) best = r;
        const int tmp = piv[c]; piv[c] = piv[best]; piv[best] = tmp;
        const double dg = A[piv[c]][c];
        if (dg == 0.0) return false;
        for (int r = c + 1; r < 3; ++r) {
            const double f = A[piv[r]][c] / dg;
            for (int k = c; k < 3; ++k) A[piv[r]][k] -= f * A[piv[c]][k];
            b[piv[r]] -= f * b[piv[c]];
        }
    }
    for (int c = 2; c >= 0; --c) {
        double s = b[piv[c]];
        for (int k = c + 1; k < 3; ++k) s -= A[piv[c]][k] * x[k];
        x[c] = s / A[piv[c]][c];
    }
    return true;
}

// Characteristic sums of an outlet particle: fluid J2 (Shepard, Eq. shepard) and the
// previous step's J2 and advection velocity of red outlet neighbours (Eq. average_old).
struct OutletSums {
    const Dev &d;
    double sw = 0, sj = 0, sjp = 0, sadv = 0;
    int nf = 0, mr = 0;
    __device__ OutletSums(const Dev &dd) : d(dd) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int j, float, float, float, double, double, double er2, bool,
                               const float4 &)
    {
        const uint8_t t = d.stag[j];
        if ((t & 0x7f) == FLUID) {
            const double w = d.ph.a2 * quintic_w(sqrt(er2) * d.ph.inv_h);
            sw += w;
            sj += w * d.AUX[j].x;
            ++nf;
        } else if (t == (OUTLET | TAG_REDP)) {
            const double2 a = d.AUX[j];
            sjp += a.x;
            sadv += a.y;
            ++mr;
        }
    }
};

template <int MIXED>
__global__ void __launch_bounds__(TPB) k_boundary(Dev d, int end_of_step)
{
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int nb = d.cnt->n_bnd;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
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
            WallSums<MIXED> f(d);
            for_neighbors<true>(d, xy.x, xy.y, cx, cy, pk.x, pk.y, f);
            const int wi = (t == WALL) ? 0 : 1;
            double pw, ug, vg;
            if (f.sw > 0.0) {
                pw = f.sp / f.sw;
                const double uf = f.su / f.sw, vf = f.sv / f.sw;
                if (ph.wall_slip[wi]) { ug = uf; vg = -vf; }
                else { ug = 2.0 * ph.wall_u[wi] - uf; vg = 2.0 * ph.wall_v[wi] - vf; }
            } else {
                pw = 0.0; ug = ph.wall_u[wi]; vg = ph.wall_v[wi];
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
            d.p[s] = pw; d.u[s] = ug; d.v[s] = vg; d.ut[s] = ug; d.vt[s] = vg;
        } else if (t == INLET && ph.has_inlet) {
            // Mirrored inlet pressure (Sec. 3.2): first-order Taylor system at the mirror
            // point k = (2 x_in - x_o, y_o) over fluid l, then p_o = p_k - (r_o - r_k).grad p_k
            // (Eq. taylor2).  No fluid in reach: p_o = 0; singular system
            // (|det| <= 1e-9 |M00 M11 M22|): the Shepard value sum p W V / sum W V.
            const double xk = 2.0 * ph.x_in - xy.x, yk = xy.y;
            const int cx = cell_coord(xk, g.x_min, g.inv_sx, g.nx);
            const int cy = cell_coord(yk, g.y_min, g.inv_sy, g.ny);
            const float rx = (float)(xk - (g.x_min + (double)cx * g.sx));
            const float ry = (float)(yk - (g.y_min + (double)cy * g.sy));
            MirrorSums<MIXED> f(d);
            for_neighbors<true>(d, xk, yk, cx, cy, rx, ry, f);
            double pk = 0.0, gxp = 0.0, gyp = 0.0;
            if (f.nl > 0) {
                const double det =
                    f.M[0][0] * (f.M[1][1] * f.M[2][2] - f.M[1][2] * f.M[2][1]) -
                    f.M[0][1] * (f.M[1][0] * f.M[2][2] - f.M[1][2] * f.M[2][0]) +
                    f.M[0][2] * (f.M[1][0] * f.M[2][1] - f.M[1][1] * f.M[2][0]);
                pk = f.b[0] / f.M[0][0];
                if (!(fabs(det) <= 1e-9 * fabs(f.M[0][0] * f.M[1][1] * f.M[2][2]))) {
                    double A[3][3], rhs[3], sol[3];
                    for (int a = 0; a < 3; ++a) {
                        rhs[a] = f.b[a];
                        for (int c = 0; c < 3; ++c) A[a][c] = f.M[a][c];
                    }
                    if (solve3(A, rhs, sol)) { pk = sol[0]; gxp = sol[1]; gyp = sol[2]; }
                }
            }
            const double po = pk - ((xy.x - xk) * gxp + (xy.y - yk) * gyp);
            if (MIXED) {
                float4 q = d.Qf[k];
                q.x = (float)po;
                d.Qf[k] = q;
            } else {
                d.PV[k].x = po;
            }
            d.p[s] = po;
        } else if (t == OUTLET && end_of_step && ph.has_outlet) {
            // Hybrid outlet (Sec. 3.4): red particles (fluid in reach) take the Shepard J2
            // of the fluid; blue ones the mean previous-step J2 of red outlet neighbours.
            // J3 = 0 gives p' = J2/2, u' = J2/(2 rho0 c); value = frozen average + acoustic
            // part (Eq. acou).  Written to the slot arrays only: the rates of this
            // evaluation still see the outlet values of the step.
            int cx, cy;
            cell_of(d, k, cx, cy);
            const float4 pk = d.P[k];
            OutletSums f(d);
            for_neighbors<true>(d, xy.x, xy.y, cx, cy, pk.x, pk.y, f);
            const bool red = f.nf > 0;
            const double J2 = red ? f.sj / f.sw : (f.mr > 0 ? f.sjp / (double)f.mr : 0.0);
            const double rc = ph.rho0 * ph.cs;
            const double un = d.ubar[s] + J2 / (2.0 * rc);
            const double adv = red ? un : (f.mr > 0 ? f.sadv / (double)f.mr : d.ubar[s]);
            d.u[s] = un;
            d.v[s] = d.vbar[s];
            d.p[s] = d.pbar[s] + 0.5 * J2;
            d.ut[s] = un;
            d.vt[s] = d.vbar[s];
            d.J2p[s] = J2;
            d.advp[s] = adv;
            d.redp[s] = red ? 1 : 0;
        }
    }
}

// ---------------------------------------------------------------------------- pass B
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
// G_i = sum_j c_ij gW, which is also the background-pressure sum.
// Solid particles counted in the drag: F_i = sum_{j fluid} c_ij [ -p~_ij gW + eta~_ij
// u_ij (gW . r_ij)/(r^2 + eta h^2) ] with u_ij = u_g,i - u_j (Eq. tvf-momentum_solid).
struct PassB32 {
    const Dev &d;
    // i-side
    float pi, Vi, rhoi, ui, vi, dui, dvi, mi_inv;
    bool solid;
    // constants
    float a2h, inv_h, c2, nu2, nue2, eh2;
    // accumulators (hi, lo) and per-cell partials
    float ax_h = 0, ax_l = 0, ay_h = 0, ay_l = 0, ap_h = 0, ap_l = 0, gx_h = 0, gx_l = 0,
          gy_h = 0, gy_l = 0;
    float cax = 0, cay = 0, cap_ = 0, cgx = 0, cgy = 0;
    float sdp = 0;
    __device__ PassB32(const Dev &dd) : d(dd)
    {
        a2h = dd.ph.a2hf; inv_h = dd.ph.inv_hf; c2 = dd.ph.c2f; nu2 = 2.0f * dd.ph.nuf;
        nue2 = 2.0f * dd.ph.nuef; eh2 = dd.ph.eh2f;
    }
    __device__ void begin_cell() { cax = cay = cap_ = cgx = cgy = 0.f; }
    __device__ void end_cell()
    {
        two_sum_acc(ax_h, ax_l, cax);
        two_sum_acc(ay_h, ay_l, cay);
        two_sum_acc(ap_h, ap_l, cap_);
        two_sum_acc(gx_h, gx_l, cgx);
        two_sum_acc(gy_h, gy_l, cgy);
    }
    __device__ void operator()(int j, float dx, float dy, float r2, double, double, double, bool,
                               const float4 &)
    {
        const float4 q = __ldg(d.Qf + j);  // (p, V, rho, m/rho)
        const float dp = q.x - pi;
        sdp += dp;
        if (solid && (d.stag[j] & 0x7f) != FLUID) return;
        const float4 bj = __ldg(d.Bf + j);  // (u, v, u~-u, v~-v)
        const float r = sqrtf(r2);
        const float dwq = quintic_dw(r * inv_h);
        const float F = r > 0.f ? a2h * dwq / r : 0.f;
        const float gx = F * dx, gy = F * dy, gdotr = F * r2;
        const float cij = Vi * Vi + q.y * q.y;
        const float inv_rs = 1.0f / (rhoi + q.z);
        const float e = rhoi * dp * inv_rs;
        // eta~_ij (gW . r_ij) / (r^2 + eta h^2) = 2 nu hf with hf = rho_i rho_j/(rho_i + rho_j) ...
        const float hf = rhoi * q.z * inv_rs * gdotr / (r2 + eh2);
        const float vis = nu2 * hf;
        const float uij = ui - bj.x, vij = vi - bj.y;
        const float cgxv = cij * gx, cgyv = cij * gy;
        cgx += cgxv;
        cgy += cgyv;
        if (solid) {
            cax += cij * (vis * uij) - e * cgxv;
            cay += cij * (vis * vij) - e * cgyv;
            return;
        }
        const float Ai = rhoi * (dui * gx + dvi * gy);
        const float Aj = q.z * (bj.z * gx + bj.w * gy);
        cax += cij * (0.5f * (ui * Ai + bj.x * Aj) + vis * uij) - e * cgxv;
        cay += cij * (0.5f * (vi * Ai + bj.y * Aj) + vis * vij) - e * cgyv;
        cap_ += rhoi * c2 * q.w * (uij * gx + vij * gy) - cij * mi_inv * nue2 * hf * dp;
    }
};

struct PassB64 {
    const Dev &d;
    double pi, Vi, rhoi, ui, vi, dui, dvi, mi_inv;
    bool solid;
    double ax = 0, ay = 0, apd = 0, gxs = 0, gys = 0, sdp = 0;
    __device__ PassB64(const Dev &dd) : d(dd) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int j, float, float, float, double dx, double dy, double r2, bool,
                               const float4 &)
    {
        const Phys &ph = d.ph;
        const double2 pv = d.PV[j];  // (p, V)
        const double dp = pv.x - pi;
        sdp += dp;
        if (solid && (d.stag[j] & 0x7f) != FLUID) return;
        const double2 rm = d.RM[j];  // (rho, m/rho)
        const double2 uv = d.UV[j];
        const double r = sqrt(r2);
        const double dwq = quintic_dw(r * ph.inv_h);
        const double F = r > 0.0 ? ph.a2h * dwq / r : 0.0;
        const double gx = F * dx, gy = F * dy, gdotr = F * r2;
        const double cij = Vi * Vi + pv.y * pv.y;
        const double inv_rs = 1.0 / (rhoi + rm.x);
        const double e = rhoi * dp * inv_rs;
        const double hf = rhoi * rm.x * inv_rs * gdotr / (r2 + ph.eh2);
        const double vis = 2.0 * ph.nu * hf;
        const double uij = ui - uv.x, vij = vi - uv.y;
        const double cgxv = cij * gx, cgyv = cij * gy;
        gxs += cgxv;
        gys += cgyv;
        if (solid) {
            ax += cij * (vis * uij) - e * cgxv;
            ay += cij * (vis * vij) - e * cgyv;
            return;
        }
        const double2 duv = d.DUV[j];
        const double Ai = rhoi * (dui * gx + dvi * gy);
        const double Aj = rm.x * (duv.x * gx + duv.y * gy);
        ax += cij * (0.5 * (ui * Ai + uv.x * Aj) + vis * uij) - e * cgxv;
        ay += cij * (0.5 * (vi * Ai + uv.y * Aj) + vis * vij) - e * cgyv;
        apd += rhoi * ph.c2 * rm.y * (uij * gx + vij * gy) - cij * mi_inv * 2.0 * ph.nu_e * hf * dp;
    }
};

template <int MIXED>
__global__ void __launch_bounds__(TPB) k_pass_b(Dev d)
{
    const Phys &ph = d.ph;
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int t = d.stag[k] & 0x7f;
        const bool fl = (t == FLUID || t == INLET);
        const bool solid = (t == WALL && ph.wall_drag[0]) || (t == SLIPWALL && ph.wall_drag[1]);
        if (!fl && !solid) continue;
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pk = d.P[k];
        const double2 xy = d.XY[k];
        const int s = d.order[k];
        const int N = d.snnb[k];
        const double mi = d.m[s];
        double sx, sy, spd, G0, G1, sdp, pi;
        if (MIXED) {
            PassB32 f(d);
            const float4 q = d.Qf[k];
            const float4 b = d.Bf[k];
            f.pi = q.x; f.Vi = q.y; f.rhoi = q.z; f.ui = b.x; f.vi = b.y; f.dui = b.z; f.dvi = b.w;
            f.mi_inv = 1.0f / pk.z;
            f.solid = solid;
            for_neighbors<false>(d, xy.x, xy.y, cx, cy, pk.x, pk.y, f);
            sx = (double)f.ax_h + (double)f.ax_l;
            sy = (double)f.ay_h + (double)f.ay_l;
            spd = (double)f.ap_h + (double)f.ap_l;
            G0 = (double)f.gx_h + (double)f.gx_l;
            G1 = (double)f.gy_h + (double)f.gy_l;
            sdp = f.sdp;
            pi = q.x;
        } else {
            PassB64 f(d);
            const double2 pv = d.PV[k], rm = d.RM[k], uv = d.UV[k], duv = d.DUV[k];
            f.pi = pv.x; f.Vi = pv.y; f.rhoi = rm.x; f.ui = uv.x; f.vi = uv.y;
            f.dui = duv.x; f.dvi = duv.y;
            f.mi_inv = 1.0 / d.Ms[k];
            f.solid = solid;
            for_neighbors<true>(d, xy.x, xy.y, cx, cy, pk.x, pk.y, f);
            sx = f.ax; sy = f.ay; spd = f.apd; G0 = f.gxs; G1 = f.gys; sdp = f.sdp;
            pi = pv.x;
        }
        // -sum c p~ gW = -sum c (pbar - p_i) gW + (p_avg - p_i) G   (with p_avg) or - p_i G
        const double corr = ph.use_pavg ? sdp / (double)N : -pi;
        if (solid) {
            d.fx[s] = sx + corr * G0;
            d.fy[s] = sy + corr * G1;
        } else {
            d.au[s] = (sx + corr * G0) / mi + ph.gx;
            d.av[s] = (sy + corr * G1) / mi + ph.gy;
            d.ap[s] = spd;
            d.abu[s] = -ph.pb / mi * G0;
            d.abv[s] = -ph.pb / mi * G1;
        }
    }
}

// Debug: exact neighbour ids of every particle, with the membership test of the passes.
struct DumpIds {
    const Dev &d;
    unsigned long long *out;
    long long pos, end;
    __device__ DumpIds(const Dev &dd, unsigned long long *o, long long b, long long e)
        : d(dd), out(o), pos(b), end(e) {}
    __device__ void begin_cell() {}
    __device__ void end_cell() {}
    __device__ void operator()(int j, float, float, float, double, double, double, bool,
                               const float4 &)
    {
        if (pos < end) out[pos] = d.id[d.order[j]];
        ++pos;
    }
};

template <int MIXED>
__global__ void k_dump(Dev d, const long long *start, unsigned long long *ids)
{
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pk = d.P[k];
        const double2 xy = d.XY[k];
        DumpIds f(d, ids, start[k], start[k + 1]);
        for_neighbors<MIXED == 0>(d, xy.x, xy.y, cx, cy, pk.x, pk.y, f);
    }
}

int grid_for(int n)
{
    int b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : b;
}

}  // namespace

int launch_pass_a(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_a<1><<<grid_for(d.cap), TPB, 0, s>>>(d);
    else k_pass_a<0><<<grid_for(d.cap), TPB, 0, s>>>(d);
    return 1;
}

int launch_boundary(const Dev &d, cudaStream_t s, int mixed, int end_of_step)
{
    if (mixed) k_boundary<1><<<grid_for(d.cap), TPB, 0, s>>>(d, end_of_step);
    else k_boundary<0><<<grid_for(d.cap), TPB, 0, s>>>(d, end_of_step);
    return 1;
}

int launch_pass_b(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_b<1><<<grid_for(d.cap), TPB, 0, s>>>(d);
    else k_pass_b<0><<<grid_for(d.cap), TPB, 0, s>>>(d);
    return 1;
}

int launch_neighbor_dump(const Dev &d, cudaStream_t s, int mixed, const long long *start,
                         unsigned long long *ids)
{
    if (mixed) k_dump<1><<<grid_for(d.cap), TPB, 0, s>>>(d, start, ids);
    else k_dump<0><<<grid_for(d.cap), TPB, 0, s>>>(d, start, ids);
    return 1;
}

}  // namespace edac
