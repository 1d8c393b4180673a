// Reverse-mode adjoint of the fp64 step: the gradient of a loss built from the step history
// (weights on the drag and lift of every step, and on the pressure energy of the fluid in an
// x-window, e.g. next to the outlet) with respect to the inlet-profile modes a_k of
// u(y) = U + sum_k a_k sin(k pi (y - y0) / H).
//
// The adjoint of every operation of a step is taken in reverse order (recycling, the second
// evaluation with the outlet update, the corrector with the time-average sample, the first
// evaluation, the predictor), with the neighbour sets, the acoustic-gate decisions, the
// red/blue outlet classes and the recycling events of the values held fixed, as in the tangent
// model.  The values each adjoint operation needs come from snapshots of the context's
// workspace: edac_adjoint_run keeps checkpoints every K steps and re-runs each segment once
// from its checkpoint, storing the workspace after the first evaluation and at the end of
// every step (cell-ordered copies and cell lists of that evaluation included) and the
// decisions of the step (tags before recycling, gate, ring write index).
//
// Every pair and boundary adjoint is a gather: the thread of a particle adds the derivatives
// of the sums it enters, its own and those of its neighbours, from coefficients its
// neighbours stored (so there are no atomics, and two runs agree bit for bit).  The
// derivatives are written out by hand from the value kernels' formulas (reverse order of the
// operations of each formula).  The adjoint fields ("lambda" of a field) are fp64 and
// slot-indexed, with per-evaluation temporaries indexed like the cell-ordered copies.  The
// pair-pass adjoints run in fp32 on the fp32 pipe, as the tangent model's pair tangents do
// (fp32 copies of the fields, separations from the cell-relative fp32 coordinates of the
// membership test, the differences that cancel taken in fp64 and rounded once); the boundary
// parts (walls, the inlet's 3x3 system, the outlet) in fp64.
#include "edac_internal.cuh"

namespace edac {
namespace {

constexpr int ATPB = 128;
constexpr int NCB = 6;   // pass B output coefficients per particle
constexpr int NBC = 10;  // boundary coefficients per particle

struct ADev {
    // lambdas of the slot fields [cap]
    double *x, *y, *u, *v, *ut, *vt, *p, *au, *av, *ap, *abu, *abv;
    double *x0, *y0, *u0, *v0, *p0;  // base-state lambdas gathered within a step
    double *ubar, *vbar, *pbar, *J2, *J2p, *advp;
    double *ring;  // [cap][NAVG_MAX][3]
    double *acc;   // [cap][T_DIR] parameter-gradient contributions of each slot
    // one evaluation, by sorted index [cap]
    double *rho, *V;  // lambdas of rho and V
    float *cb;        // [cap][NCB] pass B output coefficients (fp32)
    int *cbf;         // [cap] pass B function of the particle: 0 none, 1 fluid/inlet, 2 solid
    double *bc;       // [cap][NBC] boundary coefficients (walls, inlet mirror, outlet)
    float4 *fa, *fb;  // [cap] fp32 (V, rho, m, p) and (u, v, u~ - u, v~ - v), by sorted index
    // decisions of one step [cap] (views into rec_* at the step's record)
    uint8_t *tag_pre, *gate, *rpos_old;
    uint8_t *rec_tag, *rec_gate, *rec_rpos;  // [K][cap] the steps of a segment
    double *pe;       // [nsteps] pressure energy per step (forward)
    double *grad;     // [T_DIR] the reduced gradient
};

// ------------------------------------------------------------------------------ helpers
__device__ __forceinline__ int slot_of(const Dev &d, int k) { return d.order[k]; }

// Neighbours j of sorted particle k (self included), the membership test of the value
// kernels; f(j, dx, dy, r2) with the canonical fp64 separation r_k - r_j.
template <class F>
__device__ __forceinline__ void a_walk(const Dev &d, int k, F &&f)
{
    const Geo &g = d.g;
    const int cc = d.cellk[k];
    const float4 pk = d.P[k];
    const double2 xy = d.XY[k];
    for_block(d, cc % g.nx, cc / g.nx, [&](int ox, int oy, int j0, int j1) {
        const float rxo = pk.x - (float)ox * g.sxf, ryo = pk.y - (float)oy * g.syf;
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            if (!is_member(d, rxo, ryo, __ldg(d.P + j), j, xy.x, xy.y, dxf, dyf, r2f)) continue;
            const double2 xj = d.XY[j];
            double dx, dy;
            const double r2 = exact_r2(g, xy.x, xy.y, xj.x, xj.y, dx, dy);
            f(j, dx, dy, r2);
        }
    });
}

// quintic w, w' and w'' at q
__device__ __forceinline__ void quintic3(double q, double &w, double &w1, double &w2)
{
    const double t3 = q < 3.0 ? 3.0 - q : 0.0;
    const double t2 = q < 2.0 ? 2.0 - q : 0.0;
    const double t1 = q < 1.0 ? 1.0 - q : 0.0;
    const double a = t3 * t3, b = t2 * t2, c = t1 * t1;
    w = t3 * a * a - 6.0 * (t2 * b * b) + 15.0 * (t1 * c * c);
    w1 = -5.0 * (a * a - 6.0 * b * b + 15.0 * c * c);
    w2 = 20.0 * (t3 * a - 6.0 * (t2 * b) + 15.0 * (t1 * c));
}

// W(r) and dW/dr of the quintic spline (alpha_2 and alpha_2/h applied)
__device__ __forceinline__ void W_dW(const Phys &ph, double r, double &W, double &Wr)
{
    double w, w1, w2;
    quintic3(r * ph.inv_h, w, w1, w2);
    W = ph.a2 * w;
    Wr = ph.a2h * w1;
}

__device__ __forceinline__ double mode_shape_a(const Phys &ph, int c, double y)
{
    return sin((double)(c + 1) * 3.141592653589793 * (y - ph.in_y0) / ph.in_H);
}

// d u_in / d y of the steady inlet profile
__device__ __forceinline__ double inlet_dudy(const Phys &ph, double y)
{
    double s = 0.0;
    for (int k = 0; k < ph.n_modes; ++k) {
        const double kk = (double)(k + 1) * 3.141592653589793 / ph.in_H;
        s += ph.modes[k] * kk * cos(kk * (y - ph.in_y0));
    }
    return s;
}

// ------------------------------------------------------------- pass B pair adjoint
// The pair term of pass B for particle a with neighbour b (the value kernel's formulas,
// Eqs. tvf-momentum, tvf-p-ij-basa, p-edac, transport-vel) and the derivative of
//   S = c0 ax + c1 ay + c2 Gx + c3 Gy + c4 (p_b - p_a) + c5 ap
// with respect to both particles' inputs and the separation (dx, dy) = r_a - r_b, taking
// the operations of the formulas in reverse, in fp32.  dp = p_b - p_a and (uab, vab) =
// u_a - u_b come from the fp64 values, rounded once.  solid: the solid force's pair term (no
// A-term, no pressure rate; b is a fluid particle).
struct PIn {
    float V, rho, m, u, v, du, dv;
};
struct PGrad {
    float p, V, rho, u, v, du, dv;
};

__device__ __forceinline__ PIn pin_f(const ADev &a, int k)
{
    const float4 x = a.fa[k], y = a.fb[k];
    PIn r;
    r.V = x.x; r.rho = x.y; r.m = x.z; r.u = y.x; r.v = y.y; r.du = y.z; r.dv = y.w;
    return r;
}

__device__ __forceinline__ void pairB_adj(const Phys &ph, const PIn &A, const PIn &B, float dp,
                                          float uab, float vab, float dx, float dy, const float *c,
                                          bool solid, PGrad &gA, PGrad &gB, float &gdx, float &gdy)
{
    // forward
    const float r2 = dx * dx + dy * dy;
    const float r = sqrtf(r2);
    const float q = r * ph.inv_hf;
    const float t3 = q < 3.0f ? 3.0f - q : 0.0f;
    const float t2 = q < 2.0f ? 2.0f - q : 0.0f;
    const float t1 = q < 1.0f ? 1.0f - q : 0.0f;
    const float a3 = t3 * t3, b3 = t2 * t2, c3 = t1 * t1;
    const float w1 = -5.0f * (a3 * a3 - 6.0f * b3 * b3 + 15.0f * c3 * c3);
    const float w2 = 20.0f * (t3 * a3 - 6.0f * (t2 * b3) + 15.0f * (t1 * c3));
    const float F = r > 0.0f ? ph.a2hf * w1 / r : 0.0f;
    const float gx = F * dx, gy = F * dy, gdotr = F * r2;
    const float cij = A.V * A.V + B.V * B.V;
    const float inv_rs = 1.0f / (A.rho + B.rho);
    const float e = A.rho * dp * inv_rs;
    const float H = A.rho * B.rho * inv_rs;
    const float D = r2 + ph.eh2f;
    const float hf = H * gdotr / D;
    const float vis = 2.0f * ph.nuf * hf;
    const float cgx = cij * gx, cgy = cij * gy;
    const float Lax = c[0], Lay = c[1], LGx = c[2], LGy = c[3], Lsdp = c[4], Lap = c[5];
    // reverse
    float b_dp = Lsdp, b_cij = 0.0f, b_gx = 0.0f, b_gy = 0.0f, b_hf = 0.0f, b_uab = 0.0f, b_vab = 0.0f;
    const float b_cgx = LGx - e * Lax, b_cgy = LGy - e * Lay;
    const float b_e = -(cgx * Lax + cgy * Lay);
    if (!solid) {
        const float Ai = A.rho * (A.du * gx + A.dv * gy), Aj = B.rho * (B.du * gx + B.dv * gy);
        const float Mx = 0.5f * (A.u * Ai + B.u * Aj) + vis * uab;
        const float My = 0.5f * (A.v * Ai + B.v * Aj) + vis * vab;
        b_cij += Mx * Lax + My * Lay;
        const float bMx = cij * Lax, bMy = cij * Lay;
        gA.u += 0.5f * Ai * bMx; gB.u += 0.5f * Aj * bMx;
        gA.v += 0.5f * Ai * bMy; gB.v += 0.5f * Aj * bMy;
        const float bAi = 0.5f * (A.u * bMx + A.v * bMy), bAj = 0.5f * (B.u * bMx + B.v * bMy);
        b_hf += 2.0f * ph.nuf * (uab * bMx + vab * bMy);
        b_uab += vis * bMx; b_vab += vis * bMy;
        gA.rho += bAi * (A.du * gx + A.dv * gy);
        gA.du += bAi * A.rho * gx; gA.dv += bAi * A.rho * gy;
        b_gx += bAi * A.rho * A.du; b_gy += bAi * A.rho * A.dv;
        gB.rho += bAj * (B.du * gx + B.dv * gy);
        gB.du += bAj * B.rho * gx; gB.dv += bAj * B.rho * gy;
        b_gx += bAj * B.rho * B.du; b_gy += bAj * B.rho * B.dv;
        // ap = rho_a c^2 (m_b / rho_b) (u_ab . gW) - c_ab (2 nu_e / m_a) hf (p_b - p_a)
        const float mrb = B.m / B.rho, dv_ = uab * gx + vab * gy, difa = 2.0f * ph.nuef / A.m;
        const float b_div = Lap * A.rho * ph.c2f * mrb;
        gA.rho += Lap * ph.c2f * mrb * dv_;
        gB.rho -= Lap * A.rho * ph.c2f * dv_ * mrb / B.rho;
        b_cij -= Lap * difa * hf * dp;
        b_hf -= Lap * cij * difa * dp;
        b_dp -= Lap * cij * difa * hf;
        b_uab += b_div * gx; b_vab += b_div * gy;
        b_gx += b_div * uab; b_gy += b_div * vab;
    } else {
        const float Mx = vis * uab, My = vis * vab;
        b_cij += Mx * Lax + My * Lay;
        const float bMx = cij * Lax, bMy = cij * Lay;
        b_hf += 2.0f * ph.nuf * (uab * bMx + vab * bMy);
        b_uab += vis * bMx; b_vab += vis * bMy;
    }
    gA.u += b_uab; gB.u -= b_uab;
    gA.v += b_vab; gB.v -= b_vab;
    b_cij += gx * b_cgx + gy * b_cgy;
    b_gx += cij * b_cgx;
    b_gy += cij * b_cgy;
    const float b_H = b_hf * gdotr / D, b_gdotr = b_hf * H / D;
    float b_r2 = -b_hf * hf / D;
    const float b_inv = b_H * A.rho * B.rho + b_e * A.rho * dp;
    gA.rho += b_H * B.rho * inv_rs + b_e * dp * inv_rs;
    gB.rho += b_H * A.rho * inv_rs;
    b_dp += b_e * A.rho * inv_rs;
    const float b_s = -b_inv * inv_rs * inv_rs;
    gA.rho += b_s; gB.rho += b_s;
    gB.p += b_dp; gA.p -= b_dp;
    gA.V += 2.0f * A.V * b_cij; gB.V += 2.0f * B.V * b_cij;
    const float b_F = b_gx * dx + b_gy * dy + b_gdotr * r2;
    gdx = b_gx * F;
    gdy = b_gy * F;
    b_r2 += b_gdotr * F;
    if (r > 0.0f) {
        const float b_w1 = b_F * ph.a2hf / r;
        const float b_r = -b_F * F / r + b_w1 * w2 * ph.inv_hf;
        b_r2 += b_r / (2.0f * r);
    }
    gdx += 2.0f * dx * b_r2;
    gdy += 2.0f * dy * b_r2;
}

// Neighbours j of sorted particle k with the membership test of the value kernels; f(j, dx,
// dy, r2) with the fp32 separation r_k - r_j of the test (cell-relative coordinates).
template <class F>
__device__ __forceinline__ void a_walk_f(const Dev &d, int k, F &&f)
{
    const Geo &g = d.g;
    const int cc = d.cellk[k];
    const float4 pk = d.P[k];
    const double2 xy = d.XY[k];
    for_block(d, cc % g.nx, cc / g.nx, [&](int ox, int oy, int j0, int j1) {
        const float rxo = pk.x - (float)ox * g.sxf, ryo = pk.y - (float)oy * g.syf;
        for (int j = j0; j < j1; ++j) {
            float dxf, dyf, r2f;
            if (is_member(d, rxo, ryo, __ldg(d.P + j), j, xy.x, xy.y, dxf, dyf, r2f)) f(j, dxf, dyf, r2f);
        }
    });
}

// pass B's function of sorted particle k: 1 fluid/inlet (rates), 2 solid counted in the drag
__device__ __forceinline__ int passb_kind(const Dev &d, int k)
{
    const int t = d.stag[k] & 0x7f;
    if (t == FLUID || t == INLET) return 1;
    if (drag_mode(d.ph, t)) return 2;
    return 0;
}

// ------------------------------------------------- evaluation adjoint: coefficients
// Per particle: the output-adjoint coefficients of its pass B sums from the lambdas of its
// rates (fluid/inlet) or of its drag force (solid, weights wfx, wfy), with the sums
// G = sum c_ij gW and sum (p_j - p_i) the value kernel kept; the rate lambdas are consumed.
// Also the fp32 copies of the particle's fields and zero rho/V lambdas for the evaluation.
__global__ void a_coeff_b(Dev d, ADev a, double wfx, double wfy)
{
    const Phys &ph = d.ph;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        a.rho[k] = 0.0;
        a.V[k] = 0.0;
        const double2 pv = d.PV[k], rm = d.RM[k], uv = d.UV[k], duv = d.DUV[k];
        a.fa[k] = make_float4(d2f(pv.y), d2f(rm.x), d2f(d.Ms[k]), d2f(pv.x));
        a.fb[k] = make_float4(d2f(uv.x), d2f(uv.y), d2f(duv.x), d2f(duv.y));
        const int kind = passb_kind(d, k);
        a.cbf[k] = kind;
        float *c = a.cb + (size_t)k * NCB;
        for (int q = 0; q < NCB; ++q) c[q] = 0.0f;
        if (!kind) continue;
        const int s = slot_of(d, k);
        const double pk = pv.x;
        const double Gx = d.GS[3 * (size_t)k], Gy = d.GS[3 * (size_t)k + 1], sdp = d.GS[3 * (size_t)k + 2];
        if (kind == 1) {
            const double m = d.Ms[k];
            const double lau = a.au[s], lav = a.av[s], lap = a.ap[s], labu = a.abu[s], labv = a.abv[s];
            a.au[s] = a.av[s] = a.ap[s] = a.abu[s] = a.abv[s] = 0.0;
            const int N = d.snnb[k];
            const double corr = ph.use_pavg ? sdp / (double)N : -pk;
            c[0] = d2f(lau / m);
            c[1] = d2f(lav / m);
            c[2] = d2f((corr * lau - ph.pb * labu) / m);
            c[3] = d2f((corr * lav - ph.pb * labv) / m);
            const double lcorr = (Gx * lau + Gy * lav) / m;
            if (ph.use_pavg) c[4] = d2f(lcorr / (double)N);
            else a.p[s] -= lcorr;
            c[5] = d2f(lap);
        } else {
            // F = sum_fluid c [-pbar_ij gW + visc] = ax + (-p_i) G
            c[0] = d2f(wfx);
            c[1] = d2f(wfy);
            c[2] = d2f(-pk * wfx);
            c[3] = d2f(-pk * wfy);
            a.p[s] -= Gx * wfx + Gy * wfy;
        }
    }
}

// ------------------------------------------------- evaluation adjoint: pass B pairs
// The derivatives of every pass B sum the particle enters: its own (as particle a) and its
// neighbours' (as particle b), into the lambdas of its position, pressure, velocities and
// transport velocities (slot) and of its rho and V (sorted).
__global__ void a_gather_b(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int kk = a.cbf[k];
        const int tk = d.stag[k] & 0x7f;
        const PIn Pk = pin_f(a, k);
        const float *ck = a.cb + (size_t)k * NCB;
        const double pk = d.PV[k].x;
        const double2 uvk = d.UV[k];
        PGrad g = {0, 0, 0, 0, 0, 0, 0};
        float lx = 0.0f, ly = 0.0f;
        a_walk_f(d, k, [&](int j, float dx, float dy, float) {
            if (j == k) return;
            const int kj = a.cbf[j];
            const int tj = d.stag[j] & 0x7f;
            const bool own = kk == 1 || (kk == 2 && tj == FLUID);
            const bool rev = kj == 1 || (kj == 2 && tk == FLUID);
            if (!own && !rev) return;
            const PIn Pj = pin_f(a, j);
            const double2 uvj = d.UV[j];
            const float dp = d2f(d.PV[j].x - pk);
            const float uab = d2f(uvk.x - uvj.x), vab = d2f(uvk.y - uvj.y);
            if (own) {
                PGrad gj = {0, 0, 0, 0, 0, 0, 0};
                float gdx, gdy;
                pairB_adj(ph, Pk, Pj, dp, uab, vab, dx, dy, ck, kk == 2, g, gj, gdx, gdy);
                lx += gdx;
                ly += gdy;
            }
            if (rev) {
                PGrad gj = {0, 0, 0, 0, 0, 0, 0};
                float gdx, gdy;
                pairB_adj(ph, Pj, Pk, -dp, -uab, -vab, -dx, -dy, a.cb + (size_t)j * NCB, kj == 2, gj, g,
                          gdx, gdy);
                lx -= gdx;
                ly -= gdy;
            }
        });
        const int s = slot_of(d, k);
        a.x[s] += f2d(lx);
        a.y[s] += f2d(ly);
        a.p[s] += f2d(g.p);
        a.u[s] += f2d(g.u - g.du);
        a.v[s] += f2d(g.v - g.dv);
        a.ut[s] += f2d(g.du);
        a.vt[s] += f2d(g.dv);
        a.rho[k] += f2d(g.rho);
        a.V[k] += f2d(g.V);
    }
}

// ------------------------------------------------- evaluation adjoint: boundary values
// Per boundary particle, the coefficients its projection's derivatives take, from the
// lambdas of the values it was given in this evaluation (consumed):
//   wall (Adami, cited in Sec. 2): p_w = sum W p / sum W, u_g = 2 u_w - <u> or <u>, ...;
//     bc = [kind (1 Shepard, 2 plain mean), l_sw, l_sp, l_su, l_sv];
//   inlet (Sec. 3.2): p_o = p_k - (r_o - r_k) . grad p_k from the 3x3 system M z = b of
//     Eq. matform at the mirror point k; with lambda_z = l (1, -(x_o - x_k), -(y_o - y_k)) and
//     M^T mu = lambda_z, the derivative with respect to a fluid neighbour's inputs is that of
//     Phi_l = (p_l - z . (1, x_lk, y_lk)) (mu . (W, W_x, W_y)) V_l;
//     bc = [kind (1 mean, 2 Shepard, 3 solve), x_k, y_k, z0|p_o, z1, z2, mu0|coef, mu1, mu2];
//     the inlet particle's own position lambdas are added here (second walk).
__device__ __forceinline__ bool solve3a(double M[3][3], double b[3], double x[3])
{
    int piv[3] = {0, 1, 2};
    for (int c = 0; c < 3; ++c) {
        int best = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(M[piv[r]][c]) > fabs(M[piv[best]][c])) best = r;
        const int tmp = piv[c];
        piv[c] = piv[best];
        piv[best] = tmp;
        const double dd = M[piv[c]][c];
        if (dd == 0.0) return false;
        for (int r = c + 1; r < 3; ++r) {
            const double f = M[piv[r]][c] / dd;
            for (int q = c; q < 3; ++q) M[piv[r]][q] -= f * M[piv[c]][q];
            b[piv[r]] -= f * b[piv[c]];
        }
    }
    for (int c = 2; c >= 0; --c) {
        double s = b[piv[c]];
        for (int q = c + 1; q < 3; ++q) s -= M[piv[c]][q] * x[q];
        x[c] = s / M[piv[c]][c];
    }
    return true;
}

// Neighbours l (fluid) of the point (qx, qy): exact membership; f(l, xlk, ylk, r2) with
// r_lk = r_l - r_q, as the mirror sums take it.
template <class F>
__device__ __forceinline__ void a_walk_point(const Dev &d, double qx, double qy, F &&f)
{
    const Geo &g = d.g;
    const int cx = cell_coord(qx, g.x_min, g.inv_sx, g.nx);
    const int cy = cell_coord(qy, g.y_min, g.inv_sy, g.ny);
    for_block(d, cx, cy, [&](int, int, int j0, int j1) {
        for (int j = j0; j < j1; ++j) {
            if ((d.stag[j] & 0x7f) != FLUID) continue;
            const double2 xj = d.XY[j];
            double xlk, ylk;
            const double r2 = exact_r2(g, xj.x, xj.y, qx, qy, xlk, ylk);
            if (r2 < g.rc2) f(j, xlk, ylk, r2);
        }
    });
}

// W, W_x, W_y of the mirror sums at r_lk and their derivatives with respect to (x_lk, y_lk)
struct WDer {
    double W, Wx, Wy, Wxx, Wxy, Wyy;
};
__device__ __forceinline__ WDer wder(const Phys &ph, double xlk, double ylk, double r2)
{
    WDer o;
    if (!(r2 > 1e-30)) {
        double w, w1, w2;
        quintic3(0.0, w, w1, w2);
        o.W = ph.a2 * w;
        o.Wx = o.Wy = o.Wxx = o.Wxy = o.Wyy = 0.0;
        return o;
    }
    const double r = sqrt(r2), ir = 1.0 / r;
    double w, w1, w2;
    quintic3(r * ph.inv_h, w, w1, w2);
    const double Wr = ph.a2h * w1, Wrr = ph.a2 * ph.inv_h * ph.inv_h * w2;
    const double ex = xlk * ir, ey = ylk * ir;
    o.W = ph.a2 * w;
    o.Wx = Wr * ex;
    o.Wy = Wr * ey;
    o.Wxx = Wrr * ex * ex + Wr * (ir - ex * ex * ir);
    o.Wyy = Wrr * ey * ey + Wr * (ir - ey * ey * ir);
    o.Wxy = Wrr * ex * ey - Wr * ex * ey * ir;
    return o;
}

__global__ void a_boundary_pre(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int t = d.stag[k] & 0x7f;
        double *c = a.bc + (size_t)k * NBC;
        if (t != WALL && t != SLIPWALL && t != INLET) continue;
        for (int q = 0; q < NBC; ++q) c[q] = 0.0;
        const int s = slot_of(d, k);
        const double2 xy = d.XY[k];
        if (t == WALL || t == SLIPWALL) {
            const double lp = a.p[s], lu = a.u[s] + a.ut[s], lv = a.v[s] + a.vt[s];
            a.p[s] = a.u[s] = a.ut[s] = a.v[s] = a.vt[s] = 0.0;
            double sw = 0.0, sp = 0.0, su = 0.0, sv = 0.0, cnt = 0.0;
            a_walk(d, k, [&](int j, double, double, double r2) {
                if ((d.stag[j] & 0x7f) != FLUID) return;
                const double w = ph.a2 * quintic_w(sqrt(r2) * ph.inv_h);
                const double2 pv = d.PV[j], uv = d.UV[j];
                sw += w; sp += w * pv.x; su += w * uv.x; sv += w * uv.y;
                cnt += 1.0;
            });
            if (cnt == 0.0) continue;
            const int wi = t == WALL ? 0 : 1;
            const double luf = ph.wall_slip[wi] ? lu : -lu;
            const double lvf = -lv;
            if (sw > 0.0) {
                const double isw = 1.0 / sw;
                c[0] = 1.0;
                c[2] = lp * isw;
                c[3] = luf * isw;
                c[4] = lvf * isw;
                c[1] = -(lp * sp + luf * su + lvf * sv) * isw * isw;
            } else {
                c[0] = 2.0;
                c[2] = lp / cnt;
                c[3] = luf / cnt;
                c[4] = lvf / cnt;
            }
        } else if (ph.has_inlet) {
            const double lpo = a.p[s];
            a.p[s] = 0.0;
            const double xk = 2.0 * ph.x_in - xy.x, yk = xy.y;
            double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0};
            double nl = 0.0;
            a_walk_point(d, xk, yk, [&](int l, double xlk, double ylk, double r2) {
                const WDer W = wder(ph, xlk, ylk, r2);
                const double Vl = d.RM[l].y, pl = d.PV[l].x;
                const double row[3] = {W.W * Vl, W.Wx * Vl, W.Wy * Vl};
                for (int q = 0; q < 3; ++q) {
                    M[q][0] += row[q];
                    M[q][1] += xlk * row[q];
                    M[q][2] += ylk * row[q];
                    b[q] += pl * row[q];
                }
                nl += 1.0;
            });
            c[1] = xk;
            c[2] = yk;
            if (nl == 0.0 || lpo == 0.0) continue;
            if (!(M[0][0] > 0.0)) {
                c[0] = 1.0;
                c[6] = lpo / nl;
                continue;
            }
            const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                               M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
            const bool singular = fabs(det) <= 1e-9 * fabs(M[0][0] * M[1][1] * M[2][2]);
            double z[3] = {0, 0, 0}, mu[3] = {0, 0, 0};
            bool full = false;
            if (!singular) {
                double Ms[3][3], bs[3] = {b[0], b[1], b[2]};
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q) Ms[r][q] = M[r][q];
                full = solve3a(Ms, bs, z);
                if (full) {
                    double Mt[3][3];
                    for (int r = 0; r < 3; ++r)
                        for (int q = 0; q < 3; ++q) Mt[r][q] = M[q][r];
                    double lz[3] = {lpo, -lpo * (xy.x - xk), -lpo * (xy.y - yk)};
                    full = solve3a(Mt, lz, mu);
                }
            }
            double lxo = 0.0, lyo = 0.0;
            if (full) {
                c[0] = 3.0;
                c[3] = z[0]; c[4] = z[1]; c[5] = z[2];
                c[6] = mu[0]; c[7] = mu[1]; c[8] = mu[2];
                lxo = -2.0 * z[1] * lpo;  // p_o's (x_o - x_k) with x_k = 2 x_in - x_o
                a_walk_point(d, xk, yk, [&](int l, double xlk, double ylk, double r2) {
                    const WDer W = wder(ph, xlk, ylk, r2);
                    const double Vl = d.RM[l].y, pl = d.PV[l].x;
                    const double R = pl - z[0] - xlk * z[1] - ylk * z[2];
                    const double Q = mu[0] * W.W + mu[1] * W.Wx + mu[2] * W.Wy;
                    const double dQx = mu[0] * W.Wx + mu[1] * W.Wxx + mu[2] * W.Wxy;
                    const double dQy = mu[0] * W.Wy + mu[1] * W.Wxy + mu[2] * W.Wyy;
                    // x_lk = x_l - (2 x_in - x_o): d/dx_o = +1; y_lk = y_l - y_o: d/dy_o = -1
                    lxo += Vl * (-z[1] * Q + R * dQx);
                    lyo -= Vl * (-z[2] * Q + R * dQy);
                });
            } else {
                // Shepard value sum p W V / sum W V (gradient set to zero)
                const double po = b[0] / M[0][0], coef = lpo / M[0][0];
                c[0] = 2.0;
                c[3] = po;
                c[6] = coef;
                a_walk_point(d, xk, yk, [&](int l, double xlk, double ylk, double r2) {
                    const WDer W = wder(ph, xlk, ylk, r2);
                    const double Vl = d.RM[l].y, pl = d.PV[l].x;
                    lxo += coef * (pl - po) * W.Wx * Vl;
                    lyo -= coef * (pl - po) * W.Wy * Vl;
                });
            }
            a.x[s] += lxo;
            a.y[s] += lyo;
        }
    }
}

// The fluid and outlet sides of the boundary adjoints, one neighbour walk per particle:
//   a fluid particle adds the derivatives of the wall projections it enters (its wall
//   neighbours' coefficients), of the inlet mirror systems it enters (the inlet particles
//   whose mirror point has it within 3h, found around its own mirror image with the value
//   kernel's exact test) and, at the end of a step (outl), of its red outlet neighbours'
//   Shepard J2 (into the lambdas of its J2 and position);
//   an outlet particle red in the previous step adds the derivatives of its blue neighbours'
//   means (itself included) to the lambdas of its previous J2 and advection velocity.
__global__ void a_gather_2(Dev d, ADev a, int outl)
{
    const Phys &ph = d.ph;
    const Geo &g = d.g;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint8_t tk = d.stag[k];
        const bool fl = (tk & 0x7f) == FLUID;
        const bool prev_red = outl && tk == (OUTLET | TAG_REDP);
        if (!fl && !prev_red) continue;
        const int s = slot_of(d, k);
        const double2 xy = d.XY[k];
        const double pl = d.PV[k].x;
        const double2 uvl = d.UV[k];
        const double J2k = d.AUX[k].x;
        double lp = 0.0, lu = 0.0, lv = 0.0, lx = 0.0, ly = 0.0, lrho = 0.0, lJ = 0.0, lJp = 0.0, la = 0.0;
        a_walk(d, k, [&](int j, double dx, double dy, double r2) {
            const int tj = d.stag[j] & 0x7f;
            const double *c = a.bc + (size_t)j * NBC;
            if (fl && (tj == WALL || tj == SLIPWALL)) {
                if (c[0] == 1.0) {
                    const double r = sqrt(r2);
                    double W, Wr;
                    W_dW(ph, r, W, Wr);
                    lp += c[2] * W;
                    lu += c[3] * W;
                    lv += c[4] * W;
                    if (r > 0.0) {
                        const double coef = (c[1] + c[2] * pl + c[3] * uvl.x + c[4] * uvl.y) * Wr / r;
                        lx += coef * dx;  // d r / d x_l = (x_l - x_o) / r
                        ly += coef * dy;
                    }
                } else if (c[0] == 2.0) {
                    lp += c[2];
                    lu += c[3];
                    lv += c[4];
                }
            } else if (outl && tj == OUTLET && j != k) {
                if (fl && c[0] == 1.0) {
                    const double r = sqrt(r2);
                    double W, Wr;
                    W_dW(ph, r, W, Wr);
                    lJ += c[2] * W;
                    if (r > 0.0) {
                        const double coef = (c[1] + c[2] * J2k) * Wr / r;
                        lx += coef * dx;
                        ly += coef * dy;
                    }
                } else if (fl && c[0] == 2.0) {
                    lJ += c[2];
                } else if (prev_red && c[0] == 3.0) {
                    lJp += c[3];
                    la += c[4];
                }
            }
        });
        if (prev_red) {
            // the blue mean includes the particle itself when it was red
            const double *c = a.bc + (size_t)k * NBC;
            if (c[0] == 3.0) {
                lJp += c[3];
                la += c[4];
            }
            a.J2p[s] += lJp;
            a.advp[s] += la;
            continue;
        }
        if (ph.has_inlet && xy.x < ph.x_in + ph.L_in + sqrt(g.rc2) + g.sx) {
            const double xm = 2.0 * ph.x_in - xy.x, ym = xy.y;
            const int cx = cell_coord(xm, g.x_min, g.inv_sx, g.nx);
            const int cy = cell_coord(ym, g.y_min, g.inv_sy, g.ny);
            const double Vl = d.RM[k].y, ml = d.Ms[k], rhol = d.RM[k].x;
            for_block(d, cx, cy, [&](int, int, int j0, int j1) {
                for (int o = j0; o < j1; ++o) {
                    if ((d.stag[o] & 0x7f) != INLET) continue;
                    const double *c = a.bc + (size_t)o * NBC;
                    if (c[0] == 0.0) continue;
                    const double2 xo = d.XY[o];
                    const double xk = 2.0 * ph.x_in - xo.x, yk = xo.y;
                    double xlk, ylk;
                    const double r2 = exact_r2(g, xy.x, xy.y, xk, yk, xlk, ylk);
                    if (!(r2 < g.rc2)) continue;
                    if (c[0] == 1.0) {
                        lp += c[6];
                        continue;
                    }
                    const WDer W = wder(ph, xlk, ylk, r2);
                    if (c[0] == 3.0) {
                        const double z0 = c[3], z1 = c[4], z2 = c[5];
                        const double m0 = c[6], m1 = c[7], m2 = c[8];
                        const double R = pl - z0 - xlk * z1 - ylk * z2;
                        const double Q = m0 * W.W + m1 * W.Wx + m2 * W.Wy;
                        lp += Q * Vl;
                        lrho -= R * Q * ml / (rhol * rhol);
                        lx += Vl * (-z1 * Q + R * (m0 * W.Wx + m1 * W.Wxx + m2 * W.Wxy));
                        ly += Vl * (-z2 * Q + R * (m0 * W.Wy + m1 * W.Wxy + m2 * W.Wyy));
                    } else {
                        const double po = c[3], coef = c[6];
                        lp += coef * W.W * Vl;
                        const double cw = coef * (pl - po);
                        lx += cw * W.Wx * Vl;
                        ly += cw * W.Wy * Vl;
                        lrho -= cw * W.W * ml / (rhol * rhol);
                    }
                }
            });
        }
        a.p[s] += lp;
        a.u[s] += lu;
        a.v[s] += lv;
        a.x[s] += lx;
        a.y[s] += ly;
        a.J2[s] += lJ;
        a.rho[k] += lrho;
    }
}

// ------------------------------------------------- evaluation adjoint: pass A
// rho_i = sum_j m_j W_ij, V_i = 1 / sum_j W_ij (Eq. summation-density, Sec. 2): the position
// lambdas of particle k from its own sums and its neighbours' (fp32 pair terms).
__global__ void a_pass_a(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float mk = a.fa[k].z;
        const double Vk = d.PV[k].y;
        const float lSk = d2f(-a.V[k] * Vk * Vk), lRk = d2f(a.rho[k]);
        float lx = 0.0f, ly = 0.0f;
        a_walk_f(d, k, [&](int j, float dx, float dy, float r2) {
            if (j == k || !(r2 > 0.0f)) return;
            const double Vj = d.PV[j].y;
            const float lSj = d2f(-a.V[j] * Vj * Vj), lRj = d2f(a.rho[j]);
            const float r = sqrtf(r2);
            const float Wr = ph.a2hf * quintic_dw(r * ph.inv_hf);
            const float coef = ((lRk * a.fa[j].z + lSk) + (lRj * mk + lSj)) * Wr / r;
            lx += coef * dx;
            ly += coef * dy;
        });
        const int s = slot_of(d, k);
        a.x[s] += f2d(lx);
        a.y[s] += f2d(ly);
    }
}

// ------------------------------------------------- the hybrid outlet update (Sec. 3.4)
// Per outlet particle: its new values (u = u_bar + J2/(2 rho0 c), p = p_bar + J2/2, v = v_bar,
// u~ = u, v~ = v, the stored J2 and advection velocity) are consumed and the coefficients of
// J2's derivatives stored: bc = [kind (1 red Shepard, 2 red mean, 3 blue), l_sw, l_sf | c,
// c_J2p, c_adv]; the particle's own position lambdas are added here.
__global__ void a_outlet_pre(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    const int n = d.cell_start[d.g.ncells];  // particles of the evaluation's cell build
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if ((d.stag[k] & 0x7f) != OUTLET) continue;
        double *c = a.bc + (size_t)k * NBC;
        for (int q = 0; q < NBC; ++q) c[q] = 0.0;
        const int s = slot_of(d, k);
        double Lu = a.u[s] + a.ut[s];
        const double Lv = a.v[s] + a.vt[s], Lp = a.p[s], LJ = a.J2p[s], La = a.advp[s];
        a.u[s] = a.ut[s] = a.v[s] = a.vt[s] = a.p[s] = a.J2p[s] = a.advp[s] = 0.0;
        double sw = 0.0, sf = 0.0, cnt = 0.0, mr = 0.0;
        a_walk(d, k, [&](int j, double, double, double r2) {
            const uint8_t tj = d.stag[j];
            if ((tj & 0x7f) == FLUID) {
                const double w = ph.a2 * quintic_w(sqrt(r2) * ph.inv_h);
                sw += w;
                sf += w * d.AUX[j].x;
                cnt += 1.0;
            } else if (tj == (OUTLET | TAG_REDP)) {
                mr += 1.0;
            }
        });
        const bool red = cnt > 0.0;
        if (red) Lu += La;
        const double LJ2 = Lu * ph.inv_2rc + 0.5 * Lp + LJ;
        a.ubar[s] += Lu + ((!red && mr == 0.0) ? La : 0.0);
        a.vbar[s] += Lv;
        a.pbar[s] += Lp;
        if (red) {
            if (sw > 0.0) {
                const double J2 = sf / sw;
                c[0] = 1.0;
                c[2] = LJ2 / sw;
                c[1] = -LJ2 * J2 / sw;
                double lx = 0.0, ly = 0.0;
                a_walk(d, k, [&](int j, double dx, double dy, double r2) {
                    if ((d.stag[j] & 0x7f) != FLUID) return;
                    const double r = sqrt(r2);
                    if (!(r > 0.0)) return;
                    double W, Wr;
                    W_dW(ph, r, W, Wr);
                    const double coef = (c[1] + c[2] * d.AUX[j].x) * Wr / r;
                    lx += coef * dx;
                    ly += coef * dy;
                });
                a.x[s] += lx;
                a.y[s] += ly;
            } else {
                c[0] = 2.0;
                c[2] = LJ2 / cnt;
            }
        } else if (mr > 0.0) {
            c[0] = 3.0;
            c[3] = LJ2 / mr;
            c[4] = La / mr;
        }
    }
}

// ------------------------------------------------------------ slot-space operations
// The pressure-energy term E = sum_fluid omega(x) p^2 with the window weight
// omega = sin^2(pi (x - x0) / (x1 - x0)) on [x0, x1), 0 outside: it goes to zero smoothly at
// both edges, so that particles entering or leaving the window (or the fluid, at the outlet)
// change E continuously.
__device__ __forceinline__ double pe_weight(double x, double x0, double x1, double &dw)
{
    dw = 0.0;
    if (!(x >= x0 && x < x1)) return 0.0;
    const double k = 3.141592653589793 / (x1 - x0), t = k * (x - x0);
    const double sn = sin(t), cs = cos(t);
    dw = 2.0 * k * sn * cs;
    return sn * sn;
}

// Seed of w E at the end of a step: lambda_p += 2 w omega p, lambda_x += w omega' p^2.
__global__ void a_seed_pe(Dev d, ADev a, double w, double x0, double x1)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        if (d.tag[s] != FLUID) continue;
        double dw;
        const double om = pe_weight(d.x[s], x0, x1, dw), p = d.p[s];
        a.p[s] += 2.0 * w * om * p;
        a.x[s] += w * dw * p * p;
    }
}

// Forward value of E at the end of step n, one block (fixed-order tree).
__global__ void __launch_bounds__(1024) a_pe_value(Dev d, ADev a, int nstep, double x0, double x1)
{
    __shared__ double sh[1024];
    double v = 0.0;
    for (int s = threadIdx.x; s < d.cap; s += blockDim.x) {
        if (d.tag[s] != FLUID) continue;
        double dw;
        const double om = pe_weight(d.x[s], x0, x1, dw);
        v += om * d.p[s] * d.p[s];
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.pe[nstep] = sh[0];
}

__global__ void a_rec_rpos(Dev d, ADev a)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x)
        a.rpos_old[s] = d.rpos[s];
}

// the acoustic gate of the corrector's sample (the stage's own test on the new pressure)
__global__ void a_rec_gate(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        const double pn = d.p[s];
        a.gate[s] = (d.tag[s] == FLUID && pn * pn * ph.inv_2rc <= ph.I_thr) ? 1 : 0;
    }
}

__global__ void a_rec_tag(Dev d, ADev a)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x)
        a.tag_pre[s] = d.tag[s];
}

__device__ __forceinline__ void zero_slot(const Dev &d, const ADev &a, int s)
{
    a.x[s] = a.y[s] = a.u[s] = a.v[s] = a.ut[s] = a.vt[s] = a.p[s] = 0.0;
    a.au[s] = a.av[s] = a.ap[s] = a.abu[s] = a.abv[s] = 0.0;
    a.ubar[s] = a.vbar[s] = a.pbar[s] = a.J2[s] = a.J2p[s] = a.advp[s] = 0.0;
    for (int q = 0; q < NAVG_MAX * 3; ++q) a.ring[(size_t)s * NAVG_MAX * 3 + q] = 0.0;
    (void)d;
}

// Recycling (end of Sec. 3.4), reversed: the spawned inlet particles first (x = x_parent -
// L_in, y = y_parent, p = p_parent, u = u_in(y) at the end of the step), then the slot
// conversions.
__global__ void a_recycle_spawn(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    const int ns = d.cnt->last_spawn;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < ns; r += gridDim.x * blockDim.x) {
        const int2 pm = d.spawn_map[r];
        const int ps = pm.x, sn = pm.y;
        const double y = d.y[sn];
        const double Lu = a.u[sn] + a.ut[sn];
        a.x[ps] += a.x[sn];
        a.y[ps] += a.y[sn] + inlet_dudy(ph, y) * Lu;
        a.p[ps] += a.p[sn];
        for (int c = 0; c < T_DIR; ++c)
            a.acc[(size_t)sn * T_DIR + c] += c < ph.n_modes ? mode_shape_a(ph, c, y) * Lu : 0.0;
        zero_slot(d, a, sn);
    }
}

__global__ void a_recycle_conv(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        const uint8_t t0 = a.tag_pre[s], t1 = d.tag[s];
        if (t0 == FLUID && t1 == OUTLET) {
            // u = u_bar, v = v_bar, p = p_bar, u~ = u_bar, v~ = v_bar, adv = u_bar, J2p = 0
            a.ubar[s] += a.u[s] + a.ut[s] + a.advp[s];
            a.vbar[s] += a.v[s] + a.vt[s];
            a.pbar[s] += a.p[s];
            a.u[s] = a.v[s] = a.p[s] = a.ut[s] = a.vt[s] = a.advp[s] = a.J2p[s] = 0.0;
        } else if (t0 == INLET && t1 == FLUID) {
            // ring filled with (u, v, p), averages = (u, v, p), J2 = 0
            double su = a.ubar[s], sv = a.vbar[s], sp = a.pbar[s];
            double *rg = a.ring + (size_t)s * NAVG_MAX * 3;
            for (int q = 0; q < ph.n_avg; ++q) {
                su += rg[3 * q];
                sv += rg[3 * q + 1];
                sp += rg[3 * q + 2];
            }
            for (int q = 0; q < NAVG_MAX * 3; ++q) rg[q] = 0.0;
            a.u[s] += su;
            a.v[s] += sv;
            a.p[s] += sp;
            a.ubar[s] = a.vbar[s] = a.pbar[s] = a.J2[s] = 0.0;
        } else if (t1 == TAG_DEAD) {
            zero_slot(d, a, s);
        }
    }
}

// Stages reversed.  CORR: the corrector (tau = dt) with the time-average sample and J2 of
// the fluid (Eqs. timeevg, characteristic-vars) first; the rate lambdas go to the first
// evaluation's rates.  Otherwise the predictor (tau = dt/2), whose rate lambdas go to the
// previous step's second evaluation, and the base-state lambdas become those of the step's
// start.
template <bool CORR>
__global__ void a_stage(Dev d, ADev a, double tau)
{
    const Phys &ph = d.ph;
    const double rc = ph.rho0 * ph.cs;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        const uint8_t t = a.tag_pre[s];
        if (t == FLUID) {
            if (CORR && ph.has_outlet && ph.outlet_kind == OUT_HYBRID) {
                const double LJ = a.J2[s];
                a.J2[s] = 0.0;
                a.u[s] += rc * LJ;
                a.p[s] += LJ;
                const double lb[3] = {a.ubar[s] - rc * LJ, a.vbar[s], a.pbar[s] - LJ};
                a.ubar[s] = a.vbar[s] = a.pbar[s] = 0.0;
                double *rg = a.ring + (size_t)s * NAVG_MAX * 3;
                for (int q = 0; q < ph.n_avg; ++q)
                    for (int c = 0; c < 3; ++c) rg[3 * q + c] += lb[c] * ph.inv_navg;
                if (a.gate[s]) {
                    const int q = a.rpos_old[s];
                    a.u[s] += rg[3 * q];
                    a.v[s] += rg[3 * q + 1];
                    a.p[s] += rg[3 * q + 2];
                    rg[3 * q] = rg[3 * q + 1] = rg[3 * q + 2] = 0.0;
                }
            }
            // u = u0 + tau au; u~ = u + tau abu; x = x0 + tau u~; p = p0 + tau ap
            const double Lutx = a.ut[s] + tau * a.x[s], Luty = a.vt[s] + tau * a.y[s];
            const double Lux = a.u[s] + Lutx, Luy = a.v[s] + Luty;
            a.au[s] += tau * Lux;
            a.av[s] += tau * Luy;
            a.abu[s] += tau * Lutx;
            a.abv[s] += tau * Luty;
            a.ap[s] += tau * a.p[s];
            if (CORR) {
                a.x0[s] += a.x[s]; a.y0[s] += a.y[s]; a.u0[s] += Lux; a.v0[s] += Luy; a.p0[s] += a.p[s];
                a.x[s] = a.y[s] = a.u[s] = a.v[s] = a.p[s] = 0.0;
            } else {
                a.x[s] += a.x0[s]; a.y[s] += a.y0[s]; a.u[s] = Lux + a.u0[s]; a.v[s] = Luy + a.v0[s];
                a.p[s] += a.p0[s];
                a.x0[s] = a.y0[s] = a.u0[s] = a.v0[s] = a.p0[s] = 0.0;
            }
            a.ut[s] = a.vt[s] = 0.0;
        } else if (t == INLET) {
            // u = u_in(y), v = 0, u~ = u, x = x0 + tau u
            const double y = d.y[s];
            const double Lu = a.u[s] + a.ut[s] + tau * a.x[s];
            for (int c = 0; c < T_DIR; ++c)
                a.acc[(size_t)s * T_DIR + c] += c < ph.n_modes ? mode_shape_a(ph, c, y) * Lu : 0.0;
            a.y[s] += inlet_dudy(ph, y) * Lu;
            a.u[s] = a.ut[s] = a.v[s] = a.vt[s] = 0.0;
            if (CORR) {
                a.x0[s] += a.x[s];
                a.x[s] = 0.0;
            } else {
                a.x[s] += a.x0[s];
                a.x0[s] = 0.0;
            }
        } else if (t == OUTLET) {
            // x = x0 + tau adv
            a.advp[s] += tau * a.x[s];
            if (CORR) {
                a.x0[s] += a.x[s];
                a.x[s] = 0.0;
            } else {
                a.x[s] += a.x0[s];
                a.x0[s] = 0.0;
            }
        }
    }
}

// The set-up of an upload reversed (u~ = u, rings and averages from (u, v, p), advection
// velocity u), and the inlet particles' initial velocities u_in(y).
__global__ void a_init(Dev d, ADev a)
{
    const Phys &ph = d.ph;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        if (d.tag[s] == TAG_DEAD) continue;
        double su = a.ut[s] + a.ubar[s] + a.advp[s], sv = a.vt[s] + a.vbar[s], sp = a.pbar[s];
        const double *rg = a.ring + (size_t)s * NAVG_MAX * 3;
        for (int q = 0; q < ph.n_avg; ++q) {
            su += rg[3 * q];
            sv += rg[3 * q + 1];
            sp += rg[3 * q + 2];
        }
        a.u[s] += su;
        a.v[s] += sv;
        a.p[s] += sp;
        if (d.tag[s] == INLET) {
            const double y = d.y[s];
            for (int c = 0; c < T_DIR; ++c)
                a.acc[(size_t)s * T_DIR + c] += c < ph.n_modes ? mode_shape_a(ph, c, y) * a.u[s] : 0.0;
        }
    }
}

// dL/da_c = sum over slots of their contributions, in slot order (one block per direction).
__global__ void __launch_bounds__(1024) a_reduce(Dev d, ADev a)
{
    __shared__ double sh[1024];
    const int c = blockIdx.x;
    double v = 0.0;
    for (int s = threadIdx.x; s < d.cap; s += blockDim.x) v += a.acc[(size_t)s * T_DIR + c];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.grad[c] = sh[0];
}

// --------------------------------------------------------------------- layout
// Offsets of the adjoint arrays in the workspace (256-byte aligned); with base != nullptr the
// pointers are set.  Returns the bytes used.
size_t adev_layout(const Dev &d, int nsteps, int nrec, char *base, ADev *a)
{
    const size_t C = (size_t)d.cap;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return base ? base + o : nullptr;
    };
    ADev t;
    double **slots[] = {&t.x, &t.y, &t.u, &t.v, &t.ut, &t.vt, &t.p, &t.au, &t.av, &t.ap, &t.abu,
                        &t.abv, &t.x0, &t.y0, &t.u0, &t.v0, &t.p0, &t.ubar, &t.vbar, &t.pbar,
                        &t.J2, &t.J2p, &t.advp, &t.rho, &t.V};
    for (double **q : slots) *q = (double *)take(sizeof(double) * C);
    t.ring = (double *)take(sizeof(double) * C * NAVG_MAX * 3);
    t.acc = (double *)take(sizeof(double) * C * T_DIR);
    t.cb = (float *)take(sizeof(float) * C * NCB);
    t.cbf = (int *)take(sizeof(int) * C);
    t.bc = (double *)take(sizeof(double) * C * NBC);
    t.fa = (float4 *)take(sizeof(float4) * C);
    t.fb = (float4 *)take(sizeof(float4) * C);
    t.rec_tag = (uint8_t *)take(C * (size_t)nrec);
    t.rec_gate = (uint8_t *)take(C * (size_t)nrec);
    t.rec_rpos = (uint8_t *)take(C * (size_t)nrec);
    t.tag_pre = t.rec_tag;
    t.gate = t.rec_gate;
    t.rpos_old = t.rec_rpos;
    t.pe = (double *)take(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1));
    t.grad = (double *)take(sizeof(double) * T_DIR);
    if (a) *a = t;
    return off;
}

// the views of step record `rec`
ADev adev_of(const Dev &d, void *ws, int nsteps, int nrec, int rec)
{
    ADev a;
    adev_layout(d, nsteps, nrec, static_cast<char *>(ws), &a);
    const size_t o = (size_t)rec * (size_t)d.cap;
    a.tag_pre = a.rec_tag + o;
    a.gate = a.rec_gate + o;
    a.rpos_old = a.rec_rpos + o;
    return a;
}

size_t adev_bytes(const Dev &d, int nsteps, int nrec) { return adev_layout(d, nsteps, nrec, nullptr, nullptr); }

int ablocks(int n)
{
    int b = (n + ATPB - 1) / ATPB;
    return b < 1 ? 1 : (b > 8192 ? 8192 : b);
}

}  // namespace

size_t adjoint_bytes(const Dev &d, int nsteps, int nrec) { return adev_bytes(d, nsteps, nrec); }

// Adjoint kernels of one operation (AJ_*), on stream s; rec: the step record (of nrec) that
// the recording and the reversed stages and recycling use.
int launch_adjoint(const Dev &d, void *ws, int nsteps, int nrec, int rec, cudaStream_t s, int what,
                   double p0, double p1, double p2)
{
    const ADev a = adev_of(d, ws, nsteps, nrec, rec);
    const int gb = ablocks(d.cap);
    switch (what) {
    case AJ_ZERO:
        cudaMemsetAsync(ws, 0, adev_bytes(d, nsteps, nrec), s);
        return 1;
    case AJ_PE_VALUE: a_pe_value<<<1, 1024, 0, s>>>(d, a, (int)p0, p1, p2); return 1;
    case AJ_PE_SEED: a_seed_pe<<<gb, ATPB, 0, s>>>(d, a, p0, p1, p2); return 1;
    case AJ_REC_RPOS: a_rec_rpos<<<gb, ATPB, 0, s>>>(d, a); return 1;
    case AJ_REC_GATE: a_rec_gate<<<gb, ATPB, 0, s>>>(d, a); return 1;
    case AJ_REC_TAG: a_rec_tag<<<gb, ATPB, 0, s>>>(d, a); return 1;
    case AJ_RECYCLE:
        a_recycle_spawn<<<ablocks(LIST_MAX), ATPB, 0, s>>>(d, a);
        a_recycle_conv<<<gb, ATPB, 0, s>>>(d, a);
        return 2;
    case AJ_EVAL: {
        // p0: 1 at the second evaluation of a step (outlet update, drag weights p1, p2)
        const bool end = p0 != 0.0;
        const bool outl = end && d.ph.has_outlet && d.ph.outlet_kind == OUT_HYBRID;
        int k = 0;
        a_coeff_b<<<gb, ATPB, 0, s>>>(d, a, end ? p1 : 0.0, end ? p2 : 0.0); ++k;
        if (outl) { a_outlet_pre<<<gb, ATPB, 0, s>>>(d, a); ++k; }
        a_gather_b<<<gb, ATPB, 0, s>>>(d, a); ++k;
        a_boundary_pre<<<gb, ATPB, 0, s>>>(d, a); ++k;
        a_gather_2<<<gb, ATPB, 0, s>>>(d, a, outl ? 1 : 0); ++k;
        a_pass_a<<<gb, ATPB, 0, s>>>(d, a); ++k;
        return k;
    }
    case AJ_STAGE_CORR: a_stage<true><<<gb, ATPB, 0, s>>>(d, a, p0); return 1;
    case AJ_STAGE_PRED: a_stage<false><<<gb, ATPB, 0, s>>>(d, a, p0); return 1;
    case AJ_INIT: a_init<<<gb, ATPB, 0, s>>>(d, a); return 1;
    case AJ_REDUCE: a_reduce<<<T_DIR, 1024, 0, s>>>(d, a); return 1;
    default: return 0;
    }
}

const double *adjoint_grad(const Dev &d, const void *ws, int nsteps, int nrec)
{
    return adev_of(d, const_cast<void *>(ws), nsteps, nrec, 0).grad;
}

const double *adjoint_pe(const Dev &d, const void *ws, int nsteps, int nrec)
{
    return adev_of(d, const_cast<void *>(ws), nsteps, nrec, 0).pe;
}

}  // namespace edac
