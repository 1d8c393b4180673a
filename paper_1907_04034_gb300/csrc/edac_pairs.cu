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
#include "edac_internal.cuh"

namespace edac {

namespace {

constexpr int TPB = 128;   // threads per block of the pair passes
constexpr int LMAX = 64;   // shared-memory list entries per thread (flushed when full)
constexpr int FOLD = 8;    // pair terms summed in fp32 before a compensated fold

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

// fp32 separation of a listed neighbour (same arithmetic as the membership pre-test)
__device__ __forceinline__ int geom32(const Dev &d, unsigned e, float rx, float ry, float4 &pj,
                                      float &dx, float &dy, float &r2)
{
    const int j = (int)(e >> 4);
    const int ox = (int)((e >> 2) & 3u) - 1, oy = (int)(e & 3u) - 1;
    pj = __ldg(d.P + j);
    dx = (rx - (float)ox * d.g.sxf) - pj.x;
    dy = (ry - (float)oy * d.g.syf) - pj.y;
    r2 = dx * dx + dy * dy;
    return j;
}

// r from r^2 without the IEEE square root: r^2 * rsqrt(r^2), 0 for coincident particles
__device__ __forceinline__ float fast_r(float r2) { return r2 > 0.f ? r2 * rsqrtf(r2) : 0.f; }

// ---------------------------------------------------------------------------- pass A
// S_i = sum_j W_ij, V_i = 1/S_i (number-density volume, Sec. 2), rho_i = sum_j m_j W_ij
// (Eq. summation-density), N_i = number of neighbours (self included).
struct BodyA32 {
    const Dev &d;
    float rx, ry, a2, inv_h;
    float s = 0.f, r = 0.f, sh = 0.f, sl = 0.f, rh = 0.f, rl = 0.f;
    int n = 0;
    __device__ BodyA32(const Dev &dd, float x, float y)
        : d(dd), rx(x), ry(y), a2(dd.ph.a2f), inv_h(dd.ph.inv_hf) {}
    __device__ void operator()(unsigned e)
    {
        float4 pj;
        float dx, dy, r2;
        geom32(d, e, rx, ry, pj, dx, dy, r2);
        const float w = a2 * quintic_w(fast_r(r2) * inv_h);
        s += w;
        r += pj.z * w;
        if ((++n & (FOLD - 1)) == 0) fold();
    }
    __device__ void fold()
    {
        two_sum_acc(sh, sl, s);
        two_sum_acc(rh, rl, r);
        s = r = 0.f;
    }
};

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

template <int MIXED>
__global__ void __launch_bounds__(TPB) k_pass_a(Dev d)
{
    __shared__ unsigned lst_all[LMAX * TPB];
    unsigned *lst = lst_all + threadIdx.x;
    const int n = d.cnt->n_alive;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int cx, cy;
        cell_of(d, k, cx, cy);
        const float4 pi = d.P[k];
        const double2 xy = d.XY[k];
        const int s = d.order[k];
        if (MIXED) {
            BodyA32 f(d, pi.x, pi.y);
            listed_neighbors(d, k, xy.x, xy.y, cx, cy, pi.x, pi.y, lst, f);
            f.fold();
            // self term: W(0) = alpha_2 w(0)
            const float w0 = d.ph.w0f;
            two_sum_acc(f.sh, f.sl, w0);
            two_sum_acc(f.rh, f.rl, pi.z * w0);
            const float S = f.sh + f.sl, R = f.rh + f.rl;
            const float V = 1.0f / S;
            const float4 q = d.Qf[k];
            d.Qf[k] = make_float4(q.x, V, R, pi.z / R);
            d.snnb[k] = f.n + 1;
            d.rho[s] = (double)R;
            d.vol[s] = (double)V;
            d.nnb[s] = f.n + 1;
        } else {
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
// G_i = sum_j c_ij gW, which is also the background-pressure sum.  The self pair contributes
// nothing (gW = 0, p_j - p_i = 0) and is not listed.
// Solid particles counted in the drag: F_i = sum_{j fluid} c_ij [ -p~_ij gW + eta~_ij
// u_ij (gW . r_ij)/(r^2 + eta h^2) ] with u_ij = u_g,i - u_j (Eq. tvf-momentum_solid).
struct BodyB32 {
    const Dev &d;
    float rx, ry;
    float pi, Vi, rhoi, ui, vi, dui, dvi, mi_inv;
    bool solid;
    float a2h, inv_h, c2, nu2, nue2, eh2;
    float ax = 0, ay = 0, ap = 0, gx = 0, gy = 0;
    float axh = 0, axl = 0, ayh = 0, ayl = 0, aph = 0, apl = 0, gxh = 0, gxl = 0, gyh = 0, gyl = 0;
    float sdp = 0;
    int n = 0;
    __device__ BodyB32(const Dev &dd, float x, float y) : d(dd), rx(x), ry(y)
    {
        a2h = dd.ph.a2hf; inv_h = dd.ph.inv_hf; c2 = dd.ph.c2f; nu2 = 2.0f * dd.ph.nuf;
        nue2 = 2.0f * dd.ph.nuef; eh2 = dd.ph.eh2f;
    }
    __device__ void fold()
    {
        two_sum_acc(axh, axl, ax);
        two_sum_acc(ayh, ayl, ay);
        two_sum_acc(aph, apl, ap);
        two_sum_acc(gxh, gxl, gx);
        two_sum_acc(gyh, gyl, gy);
        ax = ay = ap = gx = gy = 0.f;
    }
    __device__ void operator()(unsigned e)
    {
        float4 pj;
        float dx, dy, r2;
        const int j = geom32(d, e, rx, ry, pj, dx, dy, r2);
        const float4 q = __ldg(d.Qf + j);  // (p, V, rho, m/rho)
        const float dp = q.x - pi;
        sdp += dp;
        if (solid && (d.stag[j] & 0x7f) != FLUID) return;
        const float4 bj = __ldg(d.Bf + j);  // (u, v, u~-u, v~-v)
        const float inv_r = r2 > 0.f ? rsqrtf(r2) : 0.f;
        const float dwq = quintic_dw(r2 * inv_r * inv_h);
        const float F = a2h * dwq * inv_r;
        const float gxv = F * dx, gyv = F * dy, gdotr = F * r2;
        const float cij = Vi * Vi + q.y * q.y;
        const float inv_rs = __fdividef(1.0f, rhoi + q.z);
        const float e_ = rhoi * dp * inv_rs;
        // eta~_ij (gW . r_ij)/(r^2 + eta h^2) = 2 nu hf,  hf = rho_i rho_j/(rho_i + rho_j) (...)
        const float hf = rhoi * q.z * inv_rs * __fdividef(gdotr, r2 + eh2);
        const float vis = nu2 * hf;
        const float uij = ui - bj.x, vij = vi - bj.y;
        const float cgx = cij * gxv, cgy = cij * gyv;
        gx += cgx;
        gy += cgy;
        if (solid) {
            ax += cij * (vis * uij) - e_ * cgx;
            ay += cij * (vis * vij) - e_ * cgy;
        } else {
            const float Ai = rhoi * (dui * gxv + dvi * gyv);
            const float Aj = q.z * (bj.z * gxv + bj.w * gyv);
            ax += cij * (0.5f * (ui * Ai + bj.x * Aj) + vis * uij) - e_ * cgx;
            ay += cij * (0.5f * (vi * Ai + bj.y * Aj) + vis * vij) - e_ * cgy;
            ap += rhoi * c2 * q.w * (uij * gxv + vij * gyv) - cij * mi_inv * nue2 * hf * dp;
        }
        if ((++n & (FOLD - 1)) == 0) fold();
    }
};

struct BodyB64 {
    const Dev &d;
    double qx, qy;
    double pi, Vi, rhoi, ui, vi, dui, dvi, mi_inv;
    bool solid;
    double ax = 0, ay = 0, apd = 0, gxs = 0, gys = 0, sdp = 0;
    __device__ BodyB64(const Dev &dd, double x, double y) : d(dd), qx(x), qy(y) {}
    __device__ void operator()(unsigned e)
    {
        const Phys &ph = d.ph;
        const int j = (int)(e >> 4);
        const double2 pv = d.PV[j];  // (p, V)
        const double dp = pv.x - pi;
        sdp += dp;
        if (solid && (d.stag[j] & 0x7f) != FLUID) return;
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

template <int MIXED>
__global__ void __launch_bounds__(TPB) k_pass_b(Dev d)
{
    __shared__ unsigned lst_all[LMAX * TPB];
    unsigned *lst = lst_all + threadIdx.x;
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
            BodyB32 f(d, pk.x, pk.y);
            const float4 q = d.Qf[k];
            const float4 b = d.Bf[k];
            f.pi = q.x; f.Vi = q.y; f.rhoi = q.z; f.ui = b.x; f.vi = b.y; f.dui = b.z; f.dvi = b.w;
            f.mi_inv = 1.0f / pk.z;
            f.solid = solid;
            listed_neighbors(d, k, xy.x, xy.y, cx, cy, pk.x, pk.y, lst, f);
            f.fold();
            sx = (double)f.axh + (double)f.axl;
            sy = (double)f.ayh + (double)f.ayl;
            spd = (double)f.aph + (double)f.apl;
            G0 = (double)f.gxh + (double)f.gxl;
            G1 = (double)f.gyh + (double)f.gyl;
            sdp = f.sdp;
            pi = q.x;
        } else {
            BodyB64 f(d, xy.x, xy.y);
            const double2 pv = d.PV[k], rm = d.RM[k], uv = d.UV[k], duv = d.DUV[k];
            f.pi = pv.x; f.Vi = pv.y; f.rhoi = rm.x; f.ui = uv.x; f.vi = uv.y;
            f.dui = duv.x; f.dvi = duv.y;
            f.mi_inv = 1.0 / d.Ms[k];
            f.solid = solid;
            listed_neighbors(d, k, xy.x, xy.y, cx, cy, pk.x, pk.y, lst, f);
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

// Lane-strided walk of the neighbours of a query point: f(j, dx, dy, r2) with the pair
// geometry in T (fp32 cell-relative for the mixed path, canonical fp64 otherwise).
template <int MIXED, class F>
__device__ __forceinline__ void lane_neighbors(const Dev &d, int lane, double qx, double qy, int cx,
                                               int cy, float rx, float ry, F &&f)
{
    for_block(d, cx, cy, [&](int ox, int oy, int j0, int j1) {
        const float rxo = rx - (float)ox * d.g.sxf, ryo = ry - (float)oy * d.g.syf;
#pragma unroll 1
        for (int j = j0 + lane; j < j1; j += 32) {
            float dxf, dyf, r2f;
            if (!is_member(d, rxo, ryo, __ldg(d.P + j), j, qx, qy, dxf, dyf, r2f)) continue;
            if (MIXED) {
                f(j, dxf, dyf, r2f);
            } else {
                const double2 xy = d.XY[j];
                double dx, dy;
                const double r2 = exact_r2(d.g, qx, qy, xy.x, xy.y, dx, dy);
                f(j, dx, dy, r2);
            }
        }
    });
}

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

template <class T>
__device__ __forceinline__ T sqrt_t(T x);
template <>
__device__ __forceinline__ float sqrt_t<float>(float x) { return fast_r(x); }
template <>
__device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }

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

template <int MIXED>
__global__ void __launch_bounds__(256) k_boundary(Dev d, int end_of_step)
{
    typedef typename std::conditional<MIXED, float, double>::type T;
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int lane = threadIdx.x & 31;
    const int nb = d.cnt->n_bnd;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const T a2 = (T)ph.a2, a2h = (T)ph.a2h, inv_h = (T)ph.inv_h;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += nwarps) {
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
            T a[4] = {0, 0, 0, 0};
            lane_neighbors<MIXED>(d, lane, xy.x, xy.y, cx, cy, pk.x, pk.y, [&](int j, T, T, T r2) {
                if ((d.stag[j] & 0x7f) != FLUID) return;
                const T w = a2 * quintic_w(sqrt_t<T>(r2) * inv_h);
                double p, u, v, mr;
                fluid_fields<MIXED>(d, j, p, u, v, mr);
                a[0] += w; a[1] += w * (T)p; a[2] += w * (T)u; a[3] += w * (T)v;
            });
            warp_sum(a);
            if (lane == 0) {
                const int wi = (t == WALL) ? 0 : 1;
                double pw, ug, vg;
                const double sw = a[0];
                if (sw > 0.0) {
                    pw = (double)a[1] / sw;
                    const double uf = (double)a[2] / sw, vf = (double)a[3] / sw;
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
            }
        } else if (t == INLET && ph.has_inlet) {
            // Mirrored inlet pressure (Sec. 3.2): first-order Taylor system (Eq. matform) at
            // the mirror point k = (2 x_in - x_o, y_o) over fluid l with r_lk = r_l - r_k and
            // V_l = m_l/rho_l, solved with partial pivoting; p_o = p_k - (r_o - r_k).grad p_k
            // (Eq. taylor2).  No fluid in reach: p_o = 0; singular system
            // (|det| <= 1e-9 |M00 M11 M22|): the Shepard value sum p W V / sum W V.
            const double xk = 2.0 * ph.x_in - xy.x, yk = xy.y;
            const int cx = cell_coord(xk, g.x_min, g.inv_sx, g.nx);
            const int cy = cell_coord(yk, g.y_min, g.inv_sy, g.ny);
            const float rx = (float)(xk - (g.x_min + (double)cx * g.sx));
            const float ry = (float)(yk - (g.y_min + (double)cy * g.sy));
            T a[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            lane_neighbors<MIXED>(d, lane, xk, yk, cx, cy, rx, ry, [&](int l, T dx, T dy, T r2) {
                if ((d.stag[l] & 0x7f) != FLUID) return;
                const T xlk = -dx, ylk = -dy;  // the walk gives r_k - r_l
                const T r = sqrt_t<T>(r2);
                double p, u, v, Vl;
                fluid_fields<MIXED>(d, l, p, u, v, Vl);
                const T w = a2 * quintic_w(r * inv_h);
                T wx = 0, wy = 0;
                if (r > (T)0) {
                    const T dw = a2h * quintic_dw(r * inv_h);
                    wx = dw * xlk / r;
                    wy = dw * ylk / r;
                }
                const T row[3] = {w * (T)Vl, wx * (T)Vl, wy * (T)Vl};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    a[3 * q + 0] += row[q];
                    a[3 * q + 1] += xlk * row[q];
                    a[3 * q + 2] += ylk * row[q];
                    a[9 + q] += (T)p * row[q];
                }
                a[12] += (T)1;
            });
            warp_sum(a);
            if (lane == 0) {
                double M[3][3], bb[3];
                for (int q = 0; q < 3; ++q) {
                    for (int c = 0; c < 3; ++c) M[q][c] = (double)a[3 * q + c];
                    bb[q] = (double)a[9 + q];
                }
                double pk = 0.0, gxp = 0.0, gyp = 0.0;
                if (a[12] > (T)0) {
                    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
                    pk = bb[0] / M[0][0];
                    if (!(fabs(det) <= 1e-9 * fabs(M[0][0] * M[1][1] * M[2][2]))) {
                        double sol[3];
                        if (solve3(M, bb, sol)) { pk = sol[0]; gxp = sol[1]; gyp = sol[2]; }
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
            }
        } else if (t == OUTLET && end_of_step && ph.has_outlet) {
            // Hybrid outlet (Sec. 3.4): red particles (fluid in reach) take the Shepard J2
            // of the fluid; blue ones the mean previous-step J2 of red outlet neighbours.
            // J3 = 0 gives p' = J2/2, u' = J2/(2 rho0 c); value = frozen average + acoustic
            // part (Eq. acou).  Written to the slot arrays only: the rates of this
            // evaluation still see the outlet values of the step.
            int cx, cy;
            cell_of(d, k, cx, cy);
            const float4 pk = d.P[k];
            T a[6] = {0, 0, 0, 0, 0, 0};
            lane_neighbors<MIXED>(d, lane, xy.x, xy.y, cx, cy, pk.x, pk.y, [&](int j, T, T, T r2) {
                const uint8_t tj = d.stag[j];
                if ((tj & 0x7f) == FLUID) {
                    const T w = a2 * quintic_w(sqrt_t<T>(r2) * inv_h);
                    a[0] += w;
                    a[1] += w * (T)d.AUX[j].x;
                    a[2] += (T)1;
                } else if (tj == (OUTLET | TAG_REDP)) {
                    const double2 x2 = d.AUX[j];
                    a[3] += (T)x2.x;
                    a[4] += (T)x2.y;
                    a[5] += (T)1;
                }
            });
            warp_sum(a);
            if (lane == 0) {
                const bool red = a[2] > (T)0;
                const double mr = (double)a[5];
                const double J2 = red ? (double)a[1] / (double)a[0] : (mr > 0 ? (double)a[3] / mr : 0.0);
                const double un = d.ubar[s] + J2 / (2.0 * ph.rho0 * ph.cs);
                const double adv = red ? un : (mr > 0 ? (double)a[4] / mr : d.ubar[s]);
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

int launch_pass_a(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_a<1><<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    else k_pass_a<0><<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    return 1;
}

int launch_boundary(const Dev &d, cudaStream_t s, int mixed, int end_of_step)
{
    // one warp per boundary particle (grid-stride); boundary particles are O(sqrt(N))
    const int blocks = min(grid_for(d.cap, 64), 152 * 16);
    if (mixed) k_boundary<1><<<blocks, 256, 0, s>>>(d, end_of_step);
    else k_boundary<0><<<blocks, 256, 0, s>>>(d, end_of_step);
    return 1;
}

int launch_pass_b(const Dev &d, cudaStream_t s, int mixed)
{
    if (mixed) k_pass_b<1><<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    else k_pass_b<0><<<grid_for(d.cap, TPB), TPB, 0, s>>>(d);
    return 1;
}

int launch_neighbor_dump(const Dev &d, cudaStream_t s, int mixed, const long long *start,
                         unsigned long long *ids)
{
    (void)mixed;
    k_dump<<<grid_for(d.cap, TPB), TPB, 0, s>>>(d, start, ids);
    return 1;
}

}  // namespace edac
