/*
 * CPU ORACLE -- test infrastructure, not part of the product path.
 *
 * A plain, slow, fp64 statement of one time step of the EDAC-TVF weakly
 * compressible SPH scheme with a mirrored-pressure inlet and the hybrid
 * (characteristic + do-nothing) outlet of Negi, Ramachandran & Haftu,
 * "An improved non-reflecting outlet boundary condition for weakly-compressible
 * SPH" (arXiv 1907.04034).  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code with the CUDA
 * path.
 *
 * Every sum over neighbours runs over j in ascending array order, and array
 * order is ascending particle id (new particles are appended, deleted ones are
 * compacted out).  Neighbours of i are { j : dx^2 + dy^2 < (3h)^2 } with the
 * minimum image taken on periodic axes; i itself is included.  The library is
 * built with -ffp-contract=off so that this predicate is evaluated exactly as
 * written.
 *
 * Readings of points the paper leaves open are listed where they are used
 * ("reading: ...").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FLUID 0
#define ORC_INLET 1
#define ORC_OUTLET 2
#define ORC_WALL 3
#define ORC_SLIPWALL 4
#define ORC_NAVG_MAX 8
/* outlet treatments: hybrid (Sec. 3.4), do-nothing (Sec. 3.1), modified do-nothing
 * (Sec. 3.1.1), method of characteristics (Sec. 3.3), mirroring (Sec. 3.2) */
#define ORC_OUT_HYBRID 0
#define ORC_OUT_DONOTHING 1
#define ORC_OUT_MOD_DONOTHING 2
#define ORC_OUT_CHARACTERISTIC 3
#define ORC_OUT_MIRROR 4
/* inlet velocity in time: steady modes; the 2D pulse (Sec. 4.2), ramp (Sec. 4.3) and
 * passing vortex (Sec. 4.4) of the outlet test problems */
#define ORC_IN_MODES 0
#define ORC_IN_PULSE 1
#define ORC_IN_RAMP 2
#define ORC_IN_VORTEX 3
#define ORC_MAX_MODES 16

typedef struct {
    double x_min, x_max, y_min, y_max;
    int periodic_x, periodic_y;
    double dx, hdx, rho0, U, nu, cs, alpha, pb, eta_reg, gx, gy, dt;
    int use_pavg;
    int has_inlet;
    double x_in;
    int n_in_layers;
    int n_modes;
    double modes[ORC_MAX_MODES];
    double inlet_y0, inlet_h;
    int inlet_kind;        /* ORC_IN_*: the inlet velocity in time (Sec. 4 test problems) */
    double inlet_prm[4];   /* its parameters (see inlet_velocity) */
    int has_outlet;
    double x_out;
    int n_out_layers;
    int n_avg;
    double i_thresh;
    int outlet_kind; /* ORC_OUT_*: the outlet treatment of Sec. 3 */
    double moc_u_ref, moc_p_ref; /* reference state of the characteristic outlet */
    int wall_slip[2];
    double wall_u[2], wall_v[2];
    int wall_drag[2];
    double drag_length;
    int neighbor_mode; /* 0: brute force over all pairs (the definition); 1: binned */
    int mirror_sign;   /* -1: Eq. (taylor2), the paper's modified extrapolation */
} orc_params;

typedef struct {
    int n, cap;
    /* particle fields, arrays of length cap */
    double *x, *y, *u, *v, *ut, *vt, *p, *m;
    unsigned char *tag;
    uint64_t *id;
    double *rho, *V;
    int *nnb;
    double *au, *av, *ap, *abu, *abv;
    double *fx, *fy;
    /* hybrid-outlet state: fluid ring buffers and time averages, outlet memory */
    double *ring; /* cap * ORC_NAVG_MAX * 3 */
    int *rpos;
    double *ubar, *vbar, *pbar, *J2;
    double *J2p, *advp;
    int *redp;
    /* stage base values */
    double *x0, *y0, *u0, *v0, *p0;
    uint64_t next_id;
    int error; /* 1: capacity exceeded, 2: particle outside the domain box */
    double t;  /* time of the state: nstep dt */
    int nstep; /* steps done */
    /* event log (may be NULL): 4 words per event (step, kind, id, other id) */
    uint64_t *ev;
    int ev_cap, ev_len;
    long long ev_dropped;
} orc_state;

/* one history record per step */
typedef struct {
    double fx, fy, mass_flux;
    double n_active, n_spawn, n_delete, n_to_outlet, pad;
} orc_hist;

/* ---------------------------------------------------------------------------
 * Quintic spline, Eq. (quintic-spline), Sec. 2:
 *   W(q) = a2 [ (3-q)^5 - 6(2-q)^5 + 15(1-q)^5 ]   0 <= q <= 1
 *          a2 [ (3-q)^5 - 6(2-q)^5 ]               1 <  q <= 2
 *          a2 (3-q)^5                              2 <  q <= 3
 *          0                                       q > 3
 *   a2 = 7 / (478 pi h^2),  q = r/h.
 * dW/dr = (a2/h) dw/dq with dw/dq = -5[ (3-q)^4 - 6(2-q)^4 + 15(1-q)^4 ] on the
 * same branches.
 * ------------------------------------------------------------------------- */
static double pow5(double a) { return a * a * a * a * a; }
static double pow4(double a) { return a * a * a * a; }

double orc_w(double q)
{
    if (q > 3.0) return 0.0;
    if (q <= 1.0) return pow5(3.0 - q) - 6.0 * pow5(2.0 - q) + 15.0 * pow5(1.0 - q);
    if (q <= 2.0) return pow5(3.0 - q) - 6.0 * pow5(2.0 - q);
    return pow5(3.0 - q);
}

double orc_dw(double q)
{
    if (q > 3.0) return 0.0;
    if (q <= 1.0) return -5.0 * (pow4(3.0 - q) - 6.0 * pow4(2.0 - q) + 15.0 * pow4(1.0 - q));
    if (q <= 2.0) return -5.0 * (pow4(3.0 - q) - 6.0 * pow4(2.0 - q));
    return -5.0 * pow4(3.0 - q);
}

static double alpha2(double h) { return 7.0 / (478.0 * M_PI * h * h); }

double orc_W(double r, double h) { return alpha2(h) * orc_w(r / h); }
double orc_dWdr(double r, double h) { return alpha2(h) / h * orc_dw(r / h); }

/* ---------------------------------------------------------------------------
 * Geometry: separation r_ij = r_i - r_j with the minimum image on periodic axes.
 * ------------------------------------------------------------------------- */
static double min_image(double d, int periodic, double L)
{
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

static double sep(const orc_params *P, double xi, double yi, double xj, double yj,
                  double *dx, double *dy)
{
    *dx = min_image(xi - xj, P->periodic_x, P->x_max - P->x_min);
    *dy = min_image(yi - yj, P->periodic_y, P->y_max - P->y_min);
    return (*dx) * (*dx) + (*dy) * (*dy);
}

static double h_of(const orc_params *P) { return P->hdx * P->dx; }
static double rc2_of(const orc_params *P)
{
    double rc = 3.0 * (P->hdx * P->dx);
    return rc * rc;
}

/* ---------------------------------------------------------------------------
 * Neighbour lists (CSR), j ascending.  Mode 0 tests every pair.  Mode 1 bins
 * particles into cells no smaller than 3h and tests only the 3x3 block of
 * cells around i; it must produce the same lists (a test pins that).
 * ------------------------------------------------------------------------- */
typedef struct {
    int *start; /* n+1 */
    int *idx;
    int total;
} nlist;

static void nlist_free(nlist *L)
{
    free(L->start);
    free(L->idx);
    L->start = NULL;
    L->idx = NULL;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* bins for mode 1 */
typedef struct {
    int nx, ny;
    double sx, sy;
    int *head; /* nx*ny+1 */
    int *items;
} bins;

static int bin_coord(double v, double lo, double s, int n)
{
    int c = (int)floor((v - lo) / s);
    if (c < 0) c = 0;
    if (c >= n) c = n - 1;
    return c;
}

static void bins_build(const orc_params *P, int n, const double *xs, const double *ys, bins *B)
{
    /* bins a little wider than 3h, so that rounding in the bin index can never
       put two particles closer than 3h more than one bin apart */
    double rc = 3.0 * h_of(P) * (1.0 + 1e-9);
    double Lx = P->x_max - P->x_min, Ly = P->y_max - P->y_min;
    B->nx = (int)floor(Lx / rc);
    B->ny = (int)floor(Ly / rc);
    if (B->nx < 1) B->nx = 1;
    if (B->ny < 1) B->ny = 1;
    B->sx = Lx / B->nx;
    B->sy = Ly / B->ny;
    int nc = B->nx * B->ny;
    B->head = (int *)calloc((size_t)nc + 1, sizeof(int));
    B->items = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cell = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) {
        int cx = bin_coord(xs[i], P->x_min, B->sx, B->nx);
        int cy = bin_coord(ys[i], P->y_min, B->sy, B->ny);
        cell[i] = cy * B->nx + cx;
        B->head[cell[i] + 1]++;
    }
    for (int c = 0; c < nc; c++) B->head[c + 1] += B->head[c];
    int *fill = (int *)malloc(sizeof(int) * (size_t)nc);
    memcpy(fill, B->head, sizeof(int) * (size_t)nc);
    for (int i = 0; i < n; i++) B->items[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
}

static void bins_free(bins *B)
{
    free(B->head);
    free(B->items);
}

/* the (unique) bins of the 3x3 block around the bin of point (x, y) */
static int block_bins(const orc_params *P, const bins *B, double x, double y, int *out)
{
    int cx = bin_coord(x, P->x_min, B->sx, B->nx);
    int cy = bin_coord(y, P->y_min, B->sy, B->ny);
    int cnt = 0;
    for (int oy = -1; oy <= 1; oy++) {
        int by = cy + oy;
        if (P->periodic_y) by = (by % B->ny + B->ny) % B->ny;
        else if (by < 0 || by >= B->ny) continue;
        for (int ox = -1; ox <= 1; ox++) {
            int bx = cx + ox;
            if (P->periodic_x) bx = (bx % B->nx + B->nx) % B->nx;
            else if (bx < 0 || bx >= B->nx) continue;
            int b = by * B->nx + bx, dup = 0;
            for (int t = 0; t < cnt; t++) dup |= (out[t] == b);
            if (!dup) out[cnt++] = b;
        }
    }
    return cnt;
}

/* neighbours of the points (qx, qy)[0..nq) among particles [0..n) that pass
 * filter (tag filter mask: bit t set = tag t admitted) */
static void build_lists(const orc_params *P, const orc_state *S, int nq, const double *qx,
                        const double *qy, unsigned mask, nlist *L)
{
    const double rc2 = rc2_of(P);
    int n = S->n;
    int *cnt = (int *)calloc((size_t)nq + 1, sizeof(int));
    int **tmp = (int **)calloc((size_t)(nq > 0 ? nq : 1), sizeof(int *));
    bins B;
    int use_bins = (P->neighbor_mode == 1);
    if (use_bins) bins_build(P, n, S->x, S->y, &B);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < nq; i++) {
        int capn = 64, c = 0;
        int *buf = (int *)malloc(sizeof(int) * (size_t)capn);
        double dx, dy;
        if (!use_bins) {
            for (int j = 0; j < n; j++) {
                if (!((mask >> S->tag[j]) & 1u)) continue;
                if (sep(P, qx[i], qy[i], S->x[j], S->y[j], &dx, &dy) < rc2) {
                    if (c == capn) { capn *= 2; buf = (int *)realloc(buf, sizeof(int) * (size_t)capn); }
                    buf[c++] = j;
                }
            }
        } else {
            int bl[9];
            int nb = block_bins(P, &B, qx[i], qy[i], bl);
            for (int t = 0; t < nb; t++) {
                for (int k = B.head[bl[t]]; k < B.head[bl[t] + 1]; k++) {
                    int j = B.items[k];
                    if (!((mask >> S->tag[j]) & 1u)) continue;
                    if (sep(P, qx[i], qy[i], S->x[j], S->y[j], &dx, &dy) < rc2) {
                        if (c == capn) { capn *= 2; buf = (int *)realloc(buf, sizeof(int) * (size_t)capn); }
                        buf[c++] = j;
                    }
                }
            }
            qsort(buf, (size_t)c, sizeof(int), cmp_int);
        }
        tmp[i] = buf;
        cnt[i] = c;
    }
    L->start = (int *)malloc(sizeof(int) * ((size_t)nq + 1));
    L->start[0] = 0;
    for (int i = 0; i < nq; i++) L->start[i + 1] = L->start[i] + cnt[i];
    L->total = L->start[nq];
    L->idx = (int *)malloc(sizeof(int) * (size_t)(L->total > 0 ? L->total : 1));
    for (int i = 0; i < nq; i++) {
        memcpy(L->idx + L->start[i], tmp[i], sizeof(int) * (size_t)cnt[i]);
        free(tmp[i]);
    }
    free(tmp);
    free(cnt);
    if (use_bins) bins_free(&B);
}

static int in_box(const orc_params *P, const orc_state *S)
{
    for (int i = 0; i < S->n; i++)
        if (!(S->x[i] >= P->x_min && S->x[i] < P->x_max && S->y[i] >= P->y_min && S->y[i] < P->y_max))
            return 0;
    return 1;
}

/* Inlet velocity profile u(y) = U + sum_k a_k sin(k pi (y - y0)/H). */
/* Inlet velocity (u, v) at height y and time t (Sec. 3 and the test problems of Sec. 4):
 *   modes:  u = U + sum_k a_k sin(k pi (y - y0) / H), v = 0 (steady);
 *   pulse:  u = U + A cos(pi (y - y0) / 12) exp(-(t - t0)^2 / delta) for t0 < t < t1, else U,
 *           v = 0, prm = (A, t0, t1, delta) (Eq. velfunc2, read with a negative exponent);
 *   ramp:   u = U min(t / T, 1), v = 0, prm = (T) (Sec. 4.3);
 *   vortex: with x_r = U (d0 - t) the distance of the vortex centre, which starts d0 upstream
 *           and moves at U, y_r = y - y_c and r^2 = x_r^2 + y_r^2:
 *           u = U + G y_r / (r^2 + c), v = -G x_r / (r^2 + c), prm = (G, c, d0, y_c)
 *           (Eqs. vortex, vortexx). */
static void inlet_velocity(const orc_params *P, double y, double t, double *u, double *v)
{
    const double *q = P->inlet_prm;
    *v = 0.0;
    if (P->inlet_kind == ORC_IN_PULSE) {
        *u = P->U;
        if (t > q[1] && t < q[2])
            *u += q[0] * cos(M_PI * (y - P->inlet_y0) / 12.0) * exp(-(t - q[1]) * (t - q[1]) / q[3]);
    } else if (P->inlet_kind == ORC_IN_RAMP) {
        *u = P->U * (t < q[0] ? t / q[0] : 1.0);
    } else if (P->inlet_kind == ORC_IN_VORTEX) {
        double xr = P->U * (q[2] - t), yr = y - q[3];
        double den = xr * xr + yr * yr + q[1];
        *u = P->U + q[0] * yr / den;
        *v = -q[0] * xr / den;
    } else {
        double uu = P->U;
        for (int k = 0; k < P->n_modes; k++)
            uu += P->modes[k] * sin((double)(k + 1) * M_PI * (y - P->inlet_y0) / P->inlet_h);
        *u = uu;
    }
}

static int is_wall(int t) { return t == ORC_WALL || t == ORC_SLIPWALL; }
static int wall_index(int t) { return t == ORC_WALL ? 0 : 1; }

/* ---------------------------------------------------------------------------
 * Pass A: summation density, Eq. (summation-density), and the number-density
 * volume V_i = 1 / sum_j W_ij (Sec. 2, below Eq. tvf-momentum), for every
 * particle whatever its tag; N_i counts all neighbours (Eq. pavg: "fluid and
 * boundary").
 * ------------------------------------------------------------------------- */
static void pass_a(const orc_params *P, orc_state *S, const nlist *L)
{
    const double h = h_of(P);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < S->n; i++) {
        double sw = 0.0, rho = 0.0, dx, dy;
        for (int t = L->start[i]; t < L->start[i + 1]; t++) {
            int j = L->idx[t];
            double r = sqrt(sep(P, S->x[i], S->y[i], S->x[j], S->y[j], &dx, &dy));
            double w = orc_W(r, h);
            sw += w;
            rho += S->m[j] * w;
        }
        S->rho[i] = rho;
        S->V[i] = 1.0 / sw;
        S->nnb[i] = L->start[i + 1] - L->start[i];
    }
}

/* ---------------------------------------------------------------------------
 * Solid walls (Sec. 2 cites Adami et al. 2012 for them).  Reading: static
 * walls, no body-force term in the pressure projection; p_w is the Shepard
 * average of fluid pressure; the ghost velocity is 2 u_wall - <u_f> for a
 * no-slip wall and (<u_f>, -<v_f>) for a slip wall whose normal is y.  With no
 * fluid neighbour: p_w = 0, u_g = u_wall.  When every fluid neighbour sits at
 * the edge of the support, where W vanishes in floating point (q rounds to 3),
 * the weights are all zero and <.> is the plain mean over those neighbours:
 * the limit of the weighted mean for one such neighbour, and a value that a
 * lower-precision W (the mixed path's) reaches for the same neighbour set.
 * ------------------------------------------------------------------------- */
static void walls(const orc_params *P, orc_state *S, const nlist *L)
{
    const double h = h_of(P);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < S->n; i++) {
        if (!is_wall(S->tag[i])) continue;
        int wi = wall_index(S->tag[i]);
        double sw = 0.0, sp = 0.0, su = 0.0, sv = 0.0, dx, dy;
        double mp = 0.0, mu = 0.0, mv = 0.0;
        int nf = 0;
        for (int t = L->start[i]; t < L->start[i + 1]; t++) {
            int j = L->idx[t];
            if (S->tag[j] != ORC_FLUID) continue;
            double r = sqrt(sep(P, S->x[i], S->y[i], S->x[j], S->y[j], &dx, &dy));
            double w = orc_W(r, h);
            sw += w;
            sp += S->p[j] * w;
            su += S->u[j] * w;
            sv += S->v[j] * w;
            mp += S->p[j];
            mu += S->u[j];
            mv += S->v[j];
            nf++;
        }
        double ug, vg, pw;
        if (nf > 0) {
            double uf, vf;
            if (sw > 0.0) {
                pw = sp / sw;
                uf = su / sw;
                vf = sv / sw;
            } else {
                pw = mp / (double)nf;
                uf = mu / (double)nf;
                vf = mv / (double)nf;
            }
            if (P->wall_slip[wi]) { ug = uf; vg = -vf; }
            else { ug = 2.0 * P->wall_u[wi] - uf; vg = 2.0 * P->wall_v[wi] - vf; }
        } else {
            pw = 0.0;
            ug = P->wall_u[wi];
            vg = P->wall_v[wi];
        }
        S->p[i] = pw;
        S->u[i] = ug;
        S->v[i] = vg;
        S->ut[i] = ug;
        S->vt[i] = vg;
    }
}

/* ---------------------------------------------------------------------------
 * Inlet pressure by mirroring (Sec. 3.2, Eqs. liu1_taylor..taylor2).
 * For inlet particle o the mirror point is k = (2 x_in - x_o, y_o).  Over the
 * fluid particles l within 3h of k, with r_lk = r_l - r_k, V_l = m_l / rho_l and
 * grad W_kl the gradient of W(x - x_k) at x = x_l, the first-order Taylor system
 *
 *   [ sum W V        sum x_lk W V        sum y_lk W V      ] [ p_k   ]   [ sum p_l W V   ]
 *   [ sum W_x V      sum x_lk W_x V      sum y_lk W_x V    ] [ p_k,x ] = [ sum p_l W_x V ]
 *   [ sum W_y V      sum x_lk W_y V      sum y_lk W_y V    ] [ p_k,y ]   [ sum p_l W_y V ]
 *
 * is solved by Gaussian elimination with partial pivoting and the inlet gets
 * p_o = p_k + sign (r_o - r_k) . grad p_k, sign = -1 (Eq. taylor2).
 * Reading: if k has no fluid neighbour, p_o = 0; if the system is singular,
 * |det M| <= 1e-9 |M00 M11 M22|, p_o is the Shepard value sum p W V / sum W V.
 * ------------------------------------------------------------------------- */
static int solve3(double A[3][3], double b[3], double xsol[3])
{
    int piv[3] = {0, 1, 2};
    for (int c = 0; c < 3; c++) {
        int best = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(A[piv[r]][c]) > fabs(A[piv[best]][c])) best = r;
        int tmp = piv[c];
        piv[c] = piv[best];
        piv[best] = tmp;
        double d = A[piv[c]][c];
        if (d == 0.0) return 0;
        for (int r = c + 1; r < 3; r++) {
            double f = A[piv[r]][c] / d;
            for (int k = c; k < 3; k++) A[piv[r]][k] -= f * A[piv[c]][k];
            b[piv[r]] -= f * b[piv[c]];
        }
    }
    for (int c = 2; c >= 0; c--) {
        double s = b[piv[c]];
        for (int k = c + 1; k < 3; k++) s -= A[piv[c]][k] * xsol[k];
        xsol[c] = s / A[piv[c]][c];
    }
    return 1;
}

static double det3(double M[3][3])
{
    return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
         - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
         + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* the values f_k and gradients of nf fields (fld[f][l]) at one mirror point k from its
 * fluid neighbours ls[0..nl); returns the fluid count.  One matrix, nf right-hand sides. */
static int mirror_values(const orc_params *P, const orc_state *S, double xk, double yk,
                         const int *ls, int nl, int nf, double *const *fld, double *fk,
                         double (*grad)[2])
{
    const double h = h_of(P);
    double M[3][3] = {{0}}, b[3][3] = {{0}}, mean[3] = {0};
    for (int t = 0; t < nl; t++) {
        int l = ls[t];
        double xlk, ylk;
        double r = sqrt(sep(P, S->x[l], S->y[l], xk, yk, &xlk, &ylk));
        double Vl = S->m[l] / S->rho[l];
        double w = orc_W(r, h);
        double wx = 0.0, wy = 0.0;
        if (r > 0.0) {
            double dw = orc_dWdr(r, h);
            wx = dw * xlk / r;
            wy = dw * ylk / r;
        }
        double row[3] = {w * Vl, wx * Vl, wy * Vl};
        for (int a = 0; a < 3; a++) {
            M[a][0] += row[a];
            M[a][1] += xlk * row[a];
            M[a][2] += ylk * row[a];
            for (int f = 0; f < nf; f++) b[f][a] += fld[f][l] * row[a];
        }
        for (int f = 0; f < nf; f++) mean[f] += fld[f][l];
    }
    for (int f = 0; f < nf; f++) grad[f][0] = grad[f][1] = 0.0;
    if (nl == 0) {
        for (int f = 0; f < nf; f++) fk[f] = 0.0;
        return 0;
    }
    if (!(M[0][0] > 0.0)) { /* all weights zero: plain mean of the fluid values */
        for (int f = 0; f < nf; f++) fk[f] = mean[f] / (double)nl;
        return nl;
    }
    double d = det3(M);
    int singular = fabs(d) <= 1e-9 * fabs(M[0][0] * M[1][1] * M[2][2]);
    for (int f = 0; f < nf; f++) {
        double A[3][3], rhs[3], sol[3];
        memcpy(A, M, sizeof(A));
        memcpy(rhs, b[f], sizeof(rhs));
        if (singular || !solve3(A, rhs, sol)) {
            fk[f] = b[f][0] / M[0][0];
            continue;
        }
        fk[f] = sol[0];
        grad[f][0] = sol[1];
        grad[f][1] = sol[2];
    }
    return nl;
}

/* the pressure alone (the inlet's field) */
static int mirror_value(const orc_params *P, const orc_state *S, double xk, double yk,
                        const int *ls, int nl, double *pk_out, double grad_out[2])
{
    double *fld[1] = {S->p};
    double g[1][2];
    int n = mirror_values(P, S, xk, yk, ls, nl, 1, fld, pk_out, g);
    grad_out[0] = g[0][0];
    grad_out[1] = g[0][1];
    return n;
}

static void inlet_mirror(const orc_params *P, orc_state *S)
{
    if (!P->has_inlet) return;
    int nq = 0;
    for (int i = 0; i < S->n; i++) nq += (S->tag[i] == ORC_INLET);
    if (nq == 0) return;
    int *who = (int *)malloc(sizeof(int) * (size_t)nq);
    double *qx = (double *)malloc(sizeof(double) * (size_t)nq);
    double *qy = (double *)malloc(sizeof(double) * (size_t)nq);
    nq = 0;
    for (int i = 0; i < S->n; i++)
        if (S->tag[i] == ORC_INLET) {
            who[nq] = i;
            qx[nq] = 2.0 * P->x_in - S->x[i];
            qy[nq] = S->y[i];
            nq++;
        }
    nlist L;
    build_lists(P, S, nq, qx, qy, 1u << ORC_FLUID, &L);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nq; t++) {
        int o = who[t];
        double pk, g[2];
        mirror_value(P, S, qx[t], qy[t], L.idx + L.start[t], L.start[t + 1] - L.start[t], &pk, g);
        double rx = S->x[o] - qx[t], ry = S->y[o] - qy[t];
        S->p[o] = pk + (double)P->mirror_sign * (rx * g[0] + ry * g[1]);
    }
    nlist_free(&L);
    free(who);
    free(qx);
    free(qy);
}

/* ---------------------------------------------------------------------------
 * Pass B: the number-density EDAC-TVF momentum equation, Eq. (tvf-momentum),
 * with p_avg of Eq. (pavg) and p~_ij of Eq. (tvf-p-ij-basa); the EDAC pressure
 * rate, Eq. (p-edac); the background-pressure part of Eq. (transport-vel); and
 * for solid particles counted in the drag the force of Eq. (tvf-momentum_solid).
 *
 *   a_i    = (1/m_i) sum_j c_ij [ -p~_ij gW + 1/2 (A_i + A_j).gW
 *                                 + eta~_ij u_ij (gW . r_ij) / (r_ij^2 + eta h^2) ] + g
 *   dp_i   = sum_j (m_j rho_i / rho_j) c^2 u_ij . gW
 *            + (c_ij / m_i) eta~e_ij p_ij (gW . r_ij) / (r_ij^2 + eta h^2)
 *   abg_i  = -(p_b / m_i) sum_j c_ij gW
 *   c_ij = V_i^2 + V_j^2,  A = rho u (x) (u~ - u)  so  A.gW = rho u ((u~ - u).gW),
 *   eta_i = rho_i nu (momentum) or rho_i nu_edac (pressure), nu_edac = alpha h c / 8
 *   (Eq. edac-nu), eta~_ij = 2 eta_i eta_j / (eta_i + eta_j), eta = eta_reg.
 * Reading: accelerations are computed for fluid and inlet particles (an inlet
 * particle that becomes fluid keeps the rate computed for it); u_ij uses the
 * momentum velocities, wall ghost velocities for wall j.  The solid force sums
 * over fluid j only, with u_ij = u_g,i - u_j, and its p~_ij is the interpolated
 * pressure (rho_j p_i + rho_i p_j)/(rho_i + rho_j) without the p_avg shift:
 * summed over all neighbours, the solid-solid pairs of that antisymmetric form
 * cancel in the total, so the fluid-only sum is the body force of Eq.
 * (tvf-momentum_solid); a p_avg,i shift on the one-sided fluid sum would instead
 * subtract about p_i times the surface element and remove the pressure drag
 * that the c_d of Table clcd (Sec. 4.6) contains.  wall_drag = 2 takes the
 * equation as printed instead: the sum runs over every neighbour (solid ones
 * included) and p~_ij carries the solid particle's own p_avg,i (Eq. pavg over
 * all its neighbours) when p_avg is on.
 * ------------------------------------------------------------------------- */
static void pass_b(const orc_params *P, orc_state *S, const nlist *L)
{
    const double h = h_of(P);
    const double c2 = P->cs * P->cs;
    const double nu_edac = P->alpha * h * P->cs / 8.0;
    const double eh2 = P->eta_reg * h * h;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < S->n; i++) {
        int ti = S->tag[i];
        int do_fluid = (ti == ORC_FLUID || ti == ORC_INLET);
        int do_solid = is_wall(ti) && P->wall_drag[wall_index(ti)];
        int literal = do_solid && P->wall_drag[wall_index(ti)] == 2;
        S->au[i] = S->av[i] = S->ap[i] = S->abu[i] = S->abv[i] = 0.0;
        S->fx[i] = S->fy[i] = 0.0;
        if (!do_fluid && !do_solid) continue;
        double pavg = 0.0;
        if (P->use_pavg && (!do_solid || literal)) {
            double sp = 0.0;
            for (int t = L->start[i]; t < L->start[i + 1]; t++) sp += S->p[L->idx[t]];
            pavg = sp / (double)S->nnb[i];
        }
        double mi = S->m[i], rhoi = S->rho[i], Vi = S->V[i];
        double Ai_f = rhoi; /* A_i.gW = rho_i u_i ((u~_i - u_i) . gW) */
        double sx = 0, sy = 0, sp_rate = 0, bx = 0, by = 0;
        double dxs, dys;
        for (int t = L->start[i]; t < L->start[i + 1]; t++) {
            int j = L->idx[t];
            if (do_solid && !literal && S->tag[j] != ORC_FLUID) continue;
            double r2 = sep(P, S->x[i], S->y[i], S->x[j], S->y[j], &dxs, &dys);
            double r = sqrt(r2);
            double gx = 0.0, gy = 0.0;
            if (r > 0.0) {
                double dw = orc_dWdr(r, h);
                gx = dw * dxs / r;
                gy = dw * dys / r;
            }
            double rhoj = S->rho[j], Vj = S->V[j];
            double cij = Vi * Vi + Vj * Vj;
            double ptil = (rhoj * (S->p[i] - pavg) + rhoi * (S->p[j] - pavg)) / (rhoi + rhoj);
            double uij = S->u[i] - S->u[j], vij = S->v[i] - S->v[j];
            double gdotr = gx * dxs + gy * dys;
            double etai = rhoi * P->nu, etaj = rhoj * P->nu;
            /* the harmonic mean of two zero viscosities (inviscid runs) is zero */
            double etil = etai + etaj > 0.0 ? 2.0 * etai * etaj / (etai + etaj) : 0.0;
            double visc = etil * gdotr / (r2 + eh2);
            if (do_solid) {
                sx += cij * (-ptil * gx + visc * uij);
                sy += cij * (-ptil * gy + visc * vij);
                continue;
            }
            double Ai = Ai_f * ((S->ut[i] - S->u[i]) * gx + (S->vt[i] - S->v[i]) * gy);
            double Aj = rhoj * ((S->ut[j] - S->u[j]) * gx + (S->vt[j] - S->v[j]) * gy);
            double Aix = Ai * S->u[i], Aiy = Ai * S->v[i];
            double Ajx = Aj * S->u[j], Ajy = Aj * S->v[j];
            sx += cij * (-ptil * gx + 0.5 * (Aix + Ajx) + visc * uij);
            sy += cij * (-ptil * gy + 0.5 * (Aiy + Ajy) + visc * vij);
            double ei = rhoi * nu_edac, ej = rhoj * nu_edac;
            double etile = ei + ej > 0.0 ? 2.0 * ei * ej / (ei + ej) : 0.0;
            sp_rate += (S->m[j] * rhoi / rhoj) * c2 * (uij * gx + vij * gy)
                     + (cij / mi) * etile * (S->p[i] - S->p[j]) * gdotr / (r2 + eh2);
            bx += cij * gx;
            by += cij * gy;
        }
        if (do_solid) {
            S->fx[i] = sx;
            S->fy[i] = sy;
        } else {
            S->au[i] = sx / mi + P->gx;
            S->av[i] = sy / mi + P->gy;
            S->ap[i] = sp_rate;
            S->abu[i] = -P->pb / mi * bx;
            S->abv[i] = -P->pb / mi * by;
        }
    }
}

/* One evaluation of all rates at the current state: lists, pass A, walls,
 * inlet mirror, pass B.  Returns 0 or an error code. */
int orc_evaluate(const orc_params *P, orc_state *S)
{
    if (P->neighbor_mode == 1 && !in_box(P, S)) {
        S->error = 2;
        return 2;
    }
    nlist L;
    build_lists(P, S, S->n, S->x, S->y, 0xFFu, &L);
    pass_a(P, S, &L);
    walls(P, S, &L);
    inlet_mirror(P, S);
    pass_b(P, S, &L);
    nlist_free(&L);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Hybrid outlet, Sec. 3.4 with the characteristic variables of Sec. 3.3.
 * Fluid side (after the corrector): the last n_avg samples of (u, v, p) of each
 * fluid particle form its time average, Eq. (timeevg); a sample is taken only
 * while the acoustic intensity p^2/(2 rho c) does not exceed
 * I = (rho U^2 / 2)^2 / (2 rho c), Eq. (acouinten).  Reading: rho is the fixed
 * reference rho0 in both; the sample is the instantaneous gauge pressure.
 * J2 = rho0 c (u - u_avg) + (p - p_avg_t), Eq. (characteristic-vars) with the
 * time averages as the reference state.
 * ------------------------------------------------------------------------- */
static double intensity_threshold(const orc_params *P)
{
    if (P->i_thresh >= 0.0) return P->i_thresh;
    double q = 0.5 * P->rho0 * P->U * P->U;
    return q * q / (2.0 * P->rho0 * P->cs);
}

static void ring_fill(const orc_params *P, orc_state *S, int i)
{
    double *rg = S->ring + (size_t)i * ORC_NAVG_MAX * 3;
    for (int k = 0; k < P->n_avg; k++) {
        rg[3 * k + 0] = S->u[i];
        rg[3 * k + 1] = S->v[i];
        rg[3 * k + 2] = S->p[i];
    }
    S->rpos[i] = 0;
    S->ubar[i] = S->u[i];
    S->vbar[i] = S->v[i];
    S->pbar[i] = S->p[i];
    S->J2[i] = 0.0;
}

static void ring_update(const orc_params *P, orc_state *S)
{
    const double I = intensity_threshold(P);
    const double rc = P->rho0 * P->cs;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < S->n; i++) {
        if (S->tag[i] != ORC_FLUID) continue;
        if (P->outlet_kind == ORC_OUT_CHARACTERISTIC) {
            /* Sec. 3.3 alone: J2 against the fixed reference state (u_ref, p_ref) */
            S->J2[i] = rc * (S->u[i] - P->moc_u_ref) + (S->p[i] - P->moc_p_ref);
            continue;
        }
        if (P->outlet_kind != ORC_OUT_HYBRID) continue;
        double *rg = S->ring + (size_t)i * ORC_NAVG_MAX * 3;
        double inten = S->p[i] * S->p[i] / (2.0 * P->rho0 * P->cs);
        if (inten <= I) {
            int k = S->rpos[i];
            rg[3 * k + 0] = S->u[i];
            rg[3 * k + 1] = S->v[i];
            rg[3 * k + 2] = S->p[i];
            S->rpos[i] = (k + 1) % P->n_avg;
        }
        double su = 0.0, sv = 0.0, sp = 0.0;
        for (int k = 0; k < P->n_avg; k++) {
            su += rg[3 * k + 0];
            sv += rg[3 * k + 1];
            sp += rg[3 * k + 2];
        }
        S->ubar[i] = su / (double)P->n_avg;
        S->vbar[i] = sv / (double)P->n_avg;
        S->pbar[i] = sp / (double)P->n_avg;
        S->J2[i] = rc * (S->u[i] - S->ubar[i]) + (S->p[i] - S->pbar[i]);
    }
}

/* Outlet side, once per step, after the corrector's evaluation.
 *
 * Hybrid (Sec. 3.4): an outlet particle with fluid neighbours ("red", Fig. io_moc)
 * takes J2 as the Shepard average of fluid J2, Eq. (shepard); one without ("blue")
 * takes the mean of the previous step's J2 of the red outlet particles in its
 * support, Eq. (average_old), or 0 if there are none (the Shepard average with all
 * weights zero is the plain mean, as for walls).  With J3 = 0: p' = J2/2,
 * u' = J2/(2 rho0 c).  The particle's value is its frozen time average plus this
 * acoustic part, Eq. (acou); v stays at its average.  The advection velocity of a
 * red particle is that u; a blue one takes the mean previous-step advection
 * velocity of the red particles in its support, else its frozen u average.
 * Reading: "previous step" values are the ones this routine stored one step
 * earlier, self included in the blue averages; the advection velocity set here
 * moves the particle in x during the next step's stages (x = x^n + tau adv, y
 * fixed), like the do-nothing update x^n = x^(n-1) + u^(n-1) dt of Sec. 3.1, so
 * outlet and fluid particles move together.
 *
 * Method of characteristics (Sec. 3.3): the same red/blue extrapolation of J2, with
 * a fixed reference state (u_ref, p_ref) instead of the time averages (the free
 * stream (U, 0) unless set; Sec. 4 fixes (1 m/s, 1 Pa) for its test problems):
 * p = p_ref + J2/2, u = u_ref + J2/(2 rho0 c); the transverse velocity keeps the
 * value frozen at the crossing.  A blue particle without red neighbours advects
 * with its own u.
 *
 * Do-nothing (Sec. 3.1): u, v, p stay frozen at their values at the crossing and
 * the particle advects with that u: nothing to update.
 *
 * Modified do-nothing (Sec. 3.1.1): values frozen as in do-nothing; the advection
 * velocity is the Shepard average of the fluid u, Eq. (shepard0), for red
 * particles; blue ones take the mean previous-step advection velocity of their red
 * neighbours (the rule Sec. 3.4 gives where the Shepard interpolation does not
 * reach), else their frozen u.
 *
 * Mirroring (Sec. 3.2 applied at the outlet): p, u and v by the Taylor
 * extrapolation of Eq. (matform) about k = (2 x_out - x_o, y_o) with the minus sign
 * of Eq. (taylor2); the particle advects with that u. */
static void outlet_mirror(const orc_params *P, orc_state *S)
{
    int nq = 0;
    for (int i = 0; i < S->n; i++) nq += (S->tag[i] == ORC_OUTLET);
    if (nq == 0) return;
    int *who = (int *)malloc(sizeof(int) * (size_t)nq);
    double *qx = (double *)malloc(sizeof(double) * (size_t)nq);
    double *qy = (double *)malloc(sizeof(double) * (size_t)nq);
    nq = 0;
    for (int i = 0; i < S->n; i++)
        if (S->tag[i] == ORC_OUTLET) {
            who[nq] = i;
            qx[nq] = 2.0 * P->x_out - S->x[i];
            qy[nq] = S->y[i];
            nq++;
        }
    nlist L;
    build_lists(P, S, nq, qx, qy, 1u << ORC_FLUID, &L);
    double *fo = (double *)malloc(sizeof(double) * 3 * (size_t)nq);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nq; t++) {
        int o = who[t];
        double *fld[3] = {S->p, S->u, S->v};
        double fk[3], g[3][2];
        mirror_values(P, S, qx[t], qy[t], L.idx + L.start[t], L.start[t + 1] - L.start[t], 3,
                      fld, fk, g);
        double rx = S->x[o] - qx[t], ry = S->y[o] - qy[t];
        for (int f = 0; f < 3; f++)
            fo[3 * t + f] = fk[f] + (double)P->mirror_sign * (rx * g[f][0] + ry * g[f][1]);
    }
    for (int t = 0; t < nq; t++) { /* written after all reads (the fields are inputs above) */
        int o = who[t];
        S->p[o] = fo[3 * t + 0];
        S->u[o] = fo[3 * t + 1];
        S->v[o] = fo[3 * t + 2];
        S->ut[o] = S->u[o];
        S->vt[o] = S->v[o];
        S->advp[o] = S->u[o];
        S->J2p[o] = 0.0;
        S->redp[o] = 0;
    }
    nlist_free(&L);
    free(fo);
    free(who);
    free(qx);
    free(qy);
}

static void outlet_update(const orc_params *P, orc_state *S, const nlist *L)
{
    const int kind = P->outlet_kind;
    if (kind == ORC_OUT_DONOTHING) return;
    if (kind == ORC_OUT_MIRROR) {
        outlet_mirror(P, S);
        return;
    }
    const double h = h_of(P);
    const double rc = P->rho0 * P->cs;
    int n = S->n;
    double *J2n = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *advn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int *redn = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int o = 0; o < n; o++) {
        if (S->tag[o] != ORC_OUTLET) continue;
        /* sf: Shepard sums of the fluid value (J2, or u for the modified do-nothing) */
        double sw = 0.0, sf = 0.0, sfm = 0.0, sjp = 0.0, sadv = 0.0, dx, dy;
        int nf = 0, mr = 0;
        for (int t = L->start[o]; t < L->start[o + 1]; t++) {
            int j = L->idx[t];
            if (S->tag[j] == ORC_FLUID) {
                double r = sqrt(sep(P, S->x[o], S->y[o], S->x[j], S->y[j], &dx, &dy));
                double w = orc_W(r, h);
                double fj = kind == ORC_OUT_MOD_DONOTHING ? S->u[j] : S->J2[j];
                sw += w;
                sf += w * fj;
                sfm += fj;
                nf++;
            } else if (S->tag[j] == ORC_OUTLET && S->redp[j]) {
                sjp += S->J2p[j];
                sadv += S->advp[j];
                mr++;
            }
        }
        int red = nf > 0;
        /* all weights zero (every fluid neighbour at the support edge): plain mean */
        double shep = red ? (sw > 0.0 ? sf / sw : sfm / (double)nf) : 0.0;
        double blue_adv = mr > 0 ? sadv / (double)mr : 0.0;
        if (kind == ORC_OUT_MOD_DONOTHING) {
            J2n[o] = 0.0;
            advn[o] = red ? shep : (mr > 0 ? blue_adv : S->ubar[o]);
            redn[o] = red;
            continue;
        }
        double J2 = red ? shep : (mr > 0 ? sjp / (double)mr : 0.0);
        double pa = 0.5 * J2, ua = J2 / (2.0 * rc);
        double u, p, adv;
        if (kind == ORC_OUT_CHARACTERISTIC) {
            u = P->moc_u_ref + ua;
            p = P->moc_p_ref + pa;
            adv = red ? u : (mr > 0 ? blue_adv : u);
        } else {
            u = S->ubar[o] + ua;
            p = S->pbar[o] + pa;
            adv = red ? u : (mr > 0 ? blue_adv : S->ubar[o]);
        }
        J2n[o] = J2;
        advn[o] = adv;
        redn[o] = red;
        S->u[o] = u;
        S->v[o] = S->vbar[o];
        S->p[o] = p;
        S->ut[o] = S->u[o];
        S->vt[o] = S->v[o];
    }
    for (int o = 0; o < n; o++) {
        if (S->tag[o] != ORC_OUTLET) continue;
        S->J2p[o] = J2n[o];
        S->advp[o] = advn[o];
        S->redp[o] = redn[o];
    }
    free(J2n);
    free(advn);
    free(redn);
}

/* move particle record from index a to index b (b <= a) */
static void move_rec(orc_state *S, int a, int b)
{
    if (a == b) return;
#define MV(f) S->f[b] = S->f[a]
    MV(x); MV(y); MV(u); MV(v); MV(ut); MV(vt); MV(p); MV(m); MV(tag); MV(id);
    MV(rho); MV(V); MV(nnb); MV(au); MV(av); MV(ap); MV(abu); MV(abv); MV(fx); MV(fy);
    MV(rpos); MV(ubar); MV(vbar); MV(pbar); MV(J2); MV(J2p); MV(advp); MV(redp);
    MV(x0); MV(y0); MV(u0); MV(v0); MV(p0);
#undef MV
    memcpy(S->ring + (size_t)b * ORC_NAVG_MAX * 3, S->ring + (size_t)a * ORC_NAVG_MAX * 3,
           sizeof(double) * ORC_NAVG_MAX * 3);
}

/* Particle recycling, end of Sec. 3.4: an inlet particle that crossed x_in
 * becomes fluid and a new inlet particle is created L_in = n_in dx upstream of
 * it; a fluid particle that crossed x_out becomes an outlet particle and keeps
 * its time averages (the other outlets: the values it has when it crosses); an
 * outlet particle past x_out + L_out is deleted.
 * Reading: transitions are taken once per step after the outlet update, in
 * ascending id; new ids are handed out in ascending parent id; the new inlet
 * particle copies its parent's y, p and m and takes u = u(y), v = 0. */
typedef struct {
    uint64_t id;
    int i;
} id_index;

static int by_id(const void *a, const void *b)
{
    uint64_t x = ((const id_index *)a)->id, y = ((const id_index *)b)->id;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Event log: the step's events, kind by kind (deletions, conversions to outlet,
 * spawns), each list already in ascending id; a step whose events do not all fit
 * is counted as dropped. */
static void log_events(orc_state *S, const id_index *del, int nd, const id_index *out, int no,
                       const id_index *par, const uint64_t *new_id, int ns)
{
    if (!S->ev) return;
    int tot = nd + no + ns;
    if (S->ev_len + tot > S->ev_cap) {
        S->ev_dropped += tot;
        return;
    }
    uint64_t *e = S->ev + 4 * (size_t)S->ev_len;
    for (int k = 0; k < tot; k++, e += 4) {
        e[0] = (uint64_t)S->nstep;
        if (k < nd) {
            e[1] = 0; e[2] = del[k].id; e[3] = 0;
        } else if (k < nd + no) {
            e[1] = 1; e[2] = out[k - nd].id; e[3] = 0;
        } else {
            e[1] = 2; e[2] = new_id[k - nd - no]; e[3] = par[k - nd - no].id;
        }
    }
    S->ev_len += tot;
}

static void recycle(const orc_params *P, orc_state *S, orc_hist *H)
{
    int n = S->n;
    double L_in = P->n_in_layers * P->dx, L_out = P->n_out_layers * P->dx;
    int nspawn = 0, ndel = 0, nout = 0;
    double mflux = 0.0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    id_index *spawn = (id_index *)malloc(sizeof(id_index) * nn);
    id_index *dels = (id_index *)malloc(sizeof(id_index) * nn);
    id_index *outs = (id_index *)malloc(sizeof(id_index) * nn);
    uint64_t *new_id = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    unsigned char *del = (unsigned char *)calloc(nn, 1);
    for (int i = 0; i < n; i++) {
        int t = S->tag[i];
        if (P->has_outlet && t == ORC_OUTLET && S->x[i] >= P->x_out + L_out) {
            del[i] = 1;
            dels[ndel].id = S->id[i];
            dels[ndel].i = i;
            ndel++;
        } else if (P->has_outlet && t == ORC_FLUID && S->x[i] >= P->x_out) {
            S->tag[i] = ORC_OUTLET;
            if (P->outlet_kind == ORC_OUT_HYBRID) {
                S->u[i] = S->ubar[i];
                S->v[i] = S->vbar[i];
                S->p[i] = S->pbar[i];
            } else { /* the other outlets freeze the values it crosses with */
                S->ubar[i] = S->u[i];
                S->vbar[i] = S->v[i];
                S->pbar[i] = S->p[i];
            }
            S->ut[i] = S->u[i];
            S->vt[i] = S->v[i];
            S->J2p[i] = 0.0;
            S->redp[i] = 0;
            S->advp[i] = S->ubar[i];
            mflux += S->m[i];
            outs[nout].id = S->id[i];
            outs[nout].i = i;
            nout++;
        } else if (P->has_inlet && t == ORC_INLET && S->x[i] >= P->x_in) {
            S->tag[i] = ORC_FLUID;
            ring_fill(P, S, i);
            spawn[nspawn].id = S->id[i];
            spawn[nspawn].i = i;
            nspawn++;
        }
    }
    /* ascending id within each kind; new ids follow the parents' order */
    qsort(spawn, (size_t)nspawn, sizeof(id_index), by_id);
    qsort(dels, (size_t)ndel, sizeof(id_index), by_id);
    qsort(outs, (size_t)nout, sizeof(id_index), by_id);
    /* new inlet particles: data taken before compaction moves the parents */
    double *nx_ = (double *)malloc(sizeof(double) * (size_t)(nspawn + 1));
    double *ny_ = (double *)malloc(sizeof(double) * (size_t)(nspawn + 1));
    double *np_ = (double *)malloc(sizeof(double) * (size_t)(nspawn + 1));
    double *nm_ = (double *)malloc(sizeof(double) * (size_t)(nspawn + 1));
    for (int k = 0; k < nspawn; k++) {
        int i = spawn[k].i;
        nx_[k] = S->x[i] - L_in;
        ny_[k] = S->y[i];
        np_[k] = S->p[i];
        nm_[k] = S->m[i];
    }
    int w = 0;
    for (int i = 0; i < n; i++) {
        if (del[i]) continue;
        move_rec(S, i, w);
        w++;
    }
    S->n = w;
    int made = 0;
    for (int k = 0; k < nspawn; k++) {
        if (S->n >= S->cap) {
            S->error = 1;
            break;
        }
        int i = S->n++;
        double uin, vin;
        inlet_velocity(P, ny_[k], S->t, &uin, &vin);
        S->x[i] = nx_[k];
        S->y[i] = ny_[k];
        S->u[i] = uin;
        S->v[i] = vin;
        S->ut[i] = uin;
        S->vt[i] = vin;
        S->p[i] = np_[k];
        S->m[i] = nm_[k];
        S->tag[i] = ORC_INLET;
        S->id[i] = S->next_id++;
        new_id[made++] = S->id[i];
        S->rho[i] = S->V[i] = 0.0;
        S->nnb[i] = 0;
        S->au[i] = S->av[i] = S->ap[i] = S->abu[i] = S->abv[i] = 0.0;
        S->fx[i] = S->fy[i] = 0.0;
        S->rpos[i] = 0;
        S->ubar[i] = S->vbar[i] = S->pbar[i] = S->J2[i] = 0.0;
        S->J2p[i] = S->advp[i] = 0.0;
        S->redp[i] = 0;
        S->x0[i] = S->y0[i] = S->u0[i] = S->v0[i] = S->p0[i] = 0.0;
    }
    H->n_spawn = nspawn;
    H->n_delete = ndel;
    H->n_to_outlet = nout;
    H->mass_flux = mflux / P->dt;
    H->n_active = S->n;
    log_events(S, dels, ndel, outs, nout, spawn, new_id, made);
    free(spawn);
    free(dels);
    free(outs);
    free(new_id);
    free(del);
    free(nx_);
    free(ny_);
    free(np_);
    free(nm_);
}

/* ---------------------------------------------------------------------------
 * Time integration.  Sec. 2 defers the integrator to the EDAC paper; reading:
 * a midpoint predictor-corrector from the same base state, stage length tau =
 * dt/2 (rates at t^n) then tau = dt (rates at t^(n+1/2)):
 *   u = u^n + tau du/dt;  u~ = u + tau a_bg  (Eq. transport-vel);
 *   x = x^n + tau u~     (Eq. advection);   p = p^n + tau dp/dt;
 * periodic axes wrap.  Inlet particles move with the prescribed u(y), v = 0;
 * outlet particles move in x only, with the advection velocity the outlet
 * update chose for them (their u, v, p stay frozen during the step).  Wall
 * particles do not move.
 * ------------------------------------------------------------------------- */
static double wrap(double v, int periodic, double lo, double hi)
{
    if (periodic) {
        if (v >= hi) v -= (hi - lo);
        else if (v < lo) v += (hi - lo);
    }
    return v;
}

static void save_base(orc_state *S)
{
    for (int i = 0; i < S->n; i++) {
        S->x0[i] = S->x[i];
        S->y0[i] = S->y[i];
        S->u0[i] = S->u[i];
        S->v0[i] = S->v[i];
        S->p0[i] = S->p[i];
    }
}

static void stage(const orc_params *P, orc_state *S, double tau)
{
    for (int i = 0; i < S->n; i++) {
        int t = S->tag[i];
        if (t == ORC_FLUID) {
            S->u[i] = S->u0[i] + tau * S->au[i];
            S->v[i] = S->v0[i] + tau * S->av[i];
            S->ut[i] = S->u[i] + tau * S->abu[i];
            S->vt[i] = S->v[i] + tau * S->abv[i];
            S->x[i] = wrap(S->x0[i] + tau * S->ut[i], P->periodic_x, P->x_min, P->x_max);
            S->y[i] = wrap(S->y0[i] + tau * S->vt[i], P->periodic_y, P->y_min, P->y_max);
            S->p[i] = S->p0[i] + tau * S->ap[i];
        } else if (t == ORC_INLET) {
            double uin, vin;
            inlet_velocity(P, S->y0[i], S->t + tau, &uin, &vin);
            S->u[i] = uin;
            S->v[i] = vin;
            S->ut[i] = uin;
            S->vt[i] = vin;
            S->x[i] = S->x0[i] + tau * uin;
        } else if (t == ORC_OUTLET) {
            S->x[i] = S->x0[i] + tau * S->advp[i];
        }
    }
}

/* Set-up: ring buffers and outlet memory from the initial fields, u~ = u, then
 * one evaluation gives the rates at t = 0. */
int orc_init(const orc_params *P, orc_state *S)
{
    S->error = 0;
    S->t = 0.0;
    S->nstep = 0;
    for (int i = 0; i < S->n; i++) {
        S->ut[i] = S->u[i];
        S->vt[i] = S->v[i];
        ring_fill(P, S, i);
        S->J2p[i] = 0.0;
        S->redp[i] = 0;
        S->advp[i] = S->u[i];
        if (S->id[i] >= S->next_id) S->next_id = S->id[i] + 1;
    }
    return orc_evaluate(P, S);
}

/* nsteps full steps; hist receives one record per step (may be NULL) */
int orc_step(const orc_params *P, orc_state *S, int nsteps, orc_hist *hist)
{
    for (int s = 0; s < nsteps; s++) {
        orc_hist H;
        memset(&H, 0, sizeof(H));
        save_base(S);
        stage(P, S, 0.5 * P->dt);
        if (orc_evaluate(P, S)) return S->error;
        stage(P, S, P->dt);
        ring_update(P, S);
        if (P->neighbor_mode == 1 && !in_box(P, S)) {
            S->error = 2;
            return 2;
        }
        nlist L;
        build_lists(P, S, S->n, S->x, S->y, 0xFFu, &L);
        pass_a(P, S, &L);
        walls(P, S, &L);
        inlet_mirror(P, S);
        pass_b(P, S, &L);
        for (int i = 0; i < S->n; i++) {
            int t = S->tag[i];
            if (is_wall(t) && P->wall_drag[wall_index(t)]) {
                H.fx += S->fx[i];
                H.fy += S->fy[i];
            }
        }
        if (P->has_outlet) outlet_update(P, S, &L);
        nlist_free(&L);
        S->nstep += 1;
        S->t = (double)S->nstep * P->dt;
        recycle(P, S, &H);
        if (hist) hist[s] = H;
        if (S->error) return S->error;
    }
    return 0;
}

/* Debug: neighbour lists of all particles at the current positions.  start has
 * n+1 entries; idx receives at most cap_idx entries.  Returns the total. */
int orc_neighbors(const orc_params *P, const orc_state *S, int *start, int *idx, int cap_idx)
{
    nlist L;
    build_lists(P, S, S->n, S->x, S->y, 0xFFu, &L);
    memcpy(start, L.start, sizeof(int) * ((size_t)S->n + 1));
    int tot = L.total;
    memcpy(idx, L.idx, sizeof(int) * (size_t)(tot < cap_idx ? tot : cap_idx));
    nlist_free(&L);
    return tot;
}

/* Debug: the mirror extrapolation for arbitrary points (pins Eq. matform). */
int orc_mirror_points(const orc_params *P, const orc_state *S, int nq, const double *qx,
                      const double *qy, double *pk, double *gradx, double *grady)
{
    nlist L;
    build_lists(P, S, nq, qx, qy, 1u << ORC_FLUID, &L);
    for (int t = 0; t < nq; t++) {
        double g[2];
        mirror_value(P, S, qx[t], qy[t], L.idx + L.start[t], L.start[t + 1] - L.start[t], &pk[t], g);
        gradx[t] = g[0];
        grady[t] = g[1];
    }
    nlist_free(&L);
    return 0;
}

/* Debug: the mirrored outlet update alone at the current fields (pins Sec. 3.2 at
 * the outlet with three fields). */
int orc_outlet_mirror(const orc_params *P, orc_state *S)
{
    outlet_mirror(P, S);
    return 0;
}

/* Probes (the measurement points of the Sec. 4 test problems): at each point the
 * Shepard average of the fluid p, u, v over fluid particles within 3h (all weights
 * zero: the plain mean; none: zeros) and their count; out[4 t + (0..3)]. */
int orc_probe(const orc_params *P, const orc_state *S, int nq, const double *qx,
              const double *qy, double *out)
{
    const double h = h_of(P), rc2 = rc2_of(P);
    for (int t = 0; t < nq; t++) {
        double sw = 0.0, sp = 0.0, su = 0.0, sv = 0.0, mp = 0.0, mu = 0.0, mv = 0.0, dx, dy;
        int nf = 0;
        for (int j = 0; j < S->n; j++) {
            if (S->tag[j] != ORC_FLUID) continue;
            double r2 = sep(P, qx[t], qy[t], S->x[j], S->y[j], &dx, &dy);
            if (!(r2 < rc2)) continue;
            double w = orc_W(sqrt(r2), h);
            sw += w;
            sp += w * S->p[j];
            su += w * S->u[j];
            sv += w * S->v[j];
            mp += S->p[j];
            mu += S->u[j];
            mv += S->v[j];
            nf++;
        }
        double *o = out + 4 * t;
        if (nf == 0) {
            o[0] = o[1] = o[2] = 0.0;
        } else if (sw > 0.0) {
            o[0] = sp / sw;
            o[1] = su / sw;
            o[2] = sv / sw;
        } else {
            o[0] = mp / (double)nf;
            o[1] = mu / (double)nf;
            o[2] = mv / (double)nf;
        }
        o[3] = (double)nf;
    }
    return 0;
}

int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_state(void) { return (int)sizeof(orc_state); }
int orc_sizeof_hist(void) { return (int)sizeof(orc_hist); }
