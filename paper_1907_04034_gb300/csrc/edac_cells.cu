// Cell-list build, time-integration stages, particle recycling and the end-of-step
// reduction of the EDAC SPH library (sm_103a).
//
// Cell build: a counting sort of live slots by cell (row-major, x fastest, cells of at
// least 3h): per-cell counts by atomics, one exclusive scan, a scatter, and a per-cell
// sort by slot that makes the order independent of the atomic order.  The gather then
// writes the cell-ordered copies the pair kernels read (fp32 cell-relative positions
// for the pre-test, fp64 positions, and the fields of the chosen precision).
#include "edac_internal.cuh"

namespace edac {

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Warp-aggregated append: every lane with `want` gets a distinct index into a list whose
// length lives at *counter; one atomic per warp.  All 32 lanes must call it.
__device__ __forceinline__ int warp_append(int *counter, bool want)
{
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask == 0u) return -1;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return want ? base + __popc(mask & ((1u << lane_id()) - 1u)) : -1;
}

// ------------------------------------------------------------------------- cell build
// Finite test on the exponent bits (integer pipe; the fp64 pipe is the scarce one here).
__device__ __forceinline__ bool finite_bits(double x)
{
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// The first step of the cell build for one live slot at (xs, ys): its cell and its place in
// the cell's count.  Run by k_cell_count, or fused into the stages, which hold the new position.
__device__ __forceinline__ void count_slot(const Dev &d, int s, double xs, double ys)
{
    const Geo &g = d.g;
    // the domain test on the unclamped cell index (integer compares; the fp64 pipe is the
    // scarce one), non-finite positions by their exponent bits
    const int cxr = __double2int_rd((xs - g.x_min) * g.inv_sx);
    const int cyr = __double2int_rd((ys - g.y_min) * g.inv_sy);
    if (!(finite_bits(xs) & finite_bits(ys) & (cxr >= 0) & (cxr < g.nx) & (cyr >= 0) &
          (cyr < g.ny))) {
        set_err(d, ERR_DOMAIN);
        if (atomicCAS(&d.cnt->err_rec, 0, 1) == 0) {
            d.cnt->err_tag = d.tag[s];
            d.cnt->err_id = d.id[s];
            d.cnt->err_x = xs;
            d.cnt->err_y = ys;
        }
    }
    const int cx = cxr < 0 ? 0 : (cxr >= g.nx ? g.nx - 1 : cxr);
    const int cy = cyr < 0 ? 0 : (cyr >= g.ny ? g.ny - 1 : cyr);
    const int c = cy * g.nx + cx;
    d.slot_cell[s] = c;
    d.within[s] = atomicAdd(d.cell_count + c, 1);
}

__global__ void k_cell_count(Dev d)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        if (d.tag[s] == TAG_DEAD) d.slot_cell[s] = -1;
        else count_slot(d, s, d.x[s], d.y[s]);
    }
}

// Exclusive scan of the per-cell counts into cell_start[0..ncells] in three launches:
// per-block totals of SCAN_TILE cells, a one-block scan of the totals (which also sets the
// live count and resets the boundary-list length), and the per-block scan with its offset.
constexpr int SCAN_TILE = 4096;  // cells per block, 4 per thread

__device__ __forceinline__ int block_exclusive_scan_1024(int v, int *sh_warp, int &total)
{
    const int t = threadIdx.x;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    if (lane_id() == 31) sh_warp[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
        int w = sh_warp[t];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (t >= o) w += y;
        }
        sh_warp[t] = w;
    }
    __syncthreads();
    total = sh_warp[31];
    const int r = x - v + ((t >> 5) > 0 ? sh_warp[(t >> 5) - 1] : 0);
    __syncthreads();
    return r;
}

__device__ __forceinline__ void scan_reduce(const Dev &d, int bid)
{
    __shared__ int sh[32];
    const int n = d.g.ncells;
    const int c0 = bid * SCAN_TILE + threadIdx.x * 4;
    int v = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) v += (c0 + q < n) ? d.cell_count[c0 + q] : 0;
    int total;
    block_exclusive_scan_1024(v, sh, total);
    if (threadIdx.x == 0) d.scan_part[bid] = total;
}

__global__ void __launch_bounds__(1024) k_scan_reduce(Dev d) { scan_reduce(d, blockIdx.x); }
__global__ void __launch_bounds__(1024) k_scan_reduce_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int) { scan_reduce(d, b); });
}

__device__ __forceinline__ void scan_top(const Dev &d, int nblk)
{
    __shared__ int sh[32];
    int run = 0;
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        const int b = b0 + (int)threadIdx.x;
        const int v = b < nblk ? d.scan_part[b] : 0;
        int total;
        const int ex = block_exclusive_scan_1024(v, sh, total);
        if (b < nblk) d.scan_part[b] = run + ex;
        run += total;
    }
    if (threadIdx.x == 0) {
        d.cell_start[d.g.ncells] = run;
        d.cnt->n_alive = run;
        d.cnt->n_bnd = 0;
    }
}

__global__ void __launch_bounds__(1024) k_scan_top(Dev d, int nblk) { scan_top(d, nblk); }
__global__ void __launch_bounds__(1024) k_scan_top_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int, int) {
        scan_top(d, (d.g.ncells + SCAN_TILE - 1) / SCAN_TILE);
    });
}

__device__ __forceinline__ void scan_down(const Dev &d, int bid)
{
    __shared__ int sh[32];
    const int n = d.g.ncells;
    const int c0 = bid * SCAN_TILE + threadIdx.x * 4;
    int v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (c0 + q < n) ? d.cell_count[c0 + q] : 0;
    int total;
    int run = block_exclusive_scan_1024(v[0] + v[1] + v[2] + v[3], sh, total) + d.scan_part[bid];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (c0 + q < n) d.cell_start[c0 + q] = run;
        run += v[q];
    }
}

__global__ void __launch_bounds__(1024) k_scan_down(Dev d) { scan_down(d, blockIdx.x); }
__global__ void __launch_bounds__(1024) k_scan_down_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int) { scan_down(d, b); });
}

__device__ __forceinline__ void cell_scatter(const Dev &d, int bid, int nblk)
{
    for (int s = bid * blockDim.x + threadIdx.x; s < d.cap; s += nblk * blockDim.x) {
        const int c = d.slot_cell[s];
        if (c < 0) continue;
        d.order_raw[d.cell_start[c] + d.within[s]] = s;
    }
}

__global__ void k_cell_scatter(Dev d) { cell_scatter(d, blockIdx.x, gridDim.x); }
__global__ void k_cell_scatter_b(BatchGrid bg) { run_member(bg, [](const Dev &d, int b, int nb) { cell_scatter(d, b, nb); }); }

// One warp per cell: rank the cell's slots (ascending slot, so the cell order does not depend
// on the order of the counting atomics), write the order, clear the cell's count for the next
// build, and gather the cell-ordered copies the pair kernels read.
template <int MIXED>
__device__ __forceinline__ void gather_one(const Dev &d, int s, int k, int c)
{
    const Geo &g = d.g;
    d.order[k] = s;
    d.cellk[k] = c;
    const int cx = c % g.nx, cy = c / g.nx;
    const double xs = d.x[s], ys = d.y[s];
    const float rx = d2f(xs - __ldg(d.org_x + cx));
    const float ry = d2f(ys - __ldg(d.org_y + cy));
    const double ms = d.m[s];
    // P.w: the fp32 pressure on the mixed path (pass A completes Qf from it), 0 on the other
    d.P[k] = make_float4(rx, ry, d2f(ms), MIXED ? d2f(d.p[s]) : 0.0f);
    d.XY[k] = make_double2(xs, ys);
    const uint8_t t = d.tag[s];
    d.stag[k] = (uint8_t)(t | ((t == OUTLET && d.redp[s]) ? TAG_REDP : 0));
    d.AUX[k] = make_double2(t == FLUID ? d.J2[s] : d.J2p[s], d.advp[s]);
    const double us = d.u[s], vs = d.v[s];
    const double dus = d.ut[s] - us, dvs = d.vt[s] - vs;
    if (MIXED) {
        d.Bf[k] = make_float4(d2f(us), d2f(vs), d2f(dus), d2f(dvs));
    } else {
        d.UV[k] = make_double2(us, vs);
        d.DUV[k] = make_double2(dus, dvs);
        d.PV[k] = make_double2(d.p[s], 0.0);
        d.Ms[k] = ms;
    }
}

// Order key of an fp64 value as an unsigned integer (the IEEE 754 ordering on the bits, on
// the integer pipe): non-negative values get the sign bit set, negative ones are inverted.
__device__ __forceinline__ unsigned long long order_key(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// One thread per particle in the scattered (atomic) order: the particle's rank among the
// particles of its cell, by x and then by slot, fixes its place in the cell order, which
// therefore does not depend on the order of the counting atomics; the thread then gathers
// the cell-ordered copies the pair kernels read.  Sorting a cell by x makes every row of
// three cells x-sorted, so that the mixed pair passes can take the candidates of a row as a
// window in x.  Cells hold ~13 particles, so the rank costs ~13 cached loads.
template <int MIXED>
__device__ __forceinline__ void cell_gather(const Dev &d, int bid, int nblk)
{
    const int n = d.cnt->n_alive;
    const int stride = nblk * blockDim.x;
    // uniform trip count per warp so that warp_append sees all 32 lanes
    for (int base = bid * blockDim.x; base < n; base += stride) {
        const int e = base + threadIdx.x;
        bool is_bnd = false;
        int k = 0;
        if (e < n) {
            const int s = d.order_raw[e];
            const int c = d.slot_cell[s];
            const int j0 = d.cell_start[c], j1 = d.cell_start[c + 1];
            const unsigned long long ks = order_key(d.x[s]);
            int rank = 0;
            for (int q = j0; q < j1; ++q) {
                const int sq = __ldg(d.order_raw + q);
                const unsigned long long kq = order_key(d.x[sq]);
                rank += (kq < ks) | ((kq == ks) & (sq < s));
            }
            k = j0 + rank;
            if (e == j0) d.cell_count[c] = 0;  // one thread per non-empty cell clears its count
            gather_one<MIXED>(d, s, k, c);
            is_bnd = d.tag[s] != FLUID;
        }
        const int slot = warp_append(&d.cnt->n_bnd, is_bnd);
        if (is_bnd) d.bnd[slot] = k;
    }
}

template <int MIXED>
__global__ void k_cell_gather(Dev d) { cell_gather<MIXED>(d, blockIdx.x, gridDim.x); }
template <int MIXED>
__global__ void k_cell_gather_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) { cell_gather<MIXED>(d, b, nb); });
}

// ---------------------------------------------------------------------------- stages
// Midpoint predictor-corrector from the base state of the step (the integrator of the
// EDAC paper is not restated in this paper; this is the library's reading):
//   fluid:  u = u^n + tau du/dt,  u~ = u + tau a_bg (Eq. transport-vel),
//           x = x^n + tau u~ (Eq. advection),  p = p^n + tau dp/dt;  periodic axes wrap;
//   inlet:  u = u(y), v = 0, x = x^n + tau u(y);
//   outlet: x = x^n + tau u_adv (y fixed), fields frozen within the step.
// The predictor (tau = dt/2) saves the base state; the corrector (tau = dt) also takes
// the time-average sample of the hybrid outlet (Eqs. timeevg, acouinten) and forms J2.
// Time-average ring of the hybrid outlet: fp64 samples on the fp64 path, fp32 samples on the
// mixed path (the average only feeds J2 and the frozen outlet values).
template <class R>
__device__ __forceinline__ void ring_sample(const Dev &d, int s, double un, double vn, double pn,
                                            double &ub, double &vb, double &pbv)
{
    const Phys &ph = d.ph;
    R *rg = reinterpret_cast<R *>(d.ring) + (size_t)s * NAVG_MAX * 3;
    // intensity p^2/(2 rho0 c) against I of Eq. (acouinten): the average only takes samples
    // below it
    if (pn * pn * ph.inv_2rc <= ph.I_thr) {
        const int k = d.rpos[s];
        rg[3 * k + 0] = narrow<R>(un); rg[3 * k + 1] = narrow<R>(vn); rg[3 * k + 2] = narrow<R>(pn);
        d.rpos[s] = (uint8_t)(k + 1 == ph.n_avg ? 0 : k + 1);
    }
    R su = 0, sv = 0, sp = 0;
    for (int k = 0; k < ph.n_avg; ++k) {
        su += rg[3 * k + 0]; sv += rg[3 * k + 1]; sp += rg[3 * k + 2];
    }
    ub = widen(su) * ph.inv_navg;
    vb = widen(sv) * ph.inv_navg;
    pbv = widen(sp) * ph.inv_navg;
}


// COUNT: also the first step of the next cell build (count_slot) at each slot's new position,
// which saves k_cell_count its pass over the positions.
template <bool CORR, int MIXED, bool COUNT>
__device__ __forceinline__ void stage(const Dev &d, double tau, int bid, int nblk)
{
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    for (int s = bid * blockDim.x + threadIdx.x; s < d.cap; s += nblk * blockDim.x) {
        const uint8_t t = d.tag[s];
        if (t == FLUID) {
            double x0, y0, u0, v0, p0;
            if (!CORR) {
                x0 = d.x[s]; y0 = d.y[s]; u0 = d.u[s]; v0 = d.v[s]; p0 = d.p[s];
                d.x0[s] = x0; d.y0[s] = y0; d.u0[s] = u0; d.v0[s] = v0; d.p0[s] = p0;
            } else {
                x0 = d.x0[s]; y0 = d.y0[s]; u0 = d.u0[s]; v0 = d.v0[s]; p0 = d.p0[s];
            }
            double au, av, ap, abu, abv;
            if (MIXED) {
                au = f2d(rate_f(d.au)[s]); av = f2d(rate_f(d.av)[s]); ap = f2d(rate_f(d.ap)[s]);
                abu = f2d(rate_f(d.abu)[s]); abv = f2d(rate_f(d.abv)[s]);
            } else {
                au = d.au[s]; av = d.av[s]; ap = d.ap[s]; abu = d.abu[s]; abv = d.abv[s];
            }
            const double un = u0 + tau * au;
            const double vn = v0 + tau * av;
            const double utn = un + tau * abu;
            const double vtn = vn + tau * abv;
            double xn = x0 + tau * utn;
            double yn = y0 + tau * vtn;
            if (g.px) { if (xn >= g.x_max) xn -= g.Lx; else if (xn < g.x_min) xn += g.Lx; }
            if (g.py) { if (yn >= g.y_max) yn -= g.Ly; else if (yn < g.y_min) yn += g.Ly; }
            const double pn = p0 + tau * ap;
            d.u[s] = un; d.v[s] = vn; d.ut[s] = utn; d.vt[s] = vtn;
            d.x[s] = xn; d.y[s] = yn; d.p[s] = pn;
            if (COUNT) count_slot(d, s, xn, yn);
            if (!(finite_bits(xn) & finite_bits(yn) & finite_bits(un) & finite_bits(vn) &
                  finite_bits(pn) & finite_bits(utn) & finite_bits(vtn)))
                set_err(d, ERR_NONFINITE);
            if (CORR && ph.has_outlet && ph.outlet_kind == OUT_HYBRID) {
                double ub, vb, pbv;
                if (MIXED) ring_sample<float>(d, s, un, vn, pn, ub, vb, pbv);
                else ring_sample<double>(d, s, un, vn, pn, ub, vb, pbv);
                d.ubar[s] = ub; d.vbar[s] = vb; d.pbar[s] = pbv;
                d.J2[s] = ph.rho0 * ph.cs * (un - ub) + (pn - pbv);
            } else if (CORR && ph.has_outlet && ph.outlet_kind == OUT_CHARACTERISTIC) {
                // Sec. 3.3 alone: J2 against the fixed reference state (u_ref, p_ref)
                d.J2[s] = ph.rho0 * ph.cs * (un - ph.moc_u_ref) + (pn - ph.moc_p_ref);
            }
        } else if (t == INLET) {
            double x0;
            if (!CORR) { x0 = d.x[s]; d.x0[s] = x0; } else { x0 = d.x0[s]; }
            double uin, vin;  // the inlet velocity at the end of the stage
            inlet_uv(ph, d.y[s], (double)d.cnt->step * ph.dt + tau, uin, vin);
            d.u[s] = uin; d.v[s] = vin; d.ut[s] = uin; d.vt[s] = vin;
            const double xn = x0 + tau * uin;
            d.x[s] = xn;
            if (COUNT) count_slot(d, s, xn, d.y[s]);
        } else if (t == OUTLET) {
            double x0;
            if (!CORR) { x0 = d.x[s]; d.x0[s] = x0; } else { x0 = d.x0[s]; }
            const double xn = x0 + tau * d.advp[s];
            d.x[s] = xn;
            if (COUNT) count_slot(d, s, xn, d.y[s]);
        } else if (COUNT) {
            if (t == TAG_DEAD) d.slot_cell[s] = -1;
            else count_slot(d, s, d.x[s], d.y[s]);  // walls: not moved by the stages
        }
    }
}

template <bool CORR, int MIXED, bool COUNT>
__global__ void k_stage(Dev d, double tau) { stage<CORR, MIXED, COUNT>(d, tau, blockIdx.x, gridDim.x); }
// batched: each member's own time step (predictor dt/2, corrector dt)
template <bool CORR, int MIXED, bool COUNT>
__global__ void k_stage_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) {
        stage<CORR, MIXED, COUNT>(d, CORR ? d.ph.dt : 0.5 * d.ph.dt, b, nb);
    });
}

// ------------------------------------------------------------------------- recycling
// Ring buffer of a particle that becomes fluid: all samples = current (u, v, p).
__device__ __forceinline__ void ring_fill(const Dev &d, int s)
{
    const double u = d.u[s], v = d.v[s], p = d.p[s];
    if (d.mixed) {
        float *rg = reinterpret_cast<float *>(d.ring) + (size_t)s * NAVG_MAX * 3;
        for (int k = 0; k < d.ph.n_avg; ++k) { rg[3 * k] = (float)u; rg[3 * k + 1] = (float)v; rg[3 * k + 2] = (float)p; }
    } else {
        double *rg = d.ring + (size_t)s * NAVG_MAX * 3;
        for (int k = 0; k < d.ph.n_avg; ++k) { rg[3 * k] = u; rg[3 * k + 1] = v; rg[3 * k + 2] = p; }
    }
    d.rpos[s] = 0;
    d.ubar[s] = u; d.vbar[s] = v; d.pbar[s] = p; d.J2[s] = 0.0;
}

// Rates of slot s set to zero, in the path's storage (fp32 on the mixed path).
__device__ __forceinline__ void zero_rates(const Dev &d, int s)
{
    if (d.mixed) {
        rate_f(d.au)[s] = rate_f(d.av)[s] = rate_f(d.ap)[s] = rate_f(d.abu)[s] = rate_f(d.abv)[s] = 0.0f;
    } else {
        d.au[s] = d.av[s] = d.ap[s] = d.abu[s] = d.abv[s] = 0.0;
    }
}

// Transitions of the end of Sec. 3.4, taken once per step after the outlet update:
// outlet past x_out + L_out -> deleted; fluid past x_out -> outlet (keeps its time
// averages; the other outlets: the values it crosses with); inlet past x_in -> fluid (a new
// inlet particle is spawned by k_end_step).
// Events go to per-kind lists by warp-aggregated appends; k_end_step puts them in
// ascending id order before ids and slots are handed out.
__device__ __forceinline__ void recycle_mark(const Dev &d, int bid, int nblk)
{
    const Phys &ph = d.ph;
    const int stride = nblk * blockDim.x;
    for (int base = bid * blockDim.x; base < d.cap; base += stride) {
        const int s = base + threadIdx.x;
        bool del = false, out = false, spawn = false;
        if (s < d.cap) {
            const uint8_t t = d.tag[s];
            if (t == OUTLET && ph.has_outlet) {
                del = d.x[s] >= ph.x_out + ph.L_out;
            } else if (t == FLUID && ph.has_outlet) {
                out = d.x[s] >= ph.x_out;
            } else if (t == INLET && ph.has_inlet) {
                spawn = d.x[s] >= ph.x_in;
            }
        }
        const int idel = warp_append(&d.cnt->n_del, del);
        const int iout = warp_append(&d.cnt->n_out, out);
        const int ispw = warp_append(&d.cnt->n_spawn, spawn);
        if (del) {
            d.tag[s] = TAG_DEAD;
            if (idel < LIST_MAX) { d.ev_del_key[idel] = d.id[s]; d.ev_del_slot[idel] = s; }
            else set_err(d, ERR_LIST);
        }
        if (out) {
            d.tag[s] = OUTLET;
            if (ph.outlet_kind == OUT_HYBRID) {  // keeps its time averages
                d.u[s] = d.ubar[s]; d.v[s] = d.vbar[s]; d.p[s] = d.pbar[s];
            } else {  // the other outlets freeze the values it crosses with
                d.ubar[s] = d.u[s]; d.vbar[s] = d.v[s]; d.pbar[s] = d.p[s];
            }
            const double ub = d.ubar[s];
            d.ut[s] = ub; d.vt[s] = d.vbar[s];
            d.J2p[s] = 0.0; d.redp[s] = 0; d.advp[s] = ub;
            if (iout < LIST_MAX) { d.ev_out_key[iout] = d.id[s]; d.ev_out_m[iout] = d.m[s]; }
            else set_err(d, ERR_LIST);
        }
        if (spawn) {
            d.tag[s] = FLUID;
            ring_fill(d, s);
            if (ispw < LIST_MAX) { d.ev_spawn_key[ispw] = d.id[s]; d.ev_spawn_slot[ispw] = s; }
            else set_err(d, ERR_LIST);
        }
    }
}

__global__ void k_recycle_mark(Dev d) { recycle_mark(d, blockIdx.x, gridDim.x); }
__global__ void k_recycle_mark_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int b, int nb) { recycle_mark(d, b, nb); });
}

// rank of key[i] among key[0..n) (keys are unique particle ids)
__device__ __forceinline__ int rank_of(const unsigned long long *key, int n, int i)
{
    const unsigned long long k = key[i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += (key[j] < k);
    return r;
}

__device__ double block_sum_1024(double v, double *sh)
{
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// End of a step, one block of 1024 threads: the drag/lift sum over the solid particles
// (Eq. tvf-momentum_solid summed over the body; fixed-shape tree), the canonical
// ordering of the recycling events, slot and id hand-out for spawned inlet particles
// (ascending parent id), the mass flux, one history record and, when a log is set, the
// step's events (deletions, conversions to outlet, spawns; each kind in ascending id) or,
// when they do not all fit, their count as dropped.
__device__ __forceinline__ void end_step(const Dev &d, double *scratch_m)
{
    __shared__ double sh[1024];
    Counters *C = d.cnt;
    const int t = threadIdx.x;
    const Phys &ph = d.ph;
    // forces
    double fx = 0.0, fy = 0.0;
    for (int i = t; i < C->n_drag; i += 1024) {
        const int s = d.drag_slots[i];
        fx += d.fx[s];
        fy += d.fy[s];
    }
    fx = block_sum_1024(fx, sh);
    fy = block_sum_1024(fy, sh);
    const int n_del = min(C->n_del, LIST_MAX);
    const int n_out = min(C->n_out, LIST_MAX);
    const int n_spawn = min(C->n_spawn, LIST_MAX);
    const int ev0 = C->ev_len, stepno = C->step + 1;
    const int n_ev = n_del + n_out + min(n_spawn, C->free_top + n_del);
    const bool logged = d.evlog != nullptr && (long long)ev0 + n_ev <= (long long)d.ev_cap;
    // mass flux: converted masses summed in ascending id order
    for (int i = t; i < n_out; i += 1024) {
        const int r = rank_of(d.ev_out_key, n_out, i);
        scratch_m[r] = d.ev_out_m[i];
        if (logged) d.evlog[ev0 + n_del + r] = EventRec{d.ev_out_key[i], 0ull, stepno, EV_TO_OUTLET};
    }
    __syncthreads();
    double ms = 0.0;
    for (int i = t; i < n_out; i += 1024) ms += scratch_m[i];
    ms = block_sum_1024(ms, sh);
    // freed slots pushed in ascending id order
    const int top0 = C->free_top;
    for (int i = t; i < n_del; i += 1024) {
        const int r = rank_of(d.ev_del_key, n_del, i);
        d.free_stack[top0 + r] = d.ev_del_slot[i];
        if (logged) d.evlog[ev0 + r] = EventRec{d.ev_del_key[i], 0ull, stepno, EV_DELETE};
    }
    __syncthreads();
    const int top1 = top0 + n_del;
    const int n_new = min(n_spawn, top1);
    const unsigned long long id0 = C->next_id;
    for (int i = t; i < n_spawn; i += 1024) {
        const int r = rank_of(d.ev_spawn_key, n_spawn, i);
        if (r >= n_new) continue;
        const int ps = d.ev_spawn_slot[i];
        const int s = d.free_stack[top1 - 1 - r];
        d.spawn_map[r] = make_int2(ps, s);
        const double yv = d.y[ps];
        double uin, vin;  // the inlet velocity at the end of the step
        inlet_uv(ph, yv, (double)(C->step + 1) * ph.dt, uin, vin);
        d.x[s] = d.x[ps] - ph.L_in;
        d.y[s] = yv;
        d.u[s] = uin; d.v[s] = vin; d.ut[s] = uin; d.vt[s] = vin;
        d.p[s] = d.p[ps];
        d.m[s] = d.m[ps];
        d.id[s] = id0 + (unsigned long long)r;
        if (logged)
            d.evlog[ev0 + n_del + n_out + r] = EventRec{id0 + (unsigned long long)r, d.ev_spawn_key[i], stepno, EV_SPAWN};
        zero_rates(d, s);
        d.fx[s] = d.fy[s] = 0.0;
        d.rho[s] = d.vol[s] = 0.0;
        d.nnb[s] = 0;
        d.rpos[s] = 0;
        d.ubar[s] = d.vbar[s] = d.pbar[s] = d.J2[s] = 0.0;
        d.J2p[s] = d.advp[s] = 0.0;
        d.redp[s] = 0;
        d.x0[s] = d.y0[s] = d.u0[s] = d.v0[s] = d.p0[s] = 0.0;
        __threadfence();
        d.tag[s] = INLET;
    }
    __syncthreads();
    if (t == 0) {
        if (n_new < n_spawn) atomicOr(&C->err, ERR_CAPACITY);
        C->free_top = top1 - n_new;
        C->next_id = id0 + (unsigned long long)n_new;
        C->last_spawn = n_new;
        C->n_alive = C->n_alive - n_del + n_new;
        const int slot = C->step % d.max_history;
        double *h = d.hist + (size_t)slot * 8;
        h[0] = fx; h[1] = fy; h[2] = ms / ph.dt; h[3] = (double)C->n_alive;
        h[4] = (double)n_spawn; h[5] = (double)n_del; h[6] = (double)n_out; h[7] = 0.0;
        C->step += 1;
        C->hist_len = min(C->hist_len + 1, d.max_history);
        C->n_del = 0; C->n_out = 0; C->n_spawn = 0;
        if (logged) C->ev_len = ev0 + n_ev;
        else if (d.evlog) C->ev_dropped += (unsigned long long)n_ev;
    }
}

__global__ void __launch_bounds__(1024) k_end_step(Dev d, double *scratch_m) { end_step(d, scratch_m); }
__global__ void __launch_bounds__(1024) k_end_step_b(BatchGrid bg)
{
    run_member(bg, [](const Dev &d, int, int) { end_step(d, d.scratch_m); });
}

// Set-up after an upload: u~ = u, ring buffers and outlet memory from the initial fields.
__global__ void k_init(Dev d)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
        if (d.tag[s] == TAG_DEAD) continue;
        d.ut[s] = d.u[s];
        d.vt[s] = d.v[s];
        ring_fill(d, s);
        d.J2p[s] = 0.0;
        d.redp[s] = 0;
        d.advp[s] = d.u[s];
        zero_rates(d, s);
        d.fx[s] = d.fy[s] = 0.0;
        d.x0[s] = d.x[s]; d.y0[s] = d.y[s]; d.u0[s] = d.u[s]; d.v0[s] = d.v[s]; d.p0[s] = d.p[s];
    }
}

int grid_for(int n)
{
    int b = (n + TPB - 1) / TPB;
    return b < 1 ? 1 : b;
}

}  // namespace

// cell_count is all zero on entry: cleared by the workspace reset at upload and by
// k_cell_gather of the previous build.
int launch_rebuild(const Dev &d, cudaStream_t s, int mixed, int counted)
{
    const int nblk = (d.g.ncells + SCAN_TILE - 1) / SCAN_TILE;
    if (!counted) k_cell_count<<<grid_for(d.cap), TPB, 0, s>>>(d);
    k_scan_reduce<<<nblk, 1024, 0, s>>>(d);
    k_scan_top<<<1, 1024, 0, s>>>(d, nblk);
    k_scan_down<<<nblk, 1024, 0, s>>>(d);
    k_cell_scatter<<<grid_for(d.cap), TPB, 0, s>>>(d);
    if (mixed) k_cell_gather<1><<<grid_for(d.cap), TPB, 0, s>>>(d);
    else k_cell_gather<0><<<grid_for(d.cap), TPB, 0, s>>>(d);
    return counted ? 5 : 6;
}

template <bool CORR, bool COUNT>
void stage_of(const Dev &d, cudaStream_t s, int mixed, double tau)
{
    const int gb = grid_for(d.cap);
    if (mixed) k_stage<CORR, 1, COUNT><<<gb, TPB, 0, s>>>(d, tau);
    else k_stage<CORR, 0, COUNT><<<gb, TPB, 0, s>>>(d, tau);
}

int launch_stage(const Dev &d, cudaStream_t s, int mixed, int corrector, int count)
{
    if (corrector) {
        if (count) stage_of<true, true>(d, s, mixed, d.ph.dt);
        else stage_of<true, false>(d, s, mixed, d.ph.dt);
    } else {
        if (count) stage_of<false, true>(d, s, mixed, 0.5 * d.ph.dt);
        else stage_of<false, false>(d, s, mixed, 0.5 * d.ph.dt);
    }
    return 1;
}

int launch_recycle(const Dev &d, cudaStream_t s)
{
    k_recycle_mark<<<grid_for(d.cap), TPB, 0, s>>>(d);
    k_end_step<<<1, 1024, 0, s>>>(d, d.scratch_m);
    return 2;
}

int launch_init(const Dev &d, cudaStream_t s)
{
    k_init<<<grid_for(d.cap), TPB, 0, s>>>(d);
    return 1;
}

// ---------------------------------------------------------------- batched launches
int launch_stage_batch(const BatchPlan &p, cudaStream_t s, int corrector)
{
    const int gb = p.total[BK_CAP];
    const BatchGrid bg = p.grid(BK_CAP);
    if (corrector) {
        if (p.mixed) k_stage_b<true, 1, true><<<gb, TPB, 0, s>>>(bg);
        else k_stage_b<true, 0, true><<<gb, TPB, 0, s>>>(bg);
    } else {
        if (p.mixed) k_stage_b<false, 1, true><<<gb, TPB, 0, s>>>(bg);
        else k_stage_b<false, 0, true><<<gb, TPB, 0, s>>>(bg);
    }
    return 1;
}

// the cell count was fused into the stages (counted)
int launch_rebuild_batch(const BatchPlan &p, cudaStream_t s)
{
    k_scan_reduce_b<<<p.total[BK_SCAN], 1024, 0, s>>>(p.grid(BK_SCAN));
    k_scan_top_b<<<p.total[BK_ONE], 1024, 0, s>>>(p.grid(BK_ONE));
    k_scan_down_b<<<p.total[BK_SCAN], 1024, 0, s>>>(p.grid(BK_SCAN));
    k_cell_scatter_b<<<p.total[BK_CAP], TPB, 0, s>>>(p.grid(BK_CAP));
    if (p.mixed) k_cell_gather_b<1><<<p.total[BK_CAP], TPB, 0, s>>>(p.grid(BK_CAP));
    else k_cell_gather_b<0><<<p.total[BK_CAP], TPB, 0, s>>>(p.grid(BK_CAP));
    return 5;
}

int launch_recycle_batch(const BatchPlan &p, cudaStream_t s)
{
    k_recycle_mark_b<<<p.total[BK_CAP], TPB, 0, s>>>(p.grid(BK_CAP));
    k_end_step_b<<<p.total[BK_ONE], 1024, 0, s>>>(p.grid(BK_ONE));
    return 2;
}

int cells_batch_blocks(const Dev &d, int kind)
{
    if (kind == BK_CAP) return grid_for(d.cap);
    if (kind == BK_SCAN) return (d.g.ncells + SCAN_TILE - 1) / SCAN_TILE;
    if (kind == BK_ONE) return 1;
    return -1;
}

}  // namespace edac

// ------------------------------------------------------------------------------ probes
namespace edac {
namespace {

// Per block and probe: [sum W, sum W p, sum W u, sum W v, sum p, sum u, sum v, count] over
// the fluid particles within 3h of the probe (exact membership test), over the slot arrays.
__global__ void __launch_bounds__(256) k_probe_part(Dev d, ProbePts q, double *part)
{
    __shared__ double red[8][8];
    const Geo &g = d.g;
    const Phys &ph = d.ph;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = 0; t < q.n; ++t) {
        double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < d.cap; s += gridDim.x * blockDim.x) {
            if (d.tag[s] != FLUID) continue;
            double dx, dy;
            const double r2 = exact_r2(g, q.x[t], q.y[t], d.x[s], d.y[s], dx, dy);
            if (!(r2 < g.rc2)) continue;
            const double wv = ph.a2 * quintic_w(sqrt(r2) * ph.inv_h);
            const double p = d.p[s], u = d.u[s], v = d.v[s];
            a[0] += wv; a[1] += wv * p; a[2] += wv * u; a[3] += wv * v;
            a[4] += p; a[5] += u; a[6] += v; a[7] += 1.0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
        if (lane == 0)
            for (int i = 0; i < 8; ++i) red[w][i] = a[i];
        __syncthreads();
        if (threadIdx.x < 8) {
            double sum = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) sum += red[k][threadIdx.x];
            part[((size_t)blockIdx.x * PROBE_MAX + t) * 8 + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

// Sum the per-block parts in block order and form (p, u, v, count) per probe: the Shepard
// average, the plain mean when every weight is zero, zeros without fluid.
__global__ void k_probe_final(ProbePts q, const double *part, int nblk, double *out)
{
    const int t = threadIdx.x;
    if (t >= q.n) return;
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nblk; ++b)
        for (int i = 0; i < 8; ++i) a[i] += part[((size_t)b * PROBE_MAX + t) * 8 + i];
    double *o = out + 4 * t;
    if (a[7] == 0.0) {
        o[0] = o[1] = o[2] = 0.0;
    } else if (a[0] > 0.0) {
        o[0] = a[1] / a[0]; o[1] = a[2] / a[0]; o[2] = a[3] / a[0];
    } else {
        o[0] = a[4] / a[7]; o[1] = a[5] / a[7]; o[2] = a[6] / a[7];
    }
    o[3] = a[7];
}

}  // namespace

int launch_probe(const Dev &d, cudaStream_t s, const ProbePts &q)
{
    k_probe_part<<<PROBE_BLK, 256, 0, s>>>(d, q, d.probe_part);
    k_probe_final<<<1, 32, 0, s>>>(q, d.probe_part, PROBE_BLK, d.probe_out);
    return 2;
}

}  // namespace edac

namespace edac {
namespace {
__global__ void k_origins(Dev d)
{
    const Geo &g = d.g;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.nx + g.ny; i += gridDim.x * blockDim.x) {
        if (i < g.nx) d.org_x[i] = g.x_min + (double)i * g.sx;
        else d.org_y[i - g.nx] = g.y_min + (double)(i - g.nx) * g.sy;
    }
}
}  // namespace

int launch_origins(const Dev &d, cudaStream_t s)
{
    k_origins<<<(d.g.nx + d.g.ny + 255) / 256, 256, 0, s>>>(d);
    return 1;
}

namespace {
// Free-slot stack after an upload of n particles into slots 0..n-1: slots cap-1 down to n.
__global__ void k_free_stack(Dev d, int n)
{
    const int m = d.cap - n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        d.free_stack[i] = d.cap - 1 - i;
}

// out[r] = src[live[r]] for the read-back in id order; kind 0: src is double, 1: int,
// 2: byte, 3: float (integer, byte and float fields are widened to double).
__global__ void k_permute(const void *src, int kind, const int *live, int n, double *out)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int s = live[r];
        out[r] = kind == 0 ? static_cast<const double *>(src)[s]
                 : kind == 1 ? (double)static_cast<const int *>(src)[s]
                 : kind == 2 ? (double)static_cast<const uint8_t *>(src)[s]
                             : (double)static_cast<const float *>(src)[s];
    }
}

__global__ void k_permute_id_tag(Dev d, const int *live, int n, unsigned long long *id,
                                 uint8_t *tag)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int s = live[r];
        id[r] = d.id[s];
        tag[r] = d.tag[s];
    }
}
}  // namespace

int launch_free_stack(const Dev &d, cudaStream_t s, int n)
{
    k_free_stack<<<grid_for(d.cap - n > 0 ? d.cap - n : 1), TPB, 0, s>>>(d, n);
    return 1;
}

int launch_permute(cudaStream_t s, const void *src, int kind, const int *live, int n, double *out)
{
    k_permute<<<grid_for(n > 0 ? n : 1), TPB, 0, s>>>(src, kind, live, n, out);
    return 1;
}

int launch_permute_id_tag(const Dev &d, cudaStream_t s, const int *live, int n,
                          unsigned long long *id, uint8_t *tag)
{
    k_permute_id_tag<<<grid_for(n > 0 ? n : 1), TPB, 0, s>>>(d, live, n, id, tag);
    return 1;
}
}  // namespace edac
