// edac_density_static: the summation density, number-density volume and neighbour count
// of a particle set, with every byte of scratch in a file-scope device array instead of
// memory the library or the caller allocates.
//
// It exists for callers that cannot allocate device memory when they need the result: a
// caller whose framework hands all device memory to its own pool allocator (a raw
// allocation would fail or fragment it), a plug-in hosted by an application that owns the
// device memory and gives it none, and real-time callers that forbid allocation on the hot
// path (cudaMalloc and cudaFree can block and synchronise the device).  The caller still
// owns and passes the input and output arrays.
//
// Scratch: one static __device__ array (EDAC_STATIC_MAX_PARTICLES particles and
// EDAC_STATIC_MAX_CELLS cells, 3.7 MB) that every GPU which loads the library holds until
// the process exits.  Host code cannot use the array's name as a device address, so the
// first call on each device (with that device current) looks the address up with
// cudaGetSymbolAddress and caches it; that first call should come before any stream
// capture.  All calls share the array: calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race.  The per-cell counters are
// cleared by every call.
#include <mutex>

#include "edac.h"
#include "edac_internal.cuh"

using namespace edac;

namespace {

constexpr int SMAX_N = EDAC_STATIC_MAX_PARTICLES;
constexpr int SMAX_C = EDAC_STATIC_MAX_CELLS;
constexpr int MAX_DEVICES = 64;

// [cell_count SMAX_C | cell_start SMAX_C + 1 | flag 1 | cell_of SMAX_N | within SMAX_N | order SMAX_N]
constexpr size_t SCRATCH_INTS = 2 * (size_t)SMAX_C + 2 + 3 * (size_t)SMAX_N;
static __device__ __align__(256) int g_scratch[SCRATCH_INTS];

std::mutex g_mutex;
int *g_ptr[MAX_DEVICES] = {};

struct StaticGrid {
    Geo g;
    double a2, inv_h;
    int n;
    int *count, *start, *flag, *cell_of, *within, *order;
};

__global__ void k_st_clear(StaticGrid s)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < s.g.ncells; c += gridDim.x * blockDim.x)
        s.count[c] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.flag = 0;
}

__global__ void k_st_count(StaticGrid s, const double *x, const double *y)
{
    const Geo &g = s.g;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const double xi = x[i], yi = y[i];
        if (!(xi >= g.x_min && xi < g.x_max && yi >= g.y_min && yi < g.y_max)) atomicOr(s.flag, 1);
        const int c = cell_coord(yi, g.y_min, g.inv_sy, g.ny) * g.nx + cell_coord(xi, g.x_min, g.inv_sx, g.nx);
        s.cell_of[i] = c;
        s.within[i] = atomicAdd(s.count + c, 1);
    }
}

// one block: exclusive scan of the counts, each thread a contiguous chunk
__global__ void __launch_bounds__(1024) k_st_scan(StaticGrid s)
{
    __shared__ int tot[1024];
    const int n = s.g.ncells, t = threadIdx.x;
    const int chunk = (n + 1023) / 1024, b = t * chunk, e = min(n, b + chunk);
    int local = 0;
    for (int c = b; c < e; ++c) local += s.count[c];
    tot[t] = local;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? tot[t - o] : 0;
        __syncthreads();
        tot[t] += v;
        __syncthreads();
    }
    int run = tot[t] - local;
    for (int c = b; c < e; ++c) {
        s.start[c] = run;
        run += s.count[c];
    }
    if (t == 1023) s.start[n] = tot[1023];
}

__global__ void k_st_scatter(StaticGrid s)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x)
        s.order[s.start[s.cell_of[i]] + s.within[i]] = i;
}

// fp64 summation density (Eq. summation-density with the quintic spline), V = 1/sum W and the
// neighbour count (self included), with the library's exact membership test
__global__ void k_st_density(StaticGrid s, const double *x, const double *y, const double *m,
                             double *rho, double *vol, int *nnb)
{
    const Geo &g = s.g;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x) {
        const double xi = x[i], yi = y[i];
        const int c = s.cell_of[i];
        const int cx = c % g.nx, cy = c / g.nx;
        double sw = 0.0, sr = 0.0;
        int cnt = 0;
        for (int oy = -1; oy <= 1; ++oy) {
            int by = cy + oy;
            if (g.py) by = by < 0 ? by + g.ny : (by >= g.ny ? by - g.ny : by);
            else if (by < 0 || by >= g.ny) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                int bx = cx + ox;
                if (g.px) bx = bx < 0 ? bx + g.nx : (bx >= g.nx ? bx - g.nx : bx);
                else if (bx < 0 || bx >= g.nx) continue;
                const int cc = by * g.nx + bx;
                for (int q = s.start[cc]; q < s.start[cc + 1]; ++q) {
                    const int j = s.order[q];
                    double dx, dy;
                    const double r2 = exact_r2(g, xi, yi, x[j], y[j], dx, dy);
                    if (!(r2 < g.rc2)) continue;
                    const double w = s.a2 * quintic_w(sqrt(r2) * s.inv_h);
                    sw += w;
                    sr += m[j] * w;
                    ++cnt;
                }
            }
        }
        rho[i] = sr;
        vol[i] = 1.0 / sw;
        nnb[i] = cnt;
    }
}

}  // namespace

extern "C" edac_status edac_density_static(const edac_params *p, int n, const double *d_x,
                                           const double *d_y, const double *d_m, double *d_rho,
                                           double *d_vol, int *d_nnb)
{
    if (!p || n < 0 || n > SMAX_N) return EDAC_E_INVALID;
    if (n > 0 && (!d_x || !d_y || !d_m || !d_rho || !d_vol || !d_nnb)) return EDAC_E_INVALID;
    if (!(p->dx > 0 && p->hdx > 0 && p->x_max > p->x_min && p->y_max > p->y_min)) return EDAC_E_INVALID;
    if (n == 0) return EDAC_OK;
    StaticGrid s;
    Geo &g = s.g;
    const double h = p->hdx * p->dx;
    const double rc = 3.0 * (p->hdx * p->dx);
    g.x_min = p->x_min; g.x_max = p->x_max; g.y_min = p->y_min; g.y_max = p->y_max;
    g.Lx = p->x_max - p->x_min;
    g.Ly = p->y_max - p->y_min;
    g.hLx = 0.5 * g.Lx;
    g.hLy = 0.5 * g.Ly;
    g.px = p->periodic_x ? 1 : 0;
    g.py = p->periodic_y ? 1 : 0;
    const double s_min = rc * (1.0 + 1e-9);  // cells a little wider than 3h, as the library's
    double nxd = floor(g.Lx / s_min), nyd = floor(g.Ly / s_min);
    if (nxd < 1) nxd = 1;
    if (nyd < 1) nyd = 1;
    if (nxd * nyd > (double)SMAX_C) return EDAC_E_CAPACITY;  // beyond the static cell table
    g.nx = (int)nxd;
    g.ny = (int)nyd;
    if ((g.px && g.nx < 3) || (g.py && g.ny < 3)) return EDAC_E_INVALID;
    g.ncells = g.nx * g.ny;
    g.sx = g.Lx / g.nx;
    g.sy = g.Ly / g.ny;
    g.inv_sx = 1.0 / g.sx;
    g.inv_sy = 1.0 / g.sy;
    g.rc2 = rc * rc;
    s.a2 = 7.0 / (478.0 * M_PI * h * h);
    s.inv_h = 1.0 / h;
    s.n = n;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return EDAC_E_CUDA;
    int *base;
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        if (!g_ptr[dev]) {
            int *ptr = nullptr;
            if (cudaGetSymbolAddress((void **)&ptr, g_scratch) != cudaSuccess || !ptr) return EDAC_E_CUDA;
            g_ptr[dev] = ptr;
        }
        base = g_ptr[dev];
    }
    s.count = base;
    s.start = base + SMAX_C;
    s.flag = s.start + SMAX_C + 1;
    s.cell_of = s.flag + 1;
    s.within = s.cell_of + SMAX_N;
    s.order = s.within + SMAX_N;
    cudaStream_t st = (cudaStream_t)p->cuda_stream;
    const int blocks = (n + 255) / 256;
    k_st_clear<<<(g.ncells + 255) / 256, 256, 0, st>>>(s);
    k_st_count<<<blocks, 256, 0, st>>>(s, d_x, d_y);
    k_st_scan<<<1, 1024, 0, st>>>(s);
    k_st_scatter<<<blocks, 256, 0, st>>>(s);
    k_st_density<<<blocks, 256, 0, st>>>(s, d_x, d_y, d_m, d_rho, d_vol, d_nnb);
    int flag = 0;
    if (cudaMemcpyAsync(&flag, s.flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return EDAC_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return EDAC_E_CUDA;
    if (cudaGetLastError() != cudaSuccess) return EDAC_E_CUDA;
    return flag ? EDAC_E_DOMAIN : EDAC_OK;
}
