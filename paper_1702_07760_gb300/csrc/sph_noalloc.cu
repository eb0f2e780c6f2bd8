// Allocation-free cell sort: the cell hash and the stable counting sort by
// (cell id, particle id) of the cell-list build, for callers that must not
// allocate device memory -- a host application whose device memory belongs to
// its own pool or allocator, or a deployment whose device memory is fixed in
// advance.  Its scratch memory is a file-scope device array of fixed size
// instead of the per-simulation buffers that sph_create allocates.  The call
// ends by copying a one-word out-of-box flag to the host and waiting for the
// stream.
#include "sph.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

namespace {

// Limits of the allocation-free entry point (see sph.h).
constexpr int NA_MAX_PARTICLES = 1 << 20;
constexpr int NA_MAX_CELLS = 1 << 20;
constexpr int NA_SCAN_THREADS = 1024, NA_SCAN_ITEMS = 4, NA_SCAN_TILE = NA_SCAN_THREADS * NA_SCAN_ITEMS;
constexpr int NA_MAX_TILES = (NA_MAX_CELLS + NA_SCAN_TILE - 1) / NA_SCAN_TILE;
// int words: count[cells], cstart[cells + 1], cell_tmp[n], slot[n], tmp[n],
// tile sums, then the out-of-box flag
constexpr size_t NA_OFF_COUNT = 0;
constexpr size_t NA_OFF_CSTART = NA_OFF_COUNT + NA_MAX_CELLS;
constexpr size_t NA_OFF_CELL = NA_OFF_CSTART + NA_MAX_CELLS + 64;
constexpr size_t NA_OFF_SLOT = NA_OFF_CELL + NA_MAX_PARTICLES;
constexpr size_t NA_OFF_TMP = NA_OFF_SLOT + NA_MAX_PARTICLES;
constexpr size_t NA_OFF_TILES = NA_OFF_TMP + NA_MAX_PARTICLES;
constexpr size_t NA_OFF_FLAGS = NA_OFF_TILES + NA_MAX_TILES + 64;
constexpr size_t NA_WORDS = NA_OFF_FLAGS + 64;

// Scratch of every call on this device (about 21 MB, held until the process
// exits).  Host code must not use this name as an address: it is resolved to
// a device address once per device by scratch_for_current_device().
static __device__ __align__(256) int g_noalloc_scratch[NA_WORDS];

}  // namespace

namespace sphgb {
int set_error(int code, const std::string &msg);  // message for sph_last_error()
}

namespace {

int na_fail(int code, const std::string &m) { return sphgb::set_error(code, m); }

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
int *g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up with
// that device current the first time it is needed and cached per device
// index (a device reset would invalidate the cached address).
int scratch_for_current_device(int **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(SPH_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(SPH_EINVAL, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return na_fail(SPH_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<int *>(p);
    }
    *out = g_na_ptr[dev];
    return SPH_OK;
}

struct NaGrid {
    int dim, nx, ny, nz;
    double lo[3];
    double cs;
};

__global__ void k_na_zero(int *a, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = 0;
}

// Cell id of every particle (x row-major, n * dim doubles), written to the
// caller's array and to the scratch copy, plus its arrival slot in the cell.
__global__ void k_na_hash(int n, NaGrid g, const double *__restrict__ x, int *cell_out, int *cell_tmp, int *slot,
                          int *count, int *outside)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int dims[3] = {g.nx, g.ny, g.nz};
    int c[3] = {0, 0, 0};
    int bad = 0;
    for (int a = 0; a < g.dim; ++a) {
        const double s = floor((x[(size_t)k * g.dim + a] - g.lo[a]) / g.cs);
        if (!(s >= 0.0 && s < (double)dims[a])) bad = 1;
        else c[a] = (int)s;
    }
    if (bad) atomicOr(outside, 1);
    const int id = c[0] + g.nx * (c[1] + g.ny * c[2]);
    cell_out[k] = id;
    cell_tmp[k] = id;
    slot[k] = atomicAdd(count + id, 1);
}

// Exclusive scan of one value per thread over a block of NA_SCAN_THREADS.
__device__ int na_block_scan(int v, int *total)
{
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int w = warp_tot[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const int res = warp_tot[wid] + inc - v;
    __syncthreads();
    return res;
}

// cstart = exclusive scan of count (m cells), tile by tile; tiles[] gets the
// tile totals.
__global__ void __launch_bounds__(NA_SCAN_THREADS) k_na_scan_tiles(const int *count, int *cstart, int *tiles, int m)
{
    __shared__ int tot;
    const int base = blockIdx.x * NA_SCAN_TILE + threadIdx.x * NA_SCAN_ITEMS;
    int v[NA_SCAN_ITEMS], sum = 0;
    for (int k = 0; k < NA_SCAN_ITEMS; ++k) {
        v[k] = base + k < m ? count[base + k] : 0;
        sum += v[k];
    }
    int ex = na_block_scan(sum, &tot);
    for (int k = 0; k < NA_SCAN_ITEMS; ++k) {
        if (base + k < m) cstart[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

// Scans the tile totals in place (one block, ntiles <= NA_SCAN_THREADS);
// cstart[m] = n.
__global__ void __launch_bounds__(NA_SCAN_THREADS) k_na_scan_tile_sums(int *cstart, int *tiles, int ntiles, int m)
{
    __shared__ int tot;
    const int t = threadIdx.x < ntiles ? tiles[threadIdx.x] : 0;
    const int ex = na_block_scan(t, &tot);
    if (threadIdx.x < ntiles) tiles[threadIdx.x] = ex;
    if (threadIdx.x == 0) cstart[m] = tot;
}

__global__ void k_na_scan_add(int *cstart, const int *tiles, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) cstart[i] += tiles[i / NA_SCAN_TILE];
}

__global__ void k_na_scatter(int n, const int *cell_tmp, const int *slot, const int *cstart, int *tmp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) tmp[cstart[cell_tmp[k]] + slot[k]] = k;
}

// Position of each particle in the sorted order: its rank by particle id (its
// index) among the particles of its cell.
__global__ void k_na_rank(int n, const int *tmp, const int *cell_tmp, const int *cstart, int *order_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int k = tmp[p];
    const int c = cell_tmp[k];
    const int b = cstart[c], e = cstart[c + 1];
    int rank = 0;
    for (int q = b; q < e; ++q) rank += tmp[q] < k;
    order_out[b + rank] = k;
}

}  // namespace

extern "C" {

int sph_cell_sort_noalloc(const sph_params *P, int64_t n, const double *x_dev, int32_t *cell_dev,
                          int32_t *order_dev, void *stream)
{
    if (!P) return na_fail(SPH_EINVAL, "params is NULL");
    if (P->dim != 2 && P->dim != 3) return na_fail(SPH_EINVAL, "dim must be 2 or 3");
    if (P->periodic != 0) return na_fail(SPH_EINVAL, "the allocation-free sort has no periodic axes");
    if (n < 0 || n > NA_MAX_PARTICLES)
        return na_fail(SPH_EINVAL, "n exceeds the allocation-free limit of 2^20 particles");
    if (!(P->cell_size > 0) || !std::isfinite(P->cell_size)) return na_fail(SPH_EINVAL, "cell_size must be positive");
    NaGrid g{};
    g.dim = P->dim;
    g.cs = P->cell_size;
    int dims[3] = {1, 1, 1};
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) g.lo[a] = a < P->dim ? P->box_lo[a] : 0.0;
    for (int a = 0; a < P->dim; ++a) {
        if (!(P->box_hi[a] > P->box_lo[a])) return na_fail(SPH_EINVAL, "box_hi must exceed box_lo");
        const double m = std::floor((P->box_hi[a] - P->box_lo[a]) / P->cell_size) + 1.0;
        if (m > (double)NA_MAX_CELLS) return na_fail(SPH_EINVAL, "cell grid exceeds the allocation-free limit of 2^20 cells");
        dims[a] = (int)m;
        ncell *= dims[a];
    }
    if (ncell > NA_MAX_CELLS) return na_fail(SPH_EINVAL, "cell grid exceeds the allocation-free limit of 2^20 cells");
    if (n == 0) return SPH_OK;
    if (!x_dev || !cell_dev || !order_dev) return na_fail(SPH_EINVAL, "a device array is NULL");
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];

    int *base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    int *count = base + NA_OFF_COUNT, *cstart = base + NA_OFF_CSTART, *cell_tmp = base + NA_OFF_CELL;
    int *slot = base + NA_OFF_SLOT, *tmp = base + NA_OFF_TMP, *tiles = base + NA_OFF_TILES;
    int *outside_flag = base + NA_OFF_FLAGS;
    cudaStream_t st = (cudaStream_t)stream;
    const int nc = (int)ncell, ni = (int)n;
    const int ntiles = (nc + NA_SCAN_TILE - 1) / NA_SCAN_TILE;
    auto nb = [](int w) { return (w + 255) / 256; };

    // the array keeps the previous call's contents: clear what starts at zero
    cudaError_t e = cudaMemsetAsync(outside_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return na_fail(SPH_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_na_zero<<<nb(nc), 256, 0, st>>>(count, nc);
    k_na_hash<<<nb(ni), 256, 0, st>>>(ni, g, x_dev, cell_dev, cell_tmp, slot, count, outside_flag);
    k_na_scan_tiles<<<ntiles, NA_SCAN_THREADS, 0, st>>>(count, cstart, tiles, nc);
    k_na_scan_tile_sums<<<1, NA_SCAN_THREADS, 0, st>>>(cstart, tiles, ntiles, nc);
    k_na_scan_add<<<nb(nc), 256, 0, st>>>(cstart, tiles, nc);
    k_na_scatter<<<nb(ni), 256, 0, st>>>(ni, cell_tmp, slot, cstart, tmp);
    k_na_rank<<<nb(ni), 256, 0, st>>>(ni, tmp, cell_tmp, cstart, order_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(SPH_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    int outside = 0;
    e = cudaMemcpyAsync(&outside, outside_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return na_fail(SPH_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    if (outside) return na_fail(SPH_EDOMAIN, "a particle lies outside the box covered by the cell grid");
    return SPH_OK;
}

}  // extern "C"
