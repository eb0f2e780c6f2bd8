// Device kernels of the two-phase WCSPH particle loop (sm_103a).
//
// Method: Wei et al., "Behavior of Oil under Breaking Waves by a Two-phase SPH
// Model", Sec. II.  Layout and arithmetic choices made for the GPU:
//   * particles live in cell order (stable by original id), structure of
//     arrays;
//   * a position used by the interaction sweeps is the particle's cell (an
//     integer index of the cell grid) plus an FP32 offset from the centre of
//     its super-cell (a block of f x f x f cells whose edge E = f * cell edge
//     is at least the list radius); a pair vector is
//     (o_i - o_j) + (S_i - S_j) * E, the super-cell difference (-1, 0 or 1
//     per axis) being packed into the pair's neighbour-list entry;
//   * the FP64 position and velocity are the integration accumulators;
//   * density is stored as the deviation drho = rho - rho0(phase) in FP32, so
//     the equation of state and the renormalisation never subtract two
//     numbers near rho0;
//   * once per step a neighbour list (radius 2h + 2 skin) is built from the
//     cell list, scanning per particle only the cells of the +/-f stencil that
//     the radius can reach, and stored column-major, so the four
//     interaction sweeps of the step read it coalesced and run without the
//     branch divergence of a candidate scan; a sweep gathers two 16-byte
//     records per neighbour.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sphgb {

enum : unsigned {
    FLAG_DOMAIN = 1u,     // a particle left the cell grid
    FLAG_NONFINITE = 2u,  // NaN/Inf in the state
    FLAG_SKIN = 4u,       // predictor displacement beyond the skin
    FLAG_LIST = 8u,       // a particle has more list neighbours than max_neighbours
};

// Constants of the physics, FP32 unless they feed an FP64 accumulator.
struct Phys {
    float inv_h;        // 1/h
    float R2;           // (2h)^2, support test
    float RL2;          // list radius^2, (2h + 2 skin)^2
    float RP;           // list radius widened by 1e-4 (conservative stencil pruning)
    float cF;           // -5 alpha_d / h^2: grad W_ij = cF (1-q/2)^3 r_ij
    float mass[2];      // per-phase particle mass
    float inv_mass[2];
    float rho0[2];      // per-phase reference density
    float inv_rho0[2];
    float beta[2];      // rho0 c0^2 / gamma
    float kvis[4];      // [2*ph_i + ph_j]: 2 mu_ij (dynamic form) or 2 nu_ij (kinematic form)
    float delta2;       // delta^2
    float alpha_s;      // surface tension coefficient
    float inv_dim;      // 1/d in Eq. csf
    float gf[3];        // gravity (FP32, added to the FP32 acceleration)
    int visc_dynamic;   // 1: Eq. visc_2 (factor 1/rho_i), 0: Eq. visc_1
    int renorm_every;   // Eq. ct_dist_3 at stage 1 of steps with step % renorm_every == 0
    int kmax;           // neighbour-list capacity per particle
    int rebuild_every;  // 0: rebuild when a particle may leave the skin; k: every k steps
    double skin;        // allowed displacement since the last build (the list's margin)
};

struct Grid {
    int nx, ny, nz;     // cells per axis (nz = 1 in 2-D)
    int f;              // cells per super-cell edge: 1 or 2 (also the stencil half-width)
    float cs;           // cell edge (FP32)
    float Es;           // super-cell edge (FP32): pair vectors
    double csd;         // cell edge (FP64): hashing
    double Ed;          // super-cell edge (FP64): offsets
    double lo[3];       // box lower corner
};

// All device arrays of one simulation (sorted order unless noted).
struct Dev {
    int n;
    // state (FP64 accumulators + FP32 density deviation)
    double *x;          // dim * n, SoA
    double *u;          // dim * n, SoA
    float *drho;        // n, rho - rho0(phase) of the state
    int *pid;           // n, original particle id
    uint8_t *tag;       // n, bit0 oil, bit1 wall
    int *cell;          // n, cell id (sorted order)
    // stage arrays
    float4 *pos;        // n, (offset from the super-cell centre xyz, +/- m/rho of the stage input; sign = phase)
    float4 *pos0;       // n, offset at the last list build (xyz): displacement since the build
    float *vd;          // n, (m/rho) * drho of the stage input
    float4 *posv;       // n, (offset xyz, +/- m/rho after renormalisation with its lowest
                        //     mantissa bit replaced by the interface flag): sweep A output
    float4 *velp;       // n, stage 1: (u^n xyz, P/rho^2 from sweep A)
    float4 *velq;       // n, stage 2: (u* xyz, P/rho^2 from sweep A); a separate buffer so
                        //     the stage-1 force sweep can write it while neighbours read velp
    float *pres;        // n, P from sweep A
    float *drho_stage;  // n, drho* of the predictor
    float *drho_eval;   // n, drho after renormalisation (stage output)
    float4 *T4;         // n, T sigma^-2 = T (m/rho)^2: 2-D (xx, xy, yy, 0); 3-D (xx, xy, xz, yy)
    float2 *T2;         // n, 3-D only: (yz, zz)
    float4 *acc;        // n, (a xyz, Drho/Dt)
    // neighbour list
    unsigned *nbr;      // kmax * n, entry k of particle i at nbr[k * n + i]
    int *ncnt;          // n, list length
    uint8_t *nflag;     // n, bit0: an other-phase particle lies within the list radius
    // cell list
    int *cstart;        // ncell + 1
    unsigned *flags;    // 1 word
    unsigned *rebuild;  // 1 word: nonzero when the cell and neighbour lists must be rebuilt
    long long *step;    // device step counter (drives the renormalisation schedule)
    long long *builds;  // number of list builds performed
};

// Neighbour-list entries a sweep loads ahead of use (one chunk in flight
// while the previous chunk is processed).
#ifndef SPH_LIST_CHUNK
#define SPH_LIST_CHUNK 4
#endif

// Neighbour-list entry: particle index in the low 26 bits; per axis a, two
// bits at 26 + 2a holding (S_i - S_j) + 1 in {0, 1, 2} (super-cells).
constexpr int NBR_IDX_BITS = 26;
constexpr unsigned NBR_IDX_MASK = (1u << NBR_IDX_BITS) - 1u;

__device__ __forceinline__ int phase_of(float w) { return __float_as_uint(w) >> 31; }

// Per-phase constant without indexing the parameter block at run time (an
// indexed parameter load would go through the constant cache per thread).
__device__ __forceinline__ float by_phase(int phase, const float (&a)[2]) { return phase ? a[1] : a[0]; }

// (S_i - S_j) * E for axis a of an entry, exact: the code e in {0, 1, 2}
// becomes the float e - 1 through the 2^23 + 2^22 mantissa trick.
__device__ __forceinline__ float entry_shift(unsigned e, int a, float E)
{
    const unsigned code = (e >> (NBR_IDX_BITS + 2 * a)) & 3u;
    return (__uint_as_float(0x4B400000u | code) - 12582913.f) * E;
}

// r_ij = x_i - x_j from super-cell offsets and the centre difference (s).
template <int DIM>
__device__ __forceinline__ float pair_vec(const float4 &oi, const float4 &oj, float sx, float sy, float sz,
                                          float &rx, float &ry, float &rz)
{
    rx = (oi.x - oj.x) + sx;
    ry = (oi.y - oj.y) + sy;
    rz = DIM == 3 ? (oi.z - oj.z) + sz : 0.f;
    float r2 = rx * rx;
    r2 = fmaf(ry, ry, r2);
    if (DIM == 3) r2 = fmaf(rz, rz, r2);
    return r2;
}

__device__ __forceinline__ void cell_coords(const Grid &g, int c, int &cx, int &cy, int &cz)
{
    cx = c % g.nx;
    const int r = c / g.nx;
    cy = r % g.ny;
    cz = r / g.ny;
}

// Gap along one axis between a particle at p (from its cell's lower corner)
// and the cell d cells away: 0 for d = 0.
__device__ __forceinline__ float axis_gap(float p, int d, float e)
{
    return d > 0 ? (float)d * e - p : (d < 0 ? p - (float)(d + 1) * e : 0.f);
}

// Scans the particles of the cells within +/-f of cell c that a sphere of
// radius Rp around the particle can reach (pruned per row), and calls
// f(j, oj, rx, ry, rz, r2, code) for those with |r_ij|^2 < R2 (j == i
// included); code is the shift part of a neighbour-list entry.
template <int DIM, class F>
__device__ __forceinline__ void for_each_candidate(const Grid &g, const int *__restrict__ cstart,
                                                   const float4 *__restrict__ pos, int c, const float4 &oi,
                                                   float R2, float Rp, F &&fn)
{
    int cx, cy, cz;
    cell_coords(g, c, cx, cy, cz);
    const int fm = g.f - 1, hw = g.f;
    const int Sx = cx >> fm, Sy = cy >> fm, Sz = cz >> fm;
    const float e = g.cs, E = g.Es;
    // position inside the cell from its lower corner: the super-cell centre
    // lies e/2 above the corner for f = 1, and e above (even cell) or at the
    // corner (odd cell) for f = 2
    const float px = oi.x + (hw == 1 ? 0.5f * e : ((cx & 1) ? 0.f : e));
    const float py = oi.y + (hw == 1 ? 0.5f * e : ((cy & 1) ? 0.f : e));
    const float pz = DIM == 3 ? oi.z + (hw == 1 ? 0.5f * e : ((cz & 1) ? 0.f : e)) : 0.f;
    const float Rp2 = Rp * Rp;
    const int z0 = DIM == 3 ? max(cz - hw, 0) : 0, z1 = DIM == 3 ? min(cz + hw, g.nz - 1) : 0;
    const int y0 = max(cy - hw, 0), y1 = min(cy + hw, g.ny - 1);
    for (int z = z0; z <= z1; ++z) {
        const float gz = DIM == 3 ? axis_gap(pz, z - cz, e) : 0.f;
        if (gz >= Rp) continue;
        const int dSz = DIM == 3 ? Sz - (z >> fm) : 0;
        const float sz = (float)dSz * E;
        for (int y = y0; y <= y1; ++y) {
            const float gy = axis_gap(py, y - cy, e);
            const float rem = Rp2 - gy * gy - gz * gz;
            if (rem <= 0.f) continue;
            const int dSy = Sy - (y >> fm);
            const float sy = (float)dSy * E;
            const float xr = sqrtf(rem);
            const int xlo = max(max(cx + (int)floorf((px - xr) / e), cx - hw), 0);
            const int xhi = min(min(cx + (int)floorf((px + xr) / e), cx + hw), g.nx - 1);
            if (xlo > xhi) continue;
            // the cells xlo..xhi of a row are contiguous in the sorted order
            const int row = (z * g.ny + y) * g.nx;
            const int jb = __ldg(cstart + row + xlo), je = __ldg(cstart + row + xhi + 1);
            // super-cell Sx covers cells [Sx*f, Sx*f + f)
            const int b1 = __ldg(cstart + row + min(max(Sx * hw, xlo), xhi + 1));
            const int b2 = __ldg(cstart + row + min(max(Sx * hw + hw, xlo), xhi + 1));
            const unsigned cyz = ((unsigned)(dSy + 1) << (NBR_IDX_BITS + 2)) |
                                 ((unsigned)(dSz + 1) << (NBR_IDX_BITS + 4));
#pragma unroll 4
            for (int j = jb; j < je; ++j) {
                const float4 oj = __ldg(pos + j);
                // super-cell of j along x: Sx - 1, Sx or Sx + 1
                const float sx = j < b1 ? E : (j < b2 ? 0.f : -E);
                const unsigned ex = j < b1 ? 2u : (j < b2 ? 1u : 0u);
                float rx, ry, rz;
                const float r2 = pair_vec<DIM>(oi, oj, sx, sy, sz, rx, ry, rz);
                if (r2 < R2) fn(j, oj, rx, ry, rz, r2, cyz | (ex << NBR_IDX_BITS));
            }
        }
    }
}

// Compensated (Kahan) accumulation.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Eq. state with gamma = 7 written in the density deviation eps = drho/rho0:
// P = beta ((1 + eps)^7 - 1) = beta eps (7 + 21 eps + 35 eps^2 + 35 eps^3
// + 21 eps^4 + 7 eps^5 + eps^6), free of the cancellation of the power form.
__device__ __forceinline__ float eos_tait7(float beta, float eps)
{
    float p = eps + 7.f;
    p = fmaf(p, eps, 21.f);
    p = fmaf(p, eps, 35.f);
    p = fmaf(p, eps, 35.f);
    p = fmaf(p, eps, 21.f);
    p = fmaf(p, eps, 7.f);
    return beta * eps * p;
}

// FP32 offset of an FP64 position from the centre of the super-cell of cell c.
template <int DIM>
__device__ __forceinline__ float4 cell_offset(const Grid &g, int c, const double xa[3])
{
    int cc[3];
    cell_coords(g, c, cc[0], cc[1], cc[2]);
    const int fm = g.f - 1;
    float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < DIM; ++a) o[a] = (float)(xa[a] - (g.lo[a] + ((double)(cc[a] >> fm) + 0.5) * g.Ed));
    return make_float4(o[0], o[1], o[2], 0.f);
}

// Signed specific volume m/rho, negative for oil.
__device__ __forceinline__ float signed_volume(const Phys &ph, int phase, float drho, float &vol)
{
    vol = by_phase(phase, ph.mass) / (by_phase(phase, ph.rho0) + drho);
    return phase ? -vol : vol;
}

// ---------------------------------------------------------------------------
// Cell list: hash, counting sort stable in particle id, reorder.

template <int DIM>
__global__ void __launch_bounds__(256) k_hash(Dev d, Grid g, int *cell_tmp, int *slot, int *count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n || !*d.rebuild) return;
    const int dims[3] = {g.nx, g.ny, g.nz};
    int c[3] = {0, 0, 0};
    unsigned bad = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double xa = d.x[(size_t)a * d.n + k];
        const double s = floor((xa - g.lo[a]) / g.csd);
        if (isnan(xa)) {
            bad |= FLAG_NONFINITE;
        } else if (!(s >= 0.0 && s < (double)dims[a])) {
            bad |= FLAG_DOMAIN;
        } else {
            c[a] = (int)s;
        }
    }
    if (bad) atomicOr(d.flags, bad);
    const int id = c[0] + g.nx * (c[1] + g.ny * c[2]);
    cell_tmp[k] = id;
    slot[k] = atomicAdd(count + id, 1);
}

// Exclusive scan of m ints, 4096 per block (1024 threads x 4).
constexpr int SCAN_THREADS = 1024, SCAN_ITEMS = 4, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; the block total is
// written to *total (shared memory).
__device__ __forceinline__ int block_exclusive_scan(int v, int *total)
{
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < nw ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;
        if (lane == nw - 1) *total = wi;
    }
    __syncthreads();
    const int res = warp_tot[wid] + inc - v;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const int *in, int *out, int *tile_sums, int m,
                                                              const unsigned *rebuild)
{
    __shared__ int s_total;
    if (!*rebuild) return;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < m ? in[base + k] : 0;
        sum += v[k];
    }
    int ex = block_exclusive_scan(sum, &s_total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < m) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s_total;
}

// Scans the tile sums in place (one block, at most SCAN_TILE tiles) and
// writes the grand total to out[m].
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(int *tile_sums, int ntiles, int *out, int m,
                                                             const unsigned *rebuild)
{
    __shared__ int s_total;
    if (!*rebuild) return;
    const int base = threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < ntiles ? tile_sums[base + k] : 0;
        sum += v[k];
    }
    int ex = block_exclusive_scan(sum, &s_total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < ntiles) tile_sums[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) out[m] = s_total;
}

__global__ void __launch_bounds__(256) k_scan_add(int *out, const int *tile_sums, int m, const unsigned *rebuild)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && *rebuild) out[i] += tile_sums[i / SCAN_TILE];
}

__global__ void __launch_bounds__(256) k_zero(int *a, int m, const unsigned *rebuild)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && *rebuild) a[i] = 0;
}

__global__ void __launch_bounds__(256) k_scatter(int n, const int *cell_tmp, const int *slot, const int *cstart, int *tmp,
                                                 const unsigned *rebuild)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !*rebuild) return;
    tmp[cstart[cell_tmp[k]] + slot[k]] = k;
}

// Final position of each particle inside its cell: its rank by original id
// among the cell's particles, so the order is (cell id, particle id).
__global__ void __launch_bounds__(256) k_rank(int n, const int *tmp, const int *cell_tmp, const int *pid,
                                              const int *cstart, int *perm, const unsigned *rebuild)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !*rebuild) return;
    const int k = tmp[p];
    const int c = cell_tmp[k];
    const int b = cstart[c], e = cstart[c + 1];
    const int me = pid[k];
    int rank = 0;
    for (int q = b; q < e; ++q) rank += pid[tmp[q]] < me;
    perm[b + rank] = k;
}

// Stage-1 records of particle k from its FP64 state.
template <int DIM>
__device__ __forceinline__ void stage_records(const Dev &d, const Grid &g, const Phys &ph, int k, int c,
                                              const double xa[3], const double ua[3], float dr, int oil)
{
    float4 p = cell_offset<DIM>(g, c, xa);
    float vol;
    p.w = signed_volume(ph, oil, dr, vol);
    d.pos[k] = p;
    d.vd[k] = vol * dr;
    d.velp[k] = make_float4((float)ua[0], (float)ua[1], (float)ua[2], 0.f);
}

// Gathers the state into the new order (into the scratch set `dst`) and
// prepares the stage-1 records and the build offsets.
template <int DIM>
__global__ void __launch_bounds__(256) k_gather(Dev src, Dev dst, Grid g, Phys ph, const int *perm, const int *cell_tmp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = src.n;
    if (k >= n || !*src.rebuild) return;
    const int o = perm[k];
    double xa[3] = {0, 0, 0}, ua[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        xa[a] = src.x[(size_t)a * n + o];
        ua[a] = src.u[(size_t)a * n + o];
        dst.x[(size_t)a * n + k] = xa[a];
        dst.u[(size_t)a * n + k] = ua[a];
    }
    const float dr = src.drho[o];
    const uint8_t tg = src.tag[o];
    const int c = cell_tmp[o];
    dst.drho[k] = dr;
    dst.pid[k] = src.pid[o];
    dst.tag[k] = tg;
    src.cell[k] = c;
    stage_records<DIM>(src, g, ph, k, c, xa, ua, dr, tg & 1);
    src.pos0[k] = src.pos[k];
}

// Copies the gathered state back into the primary set.
template <int DIM>
__global__ void __launch_bounds__(256) k_copy_back(Dev src, Dev dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = src.n;
    if (k >= n || !*dst.rebuild) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        dst.x[(size_t)a * n + k] = src.x[(size_t)a * n + k];
        dst.u[(size_t)a * n + k] = src.u[(size_t)a * n + k];
    }
    dst.drho[k] = src.drho[k];
    dst.pid[k] = src.pid[k];
    dst.tag[k] = src.tag[k];
}

// ---------------------------------------------------------------------------
// Neighbour list: every j != i within the cell edge (2h + 2 skin) at the
// positions of the build, so the list stays complete while no particle moves
// farther than the skin.
template <int DIM>
__global__ void __launch_bounds__(256, 4) k_build_list(Dev d, Grid g, Phys ph)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n || !*d.rebuild) return;
    if (i == 0) *d.builds += 1;
    const float4 oi = d.pos[i];
    const int phi_ = phase_of(oi.w);
    int cnt = 0;
    int other = 0;
    const int n = d.n, kmax = ph.kmax;
    unsigned *__restrict__ nbr = d.nbr;
    for_each_candidate<DIM>(g, d.cstart, d.pos, d.cell[i], oi, ph.RL2, ph.RP,
        [&](int j, const float4 &oj, float, float, float, float, unsigned code) {
            if (j == i) return;
            if (cnt < kmax) nbr[(size_t)cnt * n + i] = (unsigned)j | code;
            ++cnt;
            other |= phase_of(oj.w) != phi_;
        });
    if (cnt > kmax) {
        atomicOr(d.flags, FLAG_LIST);
        cnt = kmax;
    }
    d.ncnt[i] = cnt;
    d.nflag[i] = (uint8_t)other;
}

// ---------------------------------------------------------------------------
// Explicit midpoint predictor-corrector, run per particle at the end of the
// force sweep of each stage (the particle's own acceleration is then final).

// Predictor: x* = x^n + dt/2 u^n, u* = u^n + dt/2 a^n, rho* = rho^n + dt/2 Drho^n;
// the renormalised density becomes the state rho^n.  Writes the stage-2
// records (pos, vd, velq).
template <int DIM>
__device__ __forceinline__ void predict_particle(const Dev &d, const Grid &g, const Phys &ph, int k, float4 a,
                                                 double dt)
{
    const uint8_t tg = d.tag[k];
    const float dr = d.drho_eval[k];
    d.drho[k] = dr;
    const float drs = fmaf(0.5f * (float)dt, a.w, dr);
    d.drho_stage[k] = drs;
    double xs[3] = {0, 0, 0}, us[3] = {0, 0, 0};
    const double af[3] = {a.x, a.y, a.z};
    bool finite = isfinite(drs);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const double x = d.x[(size_t)c * d.n + k], u = d.u[(size_t)c * d.n + k];
        xs[c] = (tg & 2) ? x : x + 0.5 * dt * u;
        us[c] = (tg & 2) ? u : u + 0.5 * dt * af[c];
        finite = finite && isfinite(us[c]) && isfinite(xs[c]);
    }
    float4 p = cell_offset<DIM>(g, d.cell[k], xs);
    // the neighbour list stays complete while no particle is farther than the
    // skin from where it was at the build
    const float4 p0 = d.pos0[k];
    const float ex = p.x - p0.x, ey = p.y - p0.y, ez = p.z - p0.z;
    if (ex * ex + ey * ey + ez * ez > (float)(ph.skin * ph.skin)) atomicOr(d.flags, FLAG_SKIN);
    float vol;
    p.w = signed_volume(ph, tg & 1, drs, vol);
    d.pos[k] = p;
    d.vd[k] = vol * drs;
    d.velq[k] = make_float4((float)us[0], (float)us[1], (float)us[2], 0.f);
    if (!finite) atomicOr(d.flags, FLAG_NONFINITE);
}

// Corrector: x^{n+1} = x^n + dt u*, u^{n+1} = u^n + dt a*, rho^{n+1} = rho^n +
// dt Drho*, in the FP64 accumulators (walls keep x and u).  Writes the
// stage-1 records of the next step and decides whether it rebuilds the lists.
template <int DIM>
__device__ __forceinline__ void correct_particle(const Dev &d, const Grid &g, const Phys &ph, int k, float4 a,
                                                 double dt)
{
    if (k == 0) {
        const long long next = *d.step + 1;
        *d.step = next;
        if (ph.rebuild_every > 0 && next % ph.rebuild_every == 0) *d.rebuild = 1u;
    }
    const uint8_t tg = d.tag[k];
    const float dr = fmaf((float)dt, a.w, d.drho[k]);
    d.drho[k] = dr;
    bool finite = isfinite(dr);
    double xa[3] = {0, 0, 0}, ua[3] = {0, 0, 0};
    const float4 us = d.velq[k];
    const double usa[3] = {us.x, us.y, us.z};
    const double af[3] = {a.x, a.y, a.z};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        xa[c] = d.x[(size_t)c * d.n + k];
        ua[c] = d.u[(size_t)c * d.n + k];
        if (!(tg & 2)) {
            xa[c] += dt * usa[c];
            ua[c] += dt * af[c];
            d.x[(size_t)c * d.n + k] = xa[c];
            d.u[(size_t)c * d.n + k] = ua[c];
        }
        finite = finite && isfinite(xa[c]) && isfinite(ua[c]);
    }
    if (!finite) atomicOr(d.flags, FLAG_NONFINITE);
    // stage-1 records of the next step (replaced by the gather if it rebuilds)
    stage_records<DIM>(d, g, ph, k, d.cell[k], xa, ua, dr, tg & 1);
    if (ph.rebuild_every == 0 && !(tg & 2)) {
        // next step's stage positions: x^{n+1} and x^{n+1} + dt/2 u^{n+1};
        // rebuild before either can be farther than the skin from the build
        const float4 p = d.pos[k], p0 = d.pos0[k];
        const float hx = 0.5f * (float)dt * (float)ua[0], hy = 0.5f * (float)dt * (float)ua[1],
                    hz = 0.5f * (float)dt * (float)ua[2];
        const float ex = p.x - p0.x, ey = p.y - p0.y, ez = p.z - p0.z;
        const float d1 = ex * ex + ey * ey + ez * ez;
        const float d2 = (ex + hx) * (ex + hx) + (ey + hy) * (ey + hy) + (ez + hz) * (ez + hz);
        const float lim = (float)(0.98 * ph.skin);
        if (fmaxf(d1, d2) > lim * lim) atomicOr(d.rebuild, 1u);
    }
}

// ---------------------------------------------------------------------------
// Sweep A: per-phase renormalisation (Eq. ct_dist_3), colour-index gradient
// (Eq. cd) and surface stress tensor (Eq. csf), equation of state (Eq. state).
//
// Eq. ct_dist_3 with same-phase masses m_j = m_i is rewritten exactly as a
// Shepard average of the density deviation:
//   rho_i - rho0 = sum_j (m_j/rho_j) drho_j W_ij / sum_j (m_j/rho_j) W_ij,
// over i itself and its same-phase neighbours, both sums Kahan-compensated.
// The colour gradient uses the density that entered the stage:
// grad C_i = (1/V_i) sum_{j other phase} V_j^2 grad W_ij, V = m/rho = 1/sigma.
template <int DIM>
__global__ void __launch_bounds__(256) k_sweep_a(Dev d, Grid g, Phys ph, const float *__restrict__ drho_in, int stage1,
                                                 float4 *vel_s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int renorm = stage1 && ph.renorm_every > 0 && (*d.step % ph.renorm_every) == 0;
    // the lists built for this step are in place; the corrector decides the next build
    if (stage1 && i == 0) *d.rebuild = 0u;
    const float4 oi = d.pos[i];
    const int phi_ = phase_of(oi.w);
    // self term: W(0)/alpha_d = 1
    float s1 = fabsf(oi.w), c1 = 0.f, s2 = d.vd[i], c2 = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    const bool other = d.nflag[i] & 1;
    if (renorm || other) {
        const float inv_h = ph.inv_h, cs = g.Es;
        const int n = d.n, cnt = d.ncnt[i];
        const unsigned *__restrict__ col = d.nbr + i;
        const float4 *__restrict__ pos = d.pos;
        const float *__restrict__ vd = d.vd;
        constexpr int CH = SPH_LIST_CHUNK;
        unsigned ec[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) ec[c] = c < cnt ? __ldg(col + (size_t)c * n) : 0u;
        for (int k0 = 0; k0 < cnt; k0 += CH) {
            unsigned en[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int kk = k0 + CH + c;
                en[c] = kk < cnt ? __ldg(col + (size_t)kk * n) : 0u;
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (k0 + c >= cnt) break;
                const unsigned e = ec[c];
                const int j = (int)(e & NBR_IDX_MASK);
                const float4 oj = __ldg(pos + j);
                float rx, ry, rz;
                const float r2 = pair_vec<DIM>(oi, oj, entry_shift(e, 0, cs), entry_shift(e, 1, cs),
                                               DIM == 3 ? entry_shift(e, 2, cs) : 0.f, rx, ry, rz);
                // beyond the support (list entries in the skin) t clamps to 0 and
                // every kernel term vanishes
                const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
                const float t = fmaxf(fmaf(-0.5f * inv_h, r, 1.f), 0.f);
                const float t3 = t * t * t;
                if (phase_of(oj.w) == phi_) {
                    if (renorm) {
                        // W / alpha_d = t^4 (2q + 1)
                        const float w = t3 * t * fmaf(2.f * inv_h, r, 1.f);
                        kahan_add(s1, c1, fabsf(oj.w) * w);
                        kahan_add(s2, c2, __ldg(vd + j) * w);
                    }
                } else {
                    const float cc = oj.w * oj.w * t3;
                    gx = fmaf(cc, rx, gx);
                    gy = fmaf(cc, ry, gy);
                    if (DIM == 3) gz = fmaf(cc, rz, gz);
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) ec[c] = en[c];
        }
    }
    const float drho = renorm ? s2 / s1 : drho_in[i];
    d.drho_eval[i] = drho;
    const float rho = by_phase(phi_, ph.rho0) + drho;
    const float vol = by_phase(phi_, ph.mass) / rho;
    const float P = eos_tait7(by_phase(phi_, ph.beta), drho * by_phase(phi_, ph.inv_rho0));
    // grad C_i = sigma_i sum V_j^2 grad W_ij, sigma_i = 1/|V_i| (entry density)
    const float sc = ph.cF / fabsf(oi.w);
    gx *= sc;
    gy *= sc;
    gz *= sc;
    const float n2 = gx * gx + gy * gy + gz * gz;
    unsigned iface = 0u;
    float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 t2 = make_float2(0.f, 0.f);
    if (n2 > 0.f) {
        iface = 1u;
        // T sigma_i^-2 = alpha_s / |g| (|g|^2/d I - g g^T) V_i^2, V_i from the renormalised density
        const float kk = ph.alpha_s * rsqrtf(n2) * vol * vol;
        const float iso = n2 * ph.inv_dim;
        if (DIM == 2) {
            t4 = make_float4(kk * (iso - gx * gx), -kk * gx * gy, kk * (iso - gy * gy), 0.f);
        } else {
            t4 = make_float4(kk * (iso - gx * gx), -kk * gx * gy, -kk * gx * gz, kk * (iso - gy * gy));
            t2 = make_float2(-kk * gy * gz, kk * (iso - gz * gz));
        }
    }
    // signed volume (sign = phase) whose lowest mantissa bit carries the
    // interface flag: at most one unit in the last place, the size of the
    // rounding of m/rho itself
    const float vs = phi_ ? -vol : vol;
    d.posv[i] = make_float4(oi.x, oi.y, oi.z, __uint_as_float((__float_as_uint(vs) & ~1u) | iface));
    vel_s[i].w = P / (rho * rho);
    d.pres[i] = P;
    d.T4[i] = t4;
    if (DIM == 3) d.T2[i] = t2;
}

// ---------------------------------------------------------------------------
// Sweep B: pressure gradient (Eq. dist_p_1), harmonic-mean viscosity
// (Eq. visc_2 or visc_1), surface tension (F_s/rho), gravity, continuity
// (Eq. ct_dist_2).  grad_i W_ij = cF t^3 r_ij with t = 1 - q/2; the common
// factor cF is applied once per particle.
// STAGE 0: rates only; 1: then the predictor; 2: then the corrector.
template <int DIM, int STAGE>
__global__ void __launch_bounds__(256, 4) k_sweep_b(Dev d, Grid g, Phys ph, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float4 oi = d.posv[i];
    const int phi_ = phase_of(oi.w);
    const unsigned iface_i = __float_as_uint(oi.w) & 1u;
    const float4 *__restrict__ vel_s = STAGE == 2 ? d.velq : d.velp;
    const float4 ui = vel_s[i];              // w: P_i / rho_i^2
    const float4 Ti = d.T4[i];
    const float2 Ti2 = DIM == 3 ? d.T2[i] : make_float2(0.f, 0.f);
    float px = 0.f, py = 0.f, pz = 0.f;    // sum m_j (P_i/rho_i^2 + P_j/rho_j^2) t^3 r_ij
    float vx = 0.f, vy = 0.f, vz = 0.f;    // sum k_ij V_j t^3 r^2/(r^2+delta^2) u_ij
    float sx = 0.f, sy = 0.f, sz = 0.f;    // sum (T_i/sigma_i^2 + T_j/sigma_j^2) . t^3 r_ij
    float dv = 0.f;                        // sum V_j t^3 u_ij . r_ij
    const float inv_h = ph.inv_h, cs = g.Es;
    const int n = d.n, cnt = d.ncnt[i];
    // per-phase constants of the pair terms as registers (selected per pair)
    const float m_wat = ph.mass[0], m_oil = ph.mass[1];
    const float kv_wat = phi_ ? ph.kvis[2] : ph.kvis[0], kv_oil = phi_ ? ph.kvis[3] : ph.kvis[1];
    const unsigned *__restrict__ col = d.nbr + i;
    const float4 *__restrict__ posv = d.posv;
    const float4 *__restrict__ T4 = d.T4;
    const float2 *__restrict__ T2 = d.T2;
    constexpr int CH = SPH_LIST_CHUNK;
    unsigned ec[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) ec[c] = c < cnt ? __ldg(col + (size_t)c * n) : 0u;
    for (int k0 = 0; k0 < cnt; k0 += CH) {
        unsigned en[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int kk = k0 + CH + c;
            en[c] = kk < cnt ? __ldg(col + (size_t)kk * n) : 0u;
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (k0 + c >= cnt) break;
            const unsigned e = ec[c];
            const int j = (int)(e & NBR_IDX_MASK);
            const float4 oj = __ldg(posv + j);
            const float4 uj = __ldg(vel_s + j);
            float rx, ry, rz;
            const float r2 = pair_vec<DIM>(oi, oj, entry_shift(e, 0, cs), entry_shift(e, 1, cs),
                                           DIM == 3 ? entry_shift(e, 2, cs) : 0.f, rx, ry, rz);
            const bool oil_j = oj.w < 0.f;
            const float vol_j = fabsf(oj.w);
            // beyond the support (list entries in the skin) t clamps to 0 and
            // every pair term below vanishes
            const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
            const float t = fmaxf(fmaf(-0.5f * inv_h, r, 1.f), 0.f);
            const float t3 = t * t * t;
            const float pt = (oil_j ? m_oil : m_wat) * (ui.w + uj.w) * t3;
            px = fmaf(pt, rx, px);
            py = fmaf(pt, ry, py);
            if (DIM == 3) pz = fmaf(pt, rz, pz);
            const float ux = ui.x - uj.x, uy = ui.y - uj.y, uz = DIM == 3 ? ui.z - uj.z : 0.f;
            const float vt = vol_j * t3;
            const float s = (oil_j ? kv_oil : kv_wat) * vt * __fdividef(r2, r2 + ph.delta2);
            vx = fmaf(s, ux, vx);
            vy = fmaf(s, uy, vy);
            if (DIM == 3) vz = fmaf(s, uz, vz);
            float ur = ux * rx;
            ur = fmaf(uy, ry, ur);
            if (DIM == 3) ur = fmaf(uz, rz, ur);
            dv = fmaf(vt, ur, dv);
            if ((iface_i | (__float_as_uint(oj.w) & 1u)) != 0u) {
                const float4 Tj = __ldg(T4 + j);
                if (DIM == 2) {
                    const float xx = Ti.x + Tj.x, xy = Ti.y + Tj.y, yy = Ti.z + Tj.z;
                    sx = fmaf(t3, xx * rx + xy * ry, sx);
                    sy = fmaf(t3, xy * rx + yy * ry, sy);
                } else {
                    const float2 Tj2 = __ldg(T2 + j);
                    const float xx = Ti.x + Tj.x, xy = Ti.y + Tj.y, xz = Ti.z + Tj.z;
                    const float yy = Ti.w + Tj.w, yz = Ti2.x + Tj2.x, zz = Ti2.y + Tj2.y;
                    sx = fmaf(t3, xx * rx + xy * ry + xz * rz, sx);
                    sy = fmaf(t3, xy * rx + yy * ry + yz * rz, sy);
                    sz = fmaf(t3, xz * rx + yz * ry + zz * rz, sz);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) ec[c] = en[c];
    }
    const float rho = by_phase(phi_, ph.rho0) + d.drho_eval[i];
    float4 out;
    out.w = rho * ph.cF * dv;
    if (d.tag[i] & 2) {
        out.x = out.y = out.z = 0.f;
    } else {
        const float vf = ph.visc_dynamic ? ph.cF / rho : ph.cF;
        const float sf = ph.cF * by_phase(phi_, ph.inv_mass);
        out.x = -ph.cF * px + vf * vx + sf * sx + ph.gf[0];
        out.y = -ph.cF * py + vf * vy + sf * sy + ph.gf[1];
        out.z = DIM == 3 ? -ph.cF * pz + vf * vz + sf * sz + ph.gf[2] : 0.f;
    }
    d.acc[i] = out;
    if (STAGE == 1) predict_particle<DIM>(d, g, ph, i, out, dt);
    if (STAGE == 2) correct_particle<DIM>(d, g, ph, i, out, dt);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Neighbour sets and pair statistics by the sweeps' own support test.

template <int DIM>
__global__ void __launch_bounds__(256) k_nbr_count(Dev d, Grid g, Phys ph, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float4 oi = d.pos[i];
    int cnt = 0;
    for_each_candidate<DIM>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                            [&](int j, const float4 &, float, float, float, float, unsigned) { cnt += j != i; });
    count[i] = cnt;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_nbr_fill(Dev d, Grid g, Phys ph, const long long *start, int *list)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float4 oi = d.pos[i];
    long long w = start[i];
    for_each_candidate<DIM>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                            [&](int j, const float4 &, float, float, float, float, unsigned) {
                                if (j != i) list[w++] = d.pid[j];
                            });
}

// Totals of ordered neighbour pairs (j != i): [0] all, [1] of different phase.
template <int DIM>
__global__ void __launch_bounds__(256) k_pair_stats(Dev d, Grid g, Phys ph, unsigned long long *tot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int all = 0, other = 0;
    if (i < d.n) {
        const float4 oi = d.pos[i];
        const int phi_ = phase_of(oi.w);
        for_each_candidate<DIM>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                                [&](int j, const float4 &oj, float, float, float, float, unsigned) {
                                    all += j != i;
                                    other += phase_of(oj.w) != phi_;
                                });
    }
    for (int o = 16; o > 0; o >>= 1) {
        all += __shfl_down_sync(0xffffffffu, all, o);
        other += __shfl_down_sync(0xffffffffu, other, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(tot, (unsigned long long)all);
        atomicAdd(tot + 1, (unsigned long long)other);
    }
}

// ---------------------------------------------------------------------------
// Output in original order.

enum ReadKind { RK_X, RK_U, RK_RHO, RK_RHO_EVAL, RK_P, RK_ACC, RK_DRHO, RK_T, RK_CELL, RK_ORDER };

template <int DIM>
__global__ void __launch_bounds__(256) k_unpermute(Dev d, Phys ph, int kind, double *out, int *iout)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int n = d.n;
    const int p = d.pid[k];
    const int phs = d.tag[k] & 1;
    switch (kind) {
    case RK_X:
        for (int c = 0; c < DIM; ++c) out[(size_t)p * DIM + c] = d.x[(size_t)c * n + k];
        break;
    case RK_U:
        for (int c = 0; c < DIM; ++c) out[(size_t)p * DIM + c] = d.u[(size_t)c * n + k];
        break;
    case RK_RHO:
        out[p] = (double)by_phase(phs, ph.rho0) + (double)d.drho[k];
        break;
    case RK_RHO_EVAL:
        out[p] = (double)by_phase(phs, ph.rho0) + (double)d.drho_eval[k];
        break;
    case RK_P:
        out[p] = d.pres[k];
        break;
    case RK_ACC: {
        const float4 a = d.acc[k];
        const float av[3] = {a.x, a.y, a.z};
        for (int c = 0; c < DIM; ++c) out[(size_t)p * DIM + c] = av[c];
        break;
    }
    case RK_DRHO:
        out[p] = d.acc[k].w;
        break;
    case RK_T: {
        const float4 t = d.T4[k];
        // T sigma^-2 was formed with V = m/rho of the renormalised density
        const double v = (double)(by_phase(phs, ph.mass) / (by_phase(phs, ph.rho0) + d.drho_eval[k]));
        const double v2 = v * v;
        double T[9];
        if (DIM == 2) {
            T[0] = t.x; T[1] = t.y; T[2] = t.y; T[3] = t.z;
        } else {
            const float2 t2 = d.T2[k];
            T[0] = t.x; T[1] = t.y; T[2] = t.z;
            T[3] = t.y; T[4] = t.w; T[5] = t2.x;
            T[6] = t.z; T[7] = t2.x; T[8] = t2.y;
        }
        for (int c = 0; c < DIM * DIM; ++c) out[(size_t)p * DIM * DIM + c] = T[c] / v2;
        break;
    }
    case RK_CELL:
        iout[p] = d.cell[k];
        break;
    case RK_ORDER:
        iout[k] = p;
        break;
    }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: deterministic two-level reductions.

constexpr int DIAG_THREADS = 256;
constexpr int DIAG_K = 16;  // accumulated quantities per pass

__device__ __forceinline__ void block_reduce_store(double (&v)[DIAG_K], double *out)
{
    __shared__ double sm[DIAG_THREADS];
#pragma unroll 1
    for (int q = 0; q < DIAG_K; ++q) {
        sm[threadIdx.x] = v[q];
        __syncthreads();
        for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                // max for the speed slot, sum otherwise
                sm[threadIdx.x] = q == 15 ? fmax(sm[threadIdx.x], sm[threadIdx.x + s])
                                          : sm[threadIdx.x] + sm[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) out[q] = sm[0];
        __syncthreads();
    }
}

// pass 0: mass, momentum, energies, oil count and sum of oil positions, max|u|
// pass 1: covariance of oil positions about the centroid `cen`
template <int DIM>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag(Dev d, int pass, const double *cen, const double *grav,
                                                       const double *mass, double *partial)
{
    double v[DIAG_K];
#pragma unroll
    for (int q = 0; q < DIAG_K; ++q) v[q] = 0.0;
    const int n = d.n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint8_t tg = d.tag[k];
        if (tg & 2) continue;
        const int oil = tg & 1;
        double x[3] = {0, 0, 0}, u[3] = {0, 0, 0};
        for (int c = 0; c < DIM; ++c) {
            x[c] = d.x[(size_t)c * n + k];
            u[c] = d.u[(size_t)c * n + k];
        }
        if (pass == 0) {
            const double m = mass[oil];
            const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            v[0] += m;
            v[1] += m * u[0];
            v[2] += m * u[1];
            v[3] += m * u[2];
            v[4] += 0.5 * m * u2;
            v[5] -= m * (grav[0] * x[0] + grav[1] * x[1] + grav[2] * x[2]);
            if (oil) {
                v[6] += x[0];
                v[7] += x[1];
                v[8] += x[2];
                v[9] += 1.0;
            }
            v[15] = fmax(v[15], sqrt(u2));
        } else if (oil) {
            const double a = x[0] - cen[0], b = x[1] - cen[1], c = x[2] - cen[2];
            v[0] += a * a;
            v[1] += a * b;
            v[2] += a * c;
            v[3] += b * b;
            v[4] += b * c;
            v[5] += c * c;
        }
    }
    block_reduce_store(v, partial + (size_t)blockIdx.x * DIAG_K);
}

__global__ void __launch_bounds__(DIAG_K) k_diag_final(const double *partial, int nblocks, double *out)
{
    const int q = threadIdx.x;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double v = partial[(size_t)b * DIAG_K + q];
        s = q == 15 ? fmax(s, v) : s + v;
    }
    out[q] = s;
}

}  // namespace sphgb
