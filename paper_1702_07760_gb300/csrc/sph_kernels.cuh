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
//   * a neighbour list (radius 2h + 2 skin) is built from the cell list,
//     scanning per particle only the cells of the +/-f stencil that the
//     radius can reach, and stored column-major, so the four interaction
//     sweeps of a step read it coalesced and run without the branch
//     divergence of a candidate scan; a sweep gathers two 16-byte records per
//     neighbour.  The list is rebuilt only when a particle may have moved
//     farther than the skin since the last build;
//   * several independent simulations ("instances") can share one particle
//     set: they sit in disjoint regions of one box and each particle carries
//     the index of its instance, whose constants (densities, masses,
//     viscosities, tension, time-step scale) come from a small table.
//
// Every phase is a device function of one particle (or cell, or tile), used
// both by one-kernel-per-phase launches and by a persistent kernel that runs
// whole steps with grid barriers between phases.  The template flag NC
// selects read-only cached loads, which are valid only for data no phase of
// the same launch writes; the persistent kernel uses plain loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sphgb {

enum : unsigned {
    FLAG_DOMAIN = 1u,     // a particle left the cell grid
    FLAG_NONFINITE = 2u,  // NaN/Inf in the state
    FLAG_SKIN = 4u,       // predictor displacement beyond the skin
    FLAG_LIST = 8u,       // a particle has more list neighbours than max_neighbours
    FLAG_TIMEOUT = 16u,   // a grid barrier of the persistent kernel gave up waiting
    FLAG_BOUNDS = 32u,    // an index out of range (bounds-checked builds only)
};
constexpr unsigned FLAG_ERRORS = 63u;

// Bounds-checked build (-DSPH_CHECKED): every index read from device data
// (list entries, sort slots, permutations) is tested before it is used; a bad
// one raises FLAG_BOUNDS and the access is skipped instead of made.  Off in the
// ordinary build, where the indices are correct by construction.
#ifdef SPH_CHECKED
#define SPH_IN_RANGE(flags, i, n) \
    (((unsigned)(i) < (unsigned)(n)) ? true : (atomicOr((flags), FLAG_BOUNDS), false))
#else
#define SPH_IN_RANGE(flags, i, n) true
#endif

// Constants shared by all instances, FP32 unless they feed an FP64 accumulator.
struct Phys {
    float inv_h;        // 1/h
    float R2;           // (2h)^2, support test
    float RL2;          // list radius^2, (2h + 2 skin)^2
    float RP;           // list radius widened by 1e-4 (conservative stencil pruning)
    float cF;           // -5 alpha_d / h^2: grad W_ij = cF (1-q/2)^3 r_ij
    float delta2;       // delta^2
    float inv_dim;      // 1/d in Eq. csf
    float gf[3];        // gravity (FP32, added to the FP32 acceleration)
    int visc_dynamic;   // 1: Eq. visc_2 (factor 1/rho_i), 0: Eq. visc_1
    int renorm_every;   // Eq. ct_dist_3 at stage 1 of steps with step % renorm_every == 0
    int renorm_walls;   // 1: boundary particles are renormalised as water; 0: they keep their density
    int kmax;           // neighbour-list capacity per particle
    int rebuild_every;  // 0: rebuild when a particle may leave the skin; k: every k steps
    double skin;        // allowed displacement since the last build (the list's margin)
    float skin2f;       // (float)(skin * skin): the predictor's skin test
    float skin98f;      // (float)(0.98 * skin): the corrector's rebuild test
};

// Constants of one instance.
struct Inst {
    float mass[2];      // per-phase particle mass
    float inv_mass[2];
    float rho0[2];      // per-phase reference density
    float inv_rho0[2];
    float beta[2];      // rho0 c0^2 / gamma
    float kvis[4];      // [2*ph_i + ph_j]: 2 mu_ij (dynamic form) or 2 nu_ij (kinematic form)
    float vol0[2];      // per-phase m / rho0: the volume at the reference density
    float alpha_s;      // surface tension coefficient
    float pad;
    double dt_scale;    // this instance's step is dt * dt_scale
    double offset[3];   // placement of the instance's frame in the shared box
    double mass64[2];   // per-phase particle mass in FP64 (diagnostics)
};

struct Grid {
    int nx, ny, nz;     // cells per axis (nz = 1 in 2-D)
    int f;              // cells per super-cell edge: 1 or 2 (also the stencil half-width)
    float cs;           // cell edge (FP32)
    float inv_cs;       // 1 / cs (FP32): row pruning and the hash's estimate
    float Es;           // super-cell edge (FP32): pair vectors
    double csd;         // cell edge (FP64): hashing
    double Ed;          // super-cell edge (FP64): offsets
    double lo[3];       // box lower corner
    int per[3];         // 1: the axis is periodic (its cell count is a multiple of f, >= 3f)
    const double *cen;  // super-cell centres, FP64: axis a, super-cell S at cen[cen_off[a] + S],
    int cen_off[3];     //   each fma(S + 0.5, Ed, lo[a]) (a table: no int-to-FP64 work per use)
};

// All device arrays of one simulation (sorted order unless noted).
struct Dev {
    int n;
    // state (FP64 accumulators + FP32 density deviation)
    double *x;          // dim * n, SoA
    double *u;          // dim * n, SoA
    float *drho;        // n, rho - rho0(phase) of the state
    int *pid;           // n, original particle id
    int *inv;           // n, by original id: the particle's sorted position (inverse of pid)
    uint8_t *tag;       // n, bit0 oil, bit1 wall
    uint16_t *iid;      // n, instance index
    int *cell;          // n, cell id (sorted order)
    const Inst *inst;   // instance table
    // stage arrays
    float4 *pos;        // n, (offset from the super-cell centre xyz, w: (m/rho) * drho of the stage
                        //     input with its lowest mantissa bit replaced by the phase; pack_vd)
    float4 *pos0;       // n, offset at the last list build (xyz): displacement since the build
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
    int *nfcnt;         // n, the part of the list the force sweep visits while *walls_moving is 0
                        //     (static boundary particles: the leading part without static
                        //     boundary neighbours; everyone else: the whole list)
    unsigned *walls_moving;  // 1 word: nonzero when a static boundary particle has a nonzero
                        //     velocity (set by the load of a state; boundary particles keep u)
    uint8_t *nflag;     // n, bit0: an other-phase particle lies within the list radius
    int *mixed;         // n, the particles with nflag bit 0 set, in no particular order
    int *nmixed;        // 1 word: their number (reset by the hash, appended by the list build)
    // cell list
    int *cstart;        // ncell + 1
    unsigned *flags;    // 1 word
    unsigned *rebuild;  // 1 word: nonzero when the cell and neighbour lists must be rebuilt
    long long *step;    // device step counter (drives the renormalisation schedule)
    long long *builds;  // number of list builds performed
    // time and boundary motion
    double *clock;      // 2 words: [0] time t_n of the current step, [1] the step size
                        //   of the last completed step, added into [0] when the next starts
    const struct Motion *motion;  // prescribed piston motion (particles with tag bit 2)
    // periodic axes: period (0 when the axis is not periodic) and lower bound
    double period[3];
    double plo[3];
};

// Prescribed displacement X(t) of the piston particles along `axis`: for
// t <= t_end, X(t) = sum_c amp_c (sin(omega_c t + phase_c) - sin(phase_c)) and
// X'(t) = sum_c amp_c omega_c cos(omega_c t + phase_c); afterwards the piston
// rests at X(t_end).  (The flume runs drive a piston-type wave maker with a
// cosine stroke: one component with phase -pi/2.)
constexpr int MOTION_MAX = 8;
struct Motion {
    int axis;
    int ncomp;
    double t_end;
    double amp[MOTION_MAX];
    double omega[MOTION_MAX];
    double phase[MOTION_MAX];
};

__device__ __forceinline__ double motion_disp(const Motion &m, double t)
{
    const double te = t < m.t_end ? t : m.t_end;
    double X = 0.0;
    for (int c = 0; c < m.ncomp; ++c) X += m.amp[c] * (sin(m.omega[c] * te + m.phase[c]) - sin(m.phase[c]));
    return X;
}

__device__ __forceinline__ double motion_vel(const Motion &m, double t)
{
    if (t > m.t_end) return 0.0;
    double U = 0.0;
    for (int c = 0; c < m.ncomp; ++c) U += m.amp[c] * m.omega[c] * cos(m.omega[c] * t + m.phase[c]);
    return U;
}

// Coordinate wrapped into [lo, lo + L) along a periodic axis (L > 0).
__device__ __forceinline__ double wrap_coord(double v, double lo, double L)
{
    return L > 0.0 ? v - L * floor((v - lo) / L) : v;
}

// Scratch of the cell-list build.
struct Sort {
    int *count;         // ncell, particles per cell
    int *cell_tmp;      // n, cell id in the pre-sort order
    int *slot;          // n, arrival slot within the cell
    int *tmp;           // n, pre-sort index at each (unordered) sorted position
    int *perm;          // n, pre-sort index at each sorted position
    int *tile_sums;     // scan tiles
    int ncell;
    int n;              // particles
    unsigned *flags;    // the simulation's error word (bounds-checked builds)
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

// Load through the read-only cache when NC (data constant for the launch).
template <bool NC, class T>
__device__ __forceinline__ T ld(const T *p)
{
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// Neighbour-list entry load.  The list is streamed once per sweep (each
// warp reads whole 128-byte lines of it), so in launches where it is
// read-only its lines bypass L1 and leave the space to the neighbour records
// that are gathered many times (measured 1 % faster on both sweeps).
template <bool NC>
__device__ __forceinline__ unsigned ld_list(const unsigned *p)
{
    if constexpr (NC) {
        unsigned v;
        asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
        return v;
    } else {
        return *p;
    }
}

// Read-only pointer, __restrict__ only where the pointee is not written
// anywhere in the launch (NC): the persistent kernel writes every array in
// some phase and must not let the compiler route its loads through the
// non-coherent read-only path.
template <bool NC, class T>
struct RO {
    using type = const T *__restrict__;
};
template <class T>
struct RO<false, T> {
    using type = const T *;
};

__device__ __forceinline__ int phase_of(float w) { return __float_as_uint(w) >> 31; }

// Boundary particle that is not a piston (tag bit 1 without bit 2).
__device__ __forceinline__ bool static_wall(unsigned tag) { return (tag & 6u) == 2u; }

__device__ __forceinline__ float by_phase(int phase, const float (&a)[2]) { return phase ? a[1] : a[0]; }

// w of a stage-input record (pos): vd = (m/rho) drho, the volume times the
// density deviation, with its lowest mantissa bit replaced by the phase (1:
// oil; a change of at most one unit in the last place of vd).  Within a
// phase vd = V (rho - rho0) = m - rho0 V, so the record gives the volume too,
// V = m/rho0 - vd/rho0, and the renormalisation sweep reads one 16-byte
// record per neighbour.
__device__ __forceinline__ float pack_vd(float vd, int oil)
{
    return __uint_as_float((__float_as_uint(vd) & ~1u) | (unsigned)oil);
}
__device__ __forceinline__ int rec_phase(float w) { return (int)(__float_as_uint(w) & 1u); }
__device__ __forceinline__ float rec_vd(float w) { return __uint_as_float(__float_as_uint(w) & ~1u); }
__device__ __forceinline__ float rec_vol(float vd, float vol0, float inv_rho0) { return fmaf(-inv_rho0, vd, vol0); }

// (S_i - S_j) * E for axis a of an entry, exact: the code e in {0, 1, 2}
// becomes the float e - 1 through the 2^23 + 2^22 mantissa trick.
__device__ __forceinline__ float entry_shift(unsigned e, int a, float E)
{
    const unsigned code = (e >> (NBR_IDX_BITS + 2 * a)) & 3u;
    return (__uint_as_float(0x4B400000u | code) - 12582913.f) * E;
}

// Products that feed a sum are written as explicit FMAs or round-to-nearest
// multiplies throughout the sweeps and the integration, so ptxas has no
// multiply-add left to fuse: every build of a function (per-kernel launches
// and the persistent kernel, at any register budget) rounds identically.

// x^2 + y^2 + z^2 with a fixed rounding sequence.
__device__ __forceinline__ float sq3(float x, float y, float z)
{
    return fmaf(z, z, fmaf(y, y, __fmul_rn(x, x)));
}

// r_ij = x_i - x_j from super-cell offsets and the centre difference (s).
template <int DIM>
__device__ __forceinline__ float pair_vec(const float4 &oi, const float4 &oj, float sx, float sy, float sz,
                                          float &rx, float &ry, float &rz)
{
    rx = (oi.x - oj.x) + sx;
    ry = (oi.y - oj.y) + sy;
    rz = DIM == 3 ? (oi.z - oj.z) + sz : 0.f;
    float r2 = __fmul_rn(rx, rx);
    r2 = fmaf(ry, ry, r2);
    if (DIM == 3) r2 = fmaf(rz, rz, r2);
    return r2;
}

// r_ij = x_i - x_j for list entry e (returns |r_ij|^2): the offset difference
// plus the super-cell centre difference (S_i - S_j) E of each axis, whose
// codes (S_i - S_j + 1) sit at bits 26 (x), 28 (y) and 30 (z).  Each code
// becomes an exact float through the 1.5 * 2^23 mantissa trick and is fused
// into the difference with one FMA: the same value as (o_i - o_j) + (S_i - S_j) E.
template <int DIM>
__device__ __forceinline__ float entry_vec(const float4 &oi, const float4 &oj, unsigned e, float E, float &rx,
                                          float &ry, float &rz)
{
    const unsigned es = e >> NBR_IDX_BITS;
    rx = fmaf(__uint_as_float(0x4B400000u | (es & 3u)) - 12582913.f, E, oi.x - oj.x);
    ry = fmaf(__uint_as_float(0x4B400000u | ((es >> 2) & 3u)) - 12582913.f, E, oi.y - oj.y);
    rz = DIM == 3 ? fmaf(__uint_as_float(0x4B400000u | (es >> 4)) - 12582913.f, E, oi.z - oj.z) : 0.f;
    float r2 = __fmul_rn(rx, rx);
    r2 = fmaf(ry, ry, r2);
    if (DIM == 3) r2 = fmaf(rz, rz, r2);
    return r2;
}

// |r_ij| from r^2 as r^2 / sqrt(r^2).  The added 1e-30 lies far below half
// an ulp of any nonzero r^2 a list holds, so it changes nothing but r^2 = 0,
// which it keeps finite (a plain FP32 add, on the FMA pipe).
__device__ __forceinline__ float pair_dist(float r2) { return r2 * rsqrtf(r2 + 1e-30f); }

// t = 1 - q/2 = 1 - r/(2h), clamped at 0 beyond the support by the saturation
// of the fused multiply-add (t <= 1 holds anyway, r >= 0).
__device__ __forceinline__ float kernel_t(float inv_h, float r)
{
    float t;
    asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(t) : "f"(-0.5f * inv_h), "f"(r), "f"(1.f));
    return t;
}

// Padding entry of particle i's list: i itself one super-cell away along x
// and y, |r| = sqrt(2) E > 2h, so every pair term it feeds is zero.
__device__ __forceinline__ unsigned pad_entry(int i)
{
    return (unsigned)i | (2u << NBR_IDX_BITS) | (2u << (NBR_IDX_BITS + 2)) | (1u << (NBR_IDX_BITS + 4));
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
// fn(j, oj, rx, ry, rz, r2, code) for those with |r_ij|^2 < R2 (j == i
// included); code is the shift part of a neighbour-list entry.  Along a
// periodic axis the stencil wraps around the box: cells are visited at their
// unwrapped position (so the super-cell difference S_i - S_j, and with it
// r_ij, is that of the nearest image) and read at the wrapped one.
template <int DIM, bool NC, class F>
__device__ __forceinline__ void for_each_candidate(const Grid &g, typename RO<NC, int>::type cstart,
                                                   typename RO<NC, float4>::type pos, int c, const float4 &oi,
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
    int z0 = 0, z1 = 0;
    if (DIM == 3) {
        z0 = g.per[2] ? cz - hw : max(cz - hw, 0);
        z1 = g.per[2] ? cz + hw : min(cz + hw, g.nz - 1);
    }
    const int y0 = g.per[1] ? cy - hw : max(cy - hw, 0), y1 = g.per[1] ? cy + hw : min(cy + hw, g.ny - 1);
    for (int z = z0; z <= z1; ++z) {
        const float gz = DIM == 3 ? axis_gap(pz, z - cz, e) : 0.f;
        if (gz >= Rp) continue;
        const int dSz = DIM == 3 ? Sz - (z >> fm) : 0;
        const int zw = DIM == 3 ? (z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z)) : 0;
        const float sz = (float)dSz * E;
        for (int y = y0; y <= y1; ++y) {
            const float gy = axis_gap(py, y - cy, e);
            const float rem = Rp2 - gy * gy - gz * gz;
            if (rem <= 0.f) continue;
            const int dSy = Sy - (y >> fm);
            const int yw = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
            const float sy = (float)dSy * E;
            // the row's cells that reach the sphere of radius Rp; Rp exceeds
            // every search radius by 1e-4 of the list radius, far more than
            // the few-ulp error of the fast root and of the reciprocal
            // (1e-6 of a cell), so no cell holding a particle within the
            // search radius is left out
            const float xr = rem * rsqrtf(rem + 1e-30f);
            int xlo = max(cx + (int)floorf((px - xr) * g.inv_cs), cx - hw);
            int xhi = min(cx + (int)floorf((px + xr) * g.inv_cs), cx + hw);
            if (!g.per[0]) {
                xlo = max(xlo, 0);
                xhi = min(xhi, g.nx - 1);
            }
            if (xlo > xhi) continue;
            const int row = (zw * g.ny + yw) * g.nx;
            const unsigned cyz = ((unsigned)(dSy + 1) << (NBR_IDX_BITS + 2)) |
                                 ((unsigned)(dSz + 1) << (NBR_IDX_BITS + 4));
            // the particles of cells a..b of the row (one image)
            auto piece = [&](int a, int b, int off) {
                const int jb = ld<NC>(cstart + row + a - off), je = ld<NC>(cstart + row + b - off + 1);
                // super-cell Sx covers the unwrapped cells [Sx*f, Sx*f + f)
                const int b1 = ld<NC>(cstart + row + min(max(Sx * hw, a), b + 1) - off);
                const int b2 = ld<NC>(cstart + row + min(max(Sx * hw + hw, a), b + 1) - off);
#pragma unroll 4
                for (int j = jb; j < je; ++j) {
                    const float4 oj = ld<NC>(pos + j);
                    // super-cell of j along x: Sx - 1, Sx or Sx + 1
                    const float sx = j < b1 ? E : (j < b2 ? 0.f : -E);
                    const unsigned ex = j < b1 ? 2u : (j < b2 ? 1u : 0u);
                    float rx, ry, rz;
                    const float r2 = pair_vec<DIM>(oi, oj, sx, sy, sz, rx, ry, rz);
                    if (r2 < R2) fn(j, oj, rx, ry, rz, r2, cyz | (ex << NBR_IDX_BITS));
                }
            };
            if (!g.per[0]) {
                piece(xlo, xhi, 0);
            } else {
                // the unwrapped range xlo..xhi in pieces of one image each;
                // the cells of a piece are contiguous in the sorted order
                for (int img = -1; img <= 1; ++img) {
                    const int off = img * g.nx;
                    const int a = max(xlo, off), b = min(xhi, off + g.nx - 1);
                    if (a <= b) piece(a, b, off);
                }
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
    for (int a = 0; a < DIM; ++a) o[a] = (float)(xa[a] - g.cen[g.cen_off[a] + (cc[a] >> fm)]);
    return make_float4(o[0], o[1], o[2], 0.f);
}

// Every component of v finite (FP32 tests on the FMA/ALU pipes: the FP64
// pipe of this part runs at 1/64 of the FP32 rate).
__device__ __forceinline__ bool finite4(const float4 &v)
{
    return isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
}

// w of the stage-input record of a particle of the given phase and density
// deviation: (m/rho) drho with the phase bit (pack_vd).
__device__ __forceinline__ float record_w(const Inst &I, int phase, float drho)
{
    const float vol = by_phase(phase, I.mass) / (by_phase(phase, I.rho0) + drho);
    return pack_vd(vol * drho, phase);
}

// ---------------------------------------------------------------------------
// Cell list: hash, counting sort stable in particle id, reorder.

template <int DIM>
__device__ __forceinline__ void hash_one(const Dev &d, const Grid &g, const Sort &s, int k)
{
    if (k == 0) *d.nmixed = 0;  // the list build that follows appends the mixed particles
    const int dims[3] = {g.nx, g.ny, g.nz};
    int c[3] = {0, 0, 0};
    unsigned bad = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        double xa = d.x[(size_t)a * d.n + k];
        if (g.per[a] && isfinite(xa)) {
            // a periodic coordinate is wrapped into the box at every build
            xa = wrap_coord(xa, g.lo[a], d.period[a]);
            d.x[(size_t)a * d.n + k] = xa;
        }
        // floor((x - lo) / cs) of the FP64 quotient, from an FP32 estimate
        // where that is decisive: q32 = fl32(t) * fl32(1 / fl32(cs)) lies
        // within 2.4e-7 |q| of t / cs (four FP32 roundings of at most 2^-24
        // relative: cs, its reciprocal, t and the product), so when its
        // fractional part keeps 4e-7 |q| + 1e-30 away from 0 and 1 both floors
        // agree; otherwise (near a cell face, or not finite) the FP64
        // division decides, as before
        const double t = xa - g.lo[a];
        const float q32 = __fmul_rn((float)t, g.inv_cs);
        const float fl = floorf(q32), fr = q32 - fl, m = fmaf(4e-7f, fabsf(q32), 1e-30f);
        if (fr > m && fr < 1.f - m) {
            // decided by the estimate (finite, away from a face): the bounds
            // test on the FP32 cell index, off the FP64 pipe (1/64 rate)
            if (fl >= 0.f && fl < (float)dims[a]) c[a] = (int)fl;
            else bad |= FLAG_DOMAIN;
            continue;
        }
        double sc = floor(t / g.csd);
        if (g.per[a] && sc >= (double)dims[a]) sc = dims[a] - 1;  // rounding at the upper side
        if (isnan(xa)) {
            bad |= FLAG_NONFINITE;
        } else if (!(sc >= 0.0 && sc < (double)dims[a])) {
            bad |= FLAG_DOMAIN;
        } else {
            c[a] = (int)sc;
        }
    }
    if (bad) atomicOr(d.flags, bad);
    const int id = c[0] + g.nx * (c[1] + g.ny * c[2]);
    s.cell_tmp[k] = id;
    s.slot[k] = atomicAdd(s.count + id, 1);
}

// Exclusive scan of the cell counts in tiles of SCAN_TILE cells.
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

// Scans tile `tile` of `in` (m values) into `out` with whatever block size
// runs it (each thread takes SCAN_TILE / blockDim consecutive values) and
// returns the tile total (the same in every thread).
__device__ __forceinline__ int scan_tile(const int *in, int *out, int m, int tile)
{
    __shared__ int s_total;
    const int per = SCAN_TILE / blockDim.x;
    const int base = tile * SCAN_TILE + threadIdx.x * per;
    int sum = 0;
    for (int k = 0; k < per; ++k) sum += base + k < m ? in[base + k] : 0;
    int ex = block_exclusive_scan(sum, &s_total);
    for (int k = 0; k < per; ++k) {
        if (base + k < m) {
            const int v = in[base + k];
            out[base + k] = ex;
            ex += v;
        }
    }
    const int t = s_total;
    __syncthreads();
    return t;
}

// Exclusive scan of the tile totals in place (one block); writes the grand
// total to out[m].
__device__ __forceinline__ void scan_tile_sums(int *tile_sums, int ntiles, int *out, int m)
{
    __shared__ int s_total;
    const int per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int base = threadIdx.x * per;
    int sum = 0;
    for (int k = 0; k < per; ++k) sum += base + k < ntiles ? tile_sums[base + k] : 0;
    int ex = block_exclusive_scan(sum, &s_total);
    for (int k = 0; k < per; ++k) {
        if (base + k < ntiles) {
            const int v = tile_sums[base + k];
            tile_sums[base + k] = ex;
            ex += v;
        }
    }
    if (threadIdx.x == 0) out[m] = s_total;
    __syncthreads();
}

__device__ __forceinline__ void scatter_one(const Sort &s, const int *cstart, int k)
{
    const int t = cstart[s.cell_tmp[k]] + s.slot[k];
    if (SPH_IN_RANGE(s.flags, t, s.n)) s.tmp[t] = k;
}

// Final position of each particle inside its cell: its rank by original id
// among the cell's particles, so the order is (cell id, particle id).
__device__ __forceinline__ void rank_one(const Sort &s, const int *pid, const int *cstart, int p)
{
    const int k = s.tmp[p];
    const int c = s.cell_tmp[k];
    const int b = cstart[c], e = cstart[c + 1];
    const int me = pid[k];
    int rank = 0;
    for (int q = b; q < e; ++q) rank += pid[s.tmp[q]] < me;
    if (SPH_IN_RANGE(s.flags, b + rank, s.n)) s.perm[b + rank] = k;
}

// Stage-1 records of particle k from its FP64 state; returns whether every
// FP32 value of the records is finite (a non-finite FP64 position or
// velocity gives a non-finite record), and the position and velocity
// records through p_out and v_out.
template <int DIM>
__device__ __forceinline__ bool stage_records(const Dev &d, const Grid &g, const Inst &I, int k, int c,
                                              const double xa[3], const double ua[3], float dr, int oil,
                                              float4 *p_out = nullptr, float4 *v_out = nullptr)
{
    float4 p = cell_offset<DIM>(g, c, xa);
    p.w = record_w(I, oil, dr);
    const float4 v = make_float4((float)ua[0], (float)ua[1], (float)ua[2], 0.f);
    d.pos[k] = p;
    d.velp[k] = v;
    if (p_out) *p_out = p;
    if (v_out) *v_out = v;
    return finite4(p) && finite4(v);
}

// Gathers the state of sorted position k into the scratch set `dst` and
// prepares its stage-1 records and build offset.
template <int DIM>
__device__ __forceinline__ void gather_one(const Dev &src, const Dev &dst, const Grid &g, const Sort &s, int k)
{
    const int n = src.n;
    const int o = s.perm[k];
    if (!SPH_IN_RANGE(src.flags, o, n)) return;
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
    const uint16_t ii = src.iid[o];
    const int c = s.cell_tmp[o];
    dst.drho[k] = dr;
    dst.pid[k] = src.pid[o];
    dst.tag[k] = tg;
    dst.iid[k] = ii;
    src.cell[k] = c;
    stage_records<DIM>(src, g, src.inst[ii], k, c, xa, ua, dr, tg & 1);
    src.pos0[k] = src.pos[k];
}

template <int DIM>
__device__ __forceinline__ void copy_one(const Dev &src, const Dev &dst, int k)
{
    const int n = src.n;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        dst.x[(size_t)a * n + k] = src.x[(size_t)a * n + k];
        dst.u[(size_t)a * n + k] = src.u[(size_t)a * n + k];
    }
    dst.drho[k] = src.drho[k];
    dst.pid[k] = src.pid[k];
    dst.inv[src.pid[k]] = k;
    dst.tag[k] = src.tag[k];
    dst.iid[k] = src.iid[k];
}

// Neighbour list of particle i: every j != i within 2h + 2 skin at the
// positions of the build, so the list stays complete while no particle moves
// farther than the skin.
template <int DIM, bool NC>
__device__ __forceinline__ void list_one(const Dev &d, const Grid &g, const Phys &ph, int i)
{
    const float4 oi = d.pos[i];
    const int phi_ = rec_phase(oi.w);
    int cf = 0, cs = 0;  // entries at the front; static boundary entries at the back
    int other = 0;
    const int n = d.n, kmax = ph.kmax;
    unsigned *__restrict__ nbr = d.nbr;
    typename RO<NC, uint8_t>::type tag = d.tag;
    // a static boundary particle while every static boundary particle is at
    // rest: its pairs with the others feed the force sweep nothing (u_ij = 0,
    // and its own acceleration is not used), so they are written from the end
    // of its column backwards and then moved behind the rest of its list,
    // which the force sweep visits alone
    const bool split = static_wall(d.tag[i]) && *(volatile unsigned *)d.walls_moving == 0u;
    for_each_candidate<DIM, NC>(g, d.cstart, d.pos, d.cell[i], oi, ph.RL2, ph.RP,
        [&](int j, const float4 &oj, float, float, float, float, unsigned code) {
            if (j == i) return;
            const bool back = split && static_wall(ld<NC>(tag + j));
            // entries past kmax are counted, not stored (the overflow is reported)
            if (cf + cs < kmax) nbr[(size_t)(back ? kmax - 1 - cs : cf) * n + i] = (unsigned)j | code;
            cf += !back;
            cs += back;
            other |= rec_phase(oj.w) != phi_;
        });
    // lists hold whole chunks (kmax is a multiple of the chunk), so the
    // sweeps need no per-entry bound test
    int nf = cf;
    for (; nf % SPH_LIST_CHUNK; ++nf)
        if (nf + cs < kmax) nbr[(size_t)nf * n + i] = pad_entry(i);
    int cnt = nf + cs;
    if (cnt > kmax) {
        atomicOr(d.flags, FLAG_LIST);
        cnt = kmax;
        nf = min(nf, kmax);
    } else if (cs > 0) {
        // the back entries (in reverse scan order) move down to follow the
        // front part; every move goes to a lower or equal slot, in ascending
        // order, so no entry is overwritten before it is read
        for (int q = 0; q < cs; ++q) nbr[(size_t)(nf + q) * n + i] = nbr[(size_t)(kmax - cs + q) * n + i];
    }
    for (; cnt % SPH_LIST_CHUNK; ++cnt) nbr[(size_t)cnt * n + i] = pad_entry(i);
    d.ncnt[i] = cnt;
    d.nfcnt[i] = split ? nf : cnt;
    d.nflag[i] = (uint8_t)other;
    if (other) d.mixed[atomicAdd(d.nmixed, 1)] = i;
}

// ---------------------------------------------------------------------------
// Explicit midpoint predictor-corrector, run per particle at the end of the
// force sweep of each stage (the particle's own acceleration is then final).

// Predictor: x* = x^n + dt/2 u^n, u* = u^n + dt/2 a^n, rho* = rho^n + dt/2 Drho^n;
// the renormalised density becomes the state rho^n.  Writes the stage-2
// records (pos, velq).  o1 and u1 are the particle's stage-1 records
// (the FP32 offset of x^n from its super-cell centre and the FP32 u^n): the
// stage-2 offset is o1 + dt/2 u1 in one FP32 FMA per axis, within one
// rounding of the offset of the FP64 x*, and x* itself is not needed (the
// corrector integrates from x^n).  Only the velocity, which the stage keeps
// to integrate x, goes through FP64 (the FP64 pipe of this part runs at 1/64
// of the FP32 rate); the pistons' prescribed motion is evaluated in FP64.
template <int DIM>
__device__ __forceinline__ void predict_particle(const Dev &d, const Grid &g, const Phys &ph, const Inst &I, int k,
                                                 float4 a, double dt, const float4 &o1, const float4 &u1)
{
    const uint8_t tg = d.tag[k];
    const float dr = d.drho_eval[k];
    d.drho[k] = dr;
    const float hdt = 0.5f * (float)dt;
    const float drs = fmaf(hdt, a.w, dr);
    d.drho_stage[k] = drs;
    double us[3] = {0, 0, 0};
    const double af[3] = {a.x, a.y, a.z};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const double u = d.u[(size_t)c * d.n + k];
        us[c] = (tg & 2) ? u : fma(0.5 * dt, af[c], u);
    }
    float4 p;
    if (tg & 4) {
        // piston: at X(t + dt/2) with velocity X'(t + dt/2) along its axis
        const Motion &m = *d.motion;
        const double t = d.clock[0];
        const double dX = motion_disp(m, t + 0.5 * dt) - motion_disp(m, t), U = motion_vel(m, t + 0.5 * dt);
        double xs[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            xs[c] = d.x[(size_t)c * d.n + k];
            if (c == m.axis) xs[c] += dX;
            us[c] = c == m.axis ? U : 0.0;
        }
        p = cell_offset<DIM>(g, d.cell[k], xs);
    } else if (tg & 2) {
        p = make_float4(o1.x, o1.y, o1.z, 0.f);
    } else {
        p = make_float4(fmaf(hdt, u1.x, o1.x), fmaf(hdt, u1.y, o1.y), DIM == 3 ? fmaf(hdt, u1.z, o1.z) : 0.f, 0.f);
    }
    // the neighbour list stays complete while no particle is farther than the
    // skin from where it was at the build
    const float4 p0 = d.pos0[k];
    const float ex = p.x - p0.x, ey = p.y - p0.y, ez = p.z - p0.z;
    if (sq3(ex, ey, ez) > ph.skin2f) atomicOr(d.flags, FLAG_SKIN);
    p.w = record_w(I, tg & 1, drs);
    const float4 v = make_float4((float)us[0], (float)us[1], (float)us[2], 0.f);
    d.pos[k] = p;
    d.velq[k] = v;
    // a non-finite FP64 state gives non-finite FP32 records
    if (!(isfinite(drs) && finite4(p) && finite4(v))) atomicOr(d.flags, FLAG_NONFINITE);
}

// Corrector: x^{n+1} = x^n + dt u*, u^{n+1} = u^n + dt a*, rho^{n+1} = rho^n +
// dt Drho*, in the FP64 accumulators (walls keep x and u).  Writes the
// stage-1 records of the next step and decides whether it rebuilds the lists.
template <int DIM>
__device__ __forceinline__ void correct_particle(const Dev &d, const Grid &g, const Phys &ph, const Inst &I, int k,
                                                 float4 a, double dt)
{
    if (k == 0) {
        const long long next = *d.step + 1;
        *d.step = next;
        if (ph.rebuild_every > 0 && next % ph.rebuild_every == 0) *d.rebuild = 1u;
    }
    const uint8_t tg = d.tag[k];
    const float dr = fmaf((float)dt, a.w, d.drho[k]);
    d.drho[k] = dr;
    double xa[3] = {0, 0, 0}, ua[3] = {0, 0, 0};
    const float4 us = d.velq[k];
    const double usa[3] = {us.x, us.y, us.z};
    const double af[3] = {a.x, a.y, a.z};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        xa[c] = d.x[(size_t)c * d.n + k];
        ua[c] = d.u[(size_t)c * d.n + k];
        if (!(tg & 2)) {
            xa[c] = fma(dt, usa[c], xa[c]);
            ua[c] = fma(dt, af[c], ua[c]);
            d.x[(size_t)c * d.n + k] = xa[c];
            d.u[(size_t)c * d.n + k] = ua[c];
        }
    }
    if (tg & 4) {
        // piston: at X(t + dt) with velocity X'(t + dt) along its axis
        const Motion &m = *d.motion;
        const double t = d.clock[0];
        const double dX = motion_disp(m, t + dt) - motion_disp(m, t), U = motion_vel(m, t + dt);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            if (c == m.axis) xa[c] += dX;
            ua[c] = c == m.axis ? U : 0.0;
            d.x[(size_t)c * d.n + k] = xa[c];
            d.u[(size_t)c * d.n + k] = ua[c];
        }
    }
    // stage-1 records of the next step (replaced by the gather if it rebuilds);
    // a non-finite FP64 state gives non-finite FP32 records
    float4 p, v;
    const bool finite = stage_records<DIM>(d, g, I, k, d.cell[k], xa, ua, dr, tg & 1, &p, &v);
    if (!(finite && isfinite(dr))) atomicOr(d.flags, FLAG_NONFINITE);
    if (ph.rebuild_every == 0 && (!(tg & 2) || (tg & 4))) {
        // next step's stage positions: x^{n+1} and x^{n+1} + dt/2 u^{n+1};
        // rebuild before either can be farther than the skin from the build
        const float4 p0 = d.pos0[k];
        const float hdt = 0.5f * (float)dt;
        const float hx = __fmul_rn(hdt, v.x), hy = __fmul_rn(hdt, v.y), hz = __fmul_rn(hdt, v.z);
        const float ex = p.x - p0.x, ey = p.y - p0.y, ez = p.z - p0.z;
        const float d1 = sq3(ex, ey, ez);
        const float d2 = sq3(ex + hx, ey + hy, ez + hz);
        const float lim = ph.skin98f;
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
// The pair loop of sweep A for particle i.  MIXED: the list may hold
// other-phase particles (colour gradient, phase test per pair); otherwise
// every entry is same-phase.  The renormalisation sums are compensated per
// chunk of list entries: the chunk's terms are summed with FMAs, and the
// chunk sum enters the Kahan sums (s, c).
// The pair sums of sweep A over particle i's list.  Each neighbour's volume
// comes from its record (rec_vol) with the constants of its phase: own
// (vol0, irho0) for the renormalisation, the other phase's (vol0_o,
// irho0_o) for the colour gradient.
template <int DIM, bool NC, bool MIXED>
__device__ __forceinline__ void sweep_a_pairs(const Dev &d, const Grid &g, const Phys &ph, int i, const float4 &oi,
                                              int phi_, int renorm, float vol0, float irho0, float vol0_o,
                                              float irho0_o, float &s1, float &c1, float &s2, float &c2,
                                              float &gx, float &gy, float &gz)
{
    const float inv_h = ph.inv_h, cs = g.Es;
    const int n = d.n, cnt = d.ncnt[i];
    typename RO<NC, unsigned>::type col = d.nbr + i;
    typename RO<NC, float4>::type pos = d.pos;
    // the list holds whole chunks (padding entries feed zero terms)
    constexpr int CH = SPH_LIST_CHUNK;
    unsigned ec[CH];  // the first chunk lies inside the list storage (kmax >= CH) even when empty
#pragma unroll
    for (int c = 0; c < CH; ++c) ec[c] = ld_list<NC>(col + (size_t)c * n);
    for (int k0 = 0; k0 < cnt; k0 += CH) {
        unsigned en[CH];
        const bool more = k0 + CH < cnt;
#pragma unroll
        for (int c = 0; c < CH; ++c) en[c] = more ? ld_list<NC>(col + (size_t)(k0 + CH + c) * n) : 0u;
        float p1 = 0.f, p2 = 0.f;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const unsigned e = ec[c];
            const int j = (int)(e & NBR_IDX_MASK);
            if (!SPH_IN_RANGE(d.flags, j, n)) continue;
            const float4 oj = ld<NC>(pos + j);
            float rx, ry, rz;
            const float r2 = entry_vec<DIM>(oi, oj, e, cs, rx, ry, rz);
            // beyond the support (list entries in the skin) t clamps to 0 and
            // every kernel term vanishes
            const float r = pair_dist(r2);
            const float t = kernel_t(inv_h, r);
            const float t3 = t * t * t;
            const float vdj = rec_vd(oj.w);
            if (!MIXED || rec_phase(oj.w) == phi_) {
                if (renorm) {
                    // W / alpha_d = t^4 (2q + 1)
                    const float w = t3 * t * fmaf(2.f * inv_h, r, 1.f);
                    p1 = fmaf(rec_vol(vdj, vol0, irho0), w, p1);
                    p2 = fmaf(vdj, w, p2);
                }
            } else {
                const float vj = rec_vol(vdj, vol0_o, irho0_o);
                const float cc = vj * vj * t3;
                gx = fmaf(cc, rx, gx);
                gy = fmaf(cc, ry, gy);
                if (DIM == 3) gz = fmaf(cc, rz, gz);
            }
        }
        if (renorm) {
            kahan_add(s1, c1, p1);
            kahan_add(s2, c2, p2);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) ec[c] = en[c];
    }
}

template <int DIM>
__device__ __forceinline__ void sweep_a_finish(const Dev &d, const Phys &ph, const Inst &I, int i, const float4 &oi,
                                               int phi_, float vol_in, float drho, float gx, float gy, float gz,
                                               float4 *vel_s, bool write_t = true);

// skip_mixed (stage 2): the particles with an other-phase neighbour are left
// to the warp-per-particle pass (sweep_a_mixed_warp).
template <int DIM, bool NC>
__device__ __forceinline__ void sweep_a_one(const Dev &d, const Grid &g, const Phys &ph, const float *drho_in,
                                            int renorm, bool skip_mixed, float4 *vel_s, int i)
{
    const bool other = d.nflag[i] & 1;
    if (skip_mixed && other) return;
    const float4 oi = d.pos[i];
    const int phi_ = rec_phase(oi.w);
    const Inst &I = d.inst[d.iid[i]];
    // boundary particles share the fluid's continuity equation (Sec. III),
    // whose discretisation includes Eq. ct_dist_3, so by default they are
    // renormalised as water; with renorm_walls off they keep the density
    // continuity gives them and only enter the fluid's sums as water
    const int renorm_i = renorm && (ph.renorm_walls || !(d.tag[i] & 2));
    const float vol0 = by_phase(phi_, I.vol0), irho0 = by_phase(phi_, I.inv_rho0);
    const float vol0_o = by_phase(phi_ ^ 1, I.vol0), irho0_o = by_phase(phi_ ^ 1, I.inv_rho0);
    // self term: W(0)/alpha_d = 1
    const float vdi = rec_vd(oi.w), vi = rec_vol(vdi, vol0, irho0);
    float s1 = vi, c1 = 0.f, s2 = vdi, c2 = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    // particles with no other-phase neighbour (the bulk) take the loop
    // without the per-pair phase test
    if (other)
        sweep_a_pairs<DIM, NC, true>(d, g, ph, i, oi, phi_, renorm_i, vol0, irho0, vol0_o, irho0_o, s1, c1, s2, c2,
                                     gx, gy, gz);
    else if (renorm_i)
        sweep_a_pairs<DIM, NC, false>(d, g, ph, i, oi, phi_, 1, vol0, irho0, vol0_o, irho0_o, s1, c1, s2, c2, gx,
                                      gy, gz);
    // at stage 2 a particle with no other-phase particle in its list keeps the
    // zero surface tensor that stage 1 wrote (no colour gradient either time)
    sweep_a_finish<DIM>(d, ph, I, i, oi, phi_, vi, renorm_i ? s2 / s1 : drho_in[i], gx, gy, gz, vel_s, !skip_mixed);
}

// Sweep A at stage 2 (no renormalisation: only the colour gradient) for a
// particle with an other-phase neighbour, by one whole warp: lane l takes the
// list entries l, l + 32, ... and the three sums are combined by a butterfly
// of shuffles (every lane ends with the same bits).  These particles are a
// thin shell around the interface; a thread each would leave most lanes of
// their warps idle while one walks a whole list.
template <int DIM, bool NC>
__device__ __forceinline__ void sweep_a_mixed_warp(const Dev &d, const Grid &g, const Phys &ph, const float *drho_in,
                                                   float4 *vel_s, int i, int lane)
{
    const float4 oi = d.pos[i];
    const int phi_ = rec_phase(oi.w);
    const Inst &I = d.inst[d.iid[i]];
    const float vol0_o = by_phase(phi_ ^ 1, I.vol0), irho0_o = by_phase(phi_ ^ 1, I.inv_rho0);
    const float inv_h = ph.inv_h, cs = g.Es;
    const int n = d.n, cnt = d.ncnt[i];
    typename RO<NC, float4>::type pos = d.pos;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    for (int k = lane; k < cnt; k += 32) {
        const unsigned e = ld_list<NC>(d.nbr + (size_t)k * n + i);
        const int j = (int)(e & NBR_IDX_MASK);
        if (!SPH_IN_RANGE(d.flags, j, n)) continue;
        const float4 oj = ld<NC>(pos + j);
        if (rec_phase(oj.w) == phi_) continue;
        float rx, ry, rz;
        const float r2 = entry_vec<DIM>(oi, oj, e, cs, rx, ry, rz);
        const float r = pair_dist(r2);
        const float t = kernel_t(inv_h, r);
        const float vj = rec_vol(rec_vd(oj.w), vol0_o, irho0_o);
        const float cc = vj * vj * (t * t * t);
        gx = fmaf(cc, rx, gx);
        gy = fmaf(cc, ry, gy);
        if (DIM == 3) gz = fmaf(cc, rz, gz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        if (DIM == 3) gz += __shfl_xor_sync(0xffffffffu, gz, o);
    }
    if (lane == 0)
        sweep_a_finish<DIM>(d, ph, I, i, oi, phi_, rec_vol(rec_vd(oi.w), by_phase(phi_, I.vol0), by_phase(phi_, I.inv_rho0)),
                            drho_in[i], gx, gy, gz, vel_s);
}

// Sweep A's per-particle tail: stage density, equation of state, surface
// tensor, and the records the force sweep gathers.
template <int DIM>
__device__ __forceinline__ void sweep_a_finish(const Dev &d, const Phys &ph, const Inst &I, int i, const float4 &oi,
                                               int phi_, float vol_in, float drho, float gx, float gy, float gz,
                                               float4 *vel_s, bool write_t)
{
    d.drho_eval[i] = drho;
    const float rho = by_phase(phi_, I.rho0) + drho;
    const float vol = by_phase(phi_, I.mass) / rho;
    const float P = eos_tait7(by_phase(phi_, I.beta), __fmul_rn(drho, by_phase(phi_, I.inv_rho0)));
    // grad C_i = sigma_i sum V_j^2 grad W_ij, sigma_i = 1/V_i (entry density)
    const float sc = ph.cF / vol_in;
    gx *= sc;
    gy *= sc;
    gz *= sc;
    const float n2 = sq3(gx, gy, gz);
    unsigned iface = 0u;
    float4 t4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 t2 = make_float2(0.f, 0.f);
    if (n2 > 0.f) {
        iface = 1u;
        // T sigma_i^-2 = alpha_s / |g| (|g|^2/d I - g g^T) V_i^2, V_i from the renormalised density
        const float kk = I.alpha_s * rsqrtf(n2) * vol * vol;
        const float iso = n2 * ph.inv_dim;
        if (DIM == 2) {
            t4 = make_float4(kk * fmaf(-gx, gx, iso), -kk * gx * gy, kk * fmaf(-gy, gy, iso), 0.f);
        } else {
            t4 = make_float4(kk * fmaf(-gx, gx, iso), -kk * gx * gy, -kk * gx * gz, kk * fmaf(-gy, gy, iso));
            t2 = make_float2(-kk * gy * gz, kk * fmaf(-gz, gz, iso));
        }
    }
    // signed volume (sign = phase) whose lowest mantissa bit carries the
    // interface flag: at most one unit in the last place, the size of the
    // rounding of m/rho itself
    const float vs = phi_ ? -vol : vol;
    d.posv[i] = make_float4(oi.x, oi.y, oi.z, __uint_as_float((__float_as_uint(vs) & ~1u) | iface));
    vel_s[i].w = by_phase(phi_, I.mass) * P / (rho * rho);  // m_i P_i / rho_i^2
    d.pres[i] = P;
    if (write_t) {
        d.T4[i] = t4;
        if (DIM == 3) d.T2[i] = t2;
    }
}

// Epilogue prefetch of the force sweep: the fused predictor (STAGE 1) and
// corrector (STAGE 2) read the particle's FP64 state and a few records at
// the very end of its thread's work, where their latency would add to the
// block's lifetime; they are prefetched to L2 (evict-last policy) when the
// thread starts.  (Measured: 1.4 % off the force sweep; the same prefetch to
// L1 two chunks before the end of the list loop made it 14 % slower.)
__device__ __forceinline__ void prefetch_l2_last(const void *p)
{
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(p));
}
template <int DIM, int STAGE>
__device__ __forceinline__ void prefetch_epilogue(const Dev &d, int k)
{
    const size_t n = (size_t)d.n;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        prefetch_l2_last(d.u + c * n + k);
        if (STAGE == 2) prefetch_l2_last(d.x + c * n + k);
    }
    prefetch_l2_last(d.pos0 + k);
    prefetch_l2_last(d.tag + k);
    if (STAGE == 1) prefetch_l2_last(d.drho_eval + k);
    if (STAGE == 2) {
        prefetch_l2_last(d.velq + k);
        prefetch_l2_last(d.drho + k);
        prefetch_l2_last(d.cell + k);
    }
}

// ---------------------------------------------------------------------------
// Sweep B: pressure gradient (Eq. dist_p_1), harmonic-mean viscosity
// (Eq. visc_2 or visc_1), surface tension (F_s/rho), gravity, continuity
// (Eq. ct_dist_2).  grad_i W_ij = cF t^3 r_ij with t = 1 - q/2; the common
// factor cF is applied once per particle.
// STAGE 0: rates only; 1: then the predictor; 2: then the corrector.
template <int DIM, int STAGE, bool NC>
__device__ __forceinline__ void sweep_b_one(const Dev &d, const Grid &g, const Phys &ph, double dt, int i)
{
    const float4 oi = d.posv[i];
    const int phi_ = phase_of(oi.w);
    const Inst &I = d.inst[d.iid[i]];
    const unsigned iface_i = __float_as_uint(oi.w) & 1u;
    typename RO<NC, float4>::type vel_s = STAGE == 2 ? d.velq : d.velp;
    const float4 ui = vel_s[i];              // w: m_i P_i / rho_i^2
    float px = 0.f, py = 0.f, pz = 0.f;    // sum m_j (P_i/rho_i^2 + P_j/rho_j^2) t^3 r_ij
    float vx = 0.f, vy = 0.f, vz = 0.f;    // sum k_ij V_j t^3 r^2/(r^2+delta^2) u_ij
    float sx = 0.f, sy = 0.f, sz = 0.f;    // sum (T_i/sigma_i^2 + T_j/sigma_j^2) . t^3 r_ij
    float dv = 0.f;                        // sum V_j t^3 u_ij . r_ij
    const float inv_h = ph.inv_h, cs = g.Es;
    // a static boundary particle's pairs with the others (at the end of its
    // list) add exact zeros while those are at rest: u_ij = 0 in the
    // continuity term, and the acceleration of a boundary particle is not used
    const int n = d.n, cnt = ld<NC>(d.walls_moving) ? d.ncnt[i] : d.nfcnt[i];
    if (STAGE != 0) prefetch_epilogue<DIM, STAGE>(d, i);
    // per-phase constants of the pair terms as registers (selected per pair):
    // m_j P_i / rho_i^2 for a water and an oil neighbour, and the viscous factors
    const float Pi = ui.w * by_phase(phi_, I.inv_mass);
    const float mP_wat = I.mass[0] * Pi, mP_oil = I.mass[1] * Pi;
    const float kv_wat = phi_ ? I.kvis[2] : I.kvis[0], kv_oil = phi_ ? I.kvis[3] : I.kvis[1];
    typename RO<NC, unsigned>::type col = d.nbr + i;
    typename RO<NC, float4>::type posv = d.posv;
    typename RO<NC, float4>::type T4 = d.T4;
    typename RO<NC, float2>::type T2 = d.T2;
    // the list holds whole chunks (padding entries feed zero terms)
    constexpr int CH = SPH_LIST_CHUNK;
    unsigned ec[CH];  // the first chunk lies inside the list storage (kmax >= CH) even when empty
#pragma unroll
    for (int c = 0; c < CH; ++c) ec[c] = ld_list<NC>(col + (size_t)c * n);
    for (int k0 = 0; k0 < cnt; k0 += CH) {
        unsigned en[CH];
        const bool more = k0 + CH < cnt;
#pragma unroll
        for (int c = 0; c < CH; ++c) en[c] = more ? ld_list<NC>(col + (size_t)(k0 + CH + c) * n) : 0u;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const unsigned e = ec[c];
            const int j = (int)(e & NBR_IDX_MASK);
            if (!SPH_IN_RANGE(d.flags, j, n)) continue;
            const float4 oj = ld<NC>(posv + j);
            const float4 uj = ld<NC>(vel_s + j);
            float rx, ry, rz;
            const float r2 = entry_vec<DIM>(oi, oj, e, cs, rx, ry, rz);
            const bool oil_j = oj.w < 0.f;
            const float vol_j = fabsf(oj.w);
            // beyond the support (list entries in the skin) t clamps to 0 and
            // every pair term below vanishes
            const float r = pair_dist(r2);
            const float t = kernel_t(inv_h, r);
            const float t3 = t * t * t;
            // m_j (P_i/rho_i^2 + P_j/rho_j^2) t^3 with the record's m_j P_j / rho_j^2
            const float pt = ((oil_j ? mP_oil : mP_wat) + uj.w) * t3;
            px = fmaf(pt, rx, px);
            py = fmaf(pt, ry, py);
            if (DIM == 3) pz = fmaf(pt, rz, pz);
            const float ux = ui.x - uj.x, uy = ui.y - uj.y, uz = DIM == 3 ? ui.z - uj.z : 0.f;
            const float vt = vol_j * t3;
            const float s = (oil_j ? kv_oil : kv_wat) * vt * __fdividef(r2, r2 + ph.delta2);
            vx = fmaf(s, ux, vx);
            vy = fmaf(s, uy, vy);
            if (DIM == 3) vz = fmaf(s, uz, vz);
            float ur = __fmul_rn(ux, rx);
            ur = fmaf(uy, ry, ur);
            if (DIM == 3) ur = fmaf(uz, rz, ur);
            dv = fmaf(vt, ur, dv);
            if ((iface_i | (__float_as_uint(oj.w) & 1u)) != 0u) {
                // interface pairs are few: the particle's own tensor is re-read
                // here (an L1 hit) rather than held in six registers
                const float4 Ti = ld<NC>(T4 + i);
                const float2 Ti2 = DIM == 3 ? ld<NC>(T2 + i) : make_float2(0.f, 0.f);
                const float4 Tj = ld<NC>(T4 + j);
                if (DIM == 2) {
                    const float xx = Ti.x + Tj.x, xy = Ti.y + Tj.y, yy = Ti.z + Tj.z;
                    sx = fmaf(t3, fmaf(xy, ry, __fmul_rn(xx, rx)), sx);
                    sy = fmaf(t3, fmaf(yy, ry, __fmul_rn(xy, rx)), sy);
                } else {
                    const float2 Tj2 = ld<NC>(T2 + j);
                    const float xx = Ti.x + Tj.x, xy = Ti.y + Tj.y, xz = Ti.z + Tj.z;
                    const float yy = Ti.w + Tj.w, yz = Ti2.x + Tj2.x, zz = Ti2.y + Tj2.y;
                    sx = fmaf(t3, fmaf(xz, rz, fmaf(xy, ry, __fmul_rn(xx, rx))), sx);
                    sy = fmaf(t3, fmaf(yz, rz, fmaf(yy, ry, __fmul_rn(xy, rx))), sy);
                    sz = fmaf(t3, fmaf(zz, rz, fmaf(yz, ry, __fmul_rn(xz, rx))), sz);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) ec[c] = en[c];
    }
    const float rho = by_phase(phi_, I.rho0) + d.drho_eval[i];
    float4 out;
    out.w = rho * ph.cF * dv;
    if (d.tag[i] & 2) {
        out.x = out.y = out.z = 0.f;
    } else {
        const float vf = ph.visc_dynamic ? ph.cF / rho : ph.cF;
        const float sf = ph.cF * by_phase(phi_, I.inv_mass);
        out.x = fmaf(sf, sx, fmaf(vf, vx, __fmul_rn(-ph.cF, px))) + ph.gf[0];
        out.y = fmaf(sf, sy, fmaf(vf, vy, __fmul_rn(-ph.cF, py))) + ph.gf[1];
        out.z = DIM == 3 ? fmaf(sf, sz, fmaf(vf, vz, __fmul_rn(-ph.cF, pz))) + ph.gf[2] : 0.f;
    }
    d.acc[i] = out;
    if (STAGE == 1) predict_particle<DIM>(d, g, ph, I, i, out, dt * I.dt_scale, oi, ui);
    if (STAGE == 2) {
        correct_particle<DIM>(d, g, ph, I, i, out, dt * I.dt_scale);
        // the clock advances when the next step starts (every particle of
        // this launch reads clock[0] as t_n)
        if (i == 0) d.clock[1] = dt;
    }
}

__device__ __forceinline__ int renorm_now(const Dev &d, const Phys &ph, int stage1)
{
    return stage1 && ph.renorm_every > 0 && (*d.step % ph.renorm_every) == 0;
}

// ---------------------------------------------------------------------------
// One kernel per phase.  The cell-list kernels return at once unless the
// device flag `rebuild` is set.

template <int DIM>
static __global__ void __launch_bounds__(256) k_hash(Dev d, Grid g, Sort s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n || !*d.rebuild) return;
    hash_one<DIM>(d, g, s, k);
}

static __global__ void __launch_bounds__(256) k_zero(int *a, int m, const unsigned *rebuild)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && *rebuild) a[i] = 0;
}

static __global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const int *in, int *out, int *tile_sums, int m,
                                                              const unsigned *rebuild)
{
    if (!*rebuild) return;
    const int t = scan_tile(in, out, m, blockIdx.x);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

// Scans the tile sums in place (one block) and writes the grand total to out[m].
static __global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(int *tile_sums, int ntiles, int *out, int m,
                                                             const unsigned *rebuild)
{
    if (!*rebuild) return;
    scan_tile_sums(tile_sums, ntiles, out, m);
}

static __global__ void __launch_bounds__(256) k_scan_add(int *out, const int *tile_sums, int m, const unsigned *rebuild)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m && *rebuild) out[i] += tile_sums[i / SCAN_TILE];
}

static __global__ void __launch_bounds__(256) k_scatter(int n, Sort s, const int *cstart, const unsigned *rebuild)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || !*rebuild) return;
    scatter_one(s, cstart, k);
}

static __global__ void __launch_bounds__(256) k_rank(int n, Sort s, const int *pid, const int *cstart,
                                              const unsigned *rebuild)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !*rebuild) return;
    rank_one(s, pid, cstart, p);
}

template <int DIM>
static __global__ void __launch_bounds__(256) k_gather(Dev src, Dev dst, Grid g, Sort s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= src.n || !*src.rebuild) return;
    gather_one<DIM>(src, dst, g, s, k);
}

template <int DIM>
static __global__ void __launch_bounds__(256) k_copy_back(Dev src, Dev dst)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= src.n || !*dst.rebuild) return;
    copy_one<DIM>(src, dst, k);
}

template <int DIM>
static __global__ void __launch_bounds__(256, 4) k_build_list(Dev d, Grid g, Phys ph)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n || !*d.rebuild) return;
    if (i == 0) *d.builds += 1;
    list_one<DIM, true>(d, g, ph, i);
}

// Threads per block of the stage-1 sweep A.
#ifndef SPH_SWEEP_A_THREADS
#define SPH_SWEEP_A_THREADS 256
#endif
template <int DIM>
static __global__ void __launch_bounds__(SPH_SWEEP_A_THREADS)
    k_sweep_a(Dev d, Grid g, Phys ph, const float *__restrict__ drho_in, int stage1, float4 *vel_s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int renorm = renorm_now(d, ph, stage1);
    // the lists built for this step are in place; the corrector decides the next build
    if (stage1 && i == 0) {
        *d.rebuild = 0u;
        d.clock[0] += d.clock[1];
        d.clock[1] = 0.0;
    }
    sweep_a_one<DIM, true>(d, g, ph, drho_in, renorm, false, vel_s, i);
}

// Warps [0, 8 mixed_blocks) of the launch take the mixed particles one at a
// time (warp-stride over the mixed list).
template <int DIM, bool NC>
__device__ __forceinline__ void mixed_pass(const Dev &d, const Grid &g, const Phys &ph, const float *drho_in,
                                           float4 *vel_s, int warp, int nwarps, int lane)
{
    const int nm = min(*d.nmixed, d.n);
    for (int w = warp; w < nm; w += nwarps) {
        const int i = d.mixed[w];
        if (!SPH_IN_RANGE(d.flags, i, d.n)) continue;
        sweep_a_mixed_warp<DIM, NC>(d, g, ph, drho_in, vel_s, i, lane);
    }
}

// Sweep A at stage 2: the first mixed_blocks blocks run the warp-per-particle
// pass over the mixed particles (launched first, so it overlaps the rest),
// the others a thread per particle for the remaining ones.
template <int DIM>
static __global__ void __launch_bounds__(256) k_sweep_a2(Dev d, Grid g, Phys ph, const float *__restrict__ drho_in,
                                                  float4 *vel_s, int mixed_blocks)
{
    if ((int)blockIdx.x < mixed_blocks) {
        mixed_pass<DIM, true>(d, g, ph, drho_in, vel_s, (int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                              (int)(mixed_blocks * blockDim.x) >> 5, (int)threadIdx.x & 31);
        return;
    }
    const int i = (int)(blockIdx.x - mixed_blocks) * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    sweep_a_one<DIM, true>(d, g, ph, drho_in, 0, true, vel_s, i);
}

// Threads per block of the force sweep and the resident blocks per SM it is
// compiled for (1024 threads an SM: up to 64 registers a thread).
#ifndef SPH_SWEEP_B_THREADS
#define SPH_SWEEP_B_THREADS 256
#endif
#ifndef SPH_SWEEP_B_MIN_BLOCKS
#define SPH_SWEEP_B_MIN_BLOCKS (1024 / SPH_SWEEP_B_THREADS)
#endif
template <int DIM, int STAGE>
static __global__ void __launch_bounds__(SPH_SWEEP_B_THREADS, SPH_SWEEP_B_MIN_BLOCKS)
    k_sweep_b(Dev d, Grid g, Phys ph, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    sweep_b_one<DIM, STAGE, true>(d, g, ph, dt, i);
}

// ---------------------------------------------------------------------------
// Persistent form: one cooperative launch runs whole steps, every phase a
// grid-stride loop, phases separated by a grid barrier that gives up after
// one second (the launch then sets FLAG_TIMEOUT and returns).

struct GridBarrier {
    unsigned count;     // blocks arrived at the current barrier
    unsigned gen;       // barrier generation
    unsigned snapshot;  // error flags seen by the last arriving block
    unsigned work;      // next 32-particle chunk of the current phase (reset by each barrier)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier.  Thread 0 of each block arrives with a release-acquire
// add (the block's writes, ordered before it by the block barrier, become
// visible to whoever acquires later); the last block to arrive records the
// error flags, resets the arrival and chunk counters and publishes a new
// generation with a release store, which the others poll with acquire loads.
// Returns the error flags as they stood when the last block arrived (the same
// value in every block), plus FLAG_TIMEOUT if this block gave up waiting.
__device__ __forceinline__ unsigned grid_sync(GridBarrier *b, unsigned *flags)
{
    __shared__ unsigned s_snap;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the generation cannot advance before this block has arrived
        const unsigned g0 = ld_acquire_gpu(&b->gen);
        const unsigned arrived = atom_add_acq_rel_gpu(&b->count, 1u);
        unsigned mine = 0u;
        if (arrived == gridDim.x - 1) {
            b->snapshot = *(volatile unsigned *)flags;
            atomicExch(&b->work, 0u);
            atomicExch(&b->count, 0u);
            st_release_gpu(&b->gen, g0 + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(&b->gen) == g0) {
                __nanosleep(32);
                if (global_ns() - t0 > 1000000000ull) {
                    atomicOr(flags, FLAG_TIMEOUT);
                    mine = FLAG_TIMEOUT;
                    break;
                }
            }
        }
        s_snap = *(volatile unsigned *)&b->snapshot | mine;
    }
    __syncthreads();
    return s_snap;
}

// Calls f(i) for every particle i < n, handing out chunks of consecutive
// particles (32 a sub-chunk, one particle a lane) to warps from a grid-wide
// counter: warps that finish early take more chunks, so a phase ends with at
// most one chunk in flight per warp instead of a fixed share per thread.  The
// barrier before the phase resets the counter.
template <class F>
__device__ __forceinline__ void for_each_chunk(GridBarrier *bar, int n, F &&f)
{
    const int lane = threadIdx.x & 31;
    // tickets of m x 32 particles, m chosen so each thread takes about eight
    // tickets a phase (few atomics on large inputs, a short tail on small ones)
    const int m = max(1, n / (int)(gridDim.x * blockDim.x * 8u));
    for (;;) {
        unsigned c = 0u;
        if (lane == 0) c = atomicAdd(&bar->work, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        const long long base = (long long)c * 32 * m;
        if (base >= n) break;
        for (int k = 0; k < m; ++k) {
            const long long i = base + 32 * k + lane;
            if (i < n) f((int)i);
        }
    }
}

// Particle loop of one phase: dynamic chunks (above) or, with dyn == 0, a
// fixed grid-stride share per thread.
template <class F>
__device__ __forceinline__ void for_each_particle(GridBarrier *bar, int n, int dyn, F &&f)
{
    if (dyn) {
        for_each_chunk(bar, n, f);
    } else {
        const int stride = gridDim.x * blockDim.x;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) f(i);
    }
}

// Body of the persistent kernel (instantiated per block size by the host
// file): nsteps whole steps; returns early, in every block, once an error
// flag is raised or a barrier times out.
template <int DIM>
__device__ __forceinline__ void persistent_steps(Dev d, Dev scratch, Grid g, Phys ph, Sort s, GridBarrier *bar,
                                                 double dt, int nsteps, int dyn)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    const int n = d.n;
    if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
    for (int step = 0; step < nsteps; ++step) {
        // every block reads the flag after the barrier that closed the last step
        if (*(volatile unsigned *)d.rebuild) {
            for (int c = tid; c < s.ncell; c += stride) s.count[c] = 0;
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int k = tid; k < n; k += stride) hash_one<DIM>(d, g, s, k);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            const int ntiles = (s.ncell + SCAN_TILE - 1) / SCAN_TILE;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const int tot = scan_tile(s.count, d.cstart, s.ncell, t);
                if (threadIdx.x == 0) s.tile_sums[t] = tot;
            }
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            if (blockIdx.x == 0) scan_tile_sums(s.tile_sums, ntiles, d.cstart, s.ncell);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int c = tid; c < s.ncell; c += stride) d.cstart[c] += s.tile_sums[c / SCAN_TILE];
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int k = tid; k < n; k += stride) scatter_one(s, d.cstart, k);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int p = tid; p < n; p += stride) rank_one(s, d.pid, d.cstart, p);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int k = tid; k < n; k += stride) gather_one<DIM>(d, scratch, g, s, k);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            for (int k = tid; k < n; k += stride) copy_one<DIM>(scratch, d, k);
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
            if (tid == 0) *d.builds += 1;
            for_each_particle(bar, n, dyn, [&](int i) { list_one<DIM, false>(d, g, ph, i); });
            if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
        }
        const int renorm = renorm_now(d, ph, 1);
        if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;  // all blocks read rebuild and step
        if (tid == 0) {
            *d.rebuild = 0u;
            d.clock[0] += d.clock[1];
            d.clock[1] = 0.0;
        }
        for_each_particle(bar, n, dyn, [&](int i) { sweep_a_one<DIM, false>(d, g, ph, d.drho, renorm, false, d.velp, i); });
        if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
        for_each_particle(bar, n, dyn, [&](int i) { sweep_b_one<DIM, 1, false>(d, g, ph, dt, i); });
        if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
        for_each_particle(bar, n, dyn, [&](int i) { sweep_a_one<DIM, false>(d, g, ph, d.drho_stage, 0, true, d.velq, i); });
        mixed_pass<DIM, false>(d, g, ph, d.drho_stage, d.velq, tid >> 5, stride >> 5, (int)threadIdx.x & 31);
        if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
        for_each_particle(bar, n, dyn, [&](int i) { sweep_b_one<DIM, 2, false>(d, g, ph, dt, i); });
        if (grid_sync(bar, d.flags) & FLAG_ERRORS) return;
    }
}

// ---------------------------------------------------------------------------
// Neighbour sets and pair statistics by the sweeps' own support test.

template <int DIM>
static __global__ void __launch_bounds__(256) k_nbr_count(Dev d, Grid g, Phys ph, int *count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float4 oi = d.pos[i];
    int cnt = 0;
    for_each_candidate<DIM, true>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                                  [&](int j, const float4 &, float, float, float, float, unsigned) { cnt += j != i; });
    count[i] = cnt;
}

template <int DIM>
static __global__ void __launch_bounds__(256) k_nbr_fill(Dev d, Grid g, Phys ph, const long long *start, int *list)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const float4 oi = d.pos[i];
    long long w = start[i];
    for_each_candidate<DIM, true>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                                  [&](int j, const float4 &, float, float, float, float, unsigned) {
                                      if (j != i) list[w++] = d.pid[j];
                                  });
}

// Totals of ordered neighbour pairs (j != i): [0] all, [1] of different phase.
template <int DIM>
static __global__ void __launch_bounds__(256) k_pair_stats(Dev d, Grid g, Phys ph, unsigned long long *tot)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // ordered pairs: all, across phases, both static boundary particles, a
    // static boundary particle i with any other j
    int c[4] = {0, 0, 0, 0};
    if (i < d.n) {
        const float4 oi = d.pos[i];
        const int phi_ = rec_phase(oi.w);
        const bool si = static_wall(d.tag[i]);
        for_each_candidate<DIM, true>(g, d.cstart, d.pos, d.cell[i], oi, ph.R2, ph.RP,
                                      [&](int j, const float4 &oj, float, float, float, float, unsigned) {
                                          if (j == i) return;
                                          const bool sj = static_wall(d.tag[j]);
                                          c[0] += 1;
                                          c[1] += rec_phase(oj.w) != phi_;
                                          c[2] += si && sj;
                                          c[3] += si && !sj;
                                      });
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
        if ((threadIdx.x & 31) == 0) atomicAdd(tot + q, (unsigned long long)c[q]);
    }
}

// ---------------------------------------------------------------------------
// Output in original order; positions in each instance's own frame.

enum ReadKind { RK_X, RK_U, RK_RHO, RK_RHO_EVAL, RK_P, RK_ACC, RK_DRHO, RK_T, RK_CELL, RK_ORDER, RK_TAG };

template <int DIM>
static __global__ void __launch_bounds__(256) k_unpermute(Dev d, int kind, double *out, int *iout)
{
    // one thread per original id: the output is written in order (coalesced),
    // the sorted state is gathered
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n) return;
    const int n = d.n;
    const int k = d.inv[p];
    if (!SPH_IN_RANGE(d.flags, k, n)) return;
    const int phs = d.tag[k] & 1;
    const Inst &I = d.inst[d.iid[k]];
    switch (kind) {
    case RK_X:
        // periodic coordinates in the box (between builds they may lie up to
        // the skin beyond it)
        for (int c = 0; c < DIM; ++c)
            out[(size_t)p * DIM + c] = wrap_coord(d.x[(size_t)c * n + k], d.plo[c], d.period[c]) - I.offset[c];
        break;
    case RK_U:
        for (int c = 0; c < DIM; ++c) out[(size_t)p * DIM + c] = d.u[(size_t)c * n + k];
        break;
    case RK_RHO:
        out[p] = (double)by_phase(phs, I.rho0) + (double)d.drho[k];
        break;
    case RK_RHO_EVAL:
        out[p] = (double)by_phase(phs, I.rho0) + (double)d.drho_eval[k];
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
        const double v = (double)(by_phase(phs, I.mass) / (by_phase(phs, I.rho0) + d.drho_eval[k]));
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
    case RK_TAG:
        iout[p] = d.tag[k];
        break;
    }
}

// The state (x, u, rho) in original order written straight into host memory
// the GPU can address (pinned, mapped), in whole lines: a block takes 256
// consecutive particles, gathers their values from the sorted state into
// shared memory in the output's particle-major layout, and writes each
// field's contiguous stretch with 16-byte stores (x and u must start on a
// 16-byte boundary); rho, one double a particle, is contiguous across a warp
// already.  Scattered 8-byte stores at a 24-byte stride, as k_unpermute
// makes, reach a third of the host link's rate; whole-line stores reach the
// copy engines' rate, with no staging copy after the kernel.
constexpr int RS_TILE = 256;
template <int DIM>
static __global__ void __launch_bounds__(RS_TILE) k_read_state_lines(Dev d, double *x, double *u, double *rho)
{
    __shared__ double sx[RS_TILE * DIM], su[RS_TILE * DIM];
    const int n = d.n;
    const int p0 = blockIdx.x * RS_TILE, t = threadIdx.x;
    const int cnt = min(RS_TILE, n - p0);
    if (t < cnt) {
        const int p = p0 + t;
        const int k = d.inv[p];
        if (SPH_IN_RANGE(d.flags, k, n)) {
            const Inst &I = d.inst[d.iid[k]];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                sx[t * DIM + c] = wrap_coord(d.x[(size_t)c * n + k], d.plo[c], d.period[c]) - I.offset[c];
                su[t * DIM + c] = d.u[(size_t)c * n + k];
            }
            rho[p] = (double)by_phase(d.tag[k] & 1, I.rho0) + (double)d.drho[k];
        } else {
#pragma unroll
            for (int c = 0; c < DIM; ++c) sx[t * DIM + c] = su[t * DIM + c] = 0.0;
        }
    }
    __syncthreads();
    const int m = cnt * DIM;  // doubles of the tile in each of x and u
    double2 *x2 = reinterpret_cast<double2 *>(x + (size_t)p0 * DIM);
    double2 *u2 = reinterpret_cast<double2 *>(u + (size_t)p0 * DIM);
    for (int q = t; q < m / 2; q += RS_TILE) {
        x2[q] = make_double2(sx[2 * q], sx[2 * q + 1]);
        u2[q] = make_double2(su[2 * q], su[2 * q + 1]);
    }
    if ((m & 1) && t == 0) {
        x[(size_t)p0 * DIM + m - 1] = sx[m - 1];
        u[(size_t)p0 * DIM + m - 1] = su[m - 1];
    }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics of each instance: one block per instance reduces, in a
// fixed tree order, over the instance's fluid particles taken in original
// order from arrays written by k_unpermute (positions in the instance frame,
// velocities, tags).  Per instance, DIAG_STRIDE doubles:
//   [0] mass, [1..3] momentum sum m u, [4] kinetic energy, [5] potential
//   energy -sum m g.x, [6..8] oil centroid, [9] oil count, [10] max |u|,
//   [11..16] oil position covariance about the centroid (xx xy xz yy yz zz).
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_STRIDE = 20;

__device__ __forceinline__ double block_reduce(double v, double *sm, bool is_max)
{
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            sm[threadIdx.x] = is_max ? fmax(sm[threadIdx.x], sm[threadIdx.x + s]) : sm[threadIdx.x] + sm[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sm[0];
    __syncthreads();
    return r;
}

template <int DIM>
static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_inst(const long long *first, const double *x, const double *u,
                                                            const int *tag, const Inst *inst, const double *grav,
                                                            double *out)
{
    __shared__ double sm[DIAG_THREADS];
    const int q = blockIdx.x;
    const long long b = first[q], e = first[q + 1];
    const Inst &I = inst[q];
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // m, mu xyz, ekin, epot, oil sum xyz, oil count
    double umax = 0.0;
    for (long long k = b + threadIdx.x; k < e; k += DIAG_THREADS) {
        const int tg = tag[k];
        if (tg & 2) continue;
        const int oil = tg & 1;
        const double m = oil ? I.mass64[1] : I.mass64[0];
        double u2 = 0.0, gx = 0.0;
        for (int c = 0; c < DIM; ++c) {
            const double uc = u[k * DIM + c], xc = x[k * DIM + c];
            acc[1 + c] += m * uc;
            u2 += uc * uc;
            gx += grav[c] * xc;
            if (oil) acc[6 + c] += xc;
        }
        acc[0] += m;
        acc[4] += 0.5 * m * u2;
        acc[5] -= m * gx;
        acc[9] += oil;
        umax = fmax(umax, sqrt(u2));
    }
    double tot[10];
#pragma unroll 1
    for (int c = 0; c < 10; ++c) tot[c] = block_reduce(acc[c], sm, false);
    const double vmax = block_reduce(umax, sm, true);
    double cen[3] = {0, 0, 0};
    if (tot[9] > 0)
        for (int c = 0; c < DIM; ++c) cen[c] = tot[6 + c] / tot[9];
    double cv[6] = {0, 0, 0, 0, 0, 0};
    for (long long k = b + threadIdx.x; k < e; k += DIAG_THREADS) {
        const int tg = tag[k];
        if ((tg & 2) || !(tg & 1)) continue;
        double r[3] = {0, 0, 0};
        for (int c = 0; c < DIM; ++c) r[c] = x[k * DIM + c] - cen[c];
        cv[0] += r[0] * r[0];
        cv[1] += r[0] * r[1];
        cv[2] += r[0] * r[2];
        cv[3] += r[1] * r[1];
        cv[4] += r[1] * r[2];
        cv[5] += r[2] * r[2];
    }
    double ctot[6];
#pragma unroll 1
    for (int c = 0; c < 6; ++c) ctot[c] = block_reduce(cv[c], sm, false);
    if (threadIdx.x == 0) {
        double *o = out + (size_t)q * DIAG_STRIDE;
        for (int c = 0; c < 6; ++c) o[c] = tot[c];
        for (int c = 0; c < 3; ++c) o[6 + c] = cen[c];
        o[9] = tot[9];
        o[10] = vmax;
        for (int c = 0; c < 6; ++c) o[11 + c] = ctot[c];
    }
}

}  // namespace sphgb
