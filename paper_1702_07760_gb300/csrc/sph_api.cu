// Host side of the C ABI declared in include/sph.h: parameter validation,
// device memory, the per-step launch sequence, CUDA-graph replay, reads in
// original particle order, FP64 diagnostics and per-kernel event timing.
#include "sph.h"
#include "sph_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace sphgb;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CU(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(SPH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

enum KernelId {
    KI_MEMSET, KI_HASH, KI_SCAN, KI_SCATTER, KI_RANK, KI_GATHER, KI_COPY, KI_LIST, KI_SWEEP_A, KI_SWEEP_B,
    KI_COUNT
};
// sweep_b includes the predictor (stage 1) or the corrector (stage 2)
const char *k_names[KI_COUNT] = {"count_reset", "cell_hash", "cell_scan", "cell_scatter",
                                 "cell_rank", "reorder_gather", "reorder_copy", "neighbour_list",
                                 "sweep_a", "sweep_b"};

struct PendingTiming {
    int id;
    cudaEvent_t a, b;
};

}  // namespace

struct sph_sim {
    sph_params P{};
    int dim = 0;
    int n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Grid grid{};
    Phys phys{};
    int ncell = 0;
    int ntiles = 0;
    Dev buf[2]{};
    int cur = 0;
    int *cell_tmp = nullptr, *slot = nullptr, *count = nullptr, *tmp = nullptr, *perm = nullptr,
        *tile_sums = nullptr;
    unsigned *flags = nullptr;
    unsigned *rebuild = nullptr;
    long long *dstep = nullptr;
    long long *dbuilds = nullptr;
    double last_dt = 0.0;
    double *diag_partial = nullptr, *diag_small = nullptr;
    double *read_buf = nullptr;
    int *read_ibuf = nullptr;
    int64_t step = 0;
    std::vector<void *> allocs;
    // timing
    bool timing = false;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> free_events;
    int64_t t_launches[KI_COUNT] = {};
    double t_ms[KI_COUNT] = {};
    // graph of one step (gexec[0]), replayed while dt matches gdt[0]
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    double gdt[2] = {0.0, 0.0};

    Dev &D() { return buf[cur]; }

    template <class T>
    int alloc(T **p, size_t count_) {
        void *q = nullptr;
        if (count_ == 0) count_ = 1;
        cudaError_t e = cudaMalloc(&q, count_ * sizeof(T));
        if (e != cudaSuccess) {
            *p = nullptr;
            return fail(SPH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = static_cast<T *>(q);
        return SPH_OK;
    }

    cudaEvent_t get_event() {
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    // Launch wrapper: brackets the launch with events when timing is enabled.
    template <class L>
    void launch(int id, L &&l) {
        if (timing) {
            PendingTiming p{id, get_event(), get_event()};
            cudaEventRecord(p.a, stream);
            l();
            cudaEventRecord(p.b, stream);
            pending.push_back(p);
        } else {
            l();
        }
    }

    void collect_timing() {
        for (auto &p : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                t_ms[p.id] += ms;
                t_launches[p.id] += 1;
            }
            free_events.push_back(p.a);
            free_events.push_back(p.b);
        }
        pending.clear();
    }

    int blocks(int work, int threads = 256) const { return (work + threads - 1) / threads; }

    void enqueue_build_cells(bool force);
    void enqueue_eval(int stage, const float *drho_in, double dt);
    void enqueue_step(double dt);
    int check_flags();
};

// Cell hash, stable sort, reorder and neighbour list.  Every kernel returns
// at once unless the device flag `rebuild` is set (by the corrector when a
// particle may leave the skin, or here when force is true), so the same
// launch sequence serves every step of a captured graph.
void sph_sim::enqueue_build_cells(bool force)
{
    Dev &s = buf[0];
    Dev &t = buf[1];
    if (force) cudaMemsetAsync(rebuild, 0xff, sizeof(unsigned), stream);
    launch(KI_MEMSET, [&] { k_zero<<<blocks(ncell), 256, 0, stream>>>(count, ncell, rebuild); });
    launch(KI_HASH, [&] {
        if (dim == 2) k_hash<2><<<blocks(n), 256, 0, stream>>>(s, grid, cell_tmp, slot, count);
        else k_hash<3><<<blocks(n), 256, 0, stream>>>(s, grid, cell_tmp, slot, count);
    });
    launch(KI_SCAN, [&] {
        k_scan_tiles<<<ntiles, SCAN_THREADS, 0, stream>>>(count, s.cstart, tile_sums, ncell, rebuild);
        k_scan_sums<<<1, SCAN_THREADS, 0, stream>>>(tile_sums, ntiles, s.cstart, ncell, rebuild);
        k_scan_add<<<blocks(ncell), 256, 0, stream>>>(s.cstart, tile_sums, ncell, rebuild);
    });
    launch(KI_SCATTER, [&] { k_scatter<<<blocks(n), 256, 0, stream>>>(n, cell_tmp, slot, s.cstart, tmp, rebuild); });
    launch(KI_RANK, [&] { k_rank<<<blocks(n), 256, 0, stream>>>(n, tmp, cell_tmp, s.pid, s.cstart, perm, rebuild); });
    launch(KI_GATHER, [&] {
        if (dim == 2) k_gather<2><<<blocks(n), 256, 0, stream>>>(s, t, grid, phys, perm, cell_tmp);
        else k_gather<3><<<blocks(n), 256, 0, stream>>>(s, t, grid, phys, perm, cell_tmp);
    });
    launch(KI_COPY, [&] {
        if (dim == 2) k_copy_back<2><<<blocks(n), 256, 0, stream>>>(t, s);
        else k_copy_back<3><<<blocks(n), 256, 0, stream>>>(t, s);
    });
    launch(KI_LIST, [&] {
        if (dim == 2) k_build_list<2><<<blocks(n), 256, 0, stream>>>(s, grid, phys);
        else k_build_list<3><<<blocks(n), 256, 0, stream>>>(s, grid, phys);
    });
}

// One rates evaluation: sweep A then sweep B of stage 0 (rates only), 1
// (predictor fused) or 2 (corrector fused).
void sph_sim::enqueue_eval(int stage, const float *drho_in, double dt)
{
    Dev &d = buf[0];
    float4 *vel_s = stage == 2 ? d.velq : d.velp;
    const int stage1 = stage != 2;
    launch(KI_SWEEP_A, [&] {
        if (dim == 2) k_sweep_a<2><<<blocks(n), 256, 0, stream>>>(d, grid, phys, drho_in, stage1, vel_s);
        else k_sweep_a<3><<<blocks(n), 256, 0, stream>>>(d, grid, phys, drho_in, stage1, vel_s);
    });
    launch(KI_SWEEP_B, [&] {
        if (dim == 2) {
            if (stage == 0) k_sweep_b<2, 0><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
            else if (stage == 1) k_sweep_b<2, 1><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
            else k_sweep_b<2, 2><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
        } else {
            if (stage == 0) k_sweep_b<3, 0><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
            else if (stage == 1) k_sweep_b<3, 1><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
            else k_sweep_b<3, 2><<<blocks(n), 256, 0, stream>>>(d, grid, phys, dt);
        }
    });
}

void sph_sim::enqueue_step(double dt)
{
    enqueue_build_cells(false);
    Dev &d = buf[0];
    enqueue_eval(1, d.drho, dt);
    enqueue_eval(2, d.drho_stage, dt);
}

int sph_sim::check_flags()
{
    unsigned f = 0;
    CU(cudaMemcpyAsync(&f, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    if (timing) collect_timing();
    if (f == 0) return SPH_OK;
    CU(cudaMemsetAsync(flags, 0, sizeof(unsigned), stream));
    // the most specific cause first: a step too large for the skin often
    // also sends particles out of the box or produces non-finite values
    if (f & FLAG_SKIN) return fail(SPH_ECFL, "a particle moved beyond the cell skin within a step; reduce dt or enlarge cell_size");
    if (f & FLAG_NONFINITE) return fail(SPH_ENONFINITE, "a non-finite value appeared in the particle state");
    if (f & FLAG_LIST) return fail(SPH_ECAPACITY, "a particle has more neighbours than max_neighbours");
    return fail(SPH_EDOMAIN, "a particle left the box covered by the cell grid");
}

// ---------------------------------------------------------------------------

namespace sphgb {
// Records the message returned by sph_last_error() for this thread.
int set_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace sphgb

namespace {

__global__ void k_load_state(Dev d, Phys ph, int dim, const double *x, const double *u, const double *rho)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const int p = d.pid[k];
    for (int c = 0; c < dim; ++c) {
        d.x[(size_t)c * d.n + k] = x[(size_t)p * dim + c];
        d.u[(size_t)c * d.n + k] = u[(size_t)p * dim + c];
    }
    d.drho[k] = (float)(rho[p] - (double)ph.rho0[d.tag[k] & 1]);
}

__global__ void k_iota(int *p, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = k;
}

int validate(const sph_params *P, int64_t n)
{
    if (!P) return fail(SPH_EINVAL, "params is NULL");
    if (P->dim != 2 && P->dim != 3) return fail(SPH_EINVAL, "dim must be 2 or 3");
    if (P->visc_form != SPH_VISC_DYNAMIC && P->visc_form != SPH_VISC_KINEMATIC)
        return fail(SPH_EINVAL, "visc_form must be SPH_VISC_DYNAMIC or SPH_VISC_KINEMATIC");
    if (P->renorm_every < 0) return fail(SPH_EINVAL, "renorm_every must be >= 0");
    if (P->max_neighbours < 0 || P->max_neighbours > 4096)
        return fail(SPH_EINVAL, "max_neighbours must be in [0, 4096]");
    if (P->rebuild_every < 0) return fail(SPH_EINVAL, "rebuild_every must be >= 0");
    if (P->reserved != 0) return fail(SPH_EINVAL, "reserved must be 0");
    if (!(P->h > 0) || !std::isfinite(P->h)) return fail(SPH_EINVAL, "h must be positive");
    if (!(P->c0 > 0) || !std::isfinite(P->c0)) return fail(SPH_EINVAL, "c0 must be positive");
    if (P->gamma != 7.0) return fail(SPH_EINVAL, "gamma must be 7 (the exponent of the paper's equation of state)");
    if (!(P->delta >= 0)) return fail(SPH_EINVAL, "delta must be >= 0");
    if (!(P->alpha_s >= 0)) return fail(SPH_EINVAL, "alpha_s must be >= 0");
    if (!(P->skin >= 0) || !std::isfinite(P->skin)) return fail(SPH_EINVAL, "skin must be >= 0");
    if (!(P->cell_size >= P->h + P->skin) || !std::isfinite(P->cell_size))
        return fail(SPH_EINVAL, "cell_size must be >= h + skin (half the list radius 2h + 2 skin)");
    for (int k = 0; k < 2; ++k) {
        if (!(P->rho0[k] > 0)) return fail(SPH_EINVAL, "rho0 must be positive");
        if (!(P->mass[k] > 0)) return fail(SPH_EINVAL, "mass must be positive");
        if (!(P->mu[k] >= 0)) return fail(SPH_EINVAL, "mu must be >= 0");
    }
    for (int k = 0; k < P->dim; ++k) {
        if (!(P->box_hi[k] > P->box_lo[k])) return fail(SPH_EINVAL, "box_hi must exceed box_lo");
        if (!std::isfinite(P->g[k])) return fail(SPH_EINVAL, "g must be finite");
    }
    if (n < 0 || n > ((int64_t)1 << 26)) return fail(SPH_EINVAL, "n must be in [0, 2^26]");
    return SPH_OK;
}

double harmonic(double a, double b) { return a + b > 0 ? 2.0 * a * b / (a + b) : 0.0; }

// Eigenvalues of a symmetric 3x3 matrix by the trigonometric closed form.
void eig3(const double A[6], double &lmin, double &lmax)
{
    const double a = A[0], b = A[1], c = A[2], d = A[3], e = A[4], f = A[5];  // xx xy xz yy yz zz
    const double p1 = b * b + c * c + e * e;
    const double q = (a + d + f) / 3.0;
    if (p1 <= 1e-300 * (a * a + d * d + f * f + 1e-300)) {
        lmin = std::min(a, std::min(d, f));
        lmax = std::max(a, std::max(d, f));
        return;
    }
    const double p2 = (a - q) * (a - q) + (d - q) * (d - q) + (f - q) * (f - q) + 2.0 * p1;
    const double p = std::sqrt(p2 / 6.0);
    const double B0 = (a - q) / p, B1 = b / p, B2 = c / p, B3 = (d - q) / p, B4 = e / p, B5 = (f - q) / p;
    const double detB = B0 * (B3 * B5 - B4 * B4) - B1 * (B1 * B5 - B4 * B2) + B2 * (B1 * B4 - B3 * B2);
    double r = detB / 2.0;
    r = std::max(-1.0, std::min(1.0, r));
    const double phi = std::acos(r) / 3.0;
    const double pi = 3.14159265358979323846;
    lmax = q + 2.0 * p * std::cos(phi);
    lmin = q + 2.0 * p * std::cos(phi + 2.0 * pi / 3.0);
}

}  // namespace

extern "C" {

const char *sph_last_error(void) { return g_err.c_str(); }

int sph_create(const sph_params *params, int64_t n, const double *x, const double *u, const double *rho,
               const uint8_t *phase, const uint8_t *wall, void *stream, sph_handle *out)
{
    if (!out) return fail(SPH_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(params, n);
    if (rc) return rc;
    if (n > 0 && (!x || !u || !rho || !phase || !wall)) return fail(SPH_EINVAL, "an input array is NULL");
    const sph_params &P = *params;
    const int dim = P.dim;
    // host-side checks of the particle data
    for (int64_t i = 0; i < n; ++i) {
        if (phase[i] > 1) return fail(SPH_EINVAL, "phase must be 0 (water) or 1 (oil)");
        if (wall[i] > 1) return fail(SPH_EINVAL, "wall must be 0 or 1");
        if (wall[i] && phase[i] != 0) return fail(SPH_EINVAL, "wall particles must be water (phase 0)");
        if (!(rho[i] > 0) || !std::isfinite(rho[i])) return fail(SPH_EINVAL, "rho must be positive and finite");
        for (int c = 0; c < dim; ++c) {
            const double xc = x[i * dim + c];
            if (!std::isfinite(xc) || !std::isfinite(u[i * dim + c]))
                return fail(SPH_EINVAL, "x and u must be finite");
            if (xc < P.box_lo[c] || xc > P.box_hi[c]) return fail(SPH_EINVAL, "a particle lies outside the box");
        }
    }
    sph_sim *s = new sph_sim();
    s->P = P;
    s->dim = dim;
    s->n = (int)n;
    // grid
    int dims[3] = {1, 1, 1};
    int64_t ncell = 1;
    for (int c = 0; c < dim; ++c) {
        const double m = std::floor((P.box_hi[c] - P.box_lo[c]) / P.cell_size) + 1.0;
        if (m > 1e9) {
            delete s;
            return fail(SPH_EINVAL, "cell grid too large");
        }
        dims[c] = (int)m;
        ncell *= dims[c];
    }
    if (ncell > (int64_t)SCAN_TILE * SCAN_TILE) {
        delete s;
        return fail(SPH_EINVAL, "cell grid has more than 2^24 cells; enlarge cell_size or shrink the box");
    }
    s->ncell = (int)ncell;
    s->ntiles = (int)((ncell + SCAN_TILE - 1) / SCAN_TILE);
    s->grid.nx = dims[0];
    s->grid.ny = dims[1];
    s->grid.nz = dims[2];
    const double RL = 2.0 * P.h + 2.0 * P.skin;
    s->grid.f = P.cell_size >= RL ? 1 : 2;
    s->grid.csd = P.cell_size;
    s->grid.cs = (float)P.cell_size;
    s->grid.Ed = s->grid.f * P.cell_size;
    s->grid.Es = (float)s->grid.Ed;
    for (int c = 0; c < 3; ++c) s->grid.lo[c] = c < dim ? P.box_lo[c] : 0.0;
    // physics constants
    const double pi = 3.14159265358979323846;
    const double h = P.h;
    const double alpha_d = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    Phys &ph = s->phys;
    ph.inv_h = (float)(1.0 / h);
    ph.R2 = (float)(4.0 * h * h);
    ph.RL2 = (float)(RL * RL);
    ph.RP = (float)(RL * (1.0 + 1e-4));
    ph.skin = P.skin;
    ph.kmax = P.max_neighbours > 0 ? P.max_neighbours : (dim == 2 ? 48 : 128);
    ph.cF = (float)(-5.0 * alpha_d / (h * h));
    for (int k = 0; k < 2; ++k) {
        ph.mass[k] = (float)P.mass[k];
        ph.inv_mass[k] = (float)(1.0 / P.mass[k]);
        ph.rho0[k] = (float)P.rho0[k];
        ph.inv_rho0[k] = (float)(1.0 / P.rho0[k]);
        ph.beta[k] = (float)(P.rho0[k] * P.c0 * P.c0 / P.gamma);
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double kv = P.visc_form == SPH_VISC_DYNAMIC
                                  ? 2.0 * harmonic(P.mu[a], P.mu[b])
                                  : 2.0 * harmonic(P.mu[a] / P.rho0[a], P.mu[b] / P.rho0[b]);
            ph.kvis[2 * a + b] = (float)kv;
        }
    ph.delta2 = (float)(P.delta * P.delta);
    ph.alpha_s = (float)P.alpha_s;
    ph.inv_dim = (float)(1.0 / dim);
    ph.visc_dynamic = P.visc_form == SPH_VISC_DYNAMIC;
    ph.renorm_every = P.renorm_every;
    ph.rebuild_every = P.rebuild_every;
    for (int c = 0; c < 3; ++c) ph.gf[c] = c < dim ? (float)P.g[c] : 0.f;

    auto cleanup = [&](int code) {
        for (void *p : s->allocs) cudaFree(p);
        if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
        delete s;
        return code;
    };
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup(fail(SPH_ECUDA, cudaGetErrorString(e)));
        s->own_stream = true;
    }
    const size_t N = (size_t)std::max<int64_t>(n, 1);
    int err = 0;
    for (int b = 0; b < 2 && !err; ++b) {
        Dev &d = s->buf[b];
        d.n = (int)n;
        err |= s->alloc(&d.x, N * dim);
        err |= s->alloc(&d.u, N * dim);
        err |= s->alloc(&d.drho, N);
        err |= s->alloc(&d.pid, N);
        err |= s->alloc(&d.tag, N);
    }
    Dev &a0 = s->buf[0];
    if (!err) {
        err |= s->alloc(&a0.cell, N);
        err |= s->alloc(&a0.pos0, N);
        err |= s->alloc(&a0.pos, N);
        err |= s->alloc(&a0.vd, N);
        err |= s->alloc(&a0.posv, N);
        err |= s->alloc(&a0.velp, N);
        err |= s->alloc(&a0.velq, N);
        err |= s->alloc(&a0.pres, N);
        err |= s->alloc(&a0.nbr, N * (size_t)ph.kmax);
        err |= s->alloc(&a0.ncnt, N);
        err |= s->alloc(&a0.nflag, N);
        err |= s->alloc(&a0.drho_stage, N);
        err |= s->alloc(&a0.drho_eval, N);
        err |= s->alloc(&a0.T4, N);
        err |= s->alloc(&a0.T2, N);
        err |= s->alloc(&a0.acc, N);
        err |= s->alloc(&a0.cstart, (size_t)ncell + 1);
        err |= s->alloc(&s->flags, 1);
        err |= s->alloc(&s->rebuild, 1);
        err |= s->alloc(&s->dstep, 1);
        err |= s->alloc(&s->dbuilds, 1);
        err |= s->alloc(&s->cell_tmp, N);
        err |= s->alloc(&s->slot, N);
        err |= s->alloc(&s->count, (size_t)ncell);
        err |= s->alloc(&s->tmp, N);
        err |= s->alloc(&s->perm, N);
        err |= s->alloc(&s->tile_sums, (size_t)s->ntiles);
        err |= s->alloc(&s->diag_partial, (size_t)1024 * DIAG_K);
        err |= s->alloc(&s->diag_small, 64);
    }
    if (err) return cleanup(SPH_ENOMEM);
    Dev &a1 = s->buf[1];
    a1.cell = a0.cell; a1.pos0 = a0.pos0;
    a1.pos = a0.pos; a1.vd = a0.vd; a1.posv = a0.posv; a1.velp = a0.velp; a1.velq = a0.velq; a1.pres = a0.pres;
    a1.drho_stage = a0.drho_stage;
    a1.nbr = a0.nbr; a1.ncnt = a0.ncnt; a1.nflag = a0.nflag;
    a1.drho_eval = a0.drho_eval; a1.T4 = a0.T4; a1.T2 = a0.T2; a1.acc = a0.acc;
    a1.cstart = a0.cstart;
    a0.flags = a1.flags = s->flags;
    a0.step = a1.step = s->dstep;
    a0.rebuild = a1.rebuild = s->rebuild;
    a0.builds = a1.builds = s->dbuilds;

    cudaStream_t st = s->stream;
    auto cuda_fail = [&](cudaError_t e) { return cleanup(fail(SPH_ECUDA, cudaGetErrorString(e))); };
    cudaError_t e = cudaMemsetAsync(s->flags, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->dstep, 0, sizeof(long long), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->dbuilds, 0, sizeof(long long), st)) != cudaSuccess) return cuda_fail(e);
    if (n > 0) {
        std::vector<uint8_t> tag((size_t)n);
        for (int64_t i = 0; i < n; ++i) tag[i] = (uint8_t)(phase[i] | (wall[i] << 1));
        if ((e = cudaMemcpyAsync(a0.tag, tag.data(), (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e);
        k_iota<<<s->blocks((int)n), 256, 0, st>>>(a0.pid, (int)n);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    }
    s->cur = 0;
    *out = s;
    rc = sph_set_state(s, x, u, rho);
    if (rc) {
        *out = nullptr;
        return cleanup(rc);
    }
    return SPH_OK;
}

int sph_set_state(sph_handle s, const double *x, const double *u, const double *rho)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->n == 0) return SPH_OK;
    if (!x || !u || !rho) return fail(SPH_EINVAL, "an input array is NULL");
    const size_t n = (size_t)s->n, dim = (size_t)s->dim;
    // staging area: x, u (n*dim each) and rho (n) as doubles
    if (!s->read_buf) {
        if (s->alloc(&s->read_buf, n * 9 + 16)) return SPH_ENOMEM;
        if (s->alloc(&s->read_ibuf, n)) return SPH_ENOMEM;
    }
    double *dx = s->read_buf, *du = s->read_buf + n * dim, *dr = s->read_buf + 2 * n * dim;
    CU(cudaMemcpyAsync(dx, x, sizeof(double) * n * dim, cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(du, u, sizeof(double) * n * dim, cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(dr, rho, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    k_load_state<<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->phys, s->dim, dx, du, dr);
    CU(cudaGetLastError());
    CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
}

int sph_build_cells(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->n == 0) return SPH_OK;
    s->enqueue_build_cells(true);
    CU(cudaGetLastError());
    return SPH_OK;
}

int sph_eval_rates(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->n == 0) return SPH_OK;
    s->enqueue_build_cells(true);
    s->enqueue_eval(0, s->D().drho, 0.0);
    CU(cudaGetLastError());
    return SPH_OK;
}

int sph_step(sph_handle s, double dt)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (s->n > 0) {
        // the rebuild test looks half a step ahead with the previous dt
        if (dt != s->last_dt) CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
        s->last_dt = dt;
        s->enqueue_step(dt);
        CU(cudaGetLastError());
    }
    s->step += 1;
    return SPH_OK;
}

int sph_run(sph_handle s, double dt, int64_t nsteps, int graph)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    if (s->n == 0) {
        s->step += nsteps;
        return SPH_OK;
    }
    const bool use_graph = graph && !s->timing;
    if (dt != s->last_dt) CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    s->last_dt = dt;
    if (use_graph) {
        if (!s->gexec[0] || s->gdt[0] != dt) {
            cudaGraph_t gr = nullptr;
            CU(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            s->enqueue_step(dt);
            cudaError_t e = cudaStreamEndCapture(s->stream, &gr);
            if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            if (s->gexec[0]) cudaGraphExecDestroy(s->gexec[0]);
            s->gexec[0] = nullptr;
            e = cudaGraphInstantiate(&s->gexec[0], gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            s->gdt[0] = dt;
        }
        for (int64_t k = 0; k < nsteps; ++k) {
            CU(cudaGraphLaunch(s->gexec[0], s->stream));
            s->step += 1;
        }
    } else {
        for (int64_t k = 0; k < nsteps; ++k) {
            s->enqueue_step(dt);
            CU(cudaGetLastError());
            s->step += 1;
        }
    }
    return s->check_flags();
}

int sph_sync(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    return s->check_flags();
}

int sph_read(sph_handle s, int field, void *host_out, int64_t bytes)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!host_out && s->n > 0) return fail(SPH_EINVAL, "host_out is NULL");
    const size_t n = (size_t)s->n, dim = (size_t)s->dim;
    int kind = 0;
    size_t need = 0;
    bool integer = false;
    switch (field) {
    case SPH_FIELD_POS: kind = RK_X; need = n * dim * 8; break;
    case SPH_FIELD_VEL: kind = RK_U; need = n * dim * 8; break;
    case SPH_FIELD_RHO: kind = RK_RHO; need = n * 8; break;
    case SPH_FIELD_RHO_EVAL: kind = RK_RHO_EVAL; need = n * 8; break;
    case SPH_FIELD_PRESSURE: kind = RK_P; need = n * 8; break;
    case SPH_FIELD_ACC: kind = RK_ACC; need = n * dim * 8; break;
    case SPH_FIELD_DRHO: kind = RK_DRHO; need = n * 8; break;
    case SPH_FIELD_TENSOR: kind = RK_T; need = n * dim * dim * 8; break;
    case SPH_FIELD_CELL: kind = RK_CELL; need = n * 4; integer = true; break;
    case SPH_FIELD_ORDER: kind = RK_ORDER; need = n * 4; integer = true; break;
    default: return fail(SPH_EINVAL, "unknown field");
    }
    if (bytes < (int64_t)need) return fail(SPH_EINVAL, "output buffer too small for the field");
    if (n == 0) return SPH_OK;
    if (!s->read_buf) {
        if (s->alloc(&s->read_buf, n * 9 + 16)) return SPH_ENOMEM;
        if (s->alloc(&s->read_ibuf, n)) return SPH_ENOMEM;
    }
    if (s->dim == 2) k_unpermute<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->phys, kind, s->read_buf, s->read_ibuf);
    else k_unpermute<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->phys, kind, s->read_buf, s->read_ibuf);
    CU(cudaGetLastError());
    if (integer) CU(cudaMemcpyAsync(host_out, s->read_ibuf, need, cudaMemcpyDeviceToHost, s->stream));
    else CU(cudaMemcpyAsync(host_out, s->read_buf, need, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
}

int64_t sph_neighbours(sph_handle s, int64_t *start, int32_t *list, int64_t cap)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!start) return fail(SPH_EINVAL, "start is NULL");
    const int n = s->n;
    if (n == 0) {
        start[0] = 0;
        return 0;
    }
    s->enqueue_build_cells(true);
    Dev &d = s->D();
    int *cnt = s->tmp;  // scratch, free after the build
    if (s->dim == 2) k_nbr_count<2><<<s->blocks(n), 256, 0, s->stream>>>(d, s->grid, s->phys, cnt);
    else k_nbr_count<3><<<s->blocks(n), 256, 0, s->stream>>>(d, s->grid, s->phys, cnt);
    CU(cudaGetLastError());
    std::vector<int> hc(n), order(n);
    CU(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(order.data(), d.pid, sizeof(int) * n, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    // rows in original id order
    std::vector<int64_t> sorted_start(n + 1, 0);
    for (int k = 0; k < n; ++k) sorted_start[k + 1] = sorted_start[k] + hc[k];
    const int64_t total = sorted_start[n];
    std::vector<int64_t> cnt_by_id(n);
    for (int k = 0; k < n; ++k) cnt_by_id[order[k]] = hc[k];
    start[0] = 0;
    for (int i = 0; i < n; ++i) start[i + 1] = start[i] + cnt_by_id[i];
    if (total > cap || !list) return fail(SPH_EINVAL, "list capacity too small");
    long long *dstart = nullptr;
    int *dlist = nullptr;
    CU(cudaMallocAsync((void **)&dstart, sizeof(long long) * (n + 1), s->stream));
    CU(cudaMallocAsync((void **)&dlist, sizeof(int) * std::max<int64_t>(total, 1), s->stream));
    CU(cudaMemcpyAsync(dstart, sorted_start.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, s->stream));
    if (s->dim == 2) k_nbr_fill<2><<<s->blocks(n), 256, 0, s->stream>>>(d, s->grid, s->phys, dstart, dlist);
    else k_nbr_fill<3><<<s->blocks(n), 256, 0, s->stream>>>(d, s->grid, s->phys, dstart, dlist);
    CU(cudaGetLastError());
    std::vector<int> hl(total);
    CU(cudaMemcpyAsync(hl.data(), dlist, sizeof(int) * total, cudaMemcpyDeviceToHost, s->stream));
    CU(cudaFreeAsync(dstart, s->stream));
    CU(cudaFreeAsync(dlist, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        std::copy(hl.begin() + sorted_start[k], hl.begin() + sorted_start[k + 1], list + start[i]);
        std::sort(list + start[i], list + start[i + 1]);
    }
    const int rc = s->check_flags();
    if (rc) return rc;
    return total;
}

int sph_pair_stats(sph_handle s, int64_t out[2])
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    out[0] = out[1] = 0;
    if (s->n == 0) return SPH_OK;
    s->enqueue_build_cells(true);
    unsigned long long *tot = reinterpret_cast<unsigned long long *>(s->diag_small + 48);
    CU(cudaMemsetAsync(tot, 0, 2 * sizeof(unsigned long long), s->stream));
    if (s->dim == 2) k_pair_stats<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->grid, s->phys, tot);
    else k_pair_stats<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->grid, s->phys, tot);
    CU(cudaGetLastError());
    unsigned long long h[2];
    CU(cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    out[0] = (int64_t)h[0];
    out[1] = (int64_t)h[1];
    return s->check_flags();
}

int sph_diag(sph_handle s, double out[12])
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    for (int k = 0; k < 12; ++k) out[k] = 0.0;
    if (s->n == 0) return SPH_OK;
    const int nb = std::min(1024, std::max(1, s->blocks(s->n, DIAG_THREADS)));
    double *partial = s->diag_partial;
    double *res = s->diag_small;          // 16
    double *cen = s->diag_small + 16;     // 3
    double *grav = s->diag_small + 24;    // 3
    double *mass = s->diag_small + 32;    // 2
    double consts[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < s->dim; ++c) consts[c] = s->P.g[c];
    CU(cudaMemcpyAsync(grav, consts, sizeof(double) * 3, cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(mass, s->P.mass, sizeof(double) * 2, cudaMemcpyHostToDevice, s->stream));
    double r0[DIAG_K], r1[DIAG_K];
    if (s->dim == 2) k_diag<2><<<nb, DIAG_THREADS, 0, s->stream>>>(s->D(), 0, cen, grav, mass, partial);
    else k_diag<3><<<nb, DIAG_THREADS, 0, s->stream>>>(s->D(), 0, cen, grav, mass, partial);
    k_diag_final<<<1, DIAG_K, 0, s->stream>>>(partial, nb, res);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(r0, res, sizeof(r0), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    out[0] = r0[0];
    for (int c = 0; c < s->dim; ++c) out[1 + c] = r0[1 + c];
    out[4] = r0[4];
    out[5] = r0[5];
    out[10] = r0[15];
    out[11] = r0[9];
    if (r0[9] > 0) {
        double c3[3] = {r0[6] / r0[9], r0[7] / r0[9], r0[8] / r0[9]};
        for (int c = 0; c < s->dim; ++c) out[6 + c] = c3[c];
        CU(cudaMemcpyAsync(cen, c3, sizeof(c3), cudaMemcpyHostToDevice, s->stream));
        if (s->dim == 2) k_diag<2><<<nb, DIAG_THREADS, 0, s->stream>>>(s->D(), 1, cen, grav, mass, partial);
        else k_diag<3><<<nb, DIAG_THREADS, 0, s->stream>>>(s->D(), 1, cen, grav, mass, partial);
        k_diag_final<<<1, DIAG_K, 0, s->stream>>>(partial, nb, res);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(r1, res, sizeof(r1), cudaMemcpyDeviceToHost, s->stream));
        CU(cudaStreamSynchronize(s->stream));
        double lmin, lmax;
        const double no = r0[9];
        if (s->dim == 2) {
            const double a = r1[0] / no, b = r1[1] / no, d = r1[3] / no;
            const double tr = a + d, det = a * d - b * b;
            const double disc = std::sqrt(std::max(0.25 * tr * tr - det, 0.0));
            lmin = 0.5 * tr - disc;
            lmax = 0.5 * tr + disc;
        } else {
            double A[6];
            for (int k = 0; k < 6; ++k) A[k] = r1[k] / no;
            eig3(A, lmin, lmax);
        }
        out[9] = lmax > 0 ? std::sqrt(std::max(lmin, 0.0) / lmax) : 0.0;
    }
    return s->check_flags();
}

int sph_timing_enable(sph_handle s, int enable)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    s->timing = enable != 0;
    return SPH_OK;
}

int sph_timing_reset(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    CU(cudaStreamSynchronize(s->stream));
    s->collect_timing();
    for (int k = 0; k < KI_COUNT; ++k) {
        s->t_ms[k] = 0.0;
        s->t_launches[k] = 0;
    }
    return SPH_OK;
}

int sph_timing_count(void) { return KI_COUNT; }

int sph_timing_read(sph_handle s, int k, const char **name, int64_t *launches, double *total_ms)
{
    if (!s || k < 0 || k >= KI_COUNT) return fail(SPH_EINVAL, "bad handle or kernel index");
    CU(cudaStreamSynchronize(s->stream));
    s->collect_timing();
    if (name) *name = k_names[k];
    if (launches) *launches = s->t_launches[k];
    if (total_ms) *total_ms = s->t_ms[k];
    return SPH_OK;
}

int64_t sph_list_builds(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    long long b = 0;
    CU(cudaMemcpyAsync(&b, s->dbuilds, sizeof(b), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return b;
}

int64_t sph_num_particles(sph_handle s) { return s ? s->n : 0; }
int64_t sph_step_index(sph_handle s) { return s ? s->step : 0; }
int64_t sph_num_cells(sph_handle s) { return s ? s->ncell : 0; }

void sph_destroy(sph_handle s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->collect_timing();
    for (auto e : s->free_events) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k)
        if (s->gexec[k]) cudaGraphExecDestroy(s->gexec[k]);
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
