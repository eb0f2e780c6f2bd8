// Host side of the C ABI declared in include/sph.h: parameter validation,
// device memory, the per-step launch sequence, CUDA-graph replay, the
// persistent cooperative form and its launch-shape autotuner, batches of
// independent instances, reads in original particle order, FP64 diagnostics
// and per-kernel event timing.
#include "sph.h"
#include "sph_internal.h"
#include "sph_kernels.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
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
    KI_PERSISTENT, KI_COUNT
};
// sweep_b includes the predictor (stage 1) or the corrector (stage 2);
// persistent_steps is one cooperative launch running whole steps
const char *k_names[KI_COUNT] = {"count_reset", "cell_hash", "cell_scan", "cell_scatter",
                                 "cell_rank", "reorder_gather", "reorder_copy", "neighbour_list",
                                 "sweep_a", "sweep_b", "persistent_steps"};

struct PendingTiming {
    int id;
    cudaEvent_t a, b;
};

// Block sizes the persistent kernel is compiled for.  Each size has two
// register budgets: 64 registers a thread (up to 1024 resident threads an
// SM) and 128 (up to 512 threads); a shape with at most 512 threads an SM
// takes the second.
constexpr int PERSIST_BS[3] = {128, 256, 512};

template <int DIM, int BS, int TPSM>
__global__ void __launch_bounds__(BS, TPSM / BS) k_persistent_bs(Dev d, Dev scratch, Grid g, Phys ph, Sort s,
                                                                  GridBarrier *bar, double dt, int nsteps, int dyn)
{
    persistent_steps<DIM>(d, scratch, g, ph, s, bar, dt, nsteps, dyn);
}

using PersistFn = void (*)(Dev, Dev, Grid, Phys, Sort, GridBarrier *, double, int, int);

template <int DIM, int TPSM>
PersistFn persist_fn_t(int bs)
{
    if (bs == 128) return k_persistent_bs<DIM, 128, TPSM>;
    if (bs == 256) return k_persistent_bs<DIM, 256, TPSM>;
    return k_persistent_bs<DIM, 512, TPSM>;
}

PersistFn persist_fn(int dim, int bs, bool wide)
{
    if (dim == 2) return wide ? persist_fn_t<2, 512>(bs) : persist_fn_t<2, 1024>(bs);
    return wide ? persist_fn_t<3, 512>(bs) : persist_fn_t<3, 1024>(bs);
}

}  // namespace

struct sph_sim {
    sph_params P{};
    int dim = 0;
    int n = 0;
    int ninst = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Grid grid{};
    Phys phys{};
    int ncell = 0;
    int ntiles = 0;
    Dev buf[2]{};                         // buf[0]: the state; buf[1]: reorder scratch
    Sort sort{};
    std::vector<Inst> hinst;
    Inst *dinst = nullptr;
    std::vector<int64_t> first;           // instance q owns original ids [first[q], first[q+1])
    long long *dfirst = nullptr;
    unsigned *flags = nullptr;
    unsigned *rebuild = nullptr;
    long long *dstep = nullptr;
    long long *dbuilds = nullptr;
    double *clock = nullptr;              // device time, see Dev::clock
    Motion *motion = nullptr;             // device copy of the piston motion
    int64_t npiston = 0;                  // particles with wall == 2
    bool moving = false;                  // a piston motion is set
    bool evaluated = false;               // acc holds a rates evaluation
    unsigned *amax = nullptr;             // per instance, max |a|^2 (FP32 bits) for sph_suggest_dt
    std::vector<sph_params> inst_params;  // each instance's parameters as given
    unsigned *occ = nullptr;              // oil occupancy bitmap (sph_oil_occupancy_diff)
    unsigned long long *occ_cnt = nullptr;
    GridBarrier *bar = nullptr;
    unsigned long long *pair_tot = nullptr;
    double last_dt = 0.0;
    double *diag_out = nullptr, *diag_grav = nullptr;
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
    // per-launch graph of one step, replayed while dt matches
    cudaGraphExec_t gexec = nullptr;
    double gdt = 0.0;
    // persistent form: launch shape and its graph
    int pbs = 256, pgrid = 0;             // block size, grid blocks (0: as many as fit)
    int pdyn = 1;                         // particle loops: 1 dynamic chunks, 0 grid-stride
    cudaGraphExec_t pexec = nullptr;
    double pdt = 0.0;
    int64_t psteps = 0;
    int pshape = 0;
    // extension owned by the learned surrogate
    void *ext = nullptr;
    void (*ext_free)(void *) = nullptr;

    Dev &D() { return buf[0]; }

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

    // Launch wrapper: an NVTX range named after the kernel around every
    // launch (seen by profilers that attach; a no-op otherwise), and events
    // around it when timing is enabled.
    template <class L>
    void launch(int id, L &&l) {
        nvtxRangePushA(k_names[id]);
        if (timing) {
            PendingTiming p{id, get_event(), get_event()};
            cudaEventRecord(p.a, stream);
            l();
            cudaEventRecord(p.b, stream);
            pending.push_back(p);
        } else {
            l();
        }
        nvtxRangePop();
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
    int sms = 0;  // multiprocessors of the device

    void enqueue_build_cells(bool force);
    void enqueue_load(const double *x, const double *u, const double *rho, double check_dt);
    int enqueue_read(int kind, bool integer, void *out, size_t bytes, size_t staging_offset);
    void enqueue_eval(int stage, const float *drho_in, double dt);
    void enqueue_step(double dt);
    int capture_step_graph(double dt);
    int enqueue_set_state(const double *x, const double *u, const double *rho);
    int enqueue_run(double dt, int64_t nsteps, bool graph);
    int enqueue_read_state(double *x, double *u, double *rho);
    int persistent_shape(int bs, int grid_req, int *grid_out, PersistFn *fn_out);
    int launch_persistent(double dt, int nsteps);
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
    launch(KI_MEMSET, [&] { k_zero<<<blocks(ncell), 256, 0, stream>>>(sort.count, ncell, rebuild); });
    launch(KI_HASH, [&] {
        if (dim == 2) k_hash<2><<<blocks(n), 256, 0, stream>>>(s, grid, sort);
        else k_hash<3><<<blocks(n), 256, 0, stream>>>(s, grid, sort);
    });
    launch(KI_SCAN, [&] {
        k_scan_tiles<<<ntiles, SCAN_THREADS, 0, stream>>>(sort.count, s.cstart, sort.tile_sums, ncell, rebuild);
        k_scan_sums<<<1, SCAN_THREADS, 0, stream>>>(sort.tile_sums, ntiles, s.cstart, ncell, rebuild);
        k_scan_add<<<blocks(ncell), 256, 0, stream>>>(s.cstart, sort.tile_sums, ncell, rebuild);
    });
    launch(KI_SCATTER, [&] { k_scatter<<<blocks(n), 256, 0, stream>>>(n, sort, s.cstart, rebuild); });
    launch(KI_RANK, [&] { k_rank<<<blocks(n), 256, 0, stream>>>(n, sort, s.pid, s.cstart, rebuild); });
    launch(KI_GATHER, [&] {
        if (dim == 2) k_gather<2><<<blocks(n), 256, 0, stream>>>(s, t, grid, sort);
        else k_gather<3><<<blocks(n), 256, 0, stream>>>(s, t, grid, sort);
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
        if (stage1) {
            const int ta = SPH_SWEEP_A_THREADS;
            if (dim == 2) k_sweep_a<2><<<blocks(n, ta), ta, 0, stream>>>(d, grid, phys, drho_in, stage1, vel_s);
            else k_sweep_a<3><<<blocks(n, ta), ta, 0, stream>>>(d, grid, phys, drho_in, stage1, vel_s);
        } else {
            // warps for the mixed particles: up to eight blocks of eight per SM
            const int mb = std::max(1, std::min(blocks(n), 8 * std::max(sms, 1)));
            if (dim == 2) k_sweep_a2<2><<<mb + blocks(n), 256, 0, stream>>>(d, grid, phys, drho_in, vel_s, mb);
            else k_sweep_a2<3><<<mb + blocks(n), 256, 0, stream>>>(d, grid, phys, drho_in, vel_s, mb);
        }
    });
    launch(KI_SWEEP_B, [&] {
        const int tb = SPH_SWEEP_B_THREADS, nbb = blocks(n, tb);
        if (dim == 2) {
            if (stage == 0) k_sweep_b<2, 0><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
            else if (stage == 1) k_sweep_b<2, 1><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
            else k_sweep_b<2, 2><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
        } else {
            if (stage == 0) k_sweep_b<3, 0><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
            else if (stage == 1) k_sweep_b<3, 1><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
            else k_sweep_b<3, 2><<<nbb, tb, 0, stream>>>(d, grid, phys, dt);
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

namespace {
__global__ void k_rebuild_cond(cudaGraphConditionalHandle h, const unsigned *rebuild);
}  // namespace

// The replayed step as a graph: a one-thread kernel reads the rebuild flag
// into the condition of an IF node whose body is the cell-list chain, then
// the four sweeps.  On steps without a rebuild the chain is not launched at
// all (its kernels would return at once, but ten launches of n/256 blocks
// still cost several microseconds each).  The body's kernels keep their own
// flag test, so the graph and the eager sequence compute the same.
int sph_sim::capture_step_graph(double dt)
{
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t cond_set = nullptr, cond = nullptr;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {};
    size_t count = 1;
    Dev &d = buf[0];
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("graph create: ") + cudaGetErrorString(e));
    auto bail = [&](const char *what, cudaError_t err) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(stream, &junk);
        }
        cudaGraphDestroy(g);
        return fail(SPH_ECUDA, std::string(what) + ": " + cudaGetErrorString(err));
    };
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return bail("conditional handle", e);
    if ((e = cudaStreamBeginCaptureToGraph(stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return bail("graph capture", e);
    k_rebuild_cond<<<1, 32, 0, stream>>>(h, rebuild);
    if ((e = cudaStreamEndCapture(stream, &g)) != cudaSuccess) return bail("graph capture", e);
    if ((e = cudaGraphGetNodes(g, &cond_set, &count)) != cudaSuccess || count != 1)
        return bail("graph nodes", e);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&cond, g, &cond_set, nullptr, 1, &cp)) != cudaSuccess)
        return bail("conditional node", e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return bail("graph capture", e);
    enqueue_build_cells(false);
    if ((e = cudaStreamEndCapture(stream, &body)) != cudaSuccess) return bail("graph capture", e);
    if ((e = cudaStreamBeginCaptureToGraph(stream, g, &cond, nullptr, 1, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return bail("graph capture", e);
    enqueue_eval(1, d.drho, dt);
    enqueue_eval(2, d.drho_stage, dt);
    if ((e = cudaStreamEndCapture(stream, &g)) != cudaSuccess) return bail("graph capture", e);
    if ((e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess) return bail("graph instantiate", e);
    cudaGraphDestroy(g);
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = exec;
    gdt = dt;
    return SPH_OK;
}

// Grid and kernel build of a persistent launch of grid_req blocks of bs
// threads (0: as many as can be co-resident); never more blocks than fit.
int sph_sim::persistent_shape(int bs, int grid_req, int *grid_out, PersistFn *fn_out)
{
    int dev = 0, sms = 0, fit = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool wide = grid_req > 0 && bs * ((grid_req + sms - 1) / sms) <= 512;
    PersistFn fn = persist_fn(dim, bs, wide);
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, (const void *)fn, bs, 0));
    if (fit < 1) return fail(SPH_ECUDA, "the persistent kernel does not fit an SM");
    *grid_out = grid_req > 0 ? std::min(grid_req, fit * sms) : fit * sms;
    if (fn_out) *fn_out = fn;
    return SPH_OK;
}

// Cooperative launch (all blocks co-resident, or the launch fails), through
// cudaLaunchKernelEx so that it can be captured into a graph.
int sph_sim::launch_persistent(double dt, int nsteps)
{
    int gsz = 0;
    PersistFn fn = nullptr;
    int rc = persistent_shape(pbs, pgrid, &gsz, &fn);
    if (rc) return rc;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(gsz);
    cfg.blockDim = dim3(pbs);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    launch(KI_PERSISTENT, [&] {
        e = cudaLaunchKernelEx(&cfg, fn, buf[0], buf[1], grid, phys, sort, bar, dt, nsteps, pdyn);
    });
    if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}

int sph_sim::check_flags()
{
    unsigned f = 0;
    CU(cudaMemcpyAsync(&f, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CU(cudaStreamSynchronize(stream));
    if (timing) collect_timing();
    if (f == 0) return SPH_OK;
    CU(cudaMemsetAsync(flags, 0, sizeof(unsigned), stream));
    if (f & FLAG_TIMEOUT) {
        // a block gave up at a barrier: start the next launch from a clean barrier
        CU(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), stream));
        CU(cudaStreamSynchronize(stream));
        return fail(SPH_ETIMEOUT, "a grid barrier of the persistent kernel waited longer than one second");
    }
    // the most specific cause first: a step too large for the skin often
    // also sends particles out of the box or produces non-finite values
    if (f & FLAG_SKIN) return fail(SPH_ECFL, "a particle moved beyond the cell skin within a step; reduce dt or enlarge cell_size");
    if (f & FLAG_NONFINITE) return fail(SPH_ENONFINITE, "a non-finite value appeared in the particle state");
    if (f & FLAG_BOUNDS) return fail(SPH_EBOUNDS, "an index read from device data was out of range (bounds-checked build)");
    if (f & FLAG_LIST) return fail(SPH_ECAPACITY, "a particle has more neighbours than max_neighbours");
    return fail(SPH_EDOMAIN, "a particle left the box covered by the cell grid");
}

// ---------------------------------------------------------------------------

namespace sphgb {
// Records the message returned by sph_last_error() for this thread.
int set_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace sphgb

// NVTX range for the lifetime of a scope (a no-op when no profiler attaches).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

namespace {
template <int DIM>
__global__ void k_load_state(Dev d, Grid g, Phys ph, const double *x, const double *u, const double *rho,
                             double check_dt);
__global__ void k_add_step(long long *step, long long k, double *clock, double elapsed)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *step += k;
        clock[1] += elapsed;
    }
}
// Condition of the step graph's rebuild node: the device rebuild flag (set by
// the corrector, by a forced build or by a change of dt).
__global__ void k_rebuild_cond(cudaGraphConditionalHandle h, const unsigned *rebuild)
{
    if (threadIdx.x == 0) cudaGraphSetConditional(h, *rebuild != 0u ? 1u : 0u);
}
}  // namespace

namespace {

// Copies the caller's state (original order, each instance in its own frame)
// into the sorted device state.  With check_dt > 0 the cell order and the
// neighbour list are kept when they still hold the new state: the particle's
// stage-1 records are written in its current cell, and the rebuild flag is
// raised if it is farther than the skin allows from where it was at the last
// build, by the test the corrector applies (positions now and half a step of
// check_dt ahead; a wall only now).  Non-finite positions always raise it.
// With check_dt == 0 the caller forces the rebuild.
template <int DIM>
__global__ void k_load_state(Dev d, Grid g, Phys ph, const double *x, const double *u, const double *rho,
                             double check_dt)
{
    // one thread per original id: the input is read in order (coalesced), the
    // sorted state is scattered
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d.n) return;
    const int k = d.inv[p];
    if (!SPH_IN_RANGE(d.flags, k, d.n)) return;
    const Inst &I = d.inst[d.iid[k]];
    const uint8_t tg = d.tag[k];
    double xa[3] = {0, 0, 0}, ua[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        xa[c] = x[(size_t)p * DIM + c] + I.offset[c];
        ua[c] = u[(size_t)p * DIM + c];
        d.x[(size_t)c * d.n + k] = xa[c];
        d.u[(size_t)c * d.n + k] = ua[c];
    }
    const float dr = (float)(rho[p] - (double)by_phase(tg & 1, I.rho0));
    d.drho[k] = dr;
    // static boundary particles keep their velocity: one that is not at rest
    // gives the force sweep its whole lists
    if (static_wall(tg) && !(ua[0] == 0.0 && ua[1] == 0.0 && ua[2] == 0.0)) atomicOr(d.walls_moving, 1u);
    if (!(check_dt > 0)) return;
    stage_records<DIM>(d, g, I, k, d.cell[k], xa, ua, dr, tg & 1);
    const float4 q = d.pos[k], q0 = d.pos0[k];
    const float ex = q.x - q0.x, ey = q.y - q0.y, ez = q.z - q0.z;
    const float hdt = ((tg & 2) && !(tg & 4)) ? 0.f : 0.5f * (float)(check_dt * I.dt_scale);
    const float hx = __fmul_rn(hdt, (float)ua[0]), hy = __fmul_rn(hdt, (float)ua[1]), hz = __fmul_rn(hdt, (float)ua[2]);
    const float d1 = sq3(ex, ey, ez);
    const float d2 = sq3(ex + hx, ey + hy, ez + hz);
    const float lim = ph.skin98f;
    if (!(d1 <= lim * lim) || !(d2 <= lim * lim)) atomicOr(d.rebuild, 1u);
}

}  // namespace

// The device address of a caller's buffer when kernels can use it in place
// (device or managed memory); NULL for host memory, pinned or pageable, which
// goes through the handle's staging buffers with cudaMemcpyAsync unless a
// path below reads or writes it in place.
template <class T>
T *device_view(T *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return static_cast<T *>(a.devicePointer);
    return nullptr;
}

// The device address of pinned host memory the GPU can address (mapped);
// NULL for anything else.  The state is read back into such memory in place,
// in whole lines (k_read_state_lines).
template <class T>
T *pinned_view(T *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<T *>(a.devicePointer);
    return nullptr;
}

// Queues the original-order copy of one field into `out`: in place when the
// kernel can write it (device or managed memory), else through the staging
// buffer (at staging_offset doubles) and a cudaMemcpyAsync.
int sph_sim::enqueue_read(int kind, bool integer, void *out, size_t bytes, size_t staging_offset)
{
    void *dst = device_view(out);
    double *fo = integer ? nullptr : (dst ? static_cast<double *>(dst) : read_buf + staging_offset);
    int *io = integer ? (dst ? static_cast<int *>(dst) : read_ibuf) : read_ibuf;
    if (dim == 2) k_unpermute<2><<<blocks(n), 256, 0, stream>>>(D(), kind, fo, io);
    else k_unpermute<3><<<blocks(n), 256, 0, stream>>>(D(), kind, fo, io);
    CU(cudaGetLastError());
    if (!dst) {
        const void *src = integer ? static_cast<const void *>(read_ibuf) : static_cast<const void *>(read_buf + staging_offset);
        CU(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, stream));
    }
    return SPH_OK;
}

void sph_sim::enqueue_load(const double *x, const double *u, const double *rho, double check_dt)
{
    // the load raises the flag again if a static boundary particle moves
    cudaMemsetAsync(D().walls_moving, 0, sizeof(unsigned), stream);
    if (dim == 2) k_load_state<2><<<blocks(n), 256, 0, stream>>>(D(), grid, phys, x, u, rho, check_dt);
    else k_load_state<3><<<blocks(n), 256, 0, stream>>>(D(), grid, phys, x, u, rho, check_dt);
}

namespace {

// Oil occupancy: the cells of a grid of spacing dx from lo that hold at least
// one oil particle (periodic coordinates wrapped), as a bitmap.
template <int DIM>
__global__ void k_occupancy(Dev d, double3 lo, double dx, int3 dims, unsigned *bm)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const uint8_t tg = d.tag[k];
    if (!(tg & 1) || (tg & 2)) return;
    const double l[3] = {lo.x, lo.y, lo.z};
    const int nd[3] = {dims.x, dims.y, dims.z};
    long long lin = 0, stride = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double x = wrap_coord(d.x[(size_t)a * d.n + k], d.plo[a], d.period[a]);
        double c = floor((x - l[a]) / dx);
        c = c < 0.0 ? 0.0 : (c > nd[a] - 1 ? nd[a] - 1 : c);
        lin += (long long)c * stride;
        stride *= nd[a];
    }
    atomicOr(bm + (lin >> 5), 1u << (lin & 31));
}

// out[0] += |a xor b|, out[1] += |b| over `words` bitmap words.
__global__ void k_occupancy_cmp(const unsigned *a, const unsigned *b, long long words, unsigned long long *out)
{
    unsigned long long x = 0, nb = 0;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < words; w += (long long)gridDim.x * blockDim.x) {
        x += __popc(a[w] ^ b[w]);
        nb += __popc(b[w]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        nb += __shfl_down_sync(0xffffffffu, nb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, x);
        atomicAdd(out + 1, nb);
    }
}

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014): a counter-based 64-bit mixer.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// A standard normal variate for (seed, particle id, channel): two uniforms
// from the mixer and the Box-Muller transform.
__device__ __forceinline__ double gauss(unsigned long long seed, int p, int c)
{
    const unsigned long long a = splitmix64(seed ^ splitmix64(((unsigned long long)p << 3) | (unsigned)c));
    const unsigned long long b = splitmix64(a);
    const double u1 = ((a >> 11) + 1.0) * 0x1.0p-53, u2 = (b >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// Adds N(0, sigma_u^2) to each velocity component and multiplies the density
// by 1 + N(0, sigma_rho^2), fluid particles only; the variates depend on the
// original particle id, not on the sorted position.
template <int DIM>
__global__ void k_perturb(Dev d, double sigma_u, double sigma_rho, unsigned long long seed)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    const uint8_t tg = d.tag[k];
    if (tg & 2) return;
    const int p = d.pid[k];
#pragma unroll
    for (int c = 0; c < DIM; ++c) d.u[(size_t)c * d.n + k] += sigma_u * gauss(seed, p, c);
    const Inst &I = d.inst[d.iid[k]];
    const double rho0 = by_phase(tg & 1, I.rho0);
    const double rho = (rho0 + (double)d.drho[k]) * (1.0 + sigma_rho * gauss(seed, p, 3));
    d.drho[k] = (float)(rho - rho0);
}

// Largest |a|^2 over the fluid particles of each instance, from the last
// rates evaluation (non-negative FP32 values order like their bit patterns).
__global__ void k_amax(Dev d, unsigned *amax)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n || (d.tag[k] & 2)) return;
    const float4 a = d.acc[k];
    const float a2 = a.x * a.x + a.y * a.y + a.z * a.z;
    if (a2 > 0.f) atomicMax(amax + d.iid[k], __float_as_uint(a2));
}

__global__ void k_iota(int *p, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = k;
}

int validate(const sph_params *P)
{
    if (!P) return fail(SPH_EINVAL, "params is NULL");
    if (P->dim != 2 && P->dim != 3) return fail(SPH_EINVAL, "dim must be 2 or 3");
    if (P->visc_form != SPH_VISC_DYNAMIC && P->visc_form != SPH_VISC_KINEMATIC)
        return fail(SPH_EINVAL, "visc_form must be SPH_VISC_DYNAMIC or SPH_VISC_KINEMATIC");
    if (P->renorm_every < 0) return fail(SPH_EINVAL, "renorm_every must be >= 0");
    if (P->renorm_walls != 0 && P->renorm_walls != 1) return fail(SPH_EINVAL, "renorm_walls must be 0 or 1");
    if (P->reserved != 0) return fail(SPH_EINVAL, "reserved must be 0");
    if (P->max_neighbours < 0 || P->max_neighbours > 4096)
        return fail(SPH_EINVAL, "max_neighbours must be in [0, 4096]");
    if (P->rebuild_every < 0) return fail(SPH_EINVAL, "rebuild_every must be >= 0");
    if (P->periodic & ~((1 << P->dim) - 1)) return fail(SPH_EINVAL, "periodic may only set the bits of the dim axes");
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
    return SPH_OK;
}

// Parameters every instance of a batch must share (they are compiled into
// the shared constants or the shared cell grid).
bool same_shared(const sph_params &a, const sph_params &b)
{
    bool same = a.dim == b.dim && a.visc_form == b.visc_form && a.renorm_every == b.renorm_every &&
                a.renorm_walls == b.renorm_walls &&
                a.periodic == b.periodic &&
                a.max_neighbours == b.max_neighbours && a.rebuild_every == b.rebuild_every && a.h == b.h &&
                a.gamma == b.gamma && a.delta == b.delta && a.cell_size == b.cell_size && a.skin == b.skin;
    for (int c = 0; c < 3; ++c) same = same && a.g[c] == b.g[c];
    return same;
}

double harmonic(double a, double b) { return a + b > 0 ? 2.0 * a * b / (a + b) : 0.0; }

// Per-instance constants: masses, reference densities, the Tait stiffness
// rho0 c0^2 / gamma (Eq. eos), the harmonic-mean viscosity pairs (Sec. II-C)
// and the surface-tension coefficient.
Inst make_inst(const sph_params &P)
{
    Inst I{};
    for (int k = 0; k < 2; ++k) {
        I.mass[k] = (float)P.mass[k];
        I.mass64[k] = P.mass[k];
        I.inv_mass[k] = (float)(1.0 / P.mass[k]);
        I.rho0[k] = (float)P.rho0[k];
        I.inv_rho0[k] = (float)(1.0 / P.rho0[k]);
        I.vol0[k] = (float)(P.mass[k] / P.rho0[k]);
        I.beta[k] = (float)(P.rho0[k] * P.c0 * P.c0 / P.gamma);
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const double kv = P.visc_form == SPH_VISC_DYNAMIC
                                  ? 2.0 * harmonic(P.mu[a], P.mu[b])
                                  : 2.0 * harmonic(P.mu[a] / P.rho0[a], P.mu[b] / P.rho0[b]);
            I.kvis[2 * a + b] = (float)kv;
        }
    I.alpha_s = (float)P.alpha_s;
    I.dt_scale = 1.0;
    return I;
}

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

// Places instance boxes (extents w[q] along x, hgt[q] along y) on shelves in
// the x-y plane, tallest first, at least `gap` apart, each lower corner on a
// multiple of `align`; returns the corners and the extent of the packing.
void shelf_pack(const std::vector<double> &w, const std::vector<double> &hgt, double gap, double align,
                std::vector<double> &ox, std::vector<double> &oy, double &width, double &height)
{
    auto up = [align](double v) { return std::ceil(v / align - 1e-9) * align; };
    const size_t k = w.size();
    std::vector<size_t> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return hgt[a] > hgt[b]; });
    double area = 0.0, wmax = 0.0;
    for (size_t q = 0; q < k; ++q) {
        area += (w[q] + gap) * (hgt[q] + gap);
        wmax = std::max(wmax, w[q] + gap);
    }
    const double limit = std::max(wmax, 1.2 * std::sqrt(area));
    ox.assign(k, 0.0);
    oy.assign(k, 0.0);
    double x = 0.0, y = 0.0, row_h = 0.0;
    width = 0.0;
    for (size_t idx = 0; idx < k; ++idx) {
        const size_t q = order[idx];
        if (x > 0.0 && x + w[q] > limit) {
            y = up(y + row_h + gap);
            x = 0.0;
            row_h = 0.0;
        }
        ox[q] = x;
        oy[q] = y;
        x = up(x + w[q] + gap);
        row_h = std::max(row_h, hgt[q]);
        width = std::max(width, ox[q] + w[q]);
    }
    height = y + row_h;
}

// Shared creation path of sph_create and sph_create_batch.
int create_sim(const sph_params *params, int k, const int64_t *counts, const double *x, const double *u,
               const double *rho, const uint8_t *phase, const uint8_t *wall, void *stream, sph_handle *out)
{
    if (!out) return fail(SPH_EINVAL, "out is NULL");
    *out = nullptr;
    if (k < 1 || k > 65535) return fail(SPH_EINVAL, "the number of instances must be in [1, 65535]");
    int64_t n = 0;
    for (int q = 0; q < k; ++q) {
        int rc = validate(params + q);
        if (rc) return rc;
        if (!same_shared(params[0], params[q]))
            return fail(SPH_EINVAL, "instances of a batch must share dim, h, gamma, delta, g, cell_size, skin, "
                                    "visc_form, renorm_every, renorm_walls, rebuild_every and max_neighbours");
        if (counts[q] < 0) return fail(SPH_EINVAL, "instance particle counts must be >= 0");
        n += counts[q];
        if (n > ((int64_t)1 << 26)) return fail(SPH_EINVAL, "n must be in [0, 2^26]");
    }
    if (n > 0 && (!x || !u || !rho || !phase || !wall)) return fail(SPH_EINVAL, "an input array is NULL");
    const sph_params &P0 = params[0];
    if (k > 1 && P0.periodic) return fail(SPH_EINVAL, "periodic axes are not supported in a batch");
    const int dim = P0.dim;
    // host-side checks of the particle data
    {
        int64_t i = 0;
        for (int q = 0; q < k; ++q)
            for (int64_t c = 0; c < counts[q]; ++c, ++i) {
                if (phase[i] > 1) return fail(SPH_EINVAL, "phase must be 0 (water) or 1 (oil)");
                if (wall[i] > 2) return fail(SPH_EINVAL, "wall must be 0 (fluid), 1 (boundary) or 2 (piston)");
                if (wall[i] && phase[i] != 0) return fail(SPH_EINVAL, "wall particles must be water (phase 0)");
                if (!(rho[i] > 0) || !std::isfinite(rho[i])) return fail(SPH_EINVAL, "rho must be positive and finite");
                for (int a = 0; a < dim; ++a) {
                    const double xc = x[i * dim + a];
                    if (!std::isfinite(xc) || !std::isfinite(u[i * dim + a]))
                        return fail(SPH_EINVAL, "x and u must be finite");
                    if (xc < params[q].box_lo[a] || xc > params[q].box_hi[a])
                        return fail(SPH_EINVAL, "a particle lies outside the box");
                }
            }
    }
    sph_sim *s = new sph_sim();
    s->P = P0;
    s->inst_params.assign(params, params + k);
    s->dim = dim;
    s->n = (int)n;
    s->ninst = k;
    // instance placement in the shared grid: a single instance keeps its own
    // box; a batch is shelf-packed in the x-y plane with gaps wider than the
    // list radius plus two cells, so no neighbour pair joins two instances.
    // Each instance's box corner sits on a super-cell boundary of the shared
    // grid, so its particles see the same cell geometry (and the same pair
    // arithmetic, up to FP64 rounding of the shifted positions) as alone.
    const double RL = 2.0 * P0.h + 2.0 * P0.skin;
    s->hinst.resize(k);
    double box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};
    if (k == 1) {
        s->hinst[0] = make_inst(P0);
        for (int a = 0; a < dim; ++a) {
            box_lo[a] = P0.box_lo[a];
            box_hi[a] = P0.box_hi[a];
        }
    } else {
        std::vector<double> w(k), hg(k), ox, oy;
        double zmax = 0.0;
        for (int q = 0; q < k; ++q) {
            w[q] = params[q].box_hi[0] - params[q].box_lo[0];
            hg[q] = params[q].box_hi[1] - params[q].box_lo[1];
            if (dim == 3) zmax = std::max(zmax, params[q].box_hi[2] - params[q].box_lo[2]);
        }
        double width = 0.0, height = 0.0;
        const double gap = RL + 2.0 * P0.cell_size;
        const double E = (P0.cell_size >= RL ? 1.0 : 2.0) * P0.cell_size;
        shelf_pack(w, hg, gap, E, ox, oy, width, height);
        for (int q = 0; q < k; ++q) {
            Inst I = make_inst(params[q]);
            I.offset[0] = ox[q] - params[q].box_lo[0];
            I.offset[1] = oy[q] - params[q].box_lo[1];
            I.offset[2] = dim == 3 ? -params[q].box_lo[2] : 0.0;
            s->hinst[q] = I;
        }
        box_hi[0] = width;
        box_hi[1] = height;
        box_hi[2] = dim == 3 ? zmax : 0.0;
    }
    s->first.assign(k + 1, 0);
    for (int q = 0; q < k; ++q) s->first[q + 1] = s->first[q] + counts[q];
    // grid
    int dims[3] = {1, 1, 1};
    int64_t ncell = 1;
    const int fcell = P0.cell_size >= RL ? 1 : 2;   // cells per super-cell edge
    for (int c = 0; c < dim; ++c) {
        const double len = box_hi[c] - box_lo[c];
        double m = std::floor(len / P0.cell_size) + 1.0;
        if ((P0.periodic >> c) & 1) {
            // the cells must tile the period, in whole super-cells, at least
            // three of them (so a stencil never meets a cell twice)
            m = std::nearbyint(len / P0.cell_size);
            if (std::fabs(m * P0.cell_size - len) > 1e-9 * len || (int64_t)m % fcell != 0 || m < 3 * fcell) {
                delete s;
                return fail(SPH_EINVAL, "a periodic axis must span a whole number of super-cells (cell_size, or "
                                        "2 cell_size when cell_size < 2h + 2 skin), at least three");
            }
        }
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
    s->grid.f = P0.cell_size >= RL ? 1 : 2;
    s->grid.csd = P0.cell_size;
    s->grid.cs = (float)P0.cell_size;
    s->grid.inv_cs = 1.0f / s->grid.cs;
    s->grid.Ed = s->grid.f * P0.cell_size;
    s->grid.Es = (float)s->grid.Ed;
    for (int c = 0; c < 3; ++c) s->grid.lo[c] = box_lo[c];
    for (int c = 0; c < 3; ++c) s->grid.per[c] = c < dim ? (P0.periodic >> c) & 1 : 0;
    // constants shared by all instances
    const double pi = 3.14159265358979323846;
    const double h = P0.h;
    const double alpha_d = dim == 2 ? 7.0 / (4.0 * pi * h * h) : 21.0 / (16.0 * pi * h * h * h);
    Phys &ph = s->phys;
    ph.inv_h = (float)(1.0 / h);
    ph.R2 = (float)(4.0 * h * h);
    ph.RL2 = (float)(RL * RL);
    ph.RP = (float)(RL * (1.0 + 1e-4));
    ph.skin = P0.skin;
    ph.skin2f = (float)(P0.skin * P0.skin);
    ph.skin98f = (float)(0.98 * P0.skin);
    ph.kmax = P0.max_neighbours > 0 ? P0.max_neighbours : (dim == 2 ? 48 : 128);
    ph.kmax = (ph.kmax + SPH_LIST_CHUNK - 1) / SPH_LIST_CHUNK * SPH_LIST_CHUNK;  // lists hold whole chunks
    ph.cF = (float)(-5.0 * alpha_d / (h * h));
    ph.delta2 = (float)(P0.delta * P0.delta);
    ph.inv_dim = (float)(1.0 / dim);
    ph.visc_dynamic = P0.visc_form == SPH_VISC_DYNAMIC;
    ph.renorm_every = P0.renorm_every;
    ph.renorm_walls = P0.renorm_walls;
    ph.rebuild_every = P0.rebuild_every;
    for (int c = 0; c < 3; ++c) ph.gf[c] = c < dim ? (float)P0.g[c] : 0.f;

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
        if (b == 0) err |= s->alloc(&d.inv, N);
        err |= s->alloc(&d.tag, N);
        err |= s->alloc(&d.iid, N);
    }
    Dev &a0 = s->buf[0];
    if (!err) {
        err |= s->alloc(&a0.cell, N);
        err |= s->alloc(&a0.pos0, N);
        err |= s->alloc(&a0.pos, N);
        err |= s->alloc(&a0.posv, N);
        err |= s->alloc(&a0.velp, N);
        err |= s->alloc(&a0.velq, N);
        err |= s->alloc(&a0.pres, N);
        err |= s->alloc(&a0.nbr, N * (size_t)ph.kmax);
        err |= s->alloc(&a0.ncnt, N);
        err |= s->alloc(&a0.nfcnt, N);
        err |= s->alloc(&a0.walls_moving, 1);
        err |= s->alloc(&a0.nflag, N);
        err |= s->alloc(&a0.mixed, N);
        err |= s->alloc(&a0.nmixed, 1);
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
        err |= s->alloc(&s->bar, 1);
        err |= s->alloc(&s->pair_tot, 4);
        err |= s->alloc(&s->dinst, (size_t)k);
        err |= s->alloc(&s->dfirst, (size_t)k + 1);
        err |= s->alloc(&s->sort.cell_tmp, N);
        err |= s->alloc(&s->sort.slot, N);
        err |= s->alloc(&s->sort.count, (size_t)ncell);
        err |= s->alloc(&s->sort.tmp, N);
        err |= s->alloc(&s->sort.perm, N);
        err |= s->alloc(&s->sort.tile_sums, (size_t)s->ntiles);
        err |= s->alloc(&s->diag_out, (size_t)k * DIAG_STRIDE);
        err |= s->alloc(&s->diag_grav, 4);
        err |= s->alloc(&s->read_buf, N * 9 + 16);
        err |= s->alloc(&s->read_ibuf, N);
        err |= s->alloc(&s->clock, 2);
        err |= s->alloc(&s->amax, (size_t)k);
        err |= s->alloc(&s->motion, 1);
    }
    if (err) return cleanup(SPH_ENOMEM);
    s->sort.ncell = (int)ncell;
    s->sort.n = (int)n;
    s->sort.flags = s->flags;
    Dev &a1 = s->buf[1];
    a1.cell = a0.cell; a1.pos0 = a0.pos0;
    a1.pos = a0.pos; a1.posv = a0.posv; a1.velp = a0.velp; a1.velq = a0.velq; a1.pres = a0.pres;
    a1.nbr = a0.nbr; a1.ncnt = a0.ncnt; a1.nfcnt = a0.nfcnt; a1.walls_moving = a0.walls_moving; a1.nflag = a0.nflag; a1.mixed = a0.mixed; a1.nmixed = a0.nmixed;
    a1.drho_stage = a0.drho_stage; a1.drho_eval = a0.drho_eval;
    a1.T4 = a0.T4; a1.T2 = a0.T2; a1.acc = a0.acc; a1.cstart = a0.cstart;
    a0.flags = a1.flags = s->flags;
    a0.step = a1.step = s->dstep;
    a0.rebuild = a1.rebuild = s->rebuild;
    a0.builds = a1.builds = s->dbuilds;
    a0.inst = a1.inst = s->dinst;
    a0.clock = a1.clock = s->clock;
    a1.inv = a0.inv;
    a0.motion = a1.motion = s->motion;
    for (int c = 0; c < 3; ++c) {
        a0.period[c] = a1.period[c] = s->grid.per[c] ? box_hi[c] - box_lo[c] : 0.0;
        a0.plo[c] = a1.plo[c] = box_lo[c];
    }

    cudaStream_t st = s->stream;
    auto cuda_fail = [&](cudaError_t e) { return cleanup(fail(SPH_ECUDA, cudaGetErrorString(e))); };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMemsetAsync(s->flags, 0, sizeof(unsigned), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->dstep, 0, sizeof(long long), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->dbuilds, 0, sizeof(long long), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(a0.nmixed, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e);
    {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_fail(e);
    }
    {
        // super-cell centres per axis (the FP64 offsets' origins)
        std::vector<double> cen;
        const int dims3[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
        for (int a = 0; a < 3; ++a) {
            s->grid.cen_off[a] = (int)cen.size();
            const int ns = dims3[a] / s->grid.f + 2;
            for (int S = 0; S < ns; ++S) cen.push_back(std::fma((double)S + 0.5, s->grid.Ed, s->grid.lo[a]));
        }
        double *dcen = nullptr;
        if (s->alloc(&dcen, cen.size())) return cleanup(SPH_ENOMEM);
        if ((e = cudaMemcpyAsync(dcen, cen.data(), sizeof(double) * cen.size(), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return cuda_fail(e);
        s->grid.cen = dcen;
    }
    if ((e = cudaMemsetAsync(s->bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->clock, 0, 2 * sizeof(double), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemsetAsync(s->motion, 0, sizeof(Motion), st)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpyAsync(s->dinst, s->hinst.data(), sizeof(Inst) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    std::vector<long long> fl(s->first.begin(), s->first.end());
    if ((e = cudaMemcpyAsync(s->dfirst, fl.data(), sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e);
    double grav[4] = {0, 0, 0, 0};
    for (int c = 0; c < dim; ++c) grav[c] = P0.g[c];
    if ((e = cudaMemcpyAsync(s->diag_grav, grav, sizeof(grav), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e);
    if (n > 0) {
        std::vector<uint8_t> tag((size_t)n);
        std::vector<uint16_t> iid((size_t)n);
        int64_t i = 0;
        for (int q = 0; q < k; ++q)
            for (int64_t c = 0; c < counts[q]; ++c, ++i) {
                // bit 0 oil, bit 1 boundary (fixed or piston), bit 2 piston
                tag[i] = (uint8_t)(phase[i] | (wall[i] ? 2 : 0) | (wall[i] == 2 ? 4 : 0));
                s->npiston += wall[i] == 2;
                iid[i] = (uint16_t)q;
            }
        if ((e = cudaMemcpyAsync(a0.tag, tag.data(), (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e);
        if ((e = cudaMemcpyAsync(a0.iid, iid.data(), sizeof(uint16_t) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e);
        k_iota<<<s->blocks((int)n), 256, 0, st>>>(a0.pid, (int)n);
        k_iota<<<s->blocks((int)n), 256, 0, st>>>(a0.inv, (int)n);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
    *out = s;
    int rc = sph_set_state(s, x, u, rho);
    if (rc) {
        *out = nullptr;
        return cleanup(rc);
    }
    return SPH_OK;
}

}  // namespace

namespace sphgb {

SimView sim_view(sph_sim *s)
{
    SimView v{};
    v.d = s->buf[0];
    v.g = s->grid;
    v.ph = s->phys;
    v.stream = s->stream;
    v.dim = s->dim;
    v.n = s->n;
    v.ninst = s->ninst;
    v.h = s->P.h;
    v.rho0 = s->P.rho0;
    v.npiston = s->npiston;
    return v;
}

void sim_build_lists(sph_sim *s)
{
    if (s->n > 0) s->enqueue_build_cells(true);
}

int sim_check(sph_sim *s) { return s->check_flags(); }

int sim_moved(sph_sim *s, int64_t steps, double elapsed)
{
    if (s->n > 0) {
        k_add_step<<<1, 32, 0, s->stream>>>(s->dstep, (long long)steps, s->clock, elapsed);
        CU(cudaGetLastError());
        CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    }
    s->step += steps;
    return SPH_OK;
}

int sim_snapshot_device(sph_sim *s, double *x, double *u, double *rho)
{
    if (s->n == 0) return SPH_OK;
    const int nb = s->blocks(s->n);
    if (s->dim == 2) {
        k_unpermute<2><<<nb, 256, 0, s->stream>>>(s->D(), RK_X, x, s->read_ibuf);
        k_unpermute<2><<<nb, 256, 0, s->stream>>>(s->D(), RK_U, u, s->read_ibuf);
        k_unpermute<2><<<nb, 256, 0, s->stream>>>(s->D(), RK_RHO, rho, s->read_ibuf);
    } else {
        k_unpermute<3><<<nb, 256, 0, s->stream>>>(s->D(), RK_X, x, s->read_ibuf);
        k_unpermute<3><<<nb, 256, 0, s->stream>>>(s->D(), RK_U, u, s->read_ibuf);
        k_unpermute<3><<<nb, 256, 0, s->stream>>>(s->D(), RK_RHO, rho, s->read_ibuf);
    }
    CU(cudaGetLastError());
    return SPH_OK;
}

int sim_load_device(sph_sim *s, const double *x, const double *u, const double *rho)
{
    if (s->n == 0) return SPH_OK;
    s->enqueue_load(x, u, rho, 0.0);
    CU(cudaGetLastError());
    CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    return SPH_OK;
}

int sim_centroid(sph_sim *s, double c[3])
{
    std::vector<double> all((size_t)12 * s->ninst);
    const int rc = sph_diag_instances(s, all.data());
    for (int k = 0; k < 3; ++k) c[k] = all[6 + k];
    return rc;
}

// Occupancy grid of the handle: spacing d_p = (m_oil / rho0_oil)^(1/dim) of
// instance 0 from the grid's lower corner, covering the cell grid.
struct OccGrid {
    double3 lo;
    double dx;
    int3 dims;
    long long words;
};

OccGrid occ_grid(const sph_sim *s)
{
    const sph_params &P = s->inst_params[0];
    const double dp = std::pow(P.mass[1] / P.rho0[1], 1.0 / s->dim);
    OccGrid o{};
    o.lo = make_double3(s->grid.lo[0], s->grid.lo[1], s->grid.lo[2]);
    o.dx = dp;
    const int nd[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
    int m[3] = {1, 1, 1};
    for (int a = 0; a < s->dim; ++a) m[a] = (int)std::ceil(nd[a] * s->grid.csd / dp);
    o.dims = make_int3(m[0], m[1], m[2]);
    o.words = ((long long)m[0] * m[1] * m[2] + 31) / 32;
    return o;
}

int64_t sim_occupancy_words(sph_sim *s) { return occ_grid(s).words; }

int sim_occupancy(sph_sim *s, unsigned *bm)
{
    const OccGrid o = occ_grid(s);
    CU(cudaMemsetAsync(bm, 0, sizeof(unsigned) * o.words, s->stream));
    if (s->n == 0) return SPH_OK;
    if (s->dim == 2) k_occupancy<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), o.lo, o.dx, o.dims, bm);
    else k_occupancy<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), o.lo, o.dx, o.dims, bm);
    CU(cudaGetLastError());
    return SPH_OK;
}

int sim_occupancy_error(sph_sim *s, const unsigned *a, const unsigned *b, double *err)
{
    if (!s->occ_cnt && s->alloc(&s->occ_cnt, 2)) return SPH_ENOMEM;
    const long long words = occ_grid(s).words;
    CU(cudaMemsetAsync(s->occ_cnt, 0, 2 * sizeof(unsigned long long), s->stream));
    const int blocks = (int)std::min<long long>((words + 255) / 256, 1024);
    k_occupancy_cmp<<<std::max(blocks, 1), 256, 0, s->stream>>>(a, b, words, s->occ_cnt);
    CU(cudaGetLastError());
    unsigned long long c[2];
    CU(cudaMemcpyAsync(c, s->occ_cnt, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    *err = c[1] > 0 ? (double)c[0] / (double)c[1] : (c[0] > 0 ? 1.0e30 : 0.0);
    return SPH_OK;
}

void *sim_ext(sph_sim *s) { return s->ext; }

void sim_set_ext(sph_sim *s, void *p, void (*free_fn)(void *))
{
    if (s->ext && s->ext_free) s->ext_free(s->ext);
    s->ext = p;
    s->ext_free = free_fn;
}

}  // namespace sphgb

extern "C" {

const char *sph_last_error(void) { return g_err.c_str(); }

int sph_create(const sph_params *params, int64_t n, const double *x, const double *u, const double *rho,
               const uint8_t *phase, const uint8_t *wall, void *stream, sph_handle *out)
{
    if (n < 0) {
        if (out) *out = nullptr;
        return fail(SPH_EINVAL, "n must be in [0, 2^26]");
    }
    return create_sim(params, 1, &n, x, u, rho, phase, wall, stream, out);
}

int sph_create_batch(int k, const sph_params *params, const int64_t *counts, const double *x, const double *u,
                     const double *rho, const uint8_t *phase, const uint8_t *wall, void *stream, sph_handle *out)
{
    if (!params || !counts) {
        if (out) *out = nullptr;
        return fail(SPH_EINVAL, "params or counts is NULL");
    }
    return create_sim(params, k, counts, x, u, rho, phase, wall, stream, out);
}

// Queues the upload and load of a state (original order) without waiting.
int sph_sim::enqueue_set_state(const double *x, const double *u, const double *rho)
{
    const size_t nn = (size_t)n, dd = (size_t)dim;
    // device arrays are read in place by the load kernel; host arrays are
    // staged by the copy engines (a load kernel reading pinned memory in place
    // measured slower: its per-particle work and scattered writes leave too
    // few reads in flight to fill the host link)
    const double *dx = device_view(x), *du = device_view(u), *dr = device_view(rho);
    if (!dx) {
        dx = read_buf;
        CU(cudaMemcpyAsync(read_buf, x, sizeof(double) * nn * dd, cudaMemcpyHostToDevice, stream));
    }
    if (!du) {
        du = read_buf + nn * dd;
        CU(cudaMemcpyAsync(read_buf + nn * dd, u, sizeof(double) * nn * dd, cudaMemcpyHostToDevice, stream));
    }
    if (!dr) {
        dr = read_buf + 2 * nn * dd;
        CU(cudaMemcpyAsync(read_buf + 2 * nn * dd, rho, sizeof(double) * nn, cudaMemcpyHostToDevice, stream));
    }
    // the lists are kept when they still hold the new state (tested against the
    // skin with the last step size; a fixed rebuild cadence or no step yet rebuilds)
    const double check_dt = P.rebuild_every == 0 ? last_dt : 0.0;
    enqueue_load(dx, du, dr, check_dt);
    CU(cudaGetLastError());
    if (!(check_dt > 0)) CU(cudaMemsetAsync(rebuild, 0xff, sizeof(unsigned), stream));
    return SPH_OK;
}

int sph_set_state(sph_handle s, const double *x, const double *u, const double *rho)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->n == 0) return SPH_OK;
    if (!x || !u || !rho) return fail(SPH_EINVAL, "an input array is NULL");
    const int rc = s->enqueue_set_state(x, u, rho);
    if (rc != SPH_OK) return rc;
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
}

int sph_create_dev(const sph_params *params, int64_t n, const double *x_dev, const double *u_dev,
                   const double *rho_dev, const uint8_t *phase_dev, const uint8_t *wall_dev, void *stream,
                   sph_handle *out)
{
    if (out) *out = nullptr;
    if (n < 0 || n > ((int64_t)1 << 26)) return fail(SPH_EINVAL, "n must be in [0, 2^26]");
    if (!params) return fail(SPH_EINVAL, "params is NULL");
    if (params->dim != 2 && params->dim != 3) return fail(SPH_EINVAL, "dim must be 2 or 3");
    if (n > 0 && (!x_dev || !u_dev || !rho_dev || !phase_dev || !wall_dev))
        return fail(SPH_EINVAL, "an input array is NULL");
    // the creation path validates and packs on the host: stage the arrays there
    const size_t nv = (size_t)n * params->dim;
    std::vector<double> x(nv), u(nv), rho((size_t)n);
    std::vector<uint8_t> phase((size_t)n), wall((size_t)n);
    cudaStream_t st = (cudaStream_t)stream;
    if (n > 0) {
        CU(cudaMemcpyAsync(x.data(), x_dev, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(u.data(), u_dev, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(rho.data(), rho_dev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(phase.data(), phase_dev, (size_t)n, cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(wall.data(), wall_dev, (size_t)n, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
    }
    return create_sim(params, 1, &n, x.data(), u.data(), rho.data(), phase.data(), wall.data(), stream, out);
}

int sph_set_piston(sph_handle s, int axis, int ncomp, const double *amp, const double *omega, const double *phase,
                   double t_end)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->ninst != 1) return fail(SPH_EINVAL, "a piston motion needs a single-instance handle");
    if (axis < 0 || axis >= s->dim) return fail(SPH_EINVAL, "axis must be in [0, dim)");
    if (ncomp < 0 || ncomp > MOTION_MAX) return fail(SPH_EINVAL, "ncomp must be in [0, 8]");
    if (ncomp > 0 && (!amp || !omega || !phase)) return fail(SPH_EINVAL, "a component array is NULL");
    if (std::isnan(t_end) || t_end < 0) return fail(SPH_EINVAL, "t_end must be >= 0 (may be infinite)");
    Motion m{};
    m.axis = axis;
    m.ncomp = ncomp;
    m.t_end = t_end;
    for (int c = 0; c < ncomp; ++c) {
        if (!std::isfinite(amp[c]) || !std::isfinite(omega[c]) || !std::isfinite(phase[c]))
            return fail(SPH_EINVAL, "the motion components must be finite");
        m.amp[c] = amp[c];
        m.omega[c] = omega[c];
        m.phase[c] = phase[c];
    }
    CU(cudaMemcpyAsync(s->motion, &m, sizeof(Motion), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    s->moving = ncomp > 0;
    return SPH_OK;
}

int sph_get_time(sph_handle s, double *t)
{
    if (!s || !t) return fail(SPH_EINVAL, "NULL argument");
    double c[2];
    CU(cudaMemcpyAsync(c, s->clock, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    *t = c[0] + c[1];
    return s->check_flags();
}

int sph_set_time(sph_handle s, double t)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!std::isfinite(t)) return fail(SPH_EINVAL, "t must be finite");
    const double c[2] = {t, 0.0};
    CU(cudaMemcpyAsync(s->clock, c, sizeof(c), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
}

int sph_suggest_dt(sph_handle s, double *dt)
{
    if (!s || !dt) return fail(SPH_EINVAL, "NULL argument");
    const int k = s->ninst;
    std::vector<float> amax((size_t)k, 0.f);
    if (s->evaluated && s->n > 0) {
        CU(cudaMemsetAsync(s->amax, 0, sizeof(unsigned) * k, s->stream));
        k_amax<<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->amax);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(amax.data(), s->amax, sizeof(float) * k, cudaMemcpyDeviceToHost, s->stream));
        CU(cudaStreamSynchronize(s->stream));
        int rc = s->check_flags();
        if (rc) return rc;
    }
    const double h = s->P.h, pi = 3.14159265358979323846;
    double best = INFINITY;
    for (int q = 0; q < k; ++q) {
        const sph_params &P = s->inst_params[q];
        double d = 0.25 * h / P.c0;                                           // acoustic (CFL)
        const double nu = std::max(P.mu[0] / P.rho0[0], P.mu[1] / P.rho0[1]);
        if (nu > 0) d = std::min(d, 0.125 * h * h / nu);                      // viscous diffusion
        if (P.alpha_s > 0)                                                    // capillary waves
            d = std::min(d, 0.25 * std::sqrt(std::min(P.rho0[0], P.rho0[1]) * h * h * h / (2.0 * pi * P.alpha_s)));
        const double a = std::sqrt((double)amax[q]);
        if (a > 0) d = std::min(d, 0.25 * std::sqrt(h / a));                  // body force
        best = std::min(best, d / s->hinst[q].dt_scale);
    }
    *dt = best;
    return SPH_OK;
}

int sph_perturb_state(sph_handle s, double sigma_u, double sigma_rho, uint64_t seed)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(sigma_u >= 0) || !(sigma_rho >= 0) || !std::isfinite(sigma_u) || !std::isfinite(sigma_rho))
        return fail(SPH_EINVAL, "sigma_u and sigma_rho must be finite and >= 0");
    if (s->n == 0) return SPH_OK;
    if (s->dim == 2) k_perturb<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), sigma_u, sigma_rho, seed);
    else k_perturb<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), sigma_u, sigma_rho, seed);
    CU(cudaGetLastError());
    // the stage records derive from the state: rebuilt with the lists
    CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    return SPH_OK;
}

int sph_oil_occupancy_diff(sph_handle a, sph_handle b, double *err)
{
    if (!a || !b || !err) return fail(SPH_EINVAL, "NULL argument");
    const OccGrid ga = occ_grid(a), gb = occ_grid(b);
    if (a->dim != b->dim || ga.dims.x != gb.dims.x || ga.dims.y != gb.dims.y || ga.dims.z != gb.dims.z ||
        ga.dx != gb.dx || ga.lo.x != gb.lo.x || ga.lo.y != gb.lo.y || ga.lo.z != gb.lo.z)
        return fail(SPH_EINVAL, "the handles' occupancy grids differ (cell grid and oil particle volume)");
    if (!a->occ && a->alloc(&a->occ, (size_t)ga.words)) return SPH_ENOMEM;
    if (!b->occ && b->alloc(&b->occ, (size_t)gb.words)) return SPH_ENOMEM;
    int rc = sim_occupancy(a, a->occ);
    if (!rc) rc = sim_occupancy(b, b->occ);
    if (rc) return rc;
    CU(cudaStreamSynchronize(b->stream));
    if ((rc = sim_occupancy_error(a, a->occ, b->occ, err))) return rc;
    if ((rc = a->check_flags())) return rc;
    return b->check_flags();
}

int sph_set_dt_scales(sph_handle s, const double *scales)
{
    if (!s || !scales) return fail(SPH_EINVAL, "NULL argument");
    for (int q = 0; q < s->ninst; ++q)
        if (!(scales[q] > 0 && scales[q] <= 1.0)) return fail(SPH_EINVAL, "dt scales must be in (0, 1]");
    for (int q = 0; q < s->ninst; ++q) s->hinst[q].dt_scale = scales[q];
    CU(cudaMemcpyAsync(s->dinst, s->hinst.data(), sizeof(Inst) * s->ninst, cudaMemcpyHostToDevice, s->stream));
    // the rebuild test looks half a step ahead with the previous step size
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
    s->evaluated = true;
    CU(cudaGetLastError());
    return SPH_OK;
}

int sph_step(sph_handle s, double dt)
{
    NvtxScope nvtx_scope("sph_step");
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (s->n > 0) {
        // the rebuild test looks half a step ahead with the previous dt
        if (dt != s->last_dt) CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
        s->last_dt = dt;
        s->enqueue_step(dt);
        CU(cudaGetLastError());
        s->evaluated = true;
    }
    s->step += 1;
    return SPH_OK;
}

int sph_run(sph_handle s, double dt, int64_t nsteps, int graph)
{
    NvtxScope nvtx_scope("sph_run");
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    if (s->n == 0) {
        s->step += nsteps;
        return SPH_OK;
    }
    const int rc = s->enqueue_run(dt, nsteps, graph != 0);
    if (rc != SPH_OK) return rc;
    return s->check_flags();
}

// Queues nsteps steps (graph-replayed when graph) without waiting.
int sph_sim::enqueue_run(double dt, int64_t nsteps, bool graph)
{
    const bool use_graph = graph && !timing;
    if (dt != last_dt) CU(cudaMemsetAsync(rebuild, 0xff, sizeof(unsigned), stream));
    last_dt = dt;
    if (use_graph) {
        if (!gexec || gdt != dt) {
            const int rc = capture_step_graph(dt);
            if (rc != SPH_OK) return rc;
        }
        for (int64_t k = 0; k < nsteps; ++k) {
            CU(cudaGraphLaunch(gexec, stream));
            step += 1;
        }
    } else {
        for (int64_t k = 0; k < nsteps; ++k) {
            enqueue_step(dt);
            CU(cudaGetLastError());
            step += 1;
        }
    }
    if (nsteps > 0) evaluated = true;
    return SPH_OK;
}

int sph_run_persistent(sph_handle s, double dt, int64_t nsteps, int graph)
{
    NvtxScope nvtx_scope("sph_run_persistent");
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (nsteps < 0 || nsteps > 0x7fffffff) return fail(SPH_EINVAL, "nsteps must be in [0, 2^31)");
    if (s->n == 0 || nsteps == 0) {
        s->step += nsteps;
        return SPH_OK;
    }
    if (dt != s->last_dt) CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    s->last_dt = dt;
    const int shape = (s->pbs * 100000 + s->pgrid) * 2 + s->pdyn;
    if (graph && !s->timing) {
        if (!s->pexec || s->pdt != dt || s->psteps != nsteps || s->pshape != shape) {
            cudaGraph_t gr = nullptr;
            CU(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
            int rc = s->launch_persistent(dt, (int)nsteps);
            cudaError_t e = cudaStreamEndCapture(s->stream, &gr);
            if (rc) {
                if (gr) cudaGraphDestroy(gr);
                return rc;
            }
            if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            if (s->pexec) cudaGraphExecDestroy(s->pexec);
            s->pexec = nullptr;
            e = cudaGraphInstantiate(&s->pexec, gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return fail(SPH_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            s->pdt = dt;
            s->psteps = nsteps;
            s->pshape = shape;
        }
        CU(cudaGraphLaunch(s->pexec, s->stream));
    } else {
        int rc = s->launch_persistent(dt, (int)nsteps);
        if (rc) return rc;
    }
    s->step += nsteps;
    s->evaluated = true;
    return s->check_flags();
}

int sph_set_launch_shape(sph_handle s, int block, int grid_blocks, int dynamic_chunks)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (block != 128 && block != 256 && block != 512) return fail(SPH_EINVAL, "block must be 128, 256 or 512");
    if (grid_blocks < 0) return fail(SPH_EINVAL, "grid_blocks must be >= 0");
    if (dynamic_chunks != 0 && dynamic_chunks != 1) return fail(SPH_EINVAL, "dynamic_chunks must be 0 or 1");
    int gsz = 0;
    int rc = s->persistent_shape(block, grid_blocks, &gsz, nullptr);
    if (rc) return rc;
    s->pbs = block;
    s->pgrid = grid_blocks;
    s->pdyn = dynamic_chunks;
    return SPH_OK;
}

int sph_get_launch_shape(sph_handle s, int *block, int *grid_blocks, int *dynamic_chunks)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    int gsz = 0;
    int rc = s->persistent_shape(s->pbs, s->pgrid, &gsz, nullptr);
    if (rc) return rc;
    if (block) *block = s->pbs;
    if (grid_blocks) *grid_blocks = gsz;
    if (dynamic_chunks) *dynamic_chunks = s->pdyn;
    return SPH_OK;
}

int sph_autotune(sph_handle s, double dt, int trial_steps, int *best_block, int *best_grid_blocks,
                 int *best_dynamic_chunks, double *best_ms_per_step)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt) || trial_steps < 1)
        return fail(SPH_EINVAL, "dt must be positive and trial_steps >= 1");
    if (s->n == 0) return SPH_OK;
    // the trials advance the state: keep it and put it back afterwards
    const size_t n = (size_t)s->n, dim = (size_t)s->dim;
    std::vector<double> x(n * dim), u(n * dim), rho(n);
    int rc = sph_read(s, SPH_FIELD_POS, x.data(), (int64_t)(x.size() * 8));
    if (!rc) rc = sph_read(s, SPH_FIELD_VEL, u.data(), (int64_t)(u.size() * 8));
    if (!rc) rc = sph_read(s, SPH_FIELD_RHO, rho.data(), (int64_t)(rho.size() * 8));
    if (rc) return rc;
    long long dstep = 0, dbuilds = 0;
    double clock[2] = {0, 0};
    CU(cudaMemcpyAsync(clock, s->clock, sizeof(clock), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(&dstep, s->dstep, sizeof(dstep), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaMemcpyAsync(&dbuilds, s->dbuilds, sizeof(dbuilds), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // candidate shapes: every co-resident multiple of the SM count and, for
    // inputs smaller than twice such a grid's threads, fractions of the SM
    // count (fewer blocks make each grid barrier cheaper)
    struct Shape {
        int bs, grid, dyn;
    };
    std::vector<Shape> shapes;
    for (int bs : PERSIST_BS) {
        int maxg = 0;
        rc = s->persistent_shape(bs, 0, &maxg, nullptr);
        if (rc) return rc;
        std::vector<int> grids;
        for (int g = sms; g <= maxg; g += sms) grids.push_back(g);
        for (int div : {2, 4, 8, 19})
            if (sms / div >= 1 && (int64_t)(sms / div) * bs <= 2 * (int64_t)n) grids.push_back(sms / div);
        for (int g : grids)
            for (int dyn : {1, 0}) shapes.push_back({bs, g, dyn});
    }
    const int64_t host_step = s->step;
    const double host_last_dt = s->last_dt;
    const bool timing = s->timing;
    s->timing = false;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    double best = 1e300;
    int bb = s->pbs, bg = s->pgrid, bd = s->pdyn;
    for (const Shape &sh : shapes) {
        s->pbs = sh.bs;
        s->pgrid = sh.grid;
        s->pdyn = sh.dyn;
        rc = sph_set_state(s, x.data(), u.data(), rho.data());
        if (!rc) rc = sph_run_persistent(s, dt, 1, 0);  // warm-up, includes a list build
        if (rc) break;
        cudaEventRecord(e0, s->stream);
        rc = s->launch_persistent(dt, trial_steps);
        cudaEventRecord(e1, s->stream);
        if (!rc) rc = s->check_flags();
        if (rc) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / trial_steps;
        if (per < best) {
            best = per;
            bb = sh.bs;
            bg = sh.grid;
            bd = sh.dyn;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->timing = timing;
    s->pbs = bb;
    s->pgrid = bg;
    s->pdyn = bd;
    // the state and counters as they were before the trials (the next step
    // rebuilds the lists)
    int rc2 = sph_set_state(s, x.data(), u.data(), rho.data());
    CU(cudaMemcpyAsync(s->clock, clock, sizeof(clock), cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemsetAsync(s->rebuild, 0xff, sizeof(unsigned), s->stream));
    CU(cudaMemcpyAsync(s->dstep, &dstep, sizeof(dstep), cudaMemcpyHostToDevice, s->stream));
    CU(cudaMemcpyAsync(s->dbuilds, &dbuilds, sizeof(dbuilds), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    s->step = host_step;
    s->last_dt = host_last_dt;
    if (rc) return rc;
    if (rc2) return rc2;
    if (best_block) *best_block = bb;
    if (best_grid_blocks) *best_grid_blocks = bg;
    if (best_dynamic_chunks) *best_dynamic_chunks = bd;
    if (best_ms_per_step) *best_ms_per_step = best;
    return SPH_OK;
}

int sph_test_stall_barrier(sph_handle s)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    // with `count` at a value no arrival can reach from below, no block is the
    // last to arrive: every block waits out its one-second limit and returns
    int gsz = 0;
    int rc = s->persistent_shape(s->pbs, s->pgrid, &gsz, nullptr);
    if (rc) return rc;
    const unsigned count = (unsigned)gsz;
    CU(cudaMemcpyAsync(&s->bar->count, &count, sizeof(count), cudaMemcpyHostToDevice, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
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
    if (int rc = s->enqueue_read(kind, integer, host_out, need, 0)) return rc;
    CU(cudaStreamSynchronize(s->stream));
    return SPH_OK;
}

// Queues the unpermuted reads of x, u and rho without waiting.
int sph_sim::enqueue_read_state(double *x, double *u, double *rho)
{
    const size_t nn = (size_t)n, dd = (size_t)dim;
    // pinned outputs (x and u on 16-byte boundaries): one kernel writes all
    // three in place, in whole lines
    double *px = pinned_view(x), *pu = pinned_view(u), *pr = pinned_view(rho);
    if (px && pu && pr && ((uintptr_t)px % 16) == 0 && ((uintptr_t)pu % 16) == 0) {
        const int nb = blocks(n, RS_TILE);
        if (dim == 2) k_read_state_lines<2><<<nb, RS_TILE, 0, stream>>>(D(), px, pu, pr);
        else k_read_state_lines<3><<<nb, RS_TILE, 0, stream>>>(D(), px, pu, pr);
        CU(cudaGetLastError());
        return SPH_OK;
    }
    int rc = enqueue_read(RK_X, false, x, nn * dd * 8, 0);
    if (!rc) rc = enqueue_read(RK_U, false, u, nn * dd * 8, nn * dd);
    if (!rc) rc = enqueue_read(RK_RHO, false, rho, nn * 8, 2 * nn * dd);
    return rc;
}

int sph_read_state(sph_handle s, double *x, double *u, double *rho)
{
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (s->n == 0) return SPH_OK;
    if (!x || !u || !rho) return fail(SPH_EINVAL, "an output array is NULL");
    const int rc = s->enqueue_read_state(x, u, rho);
    if (rc) return rc;
    return s->check_flags();
}

int sph_advance_host(sph_handle s, double dt, int64_t nsteps, const double *x, const double *u, const double *rho,
                     double *x_out, double *u_out, double *rho_out)
{
    NvtxScope nvtx_scope("sph_advance_host");
    if (!s) return fail(SPH_EINVAL, "handle is NULL");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be positive and finite");
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    if (!x || !u || !rho) return fail(SPH_EINVAL, "an input array is NULL");
    if (!x_out || !u_out || !rho_out) return fail(SPH_EINVAL, "an output array is NULL");
    if (s->n == 0) {
        s->step += nsteps;
        return SPH_OK;
    }
    int rc = s->enqueue_set_state(x, u, rho);
    if (rc == SPH_OK) rc = s->enqueue_run(dt, nsteps, true);
    if (rc == SPH_OK) rc = s->enqueue_read_state(x_out, u_out, rho_out);
    if (rc != SPH_OK) {
        cudaStreamSynchronize(s->stream);
        return rc;
    }
    return s->check_flags();
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
    int *cnt = s->read_ibuf;
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

int sph_pair_classes(sph_handle s, int64_t out[4])
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    out[0] = out[1] = out[2] = out[3] = 0;
    if (s->n == 0) return SPH_OK;
    s->enqueue_build_cells(true);
    CU(cudaMemsetAsync(s->pair_tot, 0, 4 * sizeof(unsigned long long), s->stream));
    if (s->dim == 2) k_pair_stats<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->grid, s->phys, s->pair_tot);
    else k_pair_stats<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), s->grid, s->phys, s->pair_tot);
    CU(cudaGetLastError());
    unsigned long long h[4];
    CU(cudaMemcpyAsync(h, s->pair_tot, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    for (int q = 0; q < 4; ++q) out[q] = (int64_t)h[q];
    return s->check_flags();
}

int sph_pair_stats(sph_handle s, int64_t out[2])
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    int64_t c[4];
    const int rc = sph_pair_classes(s, c);
    out[0] = c[0];
    out[1] = c[1];
    return rc;
}

int sph_diag_instances(sph_handle s, double *out)
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    const int k = s->ninst;
    for (int q = 0; q < 12 * k; ++q) out[q] = 0.0;
    if (s->n == 0) return SPH_OK;
    const size_t n = (size_t)s->n, dim = (size_t)s->dim;
    double *x = s->read_buf, *u = s->read_buf + n * dim;
    // original-order positions (instance frames), velocities and tags
    if (s->dim == 2) {
        k_unpermute<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_X, x, s->read_ibuf);
        k_unpermute<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_U, u, s->read_ibuf);
        k_unpermute<2><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_TAG, x, s->read_ibuf);
        k_diag_inst<2><<<k, DIAG_THREADS, 0, s->stream>>>(s->dfirst, x, u, s->read_ibuf, s->dinst, s->diag_grav,
                                                           s->diag_out);
    } else {
        k_unpermute<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_X, x, s->read_ibuf);
        k_unpermute<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_U, u, s->read_ibuf);
        k_unpermute<3><<<s->blocks(s->n), 256, 0, s->stream>>>(s->D(), RK_TAG, x, s->read_ibuf);
        k_diag_inst<3><<<k, DIAG_THREADS, 0, s->stream>>>(s->dfirst, x, u, s->read_ibuf, s->dinst, s->diag_grav,
                                                           s->diag_out);
    }
    CU(cudaGetLastError());
    std::vector<double> r((size_t)k * DIAG_STRIDE);
    CU(cudaMemcpyAsync(r.data(), s->diag_out, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, s->stream));
    CU(cudaStreamSynchronize(s->stream));
    for (int q = 0; q < k; ++q) {
        const double *v = r.data() + (size_t)q * DIAG_STRIDE;
        double *o = out + (size_t)q * 12;
        o[0] = v[0];
        for (int c = 0; c < s->dim; ++c) o[1 + c] = v[1 + c];
        o[4] = v[4];
        o[5] = v[5];
        o[10] = v[10];
        o[11] = v[9];
        if (v[9] > 0) {
            for (int c = 0; c < s->dim; ++c) o[6 + c] = v[6 + c];
            const double no = v[9];
            double lmin, lmax;
            if (s->dim == 2) {
                const double a = v[11] / no, b = v[12] / no, d = v[14] / no;
                const double tr = a + d, det = a * d - b * b;
                const double disc = std::sqrt(std::max(0.25 * tr * tr - det, 0.0));
                lmin = 0.5 * tr - disc;
                lmax = 0.5 * tr + disc;
            } else {
                double A[6];
                for (int c = 0; c < 6; ++c) A[c] = v[11 + c] / no;
                eig3(A, lmin, lmax);
            }
            o[9] = lmax > 0 ? std::sqrt(std::max(lmin, 0.0) / lmax) : 0.0;
        }
    }
    return s->check_flags();
}

int sph_diag(sph_handle s, double out[12])
{
    if (!s || !out) return fail(SPH_EINVAL, "NULL argument");
    if (s->ninst == 1) return sph_diag_instances(s, out);
    std::vector<double> all((size_t)12 * s->ninst);
    const int rc = sph_diag_instances(s, all.data());
    for (int c = 0; c < 12; ++c) out[c] = all[c];
    return rc;
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
int64_t sph_num_instances(sph_handle s) { return s ? s->ninst : 0; }

void sph_destroy(sph_handle s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->ext && s->ext_free) s->ext_free(s->ext);
    s->collect_timing();
    for (auto e : s->free_events) cudaEventDestroy(e);
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->pexec) cudaGraphExecDestroy(s->pexec);
    for (void *p : s->allocs) cudaFree(p);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
