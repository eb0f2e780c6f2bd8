// Internal interface between the simulation handle (sph_api.cu) and the
// learned surrogate (mpnn.cu); not part of the C ABI.
#pragma once

#include "sph.h"
#include "sph_kernels.cuh"

#include <cuda_runtime.h>

#include <string>

namespace sphgb {

struct SimView {
    Dev d;                 // device arrays, sorted order
    Grid g;
    Phys ph;
    cudaStream_t stream;
    int dim, n, ninst;
    double h;
    const double *rho0;    // per-phase reference density of instance 0 (host)
    int64_t npiston;       // particles with a prescribed (piston) motion
};

int set_error(int code, const std::string &msg);
SimView sim_view(sph_sim *s);
// Queues a cell and neighbour-list build at the current positions.
void sim_build_lists(sph_sim *s);
// Waits for the stream and reports device error flags.
int sim_check(sph_sim *s);
// Adds `steps` to the host and device step counters and `elapsed` to the
// device clock, and marks the lists for a rebuild (the state moved by more
// than the skin allows).
int sim_moved(sph_sim *s, int64_t steps, double elapsed);
// Original-order state <-> device arrays (x, u: n * dim; rho: n).
int sim_snapshot_device(sph_sim *s, double *x, double *u, double *rho);
int sim_load_device(sph_sim *s, const double *x, const double *u, const double *rho);
// Oil centroid of instance 0 (FP64), or an error code.
int sim_centroid(sph_sim *s, double c[3]);
// Oil occupancy bitmaps (cells of spacing d_p holding oil): the words of one
// bitmap, queueing one into bm, and |a xor b| / |b| (waits for the stream).
int64_t sim_occupancy_words(sph_sim *s);
int sim_occupancy(sph_sim *s, unsigned *bm);
int sim_occupancy_error(sph_sim *s, const unsigned *a, const unsigned *b, double *err);
// Slot owned by the surrogate, freed with the handle.
void *sim_ext(sph_sim *s);
void sim_set_ext(sph_sim *s, void *p, void (*free_fn)(void *));

}  // namespace sphgb
