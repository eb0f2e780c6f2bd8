// Learned k-step surrogate of the particle loop: a message-passing network
// over the SPH neighbour graph (edges |r_ij| < 2h), BF16 operands on the
// tensor cores (umma.cuh) with FP32 accumulation, hand-written forward and
// backward kernels, Adam, and the C ABI declared in include/sph_surrogate.h.
//
// The network and its parameter format are those of surrogate_layout.py:
// encoder, two rounds of [edge MLP on (h_i, h_j, e_ij), sum over j scaled by
// 1/k_ref, residual node MLP on (h, M)], decoder.  Every dense layer is one
// tcgen05 contraction over all nodes.  The edge MLP's first layer is split
// by blocks (W1 h_i + b1 and W2 h_j are node contractions, W3 e_ij is formed
// per edge) and its second layer, being linear, is applied after the sum
// (We2 S_i + deg_i / k_ref be2), so the per-edge work is one gather, the
// SiLU and the sum.  Nodes are the particles in the simulation's sorted
// order; the edges are the entries of its neighbour list closer than 2h.
#include "sph_internal.h"
#include "sph_kernels.cuh"
#include "sph_surrogate.h"
#include "umma.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

using namespace sphgb;
using bf16 = __nv_bfloat16;

namespace {

constexpr int H = 128;        // hidden width
constexpr int FIN = 16;       // padded node input width
constexpr int FOUT = 16;      // padded output width
constexpr int EW = 256;       // threads of the edge kernels (8 warps, one node each)

#define CUR(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return set_error(SPH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Offsets of the parameter tensors in the flat vector, in the order of
// surrogate_layout.layout().
struct Layout {
    int dim = 0, nin = 0, ne = 0, nout = 0;
    int enc1w, enc1b, enc2w, enc2b;
    int w1[2], b1[2], w2[2], w3[2], we2[2], be2[2], n1[2], n1b[2], n2[2], n2b[2];
    int dec1w, dec1b, dec2w, dec2b;
    int total = 0;
};

Layout make_layout(int dim)
{
    Layout L;
    L.dim = dim;
    L.nin = 2 * dim + 4;
    L.ne = 2 * dim + 3;
    L.nout = 2 * dim + 1;
    int o = 0;
    auto take = [&](int k) {
        const int r = o;
        o += k;
        return r;
    };
    L.enc1w = take(H * L.nin);
    L.enc1b = take(H);
    L.enc2w = take(H * H);
    L.enc2b = take(H);
    for (int r = 0; r < 2; ++r) {
        L.w1[r] = take(H * H);
        L.b1[r] = take(H);
        L.w2[r] = take(H * H);
        L.w3[r] = take(H * L.ne);
        L.we2[r] = take(H * H);
        L.be2[r] = take(H);
        L.n1[r] = take(H * 2 * H);
        L.n1b[r] = take(H);
        L.n2[r] = take(H * H);
        L.n2b[r] = take(H);
    }
    L.dec1w = take(H * H);
    L.dec1b = take(H);
    L.dec2w = take(L.nout * H);
    L.dec2b = take(L.nout);
    L.total = o;
    return L;
}

struct Surrogate {
    int dim = 0, n = 0, npad = 0;
    Layout L;
    float k_ref = 1.f, t_jump = 0.f, sd_edge_u = 1.f, sd_edge_rho = 1.f;
    double t_jump64 = 0.0;       // the jump's time span (the device clock advances by it)
    std::vector<float> norm;     // mu_in, sd_in, mu_out, sd_out
    float *norm_d = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    long long adam_t = 0;
    // packed BF16 weights: forward (B operands) and transposed (backward)
    bf16 *Wenc1, *Wenc2, *Wpq[2], *We2[2], *Wn1[2], *Wn2[2], *Wd1, *Wd2;
    bf16 *Wd2T, *Wd1T, *Wn2T[2], *Wn1T[2], *We2T[2], *WpqT[2], *Wenc2T;
    float *bpq[2], *bd2;
    // forward activations (rows: nodes in sorted order, padded to npad, zero beyond n)
    bf16 *X16, *A0, *A1[2], *S[2], *G1[2], *hLb, *A2;
    __half *PQ[2];               // [P | Q] node terms of the edge MLP's first layer, FP16
    __half *PQf = nullptr;       // the same with the state-difference channels folded in (forward)
    float *Z0, *h[3], *degs, *Z1[2], *Z2, *Y;
    float4 *NF;                  // per node: u / sd_edge_u (xyz), density deviation / sd_edge_rho
    // backward
    float *dYf, *dZf, *dA, *dh, *dh2, *dS;
    bf16 *dYb, *dZb, *dAb, *dhb, *dPQ, *T1, *T2;
    double *loss_d = nullptr;
    unsigned *err = nullptr;
    // judge snapshots (original order)
    double *sx = nullptr, *su = nullptr, *sr = nullptr;
    double *vx = nullptr, *vu = nullptr, *vr = nullptr;   // last verified state
    // judge: oil occupancy bitmaps of the jump and of the plain steps, the
    // interface tolerance (0: not used to reject) and the last run's maxima
    unsigned *occ_a = nullptr, *occ_b = nullptr;
    double itol = 0.0, max_cerr = 0.0, max_ierr = 0.0;
    std::vector<void *> allocs;

    ~Surrogate()
    {
        for (void *p : allocs) cudaFree(p);
    }
};

void free_surrogate(void *p) { delete static_cast<Surrogate *>(p); }

template <class T>
int dalloc(Surrogate &S, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return set_error(SPH_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    S.allocs.push_back(q);
    cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T));
    *p = static_cast<T *>(q);
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// Kernels

// Derivative of SiLU with the fast reciprocal (relative error ~1e-6, far
// below the BF16 rounding of the network's operands).
__device__ __forceinline__ float dsilu(float z)
{
    const float s = __fdividef(1.f, 1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// dst[(row_off + r) * ld + c] = W[r][c], or transposed dst[c * ld + row_off + r].
__global__ void k_pack(const float *W, int rows, int cols, bf16 *dst, int ld, int row_off, int transpose)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows * cols) return;
    const int r = k / cols, c = k % cols;
    const bf16 v = __float2bfloat16_rn(W[k]);
    if (transpose) dst[(size_t)c * ld + row_off + r] = v;
    else dst[(size_t)(row_off + r) * ld + c] = v;
}

__global__ void k_copy_f(const float *src, float *dst, int count)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) dst[k] = src[k];
}

// Normalised node inputs [u, (rho - rho0)/rho0, oil, wall, T a,
// T (Drho/Dt)/rho0] (sorted order; the rates are those of the evaluation at
// the current state), and the per-node terms of the edge state differences.
template <int DIM>
__global__ void k_features(Dev d, const float *norm, float T, float inv_su, float inv_sr, bf16 *X, float4 *NF)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    constexpr int NIN = 2 * DIM + 4;
    const uint8_t tg = d.tag[k];
    const Inst &I = d.inst[d.iid[k]];
    const float inv_rho0 = by_phase(tg & 1, I.inv_rho0);
    const float4 a = d.acc[k];
    float raw[NIN];
#pragma unroll
    for (int c = 0; c < DIM; ++c) raw[c] = (float)d.u[(size_t)c * d.n + k];
    raw[DIM] = d.drho[k] * inv_rho0;
    raw[DIM + 1] = (float)(tg & 1);
    raw[DIM + 2] = (float)((tg >> 1) & 1);
    raw[DIM + 3] = T * a.x;
    raw[DIM + 4] = T * a.y;
    if (DIM == 3) raw[DIM + 5] = T * a.z;
    raw[2 * DIM + 3] = T * a.w * inv_rho0;
    __align__(16) bf16 out[FIN];
#pragma unroll
    for (int c = 0; c < FIN; ++c) out[c] = __float2bfloat16_rn(c < NIN ? (raw[c] - norm[c]) / norm[NIN + c] : 0.f);
#pragma unroll
    for (int c = 0; c < FIN; c += 8) *(uint4 *)(X + (size_t)k * FIN + c) = *(const uint4 *)(out + c);
    NF[k] = make_float4(raw[0] * inv_su, raw[1] * inv_su, DIM == 3 ? raw[2] * inv_su : 0.f, raw[DIM] * inv_sr);
}

// Edge features of the pair (i, j): r_ij / 2h (DIM), |r_ij| / 2h,
// phase_i != phase_j, (u_i - u_j) / sd_edge_u (DIM), density deviation
// difference / sd_edge_rho.
template <int DIM>
__device__ __forceinline__ bool edge_features(const Dev &d, const Grid &g, float R2, float inv2h, const float4 &oi,
                                              int phi, const float4 &nfi, const float4 *NF, unsigned e, int &j,
                                              float (&ef)[2 * DIM + 3])
{
    j = (int)(e & NBR_IDX_MASK);
    if (!SPH_IN_RANGE(d.flags, j, d.n)) return false;
    const float4 oj = d.pos[j];
    float rx, ry, rz;
    const float r2 = pair_vec<DIM>(oi, oj, entry_shift(e, 0, g.Es), entry_shift(e, 1, g.Es),
                                   DIM == 3 ? entry_shift(e, 2, g.Es) : 0.f, rx, ry, rz);
    if (!(r2 < R2)) return false;
    ef[0] = rx * inv2h;
    ef[1] = ry * inv2h;
    if (DIM == 3) ef[2] = rz * inv2h;
    ef[DIM] = sqrtf(r2) * inv2h;
    ef[DIM + 1] = rec_phase(oj.w) != phi ? 1.f : 0.f;
    const float4 nfj = NF[j];
    ef[DIM + 2] = nfi.x - nfj.x;
    ef[DIM + 3] = nfi.y - nfj.y;
    if (DIM == 3) ef[DIM + 4] = nfi.z - nfj.z;
    ef[2 * DIM + 2] = nfi.w - nfj.w;
    return true;
}

// The pair-only part of the edge features: r_ij / 2h (DIM), |r_ij| / 2h,
// phase_i != phase_j.  The state-difference channels of edge_features are
// linear in node quantities, so the forward pass folds them into the node
// terms (k_pq_fold) and the edge phase needs only these.
template <int DIM>
__device__ __forceinline__ bool edge_geom(const Dev &d, const Grid &g, float R2, float inv2h, const float4 &oi,
                                          int phi, unsigned e, int &j, float (&ef)[DIM + 2])
{
    j = (int)(e & NBR_IDX_MASK);
    if (!SPH_IN_RANGE(d.flags, j, d.n)) return false;
    const float4 oj = d.pos[j];
    float rx, ry, rz;
    const float r2 = pair_vec<DIM>(oi, oj, entry_shift(e, 0, g.Es), entry_shift(e, 1, g.Es),
                                   DIM == 3 ? entry_shift(e, 2, g.Es) : 0.f, rx, ry, rz);
    if (!(r2 < R2)) return false;
    ef[0] = rx * inv2h;
    ef[1] = ry * inv2h;
    if (DIM == 3) ef[2] = rz * inv2h;
    ef[DIM] = sqrtf(r2) * inv2h;
    ef[DIM + 1] = rec_phase(oj.w) != phi ? 1.f : 0.f;
    return true;
}

__device__ __forceinline__ void load4(const __half *p, float (&v)[4])
{
    const uint2 raw = *(const uint2 *)p;
    const float2 a = __half22float2(*(const __half2 *)&raw.x), b = __half22float2(*(const __half2 *)&raw.y);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

__device__ __forceinline__ void store4(bf16 *p, const float (&v)[4])
{
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 raw;
    raw.x = *(const unsigned *)&a;
    raw.y = *(const unsigned *)&b;
    *(uint2 *)p = raw;
}


// Width of a staged entry: 2 DIM + 3 edge features and the sender index,
// padded to whole 16-byte vectors.
template <int DIM>
__host__ __device__ constexpr int slot_width() { return ((2 * DIM + 4) + 3) / 4 * 4; }

// Lane-parallel decoding of up to 32 list entries of receiver i (entry
// k0 + lane on each lane): the edge features and the sender of every valid
// entry go to the warp's shared-memory slots; returns the ballot of valid
// entries.
template <int DIM>
__device__ __forceinline__ unsigned stage_entries(const Dev &d, const Grid &g, float R2, float inv2h,
                                                  const float4 &oi, int phi, const float4 &nfi, const float4 *NF,
                                                  int i, int k0, int cnt, float (*slot)[slot_width<DIM>()])
{
    constexpr int NE = 2 * DIM + 3;
    const int lane = threadIdx.x & 31;
    const int k = k0 + lane;
    bool valid = false;
    if (k < cnt) {
        int j;
        float ef[NE];
        valid = edge_features<DIM>(d, g, R2, inv2h, oi, phi, nfi, NF, d.nbr[(size_t)k * d.n + i], j, ef);
        if (valid) {
#pragma unroll
            for (int c = 0; c < NE; ++c) slot[lane][c] = ef[c];
            slot[lane][NE] = __int_as_float(j);
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    __syncwarp();
    return mask;
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// Slots of the forward edge phase: the DIM + 2 pair features and the sender.
template <int DIM>
__host__ __device__ constexpr int geom_slot_width() { return ((DIM + 3) + 3) / 4 * 4; }

// Lane-parallel decoding of up to 32 entries for the forward edge phase: the
// pair features as duplicated FP16 pairs and the sender index after them.
template <int DIM>
__device__ __forceinline__ unsigned stage_geom_h2(const Dev &d, const Grid &g, float R2, float inv2h,
                                                  const float4 &oi, int phi, int i, int k0, int cnt,
                                                  uint32_t (*slot)[geom_slot_width<DIM>()])
{
    constexpr int NG = DIM + 2;
    const int lane = threadIdx.x & 31;
    const int k = k0 + lane;
    bool valid = false;
    if (k < cnt) {
        int j;
        float ef[NG];
        valid = edge_geom<DIM>(d, g, R2, inv2h, oi, phi, d.nbr[(size_t)k * d.n + i], j, ef);
        if (valid) {
#pragma unroll
            for (int c = 0; c < NG; ++c) {
                const __half2 e2 = __float2half2_rn(ef[c]);
                slot[lane][c] = *(const uint32_t *)&e2;
            }
            slot[lane][NG] = (uint32_t)j;
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    __syncwarp();
    return mask;
}

// Folds the state-difference channels of the first edge layer into the node
// terms: with f_i the node's scaled (u, delta) channels and W3d their columns
// of W3, W3d (f_i - f_j) = W3d f_i - W3d f_j, so P'_i = P_i + W3d f_i and
// Q'_j = Q_j - W3d f_j give the same pre-activation P'_i + Q'_j + W3g e_ij.
// One thread per node and four features; FP32 sums, FP16 results.
template <int DIM>
__global__ void __launch_bounds__(256) k_pq_fold(int n, const float4 *NF, const __half *PQ, const float *W3,
                                                 __half *PQf)
{
    constexpr int NE = 2 * DIM + 3;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t >> 5);
    if (i >= n) return;
    const int f0 = (int)(t & 31) * 4;
    const float4 f = NF[i];
    const float fa[3] = {f.x, f.y, f.z};
    float pv[4], qv[4];
    load4(PQ + (size_t)i * 2 * H + f0, pv);
    load4(PQ + (size_t)i * 2 * H + H + f0, qv);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float *w = W3 + (size_t)(f0 + q) * NE;
        float sdiff = w[2 * DIM + 2] * f.w;
#pragma unroll
        for (int a = 0; a < DIM; ++a) sdiff = fmaf(w[DIM + 2 + a], fa[a], sdiff);
        pv[q] += sdiff;
        qv[q] -= sdiff;
    }
    __half2 *pp = (__half2 *)(PQf + (size_t)i * 2 * H + f0), *qq = (__half2 *)(PQf + (size_t)i * 2 * H + H + f0);
    pp[0] = __floats2half2_rn(pv[0], pv[1]);
    pp[1] = __floats2half2_rn(pv[2], pv[3]);
    qq[0] = __floats2half2_rn(qv[0], qv[1]);
    qq[1] = __floats2half2_rn(qv[2], qv[3]);
}

__device__ __forceinline__ __half2 tanh_h2(__half2 x)
{
    uint32_t r;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(r) : "r"(*(const uint32_t *)&x));
    return *(const __half2 *)&r;
}

// Forward edge phase: one warp per receiver i, four features per lane.
// S_i = (1/k_ref) sum_j SiLU(P'_i + Q'_j + W3g e_ij) over list entries with
// |r_ij| < 2h (the folded node terms of k_pq_fold and the pair features);
// degs_i = deg_i / k_ref.  Entries are decoded 32 at a time,
// one per lane; the sender rows Q_j of every valid entry of the batch are
// then copied to shared memory with cp.async (all in flight together).  The
// pre-activation and SiLU run on feature pairs in FP16 (packed FMA, and
// SiLU(z) = h + h tanh(h) with h = z/2); each batch's sum is added to an
// FP32 accumulator.
constexpr int EWF = 128;   // threads of the forward edge kernel (4 warps, one node each)

template <int DIM>
__global__ void __launch_bounds__(EWF, 4) k_edge_fwd(Dev d, Grid g, float R2, float inv2h, const __half *PQ,
                                                   const float *W3, float inv_kref, bf16 *S, float *degs)
{
    constexpr int NE = 2 * DIM + 3;   // columns of W3 (the pair features are its first NG)
    constexpr int NG = DIM + 2;
    constexpr int SWD = geom_slot_width<DIM>();
    __shared__ __align__(16) uint32_t slots[EWF / 32][32][SWD];
    __shared__ __align__(16) uint2 qrows[EWF / 32][32][32];   // [warp][entry][lane]: 4 FP16 features
    const int wid = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= d.n) return;
    const int f0 = lane * 4;
    __half2 w2[NG][2];   // W3 column c for features (f0, f0+1) and (f0+2, f0+3)
#pragma unroll
    for (int c = 0; c < NG; ++c) {
        w2[c][0] = __floats2half2_rn(W3[f0 * NE + c], W3[(f0 + 1) * NE + c]);
        w2[c][1] = __floats2half2_rn(W3[(f0 + 2) * NE + c], W3[(f0 + 3) * NE + c]);
    }
    const uint2 praw = *(const uint2 *)(PQ + (size_t)i * 2 * H + f0);
    const __half2 P0 = *(const __half2 *)&praw.x, P1 = *(const __half2 *)&praw.y;
    const __half2 half2c = __float2half2_rn(0.5f);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int deg = 0;
    const float4 oi = d.pos[i];
    const int phi = rec_phase(oi.w);
    const int cnt = d.ncnt[i];
    uint32_t(*slot)[SWD] = slots[wid];
    uint2(*qr)[32] = qrows[wid];
    for (int k0 = 0; k0 < cnt; k0 += 32) {
        const unsigned valid = stage_geom_h2<DIM>(d, g, R2, inv2h, oi, phi, i, k0, cnt, slot);
        deg += __popc(valid);
        for (unsigned m = valid; m; m &= m - 1) {
            const int sl = __ffs(m) - 1;
            cp_async8(&qr[sl][lane], PQ + (size_t)slot[sl][NG] * 2 * H + H + f0);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        __half2 s0 = __float2half2_rn(0.f), s1 = s0;
        for (unsigned m = valid; m; m &= m - 1) {
            const int sl = __ffs(m) - 1;
            const uint2 raw = qr[sl][lane];
            __half2 z0 = __hadd2(P0, *(const __half2 *)&raw.x);
            __half2 z1 = __hadd2(P1, *(const __half2 *)&raw.y);
            uint32_t e[SWD];
#pragma unroll
            for (int v4 = 0; v4 < SWD / 4; ++v4) {
                const uint4 t4 = *(const uint4 *)&slot[sl][4 * v4];
                e[4 * v4] = t4.x;
                e[4 * v4 + 1] = t4.y;
                e[4 * v4 + 2] = t4.z;
                e[4 * v4 + 3] = t4.w;
            }
#pragma unroll
            for (int c = 0; c < NG; ++c) {
                const __half2 ec = *(const __half2 *)&e[c];
                z0 = __hfma2(w2[c][0], ec, z0);
                z1 = __hfma2(w2[c][1], ec, z1);
            }
            const __half2 h0 = __hmul2(z0, half2c), h1 = __hmul2(z1, half2c);
            s0 = __hadd2(s0, __hfma2(h0, tanh_h2(h0), h0));
            s1 = __hadd2(s1, __hfma2(h1, tanh_h2(h1), h1));
        }
        const float2 a0 = __half22float2(s0), a1 = __half22float2(s1);
        acc[0] += a0.x;
        acc[1] += a0.y;
        acc[2] += a1.x;
        acc[3] += a1.y;
        __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] *= inv_kref;
    store4(S + (size_t)i * H + f0, acc);
    if (lane == 0) degs[i] = deg * inv_kref;
}

// Backward edge phase: one warp per node i.  With dZ_ij = dS_i SiLU'(z_ij) / k_ref:
// dP_i = sum_j dZ_ij, dQ_i = sum_j dZ_ji (the neighbour relation is
// symmetric, so node i gathers its own sender terms), dW3 += dZ_ij e_ij and
// db1 += dP_i, reduced per block and added with atomics.
template <int DIM>
__global__ void __launch_bounds__(EW, 2) k_edge_bwd(Dev d, Grid g, float R2, float inv2h, const float4 *NF,
                                                 const __half *PQ, const float *W3, float inv_kref, const float *dS,
                                                 bf16 *dPQ, float *gW3, float *gb1)
{
    constexpr int NE = 2 * DIM + 3;
    constexpr int SWD = slot_width<DIM>();
    __shared__ __align__(16) float slots[EW / 32][32][SWD];
    __shared__ float red[EW / 32][H * (NE + 1)];
    __shared__ float4 sw[NE][32];
    for (int t = threadIdx.x; t < NE * 32; t += EW) {
        const int c = t / 32, l = t % 32;
        sw[c][l] = make_float4(W3[(4 * l) * NE + c], W3[(4 * l + 1) * NE + c], W3[(4 * l + 2) * NE + c],
                               W3[(4 * l + 3) * NE + c]);
    }
    __syncthreads();
    const int wid = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int f0 = lane * 4;
    float gw[4][NE];
    float dP[4] = {0.f, 0.f, 0.f, 0.f}, dQ[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < NE; ++c) gw[q][c] = 0.f;
    if (i < d.n) {
        float Pi[4], Qi[4], dSi[4];
        load4(PQ + (size_t)i * 2 * H + f0, Pi);
        load4(PQ + (size_t)i * 2 * H + H + f0, Qi);
        const float4 ds4 = *(const float4 *)(dS + (size_t)i * H + f0);
        dSi[0] = ds4.x * inv_kref;
        dSi[1] = ds4.y * inv_kref;
        dSi[2] = ds4.z * inv_kref;
        dSi[3] = ds4.w * inv_kref;
        const float4 oi = d.pos[i];
        const float4 nfi = NF[i];
        const int phi = rec_phase(oi.w);
        const int cnt = d.ncnt[i];
        float(*slot)[SWD] = slots[wid];
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            unsigned mask = stage_entries<DIM>(d, g, R2, inv2h, oi, phi, nfi, NF, i, k0, cnt, slot);
            while (mask) {
                constexpr int GB = 2;
                int sl[GB];
                float Pj[GB][4], Qj[GB][4];
                float4 dSj[GB];
#pragma unroll
                for (int t = 0; t < GB; ++t) {
                    sl[t] = mask ? __ffs(mask) - 1 : -1;
                    if (mask) mask &= mask - 1;
                    if (sl[t] >= 0) {
                        const size_t j = (size_t)__float_as_int(slot[sl[t]][NE]);
                        load4(PQ + j * 2 * H + f0, Pj[t]);
                        load4(PQ + j * 2 * H + H + f0, Qj[t]);
                        dSj[t] = *(const float4 *)(dS + j * H + f0);
                    }
                }
#pragma unroll
                for (int t = 0; t < GB; ++t) {
                    if (sl[t] < 0) break;
                    float ef[NE];
#pragma unroll
                    for (int c = 0; c < NE; ++c) ef[c] = slot[sl[t]][c];
                    const float dsj[4] = {dSj[t].x, dSj[t].y, dSj[t].z, dSj[t].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float zij = Pi[q] + Qj[t][q], zji = Pj[t][q] + Qi[q];
#pragma unroll
                        for (int c = 0; c < NE; ++c) {
                            // e_ji: the relative position and the state differences change
                            // sign, the distance and the phase flag do not
                            const float ec = ef[c];
                            const float4 wc4 = sw[c][lane];
                            const float wq = q == 0 ? wc4.x : q == 1 ? wc4.y : q == 2 ? wc4.z : wc4.w;
                            zij = fmaf(wq, ec, zij);
                            zji = fmaf(wq, (c < DIM || c >= DIM + 2) ? -ec : ec, zji);
                        }
                        const float dzij = dSi[q] * dsilu(zij);
                        const float dzji = dsj[q] * inv_kref * dsilu(zji);
                        dP[q] += dzij;
                        dQ[q] += dzji;
#pragma unroll
                        for (int c = 0; c < NE; ++c) gw[q][c] = fmaf(dzij, ef[c], gw[q][c]);
                    }
                }
            }
            __syncwarp();
        }
        store4(dPQ + (size_t)i * 2 * H + f0, dP);
        store4(dPQ + (size_t)i * 2 * H + H + f0, dQ);
    }
    // block reduction of dW3 and db1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int c = 0; c < NE; ++c) red[wid][(f0 + q) * NE + c] = gw[q][c];
        red[wid][H * NE + f0 + q] = dP[q];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < H * (NE + 1); t += EW) {
        float s = 0.f;
        for (int w2 = 0; w2 < EW / 32; ++w2) s += red[w2][t];
        if (s != 0.f) {
            if (t < H * NE) atomicAdd(gW3 + t, s);
            else atomicAdd(gb1 + (t - H * NE), s);
        }
    }
}

// Column sums over n rows of src (ld), optionally weighted per row, added to dst.
__global__ void k_colsum(const float *src, int ld, int cols, int n, const float *roww, float *dst)
{
    const int c = threadIdx.x;
    const int rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
    if (c >= cols) return;
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += (roww ? roww[r] : 1.f) * src[(size_t)r * ld + c];
    if (s != 0.f) atomicAdd(dst + c, s);
}

// dst[c][r] = src[r][c] for r < rows (rows padded up to a multiple of 32), c < cols.
__global__ void k_transpose(const bf16 *src, int ld_src, int rows, int cols, bf16 *dst, int ld_dst)
{
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * ld_src + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[(size_t)c * ld_dst + r] = tile[threadIdx.x][k];
    }
}

__global__ void k_add(const float *a, int lda, const float *b, int ldb, float *out, int ldo, int rows, int cols)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows * cols) return;
    const int r = k / cols, c = k % cols;
    out[(size_t)r * ldo + c] = a[(size_t)r * lda + c] + b[(size_t)r * ldb + c];
}

// Targets from the state after k plain steps (original order, instance
// frame) against the current state (sorted), masked squared error, dL/dy.
template <int DIM>
__global__ void k_loss(Dev d, const float *norm, float T, const float *Y, const double *x1, const double *u1,
                       const double *rho1, float inv_count, float *dYf, bf16 *dYb, double *loss)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (k < d.n) {
        constexpr int NIN = 2 * DIM + 4, NOUT = 2 * DIM + 1;
        const float *mu_out = norm + 2 * NIN, *sd_out = norm + 2 * NIN + NOUT;
        const int p = d.pid[k];
        const uint8_t tg = d.tag[k];
        const Inst &I = d.inst[d.iid[k]];
        const bool wall = tg & 2;
        const float4 a = d.acc[k];
        const float av[3] = {a.x, a.y, a.z};
        float delta[NOUT];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double u0c = d.u[(size_t)c * d.n + k], u1c = u1[(size_t)p * DIM + c];
            const double dxc = x1[(size_t)p * DIM + c] - (d.x[(size_t)c * d.n + k] - I.offset[c]);
            delta[c] = (float)(dxc - (double)T * 0.5 * (u0c + u1c));
            delta[DIM + c] = (float)(u1c - u0c - (double)T * av[c]);
        }
        const double rho0 = (double)by_phase(tg & 1, I.rho0);
        delta[2 * DIM] = (float)((rho1[p] - (rho0 + (double)d.drho[k])) / rho0 - (double)T * a.w / rho0);
        float dy[FOUT];
#pragma unroll
        for (int c = 0; c < FOUT; ++c) dy[c] = 0.f;
#pragma unroll
        for (int c = 0; c < NOUT; ++c) {
            if (wall && c < 2 * DIM) continue;
            const float t = (delta[c] - mu_out[c]) / sd_out[c];
            const float e = Y[(size_t)k * FOUT + c] - t;
            l += (double)e * e;
            dy[c] = 2.f * e * inv_count;
        }
#pragma unroll
        for (int c = 0; c < FOUT; ++c) {
            dYf[(size_t)k * FOUT + c] = dy[c];
            dYb[(size_t)k * FOUT + c] = __float2bfloat16_rn(dy[c]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// Applies the de-normalised increments: x += dx, u += du on fluid particles,
// rho += drho on all.
template <int DIM>
__global__ void k_apply(Dev d, const float *norm, float T, const float *Y)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    constexpr int NIN = 2 * DIM + 4, NOUT = 2 * DIM + 1;
    const float *mu_out = norm + 2 * NIN, *sd_out = norm + 2 * NIN + NOUT;
    const uint8_t tg = d.tag[k];
    const Inst &I = d.inst[d.iid[k]];
    const float4 a = d.acc[k];
    const float av[3] = {a.x, a.y, a.z};
    float D[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) D[c] = Y[(size_t)k * FOUT + c] * sd_out[c] + mu_out[c];
    bool finite = true;
    if (!(tg & 2)) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double u0 = d.u[(size_t)c * d.n + k], du = (double)T * av[c] + (double)D[DIM + c];
            const double x = d.x[(size_t)c * d.n + k] + ((double)T * (u0 + 0.5 * du) + (double)D[c]);
            const double u = u0 + du;
            d.x[(size_t)c * d.n + k] = x;
            d.u[(size_t)c * d.n + k] = u;
            finite = finite && isfinite(x) && isfinite(u);
        }
    }
    const float dr = d.drho[k] + (T * a.w + D[2 * DIM] * by_phase(tg & 1, I.rho0));
    d.drho[k] = dr;
    if (!finite || !isfinite(dr)) atomicOr(d.flags, FLAG_NONFINITE);
}

// De-normalised increments in original order: out[p * NOUT + c].
template <int DIM>
__global__ void k_predict_out(Dev d, const float *norm, float T, const float *Y, double *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.n) return;
    constexpr int NIN = 2 * DIM + 4, NOUT = 2 * DIM + 1;
    const float *mu_out = norm + 2 * NIN, *sd_out = norm + 2 * NIN + NOUT;
    const int p = d.pid[k];
    const uint8_t tg = d.tag[k];
    const Inst &I = d.inst[d.iid[k]];
    const float4 a = d.acc[k];
    const float av[3] = {a.x, a.y, a.z};
    float D[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) D[c] = Y[(size_t)k * FOUT + c] * sd_out[c] + mu_out[c];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const double u0 = d.u[(size_t)c * d.n + k], du = (double)T * av[c] + (double)D[DIM + c];
        out[(size_t)p * NOUT + c] = (tg & 2) ? 0.0 : (double)T * (u0 + 0.5 * du) + (double)D[c];
        out[(size_t)p * NOUT + DIM + c] = (tg & 2) ? 0.0 : du;
    }
    out[(size_t)p * NOUT + 2 * DIM] = (double)(T * a.w + D[2 * DIM] * by_phase(tg & 1, I.rho0));
}

// Adam (Kingma & Ba 2015) with bias correction folded into the step size.
__global__ void k_adam(float *theta, const float *g, float *m, float *v, int count, float lr_t, float b1, float b2,
                       float eps_t)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr_t * mk / (sqrtf(vk) + eps_t);
}

// ---------------------------------------------------------------------------
// Host side

inline int nb(int work, int t = 256) { return (work + t - 1) / t; }

struct Epi {
    float *Cf = nullptr;
    int ldcf = 0;
    bf16 *Cb = nullptr;
    int ldcb = 0;
    const float *bias = nullptr;
    const float *row_scale = nullptr, *row_bias = nullptr;
    float *Z = nullptr;
    int ldz = 0;
    const float *residual = nullptr;
    int ldr = 0;
    int act = 0;
    const float *dact = nullptr;
    int lddact = 0;
    int atomic = 0;
    int k_split = 0;
    int n_store = 0;
    int cb_half = 0;
};

int mm(Surrogate &S, cudaStream_t st, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K,
       const Epi &e)
{
    umma::GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_split = e.k_split > 0 ? e.k_split : ((K + umma::BK - 1) / umma::BK) * umma::BK;
    g.Cf = e.Cf;
    g.ldcf = e.ldcf;
    g.Cb = e.Cb;
    g.ldcb = e.ldcb;
    g.bias = e.bias;
    g.row_scale = e.row_scale;
    g.row_bias = e.row_bias;
    g.Z = e.Z;
    g.ldz = e.ldz;
    g.residual = e.residual;
    g.ldr = e.ldr;
    g.act = e.act;
    g.dact = e.dact;
    g.lddact = e.lddact;
    g.atomic = e.atomic;
    g.n_store = e.n_store;
    g.cb_half = e.cb_half;
    g.err = S.err;
    cudaError_t err = umma::gemm(g, st);
    if (err != cudaSuccess) return set_error(SPH_ECUDA, std::string("gemm: ") + cudaGetErrorString(err));
    return SPH_OK;
}

// dW (rows x cols, ld cols, in the flat gradient) += dY^T X, with dY^T (rows x npad) and X^T (cols x npad).
int mm_wgrad(Surrogate &S, cudaStream_t st, const bf16 *dYT, int rows, const bf16 *XT, int cols, float *dW,
             int n_store = 0)
{
    Epi e;
    e.Cf = dW;
    e.ldcf = n_store > 0 ? n_store : cols;
    e.atomic = 1;
    e.n_store = n_store;
    e.k_split = 4096;
    return mm(S, st, dYT, S.npad, XT, S.npad, rows, cols, S.npad, e);
}

int transpose(Surrogate &S, cudaStream_t st, const bf16 *src, int ld, int cols, bf16 *dst)
{
    dim3 grid(S.npad / 32, (cols + 31) / 32);
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(src, ld, S.npad, cols, dst, S.npad);
    CUR(cudaGetLastError());
    return SPH_OK;
}

int pack_weights(Surrogate &S, cudaStream_t st)
{
    const Layout &L = S.L;
    const float *T = S.theta;
    auto pk = [&](int off, int rows, int cols, bf16 *dst, int ld, int row_off, int tr) {
        k_pack<<<nb(rows * cols), 256, 0, st>>>(T + off, rows, cols, dst, ld, row_off, tr);
    };
    pk(L.enc1w, H, L.nin, S.Wenc1, FIN, 0, 0);
    pk(L.enc2w, H, H, S.Wenc2, H, 0, 0);
    pk(L.enc2w, H, H, S.Wenc2T, H, 0, 1);
    for (int r = 0; r < 2; ++r) {
        pk(L.w1[r], H, H, S.Wpq[r], H, 0, 0);
        pk(L.w2[r], H, H, S.Wpq[r], H, H, 0);
        pk(L.w1[r], H, H, S.WpqT[r], 2 * H, 0, 1);
        pk(L.w2[r], H, H, S.WpqT[r], 2 * H, H, 1);
        pk(L.we2[r], H, H, S.We2[r], H, 0, 0);
        pk(L.we2[r], H, H, S.We2T[r], H, 0, 1);
        pk(L.n1[r], H, 2 * H, S.Wn1[r], 2 * H, 0, 0);
        pk(L.n1[r], H, 2 * H, S.Wn1T[r], H, 0, 1);
        pk(L.n2[r], H, H, S.Wn2[r], H, 0, 0);
        pk(L.n2[r], H, H, S.Wn2T[r], H, 0, 1);
        k_copy_f<<<1, H, 0, st>>>(T + L.b1[r], S.bpq[r], H);
    }
    pk(L.dec1w, H, H, S.Wd1, H, 0, 0);
    pk(L.dec1w, H, H, S.Wd1T, H, 0, 1);
    pk(L.dec2w, L.nout, H, S.Wd2, H, 0, 0);
    pk(L.dec2w, L.nout, H, S.Wd2T, FOUT, 0, 1);
    k_copy_f<<<1, 32, 0, st>>>(T + L.dec2b, S.bd2, L.nout);
    CUR(cudaGetLastError());
    return SPH_OK;
}

int alloc_surrogate(Surrogate &S)
{
    const size_t P = (size_t)S.npad;
    const size_t nt = (size_t)S.L.total;
    int e = 0;
    e |= dalloc(S, &S.theta, nt);
    e |= dalloc(S, &S.grad, nt);
    e |= dalloc(S, &S.m, nt);
    e |= dalloc(S, &S.v, nt);
    e |= dalloc(S, &S.norm_d, 64);
    e |= dalloc(S, &S.Wenc1, H * FIN);
    e |= dalloc(S, &S.Wenc2, H * H);
    e |= dalloc(S, &S.Wenc2T, H * H);
    for (int r = 0; r < 2; ++r) {
        e |= dalloc(S, &S.Wpq[r], 2 * H * H);
        e |= dalloc(S, &S.WpqT[r], 2 * H * H);
        e |= dalloc(S, &S.We2[r], H * H);
        e |= dalloc(S, &S.We2T[r], H * H);
        e |= dalloc(S, &S.Wn1[r], 2 * H * H);
        e |= dalloc(S, &S.Wn1T[r], 2 * H * H);
        e |= dalloc(S, &S.Wn2[r], H * H);
        e |= dalloc(S, &S.Wn2T[r], H * H);
        e |= dalloc(S, &S.bpq[r], 2 * H);
        e |= dalloc(S, &S.A1[r], P * 2 * H);
        e |= dalloc(S, &S.PQ[r], P * 2 * H);
        if (r == 0) e |= dalloc(S, &S.PQf, P * 2 * H);
        e |= dalloc(S, &S.S[r], P * H);
        e |= dalloc(S, &S.G1[r], P * H);
        e |= dalloc(S, &S.Z1[r], P * H);
    }
    e |= dalloc(S, &S.Wd1, H * H);
    e |= dalloc(S, &S.Wd1T, H * H);
    e |= dalloc(S, &S.Wd2, FOUT * H);
    e |= dalloc(S, &S.Wd2T, H * FOUT);
    e |= dalloc(S, &S.bd2, FOUT);
    e |= dalloc(S, &S.X16, P * FIN);
    e |= dalloc(S, &S.A0, P * H);
    e |= dalloc(S, &S.Z0, P * H);
    for (int k = 0; k < 3; ++k) e |= dalloc(S, &S.h[k], P * H);
    e |= dalloc(S, &S.degs, P);
    e |= dalloc(S, &S.hLb, P * H);
    e |= dalloc(S, &S.Z2, P * H);
    e |= dalloc(S, &S.A2, P * H);
    e |= dalloc(S, &S.Y, P * FOUT);
    e |= dalloc(S, &S.NF, P);
    e |= dalloc(S, &S.loss_d, 1);
    e |= dalloc(S, &S.err, 1);
    if (e) return SPH_ENOMEM;
    CUR(cudaDeviceSynchronize());   // the zero fills precede any use on the simulation's stream
    return SPH_OK;
}

int alloc_backward(Surrogate &S)
{
    if (S.dA) return SPH_OK;
    const size_t P = (size_t)S.npad;
    int e = 0;
    e |= dalloc(S, &S.dYf, P * FOUT);
    e |= dalloc(S, &S.dYb, P * FOUT);
    e |= dalloc(S, &S.dZf, P * H);
    e |= dalloc(S, &S.dZb, P * H);
    e |= dalloc(S, &S.dA, P * 2 * H);
    e |= dalloc(S, &S.dAb, P * 2 * H);
    e |= dalloc(S, &S.dh, P * H);
    e |= dalloc(S, &S.dh2, P * H);
    e |= dalloc(S, &S.dhb, P * H);
    e |= dalloc(S, &S.dS, P * H);
    e |= dalloc(S, &S.dPQ, P * 2 * H);
    e |= dalloc(S, &S.T1, P * 2 * H);
    e |= dalloc(S, &S.T2, P * 2 * H);
    if (e) return SPH_ENOMEM;
    CUR(cudaDeviceSynchronize());
    return SPH_OK;
}

// Forward pass at the simulation's current state (rates evaluated by the
// caller); the pre-activations the backward pass needs are stored only when
// training.
int forward(Surrogate &S, const SimView &v, bool training)
{
    const Layout &L = S.L;
    const float *T = S.theta;
    cudaStream_t st = v.stream;
    const int n = v.n;
    int rc = 0;
    const float isu = 1.f / S.sd_edge_u, isr = 1.f / S.sd_edge_rho;
    if (v.dim == 2) k_features<2><<<nb(n), 256, 0, st>>>(v.d, S.norm_d, S.t_jump, isu, isr, S.X16, S.NF);
    else k_features<3><<<nb(n), 256, 0, st>>>(v.d, S.norm_d, S.t_jump, isu, isr, S.X16, S.NF);
    CUR(cudaGetLastError());
    {
        Epi e;
        e.bias = T + L.enc1b;
        e.act = 1;
        e.Z = training ? S.Z0 : nullptr;
        e.ldz = H;
        e.Cb = S.A0;
        e.ldcb = H;
        if ((rc = mm(S, st, S.X16, FIN, S.Wenc1, FIN, n, H, FIN, e))) return rc;
    }
    {
        Epi e;
        e.bias = T + L.enc2b;
        e.Cf = S.h[0];
        e.ldcf = H;
        e.Cb = S.A1[0];
        e.ldcb = 2 * H;
        if ((rc = mm(S, st, S.A0, H, S.Wenc2, H, n, H, H, e))) return rc;
    }
    const float R2 = (float)(4.0 * v.h * v.h), inv2h = (float)(0.5 / v.h), invk = 1.f / S.k_ref;
    for (int r = 0; r < 2; ++r) {
        {
            Epi e;
            e.bias = S.bpq[r];
            e.Cb = (bf16 *)S.PQ[r];
            e.cb_half = 1;
            e.ldcb = 2 * H;
            if ((rc = mm(S, st, S.A1[r], 2 * H, S.Wpq[r], H, n, 2 * H, H, e))) return rc;
        }
        if (v.dim == 2) {
            k_pq_fold<2><<<nb(n * 32, 256), 256, 0, st>>>(n, S.NF, S.PQ[r], T + L.w3[r], S.PQf);
            k_edge_fwd<2><<<nb(n * 32, EWF), EWF, 0, st>>>(v.d, v.g, R2, inv2h, S.PQf, T + L.w3[r], invk, S.S[r],
                                                           S.degs);
        } else {
            k_pq_fold<3><<<nb(n * 32, 256), 256, 0, st>>>(n, S.NF, S.PQ[r], T + L.w3[r], S.PQf);
            k_edge_fwd<3><<<nb(n * 32, EWF), EWF, 0, st>>>(v.d, v.g, R2, inv2h, S.PQf, T + L.w3[r], invk, S.S[r],
                                                           S.degs);
        }
        CUR(cudaGetLastError());
        {
            Epi e;
            e.row_scale = S.degs;
            e.row_bias = T + L.be2[r];
            e.Cb = S.A1[r] + H;
            e.ldcb = 2 * H;
            if ((rc = mm(S, st, S.S[r], H, S.We2[r], H, n, H, H, e))) return rc;
        }
        {
            Epi e;
            e.bias = T + L.n1b[r];
            e.act = 1;
            e.Z = training ? S.Z1[r] : nullptr;
            e.ldz = H;
            e.Cb = S.G1[r];
            e.ldcb = H;
            if ((rc = mm(S, st, S.A1[r], 2 * H, S.Wn1[r], 2 * H, n, H, 2 * H, e))) return rc;
        }
        {
            Epi e;
            e.bias = T + L.n2b[r];
            e.residual = S.h[r];
            e.ldr = H;
            e.Cf = S.h[r + 1];
            e.ldcf = H;
            e.Cb = r == 0 ? S.A1[1] : S.hLb;
            e.ldcb = r == 0 ? 2 * H : H;
            if ((rc = mm(S, st, S.G1[r], H, S.Wn2[r], H, n, H, H, e))) return rc;
        }
    }
    {
        Epi e;
        e.bias = T + L.dec1b;
        e.act = 1;
        e.Z = training ? S.Z2 : nullptr;
        e.ldz = H;
        e.Cb = S.A2;
        e.ldcb = H;
        if ((rc = mm(S, st, S.hLb, H, S.Wd1, H, n, H, H, e))) return rc;
    }
    {
        Epi e;
        e.bias = S.bd2;
        e.Cf = S.Y;
        e.ldcf = FOUT;
        if ((rc = mm(S, st, S.A2, H, S.Wd2, H, n, FOUT, H, e))) return rc;
    }
    return SPH_OK;
}

// Backward pass from dY (S.dYf / S.dYb) into S.grad (zeroed here).
int backward(Surrogate &S, const SimView &v)
{
    const Layout &L = S.L;
    const float *T = S.theta;
    float *G = S.grad;
    cudaStream_t st = v.stream;
    const int n = v.n;
    const int cs_blocks = std::max(1, std::min(1024, nb(n, 512)));
    int rc = 0;
    CUR(cudaMemsetAsync(G, 0, sizeof(float) * L.total, st));
    // decoder, layer 2
    if ((rc = transpose(S, st, S.dYb, FOUT, FOUT, S.T1))) return rc;
    if ((rc = transpose(S, st, S.A2, H, H, S.T2))) return rc;
    if ((rc = mm_wgrad(S, st, S.T1, L.nout, S.T2, H, G + L.dec2w))) return rc;
    k_colsum<<<cs_blocks, 256, 0, st>>>(S.dYf, FOUT, L.nout, n, nullptr, G + L.dec2b);
    {
        Epi e;
        e.act = 2;
        e.dact = S.Z2;
        e.lddact = H;
        e.Cf = S.dZf;
        e.ldcf = H;
        e.Cb = S.dZb;
        e.ldcb = H;
        if ((rc = mm(S, st, S.dYb, FOUT, S.Wd2T, FOUT, n, H, FOUT, e))) return rc;
    }
    // decoder, layer 1
    if ((rc = transpose(S, st, S.dZb, H, H, S.T1))) return rc;
    if ((rc = transpose(S, st, S.hLb, H, H, S.T2))) return rc;
    if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, H, G + L.dec1w))) return rc;
    k_colsum<<<cs_blocks, 256, 0, st>>>(S.dZf, H, H, n, nullptr, G + L.dec1b);
    {
        Epi e;
        e.Cf = S.dh;
        e.ldcf = H;
        e.Cb = S.dhb;
        e.ldcb = H;
        if ((rc = mm(S, st, S.dZb, H, S.Wd1T, H, n, H, H, e))) return rc;
    }
    const float R2 = (float)(4.0 * v.h * v.h), inv2h = (float)(0.5 / v.h), invk = 1.f / S.k_ref;
    for (int r = 1; r >= 0; --r) {
        const bf16 *hb = r == 0 ? S.A1[0] : S.A1[1];   // h_r in BF16: left half of [h, M]
        // node MLP, layer 2 (residual: dh passes through)
        if ((rc = transpose(S, st, S.dhb, H, H, S.T1))) return rc;
        if ((rc = transpose(S, st, S.G1[r], H, H, S.T2))) return rc;
        if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, H, G + L.n2[r]))) return rc;
        k_colsum<<<cs_blocks, 256, 0, st>>>(S.dh, H, H, n, nullptr, G + L.n2b[r]);
        {
            Epi e;
            e.act = 2;
            e.dact = S.Z1[r];
            e.lddact = H;
            e.Cf = S.dZf;
            e.ldcf = H;
            e.Cb = S.dZb;
            e.ldcb = H;
            if ((rc = mm(S, st, S.dhb, H, S.Wn2T[r], H, n, H, H, e))) return rc;
        }
        // node MLP, layer 1 on [h, M]
        if ((rc = transpose(S, st, S.dZb, H, H, S.T1))) return rc;
        if ((rc = transpose(S, st, S.A1[r], 2 * H, 2 * H, S.T2))) return rc;
        if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, 2 * H, G + L.n1[r]))) return rc;
        k_colsum<<<cs_blocks, 256, 0, st>>>(S.dZf, H, H, n, nullptr, G + L.n1b[r]);
        {
            Epi e;
            e.Cf = S.dA;
            e.ldcf = 2 * H;
            e.Cb = S.dAb;
            e.ldcb = 2 * H;
            if ((rc = mm(S, st, S.dZb, H, S.Wn1T[r], H, n, 2 * H, H, e))) return rc;
        }
        // second edge layer, applied after the sum: M = S We2^T + degs be2
        if ((rc = transpose(S, st, S.dAb + H, 2 * H, H, S.T1))) return rc;
        if ((rc = transpose(S, st, S.S[r], H, H, S.T2))) return rc;
        if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, H, G + L.we2[r]))) return rc;
        k_colsum<<<cs_blocks, 256, 0, st>>>(S.dA + H, 2 * H, H, n, S.degs, G + L.be2[r]);
        {
            Epi e;
            e.Cf = S.dS;
            e.ldcf = H;
            if ((rc = mm(S, st, S.dAb + H, 2 * H, S.We2T[r], H, n, H, H, e))) return rc;
        }
        // edge phase
        if (v.dim == 2)
            k_edge_bwd<2><<<nb(n * 32, EW), EW, 0, st>>>(v.d, v.g, R2, inv2h, S.NF, S.PQ[r], T + L.w3[r], invk,
                                                         S.dS, S.dPQ, G + L.w3[r], G + L.b1[r]);
        else
            k_edge_bwd<3><<<nb(n * 32, EW), EW, 0, st>>>(v.d, v.g, R2, inv2h, S.NF, S.PQ[r], T + L.w3[r], invk,
                                                         S.dS, S.dPQ, G + L.w3[r], G + L.b1[r]);
        CUR(cudaGetLastError());
        // first edge layer, node parts: P = h W1^T + b1, Q = h W2^T
        if ((rc = transpose(S, st, S.dPQ, 2 * H, 2 * H, S.T1))) return rc;
        if ((rc = transpose(S, st, hb, 2 * H, H, S.T2))) return rc;
        if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, H, G + L.w1[r]))) return rc;
        if ((rc = mm_wgrad(S, st, S.T1 + (size_t)H * S.npad, H, S.T2, H, G + L.w2[r]))) return rc;
        // dh_r = dh_{r+1} + d[h part of n1 input] + dP W1 + dQ W2
        k_add<<<nb(n * H), 256, 0, st>>>(S.dh, H, S.dA, 2 * H, S.dh2, H, n, H);
        {
            Epi e;
            e.residual = S.dh2;
            e.ldr = H;
            e.Cf = S.dh;
            e.ldcf = H;
            e.Cb = S.dhb;
            e.ldcb = H;
            if ((rc = mm(S, st, S.dPQ, 2 * H, S.WpqT[r], 2 * H, n, H, 2 * H, e))) return rc;
        }
    }
    // encoder, layer 2
    if ((rc = transpose(S, st, S.dhb, H, H, S.T1))) return rc;
    if ((rc = transpose(S, st, S.A0, H, H, S.T2))) return rc;
    if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, H, G + L.enc2w))) return rc;
    k_colsum<<<cs_blocks, 256, 0, st>>>(S.dh, H, H, n, nullptr, G + L.enc2b);
    {
        Epi e;
        e.act = 2;
        e.dact = S.Z0;
        e.lddact = H;
        e.Cf = S.dZf;
        e.ldcf = H;
        e.Cb = S.dZb;
        e.ldcb = H;
        if ((rc = mm(S, st, S.dhb, H, S.Wenc2T, H, n, H, H, e))) return rc;
    }
    // encoder, layer 1
    if ((rc = transpose(S, st, S.dZb, H, H, S.T1))) return rc;
    if ((rc = transpose(S, st, S.X16, FIN, FIN, S.T2))) return rc;
    if ((rc = mm_wgrad(S, st, S.T1, H, S.T2, FIN, G + L.enc1w, L.nin))) return rc;
    k_colsum<<<cs_blocks, 256, 0, st>>>(S.dZf, H, H, n, nullptr, G + L.enc1b);
    CUR(cudaGetLastError());
    return SPH_OK;
}

Surrogate *get(sph_handle h)
{
    return h ? static_cast<Surrogate *>(sim_ext(h)) : nullptr;
}

int check_err(Surrogate &S, cudaStream_t st)
{
    unsigned e = 0;
    CUR(cudaMemcpyAsync(&e, S.err, sizeof(e), cudaMemcpyDeviceToHost, st));
    CUR(cudaStreamSynchronize(st));
    if (e) {
        CUR(cudaMemsetAsync(S.err, 0, sizeof(unsigned), st));
        return set_error(SPH_ETIMEOUT, "a tensor-core wait of the surrogate exceeded one second");
    }
    return SPH_OK;
}

}  // namespace

extern "C" {

int sph_mm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K, int k_split,
                int accumulate, void *stream, unsigned *err_dev)
{
    if (!A || !B || !C || !err_dev) return set_error(SPH_EINVAL, "NULL argument");
    if (M < 0 || K < 0 || (N != 16 && N != 32 && N != 64 && N != 128 && N != 256))
        return set_error(SPH_EINVAL, "N must be 16, 32, 64, 128 or 256 and M, K >= 0");
    if (K % 16 != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || ldc < N)
        return set_error(SPH_EINVAL, "K must be a multiple of 16, lda and ldb multiples of 8 and >= K");
    if (k_split <= 0) k_split = ((K + umma::BK - 1) / umma::BK) * umma::BK;
    if (k_split % umma::BK != 0) return set_error(SPH_EINVAL, "k_split must be a multiple of 64");
    if (K > k_split && !accumulate) return set_error(SPH_EINVAL, "a split K needs accumulate");
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16) return set_error(SPH_EINVAL, "A and B must be 16-byte aligned");
    umma::GemmArgs g{};
    g.A = (const bf16 *)A;
    g.lda = lda;
    g.B = (const bf16 *)B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_split = k_split;
    g.Cf = C;
    g.ldcf = ldc;
    g.atomic = accumulate ? 1 : 0;
    g.err = err_dev;
    cudaError_t e = umma::gemm(g, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(SPH_ECUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}

int sph_surrogate_init(sph_handle h, const double *weights, int64_t nweights, const double *norm, int64_t nnorm)
{
    if (!h || !weights || !norm) return set_error(SPH_EINVAL, "NULL argument");
    const SimView v = sim_view(h);
    if (v.ninst != 1) return set_error(SPH_EINVAL, "the surrogate runs on single-instance handles");
    if (v.npiston > 0) return set_error(SPH_EINVAL, "the surrogate does not move piston particles");
    const Layout L = make_layout(v.dim);
    if (nweights != L.total) return set_error(SPH_EINVAL, "weights: wrong number of parameters for this dim");
    if (nnorm != 2 * L.nin + 2 * L.nout + 4) return set_error(SPH_EINVAL, "norm: wrong length for this dim");
    for (int64_t k = 0; k < nnorm; ++k)
        if (!std::isfinite(norm[k])) return set_error(SPH_EINVAL, "norm must be finite");
    for (int c = 0; c < L.nin; ++c)
        if (!(norm[L.nin + c] > 0)) return set_error(SPH_EINVAL, "sd_in must be positive");
    for (int c = 0; c < L.nout; ++c)
        if (!(norm[2 * L.nin + L.nout + c] > 0)) return set_error(SPH_EINVAL, "sd_out must be positive");
    const int o = 2 * L.nin + 2 * L.nout;
    if (!(norm[o] > 0) || !(norm[o + 1] >= 0) || !(norm[o + 2] > 0) || !(norm[o + 3] > 0))
        return set_error(SPH_EINVAL, "k_ref, sd_edge_u and sd_edge_rho must be positive and T >= 0");
    for (int64_t k = 0; k < nweights; ++k)
        if (!std::isfinite(weights[k])) return set_error(SPH_EINVAL, "weights must be finite");
    Surrogate *S = get(h);
    if (!S || S->dim != v.dim || S->n != v.n) {
        S = new Surrogate();
        S->dim = v.dim;
        S->n = v.n;
        S->npad = std::max(128, ((v.n + 127) / 128) * 128);
        S->L = L;
        int rc = alloc_surrogate(*S);
        if (rc) {
            delete S;
            return rc;
        }
        sim_set_ext(h, S, free_surrogate);
    }
    S->k_ref = (float)norm[o];
    S->t_jump = (float)norm[o + 1];
    S->t_jump64 = norm[o + 1];
    S->sd_edge_u = (float)norm[o + 2];
    S->sd_edge_rho = (float)norm[o + 3];
    S->norm.assign(norm, norm + o);
    std::vector<float> tf(weights, weights + nweights);
    CUR(cudaMemcpyAsync(S->theta, tf.data(), sizeof(float) * nweights, cudaMemcpyHostToDevice, v.stream));
    CUR(cudaMemcpyAsync(S->norm_d, S->norm.data(), sizeof(float) * S->norm.size(), cudaMemcpyHostToDevice, v.stream));
    CUR(cudaMemsetAsync(S->m, 0, sizeof(float) * nweights, v.stream));
    CUR(cudaMemsetAsync(S->v, 0, sizeof(float) * nweights, v.stream));
    S->adam_t = 0;
    int rc = pack_weights(*S, v.stream);
    if (rc) return rc;
    CUR(cudaStreamSynchronize(v.stream));
    return SPH_OK;
}

int sph_surrogate_get_weights(sph_handle h, double *weights, int64_t nweights)
{
    Surrogate *S = get(h);
    if (!S || !weights) return set_error(SPH_EINVAL, "no surrogate on this handle, or NULL argument");
    if (nweights != S->L.total) return set_error(SPH_EINVAL, "weights: wrong length");
    const SimView v = sim_view(h);
    std::vector<float> tf(nweights);
    CUR(cudaMemcpyAsync(tf.data(), S->theta, sizeof(float) * nweights, cudaMemcpyDeviceToHost, v.stream));
    CUR(cudaStreamSynchronize(v.stream));
    for (int64_t k = 0; k < nweights; ++k) weights[k] = tf[k];
    return SPH_OK;
}

int sph_surrogate_predict(sph_handle h, double *out, int64_t bytes)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    const SimView v0 = sim_view(h);
    const size_t need = (size_t)v0.n * S->L.nout * sizeof(double);
    if (!out || bytes < (int64_t)need) return set_error(SPH_EINVAL, "output buffer too small");
    if (v0.n == 0) return SPH_OK;
    int rc0 = sph_eval_rates(h);
    if (rc0) return rc0;
    const SimView v = sim_view(h);
    int rc = forward(*S, v, false);
    if (rc) return rc;
    double *dout = nullptr;
    CUR(cudaMallocAsync((void **)&dout, need, v.stream));
    if (v.dim == 2) k_predict_out<2><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y, dout);
    else k_predict_out<3><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y, dout);
    CUR(cudaGetLastError());
    CUR(cudaMemcpyAsync(out, dout, need, cudaMemcpyDeviceToHost, v.stream));
    CUR(cudaFreeAsync(dout, v.stream));
    if ((rc = check_err(*S, v.stream))) return rc;
    return sim_check(h);
}

int sph_surrogate_advance(sph_handle h, int k_steps)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (k_steps < 1) return set_error(SPH_EINVAL, "k_steps must be >= 1");
    const SimView v0 = sim_view(h);
    if (v0.n == 0) return sim_moved(h, k_steps, S->t_jump64);
    int rc0 = sph_eval_rates(h);
    if (rc0) return rc0;
    const SimView v = sim_view(h);
    int rc = forward(*S, v, false);
    if (rc) return rc;
    if (v.dim == 2) k_apply<2><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y);
    else k_apply<3><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y);
    CUR(cudaGetLastError());
    return sim_moved(h, k_steps, S->t_jump64);
}

int sph_surrogate_train_step(sph_handle h, const double *x1, const double *u1, const double *rho1, double lr,
                             int update, double *loss_out, double *grad_out, int64_t ngrad)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (!x1 || !u1 || !rho1) return set_error(SPH_EINVAL, "target arrays are NULL");
    if (update && !(lr > 0)) return set_error(SPH_EINVAL, "lr must be positive");
    if (grad_out && ngrad != S->L.total) return set_error(SPH_EINVAL, "grad_out: wrong length");
    const SimView v0 = sim_view(h);
    if (v0.n == 0) return set_error(SPH_EINVAL, "no particles");
    int rc = alloc_backward(*S);
    if (rc) return rc;
    int rc0 = sph_eval_rates(h);
    if (rc0) return rc0;
    const SimView v = sim_view(h);
    if ((rc = forward(*S, v, true))) return rc;
    // count of (node, channel) terms: every channel of fluid nodes, the density channel of walls
    // (computed on the device side by the loss kernel's mask; the host needs the wall count)
    std::vector<uint8_t> tags(v.n);
    CUR(cudaMemcpyAsync(tags.data(), v.d.tag, v.n, cudaMemcpyDeviceToHost, v.stream));
    CUR(cudaStreamSynchronize(v.stream));
    int64_t walls = 0;
    for (uint8_t t : tags) walls += (t >> 1) & 1;
    const double count = (double)(v.n - walls) * S->L.nout + (double)walls;
    CUR(cudaMemsetAsync(S->loss_d, 0, sizeof(double), v.stream));
    if (v.dim == 2)
        k_loss<2><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y, x1, u1, rho1,
                                                 (float)(1.0 / count), S->dYf, S->dYb, S->loss_d);
    else
        k_loss<3><<<nb(v.n), 256, 0, v.stream>>>(v.d, S->norm_d, S->t_jump, S->Y, x1, u1, rho1,
                                                 (float)(1.0 / count), S->dYf, S->dYb, S->loss_d);
    CUR(cudaGetLastError());
    if ((rc = backward(*S, v))) return rc;
    if (update) {
        S->adam_t += 1;
        const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
        // theta -= lr mhat / (sqrt(vhat) + eps) with mhat = m / c1, vhat = v / c2
        const double c1 = 1.0 - std::pow(b1, (double)S->adam_t), c2 = 1.0 - std::pow(b2, (double)S->adam_t);
        const double lr_t = lr * std::sqrt(c2) / c1, eps_t = eps * std::sqrt(c2);
        k_adam<<<nb(S->L.total), 256, 0, v.stream>>>(S->theta, S->grad, S->m, S->v, S->L.total, (float)lr_t,
                                                     (float)b1, (float)b2, (float)eps_t);
        CUR(cudaGetLastError());
        if ((rc = pack_weights(*S, v.stream))) return rc;
    }
    double loss = 0.0;
    CUR(cudaMemcpyAsync(&loss, S->loss_d, sizeof(double), cudaMemcpyDeviceToHost, v.stream));
    if (grad_out) {
        std::vector<float> g(ngrad);
        CUR(cudaMemcpyAsync(g.data(), S->grad, sizeof(float) * ngrad, cudaMemcpyDeviceToHost, v.stream));
        CUR(cudaStreamSynchronize(v.stream));
        for (int64_t k = 0; k < ngrad; ++k) grad_out[k] = g[k];
    }
    if ((rc = check_err(*S, v.stream))) return rc;
    if (loss_out) *loss_out = loss / count;
    return sim_check(h);
}

int sph_snapshot(sph_handle h, double *x_dev, double *u_dev, double *rho_dev)
{
    if (!h || !x_dev || !u_dev || !rho_dev) return set_error(SPH_EINVAL, "NULL argument");
    return sim_snapshot_device(h, x_dev, u_dev, rho_dev);
}

int sph_load_snapshot(sph_handle h, const double *x_dev, const double *u_dev, const double *rho_dev)
{
    if (!h || !x_dev || !u_dev || !rho_dev) return set_error(SPH_EINVAL, "NULL argument");
    return sim_load_device(h, x_dev, u_dev, rho_dev);
}

namespace {

// Errors that mean "the jump produced an unusable state" rather than a
// failure of the library.
bool state_error(int rc)
{
    return rc == SPH_ENONFINITE || rc == SPH_EDOMAIN || rc == SPH_ECAPACITY || rc == SPH_ECFL;
}

// The plain steps that judge or replace a jump must span the time the network
// jumps (its normalisation block's t_jump): k_steps * dt = t_jump, up to the
// rounding of either.
int check_jump_span(const Surrogate &S, double dt, int k_steps)
{
    const double span = (double)k_steps * dt;
    if (!(std::fabs(span - S.t_jump64) <= 1e-9 * S.t_jump64)) {
        char m[200];
        snprintf(m, sizeof m, "k_steps * dt = %.9g s differs from the network's jump span t_jump = %.9g s", span,
                 S.t_jump64);
        return set_error(SPH_EINVAL, m);
    }
    return SPH_OK;
}

// Snapshot buffers of the judged run (allocated once per surrogate).
int judge_buffers(Surrogate &S, const SimView &v, sph_handle h)
{
    if (S.sx) return SPH_OK;
    const size_t nd = (size_t)v.n * v.dim;
    const size_t words = (size_t)sim_occupancy_words(h);
    int e = dalloc(S, &S.sx, nd) | dalloc(S, &S.su, nd) | dalloc(S, &S.sr, (size_t)v.n) |
            dalloc(S, &S.vx, nd) | dalloc(S, &S.vu, nd) | dalloc(S, &S.vr, (size_t)v.n) |
            dalloc(S, &S.occ_a, words) | dalloc(S, &S.occ_b, words);
    if (e) return SPH_ENOMEM;
    CUR(cudaDeviceSynchronize());
    return SPH_OK;
}

// One judged macro-step: the surrogate jump and k plain steps from the same
// state; the plain result is kept.  *err = |c_jump - c_plain| / d_ref for the
// oil centroids, *ierr = |O_jump xor O_plain| / |O_plain| for the oil
// occupancies (both 1e30 when the jump broke the state).  Updates the
// surrogate's maxima; *reject tells whether either tolerance is exceeded.
int judged_jump(sph_handle h, Surrogate &S, const SimView &v, double dt, int k_steps, double d_ref, double tol,
                double *err, bool *reject)
{
    int rc;
    if ((rc = sim_snapshot_device(h, S.sx, S.su, S.sr))) return rc;
    if ((rc = sph_surrogate_advance(h, k_steps))) return rc;
    double cs[3] = {0, 0, 0}, cp[3];
    const int crc = sim_centroid(h, cs);
    if (crc && !state_error(crc)) return crc;
    if (!crc && (rc = sim_occupancy(h, S.occ_a))) return rc;
    if ((rc = sim_load_device(h, S.sx, S.su, S.sr))) return rc;
    if ((rc = sim_moved(h, -k_steps, -S.t_jump64))) return rc;
    if ((rc = sph_run(h, dt, k_steps, 1))) return rc;
    if ((rc = sim_centroid(h, cp))) return rc;
    double ierr = 1.0e30;
    if (!crc) {
        if ((rc = sim_occupancy(h, S.occ_b))) return rc;
        if ((rc = sim_occupancy_error(h, S.occ_a, S.occ_b, &ierr))) return rc;
    }
    double e2 = 0.0;
    for (int c = 0; c < v.dim; ++c) e2 += (cs[c] - cp[c]) * (cs[c] - cp[c]);
    *err = crc ? 1.0e30 : std::sqrt(e2) / d_ref;
    S.max_cerr = std::max(S.max_cerr, *err);
    S.max_ierr = std::max(S.max_ierr, ierr);
    *reject = *err > tol || (S.itol > 0 && ierr > S.itol);
    return SPH_OK;
}

}  // namespace

int sph_surrogate_advance_judged(sph_handle h, double dt, int k_steps, double tol, double d_ref, double *err)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (!(dt > 0) || k_steps < 1 || !(tol > 0) || !(d_ref > 0))
        return set_error(SPH_EINVAL, "bad dt, k_steps, tol or d_ref");
    if (int e = check_jump_span(*S, dt, k_steps)) return e;
    const SimView v = sim_view(h);
    int rc = judge_buffers(*S, v, h);
    if (rc) return rc;
    double e = 0.0;
    bool reject = false;
    S->max_cerr = S->max_ierr = 0.0;
    if ((rc = judged_jump(h, *S, v, dt, k_steps, d_ref, tol, &e, &reject))) return rc;
    if (err) *err = e;
    if ((rc = check_err(*S, v.stream))) return rc;
    if ((rc = sim_check(h))) return rc;
    return reject ? set_error(SPH_EFALLBACK, "the judge rejected the surrogate jump; the state holds the plain steps")
                  : SPH_OK;
}

int sph_surrogate_set_interface_tol(sph_handle h, double tol)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (!(tol >= 0) || !std::isfinite(tol)) return set_error(SPH_EINVAL, "tol must be >= 0");
    S->itol = tol;
    return SPH_OK;
}

int sph_surrogate_judge_stats(sph_handle h, double *max_centroid_err, double *max_interface_err)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (max_centroid_err) *max_centroid_err = S->max_cerr;
    if (max_interface_err) *max_interface_err = S->max_ierr;
    return SPH_OK;
}

int sph_surrogate_run(sph_handle h, double dt, int k_steps, int64_t n_macro, int judge_every, double tol,
                      double d_ref, int64_t *n_judged, int64_t *n_rejected, double *max_err)
{
    Surrogate *S = get(h);
    if (!S) return set_error(SPH_EINVAL, "no surrogate on this handle");
    if (!(dt > 0) || k_steps < 1 || n_macro < 0 || judge_every < 0 || !(tol > 0) || !(d_ref > 0))
        return set_error(SPH_EINVAL, "bad dt, k_steps, n_macro, judge_every, tol or d_ref");
    if (int e = check_jump_span(*S, dt, k_steps)) return e;
    const SimView v = sim_view(h);
    if (int e = judge_buffers(*S, v, h)) return e;
    S->max_cerr = S->max_ierr = 0.0;
    // a state the plain method produced or accepted, and the macro-step it belongs to
    auto verify = [&](int64_t m, int64_t &mv) {
        mv = m;
        return sim_snapshot_device(h, S->vx, S->vu, S->vr);
    };
    int64_t judged = 0, rejected = 0, mv = 0;
    double worst = 0.0;
    bool fallback = false;
    int rc = verify(0, mv);
    if (rc) return rc;
    for (int64_t mstep = 0; mstep < n_macro; ++mstep) {
        const bool judge = judge_every > 0 && (mstep % judge_every) == 0;
        if (judge) {
            // surrogate jump and plain steps from the same state; the plain result is kept
            double err = 0.0;
            bool reject = false;
            rc = judged_jump(h, *S, v, dt, k_steps, d_ref, tol, &err, &reject);
            if (rc && !state_error(rc)) return rc;
            if (rc) {
                // the plain steps failed from the state the unjudged jumps left: back to
                // the last verified state, plain steps from there
                const int64_t redo = (mstep + 1 - mv) * k_steps;
                if ((rc = sim_load_device(h, S->vx, S->vu, S->vr))) return rc;
                if ((rc = sim_moved(h, -redo, -(double)(mstep + 1 - mv) * S->t_jump64))) return rc;
                if ((rc = sph_run(h, dt, redo, 1))) return rc;
                err = 1.0e30;
                reject = true;
                S->max_cerr = std::max(S->max_cerr, err);
            }
            worst = std::max(worst, err);
            ++judged;
            fallback = reject;
            rejected += fallback ? 1 : 0;
            if ((rc = verify(mstep + 1, mv))) return rc;
        } else if (fallback) {
            if ((rc = sph_run(h, dt, k_steps, 1))) return rc;
        } else {
            if ((rc = sph_surrogate_advance(h, k_steps))) return rc;
            const int crc = sim_check(h);
            if (crc && !state_error(crc)) return crc;
            if (crc) {
                // the jump broke the state: back to the last verified state, plain steps from there
                const int64_t redo = (mstep + 1 - mv) * k_steps;
                if ((rc = sim_load_device(h, S->vx, S->vu, S->vr))) return rc;
                if ((rc = sim_moved(h, -redo, -(double)(mstep + 1 - mv) * S->t_jump64))) return rc;
                if ((rc = sph_run(h, dt, redo, 1))) return rc;
                ++rejected;
                fallback = true;
                if ((rc = verify(mstep + 1, mv))) return rc;
            }
        }
    }
    if ((rc = check_err(*S, v.stream))) return rc;
    if (n_judged) *n_judged = judged;
    if (n_rejected) *n_rejected = rejected;
    if (max_err) *max_err = worst;
    return sim_check(h);
}

}  // extern "C"
