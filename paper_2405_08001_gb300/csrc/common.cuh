// Internal definitions shared by the solver's CUDA translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pncg {

// sticky device error bits (Ctrl::err); the host maps them to sim_status
enum : uint32_t {
    ERR_INVERTED = 1u,
    ERR_PENETRATION = 2u,
    ERR_NONFINITE = 4u,
    ERR_CAPACITY = 8u,
    ERR_RANGE = 16u,
    ERR_TIMEOUT = 32u,
};

// ticket counters of the "last block finishes the reduction" kernels
// TK_PAIRS, TK_PAIRS + 1: the persistent gradient pass's candidate cursor, by iteration parity
enum { TK_PREDICT = 0, TK_DOTS, TK_DIR, TK_PHP, TK_UPDATE, TK_SCAN, TK_ENERGY, TK_MISC, TK_QUERY, TK_PAIRS,
       TK_PAIRS1, TK_COUNT };

constexpr int TRACE_COLS = 8;   // beta, gp, pHp, pmax, alpha, dE, n_active, capped

// block scatter of the tet contributions: chunks of SCATTER_CHUNK consecutive tets (one block of the tet loops);
// chunks with more than SCATTER_MAXU distinct vertices fall back to global atomics
constexpr int SCATTER_CHUNK = 256;
constexpr int SCATTER_MAXU = 512;

// batching: most independent scenes one handle takes (their beta and alpha live in shared memory)
constexpr int MAX_SCENES = 1024;

// Device-resident control block: every scalar of the iteration lives here, so no host round trip is needed
// inside a time step.
struct Ctrl {
    unsigned int ticket[TK_COUNT];
    uint32_t err;          // sticky error bits
    int32_t err_step;      // time step index of the first error (-1 = none)
    int32_t n_cand;        // candidates emitted by the last build (may exceed capacity)
    int32_t n_units;       // work units listed by the last build's scan, from the end of the list (may exceed
                           // capacity)
    int32_t n_units_h;     // the heavy ones (tiles of buckets of 64+ entries), from the front
    int32_t n_active;      // active pairs appended by the current gradient pass
    int32_t n_active_last; // active pairs of the last completed iteration
    int32_t rebuild;       // 1 = candidate build needed before the next gradient pass
    uint32_t cell_bits;    // float bits of the hash cell size of the current build (atomicMax of extents)
    int32_t k;             // index of the next iteration within the step
    int32_t n_rebuilds;
    int32_t n_capped;
    int32_t n_near64;      // FP32 form: pair evaluations that took the double branch (d < 1e-3 dhat) since the
                           // step started (or since the last sim_eval_* set-up)
    int32_t iters_done;
    int32_t converged;     // eps rule fired in this step
    int32_t restarted;
    int32_t capped;
    int64_t step;          // completed time steps
    double gPg_prev;       // g^T P g of the previous iteration (PR+ denominator)
    double beta;
    double gp, pmax, pHp_vert, pHp;
    double alpha, alpha_bar, alpha_up, dE, dE0;
    double energy[4];      // inertia, elastic, pair barrier, plane barrier (sim_eval_energy)
};

// Loads of data that other blocks write during a launch (positions, directions, accumulators, candidate and hash
// arrays) go through L2 (ld.global.cg): in the persistent form one launch spans many phases, and an SM's L1 may
// still hold a line from an earlier phase.
__device__ inline double4_32a ldcg4(const double4_32a *p)
{
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
    double4_32a r;
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}
__device__ inline float4 ldcg4(const float4 *p) { return __ldcg(p); }
__device__ inline int4 ldcg4(const int4 *p) { return __ldcg(p); }

template <typename R> struct V4;
template <> struct V4<float> { typedef float4 T; };
template <> struct V4<double> { typedef double4_32a T; };

template <typename R> __host__ __device__ inline typename V4<R>::T mk4(R a, R b, R c, R d);
template <> __host__ __device__ inline float4 mk4<float>(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
template <> __host__ __device__ inline double4_32a mk4<double>(double a, double b, double c, double d) { return make_double4_32a(a, b, c, d); }

// Per-scene state of the batched form (independent scenes in one launch).  The state carried between
// iterations is double-buffered by iteration parity: iteration k reads entry (k - 1) & 1 and writes k & 1, so the
// block that writes never races the blocks still reading the previous value.
struct SegCtl {
    double gPg[2];         // g^T P g (PR+ denominator of the next iteration)
    double dE0[2];         // Delta E of iteration 0 (eps rule)
    int32_t converged[2];
    int32_t restarted, capped, iters_done, pad;
    double beta, gp, pHp, pmax, alpha, dE;   // the most recent iteration, for reporting
};

// active contact pair recorded by the gradient pass for the p^T H p pass of the same iteration
template <typename R> struct alignas(16) Active {
    int4 v;     // vertex indices (PT: point, tri; EE: edge, edge)
    R c[4];     // closest-point coefficients
    R t[3];     // t = sum c_i x_i
    R A;        // kappa (b''/d^2 - b'/d^3)
    R B;        // kappa b'/d
    R d;        // distance
    int ty;     // 0 = point-triangle, 1 = edge-edge
};

// ---------------------------------------------------------------------------------------------- block reductions

// Sums N doubles over the block in a fixed order (warp shuffles, then the warp partials by warp 0).
// The result is valid in thread 0.  sh must hold 32*N doubles.
template <int N>
__device__ inline void block_sum(double (&v)[N], double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) sh[warp * N + q] = v[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            v[q] = lane < nw ? sh[lane * N + q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        }
    }
    __syncthreads();
}

__device__ inline double block_max(double v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

// Float-float warp sum (TwoSum at every shuffle level): about 2^-46 relative accuracy of the float inputs' sum.
__device__ inline void warp_sum_ff(float &h, float &l)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
        const float s = __fadd_rn(h, h2);
        const float bp = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
        h = s;
        l = __fadd_rn(__fadd_rn(l, l2), e);
    }
}

// Block sum of N per-thread values accumulated in double.  float inputs are summed in float-float within each warp
// and in double across warps (FP64 throughput on this GPU is a small fraction of FP32, so the wide per-thread tree
// stays on the FP32 pipes); double inputs use block_sum.  Result in thread 0.
template <int N>
__device__ inline void block_sum_acc(const float (&v)[N], double (&out)[N], double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        float h = v[q], l = 0.0f;
        warp_sum_ff(h, l);
        if (lane == 0) sh[warp * N + q] = (double)h + (double)l;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            out[q] = lane < nw ? sh[lane * N + q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) out[q] += __shfl_down_sync(0xffffffffu, out[q], o);
        }
    }
    __syncthreads();
}
// the same for float-float per-thread values (heads v, tails vl)
template <int N>
__device__ inline void block_sum_acc(const float (&v)[N], const float (&vl)[N], double (&out)[N], double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        float h = v[q], l = vl[q];
        warp_sum_ff(h, l);
        if (lane == 0) sh[warp * N + q] = (double)h + (double)l;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            out[q] = lane < nw ? sh[lane * N + q] : 0.0;
            for (int o = 16; o > 0; o >>= 1) out[q] += __shfl_down_sync(0xffffffffu, out[q], o);
        }
    }
    __syncthreads();
}
template <int N>
__device__ inline void block_sum_acc(const double (&v)[N], const double (&vl)[N], double (&out)[N], double *sh)
{
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = v[q] + vl[q];
    block_sum<N>(out, sh);
}
template <int N>
__device__ inline void block_sum_acc(const double (&v)[N], double (&out)[N], double *sh)
{
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = v[q];
    block_sum<N>(out, sh);
}

__device__ inline float block_max_f(float v, float *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? sh[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

// Publishes this block's partials and returns true in every thread of the block that arrives last.
// partials[q * nblk + blockIdx.x] = v[q] (written by thread 0).  The ticket is reset by the last block.
template <int N>
__device__ inline bool publish_partials(const double (&v)[N], double *partials, unsigned int *ticket)
{
    __shared__ bool last;
    const int nblk = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) partials[q * nblk + blockIdx.x] = v[q];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned int)nblk - 1);
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last block: sums partials of quantity q over all blocks in block-index order (result in thread 0).
template <int N>
__device__ inline void finish_sums(double (&out)[N], const double *partials, double *sh)
{
    const int nblk = gridDim.x;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += __ldcg(partials + q * nblk + b);
        out[q] = s;
    }
    block_sum<N>(out, sh);
}

__device__ inline double finish_max(const double *partials, int q, double *sh)
{
    const int nblk = gridDim.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s = fmax(s, __ldcg(partials + q * nblk + b));
    return block_max(s, sh);
}

} // namespace pncg
