// Persistent form of a time step: one cooperative launch runs the prediction, the PNCG iterations and the
// velocity update, with grid-wide barriers between the phases of Algorithm 1 instead of kernel boundaries.  At
// the 98K-tet scale a phase moves a few MB out of L2 in about a microsecond, so launch gaps and per-kernel ramp-up,
// not bandwidth, bound the multi-kernel form; here every block stays resident for the whole step.
//
// Reductions: each block reduces its threads, writes one partial per quantity, and after the barrier every block
// sums all partials in block order itself (so all blocks hold bitwise identical scalars and no second barrier is
// needed).  In the FP32 form partial sums are carried as float-float (about 48 bits) on the FP32 pipes; in the FP64
// form they are doubles.
//
// One iteration has four grid barriers: gradient | beta dots | direction + p^T H p | update.  The direction
// p_{k+1} = -P g + beta p_k is not a phase of its own: the beta pass stores P g per vertex, and the p^T H p pass
// forms p_{k+1} of every vertex it touches from P g and p_k (one rounding order everywhere, so the values agree
// bitwise); the update pass then stores it as the current direction.
//
// Barrier waits are bounded: a block that waits longer than the limit sets ERR_TIMEOUT and carries on; later
// barriers do not wait once the bit is set, so the launch always terminates and the host reports SIM_ERR_TIMEOUT.
#pragma once

#include "broadphase.cuh"
#include "kernels.cuh"

namespace pncg {

// The block size PB (threads per block) and the blocks per SM of the persistent kernel are template parameters:
// the library instantiates a few shapes (persist_shapes) and can pick one per workload by timing (the block-shape
// autotuner, sim_options.block_shape = -1).
constexpr int MAXG = 1024;   // most blocks a persistent launch may have (the host caps its grid at this)
constexpr unsigned long long BARRIER_LIMIT_NS = 4000000000ull;   // a barrier wait gives up after 4 s

// Arrival counter of the grid barriers, zeroed before each launch.  Every block passes the same sequence of
// barriers, so the n-th barrier is complete once the counter reaches n * gridDim.x.
struct Bar {
    unsigned int *count;
    unsigned int n;
    // profiling (arrive = null: off): per barrier and block, globaltimer at arrival and at departure, and the
    // phase the barrier closes
    unsigned long long *arrive, *depart;
    int *kind;
    int max, phase;
};

__device__ inline unsigned int ld_relaxed(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ inline void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ inline void red_release_add(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Polls *count until it reaches target.  Every 32 polls it reads the global nanosecond timer: once limit_ns have
// passed since the first reading it sets ERR_TIMEOUT in *err and gives up, and it also gives up at once when
// another waiter has set that bit.  Returns false when it gave up.
__device__ inline bool wait_count(const unsigned int *count, unsigned int target, uint32_t *err,
                                  unsigned long long limit_ns)
{
    unsigned long long t0 = 0;
    int n = 0;
    while ((int)(ld_relaxed(count) - target) < 0) {
        if ((++n & 31) == 0) {
            if (*(volatile uint32_t *)err & ERR_TIMEOUT) return false;
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) { atomicOr(err, ERR_TIMEOUT); return false; }
        }
    }
    return true;
}

// The block's writes are ordered before its arrival by the CTA barrier and the release add (a release operation is a
// cumulative fence followed by the add, so no separate fence is needed; the add needs no round trip).  The lead
// thread polls the counter with relaxed loads and, once it has seen every arrival, orders the block's later reads
// after the other blocks' writes with one acquire fence, before the CTA barrier hands on to the block.
__device__ inline void grid_barrier(Bar &br, Ctrl *c)
{
    __syncthreads();
    br.n += 1;
    if (threadIdx.x == 0) {
        const unsigned int target = br.n * gridDim.x;
        const bool rec = br.arrive && (int)br.n <= br.max;
        if (rec) br.arrive[(size_t)(br.n - 1) * gridDim.x + blockIdx.x] = global_ns();
        red_release_add(br.count, 1u);
        wait_count(br.count, target, &c->err, BARRIER_LIMIT_NS);
        fence_acq_rel();
        if (rec) {
            br.depart[(size_t)(br.n - 1) * gridDim.x + blockIdx.x] = global_ns();
            if (blockIdx.x == 0) br.kind[br.n - 1] = br.phase;
        }
    }
    __syncthreads();
}

// --------------------------------------------------------------------------------------------------- accumulators

// R = float: float-float; R = double: double.
template <typename R> struct Acc;
template <> struct Acc<double> {
    double v = 0.0;
    __device__ inline void add(double x) { v += x; }
    __device__ inline void add_d(double x) { v += x; }
    __device__ inline void add(const Acc &o) { v += o.v; }
    __device__ inline void add_ff(double h, double l) { v += h + l; }
    __device__ inline Acc shfl_down(int o) const { Acc r; r.v = __shfl_down_sync(0xffffffffu, v, o); return r; }
    __device__ inline Acc shfl_up(int o) const { Acc r; r.v = __shfl_up_sync(0xffffffffu, v, o); return r; }
    __device__ inline double value() const { return v; }
    __device__ inline double head() const { return v; }
};
template <> struct Acc<float> {
    float h = 0.0f, l = 0.0f;
    __device__ inline void add(float x)
    {
        const float s = __fadd_rn(h, x), bp = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        h = s;
        l = __fadd_rn(l, e);
    }
    __device__ inline void add(const Acc &o)
    {
        const float s = __fadd_rn(h, o.h), bp = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(o.h, bp));
        h = s;
        l = __fadd_rn(__fadd_rn(l, o.l), e);
    }
    __device__ inline void add_ff(float oh, float ol)   // a float-float term
    {
        Acc o;
        o.h = oh;
        o.l = ol;
        add(o);
    }
    __device__ inline void add_d(double x)   // a double term: its float head and the rounding remainder
    {
        const float xh = (float)x;
        add(xh);
        l = __fadd_rn(l, (float)(x - (double)xh));
    }
    __device__ inline Acc shfl_down(int o) const
    {
        Acc r;
        r.h = __shfl_down_sync(0xffffffffu, h, o);
        r.l = __shfl_down_sync(0xffffffffu, l, o);
        return r;
    }
    __device__ inline Acc shfl_up(int o) const
    {
        Acc r;
        r.h = __shfl_up_sync(0xffffffffu, h, o);
        r.l = __shfl_up_sync(0xffffffffu, l, o);
        return r;
    }
    __device__ inline double value() const { return (double)h + (double)l; }
    __device__ inline float head() const { return h; }
};

// partial-sum storage per block and quantity
template <typename R> struct PartT;
template <> struct PartT<float> { typedef float2 T; };
template <> struct PartT<double> { typedef double T; };
__device__ inline void put_part(float2 *p, const Acc<float> &a) { *p = make_float2(a.h, a.l); }
__device__ inline void put_part(double *p, const Acc<double> &a) { *p = a.v; }
__device__ inline void get_part(const float2 *p, Acc<float> &a) { const float2 v = __ldcg(p); a.h = v.x; a.l = v.y; }
__device__ inline void get_part(const double *p, Acc<double> &a) { a.v = __ldcg(p); }


// Scalars that the lead thread of each block reads once after a reduction's barrier (instead of every thread
// reading one hot address): a counter and the error bits.
struct Fetch {
    const int *pi = nullptr;
    const uint32_t *pe = nullptr;
};

constexpr int NQ = 5;   // most quantities one grid reduction carries

// Shared memory of the persistent kernel's reductions.  The per-thread values of a reduction are stored
// transposed (one row per quantity), so that warp q reduces quantity q: few (FP64) additions per block.
__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// The block's contiguous share [b0, b1) of n items, about n / gridDim.x each.  Vertices, tets and pairs are fewer
// than (or not many more than) the grid's threads, so a grid-stride loop would leave the later blocks idle and pile
// the work, and the FP64 vertex arithmetic, on the SMs of the first ones.
struct Share { int b0, b1; };
__device__ inline Share share_of(int n)
{
    const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int b0 = min(n, (int)blockIdx.x * per);
    return {b0, min(n, b0 + per)};
}

template <typename R, int PB> struct PShared {
    Acc<R> t[NQ][PB];
    R mx[PB];
    double res[NQ + 1];   // reduced results: sums, then the max
    double o[4];          // scalars computed by thread 0 and broadcast to the block
    int oi[2];
    int fi;
    uint32_t fe;
};

// Block part of a grid reduction: N sums (and, with MX, a max of non-negative values) of the block's threads,
// written as the block's partials (quantity q at part[q * gridDim.x + block], the max in slot N).
template <typename R, int PB, int N, bool MX>
__device__ inline void block_publish(Acc<R> (&a)[N], R mx, typename PartT<R>::T *part, PShared<R, PB> &sh)
{
    static_assert(N <= NQ && N + (MX ? 1 : 0) <= PB / 32, "one warp per quantity");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) sh.t[q][threadIdx.x] = a[q];
    if (MX) sh.mx[threadIdx.x] = mx;
    __syncthreads();
    if (warp < N) {
        Acc<R> s = sh.t[warp][lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) s.add(sh.t[warp][lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_down(o));
        if (lane == 0) put_part(part + warp * gridDim.x + blockIdx.x, s);
    } else if (MX && warp == N) {
        R m = sh.mx[lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) m = fmax(m, sh.mx[lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if (lane == 0) { Acc<R> b; b.add(m); put_part(part + N * gridDim.x + blockIdx.x, b); }
    }
}

// After the barrier: every thread loads the partials of blocks t and t + PB (all quantities: one round trip to
// L2), then the block reduces them transposed like block_publish (warp q sums quantity q, warp N takes the max, in
// block order within each lane's stride); the results land in sh.res (sums in double), and thread 0 reads the
// fetched scalars.  Every block computes bitwise the same results.  Ends with a CTA barrier.
template <typename R, int PB, int N, bool MX>
__device__ inline void grid_collect(const typename PartT<R>::T *part, PShared<R, PB> &sh, const Fetch *f)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    if (f && threadIdx.x == 0) {
        if (f->pi) sh.fi = (volatile const int &)*f->pi;
        if (f->pe) sh.fe = (volatile const uint32_t &)*f->pe;
    }
    Acc<R> v[N][(MAXG + PB - 1) / PB];
    R m = R(0);
#pragma unroll
    for (int j = 0; j < (MAXG + PB - 1) / PB; ++j) {
        const int b = threadIdx.x + j * PB;
        if (b < G) {
#pragma unroll
            for (int q = 0; q < N; ++q) get_part(part + q * G + b, v[q][j]);
            if (MX) { Acc<R> w; get_part(part + N * G + b, w); m = fmax(m, w.head()); }
        }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
        Acc<R> s = v[q][0];
#pragma unroll
        for (int j = 1; j < (MAXG + PB - 1) / PB; ++j) s.add(v[q][j]);
        sh.t[q][threadIdx.x] = s;
    }
    if (MX) sh.mx[threadIdx.x] = m;
    __syncthreads();
    if (warp < N) {
        Acc<R> s = sh.t[warp][lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) s.add(sh.t[warp][lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_down(o));
        if (lane == 0) sh.res[warp] = s.value();
    } else if (MX && warp == N) {
        R mm = sh.mx[lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) mm = fmax(mm, sh.mx[lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) mm = fmax(mm, __shfl_down_sync(0xffffffffu, mm, o));
        if (lane == 0) sh.res[N] = (double)mm;
    }
    __syncthreads();
}

// Grid-wide sums of N accumulators (and a max): block part, barrier, collection into sh.res.
template <typename R, int PB, int N, bool MX>
__device__ inline void grid_reduce(Acc<R> (&a)[N], R mx, typename PartT<R>::T *part, PShared<R, PB> &sh, Bar &br,
                                   Ctrl *c, const Fetch *f = nullptr)
{
    block_publish<R, PB, N, MX>(a, mx, part, sh);
    grid_barrier(br, c);
    grid_collect<R, PB, N, MX>(part, sh, f);
}

// Grid-wide max of non-negative values of the element type (exact); one grid barrier.  `part` holds gridDim.x
// values of type R.  Returned in every thread.
template <typename R, int PB>
__device__ inline R grid_max(R v, R *part, PShared<R, PB> &sh, Bar &br, Ctrl *c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sh.mx[threadIdx.x] = v;
    __syncthreads();
    if (warp == 0) {
        R m = sh.mx[lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) m = fmax(m, sh.mx[lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if (lane == 0) part[blockIdx.x] = m;
    }
    grid_barrier(br, c);
    R m = R(0);
#pragma unroll
    for (int j = 0; j < (MAXG + PB - 1) / PB; ++j) {
        const int b = threadIdx.x + j * PB;
        if (b < (int)gridDim.x) m = fmax(m, __ldcg(part + b));
    }
    sh.mx[threadIdx.x] = m;
    __syncthreads();
    if (warp == 0) {
        R mm = sh.mx[lane];
#pragma unroll
        for (int j = 1; j < PB / 32; ++j) mm = fmax(mm, sh.mx[lane + 32 * j]);
        for (int o = 16; o > 0; o >>= 1) mm = fmax(mm, __shfl_down_sync(0xffffffffu, mm, o));
        if (lane == 0) sh.res[0] = (double)mm;
    }
    __syncthreads();
    const R r = (R)sh.res[0];
    __syncthreads();
    return r;
}

// a value that thread 0 reads once for the whole block
__device__ inline int block_read(const int *p, int *sh)
{
    if (threadIdx.x == 0) *sh = (volatile const int &)*p;
    __syncthreads();
    const int v = *sh;
    __syncthreads();
    return v;
}

struct PersistArgs {
    int do_predict, k0, n_iters, do_finish;
    unsigned int *count;          // barrier arrival counter (zeroed before the launch)
    void *part;                   // reduction partials: 2 x 8 x gridDim.x of the partial type, then 2 x gridDim.x R
    unsigned long long *stamps;   // profiling (null = off): globaltimer at the end of each phase, seen by block 0
    int *stamp_kind;              // the phase each stamp closes (K_* of sim.h order)
    int max_stamps;
    unsigned long long *arrive, *depart;   // profiling (null = off): [max_bar][gridDim.x] barrier times
    int *bar_kind;                // [max_bar] phase closed by each barrier
    int max_bar;
};

// block 0's lead thread records the end of a phase (after the barrier that closes it)
struct Stamper {
    unsigned long long *t;
    int *kind;
    int max, n = 0;
    __device__ inline void mark(int k)
    {
        if (t && blockIdx.x == 0 && threadIdx.x == 0 && n < max) { t[n] = global_ns(); kind[n] = k; }
        ++n;
    }
};

// Consecutive grid reductions alternate between two partial regions: a block writes region r only after passing
// the barrier of reduction r - 1, which every block reaches after reading region r - 2 = r.
struct RedBufs {
    void *base;
    int n;
    int sum_i = 0, max_i = 0;
    template <typename PT> __device__ inline PT *sum_region() { return (PT *)base + (size_t)(sum_i++ & 1) * 8 * n; }
    template <typename PT, typename R> __device__ inline R *max_region() { return (R *)((PT *)base + (size_t)16 * n) + (size_t)(max_i++ & 1) * n; }
};

// the displacement reference of a vertex (its position at the last candidate build): the float copy in the FP32
// form, the double position in the FP64 form; and the squared displacement of a new position from it
template <typename R> struct DispRef;
template <> struct DispRef<float> { typedef float4 T; };
template <> struct DispRef<double> { typedef double4_32a T; };
template <typename R> __device__ inline typename DispRef<R>::T disp_ref(const Dev<R> &D, int i);
template <> __device__ inline float4 disp_ref<float>(const Dev<float> &D, int i) { return ldcg4(D.xbh + i); }
template <> __device__ inline double4_32a disp_ref<double>(const Dev<double> &D, int i) { return ldcg4(D.xb + i); }
template <typename R> __device__ inline R disp2_from(const double4_32a &X, const typename DispRef<R>::T &B)
{
    if constexpr (sizeof(R) == 4) {   // the float head of the float-float copy, as disp2 forms it
        const float x = __double2float_rn(X.x) - B.x, y = __double2float_rn(X.y) - B.y, z = __double2float_rn(X.z) - B.z;
        return x * x + y * y + z * z;
    } else {
        return dist2(X, B);
    }
}

} // namespace pncg

#include "batched.cuh"

namespace pncg {

// ------------------------------------------------------------------------------------------------ the kernel

template <typename R, int PB, int MINB, bool CO = false>
__global__ void __launch_bounds__(PB, MINB) k_persistent(Dev<R> D, BPDev B, PersistArgs A)
{
    typedef typename V4<R>::T R4;
    typedef typename PartT<R>::T PT;
    static_assert(PB % 32 == 0 && PB / 32 >= NQ + 1, "one warp per reduced quantity");
    __shared__ __align__(16) unsigned char sh_raw[sizeof(PShared<R, PB>)];   // raw storage: Acc has initialisers
    PShared<R, PB> &sh = *reinterpret_cast<PShared<R, PB> *>(sh_raw);
    __shared__ int sh_i;
    // one buffer for several phases: the gradient's block-scatter accumulators, the candidate build's chunk
    // offsets, then the warps' query batches
    constexpr size_t SBUF = cmax(cmax(sizeof(R) * 6 * SCATTER_MAXU, sizeof(unsigned int) * BP_MAX_CHUNKS),
                                 sizeof(BPQWarp) * (PB / 32));
    __shared__ __align__(16) unsigned char sbuf[SBUF];
    static_assert(SBUF >= 2 * MAX_SCENES * sizeof(double), "the batched form keeps per-scene beta and alpha here");
    static_assert(SBUF >= (PB / 32) * 64 * sizeof(int), "the gradient pass queues candidates here, 64 per warp");
    // the block-aggregated scatter (options.scatter = block) covers one chunk of SCATTER_CHUNK tets per block: only
    // the shape with PB == SCATTER_CHUNK runs it (the host keeps that shape for it)
    Ctrl *c = D.ctrl;
    RedBufs rb;
    rb.base = A.part;
    rb.n = gridDim.x;
    Bar br{A.count, 0u, A.arrive, A.depart, A.bar_kind, A.max_bar, 0};
    int sred = 0;   // batched form: per-scene reductions done in this launch (round robin accumulators)
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const Share vs = share_of(D.nv), ts = share_of(D.nt);
    const int ov = vs.b0 + (int)threadIdx.x;   // this thread's own vertex (the first of its share), when < vs.b1
    // state every block reads before anyone can change it
    int rebuild = (volatile int &)c->rebuild;
    const bool skip_step = (volatile uint32_t &)c->err != 0u;
    double gPg_prev = (volatile double &)c->gPg_prev;
    double dE0 = (volatile double &)c->dE0;
    int converged = (volatile int &)c->converged;
    int ncand = (volatile int &)c->n_cand;
    const double disp_lim = 0.5 * D.pad_r * (1.0 - 1e-4);
    Stamper st{A.stamps, A.stamp_kind, A.max_stamps};
    if (lead) { c->ticket[TK_PAIRS] = 0u; c->ticket[TK_PAIRS1] = 0u; }
    grid_barrier(br, c);
    st.mark(-1);

    // ---------------------------------------------------------------- a0: prediction and iteration-0 init
    if (A.do_predict) {
        br.phase = 0;   // K_PREDICT
        R md = R(0);
        if (!skip_step) {
            for (int i = ov; i < vs.b1; i += PB) {
                double4_32a X = D.x[i];
                const double4_32a V = D.v[i];
                D.xt[i] = X;
                const int slot = D.fix_slot[i];
                double4_32a XT;
                if (slot >= 0) {
                    X.x = D.tgt[3 * slot]; X.y = D.tgt[3 * slot + 1]; X.z = D.tgt[3 * slot + 2];
                    XT = make_double4_32a(X.x, X.y, X.z, -1.0);
                    put_x<R>(D, i, X);
                } else {
                    const double h = D.h, h2 = D.h * D.h;
                    XT = make_double4_32a(X.x + h * V.x + h2 * D.grav[0], X.y + h * V.y + h2 * D.grav[1],
                                          X.z + h * V.z + h2 * D.grav[2], D.mass[i]);
                }
                D.xtil[i] = XT;
                put_xt<R>(D, i, XT);
                init_vertex<R>(D, i, X, XT, 0);
                if (D.cmark) D.cmark[i] = D.g[0][i].w != R(0) ? 1 : 0;   // within dhat of the plane at x_0
                md = fmax(md, (R)disp2<R>(D, i, X));
            }
        }
        const R m = grid_max<R, PB>(md, rb.max_region<PT, R>(), sh, br, c);
        if (!skip_step && (double)m >= disp_lim * disp_lim) rebuild = 1;
        gPg_prev = 0.0;
        dE0 = 0.0;
        converged = 0;
        if (lead) {
            c->k = 0; c->n_rebuilds = 0; c->n_capped = 0; c->n_near64 = 0; c->iters_done = 0; c->converged = 0;
            c->n_active = 0; c->dE0 = 0.0; c->gPg_prev = 0.0;
        }
        if (D.nseg > 1) seg_reset<R>(D);
        grid_barrier(br, c);
        st.mark(0);   // K_PREDICT
    }

    for (int it = 0; it < A.n_iters; ++it) {
        const int k = A.k0 + it;
        const int par = k & 1;
        // ------------------------------------------------------------ a1: candidate build when needed
        if (rebuild) {
            br.phase = 1;   // K_BP_BOXES
            // boxes, bucket counts to zero, build positions; the cell size is the grid max of the box extents
            if (lead) { c->n_cand = 0; c->n_units = 0; c->n_units_h = 0; c->n_rebuilds += 1; c->ticket[TK_QUERY] = 0u; }
            const int nprim = B.nf + B.ne;
            float ext_max = 0.0f;
            for (int j = tid; j < 3 * B.H; j += nthr) B.cnt[j] = 0u;
            for (int j = ov; j < vs.b1; j += PB) { B.xb[j] = ldcg4(B.x + j); if (B.xbh) B.xbh[j] = ldcg4(B.xh + j); }
            const Share ps = share_of(nprim);
            for (int j = ps.b0 + (int)threadIdx.x; j < ps.b1; j += PB) {
                int v[3];
                int nvp;
                if (j < B.nf) { const int4 t = B.tri[j]; v[0] = t.x; v[1] = t.y; v[2] = t.z; nvp = 3; }
                else { const int4 e = B.edge[j - B.nf]; v[0] = e.x; v[1] = e.y; nvp = 2; }
                float4 lo, hi;
                box_of(B.x, v, nvp, B.infl, lo, hi);
                B.blo[j] = lo;
                B.bhi[j] = hi;
                ext_max = fmaxf(ext_max, fmaxf(__fsub_ru(hi.x, lo.x), fmaxf(__fsub_ru(hi.y, lo.y), __fsub_ru(hi.z, lo.z))));
            }
            const float ext = (float)grid_max<R, PB>(R(ext_max), rb.max_region<PT, R>(), sh, br, c);
            if (lead) c->cell_bits = __float_as_uint(ext);
            st.mark(1);   // K_BP_BOXES
            const CellGrid cg = grid_of(ext * 1.0001f);   // as cell_size() forms it from cell_bits
            br.phase = 2;   // K_BP_COUNT
            for (int j = ps.b0 + (int)threadIdx.x; j < ps.b1; j += PB)
                for_cells(B, __ldcg(B.blo + j), __ldcg(B.bhi + j), cg, [&](int i, int jj, int kk) { atomicAdd(&B.cnt[prim_bucket(B, j, i, jj, kk)], 1u); });
            const Share ss = share_of(B.ns);
            for (int j = ss.b0 + (int)threadIdx.x; j < ss.b1; j += PB) {
                int v, cc[3];
                double4_32a X;
                if (point_cell(B, j, cg, v, X, cc)) atomicAdd(&B.cnt[point_bucket(B, cc[0], cc[1], cc[2])], 1u);
                else atomicOr(&c->err, ERR_RANGE);
            }
            grid_barrier(br, c);
            st.mark(2);   // K_BP_COUNT
            // exclusive scans of the chunks of 2^cshift buckets, one warp per chunk, four buckets per lane; the work
            // units of the triangle and edge buckets are listed on the way
            br.phase = 3;   // K_BP_SCAN
            const int cs = B.cshift_p;
            const int nchunk = (3 * B.H) >> cs;
            {
                const int gw = tid >> 5, lane = threadIdx.x & 31, nwarps = nthr >> 5;
                for (int ch = gw; ch < nchunk; ch += nwarps) {
                    unsigned int run = 0;
                    for (int base = ch << cs; base < (ch + 1) << cs; base += 128) {
                        const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(B.cnt + base) + lane);
                        {
                            const unsigned int b4 = (unsigned int)base + 4u * (unsigned int)lane;
                            const unsigned int bb[4] = {b4, b4 + 1u, b4 + 2u, b4 + 3u}, nn[4] = {v.x, v.y, v.z, v.w};
                            list_units(B, bb, nn);
                        }
                        const unsigned int tot = v.x + v.y + v.z + v.w;
                        unsigned int inc = tot;
                        for (int o = 1; o < 32; o <<= 1) {
                            const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
                            if (lane >= o) inc += n;
                        }
                        const unsigned int ex = run + inc - tot;
                        reinterpret_cast<uint4 *>(B.off + base)[lane] = make_uint4(ex, ex + v.x, ex + v.x + v.y, ex + v.x + v.y + v.z);
                        reinterpret_cast<uint4 *>(B.cnt + base)[lane] = make_uint4(0u, 0u, 0u, 0u);   // the fill cursor
                        run += __shfl_sync(0xffffffffu, inc, 31);
                    }
                    if (lane == 0) B.ctot[ch] = run;
                }
            }
            grid_barrier(br, c);
            st.mark(3);   // K_BP_SCAN
            // every block scans the chunk totals into shared memory; the buckets' global offsets go to goff for
            // the queries, and the entries to their slots
            br.phase = 4;   // K_BP_FILL
            unsigned int *choff = reinterpret_cast<unsigned int *>(sbuf);   // [BP_MAX_CHUNKS]
            {
                const int per = (nchunk + PB - 1) / PB;   // chunks per thread (nchunk <= BP_MAX_CHUNKS)
                const int c0 = threadIdx.x * per;
                unsigned int loc[(BP_MAX_CHUNKS + PB - 1) / PB];
                unsigned int tsum = 0;
#pragma unroll
                for (int q = 0; q < (BP_MAX_CHUNKS + PB - 1) / PB; ++q) {
                    loc[q] = (q < per && c0 + q < nchunk) ? __ldcg(B.ctot + c0 + q) : 0u;
                    tsum += loc[q];
                }
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                unsigned int inc = tsum;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += n;
                }
                __shared__ unsigned int wtot[PB / 32];
                if (lane == 31) wtot[warp] = inc;
                __syncthreads();
                unsigned int run = inc - tsum;
                for (int w = 0; w < warp; ++w) run += wtot[w];
#pragma unroll
                for (int q = 0; q < (BP_MAX_CHUNKS + PB - 1) / PB; ++q) {
                    if (q < per && c0 + q < nchunk) choff[c0 + q] = run;
                    run += loc[q];
                }
                __syncthreads();
            }
            for (int b = tid; b < 3 * B.H; b += nthr) B.goff[b] = choff[b >> cs] + __ldcg(B.off + b);
            {
                auto slot_of = [&](unsigned int b) { return choff[b >> cs] + __ldcg(B.off + b) + atomicAdd(&B.cnt[b], 1u); };
                for (int j = ps.b0 + (int)threadIdx.x; j < ps.b1; j += PB) fill_prim(B, j, cg, slot_of);
                for (int j = ss.b0 + (int)threadIdx.x; j < ss.b1; j += PB) fill_point(B, j, cg, slot_of);
            }
            grid_barrier(br, c);
            st.mark(4);   // K_BP_FILL
            // queries: the listed work units, the warp's staging area in sbuf; a warp takes its own unit, then
            // whichever units are left
            br.phase = 5;   // K_BP_QUERY
            {
                BPQWarp &W = reinterpret_cast<BPQWarp *>(sbuf)[threadIdx.x >> 5];
                const int nw = nthr >> 5;
                bpq_units(B, cg, W, tid >> 5, [&]() {
                    int nx = 0;
                    if ((threadIdx.x & 31) == 0) nx = nw + (int)atomicAdd(&c->ticket[TK_QUERY], 1u);
                    return __shfl_sync(0xffffffffu, nx, 0);
                });
            }
            grid_barrier(br, c);
            st.mark(5);   // K_BP_QUERY
            ncand = block_read(&c->n_cand, &sh_i);
            rebuild = 0;
        }
        // ------------------------------------------------------------ a2-a3: gradient + diagonal
        br.phase = 6;   // K_GRAD
        if (lead) {
            c->rebuild = 0;
            if (ncand > D.cand_cap) flag_error(c, ERR_CAPACITY);
        }
        {
            const Share cs = share_of(min(ncand, D.cand_cap));
            if (PB == SCATTER_CHUNK && D.scatter_block) {
                const int nch = (D.nt + SCATTER_CHUNK - 1) / SCATTER_CHUNK;
                for (int ch = blockIdx.x; ch < nch; ch += gridDim.x)
                    tet_grad_chunk<R, CO>(D, ch, par, reinterpret_cast<R *>(sbuf));
                for (int ci = cs.b0 + (int)threadIdx.x; ci < cs.b1; ci += PB) pair_grad<R>(D, ci, par);
            } else {
                // the block's share of the tets, then candidates 32 at a time per warp from a grid-wide cursor: the
                // active ones (float-float geometry) cluster in the candidate order, and a fixed share per block
                // left the blocks holding a contact patch 40 us behind the median one
                const int nts = ts.b1 - ts.b0;
                for (int q = threadIdx.x; q < nts; q += PB) {
                    TetIn<R> in;
                    load_tet_in<R>(D, ts.b0 + q, in);
                    tet_grad<R, CO>(D, ts.b0 + q, par, in);
                }
                if (lead) c->ticket[TK_PAIRS + ((k + 1) & 1)] = 0u;   // the next iteration's cursor
                unsigned int *cur = &c->ticket[TK_PAIRS + (k & 1)];
                const int nc = min(ncand, D.cand_cap), lane = threadIdx.x & 31;
                if constexpr (sizeof(R) == 4) {
                    // the float filter first; the candidates that pass it queue in shared memory (per warp) and
                    // take the float-float geometry 32 at a time, so that the long path runs with full warps (the
                    // passing ones are a fraction of each batch: a warp otherwise ran it once per batch)
                    int *wq = reinterpret_cast<int *>(sbuf) + (threadIdx.x >> 5) * 64;
                    int qn = 0;
                    const unsigned int below = (1u << lane) - 1u;
                    for (;;) {
                        int b0 = 0;
                        if (lane == 0) b0 = (int)atomicAdd(cur, 32u);
                        b0 = __shfl_sync(0xffffffffu, b0, 0);
                        if (b0 >= nc) break;
                        const int ci = b0 + lane;
                        const bool pass = ci < nc && pair_passes_filter(D, ci);
                        const unsigned int bal = __ballot_sync(0xffffffffu, pass);
                        if (pass) wq[qn + __popc(bal & below)] = ci;
                        qn += __popc(bal);
                        __syncwarp();
                        if (qn >= 32) {
                            const int cj = wq[qn - 32 + lane];
                            __syncwarp();
                            qn -= 32;
                            pair_grad<R>(D, cj, par);
                        }
                    }
                    if (lane < qn) pair_grad<R>(D, wq[lane], par);
                    __syncwarp();
                } else {
                    for (;;) {
                        int b0 = 0;
                        if (lane == 0) b0 = (int)atomicAdd(cur, 32u);
                        b0 = __shfl_sync(0xffffffffu, b0, 0);
                        if (b0 >= nc) break;
                        if (b0 + lane < nc) pair_grad<R>(D, b0 + lane, par);
                    }
                }
            }
        }
        grid_barrier(br, c);
        st.mark(6);   // K_GRAD
        if (D.segmented) {
            br.phase = 7;   // K_GATHER
            const int n4 = 4 * D.nt;
            for (int i = ov; i < vs.b1; i += PB) {
                R s6[6] = {0, 0, 0, 0, 0, 0};
                for (int q = D.v2c_off[i]; q < D.v2c_off[i + 1]; ++q) {
                    const int cc = D.v2c[q];
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk) s6[kk] += __ldcg(D.contrib + kk * n4 + cc);
                }
                R4 G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i);
                G.x += s6[0]; G.y += s6[1]; G.z += s6[2];
                Dg.x += s6[3]; Dg.y += s6[4]; Dg.z += s6[5];
                D.g[par][i] = G;
                D.dg[par][i] = Dg;
            }
            grid_barrier(br, c);
            st.mark(7);   // K_GATHER
        }
        if (D.nseg > 1) {   // batched scenes: per-scene beta, alpha (batched.cuh)
            if (batched_tail<R, PB, CO>(D, c, sh, sbuf, br, st, rb, k, par, sred, disp_lim)) rebuild = 1;
            continue;
        }
        // ------------------------------------------------------------ a4: beta (and P g for the direction)
        double beta = 0.0;
        int restarted = 0;
        int na;
        R4 oG, oDg, oPG, oP0;   // this thread's own vertex (i == ov), kept for the direction pass
        br.phase = 8;   // K_DOTS
        {
            Acc<R> s5[5];
            for (int i = ov; i < vs.b1; i += PB) {
                const R4 G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i), G0 = ldcg4(D.g[par ^ 1] + i);
                R4 P0 = ldcg4(D.p + i);
                R4 PG = mk4<R>(R(0), R(0), R(0), R(0));
                if (Dg.w > R(0)) {
                    const R gv[3] = {G.x, G.y, G.z}, dv[3] = {Dg.x, Dg.y, Dg.z}, g0[3] = {G0.x, G0.y, G0.z}, p0[3] = {P0.x, P0.y, P0.z};
                    R th[5], tl[5], pg[3];
                    beta_terms<R>(gv, dv, g0, p0, Dg.w, D.beta_rule, th, tl, pg);
#pragma unroll
                    for (int q = 0; q < 5; ++q) s5[q].add_ff(th[q], tl[q]);
                    PG = mk4<R>(pg[0], pg[1], pg[2], R(0));
                } else if (P0.x != R(0) || P0.y != R(0) || P0.z != R(0)) {
                    D.p[i] = PG;   // a kinematic vertex never moves along p
                    P0 = PG;
                }
                D.pg[i] = PG;
                if (i == ov) { oG = G; oDg = Dg; oPG = PG; oP0 = P0; }
            }
            Fetch f;
            f.pi = &c->n_active;
            grid_reduce<R, PB, 5, false>(s5, R(0), rb.sum_region<PT>(), sh, br, c, &f);
            st.mark(8);   // K_DOTS
            // beta and the restart test: scalar FP64 work, done by one thread and broadcast
            if (threadIdx.x == 0) {
                const double *t = sh.res;
                double bt = 0.0, gPg, gp_new;
                int rs = 0;
                if (D.beta_rule == 0) {
                    gPg = t[1];
                    if (k > 0) { bt = gPg_prev > 0.0 ? t[0] / gPg_prev : 0.0; if (bt < 0.0) bt = 0.0; }
                    gp_new = -gPg + bt * t[2];
                } else {
                    gPg = t[4];
                    if (k > 0) bt = fabs(t[2]) < 1e-30 ? 0.0 : t[0] / t[2] - (t[1] / t[2]) * (t[3] / t[2]);
                    gp_new = -gPg + bt * t[3];
                }
                if (gp_new >= 0.0 && bt != 0.0) { bt = 0.0; rs = 1; }
                sh.o[0] = bt;
                sh.o[1] = gPg;
                sh.oi[0] = rs;
                sh.oi[1] = sh.fi;
            }
            __syncthreads();
            beta = sh.o[0];
            gPg_prev = sh.o[1];
            restarted = sh.oi[0];
            na = sh.oi[1];
        }
        // ------------------------------------------------------------ a5-a7: direction, p^T H p and the step
        double alpha;
        double4_32a uX, uXT;
        R4 uP;
        typename DispRef<R>::T uXB;
        br.phase = 10;   // K_PHP
        {
            const R b = R(beta);
            const bool nzb = beta != 0.0;
            Acc<R> s3[3];   // g . p, p^T M p (+ half-space part), p^T H p of tets and pairs
            R pm = R(0);
            for (int i = ov; i < vs.b1; i += PB) {
                const bool own = i == ov;
                const R4 Dg = own ? oDg : ldcg4(D.dg[par] + i);
                R4 Pn = mk4<R>(R(0), R(0), R(0), R(0));
                if (Dg.w > R(0)) {
                    const R4 G = own ? oG : ldcg4(D.g[par] + i);
                    Pn = own ? dir_from<R>(oPG, oP0, b, nzb) : dir_of<R>(D, i, b, nzb);
                    const R px = Pn.x, py = Pn.y, pz = Pn.z;
                    s3[0].add(G.x * px + G.y * py + G.z * pz);
                    R mp = Dg.w * (px * px + py * py + pz * pz);
                    if (D.has_plane && G.w != R(0)) {
                        const R np = R(D.pn[0]) * px + R(D.pn[1]) * py + R(D.pn[2]) * pz;
                        mp += G.w * np * np;
                    }
                    s3[1].add(mp);
                    const R pn = D.pnorm == 0 ? sqrt(px * px + py * py + pz * pz) : fmax(fabs(px), fmax(fabs(py), fabs(pz)));
                    pm = fmax(pm, pn);
                }
                D.pnext[i] = Pn;
            }
            // the block's tets and active pairs as one list, so that no thread takes more than its share of both (the
            // vertex pass above is short)
            const Share as = share_of(na);
            const int nts = ts.b1 - ts.b0, nit = nts + (as.b1 - as.b0);
            int4 tvn = (int)threadIdx.x < nts ? D.tet[ts.b0 + threadIdx.x] : make_int4(0, 0, 0, 0);   // one tet ahead
            for (int q = threadIdx.x; q < nit; q += PB) {
                if (q < nts) {
                    const int e = ts.b0 + q;
                    const int4 tv = tvn;
                    if (q + PB < nts) tvn = D.tet[e + PB];
                    s3[2].add(tet_pHp_vec<R, CO>(D, e, tv, dir_of<R>(D, tv.x, b, nzb), dir_of<R>(D, tv.y, b, nzb),
                                             dir_of<R>(D, tv.z, b, nzb), dir_of<R>(D, tv.w, b, nzb)));
                } else {
                    Active<R> ap;
                    load_active<R>(D, as.b0 + q - nts, ap);
                    s3[2].add_d(pair_pHp_vec<R>(ap, dir_of<R>(D, ap.v.x, b, nzb), dir_of<R>(D, ap.v.y, b, nzb),
                                                dir_of<R>(D, ap.v.z, b, nzb), dir_of<R>(D, ap.v.w, b, nzb)));
                }
            }
            Fetch f;
            f.pe = &c->err;
            PT *part = rb.sum_region<PT>();
            block_publish<R, PB, 3, true>(s3, pm, part, sh);
            grid_barrier(br, c);
            // the update's loads of this thread's own vertex go out before the partial collection and the step rule
            if (ov < vs.b1) {
                uX = ldcg4(D.x + ov);
                uP = ldcg4(D.pnext + ov);
                if constexpr (sizeof(R) == 8) uXT = ldcg4(D.xtil + ov);
                uXB = disp_ref<R>(D, ov);
            }
            grid_collect<R, PB, 3, true>(part, sh, &f);
            st.mark(10);  // K_PHP (direction included)
            // the step rule (Sec. 4.3) and the predicted decrease: scalar FP64 work, done by one thread
            if (threadIdx.x == 0) {
                const double gp = sh.res[0], pHp_vert = sh.res[1], pmax = sh.res[3];
                uint32_t err = sh.fe;
                const double pHp = sh.res[2] + pHp_vert;
                const double au = pmax > 0.0 ? D.dhat / (2.0 * pmax) : 0.0;
                const double ab = -gp / pHp;
                double a;
                int capped;
                if (!(pHp > 0.0) || !isfinite(ab)) { a = au; capped = 1; }
                else if (ab < au) { a = ab; capped = 0; }
                else { a = au; capped = 1; }
                const double dE = -a * gp - 0.5 * a * a * pHp;
                if (!isfinite(a) || !isfinite(gp)) {
                    if (lead) flag_error(c, ERR_NONFINITE);
                    err |= ERR_NONFINITE;
                    a = 0.0;
                }
                if (err != 0u || converged) a = 0.0;
                if (lead) {
                    c->beta = beta; c->restarted = restarted; c->gp = gp; c->pmax = pmax; c->pHp_vert = pHp_vert;
                    c->pHp = pHp; c->alpha_bar = ab; c->alpha_up = au; c->alpha = a; c->dE = dE; c->capped = capped;
                    c->n_active_last = na;
                    c->gPg_prev = gPg_prev;
                    if (!converged && err == 0u) {
                        if (k == 0) c->dE0 = dE;
                        c->n_capped += capped;
                        c->iters_done = k + 1;
                        if (D.trace && k < D.iters) {
                            double *tr = D.trace + (size_t)k * TRACE_COLS;
                            tr[0] = beta; tr[1] = gp; tr[2] = pHp; tr[3] = pmax; tr[4] = a; tr[5] = dE;
                            tr[6] = na; tr[7] = capped;
                        }
                    }
                    c->k = k + 1;
                }
                int cv = converged;
                double e0 = dE0;
                if (!cv && err == 0u) {
                    if (k == 0) e0 = dE;
                    if (D.eps > 0.0 && dE < D.eps * e0) cv = 1;
                }
                if (lead) { c->dE0 = e0; c->converged = cv; }
                sh.o[2] = a;
                sh.o[3] = e0;
                sh.oi[0] = cv;
            }
            __syncthreads();
            alpha = sh.o[2];
            dE0 = sh.o[3];
            converged = sh.oi[0];
        }
        // ------------------------------------------------------------ a8: update
        br.phase = 11;   // K_UPDATE
        {
            R md = R(0);
            const ffl as = ff_split(alpha);
            for (int i = ov; i < vs.b1; i += PB) {
                double4_32a X, XT;
                R4 P;
                typename DispRef<R>::T XB;
                if (i == ov) { X = uX; P = uP; XT = uXT; XB = uXB; }
                else {
                    X = ldcg4(D.x + i); P = ldcg4(D.pnext + i); XB = disp_ref<R>(D, i);
                    if constexpr (sizeof(R) == 8) XT = ldcg4(D.xtil + i);
                }
                const float4 xh = update_vertex<R>(D, i, X, P, alpha, as.h, as.l, XT, par ^ 1);
                D.p[i] = P;
                if constexpr (sizeof(R) == 4) {   // the float head just written, as disp2 forms it
                    const float dx = xh.x - XB.x, dy = xh.y - XB.y, dz = xh.z - XB.z;
                    md = fmax(md, dx * dx + dy * dy + dz * dz);
                } else {
                    md = fmax(md, disp2_from<R>(X, XB));
                }
            }
            if (lead) c->n_active = 0;
            const R m = grid_max<R, PB>(md, rb.max_region<PT, R>(), sh, br, c);
            st.mark(11);  // K_UPDATE
            if ((double)m >= disp_lim * disp_lim) rebuild = 1;
        }
    }
    if (lead && rebuild) c->rebuild = 1;

    // ---------------------------------------------------------------- velocity update
    if (A.do_finish) {
        br.phase = 12;   // K_FINISH
        grid_barrier(br, c);
        const bool bad = (volatile uint32_t &)c->err != 0u;
        for (int i = ov; i < vs.b1; i += PB) {
            const double4_32a X = ldcg4(D.x + i), XT = ldcg4(D.xt + i);
            if (bad) {
                put_x<R>(D, i, XT);
            } else {
                const double ih = 1.0 / D.h;
                double4_32a V = D.v[i];
                V.x = (X.x - XT.x) * ih; V.y = (X.y - XT.y) * ih; V.z = (X.z - XT.z) * ih;
                D.v[i] = V;
            }
        }
        if (lead) {
            if (bad) { if (c->err_step < 0) c->err_step = (int)c->step; }
            else c->step += 1;
        }
        grid_barrier(br, c);
        st.mark(12);  // K_FINISH
    }
}

} // namespace pncg
