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
// Barrier waits are bounded: a block that waits longer than the limit sets ERR_TIMEOUT and carries on; later
// barriers do not wait once the bit is set, so the launch always terminates and the host reports SIM_ERR_TIMEOUT.
#pragma once

#include "broadphase.cuh"
#include "kernels.cuh"

namespace pncg {

constexpr int PB = 256;                       // threads per block of the persistent kernel
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 26;   // ~ seconds at 32 ns per poll

struct GridSync {
    unsigned int *count;
    unsigned int *gen;
};

__device__ inline unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrival: one atomic per block on `count` after a fence; release: the last block resets `count` and bumps `gen`;
// the others poll `gen` with acquire loads and fence again before the block proceeds (count and gen live on
// different 128-byte lines, so polling does not queue behind the arrivals).
__device__ inline void grid_barrier(const GridSync &gs, Ctrl *c)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int nb = gridDim.x;
        const unsigned int g = ld_acquire(gs.gen);
        __threadfence();
        if (atomicAdd(gs.count, 1u) == nb - 1) {
            atomicExch(gs.count, 0u);
            __threadfence();
            atomicAdd(gs.gen, 1u);
        } else {
            long long n = 0;
            while (ld_acquire(gs.gen) == g) {
                if ((volatile uint32_t &)c->err & ERR_TIMEOUT) break;
                if (++n > BARRIER_SPIN_LIMIT) {
                    atomicOr(&c->err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
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
    __device__ inline Acc shfl_down(int o) const { Acc r; r.v = __shfl_down_sync(0xffffffffu, v, o); return r; }
    __device__ inline double value() const { return v; }
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
    __device__ inline double value() const { return (double)h + (double)l; }
};

// partial-sum storage per block and quantity
template <typename R> struct PartT;
template <> struct PartT<float> { typedef float2 T; };
template <> struct PartT<double> { typedef double T; };
__device__ inline void put_part(float2 *p, const Acc<float> &a) { *p = make_float2(a.h, a.l); }
__device__ inline void put_part(double *p, const Acc<double> &a) { *p = a.v; }
__device__ inline void get_part(const float2 *p, Acc<float> &a) { const float2 v = __ldcg(p); a.h = v.x; a.l = v.y; }
__device__ inline void get_part(const double *p, Acc<double> &a) { a.v = __ldcg(p); }

template <typename R> struct PShared {
    Acc<R> w[PB / 32][8];
    double res[8];
    R fmax_[PB / 32];
};

// Grid-wide sum of N per-thread accumulators; the result (double) is returned in every thread of every block.
// `part` holds N x gridDim.x partials.  Contains one grid barrier.
template <typename R, int N>
__device__ inline void grid_sum(Acc<R> (&a)[N], double (&out)[N], typename PartT<R>::T *part, PShared<R> &sh,
                                const GridSync &gs, Ctrl *c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        for (int o = 16; o > 0; o >>= 1) a[q].add(a[q].shfl_down(o));
        if (lane == 0) sh.w[warp][q] = a[q];
    }
    __syncthreads();
    if (threadIdx.x < N) {
        Acc<R> b;
        for (int w = 0; w < nw; ++w) b.add(sh.w[w][threadIdx.x]);
        put_part(part + threadIdx.x * gridDim.x + blockIdx.x, b);
    }
    grid_barrier(gs, c);
    // every block: sum the partials of quantity q in block order (thread t takes blocks t, t + PB, ...)
#pragma unroll
    for (int q = 0; q < N; ++q) {
        Acc<R> s;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            Acc<R> v;
            get_part(part + q * gridDim.x + b, v);
            s.add(v);
        }
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_down(o));
        if (lane == 0) sh.w[warp][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        Acc<R> b;
        for (int w = 0; w < nw; ++w) b.add(sh.w[w][threadIdx.x]);
        sh.res[threadIdx.x] = b.value();
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = sh.res[q];
    __syncthreads();
}

// Grid-wide sum of N accumulators and max of one non-negative value with a single barrier; the max travels in the
// (N)th partial slot (its head carries the value, its tail is zero).
template <typename R, int N>
__device__ inline void grid_sum_max(Acc<R> (&a)[N], R mx, double (&out)[N], R &mx_out, typename PartT<R>::T *part,
                                    PShared<R> &sh, const GridSync &gs, Ctrl *c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        for (int o = 16; o > 0; o >>= 1) a[q].add(a[q].shfl_down(o));
        if (lane == 0) sh.w[warp][q] = a[q];
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if (lane == 0) sh.fmax_[warp] = mx;
    __syncthreads();
    if (threadIdx.x < N) {
        Acc<R> b;
        for (int w = 0; w < nw; ++w) b.add(sh.w[w][threadIdx.x]);
        put_part(part + threadIdx.x * gridDim.x + blockIdx.x, b);
    } else if (threadIdx.x == N) {
        R m = R(0);
        for (int w = 0; w < nw; ++w) m = fmax(m, sh.fmax_[w]);
        Acc<R> b;
        b.add(m);
        put_part(part + N * gridDim.x + blockIdx.x, b);
    }
    grid_barrier(gs, c);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        Acc<R> s;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            Acc<R> v;
            get_part(part + q * gridDim.x + b, v);
            s.add(v);
        }
        for (int o = 16; o > 0; o >>= 1) s.add(s.shfl_down(o));
        if (lane == 0) sh.w[warp][q] = s;
    }
    R m = R(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        Acc<R> v;
        get_part(part + N * gridDim.x + b, v);
        m = fmax(m, (R)v.value());
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) sh.fmax_[warp] = m;
    __syncthreads();
    if (threadIdx.x < N) {
        Acc<R> b;
        for (int w = 0; w < nw; ++w) b.add(sh.w[w][threadIdx.x]);
        sh.res[threadIdx.x] = b.value();
    } else if (threadIdx.x == N) {
        R r = R(0);
        for (int w = 0; w < nw; ++w) r = fmax(r, sh.fmax_[w]);
        sh.res[N] = (double)r;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = sh.res[q];
    mx_out = (R)sh.res[N];
    __syncthreads();
}

// Grid-wide max of non-negative values of the element type (exact); one grid barrier.  `part` holds gridDim.x
// values of type R.
template <typename R>
__device__ inline R grid_max(R v, R *part, PShared<R> &sh, const GridSync &gs, Ctrl *c)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) sh.fmax_[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        R m = R(0);
        for (int w = 0; w < nw; ++w) m = fmax(m, sh.fmax_[w]);
        part[blockIdx.x] = m;
    }
    grid_barrier(gs, c);
    R m = R(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = fmax(m, __ldcg(part + b));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) sh.fmax_[warp] = m;
    __syncthreads();
    R r = R(0);
    for (int w = 0; w < nw; ++w) r = fmax(r, sh.fmax_[w]);
    __syncthreads();
    return r;
}

struct PersistArgs {
    int do_predict, k0, n_iters, do_finish;
    GridSync gs;
    void *part;            // reduction partials: 2 x 8 x gridDim.x of the partial type, then 2 x gridDim.x floats
    unsigned long long *stamps;   // profiling (null = off): globaltimer at the end of each phase, seen by block 0
    int *stamp_kind;              // the phase each stamp closes (K_* of sim.h order)
    int max_stamps;
};

__device__ inline unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

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

// ------------------------------------------------------------------------------------------------ the kernel

template <typename R>
__global__ void __launch_bounds__(PB) k_persistent(Dev<R> D, BPDev B, PersistArgs A)
{
    typedef typename V4<R>::T R4;
    typedef typename PartT<R>::T PT;
    __shared__ PShared<R> sh;
    Ctrl *c = D.ctrl;
    RedBufs rb;
    rb.base = A.part;
    rb.n = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    // state every block reads before anyone can change it
    int rebuild = (volatile int &)c->rebuild;
    const bool skip_step = (volatile uint32_t &)c->err != 0u;
    double gPg_prev = (volatile double &)c->gPg_prev;
    double dE0 = (volatile double &)c->dE0;
    int converged = (volatile int &)c->converged;
    const double disp_lim = 0.5 * D.pad_r * (1.0 - 1e-4);
    Stamper st{A.stamps, A.stamp_kind, A.max_stamps};
    grid_barrier(A.gs, c);
    st.mark(-1);

    // ---------------------------------------------------------------- a0: prediction and iteration-0 init
    if (A.do_predict) {
        R md = R(0);
        if (!skip_step) {
            for (int i = tid; i < D.nv; i += nthr) {
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
                init_vertex<R>(D, i, X, XT, 0);
                md = fmax(md, (R)disp2<R>(D, i, X));
            }
        }
        const R m = grid_max<R>(md, rb.max_region<PT, R>(), sh, A.gs, c);
        if (!skip_step && (double)m >= disp_lim * disp_lim) rebuild = 1;
        gPg_prev = 0.0;
        dE0 = 0.0;
        converged = 0;
        if (lead) {
            c->k = 0; c->n_rebuilds = 0; c->n_capped = 0; c->iters_done = 0; c->converged = 0;
            c->n_active = 0; c->dE0 = 0.0; c->gPg_prev = 0.0;
        }
        grid_barrier(A.gs, c);
        st.mark(0);   // K_PREDICT
    }

    for (int it = 0; it < A.n_iters; ++it) {
        const int k = A.k0 + it;
        const int par = k & 1;
        // ------------------------------------------------------------ a1: candidate build when needed
        if (rebuild) {
            if (lead) { c->n_cand = 0; c->n_rebuilds += 1; c->cell_bits = 0u; }
            grid_barrier(A.gs, c);
            st.mark(1);   // K_BP_BOXES (set-up)
            // boxes, bucket counts to zero, build positions
            const int nprim = B.nf + B.ne;
            for (int j = tid; j < max(max(nprim, B.nv), 2 * B.H); j += nthr) {
                if (j < 2 * B.H) B.cnt[j] = 0u;
                if (j < B.nv) { B.xb[j] = ldcg4(B.x + j); if (B.xbh) B.xbh[j] = ldcg4(B.xh + j); }
                if (j < nprim) {
                    int v[3];
                    int nvp;
                    if (j < B.nf) { const int4 t = B.tri[j]; v[0] = t.x; v[1] = t.y; v[2] = t.z; nvp = 3; }
                    else { const int4 e = B.edge[j - B.nf]; v[0] = e.x; v[1] = e.y; nvp = 2; }
                    float4 lo, hi;
                    box_of(B.x, v, nvp, B.infl, lo, hi);
                    B.blo[j] = lo;
                    B.bhi[j] = hi;
                    const float ext = fmaxf(__fsub_ru(hi.x, lo.x), fmaxf(__fsub_ru(hi.y, lo.y), __fsub_ru(hi.z, lo.z)));
                    atomicMax(&c->cell_bits, __float_as_uint(ext));
                }
            }
            grid_barrier(A.gs, c);
            st.mark(1);   // K_BP_BOXES
            const float s = cell_size(B);
            for (int j = tid; j < nprim; j += nthr)
                for_cells(B, __ldcg(B.blo + j), __ldcg(B.bhi + j), s, [&](int i, int jj, int kk) { atomicAdd(&B.cnt[prim_bucket(B, j, i, jj, kk)], 1u); });
            grid_barrier(A.gs, c);
            st.mark(2);   // K_BP_COUNT
            // block-local exclusive scans of 1024-bucket chunks (one warp per chunk)
            {
                const int nchunk = 2 * B.H / BP_SCAN_N;
                const int gw = tid >> 5, lane = threadIdx.x & 31, nwarps = nthr >> 5;
                for (int ch = gw; ch < nchunk; ch += nwarps) {
                    unsigned int run = 0;
                    for (int base = ch * BP_SCAN_N; base < (ch + 1) * BP_SCAN_N; base += 32) {
                        const unsigned int v = __ldcg(B.cnt + base + lane);
                        unsigned int inc = v;
                        for (int o = 1; o < 32; o <<= 1) {
                            const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
                            if (lane >= o) inc += n;
                        }
                        B.off[base + lane] = run + inc - v;
                        B.cnt[base + lane] = 0u;
                        run += __shfl_sync(0xffffffffu, inc, 31);
                    }
                    if (lane == 0) B.boff[ch] = run;
                }
            }
            grid_barrier(A.gs, c);
            st.mark(3);   // K_BP_SCAN
            // chunk offsets: every block scans the chunk totals into shared memory
            __shared__ unsigned int choff[1024];
            {
                const int nchunk = 2 * B.H / BP_SCAN_N;
                if (threadIdx.x == 0) {
                    unsigned int run = 0;
                    for (int ch = 0; ch < nchunk && ch < 1024; ++ch) { choff[ch] = run; run += __ldcg(&B.boff[ch]); }
                }
                __syncthreads();
            }
            for (int j = tid; j < nprim; j += nthr) {
                const int prim = j < B.nf ? j : -1 - (j - B.nf);
                const float4 lo = __ldcg(B.blo + j), hi = __ldcg(B.bhi + j);
                for_cells(B, lo, hi, s, [&](int i, int jj, int kk) {
                    const unsigned int b = prim_bucket(B, j, i, jj, kk);
                    const unsigned int slot = choff[b / BP_SCAN_N] + __ldcg(B.off + b) + atomicAdd(&B.cnt[b], 1u);
                    if (slot >= (unsigned int)B.ecap) { atomicOr(&c->err, ERR_RANGE); return; }
                    B.ekey[slot] = cell_key(i, jj, kk);
                    B.eprim[slot] = prim;
                    B.eblo[slot] = lo;
                    B.ebhi[slot] = hi;
                });
            }
            grid_barrier(A.gs, c);
            st.mark(4);   // K_BP_FILL
            // queries: one warp per query primitive (offsets of the scan stored for bp_query's layout)
            if (blockIdx.x == 0) {
                const int nchunk = 2 * B.H / BP_SCAN_N;
                for (int ch = threadIdx.x; ch < nchunk && ch < 1024; ch += blockDim.x) B.boff[ch] = choff[ch];
            }
            grid_barrier(A.gs, c);
            st.mark(4);   // K_BP_FILL (offsets)
            for (int w = tid >> 5; w < B.ns + B.ne; w += nthr >> 5) bp_query_one(B, w, s);
            grid_barrier(A.gs, c);
            st.mark(5);   // K_BP_QUERY
            rebuild = 0;
        }
        // ------------------------------------------------------------ a2-a3: gradient + diagonal
        if (lead) {
            c->rebuild = 0;
            if (c->n_cand > D.cand_cap) flag_error(c, ERR_CAPACITY);
        }
        for (int e = tid; e < D.nt; e += nthr) tet_grad<R>(D, e, par);
        {
            const int nc = min((volatile int &)c->n_cand, D.cand_cap);
            for (int ci = tid; ci < nc; ci += nthr) pair_grad<R>(D, ci, par);
        }
        grid_barrier(A.gs, c);
        st.mark(6);   // K_GRAD
        if (D.segmented) {
            const int n4 = 4 * D.nt;
            for (int i = tid; i < D.nv; i += nthr) {
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
            grid_barrier(A.gs, c);
            st.mark(7);   // K_GATHER
        }
        // ------------------------------------------------------------ a4: beta
        double beta = 0.0;
        int restarted = 0;
        {
            Acc<R> s5[5];
            for (int i = tid; i < D.nv; i += nthr) {
                const R4 G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i), G0 = ldcg4(D.g[par ^ 1] + i), P0 = ldcg4(D.p + i);
                if (Dg.w > R(0)) {
                    const R gv[3] = {G.x, G.y, G.z}, dv[3] = {Dg.x, Dg.y, Dg.z}, g0[3] = {G0.x, G0.y, G0.z}, p0[3] = {P0.x, P0.y, P0.z};
                    R t5[5] = {0, 0, 0, 0, 0};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R P = precond<R>(dv[a], Dg.w);
                        const R g = gv[a], y = g - g0[a];
                        if (D.beta_rule == 0) {
                            t5[0] += g * P * y; t5[1] += g * P * g; t5[2] += g * p0[a];
                        } else {
                            t5[0] += g * P * y; t5[1] += y * P * y; t5[2] += y * p0[a]; t5[3] += p0[a] * g; t5[4] += g * P * g;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 5; ++q) s5[q].add(t5[q]);
                }
            }
            double t[5];
            grid_sum<R, 5>(s5, t, rb.sum_region<PT>(), sh, A.gs, c);
            st.mark(8);   // K_DOTS
            double gPg, gp_new;
            if (D.beta_rule == 0) {
                gPg = t[1];
                if (k > 0) { beta = gPg_prev > 0.0 ? t[0] / gPg_prev : 0.0; if (beta < 0.0) beta = 0.0; }
                gp_new = -gPg + beta * t[2];
            } else {
                gPg = t[4];
                if (k > 0) beta = fabs(t[2]) < 1e-30 ? 0.0 : t[0] / t[2] - (t[1] / t[2]) * (t[3] / t[2]);
                gp_new = -gPg + beta * t[3];
            }
            if (gp_new >= 0.0 && beta != 0.0) { beta = 0.0; restarted = 1; }
            gPg_prev = gPg;
        }
        // ------------------------------------------------------------ a5: direction
        double gp, pHp_vert, pmax;
        {
            Acc<R> s2[2];
            R pm = R(0);
            const R b = R(beta);
            for (int i = tid; i < D.nv; i += nthr) {
                const R4 G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i);
                R4 Pn = mk4<R>(R(0), R(0), R(0), R(0));
                if (Dg.w > R(0)) {
                    const R4 P0 = ldcg4(D.p + i);
                    if (beta != 0.0) {
                        Pn.x = -precond<R>(Dg.x, Dg.w) * G.x + b * P0.x;
                        Pn.y = -precond<R>(Dg.y, Dg.w) * G.y + b * P0.y;
                        Pn.z = -precond<R>(Dg.z, Dg.w) * G.z + b * P0.z;
                    } else {
                        Pn.x = -precond<R>(Dg.x, Dg.w) * G.x;
                        Pn.y = -precond<R>(Dg.y, Dg.w) * G.y;
                        Pn.z = -precond<R>(Dg.z, Dg.w) * G.z;
                    }
                    const R px = Pn.x, py = Pn.y, pz = Pn.z;
                    s2[0].add(G.x * px + G.y * py + G.z * pz);
                    R mp = Dg.w * (px * px + py * py + pz * pz);
                    if (D.has_plane && G.w != R(0)) {
                        const R np = R(D.pn[0]) * px + R(D.pn[1]) * py + R(D.pn[2]) * pz;
                        mp += G.w * np * np;
                    }
                    s2[1].add(mp);
                    const R pn = D.pnorm == 0 ? sqrt(px * px + py * py + pz * pz) : fmax(fabs(px), fmax(fabs(py), fabs(pz)));
                    pm = fmax(pm, pn);
                }
                D.p[i] = Pn;
            }
            double t[2];
            R pmr;
            grid_sum_max<R, 2>(s2, pm, t, pmr, rb.sum_region<PT>(), sh, A.gs, c);
            gp = t[0];
            pHp_vert = t[1];
            pmax = (double)pmr;
            st.mark(9);   // K_DIR
        }
        // ------------------------------------------------------------ a6-a7: p^T H p and the step
        double alpha;
        {
            Acc<R> s1[1];
            for (int e = tid; e < D.nt; e += nthr) s1[0].add(tet_pHp<R>(D, e));
            const int na = (volatile int &)c->n_active;
            for (int kk = tid; kk < na; kk += nthr) s1[0].add_d(pair_pHp<R>(D, kk));
            double t[1];
            grid_sum<R, 1>(s1, t, rb.sum_region<PT>(), sh, A.gs, c);
            st.mark(10);  // K_PHP
            const double pHp = t[0] + pHp_vert;
            const double au = pmax > 0.0 ? D.dhat / (2.0 * pmax) : 0.0;
            const double ab = -gp / pHp;
            int capped;
            if (!(pHp > 0.0) || !isfinite(ab)) { alpha = au; capped = 1; }
            else if (ab < au) { alpha = ab; capped = 0; }
            else { alpha = au; capped = 1; }
            const double dE = -alpha * gp - 0.5 * alpha * alpha * pHp;
            if (!isfinite(alpha) || !isfinite(gp)) { if (lead) flag_error(c, ERR_NONFINITE); alpha = 0.0; }
            if ((volatile uint32_t &)c->err != 0u || converged) alpha = 0.0;
            if (lead) {
                c->beta = beta; c->restarted = restarted; c->gp = gp; c->pmax = pmax; c->pHp_vert = pHp_vert;
                c->pHp = pHp; c->alpha_bar = ab; c->alpha_up = au; c->alpha = alpha; c->dE = dE; c->capped = capped;
                c->n_active_last = na;
                c->gPg_prev = gPg_prev;
                if (!converged && (volatile uint32_t &)c->err == 0u) {
                    if (k == 0) c->dE0 = dE;
                    c->n_capped += capped;
                    c->iters_done = k + 1;
                    if (D.trace && k < D.iters) {
                        double *tr = D.trace + (size_t)k * TRACE_COLS;
                        tr[0] = beta; tr[1] = gp; tr[2] = pHp; tr[3] = pmax; tr[4] = alpha; tr[5] = dE;
                        tr[6] = na; tr[7] = capped;
                    }
                }
                c->k = k + 1;
            }
            if (!converged && (volatile uint32_t &)c->err == 0u) {
                if (k == 0) dE0 = dE;
                if (D.eps > 0.0 && dE < D.eps * dE0) converged = 1;
            }
            if (lead) { c->dE0 = dE0; c->converged = converged; }
        }
        // ------------------------------------------------------------ a8: update
        {
            R md = R(0);
            for (int i = tid; i < D.nv; i += nthr) {
                double4_32a X = ldcg4(D.x + i);
                const R4 P = ldcg4(D.p + i);
                X.x += alpha * double(P.x); X.y += alpha * double(P.y); X.z += alpha * double(P.z);
                put_x<R>(D, i, X);
                init_vertex<R>(D, i, X, ldcg4(D.xtil + i), par ^ 1);
                md = fmax(md, (R)disp2<R>(D, i, X));
            }
            if (lead) c->n_active = 0;
            const R m = grid_max<R>(md, rb.max_region<PT, R>(), sh, A.gs, c);
            st.mark(11);  // K_UPDATE
            if ((double)m >= disp_lim * disp_lim) rebuild = 1;
        }
    }
    if (lead && rebuild) c->rebuild = 1;

    // ---------------------------------------------------------------- velocity update
    if (A.do_finish) {
        grid_barrier(A.gs, c);
        const bool bad = (volatile uint32_t &)c->err != 0u;
        for (int i = tid; i < D.nv; i += nthr) {
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
        grid_barrier(A.gs, c);
        st.mark(12);  // K_FINISH
    }
}

} // namespace pncg
