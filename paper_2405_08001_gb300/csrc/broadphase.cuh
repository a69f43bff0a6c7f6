// Contact-candidate pass (spatial hash over surface primitives; the paper uses grid spatial hashing for its
// broad phase, Sec. 6).  Candidates are all surface point-triangle pairs (point not in the triangle) and edge-edge
// pairs (no shared vertex) whose boxes, inflated by dhat + r, overlap at the positions of the build; pairs of one
// object closer than the exclusion radius at rest (Sec. 5.1) are dropped.  Since d changes by at most twice the
// largest vertex displacement, every pair with d < dhat is a candidate until some vertex has moved r/2.
//
// The five kernels run only when Ctrl::rebuild is set (they return at once otherwise):
//   bp_boxes  : inflated float boxes (rounded outwards), largest extent -> cell size, zero bucket counts, x_b = x
//   bp_count  : entries per hash bucket (each primitive covers at most 2 cells per axis); triangles and edges
//               have separate tables (buckets [0, H) and [H, 2H)) so each query scans one kind only
//   bp_scan   : exclusive scan of the counts (block-local scans + the last block scans the block sums)
//   bp_fill   : entries (cell key, a copy of the primitive's box with the primitive and its scene, the primitive's
//               vertices relative to the cell's corner) in bucket order, and each bucket's global first entry
//   bp_query  : batches of surface vertices (PT) or edges (EE), one warp each: exact cell-key match, box, order and
//               scene tests on every entry of the batch's buckets, then the distance at the build positions for
//               the entries that pass: only pairs with d < (dhat + r)(1 + 1e-3) become candidates
#pragma once

#include "common.cuh"
#include "geometry.cuh"

namespace pncg {

constexpr int BP_SCAN_T = 256;                 // threads per scan block
constexpr int BP_SCAN_N = 4 * BP_SCAN_T;       // buckets per scan block
constexpr int BP_B = 256;                      // threads per block, other broad-phase kernels
constexpr int BP_MAX_CHUNKS = 4096;            // scan chunks of the persistent form (chunk totals in shared memory)
constexpr int CELL_BIAS = 1 << 20;

struct BPDev {
    int nv, ns, nf, ne, H;
    const double4_32a *x;
    double4_32a *xb;
    const float4 *xh;       // FP32 form: float copy of x (null in the FP64 form)
    float4 *xbh;            // FP32 form: xh at the build
    const int *svert;       // [ns]
    const int4 *tri;        // [nf] (v0, v1, v2, object)
    const int4 *edge;       // [ne] (v0, v1, object, 0)
    const int *obj;         // [nv]
    float4 *blo, *bhi;      // [nf + ne] inflated boxes, triangles first
    unsigned int *cnt, *off, *boff;
    unsigned int *goff;     // [2H] global first entry of each bucket (written with the entries, read by queries)
    unsigned int *ctot;     // persistent form: [2H >> cshift_p] entries per scan chunk
    int cshift_p;           // persistent form: log2 of the buckets per scan chunk
    const int *vscene;      // batching: scene of each vertex (pairs of two scenes are never candidates); or null
    unsigned long long *ekey;
    float4 *eblo, *ebhi;    // the entry's primitive box (streamed with the key instead of gathered); eblo.w holds
                            // the primitive (triangle f or -1 - edge) and ebhi.w its scene, as int bits
    float4 *ev;             // [3][ecap] the primitive's vertices relative to the entry's cell corner (w: the
                            // vertex index as int bits); edges use the first two rows
    int ecap;               // entry capacity (8 per primitive)
    int4 *cand;
    int cap;
    const unsigned long long *excl;
    int nexcl;
    double infl;            // dhat + r
    float thr;              // (dhat + r)(1 + 1e-3): exact-distance threshold of a candidate
    Ctrl *ctrl;
};

__device__ inline unsigned int cell_hash(int ix, int iy, int iz, int H)
{
    return ((unsigned int)ix * 73856093u ^ (unsigned int)iy * 19349663u ^ (unsigned int)iz * 83492791u) & (unsigned int)(H - 1);
}
// bucket of primitive j's cell: triangles in [0, H), edges in [H, 2H)
__device__ inline unsigned int prim_bucket(const BPDev &B, int j, int ix, int iy, int iz)
{
    return cell_hash(ix, iy, iz, B.H) + (j < B.nf ? 0u : (unsigned int)B.H);
}
__device__ inline unsigned long long cell_key(int ix, int iy, int iz)
{
    return ((unsigned long long)(ix + CELL_BIAS) << 42) | ((unsigned long long)(iy + CELL_BIAS) << 21) |
           (unsigned long long)(iz + CELL_BIAS);
}
// the hash grid: cell size s and its reciprocal; every cell index of a build comes from floor(q * inv), which is
// monotone in q, so a point inside a box lies in one of the box's cells
struct CellGrid { float s, inv; };
__device__ inline CellGrid grid_of(float s) { return {s, 1.0f / s}; }

__device__ inline bool cell_of(float q, const CellGrid &g, int &i)
{
    const float f = floorf(q * g.inv);
    if (!(fabsf(f) < float(CELL_BIAS - 2))) return false;
    i = (int)f;
    return true;
}

// hash cell size: the largest inflated box extent of the build, with a margin so that rounding in q / s can never
// make a box span three cells along an axis
__device__ inline float cell_size(const BPDev &B) { return __uint_as_float(B.ctrl->cell_bits) * 1.0001f; }

__device__ inline void box_of(const double4_32a *x, const int *v, int n, double infl, float4 &lo, float4 &hi)
{
    double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
    for (int k = 0; k < n; ++k) {
        const double4_32a X = ldcg4(x + v[k]);
        l[0] = fmin(l[0], X.x); l[1] = fmin(l[1], X.y); l[2] = fmin(l[2], X.z);
        h[0] = fmax(h[0], X.x); h[1] = fmax(h[1], X.y); h[2] = fmax(h[2], X.z);
    }
    lo = make_float4(__double2float_rd(l[0] - infl), __double2float_rd(l[1] - infl), __double2float_rd(l[2] - infl), 0.f);
    hi = make_float4(__double2float_ru(h[0] + infl), __double2float_ru(h[1] + infl), __double2float_ru(h[2] + infl), 0.f);
}

// a position relative to the lower corner of hash cell (ix, iy, iz) of size s, formed in double and rounded once to
// float: positions within a cell or two of the corner keep ~1e-7 s in float wherever the scene sits
__device__ inline float4 rel_corner(const double4_32a &X, int ix, int iy, int iz, float s, int w)
{
    const double sd = s;
    return make_float4((float)(X.x - ix * sd), (float)(X.y - iy * sd), (float)(X.z - iz * sd), __int_as_float(w));
}

__device__ inline void prim_verts(const BPDev &B, int j, int v[3], int &nvp)
{
    if (j < B.nf) { const int4 t = B.tri[j]; v[0] = t.x; v[1] = t.y; v[2] = t.z; nvp = 3; }
    else { const int4 e = B.edge[j - B.nf]; v[0] = e.x; v[1] = e.y; v[2] = e.y; nvp = 2; }
}

// cells spanned by a box: false if a coordinate is out of the hash grid's range
__device__ inline bool box_cells(float4 lo, float4 hi, const CellGrid &g, int l[3], int h[3])
{
    return cell_of(lo.x, g, l[0]) && cell_of(lo.y, g, l[1]) && cell_of(lo.z, g, l[2]) && cell_of(hi.x, g, h[0]) &&
           cell_of(hi.y, g, h[1]) && cell_of(hi.z, g, h[2]);
}

// Writes primitive j's entries, one per cell of its box: the cell key, the box with the primitive and its scene in
// the w components, and the vertices relative to the entry's cell corner (formed once in double against the box's
// lowest cell, then shifted by whole cells in float).  slot_of(b) reserves a slot of bucket b.
template <typename F> __device__ inline void fill_prim(const BPDev &B, int j, const CellGrid &g, F slot_of)
{
    const float s = g.s;
    float4 lo = __ldcg(B.blo + j), hi = __ldcg(B.bhi + j);
    int l[3], h[3];
    if (!box_cells(lo, hi, g, l, h)) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
    int v[3], nvp;
    prim_verts(B, j, v, nvp);
    float4 r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = rel_corner(ldcg4(B.x + v[q]), l[0], l[1], l[2], s, v[q]);
    lo.w = __int_as_float(j < B.nf ? j : -1 - (j - B.nf));
    hi.w = __int_as_float(B.vscene ? B.vscene[v[0]] : 0);
    for (int i = l[0]; i <= h[0]; ++i)
        for (int jj = l[1]; jj <= h[1]; ++jj)
            for (int kk = l[2]; kk <= h[2]; ++kk) {
                const unsigned int slot = slot_of(prim_bucket(B, j, i, jj, kk));
                if (slot >= (unsigned int)B.ecap) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
                B.ekey[slot] = cell_key(i, jj, kk);
                B.eblo[slot] = lo;
                B.ebhi[slot] = hi;
                const float ox = (float)(i - l[0]) * s, oy = (float)(jj - l[1]) * s, oz = (float)(kk - l[2]) * s;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    if (q < nvp) B.ev[(size_t)q * B.ecap + slot] = make_float4(r[q].x - ox, r[q].y - oy, r[q].z - oz, r[q].w);
            }
}

static __global__ void __launch_bounds__(BP_B) bp_boxes(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const int n = max(max(B.nf + B.ne, B.nv), 2 * B.H);
    const int stride = gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) { B.ctrl->n_cand = 0; B.ctrl->n_rebuilds += 1; }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        if (j < 2 * B.H) B.cnt[j] = 0u;
        if (j < B.nv) {
            B.xb[j] = B.x[j];
            if (B.xbh) B.xbh[j] = B.xh[j];
        }
        if (j < B.nf + B.ne) {
            int v[3];
            int nvp;
            if (j < B.nf) { const int4 t = B.tri[j]; v[0] = t.x; v[1] = t.y; v[2] = t.z; nvp = 3; }
            else { const int4 e = B.edge[j - B.nf]; v[0] = e.x; v[1] = e.y; nvp = 2; }
            float4 lo, hi;
            box_of(B.x, v, nvp, B.infl, lo, hi);
            B.blo[j] = lo;
            B.bhi[j] = hi;
            float ext = fmaxf(__fsub_ru(hi.x, lo.x), fmaxf(__fsub_ru(hi.y, lo.y), __fsub_ru(hi.z, lo.z)));
            atomicMax(&B.ctrl->cell_bits, __float_as_uint(ext));
        }
    }
}

// visits the (at most 8) cells covered by [lo, hi]; returns false (and flags) on a coordinate out of range
template <typename F>
__device__ inline void for_cells(const BPDev &B, float4 lo, float4 hi, const CellGrid &g, F f)
{
    int l[3], h[3];
    if (!box_cells(lo, hi, g, l, h)) {
        atomicOr(&B.ctrl->err, ERR_RANGE);
        return;
    }
    for (int i = l[0]; i <= h[0]; ++i)
        for (int j = l[1]; j <= h[1]; ++j)
            for (int k = l[2]; k <= h[2]; ++k) f(i, j, k);
}

static __global__ void __launch_bounds__(BP_B) bp_count(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const CellGrid g = grid_of(cell_size(B));
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.nf + B.ne) return;
    for_cells(B, B.blo[j], B.bhi[j], g, [&](int i, int jj, int k) { atomicAdd(&B.cnt[prim_bucket(B, j, i, jj, k)], 1u); });
}

static __global__ void __launch_bounds__(BP_SCAN_T) bp_scan(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    __shared__ unsigned int wsum[BP_SCAN_T / 32];
    __shared__ bool last;
    const int base = blockIdx.x * BP_SCAN_N + 4 * threadIdx.x;
    uint4 c = reinterpret_cast<const uint4 *>(B.cnt)[base / 4];
    unsigned int tot = c.x + c.y + c.z + c.w;
    // inclusive warp scan of per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned int inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    unsigned int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    const unsigned int ex = wpre + inc - tot;
    uint4 o4 = make_uint4(ex, ex + c.x, ex + c.x + c.y, ex + c.x + c.y + c.z);
    reinterpret_cast<uint4 *>(B.off)[base / 4] = o4;
    reinterpret_cast<uint4 *>(B.cnt)[base / 4] = make_uint4(0u, 0u, 0u, 0u);   // becomes the fill cursor
    if (threadIdx.x == BP_SCAN_T - 1) {
        B.boff[blockIdx.x] = ex + tot;                                         // block total
        __threadfence();
        unsigned int t = atomicAdd(&B.ctrl->ticket[TK_SCAN], 1u);
        last = (t == gridDim.x - 1);
        if (last) B.ctrl->ticket[TK_SCAN] = 0u;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        unsigned int run = 0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            unsigned int v = __ldcg(&B.boff[b]);
            B.boff[b] = run;
            run += v;
        }
    }
}

static __global__ void __launch_bounds__(BP_B) bp_fill(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const CellGrid g = grid_of(cell_size(B));
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < 2 * B.H; b += gridDim.x * blockDim.x)
        B.goff[b] = B.boff[b / BP_SCAN_N] + B.off[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.nf + B.ne) return;
    fill_prim(B, j, g, [&](unsigned int b) { return B.boff[b / BP_SCAN_N] + B.off[b] + atomicAdd(&B.cnt[b], 1u); });
}

__device__ inline bool is_excluded(const BPDev &B, unsigned long long key)
{
    int lo = 0, hi = B.nexcl;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (B.excl[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo < B.nexcl && B.excl[lo] == key;
}

// ---------------------------------------------------------------------------------------------------- queries
// A warp takes a batch of BPQ_QB queries of one kind (points, or edges) and scans the entries of all their buckets
// as one list, 64 per round (two per lane, loaded together), so the batch pays the latency of its headers once and
// no lane idles at the end of a short bucket.  The batch's per-query data (cells and their keys, first entries,
// prefix counts) sit in the warp's shared area.  A round applies only the cheap tests (cell key, box, order,
// scene) to the entry's key and box; the entries that pass queue up in shared memory and get the exact distance 32
// at a time, with every lane busy.  Found pairs collect in shared memory and are appended with one atomic per 32.
constexpr int BPQ_QB = 8;       // most queries of a warp batch (lanes 0..7 form the headers)
constexpr int BPQ_QE = 6;       // edges per batch (an edge's box covers about twice the cells of a point)
constexpr int BPQ_QP = 8;       // points per batch
constexpr int BPQ_PEND = 64;    // entries past the cheap tests, awaiting the distance
constexpr int BPQ_OUT = 64;     // found pairs held before an append

struct BPQWarp {
    unsigned long long ckey[BPQ_QB][8];   // key of each cell of each query (a point has one)
    unsigned int cinc[BPQ_QB][8];   // edge: inclusive prefix over its cells of their entry counts
    unsigned int cst[BPQ_QB][8];    // first entry of each cell
    float4 qa[BPQ_QB];              // point: relative to its cell's corner (w: vertex); edge: first end relative to
                                    // the corner of its box's lowest cell (w: its vertex)
    float4 qb[BPQ_QB];              // point: float position; edge: second end as qa
    float4 lo[BPQ_QB], hi[BPQ_QB];  // edge: its box
    int4 aux[BPQ_QB];               // x: point index j or edge index a; y: scene; z: object; w: edge nx | ny << 2
    unsigned int qinc[BPQ_QB];      // inclusive prefix over the batch of the queries' entry counts
    uint2 pend[BPQ_PEND];           // (entry, query | cell << 3)
    int4 out[BPQ_OUT];
};

__device__ inline int bpq_edge_batches(const BPDev &B) { return (B.ne + BPQ_QE - 1) / BPQ_QE; }
__device__ inline int bpq_batches(const BPDev &B) { return bpq_edge_batches(B) + (B.ns + BPQ_QP - 1) / BPQ_QP; }

__device__ inline unsigned int lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// appends the warp's n held pairs (n warp-uniform; all lanes call)
__device__ inline void bpq_flush(const BPDev &B, BPQWarp &W, int &n)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (n == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&B.ctrl->n_cand, n);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < n; i += 32)
        if (base + i < B.cap) B.cand[base + i] = W.out[i];
    __syncwarp();
    n = 0;
}

// holds the lanes' found pairs (all lanes call)
__device__ inline void bpq_emit(const BPDev &B, BPQWarp &W, int &n, bool found, const int4 &cnd)
{
    const unsigned int m = __ballot_sync(0xffffffffu, found);
    if (!m) return;
    if (found) W.out[n + __popc(m & lanemask_lt())] = cnd;
    n += __popc(m);
    if (n > BPQ_OUT - 32) bpq_flush(B, W, n);
}

// queues the lanes' entries that passed the cheap tests (all lanes call)
__device__ inline void bpq_push(BPQWarp &W, int &np, bool pass, unsigned int q, unsigned int tc)
{
    const unsigned int m = __ballot_sync(0xffffffffu, pass);
    if (pass) W.pend[np + __popc(m & lanemask_lt())] = make_uint2(q, tc);
    np += __popc(m);
}

// drops the first 32 queued entries after their distances (np >= 32 on entry)
__device__ inline void bpq_shift(BPQWarp &W, int &np)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    uint2 v = make_uint2(0u, 0u);
    if (lane < np - 32) v = W.pend[32 + lane];
    __syncwarp();
    if (lane < np - 32) W.pend[lane] = v;
    __syncwarp();
    np -= 32;
}

__device__ inline v3<float> f3sub(const float4 &a, const float4 &b) { return mkv(a.x - b.x, a.y - b.y, a.z - b.z); }

// the batch's prefix counts: lane t < BPQ_QB brings its query's count; returns the batch total and leaves every
// lane the first BPQ_QB - 1 prefixes
__device__ inline unsigned int bpq_prefix(BPQWarp &W, unsigned int tot, unsigned int (&qi)[BPQ_QB - 1])
{
    const int lane = threadIdx.x & 31;
    unsigned int inc = tot;
#pragma unroll
    for (int o = 1; o < BPQ_QB; o <<= 1) {
        const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane < BPQ_QB) W.qinc[lane] = inc;
#pragma unroll
    for (int q = 0; q < BPQ_QB - 1; ++q) qi[q] = __shfl_sync(0xffffffffu, inc, q);
    __syncwarp();
    return __shfl_sync(0xffffffffu, inc, BPQ_QB - 1);
}

// the query owning item it of the batch, and the item's index within it
__device__ inline int bpq_owner(const BPQWarp &W, const unsigned int (&qi)[BPQ_QB - 1], unsigned int it, unsigned int &r)
{
    int t = 0;
#pragma unroll
    for (int q = 0; q < BPQ_QB - 1; ++q) t += qi[q] <= it ? 1 : 0;
    r = it - (t ? W.qinc[t - 1] : 0u);
    return t;
}

// offset of cell c among the cells of an edge's box (nx, ny packed in w)
__device__ inline void cell_offset(int w, int c, int &dx, int &dy, int &dz)
{
    const int nx = w & 3, ny = (w >> 2) & 3;
    dx = nx == 2 ? (c & 1) : 0;
    const int c1 = nx == 2 ? (c >> 1) : c;
    dy = ny == 2 ? (c1 & 1) : 0;
    dz = ny == 2 ? (c1 >> 1) : c1;
}

// ---- point-triangle

// cheap tests of item it of a point batch: the entry is of the point's cell, its box holds the point, same scene
__device__ inline bool pt_filter(const BPDev &B, const BPQWarp &W, const unsigned int (&qi)[BPQ_QB - 1], unsigned int it,
                                 unsigned int total, unsigned int &q, unsigned int &t)
{
    if (it >= total) return false;
    unsigned int r;
    t = bpq_owner(W, qi, it, r);
    q = W.cst[t][0] + r;
    const unsigned long long ek = __ldcg(B.ekey + q);
    const float4 lo = __ldcg(B.eblo + q), hi = __ldcg(B.ebhi + q);
    const float4 p = W.qb[t];
    return ek == W.ckey[t][0] && !(p.x < lo.x || p.x > hi.x || p.y < lo.y || p.y > hi.y || p.z < lo.z || p.z > hi.z) &&
           __float_as_int(hi.w) == W.aux[t].y;
}

// exact tests of the first n queued point-triangle entries (all lanes call)
__device__ inline void pt_exact(const BPDev &B, BPQWarp &W, int n, float thr, int &nout)
{
    const int lane = threadIdx.x & 31;
    bool found = false;
    int4 cnd = make_int4(0, 0, 0, 0);
    if (lane < n) do {
        const uint2 pd = W.pend[lane];
        const unsigned int q = pd.x;
        const int t = pd.y & 7;
        const float4 t0 = __ldcg(B.ev + q), t1 = __ldcg(B.ev + B.ecap + q), t2 = __ldcg(B.ev + 2 * (size_t)B.ecap + q);
        const float4 qa = W.qa[t];
        const int v = __float_as_int(qa.w);
        const int a0 = __float_as_int(t0.w), a1 = __float_as_int(t1.w), a2 = __float_as_int(t2.w);
        if (a0 == v || a1 == v || a2 == v) break;
        if (B.nexcl) {
            const int f = __float_as_int(__ldcg(B.eblo + q).w);
            const int4 ax = W.aux[t];
            if (B.tri[f].w == ax.z && is_excluded(B, ((unsigned long long)ax.x << 31) | (unsigned long long)f)) break;
        }
        float cc[4];
        v3<float> tv;
        const float d = pt_coeffs<float>(f3sub(qa, t0), f3sub(t1, t0), f3sub(t2, t0), cc, tv);
        if (!(d < thr)) break;
        found = true;
        cnd = make_int4(v, a0, a1, a2);
    } while (false);
    bpq_emit(B, W, nout, found, cnd);
}

// Point-triangle batch b of nb: surface points b, b + nb, b + 2 nb, ... (strided, so that a batch mixes crowded
// and sparse parts of the surface), each against the triangle table bucket of its cell.
__device__ inline void bpq_points(const BPDev &B, int b, int nb, const CellGrid &g, float thr, BPQWarp &W)
{
    const int lane = threadIdx.x & 31;
    unsigned int tot = 0;
    if (lane < BPQ_QP && b + lane * nb < B.ns) {
        const int j = b + lane * nb;
        const int v = B.svert[j];
        const double4_32a X = ldcg4(B.x + v);
        const float qx = (float)X.x, qy = (float)X.y, qz = (float)X.z;
        int ix = 0, iy = 0, iz = 0;
        if (!cell_of(qx, g, ix) || !cell_of(qy, g, iy) || !cell_of(qz, g, iz)) {
            atomicOr(&B.ctrl->err, ERR_RANGE);
        } else {
            const unsigned int b = cell_hash(ix, iy, iz, B.H);
            const unsigned int st = __ldcg(B.goff + b), len = __ldcg(B.cnt + b);
            tot = st < (unsigned int)B.ecap ? min(len, (unsigned int)B.ecap - st) : 0u;   // a fill overflow is flagged
            W.cst[lane][0] = st;
        }
        W.ckey[lane][0] = cell_key(ix, iy, iz);
        W.qa[lane] = rel_corner(X, ix, iy, iz, g.s, v);
        W.qb[lane] = make_float4(qx, qy, qz, 0.0f);
        W.aux[lane] = make_int4(j, B.vscene ? B.vscene[v] : 0, B.obj[v], 0);
    }
    unsigned int qi[BPQ_QB - 1];
    const unsigned int total = bpq_prefix(W, tot, qi);
    int np = 0, nout = 0;
    for (unsigned int base = 0; base < total; base += 64) {
        unsigned int q0 = 0, t0 = 0, q1 = 0, t1 = 0;
        const bool p0 = pt_filter(B, W, qi, base + lane, total, q0, t0);
        const bool p1 = pt_filter(B, W, qi, base + 32 + lane, total, q1, t1);
        bpq_push(W, np, p0, q0, t0);
        if (np >= 32) { __syncwarp(); pt_exact(B, W, 32, thr, nout); bpq_shift(W, np); }
        bpq_push(W, np, p1, q1, t1);
        if (np >= 32) { __syncwarp(); pt_exact(B, W, 32, thr, nout); bpq_shift(W, np); }
    }
    __syncwarp();
    if (np) pt_exact(B, W, np, thr, nout);
    bpq_flush(B, W, nout);
}

// ---- edge-edge

// cheap tests of item it of an edge batch: the entry is of its cell, numbered above the query edge, of the same
// scene, its box meets the query's, and the cell holds the lower corner of the two boxes' intersection
__device__ inline bool ee_filter(const BPDev &B, const BPQWarp &W, const unsigned int (&qi)[BPQ_QB - 1], unsigned int it,
                                 unsigned int total, const CellGrid &g, unsigned int &q, unsigned int &tc)
{
    if (it >= total) return false;
    unsigned int r;
    const int t = bpq_owner(W, qi, it, r);
    const uint4 ci0 = *reinterpret_cast<const uint4 *>(&W.cinc[t][0]);
    const uint4 ci1 = *reinterpret_cast<const uint4 *>(&W.cinc[t][4]);
    const int c = (ci0.x <= r) + (ci0.y <= r) + (ci0.z <= r) + (ci0.w <= r) + (ci1.x <= r) + (ci1.y <= r) + (ci1.z <= r);
    q = W.cst[t][c] + r - (c ? W.cinc[t][c - 1] : 0u);
    tc = (unsigned int)t | (unsigned int)c << 3;
    const unsigned long long ek = __ldcg(B.ekey + q);
    const float4 ilo = __ldcg(B.eblo + q), ihi = __ldcg(B.ebhi + q);
    if (ek != W.ckey[t][c]) return false;
    const int4 ax = W.aux[t];
    if (-1 - __float_as_int(ilo.w) <= ax.x || __float_as_int(ihi.w) != ax.y) return false;
    const float4 lo = W.lo[t], hi = W.hi[t];
    if (lo.x > ihi.x || hi.x < ilo.x || lo.y > ihi.y || hi.y < ilo.y || lo.z > ihi.z || hi.z < ilo.z) return false;
    int kx, ky, kz;
    cell_of(fmaxf(lo.x, ilo.x), g, kx);
    cell_of(fmaxf(lo.y, ilo.y), g, ky);
    cell_of(fmaxf(lo.z, ilo.z), g, kz);
    return cell_key(kx, ky, kz) == ek;
}

// exact tests of the first n queued edge-edge entries (all lanes call)
__device__ inline void ee_exact(const BPDev &B, BPQWarp &W, int n, float s, float thr, int &nout)
{
    const int lane = threadIdx.x & 31;
    bool found = false;
    int4 cnd = make_int4(0, 0, 0, 0);
    if (lane < n) do {
        const uint2 pd = W.pend[lane];
        const unsigned int q = pd.x;
        const int t = pd.y & 7, c = pd.y >> 3;
        const float4 v0 = __ldcg(B.ev + q), v1 = __ldcg(B.ev + B.ecap + q);
        const float4 pa = W.qa[t], pb = W.qb[t];
        const int ea = __float_as_int(pa.w), eb = __float_as_int(pb.w);
        const int f0 = __float_as_int(v0.w), f1 = __float_as_int(v1.w);
        if (f0 == ea || f0 == eb || f1 == ea || f1 == eb) break;
        const int4 ax = W.aux[t];
        if (B.nexcl) {
            const int bi = -1 - __float_as_int(__ldcg(B.eblo + q).w);
            if (B.edge[bi].z == ax.z &&
                is_excluded(B, (1ull << 62) | ((unsigned long long)ax.x << 31) | (unsigned long long)bi))
                break;
        }
        // the query edge's ends relative to this entry's cell corner
        int dx, dy, dz;
        cell_offset(ax.w, c, dx, dy, dz);
        const float ox = (float)dx * s, oy = (float)dy * s, oz = (float)dz * s;
        const float4 ra = make_float4(pa.x - ox, pa.y - oy, pa.z - oz, 0.f), rb = make_float4(pb.x - ox, pb.y - oy, pb.z - oz, 0.f);
        float cc[4];
        v3<float> tv;
        const float d = ee_coeffs<float>(f3sub(ra, v0), f3sub(rb, v0), f3sub(v1, v0), cc, tv);
        if (!(d < thr)) break;
        found = true;
        cnd = make_int4(-1 - ea, eb, f0, f1);
    } while (false);
    bpq_emit(B, W, nout, found, cnd);
}

// Edge-edge batch b of nb: edges b, b + nb, b + 2 nb, ... (strided), each against the edge table buckets of the
// cells of its own box (at most 2 per axis: a box is no wider than a cell).  A pair is found from the
// lower-numbered edge only, in the cell holding the lower corner of the intersection of the two boxes.
__device__ inline void bpq_edges(const BPDev &B, int b, int nb, const CellGrid &g, float thr, BPQWarp &W)
{
    const int lane = threadIdx.x & 31;
    unsigned int tot = 0;
    if (lane < BPQ_QE && b + lane * nb < B.ne) {
        const int a = b + lane * nb;
        const int4 e = B.edge[a];
        const double4_32a XA = ldcg4(B.x + e.x), XB = ldcg4(B.x + e.y);
        const float4 lo = make_float4(__double2float_rd(fmin(XA.x, XB.x)), __double2float_rd(fmin(XA.y, XB.y)),
                                      __double2float_rd(fmin(XA.z, XB.z)), 0.f);
        const float4 hi = make_float4(__double2float_ru(fmax(XA.x, XB.x)), __double2float_ru(fmax(XA.y, XB.y)),
                                      __double2float_ru(fmax(XA.z, XB.z)), 0.f);
        int l[3] = {0, 0, 0}, h[3] = {0, 0, 0};
        int nx = 1, ny = 1, ncell = 0;
        if (!box_cells(lo, hi, g, l, h)) {
            atomicOr(&B.ctrl->err, ERR_RANGE);
        } else {
            nx = h[0] - l[0] + 1;
            ny = h[1] - l[1] + 1;
            ncell = nx * ny * (h[2] - l[2] + 1);
            if (nx > 2 || ny > 2 || ncell > 8) { atomicOr(&B.ctrl->err, ERR_RANGE); ncell = 0; nx = ny = 1; }
        }
        const int w = nx | ny << 2;
        unsigned int st[8], len[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            st[c] = 0u;
            len[c] = 0u;
            if (c < ncell) {
                int dx, dy, dz;
                cell_offset(w, c, dx, dy, dz);
                const unsigned int b = cell_hash(l[0] + dx, l[1] + dy, l[2] + dz, B.H) + (unsigned int)B.H;
                st[c] = __ldcg(B.goff + b);
                len[c] = __ldcg(B.cnt + b);
                W.ckey[lane][c] = cell_key(l[0] + dx, l[1] + dy, l[2] + dz);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const unsigned int ln = st[c] < (unsigned int)B.ecap ? min(len[c], (unsigned int)B.ecap - st[c]) : 0u;
            tot += ln;
            W.cst[lane][c] = st[c];
            W.cinc[lane][c] = tot;   // cells past ncell repeat the total, so no item maps to them
        }
        W.qa[lane] = rel_corner(XA, l[0], l[1], l[2], g.s, e.x);
        W.qb[lane] = rel_corner(XB, l[0], l[1], l[2], g.s, e.y);
        W.lo[lane] = lo;
        W.hi[lane] = hi;
        W.aux[lane] = make_int4(a, B.vscene ? B.vscene[e.x] : 0, e.z, w);
    }
    unsigned int qi[BPQ_QB - 1];
    const unsigned int total = bpq_prefix(W, tot, qi);
    int np = 0, nout = 0;
    for (unsigned int base = 0; base < total; base += 64) {
        unsigned int q0 = 0, c0 = 0, q1 = 0, c1 = 0;
        const bool p0 = ee_filter(B, W, qi, base + lane, total, g, q0, c0);
        const bool p1 = ee_filter(B, W, qi, base + 32 + lane, total, g, q1, c1);
        bpq_push(W, np, p0, q0, c0);
        if (np >= 32) { __syncwarp(); ee_exact(B, W, 32, g.s, thr, nout); bpq_shift(W, np); }
        bpq_push(W, np, p1, q1, c1);
        if (np >= 32) { __syncwarp(); ee_exact(B, W, 32, g.s, thr, nout); bpq_shift(W, np); }
    }
    __syncwarp();
    if (np) ee_exact(B, W, np, g.s, thr, nout);
    bpq_flush(B, W, nout);
}

// Query batch w: edge batches first (they scan more entries), then point batches.  The candidate threshold adds
// 4e-6 s to the exact-distance one: positions within a cell or two of a corner keep ~1e-7 s each in float, and
// the differences and the distance formed from them stay well inside that.
__device__ inline void bpq_batch(const BPDev &B, int w, const CellGrid &g, BPQWarp &W)
{
    const float thr = B.thr + 4e-6f * g.s;
    const int nbe = bpq_edge_batches(B);
    if (w < nbe) bpq_edges(B, w, nbe, g, thr, W);
    else bpq_points(B, w - nbe, bpq_batches(B) - nbe, g, thr, W);
}

static __global__ void __launch_bounds__(BP_B) bp_query(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    __shared__ BPQWarp W[BP_B / 32];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w < bpq_batches(B)) bpq_batch(B, w, grid_of(cell_size(B)), W[threadIdx.x >> 5]);
}

} // namespace pncg
