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

#include <cuda_fp16.h>
#include <string.h>

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
    // entries, one per (primitive, cell of its box), in bucket order: everything the cheap tests of a query read
    // sits in two 16-byte records, the positions for the distance in the ev rows
    uint4 *erA;             // (cell key low, cell key high, v0, v1)
    uint4 *erB;             // (box (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z) as half pairs, w) with the box relative
                            // to the cell's corner in units of s, rounded outwards; w is v2 for a triangle, and for
                            // an edge the bits of the cell's offset from its box's lowest cell (x | y << 1 | z << 2)
    float4 *ev;             // [3][ecap] the primitive's vertices relative to the entry's cell corner; edges use
                            // the first two rows
    int *eprim;             // triangle f or edge index (read only where rest-pose exclusions exist)
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

__device__ inline __half2 u2h(unsigned int u) { __half2 h; memcpy(&h, &u, 4); return h; }
__device__ inline unsigned int h2u(__half2 h) { unsigned int u; memcpy(&u, &h, 4); return u; }

// A box [l, h] relative to a cell corner, in units of s, as half pairs ((l.x, l.y), (h.x, h.y), (l.z, h.z)) rounded
// outwards; 1e-6 covers the rounding of the float scaling.  Only a pre-filter reads it.
__device__ inline uint3 qbox(float lx, float ly, float lz, float hx, float hy, float hz, const CellGrid &g)
{
    const float e = 1e-6f;
    const __half2 l = __halves2half2(__float2half_rd(lx * g.inv - e), __float2half_rd(ly * g.inv - e));
    const __half2 h = __halves2half2(__float2half_ru(hx * g.inv + e), __float2half_ru(hy * g.inv + e));
    const __half2 z = __halves2half2(__float2half_rd(lz * g.inv - e), __float2half_ru(hz * g.inv + e));
    return make_uint3(h2u(l), h2u(h), h2u(z));
}
// do two such boxes meet (closed intervals on every axis)
__device__ inline bool qbox_meet(uint3 a, uint3 b)
{
    return __hble2(u2h(a.x), u2h(b.y)) & __hble2(u2h(b.x), u2h(a.y)) &
           __hble2(u2h(__byte_perm(a.z, b.z, 0x5410)), u2h(__byte_perm(b.z, a.z, 0x7632)));
}

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

// Writes primitive j's entries, one per cell of its box: the records of the cheap tests and the vertices relative
// to the entry's cell corner (formed once in double against the box's lowest cell, then shifted by whole cells in
// float).  slot_of(b) reserves a slot of bucket b; the slots of all cells are reserved before any entry is written.
template <typename F> __device__ inline void fill_prim(const BPDev &B, int j, const CellGrid &g, F slot_of)
{
    const float s = g.s;
    const float4 lo = __ldcg(B.blo + j), hi = __ldcg(B.bhi + j);
    int l[3], h[3];
    if (!box_cells(lo, hi, g, l, h)) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
    int v[3], nvp;
    prim_verts(B, j, v, nvp);
    float4 r[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) r[q] = rel_corner(ldcg4(B.x + v[q]), l[0], l[1], l[2], s, v[q]);
    // the inflated box relative to the lowest cell's corner (a pre-filter only: the 16-bit form rounds outwards)
    const float inf = (float)B.infl;
    const float mnx = fminf(fminf(r[0].x, r[1].x), r[2].x) - inf, mxx = fmaxf(fmaxf(r[0].x, r[1].x), r[2].x) + inf;
    const float mny = fminf(fminf(r[0].y, r[1].y), r[2].y) - inf, mxy = fmaxf(fmaxf(r[0].y, r[1].y), r[2].y) + inf;
    const float mnz = fminf(fminf(r[0].z, r[1].z), r[2].z) - inf, mxz = fmaxf(fmaxf(r[0].z, r[1].z), r[2].z) + inf;
    const bool tri = j < B.nf;
    const int prim = tri ? j : j - B.nf;
    auto put = [&](unsigned int slot, int dx, int dy, int dz) {
        if (slot >= (unsigned int)B.ecap) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
        const unsigned long long key = cell_key(l[0] + dx, l[1] + dy, l[2] + dz);
        const float ox = (float)dx * s, oy = (float)dy * s, oz = (float)dz * s;
        const uint3 bx = qbox(mnx - ox, mny - oy, mnz - oz, mxx - ox, mxy - oy, mxz - oz, g);
        B.erA[slot] = make_uint4((unsigned int)key, (unsigned int)(key >> 32), (unsigned int)v[0], (unsigned int)v[1]);
        const unsigned int dbits = min(dx, 1) | min(dy, 1) << 1 | min(dz, 1) << 2;
        B.erB[slot] = make_uint4(bx.x, bx.y, bx.z, tri ? (unsigned int)v[2] : dbits);
        B.eprim[slot] = prim;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q < nvp) B.ev[(size_t)q * B.ecap + slot] = make_float4(r[q].x - ox, r[q].y - oy, r[q].z - oz, 0.0f);
    };
    const int nx = h[0] - l[0] + 1, ny = h[1] - l[1] + 1, nz = h[2] - l[2] + 1;
    if (nx <= 2 && ny <= 2 && nz <= 2) {
        unsigned int slot[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if ((c & 1) < nx && ((c >> 1) & 1) < ny && (c >> 2) < nz)
                slot[c] = slot_of(prim_bucket(B, j, l[0] + (c & 1), l[1] + ((c >> 1) & 1), l[2] + (c >> 2)));
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if ((c & 1) < nx && ((c >> 1) & 1) < ny && (c >> 2) < nz) put(slot[c], c & 1, (c >> 1) & 1, c >> 2);
    } else {
        // a box wider than two cells (only when rounding at coordinates far from the origin widens it): the grid
        // cannot hold the build, which is flagged; the counted entries are still written, so every bucket is whole
        atomicOr(&B.ctrl->err, ERR_RANGE);
        for (int i = l[0]; i <= h[0]; ++i)
            for (int jj = l[1]; jj <= h[1]; ++jj)
                for (int kk = l[2]; kk <= h[2]; ++kk) put(slot_of(prim_bucket(B, j, i, jj, kk)), i - l[0], jj - l[1], kk - l[2]);
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
// A warp takes a batch of queries of one kind (points, or edges).  Its header lists the batch's non-empty
// (query, cell) segments in shared memory: the bucket's first entry, the segment's first item in the batch, the
// cell's key and the query's box relative to the cell's corner.  The warp then scans all the segments' entries as
// one list, 64 per round (two windows of 32, one item per lane each, loaded together); a lane finds its segment
// from the window's segment starts, gathered into one bit mask by a warp OR.  A round reads the two 16-byte records
// of each entry and applies the cheap tests: cell key, shared vertex, edge order, the cell rule of edge pairs and
// the overlap of the half-precision boxes.  The entries that pass queue up in shared memory and get the exact
// distance 32 at a time, with every lane busy.  Found pairs collect in shared memory and are appended with one
// atomic per 32.
//
// Edge pairs: each unordered pair is tested from one side only, the edge whose lower vertex index is smaller (two
// edges without a shared vertex have different lower vertices), and in one cell only, the cell of the lower corner
// of the intersection of the two inflated boxes.  The cell index is monotone in the coordinate, so that cell is,
// per axis, the larger of the two boxes' lowest cells; in a cell the pair shares, it is this cell exactly when on
// no axis both edges sit in their box's second cell (offset bits of the query's cell AND the entry's = 0).
constexpr int BPQ_QE = 6;       // edges per batch (an edge's box covers about twice the cells of a point)
constexpr int BPQ_QP = 8;       // points per batch
constexpr int BPQ_SEG = 48;     // (query, cell) segments of a batch: 6 edges x 8 cells, or 8 points
constexpr int BPQ_PEND = 64;    // entries past the cheap tests, awaiting the distance
constexpr int BPQ_OUT = 64;     // found pairs held before an append

struct BPQWarp {
    uint4 sa[BPQ_SEG];              // (first entry, first item, query's lower vertex, higher vertex; a point: v, v)
    unsigned long long sk[BPQ_SEG]; // the cell's key
    uint4 sb[BPQ_SEG];              // the query's box relative to the cell's corner (as the entries'), w: the cell's
                                    // offset bits (edge) | query << 8 | cell << 11
    float4 qa[BPQ_QP];              // point: relative to its cell's corner (w: vertex); edge: first end relative to
                                    // the corner of its box's lowest cell (w: its vertex)
    float4 qb[BPQ_QE];              // edge: second end as qa
    int4 aux[BPQ_QP];               // x: point index j or edge index a; y: scene; z: object; w: edge nx | ny << 2
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
__device__ inline unsigned long long key_of(const uint4 &A) { return (unsigned long long)A.y << 32 | A.x; }

// Appends the lanes' segments to the batch's list (all lanes call; ln = 0 for none): returns the segment slot of
// a lane with a segment; nseg and nitem (warp-uniform) grow by the segments and their entries.
__device__ inline int bpq_add_segments(unsigned int ln, int &nseg, unsigned int &nitem, unsigned int &first)
{
    const int lane = threadIdx.x & 31;
    const unsigned int m = __ballot_sync(0xffffffffu, ln > 0u);
    unsigned int inc = ln;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    first = nitem + inc - ln;
    const int slot = nseg + __popc(m & lanemask_lt());
    nseg += __popc(m);
    nitem += __shfl_sync(0xffffffffu, inc, 31);
    return slot;
}

// The segment of item it of the window [base, base + 32) that starts in segment k0 (all lanes call): the lanes
// bring the starts of segments k0 + 1 .. k0 + 32 (at most 32 start inside a window of 32 items, all segments being
// non-empty), one warp OR gathers them into a mask of window offsets.  Returns the lane's segment; k_next is the
// segment of the window's last item.
__device__ inline int bpq_window(const BPQWarp &W, int nseg, unsigned int base, int k0, int &k_next)
{
    const int lane = threadIdx.x & 31;
    const int k = k0 + 1 + lane;
    unsigned int bit = 0u;
    if (k < nseg) {
        const unsigned int off = W.sa[k].y - base;   // > 0: the segment starts after base
        if (off < 32u) bit = 1u << off;
    }
    const unsigned int M = __reduce_or_sync(0xffffffffu, bit);
    k_next = k0 + __popc(M);
    return k0 + __popc(M & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u)));
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

// cheap tests of an entry q of segment k of a point batch: the entry is of the point's cell, the triangle does not
// hold the point, and its box holds it
__device__ inline bool pt_filter(const BPDev &B, const BPQWarp &W, bool valid, int k, unsigned int it, unsigned int &q,
                                 unsigned int &tc)
{
    if (!valid) return false;
    const uint4 S = W.sa[k];
    q = S.x + (it - S.y);
    const uint4 A = __ldcg(B.erA + q), E = __ldcg(B.erB + q);
    const uint4 Q = W.sb[k];
    tc = Q.w >> 8;
    return (key_of(A) == W.sk[k]) & (A.z != S.z) & (A.w != S.z) & (E.w != S.z) &
           qbox_meet(make_uint3(Q.x, Q.y, Q.z), make_uint3(E.x, E.y, E.z));
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
        const uint4 A = __ldcg(B.erA + q);
        const int a2 = (int)__ldcg(&B.erB[q].w);
        const float4 qa = W.qa[t];
        const int4 ax = W.aux[t];
        const int a0 = (int)A.z, a1 = (int)A.w;
        if (B.vscene && B.vscene[a0] != ax.y) break;
        if (B.nexcl) {
            const int f = __ldcg(B.eprim + q);
            if (B.tri[f].w == ax.z && is_excluded(B, ((unsigned long long)ax.x << 31) | (unsigned long long)f)) break;
        }
        float cc[4];
        v3<float> tv;
        const float d = pt_coeffs<float>(f3sub(qa, t0), f3sub(t1, t0), f3sub(t2, t0), cc, tv);
        if (!(d < thr)) break;
        found = true;
        cnd = make_int4(__float_as_int(qa.w), a0, a1, a2);
    } while (false);
    bpq_emit(B, W, nout, found, cnd);
}

// Point-triangle batch b of nb: surface points b, b + nb, b + 2 nb, ... (strided, so that a batch mixes crowded
// and sparse parts of the surface), each against the triangle table bucket of its cell.
__device__ inline void bpq_points(const BPDev &B, int b, int nb, const CellGrid &g, float thr, BPQWarp &W)
{
    const int lane = threadIdx.x & 31;
    unsigned int ln = 0u, st = 0u;
    unsigned long long key = 0ull;
    uint3 bx = make_uint3(0u, 0u, 0u);
    int v = 0;
    if (lane < BPQ_QP && b + lane * nb < B.ns) {
        const int j = b + lane * nb;
        v = B.svert[j];
        const double4_32a X = ldcg4(B.x + v);
        int ix = 0, iy = 0, iz = 0;
        if (!cell_of((float)X.x, g, ix) || !cell_of((float)X.y, g, iy) || !cell_of((float)X.z, g, iz)) {
            atomicOr(&B.ctrl->err, ERR_RANGE);
        } else {
            const unsigned int bk = cell_hash(ix, iy, iz, B.H);
            st = __ldcg(B.goff + bk);
            const unsigned int len = __ldcg(B.cnt + bk);
            ln = st < (unsigned int)B.ecap ? min(len, (unsigned int)B.ecap - st) : 0u;   // a fill overflow is flagged
        }
        const float4 p = rel_corner(X, ix, iy, iz, g.s, v);
        bx = qbox(p.x, p.y, p.z, p.x, p.y, p.z, g);
        key = cell_key(ix, iy, iz);
        W.qa[lane] = p;
        W.aux[lane] = make_int4(j, B.vscene ? B.vscene[v] : 0, B.obj[v], 0);
    }
    int nseg = 0;
    unsigned int total = 0u, first;
    const int slot = bpq_add_segments(ln, nseg, total, first);
    if (ln > 0u) {
        W.sa[slot] = make_uint4(st, first, (unsigned int)v, (unsigned int)v);
        W.sk[slot] = key;
        W.sb[slot] = make_uint4(bx.x, bx.y, bx.z, (unsigned int)lane << 8);
    }
    __syncwarp();
    int np = 0, nout = 0, k0 = 0;
    for (unsigned int base = 0; base < total; base += 64) {
        int k1, k2;
        const int ka = bpq_window(W, nseg, base, k0, k1);
        const int kb = bpq_window(W, nseg, base + 32, k1, k2);
        k0 = k2;
        unsigned int q0 = 0, t0 = 0, q1 = 0, t1 = 0;
        const bool p0 = pt_filter(B, W, base + lane < total, ka, base + lane, q0, t0);
        const bool p1 = pt_filter(B, W, base + 32 + lane < total, kb, base + 32 + lane, q1, t1);
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

// cheap tests of an entry of segment k of an edge batch: the entry is of its cell, shares no vertex with the query
// edge and has the larger lower vertex, the cell is the pair's cell, and the boxes meet
__device__ inline bool ee_filter(const BPDev &B, const BPQWarp &W, bool valid, int k, unsigned int it, unsigned int &q,
                                 unsigned int &tc)
{
    if (!valid) return false;
    const uint4 S = W.sa[k];
    q = S.x + (it - S.y);
    const uint4 A = __ldcg(B.erA + q), E = __ldcg(B.erB + q);
    const uint4 Q = W.sb[k];
    tc = Q.w >> 8;
    const int fmn = min((int)A.z, (int)A.w), fmx = max((int)A.z, (int)A.w);
    return (key_of(A) == W.sk[k]) & (fmn > (int)S.z) & (fmn != (int)S.w) & (fmx != (int)S.w) & ((Q.w & E.w & 7u) == 0u) &
           qbox_meet(make_uint3(Q.x, Q.y, Q.z), make_uint3(E.x, E.y, E.z));
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
        const uint4 A = __ldcg(B.erA + q);
        const float4 pa = W.qa[t], pb = W.qb[t];
        const int4 ax = W.aux[t];
        const int f0 = (int)A.z, f1 = (int)A.w;
        if (B.vscene && B.vscene[f0] != ax.y) break;
        if (B.nexcl) {
            const int bi = __ldcg(B.eprim + q);
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
        cnd = make_int4(-1 - __float_as_int(pa.w), __float_as_int(pb.w), f0, f1);
    } while (false);
    bpq_emit(B, W, nout, found, cnd);
}

// Edge-edge batch b of nb: edges b, b + nb, b + 2 nb, ... (strided), each against the edge table buckets of the
// cells of its own box (at most 2 per axis: a box is no wider than a cell).  The headers take two passes of four
// edges, eight lanes per edge (one per cell), each lane forming its edge's box and cells itself.
__device__ inline void bpq_edges(const BPDev &B, int b, int nb, const CellGrid &g, float thr, BPQWarp &W)
{
    const int lane = threadIdx.x & 31, c = lane & 7;
    int nseg = 0;
    unsigned int total = 0u;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        const int t = pass * 4 + (lane >> 3);
        const int a = b + t * nb;
        unsigned int st = 0u, ln = 0u;
        unsigned long long key = 0ull;
        uint4 sb = make_uint4(0u, 0u, 0u, 0u);
        int vlo = 0, vhi = 0;
        if (t < BPQ_QE && a < B.ne) {
            const int4 e = B.edge[a];
            vlo = min(e.x, e.y);
            vhi = max(e.x, e.y);
            const double4_32a XA = ldcg4(B.x + e.x), XB = ldcg4(B.x + e.y);
            const float4 lo = make_float4(__double2float_rd(fmin(XA.x, XB.x)), __double2float_rd(fmin(XA.y, XB.y)),
                                          __double2float_rd(fmin(XA.z, XB.z)), 0.f);
            const float4 hi = make_float4(__double2float_ru(fmax(XA.x, XB.x)), __double2float_ru(fmax(XA.y, XB.y)),
                                          __double2float_ru(fmax(XA.z, XB.z)), 0.f);
            int l[3] = {0, 0, 0}, h[3] = {0, 0, 0};
            int nx = 1, ny = 1, ncell = 0;
            if (!box_cells(lo, hi, g, l, h)) {
                if (c == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
            } else {
                nx = h[0] - l[0] + 1;
                ny = h[1] - l[1] + 1;
                ncell = nx * ny * (h[2] - l[2] + 1);
                if (nx > 2 || ny > 2 || ncell > 8) {
                    if (c == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
                    ncell = 0; nx = ny = 1;
                }
            }
            const int w = nx | ny << 2;
            const float4 pa = rel_corner(XA, l[0], l[1], l[2], g.s, e.x), pb = rel_corner(XB, l[0], l[1], l[2], g.s, e.y);
            if (c < ncell) {
                int dx, dy, dz;
                cell_offset(w, c, dx, dy, dz);
                const unsigned int bk = cell_hash(l[0] + dx, l[1] + dy, l[2] + dz, B.H) + (unsigned int)B.H;
                st = __ldcg(B.goff + bk);
                const unsigned int len = __ldcg(B.cnt + bk);
                ln = st < (unsigned int)B.ecap ? min(len, (unsigned int)B.ecap - st) : 0u;   // a fill overflow is flagged
                const float ox = (float)dx * g.s, oy = (float)dy * g.s, oz = (float)dz * g.s;
                const uint3 bx = qbox(fminf(pa.x, pb.x) - ox, fminf(pa.y, pb.y) - oy, fminf(pa.z, pb.z) - oz,
                                      fmaxf(pa.x, pb.x) - ox, fmaxf(pa.y, pb.y) - oy, fmaxf(pa.z, pb.z) - oz, g);
                key = cell_key(l[0] + dx, l[1] + dy, l[2] + dz);
                sb = make_uint4(bx.x, bx.y, bx.z, (unsigned int)(dx | dy << 1 | dz << 2) | (unsigned int)t << 8 | (unsigned int)c << 11);
            }
            if (c == 0) {
                W.qa[t] = pa;
                W.qb[t] = pb;
                W.aux[t] = make_int4(a, B.vscene ? B.vscene[e.x] : 0, e.z, w);
            }
        }
        unsigned int first;
        const int slot = bpq_add_segments(ln, nseg, total, first);
        if (ln > 0u) {
            W.sa[slot] = make_uint4(st, first, (unsigned int)vlo, (unsigned int)vhi);
            W.sk[slot] = key;
            W.sb[slot] = sb;
        }
    }
    __syncwarp();
    int np = 0, nout = 0, k0 = 0;
    for (unsigned int base = 0; base < total; base += 64) {
        int k1, k2;
        const int ka = bpq_window(W, nseg, base, k0, k1);
        const int kb = bpq_window(W, nseg, base + 32, k1, k2);
        k0 = k2;
        unsigned int q0 = 0, c0 = 0, q1 = 0, c1 = 0;
        const bool p0 = ee_filter(B, W, base + lane < total, ka, base + lane, q0, c0);
        const bool p1 = ee_filter(B, W, base + 32 + lane < total, kb, base + 32 + lane, q1, c1);
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
