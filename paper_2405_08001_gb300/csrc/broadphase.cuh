// Contact-candidate pass (spatial hash over surface primitives; the paper uses grid spatial hashing for its
// broad phase, Sec. 6).  Candidates are all surface point-triangle pairs (point not in the triangle) and edge-edge
// pairs (no shared vertex) within dhat + r of each other (box test) at the positions of the build, whose distance
// there is below (dhat + r)(1 + 1e-3); pairs of one object closer than the exclusion radius at rest (Sec. 5.1) are
// dropped.  Since d changes by at most twice the largest vertex displacement, every pair with d < dhat is a
// candidate until some vertex has moved r/2.
//
// Three hash tables of H buckets each: triangles [0, H) and edges [H, 2H), each registered in every cell its box
// inflated by dhat + r covers, and surface points [2H, 3H), each in its own cell.  The five kernels run only when
// Ctrl::rebuild is set (they return at once otherwise):
//   bp_boxes  : inflated float boxes (rounded outwards), largest extent -> cell size, zero bucket counts, x_b = x
//   bp_count  : entries per bucket (a box covers at most 2 cells per axis)
//   bp_scan   : exclusive scan of the counts (block-local scans + the last block scans the block sums), and the
//               list of work units: every 32 x 32 tile (row chunk <= column chunk) of a non-empty edge bucket, and
//               every chunk of 32 rows of a non-empty triangle bucket
//   bp_fill   : entries in bucket order (the two records of the cheap tests, the vertices relative to the cell's
//               corner) and each bucket's global first entry
//   bp_query  : one warp per work unit: its 32 rows (triangles, or edges) against its columns (the points of the
//               same cells, or a chunk of 32 edges of the bucket) staged in shared memory; the pairs that pass the
//               cheap tests get the distance at the build positions, 32 at a time
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
constexpr int BP_ROWS = 32;                    // rows of a work unit (one per lane)
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
    unsigned int *goff;     // [3H] global first entry of each bucket (written with the entries, read by queries)
    unsigned int *ctot;     // persistent form: [3H >> cshift_p] entries per scan chunk
    int cshift_p;           // persistent form: log2 of the buckets per scan chunk
    const int *vscene;      // batching: scene of each vertex (pairs of two scenes are never candidates); or null
    // entries in bucket order: everything the cheap tests read sits in two 16-byte records, the positions for the
    // distance in the ev rows
    uint4 *erA;             // (cell key low, cell key high, v0, v1); a point: (key, v, v)
    uint4 *erB;             // (box (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z) as half pairs, w): the primitive's box
                            // inflated by (dhat + r)/2, so that two such boxes meet exactly when the primitives' own
                            // boxes are within dhat + r, relative to the cell's corner in units of s, rounded
                            // outwards; w is v2 for a triangle, 0 for a point, and for an edge the bits of the
                            // cell's offset from its registration box's lowest cell (x | y << 1 | z << 2)
    float4 *ev;             // [3][ecap] the primitive's vertices relative to the entry's cell corner (edges use two
                            // rows, points one)
    int *eprim;             // triangle f, edge index or surface point index (read where rest-pose exclusions exist)
    int ecap;               // entry capacity (8 per triangle or edge, 1 per point)
    uint2 *units;           // work units, listed by the scan: (bucket, row chunk | column chunk << 16) for edges,
                            // (bucket, row chunk | 0xffff << 16) for triangles
    int ucap;
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
__device__ inline unsigned int point_bucket(const BPDev &B, int ix, int iy, int iz)
{
    return cell_hash(ix, iy, iz, B.H) + 2u * (unsigned int)B.H;
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

// visits the cells covered by [lo, hi]; flags a coordinate out of the grid's range
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

// the cell of surface point j (false: out of the grid's range)
__device__ inline bool point_cell(const BPDev &B, int j, const CellGrid &g, int &v, double4_32a &X, int c[3])
{
    v = B.svert[j];
    X = ldcg4(B.x + v);
    return cell_of((float)X.x, g, c[0]) && cell_of((float)X.y, g, c[1]) && cell_of((float)X.z, g, c[2]);
}

// Writes primitive j's entries, one per cell of its registration box: the records of the cheap tests and the
// vertices relative to the entry's cell corner (formed once in double against the box's lowest cell, then shifted
// by whole cells in float).  slot_of(b) reserves a slot of bucket b; all slots are reserved before any is written.
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
    // the primitive's box inflated by half of dhat + r, relative to the lowest cell's corner
    const float inf = 0.5f * (float)B.infl;
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

// Writes surface point j's entry in its own cell: (key, v, v), its box of half of dhat + r around it, its position
// relative to the cell's corner, and j.
template <typename F> __device__ inline void fill_point(const BPDev &B, int j, const CellGrid &g, F slot_of)
{
    int v, c[3];
    double4_32a X;
    if (!point_cell(B, j, g, v, X, c)) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
    const unsigned int slot = slot_of(point_bucket(B, c[0], c[1], c[2]));
    if (slot >= (unsigned int)B.ecap) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
    const float4 p = rel_corner(X, c[0], c[1], c[2], g.s, v);
    const float inf = 0.5f * (float)B.infl;
    const uint3 bx = qbox(p.x - inf, p.y - inf, p.z - inf, p.x + inf, p.y + inf, p.z + inf, g);
    const unsigned long long key = cell_key(c[0], c[1], c[2]);
    B.erA[slot] = make_uint4((unsigned int)key, (unsigned int)(key >> 32), (unsigned int)v, (unsigned int)v);
    B.erB[slot] = make_uint4(bx.x, bx.y, bx.z, 0u);
    B.eprim[slot] = j;
    B.ev[slot] = make_float4(p.x, p.y, p.z, 0.0f);
}

// Appends the work units of the lanes' buckets (all lanes call, each with up to four buckets (b, n)): an edge
// bucket (H <= b < 2H) with n entries in t = ceil(n / 32) chunks gives its t (t + 1) / 2 tiles (r <= c), so that no
// unit is larger than 32 x 32 pairs; a triangle bucket gives its t row chunks (the points of a cell are few).  The
// tiles of edge buckets of 64 or more entries (full tiles, the densest cells) are listed from the front of the list
// and taken first by the query; the rest from the end.
__device__ inline unsigned int warp_excl(unsigned int v, unsigned int &total)
{
    const int lane = threadIdx.x & 31;
    unsigned int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}
__device__ inline void list_units(const BPDev &B, const unsigned int (&b)[4], const unsigned int (&n)[4])
{
    const int lane = threadIdx.x & 31;
    const unsigned int H = (unsigned int)B.H;
    unsigned int t[4], th = 0, tl = 0;
    bool heavy[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        t[q] = b[q] < 2u * H ? (n[q] + BP_ROWS - 1) / BP_ROWS : 0u;
        const unsigned int u = b[q] >= H ? t[q] * (t[q] + 1u) / 2u : t[q];
        heavy[q] = b[q] >= H && t[q] >= 2u;
        if (heavy[q]) th += u; else tl += u;
    }
    unsigned int wh, wl;
    const unsigned int eh = warp_excl(th, wh), el = warp_excl(tl, wl);
    if (wh + wl == 0u) return;
    unsigned int bh = 0, bl = 0;
    if (lane == 31) {
        if (wh) bh = atomicAdd((unsigned int *)&B.ctrl->n_units_h, wh);
        if (wl) bl = atomicAdd((unsigned int *)&B.ctrl->n_units, wl);
    }
    unsigned int kh = __shfl_sync(0xffffffffu, bh, 31) + eh, kl = __shfl_sync(0xffffffffu, bl, 31) + el;
    const unsigned int cap = (unsigned int)B.ucap;
    if (kh + th > cap || kl + tl > cap) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (b[q] >= H) {
            for (unsigned int r = 0; r < t[q]; ++r)
                for (unsigned int c = r; c < t[q]; ++c) {
                    const uint2 unit = make_uint2(b[q], r | c << 16);
                    if (heavy[q]) B.units[kh++] = unit; else B.units[cap - 1u - kl++] = unit;
                }
        } else {
            for (unsigned int r = 0; r < t[q]; ++r) B.units[cap - 1u - kl++] = make_uint2(b[q], r | 0xffffu << 16);
        }
    }
}

static __global__ void __launch_bounds__(BP_B) bp_boxes(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const int n = max(max(B.nf + B.ne, B.nv), 3 * B.H);
    const int stride = gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.ctrl->n_cand = 0; B.ctrl->n_units = 0; B.ctrl->n_units_h = 0; B.ctrl->n_rebuilds += 1;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        if (j < 3 * B.H) B.cnt[j] = 0u;
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

// one thread per triangle or edge (j < nf + ne) and per surface point (j < ns)
static __global__ void __launch_bounds__(BP_B) bp_count(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const CellGrid g = grid_of(cell_size(B));
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < B.nf + B.ne)
        for_cells(B, B.blo[j], B.bhi[j], g, [&](int i, int jj, int k) { atomicAdd(&B.cnt[prim_bucket(B, j, i, jj, k)], 1u); });
    if (j < B.ns) {
        int v, c[3];
        double4_32a X;
        if (point_cell(B, j, g, v, X, c)) atomicAdd(&B.cnt[point_bucket(B, c[0], c[1], c[2])], 1u);
        else atomicOr(&B.ctrl->err, ERR_RANGE);
    }
}

static __global__ void __launch_bounds__(BP_SCAN_T) bp_scan(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    __shared__ unsigned int wsum[BP_SCAN_T / 32];
    __shared__ bool last;
    const int base = blockIdx.x * BP_SCAN_N + 4 * threadIdx.x;
    uint4 c = reinterpret_cast<const uint4 *>(B.cnt)[base / 4];
    {
        const unsigned int bb[4] = {(unsigned int)base, (unsigned int)base + 1u, (unsigned int)base + 2u, (unsigned int)base + 3u};
        const unsigned int nn[4] = {c.x, c.y, c.z, c.w};
        list_units(B, bb, nn);
    }
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

// one thread per triangle or edge (j < nf + ne) and per surface point (j < ns)
static __global__ void __launch_bounds__(BP_B) bp_fill(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    const CellGrid g = grid_of(cell_size(B));
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < 3 * B.H; b += gridDim.x * blockDim.x)
        B.goff[b] = B.boff[b / BP_SCAN_N] + B.off[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    auto slot_of = [&](unsigned int b) { return B.boff[b / BP_SCAN_N] + B.off[b] + atomicAdd(&B.cnt[b], 1u); };
    if (j < B.nf + B.ne) fill_prim(B, j, g, slot_of);
    if (j < B.ns) fill_point(B, j, g, slot_of);
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
// A work unit is (bucket b, row chunk r) of the triangle or edge table.  Its warp holds 32 rows, one per lane: the
// bucket's entries 32 r .. 32 r + 31.  The columns are staged in shared memory 32 at a time: for a triangle bucket
// the entries of point bucket b + 2H (the same cells), for an edge bucket the bucket's own entries after the row's.
// Every lane tests its row against each staged column (two broadcast reads): same cell key, boxes within
// dhat + r, no shared vertex, and for edge pairs the cell rule below.  The pairs that pass queue up in shared memory
// and get the exact distance 32 at a time, with every lane busy; found pairs collect in shared memory and are
// appended with one atomic per 32.
//
// Edge pairs: two edges within dhat + r of each other are registered together in the cells from the larger of
// their registration boxes' lowest cells (per axis) to the smaller of the highest; the pair is tested in the
// lowest of those only.  In a cell the pair shares, that is this cell exactly when on no axis both edges sit past
// their box's lowest cell (offset bits of the two entries AND = 0); the cell index is monotone in the coordinate.
// A point lies in one cell, and a triangle within dhat + r of it is registered there.
constexpr int BPQ_PEND = 64;    // pairs past the cheap tests, awaiting the distance
constexpr int BPQ_OUT = 64;     // found pairs held before an append
constexpr unsigned int BPQ_PT = 0x80000000u;   // marks a point-triangle pair in the queue

struct BPQWarp {
    uint4 ca[32], cb[32];           // the staged columns' records
    uint2 pend[BPQ_PEND];           // (row entry, column entry | BPQ_PT for a point column)
    int4 out[BPQ_OUT];
};

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

__device__ inline v3<float> f3sub(const float4 &a, const float4 &b) { return mkv(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline unsigned long long key_of(const uint4 &A) { return (unsigned long long)A.y << 32 | A.x; }

// exact tests of the first n queued pairs (all lanes call); both entries of a pair are in the same cell, so their
// positions are relative to the same corner
__device__ inline void bpq_exact(const BPDev &B, BPQWarp &W, int n, float thr, int &nout)
{
    const int lane = threadIdx.x & 31;
    bool found = false;
    int4 cnd = make_int4(0, 0, 0, 0);
    if (lane < n) do {
        const uint2 pd = W.pend[lane];
        const unsigned int qr = pd.x, qc = pd.y & ~BPQ_PT;
        const uint4 Ar = __ldcg(B.erA + qr), Ac = __ldcg(B.erA + qc);
        const float4 r0 = __ldcg(B.ev + qr), r1 = __ldcg(B.ev + B.ecap + qr), c0 = __ldcg(B.ev + qc);
        float cc[4];
        v3<float> tv;
        if (pd.y & BPQ_PT) {
            // row: triangle (Ar.z, Ar.w, v2), column: point Ac.z
            const float4 r2 = __ldcg(B.ev + 2 * (size_t)B.ecap + qr);
            const int t2 = (int)__ldcg(&B.erB[qr].w), v = (int)Ac.z;
            if (B.vscene && B.vscene[v] != B.vscene[(int)Ar.z]) break;
            if (B.nexcl) {
                const int f = __ldcg(B.eprim + qr), jp = __ldcg(B.eprim + qc);
                if (B.tri[f].w == B.obj[v] && is_excluded(B, ((unsigned long long)jp << 31) | (unsigned long long)f)) break;
            }
            const float d = pt_coeffs<float>(f3sub(c0, r0), f3sub(r1, r0), f3sub(r2, r0), cc, tv);
            if (!(d < thr)) break;
            found = true;
            cnd = make_int4(v, (int)Ar.z, (int)Ar.w, t2);
        } else {
            // row: edge (Ar.z, Ar.w), column: edge (Ac.z, Ac.w)
            const float4 c1 = __ldcg(B.ev + B.ecap + qc);
            if (B.vscene && B.vscene[(int)Ar.z] != B.vscene[(int)Ac.z]) break;
            if (B.nexcl) {
                const int ea = __ldcg(B.eprim + qr), eb = __ldcg(B.eprim + qc);
                const int a = min(ea, eb), b = max(ea, eb);
                if (B.edge[a].z == B.edge[b].z &&
                    is_excluded(B, (1ull << 62) | ((unsigned long long)a << 31) | (unsigned long long)b))
                    break;
            }
            const float d = ee_coeffs<float>(f3sub(r0, c0), f3sub(r1, c0), f3sub(c1, c0), cc, tv);
            if (!(d < thr)) break;
            found = true;
            cnd = make_int4(-1 - (int)Ar.z, (int)Ar.w, (int)Ac.z, (int)Ac.w);
        }
    } while (false);
    bpq_emit(B, W, nout, found, cnd);
}

// queues the lanes' passing pairs (all lanes call); runs the exact tests once 32 are queued
__device__ inline void bpq_push(const BPDev &B, BPQWarp &W, int &np, int &nout, float thr, bool pass, unsigned int qr,
                                unsigned int qc)
{
    const unsigned int m = __ballot_sync(0xffffffffu, pass);
    if (!m) return;
    if (pass) W.pend[np + __popc(m & lanemask_lt())] = make_uint2(qr, qc);
    np += __popc(m);
    if (np >= 32) {
        __syncwarp();
        bpq_exact(B, W, 32, thr, nout);
        // drop the 32 done
        const int lane = threadIdx.x & 31;
        uint2 v = make_uint2(0u, 0u);
        if (lane < np - 32) v = W.pend[32 + lane];
        __syncwarp();
        if (lane < np - 32) W.pend[lane] = v;
        __syncwarp();
        np -= 32;
    }
}

// Work unit (b, r | c << 16) (all lanes call): rows 32 r .. 32 r + 31 of bucket b; columns 32 c .. 32 c + 31 of the
// same bucket (edges, the pairs with the row before the column), or all entries of point bucket b + 2H (c = 0xffff).
__device__ inline void bpq_unit(const BPDev &B, uint2 unit, float thr, BPQWarp &W, int &np, int &nout)
{
    const int lane = threadIdx.x & 31;
    const unsigned int b = unit.x, r = unit.y & 0xffffu, cc = unit.y >> 16;
    const bool ee = b >= (unsigned int)B.H;
    const unsigned int E = (unsigned int)B.ecap;
    const unsigned int rst = __ldcg(B.goff + b), rn = min(__ldcg(B.cnt + b), E - min(rst, E));
    unsigned int cst, c0, c1;
    if (ee) {
        cst = rst;
        c0 = cc * BP_ROWS;
        c1 = min(c0 + BP_ROWS, rn);
    } else {
        const unsigned int pb = b + 2u * (unsigned int)B.H;
        cst = __ldcg(B.goff + pb);
        c0 = 0u;
        c1 = min(__ldcg(B.cnt + pb), E - min(cst, E));
    }
    // the lane's row
    const unsigned int i = r * BP_ROWS + lane;
    const bool rv = i < rn;
    uint4 Ar = make_uint4(0u, 0u, 0u, 0u), Br = make_uint4(0u, 0u, 0u, 0u);
    if (rv) { Ar = __ldcg(B.erA + rst + i); Br = __ldcg(B.erB + rst + i); }
    const unsigned long long kr = key_of(Ar);
    const uint3 bxr = make_uint3(Br.x, Br.y, Br.z);
    const unsigned int qr = rst + i, tag = ee ? 0u : BPQ_PT;
    for (unsigned int j0 = c0; j0 < c1; j0 += 32u) {
        __syncwarp();
        if (j0 + lane < c1) { W.ca[lane] = __ldcg(B.erA + cst + j0 + lane); W.cb[lane] = __ldcg(B.erB + cst + j0 + lane); }
        __syncwarp();
        const unsigned int kn = min(32u, c1 - j0);
        for (unsigned int k = 0; k < kn; ++k) {
            const uint4 Ac = W.ca[k], Bc = W.cb[k];
            bool pass = rv & (key_of(Ac) == kr) & qbox_meet(bxr, make_uint3(Bc.x, Bc.y, Bc.z));
            if (ee) {
                pass &= (j0 + k > i) & (Ac.z != Ar.z) & (Ac.z != Ar.w) & (Ac.w != Ar.z) & (Ac.w != Ar.w) &
                        ((Br.w & Bc.w) == 0u);
            } else {
                pass &= (Ac.z != Ar.z) & (Ac.z != Ar.w) & (Ac.z != Br.w);
            }
            bpq_push(B, W, np, nout, thr, pass, qr, (cst + j0 + k) | tag);
        }
    }
}

// Work units u = first, first + stride, ... (all lanes of the warp call; its batch area in W).  The candidate
// threshold adds 4e-6 s to the exact-distance one: positions within a cell or two of a corner keep ~1e-7 s each
// in float, and the differences and the distance formed from them stay well inside that.
template <typename Next> __device__ inline void bpq_units(const BPDev &B, const CellGrid &g, BPQWarp &W, int first, Next next)
{
    const float thr = B.thr + 4e-6f * g.s;
    const int nh = ((volatile Ctrl *)B.ctrl)->n_units_h, nl = ((volatile Ctrl *)B.ctrl)->n_units;
    const int nu = nh + nl;
    if (nu > B.ucap) {   // the two ends of the list met: the build cannot be trusted
        if ((threadIdx.x & 31) == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
        return;
    }
    int np = 0, nout = 0;
    for (int u = first; u < nu; u = next())
        bpq_unit(B, __ldcg(B.units + (u < nh ? u : B.ucap - 1 - (u - nh))), thr, W, np, nout);
    __syncwarp();
    if (np) bpq_exact(B, W, np, thr, nout);
    bpq_flush(B, W, nout);
}

static __global__ void __launch_bounds__(BP_B) bp_query(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    __shared__ BPQWarp W[BP_B / 32];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    int u = w;
    bpq_units(B, grid_of(cell_size(B)), W[threadIdx.x >> 5], w, [&]() { return u += nw; });
}

} // namespace pncg
