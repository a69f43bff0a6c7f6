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
//   bp_fill   : entries (cell key, primitive, a copy of the primitive's box) in bucket order, and each bucket's
//               global first entry
//   bp_query  : per surface vertex (PT) and per edge (EE) lookup, exact cell-key match, box test, then the exact
//               distance at the build positions: only pairs with d < (dhat + r)(1 + 1e-3) become candidates
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
    int *eprim;             // triangle f or -1 - edge
    float4 *eblo, *ebhi;    // the entry's primitive box (streamed with the key instead of gathered)
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
__device__ inline bool cell_of(float q, float s, int &i)
{
    float f = floorf(q / s);
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
__device__ inline void for_cells(const BPDev &B, float4 lo, float4 hi, float s, F f)
{
    int l[3], h[3];
    if (!cell_of(lo.x, s, l[0]) || !cell_of(lo.y, s, l[1]) || !cell_of(lo.z, s, l[2]) || !cell_of(hi.x, s, h[0]) ||
        !cell_of(hi.y, s, h[1]) || !cell_of(hi.z, s, h[2])) {
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
    const float s = cell_size(B);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.nf + B.ne) return;
    for_cells(B, B.blo[j], B.bhi[j], s, [&](int i, int jj, int k) { atomicAdd(&B.cnt[prim_bucket(B, j, i, jj, k)], 1u); });
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
    const float s = cell_size(B);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < 2 * B.H; b += gridDim.x * blockDim.x)
        B.goff[b] = B.boff[b / BP_SCAN_N] + B.off[b];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B.nf + B.ne) return;
    const int prim = j < B.nf ? j : -1 - (j - B.nf);
    const float4 lo = B.blo[j], hi = B.bhi[j];
    for_cells(B, lo, hi, s, [&](int i, int jj, int k) {
        const unsigned int b = prim_bucket(B, j, i, jj, k);
        const unsigned int slot = B.boff[b / BP_SCAN_N] + B.off[b] + atomicAdd(&B.cnt[b], 1u);
        if (slot >= (unsigned int)B.ecap) { atomicOr(&B.ctrl->err, ERR_RANGE); return; }
        B.ekey[slot] = cell_key(i, jj, k);
        B.eprim[slot] = prim;
        B.eblo[slot] = lo;
        B.ebhi[slot] = hi;
    });
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

// distance of a pair at the build positions, float arithmetic on double differences (the threshold carries a
// 1e-3 relative margin, far above the float error of d)
__device__ inline float pair_dist_build(const BPDev &B, bool ee, int a, int b, int c, int d)
{
    const double4_32a X0 = ldcg4(B.x + a), X1 = ldcg4(B.x + b), X2 = ldcg4(B.x + c), X3 = ldcg4(B.x + d);
    float cc[4];
    v3<float> t;
    if (!ee) {
        return pt_coeffs<float>(rel<float>(X0.x, X0.y, X0.z, X1.x, X1.y, X1.z), rel<float>(X2.x, X2.y, X2.z, X1.x, X1.y, X1.z),
                                rel<float>(X3.x, X3.y, X3.z, X1.x, X1.y, X1.z), cc, t);
    }
    return ee_coeffs<float>(rel<float>(X0.x, X0.y, X0.z, X2.x, X2.y, X2.z), rel<float>(X1.x, X1.y, X1.z, X2.x, X2.y, X2.z),
                            rel<float>(X3.x, X3.y, X3.z, X2.x, X2.y, X2.z), cc, t);
}

__device__ inline void emit(const BPDev &B, int4 c)
{
    const int slot = atomicAdd(&B.ctrl->n_cand, 1);
    if (slot < B.cap) B.cand[slot] = c;
}

// Query j (a surface vertex for j < ns, else edge j - ns) by one warp.  The lanes take consecutive entries of the
// query's buckets (an edge's buckets are concatenated, so no lane idles at the end of a short bucket), and each
// lane loads an entry's key, primitive and box together.
__device__ inline void bp_query_one(const BPDev &B, int j, float s)
{
    const int lane = threadIdx.x & 31;
    if (j < B.ns) {
        // point-triangle: the point's own cell
        const int v = B.svert[j];
        const double4_32a X = ldcg4(B.x + v);
        const float qx = (float)X.x, qy = (float)X.y, qz = (float)X.z;
        int ix, iy, iz;
        if (!cell_of(qx, s, ix) || !cell_of(qy, s, iy) || !cell_of(qz, s, iz)) {
            if (lane == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
            return;
        }
        const unsigned long long key = cell_key(ix, iy, iz);
        const unsigned int b = cell_hash(ix, iy, iz, B.H);                 // the triangle table
        const unsigned int st = __ldcg(B.goff + b);
        const unsigned int en = min(st + __ldcg(B.cnt + b), (unsigned int)B.ecap);   // a fill overflow is flagged
        const int ov = B.obj[v];
        for (unsigned int q = st + lane; q < en; q += 32) {
            const unsigned long long ek = __ldcg(B.ekey + q);
            const float4 lo = __ldcg(B.eblo + q), hi = __ldcg(B.ebhi + q);
            const int f = __ldcg(B.eprim + q);
            if (ek != key) continue;
            if (qx < lo.x || qx > hi.x || qy < lo.y || qy > hi.y || qz < lo.z || qz > hi.z) continue;
            const int4 t = B.tri[f];
            if (t.x == v || t.y == v || t.z == v) continue;
            if (B.vscene && B.vscene[t.x] != B.vscene[v]) continue;
            if (B.nexcl && t.w == ov && is_excluded(B, ((unsigned long long)j << 31) | (unsigned long long)f)) continue;
            if (!(pair_dist_build(B, false, v, t.x, t.y, t.z) < B.thr)) continue;
            emit(B, make_int4(v, t.x, t.y, t.z));
        }
    } else if (j < B.ns + B.ne) {
        // edge-edge: cells of the edge's own box (at most 2 per axis: the box is no wider than a cell); a pair is
        // emitted from the cell holding the lower corner of the intersection of the two boxes only
        const int a = j - B.ns;
        const int4 e = B.edge[a];
        int vv[2] = {e.x, e.y};
        float4 lo, hi;
        box_of(B.x, vv, 2, 0.0, lo, hi);
        int l[3], h[3];
        if (!cell_of(lo.x, s, l[0]) || !cell_of(lo.y, s, l[1]) || !cell_of(lo.z, s, l[2]) || !cell_of(hi.x, s, h[0]) ||
            !cell_of(hi.y, s, h[1]) || !cell_of(hi.z, s, h[2])) {
            if (lane == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
            return;
        }
        const int nx = h[0] - l[0] + 1, ny = h[1] - l[1] + 1, nz = h[2] - l[2] + 1;
        const int ncell = nx * ny * nz;
        if (ncell > 8) {
            if (lane == 0) atomicOr(&B.ctrl->err, ERR_RANGE);
            return;
        }
        // lane c < ncell holds cell c's coordinates, first entry and entry count
        int cx = 0, cy = 0, cz = 0;
        unsigned int cst = 0, clen = 0;
        if (lane < ncell) {
            cx = l[0] + lane % nx;
            cy = l[1] + (lane / nx) % ny;
            cz = l[2] + lane / (nx * ny);
            const unsigned int b = cell_hash(cx, cy, cz, B.H) + (unsigned int)B.H;   // the edge table
            cst = __ldcg(B.goff + b);
            clen = __ldcg(B.cnt + b);
        }
        unsigned int inc = clen;   // inclusive prefix of the counts over lanes 0..7
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned int n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, inc, 7);
        // item it of the concatenated buckets: its cell (by the prefix of the counts) and its entry; the next
        // round's entries are loaded before the current round is tested
        struct Item { unsigned long long ek, key; float4 lo, hi; int bi; int ix, iy, iz; bool ok; };
        auto fetch = [&](unsigned int base) {
            Item r;
            const unsigned int it = base + lane;
            int c = 0;   // the cell of item it: the number of cells whose entries all come before it
#pragma unroll
            for (int k = 0; k < 8; ++k) c += (__shfl_sync(0xffffffffu, inc, k) <= it) ? 1 : 0;
            c = min(c, 7);
            const unsigned int c_inc = __shfl_sync(0xffffffffu, inc, c), c_len = __shfl_sync(0xffffffffu, clen, c);
            const unsigned int c_st = __shfl_sync(0xffffffffu, cst, c);
            r.ix = __shfl_sync(0xffffffffu, cx, c);
            r.iy = __shfl_sync(0xffffffffu, cy, c);
            r.iz = __shfl_sync(0xffffffffu, cz, c);
            const unsigned int q = c_st + (it - (c_inc - c_len));
            r.ok = it < total && q < (unsigned int)B.ecap;   // a fill overflow is flagged
            if (r.ok) {
                r.ek = __ldcg(B.ekey + q);
                r.lo = __ldcg(B.eblo + q);
                r.hi = __ldcg(B.ebhi + q);
                r.bi = -1 - __ldcg(B.eprim + q);
                r.key = cell_key(r.ix, r.iy, r.iz);
            }
            return r;
        };
        Item cur = fetch(0);
        for (unsigned int base = 0; base < total; base += 32) {
            Item nxt;
            nxt.ok = false;
            if (base + 32 < total) nxt = fetch(base + 32);   // warp-uniform
            do {
                if (!cur.ok || cur.ek != cur.key || cur.bi <= a) break;
                const float4 ilo = cur.lo, ihi = cur.hi;
                if (lo.x > ihi.x || hi.x < ilo.x || lo.y > ihi.y || hi.y < ilo.y || lo.z > ihi.z || hi.z < ilo.z) break;
                int kx, ky, kz;
                cell_of(fmaxf(lo.x, ilo.x), s, kx);
                cell_of(fmaxf(lo.y, ilo.y), s, ky);
                cell_of(fmaxf(lo.z, ilo.z), s, kz);
                if (kx != cur.ix || ky != cur.iy || kz != cur.iz) break;
                const int bi = cur.bi;
                const int4 f = B.edge[bi];
                if (f.x == e.x || f.x == e.y || f.y == e.x || f.y == e.y) break;
                if (B.vscene && B.vscene[f.x] != B.vscene[e.x]) break;
                if (B.nexcl && f.z == e.z &&
                    is_excluded(B, (1ull << 62) | ((unsigned long long)a << 31) | (unsigned long long)bi))
                    break;
                if (!(pair_dist_build(B, true, e.x, e.y, f.x, f.y) < B.thr)) break;
                emit(B, make_int4(-1 - e.x, e.y, f.x, f.y));
            } while (false);
            cur = nxt;
        }
    }
}

// One warp per query primitive.
static __global__ void __launch_bounds__(BP_B) bp_query(BPDev B)
{
    if (!B.ctrl->rebuild) return;
    bp_query_one(B, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, cell_size(B));
}

} // namespace pncg
