// Batched form of the persistent step: many independent scenes in one launch (the vertices and tets of each scene
// contiguous, scene ids non-decreasing).  Each scene is its own PNCG problem -- own beta, direction scale, max |p_v|,
// alpha and eps rule: the per-object splitting of Sec. 5.2 applied to scenes that share no contact -- while the
// gradient pass, the candidate build and the grid barriers are shared.  With split objects the groups are objects
// of one scene: the candidate pass also pairs primitives of two objects, and such a pair's p^T H p term is split
// between the two objects (each with the other's entries of p zero).
//
// With parts (split_objects = 2) every object is divided into its collision and non-collision parts for the time
// step: group 2 o + 1 holds object o's vertices in contact at x_0 (plane: marked by the prediction; pairs: marked
// from the active set of iteration 0, before its beta phase), group 2 o the rest.  A tet or pair whose vertices lie
// in several groups adds to each of them with the other groups' entries of p zero.
//
// Per-scene sums: the lanes of a warp take consecutive vertices (tets), so their scene ids are non-decreasing (with
// parts, runs of equal ids); a segmented warp scan adds up each run of equal ids and the run's last lane adds it to
// the scene's accumulator with a double atomic.  Accumulators are used round robin over three buffers: reduction r accumulates into buffer
// r % 3 and zeroes buffer (r + 1) % 3 for the next one, which every block last read before the barrier of
// reduction r - 1.  After the barrier every block computes all scenes' scalars itself (identical values) into
// shared memory; block 0 also writes them to the per-scene state.
#pragma once

// included by persistent.cuh after its accumulators, reductions and barrier

namespace pncg {

template <typename R> __device__ inline unsigned long long max_bits(R v);
template <> __device__ inline unsigned long long max_bits<float>(float v) { return (unsigned long long)__float_as_uint(v); }
template <> __device__ inline unsigned long long max_bits<double>(double v) { return (unsigned long long)__double_as_longlong(v); }
template <typename R> __device__ inline double max_value(unsigned long long b);
template <> __device__ inline double max_value<float>(unsigned long long b) { return (double)__uint_as_float((unsigned int)b); }
template <> __device__ inline double max_value<double>(unsigned long long b) { return __longlong_as_double((long long)b); }

// The group of vertex i: its scene (object), or with parts its object's collision or non-collision part.
template <typename R> __device__ inline int group_of(const Dev<R> &D, int i)
{
    return D.cmark ? 2 * D.vscene[i] + D.cmark[i] : D.vscene[i];
}

// The distinct groups of a tet's or pair's four vertices (k[0..3]): returns their number n and u[0..n).
__device__ inline int distinct4(const int k[4], int u[4])
{
    int n = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bool seen = false;
#pragma unroll
        for (int r = 0; r < q; ++r) seen |= k[r] == k[q];
        if (!seen) u[n++] = k[q];
    }
    return n;
}

// First lane of the run of equal keys that lane `lane` belongs to (runs need not be sorted: with parts a group's
// vertices can come back after another group's).
__device__ inline int run_start(int key, int lane)
{
    const int kp = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned int heads = __ballot_sync(0xffffffffu, lane == 0 || kp != key);
    return 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
}

// Segmented sum over the warp's lanes (key < 0 = no item): the last lane of each run of equal keys adds the run's
// N sums to acc[key * 8 + q0 + q].
template <typename R, int N>
__device__ inline void seg_warp_sum(Acc<R> (&a)[N], int key, double *acc, int q0)
{
    const int lane = threadIdx.x & 31;
    const int start = run_start(key, lane);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const Acc<R> u = a[q].shfl_up(o);
            if (lane - o >= start) a[q].add(u);
        }
    }
    const int kn = __shfl_down_sync(0xffffffffu, key, 1);
    if (key >= 0 && (lane == 31 || kn != key)) {
#pragma unroll
        for (int q = 0; q < N; ++q) atomicAdd(acc + (size_t)key * 8 + q0 + q, a[q].value());
    }
}

// Segmented max of non-negative values, published as bits (monotone for non-negative floats and doubles).
template <typename R>
__device__ inline void seg_warp_max(R m, int key, unsigned long long *mx)
{
    const int lane = threadIdx.x & 31;
    const int start = run_start(key, lane);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const R mu = __shfl_up_sync(0xffffffffu, m, o);
        if (lane - o >= start) m = fmax(m, mu);
    }
    const int kn = __shfl_down_sync(0xffffffffu, key, 1);
    if (key >= 0 && (lane == 31 || kn != key)) atomicMax(mx + key, max_bits<R>(m));
}

// zeroes the accumulators reduction r + 1 will use
__device__ inline void seg_zero_next(double *sacc, unsigned long long *smax, int nseg, int r, int tid, int nthr)
{
    double *a = sacc + (size_t)((r + 1) % 3) * nseg * 8;
    unsigned long long *m = smax + (size_t)((r + 1) % 3) * nseg;
    for (int q = tid; q < nseg * 8; q += nthr) a[q] = 0.0;
    for (int q = tid; q < nseg; q += nthr) m[q] = 0ull;
}

// Resets the per-scene state at the start of a time step (block 0; iteration 0 reads parity 1).
template <typename R> __device__ inline void seg_reset(const Dev<R> &D)
{
    if (blockIdx.x != 0) return;
    for (int s = threadIdx.x; s < D.nseg; s += blockDim.x) {
        D.seg[s].gPg[1] = 0.0;
        D.seg[s].dE0[1] = 0.0;
        D.seg[s].converged[1] = 0;
        D.seg[s].iters_done = 0;
    }
}

// Beta, direction + p^T H p, and update phases of iteration k for nseg > 1 scenes (three grid barriers, as in the
// single-scene form).  sbuf holds the scenes' beta and alpha (2 x MAX_SCENES doubles).  Returns 1 when some vertex
// has moved far enough since the candidate build to need a new one.
template <typename R, int PB, bool CO>
__device__ inline int batched_tail(const Dev<R> &D, Ctrl *c, PShared<R, PB> &sh, unsigned char *sbuf, Bar &br,
                                   Stamper &st, RedBufs &rb, int k, int par, int &sred, double disp_lim)
{
    typedef typename V4<R>::T R4;
    typedef typename PartT<R>::T PT;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const int ns = D.nseg;
    const int rp = (k - 1) & 1, wp = k & 1;
    double *sbeta = reinterpret_cast<double *>(sbuf);
    double *salpha = sbeta + MAX_SCENES;

    // ------------------------------------------------------------ parts: the collision parts of the time step
    if (D.cmark && k == 0) {
        br.phase = 8;   // K_DOTS
        const int na0 = min((volatile const int &)c->n_active, D.cand_cap);
        for (int kk = tid; kk < na0; kk += nthr) {
            const int4 v = __ldcg(&D.act[kk].v);
            D.cmark[v.x] = 1; D.cmark[v.y] = 1; D.cmark[v.z] = 1; D.cmark[v.w] = 1;
        }
        grid_barrier(br, c);
    }

    // ------------------------------------------------------------ beta (per scene) and P g
    br.phase = 8;   // K_DOTS
    {
        double *acc = D.sacc + (size_t)(sred % 3) * ns * 8;
        seg_zero_next(D.sacc, D.smax, ns, sred, tid, nthr);
        for (int base = tid - lane; base < D.nv; base += nthr) {
            const int i = base + lane;
            Acc<R> a5[5];
            int key = -1;
            if (i < D.nv) {
                key = group_of(D, i);
                const R4 G = ldcg4(D.g[par] + i), Dg = ldcg4(D.dg[par] + i), G0 = ldcg4(D.g[par ^ 1] + i);
                const R4 P0 = ldcg4(D.p + i);
                R4 PG = mk4<R>(R(0), R(0), R(0), R(0));
                if (Dg.w > R(0)) {
                    const R gv[3] = {G.x, G.y, G.z}, dv[3] = {Dg.x, Dg.y, Dg.z}, g0[3] = {G0.x, G0.y, G0.z}, p0[3] = {P0.x, P0.y, P0.z};
                    R th[5], tl[5], pg[3];
                    beta_terms<R>(gv, dv, g0, p0, Dg.w, D.beta_rule, th, tl, pg);
#pragma unroll
                    for (int q = 0; q < 5; ++q) a5[q].add_ff(th[q], tl[q]);
                    PG = mk4<R>(pg[0], pg[1], pg[2], R(0));
                } else if (P0.x != R(0) || P0.y != R(0) || P0.z != R(0)) {
                    D.p[i] = PG;   // a kinematic vertex never moves along p
                }
                D.pg[i] = PG;
            }
            seg_warp_sum<R, 5>(a5, key, acc, 0);
        }
        grid_barrier(br, c);
        if (threadIdx.x == 0) sh.fi = (volatile const int &)c->n_active;
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            double t[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) t[q] = __ldcg(acc + (size_t)s * 8 + q);
            const double gprev = __ldcg(&D.seg[s].gPg[rp]);
            double bt = 0.0, gPg, gp_new;
            int rs = 0;
            if (D.beta_rule == 0) {
                gPg = t[1];
                if (k > 0) { bt = gprev > 0.0 ? t[0] / gprev : 0.0; if (bt < 0.0) bt = 0.0; }
                gp_new = -gPg + bt * t[2];
            } else {
                gPg = t[4];
                if (k > 0) bt = fabs(t[2]) < 1e-30 ? 0.0 : t[0] / t[2] - (t[1] / t[2]) * (t[3] / t[2]);
                gp_new = -gPg + bt * t[3];
            }
            if (gp_new >= 0.0 && bt != 0.0) { bt = 0.0; rs = 1; }
            sbeta[s] = bt;
            if (blockIdx.x == 0) { D.seg[s].gPg[wp] = gPg; D.seg[s].beta = bt; D.seg[s].restarted = rs; }
        }
        __syncthreads();
        st.mark(8);   // K_DOTS
        ++sred;
    }
    const int na = sh.fi;

    // ------------------------------------------------------------ direction, p^T H p and the step (per scene)
    br.phase = 10;   // K_PHP
    {
        double *acc = D.sacc + (size_t)(sred % 3) * ns * 8;
        unsigned long long *mx = D.smax + (size_t)(sred % 3) * ns;
        seg_zero_next(D.sacc, D.smax, ns, sred, tid, nthr);
        for (int base = tid - lane; base < D.nv; base += nthr) {
            const int i = base + lane;
            Acc<R> a2[3];   // g^T p, p^T M p, vertices (a group without vertices takes no step)
            R pmv = R(0);
            int key = -1;
            if (i < D.nv) {
                key = group_of(D, i);
                a2[2].add(R(1));
                const double bd = sbeta[key];
                const R4 Dg = ldcg4(D.dg[par] + i);
                R4 Pn = mk4<R>(R(0), R(0), R(0), R(0));
                if (Dg.w > R(0)) {
                    const R4 G = ldcg4(D.g[par] + i);
                    Pn = dir_of<R>(D, i, R(bd), bd != 0.0);
                    const R px = Pn.x, py = Pn.y, pz = Pn.z;
                    a2[0].add(G.x * px + G.y * py + G.z * pz);
                    R mp = Dg.w * (px * px + py * py + pz * pz);
                    if (D.has_plane && G.w != R(0)) {
                        const R np = R(D.pn[0]) * px + R(D.pn[1]) * py + R(D.pn[2]) * pz;
                        mp += G.w * np * np;
                    }
                    a2[1].add(mp);
                    pmv = D.pnorm == 0 ? sqrt(px * px + py * py + pz * pz) : fmax(fabs(px), fmax(fabs(py), fabs(pz)));
                }
                D.pnext[i] = Pn;
            }
            seg_warp_sum<R, 3>(a2, key, acc, 0);
            seg_warp_max<R>(pmv, key, mx);
        }
        for (int base = tid - lane; base < D.nt; base += nthr) {
            const int e = base + lane;
            Acc<R> a1[1];
            int key = -1;
            if (e < D.nt) {
                const int4 tv = D.tet[e];
                const int vv[4] = {tv.x, tv.y, tv.z, tv.w};
                int ks[4];
                R4 pv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {   // each vertex takes the direction of its own group
                    ks[q] = group_of(D, vv[q]);
                    const double bd = sbeta[ks[q]];
                    pv[q] = dir_of<R>(D, vv[q], R(bd), bd != 0.0);
                }
                if (ks[1] == ks[0] && ks[2] == ks[0] && ks[3] == ks[0]) {
                    key = ks[0];
                    a1[0].add(tet_pHp_vec<R, CO>(D, e, tv, pv[0], pv[1], pv[2], pv[3]));
                } else {   // a tet on the border of two parts: one term per group, the others' p zero
                    const R4 z = mk4<R>(R(0), R(0), R(0), R(0));
                    int u[4];
                    const int nu = distinct4(ks, u);
                    for (int j = 0; j < nu; ++j)
                        atomicAdd(acc + (size_t)u[j] * 8 + 3,
                                  (double)tet_pHp_vec<R, CO>(D, e, tv, ks[0] == u[j] ? pv[0] : z, ks[1] == u[j] ? pv[1] : z,
                                                             ks[2] == u[j] ? pv[2] : z, ks[3] == u[j] ? pv[3] : z));
                }
            }
            seg_warp_sum<R, 1>(a1, key, acc, 4);
        }
        for (int kk = tid; kk < na; kk += nthr) {   // active pairs come in no order: one atomic each
            Active<R> ap;
            load_active<R>(D, kk, ap);
            const int vv[4] = {ap.v.x, ap.v.y, ap.v.z, ap.v.w};
            int ks[4];
            R4 pv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // each vertex takes the direction of its own group
                ks[q] = group_of(D, vv[q]);
                const double bd = sbeta[ks[q]];
                pv[q] = dir_of<R>(D, vv[q], R(bd), bd != 0.0);
            }
            // a pair whose vertices lie in several groups (objects, or parts) adds to each group's p^T H p with
            // the other groups' entries of p zero
            int u[4];
            const int nu = distinct4(ks, u);
            if (nu == 1) {
                atomicAdd(acc + (size_t)u[0] * 8 + 3, pair_pHp_vec<R>(ap, pv[0], pv[1], pv[2], pv[3]));
            } else {
                const R4 z = mk4<R>(R(0), R(0), R(0), R(0));
                for (int j = 0; j < nu; ++j)
                    atomicAdd(acc + (size_t)u[j] * 8 + 3,
                              pair_pHp_vec<R>(ap, ks[0] == u[j] ? pv[0] : z, ks[1] == u[j] ? pv[1] : z,
                                              ks[2] == u[j] ? pv[2] : z, ks[3] == u[j] ? pv[3] : z));
            }
        }
        grid_barrier(br, c);
        if (threadIdx.x == 0) sh.fe = (volatile const uint32_t &)c->err;
        __syncthreads();
        const uint32_t err = sh.fe;
        int ncap = 0;
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const double gp = __ldcg(acc + (size_t)s * 8), pMp = __ldcg(acc + (size_t)s * 8 + 1);
            const bool empty = __ldcg(acc + (size_t)s * 8 + 2) == 0.0;
            const double pHp = __ldcg(acc + (size_t)s * 8 + 4) + __ldcg(acc + (size_t)s * 8 + 3) + pMp;
            const double pmax = max_value<R>(__ldcg(mx + s));
            const double au = pmax > 0.0 ? D.dhat / (2.0 * pmax) : 0.0;
            const double ab = -gp / pHp;
            double a;
            int capped;
            if (empty) { a = 0.0; capped = 0; }
            else if (!(pHp > 0.0) || !isfinite(ab)) { a = au; capped = 1; }
            else if (ab < au) { a = ab; capped = 0; }
            else { a = au; capped = 1; }
            const double dE = -a * gp - 0.5 * a * a * pHp;
            bool bad = err != 0u;
            if (!isfinite(a) || !isfinite(gp)) { flag_error(c, ERR_NONFINITE); bad = true; }
            const int cprev = k > 0 ? __ldcg(&D.seg[s].converged[rp]) : 0;
            double e0 = k > 0 ? __ldcg(&D.seg[s].dE0[rp]) : 0.0;
            if (bad || cprev) a = 0.0;
            int cv = cprev | (empty ? 1 : 0);
            if (!cv && !bad) {
                if (k == 0) e0 = dE;
                if (D.eps > 0.0 && dE < D.eps * e0) cv = 1;
            }
            salpha[s] = a;
            if (blockIdx.x == 0) {
                SegCtl &g = D.seg[s];
                g.gp = gp; g.pHp = pHp; g.pmax = pmax; g.alpha = a; g.dE = dE; g.capped = capped;
                g.dE0[wp] = e0;
                g.converged[wp] = cv;
                if (!cprev && !bad) { g.iters_done = k + 1; ncap += capped; }
            }
        }
        if (blockIdx.x == 0 && ncap) atomicAdd(&c->n_capped, ncap);
        if (lead) {
            c->k = k + 1;
            c->n_active_last = na;
            if (err == 0u) c->iters_done = k + 1;
        }
        __syncthreads();
        st.mark(10);  // K_PHP (direction included)
        ++sred;
    }

    // ------------------------------------------------------------ update (per-scene alpha)
    br.phase = 11;   // K_UPDATE
    R md = R(0);
    for (int i = tid; i < D.nv; i += nthr) {
        double4_32a X = ldcg4(D.x + i);
        const R4 P = ldcg4(D.pnext + i);
        const double a = salpha[group_of(D, i)];
        if constexpr (sizeof(R) == 4) {
            const ffl as = ff_split(a);
            const float4 xh = update_vertex<R>(D, i, X, P, a, as.h, as.l, X, par ^ 1);
            const float4 b = ldcg4(D.xbh + i);
            const float dx = xh.x - b.x, dy = xh.y - b.y, dz = xh.z - b.z;
            md = fmax(md, dx * dx + dy * dy + dz * dz);
        } else {
            update_vertex<R>(D, i, X, P, a, 0.0f, 0.0f, ldcg4(D.xtil + i), par ^ 1);
            md = fmax(md, (R)disp2<R>(D, i, X));
        }
        D.p[i] = P;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) c->n_active = 0;
    const R m = grid_max<R, PB>(md, rb.max_region<PT, R>(), sh, br, c);
    st.mark(11);  // K_UPDATE
    return (double)m >= disp_lim * disp_lim ? 1 : 0;
}

} // namespace pncg
