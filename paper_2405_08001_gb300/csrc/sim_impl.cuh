// SimImpl<R>: device buffers, launch sequence and CUDA-graph replay of one time step (Algorithm 1).
#pragma once

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "broadphase.cuh"
#include "kernels.cuh"
#include "persist_shapes.cuh"
#include "adjoint.cuh"
#include "sim.h"

namespace pncg {

// [n][3] AoS <-> double4_32a conversions for the ABI's position arrays
static __global__ void k_pack4(const double *in, double4_32a *out, int n, int keep_w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double w = keep_w ? out[i].w : 0.0;
    out[i] = make_double4_32a(in[3 * i], in[3 * i + 1], in[3 * i + 2], w);
}
static __global__ void k_unpack4(const double4_32a *in, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4_32a v = in[i];
    out[3 * i] = v.x; out[3 * i + 1] = v.y; out[3 * i + 2] = v.z;
}
template <typename R4> __global__ void k_unpackR(const R4 *in, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const R4 v = in[i];
    out[3 * i] = double(v.x); out[3 * i + 1] = double(v.y); out[3 * i + 2] = double(v.z);
}
// writes R4 from [n][3] doubles keeping w
template <typename R4, typename R> __global__ void k_packR(const double *in, R4 *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R4 v = out[i];
    v.x = R(in[3 * i]); v.y = R(in[3 * i + 1]); v.z = R(in[3 * i + 2]);
    out[i] = v;
}
// P = diag^-1 as the direction kernel forms it (kinematic: 0)
template <typename R4, typename R> __global__ void k_precond_out(const R4 *dg, double *out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const R4 d = dg[i];
    if (!(d.w > R(0))) { out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0; return; }
    out[3 * i] = double(precond<R>(d.x, d.w));
    out[3 * i + 1] = double(precond<R>(d.y, d.w));
    out[3 * i + 2] = double(precond<R>(d.z, d.w));
}
// inertia / plane initialisation of parity par at the current x (after the caller changed x or xtil)
template <typename R> __global__ void k_reinit(Dev<R> D, int par)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nv) return;
    init_vertex<R>(D, i, D.x[i], D.xtil[i], par);
}
// refreshes the FP32 form's float-float copies of x and x~ after the host wrote either
template <typename R> __global__ void k_refresh_ff(Dev<R> D)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D.nv) {
        put_x<R>(D, i, D.x[i]);
        put_xt<R>(D, i, D.xtil[i]);
    }
}
// xtil.w = mass for every vertex (unmasked evaluation)
static __global__ void k_set_mass_w(double4_32a *xt, const double *mass, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xt[i].w = mass[i];
}
// p^T M p + plane part for sim_eval_pHp: written to ctrl->pHp_vert
template <typename R> __global__ void __launch_bounds__(VB) k_eval_vert_pHp(Dev<R> D, int par)
{
    __shared__ double sh[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s[1] = {0.0};
    if (i < D.nv) {
        const typename V4<R>::T P = D.p[i], G = D.g[par][i];
        const double px = P.x, py = P.y, pz = P.z;
        s[0] = D.mass[i] * (px * px + py * py + pz * pz);
        if (D.has_plane && G.w != R(0)) {
            const double np = D.pn[0] * px + D.pn[1] * py + D.pn[2] * pz;
            s[0] += double(G.w) * np * np;
        }
    }
    block_sum<1>(s, sh);
    if (publish_partials<1>(s, D.part, &D.ctrl->ticket[TK_MISC])) {
        double t[1];
        finish_sums<1>(t, D.part, sh);
        if (threadIdx.x == 0) D.ctrl->pHp_vert = t[0];
    }
}
// p^T H p (tets + active pairs) only, for sim_eval_pHp: ctrl->pHp = sum + pHp_vert
template <typename R, bool CO = false> __global__ void __launch_bounds__(EB) k_eval_pHp(Dev<R> D, int ntb)
{
    __shared__ double sh[32];
    double sdd[1] = {0.0};
    if ((int)blockIdx.x < ntb) {
        R s[1] = {R(0)};
        const int e = blockIdx.x * blockDim.x + threadIdx.x;
        if (e < D.nt) s[0] = tet_pHp<R, CO>(D, e);
        block_sum_acc<1>(s, sdd, sh);
    } else {
        const int na = D.ctrl->n_active;
        const int stride = (gridDim.x - ntb) * blockDim.x;
        for (int k = (blockIdx.x - ntb) * blockDim.x + threadIdx.x; k < na; k += stride) sdd[0] += pair_pHp<R>(D, k);
        block_sum<1>(sdd, sh);
    }
    if (publish_partials<1>(sdd, D.part, &D.ctrl->ticket[TK_PHP])) {
        double t[1];
        finish_sums<1>(t, D.part, sh);
        if (threadIdx.x == 0) D.ctrl->pHp = t[0] + D.ctrl->pHp_vert;
    }
}
static __global__ void k_copy_count(Ctrl *c) { c->n_active_last = c->n_active; }

#define AL3(p, n) do { sim_status st_ = dalloc(p, n); if (st_ != SIM_OK) return st_; } while (0)
#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call, __LINE__);                 \
    } while (0)

template <typename R> class SimImpl : public Sim {
    typedef typename V4<R>::T R4;

public:
    ~SimImpl() override { release(); }

    sim_status init(const HostMesh &m) override
    {
        M = m;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (M.opt.cuda_stream) { s = (cudaStream_t)M.opt.cuda_stream; own_stream = false; }
        else { CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); own_stream = true; }
        cap = M.opt.candidate_capacity > 0 ? M.opt.candidate_capacity : std::max(1 << 14, 16 * (M.ns + M.ne));
        sim_status st = alloc_all();
        if (st != SIM_OK) return st;
        if (M.nseg > 1 && !persist)
            return fail(SIM_ERR_INVALID_ARG, "batched scenes and split objects need the persistent form "
                                             "(options.persistent = 1 on a device with cooperative launch)");
        return upload_initial();
    }

    // ------------------------------------------------------------------------------------------ stepping
    sim_status step(int n, const double *targets, bool sync) override
    {
        CK(cudaSetDevice(dev));
        if (n < 0) return fail(SIM_ERR_INVALID_ARG, "n_steps < 0");
        if (M.opt.use_graph && !gexec) {
            sim_status st = capture();
            if (st != SIM_OK) return st;
        }
        for (int k = 0; k < n; ++k) {
            sim_status st = stage_targets(targets ? targets + (size_t)k * 3 * M.nfix : nullptr);
            if (st != SIM_OK) return st;
            if (tune_next >= 0 && steps_run >= 1) {
                st = tuned_step();
                if (st != SIM_OK) return st;
                ++steps_run;
                continue;
            }
            if (gexec) { CK(cudaGraphLaunch(gexec, s)); k_host = M.opt.iters; }
            else {
                st = launch_step();
                if (st != SIM_OK) return st;
            }
            ++steps_run;
        }
        if (!sync) return SIM_OK;
        return sync_and_check();
    }

    // Autotuning: the candidates are block shapes of the persistent form (options.block_shape = -1) and, with
    // options.persistent = 2, the per-phase form; from the second time step on each candidate runs TUNE_REPS time
    // steps, interleaved (c0, c1, .., c0, c1, ..), each timed on the GPU with events on the solver's stream, and the
    // candidate with the fastest step is kept.  Every tuned step is an ordinary time step of the simulation.
    static constexpr int TUNE_REPS = 2;
    void drop_graph()
    {
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    }
    // candidate c: a shape index >= 0 (persistent form) or -1 (one kernel per phase)
    void apply_config(int c)
    {
        const bool want_persist = c >= 0;
        const int want_shape = c >= 0 ? c : shape;
        if (persist != want_persist || shape != want_shape) {
            persist = want_persist;
            shape = want_shape;
            pgrid = shape_grid[shape];
            drop_graph();
        }
    }
    sim_status tuned_step()
    {
        const int nc = (int)tune_cfg.size(), cand = tune_next % nc;
        apply_config(tune_cfg[cand]);
        if (M.opt.use_graph && !gexec) {
            sim_status st = capture();
            if (st != SIM_OK) return st;
        }
        if (!tune_ev[0]) {
            CK(cudaEventCreate(&tune_ev[0]));
            CK(cudaEventCreate(&tune_ev[1]));
        }
        CK(cudaEventRecord(tune_ev[0], s));
        if (gexec) { CK(cudaGraphLaunch(gexec, s)); k_host = M.opt.iters; }
        else {
            sim_status st = launch_step();
            if (st != SIM_OK) return st;
        }
        CK(cudaEventRecord(tune_ev[1], s));
        CK(cudaEventSynchronize(tune_ev[1]));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, tune_ev[0], tune_ev[1]));
        if ((int)tune_ms.size() < nc) tune_ms.assign(nc, 3.0e38f);
        tune_ms[cand] = std::min(tune_ms[cand], ms);
        if (++tune_next == TUNE_REPS * nc) {
            int best = 0;
            for (int i = 1; i < nc; ++i)
                if (tune_ms[i] < tune_ms[best]) best = i;
            apply_config(tune_cfg[best]);
            tune_next = -1;
        }
        return SIM_OK;
    }

    sim_status begin_step(const double *targets) override
    {
        CK(cudaSetDevice(dev));
        sim_status st = stage_targets(targets);
        if (st != SIM_OK) return st;
        if (persist) CK(launch_persistent(1, 0, 0, 0));
        else launch_predict();
        k_host = 0;
        CK(cudaGetLastError());
        return SIM_OK;
    }

    sim_status iterate(int n) override
    {
        CK(cudaSetDevice(dev));
        if (persist && n > 0) {
            CK(launch_persistent(0, k_host, n, 0));
            k_host += n;
        } else {
            for (int i = 0; i < n; ++i) { launch_iteration(k_host & 1); ++k_host; }
        }
        CK(cudaGetLastError());
        return SIM_OK;
    }

    sim_status end_step() override
    {
        CK(cudaSetDevice(dev));
        launch_finish();
        CK(cudaGetLastError());
        return sync_and_check();
    }

    // ------------------------------------------------------------------------------------------ state I/O
    sim_status get_state(double *x, double *v, sim_stats *st) override
    {
        CK(cudaSetDevice(dev));
        if (x) { sim_status r = out3(D.x, x); if (r) return r; }
        if (v) { sim_status r = out3(D.v, v); if (r) return r; }
        sim_status r = sync_and_check();
        if (st) {
            std::memset(st, 0, sizeof *st);
            st->step = hctrl->step;
            st->iters_done = hctrl->iters_done;
            st->n_candidates = hctrl->n_cand;
            st->n_active = hctrl->n_active_last;
            st->n_rebuilds = hctrl->n_rebuilds;
            st->n_capped = hctrl->n_capped;
            st->n_surface_tris = M.nf; st->n_surface_edges = M.ne; st->n_surface_verts = M.ns;
            st->dE0 = hctrl->dE0;
            st->dE_last = hctrl->dE;
            st->launch_form = persist ? 1 : 0;
            st->block_threads = persist ? PSHAPE_PB[shape] : 0;
            st->blocks_per_sm = persist ? pgrid / nsm : 0;
            st->n_scenes = M.nseg;
            st->n_near_fp64 = hctrl->n_near64;
            st->n_colors = M.color_off.empty() ? 0 : (int)M.color_off.size() - 1;
        }
        return r;
    }

    sim_status set_state(const double *x, const double *v) override
    {
        CK(cudaSetDevice(dev));
        if (x) { sim_status r = in3(x, D.x); if (r) return r; }
        if (v) { sim_status r = in3(v, D.v); if (r) return r; }
        force_rebuild();
        CK(cudaStreamSynchronize(s));
        return SIM_OK;
    }

    sim_status get_iterate(double *x, double *g, double *P, double *p, double *xt, sim_iter_scalars *sc) override
    {
        CK(cudaSetDevice(dev));
        const int lp = (k_host - 1) & 1;   // parity of the last completed iteration
        const int nb = (M.nv + 255) / 256;
        if (x) { sim_status r = out3(D.x, x); if (r) return r; }
        if (xt) { sim_status r = out3(D.xtil, xt); if (r) return r; }
        if (g) { k_unpackR<R4><<<nb, 256, 0, s>>>(D.g[lp], stage, M.nv); CK(cudaMemcpyAsync(g, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); CK(cudaStreamSynchronize(s)); }
        if (P) { k_precond_out<R4, R><<<nb, 256, 0, s>>>(D.dg[lp], stage, M.nv); CK(cudaMemcpyAsync(P, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); CK(cudaStreamSynchronize(s)); }
        if (p) { k_unpackR<R4><<<nb, 256, 0, s>>>(D.p, stage, M.nv); CK(cudaMemcpyAsync(p, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); CK(cudaStreamSynchronize(s)); }
        sim_status r = sync_and_check();
        if (sc) {
            std::memset(sc, 0, sizeof *sc);
            sc->k = hctrl->k; sc->restarted = hctrl->restarted; sc->capped = hctrl->capped;
            sc->n_active = hctrl->n_active_last;
            sc->beta = hctrl->beta; sc->gp = hctrl->gp; sc->pHp = hctrl->pHp; sc->pmax = hctrl->pmax;
            sc->alpha_bar = hctrl->alpha_bar; sc->alpha_up = hctrl->alpha_up; sc->alpha = hctrl->alpha;
            sc->dE = hctrl->dE; sc->dE0 = hctrl->dE0;
        }
        return r;
    }

    sim_status set_iterate(const double *x, const double *g, const double *P, const double *p, int k,
                           double gPg) override
    {
        (void)P;
        CK(cudaSetDevice(dev));
        if (k < 0) return fail(SIM_ERR_INVALID_ARG, "k < 0");
        const int nb = (M.nv + 255) / 256;
        if (x) { sim_status r = in3(x, D.x); if (r) return r; }
        if (g) { CK(cudaMemcpyAsync(stage, g, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); k_packR<R4, R><<<nb, 256, 0, s>>>(stage, D.g[(k - 1) & 1], M.nv); }
        if (p) { CK(cudaMemcpyAsync(stage, p, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); k_packR<R4, R><<<nb, 256, 0, s>>>(stage, D.p, M.nv); }
        k_reinit<R><<<nb, 256, 0, s>>>(D, k & 1);
        CK(cudaStreamSynchronize(s));
        hctrl_sync_read();
        hctrl->k = k;
        hctrl->gPg_prev = gPg;
        CK(cudaMemcpy(&dctrl->k, &hctrl->k, sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(&dctrl->gPg_prev, &hctrl->gPg_prev, sizeof(double), cudaMemcpyHostToDevice));
        force_rebuild();
        k_host = k;
        CK(cudaStreamSynchronize(s));
        return SIM_OK;
    }

    // ------------------------------------------------------------------------------------------ evaluations
    // Runs the candidate build and the gradient pass at the given x (and xtilde) with all vertices free.
    sim_status eval_setup(const double *x, const double *xt)
    {
        CK(cudaMemcpyAsync(xsave, D.x, sizeof(double4_32a) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(xtsave, D.xtil, sizeof(double4_32a) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        sim_status r = in3(x, D.x);
        if (r) return r;
        if (xt) { r = in3(xt, D.xtil); if (r) return r; }
        const int nb = (M.nv + 255) / 256;
        k_set_mass_w<<<nb, 256, 0, s>>>(D.xtil, D.mass, M.nv);
        refresh_ff();
        k_reinit<R><<<nb, 256, 0, s>>>(D, 0);
        force_rebuild();
        zero_active();
        zero_near64();
        launch_bp();
        launch_grad(0);
        k_copy_count<<<1, 1, 0, s>>>(dctrl);
        CK(cudaGetLastError());
        return SIM_OK;
    }
    sim_status eval_restore()
    {
        CK(cudaMemcpyAsync(D.x, xsave, sizeof(double4_32a) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(D.xtil, xtsave, sizeof(double4_32a) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        refresh_ff();
        force_rebuild();
        zero_active();
        return SIM_OK;
    }

    sim_status eval_gradient(const double *x, const double *xt, double *g, double *d) override
    {
        CK(cudaSetDevice(dev));
        if (!x || !xt) return fail(SIM_ERR_INVALID_ARG, "x and xtilde are required");
        sim_status r = eval_setup(x, xt);
        if (r) return r;
        const int nb = (M.nv + 255) / 256;
        if (g) { k_unpackR<R4><<<nb, 256, 0, s>>>(D.g[0], stage, M.nv); CK(cudaMemcpyAsync(g, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); CK(cudaStreamSynchronize(s)); }
        if (d) { k_unpackR<R4><<<nb, 256, 0, s>>>(D.dg[0], stage, M.nv); CK(cudaMemcpyAsync(d, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s)); CK(cudaStreamSynchronize(s)); }
        eval_restore();
        return sync_and_check();
    }

    sim_status eval_pHp(const double *x, const double *p, double *out) override
    {
        CK(cudaSetDevice(dev));
        if (!x || !p || !out) return fail(SIM_ERR_INVALID_ARG, "x, p and out are required");
        // xtilde does not enter p^T H p: keep the current one
        sim_status r = eval_setup(x, nullptr);
        if (r) return r;
        const int nb = (M.nv + 255) / 256;
        CK(cudaMemcpyAsync(psave, D.p, sizeof(R4) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(stage, p, 24 * (size_t)M.nv, cudaMemcpyDefault, s));
        k_packR<R4, R><<<nb, 256, 0, s>>>(stage, D.p, M.nv);
        k_eval_vert_pHp<R><<<nvb, VB, 0, s>>>(D, 0);
        if (corot) k_eval_pHp<R, true><<<ntb + npb, EB, 0, s>>>(D, ntb);
        else k_eval_pHp<R><<<ntb + npb, EB, 0, s>>>(D, ntb);
        CK(cudaMemcpyAsync(D.p, psave, sizeof(R4) * (size_t)M.nv, cudaMemcpyDeviceToDevice, s));
        eval_restore();
        r = sync_and_check();
        *out = hctrl->pHp;
        return r;
    }

    sim_status eval_energy(const double *x, const double *xt, double *out, double *parts) override
    {
        CK(cudaSetDevice(dev));
        if (!x || !xt || !out) return fail(SIM_ERR_INVALID_ARG, "x, xtilde and out are required");
        sim_status r = eval_setup(x, xt);
        if (r) return r;
        k_energy<R><<<ntb + nvb + npb, EB, 0, s>>>(D, ntb, (M.nv + EB - 1) / EB);
        eval_restore();
        r = sync_and_check();
        double e = 0;
        for (int q = 0; q < 4; ++q) { e += hctrl->energy[q]; if (parts) parts[q] = hctrl->energy[q]; }
        *out = e;
        return r;
    }

    sim_status get_contacts(int32_t *idx, double *d, int32_t max, int32_t *count) override
    {
        CK(cudaSetDevice(dev));
        sim_status r = sync_and_check();
        const int n = hctrl->n_active_last;
        if (count) *count = n;
        const int m = std::min(n, std::max(max, 0));
        if (m > 0 && idx) {
            std::vector<Active<R>> h(m);
            CK(cudaMemcpy(h.data(), D.act, sizeof(Active<R>) * (size_t)m, cudaMemcpyDeviceToHost));
            for (int i = 0; i < m; ++i) {
                idx[5 * i] = h[i].ty;
                idx[5 * i + 1] = h[i].v.x; idx[5 * i + 2] = h[i].v.y; idx[5 * i + 3] = h[i].v.z; idx[5 * i + 4] = h[i].v.w;
                if (d) d[i] = double(h[i].d);
            }
        }
        return r;
    }

    sim_status get_candidates(int32_t *idx, int32_t max, int32_t *count) override
    {
        CK(cudaSetDevice(dev));
        sim_status r = sync_and_check();
        const int n = std::min(hctrl->n_cand, cap);
        if (count) *count = hctrl->n_cand;
        const int m = std::min(n, std::max(max, 0));
        if (m > 0 && idx) {
            std::vector<int4> h(m);
            CK(cudaMemcpy(h.data(), D.cand, sizeof(int4) * (size_t)m, cudaMemcpyDeviceToHost));
            for (int i = 0; i < m; ++i) {
                const bool ee = h[i].x < 0;
                idx[5 * i] = ee ? 1 : 0;
                idx[5 * i + 1] = ee ? -1 - h[i].x : h[i].x;
                idx[5 * i + 2] = h[i].y; idx[5 * i + 3] = h[i].z; idx[5 * i + 4] = h[i].w;
            }
        }
        return r;
    }

    sim_status get_trace(double *buf, int32_t max_iters, int32_t *n) override
    {
        CK(cudaSetDevice(dev));
        sim_status r = sync_and_check();
        const int m = std::min(std::min(hctrl->iters_done, M.opt.iters), std::max(max_iters, 0));
        if (n) *n = m;
        if (m > 0 && buf) CK(cudaMemcpy(buf, D.trace, sizeof(double) * TRACE_COLS * (size_t)m, cudaMemcpyDeviceToHost));
        return r;
    }

    // One time step replayed from a graph with an event-record node before and after every kernel: per-kernel
    // GPU time (summed over the step's launches of that kernel) and launch counts.
    sim_status profile_step(const double *targets, float *ms, int32_t *launches, int n_kernels) override
    {
        CK(cudaSetDevice(dev));
        if (!ms || n_kernels <= 0) return fail(SIM_ERR_INVALID_ARG, "bad profile arguments");
        sim_status st = stage_targets(targets);
        if (st != SIM_OK) return st;
        if (persist) return profile_step_persistent(ms, launches, n_kernels);
        const int n_launch = 2 + M.opt.iters * (D.segmented ? 11 : 10);
        if ((int)prof_ev.size() < n_launch + 1) {
            for (size_t i = prof_ev.size(); i < (size_t)n_launch + 1; ++i) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e));
                prof_ev.push_back(e);
            }
        }
        std::vector<int> which;
        which.reserve(n_launch);
        CK(cudaStreamSynchronize(s));
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int q = 0;
        auto mark = [&](int kernel) {
            cudaEventRecordWithFlags(prof_ev[q++], s, cudaEventRecordExternal);
            if (kernel >= 0) which.push_back(kernel);
        };
        mark(K_PREDICT); launch_predict();
        for (int k = 0; k < M.opt.iters; ++k) {
            const int par = k & 1;
            mark(K_BP_BOXES); bp_boxes<<<bpb_boxes, BP_B, 0, s>>>(B);
            mark(K_BP_COUNT); bp_count<<<bpb_prims, BP_B, 0, s>>>(B);
            mark(K_BP_SCAN); bp_scan<<<3 * B.H / BP_SCAN_N, BP_SCAN_T, 0, s>>>(B);
            mark(K_BP_FILL); bp_fill<<<bpb_prims, BP_B, 0, s>>>(B);
            mark(K_BP_QUERY); bp_query<<<bpb_query, BP_B, 0, s>>>(B);
            mark(K_GRAD); launch_grad_kernel(par);
            if (D.segmented) { mark(K_GATHER); k_gather<R><<<nvb, VB, 0, s>>>(D, par); }
            mark(K_DOTS); k_dots<R><<<nvb, VB, 0, s>>>(D, par);
            mark(K_DIR); k_dir<R><<<nvb, VB, 0, s>>>(D, par);
            mark(K_PHP); launch_pHp_kernel();
            mark(K_UPDATE); k_update<R><<<nvb, VB, 0, s>>>(D, par);
        }
        mark(K_FINISH); launch_finish();
        mark(-1);
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture", __LINE__);
        cudaGraphExec_t ge = nullptr;
        ce = cudaGraphInstantiate(&ge, g, 0);
        if (ce != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(ce, "cudaGraphInstantiate", __LINE__); }
        ce = cudaGraphLaunch(ge, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return cuda_fail(ce, "profile graph", __LINE__);
        k_host = M.opt.iters;
        const int nk = std::min(n_kernels, (int)N_PROFILED);
        for (int k = 0; k < nk; ++k) { ms[k] = 0.0f; if (launches) launches[k] = 0; }
        for (int i = 0; i < (int)which.size(); ++i) {
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, prof_ev[i], prof_ev[i + 1]));
            if (which[i] < nk) {
                ms[which[i]] += t;
                if (launches) launches[which[i]] += 1;
            }
        }
        return sync_and_check();
    }

    // the persistent step with phase stamps: time from the end of one phase to the end of the next (as block 0
    // sees it) is attributed to the later phase's kernel slot; launches count the phases
    sim_status profile_step_persistent(float *ms, int32_t *launches, int n_kernels)
    {
        const int maxst = 64 + M.opt.iters * 16;
        if (!stamp_buf) {
            AL3(stamp_buf, (size_t)maxst);
            AL3(stamp_kind, (size_t)maxst);
        }
        CK(cudaMemsetAsync(stamp_kind, 0x7F, sizeof(int) * maxst, s));   // out-of-range kind marks the end
        CK(launch_persistent(1, 0, M.opt.iters, 1, stamp_buf, stamp_kind, maxst));
        CK(cudaStreamSynchronize(s));
        std::vector<unsigned long long> t(maxst);
        std::vector<int> kd(maxst);
        CK(cudaMemcpy(t.data(), stamp_buf, sizeof(unsigned long long) * maxst, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(kd.data(), stamp_kind, sizeof(int) * maxst, cudaMemcpyDeviceToHost));
        k_host = M.opt.iters;
        const int nk = std::min(n_kernels, (int)N_PROFILED);
        for (int k = 0; k < nk; ++k) { ms[k] = 0.0f; if (launches) launches[k] = 0; }
        for (int i = 1; i < maxst; ++i) {
            const int k = kd[i];
            if (k < 0 || k >= (int)N_PROFILED) break;
            if (k < nk) {
                ms[k] += (float)((t[i] - t[i - 1]) * 1e-6);
                if (launches) launches[k] += 1;
            }
        }
        return sync_and_check();
    }

    // the persistent step with every block's arrival and departure time at every grid barrier
    sim_status profile_barriers(const double *targets, uint64_t *arrive, uint64_t *depart, int32_t *kind,
                                int32_t max_bar, int32_t *n_bar, int32_t *n_blocks) override
    {
        CK(cudaSetDevice(dev));
        if (!persist) return fail(SIM_ERR_INVALID_ARG, "barrier profiling needs the persistent step");
        if (max_bar <= 0 || !arrive || !depart || !kind) return fail(SIM_ERR_INVALID_ARG, "no output buffers");
        sim_status st = stage_targets(targets);
        if (st != SIM_OK) return st;
        const size_t nrec = (size_t)max_bar * pgrid;
        unsigned long long *da = nullptr, *dd = nullptr;
        int *dk = nullptr;
        CK(cudaMalloc(&da, nrec * sizeof(unsigned long long)));
        CK(cudaMalloc(&dd, nrec * sizeof(unsigned long long)));
        CK(cudaMalloc(&dk, max_bar * sizeof(int)));
        cudaError_t e = cudaMemsetAsync(dk, 0x7F, max_bar * sizeof(int), s);   // out-of-range kind marks the end
        if (e == cudaSuccess) e = launch_persistent(1, 0, M.opt.iters, 1, nullptr, nullptr, 0, da, dd, dk, max_bar);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(arrive, da, nrec * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(depart, dd, nrec * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(kind, dk, max_bar * sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(da); cudaFree(dd); cudaFree(dk);
        if (e != cudaSuccess) return cuda_fail(e, "profile_barriers", __LINE__);
        k_host = M.opt.iters;
        int n = 0;
        while (n < max_bar && kind[n] >= 0 && kind[n] < (int)N_PROFILED) ++n;
        *n_bar = n;
        *n_blocks = pgrid;
        return sync_and_check();
    }

    sim_status get_groups(int32_t *group) override
    {
        CK(cudaSetDevice(dev));
        sim_status r = sync_and_check();
        const int nv = M.nv;
        for (int i = 0; i < nv; ++i) group[i] = M.vscene.empty() ? 0 : M.vscene[i];
        if (D.cmark) {
            std::vector<int> mark(nv);
            CK(cudaMemcpy(mark.data(), D.cmark, sizeof(int) * nv, cudaMemcpyDeviceToHost));
            for (int i = 0; i < nv; ++i) group[i] = 2 * group[i] + mark[i];
        }
        return r;
    }

    sim_status get_scene_scalars(double *out, int32_t max_scenes, int32_t *n_scenes) override
    {
        CK(cudaSetDevice(dev));
        sim_status r = sync_and_check();
        const int n = std::min(max_scenes, M.nseg);
        *n_scenes = M.nseg;
        if (M.nseg == 1) {
            double row[11] = {hctrl->beta, hctrl->gp, hctrl->pHp, hctrl->pmax, hctrl->alpha, hctrl->dE, hctrl->dE0,
                              (double)hctrl->converged, (double)hctrl->iters_done, (double)hctrl->restarted,
                              (double)hctrl->capped};
            std::memcpy(out, row, sizeof row);
            return r;
        }
        std::vector<SegCtl> h(M.nseg);
        CK(cudaMemcpy(h.data(), D.seg, sizeof(SegCtl) * M.nseg, cudaMemcpyDeviceToHost));
        const int lp = (hctrl->k - 1) & 1;   // parity of the last completed iteration
        for (int i = 0; i < n; ++i) {
            const SegCtl &g = h[i];
            double row[11] = {g.beta, g.gp, g.pHp, g.pmax, g.alpha, g.dE, g.dE0[lp], (double)g.converged[lp],
                              (double)g.iters_done, (double)g.restarted, (double)g.capped};
            std::memcpy(out + 11 * (size_t)i, row, sizeof row);
        }
        return r;
    }

    // ------------------------------------------------------------------------------------------ differentiation
    sim_status adj_alloc()
    {
        if (adj_b) return SIM_OK;
        const size_t n3 = 3 * (size_t)M.nv;
        AL3(adj_b, n3); AL3(adj_x, n3); AL3(adj_r, n3); AL3(adj_z, n3); AL3(adj_p, n3); AL3(adj_q, n3);
        AL3(adj_av, n3); AL3(adj_ax, n3); AL3(adj_cg, (size_t)CG_N);
        AL3(adj_dE, (size_t)M.nt);
        return SIM_OK;
    }
    // q = H p at the positions of the last eval_setup
    void launch_hvp(const double *v, double *out)
    {
        const int nb = (M.nv + 127) / 128;
        k_hvp_vert<R><<<nb, 128, 0, s>>>(D, 0, v, out);
        k_hvp_tet<R><<<(M.nt + EB - 1) / EB, EB, 0, s>>>(D, v, out);
        k_hvp_pair<R><<<ncb, EB, 0, s>>>(D, v, out);
    }
    sim_status eval_hvp(const double *x, const double *v, double *out) override
    {
        CK(cudaSetDevice(dev));
        if (!x || !v || !out) return fail(SIM_ERR_INVALID_ARG, "x, v and out are required");
        sim_status r = adj_alloc();
        if (r) return r;
        r = eval_setup(x, nullptr);
        if (r) return r;
        const size_t bytes = sizeof(double) * 3 * (size_t)M.nv;
        CK(cudaMemcpyAsync(adj_p, v, bytes, cudaMemcpyDefault, s));
        launch_hvp(adj_p, adj_q);
        CK(cudaMemcpyAsync(out, adj_q, bytes, cudaMemcpyDefault, s));
        CK(cudaStreamSynchronize(s));
        eval_restore();
        return sync_and_check();
    }
    sim_status adjoint_step(const double *x1, const double *ax1, const double *av1, double *ax0, double *av0,
                            double *dE, double tol, int32_t max_iters, int32_t *iters, double *residual) override
    {
        CK(cudaSetDevice(dev));
        if (!x1 || !ax1 || !av1 || !ax0 || !av0 || max_iters <= 0 || !(tol > 0))
            return fail(SIM_ERR_INVALID_ARG, "x1, the adjoints and a positive tolerance and iteration cap are required");
        sim_status r = adj_alloc();
        if (r) return r;
        r = eval_setup(x1, nullptr);   // H at x_{t+1}: candidates, active pairs and the gradient pass there
        if (r) return r;
        const size_t n3 = 3 * (size_t)M.nv, bytes = sizeof(double) * n3;
        const int nb = (M.nv + VB - 1) / VB;
        CK(cudaMemcpyAsync(adj_ax, ax1, bytes, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(adj_av, av1, bytes, cudaMemcpyDefault, s));
        k_adj_rhs<R><<<nb, VB, 0, s>>>(D, adj_ax, adj_av, adj_b);
        unsigned int *tk = &dctrl->ticket[TK_MISC];
        k_cg_init<R><<<nb, VB, 0, s>>>(D, 0, adj_b, adj_x, adj_r, adj_z, adj_p, adj_cg, tk);
        double hcg[CG_N] = {0};
        CK(cudaMemcpyAsync(hcg, adj_cg, sizeof hcg, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const double bb = hcg[CG_BB];
        int it = 0;
        double rr = hcg[CG_RR];
        while (it < max_iters && bb > 0.0 && rr > tol * tol * bb) {
            const int batch = std::min(8, max_iters - it);
            for (int j = 0; j < batch; ++j) {
                launch_hvp(adj_p, adj_q);
                k_cg_pq<<<nb, VB, 0, s>>>((int)n3, adj_p, adj_q, D.part, adj_cg, tk);
                k_cg_update<R><<<nb, VB, 0, s>>>(D, 0, adj_x, adj_r, adj_z, adj_p, adj_q, adj_cg, tk);
                k_cg_dir<<<nb, VB, 0, s>>>((int)n3, adj_z, adj_p, adj_cg);
            }
            it += batch;
            CK(cudaMemcpyAsync(hcg, adj_cg, sizeof hcg, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            rr = hcg[CG_RR];
        }
        if (iters) *iters = it;
        if (residual) *residual = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
        k_adj_out<R><<<nb, VB, 0, s>>>(D, adj_x, adj_av, adj_ax, adj_b);
        CK(cudaMemcpyAsync(ax0, adj_ax, bytes, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(av0, adj_b, bytes, cudaMemcpyDefault, s));
        if (dE) {
            CK(cudaMemcpyAsync(adj_dE, dE, sizeof(double) * M.nt, cudaMemcpyDefault, s));
            // the elastic gradient is linear in E_e: its derivative is the gradient with E_e = 1
            Dev<R> D1 = D;
            D1.mu = R(1.0 / (2.0 * (1.0 + M.nu)));
            D1.lam = R(M.nu / ((1.0 + M.nu) * (1.0 - 2.0 * M.nu)));
            D1.escale = nullptr;
            k_adj_youngs<R><<<(M.nt + EB - 1) / EB, EB, 0, s>>>(D1, adj_x, adj_dE);
            CK(cudaMemcpyAsync(dE, adj_dE, sizeof(double) * M.nt, cudaMemcpyDefault, s));
        }
        CK(cudaStreamSynchronize(s));
        eval_restore();
        return sync_and_check();
    }

    void sizes(int32_t *out) override
    {
        out[0] = M.nv; out[1] = M.nt; out[2] = M.nf; out[3] = M.ne; out[4] = M.ns; out[5] = (int32_t)M.excl.size();
    }

private:
    HostMesh M;
    int dev = 0, nsm = 1;
    cudaStream_t s = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    Dev<R> D;
    BPDev B;
    Ctrl *dctrl = nullptr, *hctrl = nullptr;
    std::vector<void *> allocs;
    double *stage = nullptr;
    double4_32a *xsave = nullptr, *xtsave = nullptr;
    R4 *psave = nullptr;
    int cap = 0, k_host = 0;
    int nvb = 1, ntb = 1, ncb = 1, npb = 1, bpb_boxes = 1, bpb_prims = 1, bpb_query = 1;
    // colouring scatter: the per-tet inputs in colour order
    int4 *c_tet = nullptr;
    R *c_Dm = nullptr, *c_hv = nullptr, *c_es = nullptr;
    float *c_G0 = nullptr;
    std::vector<cudaEvent_t> prof_ev;
    // persistent form
    bool persist = false;
    bool corot = false;                // FP32 form with a corotated density (FCR, ARAP): its own kernel instantiations
    int shape = 0;                     // block shape of the persistent form (persist_shapes.cuh)
    int shape_grid[N_PSHAPES] = {};    // its grid (blocks), 0 = the shape cannot be launched
    std::vector<int> tune_cfg;         // autotuning candidates: shape index, or -1 = per-phase kernels
    std::vector<float> tune_ms;
    int tune_next = -1;                // the next candidate to time (-1: no tuning, or done)
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    long long steps_run = 0;
    int pgrid = 0;
    unsigned int *bar_count = nullptr;
    void *ppart = nullptr;
    unsigned long long *stamp_buf = nullptr;
    double *adj_b = nullptr, *adj_x = nullptr, *adj_r = nullptr, *adj_z = nullptr, *adj_p = nullptr, *adj_q = nullptr;
    double *adj_av = nullptr, *adj_ax = nullptr, *adj_cg = nullptr, *adj_dE = nullptr;
    int *stamp_kind = nullptr;

    sim_status fail(sim_status st, const std::string &m) { err = m; return st; }
    sim_status cuda_fail(cudaError_t e, const char *what, int line)
    {
        err = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what + " (line " + std::to_string(line) + ")";
        return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
    }

    template <typename T> sim_status dalloc(T *&p, size_t n)
    {
        p = nullptr;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __LINE__);
        allocs.push_back(q);
        p = (T *)q;
        e = cudaMemset(q, 0, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset", __LINE__);
        return SIM_OK;
    }

    void release()
    {
        if (s) cudaStreamSynchronize(s);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : prof_ev) cudaEventDestroy(e);
        for (auto &e : tune_ev) if (e) { cudaEventDestroy(e); e = nullptr; }
        prof_ev.clear();
        gexec = nullptr; graph = nullptr;
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        if (hctrl) cudaFreeHost(hctrl);
        hctrl = nullptr;
        if (own_stream && s) cudaStreamDestroy(s);
        s = nullptr;
    }

#define AL(p, n) do { sim_status st_ = dalloc(p, n); if (st_ != SIM_OK) return st_; } while (0)
#define AL2(p, n) do { sim_status st_ = dalloc(p, n); if (st_ != SIM_OK) return st_; } while (0)

    sim_status setup_persistent()
    {
        persist = false;
        corot = sizeof(R) == 4 && (M.model == MAT_FCR || M.model == MAT_ARAP);
        if (!M.opt.persistent) return SIM_OK;
        if (M.opt.scatter == SIM_SCATTER_COLOR) return SIM_OK;         // one kernel per colour: per-phase form
        if (((3 * B.H) >> B.cshift_p) > BP_MAX_CHUNKS) return SIM_OK;   // chunk offsets live in shared memory
        int coop = 0;
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (!coop) return SIM_OK;
        // every shape's grid: as many blocks per SM as it is built for and the occupancy allows
        int gmax = 0;
        for (int sh = 0; sh < N_PSHAPES; ++sh) {
            int per_sm = 0;
            if (corot && sh > 0) { shape_grid[sh] = 0; continue; }   // the corotated FP32 kernel: shape 0 only
            if constexpr (sizeof(R) == 4) {
                if (corot) CK(persist_occupancy_corot(&per_sm));
                else CK(persist_occupancy_shape<R>(sh, &per_sm));
            } else {
                CK(persist_occupancy_shape<R>(sh, &per_sm));
            }
            per_sm = std::min(per_sm, PSHAPE_MINB[sh]);
            shape_grid[sh] = per_sm > 0 ? std::min(per_sm * nsm, MAXG) : 0;
            gmax = std::max(gmax, shape_grid[sh]);
        }
        const bool block_scatter = M.opt.scatter == SIM_SCATTER_BLOCK;   // runs in shape 0 only
        shape = (block_scatter || M.opt.block_shape < 0) ? 0 : M.opt.block_shape;
        if (shape_grid[shape] <= 0) shape = 0;
        if (shape_grid[shape] <= 0) return SIM_OK;
        pgrid = shape_grid[shape];
        unsigned int *sync;
        AL2(sync, 32);                    // the barrier arrival counter on a 128-byte line of its own
        bar_count = sync;
        R4 *pg, *pnx;
        AL2(pg, (size_t)M.nv);
        AL2(pnx, (size_t)M.nv);
        D.pg = pg;
        D.pnext = pnx;
        const size_t bytes = 16 * (size_t)gmax * sizeof(typename PartT<R>::T) + 2 * (size_t)gmax * sizeof(R);
        char *pp;
        AL2(pp, bytes);
        ppart = pp;
        persist = true;
        tune_cfg.clear();
        if (M.opt.block_shape < 0 && !block_scatter) {
            for (int sh = 0; sh < N_PSHAPES; ++sh) if (shape_grid[sh] > 0) tune_cfg.push_back(sh);
        } else {
            tune_cfg.push_back(shape);
        }
        if (M.opt.persistent == 2 && M.nseg == 1) tune_cfg.push_back(-1);
        tune_next = tune_cfg.size() > 1 ? 0 : -1;
        if (tune_next < 0) tune_cfg.clear();
        tune_ms.clear();
        return SIM_OK;
    }

    sim_status alloc_candidates()
    {
        int4 *cd;
        AL(cd, (size_t)cap);
        AL(D.act, (size_t)cap);
        D.cand = cd;
        D.cand_cap = cap;
        B.cand = cd;
        B.cap = cap;
        return SIM_OK;
    }

    sim_status alloc_all()
    {
        const int nv = M.nv, nt = M.nt;
        nvb = (nv + VB - 1) / VB;
        ntb = (nt + EB - 1) / EB;
        ncb = std::max(1, std::min(2 * nsm, (cap + EB - 1) / EB));
        npb = ncb;
        D.nv = nv; D.nt = nt; D.nfix = M.nfix;
        D.has_tgt = 1;
        AL(D.x, nv); AL(D.xt, nv); AL(D.xtil, nv); AL(D.v, nv); AL(D.xb, nv);
        AL(D.g[0], nv); AL(D.g[1], nv); AL(D.dg[0], nv); AL(D.dg[1], nv); AL(D.p, nv);
        D.xh = D.xl = nullptr;
        D.xth = D.xtl = nullptr;
        D.G0 = nullptr;
        D.tS = nullptr;
        D.xbh = nullptr;
        D.pg = D.pnext = nullptr;
        if (sizeof(R) == 4) {
            AL(D.xh, nv); AL(D.xl, nv); AL(D.xbh, nv); AL(D.xth, nv); AL(D.xtl, nv);
            float *g0;
            AL(g0, 14 * (size_t)nt);
            D.G0 = g0;
            AL(D.tS, 4 * (size_t)nt);
        }
        double *mass; AL(mass, nv); D.mass = mass;
        int *fs; AL(fs, nv); D.fix_slot = fs;
        double *tg; AL(tg, 3 * (size_t)std::max(M.nfix, 1)); D.tgt = tg;
        int4 *tet; AL(tet, nt); D.tet = tet;
        R *Dm; AL(Dm, 9 * (size_t)nt); D.Dm = Dm;
        R *hv; AL(hv, nt); D.hv = hv;
        R *es = nullptr;
        if (!M.escale.empty()) AL(es, nt);
        D.escale = es;
        D.mu = R(M.mu); D.lam = R(M.lam); D.model = M.model;
        D.h = M.h; D.dhat = M.dhat; D.kappa = M.kappa; D.eps = M.opt.eps;
        // default candidate slack: r = 0.5 L - dhat (L the mean surface edge at rest) within [2, 6] dhat, so that
        // dhat + r stays below about half an edge and the candidates stay near neighbours; 6 dhat measured the
        // fewest ms per step on the twisted bar (2 to 8 dhat tried)
        D.pad_r = M.opt.pad_r > 0 ? M.opt.pad_r
                                  : M.dhat * std::min(6.0, std::max(2.0, (0.5 * M.edge_mean - M.dhat) / M.dhat));
        for (int a = 0; a < 3; ++a) D.grav[a] = M.opt.gravity[a];
        D.has_plane = M.opt.has_plane;
        if (D.has_plane) {
            double L = std::sqrt(M.opt.plane_n[0] * M.opt.plane_n[0] + M.opt.plane_n[1] * M.opt.plane_n[1] + M.opt.plane_n[2] * M.opt.plane_n[2]);
            for (int a = 0; a < 3; ++a) D.pn[a] = M.opt.plane_n[a] / L;
            D.po = M.opt.plane_o;
        }
        D.beta_rule = M.opt.beta; D.pnorm = M.opt.pnorm; D.iters = M.opt.iters;
        D.segmented = M.opt.scatter == SIM_SCATTER_SEGMENTED;
        D.scatter_block = M.opt.scatter == SIM_SCATTER_BLOCK;
        D.colored = M.opt.scatter == SIM_SCATTER_COLOR;
        D.color_tets = nullptr;
        if (D.colored) {
            int *ct; AL(ct, (size_t)nt); D.color_tets = ct;
            AL(c_tet, nt); AL(c_Dm, 9 * (size_t)nt); AL(c_hv, nt);
            if (!M.escale.empty()) AL(c_es, nt);
            if (sizeof(R) == 4) AL(c_G0, 14 * (size_t)nt);
        }
        D.nseg = M.nseg;
        D.vscene = nullptr; D.seg = nullptr; D.sacc = nullptr; D.smax = nullptr; D.cmark = nullptr;
        if (M.opt.split_objects == 2) AL(D.cmark, (size_t)nv);
        if (M.nseg > 1) {
            int *vs; AL(vs, (size_t)nv); D.vscene = vs;
            AL(D.seg, (size_t)M.nseg);
            AL(D.sacc, 3 * 8 * (size_t)M.nseg);
            AL(D.smax, 3 * (size_t)M.nseg);
        }
        D.cv_off = nullptr; D.cv = nullptr; D.tloc = nullptr;
        if (D.scatter_block) {
            int *co; AL(co, M.cv_off.size()); D.cv_off = co;
            int *cvv; AL(cvv, std::max<size_t>(M.cv.size(), 1)); D.cv = cvv;
            ushort4 *tl; AL(tl, (size_t)nt); D.tloc = tl;
        }
        D.contrib = nullptr; D.v2c_off = nullptr; D.v2c = nullptr;
        if (D.segmented) {
            R *cb; AL(cb, 6 * 4 * (size_t)nt); D.contrib = cb;
            int *vo; AL(vo, nv + 1); D.v2c_off = vo;
            int *vc; AL(vc, 4 * (size_t)nt); D.v2c = vc;
        }
        Ctrl *c; AL(c, 1); dctrl = c; D.ctrl = c;
        {
            cudaError_t e = cudaMallocHost((void **)&hctrl, sizeof(Ctrl));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost", __LINE__);
            std::memset(hctrl, 0, sizeof(Ctrl));
        }
        // the pair-block count grows with the candidate capacity up to 2 blocks per SM
        const int npb_max = std::max(npb, 2 * nsm);
        const size_t npart = (size_t)std::max(std::max(5 * nvb, 4 * (ntb + nvb + npb_max + 4)), ntb + npb_max + 8);
        AL(D.part, npart);
        AL(D.trace, (size_t)TRACE_COLS * std::max(M.opt.iters, 1));
        AL(stage, 3 * (size_t)nv);
        AL(xsave, nv); AL(xtsave, nv); AL(psave, nv);
        // broad phase
        B.nv = nv; B.ns = M.ns; B.nf = M.nf; B.ne = M.ne;
        int H = BP_SCAN_N;
        while (H < 2 * (M.nf + M.ne)) H <<= 1;
        B.H = H;
        B.x = D.x; B.xb = D.xb;
        B.xh = D.xh; B.xbh = D.xbh;
        int *sv; AL(sv, M.ns); B.svert = sv;
        int4 *tr; AL(tr, M.nf); B.tri = tr;
        int4 *ed; AL(ed, M.ne); B.edge = ed;
        int *ob; AL(ob, nv); B.obj = ob;
        AL(B.blo, (size_t)(M.nf + M.ne)); AL(B.bhi, (size_t)(M.nf + M.ne));
        // triangle, edge and point tables of H buckets each
        AL(B.cnt, 3 * (size_t)H); AL(B.off, 3 * (size_t)H); AL(B.boff, 3 * (size_t)H / BP_SCAN_N);
        AL(B.goff, 3 * (size_t)H);
        {
            // persistent scan chunks: 128 buckets (one warp, four per lane) or more, at most BP_MAX_CHUNKS chunks
            int cs = 7;
            while (((3 * (size_t)H) >> cs) > (size_t)BP_MAX_CHUNKS) ++cs;
            B.cshift_p = cs;
            AL(B.ctot, (3 * (size_t)H) >> cs);
        }
        {
            // entries: at most 8 per triangle or edge (a box spans at most 2 cells per axis), 1 per surface point;
            // work units: an edge bucket of n entries lists t (t + 1) / 2 tiles, t = ceil(n / 32), which is at most
            // n for n <= 2016; a triangle bucket one per 32 entries
            const size_t ecap = 8 * (size_t)(M.nf + M.ne) + (size_t)M.ns;
            AL(B.erA, ecap); AL(B.erB, ecap); AL(B.ev, 3 * ecap); AL(B.eprim, ecap);
            B.ecap = (int)ecap;
            const size_t ucap = ecap + std::min(2 * (size_t)H, 8 * (size_t)(M.nf + M.ne)) + 64;
            AL(B.units, ucap);
            B.ucap = (int)ucap;
        }
        unsigned long long *ex = nullptr;
        if (!M.excl.empty()) AL(ex, M.excl.size());
        B.excl = ex; B.nexcl = (int)M.excl.size();
        B.vscene = M.opt.split_objects ? nullptr : D.vscene;   // objects of one scene touch one another
        B.infl = M.dhat + D.pad_r;
        B.thr = (float)(B.infl * 1.001);
        B.ctrl = c;
        bpb_boxes = std::max(1, std::min(4 * nsm, (std::max(std::max(M.nf + M.ne, nv), 3 * H) + BP_B - 1) / BP_B));
        bpb_prims = std::max(1, (std::max(M.nf + M.ne, M.ns) + BP_B - 1) / BP_B);
        bpb_query = 4 * nsm;   // warps stride over the work units the scan listed
        {
            sim_status st = setup_persistent();
            if (st != SIM_OK) return st;
        }
        return alloc_candidates();
    }
#undef AL
#undef AL2

    template <typename T> sim_status up(const T *dst, const void *src, size_t bytes)
    {
        CK(cudaMemcpyAsync((void *)dst, src, bytes, cudaMemcpyHostToDevice, s));
        return SIM_OK;
    }

    sim_status upload_initial()
    {
        const int nv = M.nv, nt = M.nt;
        std::vector<double4_32a> x4(nv), v4(nv);
        for (int i = 0; i < nv; ++i) {
            x4[i] = make_double4_32a(M.x0[3 * i], M.x0[3 * i + 1], M.x0[3 * i + 2], 0.0);
            v4[i] = make_double4_32a(M.v0[3 * i], M.v0[3 * i + 1], M.v0[3 * i + 2], 0.0);
        }
        std::vector<int4> t4(nt);
        for (int e = 0; e < nt; ++e) t4[e] = make_int4(M.tet[4 * e], M.tet[4 * e + 1], M.tet[4 * e + 2], M.tet[4 * e + 3]);
        std::vector<R> Dm(M.Dm.begin(), M.Dm.end()), hv(M.hv.begin(), M.hv.end()), es(M.escale.begin(), M.escale.end());
        std::vector<double4_32a> xt4(nv);
        for (int i = 0; i < nv; ++i) xt4[i] = make_double4_32a(x4[i].x, x4[i].y, x4[i].z, M.fix_slot[i] >= 0 ? -1.0 : M.mass[i]);
        sim_status st;
        if ((st = up(D.x, x4.data(), sizeof(double4_32a) * nv))) return st;
        if ((st = up(D.xb, x4.data(), sizeof(double4_32a) * nv))) return st;
        if ((st = up(D.xt, x4.data(), sizeof(double4_32a) * nv))) return st;
        if ((st = up(D.xtil, xt4.data(), sizeof(double4_32a) * nv))) return st;
        if ((st = up(D.v, v4.data(), sizeof(double4_32a) * nv))) return st;
        if ((st = up(D.mass, M.mass.data(), sizeof(double) * nv))) return st;
        if ((st = up(D.fix_slot, M.fix_slot.data(), sizeof(int) * nv))) return st;
        if ((st = up(D.tet, t4.data(), sizeof(int4) * nt))) return st;
        if ((st = up(D.Dm, Dm.data(), sizeof(R) * 9 * nt))) return st;
        if ((st = up(D.hv, hv.data(), sizeof(R) * nt))) return st;
        if (D.escale && (st = up(D.escale, es.data(), sizeof(R) * nt))) return st;
        if (D.vscene && (st = up(D.vscene, M.vscene.data(), sizeof(int) * nv))) return st;
        if (D.scatter_block) {
            if ((st = up(D.cv_off, M.cv_off.data(), sizeof(int) * M.cv_off.size()))) return st;
            if (!M.cv.empty() && (st = up(D.cv, M.cv.data(), sizeof(int) * M.cv.size()))) return st;
            if ((st = up(D.tloc, M.tloc.data(), sizeof(unsigned short) * 4 * (size_t)nt))) return st;
        }
        if (D.colored && (st = up((int *)D.color_tets, M.color_tets.data(), sizeof(int) * nt))) return st;
        if (D.segmented) {
            if ((st = up(D.v2c_off, M.v2c_off.data(), sizeof(int) * (nv + 1)))) return st;
            if ((st = up(D.v2c, M.v2c.data(), sizeof(int) * 4 * nt))) return st;
        }
        std::vector<int4> tr(M.nf), ed(M.ne);
        for (int f = 0; f < M.nf; ++f) tr[f] = make_int4(M.tri[4 * f], M.tri[4 * f + 1], M.tri[4 * f + 2], M.tri[4 * f + 3]);
        for (int e = 0; e < M.ne; ++e) ed[e] = make_int4(M.edge[4 * e], M.edge[4 * e + 1], M.edge[4 * e + 2], 0);
        if ((st = up(B.svert, M.svert.data(), sizeof(int) * M.ns))) return st;
        if ((st = up(B.tri, tr.data(), sizeof(int4) * M.nf))) return st;
        if ((st = up(B.edge, ed.data(), sizeof(int4) * M.ne))) return st;
        if ((st = up(B.obj, M.obj.data(), sizeof(int) * nv))) return st;
        if (B.excl && (st = up(B.excl, M.excl.data(), sizeof(unsigned long long) * M.excl.size()))) return st;
        if (D.G0) {
            // rest metric Dm^T Dm and det Dm (six times the rest volume) per tet in double, stored as float-float
            std::vector<float> g0(14 * (size_t)nt);
            for (int e = 0; e < nt; ++e) {
                double dm[3][3];
                for (int c = 0; c < 3; ++c)
                    for (int a = 0; a < 3; ++a) dm[a][c] = M.X[3 * (size_t)M.tet[4 * e + c + 1] + a] - M.X[3 * (size_t)M.tet[4 * e] + a];
                int q = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 3; ++j, ++q) {
                        const double v = dm[0][i] * dm[0][j] + dm[1][i] * dm[1][j] + dm[2][i] * dm[2][j];
                        const float hi = (float)v;
                        g0[(size_t)q * nt + e] = hi;
                        g0[(size_t)(6 + q) * nt + e] = (float)(v - (double)hi);
                    }
                const double det = dm[0][0] * (dm[1][1] * dm[2][2] - dm[1][2] * dm[2][1]) -
                                   dm[0][1] * (dm[1][0] * dm[2][2] - dm[1][2] * dm[2][0]) +
                                   dm[0][2] * (dm[1][0] * dm[2][1] - dm[1][1] * dm[2][0]);
                const float dh = (float)det;
                g0[(size_t)12 * nt + e] = dh;
                g0[(size_t)13 * nt + e] = (float)(det - (double)dh);
            }
            if ((st = up(D.G0, g0.data(), sizeof(float) * 14 * (size_t)nt))) return st;
        }
        if (D.colored) {
            k_color_gather<R><<<(nt + 255) / 256, 256, 0, s>>>(D, c_tet, c_Dm, c_hv, c_es, c_G0);
            CK(cudaGetLastError());
        }
        refresh_ff();
        std::memset(hctrl, 0, sizeof(Ctrl));
        hctrl->err_step = -1;
        hctrl->rebuild = 1;
        CK(cudaMemcpyAsync(dctrl, hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return SIM_OK;
    }

    sim_status stage_targets(const double *targets)
    {
        // the step kernels always read the staging buffer; without targets it is refreshed from x so that the
        // kinematic vertices keep their positions
        if (M.nfix == 0) return SIM_OK;
        if (targets) CK(cudaMemcpyAsync((void *)D.tgt, targets, 24 * (size_t)M.nfix, cudaMemcpyDefault, s));
        else launch_targets_from_x();
        return SIM_OK;
    }

    void launch_targets_from_x();

    void force_rebuild()
    {
        static const int32_t one = 1;
        static const uint32_t zero = 0;
        cudaMemcpyAsync(&dctrl->rebuild, &one, sizeof one, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(&dctrl->cell_bits, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    }
    void zero_active()
    {
        static const int32_t zero = 0;
        cudaMemcpyAsync(&dctrl->n_active, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    }
    void zero_near64()
    {
        static const int32_t zero = 0;
        cudaMemcpyAsync(&dctrl->n_near64, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
    }

    void refresh_ff() { k_refresh_ff<R><<<(M.nv + 255) / 256, 256, 0, s>>>(D); }

    sim_status in3(const double *src, double4_32a *dst)
    {
        CK(cudaMemcpyAsync(stage, src, 24 * (size_t)M.nv, cudaMemcpyDefault, s));
        k_pack4<<<(M.nv + 255) / 256, 256, 0, s>>>(stage, dst, M.nv, dst == D.xtil ? 1 : 0);
        if (dst == D.x || dst == D.xtil) refresh_ff();
        CK(cudaGetLastError());
        return SIM_OK;
    }
    // enqueues the unpack and the copy out; the caller synchronises (the stream orders a following unpack into the
    // same staging buffer after this copy)
    sim_status out3(const double4_32a *src, double *dst)
    {
        k_unpack4<<<(M.nv + 255) / 256, 256, 0, s>>>(src, stage, M.nv);
        CK(cudaMemcpyAsync(dst, stage, 24 * (size_t)M.nv, cudaMemcpyDefault, s));
        return SIM_OK;
    }

    void hctrl_sync_read() { cudaMemcpy(hctrl, dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost); }

    sim_status sync_and_check()
    {
        // the control block comes back behind the stream's work (hctrl is pinned): one synchronisation
        CK(cudaMemcpyAsync(hctrl, dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const uint32_t e = hctrl->err;
        if (e == 0u) return SIM_OK;
        // report, clear the sticky error, and grow the candidate buffer on overflow
        sim_status st = SIM_ERR_NONFINITE;
        std::string what;
        if (e & ERR_INVERTED) { st = SIM_ERR_INVERTED; what = "inverted tet (det F <= 0)"; }
        else if (e & ERR_PENETRATION) { st = SIM_ERR_PENETRATION; what = "zero contact distance"; }
        else if (e & ERR_NONFINITE) { st = SIM_ERR_NONFINITE; what = "non-finite step"; }
        else if (e & ERR_CAPACITY) { st = SIM_ERR_CAPACITY; what = "contact-candidate buffer overflow"; }
        else if (e & ERR_RANGE) { st = SIM_ERR_NONFINITE; what = "positions outside the hash grid range"; }
        else if (e & ERR_TIMEOUT) { st = SIM_ERR_TIMEOUT; what = "device wait timed out"; }
        err = what + " in time step " + std::to_string(hctrl->err_step);
        const int need = hctrl->n_cand;
        hctrl->err = 0u;
        hctrl->err_step = -1;
        CK(cudaMemcpy(&dctrl->err, &hctrl->err, sizeof(uint32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(&dctrl->err_step, &hctrl->err_step, sizeof(int32_t), cudaMemcpyHostToDevice));
        if (e & ERR_CAPACITY) {
            cap = std::max(2 * cap, need + need / 2 + 1024);
            if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
            if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
            sim_status r = alloc_candidates();
            if (r != SIM_OK) return r;
            ncb = std::max(1, std::min(2 * nsm, (cap + EB - 1) / EB));
            npb = ncb;
            force_rebuild();
            CK(cudaStreamSynchronize(s));
        }
        return st;
    }

    // ------------------------------------------------------------------------------------------ launches
    void launch_predict() { k_predict<R><<<nvb, VB, 0, s>>>(D); }
    void launch_bp()
    {
        bp_boxes<<<bpb_boxes, BP_B, 0, s>>>(B);
        bp_count<<<bpb_prims, BP_B, 0, s>>>(B);
        bp_scan<<<3 * B.H / BP_SCAN_N, BP_SCAN_T, 0, s>>>(B);
        bp_fill<<<bpb_prims, BP_B, 0, s>>>(B);
        bp_query<<<bpb_query, BP_B, 0, s>>>(B);
    }
    void launch_grad(int par)
    {
        launch_grad_kernel(par);
        if (D.segmented) k_gather<R><<<nvb, VB, 0, s>>>(D, par);
    }
    void launch_iteration(int par)
    {
        launch_bp();
        launch_grad(par);
        k_dots<R><<<nvb, VB, 0, s>>>(D, par);
        k_dir<R><<<nvb, VB, 0, s>>>(D, par);
        launch_pHp_kernel();
        k_update<R><<<nvb, VB, 0, s>>>(D, par);
    }
    void launch_finish() { k_finish<R><<<nvb, VB, 0, s>>>(D); }
    // the element kernels: the FP32 corotated densities run their own instantiations
    void launch_grad_kernel(int par)
    {
        // colouring scatter: the candidates alone (no tet blocks), then one kernel per colour
        const int nt_blocks = D.colored ? 0 : ntb;
        if (corot) k_grad<R, true><<<nt_blocks + ncb, EB, 0, s>>>(D, par, nt_blocks);
        else k_grad<R><<<nt_blocks + ncb, EB, 0, s>>>(D, par, nt_blocks);
        if (D.colored) {
            Dev<R> Dc = D;
            Dc.tet = c_tet; Dc.Dm = c_Dm; Dc.hv = c_hv; Dc.escale = c_es; Dc.G0 = c_G0;
            for (size_t c = 0; c + 1 < M.color_off.size(); ++c) {
                const int t0 = M.color_off[c], n = M.color_off[c + 1] - t0;
                if (corot) k_grad_color<R, true><<<(n + EB - 1) / EB, EB, 0, s>>>(D, Dc, par, t0, n);
                else k_grad_color<R><<<(n + EB - 1) / EB, EB, 0, s>>>(D, Dc, par, t0, n);
            }
        }
    }
    void launch_pHp_kernel()
    {
        if (corot) k_pHp<R, true><<<ntb + npb, EB, 0, s>>>(D, ntb);
        else k_pHp<R><<<ntb + npb, EB, 0, s>>>(D, ntb);
    }
    cudaError_t launch_persistent(int do_predict, int k0, int n_iters, int do_finish, unsigned long long *stamps = nullptr,
                                  int *kinds = nullptr, int max_stamps = 0, unsigned long long *arrive = nullptr,
                                  unsigned long long *depart = nullptr, int *bar_kind = nullptr, int max_bar = 0)
    {
        cudaError_t e = cudaMemsetAsync(bar_count, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
        if (D.nseg > 1) {   // the batched form's round-robin accumulators start at zero
            e = cudaMemsetAsync(D.sacc, 0, sizeof(double) * 3 * 8 * (size_t)D.nseg, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(D.smax, 0, sizeof(unsigned long long) * 3 * (size_t)D.nseg, s);
            if (e != cudaSuccess) return e;
        }
        PersistArgs A;
        A.do_predict = do_predict; A.k0 = k0; A.n_iters = n_iters; A.do_finish = do_finish;
        A.count = bar_count;
        A.part = ppart;
        A.stamps = stamps; A.stamp_kind = kinds; A.max_stamps = max_stamps;
        A.arrive = arrive; A.depart = depart; A.bar_kind = bar_kind; A.max_bar = max_bar;
        if constexpr (sizeof(R) == 4) {
            if (corot) return persist_launch_corot(D, B, A, pgrid, s);
        }
        return persist_launch_shape<R>(shape, D, B, A, pgrid, s);
    }
    sim_status launch_step()
    {
        if (persist) {
            CK(launch_persistent(1, 0, M.opt.iters, 1));
            k_host = M.opt.iters;
            return SIM_OK;
        }
        launch_predict();
        for (int k = 0; k < M.opt.iters; ++k) launch_iteration(k & 1);
        launch_finish();
        k_host = M.opt.iters;
        CK(cudaGetLastError());
        return SIM_OK;
    }

    sim_status capture()
    {
        CK(cudaStreamSynchronize(s));
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            // the stream cannot be captured (e.g. the legacy default stream): replay eagerly instead
            cudaGetLastError();
            M.opt.use_graph = 0;
            return SIM_OK;
        }
        if (persist) {
            cudaError_t le = launch_persistent(1, 0, M.opt.iters, 1);
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            if (le != cudaSuccess || ee != cudaSuccess) {
                // cooperative launches that cannot be captured: launch them directly, one per step
                cudaGetLastError();
                if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
                M.opt.use_graph = 0;
                return SIM_OK;
            }
        } else {
            launch_predict();
            for (int k = 0; k < M.opt.iters; ++k) launch_iteration(k & 1);
            launch_finish();
            CK(cudaStreamEndCapture(s, &graph));
        }
        cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(graph);
            graph = nullptr;
            gexec = nullptr;
            M.opt.use_graph = 0;
        }
        return SIM_OK;
    }
};

template <typename R> __global__ void k_targets_from_x(const double4_32a *x, const int *fix_slot, double *tgt, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sl = fix_slot[i];
    if (sl < 0) return;
    const double4_32a X = x[i];
    tgt[3 * sl] = X.x; tgt[3 * sl + 1] = X.y; tgt[3 * sl + 2] = X.z;
}

template <typename R> void SimImpl<R>::launch_targets_from_x()
{
    k_targets_from_x<R><<<(M.nv + 255) / 256, 256, 0, s>>>(D.x, D.fix_slot, (double *)D.tgt, M.nv);
}

#undef CK
#undef AL3

} // namespace pncg
