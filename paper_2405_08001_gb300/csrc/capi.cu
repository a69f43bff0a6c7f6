// The C ABI of include/pncg.h: argument checks, error strings, dispatch to the precision-specific solver.
#include <cstring>
#include <new>
#include <string>

#include "sim.h"

using pncg::Sim;

struct pncg_sim {
    Sim *impl;
};

namespace {
thread_local std::string g_create_err;

sim_status guard(sim_handle h)
{
    return (h && h->impl) ? SIM_OK : SIM_ERR_INVALID_ARG;
}
} // namespace

namespace pncg {
const char *const kProfiledNames[N_PROFILED] = {"k_predict", "bp_boxes", "bp_count", "bp_scan", "bp_fill",
                                               "bp_query",  "k_grad",   "k_gather", "k_dots",  "k_dir",
                                               "k_pHp",     "k_update", "k_finish"};
}

extern "C" {

int32_t sim_abi_version(void) { return 4; }

const char *sim_status_string(sim_status s)
{
    switch (s) {
    case SIM_OK: return "SIM_OK";
    case SIM_ERR_INVALID_ARG: return "SIM_ERR_INVALID_ARG";
    case SIM_ERR_CUDA: return "SIM_ERR_CUDA";
    case SIM_ERR_OOM: return "SIM_ERR_OOM";
    case SIM_ERR_INVERTED: return "SIM_ERR_INVERTED";
    case SIM_ERR_PENETRATION: return "SIM_ERR_PENETRATION";
    case SIM_ERR_NONFINITE: return "SIM_ERR_NONFINITE";
    case SIM_ERR_TIMEOUT: return "SIM_ERR_TIMEOUT";
    case SIM_ERR_CAPACITY: return "SIM_ERR_CAPACITY";
    }
    return "unknown status";
}

sim_status sim_default_options(sim_options *o)
{
    if (!o) return SIM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof *o);
    o->precision = SIM_FP64;
    o->beta = SIM_BETA_PR_PLUS;
    o->iters = 50;
    o->eps = 0.0;
    o->pad_r = 0.0;
    o->pnorm = SIM_PNORM_VERTEX2;
    o->scatter = SIM_SCATTER_ATOMIC;
    o->excl_factor = 1.5;
    o->cuda_stream = nullptr;
    o->use_graph = 1;
    o->candidate_capacity = 0;
    o->persistent = 1;
    o->split_objects = 0;
    o->block_shape = 0;
    return SIM_OK;
}

sim_status sim_create(const sim_mesh *mesh, const sim_material *mat, double dt, double dhat, double kappa,
                      const sim_options *opt, sim_handle *out)
{
    if (!out) { g_create_err = "out is NULL"; return SIM_ERR_INVALID_ARG; }
    *out = nullptr;
    sim_options o;
    if (opt) o = *opt;
    else sim_default_options(&o);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_err = "no CUDA device: the solver has no CPU path";
        return SIM_ERR_CUDA;
    }
    pncg::HostMesh hm;
    std::string err;
    sim_status st = pncg::build_host_mesh(mesh, mat, dt, dhat, kappa, o, hm, err);
    if (st != SIM_OK) { g_create_err = err; return st; }
    Sim *impl = nullptr;
    try {
        impl = o.precision == SIM_FP32_MIXED ? pncg::make_sim_f32() : pncg::make_sim_f64();
    } catch (const std::bad_alloc &) {
        g_create_err = "out of host memory";
        return SIM_ERR_OOM;
    }
    st = impl->init(hm);
    if (st != SIM_OK) {
        g_create_err = impl->err;
        delete impl;
        return st;
    }
    pncg_sim *h = new (std::nothrow) pncg_sim;
    if (!h) { delete impl; g_create_err = "out of host memory"; return SIM_ERR_OOM; }
    h->impl = impl;
    *out = h;
    return SIM_OK;
}

sim_status sim_step(sim_handle h, int32_t n_steps, const double *targets)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->step(n_steps, targets, true);
}

sim_status sim_step_async(sim_handle h, int32_t n_steps, const double *targets)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->step(n_steps, targets, false);
}

sim_status sim_get_state(sim_handle h, double *x_out, double *v_out, sim_stats *stats)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->get_state(x_out, v_out, stats);
}

sim_status sim_set_state(sim_handle h, const double *x, const double *v)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->set_state(x, v);
}

sim_status sim_begin_step(sim_handle h, const double *targets)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->begin_step(targets);
}

sim_status sim_iterate(sim_handle h, int32_t n)
{
    if (guard(h) || n < 0) return SIM_ERR_INVALID_ARG;
    return h->impl->iterate(n);
}

sim_status sim_end_step(sim_handle h)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->end_step();
}

sim_status sim_get_iterate(sim_handle h, double *x, double *g, double *P, double *p, double *xtilde, sim_iter_scalars *s)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->get_iterate(x, g, P, p, xtilde, s);
}

sim_status sim_set_iterate(sim_handle h, const double *x, const double *g, const double *P, const double *p, int32_t k,
                           double gPg)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->set_iterate(x, g, P, p, k, gPg);
}

sim_status sim_eval_gradient(sim_handle h, const double *x, const double *xtilde, double *g, double *diag)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->eval_gradient(x, xtilde, g, diag);
}

sim_status sim_eval_pHp(sim_handle h, const double *x, const double *p, double *out)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->eval_pHp(x, p, out);
}

sim_status sim_eval_energy(sim_handle h, const double *x, const double *xtilde, double *out, double *parts)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->eval_energy(x, xtilde, out, parts);
}

sim_status sim_get_contacts(sim_handle h, int32_t *idx, double *d, int32_t max, int32_t *count)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->get_contacts(idx, d, max, count);
}

sim_status sim_get_candidates(sim_handle h, int32_t *idx, int32_t max, int32_t *count)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->get_candidates(idx, max, count);
}

sim_status sim_get_trace(sim_handle h, double *buf, int32_t max_iters, int32_t *n)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->get_trace(buf, max_iters, n);
}

sim_status sim_profile_step(sim_handle h, const double *targets, float *ms, int32_t *launches, int32_t n_kernels)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->profile_step(targets, ms, launches, n_kernels);
}

sim_status sim_profile_barriers(sim_handle h, const double *targets, uint64_t *arrive, uint64_t *depart, int32_t *kind,
                                int32_t max_barriers, int32_t *n_barriers, int32_t *n_blocks)
{
    if (guard(h) || !n_barriers || !n_blocks) return SIM_ERR_INVALID_ARG;
    return h->impl->profile_barriers(targets, arrive, depart, kind, max_barriers, n_barriers, n_blocks);
}

int32_t sim_kernel_count(void) { return pncg::N_PROFILED; }

const char *sim_kernel_name(int32_t i)
{
    return (i >= 0 && i < pncg::N_PROFILED) ? pncg::kProfiledNames[i] : "";
}

sim_status sim_eval_hvp(sim_handle h, const double *x, const double *v, double *out)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->eval_hvp(x, v, out);
}

sim_status sim_adjoint_step(sim_handle h, const double *x1, const double *ax1, const double *av1, double *ax0,
                            double *av0, double *dE, double tol, int32_t max_iters, int32_t *iters, double *residual)
{
    if (guard(h)) return SIM_ERR_INVALID_ARG;
    return h->impl->adjoint_step(x1, ax1, av1, ax0, av0, dE, tol, max_iters, iters, residual);
}

sim_status sim_get_groups(sim_handle h, int32_t *group)
{
    if (guard(h) || !group) return SIM_ERR_INVALID_ARG;
    return h->impl->get_groups(group);
}

sim_status sim_get_scene_scalars(sim_handle h, double *out, int32_t max_scenes, int32_t *n_scenes)
{
    if (guard(h) || !out || !n_scenes || max_scenes <= 0) return SIM_ERR_INVALID_ARG;
    return h->impl->get_scene_scalars(out, max_scenes, n_scenes);
}

sim_status sim_get_sizes(sim_handle h, int32_t *out)
{
    if (guard(h) || !out) return SIM_ERR_INVALID_ARG;
    h->impl->sizes(out);
    return SIM_OK;
}

void sim_destroy(sim_handle h)
{
    if (!h) return;
    delete h->impl;
    delete h;
}

sim_status sim_selftest_wait(double limit_s)
{
    return pncg::wait_selftest(limit_s, g_create_err);
}

const char *sim_last_error(sim_handle h)
{
    if (!h || !h->impl) return g_create_err.c_str();
    return h->impl->err.c_str();
}

} // extern "C"
