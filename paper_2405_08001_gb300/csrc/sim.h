// Host-side runtime interface of the solver (internal; the public ABI is include/pncg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pncg.h"
#include "common.cuh"

namespace pncg {

// Everything sim_create derives on the host from the caller's mesh and material.
struct HostMesh {
    int nv = 0, nt = 0, nf = 0, ne = 0, ns = 0, nfix = 0;
    double h = 0, dhat = 0, kappa = 0, mu = 0, lam = 0;
    int model = 0;   // energy density (SIM_MAT_*)
    double nu = 0;                         // Poisson ratio
    sim_options opt;
    std::vector<double> X, x0, v0;         // [nv][3] rest, initial positions and velocities
    std::vector<double> mass;              // [nv]
    std::vector<int> tet;                  // [nt][4]
    std::vector<double> Dm;                // [9][nt] rows of D_m^-1
    std::vector<double> hv;                // [nt] h^2 V_e
    std::vector<double> escale;            // [nt] E_e / E, empty when uniform
    std::vector<int> tri;                  // [nf][4] (v0, v1, v2, object)
    std::vector<int> edge;                 // [ne][4] (v0, v1, object, 0)
    std::vector<int> svert;                // [ns]
    std::vector<int> obj;                  // [nv]
    std::vector<int> fix_slot;             // [nv] slot in the targets array or -1
    std::vector<unsigned long long> excl;  // sorted keys (type << 62 | a << 31 | b) of excluded pairs
    double edge_mean = 0;                  // mean surface edge length at rest
    std::vector<int> v2c_off, v2c;         // vertex -> 4 * tet + corner CSR
    // block scatter: per chunk of SCATTER_CHUNK consecutive tets, its distinct vertices (sorted) and, per tet,
    // the chunk-local index of each corner
    std::vector<int> cv_off, cv;           // [nchunk + 1], [sum of distinct counts]
    std::vector<unsigned short> tloc;      // [nt][4]
    // colouring scatter: tets grouped by colour (first-fit greedy in tet order), colour c at [color_off[c],
    // color_off[c + 1])
    std::vector<int> color_off, color_tets;
    // batching: independent scenes (nseg == 1 without scene_of_vert)
    int nseg = 1;
    std::vector<int> vscene;               // [nv] scene (object) of each vertex (empty when nseg == 1)
    int nobj = 1;                          // objects (scenes); nseg = 2 nobj groups with split_objects = 2
};



// Builds the HostMesh; returns SIM_OK or an error with a message.
sim_status build_host_mesh(const sim_mesh *mesh, const sim_material *mat, double dt, double dhat, double kappa,
                           const sim_options &opt, HostMesh &out, std::string &err);

class Sim {
public:
    virtual ~Sim() {}
    std::string err;
    virtual sim_status init(const HostMesh &m) = 0;
    virtual sim_status step(int n, const double *targets, bool sync) = 0;
    virtual sim_status get_state(double *x, double *v, sim_stats *st) = 0;
    virtual sim_status set_state(const double *x, const double *v) = 0;
    virtual sim_status begin_step(const double *targets) = 0;
    virtual sim_status iterate(int n) = 0;
    virtual sim_status end_step() = 0;
    virtual sim_status get_iterate(double *x, double *g, double *P, double *p, double *xt, sim_iter_scalars *s) = 0;
    virtual sim_status set_iterate(const double *x, const double *g, const double *P, const double *p, int k,
                                   double gPg) = 0;
    virtual sim_status eval_gradient(const double *x, const double *xt, double *g, double *d) = 0;
    virtual sim_status eval_pHp(const double *x, const double *p, double *out) = 0;
    virtual sim_status eval_energy(const double *x, const double *xt, double *out, double *parts) = 0;
    virtual sim_status get_contacts(int32_t *idx, double *d, int32_t max, int32_t *count) = 0;
    virtual sim_status get_candidates(int32_t *idx, int32_t max, int32_t *count) = 0;
    virtual sim_status get_trace(double *buf, int32_t max_iters, int32_t *n) = 0;
    virtual sim_status profile_step(const double *targets, float *ms, int32_t *launches, int n_kernels) = 0;
    virtual sim_status get_scene_scalars(double *out, int32_t max_scenes, int32_t *n_scenes) = 0;
    virtual sim_status get_groups(int32_t *group) = 0;
    virtual sim_status eval_hvp(const double *x, const double *v, double *out) = 0;
    virtual sim_status adjoint_step(const double *x1, const double *ax1, const double *av1, double *ax0, double *av0,
                                    double *dE, double tol, int32_t max_iters, int32_t *iters, double *residual) = 0;
    virtual sim_status profile_barriers(const double *targets, uint64_t *arrive, uint64_t *depart, int32_t *kind,
                                        int32_t max_bar, int32_t *n_bar, int32_t *n_blocks) = 0;
    virtual void sizes(int32_t *out) = 0;
};

Sim *make_sim_f64();
sim_status wait_selftest(double limit_s, std::string &msg);
Sim *make_sim_f32();

// kernels reported by sim_profile_step, in order
enum { K_PREDICT = 0, K_BP_BOXES, K_BP_COUNT, K_BP_SCAN, K_BP_FILL, K_BP_QUERY, K_GRAD, K_GATHER, K_DOTS, K_DIR,
       K_PHP, K_UPDATE, K_FINISH, N_PROFILED };
extern const char *const kProfiledNames[N_PROFILED];

} // namespace pncg
