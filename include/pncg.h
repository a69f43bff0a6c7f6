/*
 * pncg.h -- C ABI of the GB300 (sm_103a) PNCG solver library, libpncg.so.
 *
 * The library runs the per-iteration hot path of the Jacobi-preconditioned nonlinear conjugate gradient method
 * for interior-point (IPC log-barrier) Neo-Hookean elastodynamics of Shen, Cai, Bi, Lv, "Preconditioned
 * Nonlinear Conjugate Gradient Method for Real-time Interior-point Hyperelasticity" (SIGGRAPH 2024): the
 * incremental-potential gradient, the Jacobi diagonal, p^T H p, the beta reductions, the single-pass step rule and
 * a spatial-hash contact-candidate pass, all in hand-written CUDA kernels.
 *
 * Conventions (every entry point):
 *   - Positions, velocities and vectors are double precision, array-of-structs [n_verts][3], SI units.
 *   - Inputs are copied; nothing the caller passes is kept after the call returns.  Outputs go to caller-owned
 *     buffers.  A pointer documented as "host or device" may be either: the library asks the CUDA driver which
 *     one it is and copies accordingly.
 *   - Every call returns a sim_status; nothing throws across the ABI.  Kernel errors (an inverted tet, a zero
 *     contact distance, a non-finite value, a full candidate buffer) are recorded on the device and reported by
 *     the next call that synchronises (sim_step, sim_get_state, sim_end_step, sim_eval_*).  sim_last_error()
 *     gives a one-line description of the last failure of a handle.
 *   - A handle is used by one host thread at a time.  All device work of a handle runs on its stream (the one in
 *     sim_options.cuda_stream, or a stream the library creates), in order.
 *   - There is no CPU fallback: without a CUDA device every call that needs one returns SIM_ERR_CUDA.
 */
#ifndef PNCG_H
#define PNCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pncg_sim *sim_handle; /* opaque, owned by the library; released by sim_destroy */

typedef enum {
    SIM_OK = 0,
    SIM_ERR_INVALID_ARG = 1,  /* a null or out-of-range argument, a bad mesh (index out of range, tet of
                                 non-positive rest volume) */
    SIM_ERR_CUDA = 2,         /* a CUDA runtime call failed (no device, launch failure) */
    SIM_ERR_OOM = 3,          /* device or host allocation failed */
    SIM_ERR_INVERTED = 4,     /* det F <= 0 in some tet (log I3 undefined; Sec. 3.1 gives no remedy) */
    SIM_ERR_PENETRATION = 5,  /* a contact distance (pair or plane) reached zero */
    SIM_ERR_NONFINITE = 6,    /* a non-finite gradient, p^T H p or step */
    SIM_ERR_TIMEOUT = 7,      /* a bounded device wait expired */
    SIM_ERR_CAPACITY = 8      /* the contact-candidate buffer overflowed; the step was not applied and the
                                 buffer has been enlarged for the next call */
} sim_status;

enum { SIM_FP64 = 0, SIM_FP32_MIXED = 1 };                 /* sim_options.precision */
enum { SIM_BETA_PR_PLUS = 0, SIM_BETA_DK = 1 };            /* sim_options.beta */
enum { SIM_PNORM_VERTEX2 = 0, SIM_PNORM_COMPONENT_INF = 1 }; /* sim_options.pnorm */
enum { SIM_SCATTER_ATOMIC = 0, SIM_SCATTER_SEGMENTED = 1, SIM_SCATTER_BLOCK = 2, SIM_SCATTER_COLOR = 3 }; /* sim_options.scatter */

/* Tetrahedral mesh and initial state (Sec. 3: x holds all vertex positions of the tet meshes). */
typedef struct {
    int32_t n_verts, n_tets;
    const double *rest_x;   /* [n_verts][3] host, rest positions (define D_m and the rest-pose exclusion) */
    const int32_t *tets;    /* [n_tets][4] host, vertex indices; rest volume must be positive */
    const double *x0;       /* [n_verts][3] host, initial positions; NULL = rest_x */
    const double *v0;       /* [n_verts][3] host, initial velocities; NULL = 0 */
    const uint8_t *fixed;   /* [n_verts] host, 1 = kinematic (Dirichlet) vertex whose position is prescribed
                               per step and whose g and p entries are held at zero; NULL = none */
    const int32_t *scene_of_vert; /* [n_verts] host, batching: the independent scene each vertex belongs to,
                               0 .. n_scenes-1, non-decreasing over the vertices; every tet lies in one scene and
                               the tets are ordered by scene.  Each scene is its own PNCG problem (own beta,
                               alpha, max |p_v| and eps rule: the per-object splitting of Sec. 5.2 applied to
                               independent scenes) and no contact pair spans two scenes.  At most 1024 scenes;
                               needs the persistent form.  NULL = one scene */
} sim_mesh;

/* Energy densities in the invariants I1 = tr(S) (F = R S), I2 = tr(F^T F), I3 = det F of Sec. 3.1 (sim_material.model):
 *   SIM_MAT_NH   mu/2 (I2 - 3) - mu log I3 + lambda/2 (log I3)^2   the paper's Neo-Hookean (default)
 *   SIM_MAT_SNH  mu/2 (I2 - 3) - mu (I3 - 1) + lambda/2 (I3 - 1)^2  stable Neo-Hookean
 *   SIM_MAT_FCR  mu (I2 - 2 I1 + 3) + lambda/2 (I3 - 1)^2          fixed corotated (mu |F - R|^2 + ...)
 *   SIM_MAT_ARAP mu (I2 - 2 I1 + 3)                                 as-rigid-as-possible (mu |F - R|^2)
 * Every density runs in both forms; sim_eval_hvp and sim_adjoint_step support NH only.
 * Every density treats det F <= 0 as an error (SIM_ERR_INVERTED). */
enum { SIM_MAT_NH = 0, SIM_MAT_SNH = 1, SIM_MAT_FCR = 2, SIM_MAT_ARAP = 3 };

/* Material (Sec. 3.1): mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu)). */
typedef struct {
    double density;                /* rho, kg/m^3; lumped mass m_v = sum_e rho V_e / 4 */
    double youngs, poisson;        /* E (Pa), nu */
    const double *youngs_per_tet;  /* [n_tets] host, per-tet E overriding youngs; NULL = uniform */
    int32_t model;                 /* SIM_MAT_NH (0, default), SIM_MAT_SNH, SIM_MAT_FCR or SIM_MAT_ARAP */
} sim_material;

typedef struct {
    int32_t precision;    /* SIM_FP64: all arithmetic in double.  SIM_FP32_MIXED: element and barrier arithmetic
                             in float (from double vertex differences), reductions (dot products, p^T H p,
                             energy) in double, distance re-evaluated in double when d < 1e-3 dhat */
    int32_t beta;         /* SIM_BETA_PR_PLUS (default) or SIM_BETA_DK (Sec. 4.1-4.2) */
    int32_t iters;        /* NCG iterations per time step (IterMax of Algorithm 1); default 50 */
    double eps;           /* stop when Delta E < eps Delta E_0 (Sec. 4.4); 0 = always run iters (default) */
    double gravity[3];    /* external acceleration, M^-1 f_ext (Sec. 3); default 0 */
    int32_t has_plane;    /* 1 = vertex / half-space barrier n . x >= o with the same b, kappa, dhat */
    double plane_n[3];    /* plane normal (normalised by the library) */
    double plane_o;       /* plane offset */
    double pad_r;         /* contact-candidate padding r: candidates are rebuilt when some vertex has moved r/2
                             since the last build; <= 0 = default: half the mean surface edge length at rest
                             minus dhat, clamped to [2, 6] dhat */
    int32_t pnorm;        /* norm of p in alpha_upper = dhat / (2 ||p||): SIM_PNORM_VERTEX2 (largest per-vertex
                             Euclidean length, default) or SIM_PNORM_COMPONENT_INF (largest component) */
    int32_t scatter;      /* gradient / diagonal scatter of the tets: SIM_SCATTER_ATOMIC (default: one global
                             atomic add per tet corner), SIM_SCATTER_BLOCK (each block of 256 consecutive tets
                             sums its contributions per distinct vertex in shared memory and adds them to the
                             global accumulators once), SIM_SCATTER_SEGMENTED (per-vertex gather over a
                             vertex-to-(tet, corner) CSR list, deterministic) or SIM_SCATTER_COLOR (the tets
                             greedily coloured so that no two of a colour share a vertex, one kernel per colour
                             adding without atomics; deterministic; one kernel per phase only: in the persistent
                             form every colour would be a grid barrier) */
    double excl_factor;   /* rest-pose exclusion radius in units of dhat (Sec. 5.1: 1.5; default 1.5; 0 = off) */
    void *cuda_stream;    /* cudaStream_t for all work of the handle; NULL = a stream owned by the library */
    int32_t use_graph;    /* 1 (default) = each time step is replayed from a captured CUDA graph */
    int32_t candidate_capacity; /* initial candidate-buffer capacity in pairs; <= 0 = automatic */
    int32_t persistent;   /* 1 (default) = each time step (and each sim_iterate call) is one cooperative launch
                             whose blocks stay resident and meet at grid barriers between the phases of
                             Algorithm 1; 0 = one kernel per phase; 2 = autotuned: from the second time step on,
                             two steps run persistent and two per phase (interleaved), each timed on the GPU (those
                             steps synchronise), and the faster form runs from then on (sim_stats.launch_form).  Falls
                             back to 0 when the device cannot launch cooperative kernels; batched scenes always run
                             persistent. */
    int32_t split_objects; /* 0 (default) = the groups of sim_mesh.scene_of_vert are independent scenes (no pair
                             spans two of them).  1 = they are objects of ONE scene that may touch one another
                             (pairs between two objects are contact candidates), each with its own beta, direction,
                             max |p_v|, alpha and eps rule: the per-object splitting of Sec. 5.2.  Object o steps
                             along p_o (p with every other object's entries zero) by alpha_o = min(dhat / (2 max_o
                             |p_v|), -g^T p_o / p_o^T H p_o); a pair between objects a and b adds to p_a^T H p_a
                             and to p_b^T H p_b, each with the other object's entries of p zero.  Needs the
                             persistent form, like batched scenes.
                             2 = as 1, and every object is further divided into its collision and non-collision
                             parts at the start of each time step (Sec. 5.2, the long-noodles example): the vertices
                             of the pairs with d < dhat at x_0 (after the prediction and the kinematic targets) and
                             those within dhat of the plane form the object's collision part, the rest its
                             non-collision part; the parts stay fixed for the time step and iterate as the groups
                             above (a tet or pair spanning groups adds to each group's p^T H p with the other groups'
                             entries of p zero).  Group g = 2 object + (1 for the collision part); a group without
                             vertices takes no step.  Works without scene_of_vert (one object, two groups). */
    int32_t block_shape;  /* block shape of the persistent form: 0 (default) = 256 threads x 2 blocks per SM,
                             1 = 512 x 1, 2 = 256 x 3, 3 = 256 x 1, 4 = 384 x 1 (the compiler fits the registers
                             per thread to the shape: 128, 128, 85, 255, 168); -1 = autotuned: from the second time
                             step on, each shape runs two time steps (interleaved), timed on the GPU (those steps
                             synchronise), and the shape of the fastest step runs from then on
                             (sim_stats.block_threads, blocks_per_sm).
                             With persistent = 2 the per-phase form is timed as one more candidate.
                             SIM_SCATTER_BLOCK keeps shape 0. */
} sim_options;

/* Statistics of the last completed time step. */
typedef struct {
    int64_t step;          /* number of completed time steps */
    int32_t iters_done;    /* iterations of the last step (< iters when the eps rule fired) */
    int32_t n_candidates;  /* contact candidates of the last build */
    int32_t n_active;      /* active pairs (d < dhat) in the last iteration */
    int32_t n_rebuilds;    /* candidate builds during the last step */
    int32_t n_capped;      /* iterations of the last step that took alpha = alpha_upper */
    int32_t n_surface_tris, n_surface_edges, n_surface_verts;
    double dE0, dE_last;   /* Delta E of the first and the last iteration */
    int32_t launch_form;   /* the form time steps run in now: 1 = persistent, 0 = one kernel per phase */
    int32_t n_scenes;      /* groups with their own scalars: independent scenes, objects (split_objects = 1) or
                              object parts (split_objects = 2: two per object); 1 without scene_of_vert and parts */
    int32_t n_near_fp64;   /* FP32 form: pair evaluations of the last step (or of the last sim_eval_* call) whose
                              distance fell below 1e-3 dhat, where the barrier terms are evaluated in double */
    int32_t block_threads; /* persistent form: threads per block and blocks per SM of the shape in use (0 in the */
    int32_t blocks_per_sm; /*   per-phase form) */
    int32_t n_colors;      /* scatter SIM_SCATTER_COLOR: colours of the tet colouring (gradient kernels per
                              iteration); 0 with the other scatters */
} sim_stats;

/* Scalars of the most recent iteration (Algorithm 1). */
typedef struct {
    int32_t k;             /* index of the next iteration within the step */
    int32_t restarted;     /* 1 when the direction was restarted (beta = 0 because g^T p >= 0) */
    int32_t capped;        /* 1 when alpha = alpha_upper */
    int32_t n_active;      /* active contact pairs */
    double beta, gp, pHp, pmax, alpha_bar, alpha_up, alpha, dE, dE0;
} sim_iter_scalars;

/* Fills *opt with the defaults listed above.  Returns SIM_ERR_INVALID_ARG when opt is NULL. */
sim_status sim_default_options(sim_options *opt);

/*
 * Creates a solver for the problem of Sec. 3 (Eqs. 1, E): minimise, per time step of length dt,
 *   E(x) = 1/2 (x - xt)^T M (x - xt) + dt^2 Psi(x) + kappa sum_{k in C} b(d_k(x)),
 * with Neo-Hookean Psi, the IPC barrier b (Eq. barrier) of threshold dhat and stiffness kappa over surface
 * point-triangle and edge-edge pairs (Sec. 3.2).  Host work: D_m^-1, volumes, lumped masses, the surface
 * (faces used by one tet, their edges and vertices), objects (connected components) and the rest-pose exclusion
 * of same-object pairs closer than excl_factor * dhat (Sec. 5.1).  Device buffers are allocated here.
 *   mesh, mat: host descriptions, copied.  opt: NULL = defaults.  out: receives the handle.
 * Errors: SIM_ERR_INVALID_ARG (null pointer, dt/dhat <= 0, kappa < 0, bad index or volume), SIM_ERR_CUDA,
 * SIM_ERR_OOM.  On error *out is NULL.
 */
sim_status sim_create(const sim_mesh *mesh, const sim_material *mat, double dt, double dhat, double kappa,
                      const sim_options *opt, sim_handle *out);

/*
 * Advances n_steps time steps, each one Algorithm 1: prediction xt = x + dt v + dt^2 gravity, kinematic vertices
 * moved to their targets, `iters` PNCG iterations (constraint set, gradient + Jacobi preconditioner, beta,
 * direction, p^T H p, step alpha = min(dhat / (2 ||p||), -g^T p / p^T H p), update), then v = (x - x^t) / dt.
 *   targets: host or device, [n_steps][n_fixed][3] positions of the kinematic vertices (in increasing vertex
 *            order) at the end of each step; NULL = kinematic vertices stay where they are.
 * Synchronises the handle's stream before returning.  On a kernel error the failing step is not applied (the
 * state is the one before it), later steps are skipped, and the error status is returned.
 */
sim_status sim_step(sim_handle h, int32_t n_steps, const double *targets);

/* Launches n_steps steps like sim_step but returns without synchronising (errors surface at the next
   synchronising call).  targets must stay valid until the stream reaches the copy. */
sim_status sim_step_async(sim_handle h, int32_t n_steps, const double *targets);

/*
 * Copies the state out.  x_out, v_out: host or device, [n_verts][3], NULL = skip.  stats: host, NULL = skip.
 * Synchronises.  Reports a pending kernel error.
 */
sim_status sim_get_state(sim_handle h, double *x_out, double *v_out, sim_stats *stats);

/* Replaces positions and velocities (checkpoint / resume).  x, v: host or device [n_verts][3], NULL = keep. */
sim_status sim_set_state(sim_handle h, const double *x, const double *v);

/*
 * The three phases of sim_step, run eagerly (no graph), for step-by-step inspection:
 * sim_begin_step: prediction, kinematic targets (targets: host or device [n_fixed][3] or NULL) and the first
 * candidate build; sim_iterate: n PNCG iterations; sim_end_step: velocity update (synchronises, reports errors).
 */
sim_status sim_begin_step(sim_handle h, const double *targets);
sim_status sim_iterate(sim_handle h, int32_t n);
sim_status sim_end_step(sim_handle h);

/*
 * Solver vectors after the most recent iteration, all host or device [n_verts][3], NULL = skip:
 *   x: current iterate x_k; g: gradient g_k (evaluated at x_{k-1}, kinematic entries zero); P: Jacobi
 *   preconditioner diag(H)^-1 (1/m_v where diag <= 0, zero on kinematic vertices); p: direction p_k;
 *   xtilde: the prediction xt.  s: host, NULL = skip.  Synchronises.
 */
sim_status sim_get_iterate(sim_handle h, double *x, double *g, double *P, double *p, double *xtilde,
                           sim_iter_scalars *s);

/*
 * Overwrites the solver vectors before the next sim_iterate (lock-step comparison): any of x, g, P, p may be
 * NULL to keep it; k is the iteration index the next iteration takes (0 = first of the step); gPg is
 * g^T P g of the given g and P (the PR+ denominator; ignored when k = 0).
 */
sim_status sim_set_iterate(sim_handle h, const double *x, const double *g, const double *P, const double *p,
                           int32_t k, double gPg);

/*
 * Evaluates, with the library's kernels, at arbitrary positions (candidates rebuilt at x, active set d < dhat):
 *   sim_eval_gradient: g = dE/dx and diag(H) (Eqs. E, Hessian; unmasked), host or device [n_verts][3].
 *   sim_eval_pHp: *out = p^T H p at x (Eqs. Hessian, 12, 13; frozen closest-point coefficients).
 *   sim_eval_energy: *out = E(x) with the given prediction xtilde; parts (host double[4], NULL = skip) =
 *     {inertia, dt^2 Psi, kappa sum_pairs b, kappa sum_plane b}.
 * These calls use the handle's iteration buffers: run them between steps, not inside a begin/end pair whose
 * iterate you still need.  Synchronise; report kernel errors.
 */
sim_status sim_eval_gradient(sim_handle h, const double *x, const double *xtilde, double *g, double *diag);
sim_status sim_eval_pHp(sim_handle h, const double *x, const double *p, double *out);
sim_status sim_eval_energy(sim_handle h, const double *x, const double *xtilde, double *out, double *parts);

/*
 * Active contact pairs of the most recent gradient evaluation: rows (type, v0, v1, v2, v3) with type 0 =
 * point-triangle (v0 the point) and 1 = edge-edge (v0-v1, v2-v3), and their distances.  idx: host [max][5],
 * d: host [max] (NULL = skip).  *count receives the number of pairs (may exceed max).  Synchronises.
 */
sim_status sim_get_contacts(sim_handle h, int32_t *idx, double *d, int32_t max, int32_t *count);

/*
 * Contact candidates of the most recent build, rows (type, v0, v1, v2, v3) as in sim_get_contacts.
 * idx: host [max][5].  *count receives the number of candidates.  Synchronises.
 */
sim_status sim_get_candidates(sim_handle h, int32_t *idx, int32_t max, int32_t *count);

/*
 * Per-iteration trace of the last step: rows {beta, g^T p, p^T H p, pmax, alpha, Delta E, n_active, capped},
 * host [max_iters][8].  *n receives the number of rows written.  Synchronises.
 */
sim_status sim_get_trace(sim_handle h, double *buf, int32_t max_iters, int32_t *n);

/*
 * Advances one time step like sim_step (targets as there, for this one step) and times it kernel by kernel, on
 * the GPU.  Per-phase form: the step is replayed from a CUDA graph with an event-record node before and after every
 * kernel.  Persistent form (one cooperative kernel per step): block 0 stamps the GPU global timer after the grid
 * barrier that closes each phase, and a phase's time runs from the previous stamp.  ms: host [n_kernels],
 * milliseconds spent in each kernel (phase) over the step (all its launches); launches: host [n_kernels] or NULL,
 * launch (phase) counts; kernel i is named by sim_kernel_name(i).  Synchronises.
 */
sim_status sim_profile_step(sim_handle h, const double *targets, float *ms, int32_t *launches, int32_t n_kernels);

/*
 * Persistent form only: advances one time step like sim_step and records, for every grid barrier of the step and
 * every block of the cooperative launch, the GPU global timer (ns) when the block arrived and when it left.
 * arrive, depart: host [max_barriers][n_blocks] (n_blocks = the launch's grid, at most 4 x the SM count);
 * kind: host [max_barriers], the sim_kernel_name index of the phase each barrier closes.  *n_barriers receives the
 * number of barriers recorded (at most max_barriers), *n_blocks the grid size.  SIM_ERR_INVALID_ARG when the
 * handle runs the per-phase form.  Synchronises.  A profiling aid: the paper has no counterpart.
 */
sim_status sim_profile_barriers(sim_handle h, const double *targets, uint64_t *arrive, uint64_t *depart,
                                int32_t *kind, int32_t max_barriers, int32_t *n_barriers, int32_t *n_blocks);
int32_t sim_kernel_count(void);
const char *sim_kernel_name(int32_t i);

/*
 * sim_pHp_noalloc: p^T H p of a Neo-Hookean tet mesh (inertia plus elastic terms, no contact), for callers that
 * cannot allocate device memory -- a host application that owns the whole device-memory budget through its own
 * allocator (a game engine or a renderer that loads this library as a plugin), or a real-time thread that must
 * never block in the driver's allocator.  The paper has no counterpart: it is an allocation-free variant of the
 * library's p^T H p reduction (the sum sim_eval_pHp returns for a scene without contact).
 *   x, p, rest_x: device [n_verts][3]; tets: device [n_tets][4], every rest tet positively oriented
 *   (det[X1-X0, X2-X0, X3-X0] > 0); mass: device [n_verts] (lumped masses);
 *   youngs, poisson: Neo-Hookean material; dt: time step (the elastic term is scaled by dt^2);
 *   out: device, one double receiving p^T M p + dt^2 sum_e V_e p_e^T (d2 Psi / dx2) p_e; NaN if a current tet is
 *   inverted or a rest tet has non-positive volume (the buffers are not read back, so no status reports it);
 *   cuda_stream: cudaStream_t to launch on (NULL = the legacy default stream).  Asynchronous: *out is ready when the
 *   stream reaches it.
 *   Every buffer and the stream must belong to the calling thread's current device (the scratch is looked up for
 *   that device); tet indices must lie in [0, n_verts): they are not checked on the device.
 * No memory is allocated: the kernel's scratch (one partial sum per block of 256 threads and an arrival counter)
 * is a file-scope __device__ array of 512 KiB that every GPU loading the library keeps until the process exits.
 * Limits: n_verts and n_tets at most 16,777,216 each (65,536 blocks); larger sizes return SIM_ERR_INVALID_ARG
 * and sim_noalloc_last_error() says why.  The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress) for that device: make it before any stream capture.  Every call on a device shares the
 * one scratch array, which keeps the last call's contents (the counter is cleared at the start of each call):
 * calls that may overlap on the GPU (different streams, or threads) race and must be serialised by the caller.
 * Errors: SIM_ERR_INVALID_ARG (null pointer, size, parameters), SIM_ERR_CUDA (no device, launch failure).
 */
sim_status sim_pHp_noalloc(int32_t n_verts, int32_t n_tets, const double *x, const double *p, const double *rest_x,
                           const int32_t *tets, const double *mass, double youngs, double poisson, double dt,
                           double *out, void *cuda_stream);

/* One-line description of the last failure of sim_pHp_noalloc on the calling thread. */
const char *sim_noalloc_last_error(void);

/* Sizes: out[0..5] = n_verts, n_tets, n_surface_tris, n_surface_edges, n_surface_verts, n_excluded_pairs. */
sim_status sim_get_sizes(sim_handle h, int32_t *out);

/* Releases the handle and its device buffers (synchronises its stream first).  NULL is ignored. */
void sim_destroy(sim_handle h);

/* One-line description of the last failure of h (or of the last failed sim_create or sim_selftest_wait when h is
   NULL). */
const char *sim_last_error(sim_handle h);

/*
 * Failure-detection self-test (no handle).  Runs one bounded device wait that nothing completes: a one-block kernel
 * arrives at a counter that expects two arrivals and polls it with the grid barriers' wait, whose limit is limit_s
 * seconds here (0 < limit_s <= 4) instead of 4 s.  Returns SIM_ERR_TIMEOUT, the expected outcome, after about
 * limit_s, and leaves the context usable; SIM_ERR_INVALID_ARG for a limit out of range; SIM_ERR_CUDA without a
 * device.  sim_last_error(NULL) describes the outcome.
 */
sim_status sim_selftest_wait(double limit_s);

/* Name of a status code. */
const char *sim_status_string(sim_status s);

/* ABI version of the library (incremented on incompatible changes). */
int32_t sim_abi_version(void);

/*
 * Differentiation (the adjoint of a time step, read as the exact minimiser of Algorithm 1's incremental potential
 * E(x; x~, theta); the paper has no adjoint).
 *
 * sim_eval_hvp: out = H(x) v, H the Hessian of E at x as the p^T H p pass sees it (the Sec. 3.1 split of the
 * handle's density, the I1 term of the fixed corotated and as-rigid-as-possible densities included; the barrier with the closest points frozen, Eqs. 12-13, the half-space barrier and the lumped mass), candidates
 * and active pairs taken at x.  Rows and columns of kinematic vertices are dropped (their out entries are 0).
 * x, v, out: [n_verts][3], host or device.  The handle's state is kept.  Synchronises.
 */
sim_status sim_eval_hvp(sim_handle h, const double *x, const double *v, double *out);

/*
 * sim_adjoint_step: the reverse of one time step x_t -> x_{t+1} (v_{t+1} = (x_{t+1} - x_t)/h).  Given the loss's
 * adjoints ax1 = dL/dx_{t+1} and av1 = dL/dv_{t+1}, solves H(x_{t+1}) lambda = ax1 + av1/h by Jacobi-preconditioned
 * linear CG (the preconditioner of Sec. 4.2) to a relative residual tol or max_iters iterations, and writes
 *   ax0 = dL/dx_t = M lambda - av1/h,   av0 = dL/dv_t = h M lambda
 * (kinematic vertices: ax0 = -av1/h, av0 = 0) and, when dE is not NULL, adds dL/dE_e = -lambda_e . dg_e/dE_e to
 * dE[e] for every tet (the per-tet Young's modulus; g_e the tet's elastic gradient).
 * x1, ax1, av1, ax0, av0: [n_verts][3]; dE: [n_tets]; host or device.  *iters and *residual (nullable) receive the
 * CG iterations and the final relative residual.  The handle's state is kept.  Synchronises.
 */
sim_status sim_adjoint_step(sim_handle h, const double *x1, const double *ax1, const double *av1, double *ax0,
                            double *av0, double *dE, double tol, int32_t max_iters, int32_t *iters, double *residual);

/*
 * Batching: the scalars of the most recent iteration per scene, rows {beta, g^T p, p^T H p (with p^T M p),
 * max_v |p_v|, alpha, Delta E, Delta E of iteration 0, converged, iterations done, restarted, capped}.
 * out: host [max_scenes][11]; *n_scenes receives the number of scenes (1 without scene_of_vert, whose row repeats
 * the sim_iter_scalars of sim_get_iterate).  Synchronises.
 */
sim_status sim_get_scene_scalars(sim_handle h, double *out, int32_t max_scenes, int32_t *n_scenes);

/*
 * The group of every vertex in the current time step: with split_objects = 2 the part label 2 object + (1 when
 * the vertex is in its object's collision part; set by the step's first iteration), otherwise scene_of_vert (0
 * without it).  The rows of sim_get_scene_scalars follow these labels.  group: host [n_verts].  Synchronises.
 */
sim_status sim_get_groups(sim_handle h, int32_t *group);

#ifdef __cplusplus
}
#endif

#endif /* PNCG_H */
