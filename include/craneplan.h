/*
 * craneplan.h -- C ABI of the GB300 (sm_103a) library for the stochastic B-spline path
 * optimisation of a forestry crane (arXiv 2503.14160, Sec. 4.1, Algorithm 1).
 *
 * One planning query searches joint space for a short, collision-free path from q_0 to
 * q_d. The path is a cubic B-spline whose K free control points ("waypoints") are drawn
 * each iteration from N(mu, sigma^2 C) (Algorithm 1 step (1)); every candidate is scored
 * with J = J_p + w_c J_c + w_l J_l over n_s = (K+3) S checkpoints (Eq. path opt; step
 * (2)); the candidates are ranked (step (3)); the nu best get log-rank weights (step (4));
 * and mu and C are replaced by the weighted mean and covariance of those elites (steps
 * (5)-(6)).
 *
 * Conventions for every entry point:
 *  - Return value: CP_OK (0) on success, a negative cp_status on failure; then
 *    cp_last_error() (thread-local) describes the failure. No call aborts the process.
 *  - "d_" pointers are CUDA device pointers owned by the caller; "h_" pointers and
 *    struct pointers are host memory owned by the caller. The library keeps no caller
 *    pointer after a call returns.
 *  - All device work of a planner is ordered on the stream given to cp_plan_init (a
 *    cudaStream_t passed as void*; NULL = the legacy default stream). Calls that take
 *    device pointers only enqueue work and return before it completes; calls that take
 *    "h_" outputs synchronise that stream.
 *  - Layouts: a candidate is K control points of 4 joints (q1 slew [rad], q2 boom pitch
 *    [rad], q3 jib pitch [rad], q4 telescope [m]), stored point-major as float[K][4]
 *    (one float4 per point); a population is float[N][K][4]. Means and covariances are
 *    double, flattened point-major: index 4*point + joint, D = 4K.
 *  - The library allocates device memory only in cp_plan_init (its workspace) and frees
 *    it in cp_destroy.
 */
#ifndef CRANEPLAN_H
#define CRANEPLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CP_MAX_SPHERES 16
#define CP_MAX_WAYPOINTS 32
#define CP_VERSION 1

typedef enum cp_status {
    CP_OK = 0,
    CP_ERR_ARG = -1,      /* an argument is out of range or NULL where it may not be */
    CP_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    CP_ERR_TIMEOUT = -3,  /* a bounded device-side wait gave up */
    CP_ERR_STATE = -4,    /* the planner is not ready for this call (e.g. no end points) */
    CP_ERR_OOM = -5,      /* device allocation failed */
    CP_ERR_NUMERIC = -6   /* the covariance lost positive definiteness */
} cp_status;

/* One link-bounding sphere (Sec. 3.1 collision geometry, here spheres on the links).
 * Its centre, with O the slew/boom pivot, J the jib pivot, T the tip, e_b and e_j the
 * boom and jib directions and t = offset:
 *   link 0 (boom)      O + t e_b
 *   link 1 (jib)       J + t e_j
 *   link 2 (telescope) J + (jib_len + t q4) e_j
 *   link 3 (grapple)   T - t z      (the grapple hangs plumb below the tip) */
typedef struct cp_sphere {
    int32_t link;
    double offset;   /* m */
    double radius;   /* m, > 0 */
} cp_sphere;

/* The actuated crane chain (Sec. 2, Eq. FK): slew q1 about world z at the origin; boom
 * pivot at height base_z; boom pitch q2 measured from horizontal; jib pitch q3 relative
 * to the boom in the same vertical plane; telescope q4 extends the jib axis.
 *   e_b = (cos q2 cos q1, cos q2 sin q1, sin q2),  e_j = same with q2 + q3,
 *   O = (0, 0, base_z),  J = O + boom_len e_b,  T = J + (jib_len + q4) e_j.
 * q_min/q_max are the joint limits used by J_l (Eq. path opt); the kinematics use the
 * raw, unclamped q. */
typedef struct cp_model {
    double base_z;
    double boom_len;
    double jib_len;
    double q_min[4];
    double q_max[4];
    int32_t n_spheres;                    /* 1..CP_MAX_SPHERES */
    cp_sphere spheres[CP_MAX_SPHERES];
} cp_model;

/* Vertical capped cylinder {(x-cx)^2 + (y-cy)^2 <= radius^2, z_lo <= z <= z_hi}. */
typedef struct cp_cylinder {
    double cx, cy, radius, z_lo, z_hi;
} cp_cylinder;

/* Axis-aligned box [lo, hi]. */
typedef struct cp_box {
    double lo[3];
    double hi[3];
} cp_box;

/* Obstacle scene in HOST memory. The signed distance d(q) of Sec. 3.1 is the minimum
 * over link spheres and obstacles of (obstacle signed distance at the sphere centre)
 * minus the sphere radius; d < 0 is a collision. */
typedef struct cp_scene {
    int32_t n_cyl;
    const cp_cylinder *cyl;
    int32_t n_box;
    const cp_box *box;
} cp_scene;

/* Search parameters of Algorithm 1 and of the cost (Eq. path opt). */
typedef struct cp_params {
    int32_t n_candidates;   /* lambda = N, the population size, >= 2 */
    int32_t n_waypoints;    /* K free control points, 1..CP_MAX_WAYPOINTS */
    int32_t substeps;       /* S checkpoints per moving spline span; n_s = (K+3) S */
    int32_t n_elites;       /* nu; 0 selects floor(N/2) */
    double w_c;             /* weight of J_c */
    double w_l;             /* weight of J_l */
    double lambda_c;        /* r_c(q) = lambda_c max(0, -d(q)) */
    double sigma;           /* step size: samples are N(mu, sigma^2 C) */
    double eps;             /* covariance regulariser eps I of step (6) */
    double init_std_frac;   /* C_0 = diag((init_std_frac (q_max - q_min))^2) */
    uint64_t seed;          /* Philox key */
    uint32_t query;         /* fourth Philox counter word (query id) */
    int32_t max_cylinders;  /* capacity of the scene buffers (cp_set_scene); 0 = scene's */
    int32_t max_boxes;
    double grid_cell;       /* > 0: evaluate through a polar index of the obstacles about the
                               slew axis (256 angular bins, rings of this width in m), from
                               which every checkpoint takes the obstacles near the vertical
                               plane of its slew angle without scanning the scene (for large
                               scenes); 0: scan every obstacle (broad phase or exhaustive). The
                               results are the same bit for bit. */
    double grid_half_extent;/* outer radius of the index's last closed ring (m); obstacles
                               beyond it share one open ring. 0 = boom_len + jib_len +
                               max|q4 limit| + 4 */
    int64_t max_grid_items; /* capacity of the index's cell lists; 0 = bound of the initial
                               scene */
    double smooth_margin;   /* differentiable form: softplus margin m (m); 0 selects 0.05 */
    double smooth_beta;     /* differentiable form: softplus width beta (m); 0 selects 0.01 */
    int32_t eval_ctas_per_sm; /* launch shape of the evaluation kernel: CTAs per SM of its
                                 persistent grid (0: as many as fit) */
    int32_t debug_withhold_staging; /* test hook, 0 in use: 1 makes the brute-force
                                 evaluation issue no shared-memory staging copy, 2 makes the
                                 tensor-core elite sampler issue no copy of its operand
                                 chunks, so that the bounded wait runs out and
                                 CP_ERR_TIMEOUT is reported */
    int32_t eval_exhaustive; /* 1: test every sphere against every obstacle; 0 (default): a
                                broad phase first drops, per 32 checkpoints of a candidate,
                                the obstacles out of reach of all their spheres. Both give
                                the same results bit for bit; only the time differs. Not
                                used by the grid form (grid_cell > 0). */
    int32_t update_rule;    /* steps (5)-(6): CP_UPDATE_PAPER (0) as Algorithm 1 prints them
                               (covariance about the new mean plus eps I, sigma fixed), or
                               CP_UPDATE_CMAES (1), the CMA-ES update the method is modelled
                               on: a cumulated step-size path adapts sigma, and C takes a
                               rank-one (evolution path) and a rank-mu (elites about the OLD
                               mean) update with the default learning rates; no eps. */
    int32_t collision_model;/* d(q) of Sec. 3.1 in the path cost: CP_COLLISION_SPHERES (0), the
                               link spheres of cp_model against the obstacles (the exact,
                               exhaustive, broad-phase and grid forms), or CP_COLLISION_HULLS
                               (1), the link boxes of cp_set_hull_model against boxes and
                               octagonal prisms by separating axes (cp_hull_penetration's model;
                               no grid: every obstacle is scanned per checkpoint). Only the
                               penetration depth enters J_c and the flags. */
    int32_t sampler;        /* step (1): CP_SAMPLE_FACTOR (0) draws xi = mu + L z with L the
                               FP64 Cholesky factor of sigma^2 C; CP_SAMPLE_ELITES (1), with
                               CP_UPDATE_PAPER only, draws the same N(mu, sigma^2 C) from the
                               last update's elites without forming C or its factor:
                               xi = mu + sigma (sum_j sqrt(w_j)(x_(j) - mu) g_j + sqrt(eps) g').
                               The product of the N x nu normals g and the scaled elite
                               deviations runs on the tensor cores in TF32 with a hi/lo split of
                               both operands (FP32 accuracy; FP32 accumulation). The first
                               sample after cp_set_endpoints or cp_set_distribution uses the
                               factor. C and L are formed only when cp_get_distribution or
                               cp_get_factor asks for them. */
} cp_params;

#define CP_UPDATE_PAPER 0
#define CP_UPDATE_CMAES 1
#define CP_SAMPLE_FACTOR 0
#define CP_SAMPLE_ELITES 1
#define CP_COLLISION_SPHERES 0
#define CP_COLLISION_HULLS 1

/* Cost terms of the final mean path and the state of a finished plan. */
typedef struct cp_plan_stats {
    double J, Jp, Jc, Jl;   /* cost of the final mean path and its three terms */
    double length;          /* sum_k |q(s_k) - q(s_{k-1})| of the final mean path */
    int32_t flag;           /* 1 when the final mean path collides at some checkpoint */
    int32_t n_flagged;      /* checkpoints of the final mean path in collision */
    int32_t iterations;     /* iterations run by this call */
    int32_t iteration;      /* the planner's iteration counter after the call */
    double best_J;          /* lowest candidate cost of the last iteration */
} cp_plan_stats;

/* Accumulated device time per stage while timing is on (CUDA events on the planner's
 * stream around each stage's launches), and the work the evaluation kernel did. */
typedef struct cp_timing {
    double eval_ms;   int64_t eval_launches;    /* FK + collision + cost kernel only */
    double sample_ms; int64_t sample_launches;
    double factor_ms; int64_t factor_launches;
    double update_ms; int64_t update_launches;  /* rank, weights, mean, covariance */
    int64_t eval_units;           /* work units evaluated: candidates x ceil(n_s / 32) */
    int64_t eval_obstacle_tests;  /* obstacles whose per-sphere filter passed somewhere: in the
                                     broad-phase form the (unit, obstacle) survivors of the unit
                                     box, in the exhaustive form every obstacle of every unit
                                     (both per 32 lanes), in the polar-index form the (lane,
                                     obstacle) pairs that passed (counted on the device) */
    int64_t eval_pair_tests;      /* (checkpoint, sphere, obstacle) filter tests run: 32 x
                                     spheres x eval_obstacle_tests, or, in the polar-index form,
                                     spheres x eval_box_tests */
    int64_t eval_box_tests;       /* (lane, listed obstacle) tests of the polar-index form
                                     (counted on the device; -1 for the other forms) */
} cp_timing;

typedef struct cp_planner cp_planner;

/* Description of the last failure on this thread ("" when none). */
const char *cp_last_error(void);

/* CP_VERSION of the loaded library. */
int32_t cp_version(void);

/* Number of kernels this library has launched in this process (all planners); a replay of a
 * batch graph counts the kernels recorded in it. */
int64_t cp_launch_count(void);

/* Test hook: the next n planner workspace allocations (cp_plan_init's one device
 * allocation) fail as if the device were out of memory, so that cp_plan_init returns
 * CP_ERR_OOM after releasing what it holds. n = 0 turns it off; no other effect. */
void cp_debug_fail_allocations(int32_t n);

/* Create a planner on the current CUDA device: validates the model, scene and parameters,
 * allocates the device workspace for N candidates, stages the scene (host -> device) and
 * tabulates the spline basis. End points must be set with cp_set_endpoints before
 * sampling or planning. On failure *out is NULL and nothing stays allocated.
 * Errors: CP_ERR_ARG (invalid input), CP_ERR_OOM, CP_ERR_CUDA. */
int cp_plan_init(const cp_model *model, const cp_scene *scene, const cp_params *params,
                 void *stream, cp_planner **out);

/* Release the workspace (synchronises the planner's stream first). NULL is ignored. */
void cp_destroy(cp_planner *p);

/* Replace the obstacle scene (host memory, copied to the device on the planner's
 * stream). Capacities are those given at init. Errors: CP_ERR_ARG, CP_ERR_CUDA. */
int cp_set_scene(cp_planner *p, const cp_scene *scene);

/* Set start q_0 and goal q_d (host, 4 doubles each) and reset the search: mu <- the K
 * interior points evenly spaced on the segment q_0 -> q_d (Sec. 4.1 initial guess),
 * C <- diag((init_std_frac (q_max - q_min))^2), iteration counter <- 0, and factor
 * sigma^2 C. Errors: CP_ERR_ARG, CP_ERR_CUDA. */
int cp_set_endpoints(cp_planner *p, const double h_q0[4], const double h_qd[4]);

/* Algorithm 1 step (1): d_xi[i] = mu + L z_i for i < N, L L^T = sigma^2 C, z_i the D
 * standard normals of Philox4x32-10 at counter (block j, candidate i, iteration `iter`,
 * query) under key seed, through Box-Muller (block j gives z[4j..4j+3]). d_xi is
 * float[N][K][4] on the device. Every candidate array of this API (d_xi here and in
 * cp_evaluate, cp_update, cp_smooth_cost, cp_smooth_cost_grad, cp_polish) is read and
 * written one control point (16 bytes) at a time and must be 16-byte aligned; an
 * unaligned pointer is CP_ERR_ARG. Errors: CP_ERR_STATE (no end points), CP_ERR_ARG. */
int cp_sample(cp_planner *p, int32_t iter, float *d_xi);

/* Algorithm 1 step (2): the cost of Eq. path opt for n candidates d_xi (float[n][K][4],
 * n <= N). Outputs (device; all but d_J may be NULL):
 *   d_J              double[n]       J = J_p + w_c J_c + w_l J_l
 *   d_flag           uint8[n]        1 when d(q(s_k)) < 0 at some checkpoint k = 1..n_s
 *   d_terms          double[n][5]    J_p, J_c, J_l, path length, checkpoints in collision
 *   d_substep_flags  uint32[n][W]    W = ceil(n_s / 32); bit b of word w is checkpoint
 *                                    k = 32 w + b + 1 in collision
 *   d_pen            float[n][n_s]   max(0, -d(q(s_k))) at k = 1..n_s
 * Errors: CP_ERR_STATE (no end points), CP_ERR_ARG. */
int cp_evaluate(cp_planner *p, const float *d_xi, int32_t n, double *d_J, uint8_t *d_flag,
                double *d_terms, uint32_t *d_substep_flags, float *d_pen);

/* Algorithm 1 steps (3)-(6) for the N candidates d_xi with costs d_J (double[N], NaN
 * ranks last, ties go to the lower index): mu <- sum_j w_j xi_(j),
 * C <- sum_j w_j (xi_(j) - mu)(xi_(j) - mu)^T + eps I with the new mu, then factor
 * sigma^2 C for the next sample and advance the iteration counter.
 * Errors: CP_ERR_STATE, CP_ERR_ARG, CP_ERR_NUMERIC (reported by the next host-synchronising call). */
int cp_update(cp_planner *p, const double *d_J, const float *d_xi);

/* Synchronise the planner's stream and report a device-side failure of earlier
 * asynchronous calls (CP_ERR_NUMERIC for a non-positive-definite covariance met by the
 * factorisation, CP_ERR_TIMEOUT for a bounded wait that gave up); the report is cleared. */
int cp_synchronize(cp_planner *p);

/* Run `iters` iterations of Algorithm 1 (sample, evaluate, update) from the current
 * state, then evaluate the mean path. h_ctrl (host, may be NULL) receives the K+8
 * control points of the result, double[K+8][4]: four copies of q_0, mu, four copies of
 * q_d. stats (host, may be NULL) receives the cost terms of the mean path.
 * Synchronises the planner's stream. Errors: CP_ERR_STATE, CP_ERR_ARG, CP_ERR_CUDA,
 * CP_ERR_NUMERIC. */
int cp_plan(cp_planner *p, int32_t iters, double *h_ctrl, cp_plan_stats *stats);

/* Sec. 3.1 signed distance d(q) (float, device) for n configurations d_q (float[n][4],
 * device); +inf for an empty scene. Errors: CP_ERR_ARG. */
int cp_signed_distance(cp_planner *p, const float *d_q, int32_t n, float *d_d);

/* Forward kinematics of Sec. 2 (Eq. FK) for n configurations d_q (float[n][4], device,
 * 16-byte aligned): the link-sphere centres d_centres (float[n][n_spheres][3], or NULL) by
 * the placement rule of cp_model, and the tip T = O + boom_len e_b + (jib_len + q4) e_j
 * (float[n][3], or NULL); the grapple centre hangs plumb below T. FP32, asynchronous on
 * the planner's stream. Errors: CP_ERR_ARG (n < 0, NULL or misaligned d_q). */
int cp_forward_kinematics(cp_planner *p, const float *d_q, int32_t n, float *d_centres, float *d_tip);

/* Convex-hull collision checking of Sec. 3.1 (the crane's links as convex hulls against the
 * obstacles by the separating axis theorem), batched. The paper's crane meshes are not
 * available; synthetic hulls stand in: the boom, the jib and the telescope as oriented boxes
 * along their axes (axes e, n, e x n with n the normal of the crane's vertical plane; half
 * extents (length/2 + pad, w, h); the telescope spans max(q4, 0)), the grapple as an upright
 * box of half width grapple_w and height grapple_len below the tip. Obstacles: the boxes, and
 * each cylinder as the regular octagonal prism circumscribing it (side normals at multiples
 * of 45 degrees). For each configuration d_pen receives the largest penetration depth over
 * links and obstacles (the shortest translation that separates the pair; 0 when every pair
 * is disjoint). FP32. Arguments: d_q float[n][4] (device, 16-byte aligned), hulls (host, or
 * NULL for the defaults w = h = (0.2, 0.2, 0.15) m, pad 0.2 m, grapple 0.25 x 1.0 m), d_pen
 * float[n] (device). Asynchronous on the planner's stream. Errors: CP_ERR_ARG. */
typedef struct cp_hull_model {
    double w[3];          /* half extents across the crane plane: boom, jib, telescope (m) */
    double h[3];          /* half extents in the plane, across the link */
    double pad;           /* added to each arm box's half length (m) */
    double grapple_w;     /* half width of the grapple box (m) */
    double grapple_len;   /* height of the grapple box below the tip (m) */
} cp_hull_model;

int cp_hull_penetration(cp_planner *p, const float *d_q, int32_t n, const cp_hull_model *hulls, float *d_pen);

/* The hull model the planner's path cost uses under CP_COLLISION_HULLS (host struct, copied;
 * NULL restores the defaults of cp_hull_penetration). Errors: CP_ERR_ARG. */
int cp_set_hull_model(cp_planner *p, const cp_hull_model *hulls);

/* Collision-free inverse kinematics of Sec. 3.2 (Eq. IK opt), batched: for each target
 * pose (x, y, z, psi) the configuration q that minimises |r(q)|^2 with
 *   r[0..2] = p_g(q) - (x, y, z)      p_g = the grapple centre, grapple_len below the tip
 *                                     (the passive joints hang plumb at equilibrium, so the
 *                                     equilibrium residual r_e is zero and not a row);
 *   r[3]    = lambda_q * wrap(q1 - psi)  the grapple's orientation is Rz(q1), so the SO(3)
 *                                     log of R_d^T R_g is the yaw error wrapped to [-pi, pi];
 *   r[4]    = lambda_c * max(0, -d(q))  d(q) the signed distance of Sec. 3.1.
 * Solver: damped Gauss-Newton (Levenberg-Marquardt): solve (H + mu (diag H + 1e-6)) s = -g
 * with H = J^T J and g = J^T r, clip q + s to the joint limits, accept when |r|^2
 * decreases (mu / 3, floor 1e-12), else mu * 4 (cap 1e12); `iters` iterations from each of
 * `restarts` starting points, the best (lowest |r|^2, the lower start on ties) kept. Start
 * k of target t is four uniforms of one Philox4x32-10 block, counter (k, t, 0x494B5354,
 * query), key = seed, top 24 bits of each word spread over the joint limits; with
 * d_q_init non-NULL start 0 is d_q_init[t] instead (a warm start). Arithmetic is FP32.
 * Arguments (device pointers, row-major, owned by the caller; d_targets, d_q_init and d_q
 * 16-byte aligned, each row read or written as one 16-byte word):
 *   d_targets   float[n][4]   x, y, z (m) and psi (rad)
 *   d_q_init    float[n][4]   or NULL
 *   d_q         float[n][4]   result
 *   d_f         float[n]      |r(q)|^2 at the result
 *   d_restart   int32[n]      or NULL: the start that won
 *   d_r         float[n][5]   or NULL: r at the result
 * A NaN target gives a NaN |r|^2 (ranked last among the starts). Asynchronous on the
 * planner's stream. Errors: CP_ERR_ARG (n < 0, restarts outside 1..CP_IK_MAX_RESTARTS,
 * iters < 0, a negative scale or grapple length, mu0 <= 0, NULL or misaligned buffers). */
#define CP_IK_MAX_RESTARTS 1024
typedef struct cp_ik_params {
    double lambda_q;      /* m per rad of yaw error */
    double lambda_c;      /* scale of the collision residual */
    double grapple_len;   /* tip to grapple centre (m) */
    double mu0;           /* initial damping */
    uint64_t seed;        /* Philox key of the starting points */
    uint32_t query;       /* fourth Philox counter word: separates batches */
    int32_t restarts;
    int32_t iters;
} cp_ik_params;

int cp_ik(cp_planner *p, const float *d_targets, int32_t n, const cp_ik_params *ik,
          const float *d_q_init, float *d_q, float *d_f, int32_t *d_restart, float *d_r);

/* Copy the current mean (double[D]) and covariance (double[D][D]) to device buffers
 * (either may be NULL). */
int cp_get_distribution(const cp_planner *p, double *d_mu, double *d_C);

/* Replace mean and covariance from device buffers, set the iteration counter to `iter`
 * and factor sigma^2 C (a checkpoint restore: with the same seed the remaining
 * iterations repeat bit for bit). Errors: CP_ERR_STATE (no end points), CP_ERR_ARG. */
int cp_set_distribution(cp_planner *p, const double *d_mu, const double *d_C, int32_t iter);

/* State of the CMA-ES update rule beyond (mu, C): double[1 + 2D] = {sigma, p_sigma[D],
 * p_c[D]} (device buffers). cp_set_endpoints resets it to {params.sigma, 0, 0};
 * cp_set_cma_state replaces it and factors sigma^2 C again (with cp_set_distribution it
 * restores a checkpoint of the CMA-ES rule). Under CP_UPDATE_PAPER the state holds the
 * fixed sigma and zero paths. Errors: CP_ERR_ARG, CP_ERR_STATE (no end points). */
int cp_get_cma_state(const cp_planner *p, double *d_state);
int cp_set_cma_state(cp_planner *p, const double *d_state);

/* Copy the current Cholesky factor L (double[D][D], lower, L L^T = sigma^2 C). */
int cp_get_factor(const cp_planner *p, double *d_L);

/* Copy the candidate indices of the last update in rank order (int32[nu]). */
int cp_get_elites(const cp_planner *p, int32_t *d_idx);

/* Per-iteration metrics of cp_plan (off by default; on costs one small kernel per
 * iteration). Each iteration of cp_plan while on writes one row {iteration, best J of the
 * population, mean J of the population, tr C of the updated distribution, fraction of the
 * population without a checkpoint in collision} (tr C of the factor-free sampler's
 * distribution is taken from the elites: sum_j w_j |x_(j) - mu|^2 + D eps) into a device ring
 * of the last 256 iterations. cp_set_endpoints restarts the record. */
int cp_set_metrics(cp_planner *p, int32_t on);

/* Copy up to max_rows of the most recent metric rows (host double[rows][5], oldest first)
 * and their count to *n_rows (synchronises the planner's stream). Errors: CP_ERR_ARG. */
int cp_get_metrics(cp_planner *p, double *h_rows, int32_t max_rows, int32_t *n_rows);

/* Copy the population of the last iteration of cp_plan (or of a batch run) and its costs:
 * d_xi float[N][K][4], d_J double[N] (either may be NULL). Only the planner's own draws
 * are kept here; cp_sample and cp_evaluate write the caller's buffers. */
int cp_get_population(const cp_planner *p, float *d_xi, double *d_J);

/* Philox4x32-10 (Salmon et al., SC'11) of n counters d_ctr (uint32[n][4], device) under
 * key = (uint32)seed, (uint32)(seed >> 32); d_out is uint32[n][4]. `stream` as above. */
int cp_philox4x32_10(const uint32_t *d_ctr, uint64_t key, int64_t n, uint32_t *d_out,
                     void *stream);

/* Differentiable form of the cost (the smooth surrogate of Eq. path opt used for gradient
 * polish): J_s = J_p + w_c lambda_c sum_k sum_{sphere, obstacle} beta softplus((m - sd) / beta)
 * + w_l J_l, with sd the pair's signed distance (Sec. 3.1), m = smooth_margin and
 * beta = smooth_beta. Pairs with sd > m + 30 beta are skipped (each would add less than
 * 1e-13 beta). d_xi is float[n][K][4] (n <= N); d_J receives double[n].
 * Errors: CP_ERR_STATE (no end points), CP_ERR_ARG. */
int cp_smooth_cost(cp_planner *p, const float *d_xi, int32_t n, double *d_J);

/* Adjoint of cp_smooth_cost: d_dxi[i] = gJ[i] * dJ_s(xi_i)/dxi_i (float[n][K][4]), with
 * d_gJ double[n] (NULL: all ones); d_J (may be NULL) receives J_s as in cp_smooth_cost. The
 * forward pass is recomputed per checkpoint (no tape in memory); per-candidate sums are
 * taken in a fixed order, so results are deterministic. Errors as cp_smooth_cost. */
int cp_smooth_cost_grad(cp_planner *p, const float *d_xi, int32_t n, const double *d_gJ,
                        double *d_J, float *d_dxi);

/* Gradient polish: `steps` plain gradient-descent steps xi <- xi - alpha dJ_s/dxi on the n
 * candidates d_xi (float[n][K][4], updated in place), e.g. the best candidates of a plan
 * before they are handed to a trajectory optimiser. Errors as cp_smooth_cost. */
int cp_polish(cp_planner *p, float *d_xi, int32_t n, int32_t steps, double alpha);

/* ------------------------------------------------------------------ batched form */

/* One planning query of a batch: its obstacle scene (host memory, copied at
 * cp_batch_init), its search parameters (sizes may differ between queries) and its start and
 * goal configurations. */
typedef struct cp_query {
    cp_scene scene;
    cp_params params;
    double q0[4];
    double qd[4];
} cp_query;

/* Result of one query: the control points of the final mean path (the first (K+8)*4
 * entries, four copies of q0, the K waypoints, four copies of qd) and its cost terms. */
typedef struct cp_batch_result {
    cp_plan_stats stats;
    double ctrl[(CP_MAX_WAYPOINTS + 8) * 4];
} cp_batch_result;

typedef struct cp_batch cp_batch;

/* Batched serving form of Algorithm 1 (Sec. 4.1; the many-query setting of Sec. 5.1):
 * nq independent queries planned together for `iters` iterations each, every stage of an
 * iteration one launch for all queries. The evaluation of step (2) is one persistent launch
 * per iteration: CTAs take tiles of (query, consecutive work items) from a device counter
 * and restage the query's obstacle index and spline table when the query of their tile
 * changes. Sampling (step 1), costs, the stable ranking (steps 3-4; a radix sort of all
 * queries' costs followed by passes on the query), the elites' moments (steps 5-6) and the
 * factors are segmented by query through block tables. Each query keeps its own planner
 * workspace, and its results equal those of its planner planning alone with cp_plan bit
 * for bit. The whole run (end points in, initial distributions, the iterations, the mean
 * paths' evaluation, results out) is recorded once as one CUDA graph. Every query must use
 * the polar obstacle index (grid_cell > 0), the paper's update rule, the factor sampler and
 * the sphere collision model, with one crane model for all. Allocation happens here only.
 * Errors: CP_ERR_ARG (a query outside that form; the message names it), as cp_plan_init
 * (for the first query that fails), CP_ERR_CUDA. */
int cp_batch_init(const cp_model *model, const cp_query *queries, int32_t nq, int32_t iters,
                  cp_batch **out);

/* Change the start and goal of query q for the next cp_batch_run (host values). */
int cp_batch_set_endpoints(cp_batch *b, int32_t q, const double h_q0[4], const double h_qd[4]);

/* Run every query once: one launch of the recorded graph, then wait for it. results (host,
 * nq entries, may be NULL) receives each query's result. Errors: CP_ERR_NUMERIC when a
 * query's covariance lost positive definiteness, CP_ERR_ARG when a query's obstacle index
 * overflowed, CP_ERR_CUDA. */
int cp_batch_run(cp_batch *b, cp_batch_result *results);

/* Launch shape of the batched evaluation (picked by the autotuner). Results do not depend
 * on it: an item's arithmetic and the order of its sums are fixed by the query alone. */
typedef struct cp_batch_shape {
    int32_t threads;          /* CTA size: 128, 256 or 512 */
    int32_t ctas_per_sm;      /* resident CTAs per SM (0: as many as fit) */
    int32_t items_per_warp;   /* work items per warp in a tile (1..64): a tile holds
                                 threads / 32 * items_per_warp consecutive items */
} cp_batch_shape;

/* Set the launch shape (default {256, 0, 2}) and record the graph again. Errors:
 * CP_ERR_ARG (a field outside its range), CP_ERR_CUDA. */
int cp_batch_set_shape(cp_batch *b, const cp_batch_shape *shape);

/* Time the batched evaluation alone: `reps` launches over every query's current population
 * (whatever the last run left), CUDA events around each launch; *ms = the mean duration.
 * Errors: CP_ERR_ARG, CP_ERR_CUDA. */
int cp_batch_evaluate(cp_batch *b, int32_t reps, double *ms);

typedef struct cp_batch_info {
    int64_t kernel_nodes;     /* kernels recorded in the graph (one cp_batch_run) */
    int64_t eval_tiles;       /* tiles of one iteration's evaluation */
    int32_t eval_ctas;        /* CTAs of the persistent evaluation launch */
    int32_t eval_launches;    /* persistent evaluation launches per run (iterations + 1) */
    int64_t candidates;       /* sum of the queries' N */
    double last_run_ms;       /* device time of the last cp_batch_run (CUDA events around the
                                 graph launch: input copy to result copy), 0 before the first */
} cp_batch_info;

int cp_batch_get_info(const cp_batch *b, cp_batch_info *out);

/* The planner behind query q (owned by the batch): it holds the query's state after a run
 * (cp_get_distribution, cp_get_elites), and can plan the query alone with cp_plan; do not
 * use it while cp_batch_run is running. NULL when q is out of range. */
cp_planner *cp_batch_planner(cp_batch *b, int32_t q);

/* Release the batch, its planners, stream and graph. NULL is ignored. */
void cp_batch_destroy(cp_batch *b);

/* ------------------------------------------------------------------ trajectory step */

/* Trajectory tracking optimisation of Sec. 4.2 (Eq. discrete), batched: each planned path
 * q*(s) becomes a near-time-optimal trajectory by trapezoidal direct collocation on N
 * intervals,
 *   min  t_F + omega_s sum_{k=1..N} u_k^T R u_k + omega_t sum_{k=1..N} |q_a,k - q*(k/N)|^2
 *   s.t. x_{k+1} - x_k = h/2 (f(x_k, u_k) + f(x_{k+1}, u_{k+1})),  h = t_F / N,
 *        x_0 = (q*(0), 0), x_N = (q*(1), 0),  x_min <= x_k <= x_max.
 * The model f has the structure of Sec. 2.1 with synthetic parameters (the paper gives none):
 * x = (q1..q4, alpha, beta, dq1..dq4, dalpha, dbeta), u = (ddq1..ddq4): the actuated joints
 * driven through their accelerations (subordinate velocity controllers), and the grapple's
 * two passive swing angles, a point mass on a rigid link of length grapple_len under the tip
 * (plumb at alpha = beta = 0, direction (sin a, cos a sin b, -cos a cos b)), whose
 * accelerations follow from the pendulum's Euler-Lagrange equations with the tip's
 * acceleration. Bounds: the cp_model joint limits, |dq_j| <= dq_max[j], |alpha|, |beta| <=
 * swing_max. Solver (the paper uses IPOPT): augmented Lagrangian on the equalities
 * (multipliers updated `outer` times, lambda += rho c), quadratic penalty rho_b on the bounds,
 * `inner` Levenberg-Marquardt steps (J^T J + mu (diag J^T J + 1e-9)) dz = -(e_t + J^T r) per
 * update, a step kept when t_F + 1/2 |r|^2 decreases (mu / 3, else mu * 4, from mu0). FP64.
 * The variables of one trajectory are z = (t_F, w_0, ..., w_N), w_k = (x_k, u_k): 1 + 16 (N+1)
 * doubles. */
typedef struct cp_traj_params {
    int32_t N;            /* collocation intervals, 2..255 */
    double omega_s;       /* effort weight */
    double omega_t;       /* tracking weight */
    double R[4];          /* diagonal of R (>= 0) */
    double dq_max[4];     /* velocity limits of q1..q4 (> 0; rad/s, m/s) */
    double swing_max;     /* bound of the swing angles (rad, 0 < swing_max < 1.5) */
    double grapple_len;   /* link length of the grapple pendulum (m, > 0) */
    double rho;           /* augmented-Lagrangian weight (> 0) */
    double rho_b;         /* bound-penalty weight (>= 0) */
    int32_t outer;        /* multiplier updates */
    int32_t inner;        /* Levenberg-Marquardt steps per update */
    double mu0;           /* initial damping (> 0) */
} cp_traj_params;

typedef struct cp_traj cp_traj;

/* Create a batched trajectory solver on the current device for up to max_paths trajectories:
 * validates, allocates its workspace (about 5 KB per grid point per trajectory) and keeps the
 * stream. Errors: CP_ERR_ARG, CP_ERR_CUDA. */
int cp_traj_init(const cp_model *model, const cp_traj_params *tp, int32_t max_paths, void *stream,
                 cp_traj **out);

/* Release the solver (synchronises its stream first). NULL is ignored. */
void cp_traj_destroy(cp_traj *t);

/* The targets q*(k / N), k = 0..N, of n planned paths given by their control points d_ctrl
 * (double[n][K+8][4], the layout cp_plan returns): the cubic B-spline of Sec. 4.1 on the K + 3
 * moving spans. d_q_star receives double[n][N+1][4]. Errors: CP_ERR_ARG. */
int cp_traj_targets(cp_traj *t, const double *d_ctrl, int32_t K, int32_t n, double *d_q_star);

/* The solver's starting point from the targets: q_a = q*_k, velocities by central differences
 * and inputs by second differences over t_F, the swing at rest, t_F = 1.5 x the largest
 * (total variation of a joint over its velocity limit). d_z receives double[n][1 + 16 (N+1)].
 * Errors: CP_ERR_ARG. */
int cp_traj_initial_guess(cp_traj *t, const double *d_q_star, int32_t n, double *d_z);

/* One Levenberg-Marquardt step dz (double[n][1 + 16 (N+1)]) at z with multipliers d_lam
 * (double[n][12 (N+2)]: the N defects, then the start and end states) and damping mu, without
 * acceptance (for tests and diagnostics). Errors: CP_ERR_ARG. */
int cp_traj_step(cp_traj *t, const double *d_q_star, int32_t n, const double *d_z, const double *d_lam,
                 double mu, double *d_dz);

/* Solve the n trajectories from their starting points d_z (updated in place to the result).
 * d_stats receives double[n][4]: t_F, the final objective t_F + 1/2 |r|^2, the largest
 * equality-constraint error and the largest bound violation. Asynchronous on the solver's
 * stream. Errors: CP_ERR_ARG. */
int cp_traj_solve(cp_traj *t, const double *d_q_star, int32_t n, double *d_z, double *d_stats);

/* Size of the fixed device scratch behind cp_evaluate_static (bytes, per GPU). */
#define CP_STATIC_SCRATCH_BYTES (32u << 20)

/* Candidate costs as cp_evaluate computes them with the link-sphere collision model (the
 * broad-phase form; the convex-hull model and the grid are not available here), for callers
 * that may not allocate device memory: it calls no cudaMalloc, cudaFree or other allocating
 * routine and needs no planner. The paper has no counterpart; this entry point exists for
 * callers such as a real-time control loop, where cudaMalloc may stall the device for an
 * unbounded time, or a plug-in whose host application owns all device memory.
 * All scratch (a status word, obstacle records, spline table, partial sums: about 20 bytes
 * per candidate per 32 checkpoints plus 32 bytes per obstacle and per checkpoint of a span)
 * lives in one fixed array of CP_STATIC_SCRATCH_BYTES that every GPU loading the library
 * keeps until the process exits; larger requests fail with CP_ERR_ARG and say how much they
 * need. Inputs, all on the current device except model, h_q0 and h_qd (host): d_cyl[n_cyl]
 * and d_box[n_box] in the cp_cylinder / cp_box layout, the candidates d_xi (float[n][K][4]).
 * Outputs as in cp_evaluate: d_J (required), d_flag and d_terms (may be NULL). Work is
 * ordered on `stream`; the call returns before it completes. If the bounded wait for the
 * obstacle staging gives up on the device, every d_J of the call is NaN, every d_flag is 1
 * and the d_terms are NaN (the failure is visible without a synchronisation).
 * The first call on a device looks up the scratch array's device address (make that first
 * call before any stream capture); the address is kept, so do not call this after a
 * cudaDeviceReset of the host application. Every call reuses the same scratch and
 * overwrites all of it that it reads, so two calls that overlap on the GPU (different
 * streams, or different host threads) race with each other: serialise them. */
int cp_evaluate_static(const cp_model *model, const cp_cylinder *d_cyl, int32_t n_cyl,
                       const cp_box *d_box, int32_t n_box, int32_t n_waypoints,
                       int32_t substeps, double w_c, double w_l, double lambda_c,
                       const double h_q0[4], const double h_qd[4], const float *d_xi,
                       int32_t n, double *d_J, uint8_t *d_flag, double *d_terms,
                       void *stream);

/* Test hook: while on (1), cp_evaluate_static issues no staging copy, so that its bounded
 * wait runs out on the device (about one second) and the call's results read as failed.
 * 0 turns it off; no other effect. */
void cp_debug_static_withhold_staging(int32_t on);

/* Turn per-stage timing on (1) or off (0); turning it on clears the accumulators. */
int cp_set_timing(cp_planner *p, int32_t on);

/* Synchronise the planner's stream and return the accumulated stage times. */
int cp_get_timing(cp_planner *p, cp_timing *out);

/* Measured throughput of the FP32 and the FP64 FMA pipes of the current device (TFLOP/s,
 * an FMA counted as 2 flops): compute-only kernels of eight independent FMA chains per
 * thread, eight CTAs of 256 threads per SM, the faster of two timed launches after one
 * warm-up. The paper has no counterpart; these are the denominators of the reported FP32
 * and FP64 utilisation. Takes a few milliseconds; allocates and frees a small buffer. */
int cp_alu_peaks(double *fp32_tflops, double *fp64_tflops);

#ifdef __cplusplus
}
#endif

#endif /* CRANEPLAN_H */
