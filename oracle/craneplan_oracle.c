/*
 * craneplan_oracle.c -- plain, slow, FP64 CPU oracle of the stochastic B-spline path
 * optimisation of "GPU-Accelerated Motion Planning of an Underactuated Forestry Crane
 * in Cluttered Environments" (arXiv 2503.14160), Sec. 4.1.
 *
 * TEST INFRASTRUCTURE. This file is the checker the CUDA library is compared against.
 * Only the test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark load it; the product path never does. It shares no code, header, table
 * or constant generator with the CUDA library.
 *
 * Everything is IEEE double, evaluated in the order the definitions are written.
 * Compile with -ffp-contract=off so that x86 and Arm give identical results.
 *
 * What is here (paper section / reading it follows):
 *   o_philox4x32_10     counter-based generator, Salmon et al. SC'11 (Philox4x32, 10 rounds)
 *   o_normals           Box-Muller on Philox words: the z of Algorithm 1 step (1)
 *   o_fk                crane chain forward kinematics (Sec. 2, Eq. FK; chain read as below)
 *   o_sdf_cylinder      signed distance to a vertical capped cylinder (Sec. 3.1, d<0 = collision)
 *   o_sdf_box           signed distance to an axis-aligned box (Sec. 3.1)
 *   o_signed_distance   d(q) = min over link spheres and obstacles (Sec. 3.1), brute force
 *   o_bspline           q(s) = sum_i P_i N_i^3(s), Cox-de Boor on a uniform knot vector (Sec. 4.1)
 *   o_path_cost         J = J_p + w_c J_c + w_l J_l (Eq. path opt, all three sums)
 *   o_path_cost_batch   the same for N candidates (Algorithm 1 step (2)); OpenMP over candidates
 *   o_path_cost_batch_grid  the same with d(q) through a uniform obstacle grid (equal to
 *                       the brute force in every cost term and flag; for timing large scenes)
 *   o_smooth_cost       the softplus-penalty variant of J used by the differentiable form
 *   o_smooth_grad       its analytic gradient with respect to the K free control points
 *   o_ik_residual       residual and Jacobian of the collision-free IK (Sec. 3.2, Eq. IK opt)
 *   o_fk_tip_batch      the tip of o_fk for many configurations
 *
 * Readings of the paper that the code depends on (the paper is silent or garbled here):
 *   chain   slew q1 about world z; boom pitch q2 (elevation from horizontal); jib pitch q3
 *           relative to the boom in the same vertical plane; telescope q4 extends the jib
 *           axis; the grapple hangs plumb below the tip (passive joints at equilibrium).
 *           e_b = (cos q2 cos q1, cos q2 sin q1, sin q2), e_j the same with q2+q3,
 *           O = (0,0,base_z), J = O + L_b e_b, T = J + (L_j + q4) e_j.
 *   spheres link 0: O + t e_b; link 1: J + t e_j; link 2: J + (L_j + t q4) e_j;
 *           link 3: T - t z.  (t = the sphere's offset)
 *   spline  n_c = K + 8 control points: P_0..P_3 = q_0, P_4..P_{K+3} = the K free points,
 *           P_{K+4}..P_{K+7} = q_d; uniform knots t_i = i; the K+3 spans that move
 *           ([4, K+7] in knot units) carry s in [0,1]: tau(s) = 4 + (K+3) s.
 *   checkpoints s_k = k / n_s, n_s = (K+3) S, k = 0..n_s; the sums of Eq. path opt run
 *           over k = 1..n_s.
 *   r_c     r_c(q) = lambda_c * max(0, -d(q))  (the IK collision residual of Sec. 3.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_MAX_SPHERES 32

typedef struct {
    double base_z;       /* height of the slew / boom pivot above the ground (m) */
    double boom_len;     /* L_b: boom pivot to jib pivot (m) */
    double jib_len;      /* L_j: jib pivot to the tip at zero telescope extension (m) */
    double q_min[4];
    double q_max[4];
    int32_t n_spheres;
    int32_t link[O_MAX_SPHERES];   /* 0 boom, 1 jib, 2 telescope, 3 grapple */
    double offset[O_MAX_SPHERES];  /* t of the placement rule above */
    double radius[O_MAX_SPHERES];
} o_model;

typedef struct {
    int32_t n_cyl;
    const double *cyl;   /* [n_cyl][5]: cx, cy, R, z_lo, z_hi */
    int32_t n_box;
    const double *box;   /* [n_box][6]: lo_x, lo_y, lo_z, hi_x, hi_y, hi_z */
} o_scene;

typedef struct {
    int32_t K;           /* free control points (waypoints) */
    int32_t S;           /* checkpoints per moving span */
    double w_c, w_l;     /* weights of J_c and J_l in Eq. path opt */
    double lambda_c;     /* scale of r_c */
    double margin;       /* smooth form: penalty margin m (m) */
    double beta;         /* smooth form: softplus width (m) */
} o_cost_params;

/* ------------------------------------------------------------------ Philox4x32-10 */

/* One Philox4x32 round (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32->64 products
 * of words 0 and 2 with the round multipliers, the high halves xor-ed with the other
 * words and the round key, the low halves passed through. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

/* Philox4x32 with 10 rounds; the key is bumped by the Weyl constants between rounds. */
void o_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

void o_philox4x32_10_batch(const uint32_t *ctr, const uint32_t key[2], int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) o_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Box-Muller (Box & Muller 1958) on two Philox words: the top 24 bits of each word give
 * u1 = (a+1) 2^-24 in (0,1] and u2 = b 2^-24 in [0,1), both exact in binary32;
 * z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2). */
static void box_muller(uint32_t x0, uint32_t x1, double *z0, double *z1)
{
    const double u1 = ((double)(x0 >> 8) + 1.0) * 0x1p-24;
    const double u2 = (double)(x1 >> 8) * 0x1p-24;
    const double r = sqrt(-2.0 * log(u1));
    const double a = 2.0 * M_PI * u2;
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

/* The D = 4K standard normals of candidate i at iteration t of query q (Algorithm 1 step
 * (1)). Block j of the counter (j, i, t, q) under key (seed_lo, seed_hi) gives the four
 * normals z[4j..4j+3] (control point j, joints 1..4). */
void o_normals(uint64_t seed, uint32_t t, uint32_t q, int32_t i, int32_t K, double *z)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t j = 0; j < K; ++j) {
        const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)i, t, q};
        uint32_t x[4];
        o_philox4x32_10(ctr, key, x);
        box_muller(x[0], x[1], &z[4 * j + 0], &z[4 * j + 1]);
        box_muller(x[2], x[3], &z[4 * j + 2], &z[4 * j + 3]);
    }
}

void o_normals_batch(uint64_t seed, uint32_t t, uint32_t q, int32_t n, int32_t K, double *z)
{
    for (int32_t i = 0; i < n; ++i) o_normals(seed, t, q, i, K, z + (int64_t)i * 4 * K);
}

/* ------------------------------------------------------------------ kinematics */

/* Sphere centres of the crane at configuration q (Sec. 2, Eq. FK with the chain read
 * as in the file header). Also returns the jib pivot J and the tip T when asked. */
void o_fk(const o_model *m, const double q[4], double *centres /* [n][3] */,
          double *jib_pivot /* [3] or NULL */, double *tip /* [3] or NULL */)
{
    const double eb[3] = {cos(q[1]) * cos(q[0]), cos(q[1]) * sin(q[0]), sin(q[1])};
    const double a = q[1] + q[2];
    const double ej[3] = {cos(a) * cos(q[0]), cos(a) * sin(q[0]), sin(a)};
    const double O[3] = {0.0, 0.0, m->base_z};
    double J[3], T[3];
    for (int c = 0; c < 3; ++c) J[c] = O[c] + m->boom_len * eb[c];
    for (int c = 0; c < 3; ++c) T[c] = J[c] + (m->jib_len + q[3]) * ej[c];
    for (int s = 0; s < m->n_spheres; ++s) {
        const double t = m->offset[s];
        double *p = centres + 3 * s;
        switch (m->link[s]) {
        case 0: for (int c = 0; c < 3; ++c) p[c] = O[c] + t * eb[c]; break;
        case 1: for (int c = 0; c < 3; ++c) p[c] = J[c] + t * ej[c]; break;
        case 2: for (int c = 0; c < 3; ++c) p[c] = J[c] + (m->jib_len + t * q[3]) * ej[c]; break;
        default:
            p[0] = T[0];
            p[1] = T[1];
            p[2] = T[2] - t;
            break;
        }
    }
    if (jib_pivot) memcpy(jib_pivot, J, sizeof J);
    if (tip) memcpy(tip, T, sizeof T);
}

/* ------------------------------------------------------------------ signed distances */

/* Exact signed distance from point p to the vertical capped cylinder {rho <= R,
 * z_lo <= z <= z_hi}: the standard two-component form, with a = rho - R (radial) and
 * b = max(z_lo - z, z - z_hi) (axial): min(max(a, b), 0) + |(max(a,0), max(b,0))|. */
double o_sdf_cylinder(const double p[3], const double *cyl /* cx, cy, R, z_lo, z_hi */)
{
    const double rho = hypot(p[0] - cyl[0], p[1] - cyl[1]);
    const double a = rho - cyl[2];
    const double b = fmax(cyl[3] - p[2], p[2] - cyl[4]);
    return fmin(fmax(a, b), 0.0) + hypot(fmax(a, 0.0), fmax(b, 0.0));
}

/* Exact signed distance from p to the axis-aligned box [lo, hi]: with centre c and
 * half-extent h, q_i = |p_i - c_i| - h_i, d = |max(q, 0)| + min(max_i q_i, 0). */
double o_sdf_box(const double p[3], const double *box /* lo[3], hi[3] */)
{
    double qv[3], outside = 0.0, inner = -HUGE_VAL;
    for (int c = 0; c < 3; ++c) {
        const double centre = 0.5 * (box[c] + box[3 + c]);
        const double half = 0.5 * (box[3 + c] - box[c]);
        qv[c] = fabs(p[c] - centre) - half;
        outside += fmax(qv[c], 0.0) * fmax(qv[c], 0.0);
        inner = fmax(inner, qv[c]);
    }
    return sqrt(outside) + fmin(inner, 0.0);
}

/* d(q): minimum over all link spheres and all obstacles of (obstacle SDF at the
 * sphere centre) - (sphere radius); d < 0 means collision (Sec. 3.1). +inf when the
 * scene is empty. Brute force over every pair. */
double o_signed_distance(const o_model *m, const o_scene *sc, const double q[4])
{
    double centres[3 * O_MAX_SPHERES];
    o_fk(m, q, centres, NULL, NULL);
    double d = HUGE_VAL;
    for (int s = 0; s < m->n_spheres; ++s) {
        const double *p = centres + 3 * s;
        for (int o = 0; o < sc->n_cyl; ++o)
            d = fmin(d, o_sdf_cylinder(p, sc->cyl + 5 * o) - m->radius[s]);
        for (int o = 0; o < sc->n_box; ++o)
            d = fmin(d, o_sdf_box(p, sc->box + 6 * o) - m->radius[s]);
    }
    return d;
}

/* Tips T of n configurations (o_fk, one after another): tips[n][3]. */
void o_fk_tip_batch(const o_model *m, const double *q, int64_t n, double *tips)
{
    double centres[3 * O_MAX_SPHERES];
    for (int64_t i = 0; i < n; ++i) o_fk(m, q + 4 * i, centres, NULL, tips + 3 * i);
}

void o_signed_distance_batch(const o_model *m, const o_scene *sc, const double *q, int64_t n,
                             double *d)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) d[i] = o_signed_distance(m, sc, q + 4 * i);
}

/* ------------------------------------------------------------------ B-spline */

/* All cubic basis functions N_{i,3}(tau), i = 0..n_c-1, on the uniform knots t_i = i
 * (i = 0..n_c+3), by the Cox-de Boor recursion written out degree by degree:
 *   N_{i,0}(tau) = 1 if t_i <= tau < t_{i+1}, else 0
 *   N_{i,p}(tau) = (tau - t_i)/(t_{i+p} - t_i) N_{i,p-1}(tau)
 *                + (t_{i+p+1} - tau)/(t_{i+p+1} - t_{i+1}) N_{i+1,p-1}(tau). */
void o_bspline_basis(int32_t n_c, double tau, double *basis /* [n_c] */)
{
    const int n_knots = n_c + 4;
    double N[64 + 4];
    for (int i = 0; i < n_knots - 1; ++i) {
        const double ti = (double)i, ti1 = (double)(i + 1);
        N[i] = (ti <= tau && tau < ti1) ? 1.0 : 0.0;
    }
    for (int p = 1; p <= 3; ++p) {
        for (int i = 0; i < n_knots - 1 - p; ++i) {
            const double ti = (double)i, tip = (double)(i + p);
            const double ti1 = (double)(i + 1), tip1 = (double)(i + p + 1);
            N[i] = (tau - ti) / (tip - ti) * N[i] + (tip1 - tau) / (tip1 - ti1) * N[i + 1];
        }
    }
    for (int i = 0; i < n_c; ++i) basis[i] = N[i];
}

/* q(tau) = sum_i P_i N_{i,3}(tau) for control points P[n_c][4]. */
void o_bspline(const double *P, int32_t n_c, double tau, double q[4])
{
    double basis[64];
    o_bspline_basis(n_c, tau, basis);
    for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int i = 0; i < n_c; ++i) acc += P[4 * i + c] * basis[i];
        q[c] = acc;
    }
}

/* The n_c = K + 8 control points of a candidate: four copies of q_0, the K free points
 * xi[K][4], four copies of q_d (Sec. 4.1, end-point clamping). */
static void assemble_control_points(int32_t K, const double *xi, const double q0[4],
                                    const double qd[4], double *P)
{
    for (int i = 0; i < 4; ++i) memcpy(P + 4 * i, q0, 4 * sizeof(double));
    memcpy(P + 16, xi, (size_t)K * 4 * sizeof(double));
    for (int i = 0; i < 4; ++i) memcpy(P + 4 * (K + 4 + i), qd, 4 * sizeof(double));
}

/* Path parameter of checkpoint k: s_k = k / n_s, mapped onto the moving spans. */
static double checkpoint_tau(int32_t K, int32_t S, int64_t k)
{
    const int64_t n_s = (int64_t)(K + 3) * S;
    const double s = (double)k / (double)n_s;
    return 4.0 + (double)(K + 3) * s;
}

/* ------------------------------------------------------------------ path cost */

typedef struct {
    double J, Jp, Jc, Jl;  /* total and the three terms of Eq. path opt */
    double length;         /* sum_k |q(s_k) - q(s_{k-1})|, the path length that is reported */
    int32_t flag;          /* 1 when d(q(s_k)) < 0 at some k = 1..n_s */
    int32_t n_flagged;     /* how many checkpoints are in collision */
} o_cost;

/* A distance function d(q) for the path cost: the brute-force o_signed_distance, or the
 * grid form below (equal wherever d < 0, which is all the cost uses). */
typedef double (*o_distance_fn)(const o_model *m, const o_scene *sc, const void *ctx, const double q[4]);

static double brute_distance(const o_model *m, const o_scene *sc, const void *ctx, const double q[4])
{
    (void)ctx;
    return o_signed_distance(m, sc, q);
}

/* Eq. path opt for one candidate with the distance function `dist`. d_out (optional,
 * [n_s + 1]) receives d(q(s_k)). */
static void path_cost_with(const o_model *m, const o_scene *sc, o_distance_fn dist, const void *ctx,
                           const o_cost_params *cp, const double *xi /* [K][4] */, const double q0[4],
                           const double qd[4], o_cost *out, double *d_out)
{
    const int32_t K = cp->K, n_c = K + 8;
    const int64_t n_s = (int64_t)(K + 3) * cp->S;
    double P[4 * 72];
    assemble_control_points(K, xi, q0, qd, P);
    double q_prev[4];
    o_bspline(P, n_c, checkpoint_tau(K, cp->S, 0), q_prev);
    if (d_out) d_out[0] = dist(m, sc, ctx, q_prev);
    double Jp = 0.0, Jc = 0.0, Jl = 0.0, len = 0.0;
    int32_t flag = 0, n_flagged = 0;
    for (int64_t k = 1; k <= n_s; ++k) {
        double q[4];
        o_bspline(P, n_c, checkpoint_tau(K, cp->S, k), q);
        double step2 = 0.0;
        for (int c = 0; c < 4; ++c) step2 += (q[c] - q_prev[c]) * (q[c] - q_prev[c]);
        Jp += step2;
        len += sqrt(step2);
        const double d = dist(m, sc, ctx, q);
        if (d_out) d_out[k] = d;
        Jc += cp->lambda_c * fmax(0.0, -d);
        if (d < 0.0) {
            flag = 1;
            ++n_flagged;
        }
        for (int c = 0; c < 4; ++c) {
            const double hi = fmax(0.0, q[c] - m->q_max[c]);
            const double lo = fmax(0.0, m->q_min[c] - q[c]);
            Jl += hi * hi + lo * lo;
        }
        memcpy(q_prev, q, sizeof q);
    }
    out->Jp = Jp;
    out->Jc = Jc;
    out->Jl = Jl;
    out->J = Jp + cp->w_c * Jc + cp->w_l * Jl;
    out->length = len;
    out->flag = flag;
    out->n_flagged = n_flagged;
}

/* Eq. path opt for one candidate, d(q) by brute force over every pair. */
void o_path_cost(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                 const double *xi /* [K][4] */, const double q0[4], const double qd[4],
                 o_cost *out, double *d_out)
{
    path_cost_with(m, sc, brute_distance, NULL, cp, xi, q0, qd, out, d_out);
}

/* Algorithm 1 step (2) for n candidates xi[n][K][4]. d_out (optional) is [n][n_s+1]. */
void o_path_cost_batch(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                       const double *xi, int64_t n, const double q0[4], const double qd[4],
                       o_cost *out, double *d_out)
{
    const int64_t n_s = (int64_t)(cp->K + 3) * cp->S;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        o_path_cost(m, sc, cp, xi + i * 4 * cp->K, q0, qd, out + i,
                    d_out ? d_out + i * (n_s + 1) : NULL);
}

/* ------------------------------------------------------------------ grid form (timing) */

/* A uniform 2-D grid of the obstacles, for timing the oracle on large scenes only (the
 * parity tests use the brute-force d(q)). Cells of side h cover the bounding box of every
 * obstacle's footprint dilated by the largest sphere radius (plus 1 mm); each obstacle is
 * listed in every cell its dilated footprint overlaps. A sphere that penetrates an obstacle
 * has its centre inside that footprint, so the obstacles listed in the cell of the centre
 * include every one the sphere penetrates, and the minimum over them equals the brute-force
 * d(q) wherever that is negative; elsewhere it is non-negative (or +inf), so the penalty
 * max(0, -d) and the collision flags of Eq. path opt are those of the brute force. */
typedef struct {
    double x0, y0, h;
    int32_t nx, ny;
    int32_t *start;   /* [nx ny + 1] */
    int32_t *items;   /* obstacle ids: cylinders 0..n_cyl-1, then boxes */
} o_grid;

static void footprint(const o_scene *sc, double r, int id, double f[4] /* x0, x1, y0, y1 */)
{
    if (id < sc->n_cyl) {
        const double *c = sc->cyl + 5 * id;
        const double reach = c[2] + r;
        f[0] = c[0] - reach;
        f[1] = c[0] + reach;
        f[2] = c[1] - reach;
        f[3] = c[1] + reach;
    } else {
        const double *b = sc->box + 6 * (id - sc->n_cyl);
        f[0] = b[0] - r;
        f[1] = b[3] + r;
        f[2] = b[1] - r;
        f[3] = b[4] + r;
    }
}

static void cell_span(const o_grid *g, const double f[4], int c[4] /* ix0, ix1, iy0, iy1 */)
{
    c[0] = (int)floor((f[0] - g->x0) / g->h);
    c[1] = (int)floor((f[1] - g->x0) / g->h);
    c[2] = (int)floor((f[2] - g->y0) / g->h);
    c[3] = (int)floor((f[3] - g->y0) / g->h);
    if (c[0] < 0) c[0] = 0;
    if (c[2] < 0) c[2] = 0;
    if (c[1] > g->nx - 1) c[1] = g->nx - 1;
    if (c[3] > g->ny - 1) c[3] = g->ny - 1;
}

/* Build the grid (returns 0, or -1 when memory runs out); free with o_grid_free. */
static int grid_build(const o_model *m, const o_scene *sc, double h, o_grid *g)
{
    double r = 0.0;
    for (int s = 0; s < m->n_spheres; ++s) r = fmax(r, m->radius[s]);
    r += 1e-3;
    const int n_obs = sc->n_cyl + sc->n_box;
    double lo_x = 0.0, hi_x = 0.0, lo_y = 0.0, hi_y = 0.0;
    for (int id = 0; id < n_obs; ++id) {
        double f[4];
        footprint(sc, r, id, f);
        if (id == 0 || f[0] < lo_x) lo_x = f[0];
        if (id == 0 || f[1] > hi_x) hi_x = f[1];
        if (id == 0 || f[2] < lo_y) lo_y = f[2];
        if (id == 0 || f[3] > hi_y) hi_y = f[3];
    }
    g->h = h;
    g->x0 = lo_x;
    g->y0 = lo_y;
    g->nx = (int)floor((hi_x - lo_x) / h) + 1;
    g->ny = (int)floor((hi_y - lo_y) / h) + 1;
    const int64_t cells = (int64_t)g->nx * g->ny;
    g->start = calloc((size_t)cells + 1, sizeof(int32_t));
    int32_t *fill = calloc((size_t)cells, sizeof(int32_t));
    if (!g->start || !fill) {
        free(g->start);
        free(fill);
        return -1;
    }
    for (int pass = 0; pass < 2; ++pass) {   /* count, then fill */
        for (int id = 0; id < n_obs; ++id) {
            double f[4];
            int c[4];
            footprint(sc, r, id, f);
            cell_span(g, f, c);
            for (int iy = c[2]; iy <= c[3]; ++iy)
                for (int ix = c[0]; ix <= c[1]; ++ix) {
                    const int64_t cell = (int64_t)iy * g->nx + ix;
                    if (pass == 0) g->start[cell + 1] += 1;
                    else g->items[g->start[cell] + fill[cell]++] = id;
                }
        }
        if (pass == 0) {
            for (int64_t cell = 0; cell < cells; ++cell) g->start[cell + 1] += g->start[cell];
            g->items = malloc(sizeof(int32_t) * (size_t)(g->start[cells] > 0 ? g->start[cells] : 1));
            if (!g->items) {
                free(g->start);
                free(fill);
                return -1;
            }
        }
    }
    free(fill);
    return 0;
}

static void grid_free(o_grid *g)
{
    free(g->start);
    free(g->items);
}

/* d(q) over the obstacles listed in the cells of the sphere centres (see above). */
static double grid_distance(const o_model *m, const o_scene *sc, const void *ctx, const double q[4])
{
    const o_grid *g = (const o_grid *)ctx;
    double centres[3 * O_MAX_SPHERES];
    o_fk(m, q, centres, NULL, NULL);
    double d = HUGE_VAL;
    for (int s = 0; s < m->n_spheres; ++s) {
        const double *p = centres + 3 * s;
        const double fx = floor((p[0] - g->x0) / g->h), fy = floor((p[1] - g->y0) / g->h);
        if (!(fx >= 0.0 && fy >= 0.0 && fx < (double)g->nx && fy < (double)g->ny)) continue;
        const int64_t cell = (int64_t)fy * g->nx + (int64_t)fx;
        for (int32_t it = g->start[cell]; it < g->start[cell + 1]; ++it) {
            const int id = g->items[it];
            if (id < sc->n_cyl) d = fmin(d, o_sdf_cylinder(p, sc->cyl + 5 * id) - m->radius[s]);
            else d = fmin(d, o_sdf_box(p, sc->box + 6 * (id - sc->n_cyl)) - m->radius[s]);
        }
    }
    return d;
}

/* o_path_cost_batch with d(q) through a uniform grid of cell side h (m): the same J, terms,
 * flags and collision counts as the brute force (see above). Returns 0, or -1 when the
 * grid could not be allocated. d_out, when given, holds the grid distances (equal to the
 * brute force's where negative). */
int32_t o_path_cost_batch_grid(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                               const double *xi, int64_t n, const double q0[4], const double qd[4],
                               double h, o_cost *out, double *d_out)
{
    o_grid g;
    if (!(h > 0.0) || grid_build(m, sc, h, &g) != 0) return -1;
    const int64_t n_s = (int64_t)(cp->K + 3) * cp->S;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        path_cost_with(m, sc, grid_distance, &g, cp, xi + i * 4 * cp->K, q0, qd, out + i,
                       d_out ? d_out + i * (n_s + 1) : NULL);
    grid_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ smooth form */

/* softplus(x) = ln(1 + e^x), evaluated without overflow. */
static double softplus(double x)
{
    return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

/* Smooth collision penalty at configuration q: lambda_c times the sum over every
 * sphere-obstacle pair of beta * softplus((margin - sd) / beta), sd the pair's signed
 * distance. It replaces max(0, -d) by a C-infinity surrogate so that the cost has a
 * gradient everywhere. */
double o_smooth_penalty(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                        const double q[4])
{
    double centres[3 * O_MAX_SPHERES];
    o_fk(m, q, centres, NULL, NULL);
    double acc = 0.0;
    for (int s = 0; s < m->n_spheres; ++s) {
        const double *p = centres + 3 * s;
        for (int o = 0; o < sc->n_cyl; ++o) {
            const double sd = o_sdf_cylinder(p, sc->cyl + 5 * o) - m->radius[s];
            acc += cp->beta * softplus((cp->margin - sd) / cp->beta);
        }
        for (int o = 0; o < sc->n_box; ++o) {
            const double sd = o_sdf_box(p, sc->box + 6 * o) - m->radius[s];
            acc += cp->beta * softplus((cp->margin - sd) / cp->beta);
        }
    }
    return cp->lambda_c * acc;
}

/* J_smooth = J_p + w_c sum_k smooth_penalty(q(s_k)) + w_l J_l, k = 1..n_s. */
double o_smooth_cost(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                     const double *xi, const double q0[4], const double qd[4])
{
    const int32_t K = cp->K, n_c = K + 8;
    const int64_t n_s = (int64_t)(K + 3) * cp->S;
    double P[4 * 72];
    assemble_control_points(K, xi, q0, qd, P);
    double q_prev[4];
    o_bspline(P, n_c, checkpoint_tau(K, cp->S, 0), q_prev);
    double Jp = 0.0, Jc = 0.0, Jl = 0.0;
    for (int64_t k = 1; k <= n_s; ++k) {
        double q[4];
        o_bspline(P, n_c, checkpoint_tau(K, cp->S, k), q);
        for (int c = 0; c < 4; ++c) Jp += (q[c] - q_prev[c]) * (q[c] - q_prev[c]);
        Jc += o_smooth_penalty(m, sc, cp, q);
        for (int c = 0; c < 4; ++c) {
            const double hi = fmax(0.0, q[c] - m->q_max[c]);
            const double lo = fmax(0.0, m->q_min[c] - q[c]);
            Jl += hi * hi + lo * lo;
        }
        memcpy(q_prev, q, sizeof q);
    }
    return Jp + cp->w_c * Jc + cp->w_l * Jl;
}

void o_smooth_cost_batch(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                         const double *xi, int64_t n, const double q0[4], const double qd[4],
                         double *J)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) J[i] = o_smooth_cost(m, sc, cp, xi + i * 4 * cp->K, q0, qd);
}

/* ------------------------------------------------------------------ gradient */

/* Jacobian of every sphere centre with respect to q: jac[s][c][j] = d centre_s[c] / d q_j,
 * from the chain of o_fk (each link point is a sum of terms in e_b, e_j and z). */
static void fk_jacobian(const o_model *m, const double q[4], double *jac /* [n][3][4] */)
{
    const double c1 = cos(q[0]), s1 = sin(q[0]);
    const double c2 = cos(q[1]), s2 = sin(q[1]);
    const double a = q[1] + q[2];
    const double c23 = cos(a), s23 = sin(a);
    /* e_b and its derivatives by q1, q2; e_j and its derivatives by q1, q2 (= by q3) */
    const double eb[3] = {c2 * c1, c2 * s1, s2};
    const double deb1[3] = {-c2 * s1, c2 * c1, 0.0};
    const double deb2[3] = {-s2 * c1, -s2 * s1, c2};
    const double ej[3] = {c23 * c1, c23 * s1, s23};
    const double dej1[3] = {-c23 * s1, c23 * c1, 0.0};
    const double dej2[3] = {-s23 * c1, -s23 * s1, c23};
    (void)eb;
    for (int s = 0; s < m->n_spheres; ++s) {
        const double t = m->offset[s];
        double A = 0.0, B = 0.0, G = 0.0;   /* centre = O + A e_b + (B + G q4) e_j + ... */
        switch (m->link[s]) {
        case 0: A = t; break;
        case 1: A = m->boom_len; B = t; break;
        case 2: A = m->boom_len; B = m->jib_len; G = t; break;
        default: A = m->boom_len; B = m->jib_len; G = 1.0; break;
        }
        const double L = B + G * q[3];
        double *J = jac + 12 * s;
        for (int c = 0; c < 3; ++c) {
            J[4 * c + 0] = A * deb1[c] + L * dej1[c];
            J[4 * c + 1] = A * deb2[c] + L * dej2[c];
            J[4 * c + 2] = L * dej2[c];
            J[4 * c + 3] = G * ej[c];
        }
    }
}

/* Gradient of the capped-cylinder SDF at p (the SDF is piecewise smooth: radial on the
 * side, axial on the caps, along (a, b) off the rim; inside, the nearer face). */
static void sdf_cylinder_grad(const double p[3], const double *cyl, double g[3])
{
    const double dx = p[0] - cyl[0], dy = p[1] - cyl[1];
    const double rho = hypot(dx, dy);
    const double a = rho - cyl[2];
    const double up = p[2] - cyl[4], down = cyl[3] - p[2];
    const double b = fmax(down, up);
    const double sz = up >= down ? 1.0 : -1.0;
    const double ux = rho > 0.0 ? dx / rho : 0.0, uy = rho > 0.0 ? dy / rho : 0.0;
    if (a > 0.0 && b > 0.0) {
        const double h = hypot(a, b);
        g[0] = a / h * ux;
        g[1] = a / h * uy;
        g[2] = b / h * sz;
    } else if (a >= b) {
        g[0] = ux;
        g[1] = uy;
        g[2] = 0.0;
    } else {
        g[0] = 0.0;
        g[1] = 0.0;
        g[2] = sz;
    }
}

/* Gradient of the box SDF at p: outside, along the clamped offset; inside, the face of the
 * largest q_i. */
static void sdf_box_grad(const double p[3], const double *box, double g[3])
{
    double qv[3], sg[3], out = 0.0;
    int imax = 0;
    for (int c = 0; c < 3; ++c) {
        const double centre = 0.5 * (box[c] + box[3 + c]);
        const double half = 0.5 * (box[3 + c] - box[c]);
        sg[c] = p[c] >= centre ? 1.0 : -1.0;
        qv[c] = fabs(p[c] - centre) - half;
        out += fmax(qv[c], 0.0) * fmax(qv[c], 0.0);
        if (qv[c] > qv[imax]) imax = c;
    }
    if (out > 0.0) {
        const double n = sqrt(out);
        for (int c = 0; c < 3; ++c) g[c] = fmax(qv[c], 0.0) / n * sg[c];
    } else {
        for (int c = 0; c < 3; ++c) g[c] = c == imax ? sg[c] : 0.0;
    }
}

/* logistic(x) = d softplus / dx */
static double logistic(double x)
{
    return x >= 0.0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x));
}

/* d/dq of the smooth collision penalty at q (4 values). */
static void smooth_penalty_grad(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                                const double q[4], double g[4])
{
    double centres[3 * O_MAX_SPHERES], jac[12 * O_MAX_SPHERES];
    o_fk(m, q, centres, NULL, NULL);
    fk_jacobian(m, q, jac);
    for (int j = 0; j < 4; ++j) g[j] = 0.0;
    for (int s = 0; s < m->n_spheres; ++s) {
        const double *p = centres + 3 * s;
        double dp[3] = {0.0, 0.0, 0.0};   /* d penalty / d centre */
        for (int o = 0; o < sc->n_cyl; ++o) {
            const double sd = o_sdf_cylinder(p, sc->cyl + 5 * o) - m->radius[s];
            const double w = -logistic((cp->margin - sd) / cp->beta);
            double gs[3];
            sdf_cylinder_grad(p, sc->cyl + 5 * o, gs);
            for (int c = 0; c < 3; ++c) dp[c] += w * gs[c];
        }
        for (int o = 0; o < sc->n_box; ++o) {
            const double sd = o_sdf_box(p, sc->box + 6 * o) - m->radius[s];
            const double w = -logistic((cp->margin - sd) / cp->beta);
            double gs[3];
            sdf_box_grad(p, sc->box + 6 * o, gs);
            for (int c = 0; c < 3; ++c) dp[c] += w * gs[c];
        }
        const double *J = jac + 12 * s;
        for (int j = 0; j < 4; ++j)
            for (int c = 0; c < 3; ++c) g[j] += cp->lambda_c * dp[c] * J[4 * c + j];
    }
}

/* Gradient of J_smooth (o_smooth_cost) with respect to the K free control points xi[K][4].
 * q(s_k) = sum_i N_i(tau_k) P_i is linear in the control points, so with r_k = dJ/dq(s_k),
 * dJ/dxi_f = sum_k r_k N_{4+f}(tau_k), where
 *   r_k = 2 (q_k - q_{k-1}) [k >= 1] - 2 (q_{k+1} - q_k) [k < n_s]
 *       + w_c d(penalty)/dq (q_k) + w_l d(J_l terms)/dq (q_k)   [k >= 1]. */
void o_smooth_grad(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                   const double *xi, const double q0[4], const double qd[4], double *grad)
{
    const int32_t K = cp->K, n_c = K + 8;
    const int64_t n_s = (int64_t)(K + 3) * cp->S;
    double P[4 * 72];
    assemble_control_points(K, xi, q0, qd, P);
    double *Q = (double *)malloc(sizeof(double) * 4 * (size_t)(n_s + 1));
    for (int64_t k = 0; k <= n_s; ++k) o_bspline(P, n_c, checkpoint_tau(K, cp->S, k), Q + 4 * k);
    for (int i = 0; i < 4 * K; ++i) grad[i] = 0.0;
    for (int64_t k = 0; k <= n_s; ++k) {
        const double *q = Q + 4 * k;
        double r[4] = {0.0, 0.0, 0.0, 0.0};
        if (k >= 1)
            for (int c = 0; c < 4; ++c) r[c] += 2.0 * (q[c] - Q[4 * (k - 1) + c]);
        if (k < n_s)
            for (int c = 0; c < 4; ++c) r[c] -= 2.0 * (Q[4 * (k + 1) + c] - q[c]);
        if (k >= 1) {
            double gp[4];
            smooth_penalty_grad(m, sc, cp, q, gp);
            for (int c = 0; c < 4; ++c) {
                const double hi = fmax(0.0, q[c] - m->q_max[c]);
                const double lo = fmax(0.0, m->q_min[c] - q[c]);
                r[c] += cp->w_c * gp[c] + cp->w_l * 2.0 * (hi - lo);
            }
        }
        double basis[64];
        o_bspline_basis(n_c, checkpoint_tau(K, cp->S, k), basis);
        for (int f = 0; f < K; ++f) {
            const double b = basis[4 + f];
            if (b != 0.0)
                for (int c = 0; c < 4; ++c) grad[4 * f + c] += r[c] * b;
        }
    }
    free(Q);
}

void o_smooth_grad_batch(const o_model *m, const o_scene *sc, const o_cost_params *cp,
                         const double *xi, int64_t n, const double q0[4], const double qd[4],
                         double *grad)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        o_smooth_grad(m, sc, cp, xi + i * 4 * cp->K, q0, qd, grad + i * 4 * cp->K);
}

/* ------------------------------------------------------------------ collision-free IK */

/* Residual of the collision-free IK of Sec. 3.2 (Eq. IK opt) at q for the target
 * (x, y, z, psi) and its Jacobian with respect to q (jac[5][4], may be NULL):
 *   r[0..2] = p_g - p_d, with p_g = T - (0, 0, grapple_len) the grapple centre (plumb);
 *   r[3]    = lambda_q Log(R_d^T R_g): the grapple hangs plumb, so R_g = Rz(q1) and the log
 *             map has one component, the angle q1 - psi wrapped to [-pi, pi];
 *   r[4]    = lambda_c max(0, -d(q));
 *   r_e     = 0 identically (the passive joints are at their equilibrium by the chain's
 *             reading), so it is not a row.
 * d/dq of r[4] is -lambda_c times the gradient of the pair that attains d(q) (the first
 * minimum in the order spheres, then cylinders, then boxes) when d < 0, else 0. */
void o_ik_residual(const o_model *m, const o_scene *sc, const double q[4], const double target[4],
                   double lambda_q, double lambda_c, double grapple_len, double r[5], double *jac)
{
    double centres[3 * O_MAX_SPHERES], T[3];
    o_fk(m, q, centres, NULL, T);
    r[0] = T[0] - target[0];
    r[1] = T[1] - target[1];
    r[2] = T[2] - grapple_len - target[2];
    r[3] = lambda_q * remainder(q[0] - target[3], 2.0 * M_PI);
    double d = HUGE_VAL;
    int s_min = -1, o_min = -1;   /* o_min >= n_cyl: box o_min - n_cyl */
    for (int s = 0; s < m->n_spheres; ++s) {
        const double *p = centres + 3 * s;
        for (int o = 0; o < sc->n_cyl; ++o) {
            const double v = o_sdf_cylinder(p, sc->cyl + 5 * o) - m->radius[s];
            if (v < d) { d = v; s_min = s; o_min = o; }
        }
        for (int o = 0; o < sc->n_box; ++o) {
            const double v = o_sdf_box(p, sc->box + 6 * o) - m->radius[s];
            if (v < d) { d = v; s_min = s; o_min = sc->n_cyl + o; }
        }
    }
    r[4] = lambda_c * fmax(0.0, -d);
    if (!jac) return;
    double sj[12 * O_MAX_SPHERES];
    fk_jacobian(m, q, sj);
    /* the tip T is the link-3 point at offset 0: O + L_b e_b + (L_j + q4) e_j */
    const double c1 = cos(q[0]), s1 = sin(q[0]), c2 = cos(q[1]), s2 = sin(q[1]);
    const double c23 = cos(q[1] + q[2]), s23 = sin(q[1] + q[2]);
    const double Lb = m->boom_len, L = m->jib_len + q[3];
    const double dT[3][4] = {
        {-s1 * (Lb * c2 + L * c23), -c1 * (Lb * s2 + L * s23), -c1 * L * s23, c1 * c23},
        {c1 * (Lb * c2 + L * c23), -s1 * (Lb * s2 + L * s23), -s1 * L * s23, s1 * c23},
        {0.0, Lb * c2 + L * c23, L * c23, s23}};
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 4; ++j) jac[4 * c + j] = dT[c][j];
    jac[12] = lambda_q;
    jac[13] = jac[14] = jac[15] = 0.0;
    for (int j = 0; j < 4; ++j) jac[16 + j] = 0.0;
    if (d < 0.0 && s_min >= 0) {
        double g[3];
        const double *p = centres + 3 * s_min;
        if (o_min < sc->n_cyl) sdf_cylinder_grad(p, sc->cyl + 5 * o_min, g);
        else sdf_box_grad(p, sc->box + 6 * (o_min - sc->n_cyl), g);
        const double *J = sj + 12 * s_min;
        for (int j = 0; j < 4; ++j)
            jac[16 + j] = -lambda_c * (g[0] * J[j] + g[1] * J[4 + j] + g[2] * J[8 + j]);
    }
}

/* ------------------------------------------------------------------ threads */

void o_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int32_t o_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
