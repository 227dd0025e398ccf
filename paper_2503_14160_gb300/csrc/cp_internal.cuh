// Internal declarations of the craneplan CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/craneplan.h"

namespace cp {

// ------------------------------------------------------------------ error plumbing

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
void count_launch();

#define CP_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return ::cp::cuda_fail(e_, #call);  \
    } while (0)

#define CP_LAUNCHED(what)                                          \
    do {                                                           \
        ::cp::count_launch();                                      \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return ::cp::cuda_fail(e_, what);   \
    } while (0)

// Status word written by kernels (0 = fine). Bits:
enum : uint32_t {
    DEV_ERR_TIMEOUT = 1u,      // a bounded wait gave up
    DEV_ERR_NOT_PD = 2u,       // Cholesky met a non-positive pivot
    DEV_ERR_OVERFLOW = 4u,     // an index build met more entries than its capacity
};

// ------------------------------------------------------------------ division by an invariant

// Unsigned division by a divisor d >= 1 fixed for a launch, as a multiply-high and shifts
// (Granlund and Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994, Fig. 4.1 with N = 32): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// sh1 = min(l, 1), sh2 = max(l - 1, 0); then n / d = (t + ((n - t) >> sh1)) >> sh2 with
// t = mulhi(m, n), exact for every 32-bit n.
struct FastDiv {
    uint32_t m, sh1, sh2;
};

inline FastDiv fast_div(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    FastDiv f;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.sh1 = l < 1 ? l : 1;
    f.sh2 = l > 1 ? l - 1 : 0;
    return f;
}

#ifdef __CUDACC__
static __device__ __forceinline__ uint32_t fdiv(uint32_t n, FastDiv f)
{
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.sh1)) >> f.sh2;
}
#endif

// ------------------------------------------------------------------ geometry records

// Sphere placement in the linear form used by the kernels:
//   centre = O + alpha e_b + (beta + gamma q4) e_j - delta z
struct SphereLin {
    float alpha, beta, gamma, delta, radius;
};

constexpr int kMaxSpheres = CP_MAX_SPHERES;

struct ModelDev {
    float base_z;
    float q_min[4], q_max[4];
    int n_spheres;
    float r_max;                       // largest sphere radius (filter bound)
    SphereLin sph[kMaxSpheres];
    float boom_len, jib_len;           // L_b and L_j: the tip is O + L_b e_b + (L_j + q4) e_j
    // the same placement constants of spheres 2p and 2p + 1 side by side (alpha, beta, gamma,
    // -delta), the operands of the kinematics' packed FP32x2 arithmetic
    float2 pk_alpha[kMaxSpheres / 2], pk_beta[kMaxSpheres / 2], pk_gamma[kMaxSpheres / 2],
        pk_ndelta[kMaxSpheres / 2];
    float2 pk_qmin[2], pk_nqmax[2];   // (q_min, -q_max) of joints (1, 2) and (3, 4)
};

// Cylinder records in device memory (float32):
//   filt[o]  = {cx, cy, W, 0}, W = cx^2 + cy^2 - (R + r_max)^2 (rounded from fp64)
//   exact[o] = {R, z_lo, z_hi, 0}
// Box records: centre {cx, cy, cz, 0} and half extent {hx, hy, hz, 0}.
struct SceneDev {
    const float4 *cyl_filt;
    const float4 *cyl_exact;
    int n_cyl;
    const float4 *box_c;
    const float4 *box_h;
    int n_box;
    const float4 *cyl_group;   // [n_groups(n_cyl)] {gx, gy, 0, radius}: circle that holds every
                               // member's reach (kGroup consecutive cylinders per group)
    float z_lo_all = -1e30f;   // lowest z_lo and highest z_hi over all obstacles (unbounded
    float z_hi_all = 1e30f;    // where the caller does not know them)
};

// Vertical gate of the collision tests: only penetration counts, so a sphere whose centre
// lies below an obstacle's z_lo or above its z_hi by more than r_max (plus 1 mm, far above
// the FP32 rounding of z) cannot penetrate it and needs no distance.
constexpr float kZGate = 1e-3f;

constexpr int kGroup = 8;    // cylinders per broad-phase group
__host__ __device__ inline int n_groups(int n_cyl) { return (n_cyl + kGroup - 1) / kGroup; }

// Polar index of the obstacles for large scenes. The plane around the slew axis is cut into
// n_ang angular bins over [-pi, pi) and rings of width dr about the axis (the last ring open
// outwards). Every obstacle is listed in each angular bin that its reach disk (the centre
// and the broad-phase reach of its record) overlaps, in the ring of its centre; cells are
// stored bin-major, so the rings r0..r1 of one bin are one contiguous range of entries. A
// sphere at distance |h| from the axis can only reach obstacles of the bin of its angle whose
// centre lies within w_max (the largest reach) of |h|.
struct PolarDev {
    int n_ang, n_ring;
    float inv_da;            // n_ang / (2 pi)
    float inv_dr;            // 1 / dr
    float w_max;             // largest reach of any obstacle record of the scene (m)
    const int *cell_start;   // [n_ang n_ring + 1]
    const float4 *items;     // {cx, cy, bound, id (int bits)}: bound = the square of the radius
                             // within which a sphere centre can touch it ((R + r_max)^2 + margin
                             // for a cylinder, (half diagonal + r_max + slack)^2 for a box);
                             // id < n_cyl a cylinder, else box id - n_cyl
    int capacity;            // entries allocated: the build writes and the query reads no more
};

// Margin of the fast 2-D cylinder filter, in m^2: a pair reaches the exact distance test
// when (rho^2 - (R + r_max)^2), evaluated in float32 in expanded form, is below it. The
// rounding error of that form for a pair within reach of the crane is below 3e-4 m^2.
constexpr float kFilterMargin = 2.0e-3f;

// (ii, jj), 0 <= jj <= ii, of the e-th entry of a lower triangle stored row by row.
static __device__ __forceinline__ void tri_index(int e, int &ii, int &jj)
{
    int r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    if ((r + 1) * (r + 2) / 2 <= e) ++r;
    if (r * (r + 1) / 2 > e) --r;
    ii = r;
    jj = e - r * (r + 1) / 2;
}


int validate_model(const cp_model *m);
ModelDev make_model(const cp_model *m);

// ------------------------------------------------------------------ launchers

// Work of an evaluation launch: unit = (candidate, 32 consecutive checkpoints), one per
// lane; item = (candidate, G consecutive units), taken by one warp, which adds its units'
// sums in FP64 in unit order. G depends only on the launch's size (eval_units_per_item), so
// every evaluation form sums in the same order.
struct EvalArgs {
    const float4 *xi;           // [n][K]
    int n, K, S, n_s, chunks;   // chunks = ceil(n_s / 32) units per candidate
    int G, P;                   // units per item, items per candidate (P = ceil(chunks / G))
    FastDiv div_S, div_P;       // division by S and by P
    float4 q0, qd;              // end points, used when `ends` is null
    const float4 *ends;         // optional device copy {q0, qd}, read at run time
    int ctas_per_sm;            // persistent-grid CTAs per SM (0: as many as fit)
    int withhold_staging;       // test hook: issue no staging copy, so its wait runs out
    int broadphase;             // 1: per-unit broad phase before the per-sphere filter
    unsigned long long *work;   // optional [2]: += obstacles that passed the unit box test,
                                // += (unit, obstacle) box tests run (polar index form)
    uint32_t *status;           // device status word (DEV_ERR_*) or null
    int *queue;                 // polar form: the next work item to take (zeroed before each
                                // launch); null: items in a fixed stride over the warps
    const float4 *basis;        // [S][2]: {b0..b3}(u_m), {b0..b3}(u_m) - {b0..b3}(u_{m-1})
    double *item_sum;           // [n][P][4] {J_p, sum pen, J_l, length}
    uint32_t *item_count;       // [n][P] checkpoints in collision
    uint32_t *words_out;        // optional [n][chunks]: ballot word of checkpoints in collision
    float *pen_out;             // optional [n][n_s]
};

// Units per item for n candidates of `chunks` units: about 2^15 items per launch at most, a
// whole number of units each and at most half a candidate (rounded up). Larger items share
// a candidate's control points, its index neighbourhood in L1 and the item overhead over more
// units; the warps take items from a queue, and at least two items per candidate keep the
// last ones short. The items of a launch, n ceil(chunks / G), are then at most
// eval_item_capacity(n, chunks).
inline int eval_units_per_item(int n, int chunks)
{
    const long long units = (long long)n * chunks;
    long long g = units >> 15;
    if (g > (chunks + 1) / 2) g = (chunks + 1) / 2;
    if (g < 1) g = 1;
    return (int)g;
}

// Work items of an evaluation of at most n candidates: min(n chunks, max(2^16 + n, 2 n)).
inline size_t eval_item_capacity(size_t n, size_t chunks)
{
    const size_t a = ((size_t)1 << 16) + n, b = 2 * n, c = a > b ? a : b, all = n * chunks;
    return all < c ? all : c;
}

int launch_eval(const ModelDev &m, const SceneDev &sc, const EvalArgs &a, int num_sms,
                cudaStream_t st);
int launch_eval_finalize(const double *item_sum, const uint32_t *item_count, int n, int P,
                         double w_c, double w_l, double lambda_c, double *J, uint8_t *flag,
                         double *terms, cudaStream_t st,
                         const uint32_t *status = nullptr);   // nonzero *status: NaN J, flagged
int launch_signed_distance(const ModelDev &m, const SceneDev &sc, const float *q, int n,
                           float *d, cudaStream_t st);
int launch_ik(const ModelDev &m, const SceneDev &sc, const float *targets, const float *q_init, int n,
              int restarts, int iters, float lambda_q, float lambda_c, float grapple_len, float mu0,
              uint64_t seed, uint32_t query, float *q_out, float *f_out, int *restart_out, float *r_out,
              cudaStream_t st);
int launch_forward_kinematics(const ModelDev &m, const float *q, int n, float *centres, float *tip,
                              cudaStream_t st);
// Link boxes of the convex-hull collision model (half extents across the plane w and in it
// hh for boom, jib, telescope; end pad; grapple half width and height).
struct HullDims {
    float w[3], hh[3], pad, gw, glen;
    float reach_extra;   // how far an obstacle's octagonal prism can reach beyond the
                         // sphere forms' record reach (set per scene by the planner)
};
int launch_hull_penetration(const ModelDev &m, const SceneDev &sc, const HullDims &d, const float *q, int n, float *pen,
                            cudaStream_t st);
int launch_eval_hulls(const ModelDev &m, const SceneDev &sc, const HullDims &d, const EvalArgs &a, int num_sms,
                      cudaStream_t st);
size_t eval_smem_bytes(int n_cyl, int n_box, int S);
int eval_configure(size_t smem_bytes);
int eval_ensure_smem(size_t smem_bytes);

int64_t polar_items_bound(const cp_scene *sc, double r_max, int n_ang);
float polar_reach_max(const cp_scene *sc, double r_max);
int launch_polar_build(const SceneDev &sc, const PolarDev &g, int *count, int *cursor, int *start,
                       float4 *items, uint32_t *status, cudaStream_t st);
int launch_eval_polar(const ModelDev &m, const SceneDev &sc, const PolarDev &g, const EvalArgs &a,
                      int num_sms, cudaStream_t st);

size_t smooth_smem_bytes(int n_cyl, int n_box, int S, int K);
int launch_smooth(const ModelDev &m, const SceneDev &sc, const float *xi, int n, int K, int S,
                  float4 q0, float4 qd, const float4 *basis, double margin, double beta,
                  double wc_lc, double w_l, const double *gJ, double *J, float *dxi, float *part_g,
                  double *part_J, int *queue, int num_sms, cudaStream_t st);   // queue: item counter or null
int64_t smooth_partial_units(int num_sms);
int launch_axpy(float *x, const float *y, double alpha, int64_t n, cudaStream_t st);

int launch_prepare_scene(const cp_cylinder *d_cyl_in, int n_cyl, const cp_box *d_box_in,
                         int n_box, float r_max, float4 *cyl_filt, float4 *cyl_exact, float4 *cyl_group,
                         float4 *box_c, float4 *box_h, cudaStream_t st);
int launch_basis_table(int S, float4 *basis, cudaStream_t st);
int launch_init_distribution(const double *q0, const double *qd, const double *q_min,
                             const double *q_max, int K, double init_std_frac, double *mu,
                             double *C, float4 *ends_f, cudaStream_t st);
int launch_mean_to_candidate(const double *mu, int D, float *xi, cudaStream_t st);
int launch_control_points(const double *q0, const double *qd, const double *mu, int K,
                          double *ctrl, cudaStream_t st);

int launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t *out,
                  cudaStream_t st);
int launch_factor(const double *C, double sigma2, const double *sigma_dev, int D, double *L,
                  float *Lt_f, uint32_t *status, cudaStream_t st);
int factor_configure();
int launch_sample(const double *mu, const float *Lt_f, int N, int K, uint64_t seed,
                  uint32_t iter, uint32_t query, float *xi, cudaStream_t st);
int sample_configure();

int launch_weights(int nu, double *w, cudaStream_t st);
int launch_rank(const double *J, int N, int nu, int *rank, cudaStream_t st);
int launch_scatter(int *rank, const double *J, const float *xi, int N, int nu, int D,
                   int *elite, float *elites, double *best_J, cudaStream_t st);
// yw: scratch of 2 nu D doubles (the elites' FP64 deviations and their weighted copies).
int launch_moments(const float *elites, const double *w, int nu, int D, double eps, double *yw,
                   double *s2p, double *s1p, double *mu, double *C, cudaStream_t st);

// Learning rates of the CMA-ES update (Hansen, "The CMA Evolution Strategy: A Tutorial",
// default parameters) for dimension D and the log-rank weights of nu elites.
struct CmaConsts {
    double mu_eff, c_sigma, d_sigma, c_c, c_1, c_mu, chi_n;
};
CmaConsts cma_consts(int D, int nu);
int launch_cma_reset(double sigma0, int D, double *cma, double *p_sigma, double *p_c, cudaStream_t st);
int launch_cma_update(const float *elites, const double *w, int nu, int D, const double *mu_prev,
                      const double *L, const CmaConsts &k, int t, double *yw, double *s2p, double *s1p, double *mu,
                      double *C, double *p_sigma, double *p_c, double *cma, cudaStream_t st);
int elite_slices(int N, int D, int nu, int num_sms);
size_t elite_operand_floats(int nu, int D);   // packed Y_hi / Y_lo of the tensor-core sampler
int launch_elite_weights(const double *w, int nu, double sigma, float *sw, cudaStream_t st);
int elite_update_blocks(int nu, int num_sms);
int launch_elite_update(const float *elites, const double *w, const float *sw, int nu, int D, int blocks,
                        double *part, unsigned int *bar, double *mu, float *mu_f, float *mu_lo, float *Yp,
                        uint32_t *status, cudaStream_t st);
int launch_sample_elites(const float *Yp, const float *mu_f, int N, int K, int nu, int slices, double sigma,
                         double eps, uint64_t seed, uint32_t iter, uint32_t query, float *P, float *xi,
                         uint32_t *status, bool withhold, cudaStream_t st);
int update_chunks(int nu, int D);
int radix_tiles(int N);
size_t radix_hist_ints(int N);   // ints of the histogram scratch of launch_radix_rank
int launch_radix_rank(const double *J, int N, unsigned long long *key_a, unsigned long long *key_b,
                      int *val_a, int *val_b, int *hist, cudaStream_t st);
int launch_gather_elites(const int *sorted, const double *J, const float *xi, int nu, int D,
                         int *elite, float *elites, double *best_J, cudaStream_t st);
constexpr int kRadixMinN = 8193;   // the radix sort ranks populations above 8192
int update_configure();

// Per-iteration metrics row {iteration, best J, mean J, tr C, collision-free fraction}; C
// null: tr C from the elites about mu (factor-free sampler).
constexpr int kMetricsCols = 5;
constexpr int kMetricsRing = 256;   // rows kept (the last kMetricsRing iterations)
constexpr int kMetricsBlocks = 128; // blocks of the partial sums (part holds 3 kMetricsBlocks)
int launch_iter_metrics(const double *J, const uint8_t *flag, int N, const double *best, const double *C,
                        const float *elites, const double *w, const double *mu, int nu, int D, double eps,
                        int iteration, double *part, double *row, cudaStream_t st);

// ------------------------------------------------------------------ batched form
// One launch of each stage serves every query of a batch. Each query keeps its own planner
// workspace; the batched kernels reach it through this per-query view, and a block finds its
// query in a table of {query, block within the query} built once per batch, so that every
// query's arithmetic is that of its planner run alone.
struct BatchEvalDev {          // what the evaluation of one query reads (restaged per query)
    EvalArgs a;
    SceneDev sc;
    PolarDev g;
};

struct BatchQueryDev {
    int N, K, D, nu;
    double *J;                       // [N] costs of the population
    uint8_t *flag;                   // [N]
    const double *item_sum;          // [N][P][4] of the population's evaluation
    const uint32_t *item_count;
    int P;                           // items per candidate of the population's evaluation
    double w_c, w_l, lambda_c;
    float *xi;                       // [N][D] population
    double *mu, *C, *L;
    float *Lt;
    uint32_t seed_lo, seed_hi, query;
    double sigma2;                   // sigma^2 of the factor
    int *elite;                      // [nu] elite indices in rank order
    float *elites;                   // [nu][D]
    const double *w;                 // [nu] elite weights
    double *best;                    // cost of the best candidate
    double *s2p, *s1p;               // moment partials
    double *mom_y;                   // [2][nu][D] the elites' FP64 deviations, then weighted
    double eps;
    int per, n_chunks;               // elites per moment chunk, chunks
    int cand_off;                    // first position of the query in the concatenated ranking
    uint32_t *status;
    double *consts;                  // q0[4], qd[4], q_min[4], q_max[4]
    double init_std_frac;
    float4 *ends;                    // {q0, qd} in float
    float *mean_xi;
    double *mean_J, *mean_terms;
    uint8_t *mean_flag;
    double *ctrl;                    // [K + 8][4]
};

// Block-to-query tables: entry b = {query, block index within the query}.
int launch_batch_init(const BatchQueryDev *qd, const int2 *tab, int blocks, const double *inputs, cudaStream_t st);
int launch_batch_factor(const BatchQueryDev *qd, int nq, int max_D, cudaStream_t st);
int launch_batch_sample(const BatchQueryDev *qd, const int2 *tab, int blocks, int max_K, uint32_t iter,
                        cudaStream_t st);
constexpr int kBatchSampleCands = 256;   // candidates per block of the batched sampler
int batch_eval_configure();
int launch_batch_eval_polar(const ModelDev &m, const BatchEvalDev *qd, const int4 *tiles, int n_tiles, int *queue,
                            int max_S, int threads, int blocks, cudaStream_t st);
int batch_eval_max_blocks(const ModelDev &m, int threads, int max_S, int num_sms);
// tab non-null: the populations (blocks of 256 candidates); null: the mean candidates of
// `blocks` queries, whose evaluation is described by mean_ev.
int launch_batch_finalize(const BatchQueryDev *qd, const int2 *tab, int blocks, const BatchEvalDev *mean_ev,
                          cudaStream_t st);
int launch_batch_radix_rank(const BatchQueryDev *qd, const int2 *tab, int blocks, int total, int nq,
                            const uint16_t *qid, unsigned long long *key_a, unsigned long long *key_b,
                            int *val_a, int *val_b, int *hist, int **sorted, cudaStream_t st);
int launch_batch_gather(const BatchQueryDev *qd, const int2 *tab, int blocks, const int *sorted, cudaStream_t st);
int launch_batch_moments(const BatchQueryDev *qd, int nq, const int2 *tab_prep, int blocks_prep,
                         const int2 *tab_partial, int blocks_partial, const int2 *tab_combine, int blocks_combine,
                         cudaStream_t st);
int moments_chunking(int nu, int D, int *per);   // chunks of the moment partials and elites per chunk
int launch_batch_outputs(const BatchQueryDev *qd, int nq, bool mean_candidate, double *out, int out_stride,
                         cudaStream_t st);

}  // namespace cp
