// C ABI of the craneplan library (declared in include/craneplan.h): validation, the
// planner's device workspace, and the order of the kernel launches of Algorithm 1
// (arXiv 2503.14160, Sec. 4.1). All arithmetic of the method runs in the kernels; host
// code here only checks arguments, copies inputs and results, and sequences launches.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cp_internal.cuh"

namespace cp {

namespace {
thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};
std::atomic<int32_t> g_fail_allocs{0};   // test hook: workspace allocations still to fail
}  // namespace

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? CP_ERR_OOM : CP_ERR_CUDA;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace cp

using namespace cp;

namespace {

enum Stage { ST_EVAL = 0, ST_SAMPLE = 1, ST_FACTOR = 2, ST_UPDATE = 3, ST_COUNT = 4 };

struct Timer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[ST_COUNT];
    cudaEvent_t open = nullptr;
    int64_t units = 0, tests = 0;   // evaluation work while on (tests: exhaustive form)
    bool grid = false;

    int begin(cudaStream_t st)
    {
        if (!on) return CP_OK;
        cudaEvent_t e;
        int rc = take(&e);
        if (rc != CP_OK) return rc;
        CP_CUDA(cudaEventRecord(e, st));
        open = e;
        return CP_OK;
    }
    int end(Stage s, cudaStream_t st)
    {
        if (!on) return CP_OK;
        cudaEvent_t e;
        int rc = take(&e);
        if (rc != CP_OK) return rc;
        CP_CUDA(cudaEventRecord(e, st));
        spans[s].emplace_back(open, e);
        return CP_OK;
    }
    int take(cudaEvent_t *e)
    {
        if (used == pool.size()) {
            cudaEvent_t ev;
            CP_CUDA(cudaEventCreate(&ev));
            pool.push_back(ev);
        }
        *e = pool[used++];
        return CP_OK;
    }
    void clear()
    {
        used = 0;
        for (auto &s : spans) s.clear();
        units = tests = 0;
        grid = false;
    }
    void destroy()
    {
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
        clear();
    }
};

// Bump allocator over one device allocation (256-byte aligned pieces).
struct Layout {
    size_t bytes = 0;
    template <typename T>
    size_t take(size_t count)
    {
        const size_t off = bytes;
        bytes += (count * sizeof(T) + 255) & ~(size_t)255;
        return off;
    }
};

bool is_finite(double v) { return std::isfinite(v); }

// Candidate arrays are read and written one control point (four floats) at a time.
bool aligned16(const void *ptr) { return ((uintptr_t)ptr & 15u) == 0; }

constexpr int kPolarBins = 256;   // angular bins of the polar obstacle index

// An NVTX range over a scope (host side: it brackets the enqueue of a stage's launches; a
// profiler attributes the kernels launched inside it to the range). No-ops without a tool.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace

struct cp_planner {
    cudaStream_t st = nullptr;
    int device = 0, num_sms = 1;
    cp_params prm{};
    int N = 0, K = 0, S = 0, D = 0, n_s = 0, chunks = 0, nu = 0, n_mean_chunks = 0;
    int cap_cyl = 0, cap_box = 0;
    ModelDev mdev{};
    SceneDev sdev{};
    char *base = nullptr;
    // workspace pieces
    cp_cylinder *cyl_in = nullptr;
    cp_box *box_in = nullptr;
    float4 *cyl_filt = nullptr, *cyl_exact = nullptr, *box_c = nullptr, *box_h = nullptr;
    float4 *cyl_group = nullptr;
    std::vector<cp_cylinder> cyl_sorted;   // host copy of the scene in staging order
    float4 *basis = nullptr;
    double *consts = nullptr;   // q0[4], qd[4], q_min[4], q_max[4]
    double *mu = nullptr, *C = nullptr, *L = nullptr;
    float *Lt = nullptr;
    float *xi = nullptr;
    double *J = nullptr, *terms = nullptr;
    uint8_t *flag = nullptr;
    double *item_sum = nullptr;     // [N][P][4] FP64 sums of the evaluation's work items
    uint32_t *item_count = nullptr; // [N][P]
    int *rank = nullptr, *elite = nullptr;
    float *elites = nullptr;
    double *w = nullptr, *mean_part = nullptr, *cov_part = nullptr;
    double *mom_y = nullptr;    // [2][nu][D] FP64 deviations of the elites for the moments
    double *best = nullptr;
    uint32_t *status = nullptr;
    double *ctrl = nullptr;
    float *mean_xi = nullptr;
    double *mean_J = nullptr, *mean_terms = nullptr;
    uint8_t *mean_flag = nullptr;
    float *grad = nullptr;      // [N][D] gradient buffer for polish
    float4 *ends_f = nullptr;   // [2] {q0, qd} in float, written with the end points
    unsigned long long *work = nullptr;   // [2] broad-phase survivors and box tests while timing
    int *eval_queue = nullptr;            // the polar evaluation's item counter
    size_t item_cap = 0;                  // work items the item_sum / item_count buffers hold
    unsigned long long *rkey_a = nullptr, *rkey_b = nullptr;   // radix sort scratch
    int *rval_a = nullptr, *rval_b = nullptr, *rhist = nullptr;
    double *cma = nullptr;      // CMA-ES rule: {sigma, sigma before the update, h_sigma, |p_sigma|}
    double *p_sigma = nullptr, *p_c = nullptr, *mu_prev = nullptr;
    CmaConsts cmak{};
    // factor-free sampler: scaled elite deviations Y (TF32 pair, packed in the tensor-core
    // operand layout), the mean in FP32, the slice partials [slices][N][D]; elites_ready
    // when the last step was such an update
    float *elite_Y = nullptr, *mu_f = nullptr, *mu_lo = nullptr, *sample_part = nullptr;
    float *elite_sw = nullptr;        // sigma sqrt(w_j)
    double *elite_mean_part = nullptr;   // per-block partial sums of the mean
    unsigned int *elite_bar = nullptr;   // grid barrier of the elite update (count, generation)
    int elite_slices = 1;
    bool elites_ready = false;
    HullDims hulls{{0.2f, 0.2f, 0.15f}, {0.2f, 0.2f, 0.15f}, 0.2f, 0.25f, 1.0f, 0.f};   // CP_COLLISION_HULLS
    float hull_reach_extra = 0.f;   // per scene: prism reach beyond the records' sphere reach
    float *smooth_part_g = nullptr;   // partial gradients when few candidates share the GPU
    double *smooth_part_J = nullptr;
    int smem_optin = 0;
    bool use_grid = false;
    PolarDev gdev{};                  // polar obstacle index (grid_cell > 0)
    int64_t grid_cap = 0;
    int *grid_count = nullptr, *grid_cursor = nullptr, *grid_start = nullptr;
    float4 *grid_items = nullptr;
    bool have_endpoints = false;
    float4 q0f{}, qdf{};
    int iteration = 0;
    Timer timer;
    // cp_plan's iterations recorded as one CUDA graph (launch gaps between the small
    // dependent kernels vanish); valid for one start iteration, count, scene and end points
    cudaGraphExec_t plan_exec = nullptr;
    int plan_start = -1, plan_iters = -1;
    float4 plan_q0{}, plan_qd{};
    SceneDev plan_sdev{};
    PolarDev plan_gdev{};
    bool plan_ready_before = false, plan_ready_after = false;
    bool plan_metrics = false;
    int64_t plan_nodes = 0;   // kernels in the recorded graph
    // per-iteration metrics of cp_plan: ring of kMetricsRing rows (slot = iteration mod ring)
    bool metrics_on = false;
    double *metrics = nullptr;
    double *metrics_part = nullptr;   // [kMetricsBlocks][3] partial sums of a row
    int64_t metrics_count = 0;   // rows written since the end points were set
};

namespace cp {

int validate_model(const cp_model *m)
{
    if (!m) return set_error("model is NULL"), CP_ERR_ARG;
    if (m->n_spheres < 1 || m->n_spheres > CP_MAX_SPHERES)
        return set_error("n_spheres %d outside 1..%d", m->n_spheres, CP_MAX_SPHERES), CP_ERR_ARG;
    if (!is_finite(m->base_z) || !is_finite(m->boom_len) || !is_finite(m->jib_len))
        return set_error("model lengths must be finite"), CP_ERR_ARG;
    for (int j = 0; j < 4; ++j)
        if (!is_finite(m->q_min[j]) || !is_finite(m->q_max[j]) || !(m->q_min[j] < m->q_max[j]))
            return set_error("joint %d limits must be finite with q_min < q_max", j), CP_ERR_ARG;
    for (int s = 0; s < m->n_spheres; ++s) {
        const cp_sphere &sp = m->spheres[s];
        if (sp.link < 0 || sp.link > 3) return set_error("sphere %d: link %d outside 0..3", s, sp.link), CP_ERR_ARG;
        if (!is_finite(sp.offset) || !(sp.radius > 0.0) || !is_finite(sp.radius))
            return set_error("sphere %d: offset must be finite and radius > 0", s), CP_ERR_ARG;
    }
    return CP_OK;
}

CmaConsts cma_consts(int D, int nu)
{
    // the log-rank weights of step (4), as k_weights forms them
    std::vector<double> w(nu);
    double sum = 0.0;
    for (int j = 0; j < nu; ++j) sum += (w[j] = std::log(nu + 0.5) - std::log(j + 1.0));
    double s2 = 0.0;
    for (int j = 0; j < nu; ++j) s2 += (w[j] / sum) * (w[j] / sum);
    CmaConsts k{};
    const double n = D;
    k.mu_eff = 1.0 / s2;
    k.c_sigma = (k.mu_eff + 2.0) / (n + k.mu_eff + 5.0);
    k.d_sigma = 1.0 + 2.0 * std::max(0.0, std::sqrt((k.mu_eff - 1.0) / (n + 1.0)) - 1.0) + k.c_sigma;
    k.c_c = (4.0 + k.mu_eff / n) / (n + 4.0 + 2.0 * k.mu_eff / n);
    k.c_1 = 2.0 / ((n + 1.3) * (n + 1.3) + k.mu_eff);
    k.c_mu = std::min(1.0 - k.c_1, 2.0 * (k.mu_eff - 2.0 + 1.0 / k.mu_eff) / ((n + 2.0) * (n + 2.0) + k.mu_eff));
    k.chi_n = std::sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n));
    return k;
}

ModelDev make_model(const cp_model *m)
{
    ModelDev d{};
    d.base_z = (float)m->base_z;
    for (int j = 0; j < 4; ++j) {
        d.q_min[j] = (float)m->q_min[j];
        d.q_max[j] = (float)m->q_max[j];
    }
    d.n_spheres = m->n_spheres;
    float r_max = 0.f;
    for (int s = 0; s < kMaxSpheres; ++s) {
        SphereLin l{0.f, 0.f, 0.f, 0.f, -1e30f};   // padding: never the nearest pair
        if (s < m->n_spheres) {
            const cp_sphere &sp = m->spheres[s];
            const float t = (float)sp.offset, Lb = (float)m->boom_len, Lj = (float)m->jib_len;
            switch (sp.link) {
            case 0: l = {t, 0.f, 0.f, 0.f, 0.f}; break;
            case 1: l = {Lb, t, 0.f, 0.f, 0.f}; break;
            case 2: l = {Lb, Lj, t, 0.f, 0.f}; break;
            default: l = {Lb, Lj, 1.f, t, 0.f}; break;
            }
            l.radius = (float)sp.radius;
            if (l.radius > r_max) r_max = l.radius;
        }
        d.sph[s] = l;
    }
    d.r_max = r_max;
    d.boom_len = (float)m->boom_len;
    d.jib_len = (float)m->jib_len;
    for (int q = 0; q < kMaxSpheres / 2; ++q) {
        const SphereLin &a = d.sph[2 * q], &b = d.sph[2 * q + 1];
        d.pk_alpha[q] = make_float2(a.alpha, b.alpha);
        d.pk_beta[q] = make_float2(a.beta, b.beta);
        d.pk_gamma[q] = make_float2(a.gamma, b.gamma);
        d.pk_ndelta[q] = make_float2(-a.delta, -b.delta);
    }
    for (int q = 0; q < 2; ++q) {
        d.pk_qmin[q] = make_float2(d.q_min[2 * q], d.q_min[2 * q + 1]);
        d.pk_nqmax[q] = make_float2(-d.q_max[2 * q], -d.q_max[2 * q + 1]);
    }
    return d;
}

}  // namespace cp

namespace {

int validate_scene(const cp_scene *sc)
{
    if (!sc) return set_error("scene is NULL"), CP_ERR_ARG;
    if (sc->n_cyl < 0 || sc->n_box < 0) return set_error("negative obstacle count"), CP_ERR_ARG;
    if (sc->n_cyl > 0 && !sc->cyl) return set_error("scene.cyl is NULL"), CP_ERR_ARG;
    if (sc->n_box > 0 && !sc->box) return set_error("scene.box is NULL"), CP_ERR_ARG;
    for (int i = 0; i < sc->n_cyl; ++i) {
        const cp_cylinder &c = sc->cyl[i];
        if (!is_finite(c.cx) || !is_finite(c.cy) || !is_finite(c.z_lo) || !is_finite(c.z_hi) ||
            !(c.radius > 0.0) || !is_finite(c.radius) || !(c.z_lo <= c.z_hi))
            return set_error("cylinder %d is invalid (radius > 0, z_lo <= z_hi, finite)", i), CP_ERR_ARG;
    }
    for (int i = 0; i < sc->n_box; ++i) {
        const cp_box &b = sc->box[i];
        for (int c = 0; c < 3; ++c)
            if (!is_finite(b.lo[c]) || !is_finite(b.hi[c]) || !(b.lo[c] <= b.hi[c]))
                return set_error("box %d is invalid (finite, lo <= hi)", i), CP_ERR_ARG;
    }
    return CP_OK;
}

int validate_params(const cp_params *p)
{
    if (!p) return set_error("params is NULL"), CP_ERR_ARG;
    if (p->n_candidates < 2 || p->n_candidates > (1 << 22))
        return set_error("n_candidates %d outside 2..%d", p->n_candidates, 1 << 22), CP_ERR_ARG;
    if (p->n_waypoints < 1 || p->n_waypoints > CP_MAX_WAYPOINTS)
        return set_error("n_waypoints %d outside 1..%d", p->n_waypoints, CP_MAX_WAYPOINTS), CP_ERR_ARG;
    if (p->substeps < 1 || p->substeps > 4096)
        return set_error("substeps %d outside 1..4096", p->substeps), CP_ERR_ARG;
    if (p->debug_withhold_staging < 0 || p->debug_withhold_staging > 2)
        return set_error("debug_withhold_staging %d outside 0..2", p->debug_withhold_staging), CP_ERR_ARG;
    if (p->n_elites < 0 || p->n_elites > p->n_candidates)
        return set_error("n_elites %d outside 0..n_candidates", p->n_elites), CP_ERR_ARG;
    if (!(p->sigma > 0.0) || !is_finite(p->sigma)) return set_error("sigma must be > 0"), CP_ERR_ARG;
    if (!(p->eps >= 0.0) || !is_finite(p->eps)) return set_error("eps must be >= 0"), CP_ERR_ARG;
    if (!(p->init_std_frac > 0.0) || !is_finite(p->init_std_frac))
        return set_error("init_std_frac must be > 0"), CP_ERR_ARG;
    if (!(p->w_c >= 0.0) || !(p->w_l >= 0.0) || !(p->lambda_c >= 0.0) || !is_finite(p->w_c) ||
        !is_finite(p->w_l) || !is_finite(p->lambda_c))
        return set_error("cost weights must be finite and >= 0"), CP_ERR_ARG;
    if (p->max_cylinders < 0 || p->max_boxes < 0) return set_error("negative capacity"), CP_ERR_ARG;
    if (p->eval_ctas_per_sm < 0) return set_error("eval_ctas_per_sm must be >= 0"), CP_ERR_ARG;
    if (p->eval_exhaustive != 0 && p->eval_exhaustive != 1)
        return set_error("eval_exhaustive must be 0 or 1"), CP_ERR_ARG;
    if (p->update_rule != CP_UPDATE_PAPER && p->update_rule != CP_UPDATE_CMAES)
        return set_error("update_rule must be CP_UPDATE_PAPER or CP_UPDATE_CMAES"), CP_ERR_ARG;
    if (p->collision_model != CP_COLLISION_SPHERES && p->collision_model != CP_COLLISION_HULLS)
        return set_error("collision_model must be CP_COLLISION_SPHERES or CP_COLLISION_HULLS"), CP_ERR_ARG;
    if (p->sampler != CP_SAMPLE_FACTOR && p->sampler != CP_SAMPLE_ELITES)
        return set_error("sampler must be CP_SAMPLE_FACTOR or CP_SAMPLE_ELITES"), CP_ERR_ARG;
    if (p->sampler == CP_SAMPLE_ELITES && p->update_rule != CP_UPDATE_PAPER)
        return set_error("CP_SAMPLE_ELITES draws the covariance of the paper's update; it needs CP_UPDATE_PAPER"),
               CP_ERR_ARG;
    if (!(p->grid_cell >= 0.0) || !is_finite(p->grid_cell) || !(p->grid_half_extent >= 0.0) ||
        !is_finite(p->grid_half_extent) || p->max_grid_items < 0 || !(p->smooth_margin >= 0.0) ||
        !is_finite(p->smooth_margin) || !(p->smooth_beta >= 0.0) || !is_finite(p->smooth_beta))
        return set_error("grid and smooth-penalty parameters must be finite and >= 0"), CP_ERR_ARG;
    const int64_t n_s = (int64_t)(p->n_waypoints + 3) * p->substeps;
    if ((int64_t)p->n_candidates * ((n_s + 31) / 32) > 0x7FFFFFFF)
        return set_error("n_candidates * ceil(n_s / 32) exceeds 2^31 - 1"), CP_ERR_ARG;
    return CP_OK;
}

// Cylinders sorted by the Z-order (Morton) code of their centres on a 65536 x 65536 lattice
// over the scene's bounding box; ties keep the caller's order.
void morton_order(const cp_cylinder *cyl, int n, std::vector<cp_cylinder> &out)
{
    double x0 = cyl[0].cx, x1 = x0, y0 = cyl[0].cy, y1 = y0;
    for (int i = 1; i < n; ++i) {
        x0 = std::min(x0, cyl[i].cx);
        x1 = std::max(x1, cyl[i].cx);
        y0 = std::min(y0, cyl[i].cy);
        y1 = std::max(y1, cyl[i].cy);
    }
    const double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
    auto spread = [](uint32_t v) {   // bits of v to the even positions
        uint64_t x = v & 0xFFFFu;
        x = (x | (x << 8)) & 0x00FF00FFu;
        x = (x | (x << 4)) & 0x0F0F0F0Fu;
        x = (x | (x << 2)) & 0x33333333u;
        x = (x | (x << 1)) & 0x55555555u;
        return (uint32_t)x;
    };
    std::vector<std::pair<uint32_t, int>> key((size_t)n);
    for (int i = 0; i < n; ++i) {
        const uint32_t qx = (uint32_t)((cyl[i].cx - x0) * sx), qy = (uint32_t)((cyl[i].cy - y0) * sy);
        key[i] = {spread(qx) | (spread(qy) << 1), i};
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<uint32_t, int> &a, const std::pair<uint32_t, int> &b) {
                         return a.first < b.first;
                     });
    out.resize((size_t)n);
    for (int i = 0; i < n; ++i) out[i] = cyl[key[i].second];
}

int stage_scene(cp_planner *p, const cp_scene *sc)
{
    if (sc->n_cyl > p->cap_cyl || sc->n_box > p->cap_box)
        return set_error("scene (%d cylinders, %d boxes) exceeds the capacity (%d, %d) set at init",
                         sc->n_cyl, sc->n_box, p->cap_cyl, p->cap_box), CP_ERR_ARG;
    if (sc->n_cyl > 0) {
        // staged in Z order of the centres, so that the groups of kGroup consecutive cylinders
        // are compact (every kernel takes a minimum or a sum over all of them; the order only
        // changes which obstacles share a group)
        morton_order(sc->cyl, sc->n_cyl, p->cyl_sorted);
        CP_CUDA(cudaMemcpyAsync(p->cyl_in, p->cyl_sorted.data(), sizeof(cp_cylinder) * sc->n_cyl,
                                cudaMemcpyHostToDevice, p->st));
        CP_CUDA(cudaStreamSynchronize(p->st));   // the host copy may change on the next call
    }
    if (sc->n_box > 0)
        CP_CUDA(cudaMemcpyAsync(p->box_in, sc->box, sizeof(cp_box) * sc->n_box,
                                cudaMemcpyHostToDevice, p->st));
    int rc = launch_prepare_scene(p->cyl_in, sc->n_cyl, p->box_in, sc->n_box, p->mdev.r_max,
                                  p->cyl_filt, p->cyl_exact, p->cyl_group, p->box_c, p->box_h,
                                  p->st);
    if (rc != CP_OK) return rc;
    p->sdev.n_cyl = sc->n_cyl;
    p->sdev.n_box = sc->n_box;
    double zlo = 1e30, zhi = -1e30;
    for (int i = 0; i < sc->n_cyl; ++i) {
        zlo = std::min(zlo, sc->cyl[i].z_lo);
        zhi = std::max(zhi, sc->cyl[i].z_hi);
    }
    for (int i = 0; i < sc->n_box; ++i) {
        zlo = std::min(zlo, sc->box[i].lo[2]);
        zhi = std::max(zhi, sc->box[i].hi[2]);
    }
    p->sdev.z_lo_all = (float)zlo;
    p->sdev.z_hi_all = (float)zhi;
    // the octagonal prism of a cylinder reaches R / cos(pi/8); the records' reach is at least
    // R + r_max, so the hull form dilates the broad phase by the difference where positive
    double rmax_cyl = 0.0;
    for (int i = 0; i < sc->n_cyl; ++i) rmax_cyl = std::max(rmax_cyl, sc->cyl[i].radius);
    p->hull_reach_extra = (float)(std::max(0.0, rmax_cyl / std::cos(M_PI / 8.0) - rmax_cyl - (double)p->mdev.r_max) + 1e-3);
    if (p->use_grid) {
        const int64_t need = polar_items_bound(sc, p->mdev.r_max, p->gdev.n_ang);
        if (need > p->grid_cap)
            return set_error("scene may need %lld index entries; capacity %lld (max_grid_items)",
                             (long long)need, (long long)p->grid_cap), CP_ERR_ARG;
        p->gdev.w_max = polar_reach_max(sc, p->mdev.r_max);
        rc = launch_polar_build(p->sdev, p->gdev, p->grid_count, p->grid_cursor, p->grid_start, p->grid_items,
                                p->status, p->st);
        if (rc != CP_OK) return rc;
    }
    return CP_OK;
}

int run_eval(cp_planner *p, const float *d_xi, int n, double *d_J, uint8_t *d_flag,
             double *d_terms, uint32_t *d_words, float *d_pen)
{
    NvtxRange range("craneplan:evaluate");
    EvalArgs a{};
    a.xi = (const float4 *)d_xi;
    a.n = n;
    a.K = p->K;
    a.S = p->S;
    a.n_s = p->n_s;
    a.chunks = p->chunks;
    a.G = eval_units_per_item(n, p->chunks);
    a.P = (p->chunks + a.G - 1) / a.G;
    if ((size_t)n * a.P > p->item_cap)   // the buffers are sized by the same rule: never expected
        return set_error("%d candidates need %lld work items; the planner holds %lld", n,
                         (long long)n * a.P, (long long)p->item_cap), CP_ERR_STATE;
    a.div_S = fast_div((uint32_t)p->S);
    a.div_P = fast_div((uint32_t)a.P);
    a.q0 = p->q0f;
    a.qd = p->qdf;
    a.ends = p->ends_f;
    a.ctas_per_sm = p->prm.eval_ctas_per_sm;
    a.withhold_staging = p->prm.debug_withhold_staging == 1;
    a.broadphase = p->prm.eval_exhaustive ? 0 : 1;
    a.work = p->timer.on ? p->work : nullptr;
    if (p->timer.on) {
        p->timer.units += (int64_t)n * p->chunks;
        if (p->use_grid) p->timer.grid = true;
        else if (!a.broadphase) p->timer.tests += (int64_t)n * p->chunks * (p->sdev.n_cyl + p->sdev.n_box);
    }
    a.status = p->status;
    a.queue = p->eval_queue;
    a.basis = p->basis;
    a.item_sum = p->item_sum;
    a.item_count = p->item_count;
    a.words_out = d_words;
    a.pen_out = d_pen;
    int rc = p->timer.begin(p->st);
    if (rc != CP_OK) return rc;
    if (p->prm.collision_model == CP_COLLISION_HULLS) {
        HullDims d = p->hulls;
        d.reach_extra = p->hull_reach_extra;
        rc = launch_eval_hulls(p->mdev, p->sdev, d, a, p->num_sms, p->st);
    }
    else
        rc = p->use_grid ? launch_eval_polar(p->mdev, p->sdev, p->gdev, a, p->num_sms, p->st)
                         : launch_eval(p->mdev, p->sdev, a, p->num_sms, p->st);
    if (rc != CP_OK) return rc;
    rc = p->timer.end(ST_EVAL, p->st);
    if (rc != CP_OK) return rc;
    return launch_eval_finalize(p->item_sum, p->item_count, n, a.P, p->prm.w_c, p->prm.w_l, p->prm.lambda_c,
                                d_J, d_flag, d_terms, p->st);
}

int run_factor(cp_planner *p)
{
    NvtxRange range("craneplan:factor");
    int rc = p->timer.begin(p->st);
    if (rc != CP_OK) return rc;
    rc = launch_factor(p->C, p->prm.sigma * p->prm.sigma, p->prm.update_rule == CP_UPDATE_CMAES ? p->cma : nullptr,
                       p->D, p->L, p->Lt, p->status, p->st);
    if (rc != CP_OK) return rc;
    return p->timer.end(ST_FACTOR, p->st);
}

int run_sample(cp_planner *p, int iter, float *d_xi)
{
    NvtxRange range("craneplan:sample");
    int rc = p->timer.begin(p->st);
    if (rc != CP_OK) return rc;
    if (p->elites_ready)
        rc = launch_sample_elites(p->elite_Y, p->mu_f, p->N, p->K, p->nu, p->elite_slices, p->prm.sigma,
                                  p->prm.eps, p->prm.seed, (uint32_t)iter, p->prm.query, p->sample_part, d_xi,
                                  p->status, p->prm.debug_withhold_staging == 2, p->st);
    else
        rc = launch_sample(p->mu, p->Lt, p->N, p->K, p->prm.seed, (uint32_t)iter, p->prm.query, d_xi,
                           p->st);
    if (rc != CP_OK) return rc;
    return p->timer.end(ST_SAMPLE, p->st);
}

int run_update(cp_planner *p, const double *d_J, const float *d_xi)
{
    NvtxRange range("craneplan:update");
    int rc = p->timer.begin(p->st);
    if (rc != CP_OK) return rc;
    if (p->N >= kRadixMinN) {
        if ((rc = launch_radix_rank(d_J, p->N, p->rkey_a, p->rkey_b, p->rval_a, p->rval_b, p->rhist,
                                    p->st)) != CP_OK)
            return rc;
        if ((rc = launch_gather_elites(p->rval_a, d_J, d_xi, p->nu, p->D, p->elite, p->elites, p->best,
                                       p->st)) != CP_OK)
            return rc;
    } else {
        if ((rc = launch_rank(d_J, p->N, p->nu, p->rank, p->st)) != CP_OK) return rc;
        if ((rc = launch_scatter(p->rank, d_J, d_xi, p->N, p->nu, p->D, p->elite, p->elites, p->best,
                                 p->st)) != CP_OK)
            return rc;
    }
    if (p->prm.update_rule == CP_UPDATE_CMAES) {
        CP_CUDA(cudaMemcpyAsync(p->mu_prev, p->mu, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
        if ((rc = launch_cma_update(p->elites, p->w, p->nu, p->D, p->mu_prev, p->L, p->cmak, p->iteration,
                                    p->mom_y, p->cov_part, p->mean_part, p->mu, p->C, p->p_sigma, p->p_c, p->cma,
                                    p->st)) != CP_OK)
            return rc;
    } else if (p->prm.sampler == CP_SAMPLE_ELITES) {
        // the next draw comes from these elites: the mean and the scaled deviations, no C
        if ((rc = launch_elite_update(p->elites, p->w, p->elite_sw, p->nu, p->D,
                                      elite_update_blocks(p->nu, p->num_sms), p->elite_mean_part,
                                      p->elite_bar, p->mu, p->mu_f, p->mu_lo, p->elite_Y, p->status,
                                      p->st)) != CP_OK)
            return rc;
        if ((rc = p->timer.end(ST_UPDATE, p->st)) != CP_OK) return rc;
        p->elites_ready = true;
        p->iteration += 1;
        return CP_OK;
    } else if ((rc = launch_moments(p->elites, p->w, p->nu, p->D, p->prm.eps, p->mom_y, p->cov_part, p->mean_part,
                                    p->mu, p->C, p->st)) != CP_OK) {
        return rc;
    }
    if ((rc = p->timer.end(ST_UPDATE, p->st)) != CP_OK) return rc;
    if ((rc = run_factor(p)) != CP_OK) return rc;
    p->iteration += 1;
    return CP_OK;
}

// With the factor-free sampler after an update, C (and its factor) exist only on request:
// the moments of the current elites, with the mean written to scratch so that the mean the
// sampler uses keeps its bits.
int materialise_distribution(const cp_planner *p)
{
    if (!p->elites_ready) return CP_OK;
    cp_planner *q = const_cast<cp_planner *>(p);
    int rc = launch_moments(q->elites, q->w, q->nu, q->D, q->prm.eps, q->mom_y, q->cov_part, q->mean_part, q->mu_prev, q->C,
                            q->st);
    if (rc != CP_OK) return rc;
    return launch_factor(q->C, q->prm.sigma * q->prm.sigma, nullptr, q->D, q->L, q->Lt, q->status, q->st);
}

// The metrics row of the iteration just completed by cp_plan (after run_update).
int record_metrics(cp_planner *p)
{
    if (!p->metrics_on) return CP_OK;
    const int it = p->iteration - 1;
    double *row = p->metrics + (size_t)(it % kMetricsRing) * kMetricsCols;
    const bool no_C = p->elites_ready;   // the factor-free sampler's update forms no C
    return launch_iter_metrics(p->J, p->flag, p->N, p->best, no_C ? nullptr : p->C, p->elites, p->w, p->mu, p->nu,
                               p->D, p->prm.eps, it, p->metrics_part, row, p->st);
}

// One iteration of cp_plan: steps (1)-(6) and the metrics row when on.
int run_iteration(cp_planner *p)
{
    int rc;
    if ((rc = run_sample(p, p->iteration, p->xi)) != CP_OK) return rc;
    if ((rc = run_eval(p, p->xi, p->N, p->J, p->flag, nullptr, nullptr, nullptr)) != CP_OK) return rc;
    if ((rc = run_update(p, p->J, p->xi)) != CP_OK) return rc;
    return record_metrics(p);
}

int check_status(cp_planner *p)
{
    uint32_t s = 0;
    CP_CUDA(cudaMemcpyAsync(&s, p->status, sizeof s, cudaMemcpyDeviceToHost, p->st));
    CP_CUDA(cudaStreamSynchronize(p->st));
    if (s & DEV_ERR_NOT_PD) {
        CP_CUDA(cudaMemsetAsync(p->status, 0, sizeof(uint32_t), p->st));
        return set_error("the covariance is not positive definite (Cholesky pivot <= 0)"), CP_ERR_NUMERIC;
    }
    if (s & DEV_ERR_TIMEOUT) {
        CP_CUDA(cudaMemsetAsync(p->status, 0, sizeof(uint32_t), p->st));
        return set_error("a bounded device wait gave up"), CP_ERR_TIMEOUT;
    }
    if (s & DEV_ERR_OVERFLOW) {
        CP_CUDA(cudaMemsetAsync(p->status, 0, sizeof(uint32_t), p->st));
        return set_error("the obstacle index met more entries than its capacity (max_grid_items)"), CP_ERR_ARG;
    }
    return CP_OK;
}

}  // namespace

extern "C" {

const char *cp_last_error(void) { return g_err; }

int32_t cp_version(void) { return CP_VERSION; }

int64_t cp_launch_count(void) { return g_launches.load(); }

void cp_debug_fail_allocations(int32_t n) { g_fail_allocs.store(n > 0 ? n : 0); }

int cp_plan_init(const cp_model *model, const cp_scene *scene, const cp_params *params,
                 void *stream, cp_planner **out)
{
    g_err[0] = 0;
    if (!out) return set_error("out is NULL"), CP_ERR_ARG;
    *out = nullptr;
    int rc;
    if ((rc = validate_model(model)) != CP_OK) return rc;
    if ((rc = validate_scene(scene)) != CP_OK) return rc;
    if ((rc = validate_params(params)) != CP_OK) return rc;

    cp_planner *p = new (std::nothrow) cp_planner();
    if (!p) return set_error("host allocation failed"), CP_ERR_OOM;
    p->st = (cudaStream_t)stream;
    p->prm = *params;
    if (p->prm.smooth_margin == 0.0) p->prm.smooth_margin = 0.05;
    if (p->prm.smooth_beta == 0.0) p->prm.smooth_beta = 0.01;
    p->N = params->n_candidates;
    p->K = params->n_waypoints;
    p->S = params->substeps;
    p->D = 4 * p->K;
    p->n_s = (p->K + 3) * p->S;
    p->chunks = (p->n_s + 31) / 32;
    p->nu = params->n_elites > 0 ? params->n_elites : p->N / 2;
    if (p->nu < 1) p->nu = 1;
    p->n_mean_chunks = update_chunks(p->nu, p->D);
    p->cap_cyl = params->max_cylinders > scene->n_cyl ? params->max_cylinders : scene->n_cyl;
    p->cap_box = params->max_boxes > scene->n_box ? params->max_boxes : scene->n_box;
    p->mdev = make_model(model);

    auto fail = [&](int code) {
        if (p->base) cudaFree(p->base);
        delete p;
        return code;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
    int smem_optin = 0;
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->smem_optin = smem_optin;
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaDeviceGetAttribute"));
    p->use_grid = params->grid_cell > 0.0;
    int64_t cells = 0;
    if (p->use_grid) {
        // polar index: kPolarBins angular bins, rings of width grid_cell out to
        // grid_half_extent (the last ring open outwards)
        const double h = params->grid_cell;
        double W = params->grid_half_extent;
        if (W <= 0.0)
            W = model->boom_len + model->jib_len +
                std::fmax(std::fabs(model->q_min[3]), std::fabs(model->q_max[3])) + 4.0;
        const int64_t n_ring = (int64_t)std::ceil(W / h);
        if (n_ring < 1 || n_ring * kPolarBins > (1 << 22)) {
            set_error("polar index of %d x %lld cells is outside 1..2^22 cells", kPolarBins, (long long)n_ring);
            return fail(CP_ERR_ARG);
        }
        cells = n_ring * kPolarBins;
        p->gdev.n_ang = kPolarBins;
        p->gdev.n_ring = (int)n_ring;
        p->gdev.inv_da = (float)(kPolarBins / (2.0 * M_PI));
        p->gdev.inv_dr = (float)(1.0 / h);
        p->grid_cap = params->max_grid_items > 0
                          ? params->max_grid_items
                          : polar_items_bound(scene, p->mdev.r_max, kPolarBins);
        if (p->grid_cap < 1) p->grid_cap = 1;
    }
    const size_t eval_smem = p->use_grid ? 0 : eval_smem_bytes(p->cap_cyl, p->cap_box, p->S);
    if (eval_smem > (size_t)smem_optin) {
        set_error("scene capacity (%d cylinders, %d boxes) needs %zu B of shared memory; the "
                  "device allows %d B per block", p->cap_cyl, p->cap_box, eval_smem, smem_optin);
        return fail(CP_ERR_ARG);
    }
    if ((rc = eval_configure(eval_smem > 48 * 1024 ? eval_smem : 48 * 1024)) != CP_OK) return fail(rc);
    if ((rc = factor_configure()) != CP_OK) return fail(rc);
    if ((rc = sample_configure()) != CP_OK) return fail(rc);
    if ((rc = update_configure()) != CP_OK) return fail(rc);

    const size_t N = p->N, D = p->D, nu = p->nu, ch = p->chunks, mc = p->n_mean_chunks;
    Layout L;
    const size_t o_cyl_in = L.take<cp_cylinder>(p->cap_cyl + 1);
    const size_t o_box_in = L.take<cp_box>(p->cap_box + 1);
    const size_t o_filt = L.take<float4>(p->cap_cyl + 1);
    const size_t o_exact = L.take<float4>(p->cap_cyl + 1);
    const size_t o_group = L.take<float4>(n_groups(p->cap_cyl) + 1);
    const size_t o_bc = L.take<float4>(p->cap_box + 1);
    const size_t o_bh = L.take<float4>(p->cap_box + 1);
    const size_t o_basis = L.take<float4>(2 * (size_t)p->S);
    const size_t o_consts = L.take<double>(16);
    const size_t o_mu = L.take<double>(D);
    const size_t o_C = L.take<double>(D * D);
    const size_t o_L = L.take<double>(D * D);
    const size_t o_Lt = L.take<float>(D * D);
    const size_t o_xi = L.take<float>(N * D);
    const size_t o_J = L.take<double>(N);
    const size_t o_terms = L.take<double>(N * 5);
    const size_t o_flag = L.take<uint8_t>(N);
    // work items of an evaluation of n <= N candidates: n P(n) <= eval_item_capacity(N, chunks)
    const size_t item_cap = eval_item_capacity(N, ch);
    const size_t o_item_sum = L.take<double>(item_cap * 4);
    const size_t o_item_count = L.take<uint32_t>(item_cap);
    p->item_cap = item_cap;
    const size_t o_rank = L.take<int>(N);
    const size_t o_elite = L.take<int>(nu);
    const size_t o_elites = L.take<float>(nu * D);
    const size_t o_w = L.take<double>(nu);
    const size_t o_mean_part = L.take<double>((mc + 1) * D);   // chunk partials, then S1
    const size_t o_cov_part = L.take<double>(mc * D * D);
    const size_t o_mom_y = L.take<double>(2 * nu * D);
    const size_t o_best = L.take<double>(1);
    const size_t o_status = L.take<uint32_t>(1);
    const size_t o_ctrl = L.take<double>(4 * ((size_t)p->K + 8));
    const size_t o_mean_xi = L.take<float>(D);
    const size_t o_mean_J = L.take<double>(1);
    const size_t o_mean_terms = L.take<double>(5);
    const size_t o_mean_flag = L.take<uint8_t>(1);
    const size_t o_grid_count = L.take<int>((size_t)cells + 1);
    const size_t o_grid_cursor = L.take<int>((size_t)cells + 1);
    const size_t o_grid_start = L.take<int>((size_t)cells + 1);
    const size_t o_grid_items = L.take<float4>(p->use_grid ? (size_t)p->grid_cap : 1);
    const size_t o_grad = L.take<float>(N * D);
    const size_t o_ends_f = L.take<float4>(2);
    const size_t units_max = (size_t)smooth_partial_units(p->num_sms);
    const size_t o_sp_g = L.take<float>(units_max * D);
    const size_t o_sp_J = L.take<double>(units_max);
    const size_t o_work = L.take<unsigned long long>(2);
    const size_t o_eval_queue = L.take<int>(1);
    const size_t o_metrics = L.take<double>((size_t)kMetricsRing * kMetricsCols);
    const size_t o_metrics_part = L.take<double>(3 * (size_t)kMetricsBlocks);
    const size_t o_cma = L.take<double>(4);
    const size_t o_psig = L.take<double>(D);
    const size_t o_pc = L.take<double>(D);
    const size_t o_mu_prev = L.take<double>(D);
    const bool elite_sampler = p->prm.sampler == CP_SAMPLE_ELITES;
    p->elite_slices = elite_sampler ? elite_slices(p->N, p->D, p->nu, p->num_sms) : 1;
    const size_t o_elite_Y = L.take<float>(elite_sampler ? elite_operand_floats(p->nu, p->D) : 1);
    const size_t o_mu_f = L.take<float>(D);
    const size_t o_mu_lo = L.take<float>(D);
    const size_t o_elite_sw = L.take<float>(elite_sampler ? nu : 1);
    const size_t o_elite_mp =
        L.take<double>(elite_sampler ? (size_t)elite_update_blocks(p->nu, p->num_sms) * D : 1);
    const size_t o_elite_bar = L.take<unsigned int>(2);
    const size_t o_sample_part = L.take<float>(elite_sampler ? (size_t)p->elite_slices * N * D : 1);
    const bool radix = p->N >= kRadixMinN;
    const size_t o_rka = L.take<unsigned long long>(radix ? N : 1);
    const size_t o_rkb = L.take<unsigned long long>(radix ? N : 1);
    const size_t o_rva = L.take<int>(radix ? N : 1);
    const size_t o_rvb = L.take<int>(radix ? N : 1);
    const size_t o_rh = L.take<int>(radix ? radix_hist_ints(p->N) : 1);
    int32_t left = g_fail_allocs.load();
    while (left > 0 && !g_fail_allocs.compare_exchange_weak(left, left - 1)) {
    }
    e = left > 0 ? cudaErrorMemoryAllocation : cudaMalloc((void **)&p->base, L.bytes);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(workspace)"));
    char *b = p->base;
    p->cyl_in = (cp_cylinder *)(b + o_cyl_in);
    p->box_in = (cp_box *)(b + o_box_in);
    p->cyl_filt = (float4 *)(b + o_filt);
    p->cyl_group = (float4 *)(b + o_group);
    p->cyl_exact = (float4 *)(b + o_exact);
    p->box_c = (float4 *)(b + o_bc);
    p->box_h = (float4 *)(b + o_bh);
    p->basis = (float4 *)(b + o_basis);
    p->consts = (double *)(b + o_consts);
    p->mu = (double *)(b + o_mu);
    p->C = (double *)(b + o_C);
    p->L = (double *)(b + o_L);
    p->Lt = (float *)(b + o_Lt);
    p->xi = (float *)(b + o_xi);
    p->J = (double *)(b + o_J);
    p->terms = (double *)(b + o_terms);
    p->flag = (uint8_t *)(b + o_flag);
    p->item_sum = (double *)(b + o_item_sum);
    p->item_count = (uint32_t *)(b + o_item_count);
    p->rank = (int *)(b + o_rank);
    p->elite = (int *)(b + o_elite);
    p->elites = (float *)(b + o_elites);
    p->w = (double *)(b + o_w);
    p->mean_part = (double *)(b + o_mean_part);
    p->cov_part = (double *)(b + o_cov_part);
    p->mom_y = (double *)(b + o_mom_y);
    p->best = (double *)(b + o_best);
    p->status = (uint32_t *)(b + o_status);
    p->ctrl = (double *)(b + o_ctrl);
    p->mean_xi = (float *)(b + o_mean_xi);
    p->mean_J = (double *)(b + o_mean_J);
    p->mean_terms = (double *)(b + o_mean_terms);
    p->mean_flag = (uint8_t *)(b + o_mean_flag);
    p->grad = (float *)(b + o_grad);
    p->ends_f = (float4 *)(b + o_ends_f);
    p->work = (unsigned long long *)(b + o_work);
    p->eval_queue = (int *)(b + o_eval_queue);
    p->metrics = (double *)(b + o_metrics);
    p->metrics_part = (double *)(b + o_metrics_part);
    p->cma = (double *)(b + o_cma);
    p->p_sigma = (double *)(b + o_psig);
    p->p_c = (double *)(b + o_pc);
    p->mu_prev = (double *)(b + o_mu_prev);
    p->elite_Y = (float *)(b + o_elite_Y);
    p->mu_f = (float *)(b + o_mu_f);
    p->mu_lo = (float *)(b + o_mu_lo);
    p->elite_sw = (float *)(b + o_elite_sw);
    p->elite_mean_part = (double *)(b + o_elite_mp);
    p->elite_bar = (unsigned int *)(b + o_elite_bar);
    p->sample_part = (float *)(b + o_sample_part);
    p->cmak = cma_consts(p->D, p->nu);
    p->rkey_a = (unsigned long long *)(b + o_rka);
    p->rkey_b = (unsigned long long *)(b + o_rkb);
    p->rval_a = (int *)(b + o_rva);
    p->rval_b = (int *)(b + o_rvb);
    p->rhist = (int *)(b + o_rh);
    p->smooth_part_g = (float *)(b + o_sp_g);
    p->smooth_part_J = (double *)(b + o_sp_J);
    p->grid_count = (int *)(b + o_grid_count);
    p->grid_cursor = (int *)(b + o_grid_cursor);
    p->grid_start = (int *)(b + o_grid_start);
    p->grid_items = (float4 *)(b + o_grid_items);
    p->gdev.cell_start = p->grid_start;
    p->gdev.items = p->grid_items;
    p->gdev.capacity = (int)std::min<int64_t>(p->grid_cap, 0x7FFFFFFF);
    p->sdev.cyl_filt = p->cyl_filt;
    p->sdev.cyl_group = p->cyl_group;
    p->sdev.cyl_exact = p->cyl_exact;
    p->sdev.box_c = p->box_c;
    p->sdev.box_h = p->box_h;

    e = cudaMemsetAsync(p->base, 0, L.bytes, p->st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(workspace)"));
    double lim[8];
    for (int j = 0; j < 4; ++j) {
        lim[j] = model->q_min[j];
        lim[4 + j] = model->q_max[j];
    }
    e = cudaMemcpyAsync(p->consts + 8, lim, sizeof lim, cudaMemcpyHostToDevice, p->st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpyAsync(limits)"));
    if ((rc = stage_scene(p, scene)) != CP_OK) return fail(rc);
    if ((rc = launch_basis_table(p->S, p->basis, p->st)) != CP_OK) return fail(rc);
    if ((rc = launch_weights(p->nu, p->w, p->st)) != CP_OK) return fail(rc);
    if (p->prm.sampler == CP_SAMPLE_ELITES &&
        (rc = launch_elite_weights(p->w, p->nu, p->prm.sigma, p->elite_sw, p->st)) != CP_OK)
        return fail(rc);
    e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamSynchronize(init)"));
    *out = p;
    return CP_OK;
}

void cp_destroy(cp_planner *p)
{
    if (!p) return;
    cudaStreamSynchronize(p->st);
    p->timer.destroy();
    if (p->plan_exec) cudaGraphExecDestroy(p->plan_exec);
    if (p->base) cudaFree(p->base);
    delete p;
}

int cp_set_scene(cp_planner *p, const cp_scene *scene)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    int rc = validate_scene(scene);
    if (rc != CP_OK) return rc;
    return stage_scene(p, scene);
}

int cp_set_endpoints(cp_planner *p, const double h_q0[4], const double h_qd[4])
{
    if (!p || !h_q0 || !h_qd) return set_error("NULL argument"), CP_ERR_ARG;
    for (int j = 0; j < 4; ++j)
        if (!is_finite(h_q0[j]) || !is_finite(h_qd[j])) return set_error("end points must be finite"), CP_ERR_ARG;
    double ends[8];
    memcpy(ends, h_q0, 4 * sizeof(double));
    memcpy(ends + 4, h_qd, 4 * sizeof(double));
    CP_CUDA(cudaMemcpyAsync(p->consts, ends, sizeof ends, cudaMemcpyHostToDevice, p->st));
    // the rank counters are zero between updates; a reset restores that after any failure
    CP_CUDA(cudaMemsetAsync(p->rank, 0, sizeof(int) * p->N, p->st));
    p->q0f = make_float4((float)h_q0[0], (float)h_q0[1], (float)h_q0[2], (float)h_q0[3]);
    p->qdf = make_float4((float)h_qd[0], (float)h_qd[1], (float)h_qd[2], (float)h_qd[3]);
    int rc = launch_init_distribution(p->consts, p->consts + 4, p->consts + 8, p->consts + 12, p->K,
                                      p->prm.init_std_frac, p->mu, p->C, p->ends_f, p->st);
    if (rc != CP_OK) return rc;
    if ((rc = launch_cma_reset(p->prm.sigma, p->D, p->cma, p->p_sigma, p->p_c, p->st)) != CP_OK) return rc;
    p->iteration = 0;
    p->elites_ready = false;
    p->have_endpoints = true;
    p->metrics_count = 0;
    return run_factor(p);
}

int cp_sample(cp_planner *p, int32_t iter, float *d_xi)
{
    if (!p || !d_xi) return set_error("NULL argument"), CP_ERR_ARG;
    if (!aligned16(d_xi)) return set_error("d_xi is not 16-byte aligned"), CP_ERR_ARG;
    if (iter < 0) return set_error("iteration must be >= 0"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    return run_sample(p, iter, d_xi);
}

int cp_evaluate(cp_planner *p, const float *d_xi, int32_t n, double *d_J, uint8_t *d_flag,
                double *d_terms, uint32_t *d_substep_flags, float *d_pen)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (n < 0 || n > p->N) return set_error("n = %d outside 0..N = %d", n, p->N), CP_ERR_ARG;
    if (n > 0 && (!d_xi || !d_J)) return set_error("d_xi and d_J are required"), CP_ERR_ARG;
    if (!aligned16(d_xi)) return set_error("d_xi is not 16-byte aligned"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    if (n == 0) return CP_OK;
    return run_eval(p, d_xi, n, d_J, d_flag, d_terms, d_substep_flags, d_pen);
}

int cp_update(cp_planner *p, const double *d_J, const float *d_xi)
{
    if (!p || !d_J || !d_xi) return set_error("NULL argument"), CP_ERR_ARG;
    if (!aligned16(d_xi)) return set_error("d_xi is not 16-byte aligned"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    return run_update(p, d_J, d_xi);
}

bool same_scene(const SceneDev &a, const SceneDev &b)
{
    return a.cyl_filt == b.cyl_filt && a.cyl_exact == b.cyl_exact && a.n_cyl == b.n_cyl && a.box_c == b.box_c &&
           a.box_h == b.box_h && a.n_box == b.n_box && a.cyl_group == b.cyl_group &&
           memcmp(&a.z_lo_all, &b.z_lo_all, sizeof(float)) == 0 && memcmp(&a.z_hi_all, &b.z_hi_all, sizeof(float)) == 0;
}

bool same_grid(const PolarDev &a, const PolarDev &b)
{
    return a.n_ang == b.n_ang && a.n_ring == b.n_ring && memcmp(&a.inv_da, &b.inv_da, sizeof(float)) == 0 &&
           memcmp(&a.inv_dr, &b.inv_dr, sizeof(float)) == 0 && memcmp(&a.w_max, &b.w_max, sizeof(float)) == 0 &&
           a.cell_start == b.cell_start && a.items == b.items && a.capacity == b.capacity;
}

// The iterations of cp_plan from p->iteration as one CUDA graph launch, recorded on first
// use and again whenever the start iteration, the count, the scene records or the end
// points (kernel arguments of the recorded launches) differ from the recorded ones.
int run_plan_graph(cp_planner *p, int iters)
{
    const bool same = p->plan_exec && p->plan_start == p->iteration && p->plan_iters == iters &&
                      p->plan_ready_before == p->elites_ready && p->plan_metrics == p->metrics_on &&
                      same_scene(p->plan_sdev, p->sdev) && same_grid(p->plan_gdev, p->gdev) &&
                      memcmp(&p->plan_q0, &p->q0f, sizeof(float4)) == 0 &&
                      memcmp(&p->plan_qd, &p->qdf, sizeof(float4)) == 0;
    const int start = p->iteration;
    const bool ready_before = p->elites_ready;
    if (!same) {
        if (p->plan_exec) {
            cudaGraphExecDestroy(p->plan_exec);
            p->plan_exec = nullptr;
        }
        const int64_t launches_before = g_launches.load();
        const cudaError_t e_begin = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
        if (e_begin != cudaSuccess) {
            cudaGetLastError();   // clear it, so that later launch checks do not see it
            return cuda_fail(e_begin, "cudaStreamBeginCapture");
        }
        int rc = CP_OK;
        for (int it = 0; it < iters && rc == CP_OK; ++it) rc = run_iteration(p);
        cudaGraph_t graph = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(p->st, &graph);
        p->iteration = start;
        p->plan_ready_before = ready_before;
        p->plan_ready_after = p->elites_ready;
        p->elites_ready = ready_before;
        p->plan_nodes = g_launches.load() - launches_before;   // recorded, not run
        g_launches.fetch_sub(p->plan_nodes);
        if (rc != CP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e_end != cudaSuccess) return cuda_fail(e_end, "cudaStreamEndCapture");
        const cudaError_t e_inst = cudaGraphInstantiate(&p->plan_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e_inst != cudaSuccess) {
            p->plan_exec = nullptr;
            return cuda_fail(e_inst, "cudaGraphInstantiate");
        }
        p->plan_start = start;
        p->plan_iters = iters;
        p->plan_metrics = p->metrics_on;
        p->plan_sdev = p->sdev;
        p->plan_gdev = p->gdev;
        p->plan_q0 = p->q0f;
        p->plan_qd = p->qdf;
    }
    CP_CUDA(cudaGraphLaunch(p->plan_exec, p->st));
    g_launches.fetch_add(p->plan_nodes, std::memory_order_relaxed);
    p->iteration = start + iters;
    if (p->plan_metrics) p->metrics_count += iters;
    p->elites_ready = p->plan_ready_after;
    return CP_OK;
}

int cp_plan(cp_planner *p, int32_t iters, double *h_ctrl, cp_plan_stats *stats)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (iters < 0) return set_error("iters must be >= 0"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    int rc;
    // graphs are recorded from a stream of the caller's; the legacy default stream cannot
    // be captured, so plans on it (and timed plans, whose stage events sit between the
    // kernels) launch kernel by kernel
    const bool capturable = p->st != nullptr && p->st != cudaStreamLegacy && p->st != cudaStreamPerThread;
    NvtxRange range("craneplan:plan");
    if (p->timer.on || iters == 0 || !capturable) {
        for (int it = 0; it < iters; ++it) {
            if ((rc = run_iteration(p)) != CP_OK) return rc;
            if (p->metrics_on) p->metrics_count += 1;
        }
    } else if ((rc = run_plan_graph(p, iters)) != CP_OK) {
        return rc;
    }
    if ((rc = launch_mean_to_candidate(p->mu, p->D, p->mean_xi, p->st)) != CP_OK) return rc;
    if ((rc = run_eval(p, p->mean_xi, 1, p->mean_J, p->mean_flag, p->mean_terms, nullptr, nullptr)) != CP_OK)
        return rc;
    if ((rc = launch_control_points(p->consts, p->consts + 4, p->mu, p->K, p->ctrl, p->st)) != CP_OK)
        return rc;
    double host[8];
    CP_CUDA(cudaMemcpyAsync(host, p->mean_J, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CP_CUDA(cudaMemcpyAsync(host + 1, p->mean_terms, 5 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CP_CUDA(cudaMemcpyAsync(host + 6, p->best, sizeof(double), cudaMemcpyDeviceToHost, p->st));
    if (h_ctrl)
        CP_CUDA(cudaMemcpyAsync(h_ctrl, p->ctrl, sizeof(double) * 4 * (p->K + 8),
                                cudaMemcpyDeviceToHost, p->st));
    if ((rc = check_status(p)) != CP_OK) return rc;   // synchronises
    if (stats) {
        stats->J = host[0];
        stats->Jp = host[1];
        stats->Jc = host[2];
        stats->Jl = host[3];
        stats->length = host[4];
        stats->n_flagged = (int32_t)host[5];
        stats->flag = stats->n_flagged > 0;
        stats->iterations = iters;
        stats->iteration = p->iteration;
        stats->best_J = host[6];
    }
    return CP_OK;
}

static int smooth_check(cp_planner *p, int n, const void *xi)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (n < 0 || n > p->N) return set_error("n = %d outside 0..N = %d", n, p->N), CP_ERR_ARG;
    if (n > 0 && !xi) return set_error("d_xi is NULL"), CP_ERR_ARG;
    if (!aligned16(xi)) return set_error("d_xi is not 16-byte aligned"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    const size_t smem = smooth_smem_bytes(p->sdev.n_cyl, p->sdev.n_box, p->S, p->K);
    if (smem > (size_t)p->smem_optin)
        return set_error("the smooth cost stages %zu B of obstacles per block; the device allows "
                         "%d B", smem, p->smem_optin), CP_ERR_ARG;
    return CP_OK;
}

static int run_smooth(cp_planner *p, const float *xi, int n, const double *gJ, double *J, float *dxi)
{
    return launch_smooth(p->mdev, p->sdev, xi, n, p->K, p->S, p->q0f, p->qdf, p->basis,
                         p->prm.smooth_margin, p->prm.smooth_beta, p->prm.w_c * p->prm.lambda_c,
                         p->prm.w_l, gJ, J, dxi, p->smooth_part_g, p->smooth_part_J, p->eval_queue,
                         p->num_sms, p->st);
}

int cp_smooth_cost(cp_planner *p, const float *d_xi, int32_t n, double *d_J)
{
    int rc = smooth_check(p, n, d_xi);
    if (rc != CP_OK) return rc;
    if (n > 0 && !d_J) return set_error("d_J is NULL"), CP_ERR_ARG;
    return run_smooth(p, d_xi, n, nullptr, d_J, nullptr);
}

int cp_smooth_cost_grad(cp_planner *p, const float *d_xi, int32_t n, const double *d_gJ,
                        double *d_J, float *d_dxi)
{
    NvtxRange range("craneplan:smooth_cost_grad");
    int rc = smooth_check(p, n, d_xi);
    if (rc != CP_OK) return rc;
    if (n > 0 && !d_dxi) return set_error("d_dxi is NULL"), CP_ERR_ARG;
    return run_smooth(p, d_xi, n, d_gJ, d_J, d_dxi);
}

int cp_polish(cp_planner *p, float *d_xi, int32_t n, int32_t steps, double alpha)
{
    NvtxRange range("craneplan:polish");
    int rc = smooth_check(p, n, d_xi);
    if (rc != CP_OK) return rc;
    if (steps < 0 || !is_finite(alpha)) return set_error("steps >= 0 and finite alpha"), CP_ERR_ARG;
    for (int s = 0; s < steps; ++s) {
        if ((rc = run_smooth(p, d_xi, n, nullptr, nullptr, p->grad)) != CP_OK) return rc;
        if ((rc = launch_axpy(d_xi, p->grad, alpha, (int64_t)n * p->D, p->st)) != CP_OK) return rc;
    }
    return CP_OK;
}

int cp_signed_distance(cp_planner *p, const float *d_q, int32_t n, float *d_d)
{
    NvtxRange range("craneplan:signed_distance");
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (n < 0 || (n > 0 && (!d_q || !d_d))) return set_error("invalid arguments"), CP_ERR_ARG;
    return launch_signed_distance(p->mdev, p->sdev, d_q, n, d_d, p->st);
}

int cp_forward_kinematics(cp_planner *p, const float *d_q, int32_t n, float *d_centres, float *d_tip)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (n < 0 || (n > 0 && !d_q)) return set_error("invalid arguments"), CP_ERR_ARG;
    if ((uintptr_t)d_q & 15u) return set_error("d_q must be 16-byte aligned"), CP_ERR_ARG;
    return launch_forward_kinematics(p->mdev, d_q, n, d_centres, d_tip, p->st);
}

namespace {

int hull_dims(const cp_hull_model *hulls, HullDims &d)
{
    const cp_hull_model def = {{0.2, 0.2, 0.15}, {0.2, 0.2, 0.15}, 0.2, 0.25, 1.0};
    const cp_hull_model &h = hulls ? *hulls : def;
    for (int k = 0; k < 3; ++k) {
        if (!(h.w[k] > 0.0) || !(h.h[k] > 0.0) || !is_finite(h.w[k]) || !is_finite(h.h[k]))
            return set_error("hull half extents must be finite and > 0"), CP_ERR_ARG;
        d.w[k] = (float)h.w[k];
        d.hh[k] = (float)h.h[k];
    }
    if (!(h.pad >= 0.0) || !(h.grapple_w > 0.0) || !(h.grapple_len > 0.0) || !is_finite(h.pad) ||
        !is_finite(h.grapple_w) || !is_finite(h.grapple_len))
        return set_error("hull pad must be >= 0 and the grapple box > 0"), CP_ERR_ARG;
    d.pad = (float)h.pad;
    d.gw = (float)h.grapple_w;
    d.glen = (float)h.grapple_len;
    return CP_OK;
}

}  // namespace

int cp_hull_penetration(cp_planner *p, const float *d_q, int32_t n, const cp_hull_model *hulls, float *d_pen)
{
    NvtxRange range("craneplan:hull_penetration");
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (n < 0 || (n > 0 && (!d_q || !d_pen))) return set_error("invalid arguments"), CP_ERR_ARG;
    if ((uintptr_t)d_q & 15u) return set_error("d_q must be 16-byte aligned"), CP_ERR_ARG;
    HullDims d{};
    const int rc = hull_dims(hulls, d);
    if (rc != CP_OK) return rc;
    return launch_hull_penetration(p->mdev, p->sdev, d, d_q, n, d_pen, p->st);
}

int cp_set_hull_model(cp_planner *p, const cp_hull_model *hulls)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    HullDims d{};
    const int rc = hull_dims(hulls, d);
    if (rc != CP_OK) return rc;
    p->hulls = d;
    if (p->plan_exec) {   // the recorded plan holds the old model as a kernel argument
        cudaGraphExecDestroy(p->plan_exec);
        p->plan_exec = nullptr;
    }
    return CP_OK;
}

int cp_ik(cp_planner *p, const float *d_targets, int32_t n, const cp_ik_params *ik,
          const float *d_q_init, float *d_q, float *d_f, int32_t *d_restart, float *d_r)
{
    NvtxRange range("craneplan:ik");
    if (!p || !ik) return set_error("NULL argument"), CP_ERR_ARG;
    if (n < 0 || (n > 0 && (!d_targets || !d_q || !d_f))) return set_error("invalid arguments"), CP_ERR_ARG;
    if (ik->restarts < 1 || ik->restarts > CP_IK_MAX_RESTARTS)
        return set_error("restarts must be in 1..%d", CP_IK_MAX_RESTARTS), CP_ERR_ARG;
    if (ik->iters < 0) return set_error("iters must be >= 0"), CP_ERR_ARG;
    if (((uintptr_t)d_targets | (uintptr_t)d_q_init | (uintptr_t)d_q) & 15u)
        return set_error("d_targets, d_q_init and d_q must be 16-byte aligned"), CP_ERR_ARG;
    if (!(ik->lambda_q >= 0.0) || !(ik->lambda_c >= 0.0) || !(ik->grapple_len >= 0.0) || !(ik->mu0 > 0.0) ||
        !is_finite(ik->lambda_q) || !is_finite(ik->lambda_c) || !is_finite(ik->grapple_len) || !is_finite(ik->mu0))
        return set_error("IK scales must be finite and >= 0, mu0 > 0"), CP_ERR_ARG;
    return launch_ik(p->mdev, p->sdev, d_targets, d_q_init, n, ik->restarts, ik->iters, (float)ik->lambda_q,
                     (float)ik->lambda_c, (float)ik->grapple_len, (float)ik->mu0, ik->seed, ik->query, d_q, d_f,
                     d_restart, d_r, p->st);
}

int cp_get_distribution(const cp_planner *p, double *d_mu, double *d_C)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (d_C) {
        const int rc = materialise_distribution(p);
        if (rc != CP_OK) return rc;
    }
    if (d_mu) CP_CUDA(cudaMemcpyAsync(d_mu, p->mu, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    if (d_C)
        CP_CUDA(cudaMemcpyAsync(d_C, p->C, sizeof(double) * p->D * p->D, cudaMemcpyDeviceToDevice, p->st));
    return CP_OK;
}

int cp_set_distribution(cp_planner *p, const double *d_mu, const double *d_C, int32_t iter)
{
    if (!p || !d_mu || !d_C) return set_error("NULL argument"), CP_ERR_ARG;
    if (iter < 0) return set_error("iteration must be >= 0"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    CP_CUDA(cudaMemcpyAsync(p->mu, d_mu, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    CP_CUDA(cudaMemcpyAsync(p->C, d_C, sizeof(double) * p->D * p->D, cudaMemcpyDeviceToDevice, p->st));
    p->iteration = iter;
    p->elites_ready = false;
    return run_factor(p);
}

int cp_get_factor(const cp_planner *p, double *d_L)
{
    if (!p || !d_L) return set_error("NULL argument"), CP_ERR_ARG;
    const int rc = materialise_distribution(p);
    if (rc != CP_OK) return rc;
    CP_CUDA(cudaMemcpyAsync(d_L, p->L, sizeof(double) * p->D * p->D, cudaMemcpyDeviceToDevice, p->st));
    return CP_OK;
}

int cp_get_cma_state(const cp_planner *p, double *d_state)
{
    if (!p || !d_state) return set_error("NULL argument"), CP_ERR_ARG;
    CP_CUDA(cudaMemcpyAsync(d_state, p->cma, sizeof(double), cudaMemcpyDeviceToDevice, p->st));
    CP_CUDA(cudaMemcpyAsync(d_state + 1, p->p_sigma, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    CP_CUDA(cudaMemcpyAsync(d_state + 1 + p->D, p->p_c, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    return CP_OK;
}

int cp_set_cma_state(cp_planner *p, const double *d_state)
{
    if (!p || !d_state) return set_error("NULL argument"), CP_ERR_ARG;
    if (!p->have_endpoints) return set_error("set the end points first"), CP_ERR_STATE;
    CP_CUDA(cudaMemcpyAsync(p->cma, d_state, sizeof(double), cudaMemcpyDeviceToDevice, p->st));
    CP_CUDA(cudaMemcpyAsync(p->p_sigma, d_state + 1, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    CP_CUDA(cudaMemcpyAsync(p->p_c, d_state + 1 + p->D, sizeof(double) * p->D, cudaMemcpyDeviceToDevice, p->st));
    return run_factor(p);
}

int cp_get_elites(const cp_planner *p, int32_t *d_idx)
{
    if (!p || !d_idx) return set_error("NULL argument"), CP_ERR_ARG;
    CP_CUDA(cudaMemcpyAsync(d_idx, p->elite, sizeof(int32_t) * p->nu, cudaMemcpyDeviceToDevice, p->st));
    return CP_OK;
}

int cp_get_population(const cp_planner *p, float *d_xi, double *d_J)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    if (d_xi && !aligned16(d_xi)) return set_error("d_xi must be 16-byte aligned"), CP_ERR_ARG;
    if (d_xi)
        CP_CUDA(cudaMemcpyAsync(d_xi, p->xi, sizeof(float) * (size_t)p->N * p->D, cudaMemcpyDeviceToDevice, p->st));
    if (d_J) CP_CUDA(cudaMemcpyAsync(d_J, p->J, sizeof(double) * (size_t)p->N, cudaMemcpyDeviceToDevice, p->st));
    return CP_OK;
}

int cp_set_metrics(cp_planner *p, int32_t on)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    p->metrics_on = on != 0;
    return CP_OK;
}

int cp_get_metrics(cp_planner *p, double *h_rows, int32_t max_rows, int32_t *n_rows)
{
    if (!p || !n_rows || max_rows < 0 || (max_rows > 0 && !h_rows)) return set_error("invalid arguments"), CP_ERR_ARG;
    int64_t n = std::min<int64_t>(p->metrics_count, kMetricsRing);
    n = std::min<int64_t>(n, max_rows);
    n = std::min<int64_t>(n, p->iteration);
    *n_rows = (int32_t)n;
    if (n == 0) return CP_OK;
    double ring[kMetricsRing * kMetricsCols];
    CP_CUDA(cudaMemcpyAsync(ring, p->metrics, sizeof ring, cudaMemcpyDeviceToHost, p->st));
    CP_CUDA(cudaStreamSynchronize(p->st));
    const int first = p->iteration - (int)n;   // oldest iteration returned
    for (int64_t r = 0; r < n; ++r)
        memcpy(h_rows + r * kMetricsCols, ring + (size_t)((first + r) % kMetricsRing) * kMetricsCols,
               sizeof(double) * kMetricsCols);
    return CP_OK;
}

int cp_philox4x32_10(const uint32_t *d_ctr, uint64_t key, int64_t n, uint32_t *d_out, void *stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return set_error("invalid arguments"), CP_ERR_ARG;
    return launch_philox(d_ctr, (uint32_t)key, (uint32_t)(key >> 32), n, d_out, (cudaStream_t)stream);
}

int cp_set_timing(cp_planner *p, int32_t on)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    CP_CUDA(cudaStreamSynchronize(p->st));
    p->timer.clear();
    p->timer.on = on != 0;
    CP_CUDA(cudaMemsetAsync(p->work, 0, sizeof(unsigned long long), p->st));
    CP_CUDA(cudaStreamSynchronize(p->st));
    return CP_OK;
}

int cp_get_timing(cp_planner *p, cp_timing *out)
{
    if (!p || !out) return set_error("NULL argument"), CP_ERR_ARG;
    CP_CUDA(cudaStreamSynchronize(p->st));
    double ms[ST_COUNT] = {0, 0, 0, 0};
    int64_t cnt[ST_COUNT] = {0, 0, 0, 0};
    for (int s = 0; s < ST_COUNT; ++s) {
        for (auto &pr : p->timer.spans[s]) {
            float t = 0.f;
            CP_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
            ms[s] += t;
            cnt[s] += 1;
        }
    }
    out->eval_ms = ms[ST_EVAL];
    out->eval_launches = cnt[ST_EVAL];
    out->sample_ms = ms[ST_SAMPLE];
    out->sample_launches = cnt[ST_SAMPLE];
    out->factor_ms = ms[ST_FACTOR];
    out->factor_launches = cnt[ST_FACTOR];
    out->update_ms = ms[ST_UPDATE];
    out->update_launches = cnt[ST_UPDATE];
    unsigned long long work[2] = {0, 0};
    CP_CUDA(cudaMemcpy(work, p->work, sizeof(work), cudaMemcpyDeviceToHost));
    out->eval_units = p->timer.units;
    out->eval_obstacle_tests = p->timer.tests + (int64_t)work[0];
    out->eval_box_tests = p->timer.grid ? (int64_t)work[1] : -1;
    // per-unit forms: every survivor takes the filter for 32 lanes x the spheres; the polar
    // form: every listed obstacle of a lane takes it for the lane's spheres
    out->eval_pair_tests = p->timer.grid ? out->eval_box_tests * p->mdev.n_spheres
                                         : out->eval_obstacle_tests * 32 * p->mdev.n_spheres;
    p->timer.clear();
    CP_CUDA(cudaMemsetAsync(p->work, 0, 2 * sizeof(unsigned long long), p->st));
    CP_CUDA(cudaStreamSynchronize(p->st));
    return CP_OK;
}

int cp_synchronize(cp_planner *p)
{
    if (!p) return set_error("planner is NULL"), CP_ERR_ARG;
    return check_status(p);
}

}  // extern "C"

// ------------------------------------------------------------------ batched form

struct cp_batch {
    int nq = 0, iters = 0;
    cudaStream_t st = nullptr;
    std::vector<cp_planner *> planners;
    ModelDev mdev{};
    int num_sms = 1, max_K = 0, max_S = 0, max_D = 0;
    int64_t total = 0;                 // sum of N
    double *h_in = nullptr;            // pinned [nq][8]: q0, qd
    double *h_out = nullptr;           // pinned [nq][kOutStride]
    char *base = nullptr;              // device memory of the batch
    double *d_in = nullptr, *d_out = nullptr;
    BatchQueryDev *qdev = nullptr;
    BatchEvalDev *ev_pop = nullptr, *ev_mean = nullptr;
    int2 *tab_init = nullptr, *tab_sample = nullptr, *tab_cand = nullptr, *tab_gather = nullptr;
    int2 *tab_mprep = nullptr, *tab_mpart = nullptr, *tab_mcomb = nullptr;
    int n_init = 0, n_sample = 0, n_cand = 0, n_gather = 0, n_mprep = 0, n_mpart = 0, n_mcomb = 0;
    int4 *tiles_pop = nullptr, *tiles_mean = nullptr;
    int64_t tiles_cap = 0;
    int n_tiles_pop = 0, n_tiles_mean = 0;
    int *queue = nullptr;              // [iters + 2] tile counters (the last one for cp_batch_evaluate)
    uint16_t *qid = nullptr;           // [total] query of each ranking position
    unsigned long long *key_a = nullptr, *key_b = nullptr;
    int *val_a = nullptr, *val_b = nullptr, *hist = nullptr;
    std::vector<int> order;            // queries by decreasing work per item (tile order)
    std::vector<int> items_pop, items_mean;
    cp_batch_shape shape{256, 0, 2};
    int eval_blocks = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t kernel_nodes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_run_ms = 0.0;          // device time of the last cp_batch_run
};

namespace {

constexpr int kOutStride = 8 + (CP_MAX_WAYPOINTS + 8) * 4;   // J, terms[5], best, status, ctrl

// The form the batched kernels implement, for query q.
int batch_query_ok(const cp_query &qr, int q, const cp_model *model)
{
    const cp_params &p = qr.params;
    if (!(p.grid_cell > 0.0))
        return set_error("query %d: the batched form evaluates with the polar obstacle index (grid_cell > 0)", q),
               CP_ERR_ARG;
    if (p.update_rule != CP_UPDATE_PAPER || p.sampler != CP_SAMPLE_FACTOR || p.collision_model != CP_COLLISION_SPHERES)
        return set_error("query %d: the batched form runs the paper's update rule, the factor sampler and the "
                         "sphere collision model", q),
               CP_ERR_ARG;
    if (p.debug_withhold_staging != 0) return set_error("query %d: no test hooks in the batched form", q), CP_ERR_ARG;
    (void)model;
    return CP_OK;
}

// Tiles of consecutive items of each query, queries in the given order.
void build_tiles(const std::vector<int> &order, const std::vector<int> &items, int per_tile, std::vector<int4> &out)
{
    out.clear();
    for (int q : order)
        for (int b = 0; b < items[q]; b += per_tile) out.push_back(make_int4(q, b, std::min(items[q], b + per_tile), 0));
}

int batch_upload_tiles(cp_batch *b)
{
    const int per_tile = b->shape.threads / 32 * b->shape.items_per_warp;
    std::vector<int4> pop, mean;
    build_tiles(b->order, b->items_pop, per_tile, pop);
    build_tiles(b->order, b->items_mean, per_tile, mean);
    if ((int64_t)pop.size() > b->tiles_cap || (int64_t)mean.size() > b->tiles_cap)
        return set_error("batched evaluation: %zu tiles exceed the %lld allocated", pop.size(), (long long)b->tiles_cap),
               CP_ERR_ARG;
    CP_CUDA(cudaMemcpyAsync(b->tiles_pop, pop.data(), sizeof(int4) * pop.size(), cudaMemcpyHostToDevice, b->st));
    CP_CUDA(cudaMemcpyAsync(b->tiles_mean, mean.data(), sizeof(int4) * mean.size(), cudaMemcpyHostToDevice, b->st));
    CP_CUDA(cudaStreamSynchronize(b->st));
    b->n_tiles_pop = (int)pop.size();
    b->n_tiles_mean = (int)mean.size();
    const int max_blocks = batch_eval_max_blocks(b->mdev, b->shape.threads, b->max_S, b->num_sms);
    if (max_blocks < 0) return CP_ERR_ARG;
    int blocks = max_blocks;
    if (b->shape.ctas_per_sm > 0) blocks = std::min(blocks, b->shape.ctas_per_sm * b->num_sms);
    b->eval_blocks = std::max(1, std::min(blocks, b->n_tiles_pop));
    return CP_OK;
}

// One run of the batch as stream work (recorded into the graph).
int record_batch(cp_batch *b)
{
    int rc;
    CP_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int) * (size_t)(b->iters + 2), b->st));
    CP_CUDA(cudaMemcpyAsync(b->d_in, b->h_in, sizeof(double) * 8 * b->nq, cudaMemcpyHostToDevice, b->st));
    if ((rc = launch_batch_init(b->qdev, b->tab_init, b->n_init, b->d_in, b->st)) != CP_OK) return rc;
    if ((rc = launch_batch_factor(b->qdev, b->nq, b->max_D, b->st)) != CP_OK) return rc;
    for (int t = 0; t < b->iters; ++t) {
        if ((rc = launch_batch_sample(b->qdev, b->tab_sample, b->n_sample, b->max_K, (uint32_t)t, b->st)) != CP_OK)
            return rc;
        if ((rc = launch_batch_eval_polar(b->mdev, b->ev_pop, b->tiles_pop, b->n_tiles_pop, b->queue + t, b->max_S,
                                          b->shape.threads, b->eval_blocks, b->st)) != CP_OK)
            return rc;
        if ((rc = launch_batch_finalize(b->qdev, b->tab_cand, b->n_cand, nullptr, b->st)) != CP_OK) return rc;
        int *sorted = nullptr;
        if ((rc = launch_batch_radix_rank(b->qdev, b->tab_cand, b->n_cand, (int)b->total, b->nq, b->qid, b->key_a,
                                          b->key_b, b->val_a, b->val_b, b->hist, &sorted, b->st)) != CP_OK)
            return rc;
        if ((rc = launch_batch_gather(b->qdev, b->tab_gather, b->n_gather, sorted, b->st)) != CP_OK) return rc;
        if ((rc = launch_batch_moments(b->qdev, b->nq, b->tab_mprep, b->n_mprep, b->tab_mpart, b->n_mpart, b->tab_mcomb,
                                       b->n_mcomb, b->st)) != CP_OK)
            return rc;
        if ((rc = launch_batch_factor(b->qdev, b->nq, b->max_D, b->st)) != CP_OK) return rc;
    }
    if ((rc = launch_batch_outputs(b->qdev, b->nq, true, nullptr, 0, b->st)) != CP_OK) return rc;
    const int mean_blocks = std::max(1, std::min(b->eval_blocks, b->n_tiles_mean));
    if ((rc = launch_batch_eval_polar(b->mdev, b->ev_mean, b->tiles_mean, b->n_tiles_mean, b->queue + b->iters,
                                      b->max_S, b->shape.threads, mean_blocks, b->st)) != CP_OK)
        return rc;
    if ((rc = launch_batch_finalize(b->qdev, nullptr, b->nq, b->ev_mean, b->st)) != CP_OK) return rc;
    if ((rc = launch_batch_outputs(b->qdev, b->nq, false, b->d_out, kOutStride, b->st)) != CP_OK) return rc;
    CP_CUDA(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * kOutStride * b->nq, cudaMemcpyDeviceToHost, b->st));
    return CP_OK;
}

int batch_record_graph(cp_batch *b)
{
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    CP_CUDA(cudaStreamSynchronize(b->st));
    const int64_t launches_before = g_launches.load();
    const cudaError_t e_begin = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e_begin != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e_begin, "cudaStreamBeginCapture");
    }
    const int rc = record_batch(b);
    cudaGraph_t graph = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(b->st, &graph);
    b->kernel_nodes = g_launches.load() - launches_before;   // recorded, not run
    g_launches.fetch_sub(b->kernel_nodes);
    if (rc != CP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e_end != cudaSuccess) return cuda_fail(e_end, "cudaStreamEndCapture");
    const cudaError_t e_inst = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e_inst != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e_inst, "cudaGraphInstantiate");
    }
    return CP_OK;
}

void batch_free(cp_batch *b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto *p : b->planners) cp_destroy(p);
    if (b->base) cudaFree(b->base);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->st) cudaStreamDestroy(b->st);
    if (b->h_in) cudaFreeHost(b->h_in);
    if (b->h_out) cudaFreeHost(b->h_out);
    delete b;
}

// Block table: for each query, `count(q)` entries {q, 0..count(q)-1}.
template <typename F>
void block_table(int nq, F count, std::vector<int2> &out)
{
    out.clear();
    for (int q = 0; q < nq; ++q) {
        const int c = count(q);
        for (int i = 0; i < c; ++i) out.push_back(make_int2(q, i));
    }
}

}  // namespace

extern "C" {

int cp_batch_init(const cp_model *model, const cp_query *queries, int32_t nq, int32_t iters,
                  cp_batch **out)
{
    g_err[0] = 0;
    if (!out) return set_error("out is NULL"), CP_ERR_ARG;
    *out = nullptr;
    if (!queries || nq < 1 || nq > 4096) return set_error("nq = %d outside 1..4096", nq), CP_ERR_ARG;
    if (iters < 0) return set_error("iters must be >= 0"), CP_ERR_ARG;
    int rc;
    if ((rc = validate_model(model)) != CP_OK) return rc;
    for (int q = 0; q < nq; ++q) {
        for (int j = 0; j < 4; ++j)
            if (!is_finite(queries[q].q0[j]) || !is_finite(queries[q].qd[j]))
                return set_error("query %d: end points must be finite", q), CP_ERR_ARG;
        if ((rc = batch_query_ok(queries[q], q, model)) != CP_OK) return rc;
    }
    cp_batch *b = new (std::nothrow) cp_batch();
    if (!b) return set_error("host allocation failed"), CP_ERR_OOM;
    b->nq = nq;
    b->iters = iters;
    auto fail = [&](int code) {
        batch_free(b);
        return code;
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaStreamCreateWithFlags"));
    if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaMallocHost((void **)&b->h_in, sizeof(double) * 8 * nq)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&b->h_out, sizeof(double) * kOutStride * nq)) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMallocHost"));
    for (int q = 0; q < nq; ++q) {
        cp_planner *p = nullptr;
        rc = cp_plan_init(model, &queries[q].scene, &queries[q].params, b->st, &p);
        if (rc != CP_OK) {
            char msg[512];
            snprintf(msg, sizeof msg, "query %d: %s", q, g_err);
            set_error("%s", msg);
            return fail(rc);
        }
        b->planners.push_back(p);
        p->have_endpoints = true;
        memcpy(b->h_in + 8 * q, queries[q].q0, 4 * sizeof(double));
        memcpy(b->h_in + 8 * q + 4, queries[q].qd, 4 * sizeof(double));
    }
    b->mdev = b->planners[0]->mdev;
    b->num_sms = b->planners[0]->num_sms;
    std::vector<BatchQueryDev> qh(nq);
    std::vector<BatchEvalDev> eh(nq), mh(nq);
    std::vector<int> G(nq);
    b->items_pop.resize(nq);
    b->items_mean.resize(nq);
    int64_t off = 0;
    for (int q = 0; q < nq; ++q) {
        cp_planner *p = b->planners[q];
        b->max_K = std::max(b->max_K, p->K);
        b->max_S = std::max(b->max_S, p->S);
        b->max_D = std::max(b->max_D, p->D);
        BatchQueryDev &d = qh[q];
        d.N = p->N;
        d.K = p->K;
        d.D = p->D;
        d.nu = p->nu;
        d.J = p->J;
        d.flag = p->flag;
        d.item_sum = p->item_sum;
        d.item_count = p->item_count;
        d.w_c = p->prm.w_c;
        d.w_l = p->prm.w_l;
        d.lambda_c = p->prm.lambda_c;
        d.xi = p->xi;
        d.mu = p->mu;
        d.C = p->C;
        d.L = p->L;
        d.Lt = p->Lt;
        d.seed_lo = (uint32_t)p->prm.seed;
        d.seed_hi = (uint32_t)(p->prm.seed >> 32);
        d.query = p->prm.query;
        d.sigma2 = p->prm.sigma * p->prm.sigma;
        d.elite = p->elite;
        d.elites = p->elites;
        d.w = p->w;
        d.best = p->best;
        d.s2p = p->cov_part;
        d.s1p = p->mean_part;
        d.eps = p->prm.eps;
        d.n_chunks = moments_chunking(p->nu, p->D, &d.per);
        d.mom_y = p->mom_y;
        d.cand_off = (int)off;
        d.status = p->status;
        d.consts = p->consts;
        d.init_std_frac = p->prm.init_std_frac;
        d.ends = p->ends_f;
        d.mean_xi = p->mean_xi;
        d.mean_J = p->mean_J;
        d.mean_terms = p->mean_terms;
        d.mean_flag = p->mean_flag;
        d.ctrl = p->ctrl;
        // the evaluation arguments of cp_plan's launches (run_eval) for the population and
        // the mean candidate
        for (int m = 0; m < 2; ++m) {
            EvalArgs a{};
            const int n = m == 0 ? p->N : 1;
            a.xi = (const float4 *)(m == 0 ? p->xi : p->mean_xi);
            a.n = n;
            a.K = p->K;
            a.S = p->S;
            a.n_s = p->n_s;
            a.chunks = p->chunks;
            a.G = eval_units_per_item(n, p->chunks);
            a.P = (p->chunks + a.G - 1) / a.G;
            a.div_S = fast_div((uint32_t)p->S);
            a.div_P = fast_div((uint32_t)a.P);
            a.ends = p->ends_f;
            a.broadphase = 1;
            a.status = p->status;
            a.basis = p->basis;
            a.item_sum = p->item_sum;
            a.item_count = p->item_count;
            BatchEvalDev &ev = m == 0 ? eh[q] : mh[q];
            ev.a = a;
            ev.sc = p->sdev;
            ev.g = p->gdev;
            if ((size_t)n * a.P > p->item_cap)
                return fail((set_error("query %d: %d candidates need more work items than its planner holds", q, n),
                             CP_ERR_STATE));
            (m == 0 ? b->items_pop : b->items_mean)[q] = n * a.P;
            if (m == 0) {
                d.P = a.P;
                G[q] = a.G;
            }
        }
        off += p->N;
    }
    b->total = off;
    if (b->total > (1ll << 30)) return fail((set_error("the batch holds %lld candidates; at most 2^30", (long long)off), CP_ERR_ARG));
    b->order.resize(nq);
    for (int q = 0; q < nq; ++q) b->order[q] = q;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return G[x] > G[y]; });

    std::vector<int2> t_init, t_sample, t_cand, t_gather, t_mprep, t_mpart, t_mcomb;
    block_table(nq, [&](int q) { return (qh[q].D * qh[q].D + 255) / 256; }, t_init);
    block_table(nq, [&](int q) { return (qh[q].N + kBatchSampleCands - 1) / kBatchSampleCands; }, t_sample);
    block_table(nq, [&](int q) { return (qh[q].N + 255) / 256; }, t_cand);
    block_table(nq, [&](int q) { return (qh[q].nu + 7) / 8; }, t_gather);
    block_table(nq, [&](int q) { return (qh[q].nu * qh[q].D + 255) / 256; }, t_mprep);
    block_table(nq, [&](int q) {
        const int nt = (qh[q].D + 15) / 16;
        return nt * (nt + 1) / 2 * qh[q].n_chunks;
    }, t_mpart);
    block_table(nq, [&](int q) { return (qh[q].D * (qh[q].D + 1) / 2 + 31) / 32; }, t_mcomb);
    int64_t max_tiles = 0;
    for (int q = 0; q < nq; ++q) max_tiles += std::max(b->items_pop[q], b->items_mean[q]);   // tiles of >= 1 item
    b->tiles_cap = max_tiles;

    Layout L;
    const size_t o_in = L.take<double>(8 * (size_t)nq);
    const size_t o_out = L.take<double>((size_t)kOutStride * nq);
    const size_t o_q = L.take<BatchQueryDev>(nq);
    const size_t o_ep = L.take<BatchEvalDev>(nq);
    const size_t o_em = L.take<BatchEvalDev>(nq);
    const size_t o_ti = L.take<int2>(t_init.size());
    const size_t o_ts = L.take<int2>(t_sample.size());
    const size_t o_tc = L.take<int2>(t_cand.size());
    const size_t o_tg = L.take<int2>(t_gather.size());
    const size_t o_tq = L.take<int2>(t_mprep.size());
    const size_t o_tp = L.take<int2>(t_mpart.size());
    const size_t o_tm = L.take<int2>(t_mcomb.size());
    const size_t o_tilp = L.take<int4>((size_t)max_tiles);
    const size_t o_tilm = L.take<int4>((size_t)max_tiles);
    const size_t o_queue = L.take<int>((size_t)iters + 2);
    const size_t o_qid = L.take<uint16_t>((size_t)b->total);
    const size_t o_ka = L.take<unsigned long long>((size_t)b->total);
    const size_t o_kb = L.take<unsigned long long>((size_t)b->total);
    const size_t o_va = L.take<int>((size_t)b->total);
    const size_t o_vb = L.take<int>((size_t)b->total);
    const size_t o_h = L.take<int>(radix_hist_ints((int)b->total));
    if ((e = cudaMalloc((void **)&b->base, L.bytes)) != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(batch)"));
    char *base = b->base;
    b->d_in = (double *)(base + o_in);
    b->d_out = (double *)(base + o_out);
    b->qdev = (BatchQueryDev *)(base + o_q);
    b->ev_pop = (BatchEvalDev *)(base + o_ep);
    b->ev_mean = (BatchEvalDev *)(base + o_em);
    b->tab_init = (int2 *)(base + o_ti);
    b->tab_sample = (int2 *)(base + o_ts);
    b->tab_cand = (int2 *)(base + o_tc);
    b->tab_gather = (int2 *)(base + o_tg);
    b->tab_mprep = (int2 *)(base + o_tq);
    b->tab_mpart = (int2 *)(base + o_tp);
    b->tab_mcomb = (int2 *)(base + o_tm);
    b->tiles_pop = (int4 *)(base + o_tilp);
    b->tiles_mean = (int4 *)(base + o_tilm);
    b->queue = (int *)(base + o_queue);
    b->qid = (uint16_t *)(base + o_qid);
    b->key_a = (unsigned long long *)(base + o_ka);
    b->key_b = (unsigned long long *)(base + o_kb);
    b->val_a = (int *)(base + o_va);
    b->val_b = (int *)(base + o_vb);
    b->hist = (int *)(base + o_h);
    b->n_init = (int)t_init.size();
    b->n_sample = (int)t_sample.size();
    b->n_cand = (int)t_cand.size();
    b->n_gather = (int)t_gather.size();
    b->n_mprep = (int)t_mprep.size();
    b->n_mpart = (int)t_mpart.size();
    b->n_mcomb = (int)t_mcomb.size();
    std::vector<uint16_t> qid((size_t)b->total);
    for (int q = 0; q < nq; ++q)
        std::fill(qid.begin() + qh[q].cand_off, qid.begin() + qh[q].cand_off + qh[q].N, (uint16_t)q);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes == 0 ? cudaSuccess : cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->st);
    };
    if ((e = up(b->qdev, qh.data(), sizeof(BatchQueryDev) * nq)) != cudaSuccess ||
        (e = up(b->ev_pop, eh.data(), sizeof(BatchEvalDev) * nq)) != cudaSuccess ||
        (e = up(b->ev_mean, mh.data(), sizeof(BatchEvalDev) * nq)) != cudaSuccess ||
        (e = up(b->tab_init, t_init.data(), sizeof(int2) * t_init.size())) != cudaSuccess ||
        (e = up(b->tab_sample, t_sample.data(), sizeof(int2) * t_sample.size())) != cudaSuccess ||
        (e = up(b->tab_cand, t_cand.data(), sizeof(int2) * t_cand.size())) != cudaSuccess ||
        (e = up(b->tab_gather, t_gather.data(), sizeof(int2) * t_gather.size())) != cudaSuccess ||
        (e = up(b->tab_mprep, t_mprep.data(), sizeof(int2) * t_mprep.size())) != cudaSuccess ||
        (e = up(b->tab_mpart, t_mpart.data(), sizeof(int2) * t_mpart.size())) != cudaSuccess ||
        (e = up(b->tab_mcomb, t_mcomb.data(), sizeof(int2) * t_mcomb.size())) != cudaSuccess ||
        (e = up(b->qid, qid.data(), sizeof(uint16_t) * qid.size())) != cudaSuccess)
        return fail(cuda_fail(e, "cudaMemcpyAsync(batch tables)"));
    if ((rc = batch_upload_tiles(b)) != CP_OK) return fail(rc);   // synchronises
    if ((rc = batch_record_graph(b)) != CP_OK) return fail(rc);
    *out = b;
    return CP_OK;
}

int cp_batch_set_endpoints(cp_batch *b, int32_t q, const double h_q0[4], const double h_qd[4])
{
    if (!b || !h_q0 || !h_qd || q < 0 || q >= b->nq) return set_error("invalid arguments"), CP_ERR_ARG;
    for (int j = 0; j < 4; ++j)
        if (!is_finite(h_q0[j]) || !is_finite(h_qd[j])) return set_error("end points must be finite"), CP_ERR_ARG;
    CP_CUDA(cudaStreamSynchronize(b->st));   // the graph may be reading the inputs
    memcpy(b->h_in + 8 * q, h_q0, 4 * sizeof(double));
    memcpy(b->h_in + 8 * q + 4, h_qd, 4 * sizeof(double));
    return CP_OK;
}

int cp_batch_run(cp_batch *b, cp_batch_result *results)
{
    if (!b) return set_error("batch is NULL"), CP_ERR_ARG;
    NvtxRange range("craneplan:batch_run");
    CP_CUDA(cudaEventRecord(b->ev0, b->st));
    CP_CUDA(cudaGraphLaunch(b->exec, b->st));
    g_launches.fetch_add(b->kernel_nodes, std::memory_order_relaxed);
    CP_CUDA(cudaEventRecord(b->ev1, b->st));
    CP_CUDA(cudaStreamSynchronize(b->st));
    float run_ms = 0.f;
    CP_CUDA(cudaEventElapsedTime(&run_ms, b->ev0, b->ev1));
    b->last_run_ms = run_ms;
    int rc = CP_OK;
    for (int q = 0; q < b->nq; ++q) {
        const double *o = b->h_out + kOutStride * q;
        cp_planner *p = b->planners[q];
        // the query's planner now holds the state after `iters` iterations from the start
        p->iteration = b->iters;
        p->elites_ready = false;
        const double *in = b->h_in + 8 * q;
        p->q0f = make_float4((float)in[0], (float)in[1], (float)in[2], (float)in[3]);
        p->qdf = make_float4((float)in[4], (float)in[5], (float)in[6], (float)in[7]);
        if (results) {
            cp_batch_result &r = results[q];
            memset(&r, 0, sizeof r);
            r.stats.J = o[0];
            r.stats.Jp = o[1];
            r.stats.Jc = o[2];
            r.stats.Jl = o[3];
            r.stats.length = o[4];
            r.stats.n_flagged = (int32_t)o[5];
            r.stats.flag = r.stats.n_flagged > 0;
            r.stats.iterations = b->iters;
            r.stats.iteration = b->iters;
            r.stats.best_J = o[6];
            memcpy(r.ctrl, o + 8, sizeof(double) * 4 * (p->K + 8));
        }
        const uint32_t status = (uint32_t)o[7];
        if (status != 0 && rc == CP_OK) {
            if (status & DEV_ERR_NOT_PD) {
                set_error("query %d: the covariance is not positive definite", q);
                rc = CP_ERR_NUMERIC;
            } else {
                set_error("query %d: the obstacle index met more entries than its capacity, or the ranking "
                          "placed a foreign candidate in the query's range (status %u)", q, status);
                rc = CP_ERR_ARG;
            }
        }
    }
    return rc;
}

int cp_batch_set_shape(cp_batch *b, const cp_batch_shape *shape)
{
    if (!b || !shape) return set_error("invalid arguments"), CP_ERR_ARG;
    if (shape->threads != 128 && shape->threads != 256 && shape->threads != 512)
        return set_error("threads = %d is not 128, 256 or 512", shape->threads), CP_ERR_ARG;
    if (shape->ctas_per_sm < 0 || shape->ctas_per_sm > 32)
        return set_error("ctas_per_sm = %d outside 0..32", shape->ctas_per_sm), CP_ERR_ARG;
    if (shape->items_per_warp < 1 || shape->items_per_warp > 64)
        return set_error("items_per_warp = %d outside 1..64", shape->items_per_warp), CP_ERR_ARG;
    CP_CUDA(cudaStreamSynchronize(b->st));
    const cp_batch_shape old = b->shape;
    b->shape = *shape;
    int rc = batch_upload_tiles(b);
    if (rc == CP_OK) rc = batch_record_graph(b);
    if (rc != CP_OK) {
        b->shape = old;
        batch_upload_tiles(b);
        batch_record_graph(b);
    }
    return rc;
}

int cp_batch_evaluate(cp_batch *b, int32_t reps, double *ms)
{
    if (!b || !ms || reps < 1) return set_error("invalid arguments"), CP_ERR_ARG;
    int *counter = b->queue + b->iters + 1;
    double total = 0.0;
    for (int r = 0; r < reps; ++r) {
        CP_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), b->st));
        CP_CUDA(cudaEventRecord(b->ev0, b->st));
        int rc = launch_batch_eval_polar(b->mdev, b->ev_pop, b->tiles_pop, b->n_tiles_pop, counter, b->max_S,
                                         b->shape.threads, b->eval_blocks, b->st);
        if (rc != CP_OK) return rc;
        CP_CUDA(cudaEventRecord(b->ev1, b->st));
        CP_CUDA(cudaEventSynchronize(b->ev1));
        float t = 0.f;
        CP_CUDA(cudaEventElapsedTime(&t, b->ev0, b->ev1));
        total += t;
    }
    *ms = total / reps;
    return CP_OK;
}

int cp_batch_get_info(const cp_batch *b, cp_batch_info *out)
{
    if (!b || !out) return set_error("invalid arguments"), CP_ERR_ARG;
    out->kernel_nodes = b->kernel_nodes;
    out->eval_tiles = b->n_tiles_pop;
    out->eval_ctas = b->eval_blocks;
    out->eval_launches = b->iters + 1;
    out->candidates = b->total;
    out->last_run_ms = b->last_run_ms;
    return CP_OK;
}

cp_planner *cp_batch_planner(cp_batch *b, int32_t q)
{
    if (!b || q < 0 || q >= b->nq) return nullptr;
    return b->planners[q];
}

void cp_batch_destroy(cp_batch *b)
{
    if (!b) return;
    batch_free(b);
}

}  // extern "C"
