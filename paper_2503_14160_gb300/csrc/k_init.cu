// Set-up kernels: obstacle records for the evaluation kernel, the uniform cubic B-spline
// basis table, the initial sampling distribution (Sec. 4.1: linear interpolation with
// evenly spaced interior control points) and small format conversions.
#include "cp_internal.cuh"

namespace cp {
namespace {

__global__ void k_prepare_scene(const cp_cylinder *__restrict__ cyl, int n_cyl,
                                const cp_box *__restrict__ box, int n_box, float r_max,
                                float4 *cyl_filt, float4 *cyl_exact, float4 *box_c,
                                float4 *box_h)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cyl) {
        const cp_cylinder c = cyl[i];
        const double reach = c.radius + (double)r_max;
        const double W = c.cx * c.cx + c.cy * c.cy - reach * reach;
        // w: broad-phase reach, the filter's bound sqrt(reach^2 + margin) with slack
        const double cull = sqrt(reach * reach + 0.01) + 0.01;
        cyl_filt[i] = make_float4((float)c.cx, (float)c.cy, (float)W, (float)cull);
        // w: (R + r_max)^2 plus the filter margin, the bound of the filter in polar form
        cyl_exact[i] = make_float4((float)c.radius, (float)c.z_lo, (float)c.z_hi,
                                   (float)(reach * reach + (double)kFilterMargin));
    }
    if (i < n_box) {
        const cp_box b = box[i];
        // w: broad-phase reach, the half diagonal of the footprint plus a sphere, with slack
        const double hx = 0.5 * (b.hi[0] - b.lo[0]), hy = 0.5 * (b.hi[1] - b.lo[1]);
        const double cull = sqrt(hx * hx + hy * hy) + (double)r_max + 0.01;
        box_c[i] = make_float4((float)(0.5 * (b.lo[0] + b.hi[0])), (float)(0.5 * (b.lo[1] + b.hi[1])),
                               (float)(0.5 * (b.lo[2] + b.hi[2])), (float)cull);
        box_h[i] = make_float4((float)(0.5 * (b.hi[0] - b.lo[0])), (float)(0.5 * (b.hi[1] - b.lo[1])),
                               (float)(0.5 * (b.hi[2] - b.lo[2])), 0.f);
    }
}

// Group g of kGroup consecutive cylinders: a circle {gx, gy, 0, radius} that holds the reach
// disk of every member (centre plus its broad-phase reach w), so that an obstacle box test
// that passes for a member passes for its group. The centre is the middle of the members'
// bounding box; the radius is taken in FP64 and padded by 1e-5 m plus 1e-6 of the centre's
// distance from the origin, far above the FP32 rounding of the rotated coordinates.
__global__ void k_prepare_groups(const float4 *__restrict__ cyl_filt, int n_cyl, float4 *group)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups(n_cyl)) return;
    const int b = g * kGroup, e = min(n_cyl, b + kGroup);
    float x0 = cyl_filt[b].x, x1 = x0, y0 = cyl_filt[b].y, y1 = y0;
    for (int i = b + 1; i < e; ++i) {
        x0 = fminf(x0, cyl_filt[i].x);
        x1 = fmaxf(x1, cyl_filt[i].x);
        y0 = fminf(y0, cyl_filt[i].y);
        y1 = fmaxf(y1, cyl_filt[i].y);
    }
    const float gx = 0.5f * (x0 + x1), gy = 0.5f * (y0 + y1);
    double r = 0.0;
    for (int i = b; i < e; ++i) {
        const double dx = (double)cyl_filt[i].x - gx, dy = (double)cyl_filt[i].y - gy;
        r = fmax(r, sqrt(dx * dx + dy * dy) + (double)cyl_filt[i].w);
    }
    r += 1e-5 + 1e-6 * sqrt((double)gx * gx + (double)gy * gy);
    group[g] = make_float4(gx, gy, 0.f, (float)(r * (1.0 + 1e-6)));
}

// Uniform cubic B-spline basis on one span at u in [0, 1] (basis-matrix form):
//   b0 = (1-u)^3 / 6, b1 = (3u^3 - 6u^2 + 4) / 6, b2 = (-3u^3 + 3u^2 + 3u + 1) / 6, b3 = u^3 / 6
__device__ void cubic_basis(double u, double b[4])
{
    const double v = 1.0 - u;
    b[0] = v * v * v / 6.0;
    b[1] = (3.0 * u * u * u - 6.0 * u * u + 4.0) / 6.0;
    b[2] = (-3.0 * u * u * u + 3.0 * u * u + 3.0 * u + 1.0) / 6.0;
    b[3] = u * u * u / 6.0;
}

// basis[2(m-1)] = b(m/S), basis[2(m-1)+1] = b(m/S) - b((m-1)/S), m = 1..S, differences
// taken in FP64 before rounding so that increments keep their relative accuracy.
__global__ void k_basis_table(int S, float4 *basis)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (m > S) return;
    double b[4], b0[4];
    cubic_basis((double)m / (double)S, b);
    cubic_basis((double)(m - 1) / (double)S, b0);
    basis[2 * (m - 1)] = make_float4((float)b[0], (float)b[1], (float)b[2], (float)b[3]);
    basis[2 * (m - 1) + 1] = make_float4((float)(b[0] - b0[0]), (float)(b[1] - b0[1]),
                                         (float)(b[2] - b0[2]), (float)(b[3] - b0[3]));
}

// mu[4f + c] = q0[c] + (f+1)/(K+1) (qd[c] - q0[c]); C = diag((frac (q_max - q_min))^2).
__device__ __forceinline__ void init_entry(int idx, const double *q0, const double *qd, const double *q_min,
                                           const double *q_max, int K, double frac, double *mu, double *C)
{
    const int D = 4 * K;
    const int r = idx / D, c = idx - r * D;
    double v = 0.0;
    if (r == c) {
        const int j = r & 3;
        const double sd = frac * (q_max[j] - q_min[j]);
        v = sd * sd;
    }
    C[idx] = v;
    if (idx < D) {
        const int f = idx >> 2, j = idx & 3;
        mu[idx] = q0[j] + (double)(f + 1) / (double)(K + 1) * (qd[j] - q0[j]);
    }
}

__device__ __forceinline__ void ends_to_float(const double *q0, const double *qd, float4 *ends_f)
{
    ends_f[0] = make_float4((float)q0[0], (float)q0[1], (float)q0[2], (float)q0[3]);
    ends_f[1] = make_float4((float)qd[0], (float)qd[1], (float)qd[2], (float)qd[3]);
}

__global__ void k_init_distribution(const double *q0, const double *qd, const double *q_min,
                                    const double *q_max, int K, double frac, double *mu,
                                    double *C, float4 *ends_f)
{
    const int D = 4 * K;
    if (blockIdx.x == 0 && threadIdx.x == 0 && ends_f != nullptr) ends_to_float(q0, qd, ends_f);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < D * D;
         idx += gridDim.x * blockDim.x)
        init_entry(idx, q0, qd, q_min, q_max, K, frac, mu, C);
}

// The start of every query of a batch: end points from inputs[q][8] = {q0, qd} into the
// query's constants and float copy, its status cleared, and its initial distribution (block
// b of query q: entries 256 b .. of C).
__global__ void __launch_bounds__(256)
k_batch_init(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab, const double *__restrict__ inputs)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    const double *in = inputs + 8 * e.x;
    if (e.y == 0 && threadIdx.x < 8) q.consts[threadIdx.x] = in[threadIdx.x];
    if (e.y == 0 && threadIdx.x == 0) {
        ends_to_float(in, in + 4, q.ends);
        *q.status = 0u;
    }
    const int idx = e.y * 256 + (int)threadIdx.x;
    if (idx < q.D * q.D) init_entry(idx, in, in + 4, q.consts + 8, q.consts + 12, q.K, q.init_std_frac, q.mu, q.C);
}

__global__ void k_mean_to_candidate(const double *mu, int D, float *xi)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < D) xi[r] = (float)mu[r];
}

__device__ __forceinline__ double control_point(const double *q0, const double *qd, const double *mu, int K,
                                                int idx)
{
    const int point = idx >> 2, j = idx & 3;
    return point < 4 ? q0[j] : (point >= K + 4 ? qd[j] : mu[4 * (point - 4) + j]);
}

__global__ void k_control_points(const double *q0, const double *qd, const double *mu, int K,
                                 double *ctrl)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // 0 .. 4(K+8)-1
    if (idx >= 4 * (K + 8)) return;
    ctrl[idx] = control_point(q0, qd, mu, K, idx);
}

// One block per query. mean_candidate: the mean as an FP32 candidate. Otherwise the
// query's results into out[q][stride]: the mean's cost and terms[5], the best cost, the
// status word, then the control points of the mean path (also kept in the query's ctrl).
__global__ void __launch_bounds__(256)
k_batch_outputs(const BatchQueryDev *__restrict__ qd, int mean_candidate, double *out, int stride)
{
    const BatchQueryDev &q = qd[blockIdx.x];
    if (mean_candidate) {
        for (int r = threadIdx.x; r < q.D; r += blockDim.x) q.mean_xi[r] = (float)q.mu[r];
        return;
    }
    double *o = out + (size_t)stride * blockIdx.x;
    for (int idx = threadIdx.x; idx < 4 * (q.K + 8); idx += blockDim.x) {
        const double v = control_point(q.consts, q.consts + 4, q.mu, q.K, idx);
        q.ctrl[idx] = v;
        o[8 + idx] = v;
    }
    if (threadIdx.x == 0) {
        o[0] = *q.mean_J;
        for (int t = 0; t < 5; ++t) o[1 + t] = q.mean_terms[t];
        o[6] = *q.best;
        o[7] = (double)*q.status;
    }
}

}  // namespace

int launch_prepare_scene(const cp_cylinder *d_cyl_in, int n_cyl, const cp_box *d_box_in,
                         int n_box, float r_max, float4 *cyl_filt, float4 *cyl_exact, float4 *cyl_group,
                         float4 *box_c, float4 *box_h, cudaStream_t st)
{
    const int n = n_cyl > n_box ? n_cyl : n_box;
    if (n == 0) return CP_OK;
    k_prepare_scene<<<(n + 127) / 128, 128, 0, st>>>(d_cyl_in, n_cyl, d_box_in, n_box, r_max,
                                                     cyl_filt, cyl_exact, box_c, box_h);
    CP_LAUNCHED("k_prepare_scene");
    if (n_cyl > 0) {
        k_prepare_groups<<<(n_groups(n_cyl) + 127) / 128, 128, 0, st>>>(cyl_filt, n_cyl, cyl_group);
        CP_LAUNCHED("k_prepare_groups");
    }
    return CP_OK;
}

int launch_basis_table(int S, float4 *basis, cudaStream_t st)
{
    k_basis_table<<<(S + 127) / 128, 128, 0, st>>>(S, basis);
    CP_LAUNCHED("k_basis_table");
    return CP_OK;
}

int launch_init_distribution(const double *q0, const double *qd, const double *q_min,
                             const double *q_max, int K, double init_std_frac, double *mu,
                             double *C, float4 *ends_f, cudaStream_t st)
{
    const int D = 4 * K;
    const int threads = 256;
    const int blocks = (D * D + threads - 1) / threads;
    k_init_distribution<<<blocks, threads, 0, st>>>(q0, qd, q_min, q_max, K, init_std_frac, mu, C,
                                                    ends_f);
    CP_LAUNCHED("k_init_distribution");
    return CP_OK;
}

int launch_mean_to_candidate(const double *mu, int D, float *xi, cudaStream_t st)
{
    k_mean_to_candidate<<<1, 128, 0, st>>>(mu, D, xi);
    CP_LAUNCHED("k_mean_to_candidate");
    return CP_OK;
}

int launch_control_points(const double *q0, const double *qd, const double *mu, int K,
                          double *ctrl, cudaStream_t st)
{
    const int n = 4 * (K + 8);
    k_control_points<<<(n + 127) / 128, 128, 0, st>>>(q0, qd, mu, K, ctrl);
    CP_LAUNCHED("k_control_points");
    return CP_OK;
}

int launch_batch_init(const BatchQueryDev *qd, const int2 *tab, int blocks, const double *inputs, cudaStream_t st)
{
    k_batch_init<<<blocks, 256, 0, st>>>(qd, tab, inputs);
    CP_LAUNCHED("k_batch_init");
    return CP_OK;
}

int launch_batch_outputs(const BatchQueryDev *qd, int nq, bool mean_candidate, double *out, int out_stride,
                         cudaStream_t st)
{
    k_batch_outputs<<<nq, 256, 0, st>>>(qd, mean_candidate ? 1 : 0, out, out_stride);
    CP_LAUNCHED("k_batch_outputs");
    return CP_OK;
}

}  // namespace cp
