// Step (1) of Algorithm 1 drawn from the elites of the last update, with no factor
// (arXiv 2503.14160, Sec. 4.1). With C = sum_j w_j (x_(j) - mu)(x_(j) - mu)^T + eps I (steps
// (5)-(6), mu the new mean)
//     xi_i = mu + sigma (sum_j sqrt(w_j) (x_(j) - mu) g_ij + sqrt(eps) g'_i)
// is normal with mean mu and covariance sigma^2 C exactly, so the FP64 moments and the FP64
// Cholesky factor (whose dependent chains are slow on this part) leave the iteration; the
// draw is an FP32 product of N x nu normals and the nu x D scaled elite deviations.
//   k_elite_weights  sigma sqrt(w_j), once per planner
//   k_elite_mean     mu (FP64, about the best elite, fixed order) and Y[j][d] =
//                    sigma sqrt(w_j) (x_(j)d - mu_d) in FP32
//   k_sample_elites  partial products over a slice of the elites: a CTA takes 64 candidates
//                    x 64 coordinates, stages 32 elites of Y and the matching 32 x 64
//                    normals (Philox blocks generated in place) in shared memory, each
//                    thread accumulating 8 x 4 outputs
//   k_sample_reduce  xi = mu + sum of the slices (fixed order) + sigma sqrt(eps) g'
// Normals: candidate i at iteration t has the stream of Philox blocks (b, i, t, query), four
// standard normals per block (Box-Muller on words 0-1 and 2-3); g_ij is normal j, g'_id
// normal nu + d.
#include "cp_internal.cuh"
#include "philox.cuh"

namespace cp {
namespace {

constexpr int kTileC = 64;     // candidates per CTA tile
constexpr int kTileD = 64;     // coordinates per CTA tile
constexpr int kChunkE = 32;    // elites per staged chunk
constexpr int kSEThreads = 128;   // 8 candidates x 4 coordinates a thread

// Normal number j of candidate i (a block of four per Philox call).
__device__ __forceinline__ float normal_at(uint32_t i, uint32_t j, uint32_t iter, uint32_t query, uint32_t k0,
                                           uint32_t k1)
{
    const uint4 x = philox4x32_10(make_uint4(j >> 2, i, iter, query), k0, k1);
    float z0, z1;
    if ((j & 2) == 0)
        box_muller(x.x, x.y, z0, z1);
    else
        box_muller(x.z, x.w, z0, z1);
    return (j & 1) ? z1 : z0;
}

// One block per coordinate d: mu_d = x_(1)d + sum_j w_j (x_(j)d - x_(1)d), then the column d
// of Y. The sum runs over the elites in a fixed partition (thread t takes j = t, t + 256, ...)
// and a fixed reduction tree.
__global__ void k_elite_weights(const double *__restrict__ w, int nu, double sigma, double *sw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nu) sw[k] = sigma * sqrt(w[k]);
}

__global__ void __launch_bounds__(256)
k_elite_mean(const float *__restrict__ elites, const double *__restrict__ w, const double *__restrict__ sw,
             int nu, int D, double *mu, float *mu_f, float *Y)
{
    __shared__ double s_part[8];
    __shared__ double s_mu;
    const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const double x1 = (double)elites[d];
    double a0 = 0.0, a1 = 0.0;
    int j = tid;
    for (; j + 256 < nu; j += 512) {
        a0 = fma(w[j], (double)elites[(size_t)j * D + d] - x1, a0);
        a1 = fma(w[j + 256], (double)elites[(size_t)(j + 256) * D + d] - x1, a1);
    }
    if (j < nu) a0 = fma(w[j], (double)elites[(size_t)j * D + d] - x1, a0);
    double v = a0 + a1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_part[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int k = 0; k < 8; ++k) sum += s_part[k];
        s_mu = x1 + sum;
        mu[d] = s_mu;
        mu_f[d] = (float)s_mu;
    }
    __syncthreads();
    const double m = s_mu;
    for (int k = tid; k < nu; k += 256)
        Y[(size_t)k * D + d] = (float)(sw[k] * ((double)elites[(size_t)k * D + d] - m));
}

// Slice s of the elites [j_begin, j_end) for the tile (candidates c0.., coordinates d0..):
// P[s][i][d] = sum_{j in slice} g_ij Y[j][d].
__global__ void __launch_bounds__(kSEThreads)
k_sample_elites(const float *__restrict__ Y, int N, int D, int nu, int per_slice, uint32_t k0, uint32_t k1,
                uint32_t iter, uint32_t query, float *P)
{
    __shared__ __align__(16) float s_g[kChunkE][kTileC];   // normals [elite][candidate]
    __shared__ __align__(16) float s_y[kChunkE][kTileD];   // Y chunk [elite][coordinate]
    const int c0 = blockIdx.x * kTileC, d0 = blockIdx.y * kTileD, slice = blockIdx.z;
    const int j_begin = slice * per_slice, j_end = min(nu, j_begin + per_slice);
    const int tid = threadIdx.x, tc = tid & 7, td = tid >> 3;   // 8 candidates x 4 coordinates
    float acc[8][4] = {};
    for (int j0 = j_begin; j0 < j_end; j0 += kChunkE) {
        __syncthreads();
        // normals: 64 candidates x 8 Philox blocks of 4
        for (int e = tid; e < kTileC * (kChunkE / 4); e += kSEThreads) {
            const int c = e & (kTileC - 1), b = e / kTileC;
            const int i = c0 + c, jj = j0 + 4 * b;
            float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
            if (i < N) {
                const uint4 x = philox4x32_10(make_uint4((uint32_t)(jj >> 2), (uint32_t)i, iter, query), k0, k1);
                box_muller(x.x, x.y, z0, z1);
                box_muller(x.z, x.w, z2, z3);
            }
            s_g[4 * b + 0][c] = z0;
            s_g[4 * b + 1][c] = z1;
            s_g[4 * b + 2][c] = z2;
            s_g[4 * b + 3][c] = z3;
        }
        // scaled deviations: rows j0.. of Y for the tile's coordinates (zero past nu or D)
        for (int e = tid; e < kChunkE * kTileD; e += kSEThreads) {
            const int k = e / kTileD, d = e - k * kTileD;
            const int dd = d0 + d, j = j0 + k;
            s_y[k][d] = dd < D && j < j_end ? Y[(size_t)j * D + dd] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kChunkE; ++k) {
            const float4 g0 = *reinterpret_cast<const float4 *>(&s_g[k][8 * tc]);
            const float4 g1 = *reinterpret_cast<const float4 *>(&s_g[k][8 * tc + 4]);
            const float4 y = *reinterpret_cast<const float4 *>(&s_y[k][4 * td]);
            const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(gv[a], yv[b], acc[a][b]);
        }
    }
    float *out = P + (size_t)slice * N * D;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int i = c0 + 8 * tc + a;
        if (i >= N) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int d = d0 + 4 * td + b;
            if (d < D) out[(size_t)i * D + d] = acc[a][b];
        }
    }
}

// xi[i][d] = mu_d + sum_s P[s][i][d] (slices in order) + sigma sqrt(eps) g'_id.
__global__ void k_sample_reduce(const float *__restrict__ P, int slices, const float *__restrict__ mu_f, int N,
                                int D, int nu, float eps_scale, uint32_t k0, uint32_t k1, uint32_t iter,
                                uint32_t query, float *xi)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * D) return;
    const int i = (int)(e / D), d = (int)(e - (int64_t)i * D);
    float v = 0.f;
    for (int s = 0; s < slices; ++s) v += P[(size_t)s * N * D + e];
    const float g = normal_at((uint32_t)i, (uint32_t)(nu + d), iter, query, k0, k1);
    xi[e] = mu_f[d] + fmaf(eps_scale, g, v);
}

}  // namespace

// Slices of the elites for N candidates and D coordinates: about twelve CTAs per SM, so
// that the last wave is a small part of the launch (at most 32 slices, at least one chunk
// each).
int elite_slices(int N, int D, int nu, int num_sms)
{
    const int tiles = ((N + kTileC - 1) / kTileC) * ((D + kTileD - 1) / kTileD);
    int s = (12 * num_sms + tiles - 1) / tiles;
    const int max_s = (nu + kChunkE - 1) / kChunkE;
    if (s > max_s) s = max_s;
    if (s > 32) s = 32;
    return s < 1 ? 1 : s;
}

int launch_elite_weights(const double *w, int nu, double sigma, double *sw, cudaStream_t st)
{
    k_elite_weights<<<(nu + 255) / 256, 256, 0, st>>>(w, nu, sigma, sw);
    CP_LAUNCHED("k_elite_weights");
    return CP_OK;
}

int launch_elite_mean(const float *elites, const double *w, const double *sw, int nu, int D, double *mu, float *mu_f,
                      float *Y, cudaStream_t st)
{
    k_elite_mean<<<D, 256, 0, st>>>(elites, w, sw, nu, D, mu, mu_f, Y);
    CP_LAUNCHED("k_elite_mean");
    return CP_OK;
}

int launch_sample_elites(const float *Y, const float *mu_f, int N, int K, int nu, int slices, double sigma,
                         double eps, uint64_t seed, uint32_t iter, uint32_t query, float *P, float *xi,
                         cudaStream_t st)
{
    const int D = 4 * K;
    int per = (nu + slices - 1) / slices;
    per = (per + kChunkE - 1) / kChunkE * kChunkE;   // slices start on a chunk (and Philox block) boundary
    const int used = (nu + per - 1) / per;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    dim3 grid((N + kTileC - 1) / kTileC, (D + kTileD - 1) / kTileD, used);
    k_sample_elites<<<grid, kSEThreads, 0, st>>>(Y, N, D, nu, per, k0, k1, iter, query, P);
    CP_LAUNCHED("k_sample_elites");
    const int64_t total = (int64_t)N * D;
    k_sample_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, used, mu_f, N, D, nu,
                                                                     (float)(sigma * sqrt(eps)), k0, k1, iter,
                                                                     query, xi);
    CP_LAUNCHED("k_sample_reduce");
    return CP_OK;
}

}  // namespace cp
