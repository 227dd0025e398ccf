// Algorithm 1 steps (3)-(6) (arXiv 2503.14160, Sec. 4.1):
//   k_weights        w_j = (ln(nu + 1/2) - ln j) / sum_k (ln(nu + 1/2) - ln k), FP64, once
//   k_rank_count     rank of every candidate = number of candidates before it in the order
//                    (J ascending, NaN as +inf, ties by index): an all-pairs count, split
//                    over the grid's y dimension and summed with integer atomics
//   k_scatter        elite list in rank order, the elite rows gathered contiguously
//   k_mean_partial / k_mean_combine   mu = sum_j w_j xi_(j), FP64, fixed order
//   k_cov_partial / k_cov_combine     C = sum_j w_j (xi_(j) - mu)(xi_(j) - mu)^T + eps I,
//                    FP64, about the new mean, 16x16 output tiles x chunks of elites,
//                    chunk partials summed in chunk order (deterministic)
#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr int kChunk = 128;         // elites per partial
constexpr int kRankThreads = 256;
constexpr int kRankSplit = 256;     // j-range per grid row of k_rank_count

// Order-preserving map of a double to uint64 (NaN -> +inf, -0 -> +0).
__device__ __forceinline__ unsigned long long order_key(double v)
{
    if (isnan(v)) v = __longlong_as_double(0x7FF0000000000000ll);
    if (v == 0.0) v = 0.0;
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_weights(int nu, double *w)
{
    __shared__ double part[1024];
    const double top = log((double)nu + 0.5);
    double acc = 0.0;
    for (int j = threadIdx.x; j < nu; j += blockDim.x) acc += top - log((double)(j + 1));
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    const double total = part[0];
    for (int j = threadIdx.x; j < nu; j += blockDim.x) w[j] = (top - log((double)(j + 1))) / total;
}

__global__ void __launch_bounds__(kRankThreads)
k_rank_count(const double *__restrict__ J, int N, int *rank)
{
    __shared__ unsigned long long s_key[kRankThreads];
    const int i = blockIdx.x * kRankThreads + threadIdx.x;
    const unsigned long long ki = i < N ? order_key(J[i]) : ~0ull;
    const int j_begin = blockIdx.y * kRankSplit;
    const int j_end = min(N, j_begin + kRankSplit);
    int cnt = 0;
    for (int base = j_begin; base < j_end; base += kRankThreads) {
        __syncthreads();
        const int j = base + threadIdx.x;
        s_key[threadIdx.x] = j < j_end ? order_key(J[j]) : ~0ull;
        __syncthreads();
        const int lim = min(kRankThreads, j_end - base);
        for (int t = 0; t < lim; ++t) {
            const unsigned long long kj = s_key[t];
            cnt += (kj < ki) || (kj == ki && base + t < i);
        }
    }
    if (i < N && cnt > 0) atomicAdd(rank + i, cnt);
}

// One warp per candidate: a candidate of rank r < nu writes its index to elite[r] and its
// row to elites[r][:]; rank 0 also records its cost.
__global__ void k_scatter(const int *__restrict__ rank, const double *__restrict__ J,
                          const float *__restrict__ xi, int N, int nu, int D, int *elite,
                          float *elites, double *best_J)
{
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int r = rank[warp];
    if (r >= nu) return;
    if (lane == 0) {
        elite[r] = warp;
        if (r == 0 && best_J != nullptr) *best_J = J[warp];
    }
    for (int c = lane; c < D; c += 32) elites[(size_t)r * D + c] = xi[(size_t)warp * D + c];
}

// Chunk p of kChunk elites: partial[p][c] = sum_{j in chunk} w_j elites[j][c].
__global__ void k_mean_partial(const float *__restrict__ elites, const double *__restrict__ w,
                               int nu, int D, double *partial)
{
    const int p = blockIdx.x, c = threadIdx.x;
    if (c >= D) return;
    const int j0 = p * kChunk, j1 = min(nu, j0 + kChunk);
    double acc = 0.0;
    for (int j = j0; j < j1; ++j) acc += w[j] * (double)elites[(size_t)j * D + c];
    partial[(size_t)p * D + c] = acc;
}

__global__ void k_mean_combine(const double *__restrict__ partial, int n_chunks, int D, double *mu)
{
    const int c = threadIdx.x;
    if (c >= D) return;
    double acc = 0.0;
    for (int p = 0; p < n_chunks; ++p) acc += partial[(size_t)p * D + c];
    mu[c] = acc;
}

// Block (tile t of the lower triangle of 16x16 tiles, chunk p): one output per thread.
__global__ void __launch_bounds__(256)
k_cov_partial(const float *__restrict__ elites, const double *__restrict__ w,
              const double *__restrict__ mu, int nu, int D, double *partial)
{
    __shared__ double yr[kChunk][16];
    __shared__ double yc[kChunk][16];
    __shared__ double ws[kChunk];
    // tile index -> (tile row tr >= tile col tc)
    int t = blockIdx.x, tr = 0;
    while (t > tr) {
        t -= tr + 1;
        ++tr;
    }
    const int tc = t;
    const int p = blockIdx.y;
    const int j0 = p * kChunk, cnt = min(nu - j0, kChunk);
    for (int idx = threadIdx.x; idx < cnt * 16; idx += blockDim.x) {
        const int j = idx >> 4, k = idx & 15;
        const int r = tr * 16 + k, c = tc * 16 + k;
        yr[j][k] = r < D ? (double)elites[(size_t)(j0 + j) * D + r] - mu[r] : 0.0;
        yc[j][k] = c < D ? (double)elites[(size_t)(j0 + j) * D + c] - mu[c] : 0.0;
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) ws[j] = w[j0 + j];
    __syncthreads();
    const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    double acc = 0.0;
    for (int j = 0; j < cnt; ++j) acc += ws[j] * yr[j][a] * yc[j][b];
    const int r = tr * 16 + a, c = tc * 16 + b;
    if (r < D && c < D) partial[((size_t)p * D + r) * D + c] = acc;
}

__global__ void k_cov_combine(const double *__restrict__ partial, int n_chunks, int D, double eps,
                              double *C)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= D * D) return;
    int r = idx / D, c = idx - r * D;
    const int lr = r >= c ? r : c, lc = r >= c ? c : r;     // lower-triangle source
    double acc = 0.0;
    for (int p = 0; p < n_chunks; ++p) acc += partial[((size_t)p * D + lr) * D + lc];
    if (r == c) acc += eps;
    C[idx] = acc;
}

}  // namespace

int update_chunk_size() { return kChunk; }

int launch_weights(int nu, double *w, cudaStream_t st)
{
    k_weights<<<1, 1024, 0, st>>>(nu, w);
    CP_LAUNCHED("k_weights");
    return CP_OK;
}

// rank must be zeroed by the caller; elite, elites and best_J are written.
int launch_rank(const double *J, int N, int nu, int *rank, cudaStream_t st)
{
    dim3 grid((N + kRankThreads - 1) / kRankThreads, (N + kRankSplit - 1) / kRankSplit);
    k_rank_count<<<grid, kRankThreads, 0, st>>>(J, N, rank);
    CP_LAUNCHED("k_rank_count");
    (void)nu;
    return CP_OK;
}

int launch_scatter(const int *rank, const double *J, const float *xi, int N, int nu, int D,
                   int *elite, float *elites, double *best_J, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = (N * 32 + threads - 1) / threads;
    k_scatter<<<blocks, threads, 0, st>>>(rank, J, xi, N, nu, D, elite, elites, best_J);
    CP_LAUNCHED("k_scatter");
    return CP_OK;
}

int launch_mean(const float *elites, const double *w, int nu, int D, double *partial,
                double *mu, cudaStream_t st)
{
    const int n_chunks = (nu + kChunk - 1) / kChunk;
    k_mean_partial<<<n_chunks, 128, 0, st>>>(elites, w, nu, D, partial);
    CP_LAUNCHED("k_mean_partial");
    k_mean_combine<<<1, 128, 0, st>>>(partial, n_chunks, D, mu);
    CP_LAUNCHED("k_mean_combine");
    return CP_OK;
}

int launch_cov(const float *elites, const double *w, const double *mu, int nu, int D,
               double eps, double *partial, double *C, cudaStream_t st)
{
    const int n_chunks = (nu + kChunk - 1) / kChunk;
    const int tiles = (D + 15) / 16;
    dim3 grid(tiles * (tiles + 1) / 2, n_chunks);
    k_cov_partial<<<grid, 256, 0, st>>>(elites, w, mu, nu, D, partial);
    CP_LAUNCHED("k_cov_partial");
    k_cov_combine<<<(D * D + 255) / 256, 256, 0, st>>>(partial, n_chunks, D, eps, C);
    CP_LAUNCHED("k_cov_combine");
    return CP_OK;
}

}  // namespace cp
