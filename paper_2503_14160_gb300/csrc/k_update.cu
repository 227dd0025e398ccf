// Algorithm 1 steps (3)-(6) (arXiv 2503.14160, Sec. 4.1):
//   k_weights        w_j = (ln(nu + 1/2) - ln j) / sum_k (ln(nu + 1/2) - ln k), FP64, once
//   k_rank_count     rank of every candidate = number of candidates before it in the order
//                    (J ascending, NaN as +inf, ties by index): an all-pairs count, split
//                    over the grid's y dimension and summed with integer atomics
//   k_scatter        elite list in rank order, the elite rows gathered contiguously; the
//                    rank counters are cleared for the next ranking
//   k_radix_*        for large N instead: a stable LSD radix sort of the keys (8 x 8 bits)
//   k_moments_partial / k_moments_combine   mu = sum_j w_j xi_(j) and
//                    C = sum_j w_j (xi_(j) - mu)(xi_(j) - mu)^T + eps I (about the new
//                    mean) in one FP64 pass about the best elite, 16x16 output tiles x
//                    chunks of elites, chunk partials summed in a fixed order (deterministic)
#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr int kChunk = 32;          // elites staged at a time
constexpr int kMaxChunks = 512;     // bound on the partial buffers
constexpr int kRankThreads = 256;
constexpr int kRankPer = 128;       // j-range per grid row of k_rank_count

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

// Block (x, y): candidates i of block x against the candidates j of the y-th range of
// kRankPer. Candidate j precedes i when k_j < k_i, or k_j == k_i and j < i; for j < i that
// is k_j < k_i + 1 (the key of a real cost stays below 2^64 - 1), for j >= i k_j < k_i, so
// each comparison is one 64-bit compare against a threshold that changes once per range.
__global__ void __launch_bounds__(kRankThreads)
k_rank_count(const double *__restrict__ J, int N, int *rank)
{
    __shared__ unsigned long long s_key[kRankPer];
    const int i = blockIdx.x * kRankThreads + threadIdx.x;
    const unsigned long long ki = i < N ? order_key(J[i]) : 0ull;
    const int j0 = blockIdx.y * kRankPer;
    const int len = min(kRankPer, N - j0);
    for (int t = threadIdx.x; t < len; t += kRankThreads) s_key[t] = order_key(J[j0 + t]);
    __syncthreads();
    const int split = min(max(i - j0, 0), len);   // j0 + split: the first j >= i
    const unsigned long long ki1 = ki + 1;
    int cnt = 0;
    for (int t = 0; t < split; ++t) cnt += s_key[t] < ki1;
#pragma unroll 4
    for (int t = split; t < len; ++t) cnt += s_key[t] < ki;
    if (i < N && cnt > 0) atomicAdd(rank + i, cnt);
}

// One warp per candidate: a candidate of rank r < nu writes its index to elite[r] and its
// row to elites[r][:]; rank 0 also records its cost. The rank counter goes back to zero for
// the next ranking.
__global__ void k_scatter(int *__restrict__ rank, const double *__restrict__ J,
                          const float *__restrict__ xi, int N, int nu, int D, int *elite,
                          float *elites, double *best_J)
{
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int r = rank[warp];
    __syncwarp();
    if (lane == 0) rank[warp] = 0;
    if (r >= nu) return;
    if (lane == 0) {
        elite[r] = warp;
        if (r == 0 && best_J != nullptr) *best_J = J[warp];
    }
    for (int c = lane; c < D; c += 32) elites[(size_t)r * D + c] = xi[(size_t)warp * D + c];
}

// Steps (5)-(6) in one pass over the elites, about the best elite m0 = xi_(1): with
// y_j = xi_(j) - m0 (exact in FP64 for the FP32 rows), S1 = sum_j w_j y_j and
// S2 = sum_j w_j y_j y_j^T give mu = m0 + S1 and, since the weights sum to one,
// C = sum_j w_j (xi_(j) - mu)(xi_(j) - mu)^T + eps I = S2 - S1 S1^T + eps I. The best elite
// lies within the spread of the elites, so S1 S1^T is of the size of C and the subtraction
// loses no more than a few FP64 roundings.
//
// Block (tile t of the lower triangle of 16x16 tiles, chunk p of kChunk-row groups): one
// S2 entry per thread, and S1 of the tile's rows on diagonal tiles. Partials are stored
// chunk-major ([chunk][row][col] and [chunk][row]): a tile's writes are rows of 16
// consecutive entries, and the combine (one thread per entry) reads one chunk of
// consecutive entries per load.
__device__ __forceinline__ void moments_partial_body(const double *__restrict__ Y, const double *__restrict__ WY,
                                                    int nu, int D, int per, int n_chunks, double *s2p, double *s1p,
                                                    int t, int p)
{
    __shared__ double wyr[kChunk][17];
    __shared__ double yc[kChunk][17];
    int tr = 0;   // tile index -> (tile row tr >= tile col tc)
    while (t > tr) {
        t -= tr + 1;
        ++tr;
    }
    const int tc = t;
    const bool diag = tr == tc;
    // the thread's entry (a, b) of the tile: all 256 of an off-diagonal tile; the 136 with
    // b <= a of a diagonal tile (warps 5-7 idle there)
    int a = threadIdx.x >> 4, b = threadIdx.x & 15;
    const bool active = !diag || threadIdx.x < 136;
    if (diag && active) tri_index(threadIdx.x, a, b);
    const int j_end = min(nu, (p + 1) * per);
    // four interleaved accumulators: a dependent FP64 FMA waits tens of cycles, so one
    // running sum would leave the FP64 pipe idle between its steps
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, acc1 = 0.0;
    for (int j0 = p * per; j0 < j_end; j0 += kChunk) {
        const int cnt = min(j_end - j0, kChunk);
        __syncthreads();
        for (int idx = threadIdx.x; idx < cnt * 16; idx += blockDim.x) {
            const int j = idx >> 4, k = idx & 15;
            const int r = tr * 16 + k, c = tc * 16 + k;
            const size_t row = (size_t)(j0 + j) * D;
            wyr[j][k] = r < D ? WY[row + r] : 0.0;
            yc[j][k] = c < D ? Y[row + c] : 0.0;
        }
        __syncthreads();
        if (active) {
            int j = 0;
            for (; j + 3 < cnt; j += 4) {
                a0 = fma(wyr[j][a], yc[j][b], a0);
                a1 = fma(wyr[j + 1][a], yc[j + 1][b], a1);
                a2 = fma(wyr[j + 2][a], yc[j + 2][b], a2);
                a3 = fma(wyr[j + 3][a], yc[j + 3][b], a3);
            }
            for (; j < cnt; ++j) a0 = fma(wyr[j][a], yc[j][b], a0);
            if (diag && b == 0)
                for (int j = 0; j < cnt; ++j) acc1 += wyr[j][a];
        }
    }
    const int r = tr * 16 + a, c = tc * 16 + b;
    if (active && r < D && c <= r) s2p[(size_t)p * D * D + (size_t)r * D + c] = (a0 + a1) + (a2 + a3);
    if (active && diag && b == 0 && r < D) s1p[(size_t)p * D + r] = acc1;
}

// The elites' deviations from the best elite in FP64, y_j = x_(j) - x_(1) (exact: both are
// FP32), and w_j y_j, once per update for every tile of the moments.
__device__ __forceinline__ void moments_prep_body(const float *__restrict__ elites, const double *__restrict__ w,
                                                 int nu, int D, double *Y, double *WY, int idx)
{
    if (idx >= nu * D) return;
    const int j = idx / D, r = idx - j * D;
    const double y = (double)elites[idx] - (double)elites[r];
    Y[idx] = y;
    WY[idx] = w[j] * y;
}

__global__ void k_moments_prep(const float *__restrict__ elites, const double *__restrict__ w, int nu, int D,
                               double *Y, double *WY)
{
    moments_prep_body(elites, w, nu, D, Y, WY, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256)
k_moments_partial(const double *__restrict__ Y, const double *__restrict__ WY, int nu, int D,
                  int per, int n_chunks, double *s2p, double *s1p)
{
    moments_partial_body(Y, WY, nu, D, per, n_chunks, s2p, s1p, blockIdx.x, blockIdx.y);
}

// Every query's deviations in one launch (block b of query q: entries 256 b ..).
__global__ void __launch_bounds__(256)
k_batch_moments_prep(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    moments_prep_body(q.elites, q.w, q.nu, q.D, q.mom_y, q.mom_y + (size_t)q.nu * q.D, e.y * 256 + (int)threadIdx.x);
}

// Every query's partials in one launch: block b of query q is tile b % tiles, chunk b / tiles
// of that query (tiles = its lower-triangle tile count).
__global__ void __launch_bounds__(256)
k_batch_moments_partial(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    const int nt = (q.D + 15) / 16, tiles = nt * (nt + 1) / 2;
    moments_partial_body(q.mom_y, q.mom_y + (size_t)q.nu * q.D, q.nu, q.D, q.per, q.n_chunks, q.s2p, q.s1p,
                         e.y % tiles, e.y / tiles);
}

// Sum of the n values v[0], v[stride], ..., v[(n - 1) stride] in a fixed order: 32 running
// sums, sum l taking the terms q = l, l + 32, l + 64, ... in turn, then pairwise at distances
// 16, 8, 4, 2, 1 (sum l of the first 16 plus sum l + 16, and so on down to sums 0 and 1).
// It is the order of a warp's lane-strided sums and xor-shuffle tree. Here G aligned lanes
// (sub = 0 .. G-1) share one sum: lane sub keeps the running sums sub P .. sub P + P - 1
// (P = 32 / G), the pairings across lanes go through xor shuffles within the group and the
// rest inside the lane, so the additions are the same and so are the bits. Every lane of the
// warp calls it (full-warp shuffles); the total is returned on every lane of the group.
template <int G>
__device__ __forceinline__ double tree_sum(const double *__restrict__ v, int n, size_t stride, int sub)
{
    constexpr int P = 32 / G;
    double s[P];
#pragma unroll
    for (int i = 0; i < P; ++i) s[i] = 0.0;
    const int l0 = sub * P;
    for (int q0 = 0; q0 < n; q0 += 32) {
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (q0 + l0 + i < n) s[i] += v[(size_t)(q0 + l0 + i) * stride];
    }
#pragma unroll
    for (int off = 16; off >= P; off >>= 1) {   // partner lane sub + off / P holds sums l + off
#pragma unroll
        for (int i = 0; i < P; ++i) s[i] += __shfl_xor_sync(0xffffffffu, s[i], off / P);
    }
#pragma unroll
    for (int off = P / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < off; ++i) s[i] += s[i + off];
    }
    return G > 1 ? __shfl_sync(0xffffffffu, s[0], (int)(threadIdx.x & 31) & ~(G - 1)) : s[0];
}

// Lanes per sum of the moment combine: four lanes, eight running sums each.
constexpr int kSumLanes = 4;

// S1 of rows 0 .. r_last into shared memory (one thread per row), for the entries of a block.
__device__ __forceinline__ void stage_s1(const double *__restrict__ s1p, int n_chunks, int D, int r_last,
                                         double *s_s1)
{
    for (int r = threadIdx.x; r <= r_last && r < D; r += blockDim.x) s_s1[r] = tree_sum<1>(s1p + r, n_chunks, D, 0);
    __syncthreads();
}

// Row of the last lower-triangle entry a block of blockDim.x threads starting at entry e0 holds.
__device__ __forceinline__ int last_row(int e0, int D)
{
    int r, c;
    tri_index(min(e0 + (int)blockDim.x, D * (D + 1) / 2) - 1, r, c);
    return r;
}

// S1 of row r (its chunk partials summed in the fixed order above, kSumLanes lanes per row),
// stored after the chunk partials of s1p, and mu_r = m0_r + S1_r. Called by whole warps.
__device__ __forceinline__ void moments_s1_body(double *s1p, int n_chunks, int D, const float *__restrict__ elites,
                                               double *mu, int r, int sub)
{
    const double s = tree_sum<kSumLanes>(s1p + min(r, D - 1), n_chunks, D, sub);
    if (r < D && sub == 0) {
        s1p[(size_t)n_chunks * D + r] = s;
        mu[r] = (double)elites[r] + s;
    }
}

// Lower-triangle entry e (r >= c), kSumLanes lanes per entry:
// C[r][c] = C[c][r] = S2 - S1_r S1_c + eps [r = c], with S1 from moments_s1_body. Called by
// whole warps.
__device__ __forceinline__ void moments_combine_body(const double *__restrict__ s2p, const double *__restrict__ s1,
                                                    int n_chunks, int D, double eps, double *C, int e, int sub)
{
    const int entries = D * (D + 1) / 2;
    int r, c;
    tri_index(min(e, entries - 1), r, c);
    const double s2 = tree_sum<kSumLanes>(s2p + (size_t)r * D + c, n_chunks, (size_t)D * D, sub);
    if (e >= entries || sub != 0) return;
    double v = fma(-s1[r], s1[c], s2);
    if (r == c) v += eps;
    C[(size_t)r * D + c] = v;
    C[(size_t)c * D + r] = v;
}

// Blocks of 128 threads: 32 rows (entries) per block, kSumLanes lanes each.
__global__ void __launch_bounds__(128)
k_moments_s1(double *s1p, int n_chunks, int D, const float *__restrict__ elites, double *mu)
{
    const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    moments_s1_body(s1p, n_chunks, D, elites, mu, g / kSumLanes, g % kSumLanes);
}

__global__ void __launch_bounds__(128)
k_moments_combine(const double *__restrict__ s2p, const double *__restrict__ s1, int n_chunks, int D, double eps,
                  double *C)
{
    const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    moments_combine_body(s2p, s1, n_chunks, D, eps, C, g / kSumLanes, g % kSumLanes);
}

// Block (x, q): S1 and the mean of rows 32 x .. 32 x + 31 of query q.
__global__ void __launch_bounds__(128)
k_batch_moments_s1(const BatchQueryDev *__restrict__ qd)
{
    const BatchQueryDev &q = qd[blockIdx.y];
    const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    moments_s1_body(q.s1p, q.n_chunks, q.D, q.elites, q.mu, g / kSumLanes, g % kSumLanes);
}

// Block b of query q combines the entries 32 b .. 32 b + 31 of that query.
__global__ void __launch_bounds__(128)
k_batch_moments_combine(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    moments_combine_body(q.s2p, q.s1p + (size_t)q.n_chunks * q.D, q.n_chunks, q.D, q.eps, q.C,
                         e.y * 32 + (int)threadIdx.x / kSumLanes, (int)threadIdx.x % kSumLanes);
}

// ---------------------------------------------------------------- LSD radix sort (large N)
// Stable ascending sort of (key, index) by the order-preserving 64-bit keys: eight passes of
// 8-bit digits; tiles of kRadixTile consecutive elements; per pass a tile histogram, an
// exclusive scan in (digit, tile) order, and a stable scatter (ranks inside a warp from
// __match_any_sync, across warps and passes from per-digit prefixes).
constexpr int kRadixTile = 1024;
constexpr int kRadixThreads = 256;
constexpr int kRadixTotals = 10 * 256;   // per-digit totals of up to ten passes

__global__ void k_radix_init(const double *__restrict__ J, int N, unsigned long long *key, int *val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        key[i] = order_key(J[i]);
        val[i] = i;
    }
}

// The digit of a pass: 8 bits of the key, or (kByQuery) 8 bits of the query of the element's
// value (qid[value]), for the last passes of the batched ranking.
template <bool kByQuery>
__device__ __forceinline__ int radix_digit(unsigned long long k, int v, int shift, const uint16_t *__restrict__ qid)
{
    if (kByQuery) return (int)((qid[v] >> shift) & 255u);
    return (int)((k >> shift) & 255ull);
}

// Tile histograms of one pass, digit-major (hist[d * tiles + tile]), and each digit's count
// over all tiles added into totals[d] (zero before the pass).
template <bool kByQuery = false>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const unsigned long long *__restrict__ key, int N, int shift, int tiles, int *hist, int *totals,
             const int *__restrict__ val = nullptr, const uint16_t *__restrict__ qid = nullptr)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int b = blockIdx.x * kRadixTile, e = min(N, b + kRadixTile);
    for (int i = b + threadIdx.x; i < e; i += kRadixThreads)
        atomicAdd(&h[radix_digit<kByQuery>(kByQuery ? 0ull : key[i], kByQuery ? val[i] : 0, shift, qid)], 1);
    __syncthreads();
    hist[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];   // digit-major
    if (h[threadIdx.x] != 0) atomicAdd(totals + threadIdx.x, h[threadIdx.x]);
}

// Exclusive scan of the digit-major histogram in place, one block per digit d: the element
// (d, tile) becomes the count of all digits below d (from the per-digit totals) plus the
// counts of digit d in the tiles before `tile`, 256 tiles at a time (block scan by warp
// shuffles, the running total carried to the next 256). Integer sums: the same offsets as
// any other order of the scan.
__global__ void __launch_bounds__(256) k_radix_scan(int *hist, int tiles, const int *__restrict__ totals)
{
    __shared__ int warp_tot[8];
    __shared__ int carry_s;
    const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int below = __reduce_add_sync(0xffffffffu, t < d ? totals[t] : 0);
    if (lane == 0) warp_tot[warp] = below;
    __syncthreads();
    if (t == 0) {
        int c = 0;
        for (int w = 0; w < 8; ++w) c += warp_tot[w];
        carry_s = c;
    }
    int *row = hist + (size_t)d * tiles;
    for (int base = 0; base < tiles; base += 256) {
        __syncthreads();   // carry_s written, warp_tot free
        const int i = base + t;
        const int c = i < tiles ? row[i] : 0;
        int x = c;         // inclusive scan within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        int pre = carry_s;
        for (int w = 0; w < warp; ++w) pre += warp_tot[w];
        if (i < tiles) row[i] = pre + x - c;
        __syncthreads();   // every thread has read carry_s
        if (t == 255) carry_s = pre + x;
    }
}

template <bool kByQuery = false>
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const unsigned long long *__restrict__ key_in, const int *__restrict__ val_in, int N,
                int shift, int tiles, const int *__restrict__ offsets, unsigned long long *key_out,
                int *val_out, const uint16_t *__restrict__ qid = nullptr)
{
    __shared__ int run[256];            // elements of each digit placed by earlier passes
    __shared__ int wcount[8][256];      // per-warp digit counts of the current pass
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    run[threadIdx.x] = offsets[threadIdx.x * tiles + blockIdx.x];
    const int b = blockIdx.x * kRadixTile, e = min(N, b + kRadixTile);
    const unsigned lt = (1u << lane) - 1u;
    for (int r = b; r < e; r += kRadixThreads) {
        for (int w = 0; w < 8; ++w) wcount[w][threadIdx.x] = 0;
        __syncthreads();
        const int i = r + threadIdx.x;
        const bool valid = i < e;
        unsigned long long k = 0;
        int v = 0, d = 256 + lane;      // invalid lanes get digits no valid lane has
        if (valid) {
            k = key_in[i];
            v = val_in[i];
            d = radix_digit<kByQuery>(k, v, shift, qid);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int in_warp = __popc(peers & lt);
        if (valid && in_warp == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        int before = 0;                 // same digit in earlier warps of this pass
        if (valid)
            for (int w = 0; w < warp; ++w) before += wcount[w][d];
        if (valid) {
            const int pos = run[d] + before + in_warp;
            key_out[pos] = k;
            val_out[pos] = v;
        }
        __syncthreads();
        int total = 0;
        for (int w = 0; w < 8; ++w) total += wcount[w][threadIdx.x];
        run[threadIdx.x] += total;
        __syncthreads();
    }
}

// Elite list and rows from the sorted indices; rank 0 also records its cost.
__device__ __forceinline__ void gather_body(const int *__restrict__ sorted, int base, const double *__restrict__ J,
                                            const float *__restrict__ xi, int nu, int D, int *elite, float *elites,
                                            double *best_J, int r, int n_valid = 0x7FFFFFFF,
                                            uint32_t *status = nullptr)
{
    const int lane = threadIdx.x & 31;
    if (r >= nu) return;
    const int i = sorted[r] - base;
    if (i < 0 || i >= n_valid) {   // not one of this query's candidates: report, touch nothing
        if (lane == 0 && status != nullptr) atomicOr(status, DEV_ERR_OVERFLOW);
        return;
    }
    if (lane == 0) {
        elite[r] = i;
        if (r == 0 && best_J != nullptr) *best_J = J[i];
    }
    for (int c = lane; c < D; c += 32) elites[(size_t)r * D + c] = xi[(size_t)i * D + c];
}

__global__ void k_gather_elites(const int *__restrict__ sorted, const double *__restrict__ J,
                                const float *__restrict__ xi, int nu, int D, int *elite,
                                float *elites, double *best_J)
{
    gather_body(sorted, 0, J, xi, nu, D, elite, elites, best_J, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5));
}

// The batched ranking: key and value of every query's candidates at the query's offset in
// the concatenated arrays (value = that position), and the query of each position.
__global__ void k_batch_radix_init(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab,
                                   unsigned long long *key, int *val)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    const int i = e.y * 256 + (int)threadIdx.x;
    if (i < q.N) {
        key[q.cand_off + i] = order_key(q.J[i]);
        val[q.cand_off + i] = q.cand_off + i;
    }
}

// Elites of every query from its sorted range (block b of query q: ranks 8 b .. 8 b + 7).
__global__ void __launch_bounds__(256)
k_batch_gather(const BatchQueryDev *__restrict__ qd, const int2 *__restrict__ tab, const int *__restrict__ sorted)
{
    const int2 e = tab[blockIdx.x];
    const BatchQueryDev &q = qd[e.x];
    gather_body(sorted + q.cand_off, q.cand_off, q.J, q.xi, q.nu, q.D, q.elite, q.elites, q.best,
                e.y * 8 + (int)(threadIdx.x >> 5), q.N, q.status);
}

// ---------------------------------------------------------------- CMA-ES update rule
// The update of the CMA-ES tutorial (Hansen 2016) in place of steps (5)-(6), from the same
// per-chunk moments about the best elite x_(1): S1 = sum_j w_j y_j, S2 = sum_j w_j y_j y_j^T,
// y_j = x_(j) - x_(1). State cma[4] = {sigma, sigma before the update, h_sigma, |p_sigma|}.
constexpr int kCmaThreads = 4 * CP_MAX_WAYPOINTS;   // one thread per coordinate, D <= 128

__global__ void k_cma_reset(double sigma0, int D, double *cma, double *p_sigma, double *p_c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < D) {
        p_sigma[i] = 0.0;
        p_c[i] = 0.0;
    }
    if (i == 0) {
        cma[0] = sigma0;
        cma[1] = sigma0;
        cma[2] = 1.0;
        cma[3] = 0.0;
    }
}

// One CTA: the new mean m' = x_(1) + S1, the mean shift m' - m, z = L^-1 (m' - m) by forward
// substitution with the current factor L (L L^T = sigma^2 C, so z = L_C^-1 (m' - m) / sigma
// with L_C the Cholesky factor of C), the step-size path and its length, h_sigma, the
// covariance path, and sigma'. L is staged in shared memory (row stride D + 1); warp 0
// runs the substitution column by column, lane l holding rows l, l + 32, l + 64, l + 96,
// each new z_j passed by a shuffle, so the dependent chain has no block barrier.
__global__ void __launch_bounds__(kCmaThreads)
k_cma_paths(const double *__restrict__ s1p, int n_chunks, int D, const float *__restrict__ elites,
            const double *__restrict__ mu_prev, const double *__restrict__ L, CmaConsts k, int t,
            double *mu, double *p_sigma, double *p_c, double *cma)
{
    extern __shared__ double s_L[];   // [D][D + 1]
    __shared__ double s_b[kCmaThreads];
    __shared__ double s_red[kCmaThreads / 32];
    const int r = threadIdx.x, lane = r & 31;
    const int ld = D + 1;
    for (int idx = r; idx < D * D; idx += kCmaThreads) {
        const int i = idx / D, j = idx - i * D;
        if (j <= i) s_L[i * ld + j] = L[idx];
    }
    double shift = 0.0;
    if (r < D) {
        double s1 = 0.0;
        for (int c = 0; c < n_chunks; ++c) s1 += s1p[(size_t)c * D + r];
        const double m_new = (double)elites[r] + s1;
        shift = m_new - mu_prev[r];
        mu[r] = m_new;
        s_b[r] = shift;
    }
    __syncthreads();
    if (r < 32) {
        double b[4], rinv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = lane + 32 * i;
            b[i] = row < D ? s_b[row] : 0.0;
            rinv[i] = row < D ? 1.0 / s_L[row * ld + row] : 0.0;
        }
#pragma unroll
        for (int slot = 0; slot < 4; ++slot) {
            for (int jj = 0; jj < 32; ++jj) {
                const int j = slot * 32 + jj;
                if (j >= D) break;
                const double zj = __shfl_sync(0xffffffffu, b[slot] * rinv[slot], jj);
                if (lane == jj) s_b[j] = zj;   // z_j replaces b_j
#pragma unroll
                for (int i = slot; i < 4; ++i) {
                    const int row = lane + 32 * i;
                    if (row > j && row < D) b[i] = fma(-s_L[row * ld + j], zj, b[i]);
                }
            }
        }
    }
    __syncthreads();
    const double z = r < D ? s_b[r] : 0.0;
    const double sigma = cma[0];
    double ps = 0.0;
    if (r < D) {
        ps = fma(1.0 - k.c_sigma, p_sigma[r], sqrt(k.c_sigma * (2.0 - k.c_sigma) * k.mu_eff) * z);
        p_sigma[r] = ps;
    }
    double v = ps * ps;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[r >> 5] = v;
    __syncthreads();
    double n2 = 0.0;
    for (int w = 0; w < kCmaThreads / 32; ++w) n2 += s_red[w];
    const double norm = sqrt(n2);
    const double h = norm / sqrt(1.0 - pow(1.0 - k.c_sigma, 2.0 * (t + 1)))
                     < (1.4 + 2.0 / (D + 1)) * k.chi_n ? 1.0 : 0.0;
    if (r < D) p_c[r] = fma(1.0 - k.c_c, p_c[r], h * sqrt(k.c_c * (2.0 - k.c_c) * k.mu_eff) * (shift / sigma));
    if (r == 0) {
        cma[1] = sigma;
        cma[2] = h;
        cma[3] = norm;
        cma[0] = sigma * exp((k.c_sigma / k.d_sigma) * (norm / k.chi_n - 1.0));
    }
}

// One thread per lower-triangle entry: the elites' weighted scatter about the OLD mean m from
// the moments about x_(1) (with d = x_(1) - m and weights summing to one:
// S2 + S1 d^T + d S1^T + d d^T), then C' = a C + c_1 p_c p_c^T + c_mu scatter / sigma^2 with
// a = 1 + c_1 (1 - h_sigma) c_c (2 - c_c) - c_1 - c_mu.
__global__ void __launch_bounds__(256) k_cma_cov(const double *__restrict__ s2p, const double *__restrict__ s1p, int n_chunks,
                          int D, const float *__restrict__ elites, const double *__restrict__ mu_prev,
                          const double *__restrict__ p_c, const double *__restrict__ cma, CmaConsts k,
                          double *C)
{
    __shared__ double s_s1[4 * CP_MAX_WAYPOINTS];
    const int e0 = (int)(blockIdx.x * blockDim.x);
    stage_s1(s1p, n_chunks, D, last_row(e0, D), s_s1);
    const int e = e0 + (int)threadIdx.x;
    if (e >= D * (D + 1) / 2) return;
    int r, c;
    tri_index(e, r, c);
    const double s2 = tree_sum<1>(s2p + (size_t)r * D + c, n_chunks, (size_t)D * D, 0);
    const double sr = s_s1[r], sc = s_s1[c];
    const double dr = (double)elites[r] - mu_prev[r], dc = (double)elites[c] - mu_prev[c];
    const double scatter = fma(dr, dc, fma(dr, sc, fma(sr, dc, s2)));
    const double sig = cma[1], h = cma[2];
    const double a = 1.0 + k.c_1 * (1.0 - h) * k.c_c * (2.0 - k.c_c) - k.c_1 - k.c_mu;
    const double v = fma(a, C[(size_t)r * D + c], fma(k.c_1 * p_c[r], p_c[c], k.c_mu * scatter / (sig * sig)));
    C[(size_t)r * D + c] = v;
    C[(size_t)c * D + r] = v;
}

}  // namespace

int radix_tiles(int N) { return (N + kRadixTile - 1) / kRadixTile; }

size_t radix_hist_ints(int N) { return 256 * (size_t)radix_tiles(N) + kRadixTotals; }

// Sorted candidate order by (J, index) into `sorted` (N ints); scratch: two key buffers of
// N, one value buffer of N, hist of radix_hist_ints(N) ints (tile histograms, then the
// per-digit totals of every pass).
int launch_radix_rank(const double *J, int N, unsigned long long *key_a, unsigned long long *key_b,
                      int *val_a, int *val_b, int *hist, cudaStream_t st)
{
    const int tiles = radix_tiles(N);
    int *totals = hist + 256 * (size_t)tiles;   // [pass][digit]
    CP_CUDA(cudaMemsetAsync(totals, 0, sizeof(int) * kRadixTotals, st));
    k_radix_init<<<(N + 255) / 256, 256, 0, st>>>(J, N, key_a, val_a);
    CP_LAUNCHED("k_radix_init");
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        int *tot = totals + 256 * pass;
        k_radix_hist<false><<<tiles, kRadixThreads, 0, st>>>(key_a, N, shift, tiles, hist, tot);
        CP_LAUNCHED("k_radix_hist");
        k_radix_scan<<<256, 256, 0, st>>>(hist, tiles, tot);
        CP_LAUNCHED("k_radix_scan");
        k_radix_scatter<false><<<tiles, kRadixThreads, 0, st>>>(key_a, val_a, N, shift, tiles, hist, key_b, val_b);
        CP_LAUNCHED("k_radix_scatter");
        unsigned long long *tk = key_a;
        key_a = key_b;
        key_b = tk;
        int *tv = val_a;
        val_a = val_b;
        val_b = tv;
    }
    return CP_OK;   // after an even number of passes the result is back in val_a
}

int launch_gather_elites(const int *sorted, const double *J, const float *xi, int nu, int D,
                         int *elite, float *elites, double *best_J, cudaStream_t st)
{
    const int threads = 256;
    k_gather_elites<<<(nu * 32 + threads - 1) / threads, threads, 0, st>>>(sorted, J, xi, nu, D, elite,
                                                                          elites, best_J);
    CP_LAUNCHED("k_gather_elites");
    return CP_OK;
}

// Number of partials (chunks of elites) the update uses for nu elites of dimension D, and
// elites per chunk: chunks of 32 elites, doubled (up to 256) while the partial launch would
// have more than 1024 blocks, at most kMaxChunks chunks. A function of (nu, D) alone, so the
// order of the sums does not depend on the device.
int update_chunks(int nu, int D)
{
    const int nt = (D + 15) / 16, tiles = nt * (nt + 1) / 2;
    int e = kChunk;
    while (e < 256 && (long long)((nu + e - 1) / e) * tiles > 1024) e *= 2;
    const int n = (nu + e - 1) / e;
    return n < kMaxChunks ? n : kMaxChunks;
}

static int per_chunk(int nu, int D)
{
    const int n = update_chunks(nu, D);
    const int per = (nu + n - 1) / n;
    return (per + kChunk - 1) / kChunk * kChunk;
}

int update_configure()
{
    const int Dm = 4 * CP_MAX_WAYPOINTS;
    CP_CUDA(cudaFuncSetAttribute(k_cma_paths, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(double) * Dm * (Dm + 1))));
    return CP_OK;
}

int launch_weights(int nu, double *w, cudaStream_t st)
{
    k_weights<<<1, 1024, 0, st>>>(nu, w);
    CP_LAUNCHED("k_weights");
    return CP_OK;
}

// rank must be zero on entry (the workspace starts cleared and k_scatter clears it again).
int launch_rank(const double *J, int N, int nu, int *rank, cudaStream_t st)
{
    dim3 grid((N + kRankThreads - 1) / kRankThreads, (N + kRankPer - 1) / kRankPer);
    k_rank_count<<<grid, kRankThreads, 0, st>>>(J, N, rank);
    CP_LAUNCHED("k_rank_count");
    (void)nu;
    return CP_OK;
}

int launch_scatter(int *rank, const double *J, const float *xi, int N, int nu, int D,
                   int *elite, float *elites, double *best_J, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = (N * 32 + threads - 1) / threads;
    k_scatter<<<blocks, threads, 0, st>>>(rank, J, xi, N, nu, D, elite, elites, best_J);
    CP_LAUNCHED("k_scatter");
    return CP_OK;
}

int launch_cma_reset(double sigma0, int D, double *cma, double *p_sigma, double *p_c, cudaStream_t st)
{
    k_cma_reset<<<(D + 127) / 128, 128, 0, st>>>(sigma0, D, cma, p_sigma, p_c);
    CP_LAUNCHED("k_cma_reset");
    return CP_OK;
}

// CMA-ES update: mu_prev must hold the mean before the update; mu, C, p_sigma, p_c and cma
// are updated in place (L is the factor of sigma^2 C before the update).
static int launch_moments_partial(const float *elites, const double *w, int nu, int D, double *yw, double *s2p,
                                  double *s1p, int *n_chunks_out, cudaStream_t st)
{
    const int per = per_chunk(nu, D);
    const int n_chunks = (nu + per - 1) / per;
    const int tiles = (D + 15) / 16;
    double *Y = yw, *WY = yw + (size_t)nu * D;
    k_moments_prep<<<(nu * D + 255) / 256, 256, 0, st>>>(elites, w, nu, D, Y, WY);
    CP_LAUNCHED("k_moments_prep");
    dim3 grid(tiles * (tiles + 1) / 2, n_chunks);
    k_moments_partial<<<grid, 256, 0, st>>>(Y, WY, nu, D, per, n_chunks, s2p, s1p);
    CP_LAUNCHED("k_moments_partial");
    *n_chunks_out = n_chunks;
    return CP_OK;
}

int launch_cma_update(const float *elites, const double *w, int nu, int D, const double *mu_prev,
                      const double *L, const CmaConsts &k, int t, double *yw, double *s2p, double *s1p, double *mu,
                      double *C, double *p_sigma, double *p_c, double *cma, cudaStream_t st)
{
    int n_chunks = 0;
    int rc = launch_moments_partial(elites, w, nu, D, yw, s2p, s1p, &n_chunks, st);
    if (rc != CP_OK) return rc;
    const size_t smem = sizeof(double) * (size_t)D * (D + 1);
    k_cma_paths<<<1, kCmaThreads, smem, st>>>(s1p, n_chunks, D, elites, mu_prev, L, k, t, mu, p_sigma, p_c, cma);
    CP_LAUNCHED("k_cma_paths");
    const int entries = D * (D + 1) / 2;
    k_cma_cov<<<(entries + 255) / 256, 256, 0, st>>>(s2p, s1p, n_chunks, D, elites, mu_prev, p_c, cma, k, C);
    CP_LAUNCHED("k_cma_cov");
    return CP_OK;
}

int moments_chunking(int nu, int D, int *per)
{
    *per = per_chunk(nu, D);
    return (nu + *per - 1) / *per;
}

// Stable LSD ranking of every query's candidates at once: the eight key passes order all
// positions by (J, position); the query passes then move each query's candidates, in that
// order, to its own range (a query's positions are contiguous and increase with the index,
// so ties keep the index order of the plain ranking).
int launch_batch_radix_rank(const BatchQueryDev *qd, const int2 *tab, int blocks, int total, int nq,
                            const uint16_t *qid, unsigned long long *key_a, unsigned long long *key_b,
                            int *val_a, int *val_b, int *hist, int **sorted, cudaStream_t st)
{
    const int tiles = radix_tiles(total);
    int *totals = hist + 256 * (size_t)tiles;   // [pass][digit]
    CP_CUDA(cudaMemsetAsync(totals, 0, sizeof(int) * kRadixTotals, st));
    k_batch_radix_init<<<blocks, 256, 0, st>>>(qd, tab, key_a, val_a);
    CP_LAUNCHED("k_batch_radix_init");
    const int q_passes = nq > 256 ? 2 : (nq > 1 ? 1 : 0);
    for (int pass = 0; pass < 8 + q_passes; ++pass) {
        const bool byq = pass >= 8;
        const int shift = byq ? 8 * (pass - 8) : 8 * pass;
        int *tot = totals + 256 * pass;
        if (byq)
            k_radix_hist<true><<<tiles, kRadixThreads, 0, st>>>(key_a, total, shift, tiles, hist, tot, val_a, qid);
        else
            k_radix_hist<false><<<tiles, kRadixThreads, 0, st>>>(key_a, total, shift, tiles, hist, tot);
        CP_LAUNCHED("k_radix_hist");
        k_radix_scan<<<256, 256, 0, st>>>(hist, tiles, tot);
        CP_LAUNCHED("k_radix_scan");
        if (byq)
            k_radix_scatter<true><<<tiles, kRadixThreads, 0, st>>>(key_a, val_a, total, shift, tiles, hist, key_b,
                                                                   val_b, qid);
        else
            k_radix_scatter<false><<<tiles, kRadixThreads, 0, st>>>(key_a, val_a, total, shift, tiles, hist, key_b,
                                                                    val_b);
        CP_LAUNCHED("k_radix_scatter");
        unsigned long long *tk = key_a;
        key_a = key_b;
        key_b = tk;
        int *tv = val_a;
        val_a = val_b;
        val_b = tv;
    }
    *sorted = val_a;
    return CP_OK;
}

int launch_batch_gather(const BatchQueryDev *qd, const int2 *tab, int blocks, const int *sorted, cudaStream_t st)
{
    if (blocks == 0) return CP_OK;
    k_batch_gather<<<blocks, 256, 0, st>>>(qd, tab, sorted);
    CP_LAUNCHED("k_batch_gather");
    return CP_OK;
}

int launch_batch_moments(const BatchQueryDev *qd, int nq, const int2 *tab_prep, int blocks_prep,
                         const int2 *tab_partial, int blocks_partial, const int2 *tab_combine, int blocks_combine,
                         cudaStream_t st)
{
    k_batch_moments_prep<<<blocks_prep, 256, 0, st>>>(qd, tab_prep);
    CP_LAUNCHED("k_batch_moments_prep");
    k_batch_moments_partial<<<blocks_partial, 256, 0, st>>>(qd, tab_partial);
    CP_LAUNCHED("k_batch_moments_partial");
    k_batch_moments_s1<<<dim3(CP_MAX_WAYPOINTS * 4 / 32, nq), 128, 0, st>>>(qd);
    CP_LAUNCHED("k_batch_moments_s1");
    k_batch_moments_combine<<<blocks_combine, 128, 0, st>>>(qd, tab_combine);
    CP_LAUNCHED("k_batch_moments_combine");
    return CP_OK;
}

int launch_moments(const float *elites, const double *w, int nu, int D, double eps, double *yw,
                   double *s2p, double *s1p, double *mu, double *C, cudaStream_t st)
{
    int n_chunks = 0;
    int rc = launch_moments_partial(elites, w, nu, D, yw, s2p, s1p, &n_chunks, st);
    if (rc != CP_OK) return rc;
    const int entries = D * (D + 1) / 2;
    k_moments_s1<<<(D + 31) / 32, 128, 0, st>>>(s1p, n_chunks, D, elites, mu);
    CP_LAUNCHED("k_moments_s1");
    k_moments_combine<<<(entries + 31) / 32, 128, 0, st>>>(s2p, s1p + (size_t)n_chunks * D, n_chunks, D, eps, C);
    CP_LAUNCHED("k_moments_combine");
    return CP_OK;
}

}  // namespace cp
