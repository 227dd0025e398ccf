// The last part of Algorithm 1 step (2): per candidate, the FP32 partial sums of its work
// units (32 checkpoints each: J_p, the penetration sum, J_l, the path length, and the
// ballot word of checkpoints in collision) summed in FP64 into
// J = J_p + w_c lambda_c sum_k pen_k + w_l J_l (Eq. path opt; arXiv 2503.14160, Sec. 4.1).
//
// Eight lanes per candidate: lane g of the group loads the unit records g, g + 8, ... first
// (independent loads in flight together), then adds them in FP64 in that order, and three
// shuffle steps combine the eight sums in a fixed tree, so results are deterministic. FP64
// adds have a long dependent latency on this part; the split keeps every chain short.
#include "cp_internal.cuh"

namespace cp {
namespace {

constexpr int kFinalizeLanes = 8;
constexpr int kFinalizeBatch = 4;   // unit records loaded before they are added

__global__ void __launch_bounds__(256)
k_eval_finalize(const float4 *__restrict__ partial, const uint32_t *__restrict__ flagword, int n, int chunks,
                double w_c, double w_l, double lambda_c, double *J, uint8_t *flag, double *terms,
                uint32_t *substep_flags, const uint32_t *status)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / kFinalizeLanes, g = t % kFinalizeLanes;
    const bool active = i < n;
    double jp = 0.0, jc = 0.0, jl = 0.0, len = 0.0;
    int n_flagged = 0;
    if (active) {
        const float4 *row = partial + (size_t)i * chunks;
        const uint32_t *frow = flagword + (size_t)i * chunks;
        for (int c0 = g; c0 < chunks; c0 += kFinalizeLanes * kFinalizeBatch) {
            float4 v[kFinalizeBatch];
            uint32_t w[kFinalizeBatch];
#pragma unroll
            for (int b = 0; b < kFinalizeBatch; ++b) {
                const int c = c0 + b * kFinalizeLanes;
                v[b] = c < chunks ? row[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                w[b] = c < chunks ? frow[c] : 0u;
            }
#pragma unroll
            for (int b = 0; b < kFinalizeBatch; ++b) {
                jp += (double)v[b].x;
                jc += (double)v[b].y;
                jl += (double)v[b].z;
                len += (double)v[b].w;
                n_flagged += __popc(w[b]);
                const int c = c0 + b * kFinalizeLanes;
                if (substep_flags != nullptr && c < chunks) substep_flags[(size_t)i * chunks + c] = w[b];
            }
        }
    }
#pragma unroll
    for (int off = 1; off < kFinalizeLanes; off <<= 1) {   // every lane of the warp takes part
        jp += __shfl_xor_sync(0xffffffffu, jp, off);
        jc += __shfl_xor_sync(0xffffffffu, jc, off);
        jl += __shfl_xor_sync(0xffffffffu, jl, off);
        len += __shfl_xor_sync(0xffffffffu, len, off);
        n_flagged += __shfl_xor_sync(0xffffffffu, n_flagged, off);
    }
    if (!active || g != 0) return;
    jc *= lambda_c;
    J[i] = jp + w_c * jc + w_l * jl;
    if (flag != nullptr) flag[i] = n_flagged > 0 ? 1 : 0;
    if (status != nullptr && *status != 0u) {
        // the evaluation gave up on a bounded wait: some partials are stale, so no result
        // of this call is valid (NaN cost, flagged)
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        jp = jc = jl = len = nan;
        J[i] = nan;
        if (flag != nullptr) flag[i] = 1;
    }
    if (terms != nullptr) {
        double *tm = terms + (size_t)i * 5;
        tm[0] = jp;
        tm[1] = jc;
        tm[2] = jl;
        tm[3] = len;
        tm[4] = (double)n_flagged;
    }
}

}  // namespace

int launch_eval_finalize(const float4 *partial, const uint32_t *flagword, int n, int chunks,
                         double w_c, double w_l, double lambda_c, double *J, uint8_t *flag,
                         double *terms, uint32_t *substep_flags, cudaStream_t st,
                         const uint32_t *status)
{
    if (n == 0) return CP_OK;
    const int threads = 256;
    const int64_t total = (int64_t)n * kFinalizeLanes;
    k_eval_finalize<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
        partial, flagword, n, chunks, w_c, w_l, lambda_c, J, flag, terms, substep_flags, status);
    CP_LAUNCHED("k_eval_finalize");
    return CP_OK;
}

}  // namespace cp
