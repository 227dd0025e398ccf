// How the warps of an evaluation launch take its work items. With a counter
// (EvalArgs::queue, zeroed before the launch) lane 0 takes the next item and the warp shares
// it, so candidates of uneven cost (those in contact take the exact distances) even out over
// the warps; without one the items go round the warps in a fixed stride. The counter only
// grows, so every warp leaves once the items are handed out. Called by whole warps.
#pragma once

#include "cp_internal.cuh"

namespace cp {

__device__ __forceinline__ int queue_next(const EvalArgs &a, int it, int n_warps, int lane)
{
    if (a.queue == nullptr) return it + n_warps;
    int v = 0;
    if (lane == 0) v = atomicAdd(a.queue, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ int queue_first(const EvalArgs &a, int warp, int lane)
{
    return a.queue == nullptr ? warp : queue_next(a, 0, 0, lane);
}

}  // namespace cp
