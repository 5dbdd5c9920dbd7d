// kern.cuh -- launch and reduction helpers shared by the cycle kernels of
// one right-hand side (cycle.cu) and of interleaved blocks of right-hand
// sides (block.cu).
#pragma once

#include <utility>

#include "gw_internal.cuh"

namespace gw {

constexpr int BS = 256;  // threads per block of every cycle and CG kernel

#define ROWS(i, n) for (int i = blockIdx.x * BS + threadIdx.x; i < (n); i += gridDim.x * BS)

// Programmatic dependent launch: every kernel of the cycle and of CG is
// launched so that the next kernel in the stream may be scheduled while this
// one runs; each kernel waits for its predecessors to complete (and their
// writes to be visible) before it touches global memory, then lets its own
// dependents launch.  Inside captured graphs this hides the launch gap
// between the 20-30 dependent kernels of a CG iteration.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GW_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}


// ------------------------------------------------------------- reductions --
__device__ __forceinline__ double warp_sum(double v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// block sum in a fixed order (shuffle tree, then warp 0 adds the 8 warp sums)
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < BS / 32 ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;  // valid in thread 0
}

// Writes this block's partial sums; returns true in the last block to arrive,
// which then holds the grand totals (summed over blocks in index order) in tot[].
template <int K>
__device__ __forceinline__ bool reduce_last(const double (&loc)[K], double *part, unsigned *cnt, double (&tot)[K])
{
    __shared__ double sh[32];
    __shared__ unsigned ticket;
    for (int k = 0; k < K; ++k) {
        double s = block_sum(loc[k], sh);
        if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return false;
    __threadfence();
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += BS) s += __ldcg(part + (size_t)k * gridDim.x + b);
        tot[k] = block_sum(s, sh);
    }
    if (threadIdx.x == 0) *cnt = 0u;
    return true;
}

__device__ __forceinline__ bool finished(const Ctl *c) { return c && *(volatile const int *)&c->done; }

}  // namespace gw
