// kern.cuh -- launch and reduction helpers shared by the cycle kernels of
// one right-hand side (cycle.cu) and of interleaved blocks of right-hand
// sides (block.cu).
#pragma once

#include <algorithm>
#include <utility>

#include "gw_internal.cuh"

namespace gw {

constexpr int BS = 256;  // threads per block of every cycle and CG kernel

// Blocks a grid-stride loop over `threads` work items asks for.
static inline int blocks_for(long long threads)
{
    const long long b = (threads + BS - 1) / BS;
    return (int)std::max(1LL, std::min<long long>(b, 1LL << 30));
}

#ifndef GW_GRID_BALANCE
#define GW_GRID_BALANCE 0
#endif

// The grid actually launched for `blocks`: at most one wave of the kernel
// (its resident blocks per SM times the SMs, from the occupancy calculator),
// and within that as few blocks as give every thread the same number of
// grid-stride iterations.
static inline int wave_grid(const void *fn, int blocks)
{
    const int cap = kernel_wave(fn, BS);
    if (blocks <= cap) return std::max(1, blocks);
    if (!GW_GRID_BALANCE) return cap;
    const int iters = (blocks + cap - 1) / cap;
    return (blocks + iters - 1) / iters;
}

#define ROWS(i, n) for (int i = blockIdx.x * BS + threadIdx.x; i < (n); i += gridDim.x * BS)

// The block index and block count a kernel body works with: the launch's own
// grid, or, in a batched launch that runs one pass for several solves, the
// virtual grid of one solve (each solve keeps its own row partition and
// reduction order, so its results do not depend on what else runs).
struct VB {
    int bid, nb;
};
__device__ __forceinline__ VB vb_grid() { return VB{(int)blockIdx.x, (int)gridDim.x}; }

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
    cfg.gridDim = dim3((unsigned)wave_grid((const void *)kernel, grid));
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
// A thread's share of an FP32 dot product without FP32 rounding of the sum:
// each product is split exactly into p + e (e by a fused multiply-add) and
// the products are added in two FP32 words by the error-free TwoSum, which
// keeps about 46 bits; the pair becomes an FP64 value at the reduction.  FP32
// operations only (FP64 throughput is scarce on this GPU); explicitly rounded
// intrinsics keep the compiler from contracting the transformations.
struct Sum2 {
    float hi = 0.f, lo = 0.f;
};
__device__ __forceinline__ void sum2_prod(Sum2 &s, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s.hi, p);
    const float bp = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double sum2_value(const Sum2 &s) { return (double)s.hi + (double)s.lo; }

// A thread's running share of a dot product over all its rows: for FP32
// operands the error-free pair above, carried from row block to row block
// and turned into FP64 once, when the block reduces (one conversion a thread
// instead of one a row block: FP64 issue, about 2 operations a cycle an SM,
// is the scarce unit on this GPU); for FP64 operands a plain FP64 sum.
struct DAcc {
    Sum2 s;
    double d = 0.0;
};
__device__ __forceinline__ double dacc_value(const DAcc &a) { return a.d + sum2_value(a.s); }

// adds the dot product of R consecutive entries
template <int R, class T, class U>
__device__ __forceinline__ void dot_add(DAcc &acc, const T (&a)[R], const U (&b)[R])
{
    if constexpr (sizeof(T) == 4 && sizeof(U) == 4) {
#pragma unroll
        for (int k = 0; k < R; ++k) sum2_prod(acc.s, (float)a[k], (float)b[k]);
    } else {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < R; ++k) s += (double)a[k] * (double)b[k];
        acc.d += s;
    }
}
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
__device__ __forceinline__ bool reduce_last(VB vb, const double (&loc)[K], double *part, unsigned *cnt,
                                            double (&tot)[K])
{
    constexpr int W = BS / 32;
    __shared__ double sh[K][W];
    __shared__ unsigned ticket;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // warps (shuffle tree), then one thread per value adds the warps in order
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double v = warp_sum(loc[k]);
        if (lane == 0) sh[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < W; ++q) s += sh[threadIdx.x][q];
        part[(size_t)threadIdx.x * vb.nb + vb.bid] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
    __syncthreads();
    if (ticket != (unsigned)vb.nb - 1) return false;
    __threadfence();
    // last block: every thread adds the partials b = t, t + BS, ... (their
    // loads issued together), then the warps' shuffle trees and the warps in
    // order, a fixed order for a given block count
    __shared__ double fin[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
#pragma unroll 8
        for (int b = threadIdx.x; b < vb.nb; b += BS) s += __ldcg(part + (size_t)k * vb.nb + b);
        s = warp_sum(s);
        if (lane == 0) sh[k][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < W; ++q) s += sh[threadIdx.x][q];
        fin[threadIdx.x] = s;
    }
    if (threadIdx.x == 0) *cnt = 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = fin[k];
    return true;
}

template <int K>
__device__ __forceinline__ bool reduce_last(const double (&loc)[K], double *part, unsigned *cnt, double (&tot)[K])
{
    return reduce_last<K>(vb_grid(), loc, part, cnt, tot);
}

__device__ __forceinline__ bool finished(const Ctl *c) { return c && *(volatile const int *)&c->done; }

// Ends the solve with the given status.  Under a graph while node the loop
// itself is ended by the kernel that checks the true residual (k_rel_res, or
// k_cg_true in the FP64 form): it stops the loop when it finds the solve done
// on entry, or when it finds it converged, so that the heavy kernels make no
// device graph call (profilers skip kernels that make one).
__device__ __forceinline__ void ctl_stop(Ctl *c, int status)
{
    c->status = status;
    c->done = 1;
}

// ends the while loop of the solve's graph (one thread: the condition is
// never set concurrently)
__device__ __forceinline__ void ctl_end_loop(const Ctl *c)
{
    if (c->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)c->cond, 0u);
}

}  // namespace gw
