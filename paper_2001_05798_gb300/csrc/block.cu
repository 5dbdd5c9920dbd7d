// block.cu -- several right-hand sides solved together on one hierarchy.
//
// Systems that share a matrix reuse its preconditioner (Introduction, on the
// dual delineation approach).  Here KB right-hand sides (KB = 4 or 8) run
// as KB independent preconditioned CG recurrences whose vectors are
// interleaved: entry j of row i sits at i*KB + j.  Every pass of the V-cycle
// and of CG then reads each level matrix (values, indices, the level-0
// stencil coefficients) once for all KB columns, and a gathered neighbour
// supplies KB consecutive values.  One thread handles CW consecutive columns
// of one row with a single 16-byte access.
//
// The arithmetic per column is the mixed form of the single-vector solver:
// FP32 hierarchy, FP32 recurrence with the flexible beta, FP64 solution by
// reliable updates against the FP64 level-0 operator, and the stop on the
// FP64 residual.  Each column carries its own scalars (alpha, beta, rz, ...)
// in a device control block; a column that has converged or failed keeps
// alpha = 0, so its solution no longer changes, while the others go on.  The
// passes are captured in CUDA graphs and replayed until every column is done.
#include <string.h>

#include <memory>
#include <type_traits>
#include <vector>

#include "gw_internal.cuh"
#include "kern.cuh"

namespace gw {

constexpr int KB_MAX = 8;

// Column scalars of one block solve.
struct BlkCtl {
    Ctl col[KB_MAX];
    unsigned cnt[4];
    int done;       // every column has finished
    int any_check;  // some column asks for a reliable update
};

// ------------------------------------------------------------- vectors --
template <class T, int CW>
struct alignas(sizeof(T) * CW) CV {
    T v[CW];
};

template <int CW, class T>
__device__ __forceinline__ CV<T, CW> cld(const T *p)
{
    return *reinterpret_cast<const CV<T, CW> *>(p);
}

template <int CW, class T>
__device__ __forceinline__ void cst(T *p, const CV<T, CW> &a)
{
    *reinterpret_cast<CV<T, CW> *>(p) = a;
}

template <int CW, class T>
__device__ __forceinline__ void cacc(CV<T, CW> &acc, T c, const CV<T, CW> &x)
{
#pragma unroll
    for (int u = 0; u < CW; ++u) acc.v[u] += c * x.v[u];
}

// gathered value functors; x is already offset to the thread's first column
template <class T, int CW, int KB>
struct BVec {
    const T *x;
    __device__ __forceinline__ CV<T, CW> operator()(int c) const { return cld<CW>(x + c * KB); }
};

// c0 dw_c b_c: the first Chebyshev correction from a zero guess
template <int CW, int KB>
struct BProd {
    const float *dw;
    const float *b;
    float c0;
    __device__ __forceinline__ CV<float, CW> operator()(int c) const
    {
        const float w = dw[c];
        CV<float, CW> o = cld<CW>(b + c * KB);
#pragma unroll
        for (int u = 0; u < CW; ++u) o.v[u] = c0 * (w * o.v[u]);
        return o;
    }
};

// z_c + beta p_c: the new CG direction, formed where it is gathered
template <int CW, int KB>
struct BDir {
    const float *z;
    const float *p;
    CV<float, CW> beta;
    __device__ __forceinline__ CV<float, CW> operator()(int c) const
    {
        const CV<float, CW> zz = cld<CW>(z + c * KB), pp = cld<CW>(p + c * KB);
        CV<float, CW> o;
#pragma unroll
        for (int u = 0; u < CW; ++u) o.v[u] = zz.v[u] + beta.v[u] * pp.v[u];
        return o;
    }
};

// ---------------------------------------------------------- matrix views --
// Row products of CW columns.  Terms are added in the order of the
// single-vector views (stencil: -z, -y, -x, diagonal, +x, +y, +z; sliced
// ELL: slot order), so a column's product equals the single-vector one.
template <class T>
struct BSten {
    const T *__restrict__ d;
    const T *__restrict__ ox;
    const T *__restrict__ oy;
    const T *__restrict__ oz;
    int n, nx, sxy;
    template <int CW, class F>
    __device__ __forceinline__ CV<T, CW> dot(int i, F f) const
    {
        CV<T, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0;
        if (i >= sxy) cacc(acc, __ldg(oz + i - sxy), f(i - sxy));
        if (i >= nx) cacc(acc, __ldg(oy + i - nx), f(i - nx));
        if (i >= 1) cacc(acc, __ldg(ox + i - 1), f(i - 1));
        cacc(acc, __ldg(d + i), f(i));
        if (i + 1 < n) cacc(acc, __ldg(ox + i), f(i + 1));
        if (i + nx < n) cacc(acc, __ldg(oy + i), f(i + nx));
        if (i + sxy < n) cacc(acc, __ldg(oz + i), f(i + sxy));
        return acc;
    }
};

template <class T>
struct BSell {
    const int *__restrict__ sp;
    const int *__restrict__ ci;
    const T *__restrict__ v;
    const int *__restrict__ perm;  // row of slot row r (null: r); restriction matrices only
    __device__ __forceinline__ int out_row(int r) const { return perm ? __ldg(perm + r) : r; }
    template <int CW, class F>
    __device__ __forceinline__ CV<T, CW> dot(int r, F f) const
    {
        constexpr int V = SellV<T>::V;
        const int s = r >> 5, lane = r & 31;
        const int base = sp[s];
        const int nch = (sp[s + 1] - base) / (SELL_C * V);
        CV<T, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0;
        // two chunks at a time: values and columns, then the gathers, then the
        // products in chunk order, so that a row's loads overlap
        for (int c = 0; c < nch; c += 2) {
            const bool two = c + 1 < nch;
            const int e0 = base + c * SELL_C * V + lane * V, e1 = e0 + SELL_C * V;
            T a0[V], a1[V];
            int j0[V], j1[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                a0[k] = __ldg(v + e0 + k);
                j0[k] = __ldg(ci + e0 + k);
                a1[k] = two ? __ldg(v + e1 + k) : T(0);
                j1[k] = two ? __ldg(ci + e1 + k) : 0;
            }
            decltype(f(0)) g0[V], g1[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                g0[k] = f(j0[k]);
                if (two) g1[k] = f(j1[k]);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) cacc(acc, a0[k], g0[k]);
            if (two) {
#pragma unroll
                for (int k = 0; k < V; ++k) cacc(acc, a1[k], g1[k]);
            }
        }
        return acc;
    }
};

template <class T>
struct BCsr {
    const int *__restrict__ rp;
    const int *__restrict__ ci;
    const T *__restrict__ v;
    template <int CW, class F>
    __device__ __forceinline__ CV<T, CW> dot(int i, F f) const
    {
        CV<T, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0;
        const int e1 = rp[i + 1];
        for (int e = rp[i]; e < e1; ++e) cacc(acc, __ldg(v + e), f(__ldg(ci + e)));
        return acc;
    }
};

struct BStenB {
    const float *__restrict__ d;
    const __nv_bfloat16 *__restrict__ ox;
    const __nv_bfloat16 *__restrict__ oy;
    const __nv_bfloat16 *__restrict__ oz;
    int n, nx, sxy;
    template <int CW, class F>
    __device__ __forceinline__ CV<float, CW> dot(int i, F f) const
    {
        CV<float, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0.f;
        if (i >= sxy) cacc(acc, __bfloat162float(oz[i - sxy]), f(i - sxy));
        if (i >= nx) cacc(acc, __bfloat162float(oy[i - nx]), f(i - nx));
        if (i >= 1) cacc(acc, __bfloat162float(ox[i - 1]), f(i - 1));
        cacc(acc, __ldg(d + i), f(i));
        if (i + 1 < n) cacc(acc, __bfloat162float(ox[i]), f(i + 1));
        if (i + nx < n) cacc(acc, __bfloat162float(oy[i]), f(i + nx));
        if (i + sxy < n) cacc(acc, __bfloat162float(oz[i]), f(i + sxy));
        return acc;
    }
};

struct BStenH {
    const float *__restrict__ sd;
    const __half *__restrict__ dd;
    const __half *__restrict__ ox;
    const __half *__restrict__ oy;
    const __half *__restrict__ oz;
    int n, nx, sxy;
    template <int CW>
    __device__ __forceinline__ CV<float, CW> scaled(float s, const CV<float, CW> &x) const
    {
        CV<float, CW> o;
#pragma unroll
        for (int u = 0; u < CW; ++u) o.v[u] = s * x.v[u];
        return o;
    }
    template <int CW, class F>
    __device__ __forceinline__ CV<float, CW> dot(int i, F f) const
    {
        CV<float, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0.f;
        const float si = __ldg(sd + i);
        if (i >= sxy) cacc(acc, __half2float(oz[i - sxy]), scaled<CW>(__ldg(sd + i - sxy), f(i - sxy)));
        if (i >= nx) cacc(acc, __half2float(oy[i - nx]), scaled<CW>(__ldg(sd + i - nx), f(i - nx)));
        if (i >= 1) cacc(acc, __half2float(ox[i - 1]), scaled<CW>(__ldg(sd + i - 1), f(i - 1)));
        cacc(acc, 1.f + __half2float(dd[i]), scaled<CW>(si, f(i)));
        if (i + 1 < n) cacc(acc, __half2float(ox[i]), scaled<CW>(__ldg(sd + i + 1), f(i + 1)));
        if (i + nx < n) cacc(acc, __half2float(oy[i]), scaled<CW>(__ldg(sd + i + nx), f(i + nx)));
        if (i + sxy < n) cacc(acc, __half2float(oz[i]), scaled<CW>(__ldg(sd + i + sxy), f(i + sxy)));
        return scaled<CW>(si, acc);
    }
};

template <class T, class F>
static void with_bmat(const MatStore<T> &M, F f)
{
    switch (M.fmt) {
    case FMT_SELL: f(BSell<T>{M.sell.sp.p, M.sell.ci.p, M.sell.v.p, M.sell.perm.p}); break;
    case FMT_CSR4:
    case FMT_CSR8:
    case FMT_CSR32: f(BCsr<T>{M.csr.rp.p, M.csr.ci.p, M.csr.v.p}); break;
    case FMT_STEN: {
        const StenT<T> &S = M.sten;
        f(BSten<T>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, S.nx * S.ny});
        break;
    }
    case FMT_STENB:
        if constexpr (sizeof(T) == 4) {
            const StenB &S = M.stenb;
            f(BStenB{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, S.nx * S.ny});
            break;
        }
        [[fallthrough]];
    case FMT_STENH:
        if constexpr (sizeof(T) == 4) {
            const StenH &S = M.stenh;
            f(BStenH{S.sd.p, S.dd.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, S.nx * S.ny});
            break;
        }
        [[fallthrough]];
    default: fail(GW_ERR_ARG, "interleaved solves need P, R and the coarse operators uncompressed");
    }
}

// thread -> (row, first column): TPR = KB / CW threads per row
#define BLOCK_ROWS(n, KB, CW)                                                                         \
    for (int t_ = blockIdx.x * BS + threadIdx.x, i = t_ / ((KB) / (CW)), off = (t_ % ((KB) / (CW))) * (CW); \
         i < (n); t_ += gridDim.x * BS, i = t_ / ((KB) / (CW)), off = (t_ % ((KB) / (CW))) * (CW))

// first column of this thread (fixed: the grid stride is a multiple of KB / CW)
template <int KB, int CW>
__device__ __forceinline__ int first_col()
{
    return (int)((blockIdx.x * BS + threadIdx.x) % (KB / CW)) * CW;
}

__device__ __forceinline__ bool bfinished(const BlkCtl *c) { return *(volatile const int *)&c->done; }

// ----------------------------------------------------------- reductions --
// Per-column sums of NV quantities.  A thread holds CW columns (its first
// column is (lane mod TPR) * CW); lanes of equal first column are added by a
// shuffle tree, the warps in order, the blocks in order by the last block to
// arrive, so every sum is reproducible.  Returns true in that last block, with
// tot[v * KB + j] valid in every thread after the call.
template <int KB, int CW, int NV>
__device__ __forceinline__ bool reduce_cols(const double (&loc)[NV][CW], double *part, unsigned *cnt, double *tot)
{
    constexpr int TPR = KB / CW, W = BS / 32;
    __shared__ double sh[NV * KB][W];
    __shared__ unsigned ticket;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            double s = loc[v][u];
#pragma unroll
            for (int o = 16; o >= TPR; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane < TPR) sh[v * KB + lane * CW + u][w] = s;
        }
    __syncthreads();
    if (threadIdx.x < NV * KB) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < W; ++k) s += sh[threadIdx.x][k];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
    __syncthreads();
    if (ticket != gridDim.x - 1) return false;
    __threadfence();
    for (int q = w; q < NV * KB; q += W) {
        double s = 0.0;
#pragma unroll 8
        for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)q * gridDim.x + b);
        s = warp_sum(s);
        if (lane == 0) tot[q] = s;
    }
    if (threadIdx.x == 0) *cnt = 0u;
    __syncthreads();
    return true;
}

// after the column updates of an epilogue (thread 0 of the last block)
template <int KB>
__device__ __forceinline__ void refresh_done(BlkCtl *c)
{
    int all = 1, chk = 0;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
        all &= c->col[j].done ? 1 : 0;
        chk |= (!c->col[j].done && c->col[j].check) ? 1 : 0;
    }
    c->done = all;
    c->any_check = chk;
}

__device__ __forceinline__ void col_stop(Ctl &c, int status)
{
    c.status = status;
    c.done = 1;
    c.alpha = 0.0;
    c.beta = 0.0;
    c.check = 0;
}

// Epilogue of the last kernel of a preconditioner application: rz = (r, z);
// mode 1 also forms the flexible beta = -alpha (q, z) / rz_old.
template <int KB, int CW>
__device__ __forceinline__ void rz_cols(const double (&loc)[2][CW], double *part, BlkCtl *c, int mode)
{
    __shared__ double tot[2 * KB];
    if (!reduce_cols<KB, CW, 2>(loc, part, &c->cnt[0], tot)) return;
    if (threadIdx.x < KB) {
        Ctl &cj = c->col[threadIdx.x];
        if (!cj.done) {
            const double rz_new = tot[threadIdx.x];
            if (mode == 1) {
                const double beta = -cj.alpha * tot[KB + threadIdx.x] / cj.rz;
                cj.beta = beta;
                if (!isfinite(beta) || !isfinite(rz_new)) col_stop(cj, GW_ERR_BREAKDOWN);
            }
            cj.rz = rz_new;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) refresh_done<KB>(c);
}

// A thread's per-column dot-product shares are error-free FP32 pairs carried
// over all its rows (FP32 operations only) and become FP64 once, before the
// block reduction, as in the single-vector passes.
template <int NV, int CW>
__device__ __forceinline__ void pairs_to_double(const Sum2 (&a)[NV][CW], double (&d)[NV][CW])
{
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int u = 0; u < CW; ++u) d[v][u] = sum2_value(a[v][u]);
}

template <int KB, int CW>
__device__ __forceinline__ void rz_cols(const Sum2 (&acc)[2][CW], double *part, BlkCtl *c, int mode)
{
    double loc[2][CW];
    pairs_to_double(acc, loc);
    rz_cols<KB, CW>(loc, part, c, mode);
}

template <int CW>
__device__ __forceinline__ void dot_cols(const float *b, const CV<float, CW> &z, const float *q, Sum2 (&loc)[2][CW])
{
    const CV<float, CW> bb = cld<CW>(b);
#pragma unroll
    for (int u = 0; u < CW; ++u) sum2_prod(loc[0][u], bb.v[u], z.v[u]);
    if (q) {
        const CV<float, CW> qq = cld<CW>(q);
#pragma unroll
        for (int u = 0; u < CW; ++u) sum2_prod(loc[1][u], qq.v[u], z.v[u]);
    }
}

// ------------------------------------------------------- V-cycle kernels --
// The same passes as the single-vector cycle, on KB interleaved columns.
// DOT: the pass writes the CG's z and reduces (r, z) and (q, z) per column.

// first two Chebyshev steps from zero: d0 = c0 dw b, r1 = b - A d0,
// d1 = c1 d0 + c2 dw r1, x = d0 + d1
template <int KB, int CW, class M, bool DOT>
__global__ void __launch_bounds__(BS) kb_cheb_zero2(M A, int n, const float *__restrict__ dw,
                                                    const float *__restrict__ b, float *__restrict__ x,
                                                    float *__restrict__ r, float *__restrict__ d,
                                                    float *__restrict__ xo, float c0, float c1, float c2, int keep,
                                                    const float *__restrict__ q, double *part, BlkCtl *c, int mode)
{
    pdl_enter();
    if (bfinished(c)) return;
    Sum2 loc[2][CW];
    BLOCK_ROWS(n, KB, CW)
    {
        const CV<float, CW> ad = A.template dot<CW>(i, BProd<CW, KB>{dw, b + off, c0});
        const size_t e = (size_t)i * KB + off;
        const CV<float, CW> bi = cld<CW>(b + e);
        const float w = dw[i];
        CV<float, CW> rv, dv, xv;
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            const float d0 = c0 * (w * bi.v[u]);
            rv.v[u] = bi.v[u] - ad.v[u];
            dv.v[u] = c1 * d0 + c2 * (w * rv.v[u]);
            xv.v[u] = d0 + dv.v[u];
        }
        if (keep) {
            cst<CW>(r + e, rv);
            cst<CW>(d + e, dv);
        }
        if constexpr (DOT) {
            cst<CW>(xo + e, xv);
            dot_cols<CW>(b + e, xv, q ? q + e : nullptr, loc);
        } else {
            cst<CW>(x + e, xv);
        }
    }
    if constexpr (DOT) rz_cols<KB, CW>(loc, part, c, mode);
}

// Chebyshev first step: r = b - A x (r = b when x0zero), d = c0 dw r;
// with x0zero x = d, otherwise the next step adds d.  DOT: z = x + d.
template <int KB, int CW, class M, bool DOT>
__global__ void __launch_bounds__(BS) kb_cheb0(M A, int n, const float *__restrict__ dw, const float *__restrict__ b,
                                               float *x, float *__restrict__ r, float *__restrict__ d,
                                               float *__restrict__ xo, float c0, int x0zero,
                                               const float *__restrict__ q, double *part, BlkCtl *c, int mode)
{
    pdl_enter();
    if (bfinished(c)) return;
    Sum2 loc[2][CW];
    BLOCK_ROWS(n, KB, CW)
    {
        CV<float, CW> ax;
#pragma unroll
        for (int u = 0; u < CW; ++u) ax.v[u] = 0.f;
        if (!x0zero) ax = A.template dot<CW>(i, BVec<float, CW, KB>{x + off});
        const size_t e = (size_t)i * KB + off;
        const CV<float, CW> bi = cld<CW>(b + e);
        const float w = dw[i];
        CV<float, CW> ro, dv;
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            ro.v[u] = bi.v[u] - ax.v[u];
            dv.v[u] = c0 * (w * ro.v[u]);
        }
        cst<CW>(r + e, ro);
        cst<CW>(d + e, dv);
        if constexpr (DOT) {
            CV<float, CW> xn;
            if (x0zero) {
                xn = dv;
            } else {
                xn = cld<CW>(x + e);
#pragma unroll
                for (int u = 0; u < CW; ++u) xn.v[u] += dv.v[u];
            }
            cst<CW>(xo + e, xn);
            dot_cols<CW>(b + e, xn, q ? q + e : nullptr, loc);
        } else if (x0zero) {
            cst<CW>(x + e, dv);
        }
    }
    if constexpr (DOT) rz_cols<KB, CW>(loc, part, c, mode);
}

// Chebyshev step k >= 2: r -= A d; dn = c1 d + c2 dw r; x += (add_prev ? d : 0) + dn
template <int KB, int CW, class M, bool DOT>
__global__ void __launch_bounds__(BS) kb_chebk(M A, int n, const float *__restrict__ dw, float *__restrict__ r,
                                               const float *__restrict__ d, float *__restrict__ dn, float *x,
                                               float *__restrict__ xo, float c1, float c2, int add_prev,
                                               const float *__restrict__ b0, const float *__restrict__ q,
                                               double *part, BlkCtl *c, int mode)
{
    pdl_enter();
    if (bfinished(c)) return;
    Sum2 loc[2][CW];
    BLOCK_ROWS(n, KB, CW)
    {
        const CV<float, CW> ad = A.template dot<CW>(i, BVec<float, CW, KB>{d + off});
        const size_t e = (size_t)i * KB + off;
        const CV<float, CW> rv = cld<CW>(r + e), dp = cld<CW>(d + e), xv = cld<CW>(x + e);
        const float w = dw[i];
        CV<float, CW> ro, dv, xn;
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            ro.v[u] = rv.v[u] - ad.v[u];
            dv.v[u] = c1 * dp.v[u] + c2 * (w * ro.v[u]);
            xn.v[u] = xv.v[u] + (add_prev ? dp.v[u] : 0.f) + dv.v[u];
        }
        cst<CW>(r + e, ro);
        cst<CW>(dn + e, dv);
        if constexpr (DOT) {
            cst<CW>(xo + e, xn);
            dot_cols<CW>(b0 + e, xn, q ? q + e : nullptr, loc);
        } else {
            cst<CW>(x + e, xn);
        }
    }
    if constexpr (DOT) rz_cols<KB, CW>(loc, part, c, mode);
}

// damped Jacobi: xo = x + dw (b - A x) (x = null: a zero guess)
template <int KB, int CW, class M, bool DOT>
__global__ void __launch_bounds__(BS) kb_jacobi(M A, int n, const float *__restrict__ dw, const float *__restrict__ b,
                                                const float *__restrict__ x, float *__restrict__ xo,
                                                const float *__restrict__ q, double *part, BlkCtl *c, int mode)
{
    pdl_enter();
    if (bfinished(c)) return;
    Sum2 loc[2][CW];
    BLOCK_ROWS(n, KB, CW)
    {
        CV<float, CW> ax, xv;
#pragma unroll
        for (int u = 0; u < CW; ++u) ax.v[u] = xv.v[u] = 0.f;
        const size_t e = (size_t)i * KB + off;
        if (x) {
            ax = A.template dot<CW>(i, BVec<float, CW, KB>{x + off});
            xv = cld<CW>(x + e);
        }
        const CV<float, CW> bi = cld<CW>(b + e);
        const float w = dw[i];
        CV<float, CW> xn;
#pragma unroll
        for (int u = 0; u < CW; ++u) xn.v[u] = xv.v[u] + w * (bi.v[u] - ax.v[u]);
        cst<CW>(xo + e, xn);
        if constexpr (DOT) dot_cols<CW>(b + e, xn, q ? q + e : nullptr, loc);
    }
    if constexpr (DOT) rz_cols<KB, CW>(loc, part, c, mode);
}

template <int KB>
__global__ void __launch_bounds__(BS) kb_axpy(long long m, const float *__restrict__ d, float *__restrict__ x,
                                              const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    for (long long e = blockIdx.x * (long long)BS + threadIdx.x; e < m; e += (long long)gridDim.x * BS) x[e] += d[e];
}

// r = b - A x
template <int KB, int CW, class M>
__global__ void __launch_bounds__(BS) kb_residual(M A, int n, const float *__restrict__ b, const float *__restrict__ x,
                                                  float *__restrict__ r, const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    BLOCK_ROWS(n, KB, CW)
    {
        const CV<float, CW> ax = A.template dot<CW>(i, BVec<float, CW, KB>{x + off});
        const size_t e = (size_t)i * KB + off;
        CV<float, CW> ro = cld<CW>(b + e);
#pragma unroll
        for (int u = 0; u < CW; ++u) ro.v[u] -= ax.v[u];
        cst<CW>(r + e, ro);
    }
}

// y = R x (restriction)
template <int KB, int CW, class M>
__global__ void __launch_bounds__(BS) kb_spmv(M Rm, int n, const float *__restrict__ x, float *__restrict__ y,
                                              const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    BLOCK_ROWS(n, KB, CW)
    {
        const CV<float, CW> s = Rm.template dot<CW>(i, BVec<float, CW, KB>{x + off});
        int o = i;
        if constexpr (std::is_same<M, BSell<float>>::value) o = Rm.out_row(i);
        cst<CW>(y + (size_t)o * KB + off, s);
    }
}

// x += P e (interpolate and correct)
template <int KB, int CW, class M>
__global__ void __launch_bounds__(BS) kb_prolong(M P, int n, const float *__restrict__ ec, float *__restrict__ x,
                                                 const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    BLOCK_ROWS(n, KB, CW)
    {
        const CV<float, CW> s = P.template dot<CW>(i, BVec<float, CW, KB>{ec + off});
        const size_t e = (size_t)i * KB + off;
        CV<float, CW> xv = cld<CW>(x + e);
#pragma unroll
        for (int u = 0; u < CW; ++u) xv.v[u] += s.v[u];
        cst<CW>(x + e, xv);
    }
}

// x += P e on level 0 with the implicit prolongator (ImplP)
template <int KB, int CW>
__global__ void __launch_bounds__(BS) kb_prolong_imp(const int *__restrict__ agg, const float *__restrict__ s,
                                                     const float *__restrict__ fx, const float *__restrict__ fy,
                                                     const float *__restrict__ fz, int n, int nx, int sxy, float w0,
                                                     const float *__restrict__ ec, float *__restrict__ x,
                                                     const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    BLOCK_ROWS(n, KB, CW)
    {
        const float *eo = ec + off;
        CV<float, CW> acc;
#pragma unroll
        for (int u = 0; u < CW; ++u) acc.v[u] = 0.f;
        if (i >= sxy) cacc(acc, __ldg(fz + i - sxy), cld<CW>(eo + __ldg(agg + i - sxy) * KB));
        if (i >= nx) cacc(acc, __ldg(fy + i - nx), cld<CW>(eo + __ldg(agg + i - nx) * KB));
        if (i >= 1) cacc(acc, __ldg(fx + i - 1), cld<CW>(eo + __ldg(agg + i - 1) * KB));
        if (i + 1 < n) cacc(acc, __ldg(fx + i), cld<CW>(eo + __ldg(agg + i + 1) * KB));
        if (i + nx < n) cacc(acc, __ldg(fy + i), cld<CW>(eo + __ldg(agg + i + nx) * KB));
        if (i + sxy < n) cacc(acc, __ldg(fz + i), cld<CW>(eo + __ldg(agg + i + sxy) * KB));
        const float si = __ldg(s + i), w = si != 0.f ? w0 : 1.f;
        const CV<float, CW> ev = cld<CW>(eo + __ldg(agg + i) * KB);
        const size_t e = (size_t)i * KB + off;
        CV<float, CW> xv = cld<CW>(x + e);
#pragma unroll
        for (int u = 0; u < CW; ++u) xv.v[u] += w * ev.v[u] - si * acc.v[u];
        cst<CW>(x + e, xv);
    }
}

// x = Ainv b on the coarsest level (dense FP64 inverse), one warp per row,
// KB columns at once
template <int KB>
__global__ void __launch_bounds__(BS) kb_coarse(int n, const double *__restrict__ Ainv, const float *__restrict__ b,
                                                float *__restrict__ x, const BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    const int lane = threadIdx.x & 31;
    for (int row = (blockIdx.x * BS + threadIdx.x) >> 5; row < n; row += (gridDim.x * BS) >> 5) {
        const double *a = Ainv + (size_t)row * n;
        double s[KB];
#pragma unroll
        for (int j = 0; j < KB; ++j) s[j] = 0.0;
        for (int k = lane; k < n; k += 32) {
            const double akj = a[k];
            const CV<float, 4> *bb = reinterpret_cast<const CV<float, 4> *>(b + (size_t)k * KB);
#pragma unroll
            for (int h = 0; h < KB / 4; ++h) {
                const CV<float, 4> v = bb[h];
#pragma unroll
                for (int u = 0; u < 4; ++u) s[4 * h + u] += akj * (double)v.v[u];
            }
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) s[j] = warp_sum(s[j]);
        if (lane < KB) {
            double mine = 0.0;
#pragma unroll
            for (int j = 0; j < KB; ++j)
                if (j == lane) mine = s[j];
            x[(size_t)row * KB + lane] = (float)mine;
        }
    }
}

// ------------------------------------------------------------ CG kernels --
// x64 = 0, xs = 0, r = b, both direction buffers 0; per column ||b||^2
template <int KB>
__global__ void __launch_bounds__(BS) kb_init(int n, const double *__restrict__ b, double *__restrict__ x,
                                              float *__restrict__ xs, float *__restrict__ r, float *__restrict__ pa,
                                              float *__restrict__ pb, double *part, BlkCtl *c)
{
    pdl_enter();
    __shared__ double tot[KB];
    double loc[1][1] = {{0.0}};
    BLOCK_ROWS(n, KB, 1)
    {
        const size_t e = (size_t)i * KB + off;
        const double bi = b[e];
        x[e] = 0.0;
        xs[e] = 0.f;
        r[e] = (float)bi;
        pa[e] = 0.f;
        pb[e] = 0.f;
        loc[0][0] += bi * bi;
    }
    if (!reduce_cols<KB, 1, 1>(loc, part, &c->cnt[0], tot)) return;
    if (threadIdx.x < KB) {
        Ctl &cj = c->col[threadIdx.x];
        const double b2 = tot[threadIdx.x];
        cj.bnorm2 = b2;
        cj.rmax2 = b2;
        cj.it = 0;
        cj.check = 0;
        cj.status = isfinite(b2) ? GW_OK : GW_ERR_ARG;  // a non-finite right-hand side entry
        cj.rz = cj.pq = cj.alpha = cj.beta = cj.rr = cj.rt2 = cj.qz = 0.0;
        cj.relres = isfinite(b2) ? (b2 > 0.0 ? 1.0 : 0.0) : b2;
        cj.done = (b2 > 0.0 && isfinite(b2)) ? 0 : 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) refresh_done<KB>(c);
}

// p_new = z + beta p_old (formed where gathered), q = A p_new, pq = (p_new, q),
// alpha = rz / pq per column; a column at maxit stops here
template <int KB, int CW, class M>
__global__ void __launch_bounds__(BS) kb_dir_spmv(M A, int n, const float *__restrict__ z,
                                                  const float *__restrict__ pold, float *__restrict__ pnew,
                                                  float *__restrict__ q, double *part, BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    __shared__ double tot[KB];
    Sum2 acc[1][CW];
    CV<float, CW> beta;  // a thread keeps its columns: the grid stride is a multiple of KB / CW
#pragma unroll
    for (int u = 0; u < CW; ++u) beta.v[u] = (float)c->col[first_col<KB, CW>() + u].beta;
    BLOCK_ROWS(n, KB, CW)
    {
        const BDir<CW, KB> f{z + off, pold + off, beta};
        const CV<float, CW> qi = A.template dot<CW>(i, f);
        const CV<float, CW> pi = f(i);
        const size_t e = (size_t)i * KB + off;
        cst<CW>(q + e, qi);
        cst<CW>(pnew + e, pi);
#pragma unroll
        for (int u = 0; u < CW; ++u) sum2_prod(acc[0][u], pi.v[u], qi.v[u]);
    }
    double loc[1][CW];
    pairs_to_double(acc, loc);
    if (!reduce_cols<KB, CW, 1>(loc, part, &c->cnt[0], tot)) return;
    if (threadIdx.x < KB) {
        Ctl &cj = c->col[threadIdx.x];
        if (!cj.done) {
            if (cj.it >= cj.maxit) {
                col_stop(cj, GW_ERR_NOT_CONVERGED);
            } else {
                const double pq = tot[threadIdx.x];
                cj.pq = pq;
                cj.it += 1;
                if (!(pq > 0.0) || !isfinite(pq)) col_stop(cj, GW_ERR_BREAKDOWN);
                else cj.alpha = cj.rz / pq;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) refresh_done<KB>(c);
}

// xs += alpha p; r -= alpha q; rr = (r, r) per column; a column whose
// recursive residual passes the test, or fell by delta since its last
// reliable update, asks for one
template <int KB, int CW>
__global__ void __launch_bounds__(BS) kb_update(int n, float *__restrict__ xs, float *__restrict__ r,
                                                const float *__restrict__ p, const float *__restrict__ q, double *part,
                                                BlkCtl *c)
{
    pdl_enter();
    if (bfinished(c)) return;
    __shared__ double tot[KB];
    Sum2 acc[1][CW];
    CV<float, CW> a;
#pragma unroll
    for (int u = 0; u < CW; ++u) a.v[u] = (float)c->col[first_col<KB, CW>() + u].alpha;
    BLOCK_ROWS(n, KB, CW)
    {
        const size_t e = (size_t)i * KB + off;
        CV<float, CW> xv = cld<CW>(xs + e), rv = cld<CW>(r + e);
        const CV<float, CW> pv = cld<CW>(p + e), qv = cld<CW>(q + e);
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            xv.v[u] += a.v[u] * pv.v[u];
            rv.v[u] -= a.v[u] * qv.v[u];
            sum2_prod(acc[0][u], rv.v[u], rv.v[u]);
        }
        cst<CW>(xs + e, xv);
        cst<CW>(r + e, rv);
    }
    double loc[1][CW];
    pairs_to_double(acc, loc);
    if (!reduce_cols<KB, CW, 1>(loc, part, &c->cnt[0], tot)) return;
    if (threadIdx.x < KB) {
        Ctl &cj = c->col[threadIdx.x];
        if (!cj.done) {
            const double rr = tot[threadIdx.x];
            cj.rr = rr;
            if (!isfinite(rr)) col_stop(cj, GW_ERR_BREAKDOWN);
            else if (rr <= cj.tol2 * cj.bnorm2 || rr <= cj.delta2 * cj.rmax2) cj.check = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) refresh_done<KB>(c);
}

// reliable update part 1: x64 += xs; xs = 0 (columns asking for it, or all)
template <int KB>
__global__ void __launch_bounds__(BS) kb_rel_fold(int n, double *__restrict__ x, float *__restrict__ xs,
                                                  const BlkCtl *c, int force)
{
    pdl_enter();
    if (!force && (bfinished(c) || !c->any_check)) return;
    if (!force && !c->col[first_col<KB, 1>()].check) return;
    BLOCK_ROWS(n, KB, 1)
    {
        const size_t e = (size_t)i * KB + off;
        x[e] += (double)xs[e];
        xs[e] = 0.f;
    }
}

// reliable update part 2: r = b - A64 x64 in FP64 (stored as FP32) for the
// columns asking for it; a column stops when ||r|| passes, else remembers
// ||r||^2.  force: only the final relative residual of every column.
template <int KB, int CW, class M>
__global__ void __launch_bounds__(BS) kb_rel_res(M A, int n, const double *__restrict__ b,
                                                 const double *__restrict__ x, float *__restrict__ r, double *part,
                                                 BlkCtl *c, int force)
{
    pdl_enter();
    if (!force && (bfinished(c) || !c->any_check)) return;
    __shared__ double tot[KB];
    double loc[1][CW] = {};
    bool act = force != 0, mine[CW];
#pragma unroll
    for (int u = 0; u < CW; ++u) {
        mine[u] = !force && c->col[first_col<KB, CW>() + u].check != 0;
        act |= mine[u];
    }
    BLOCK_ROWS(n, KB, CW)
    {
        if (!act) break;
        const CV<double, CW> ax = A.template dot<CW>(i, BVec<double, CW, KB>{x + off});
        const size_t e = (size_t)i * KB + off;
        const CV<double, CW> bv = cld<CW>(b + e);
#pragma unroll
        for (int u = 0; u < CW; ++u) {
            const double t = bv.v[u] - ax.v[u];
            loc[0][u] += t * t;
            if (mine[u]) r[e + u] = (float)t;
        }
    }
    if (!reduce_cols<KB, CW, 1>(loc, part, &c->cnt[0], tot)) return;
    if (threadIdx.x < KB) {
        Ctl &cj = c->col[threadIdx.x];
        const double rt2 = tot[threadIdx.x];
        if (force) {
            cj.rt2 = rt2;
            cj.relres = cj.bnorm2 > 0.0 ? sqrt(rt2 / cj.bnorm2) : 0.0;
        } else if (cj.check && !cj.done) {
            cj.rt2 = rt2;
            cj.relres = cj.bnorm2 > 0.0 ? sqrt(rt2 / cj.bnorm2) : 0.0;
            if (rt2 <= cj.tol2 * cj.bnorm2) {
                col_stop(cj, GW_OK);
            } else {
                cj.rmax2 = rt2;
                cj.check = 0;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) refresh_done<KB>(c);
}

// column-major n x kk block (column j at B + j*n) <-> interleaved n x KB;
// columns kk..KB-1 of the interleaved block are zero
template <int KB>
__global__ void kb_gather(int n, int kk, const double *__restrict__ B, double *__restrict__ b)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * KB;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / KB), j = (int)(e % KB);
        b[e] = j < kk ? B[(size_t)j * n + i] : 0.0;
    }
}

template <int KB>
__global__ void kb_scatter(int n, int kk, const double *__restrict__ x, double *__restrict__ X)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * kk;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), i = (int)(e % n);
        X[e] = x[(size_t)i * KB + j];
    }
}

// ------------------------------------------------------------------ driver --
struct BlockLevel {
    DBuf<float> x, b, r, d, d2;
};

struct BlockState {
    int kb = 0;  // columns of the captured graphs
    std::vector<BlockLevel> lv;
    DBuf<double> b64, x64, stage, part;
    DBuf<float> xs, r, z, p, pb, q;
    DBuf<BlkCtl> ctl;
    BlkCtl *ctl_host = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t ginit = nullptr, gexec = nullptr;
    long long init_kernels = 0, iter_kernels = 0;
    ~BlockState()
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (ginit) cudaGraphExecDestroy(ginit);
        if (cap) cudaStreamDestroy(cap);
        if (ctl_host) host_free(ctl_host);
    }
};

void block_free(BlockState *s) { delete s; }

void block_drop_graphs(BlockState *s)
{
    if (!s) return;
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->ginit) cudaGraphExecDestroy(s->ginit);
    s->gexec = s->ginit = nullptr;
    s->kb = 0;
}

static constexpr int BGRAPH_ITERS = 4;  // even: the direction buffers alternate

static int bgrid(const Hier &, long long threads) { return blocks_for(threads); }

template <int KB>
struct BCyc {
    static constexpr int CW = 4;  // float columns per thread
    static constexpr int TPR = KB / CW;
    Hier &H;
    BlockState &S;
    BlkCtl *c;
    double *part;
    cudaStream_t st;

    int g(int n) const { return bgrid(H, (long long)n * TPR); }

    // one smoothing application on level l (the single-vector smoother's steps)
    void smooth(int l, const float *b, bool x0zero, bool last, float *zout, const float *q, int mode)
    {
        CycLevel<float> &lv = H.cf[l];
        BlockLevel &bl = S.lv[l];
        const int n = lv.n, nu = std::max(1, H.o.nu);
        with_bmat(lv.A, [&](auto A) {
            using M = decltype(A);
            if (H.o.smoother == GW_SMOOTH_JACOBI) {
                float *cur = bl.x.p, *nxt = bl.r.p;
                for (int s = 0; s < nu; ++s) {
                    const bool first = x0zero && s == 0, fin = last && s == nu - 1;
                    const float *xi = first ? nullptr : cur;
                    if (fin)
                        launch_pdl(kb_jacobi<KB, CW, M, true>, g(n), st, A, n, lv.dw.p, b, xi, zout, q, part, c, mode);
                    else
                        launch_pdl(kb_jacobi<KB, CW, M, false>, g(n), st, A, n, lv.dw.p, b, xi, nxt, q, part, c,
                                   mode);
                    if (!fin) std::swap(cur, nxt);
                }
                if (!last && cur != bl.x.p)
                    GW_CUDA(cudaMemcpyAsync(bl.x.p, cur, (size_t)n * KB * sizeof(float), cudaMemcpyDeviceToDevice,
                                            st));
                return;
            }
            const int m = std::max(1, H.o.degree);
            for (int s = 0; s < nu; ++s) {
                const int zero = x0zero && s == 0;
                const bool fin = last && s == nu - 1;
                float *d = bl.d.p, *dnx = bl.d2.p;
                if (fin && m == 1) {
                    launch_pdl(kb_cheb0<KB, CW, M, true>, g(n), st, A, n, lv.dw.p, b, bl.x.p, bl.r.p, d, zout,
                               (float)lv.c0, zero, q, part, c, mode);
                    continue;
                }
                if (zero && m >= 2) {
                    const bool f2 = fin && m == 2;
                    const int keep = m > 2;
                    if (f2)
                        launch_pdl(kb_cheb_zero2<KB, CW, M, true>, g(n), st, A, n, lv.dw.p, b, bl.x.p, bl.r.p, d,
                                   zout, (float)lv.c0, (float)lv.c1[1], (float)lv.c2[1], keep, q, part, c, mode);
                    else
                        launch_pdl(kb_cheb_zero2<KB, CW, M, false>, g(n), st, A, n, lv.dw.p, b, bl.x.p, bl.r.p, d,
                                   (float *)nullptr, (float)lv.c0, (float)lv.c1[1], (float)lv.c2[1], keep, q, part, c,
                                   mode);
                    for (int k = 2; k < m; ++k) {
                        const bool f3 = fin && k == m - 1;
                        if (f3)
                            launch_pdl(kb_chebk<KB, CW, M, true>, g(n), st, A, n, lv.dw.p, bl.r.p, d, dnx, bl.x.p,
                                       zout, (float)lv.c1[k], (float)lv.c2[k], 0, b, q, part, c, mode);
                        else
                            launch_pdl(kb_chebk<KB, CW, M, false>, g(n), st, A, n, lv.dw.p, bl.r.p, d, dnx, bl.x.p,
                                       (float *)nullptr, (float)lv.c1[k], (float)lv.c2[k], 0, (const float *)nullptr,
                                       q, part, c, mode);
                        std::swap(d, dnx);
                    }
                    continue;
                }
                launch_pdl(kb_cheb0<KB, CW, M, false>, g(n), st, A, n, lv.dw.p, b, bl.x.p, bl.r.p, d,
                           (float *)nullptr, (float)lv.c0, zero, q, part, c, mode);
                if (m == 1) {
                    if (!zero) launch_pdl(kb_axpy<KB>, bgrid(H, (long long)n * KB), st, (long long)n * KB, d, bl.x.p, c);
                    continue;
                }
                for (int k = 1; k < m; ++k) {
                    const bool f2 = fin && k == m - 1;
                    const int add_prev = (k == 1 && !zero) ? 1 : 0;
                    if (f2)
                        launch_pdl(kb_chebk<KB, CW, M, true>, g(n), st, A, n, lv.dw.p, bl.r.p, d, dnx, bl.x.p, zout,
                                   (float)lv.c1[k], (float)lv.c2[k], add_prev, b, q, part, c, mode);
                    else
                        launch_pdl(kb_chebk<KB, CW, M, false>, g(n), st, A, n, lv.dw.p, bl.r.p, d, dnx, bl.x.p,
                                   (float *)nullptr, (float)lv.c1[k], (float)lv.c2[k], add_prev,
                                   (const float *)nullptr, q, part, c, mode);
                    std::swap(d, dnx);
                }
            }
        });
    }

    // z = M^-1 r on KB interleaved columns; the last pass reduces (r, z), (q, z)
    void vcycle(const float *r, float *z, const float *q, int mode)
    {
        const int L = H.L;
        for (int l = 0; l < L - 1; ++l) {
            CycLevel<float> &lv = H.cf[l];
            BlockLevel &bl = S.lv[l];
            const int n = lv.n;
            const float *b = l == 0 ? r : bl.b.p;
            smooth(l, b, true, false, nullptr, q, mode);
            with_bmat(lv.A, [&](auto A) {
                using M = decltype(A);
                launch_pdl(kb_residual<KB, CW, M>, g(n), st, A, n, b, (const float *)bl.x.p, bl.r.p, (const BlkCtl *)c);
            });
            with_bmat(lv.R, [&](auto Rm) {
                using M = decltype(Rm);
                launch_pdl(kb_spmv<KB, CW, M>, g(lv.R.nr), st, Rm, lv.R.nr, (const float *)bl.r.p, S.lv[l + 1].b.p,
                           (const BlkCtl *)c);
            });
        }
        const int nc = H.cf[L - 1].n;
        launch_pdl(kb_coarse<KB>, std::max(1, std::min(H.max_blocks, (nc * 32 + BS - 1) / BS)), st, nc,
                   (const double *)H.Ainv.p, (const float *)S.lv[L - 1].b.p, S.lv[L - 1].x.p, (const BlkCtl *)c);
        for (int l = L - 2; l >= 0; --l) {
            CycLevel<float> &lv = H.cf[l];
            BlockLevel &bl = S.lv[l];
            const int n = lv.n;
            if (l == 0 && H.p0.n) {
                const ImplP &I = H.p0;
                launch_pdl(kb_prolong_imp<KB, CW>, g(n), st, I.agg, (const float *)I.s.p, (const float *)I.fx.p,
                           (const float *)I.fy.p, (const float *)I.fz.p, I.n, I.nx, I.sxy, I.w0,
                           (const float *)S.lv[1].x.p, bl.x.p, (const BlkCtl *)c);
                smooth(l, r, false, true, z, q, mode);
                continue;
            }
            with_bmat(lv.P, [&](auto P) {
                using M = decltype(P);
                launch_pdl(kb_prolong<KB, CW, M>, g(n), st, P, n, (const float *)S.lv[l + 1].x.p, bl.x.p,
                           (const BlkCtl *)c);
            });
            smooth(l, l == 0 ? r : bl.b.p, false, l == 0, z, q, mode);
        }
        GW_LAUNCH_CHECK();
    }

    void rel_update(int force)
    {
        const int n = H.n;
        launch_pdl(kb_rel_fold<KB>, bgrid(H, (long long)n * KB), st, n, S.x64.p, S.xs.p, (const BlkCtl *)c, force);
        with_bmat(H.A64, [&](auto A) {
            using M = decltype(A);
            launch_pdl(kb_rel_res<KB, 2, M>, bgrid(H, (long long)n * (KB / 2)), st, A, n, (const double *)S.b64.p,
                       (const double *)S.x64.p, S.r.p, part, c, force);
        });
    }

    void init()
    {
        const int n = H.n;
        launch_pdl(kb_init<KB>, bgrid(H, (long long)n * KB), st, n, (const double *)S.b64.p, S.x64.p, S.xs.p, S.r.p,
                   S.p.p, S.pb.p, part, c);
        vcycle(S.r.p, S.z.p, nullptr, 0);
    }

    void iteration(int parity)
    {
        const int n = H.n;
        float *pold = parity ? S.pb.p : S.p.p, *pnew = parity ? S.p.p : S.pb.p;
        with_bmat(cg_op32(H), [&](auto A) {
            using M = decltype(A);
            launch_pdl(kb_dir_spmv<KB, CW, M>, g(n), st, A, n, (const float *)S.z.p, (const float *)pold, pnew, S.q.p,
                       part, c);
        });
        launch_pdl(kb_update<KB, CW>, g(n), st, n, S.xs.p, S.r.p, (const float *)pnew, (const float *)S.q.p, part, c);
        rel_update(0);
        vcycle(S.r.p, S.z.p, S.q.p, 1);
    }
};

template <class F>
static cudaGraphExec_t bcapture(BlockState &S, F body, long long *nkernels)
{
    if (!S.cap) GW_CUDA(cudaStreamCreateWithFlags(&S.cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CaptureScope scope;
    GW_CUDA(cudaStreamBeginCapture(S.cap, cudaStreamCaptureModeThreadLocal));
    try {
        body(S.cap);
    } catch (...) {
        cudaStreamEndCapture(S.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    GW_CUDA(cudaStreamEndCapture(S.cap, &g));
    size_t num = 0;
    GW_CUDA(cudaGraphGetNodes(g, nullptr, &num));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    GW_CUDA(e);
    *nkernels = (long long)num;
    return ex;
}

static void ensure_state(Hier &H)
{
    if (H.blk) return;
    std::unique_ptr<BlockState> s(new BlockState());
    const size_t n = (size_t)H.n, m = n * KB_MAX;
    s->lv.resize(H.L);
    for (int l = 0; l < H.L; ++l) {
        const size_t ml = (size_t)H.cf[l].n * KB_MAX;
        BlockLevel &b = s->lv[l];
        if (l > 0) b.b.alloc(ml);
        b.x.alloc(ml);
        if (l < H.L - 1) {
            b.r.alloc(ml);
            b.d.alloc(ml);
            b.d2.alloc(ml);
        }
    }
    s->b64.alloc(m);
    s->x64.alloc(m);
    s->stage.alloc(m);
    s->xs.alloc(m);
    s->r.alloc(m);
    s->z.alloc(m);
    s->p.alloc(m);
    s->pb.alloc(m);
    s->q.alloc(m);
    s->part.alloc((size_t)2 * KB_MAX * RED_MAX_BLOCKS);
    s->ctl.alloc(1);
    GW_CUDA(cudaMemset(s->ctl.p, 0, sizeof(BlkCtl)));
    GW_CUDA(host_malloc((void **)&s->ctl_host, sizeof(BlkCtl)));
    H.blk = s.release();
}

template <int KB>
static void ensure_bgraphs(Hier &H)
{
    BlockState &S = *H.blk;
    if (S.kb == KB && S.ginit && S.gexec) return;
    block_drop_graphs(&S);
    S.ginit = bcapture(S, [&](cudaStream_t s) {
        BCyc<KB>{H, S, S.ctl.p, S.part.p, s}.init();
    }, &S.init_kernels);
    S.gexec = bcapture(S, [&](cudaStream_t s) {
        BCyc<KB> cyc{H, S, S.ctl.p, S.part.p, s};
        for (int k = 0; k < BGRAPH_ITERS; ++k) cyc.iteration(k & 1);
    }, &S.iter_kernels);
    S.kb = KB;
}

// One block of kk <= KB columns: B and X column-major with leading dimension n.
template <int KB>
static void block_run(Hier &H, int kk, const double *B, double *X, double tol, int maxit, int *iters,
                      double *relres, int *status, cudaStream_t st)
{
    ensure_state(H);
    ensure_bgraphs<KB>(H);
    BlockState &S = *H.blk;
    const int n = H.n;
    const size_t cols = (size_t)n * kk * sizeof(double);
    const int gg = std::min(bgrid(H, (long long)n * KB), H.max_blocks);
    const double *Bd = B;
    if (!is_device_ptr(B)) {
        GW_CUDA(cudaMemcpyAsync(S.stage.p, B, cols, cudaMemcpyHostToDevice, st));
        Bd = S.stage.p;
    }
    gw_launch(kb_gather<KB>, gg, BS, 0, st, n, kk, Bd, S.b64.p);
    BlkCtl init;
    memset(&init, 0, sizeof init);
    for (int j = 0; j < KB; ++j) {
        init.col[j].tol2 = tol * tol;
        init.col[j].maxit = maxit;
        init.col[j].flexible = 1;
        init.col[j].delta2 = H.o.delta * H.o.delta;
    }
    *S.ctl_host = init;
    GW_CUDA(cudaMemcpyAsync(S.ctl.p, S.ctl_host, sizeof(BlkCtl), cudaMemcpyHostToDevice, st));
    GW_CUDA(cudaGraphLaunch(S.ginit, st));
    H.launches += S.init_kernels + 1;
    const int max_launches = (maxit + BGRAPH_ITERS - 1) / BGRAPH_ITERS + 2;
    for (int k = 0; k < max_launches; ++k) {
        GW_CUDA(cudaGraphLaunch(S.gexec, st));
        H.launches += S.iter_kernels;
        GW_CUDA(cudaMemcpyAsync(S.ctl_host, S.ctl.p, sizeof(BlkCtl), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
        if (S.ctl_host->done) break;
    }
    // fold what is left of every correction and take the final residuals
    BCyc<KB>{H, S, S.ctl.p, S.part.p, st}.rel_update(1);
    H.launches += 2;
    double *Xd = is_device_ptr(X) ? X : S.stage.p;
    gw_launch(kb_scatter<KB>, gg, BS, 0, st, n, kk, S.x64.p, Xd);
    H.launches += 2;
    GW_LAUNCH_CHECK();
    if (Xd != X) GW_CUDA(cudaMemcpyAsync(X, Xd, cols, cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaMemcpyAsync(S.ctl_host, S.ctl.p, sizeof(BlkCtl), cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < kk; ++j) {
        const Ctl &cj = S.ctl_host->col[j];
        if (iters) iters[j] = cj.it;
        if (relres) relres[j] = cj.relres;
        status[j] = cj.done ? cj.status : GW_ERR_NOT_CONVERGED;
    }
    H.solves += kk;
}

bool block_supported(const Hier &H)
{
    if (H.o.prec != GW_PREC_MIXED32 || H.L < 2) return false;
    return (long long)H.n * KB_MAX <= 0x7fffffffLL;
}

// k columns in blocks of 8 (a last block of 1-4 columns runs 4 wide)
int block_solve(Hier &H, int k, const double *B, double *X, double tol, int maxit, int *iters, double *relres,
                cudaStream_t st)
{
    int worst = GW_OK;
    const size_t n = (size_t)H.n;
    std::vector<int> stat(KB_MAX);
    for (int c0 = 0; c0 < k; c0 += KB_MAX) {
        const int kk = std::min(KB_MAX, k - c0);
        if (kk > 4)
            block_run<8>(H, kk, B + c0 * n, X + c0 * n, tol, maxit, iters ? iters + c0 : nullptr,
                         relres ? relres + c0 : nullptr, stat.data(), st);
        else
            block_run<4>(H, kk, B + c0 * n, X + c0 * n, tol, maxit, iters ? iters + c0 : nullptr,
                         relres ? relres + c0 : nullptr, stat.data(), st);
        for (int j = 0; j < kk; ++j)
            if (stat[j] != GW_OK && worst == GW_OK) worst = stat[j];
    }
    return worst;
}

}  // namespace gw
