// cycle.cu -- the V-cycle preconditioner and the outer conjugate-gradient loop.
//
// V-cycle (Introduction): on each level a smoothing step and the residual,
// restriction of the residual to the next level, a direct solve on the
// coarsest level, interpolation and correction on the way up, and a final
// smoothing step; the passes are sparse matrix-vector products.  The
// smoothers are damped Jacobi (weight 4/3 over the Gershgorin bound) or
// Chebyshev polynomials of D^-1 A (Adams et al. 2003), fused with the residual
// they need.  The coarsest level multiplies by its dense FP64 inverse.
//
// Every kernel is written once against a matrix view: the index-free 7-point
// stencil of level 0, sliced ELL (one thread per row) for short rows, and CSR
// read by groups of 8 or 32 lanes per row for the long rows of the Galerkin
// levels, so small levels still spread over every SM.
//
// CG (Saad, Algorithm 9.1) runs in FP64 with all scalars on the device: dot
// products are reduced deterministically (fixed grid, per-block partial sums,
// the last block to arrive adds them in a fixed order) and every kernel
// leaves at once when the control block says the solve has finished, so a
// captured graph of several iterations can be replayed without a host round
// trip per iteration.
#include <string.h>

#include <memory>

#include "gw_internal.cuh"
#include "kern.cuh"

namespace gw {


// chunks of a sliced-ELL row whose loads the compiler may issue together
#ifndef GW_SELL_UNROLL
#define GW_SELL_UNROLL 1
#endif
constexpr int SELL_UNROLL = GW_SELL_UNROLL;
// chunks of a sliced-ELL row read before their gathers (a thread per row)
#ifndef GW_SELL_BATCH
#define GW_SELL_BATCH 2
#endif
constexpr int SELL_BATCH = GW_SELL_BATCH;

// ------------------------------------------------------------ matrix views --
// R consecutive values handled by one thread (R = 4 floats or 2 doubles is
// one 16-byte load or store).
template <class T, int R>
struct VecN {
    T v[R];
};

template <int R, class T>
__device__ __forceinline__ VecN<T, R> ld_ro(const T *__restrict__ p)
{
    VecN<T, R> o;
    if constexpr (R == 8 && sizeof(T) == 4) {
        const float4 t0 = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 t1 = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        o.v[0] = t0.x, o.v[1] = t0.y, o.v[2] = t0.z, o.v[3] = t0.w;
        o.v[4] = t1.x, o.v[5] = t1.y, o.v[6] = t1.z, o.v[7] = t1.w;
    } else if constexpr (R == 4 && sizeof(T) == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        o.v[0] = t.x, o.v[1] = t.y, o.v[2] = t.z, o.v[3] = t.w;
    } else if constexpr (R == 2 && sizeof(T) == 8) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        o.v[0] = t.x, o.v[1] = t.y;
    } else if constexpr (R == 4 && sizeof(T) == 8) {
        const double2 t0 = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 t1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        o.v[0] = t0.x, o.v[1] = t0.y, o.v[2] = t1.x, o.v[3] = t1.y;
    } else if constexpr (R == 2 && sizeof(T) == 4) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        o.v[0] = t.x, o.v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = __ldg(p + k);
    }
    return o;
}

// coherent load (the array is written by this kernel, each element by its own thread)
template <int R, class T>
__device__ __forceinline__ VecN<T, R> ld_rw(const T *p)
{
    VecN<T, R> o;
    if constexpr (R == 8 && sizeof(T) == 4) {
        const float4 t0 = reinterpret_cast<const float4 *>(p)[0];
        const float4 t1 = reinterpret_cast<const float4 *>(p)[1];
        o.v[0] = t0.x, o.v[1] = t0.y, o.v[2] = t0.z, o.v[3] = t0.w;
        o.v[4] = t1.x, o.v[5] = t1.y, o.v[6] = t1.z, o.v[7] = t1.w;
    } else if constexpr (R == 4 && sizeof(T) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o.v[0] = t.x, o.v[1] = t.y, o.v[2] = t.z, o.v[3] = t.w;
    } else if constexpr (R == 2 && sizeof(T) == 8) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        o.v[0] = t.x, o.v[1] = t.y;
    } else if constexpr (R == 4 && sizeof(T) == 8) {
        const double2 t0 = reinterpret_cast<const double2 *>(p)[0];
        const double2 t1 = reinterpret_cast<const double2 *>(p)[1];
        o.v[0] = t0.x, o.v[1] = t0.y, o.v[2] = t1.x, o.v[3] = t1.y;
    } else if constexpr (R == 2 && sizeof(T) == 4) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        o.v[0] = t.x, o.v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = p[k];
    }
    return o;
}

template <int R, class T>
__device__ __forceinline__ void st(T *p, const VecN<T, R> &o)
{
    if constexpr (R == 8 && sizeof(T) == 4) {
        reinterpret_cast<float4 *>(p)[0] = make_float4(o.v[0], o.v[1], o.v[2], o.v[3]);
        reinterpret_cast<float4 *>(p)[1] = make_float4(o.v[4], o.v[5], o.v[6], o.v[7]);
    } else if constexpr (R == 4 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(o.v[0], o.v[1], o.v[2], o.v[3]);
    } else if constexpr (R == 2 && sizeof(T) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(o.v[0], o.v[1]);
    } else if constexpr (R == 4 && sizeof(T) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(o.v[0], o.v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(o.v[2], o.v[3]);
    } else if constexpr (R == 2 && sizeof(T) == 4) {
        *reinterpret_cast<float2 *>(p) = make_float2(o.v[0], o.v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) p[k] = o.v[k];
    }
}

template <class U, class T, int R>
__device__ __forceinline__ VecN<U, R> cvt(const VecN<T, R> &a)
{
    VecN<U, R> o;
#pragma unroll
    for (int k = 0; k < R; ++k) o.v[k] = (U)a.v[k];
    return o;
}

// gathered operands: p[j] converted to T, and dw[j] * b[j]
template <class T, class S>
struct GVec {
    const S *__restrict__ p;
    __device__ __forceinline__ T operator()(int j) const { return (T)__ldg(p + j); }
    template <int R>
    __device__ __forceinline__ VecN<T, R> vec(int j0) const
    {
        return cvt<T>(ld_ro<R>(p + j0));
    }
};

template <class T, class S>
struct GProd {
    const T *__restrict__ dw;
    const S *__restrict__ b;
    __device__ __forceinline__ T operator()(int j) const { return __ldg(dw + j) * (T)__ldg(b + j); }
    template <int R>
    __device__ __forceinline__ VecN<T, R> vec(int j0) const
    {
        const VecN<T, R> w = ld_ro<R>(dw + j0);
        const VecN<T, R> bb = cvt<T>(ld_ro<R>(b + j0));
        VecN<T, R> o;
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = w.v[k] * bb.v[k];
        return o;
    }
};

// c * dw[j] * b[j]: the first Chebyshev correction from a zero guess
template <class T, class S>
struct GProdC {
    const T *__restrict__ dw;
    const S *__restrict__ b;
    T c;
    __device__ __forceinline__ T operator()(int j) const { return c * (__ldg(dw + j) * (T)__ldg(b + j)); }
    template <int R>
    __device__ __forceinline__ VecN<T, R> vec(int j0) const
    {
        const VecN<T, R> w = ld_ro<R>(dw + j0);
        const VecN<T, R> bb = cvt<T>(ld_ro<R>(b + j0));
        VecN<T, R> o;
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = c * (w.v[k] * bb.v[k]);
        return o;
    }
};

// z[j] + beta * p[j]: the new CG direction, formed where it is gathered
template <class T>
struct GDir {
    const T *__restrict__ z;
    const T *__restrict__ p;
    T beta;
    __device__ __forceinline__ T operator()(int j) const { return __ldg(z + j) + beta * __ldg(p + j); }
    template <int R>
    __device__ __forceinline__ VecN<T, R> vec(int j0) const
    {
        const VecN<T, R> zz = ld_ro<R>(z + j0), pp = ld_ro<R>(p + j0);
        VecN<T, R> o;
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = zz.v[k] + beta * pp.v[k];
        return o;
    }
};

template <class T>
struct SV {
    const int *__restrict__ sp;
    const int *__restrict__ ci;
    const T *__restrict__ v;
    int nr;
    const int *__restrict__ perm;  // row of slot row r (null: r); restriction matrices only
};

template <class T>
struct VecT;
template <>
struct VecT<float> {
    using V = float4;
    using I = int4;
};
template <>
struct VecT<double> {
    using V = double2;
    using I = int2;
};

// Sliced ELL, G lanes per row (lane g of a row takes chunks g, g + G, ...,
// so a warp still reads whole 16-byte vectors of consecutive rows); V slots
// per 16-byte load; every lane of the group gets the sum.
template <class T, int G_ = 1>
struct MSell {
    using value_type = T;
    static constexpr int G = G_, R = 1;
    SV<T> a;
    template <class F>
    __device__ __forceinline__ VecN<T, 1> dot(int r, int lane, F f) const
    {
        using VV = typename VecT<T>::V;
        using VI = typename VecT<T>::I;
        constexpr int V = SellV<T>::V;
        T acc = 0;
        if constexpr (G == 1) {
            // a thread per row: SELL_BATCH chunks' values and columns first,
            // then their gathers, then the products in chunk order, so that
            // a batch's loads are in flight together
            if (r < a.nr || G == 1) {
                const int s = r >> 5, rl = r & 31;
                const int base = a.sp[s];
                const int nch = (a.sp[s + 1] - base) / (SELL_C * V);
                const VV *vv = reinterpret_cast<const VV *>(a.v + base) + rl;
                const VI *cc = reinterpret_cast<const VI *>(a.ci + base) + rl;
                for (int c0 = 0; c0 < nch; c0 += SELL_BATCH) {
                    VV x[SELL_BATCH];
                    VI j[SELL_BATCH];
#pragma unroll
                    for (int b = 0; b < SELL_BATCH; ++b)
                        if (c0 + b < nch) {
                            x[b] = __ldg(vv + (c0 + b) * SELL_C);
                            j[b] = __ldg(cc + (c0 + b) * SELL_C);
                        }
                    T g[SELL_BATCH][V];
#pragma unroll
                    for (int b = 0; b < SELL_BATCH; ++b)
                        if (c0 + b < nch) {
                            if constexpr (V == 4) {
                                g[b][0] = f(j[b].x);
                                g[b][1] = f(j[b].y);
                                g[b][2] = f(j[b].z);
                                g[b][3] = f(j[b].w);
                            } else {
                                g[b][0] = f(j[b].x);
                                g[b][1] = f(j[b].y);
                            }
                        }
#pragma unroll
                    for (int b = 0; b < SELL_BATCH; ++b)
                        if (c0 + b < nch) {
                            if constexpr (V == 4) {
                                acc += x[b].x * g[b][0];
                                acc += x[b].y * g[b][1];
                                acc += x[b].z * g[b][2];
                                acc += x[b].w * g[b][3];
                            } else {
                                acc += x[b].x * g[b][0];
                                acc += x[b].y * g[b][1];
                            }
                        }
                }
            }
            return VecN<T, 1>{{acc}};
        }
        if (G == 1 || r < a.nr) {
            const int s = r >> 5, rl = r & 31;
            const int base = a.sp[s];
            const int nch = (a.sp[s + 1] - base) / (SELL_C * V);
            const VV *vv = reinterpret_cast<const VV *>(a.v + base) + rl;
            const VI *cc = reinterpret_cast<const VI *>(a.ci + base) + rl;
#pragma unroll SELL_UNROLL
            for (int c = (G == 1 ? 0 : lane); c < nch; c += G) {
                const VV x = __ldg(vv + c * SELL_C);
                const VI j = __ldg(cc + c * SELL_C);
                if constexpr (V == 4) {
                    acc += x.x * f(j.x);
                    acc += x.y * f(j.y);
                    acc += x.z * f(j.z);
                    acc += x.w * f(j.w);
                } else {
                    acc += x.x * f(j.x);
                    acc += x.y * f(j.y);
                }
            }
        }
        if constexpr (G > 1) {
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, G);
        }
        return VecN<T, 1>{{acc}};
    }
};

// output row of a row product: the slot row's row for a length-sorted sliced
// ELL, the row itself otherwise
template <class M>
__device__ __forceinline__ int out_row(const M &, int i)
{
    return i;
}
template <class T, int G>
__device__ __forceinline__ int out_row(const MSell<T, G> &m, int i)
{
    return m.a.perm ? __ldg(m.a.perm + i) : i;
}

// CSR read by a group of G lanes per row; every lane of the group gets the sum.
template <class T, int G_>
struct MCsr {
    using value_type = T;
    static constexpr int G = G_, R = 1;
    const int *__restrict__ rp;
    const int *__restrict__ ci;
    const T *__restrict__ v;
    int n;
    template <class F>
    __device__ __forceinline__ VecN<T, 1> dot(int i, int lane, F f) const
    {
        T s = 0;
        if (i < n) {
            const int e1 = rp[i + 1];
            for (int e = rp[i] + lane; e < e1; e += G) s += __ldg(v + e) * f(__ldg(ci + e));
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, G);
        return VecN<T, 1>{{s}};
    }
};

// Index-free 7-point stencil, R consecutive rows per thread (R = 1 for any
// grid; R = 16 bytes / sizeof(T) when nx and n are multiples of R, so every
// coefficient and vector access is one aligned 16-byte load).  Terms are added
// in ascending column order: -z, -y, -x, diagonal, +x, +y, +z.
template <class T, int R_>
struct MSten {
    using value_type = T;
    static constexpr int G = 1, R = R_;
    const T *__restrict__ d;
    const T *__restrict__ ox;
    const T *__restrict__ oy;
    const T *__restrict__ oz;
    int n, nx, sxy;
    template <class F>
    __device__ __forceinline__ VecN<T, R> dot(int i0, int, F f) const
    {
        VecN<T, R> acc;
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] = 0;
        if (i0 >= sxy) {
            const VecN<T, R> c = ld_ro<R>(oz + i0 - sxy);
            const VecN<T, R> x = f.template vec<R>(i0 - sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        if (i0 >= nx) {
            const VecN<T, R> c = ld_ro<R>(oy + i0 - nx);
            const VecN<T, R> x = f.template vec<R>(i0 - nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        const VecN<T, R> cx = ld_ro<R>(ox + i0);
        const VecN<T, R> xc = f.template vec<R>(i0);
        const T cxm = i0 >= 1 ? __ldg(ox + i0 - 1) : T(0);
        const T xm = i0 >= 1 ? f(i0 - 1) : T(0);
        const T xp = i0 + R < n ? f(i0 + R) : T(0);
        acc.v[0] += cxm * xm;
#pragma unroll
        for (int k = 1; k < R; ++k) acc.v[k] += cx.v[k - 1] * xc.v[k - 1];
        const VecN<T, R> dg = ld_ro<R>(d + i0);
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] += dg.v[k] * xc.v[k];
#pragma unroll
        for (int k = 0; k < R - 1; ++k) acc.v[k] += cx.v[k] * xc.v[k + 1];
        acc.v[R - 1] += cx.v[R - 1] * xp;
        if (i0 + nx < n) {
            const VecN<T, R> c = ld_ro<R>(oy + i0);
            const VecN<T, R> x = f.template vec<R>(i0 + nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        if (i0 + sxy < n) {
            const VecN<T, R> c = ld_ro<R>(oz + i0);
            const VecN<T, R> x = f.template vec<R>(i0 + sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        return acc;
    }
};

// R BF16 values (R = 4: one 8-byte load) widened to FP32
template <int R>
__device__ __forceinline__ VecN<float, R> ld_bf(const __nv_bfloat16 *p)
{
    VecN<float, R> o;
    if constexpr (R == 4) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        o.v[0] = __uint_as_float(w.x << 16);
        o.v[1] = __uint_as_float(w.x & 0xffff0000u);
        o.v[2] = __uint_as_float(w.y << 16);
        o.v[3] = __uint_as_float(w.y & 0xffff0000u);
    } else if constexpr (R == 2) {
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(p));
        o.v[0] = __uint_as_float(w << 16);
        o.v[1] = __uint_as_float(w & 0xffff0000u);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = __bfloat162float(p[k]);
    }
    return o;
}

// The level-0 stencil with BF16 couplings and an FP32 diagonal (10 bytes a
// row instead of 16); same row blocking and term order as MSten.
template <int R_>
struct MStenB {
    using value_type = float;
    static constexpr int G = 1, R = R_;
    const float *__restrict__ d;
    const __nv_bfloat16 *__restrict__ ox;
    const __nv_bfloat16 *__restrict__ oy;
    const __nv_bfloat16 *__restrict__ oz;
    int n, nx, sxy;
    template <class F>
    __device__ __forceinline__ VecN<float, R> dot(int i0, int, F f) const
    {
        VecN<float, R> acc;
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] = 0.f;
        if (i0 >= sxy) {
            const VecN<float, R> c = ld_bf<R>(oz + i0 - sxy);
            const VecN<float, R> x = f.template vec<R>(i0 - sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        if (i0 >= nx) {
            const VecN<float, R> c = ld_bf<R>(oy + i0 - nx);
            const VecN<float, R> x = f.template vec<R>(i0 - nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        const VecN<float, R> cx = ld_bf<R>(ox + i0);
        const VecN<float, R> xc = f.template vec<R>(i0);
        const float cxm = i0 >= 1 ? __bfloat162float(ox[i0 - 1]) : 0.f;
        const float xm = i0 >= 1 ? f(i0 - 1) : 0.f;
        const float xp = i0 + R < n ? f(i0 + R) : 0.f;
        acc.v[0] += cxm * xm;
#pragma unroll
        for (int k = 1; k < R; ++k) acc.v[k] += cx.v[k - 1] * xc.v[k - 1];
        const VecN<float, R> dg = ld_ro<R>(d + i0);
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] += dg.v[k] * xc.v[k];
#pragma unroll
        for (int k = 0; k < R - 1; ++k) acc.v[k] += cx.v[k] * xc.v[k + 1];
        acc.v[R - 1] += cx.v[R - 1] * xp;
        if (i0 + nx < n) {
            const VecN<float, R> c = ld_bf<R>(oy + i0);
            const VecN<float, R> x = f.template vec<R>(i0 + nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        if (i0 + sxy < n) {
            const VecN<float, R> c = ld_bf<R>(oz + i0);
            const VecN<float, R> x = f.template vec<R>(i0 + sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * x.v[k];
        }
        return acc;
    }
};

// R FP16 values (R = 4: one 8-byte load) widened to FP32
template <int R>
__device__ __forceinline__ VecN<float, R> ld_h(const __half *p)
{
    VecN<float, R> o;
    if constexpr (R == 4) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        __half2 a, b;
        memcpy(&a, &w.x, sizeof a);
        memcpy(&b, &w.y, sizeof b);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        o.v[0] = fa.x, o.v[1] = fa.y, o.v[2] = fb.x, o.v[3] = fb.y;
    } else if constexpr (R == 2) {
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(p));
        __half2 a;
        memcpy(&a, &w, sizeof a);
        const float2 fa = __half22float2(a);
        o.v[0] = fa.x, o.v[1] = fa.y;
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = __half2float(p[k]);
    }
    return o;
}

// The scaled FP16 stencil (StenH): (A x)_i = sd_i ((1 + dd_i) sd_i x_i +
// sum_j c_ij sd_j x_j), 12 bytes a row; sd is gathered at the neighbours.
// Same row blocking and term order as MSten.
template <int R_>
struct MStenH {
    using value_type = float;
    static constexpr int G = 1, R = R_;
    const float *__restrict__ sd;
    const __half *__restrict__ dd;
    const __half *__restrict__ ox;
    const __half *__restrict__ oy;
    const __half *__restrict__ oz;
    int n, nx, sxy;
    template <class F>
    __device__ __forceinline__ VecN<float, R> dot(int i0, int, F f) const
    {
        VecN<float, R> acc;
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] = 0.f;
        if (i0 >= sxy) {
            const VecN<float, R> c = ld_h<R>(oz + i0 - sxy), s = ld_ro<R>(sd + i0 - sxy);
            const VecN<float, R> x = f.template vec<R>(i0 - sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * (s.v[k] * x.v[k]);
        }
        if (i0 >= nx) {
            const VecN<float, R> c = ld_h<R>(oy + i0 - nx), s = ld_ro<R>(sd + i0 - nx);
            const VecN<float, R> x = f.template vec<R>(i0 - nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * (s.v[k] * x.v[k]);
        }
        const VecN<float, R> cx = ld_h<R>(ox + i0), sc = ld_ro<R>(sd + i0), dg = ld_h<R>(dd + i0);
        const VecN<float, R> xc = f.template vec<R>(i0);
        const float cxm = i0 >= 1 ? __half2float(ox[i0 - 1]) : 0.f;
        const float sxm = i0 >= 1 ? __ldg(sd + i0 - 1) * f(i0 - 1) : 0.f;
        const float sxp = i0 + R < n ? __ldg(sd + i0 + R) * f(i0 + R) : 0.f;
        acc.v[0] += cxm * sxm;
#pragma unroll
        for (int k = 1; k < R; ++k) acc.v[k] += cx.v[k - 1] * (sc.v[k - 1] * xc.v[k - 1]);
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] += (1.f + dg.v[k]) * (sc.v[k] * xc.v[k]);
#pragma unroll
        for (int k = 0; k < R - 1; ++k) acc.v[k] += cx.v[k] * (sc.v[k + 1] * xc.v[k + 1]);
        acc.v[R - 1] += cx.v[R - 1] * sxp;
        if (i0 + nx < n) {
            const VecN<float, R> c = ld_h<R>(oy + i0), s = ld_ro<R>(sd + i0 + nx);
            const VecN<float, R> x = f.template vec<R>(i0 + nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * (s.v[k] * x.v[k]);
        }
        if (i0 + sxy < n) {
            const VecN<float, R> c = ld_h<R>(oz + i0), s = ld_ro<R>(sd + i0 + sxy);
            const VecN<float, R> x = f.template vec<R>(i0 + sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc.v[k] += c.v[k] * (s.v[k] * x.v[k]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) acc.v[k] *= sc.v[k];
        return acc;
    }
};

// rows per thread of the level-0 stencil: 4 (16 bytes of FP32, 32 bytes of
// FP64 per array); 8 FP32 rows per thread measured slower (more registers,
// fewer resident blocks)
template <class T>
constexpr int sten_r()
{
    return 4;
}

// rows longer than this on average are read by GW_SELL_LANES lanes each
constexpr int SELL_LONG_ROW = 12;
#ifndef GW_SELL_LANES
#define GW_SELL_LANES 1
#endif

template <class T, class F>
static void with_mat(const MatStore<T> &M, F f)
{
    switch (M.fmt) {
    case FMT_SELL: {
        const SV<T> sv{M.sell.sp.p, M.sell.ci.p, M.sell.v.p, M.sell.nr, M.sell.perm.p};
        if (M.nnz > (long long)SELL_LONG_ROW * M.nr) f(MSell<T, GW_SELL_LANES>{sv});
        else f(MSell<T, 1>{sv});
        break;
    }
    case FMT_CSR4: f(MCsr<T, 4>{M.csr.rp.p, M.csr.ci.p, M.csr.v.p, M.csr.nr}); break;
    case FMT_CSR8: f(MCsr<T, 8>{M.csr.rp.p, M.csr.ci.p, M.csr.v.p, M.csr.nr}); break;
    case FMT_CSR32: f(MCsr<T, 32>{M.csr.rp.p, M.csr.ci.p, M.csr.v.p, M.csr.nr}); break;
    case FMT_STENH:
        if constexpr (sizeof(T) == 4) {
            const StenH &S = M.stenh;
            const int sxy = S.nx * S.ny;
            if (S.n % 4 == 0 && S.nx % 4 == 0)
                f(MStenH<4>{S.sd.p, S.dd.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
            else if (S.n % 2 == 0 && S.nx % 2 == 0)
                f(MStenH<2>{S.sd.p, S.dd.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
            else
                f(MStenH<1>{S.sd.p, S.dd.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
        } else {
            fail(GW_ERR_SETUP, "an FP16 stencil in an FP64 hierarchy");
        }
        break;
    case FMT_STENB:
        if constexpr (sizeof(T) == 4) {
            const StenB &S = M.stenb;
            const int sxy = S.nx * S.ny;
            if (S.n % 4 == 0 && S.nx % 4 == 0) f(MStenB<4>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
            else if (S.n % 2 == 0 && S.nx % 2 == 0) f(MStenB<2>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
            else f(MStenB<1>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
        } else {
            fail(GW_ERR_SETUP, "a BF16 stencil in an FP64 hierarchy");
        }
        break;
    default: {
        constexpr int RV = sten_r<T>(), RH = RV / 2;
        const StenT<T> &S = M.sten;
        const int sxy = S.nx * S.ny;
        if (S.n % RV == 0 && S.nx % RV == 0)
            f(MSten<T, RV>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
        else if (S.n % RH == 0 && S.nx % RH == 0)
            f(MSten<T, RH>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
        else
            f(MSten<T, 1>{S.d.p, S.ox.p, S.oy.p, S.oz.p, S.n, S.nx, sxy});
    }
    }
}

// Row blocks a thread's loop takes per unrolled step: two for the FP32
// level-0 stencil (the second block's loads then overlap the first's; the
// sliced-ELL and CSR forms measured slower unrolled), one otherwise.
template <class M>
struct RowUnroll {
    static constexpr int v = 1;
};
template <>
struct RowUnroll<MSten<float, 4>> {
    static constexpr int v = 2;
};

// Row blocks of M::R rows handled by groups of M::G lanes.  The loop keeps
// whole warps together (so the group reductions may shuffle); a group whose
// block starts at or past n does no epilogue.
#define GROUP_ROWS(M, n)                                                                                  \
    const int lane = M::G == 1 ? 0 : (int)(threadIdx.x & (M::G - 1));                                    \
    _Pragma("unroll (RowUnroll<M>::v)")                                                                  \
    for (int i = (int)((vb.bid * (long long)BS + threadIdx.x) / M::G) * M::R,                             \
             stride_ = vb.nb * (BS / M::G) * M::R;                                                        \
         M::G == 1 ? (i < (n)) : __any_sync(0xffffffffu, i < (n)); i += stride_)

// blocks asked for by a pass over n rows (launch_pdl fits them to one wave)
template <class M>
static inline int grid_for(const Hier &, long long n)
{
    long long groups = (n + M::R - 1) / M::R;
    return blocks_for(groups * M::G);
}

static inline int vgrid(const Hier &, long long n) { return blocks_for(n); }


// ------------------------------------------------------- V-cycle kernels --
// Epilogue of the last kernel of a preconditioner application inside CG:
// rz = (r, z); mode 1 also forms beta (flexible: -alpha (q,z) / rz_old).
__device__ __forceinline__ void cg_rz_epilogue(VB vb, double lrz, double lqz, double *part, Ctl *c, int mode)
{
    if (!c) return;
    double loc[2] = {lrz, lqz}, tot[2];
    if (reduce_last<2>(vb, loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        const double rz_new = tot[0];
        if (mode == 1) {
            const double beta = c->flexible ? -c->alpha * tot[1] / c->rz : rz_new / c->rz;
            c->beta = beta;
            if (!isfinite(beta) || !isfinite(rz_new)) {
                ctl_stop(c, GW_ERR_BREAKDOWN);
            }
        }
        c->rz = rz_new;
    }
}

// (b, z) and (q, z) contributions of R rows: products summed in T over the
// R rows, then accumulated in FP64 across rows and threads
template <int R, class T, class OT>
__device__ __forceinline__ void dot_rows(int i, const T *b, const OT (&z)[R], const T *q, DAcc &lrz, DAcc &lqz)
{
    const VecN<T, R> bb = ld_ro<R>(b + i);
    T zz[R];
#pragma unroll
    for (int k = 0; k < R; ++k) zz[k] = (T)z[k];
    dot_add<R>(lrz, bb.v, zz);
    if (q) {
        const VecN<T, R> qq = ld_ro<R>(q + i);
        dot_add<R>(lqz, qq.v, zz);
    }
}

// x = dw * b ; r = b - A x   (first Jacobi step from zero, fused with the residual)
template <class M, class BT>
__device__ __forceinline__ void b_jac0_res(VB vb, M A, int n, const typename M::value_type *__restrict__ dw,
                                                 const BT *__restrict__ b, typename M::value_type *__restrict__ x,
                                                 typename M::value_type *__restrict__ r, const Ctl *ctl) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    GROUP_ROWS(M, n)
    {
        const VecN<T, R> ax = A.dot(i, lane, GProd<T, BT>{dw, b});
        if (i < n && lane == 0) {
            const VecN<T, R> bi = cvt<T>(ld_ro<R>(b + i));
            const VecN<T, R> w = ld_ro<R>(dw + i);
            VecN<T, R> xo, ro;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                xo.v[k] = w.v[k] * bi.v[k];
                ro.v[k] = bi.v[k] - ax.v[k];
            }
            st<R>(x + i, xo);
            st<R>(r + i, ro);
        }
    }
}

template <class M, class BT>
__global__ void __launch_bounds__(BS) k_jac0_res(M A, int n, const typename M::value_type *__restrict__ dw,
                                                 const BT *__restrict__ b, typename M::value_type *__restrict__ x,
                                                 typename M::value_type *__restrict__ r, const Ctl *ctl)
{
    pdl_enter();
    b_jac0_res<M, BT>(vb_grid(), A, n, dw, b, x, r, ctl);
}

// xo = xi + dw * (b - A xi); xi == nullptr means xi = 0.  With DOT, xo is the
// CG's z (double) and (b, z) [and (q, z)] are reduced.
template <class M, class BT, class OT, bool DOT>
__device__ __forceinline__ void b_jacobi(VB vb, M A, int n, const typename M::value_type *__restrict__ dw,
                                               const BT *__restrict__ b, const typename M::value_type *__restrict__ xi,
                                               OT *__restrict__ xo, const typename M::value_type *__restrict__ q,
                                               double *part, Ctl *ctl, int mode) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    DAcc lrz, lqz;
    GROUP_ROWS(M, n)
    {
        VecN<T, R> ax;
        if (xi) ax = A.dot(i, lane, GVec<T, T>{xi});
        if (i < n && lane == 0) {
            const VecN<T, R> bi = cvt<T>(ld_ro<R>(b + i));
            const VecN<T, R> w = ld_ro<R>(dw + i);
            VecN<T, R> xv;
            if (xi) xv = ld_ro<R>(xi + i);
            OT out[R];
            VecN<OT, R> o;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const T xn = xi ? xv.v[k] + w.v[k] * (bi.v[k] - ax.v[k]) : w.v[k] * bi.v[k];
                o.v[k] = (OT)xn;
                out[k] = (OT)xn;
            }
            st<R>(xo + i, o);
            if constexpr (DOT) dot_rows<R>(i, b, out, q, lrz, lqz);
        }
    }
    if constexpr (DOT) cg_rz_epilogue(vb, dacc_value(lrz), dacc_value(lqz), part, ctl, mode);
}

template <class M, class BT, class OT, bool DOT>
__global__ void __launch_bounds__(BS) k_jacobi(M A, int n, const typename M::value_type *__restrict__ dw,
                                               const BT *__restrict__ b, const typename M::value_type *__restrict__ xi,
                                               OT *__restrict__ xo, const typename M::value_type *__restrict__ q,
                                               double *part, Ctl *ctl, int mode)
{
    pdl_enter();
    b_jacobi<M, BT, OT, DOT>(vb_grid(), A, n, dw, b, xi, xo, q, part, ctl, mode);
}

// r = b - A x
template <class M, class BT>
__device__ __forceinline__ void b_residual(VB vb, M A, int n, const BT *__restrict__ b,
                                                 const typename M::value_type *__restrict__ x,
                                                 typename M::value_type *__restrict__ r, const Ctl *ctl) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    GROUP_ROWS(M, n)
    {
        const VecN<T, R> ax = A.dot(i, lane, GVec<T, T>{x});
        if (i < n && lane == 0) {
            const VecN<T, R> bi = cvt<T>(ld_ro<R>(b + i));
            VecN<T, R> ro;
#pragma unroll
            for (int k = 0; k < R; ++k) ro.v[k] = bi.v[k] - ax.v[k];
            st<R>(r + i, ro);
        }
    }
}

template <class M, class BT>
__global__ void __launch_bounds__(BS) k_residual(M A, int n, const BT *__restrict__ b,
                                                 const typename M::value_type *__restrict__ x,
                                                 typename M::value_type *__restrict__ r, const Ctl *ctl)
{
    pdl_enter();
    b_residual<M, BT>(vb_grid(), A, n, b, x, r, ctl);
}

// y = R x (restriction)
template <class M>
__device__ __forceinline__ void b_spmv(VB vb, M Rm, int n, const typename M::value_type *__restrict__ x,
                                             typename M::value_type *__restrict__ y, const Ctl *ctl) {
    using T = typename M::value_type;
    if (finished(ctl)) return;
    GROUP_ROWS(M, n)
    {
        const VecN<T, M::R> s = Rm.dot(i, lane, GVec<T, T>{x});
        if (i < n && lane == 0) {
            if constexpr (M::R == 1) y[out_row(Rm, i)] = s.v[0];
            else st<M::R>(y + i, s);
        }
    }
}

template <class M>
__global__ void __launch_bounds__(BS) k_spmv(M Rm, int n, const typename M::value_type *__restrict__ x,
                                             typename M::value_type *__restrict__ y, const Ctl *ctl)
{
    pdl_enter();
    b_spmv<M>(vb_grid(), Rm, n, x, y, ctl);
}

// x += P e (interpolate and correct)
template <class M>
__device__ __forceinline__ void b_prolong(VB vb, M P, int n, const typename M::value_type *__restrict__ e,
                                                typename M::value_type *__restrict__ x, const Ctl *ctl) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    GROUP_ROWS(M, n)
    {
        const VecN<T, R> s = P.dot(i, lane, GVec<T, T>{e});
        if (i < n && lane == 0) {
            VecN<T, R> xv = ld_rw<R>(x + i);
#pragma unroll
            for (int k = 0; k < R; ++k) xv.v[k] += s.v[k];
            st<R>(x + i, xv);
        }
    }
}

template <class M>
__global__ void __launch_bounds__(BS) k_prolong(M P, int n, const typename M::value_type *__restrict__ e,
                                                typename M::value_type *__restrict__ x, const Ctl *ctl)
{
    pdl_enter();
    b_prolong<M>(vb_grid(), P, n, e, x, ctl);
}

// x += P e on level 0 with the implicit prolongator (ImplP), R rows a thread:
// x_i += w_i e[agg_i] - s_i sum_j f_ij e[agg_j], neighbours in the order
// -z, -y, -x, +x, +y, +z
template <int R>
__device__ __forceinline__ VecN<int, R> ld_int(const int *__restrict__ p)
{
    VecN<int, R> o;
    if constexpr (R == 4) {
        const int4 t = __ldg(reinterpret_cast<const int4 *>(p));
        o.v[0] = t.x, o.v[1] = t.y, o.v[2] = t.z, o.v[3] = t.w;
    } else if constexpr (R == 2) {
        const int2 t = __ldg(reinterpret_cast<const int2 *>(p));
        o.v[0] = t.x, o.v[1] = t.y;
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) o.v[k] = __ldg(p + k);
    }
    return o;
}

struct PImpl {
    const int *__restrict__ agg;
    const float *__restrict__ s;
    const float *__restrict__ fx;
    const float *__restrict__ fy;
    const float *__restrict__ fz;
    int n, nx, sxy;
    float w0;
};

template <int R>
__device__ __forceinline__ void b_prolong_imp(VB vb, PImpl P, const float *__restrict__ e, float *__restrict__ x,
                                                    const Ctl *ctl) {
    if (finished(ctl)) return;
    const int n = P.n, nx = P.nx, sxy = P.sxy;
    for (int i0 = R * (vb.bid * BS + threadIdx.x); i0 < n; i0 += R * vb.nb * BS) {
        // every aggregate id first, then every gather of e, so that the loads
        // of the six neighbours are in flight together; the sums keep the
        // order -z, -y, -x, +x, +y, +z
        const bool zm = i0 >= sxy, ym = i0 >= nx, xm = i0 >= 1, xp = i0 + R < n, yp = i0 + nx < n,
                   zp = i0 + sxy < n;
        const VecN<int, R> ai = ld_int<R>(P.agg + i0);
        VecN<int, R> azm, aym, ayp, azp;
        int axm = 0, axp = 0;
        if (zm) azm = ld_int<R>(P.agg + i0 - sxy);
        if (ym) aym = ld_int<R>(P.agg + i0 - nx);
        if (xm) axm = __ldg(P.agg + i0 - 1);
        if (xp) axp = __ldg(P.agg + i0 + R);
        if (yp) ayp = ld_int<R>(P.agg + i0 + nx);
        if (zp) azp = ld_int<R>(P.agg + i0 + sxy);
        VecN<float, R> ev, ezm, eym, eyp, ezp;
        float exm = 0.f, exp_ = 0.f;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            ev.v[k] = __ldg(e + ai.v[k]);
            ezm.v[k] = zm ? __ldg(e + azm.v[k]) : 0.f;
            eym.v[k] = ym ? __ldg(e + aym.v[k]) : 0.f;
            eyp.v[k] = yp ? __ldg(e + ayp.v[k]) : 0.f;
            ezp.v[k] = zp ? __ldg(e + azp.v[k]) : 0.f;
        }
        if (xm) exm = __ldg(e + axm);
        if (xp) exp_ = __ldg(e + axp);
        float acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = 0.f;
        if (zm) {
            const VecN<float, R> c = ld_ro<R>(P.fz + i0 - sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * ezm.v[k];
        }
        if (ym) {
            const VecN<float, R> c = ld_ro<R>(P.fy + i0 - nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * eym.v[k];
        }
        const VecN<float, R> cx = ld_ro<R>(P.fx + i0);
        if (xm) acc[0] += __ldg(P.fx + i0 - 1) * exm;
#pragma unroll
        for (int k = 1; k < R; ++k) acc[k] += cx.v[k - 1] * ev.v[k - 1];
#pragma unroll
        for (int k = 0; k < R - 1; ++k) acc[k] += cx.v[k] * ev.v[k + 1];
        if (xp) acc[R - 1] += cx.v[R - 1] * exp_;
        if (yp) {
            const VecN<float, R> c = ld_ro<R>(P.fy + i0);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * eyp.v[k];
        }
        if (zp) {
            const VecN<float, R> c = ld_ro<R>(P.fz + i0);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * ezp.v[k];
        }
        const VecN<float, R> sv = ld_ro<R>(P.s + i0);
        VecN<float, R> xv = ld_rw<R>(x + i0);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float w = sv.v[k] != 0.f ? P.w0 : 1.f;
            xv.v[k] += w * ev.v[k] - sv.v[k] * acc[k];
        }
        st<R>(x + i0, xv);
    }
}

template <int R>
__global__ void __launch_bounds__(BS) k_prolong_imp(PImpl P, const float *__restrict__ e, float *__restrict__ x,
                                                    const Ctl *ctl)
{
    pdl_enter();
    b_prolong_imp<R>(vb_grid(), P, e, x, ctl);
}

// u_j = w_j r_j - sum_i f_ij s_i r_i over the six neighbours (the first half
// of r_c = (P^T r)_c on level 0), R rows a thread, neighbours in the order
// -z, -y, -x, +x, +y, +z
template <int R>
__device__ __forceinline__ void b_restrict_u(VB vb, PImpl P, const float *__restrict__ r, float *__restrict__ u,
                                                   const Ctl *ctl) {
    if (finished(ctl)) return;
    const int n = P.n, nx = P.nx, sxy = P.sxy;
    for (int i0 = R * (vb.bid * BS + threadIdx.x); i0 < n; i0 += R * vb.nb * BS) {
        float acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = 0.f;
        if (i0 >= sxy) {
            const VecN<float, R> c = ld_ro<R>(P.fz + i0 - sxy), sv = ld_ro<R>(P.s + i0 - sxy),
                                 rv = ld_ro<R>(r + i0 - sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * (sv.v[k] * rv.v[k]);
        }
        if (i0 >= nx) {
            const VecN<float, R> c = ld_ro<R>(P.fy + i0 - nx), sv = ld_ro<R>(P.s + i0 - nx),
                                 rv = ld_ro<R>(r + i0 - nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * (sv.v[k] * rv.v[k]);
        }
        const VecN<float, R> s0 = ld_ro<R>(P.s + i0), r0 = ld_ro<R>(r + i0), cx = ld_ro<R>(P.fx + i0);
        if (i0 >= 1) acc[0] += __ldg(P.fx + i0 - 1) * (__ldg(P.s + i0 - 1) * __ldg(r + i0 - 1));
#pragma unroll
        for (int k = 1; k < R; ++k) acc[k] += cx.v[k - 1] * (s0.v[k - 1] * r0.v[k - 1]);
#pragma unroll
        for (int k = 0; k < R - 1; ++k) acc[k] += cx.v[k] * (s0.v[k + 1] * r0.v[k + 1]);
        if (i0 + R < n) acc[R - 1] += cx.v[R - 1] * (__ldg(P.s + i0 + R) * __ldg(r + i0 + R));
        if (i0 + nx < n) {
            const VecN<float, R> c = ld_ro<R>(P.fy + i0), sv = ld_ro<R>(P.s + i0 + nx), rv = ld_ro<R>(r + i0 + nx);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * (sv.v[k] * rv.v[k]);
        }
        if (i0 + sxy < n) {
            const VecN<float, R> c = ld_ro<R>(P.fz + i0), sv = ld_ro<R>(P.s + i0 + sxy),
                                 rv = ld_ro<R>(r + i0 + sxy);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] += c.v[k] * (sv.v[k] * rv.v[k]);
        }
        VecN<float, R> uo;
#pragma unroll
        for (int k = 0; k < R; ++k) uo.v[k] = (s0.v[k] != 0.f ? P.w0 : 1.f) * r0.v[k] - acc[k];
        st<R>(u + i0, uo);
    }
}

template <int R>
__global__ void __launch_bounds__(BS) k_restrict_u(PImpl P, const float *__restrict__ r, float *__restrict__ u,
                                                   const Ctl *ctl)
{
    pdl_enter();
    b_restrict_u<R>(vb_grid(), P, r, u, ctl);
}

// r_c = sum of u over the members of aggregate c: four lanes per aggregate,
// lane g adding members g, g + 4, ... in order, then a fixed shuffle tree.
// A lane takes its members RS_CHUNK at a time: the member indices first, then
// the gathered u values, then the additions in order, so that the loads of a
// chunk are in flight together instead of one dependent pair per member.
constexpr int RS_LANES = 4, RS_CHUNK = 4;
__device__ __forceinline__ void b_restrict_sum(VB vb, int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                                                     const float *__restrict__ u, float *__restrict__ rc,
                                                     const Ctl *ctl) {
    if (finished(ctl)) return;
    const int g = threadIdx.x & (RS_LANES - 1);
    for (int c = (int)((vb.bid * (long long)BS + threadIdx.x) / RS_LANES), stride = vb.nb * (BS / RS_LANES);
         __any_sync(0xffffffffu, c < nc); c += stride) {
        float acc = 0.f;
        if (c < nc) {
            const int e1 = __ldg(mptr + c + 1);
            for (int e = __ldg(mptr + c) + g; e < e1; e += RS_LANES * RS_CHUNK) {
                int m[RS_CHUNK];
                float v[RS_CHUNK];
#pragma unroll
                for (int k = 0; k < RS_CHUNK; ++k) m[k] = e + k * RS_LANES < e1 ? __ldg(mem + e + k * RS_LANES) : -1;
#pragma unroll
                for (int k = 0; k < RS_CHUNK; ++k) v[k] = m[k] >= 0 ? __ldg(u + m[k]) : 0.f;
#pragma unroll
                for (int k = 0; k < RS_CHUNK; ++k)
                    if (m[k] >= 0) acc += v[k];
            }
        }
#pragma unroll
        for (int off = RS_LANES / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, RS_LANES);
        if (c < nc && g == 0) rc[c] = acc;
    }
}

__global__ void __launch_bounds__(BS) k_restrict_sum(int nc, const int *__restrict__ mptr, const int *__restrict__ mem,
                                                     const float *__restrict__ u, float *__restrict__ rc,
                                                     const Ctl *ctl)
{
    pdl_enter();
    b_restrict_sum(vb_grid(), nc, mptr, mem, u, rc, ctl);
}

static void restrict_imp(Hier &H, const float *r, float *u, float *rc, const Ctl *ctl, cudaStream_t st)
{
    const ImplP &I = H.p0;
    const PImpl P{I.agg, I.s.p, I.fx.p, I.fy.p, I.fz.p, I.n, I.nx, I.sxy, I.w0};
    if (I.n % 4 == 0 && I.nx % 4 == 0) launch_pdl(k_restrict_u<4>, vgrid(H, I.n / 4), st, P, r, u, ctl);
    else launch_pdl(k_restrict_u<1>, vgrid(H, I.n), st, P, r, u, ctl);
    launch_pdl(k_restrict_sum, vgrid(H, (long long)I.nc * RS_LANES), st, I.nc, (const int *)I.mptr.p, (const int *)I.mem.p, (const float *)u,
               rc, ctl);
}

static void prolong_imp(Hier &H, const float *e, float *x, const Ctl *ctl, cudaStream_t st)
{
    const ImplP &I = H.p0;
    const PImpl P{I.agg, I.s.p, I.fx.p, I.fy.p, I.fz.p, I.n, I.nx, I.sxy, I.w0};
    if (I.n % 4 == 0 && I.nx % 4 == 0) launch_pdl(k_prolong_imp<4>, vgrid(H, I.n / 4), st, P, e, x, ctl);
    else launch_pdl(k_prolong_imp<1>, vgrid(H, I.n), st, P, e, x, ctl);
}

// x = Ainv b on the coarsest level (dense FP64 inverse), one warp per row
template <class T>
__device__ __forceinline__ void b_coarse(VB vb, int n, const double *__restrict__ Ainv, const T *__restrict__ b,
                                               T *__restrict__ x, const Ctl *ctl) {
    if (finished(ctl)) return;
    const int lane = threadIdx.x & 31;
    for (int row = (vb.bid * BS + threadIdx.x) >> 5; row < n; row += (vb.nb * BS) >> 5) {
        const double *a = Ainv + (size_t)row * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s += a[j] * (double)b[j];
        s = warp_sum(s);
        if (lane == 0) x[row] = (T)s;
    }
}

template <class T>
__global__ void __launch_bounds__(BS) k_coarse(int n, const double *__restrict__ Ainv, const T *__restrict__ b,
                                               T *__restrict__ x, const Ctl *ctl)
{
    pdl_enter();
    b_coarse<T>(vb_grid(), n, Ainv, b, x, ctl);
}

// Chebyshev first step: r = b - A x (r = b when x0zero), d = c0 dw r.  x is
// gathered here, so it is not written in place: with x0zero x = d; otherwise
// the next step (or k_axpy) adds d.  DOT: xo = x + d is the CG's z.
template <class M, class BT, class OT, bool DOT>
__device__ __forceinline__ void b_cheb0(VB vb, M A, int n, const typename M::value_type *__restrict__ dw,
                                              const BT *__restrict__ b, typename M::value_type *x,
                                              typename M::value_type *__restrict__ r,
                                              typename M::value_type *__restrict__ d, OT *__restrict__ xo,
                                              typename M::value_type c0, int x0zero,
                                              const typename M::value_type *__restrict__ q, double *part, Ctl *ctl,
                                              int mode) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    DAcc lrz, lqz;
    GROUP_ROWS(M, n)
    {
        VecN<T, R> ax;
#pragma unroll
        for (int k = 0; k < R; ++k) ax.v[k] = 0;
        if (!x0zero) ax = A.dot(i, lane, GVec<T, T>{x});
        if (i < n && lane == 0) {
            const VecN<T, R> bi = cvt<T>(ld_ro<R>(b + i));
            const VecN<T, R> w = ld_ro<R>(dw + i);
            VecN<T, R> ro, dv, xv;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                ro.v[k] = bi.v[k] - ax.v[k];
                dv.v[k] = c0 * (w.v[k] * ro.v[k]);
            }
            st<R>(r + i, ro);
            st<R>(d + i, dv);
            if constexpr (DOT) {
                if (!x0zero) xv = ld_rw<R>(x + i);
                OT out[R];
                VecN<OT, R> o;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const T xn = (x0zero ? (T)0 : xv.v[k]) + dv.v[k];
                    o.v[k] = (OT)xn;
                    out[k] = (OT)xn;
                }
                st<R>(xo + i, o);
                dot_rows<R>(i, b, out, q, lrz, lqz);
            } else {
                if (x0zero) st<R>(x + i, dv);
            }
        }
    }
    if constexpr (DOT) cg_rz_epilogue(vb, dacc_value(lrz), dacc_value(lqz), part, ctl, mode);
}

template <class M, class BT, class OT, bool DOT>
__global__ void __launch_bounds__(BS) k_cheb0(M A, int n, const typename M::value_type *__restrict__ dw,
                                              const BT *__restrict__ b, typename M::value_type *x,
                                              typename M::value_type *__restrict__ r,
                                              typename M::value_type *__restrict__ d, OT *__restrict__ xo,
                                              typename M::value_type c0, int x0zero,
                                              const typename M::value_type *__restrict__ q, double *part, Ctl *ctl,
                                              int mode)
{
    pdl_enter();
    b_cheb0<M, BT, OT, DOT>(vb_grid(), A, n, dw, b, x, r, d, xo, c0, x0zero, q, part, ctl, mode);
}

// Chebyshev step k >= 2: r -= A d; dn = c1 d + c2 dw r; x += (add_prev ? d : 0) + dn
template <class M, class OT, bool DOT>
__device__ __forceinline__ void b_chebk(VB vb, M A, int n, const typename M::value_type *__restrict__ dw,
                                              typename M::value_type *__restrict__ r,
                                              const typename M::value_type *__restrict__ d,
                                              typename M::value_type *__restrict__ dn, typename M::value_type *x,
                                              OT *__restrict__ xo, typename M::value_type c1,
                                              typename M::value_type c2, int add_prev,
                                              const typename M::value_type *__restrict__ b0,
                                              const typename M::value_type *__restrict__ q, double *part, Ctl *ctl,
                                              int mode) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    DAcc lrz, lqz;
    GROUP_ROWS(M, n)
    {
        const VecN<T, R> ad = A.dot(i, lane, GVec<T, T>{d});
        if (i < n && lane == 0) {
            const VecN<T, R> rv = ld_rw<R>(r + i);
            const VecN<T, R> dp = ld_ro<R>(d + i);
            const VecN<T, R> w = ld_ro<R>(dw + i);
            const VecN<T, R> xv = ld_rw<R>(x + i);
            VecN<T, R> ro, dv, xn;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                ro.v[k] = rv.v[k] - ad.v[k];
                dv.v[k] = c1 * dp.v[k] + c2 * (w.v[k] * ro.v[k]);
                xn.v[k] = xv.v[k] + (add_prev ? dp.v[k] : (T)0) + dv.v[k];
            }
            st<R>(r + i, ro);
            st<R>(dn + i, dv);
            if constexpr (DOT) {
                OT out[R];
                VecN<OT, R> o;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    o.v[k] = (OT)xn.v[k];
                    out[k] = (OT)xn.v[k];
                }
                st<R>(xo + i, o);
                dot_rows<R>(i, b0, out, q, lrz, lqz);
            } else {
                st<R>(x + i, xn);
            }
        }
    }
    if constexpr (DOT) cg_rz_epilogue(vb, dacc_value(lrz), dacc_value(lqz), part, ctl, mode);
}

template <class M, class OT, bool DOT>
__global__ void __launch_bounds__(BS) k_chebk(M A, int n, const typename M::value_type *__restrict__ dw,
                                              typename M::value_type *__restrict__ r,
                                              const typename M::value_type *__restrict__ d,
                                              typename M::value_type *__restrict__ dn, typename M::value_type *x,
                                              OT *__restrict__ xo, typename M::value_type c1,
                                              typename M::value_type c2, int add_prev,
                                              const typename M::value_type *__restrict__ b0,
                                              const typename M::value_type *__restrict__ q, double *part, Ctl *ctl,
                                              int mode)
{
    pdl_enter();
    b_chebk<M, OT, DOT>(vb_grid(), A, n, dw, r, d, dn, x, xo, c1, c2, add_prev, b0, q, part, ctl, mode);
}

// The first two Chebyshev steps from a zero guess in one pass: with
// d0 = c0 dw b (formed where gathered), r1 = b - A d0, d1 = c1 d0 + c2 dw r1,
// x = d0 + d1.  r1 and d1 are stored only when more steps follow (keep).
// DOT: x is the CG's z and (b, z), (q, z) are reduced.
template <class M, class OT, bool DOT>
__device__ __forceinline__ void b_cheb_zero2(VB vb, M A, int n, const typename M::value_type *__restrict__ dw,
                                                   const typename M::value_type *__restrict__ b,
                                                   typename M::value_type *__restrict__ x,
                                                   typename M::value_type *__restrict__ r,
                                                   typename M::value_type *__restrict__ d, OT *__restrict__ xo,
                                                   typename M::value_type c0, typename M::value_type c1,
                                                   typename M::value_type c2, int keep,
                                                   const typename M::value_type *__restrict__ q, double *part,
                                                   Ctl *ctl, int mode) {
    using T = typename M::value_type;
    constexpr int R = M::R;
    if (finished(ctl)) return;
    DAcc lrz, lqz;
    GROUP_ROWS(M, n)
    {
        const VecN<T, R> ad = A.dot(i, lane, GProdC<T, T>{dw, b, c0});
        if (i < n && lane == 0) {
            const VecN<T, R> bi = ld_ro<R>(b + i);
            const VecN<T, R> w = ld_ro<R>(dw + i);
            VecN<T, R> rv, dv, xv;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const T d0 = c0 * (w.v[k] * bi.v[k]);
                rv.v[k] = bi.v[k] - ad.v[k];
                dv.v[k] = c1 * d0 + c2 * (w.v[k] * rv.v[k]);
                xv.v[k] = d0 + dv.v[k];
            }
            if (keep) {
                st<R>(r + i, rv);
                st<R>(d + i, dv);
            }
            if constexpr (DOT) {
                OT out[R];
                VecN<OT, R> o;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    o.v[k] = (OT)xv.v[k];
                    out[k] = (OT)xv.v[k];
                }
                st<R>(xo + i, o);
                dot_rows<R>(i, b, out, q, lrz, lqz);
            } else {
                st<R>(x + i, xv);
            }
        }
    }
    if constexpr (DOT) cg_rz_epilogue(vb, dacc_value(lrz), dacc_value(lqz), part, ctl, mode);
}

template <class M, class OT, bool DOT>
__global__ void __launch_bounds__(BS) k_cheb_zero2(M A, int n, const typename M::value_type *__restrict__ dw,
                                                   const typename M::value_type *__restrict__ b,
                                                   typename M::value_type *__restrict__ x,
                                                   typename M::value_type *__restrict__ r,
                                                   typename M::value_type *__restrict__ d, OT *__restrict__ xo,
                                                   typename M::value_type c0, typename M::value_type c1,
                                                   typename M::value_type c2, int keep,
                                                   const typename M::value_type *__restrict__ q, double *part,
                                                   Ctl *ctl, int mode)
{
    pdl_enter();
    b_cheb_zero2<M, OT, DOT>(vb_grid(), A, n, dw, b, x, r, d, xo, c0, c1, c2, keep, q, part, ctl, mode);
}

template <class T>
__device__ __forceinline__ void b_axpy(VB vb, int n, const T *__restrict__ d, T *__restrict__ x, const Ctl *ctl) {
    if (finished(ctl)) return;
    for (int i = vb.bid * BS + threadIdx.x; i < n; i += vb.nb * BS) x[i] += d[i];
}

template <class T>
__global__ void __launch_bounds__(BS) k_axpy(int n, const T *__restrict__ d, T *__restrict__ x, const Ctl *ctl)
{
    pdl_enter();
    b_axpy<T>(vb_grid(), n, d, x, ctl);
}

// ---------------------------------------------------------- V-cycle driver --
// Algorithmic bytes of each launch (every array counted once, a gathered
// vector once, padding slots not counted) are added to H.prof_bytes while a
// profiled graph is captured.
static inline double vbytes(const Hier &H, double b) { return H.prof_capture ? b : 0.0; }

static void mark_begin(Hier &H, int kind, cudaStream_t st)
{
    if (!H.prof_capture) return;
    Hier::Mark m;
    m.kind = kind;
    m.iter = H.cap_iter;
    m.bytes = 0.0;
    GW_CUDA(cudaEventCreate(&m.a));
    GW_CUDA(cudaEventCreate(&m.b));
    GW_CUDA(cudaEventRecordWithFlags(m.a, st, cudaEventRecordExternal));
    H.marks.push_back(m);
    H.prof_bytes = 0.0;
}

static void mark_end(Hier &H, cudaStream_t st)
{
    if (!H.prof_capture) return;
    Hier::Mark &m = H.marks.back();
    GW_CUDA(cudaEventRecordWithFlags(m.b, st, cudaEventRecordExternal));
    m.bytes = H.prof_bytes;
}

// bytes of the matrix itself: values + indices (none for the stencil)
template <class T>
static double mat_bytes(const MatStore<T> &M)
{
    if (M.fmt == FMT_STEN) return 4.0 * M.nr * sizeof(T);
    if (M.fmt == FMT_STENB) return 10.0 * M.nr;
    if (M.fmt == FMT_STENH) return 12.0 * M.nr;
    return (double)M.nnz * (sizeof(T) + 4.0);
}

// Runs one launch, bracketed by profiling events of the given kind (kind < 0:
// not profiled).  The launch's algorithmic bytes are added inside.
template <class F>
static void timed(Hier &H, int kind, cudaStream_t st, F f)
{
    if (kind >= 0) mark_begin(H, kind, st);
    f();
    if (kind >= 0) mark_end(H, st);
}

// One smoothing application on level l.  k1/k2: profiling kinds of the first
// kernel and of the following ones (-1: not profiled).
template <class T>
static void smooth(Hier &H, std::vector<CycLevel<T>> &C, int l, const T *b, bool x0zero, bool last, T *zout,
                   Ctl *ctl, const T *q, int mode, int k1, int k2, cudaStream_t st)
{
    CycLevel<T> &lv = C[l];
    const int nu = std::max(1, H.o.nu);
    double *part = H.part.p;
    const int n = lv.n;
    const double dn = n, sx = sizeof(T);
    const double amat = mat_bytes(lv.A);
    int launched = 0;
    auto kind = [&]() { return launched++ == 0 ? k1 : k2; };
    with_mat(lv.A, [&](auto A) {
        using M = decltype(A);
        const int g = grid_for<M>(H, n);
        if (H.o.smoother == GW_SMOOTH_JACOBI) {
            T *cur = lv.x.p, *nxt = lv.t.p;
            for (int s = 0; s < nu; ++s) {
                const bool first = x0zero && s == 0;
                const bool fin = last && s == nu - 1;
                const T *xi = first ? nullptr : cur;
                timed(H, kind(), st, [&] {
                    H.prof_bytes += vbytes(H, (first ? 0.0 : amat + dn * sx) + 3.0 * dn * sx + (fin && q ? dn * sx : 0.0));
                    if (fin)
                        launch_pdl(k_jacobi<M, T, T, true>, g, st, A, n, lv.dw.p, b, xi, zout, q, part, ctl, mode);
                    else
                        launch_pdl(k_jacobi<M, T, T, false>, g, st, A, n, lv.dw.p, b, xi, nxt, q, part, ctl, mode);
                });
                if (!fin) std::swap(cur, nxt);
            }
            if (cur != lv.x.p)
                GW_CUDA(cudaMemcpyAsync(lv.x.p, cur, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, st));
            return;
        }
        // Chebyshev of degree m, nu times
        const int m = std::max(1, H.o.degree);
        for (int s = 0; s < nu; ++s) {
            const int zero = x0zero && s == 0;
            const bool fin = last && s == nu - 1;
            T *d = lv.d.p, *dnx = lv.d2.p;
            const double b0 = 2.0 * dn * sx + (zero ? 0.0 : amat + dn * sx);
            if (fin && m == 1) {
                timed(H, kind(), st, [&] {
                    H.prof_bytes += vbytes(H, b0 + 3.0 * dn * sx + (q ? dn * sx : 0.0));
                    launch_pdl(k_cheb0<M, T, T, true>, g, st, A, n, lv.dw.p, b, lv.x.p, lv.r.p, d, zout, (T)lv.c0,
                               zero, q, part, ctl, mode);
                });
                continue;
            }
            if (zero && m >= 2) {
                // first two steps from zero fused: x = d0 + d1
                const bool f2 = fin && m == 2;
                const int keep = m > 2;
                timed(H, kind(), st, [&] {
                    H.prof_bytes += vbytes(H, amat + 2.0 * dn * sx + (keep ? 3.0 : 1.0) * dn * sx +
                                                  (f2 ? dn * sx * (q ? 2.0 : 1.0) : 0.0));
                    if (f2)
                        launch_pdl(k_cheb_zero2<M, T, true>, g, st, A, n, lv.dw.p, b, lv.x.p, lv.r.p, d, zout,
                                   (T)lv.c0, (T)lv.c1[1], (T)lv.c2[1], keep, q, part, ctl, mode);
                    else
                        launch_pdl(k_cheb_zero2<M, T, false>, g, st, A, n, lv.dw.p, b, lv.x.p, lv.r.p, d,
                                   (T *)nullptr, (T)lv.c0, (T)lv.c1[1], (T)lv.c2[1], keep, q, part, ctl, mode);
                });
                for (int k = 2; k < m; ++k) {
                    const bool f3 = fin && k == m - 1;
                    timed(H, kind(), st, [&] {
                        H.prof_bytes += vbytes(H, amat + dn * sx * 7.0 + (f3 ? dn * sx * (q ? 2.0 : 1.0) : 0.0));
                        if (f3)
                            launch_pdl(k_chebk<M, T, true>, g, st, A, n, lv.dw.p, lv.r.p, d, dnx, lv.x.p, zout,
                                       (T)lv.c1[k], (T)lv.c2[k], 0, b, q, part, ctl, mode);
                        else
                            launch_pdl(k_chebk<M, T, false>, g, st, A, n, lv.dw.p, lv.r.p, d, dnx, lv.x.p,
                                       (T *)nullptr, (T)lv.c1[k], (T)lv.c2[k], 0, (const T *)nullptr, q, part, ctl,
                                       mode);
                    });
                    std::swap(d, dnx);
                }
                continue;
            }
            timed(H, kind(), st, [&] {
                H.prof_bytes += vbytes(H, b0 + (zero ? 3.0 : 2.0) * dn * sx);
                launch_pdl(k_cheb0<M, T, T, false>, g, st, A, n, lv.dw.p, b, lv.x.p, lv.r.p, d, (T *)nullptr,
                           (T)lv.c0, zero, q, part, ctl, mode);
            });
            if (m == 1) {
                if (!zero)
                    timed(H, kind(), st, [&] {
                        H.prof_bytes += vbytes(H, 3.0 * dn * sx);
                        launch_pdl(k_axpy<T>, vgrid(H, n), st, n, d, lv.x.p, ctl);
                    });
                continue;
            }
            for (int k = 1; k < m; ++k) {
                const bool f2 = fin && k == m - 1;
                const int add_prev = (k == 1 && !zero) ? 1 : 0;
                timed(H, kind(), st, [&] {
                    H.prof_bytes += vbytes(H, amat + dn * sx * 7.0 + (f2 ? dn * sx * (q ? 2.0 : 1.0) : 0.0));
                    if (f2)
                        launch_pdl(k_chebk<M, T, true>, g, st, A, n, lv.dw.p, lv.r.p, d, dnx, lv.x.p, zout,
                                   (T)lv.c1[k], (T)lv.c2[k], add_prev, b, q, part, ctl, mode);
                    else
                        launch_pdl(k_chebk<M, T, false>, g, st, A, n, lv.dw.p, lv.r.p, d, dnx, lv.x.p, (T *)nullptr,
                                   (T)lv.c1[k], (T)lv.c2[k], add_prev, (const T *)nullptr, q, part, ctl, mode);
                });
                std::swap(d, dnx);
            }
        }
    });
}

// One V-cycle z = M^-1 r on the hierarchy stored in T; r and z are level-0
// vectors in T.  With ctl, the last kernel reduces (r, z) (and (q, z)).
// Level-0 kernels are profiled one by one; the coarser levels as three
// groups (level 1 down, levels >= 2, level 1 up).
template <class T>
static void vcycle_t(Hier &H, std::vector<CycLevel<T>> &C, const T *r, T *z, Ctl *ctl, const T *q, int mode,
                     cudaStream_t st)
{
    const int L = H.L;
    if (L == 1) fail(GW_ERR_SETUP, "a one-level hierarchy is not supported by the V-cycle");
    const double sx = sizeof(T);
    for (int l = 0; l < L - 1; ++l) {
        CycLevel<T> &lv = C[l];
        const int n = lv.n;
        const double dn = n, amat = mat_bytes(lv.A);
        const T *bl = l == 0 ? r : lv.b.p;
        const bool l0 = l == 0;
        if (H.o.smoother == GW_SMOOTH_JACOBI && H.o.nu <= 1) {
            timed(H, l0 ? GW_PK_PRE1 : -1, st, [&] {
                H.prof_bytes += vbytes(H, amat + 4.0 * dn * sx);
                with_mat(lv.A, [&](auto A) {
                    using M = decltype(A);
                    launch_pdl(k_jac0_res<M, T>, grid_for<M>(H, n), st, A, n, lv.dw.p, bl, lv.x.p, lv.r.p, ctl);
                });
            });
        } else {
            smooth<T>(H, C, l, bl, true, false, nullptr, ctl, q, mode, l0 ? GW_PK_PRE1 : -1, l0 ? GW_PK_PRE2 : -1,
                      st);
            timed(H, l0 ? GW_PK_RESID : -1, st, [&] {
                H.prof_bytes += vbytes(H, amat + 3.0 * dn * sx);
                with_mat(lv.A, [&](auto A) {
                    using M = decltype(A);
                    launch_pdl(k_residual<M, T>, grid_for<M>(H, n), st, A, n, bl, lv.x.p, lv.r.p, ctl);
                });
            });
        }
        timed(H, l0 ? GW_PK_RESTRICT : -1, st, [&] {
            if constexpr (sizeof(T) == 4) {
                if (l0 && H.p0.n) {
                    // u pass: r, s, fx, fy, fz read, u written; sum pass: mem and u read,
                    // mptr read and r_c written per aggregate
                    H.prof_bytes += vbytes(H, 24.0 * dn + 8.0 * dn + 8.0 * (double)H.p0.nc);
                    restrict_imp(H, lv.r.p, lv.t.p, C[1].b.p, ctl, st);
                    return;
                }
            }
            H.prof_bytes += vbytes(H, mat_bytes(lv.R) + dn * sx + (double)lv.R.nr * sx);
            with_mat(lv.R, [&](auto Rm) {
                using M = decltype(Rm);
                launch_pdl(k_spmv<M>, grid_for<M>(H, lv.R.nr), st, Rm, lv.R.nr, lv.r.p, C[l + 1].b.p, ctl);
            });
        });
        GW_LAUNCH_CHECK();
        if (l == 0) {
            mark_begin(H, L > 2 ? GW_PK_L1DOWN : GW_PK_DEEP, st);
        } else if (l == 1) {
            mark_end(H, st);
            mark_begin(H, GW_PK_DEEP, st);
        }
    }
    {
        CycLevel<T> &lc = C[L - 1];
        H.prof_bytes += vbytes(H, (double)lc.n * lc.n * 8.0 + 2.0 * lc.n * sx);
        launch_pdl(k_coarse<T>, std::max(1, std::min(H.max_blocks, (lc.n * 32 + BS - 1) / BS)), st, lc.n, H.Ainv.p,
                   lc.b.p, lc.x.p, ctl);
    }
    for (int l = L - 2; l >= 0; --l) {
        CycLevel<T> &lv = C[l];
        const int n = lv.n;
        const double dn = n;
        const bool l0 = l == 0;
        if (l == 1) {
            mark_end(H, st);
            mark_begin(H, GW_PK_L1UP, st);
        }
        if (l == 0) mark_end(H, st);
        timed(H, l0 ? GW_PK_PROLONG : -1, st, [&] {
            if constexpr (sizeof(T) == 4) {
                if (l0 && H.p0.n) {
                    // s, fx, fy, fz, agg once, the coarse vector once, x read and written
                    H.prof_bytes += vbytes(H, 20.0 * dn + (double)C[1].n * sx + 2.0 * dn * sx);
                    prolong_imp(H, C[1].x.p, lv.x.p, ctl, st);
                    return;
                }
            }
            H.prof_bytes += vbytes(H, mat_bytes(lv.P) + (double)lv.P.nc * sx + 2.0 * dn * sx);
            with_mat(lv.P, [&](auto P) {
                using M = decltype(P);
                launch_pdl(k_prolong<M>, grid_for<M>(H, n), st, P, n, C[l + 1].x.p, lv.x.p, ctl);
            });
        });
        smooth<T>(H, C, l, l == 0 ? r : lv.b.p, false, l == 0, z, ctl, q, mode, l0 ? GW_PK_POST1 : -1,
                  l0 ? GW_PK_POST2 : -1, st);
        GW_LAUNCH_CHECK();
    }
}

template <class A, class B>
__global__ void k_convert(int n, const A *__restrict__ a, B *__restrict__ b)
{
    pdl_enter();
    ROWS(i, n) b[i] = (B)a[i];
}

// Standalone V-cycle on FP64 vectors (the mixed hierarchy converts in and out).
void vcycle_enqueue(Hier &H, const double *r, double *z, Ctl *ctl, bool dot, cudaStream_t st)
{
    (void)dot;
    if (H.o.prec == GW_PREC_FP64) {
        vcycle_t<double>(H, H.cd, r, z, ctl, nullptr, 0, st);
        return;
    }
    const int n = H.n;
    launch_pdl(k_convert<double, float>, vgrid(H, n), st, n, r, H.r32.p);
    vcycle_t<float>(H, H.cf, H.r32.p, H.z32.p, ctl, nullptr, 0, st);
    launch_pdl(k_convert<float, double>, vgrid(H, n), st, n, H.z32.p, z);
    GW_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- CG kernels --
// Two forms share these kernels.  FP64: every vector and the matrix of the
// CG recurrence in FP64.  Mixed: the CG recurrence (p, q, r, z and the
// correction xs) runs in FP32 against the FP32 level-0 operator, dot
// products are summed in FP64 across threads, and the solution is kept in
// FP64 by reliable updates (van der Vorst & Ye 2000): whenever the recursive
// residual has dropped by the factor delta since the last update, or passes
// the stopping test, xs is folded into the FP64 solution and the residual is
// recomputed as b - A x with the FP64 operator in FP64 arithmetic.

// x = 0, r = b (FP64 form) or x64 = 0, xs = 0, r32 = b (mixed form), both
// direction buffers 0, beta = 0; ||b||^2
template <class V>
__global__ void __launch_bounds__(BS) k_cg_init(int n, const double *__restrict__ b, double *__restrict__ x,
                                                V *__restrict__ xs, V *__restrict__ r, V *__restrict__ pa,
                                                V *__restrict__ pb, double *part, Ctl *c)
{
    pdl_enter();
    double loc[1] = {0.0}, tot[1];
    ROWS(i, n)
    {
        const double bi = b[i];
        x[i] = 0.0;
        if (xs) xs[i] = (V)0;
        r[i] = (V)bi;
        pa[i] = (V)0;
        pb[i] = (V)0;
        loc[0] += bi * bi;
    }
    if (reduce_last<1>(loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        c->bnorm2 = tot[0];
        c->rmax2 = tot[0];
        c->it = 0;
        c->check = 0;
        const bool fin = isfinite(tot[0]);  // false: b has a non-finite entry
        c->status = GW_OK;
        c->done = 0;
        c->rz = c->pq = c->alpha = c->beta = c->rr = c->rt2 = c->qz = 0.0;
        c->relres = fin ? (tot[0] > 0.0 ? 1.0 : 0.0) : tot[0];
        if (!fin) ctl_stop(c, GW_ERR_ARG);
        else if (!(tot[0] > 0.0)) ctl_stop(c, GW_OK);
    }
}

template <class V>
__global__ void __launch_bounds__(BS) k_copy(int n, const V *__restrict__ a, V *__restrict__ b, const Ctl *c)
{
    pdl_enter();
    if (finished(c)) return;
    ROWS(i, n) b[i] = a[i];
}

// q = A p, pq = (p, q); alpha = rz / pq
template <class M>
__global__ void __launch_bounds__(BS) k_cg_spmv_dot(M A, int n, const typename M::value_type *__restrict__ p,
                                                    typename M::value_type *__restrict__ q, double *part, Ctl *c)
{
    const VB vb = vb_grid();
    pdl_enter();
    using V = typename M::value_type;
    constexpr int R = M::R;
    if (finished(c)) return;
    if (c->it >= c->maxit) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ctl_stop(c, GW_ERR_NOT_CONVERGED);
        }
        return;
    }
    double loc[1] = {0.0}, tot[1];
    GROUP_ROWS(M, n)
    {
        const VecN<V, R> qi = A.dot(i, lane, GVec<V, V>{p});
        if (i < n && lane == 0) {
            st<R>(q + i, qi);
            const VecN<V, R> pi = ld_ro<R>(p + i);
            V s = 0;
#pragma unroll
            for (int k = 0; k < R; ++k) s += pi.v[k] * qi.v[k];
            loc[0] += (double)s;
        }
    }
    if (reduce_last<1>(loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        c->pq = pq;
        c->it += 1;
        if (!(pq > 0.0) || !isfinite(pq)) {
            ctl_stop(c, GW_ERR_BREAKDOWN);
        } else {
            c->alpha = c->rz / pq;
        }
    }
}

// The direction update fused into the product: p_new = z + beta p_old (formed
// where gathered, stored for the own rows), q = A p_new, pq = (p_new, q),
// alpha = rz / pq.  The direction lives in two buffers that swap roles every
// iteration: p_old is pa in even iterations (c->it even at the start) and pb
// in odd ones, p_new the other one.
template <class M>
__device__ __forceinline__ void b_cg_dir_spmv(VB vb, M A, int n, const typename M::value_type *__restrict__ z,
                                                    typename M::value_type *pa, typename M::value_type *pb,
                                                    typename M::value_type *__restrict__ q, double *part, Ctl *c) {
    using V = typename M::value_type;
    constexpr int R = M::R;
    if (finished(c)) return;
    const int odd = c->it & 1;
    const V *__restrict__ pold = odd ? pb : pa;
    V *__restrict__ pnew = odd ? pa : pb;
    if (c->it >= c->maxit) {
        if (vb.bid == 0 && threadIdx.x == 0) {
            ctl_stop(c, GW_ERR_NOT_CONVERGED);
        }
        return;
    }
    const V beta = (V)c->beta;
    DAcc acc;
    GROUP_ROWS(M, n)
    {
        const VecN<V, R> qi = A.dot(i, lane, GDir<V>{z, pold, beta});
        if (i < n && lane == 0) {
            st<R>(q + i, qi);
            const VecN<V, R> pi = GDir<V>{z, pold, beta}.template vec<R>(i);
            st<R>(pnew + i, pi);
            dot_add<R>(acc, pi.v, qi.v);
        }
    }
    double loc[1] = {dacc_value(acc)}, tot[1];
    if (reduce_last<1>(vb, loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        c->pq = pq;
        c->it += 1;
        if (!(pq > 0.0) || !isfinite(pq)) {
            ctl_stop(c, GW_ERR_BREAKDOWN);
        } else {
            c->alpha = c->rz / pq;
        }
    }
}

template <class M>
__global__ void __launch_bounds__(BS) k_cg_dir_spmv(M A, int n, const typename M::value_type *__restrict__ z,
                                                    typename M::value_type *pa, typename M::value_type *pb,
                                                    typename M::value_type *__restrict__ q, double *part, Ctl *c)
{
    pdl_enter();
    b_cg_dir_spmv<M>(vb_grid(), A, n, z, pa, pb, q, part, c);
}

// x += alpha p; r -= alpha q; rr = (r, r).  Sets check when r passes the
// stopping test, or (mixed form) when it fell below delta times the residual
// of the last reliable update.  With pb, p is the new direction of the two
// alternating buffers (pb after an even iteration, pa after an odd one).
template <class V, int R>
__device__ __forceinline__ void b_cg_update(VB vb, int n, V *__restrict__ x, V *__restrict__ r, const V *pa,
                                                  const V *pb, const V *__restrict__ q, double *part, Ctl *c,
                                                  int reliable) {
    if (finished(c)) return;
    const V *__restrict__ p = (pb && !((c->it - 1) & 1)) ? pb : pa;
    const V a = (V)c->alpha;
    DAcc acc;
    // two of the thread's row groups per step, all their loads issued first
    // (the second group's loads no longer wait for the first's); the groups
    // are added to the dot in the same order as one at a time
    const int stride = R * vb.nb * BS;
    for (int i = R * (vb.bid * BS + threadIdx.x); i < n; i += 2 * stride) {
        const int i2 = i + stride;
        const bool two = i2 < n;
        VecN<V, R> xv = ld_rw<R>(x + i), rv = ld_rw<R>(r + i), xv2, rv2;
        const VecN<V, R> pv = ld_ro<R>(p + i), qv = ld_ro<R>(q + i);
        VecN<V, R> pv2, qv2;
        if (two) {
            xv2 = ld_rw<R>(x + i2);
            rv2 = ld_rw<R>(r + i2);
            pv2 = ld_ro<R>(p + i2);
            qv2 = ld_ro<R>(q + i2);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            xv.v[k] += a * pv.v[k];
            rv.v[k] -= a * qv.v[k];
        }
        dot_add<R>(acc, rv.v, rv.v);
        st<R>(x + i, xv);
        st<R>(r + i, rv);
        if (two) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                xv2.v[k] += a * pv2.v[k];
                rv2.v[k] -= a * qv2.v[k];
            }
            dot_add<R>(acc, rv2.v, rv2.v);
            st<R>(x + i2, xv2);
            st<R>(r + i2, rv2);
        }
    }
    double loc[1] = {dacc_value(acc)}, tot[1];
    if (reduce_last<1>(vb, loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        c->rr = tot[0];
        if (!isfinite(tot[0])) {
            ctl_stop(c, GW_ERR_BREAKDOWN);
        } else if (tot[0] <= c->tol2 * c->bnorm2 || (reliable && tot[0] <= c->delta2 * c->rmax2)) {
            c->check = 1;
        }
    }
}

template <class V, int R>
__global__ void __launch_bounds__(BS) k_cg_update(int n, V *__restrict__ x, V *__restrict__ r, const V *pa,
                                                  const V *pb, const V *__restrict__ q, double *part, Ctl *c,
                                                  int reliable)
{
    pdl_enter();
    b_cg_update<V, R>(vb_grid(), n, x, r, pa, pb, q, part, c, reliable);
}

// FP64 form: when the recursive residual passed, r = b - A x; stop if it passes too
template <class M>
__global__ void __launch_bounds__(BS) k_cg_true(M A, int n, const double *__restrict__ b, const double *__restrict__ x,
                                                double *__restrict__ r, double *part, Ctl *c, int force)
{
    const VB vb = vb_grid();
    pdl_enter();
    constexpr int R = M::R;
    if (!force && finished(c)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl_end_loop(c);
        return;
    }
    if (!force && !c->check) return;
    double loc[1] = {0.0}, tot[1];
    GROUP_ROWS(M, n)
    {
        const VecN<double, R> ax = A.dot(i, lane, GVec<double, double>{x});
        if (i < n && lane == 0) {
            const VecN<double, R> bv = ld_ro<R>(b + i);
            VecN<double, R> rv;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                rv.v[k] = bv.v[k] - ax.v[k];
                loc[0] += rv.v[k] * rv.v[k];
            }
            if (!force && r) st<R>(r + i, rv);
        }
    }
    if (reduce_last<1>(loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        c->rt2 = tot[0];
        const double rel = c->bnorm2 > 0.0 ? sqrt(tot[0] / c->bnorm2) : 0.0;
        if (force) {
            c->relres = rel;
        } else if (tot[0] <= c->tol2 * c->bnorm2) {
            c->relres = rel;
            ctl_stop(c, GW_OK);
            ctl_end_loop(c);
        } else {
            c->check = 0;
        }
    }
}

// mixed form, reliable update part 1: x64 += xs; xs = 0
template <int R>
__device__ __forceinline__ void b_rel_fold(VB vb, int n, double *__restrict__ x, float *__restrict__ xs, const Ctl *c,
                                                 int force) {
    if (!force && (finished(c) || !c->check)) return;
    for (int i = R * (vb.bid * BS + threadIdx.x); i < n; i += R * vb.nb * BS) {
        VecN<double, R> xv = ld_rw<R>(x + i);
        const VecN<float, R> sv = ld_rw<R>(xs + i);
        VecN<float, R> zero;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            xv.v[k] += (double)sv.v[k];
            zero.v[k] = 0.f;
        }
        st<R>(x + i, xv);
        st<R>(xs + i, zero);
    }
}

template <int R>
__global__ void __launch_bounds__(BS) k_rel_fold(int n, double *__restrict__ x, float *__restrict__ xs, const Ctl *c,
                                                 int force)
{
    pdl_enter();
    b_rel_fold<R>(vb_grid(), n, x, xs, c, force);
}

// mixed form, reliable update part 2: r = b - A64 x64 in FP64, stored as FP32;
// stop if ||r|| passes the test, else remember ||r||^2 for the next update
template <class M>
__device__ __forceinline__ void b_rel_res(VB vb, M A, int n, const double *__restrict__ b, const double *__restrict__ x,
                                                float *__restrict__ r, double *part, Ctl *c, int force) {
    constexpr int R = M::R;
    if (!force && finished(c)) {
        if (vb.bid == 0 && threadIdx.x == 0) ctl_end_loop(c);
        return;
    }
    if (!force && !c->check) return;
    double loc[1] = {0.0}, tot[1];
    GROUP_ROWS(M, n)
    {
        const VecN<double, R> ax = A.dot(i, lane, GVec<double, double>{x});
        if (i < n && lane == 0) {
            const VecN<double, R> bv = ld_ro<R>(b + i);
            VecN<float, R> rv;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const double t = bv.v[k] - ax.v[k];
                rv.v[k] = (float)t;
                loc[0] += t * t;
            }
            if (!force) st<R>(r + i, rv);
        }
    }
    if (reduce_last<1>(vb, loc, part, &c->cnt[0], tot) && threadIdx.x == 0) {
        c->rt2 = tot[0];
        const double rel = c->bnorm2 > 0.0 ? sqrt(tot[0] / c->bnorm2) : 0.0;
        c->relres = rel;
        if (!force) {
            if (tot[0] <= c->tol2 * c->bnorm2) {
                ctl_stop(c, GW_OK);
                ctl_end_loop(c);
            } else {
                c->rmax2 = tot[0];
                c->check = 0;
            }
        }
    }
}

template <class M>
__global__ void __launch_bounds__(BS) k_rel_res(M A, int n, const double *__restrict__ b, const double *__restrict__ x,
                                                float *__restrict__ r, double *part, Ctl *c, int force)
{
    pdl_enter();
    b_rel_res<M>(vb_grid(), A, n, b, x, r, part, c, force);
}

// p = z + beta p
template <class V, int R>
__global__ void __launch_bounds__(BS) k_cg_p(int n, const V *__restrict__ z, V *__restrict__ p, const Ctl *c)
{
    pdl_enter();
    if (finished(c)) return;
    const V beta = (V)c->beta;
    for (int i = R * (blockIdx.x * BS + threadIdx.x); i < n; i += R * gridDim.x * BS) {
        const VecN<V, R> zv = ld_ro<R>(z + i);
        VecN<V, R> pv = ld_rw<R>(p + i);
#pragma unroll
        for (int k = 0; k < R; ++k) pv.v[k] = zv.v[k] + beta * pv.v[k];
        st<R>(p + i, pv);
    }
}

// ------------------------------------------------------------------ CG loop --
static const MatStore<double> &fine64(Hier &H) { return H.o.prec == GW_PREC_FP64 ? H.cd[0].A : H.A64; }

// pb: p is the new one of the two alternating direction buffers (pa, pb)
template <class V>
static void cg_vec_update(Hier &H, V *x, V *r, const V *pa, const V *pb, const V *q, int reliable, cudaStream_t st)
{
    const int n = H.n;
    constexpr int R = 16 / sizeof(V);
    if (n % R == 0)
        launch_pdl(k_cg_update<V, R>, vgrid(H, n / R), st, n, x, r, pa, pb, q, H.part.p, H.ctl.p, reliable);
    else launch_pdl(k_cg_update<V, 1>, vgrid(H, n), st, n, x, r, pa, pb, q, H.part.p, H.ctl.p, reliable);
}

template <class V>
static void cg_vec_p(Hier &H, const V *z, V *p, cudaStream_t st)
{
    const int n = H.n;
    constexpr int R = 16 / sizeof(V);
    if (n % R == 0) launch_pdl(k_cg_p<V, R>, vgrid(H, n / R), st, n, z, p, H.ctl.p);
    else launch_pdl(k_cg_p<V, 1>, vgrid(H, n), st, n, z, p, H.ctl.p);
}

static void rel_update(Hier &H, int force, cudaStream_t st)
{
    const int n = H.n;
    if (n % 2 == 0) launch_pdl(k_rel_fold<2>, vgrid(H, n / 2), st, n, H.x.p, H.xs32.p, H.ctl.p, force);
    else launch_pdl(k_rel_fold<1>, vgrid(H, n), st, n, H.x.p, H.xs32.p, H.ctl.p, force);
    with_mat(H.A64, [&](auto A) {
        using M = decltype(A);
        launch_pdl(k_rel_res<M>, grid_for<M>(H, n), st, A, n, H.b.p, H.x.p, H.r32.p, H.part.p, H.ctl.p, force);
    });
}

// One CG iteration.  The direction lives in two buffers that swap roles
// every iteration (parity = iteration number mod 2), so the captured graph
// holds an even number of iterations.
static void cg_iteration(Hier &H, int parity, cudaStream_t st)
{
    const int n = H.n;
    Ctl *c = H.ctl.p;
    const double dn = n;
    if (H.o.prec == GW_PREC_FP64) {
        // FP64 form: the direction update stays a separate pass, because
        // forming z + beta p at every gathered neighbour would add FP64
        // multiply-adds, the scarce resource of this GPU
        (void)parity;
        const MatStore<double> &A64 = H.cd[0].A;
        timed(H, GW_PK_SPMV, st, [&] {
            H.prof_bytes += vbytes(H, mat_bytes(A64) + 16.0 * dn);
            with_mat(A64, [&](auto A) {
                using M = decltype(A);
                launch_pdl(k_cg_spmv_dot<M>, grid_for<M>(H, n), st, A, n, (const double *)H.p.p, H.q.p, H.part.p, c);
            });
        });
        timed(H, GW_PK_UPDATE, st, [&] {
            H.prof_bytes += vbytes(H, 48.0 * dn);
            cg_vec_update<double>(H, H.x.p, H.r.p, H.p.p, (const double *)nullptr, H.q.p, 0, st);
        });
        with_mat(A64, [&](auto A) {
            using M = decltype(A);
            launch_pdl(k_cg_true<M>, grid_for<M>(H, n), st, A, n, H.b.p, H.x.p, H.r.p, H.part.p, c, 0);
        });
        vcycle_t<double>(H, H.cd, H.r.p, H.z.p, c, nullptr, 1, st);
        timed(H, GW_PK_PUPDATE, st, [&] {
            H.prof_bytes += vbytes(H, 24.0 * dn);
            cg_vec_p<double>(H, H.z.p, H.p.p, st);
        });
        GW_LAUNCH_CHECK();
        return;
    }
    const MatStore<float> &A32 = cg_op32(H);
    (void)parity;
    timed(H, GW_PK_SPMV, st, [&] {
        H.prof_bytes += vbytes(H, mat_bytes(A32) + 16.0 * dn);  // z, p_old read; p_new, q written
        with_mat(A32, [&](auto A) {
            using M = decltype(A);
            launch_pdl(k_cg_dir_spmv<M>, grid_for<M>(H, n), st, A, n, (const float *)H.z32.p, H.p32.p, H.p32b.p,
                       H.q32.p, H.part.p, c);
        });
    });
    timed(H, GW_PK_UPDATE, st, [&] {
        H.prof_bytes += vbytes(H, 24.0 * dn);
        cg_vec_update<float>(H, H.xs32.p, H.r32.p, H.p32.p, H.p32b.p, H.q32.p, 1, st);
    });
    rel_update(H, 0, st);
    vcycle_t<float>(H, H.cf, H.r32.p, H.z32.p, c, H.q32.p, 1, st);
    GW_LAUNCH_CHECK();
}

// Iterations per replay of the profiled iteration graph (events cannot sit
// inside a while node's body, so the profiled solve keeps host-polled replays)
static constexpr int GRAPH_ITERS = 4;

static size_t kernel_nodes(cudaGraph_t g)
{
    size_t num = 0;
    GW_CUDA(cudaGraphGetNodes(g, nullptr, &num));
    std::vector<cudaGraphNode_t> nodes(num);
    if (num) GW_CUDA(cudaGraphGetNodes(g, nodes.data(), &num));
    size_t k = 0;
    for (size_t i = 0; i < num; ++i) {
        cudaGraphNodeType t;
        GW_CUDA(cudaGraphNodeGetType(nodes[i], &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

template <class F>
static cudaGraphExec_t capture(Hier &H, F body, long long *nkernels)
{
    if (!H.cap) GW_CUDA(cudaStreamCreateWithFlags(&H.cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CaptureScope scope;  // no allocation or free of this library runs meanwhile
    GW_CUDA(cudaStreamBeginCapture(H.cap, cudaStreamCaptureModeThreadLocal));
    try {
        body(H.cap);
    } catch (...) {
        cudaStreamEndCapture(H.cap, &g);
        if (g) cudaGraphDestroy(g);
        H.prof_capture = false;
        throw;
    }
    GW_CUDA(cudaStreamEndCapture(H.cap, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) *nkernels = (long long)kernel_nodes(g);
    cudaGraphDestroy(g);
    GW_CUDA(e);
    return ex;
}

// The whole solve as one graph: the start (b -> r, the first V-cycle), then a
// while node whose body is one CG iteration.  The loop's condition starts at
// 1 on every launch; the kernel that finishes the solve (converged, maxit,
// breakdown) sets it to 0 through the handle kept in the control block.
// init_kernels / iter_kernels receive the kernels of the start and of the body.
template <class FI, class FB>
static cudaGraphExec_t capture_loop(Hier &H, FI init, FB iteration, unsigned long long *handle)
{
    if (!H.cap) GW_CUDA(cudaStreamCreateWithFlags(&H.cap, cudaStreamNonBlocking));
    if (!H.cap2) GW_CUDA(cudaStreamCreateWithFlags(&H.cap2, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr, body = nullptr;
    CaptureScope scope;
    GW_CUDA(cudaStreamBeginCapture(H.cap, cudaStreamCaptureModeThreadLocal));
    bool body_open = false;
    try {
        init(H.cap);
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        GW_CUDA(cudaStreamGetCaptureInfo(H.cap, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
        cudaGraphConditionalHandle h = 0;
        GW_CUDA(cudaGraphConditionalHandleCreate(&h, cg, 1u, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t loop = nullptr;
        GW_CUDA(cudaGraphAddNode(&loop, cg, deps, nullptr, ndeps, &np));
        body = np.conditional.phGraph_out[0];
        GW_CUDA(cudaStreamUpdateCaptureDependencies(H.cap, &loop, nullptr, 1, cudaStreamSetCaptureDependencies));
        GW_CUDA(cudaStreamBeginCaptureToGraph(H.cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        body_open = true;
        iteration(H.cap2);
        body_open = false;
        cudaGraph_t bout = nullptr;
        GW_CUDA(cudaStreamEndCapture(H.cap2, &bout));
        *handle = (unsigned long long)h;
    } catch (...) {
        cudaGraph_t t = nullptr;
        if (body_open) cudaStreamEndCapture(H.cap2, &t);
        cudaStreamEndCapture(H.cap, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    GW_CUDA(cudaStreamEndCapture(H.cap, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) {
        H.iter_kernels = (long long)kernel_nodes(body);
        H.init_kernels = (long long)kernel_nodes(g);  // the while node is not a kernel node
    }
    cudaGraphDestroy(g);
    GW_CUDA(e);
    return ex;
}

void drop_graphs(Hier &H)
{
    block_drop_graphs(H.blk);
    if (H.gexec) cudaGraphExecDestroy(H.gexec);
    if (H.ginit) cudaGraphExecDestroy(H.ginit);
    if (H.gsolve) cudaGraphExecDestroy(H.gsolve);
    H.gexec = H.ginit = H.gsolve = nullptr;
    H.cond = 0;
    for (auto &m : H.marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    H.marks.clear();
}

// the start of a solve: x = 0, r = b, the first V-cycle, p = z (FP64 form)
static void cg_start(Hier &H, cudaStream_t s)
{
    const int n = H.n, g = vgrid(H, n);
    if (H.o.prec == GW_PREC_FP64) {
        launch_pdl(k_cg_init<double>, g, s, n, (const double *)H.b.p, H.x.p, (double *)nullptr, H.r.p, H.p.p,
                   H.p2.p, H.part.p, H.ctl.p);
        vcycle_t<double>(H, H.cd, H.r.p, H.z.p, H.ctl.p, nullptr, 0, s);
        launch_pdl(k_copy<double>, g, s, n, (const double *)H.z.p, H.p.p, H.ctl.p);
    } else {
        launch_pdl(k_cg_init<float>, g, s, n, (const double *)H.b.p, H.x.p, H.xs32.p, H.r32.p, H.p32.p, H.p32b.p,
                   H.part.p, H.ctl.p);
        vcycle_t<float>(H, H.cf, H.r32.p, H.z32.p, H.ctl.p, nullptr, 0, s);
    }
    GW_LAUNCH_CHECK();
}

static void ensure_graphs(Hier &H)
{
    if (H.prof_on) {
        if (H.gexec && H.ginit) return;
        drop_graphs(H);
        H.ginit = capture(H, [&](cudaStream_t s) { cg_start(H, s); }, &H.init_kernels);
        H.prof_capture = true;
        H.gexec = capture(H, [&](cudaStream_t s) {
            for (int k = 0; k < GRAPH_ITERS; ++k) {
                H.cap_iter = k;
                cg_iteration(H, k & 1, s);
            }
        }, &H.iter_kernels);
        H.prof_capture = false;
        H.graph_iters = GRAPH_ITERS;
        return;
    }
    if (H.gsolve) return;
    drop_graphs(H);
    H.gsolve = capture_loop(H, [&](cudaStream_t s) { cg_start(H, s); },
                            [&](cudaStream_t s) { cg_iteration(H, 0, s); }, &H.cond);
    H.graph_iters = 1;
}

// accumulate the profiled level-0 kernel times of one replay of the iteration
// graph; only iterations that ran to the end (iteration number < it_now, or
// all of them while the solve continues) are counted
static void collect_marks(Hier &H, int first_iter, int it_now, bool done)
{
    for (auto &m : H.marks) {
        const int iter = first_iter + m.iter;
        if (done && iter >= it_now) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        H.prof_ms[m.kind] += ms;
        H.prof_cnt[m.kind] += 1;
        H.prof_b[m.kind] = m.bytes;
    }
}

void pcg_prepare(Hier &H) { ensure_graphs(H); }

int pcg_run(Hier &H, double tol, int maxit, int *iters, double *relres, cudaStream_t st)
{
    NvtxRange range("gw solve");
    Ctl *c = H.ctl.p;
    ensure_graphs(H);
    Ctl init;
    memset(&init, 0, sizeof init);
    init.tol2 = tol * tol;
    init.maxit = maxit;
    init.flexible = H.o.prec == GW_PREC_FP64 ? 0 : 1;
    init.delta2 = H.o.delta * H.o.delta;
    init.cond = H.gsolve ? H.cond : 0ULL;
    *H.ctl_host = init;
    GW_CUDA(cudaMemcpyAsync(c, H.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    if (H.gsolve) {
        // one launch runs the solve to its stop
        GW_CUDA(cudaGraphLaunch(H.gsolve, st));
        GW_CUDA(cudaMemcpyAsync(H.ctl_host, c, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
        H.launches += H.init_kernels + (long long)std::max(1, H.ctl_host->it) * H.iter_kernels;
    } else {
        GW_CUDA(cudaGraphLaunch(H.ginit, st));
        H.launches += H.init_kernels;
        const int max_launches = (maxit + GRAPH_ITERS - 1) / GRAPH_ITERS + 2;
        for (int k = 0; k < max_launches; ++k) {
            GW_CUDA(cudaGraphLaunch(H.gexec, st));
            H.launches += H.iter_kernels;
            GW_CUDA(cudaMemcpyAsync(H.ctl_host, c, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
            GW_CUDA(cudaStreamSynchronize(st));
            if (!H.marks.empty()) collect_marks(H, k * GRAPH_ITERS + 1, H.ctl_host->it, H.ctl_host->done);
            if (H.ctl_host->done) break;
        }
    }
    if (H.ctl_host->status == GW_ERR_NOT_CONVERGED || !H.ctl_host->done) {
        if (H.o.prec == GW_PREC_FP64) {
            with_mat(fine64(H), [&](auto A) {
                using M = decltype(A);
                launch_pdl(k_cg_true<M>, grid_for<M>(H, H.n), st, A, H.n, H.b.p, H.x.p, H.r.p, H.part.p, c, 1);
            });
            H.launches += 1;
        } else {
            rel_update(H, 1, st);
            H.launches += 2;
        }
        GW_LAUNCH_CHECK();
        GW_CUDA(cudaMemcpyAsync(H.ctl_host, c, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
        if (!H.ctl_host->done) H.ctl_host->status = GW_ERR_NOT_CONVERGED;
    }
    H.solves += 1;
    if (iters) *iters = H.ctl_host->it;
    if (relres) *relres = H.ctl_host->relres;
    return H.ctl_host->status;
}


// =============================================================================
// Batched solves (serving): the same pass of every active solve in one launch.
//
// Concurrent solves of different grids and fields (the sensitivity sweeps the
// Abstract motivates) each keep their own resident hierarchy.  A batch holds
// up to max_slots of them.  A device slot table describes every slot: per
// level its matrices (the level-0 stencil, sliced ELL or warp-CSR on the
// coarser levels), smoother data, vectors and Chebyshev coefficients, the
// implicit level-0 transfer, the coarsest inverse and the CG vectors and
// control block.  One CG iteration of the mixed form is a fixed sequence of
// passes (the CG product and update, the reliable update, and the V-cycle's
// passes level by level, padded to the deepest hierarchy); each pass is one
// launch whose work list holds (slot, virtual block) items for every slot
// that has that pass.  A slot's passes use a virtual grid fixed by its own
// size, and its reductions use its own partial-sum array and counters, so a
// solve gives the same bits alone and in any mix.  The iteration is captured
// once as a CUDA graph and replayed; admission and removal of slots between
// replays only rewrite the device slot table and work lists.  Slots finish
// independently: a finished slot's passes return at once until it is taken.

constexpr int BATCH_MAXL = 12;   // levels of a hierarchy in a batch
constexpr int BATCH_NB_CAP = 1024;  // virtual blocks of one pass of one slot

enum { BM_NONE = 0, BM_STEN4, BM_STEN2, BM_STEN1, BM_SELL, BM_CSR32 };

// a matrix of a slot, dispatched on fmt inside the batched kernels
struct BMat {
    int fmt, nr;
    const float *d, *ox, *oy, *oz;  // stencil (n = nr)
    int nx, sxy;
    const int *sp, *ci, *perm, *rp;  // sliced ELL (sp, ci, perm) or CSR (rp, ci)
    const float *v;
};

struct BLev {
    int n;
    BMat A, P, R;
    const float *dw;
    float *x, *b, *r, *t, *d, *d2;
    float c0, c1[8], c2[8];
};

struct BSlot {
    int L, active;
    BLev lv[BATCH_MAXL];
    BMat A32;                                   // operator of the CG recurrence (level-0 stencil)
    const double *ad, *ax, *ay, *az;            // FP64 level-0 stencil of the reliable updates
    int a64r;                                   // its rows per thread (4, 2 or 1)
    PImpl p0;                                   // implicit level-0 prolongator / restriction
    int p0r;                                    // its rows per thread (4 or 1)
    const int *mptr, *mem;
    int nc0;                                    // aggregates of level 0 (rows of level 1)
    const double *Ainv;
    float *xs, *r32, *p32, *p32b, *q32, *z32;
    double *x, *b;
    double *part;
    Ctl *ctl;
};

// one launch of the batched iteration: pass kind, level, Chebyshev step and
// whether the step reads d2 and writes d (the two direction buffers alternate)
enum {
    BP_DIR_SPMV = 0, BP_UPDATE, BP_REL_FOLD, BP_REL_RES, BP_ZERO2, BP_CHEBK, BP_RESID, BP_RESTRICT_U,
    BP_RESTRICT_SUM, BP_SPMV, BP_COARSE, BP_PROLONG, BP_PROLONG_IMP, BP_CHEB0, BP_CHEBK_DOT
};

struct BLaunch {
    int kind, level, step, swap, add_prev, keep;
};

// per-slot summary written at the end of every replay
struct BSum {
    int done, status, it, pad;
    double relres;
};

template <class F>
__device__ __forceinline__ void with_bmat(const BMat &m, F f)
{
    switch (m.fmt) {
    case BM_STEN4: f(MSten<float, 4>{m.d, m.ox, m.oy, m.oz, m.nr, m.nx, m.sxy}); break;
    case BM_STEN2: f(MSten<float, 2>{m.d, m.ox, m.oy, m.oz, m.nr, m.nx, m.sxy}); break;
    case BM_STEN1: f(MSten<float, 1>{m.d, m.ox, m.oy, m.oz, m.nr, m.nx, m.sxy}); break;
    case BM_SELL: f(MSell<float, 1>{SV<float>{m.sp, m.ci, m.v, m.nr, m.perm}}); break;
    case BM_CSR32: f(MCsr<float, 32>{m.rp, m.ci, m.v, m.nr}); break;
    default: break;
    }
}

template <int KIND>
__global__ void __launch_bounds__(BS) kb_pass(const BSlot *__restrict__ slots, const int4 *__restrict__ work,
                                              const int *__restrict__ wcnt, int launch, BLaunch Lc)
{
    pdl_enter();
    const int cnt = wcnt[2 * launch + 1], off = wcnt[2 * launch];
    for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
        const int4 item = work[off + w];
        const BSlot &S = slots[item.x];
        const VB vb{item.y, item.z};
        const int l = Lc.level;
        if constexpr (KIND == BP_DIR_SPMV) {
            with_bmat(S.A32, [&](auto A) {
                b_cg_dir_spmv(vb, A, S.lv[0].n, (const float *)S.z32, S.p32, S.p32b, S.q32, S.part, S.ctl);
            });
        } else if constexpr (KIND == BP_UPDATE) {
            if (S.lv[0].n % 4 == 0)
                b_cg_update<float, 4>(vb, S.lv[0].n, S.xs, S.r32, S.p32, S.p32b, S.q32, S.part, S.ctl, 1);
            else
                b_cg_update<float, 1>(vb, S.lv[0].n, S.xs, S.r32, S.p32, S.p32b, S.q32, S.part, S.ctl, 1);
        } else if constexpr (KIND == BP_REL_FOLD) {
            if (S.lv[0].n % 2 == 0) b_rel_fold<2>(vb, S.lv[0].n, S.x, S.xs, S.ctl, 0);
            else b_rel_fold<1>(vb, S.lv[0].n, S.x, S.xs, S.ctl, 0);
        } else if constexpr (KIND == BP_REL_RES) {
            const int n = S.lv[0].n, nx = S.A32.nx, sxy = S.A32.sxy;
            if (S.a64r == 4)
                b_rel_res(vb, MSten<double, 4>{S.ad, S.ax, S.ay, S.az, n, nx, sxy}, n, S.b, S.x, S.r32, S.part, S.ctl, 0);
            else if (S.a64r == 2)
                b_rel_res(vb, MSten<double, 2>{S.ad, S.ax, S.ay, S.az, n, nx, sxy}, n, S.b, S.x, S.r32, S.part, S.ctl, 0);
            else
                b_rel_res(vb, MSten<double, 1>{S.ad, S.ax, S.ay, S.az, n, nx, sxy}, n, S.b, S.x, S.r32, S.part, S.ctl, 0);
        } else if constexpr (KIND == BP_ZERO2) {
            const BLev &v = S.lv[l];
            const float *bl = l == 0 ? S.r32 : v.b;
            with_bmat(v.A, [&](auto A) {
                using M = decltype(A);
                b_cheb_zero2<M, float, false>(vb, A, v.n, v.dw, bl, v.x, v.r, v.d, (float *)nullptr, v.c0, v.c1[1],
                                              v.c2[1], Lc.keep, S.q32, S.part, S.ctl, 1);
            });
        } else if constexpr (KIND == BP_CHEBK || KIND == BP_CHEBK_DOT) {
            const BLev &v = S.lv[l];
            float *d = Lc.swap ? v.d2 : v.d, *dn = Lc.swap ? v.d : v.d2;
            with_bmat(v.A, [&](auto A) {
                using M = decltype(A);
                if constexpr (KIND == BP_CHEBK_DOT)
                    b_chebk<M, float, true>(vb, A, v.n, v.dw, v.r, d, dn, v.x, S.z32, v.c1[Lc.step], v.c2[Lc.step],
                                            Lc.add_prev, (const float *)S.r32, S.q32, S.part, S.ctl, 1);
                else
                    b_chebk<M, float, false>(vb, A, v.n, v.dw, v.r, d, dn, v.x, (float *)nullptr, v.c1[Lc.step],
                                             v.c2[Lc.step], Lc.add_prev, (const float *)nullptr, S.q32, S.part,
                                             S.ctl, 1);
            });
        } else if constexpr (KIND == BP_CHEB0) {
            const BLev &v = S.lv[l];
            const float *bl = l == 0 ? S.r32 : v.b;
            with_bmat(v.A, [&](auto A) {
                using M = decltype(A);
                b_cheb0<M, float, float, false>(vb, A, v.n, v.dw, bl, v.x, v.r, v.d, (float *)nullptr, v.c0, 0,
                                                S.q32, S.part, S.ctl, 1);
            });
        } else if constexpr (KIND == BP_RESID) {
            const BLev &v = S.lv[l];
            const float *bl = l == 0 ? S.r32 : v.b;
            with_bmat(v.A, [&](auto A) { b_residual(vb, A, v.n, bl, (const float *)v.x, v.r, S.ctl); });
        } else if constexpr (KIND == BP_RESTRICT_U) {
            if (S.p0r == 4) b_restrict_u<4>(vb, S.p0, S.lv[0].r, S.lv[0].t, S.ctl);
            else b_restrict_u<1>(vb, S.p0, S.lv[0].r, S.lv[0].t, S.ctl);
        } else if constexpr (KIND == BP_RESTRICT_SUM) {
            b_restrict_sum(vb, S.nc0, S.mptr, S.mem, S.lv[0].t, S.lv[1].b, S.ctl);
        } else if constexpr (KIND == BP_SPMV) {
            const BLev &v = S.lv[l];
            with_bmat(v.R, [&](auto R) { b_spmv(vb, R, v.R.nr, (const float *)v.r, S.lv[l + 1].b, S.ctl); });
        } else if constexpr (KIND == BP_COARSE) {
            const BLev &v = S.lv[l];
            b_coarse<float>(vb, v.n, S.Ainv, v.b, v.x, S.ctl);
        } else if constexpr (KIND == BP_PROLONG) {
            const BLev &v = S.lv[l];
            with_bmat(v.P, [&](auto P) { b_prolong(vb, P, v.n, (const float *)S.lv[l + 1].x, v.x, S.ctl); });
        } else if constexpr (KIND == BP_PROLONG_IMP) {
            if (S.p0r == 4) b_prolong_imp<4>(vb, S.p0, S.lv[1].x, S.lv[0].x, S.ctl);
            else b_prolong_imp<1>(vb, S.p0, S.lv[1].x, S.lv[0].x, S.ctl);
        }
    }
}

// copies every active slot's control block into the summary array
__global__ void kb_summary(const BSlot *__restrict__ slots, int nslots, BSum *__restrict__ out)
{
    pdl_enter();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nslots; s += gridDim.x * blockDim.x) {
        BSum o{1, GW_OK, 0, 0, 0.0};
        if (slots[s].active) {
            const Ctl *c = slots[s].ctl;
            o.done = *(volatile const int *)&c->done;
            o.status = c->status;
            o.it = c->it;
            o.relres = c->relres;
        }
        out[s] = o;
    }
}

struct Batch {
    int max_slots = 0, dev = 0, degree = 0, lmax = 0, graph_lmax = 0;
    cudaStream_t st = nullptr, cap = nullptr;
    cudaGraphExec_t g = nullptr;
    std::vector<Hier *> slot_h;
    std::vector<int> state;           // 0 free, 1 running, 2 finished (not yet taken)
    std::vector<BSlot> hslots;        // host image of the slot table
    std::vector<BLaunch> launches;    // the iteration's pass sequence for lmax levels
    DBuf<BSlot> dslots;
    DBuf<int4> work;
    DBuf<int> wcnt;                   // per launch: offset and count of its items
    DBuf<BSum> dsum;
    BSum *hsum = nullptr;             // pinned
    int4 *hwork = nullptr;            // pinned staging of the work lists
    int *hwcnt = nullptr;
    BSlot *hstage = nullptr;
    size_t work_cap = 0;
    long long iter_kernels = 0, launches_run = 0;
    ~Batch()
    {
        if (g) cudaGraphExecDestroy(g);
        if (hsum) host_free(hsum);
        if (hwork) host_free(hwork);
        if (hwcnt) host_free(hwcnt);
        if (hstage) host_free(hstage);
        if (cap) cudaStreamDestroy(cap);
        if (st) cudaStreamDestroy(st);
    }
};

static BMat bmat_of(const MatStore<float> &M)
{
    BMat b;
    memset(&b, 0, sizeof b);
    b.nr = M.nr;
    switch (M.fmt) {
    case FMT_STEN: {
        const StenT<float> &S = M.sten;
        b.fmt = (S.n % 4 == 0 && S.nx % 4 == 0) ? BM_STEN4 : (S.n % 2 == 0 && S.nx % 2 == 0) ? BM_STEN2 : BM_STEN1;
        b.d = S.d.p, b.ox = S.ox.p, b.oy = S.oy.p, b.oz = S.oz.p;
        b.nr = S.n, b.nx = S.nx, b.sxy = S.nx * S.ny;
        break;
    }
    case FMT_SELL:
        if (M.nnz > (long long)SELL_LONG_ROW * M.nr && GW_SELL_LANES != 1) fail(GW_ERR_ARG, "batch: unsupported lanes");
        b.fmt = BM_SELL;
        b.sp = M.sell.sp.p, b.ci = M.sell.ci.p, b.v = M.sell.v.p, b.perm = M.sell.perm.p;
        b.nr = M.sell.nr;
        break;
    case FMT_CSR32:
        b.fmt = BM_CSR32;
        b.rp = M.csr.rp.p, b.ci = M.csr.ci.p, b.v = M.csr.v.p;
        b.nr = M.csr.nr;
        break;
    default: fail(GW_ERR_ARG, "batch: a level format the batched kernels do not read (%d)", M.fmt);
    }
    return b;
}

// virtual blocks of one pass of one slot (a function of the slot alone)
static int bnb(long long threads) { return (int)std::max(1LL, std::min<long long>((threads + BS - 1) / BS, BATCH_NB_CAP)); }

static int bmat_rows_per_thread(const BMat &m) { return m.fmt == BM_STEN4 ? 4 : m.fmt == BM_STEN2 ? 2 : 1; }

static long long bmat_threads(const BMat &m, int n)
{
    if (m.fmt == BM_CSR32) return 32LL * n;
    return (n + bmat_rows_per_thread(m) - 1) / bmat_rows_per_thread(m);
}

static int pass_nb(const BSlot &S, const BLaunch &c)
{
    const int n0 = S.lv[0].n;
    switch (c.kind) {
    case BP_DIR_SPMV: return bnb(bmat_threads(S.A32, n0));
    case BP_UPDATE: return bnb(n0 % 4 == 0 ? n0 / 4 : n0);
    case BP_REL_FOLD: return bnb(n0 % 2 == 0 ? n0 / 2 : n0);
    case BP_REL_RES: return bnb((n0 + S.a64r - 1) / S.a64r);
    case BP_RESTRICT_U:
    case BP_PROLONG_IMP: return bnb(n0 / S.p0r);
    case BP_RESTRICT_SUM: return bnb(4LL * S.nc0);
    case BP_COARSE: return bnb(32LL * S.lv[c.level].n);
    case BP_SPMV: return bnb(bmat_threads(S.lv[c.level].R, S.lv[c.level].R.nr));
    case BP_PROLONG: return bnb(bmat_threads(S.lv[c.level].P, S.lv[c.level].n));
    default: return bnb(bmat_threads(S.lv[c.level].A, S.lv[c.level].n));
    }
}

// does slot S take part in launch c
static bool pass_has(const BSlot &S, const BLaunch &c)
{
    if (!S.active) return false;
    const int l = c.level;
    switch (c.kind) {
    case BP_DIR_SPMV:
    case BP_UPDATE:
    case BP_REL_FOLD:
    case BP_REL_RES: return true;
    case BP_COARSE: return l == S.L - 1;
    default: return l < S.L - 1;
    }
}

// the pass sequence of one CG iteration for hierarchies of up to lmax levels
// and Chebyshev degree m, one application before and after the coarse
// correction (the order of cg_iteration, vcycle_t and smooth)
static std::vector<BLaunch> batch_sequence(int lmax, int m)
{
    std::vector<BLaunch> q;
    auto add = [&](int kind, int level, int step = 0, int swap = 0, int add_prev = 0, int keep = 0) {
        q.push_back(BLaunch{kind, level, step, swap, add_prev, keep});
    };
    add(BP_DIR_SPMV, 0);
    add(BP_UPDATE, 0);
    add(BP_REL_FOLD, 0);
    add(BP_REL_RES, 0);
    for (int l = 0; l < lmax; ++l) {
        if (l < lmax - 1) {
            add(BP_ZERO2, l, 1, 0, 0, m > 2);
            for (int k = 2; k < m; ++k) add(BP_CHEBK, l, k, (k % 2) ? 1 : 0, 0);  // k = 2 reads d, writes d2
            add(BP_RESID, l);
            if (l == 0) {
                add(BP_RESTRICT_U, 0);
                add(BP_RESTRICT_SUM, 0);
            } else {
                add(BP_SPMV, l);
            }
        }
        if (l >= 1) add(BP_COARSE, l);
    }
    for (int l = lmax - 2; l >= 0; --l) {
        add(l == 0 ? BP_PROLONG_IMP : BP_PROLONG, l);
        add(BP_CHEB0, l);
        for (int k = 1; k < m; ++k)
            add(l == 0 && k == m - 1 ? BP_CHEBK_DOT : BP_CHEBK, l, k, (k % 2) ? 0 : 1, k == 1 ? 1 : 0);
    }
    return q;
}

template <int KIND>
static void kb_launch(Batch &B, int idx, cudaStream_t s)
{
    launch_pdl(kb_pass<KIND>, kernel_wave((const void *)kb_pass<KIND>, BS), s, (const BSlot *)B.dslots.p,
               (const int4 *)B.work.p, (const int *)B.wcnt.p, idx, B.launches[(size_t)idx]);
}

static void batch_enqueue_iteration(Batch &B, cudaStream_t s)
{
    for (int i = 0; i < (int)B.launches.size(); ++i) {
        switch (B.launches[(size_t)i].kind) {
        case BP_DIR_SPMV: kb_launch<BP_DIR_SPMV>(B, i, s); break;
        case BP_UPDATE: kb_launch<BP_UPDATE>(B, i, s); break;
        case BP_REL_FOLD: kb_launch<BP_REL_FOLD>(B, i, s); break;
        case BP_REL_RES: kb_launch<BP_REL_RES>(B, i, s); break;
        case BP_ZERO2: kb_launch<BP_ZERO2>(B, i, s); break;
        case BP_CHEBK: kb_launch<BP_CHEBK>(B, i, s); break;
        case BP_RESID: kb_launch<BP_RESID>(B, i, s); break;
        case BP_RESTRICT_U: kb_launch<BP_RESTRICT_U>(B, i, s); break;
        case BP_RESTRICT_SUM: kb_launch<BP_RESTRICT_SUM>(B, i, s); break;
        case BP_SPMV: kb_launch<BP_SPMV>(B, i, s); break;
        case BP_COARSE: kb_launch<BP_COARSE>(B, i, s); break;
        case BP_PROLONG: kb_launch<BP_PROLONG>(B, i, s); break;
        case BP_PROLONG_IMP: kb_launch<BP_PROLONG_IMP>(B, i, s); break;
        case BP_CHEB0: kb_launch<BP_CHEB0>(B, i, s); break;
        case BP_CHEBK_DOT: kb_launch<BP_CHEBK_DOT>(B, i, s); break;
        default: break;
        }
    }
    launch_pdl(kb_summary, 1, s, (const BSlot *)B.dslots.p, B.max_slots, B.dsum.p);
    GW_CUDA(cudaMemcpyAsync(B.hsum, B.dsum.p, sizeof(BSum) * (size_t)B.max_slots, cudaMemcpyDeviceToHost, s));
    GW_LAUNCH_CHECK();
}

// rewrites the work lists of every launch from the slot table
static void batch_rebuild_work(Batch &B)
{
    const int nl = (int)B.launches.size();
    size_t total = 0;
    for (int i = 0; i < nl; ++i)
        for (int s = 0; s < B.max_slots; ++s)
            if (pass_has(B.hslots[(size_t)s], B.launches[(size_t)i])) total += (size_t)pass_nb(B.hslots[(size_t)s], B.launches[(size_t)i]);
    if (total > B.work_cap) fail(GW_ERR_OOM, "batch: work lists exceed their capacity");
    size_t k = 0;
    for (int i = 0; i < nl; ++i) {
        B.hwcnt[2 * i] = (int)k;
        for (int s = 0; s < B.max_slots; ++s) {
            const BSlot &S = B.hslots[(size_t)s];
            if (!pass_has(S, B.launches[(size_t)i])) continue;
            const int nb = pass_nb(S, B.launches[(size_t)i]);
            for (int v = 0; v < nb; ++v) B.hwork[k++] = make_int4(s, v, nb, 0);
        }
        B.hwcnt[2 * i + 1] = (int)(k - (size_t)B.hwcnt[2 * i]);
    }
    GW_CUDA(cudaMemcpyAsync(B.wcnt.p, B.hwcnt, sizeof(int) * 2 * (size_t)nl, cudaMemcpyHostToDevice, B.st));
    if (k) GW_CUDA(cudaMemcpyAsync(B.work.p, B.hwork, sizeof(int4) * k, cudaMemcpyHostToDevice, B.st));
}

// (re)captures the iteration graph for hierarchies of up to lmax levels
static void batch_capture(Batch &B, int lmax)
{
    if (B.g && B.graph_lmax >= lmax) return;
    lmax = std::max(lmax, B.graph_lmax);
    std::vector<BLaunch> seq = batch_sequence(lmax, B.degree);
    const size_t nl = seq.size();
    // launch table and work-list capacity for this sequence
    DBuf<int> wcnt(2 * nl);
    size_t cap = nl * (size_t)B.max_slots * BATCH_NB_CAP;
    DBuf<int4> work(cap);
    int *hw = nullptr;
    int4 *hk = nullptr;
    GW_CUDA(host_malloc((void **)&hw, sizeof(int) * 2 * nl));
    GW_CUDA(host_malloc((void **)&hk, sizeof(int4) * cap));
    if (B.hwcnt) host_free(B.hwcnt);
    if (B.hwork) host_free(B.hwork);
    B.hwcnt = hw;
    B.hwork = hk;
    B.wcnt = std::move(wcnt);
    B.work = std::move(work);
    B.work_cap = cap;
    B.launches = seq;
    if (B.g) cudaGraphExecDestroy(B.g);
    B.g = nullptr;
    for (int i = 0; i < (int)nl; ++i) {  // kernels are loaded outside the capture
        B.hwcnt[2 * i] = 0;
        B.hwcnt[2 * i + 1] = 0;
    }
    GW_CUDA(cudaMemcpyAsync(B.wcnt.p, B.hwcnt, sizeof(int) * 2 * nl, cudaMemcpyHostToDevice, B.st));
    batch_enqueue_iteration(B, B.st);
    GW_CUDA(cudaStreamSynchronize(B.st));
    cudaGraph_t g = nullptr;
    {
        CaptureScope scope;
        GW_CUDA(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
        try {
            batch_enqueue_iteration(B, B.cap);
        } catch (...) {
            cudaStreamEndCapture(B.cap, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        GW_CUDA(cudaStreamEndCapture(B.cap, &g));
    }
    cudaError_t e = cudaGraphInstantiate(&B.g, g, 0);
    if (e == cudaSuccess) B.iter_kernels = (long long)kernel_nodes(g);
    cudaGraphDestroy(g);
    GW_CUDA(e);
    B.graph_lmax = lmax;
    batch_rebuild_work(B);
}

Batch *batch_create(int max_slots)
{
    if (max_slots < 1 || max_slots > 256) fail(GW_ERR_ARG, "gw_batch_create: max_slots must be in 1..256");
    std::unique_ptr<Batch> B(new Batch);
    B->max_slots = max_slots;
    GW_CUDA(cudaGetDevice(&B->dev));
    GW_CUDA(cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
    B->slot_h.assign((size_t)max_slots, nullptr);
    B->state.assign((size_t)max_slots, 0);
    B->hslots.resize((size_t)max_slots);
    memset(B->hslots.data(), 0, sizeof(BSlot) * (size_t)max_slots);
    B->dslots.alloc((size_t)max_slots);
    B->dsum.alloc((size_t)max_slots);
    GW_CUDA(host_malloc((void **)&B->hsum, sizeof(BSum) * (size_t)max_slots));
    GW_CUDA(host_malloc((void **)&B->hstage, sizeof(BSlot) * (size_t)max_slots));
    memcpy(B->hstage, B->hslots.data(), sizeof(BSlot) * (size_t)max_slots);
    GW_CUDA(cudaMemcpyAsync(B->dslots.p, B->hstage, sizeof(BSlot) * (size_t)max_slots, cudaMemcpyHostToDevice, B->st));
    GW_CUDA(cudaStreamSynchronize(B->st));
    return B.release();
}

void batch_free(Batch *B)
{
    if (!B) return;
    cudaStreamSynchronize(B->st);
    for (Hier *H : B->slot_h)
        if (H) H->batch = nullptr;  // solves not taken are abandoned; their hierarchies stay usable
    delete B;
}

static void batch_upload_slots(Batch &B)
{
    memcpy(B.hstage, B.hslots.data(), sizeof(BSlot) * (size_t)B.max_slots);
    GW_CUDA(cudaMemcpyAsync(B.dslots.p, B.hstage, sizeof(BSlot) * (size_t)B.max_slots, cudaMemcpyHostToDevice, B.st));
}

// Why a hierarchy cannot join a batch (nullptr: it can).
static const char *batch_unsupported(const Hier &H, int degree)
{
    if (H.o.prec != GW_PREC_MIXED32 || H.o.half_storage) return "batched solves run the mixed form with FP32 storage";
    if (H.o.smoother != GW_SMOOTH_CHEBYSHEV || H.o.nu != 1 || H.o.degree < 2)
        return "batched solves run Chebyshev smoothing of degree >= 2 with nu = 1";
    if (degree && H.o.degree != degree) return "every solve of a batch has the same Chebyshev degree";
    if (H.L < 2 || H.L > BATCH_MAXL) return "batched solves need 2 to 12 levels";
    if (!H.p0.n) return "batched solves need the implicit level-0 transfer of a 7-point grid";
    if (H.cf[0].A.fmt != FMT_STEN || cg_op32(H).fmt != FMT_STEN || H.A64.fmt != FMT_STEN)
        return "batched solves need the level-0 stencil";
    return nullptr;
}

int batch_add(Batch &B, Hier &H, const double *b, double tol, int maxit)
{
    AllocStream alloc_scope(B.st);
    if (const char *why = batch_unsupported(H, B.degree)) fail(GW_ERR_ARG, "gw_batch_add: %s", why);
    if (H.dev != B.dev) fail(GW_ERR_ARG, "gw_batch_add: the hierarchy lives on another device");
    for (int s = 0; s < B.max_slots; ++s)
        if (B.slot_h[(size_t)s] == &H) fail(GW_ERR_ARG, "gw_batch_add: the hierarchy is already in this batch");
    int slot = -1;
    for (int s = 0; s < B.max_slots; ++s)
        if (!B.state[(size_t)s]) {
            slot = s;
            break;
        }
    if (slot < 0) fail(GW_ERR_ARG, "gw_batch_add: every slot is in use");
    B.degree = H.o.degree;
    // the slot's description
    BSlot S;
    memset(&S, 0, sizeof S);
    S.L = H.L;
    S.active = 1;
    for (int l = 0; l < H.L; ++l) {
        CycLevel<float> &c = H.cf[(size_t)l];
        BLev &v = S.lv[l];
        v.n = c.n;
        if (l < H.L - 1) {
            v.A = bmat_of(c.A);
            if (l >= 1) {
                v.P = bmat_of(c.P);
                v.R = bmat_of(c.R);
            }
        }
        v.dw = c.dw.p;
        v.x = c.x.p, v.b = c.b.p, v.r = c.r.p, v.t = c.t.p, v.d = c.d.p, v.d2 = c.d2.p;
        v.c0 = (float)c.c0;
        for (int k = 0; k < 8; ++k) {
            v.c1[k] = (float)c.c1[k];
            v.c2[k] = (float)c.c2[k];
        }
    }
    S.A32 = bmat_of(cg_op32(H));
    {
        const StenT<double> &D = H.A64.sten;
        S.ad = D.d.p, S.ax = D.ox.p, S.ay = D.oy.p, S.az = D.oz.p;
        constexpr int RV = sten_r<double>(), RH = RV / 2;
        S.a64r = (D.n % RV == 0 && D.nx % RV == 0) ? RV : (D.n % RH == 0 && D.nx % RH == 0) ? RH : 1;
    }
    {
        const ImplP &I = H.p0;
        S.p0 = PImpl{I.agg, I.s.p, I.fx.p, I.fy.p, I.fz.p, I.n, I.nx, I.sxy, I.w0};
        S.p0r = (I.n % 4 == 0 && I.nx % 4 == 0) ? 4 : 1;
        S.mptr = I.mptr.p;
        S.mem = I.mem.p;
        S.nc0 = I.nc;
    }
    S.Ainv = H.Ainv.p;
    S.xs = H.xs32.p, S.r32 = H.r32.p, S.p32 = H.p32.p, S.p32b = H.p32b.p, S.q32 = H.q32.p, S.z32 = H.z32.p;
    S.x = H.x.p, S.b = H.b.p;
    S.part = H.part.p;
    S.ctl = H.ctl.p;
    // the right-hand side and the start of the solve (x = 0, r = b, the first V-cycle)
    GW_CUDA(cudaMemcpyAsync(H.b.p, b, (size_t)H.n * sizeof(double), cudaMemcpyDefault, B.st));
    Ctl init;
    memset(&init, 0, sizeof init);
    init.tol2 = tol * tol;
    init.maxit = maxit;
    init.flexible = 1;
    init.delta2 = H.o.delta * H.o.delta;
    init.cond = 0;
    *H.ctl_host = init;
    GW_CUDA(cudaMemcpyAsync(H.ctl.p, H.ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, B.st));
    cg_start(H, B.st);
    H.launches += H.init_kernels;
    B.slot_h[(size_t)slot] = &H;
    B.state[(size_t)slot] = 1;
    H.batch = &B;
    B.hslots[(size_t)slot] = S;
    B.lmax = std::max(B.lmax, H.L);
    batch_upload_slots(B);
    if (!B.g || B.graph_lmax < B.lmax) batch_capture(B, B.lmax);
    else batch_rebuild_work(B);
    GW_CUDA(cudaStreamSynchronize(B.st));  // the staging buffers are reused by the next call
    return slot;
}

// Replays the iteration graph up to `iterations` times, stopping early once
// some running solve has finished; returns the number of finished solves
// waiting to be taken.
int batch_run(Batch &B, int iterations)
{
    AllocStream alloc_scope(B.st);
    NvtxRange range("gw batch replays");
    int running = 0;
    for (int s = 0; s < B.max_slots; ++s) running += B.state[(size_t)s] == 1;
    for (int k = 0; k < iterations && running && B.g; ++k) {
        GW_CUDA(cudaGraphLaunch(B.g, B.st));
        B.launches_run += B.iter_kernels;
        GW_CUDA(cudaStreamSynchronize(B.st));
        bool any = false;
        for (int s = 0; s < B.max_slots; ++s)
            if (B.state[(size_t)s] == 1 && B.hsum[s].done) {
                B.state[(size_t)s] = 2;
                any = true;
            }
        if (any) break;
    }
    int fin = 0;
    for (int s = 0; s < B.max_slots; ++s) fin += B.state[(size_t)s] == 2;
    return fin;
}

int batch_state(const Batch &B, int slot) { return slot >= 0 && slot < B.max_slots ? B.state[(size_t)slot] : -1; }

// Takes a finished solve out of the batch: its heads into h (host or device),
// its iterations and true relative residual; frees the slot.
int batch_take(Batch &B, int slot, double *h, int *iters, double *relres)
{
    AllocStream alloc_scope(B.st);
    if (slot < 0 || slot >= B.max_slots || B.state[(size_t)slot] != 2)
        fail(GW_ERR_ARG, "gw_batch_take: slot %d holds no finished solve", slot);
    Hier &H = *B.slot_h[(size_t)slot];
    Ctl *c = H.ctl.p;
    GW_CUDA(cudaMemcpyAsync(H.ctl_host, c, sizeof(Ctl), cudaMemcpyDeviceToHost, B.st));
    GW_CUDA(cudaStreamSynchronize(B.st));
    if (H.ctl_host->status == GW_ERR_NOT_CONVERGED || !H.ctl_host->done) {
        rel_update(H, 1, B.st);  // fold the correction in and state the true residual
        GW_LAUNCH_CHECK();
        GW_CUDA(cudaMemcpyAsync(H.ctl_host, c, sizeof(Ctl), cudaMemcpyDeviceToHost, B.st));
        GW_CUDA(cudaStreamSynchronize(B.st));
        if (!H.ctl_host->done) H.ctl_host->status = GW_ERR_NOT_CONVERGED;
    }
    if (h) GW_CUDA(cudaMemcpyAsync(h, H.x.p, (size_t)H.n * sizeof(double), cudaMemcpyDefault, B.st));
    const int status = H.ctl_host->status;
    if (iters) *iters = H.ctl_host->it;
    if (relres) *relres = H.ctl_host->relres;
    H.solves += 1;
    memset(&B.hslots[(size_t)slot], 0, sizeof(BSlot));
    H.batch = nullptr;
    B.slot_h[(size_t)slot] = nullptr;
    B.state[(size_t)slot] = 0;
    B.lmax = 0;
    for (int s = 0; s < B.max_slots; ++s)
        if (B.state[(size_t)s]) B.lmax = std::max(B.lmax, B.hslots[(size_t)s].L);
    batch_upload_slots(B);
    batch_rebuild_work(B);
    GW_CUDA(cudaStreamSynchronize(B.st));
    return status;
}

long long batch_kernel_launches(const Batch &B) { return B.launches_run; }

// A hierarchy that is freed while its solve is in the batch leaves it.
void batch_forget(Batch &B, Hier *H)
{
    for (int s = 0; s < B.max_slots; ++s)
        if (B.slot_h[(size_t)s] == H) {
            cudaStreamSynchronize(B.st);
            memset(&B.hslots[(size_t)s], 0, sizeof(BSlot));
            B.slot_h[(size_t)s] = nullptr;
            B.state[(size_t)s] = 0;
            try {
                batch_upload_slots(B);
                batch_rebuild_work(B);
                GW_CUDA(cudaStreamSynchronize(B.st));
            } catch (...) {
            }
        }
    H->batch = nullptr;
}

}  // namespace gw
