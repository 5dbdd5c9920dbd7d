// setup.cu -- the AMG setup phase on the GPU (Introduction: the hierarchy,
// prolongation and restriction are built automatically; "CG/AMG/SA" smoothed
// aggregation, Results section).
//
// Stages per level: symmetrised strength of connection, distance-2 maximal
// independent set by parallel rounds with hashed priorities, aggregation,
// filtered matrix and Gershgorin bound, Jacobi-smoothed prolongator,
// transpose, Galerkin product by a two-pass SpGEMM.  Then the dense inverse of
// the coarsest level and the conversion of every level to sliced ELL.
//
// Every floating-point operation that decides the hierarchy is an explicitly
// rounded intrinsic (__dmul_rn, __dadd_rn, __ddiv_rn), so no multiply-add is
// fused, and every sum runs in ascending column order of its row -- the same
// order a serial FP64 implementation follows -- so aggregates, patterns and
// values match such an implementation exactly.
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "gw_internal.cuh"

namespace gw {

static inline int nblk(long long n, int bs, long long cap = 152LL * 32)
{
    long long b = (n + bs - 1) / bs;
    return (int)std::max(1LL, std::min(b, cap));
}

#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// Row-parallel form of the SpGEMM and prolongator passes: chosen per product
// from the row counts and lengths (0), or forced to a thread a row (1) or a
// warp a row (2) by GW_SETUP_FORMS=thread|warp in the environment, read once,
// so that tests can check both forms against the oracle on any problem.  Both
// forms give the same bits.
// Lanes that share a row in the per-row setup passes: one for the short rows
// of the fine grid, a group of 8 or a warp for the long rows of the coarse
// levels (a thread walking a row of a hundred entries alone leaves a
// 6k-row level on a few dozen SMs).
static int row_lanes(const DCSR &A)
{
    const double per_row = A.nr ? (double)A.nnz / A.nr : 0.0;
    return per_row <= 12.0 ? 1 : per_row <= 48.0 ? 8 : 32;
}

// Rows handed to groups of G lanes; whole warps stay in the loop when G > 1
// (the groups' shuffles need every lane), so the row index may be >= n.
#define GROUP_LOOP(G, ii, n)                                                                       \
    for (long long ii = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / (G),                \
                   ii##_step = (long long)gridDim.x * (blockDim.x / (G));                        \
         (G) == 1 ? ii < (n) : __any_sync(0xffffffffu, ii < (n)); ii += ii##_step)

static int setup_forms()
{
    static const int f = [] {
        const char *e = getenv("GW_SETUP_FORMS");
        if (!e) return 0;
        if (!strcmp(e, "thread")) return 1;
        if (!strcmp(e, "warp")) return 2;
        return 0;
    }();
    return f;
}

// SplitMix64 (Steele, Lea & Flood 2014): finaliser of x + golden gamma.
__device__ __forceinline__ uint64_t smix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t prio_key(uint64_t seed, int level, int i)
{
    return smix64(seed ^ ((uint64_t)level << 48) ^ (uint64_t)(uint32_t)i);
}

__device__ __forceinline__ bool prio_gt(uint64_t k1, int i1, uint64_t k2, int i2)
{
    return k1 > k2 || (k1 == k2 && i1 > i2);
}

// Block-wide maximum of non-negative doubles given as their bit patterns
// (ordered like the values), then one atomicMax per block.  Every thread of
// the block must call it.
__device__ __forceinline__ void block_atomic_max(unsigned long long v, unsigned long long *dst)
{
    __shared__ unsigned long long sm[32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) m = sm[k] > m ? sm[k] : m;
        if (m) atomicMax(dst, m);
    }
}

// ----------------------------------------------------------------- strength --
__global__ void k_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                       double *__restrict__ d)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double dd = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i) {
                dd = v[e];
                break;
            }
        d[i] = dd;
    }
}

// (i,j) strong iff a_ij^2 > theta2 * (a_ii * a_jj), i != j
template <int G>
__global__ void k_strength_raw(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                               const double *__restrict__ v, const double *__restrict__ d, double theta2,
                               unsigned char *__restrict__ raw)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        if (ii >= n) continue;
        const int i = (int)ii;
        const double di = d[i];
        for (int e = rp[i] + lane; e < rp[i + 1]; e += G) {
            const int j = ci[e];
            if (j == i) {
                raw[e] = 0;
                continue;
            }
            const double a = v[e];
            const double lhs = __dmul_rn(a, a);
            double rhs = __dmul_rn(di, d[j]);
            rhs = __dmul_rn(theta2, rhs);
            raw[e] = lhs > rhs;
        }
    }
}

__device__ __forceinline__ int row_find(const int *__restrict__ rp, const int *__restrict__ ci, int row, int col)
{
    int lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = ci[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// S = raw OR raw^T
template <int G>
__global__ void k_strength_sym(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                               const unsigned char *__restrict__ raw, unsigned char *__restrict__ S)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        if (ii >= n) continue;
        const int i = (int)ii;
        for (int e = rp[i] + lane; e < rp[i + 1]; e += G) {
            const int j = ci[e];
            unsigned char s = raw[e];
            if (!s && j != i) {
                int t = row_find(rp, ci, j, i);
                if (t >= 0) s = raw[t];
            }
            S[e] = s;
        }
    }
}

void setup_strength(const DCSR &A, double theta2, DBuf<unsigned char> &S, cudaStream_t st)
{
    DBuf<double> d((size_t)A.nr);
    DBuf<unsigned char> raw((size_t)A.nnz + 1);
    S.alloc((size_t)A.nnz + 1);
    gw_launch(k_diag, nblk(A.nr, 256), 256, 0, st, A.nr, A.rp.p, A.ci.p, A.v.p, d.p);
    const int G = row_lanes(A), gg = nblk((long long)A.nr * G, 256);
    if (G == 1) {
        gw_launch(k_strength_raw<1>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, A.v.p, d.p, theta2, raw.p);
        gw_launch(k_strength_sym<1>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, raw.p, S.p);
    } else if (G == 8) {
        gw_launch(k_strength_raw<8>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, A.v.p, d.p, theta2, raw.p);
        gw_launch(k_strength_sym<8>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, raw.p, S.p);
    } else {
        gw_launch(k_strength_raw<32>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, A.v.p, d.p, theta2, raw.p);
        gw_launch(k_strength_sym<32>, gg, 256, 0, st, A.nr, A.rp.p, A.ci.p, raw.p, S.p);
    }
    GW_LAUNCH_CHECK();
    GW_CUDA(cudaStreamSynchronize(st));
}

// -------------------------------------------------------------------- MIS-2 --
// Parallel rounds with fixed priorities (key, index).  A node joins the set
// when it beats every undecided node within two hops of the strength graph
// (the hops pass through nodes in any state); nodes within two hops of a
// selected node leave.  With fixed priorities this yields the same set as
// visiting the nodes in descending priority (Blelloch, Fineman & Shun 2012).
enum : unsigned char { MIS_UNDECIDED = 0, MIS_ROOT = 1, MIS_OUT = 2 };

// the larger of two (key, index) candidates, -1 meaning none (a strict
// total order, so the maximum over a group does not depend on its order)
__device__ __forceinline__ void prio_take(uint64_t &bk, int &bi, uint64_t k, int i)
{
    if (i >= 0 && (bi < 0 || prio_gt(k, i, bk, bi))) {
        bk = k;
        bi = i;
    }
}

template <int G>
__device__ __forceinline__ void prio_group_max(uint64_t &bk, int &bi)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const uint64_t k = __shfl_xor_sync(0xffffffffu, (unsigned long long)bk, off, G);
        const int i = __shfl_xor_sync(0xffffffffu, bi, off, G);
        prio_take(bk, bi, k, i);
    }
}

template <int G>
__device__ __forceinline__ bool group_any(bool f)
{
    unsigned v = f ? 1u : 0u;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, off, G);
    return v != 0;
}

// m1(i) = max undecided (key, index) over {i} and its strong neighbours
template <int G>
__global__ void k_mis_max1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const unsigned char *__restrict__ S, const unsigned char *__restrict__ state,
                           uint64_t seed, int level, unsigned long long *__restrict__ mk, int *__restrict__ mi)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        const int i = (int)ii;
        uint64_t bk = 0;
        int bi = -1;
        if (ii < n) {
            if (lane == 0 && state[i] == MIS_UNDECIDED) prio_take(bk, bi, prio_key(seed, level, i), i);
            for (int e = rp[i] + lane; e < rp[i + 1]; e += G) {
                if (!S[e]) continue;
                const int j = ci[e];
                if (state[j] != MIS_UNDECIDED) continue;
                prio_take(bk, bi, prio_key(seed, level, j), j);
            }
        }
        prio_group_max<G>(bk, bi);
        if (lane == 0 && ii < n) {
            mk[i] = bk;
            mi[i] = bi;
        }
    }
}

// an undecided i whose m2 = max of m1 over {i} and its strong neighbours is
// i itself becomes a root
template <int G>
__global__ void k_mis_select(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const unsigned char *__restrict__ S, unsigned char *__restrict__ state,
                             const unsigned long long *__restrict__ mk, const int *__restrict__ mi)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        const int i = (int)ii;
        const bool live = ii < n && state[i] == MIS_UNDECIDED;
        uint64_t bk = 0;
        int bi = -1;
        if (live) {
            if (lane == 0) prio_take(bk, bi, mk[i], mi[i]);
            for (int e = rp[i] + lane; e < rp[i + 1]; e += G) {
                if (!S[e]) continue;
                const int j = ci[e];
                prio_take(bk, bi, mk[j], mi[j]);
            }
        }
        prio_group_max<G>(bk, bi);
        if (lane == 0 && live && bi == i) state[i] = MIS_ROOT;
    }
}

// near1(i): i is a root or has a strong neighbour that is one
template <int G>
__global__ void k_mis_near1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            const unsigned char *__restrict__ S, const unsigned char *__restrict__ state,
                            unsigned char *__restrict__ near1)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        const int i = (int)ii;
        bool f = false;
        if (ii < n) {
            f = lane == 0 && state[i] == MIS_ROOT;
            for (int e = rp[i] + lane; e < rp[i + 1] && !f; e += G)
                if (S[e] && state[ci[e]] == MIS_ROOT) f = true;
        }
        f = group_any<G>(f);
        if (lane == 0 && ii < n) near1[i] = f;
    }
}

// an undecided node within two hops of a root leaves; the others are counted
template <int G>
__global__ void k_mis_remove(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const unsigned char *__restrict__ S, unsigned char *__restrict__ state,
                             const unsigned char *__restrict__ near1, int *__restrict__ undecided)
{
    const int lane = threadIdx.x & (G - 1);
    GROUP_LOOP(G, ii, n)
    {
        const int i = (int)ii;
        const bool live = ii < n && state[i] == MIS_UNDECIDED;
        bool f = false;
        if (live) {
            f = lane == 0 && near1[i];
            for (int e = rp[i] + lane; e < rp[i + 1] && !f; e += G)
                if (S[e] && near1[ci[e]]) f = true;
        }
        f = group_any<G>(f);
        if (lane == 0 && live) {
            if (f) state[i] = MIS_OUT;
            else atomicAdd(undecided, 1);
        }
    }
}

__global__ void k_mis_roots(int n, const unsigned char *__restrict__ state, unsigned char *__restrict__ root)
{
    GRID_STRIDE(i, n) root[i] = state[i] == MIS_ROOT;
}

int setup_mis2(const DCSR &A, const unsigned char *S, uint64_t seed, int level, DBuf<unsigned char> &root,
               int max_rounds, cudaStream_t st)
{
    const int n = A.nr;
    DBuf<unsigned char> state((size_t)n), near1((size_t)n);
    DBuf<unsigned long long> mk((size_t)n);
    DBuf<int> mi((size_t)n), cnt(1);
    root.alloc((size_t)n);
    GW_CUDA(cudaMemsetAsync(state.p, 0, (size_t)n, st));
    const int g = nblk(n, 256);
    const int G = row_lanes(A), gg = nblk((long long)n * G, 256);
    auto mis_round = [&](auto lanes) {
        constexpr int L = decltype(lanes)::value;
        gw_launch(k_mis_max1<L>, gg, 256, 0, st, n, A.rp.p, A.ci.p, S, state.p, seed, level, mk.p, mi.p);
        gw_launch(k_mis_select<L>, gg, 256, 0, st, n, A.rp.p, A.ci.p, S, state.p, mk.p, mi.p);
        gw_launch(k_mis_near1<L>, gg, 256, 0, st, n, A.rp.p, A.ci.p, S, state.p, near1.p);
        gw_launch(k_mis_remove<L>, gg, 256, 0, st, n, A.rp.p, A.ci.p, S, state.p, near1.p, cnt.p);
    };
    int rounds = 0;
    for (;;) {
        if (rounds >= max_rounds) fail(GW_ERR_SETUP, "MIS-2 did not finish in %d rounds on level %d", max_rounds, level);
        ++rounds;
        GW_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int), st));
        if (G == 1) mis_round(std::integral_constant<int, 1>());
        else if (G == 8) mis_round(std::integral_constant<int, 8>());
        else mis_round(std::integral_constant<int, 32>());
        GW_LAUNCH_CHECK();
        if (read_int(cnt.p, st) == 0) break;
    }
    gw_launch(k_mis_roots, g, 256, 0, st, n, state.p, root.p);
    GW_LAUNCH_CHECK();
    return rounds;
}

// -------------------------------------------------------------- aggregates --
__global__ void k_root_flag(int n, const unsigned char *__restrict__ root, int *__restrict__ f)
{
    GRID_STRIDE(i, n) f[i] = root[i] ? 1 : 0;
}

// roots take their scan index; strong neighbours of a root join it
__global__ void k_join1(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                        const unsigned char *__restrict__ S, const unsigned char *__restrict__ root,
                        const int *__restrict__ id, int *__restrict__ agg1, int *__restrict__ rootof)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        int a = -1, r = -1;
        if (root[i]) {
            a = id[i];
            r = i;
        } else {
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int j = ci[e];
                if (S[e] && j != i && root[j]) {
                    a = id[j];
                    r = j;
                    break;
                }
            }
        }
        agg1[i] = a;
        rootof[i] = r;
    }
}

// remaining nodes join the step-1 neighbour whose root has the largest (key, index)
__global__ void k_join2(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                        const unsigned char *__restrict__ S, const int *__restrict__ agg1,
                        const int *__restrict__ rootof, uint64_t seed, int level, int *__restrict__ agg,
                        int *__restrict__ bad)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        if (agg1[i] >= 0) {
            agg[i] = agg1[i];
            continue;
        }
        int best = -1;
        uint64_t bk = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (!S[e] || j == i || agg1[j] < 0) continue;
            const int r = rootof[j];
            const uint64_t k = prio_key(seed, level, r);
            if (best < 0 || k > bk || (k == bk && r > best)) {
                best = r;
                bk = k;
            }
        }
        if (best < 0) {
            agg[i] = -1;
            atomicAdd(bad, 1);
        } else {
            agg[i] = agg1[best];
        }
    }
}

int setup_aggregate(const DCSR &A, const unsigned char *S, const unsigned char *root, uint64_t seed, int level,
                    DBuf<int> &agg, cudaStream_t st)
{
    const int n = A.nr;
    DBuf<int> id((size_t)n + 1), agg1((size_t)n), rootof((size_t)n), bad(1);
    agg.alloc((size_t)n);
    const int g = nblk(n, 256);
    gw_launch(k_root_flag, g, 256, 0, st, n, root, id.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(id.p, id.p, n, st);
    gw_launch(k_join1, g, 256, 0, st, n, A.rp.p, A.ci.p, S, root, id.p, agg1.p, rootof.p);
    GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    gw_launch(k_join2, g, 256, 0, st, n, A.rp.p, A.ci.p, S, agg1.p, rootof.p, seed, level, agg.p, bad.p);
    GW_LAUNCH_CHECK();
    if (read_int(bad.p, st)) fail(GW_ERR_SETUP, "aggregation left nodes unassigned on level %d", level);
    return read_int(id.p + n, st);
}

// ------------------------------------------------------ smoothed prolongator --
// A_F: weak off-diagonals dropped and added to the diagonal in ascending
// column order; rho = max over rows with a strong neighbour of
// (sum_j |a^F_ij|, ascending j) / a^F_ii.
__global__ void k_filter(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const double *__restrict__ v, const unsigned char *__restrict__ S,
                         const double *__restrict__ d, double *__restrict__ aF, unsigned char *__restrict__ hs,
                         unsigned long long *__restrict__ rho_bits)
{
    unsigned long long best = 0;
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double di = d[i];
        unsigned char h = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (j == i) continue;
            if (S[e]) h = 1;
            else di = __dadd_rn(di, v[e]);
        }
        aF[i] = di;
        hs[i] = h;
        if (!h) continue;
        double s = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (j == i) s = __dadd_rn(s, fabs(di));
            else if (S[e]) s = __dadd_rn(s, fabs(v[e]));
        }
        const double ratio = __ddiv_rn(s, di);
        if (ratio > 0.0 && isfinite(ratio)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(ratio);
            best = b > best ? b : best;
        }
    }
    block_atomic_max(best, rho_bits);
}

__device__ __forceinline__ bool p_member(int i, int j, unsigned char s) { return j == i || s; }

__global__ void k_p_count(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                          const unsigned char *__restrict__ S, const int *__restrict__ agg,
                          const unsigned char *__restrict__ hs, int *__restrict__ cnt)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        if (!hs[i]) {
            cnt[i] = 1;
            continue;
        }
        int c = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (!p_member(i, j, S[e])) continue;
            const int a = agg[j];
            bool dup = false;
            for (int f = rp[i]; f < e && !dup; ++f)
                if (p_member(i, ci[f], S[f]) && agg[ci[f]] == a) dup = true;
            if (!dup) ++c;
        }
        cnt[i] = c;
    }
}

// P(i,c) = [c == agg(i)] - s_i * sum_{j in {i} U S(i), agg(j) = c} a^F_ij,
// s_i = omega / a^F_ii, sums in ascending j; columns ascending.
__global__ void k_p_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                         const double *__restrict__ v, const unsigned char *__restrict__ S,
                         const int *__restrict__ agg, const unsigned char *__restrict__ hs,
                         const double *__restrict__ aF, double omega, const int *__restrict__ prp,
                         int *__restrict__ pci, double *__restrict__ pv)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        int o = prp[i];
        const int ai = agg[i];
        if (!hs[i]) {
            pci[o] = ai;
            pv[o] = 1.0;
            continue;
        }
        const double s = __ddiv_rn(omega, aF[i]);
        const int cnt = prp[i + 1] - o;
        int last = -1;
        for (int t = 0; t < cnt; ++t) {
            int c = 0x7fffffff;
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int j = ci[e];
                if (!p_member(i, j, S[e])) continue;
                const int a = agg[j];
                if (a > last && a < c) c = a;
            }
            double acc = 0.0;
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int j = ci[e];
                if (!p_member(i, j, S[e]) || agg[j] != c) continue;
                acc = __dadd_rn(acc, j == i ? aF[i] : v[e]);
            }
            const double delta = c == ai ? 1.0 : 0.0;
            pci[o + t] = c;
            pv[o + t] = __dsub_rn(delta, __dmul_rn(s, acc));
            last = c;
        }
    }
}

// The same two passes with a warp per row, for levels whose rows are long
// (the thread-per-row passes above are quadratic in the row length).  The
// row's member aggregates (j = i or strong) go to shared memory; an entry is
// the first occurrence of its aggregate if no earlier entry has it; the
// first occurrences are counted, and each one's column is its rank among
// them, its value the sum over the row's entries of that aggregate in
// ascending j, as in k_p_fill.  Rows of more than PW_MAX entries take the
// serial path on lane 0.
constexpr int PW_MAX = 256, PW_WARPS = 8;

__device__ void pw_load(int i, int e0, int len, const int *__restrict__ ci, const unsigned char *__restrict__ S,
                        const int *__restrict__ agg, int *sagg, unsigned char *sfirst, int lane)
{
    for (int t = lane; t < len; t += 32) {
        const int j = ci[e0 + t];
        sagg[t] = p_member(i, j, S[e0 + t]) ? agg[j] : -1;
    }
    __syncwarp();
    for (int t = lane; t < len; t += 32) {
        const int a = sagg[t];
        bool first = a >= 0;
        for (int u = 0; u < t && first; ++u)
            if (sagg[u] == a) first = false;
        sfirst[t] = first;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * PW_WARPS) k_p_count_w(int n, const int *__restrict__ rp,
                                                            const int *__restrict__ ci,
                                                            const unsigned char *__restrict__ S,
                                                            const int *__restrict__ agg,
                                                            const unsigned char *__restrict__ hs,
                                                            int *__restrict__ cnt)
{
    __shared__ int sagg_all[PW_WARPS][PW_MAX];
    __shared__ unsigned char sfirst_all[PW_WARPS][PW_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long ii = (long long)blockIdx.x * PW_WARPS + w; ii < n; ii += (long long)gridDim.x * PW_WARPS) {
        const int i = (int)ii, e0 = rp[i], len = rp[i + 1] - e0;
        if (!hs[i]) {
            if (lane == 0) cnt[i] = 1;
            continue;
        }
        int c = 0;
        if (len > PW_MAX) {
            if (lane == 0) {
                for (int e = e0; e < e0 + len; ++e) {
                    const int j = ci[e];
                    if (!p_member(i, j, S[e])) continue;
                    const int a = agg[j];
                    bool dup = false;
                    for (int f = e0; f < e && !dup; ++f)
                        if (p_member(i, ci[f], S[f]) && agg[ci[f]] == a) dup = true;
                    if (!dup) ++c;
                }
                cnt[i] = c;
            }
            continue;
        }
        pw_load(i, e0, len, ci, S, agg, sagg_all[w], sfirst_all[w], lane);
        for (int t = lane; t < len; t += 32) c += sfirst_all[w][t];
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (lane == 0) cnt[i] = c;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * PW_WARPS) k_p_fill_w(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ ci, const double *__restrict__ v,
                                                           const unsigned char *__restrict__ S,
                                                           const int *__restrict__ agg,
                                                           const unsigned char *__restrict__ hs,
                                                           const double *__restrict__ aF, double omega,
                                                           const int *__restrict__ prp, int *__restrict__ pci,
                                                           double *__restrict__ pv)
{
    __shared__ int sagg_all[PW_WARPS][PW_MAX];
    __shared__ unsigned char sfirst_all[PW_WARPS][PW_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *sagg = sagg_all[w];
    unsigned char *sfirst = sfirst_all[w];
    for (long long ii = (long long)blockIdx.x * PW_WARPS + w; ii < n; ii += (long long)gridDim.x * PW_WARPS) {
        const int i = (int)ii, e0 = rp[i], len = rp[i + 1] - e0;
        const int o = prp[i], ai = agg[i];
        if (!hs[i]) {
            if (lane == 0) {
                pci[o] = ai;
                pv[o] = 1.0;
            }
            continue;
        }
        const double s = __ddiv_rn(omega, aF[i]);
        if (len > PW_MAX) {
            if (lane == 0) {
                const int cnt = prp[i + 1] - o;
                int last = -1;
                for (int t = 0; t < cnt; ++t) {
                    int c = 0x7fffffff;
                    for (int e = e0; e < e0 + len; ++e) {
                        const int j = ci[e];
                        if (!p_member(i, j, S[e])) continue;
                        const int a = agg[j];
                        if (a > last && a < c) c = a;
                    }
                    double acc = 0.0;
                    for (int e = e0; e < e0 + len; ++e) {
                        const int j = ci[e];
                        if (!p_member(i, j, S[e]) || agg[j] != c) continue;
                        acc = __dadd_rn(acc, j == i ? aF[i] : v[e]);
                    }
                    pci[o + t] = c;
                    pv[o + t] = __dsub_rn(c == ai ? 1.0 : 0.0, __dmul_rn(s, acc));
                    last = c;
                }
            }
            continue;
        }
        pw_load(i, e0, len, ci, S, agg, sagg, sfirst, lane);
        for (int t = lane; t < len; t += 32) {
            if (!sfirst[t]) continue;
            const int a = sagg[t];
            int rank = 0;
            for (int u = 0; u < len; ++u) rank += sfirst[u] && sagg[u] < a;
            double acc = 0.0;
            for (int u = t; u < len; ++u)
                if (sagg[u] == a) acc = __dadd_rn(acc, ci[e0 + u] == i ? aF[i] : v[e0 + u]);
            pci[o + rank] = a;
            pv[o + rank] = __dsub_rn(a == ai ? 1.0 : 0.0, __dmul_rn(s, acc));
        }
        __syncwarp();
    }
}

void setup_smooth_p(const DCSR &A, const unsigned char *S, const int *agg, int nagg, DCSR &P, double *omega,
                    double *rho, cudaStream_t st)
{
    const int n = A.nr;
    DBuf<double> d((size_t)n), aF((size_t)n);
    DBuf<unsigned char> hs((size_t)n);
    DBuf<unsigned long long> rb(1);
    const int g = nblk(n, 256);
    gw_launch(k_diag, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, d.p);
    GW_CUDA(cudaMemsetAsync(rb.p, 0, sizeof(unsigned long long), st));
    gw_launch(k_filter, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, S, d.p, aF.p, hs.p, rb.p);
    GW_LAUNCH_CHECK();
    unsigned long long bits = 0;
    GW_CUDA(cudaMemcpyAsync(&bits, rb.p, sizeof bits, cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    double r;
    memcpy(&r, &bits, sizeof r);
    *rho = r;
    *omega = r > 0.0 ? (4.0 / 3.0) / r : 0.0;
    P.nr = n;
    P.nc = nagg;
    P.rp.alloc((size_t)n + 1);
    // a warp a row where rows are long (the coarse levels), a thread a row otherwise
    const bool warp_rows = setup_forms() ? setup_forms() == 2 : n > 0 && (double)A.nnz / n > 12.0;
    const int gw_ = (int)std::max(1LL, std::min<long long>(((long long)n + PW_WARPS - 1) / PW_WARPS, 152LL * 64));
    if (warp_rows) gw_launch(k_p_count_w, gw_, 32 * PW_WARPS, 0, st, n, A.rp.p, A.ci.p, S, agg, hs.p, P.rp.p);
    else gw_launch(k_p_count, g, 256, 0, st, n, A.rp.p, A.ci.p, S, agg, hs.p, P.rp.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(P.rp.p, P.rp.p, n, st);
    P.nnz = read_int(P.rp.p + n, st);
    P.ci.alloc((size_t)P.nnz);
    P.v.alloc((size_t)P.nnz);
    if (warp_rows)
        gw_launch(k_p_fill_w, gw_, 32 * PW_WARPS, 0, st, n, A.rp.p, A.ci.p, A.v.p, S, agg, hs.p, aF.p, *omega, P.rp.p,
                  P.ci.p, P.v.p);
    else
        gw_launch(k_p_fill, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, S, agg, hs.p, aF.p, *omega, P.rp.p, P.ci.p,
                  P.v.p);
    GW_LAUNCH_CHECK();
}

// s_i and the strong +x, +y, +z couplings of the implicit level-0 prolongator
__global__ void k_p_implicit(int n, int nx, int sxy, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, const unsigned char *__restrict__ S,
                             const double *__restrict__ aF, const unsigned char *__restrict__ hs, double omega,
                             float *__restrict__ s, float *__restrict__ fx, float *__restrict__ fy,
                             float *__restrict__ fz, int *__restrict__ bad)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double a = 0.0, b = 0.0, c = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const long long j = ci[e];
            if (j == i) continue;
            const double x = S[e] ? v[e] : 0.0;
            if (j == (long long)i + sxy) c = x;
            else if (j == (long long)i + nx) b = x;
            else if (j == (long long)i + 1) a = x;
            else if (!(j == (long long)i - sxy || j == (long long)i - nx || j == (long long)i - 1)) atomicAdd(bad, 1);
        }
        s[i] = hs[i] ? (float)__ddiv_rn(omega, aF[i]) : 0.f;
        fx[i] = (float)a;
        fy[i] = (float)b;
        fz[i] = (float)c;
    }
}

__global__ void k_tent(int n, const int *__restrict__ agg, int *__restrict__ rp, int *__restrict__ ci,
                       double *__restrict__ v)
{
    GRID_STRIDE(i, (long long)n + 1)
    {
        rp[i] = (int)i;
        if (i < n) {
            ci[i] = agg[i];
            v[i] = 1.0;
        }
    }
}

void setup_transpose(const DCSR &P, DCSR &R, cudaStream_t st);

bool setup_implicit_p(const DCSR &A, const unsigned char *S, const int *agg, int nagg, double omega, int nx, int ny,
                      int nz, ImplP &out, cudaStream_t st)
{
    out = ImplP();
    const int n = A.nr;
    if (nx < 1 || (long long)nx * ny * nz != n || !(omega > 0.0)) return false;
    DBuf<double> d((size_t)n), aF((size_t)n);
    DBuf<unsigned char> hs((size_t)n);
    DBuf<unsigned long long> rb(1);
    DBuf<int> bad(1);
    const int g = nblk(n, 256);
    gw_launch(k_diag, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, d.p);
    GW_CUDA(cudaMemsetAsync(rb.p, 0, sizeof(unsigned long long), st));
    GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    gw_launch(k_filter, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, S, d.p, aF.p, hs.p, rb.p);
    out.s.alloc((size_t)n);
    out.fx.alloc((size_t)n);
    out.fy.alloc((size_t)n);
    out.fz.alloc((size_t)n);
    gw_launch(k_p_implicit, g, 256, 0, st, n, nx, nx * ny, A.rp.p, A.ci.p, A.v.p, S, aF.p, hs.p, omega, out.s.p, out.fx.p,
                                    out.fy.p, out.fz.p, bad.p);
    GW_LAUNCH_CHECK();
    if (read_int(bad.p, st) != 0) {
        out = ImplP();
        return false;
    }
    // member lists: rows of the tentative prolongator's transpose
    DCSR Pt, Rt;
    Pt.nr = n;
    Pt.nc = nagg;
    Pt.nnz = n;
    Pt.rp.alloc((size_t)n + 1);
    Pt.ci.alloc((size_t)n);
    Pt.v.alloc((size_t)n);
    gw_launch(k_tent, nblk((long long)n + 1, 256), 256, 0, st, n, agg, Pt.rp.p, Pt.ci.p, Pt.v.p);
    GW_LAUNCH_CHECK();
    setup_transpose(Pt, Rt, st);
    out.mptr = std::move(Rt.rp);
    out.mem = std::move(Rt.ci);
    out.nc = nagg;
    out.n = n;
    out.nx = nx;
    out.sxy = nx * ny;
    out.w0 = (float)(1.0 - omega);
    return true;
}

// ---------------------------------------------------------------- transpose --
__global__ void k_tr_count(int nnz, const int *__restrict__ ci, int *__restrict__ cnt)
{
    GRID_STRIDE(e, nnz) atomicAdd(&cnt[ci[e]], 1);
}

__global__ void k_tr_scatter(int nr, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, const int *__restrict__ rrp, int *__restrict__ fill,
                             int *__restrict__ tci, double *__restrict__ tv)
{
    GRID_STRIDE(ii, nr)
    {
        const int i = (int)ii;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int c = ci[e];
            const int pos = rrp[c] + atomicAdd(&fill[c], 1);
            tci[pos] = i;
            tv[pos] = v[e];
        }
    }
}

// one warp per row: every entry moves to its rank among the row's (unique) keys
__global__ void k_rank_sort_rows(int nr, const int *__restrict__ rp, const int *__restrict__ kin,
                                 const double *__restrict__ vin, int *__restrict__ kout, double *__restrict__ vout)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = w0; r < nr; r += nw) {
        const int b = rp[r], m = rp[r + 1] - b;
        for (int k = lane; k < m; k += 32) {
            const int key = kin[b + k];
            int rank = 0;
            for (int t = 0; t < m; ++t) rank += kin[b + t] < key;
            kout[b + rank] = key;
            vout[b + rank] = vin[b + k];
        }
    }
}

void setup_transpose(const DCSR &P, DCSR &R, cudaStream_t st)
{
    R.nr = P.nc;
    R.nc = P.nr;
    R.nnz = P.nnz;
    R.rp.alloc((size_t)R.nr + 1);
    R.ci.alloc((size_t)R.nnz);
    R.v.alloc((size_t)R.nnz);
    DBuf<int> fill((size_t)R.nr), tci((size_t)R.nnz);
    DBuf<double> tv((size_t)R.nnz);
    GW_CUDA(cudaMemsetAsync(R.rp.p, 0, ((size_t)R.nr + 1) * sizeof(int), st));
    GW_CUDA(cudaMemsetAsync(fill.p, 0, (size_t)R.nr * sizeof(int), st));
    gw_launch(k_tr_count, nblk(P.nnz, 256), 256, 0, st, P.nnz, P.ci.p, R.rp.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(R.rp.p, R.rp.p, R.nr, st);
    gw_launch(k_tr_scatter, nblk(P.nr, 256), 256, 0, st, P.nr, P.rp.p, P.ci.p, P.v.p, R.rp.p, fill.p, tci.p, tv.p);
    gw_launch(k_rank_sort_rows, nblk((long long)R.nr * 32, 256), 256, 0, st, R.nr, R.rp.p, tci.p, tv.p, R.ci.p, R.v.p);
    GW_LAUNCH_CHECK();
    GW_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------- SpGEMM --
// C = L * Rm.  Pass 1 (symbolic) collects the distinct columns of each output
// row in a per-warp open-addressing table in shared memory and counts them;
// after a scan of the counts, pass 2 (numeric) rebuilds the set, sorts it
// (rank sort), and accumulates C(i,c) = sum over L's row i in ascending
// column k of L(i,k) * Rm(k,c): the warp walks L's row in order and its lanes
// take the entries of Rm's row k, which have distinct columns, so every
// output entry receives its terms in ascending k.
constexpr int SG_HMAX = 8192;
constexpr int SG_SMEM_MAX = 96 << 10;  // per block: W warps x 12 bytes x H <= 96 KB

__global__ void k_sg_bound(int nr, int ncol, const int *__restrict__ lrp, const int *__restrict__ lci,
                           const int *__restrict__ rrp, int *__restrict__ maxub)
{
    int best = 0;
    GRID_STRIDE(ii, nr)
    {
        const int i = (int)ii;
        long long ub = 0;
        for (int e = lrp[i]; e < lrp[i + 1]; ++e) {
            const int k = lci[e];
            ub += rrp[k + 1] - rrp[k];
        }
        best = max(best, (int)(ub < (long long)ncol ? ub : (long long)ncol));
    }
    atomicMax(maxub, best);
}

__device__ __forceinline__ unsigned sg_hash(int c) { return (unsigned)c * 2654435761u; }

__device__ __forceinline__ int sg_insert(int *keys, int H, int c)
{
    unsigned h = sg_hash(c) & (unsigned)(H - 1);
    for (int probe = 0; probe < H; ++probe) {
        int old = atomicCAS(&keys[h], -1, c);
        if (old == -1) return 1;
        if (old == c) return 0;
        h = (h + 1) & (unsigned)(H - 1);
    }
    return -1000000;  // table full: flagged by the caller through the count
}

// Table size for one row: the smallest power of two (at least 32, at most H)
// of at least twice the row's bound on distinct columns.
__device__ __forceinline__ int sg_row_table(const int *__restrict__ lrp, const int *__restrict__ lci,
                                            const int *__restrict__ rrp, int row, int H, int lane)
{
    int ub = 0;
    for (int e = lrp[row] + lane; e < lrp[row + 1]; e += 32) ub += rrp[lci[e] + 1] - rrp[lci[e]];
    for (int off = 16; off > 0; off >>= 1) ub += __shfl_xor_sync(0xffffffffu, ub, off);
    int h = 32;
    while (h < 2 * ub && h < H) h <<= 1;
    return h;
}

__device__ int sg_build_set(const int *__restrict__ lrp, const int *__restrict__ lci, const int *__restrict__ rrp,
                            const int *__restrict__ rci, int row, int *keys, int H, int lane)
{
    for (int t = lane; t < H; t += 32) keys[t] = -1;
    __syncwarp();
    int mine = 0;
    for (int e = lrp[row]; e < lrp[row + 1]; ++e) {
        const int k = lci[e];
        for (int f = rrp[k] + lane; f < rrp[k + 1]; f += 32) mine += sg_insert(keys, H, rci[f]);
    }
    __syncwarp();
    for (int off = 16; off > 0; off >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, off);
    return mine;
}

// Distinct columns of every row (table per row sized by its own bound), and
// their maximum, which sizes the numeric pass's tables.
__global__ void k_sg_symbolic(int nr, const int *__restrict__ rows, const int *__restrict__ lrp,
                              const int *__restrict__ lci, const int *__restrict__ rrp, const int *__restrict__ rci,
                              int H, int *__restrict__ cnt, int *__restrict__ overflow, int *__restrict__ maxu)
{
    extern __shared__ int sg_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    int *keys = sg_smem + (size_t)w * H;
    int best = 0;
    for (long long rr = (long long)blockIdx.x * W + w; rr < nr; rr += (long long)gridDim.x * W) {
        const int row = rows ? rows[rr] : (int)rr;
        const int Hr = sg_row_table(lrp, lci, rrp, (int)row, H, lane);
        int u = sg_build_set(lrp, lci, rrp, rci, (int)row, keys, Hr, lane);
        if (lane == 0) {
            if (u < 0 || u > Hr / 2) atomicOr(overflow, 1);
            cnt[row] = u < 0 ? 0 : u;
        }
        best = max(best, u);
        __syncwarp();
    }
    if (lane == 0 && best > 0) atomicMax(maxu, best);
}

__global__ void k_sg_numeric(int nr, const int *__restrict__ rows, const int *__restrict__ lrp,
                             const int *__restrict__ lci, const double *__restrict__ lv, const int *__restrict__ rrp,
                             const int *__restrict__ rci, const double *__restrict__ rv, int H,
                             const int *__restrict__ crp, int *__restrict__ cci, double *__restrict__ cv)
{
    extern __shared__ int sg_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, W = blockDim.x >> 5;
    // per warp: keys[H] ints, list[H] ints, acc[H/2] doubles
    char *base = (char *)sg_smem + (size_t)w * (size_t)H * 12;
    int *keys = (int *)base;
    int *list = keys + H;
    double *acc = (double *)(list + H);
    for (long long rr = (long long)blockIdx.x * W + w; rr < nr; rr += (long long)gridDim.x * W) {
        const int row = rows ? rows[rr] : (int)rr;
        sg_build_set(lrp, lci, rrp, rci, row, keys, H, lane);
        // compact the table into list (any order), then rank-sort into keys
        int u = 0;
        for (int t0 = 0; t0 < H; t0 += 32) {
            const int t = t0 + lane;
            const int c = keys[t];
            const unsigned m = __ballot_sync(0xffffffffu, c != -1);
            if (c != -1) list[u + __popc(m & ((1u << lane) - 1u))] = c;
            u += __popc(m);
        }
        __syncwarp();
        const int o = crp[row];
        for (int k = lane; k < u; k += 32) {
            const int c = list[k];
            int rank = 0;
            for (int t = 0; t < u; ++t) rank += list[t] < c;
            keys[rank] = c;
            cci[o + rank] = c;
        }
        for (int k = lane; k < u; k += 32) acc[k] = 0.0;
        __syncwarp();
        for (int e = lrp[row]; e < lrp[row + 1]; ++e) {
            const int k = lci[e];
            const double a = lv[e];
            for (int f = rrp[k] + lane; f < rrp[k + 1]; f += 32) {
                const int c = rci[f];
                int lo = 0, hi = u - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (keys[mid] < c) lo = mid + 1;
                    else hi = mid;
                }
                acc[lo] = __dadd_rn(acc[lo], __dmul_rn(a, rv[f]));
            }
            __syncwarp();
        }
        for (int k = lane; k < u; k += 32) cv[o + k] = acc[k];
        __syncwarp();
    }
}

// Short rows, one thread each: the distinct columns of the row kept as a
// sorted list in shared memory (entry t of thread x at [t * SGT_BS + x], so
// the threads of a warp touch distinct banks).  Symbolic: counts the row's
// distinct columns; a row with more than SGT_CAP of them goes to the warp
// kernels' row list instead.  Numeric: inserts each product L(i,k) Rm(k,c)
// in L's column order k, so every output entry receives its terms in
// ascending k, the same sums as the warp kernel forms.
constexpr int SGT_BS = 128, SGT_CAP = 64;

__device__ __forceinline__ int sgt_find(const int *list, int u, int c)
{
    int lo = 0, hi = u;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (list[mid * SGT_BS] < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(SGT_BS) k_sgt_symbolic(int nr, const int *__restrict__ lrp, const int *__restrict__ lci,
                                                        const int *__restrict__ rrp, const int *__restrict__ rci,
                                                        int *__restrict__ cnt, int *__restrict__ long_rows,
                                                        int *__restrict__ nlong, int *__restrict__ maxu)
{
    __shared__ int sl[SGT_CAP * SGT_BS];
    int *list = sl + threadIdx.x;
    int best = 0;
    GRID_STRIDE(ii, nr)
    {
        const int i = (int)ii;
        int u = 0;
        bool over = false;
        for (int e = lrp[i]; e < lrp[i + 1] && !over; ++e) {
            const int k = lci[e];
            for (int f = rrp[k]; f < rrp[k + 1]; ++f) {
                const int c = rci[f];
                const int pos = sgt_find(list, u, c);
                if (pos < u && list[pos * SGT_BS] == c) continue;
                if (u == SGT_CAP) {
                    over = true;
                    break;
                }
                for (int t = u; t > pos; --t) list[t * SGT_BS] = list[(t - 1) * SGT_BS];
                list[pos * SGT_BS] = c;
                ++u;
            }
        }
        if (over) {
            long_rows[atomicAdd(nlong, 1)] = i;
        } else {
            cnt[i] = u;
            best = max(best, u);
        }
    }
    if (best > 0) atomicMax(maxu, best);
}

template <int CAP>
__global__ void __launch_bounds__(SGT_BS) k_sgt_numeric(int nr, const int *__restrict__ lrp, const int *__restrict__ lci,
                                                       const double *__restrict__ lv, const int *__restrict__ rrp,
                                                       const int *__restrict__ rci, const double *__restrict__ rv,
                                                       const int *__restrict__ crp, int *__restrict__ cci,
                                                       double *__restrict__ cv)
{
    extern __shared__ double sgt_smem[];  // acc[CAP * SGT_BS] doubles, then list[CAP * SGT_BS] ints
    double *acc = sgt_smem + threadIdx.x;
    int *list = (int *)(sgt_smem + CAP * SGT_BS) + threadIdx.x;
    GRID_STRIDE(ii, nr)
    {
        const int i = (int)ii;
        const int o = crp[i], cnt = crp[i + 1] - o;
        if (cnt > CAP) continue;  // a long row: the warp kernel's
        int u = 0;
        for (int e = lrp[i]; e < lrp[i + 1]; ++e) {
            const int k = lci[e];
            const double a = lv[e];
            for (int f = rrp[k]; f < rrp[k + 1]; ++f) {
                const int c = rci[f];
                const int pos = sgt_find(list, u, c);
                if (!(pos < u && list[pos * SGT_BS] == c)) {
                    for (int t = u; t > pos; --t) {
                        list[t * SGT_BS] = list[(t - 1) * SGT_BS];
                        acc[t * SGT_BS] = acc[(t - 1) * SGT_BS];
                    }
                    list[pos * SGT_BS] = c;
                    acc[pos * SGT_BS] = 0.0;
                    ++u;
                }
                acc[pos * SGT_BS] = __dadd_rn(acc[pos * SGT_BS], __dmul_rn(a, rv[f]));
            }
        }
        for (int t = 0; t < u; ++t) {
            cci[o + t] = list[t * SGT_BS];
            cv[o + t] = acc[t * SGT_BS];
        }
    }
}

void setup_spgemm(const DCSR &L, const DCSR &Rm, DCSR &C, cudaStream_t st)
{
    // 0: long rows, 1: their count, 2: largest distinct count of the short rows,
    // 3: bound of the long rows, 4: overflow, 5: largest distinct count of the long rows
    DBuf<int> ctr(6), long_rows;
    GW_CUDA(cudaMemsetAsync(ctr.p, 0, ctr.bytes(), st));
    C.nr = L.nr;
    C.nc = Rm.nc;
    C.rp.alloc((size_t)C.nr + 1);
    // A thread a row pays off for many short rows (the level-0 products A P
    // with about 24 products a row, 2M rows); with few rows or hundreds of
    // products a row a warp a row is faster.  Products a row estimated from
    // the mean row lengths.
    const double per_row = L.nr ? (double)L.nnz / L.nr * ((double)Rm.nnz / std::max(1, Rm.nr)) : 0.0;
    const bool thread_rows = setup_forms() ? setup_forms() == 1 : L.nr >= 32768 && per_row <= 128.0;
    const int gt = nblk(L.nr, SGT_BS, 152LL * 64);
    int nlong = L.nr, mu_short = 0;
    if (thread_rows) {
        long_rows.alloc((size_t)L.nr);
        gw_launch(k_sgt_symbolic, gt, SGT_BS, 0, st, L.nr, L.rp.p, L.ci.p, Rm.rp.p, Rm.ci.p, C.rp.p, long_rows.p,
                  ctr.p + 1, ctr.p + 2);
        GW_LAUNCH_CHECK();
        int hc[2];
        GW_CUDA(cudaMemcpyAsync(hc, ctr.p + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
        nlong = hc[0];
        mu_short = hc[1];
    }
    const int *rows = thread_rows ? (const int *)long_rows.p : nullptr;
    // The attribute is global to the kernel, and setups may run concurrently on
    // several threads: always set the same value, the largest any launch uses.
    GW_CUDA(cudaFuncSetAttribute(k_sg_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize, SG_SMEM_MAX));
    GW_CUDA(cudaFuncSetAttribute(k_sg_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, SG_SMEM_MAX));
    int Hn = 0, Wn = 0;
    if (nlong > 0) {
        // rows with more than SGT_CAP distinct columns: a warp each
        gw_launch(k_sg_bound, nblk(L.nr, 256), 256, 0, st, L.nr, Rm.nc, L.rp.p, L.ci.p, Rm.rp.p, ctr.p + 3);
        GW_LAUNCH_CHECK();
        const int ub = read_int(ctr.p + 3, st);
        int H = 32;
        while (H < 2 * ub && H < SG_HMAX) H <<= 1;
        // warps per block so that a block's tables stay within 96 KB
        const int W = (int)std::max<size_t>(1, std::min<size_t>(8, (96u << 10) / ((size_t)H * sizeof(int))));
        const size_t smem_sym = (size_t)W * H * sizeof(int);
        if (smem_sym > (size_t)SG_SMEM_MAX)
            fail(GW_ERR_SETUP, "SpGEMM shared memory %zu exceeds %d", smem_sym, SG_SMEM_MAX);
        const int grid = (int)std::max(1LL, std::min<long long>(((long long)nlong + W - 1) / W, 152LL * 64));
        gw_launch(k_sg_symbolic, grid, 32 * W, smem_sym, st, nlong, rows, L.rp.p, L.ci.p,
                  Rm.rp.p, Rm.ci.p, H, C.rp.p, ctr.p + 4, ctr.p + 5);
        GW_LAUNCH_CHECK();
        int hl[2];
        GW_CUDA(cudaMemcpyAsync(hl, ctr.p + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
        if (hl[0]) fail(GW_ERR_SETUP, "SpGEMM row has more than %d distinct columns", H / 2);
        // the numeric pass knows every row's distinct count: tables of twice the largest
        Hn = 32;
        while (Hn < 2 * hl[1]) Hn <<= 1;
        const size_t per_warp_num = (size_t)Hn * 12;
        Wn = (int)std::max<size_t>(1, std::min<size_t>(8, (96u << 10) / per_warp_num));
        if ((size_t)Wn * per_warp_num > (size_t)SG_SMEM_MAX)
            fail(GW_ERR_SETUP, "SpGEMM shared memory %zu exceeds %d", (size_t)Wn * per_warp_num, SG_SMEM_MAX);
    }
    exclusive_scan(C.rp.p, C.rp.p, C.nr, st);
    C.nnz = read_int(C.rp.p + C.nr, st);
    C.ci.alloc((size_t)C.nnz);
    C.v.alloc((size_t)C.nnz);
    if (mu_short > 0) {
        auto numeric = [&](auto kernel, int cap) {
            GW_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SGT_CAP * SGT_BS * 12));
            gw_launch(kernel, gt, SGT_BS, (size_t)cap * SGT_BS * 12, st, L.nr, L.rp.p, L.ci.p, L.v.p, Rm.rp.p,
                      Rm.ci.p, Rm.v.p, C.rp.p, C.ci.p, C.v.p);
        };
        if (mu_short <= 16) numeric(k_sgt_numeric<16>, 16);
        else if (mu_short <= 32) numeric(k_sgt_numeric<32>, 32);
        else numeric(k_sgt_numeric<SGT_CAP>, SGT_CAP);
        GW_LAUNCH_CHECK();
    }
    if (nlong > 0) {
        const size_t smem_num = (size_t)Wn * Hn * 12;
        const int grid_n = (int)std::max(1LL, std::min<long long>(((long long)nlong + Wn - 1) / Wn, 152LL * 64));
        gw_launch(k_sg_numeric, grid_n, 32 * Wn, smem_num, st, nlong, rows, L.rp.p, L.ci.p,
                  L.v.p, Rm.rp.p, Rm.ci.p, Rm.v.p, Hn, C.rp.p, C.ci.p, C.v.p);
        GW_LAUNCH_CHECK();
    }
    GW_CUDA(cudaStreamSynchronize(st));
}

// ---------------------------------------------------------- coarsest level --
// Dense inverse of the coarsest level by block Gauss-Jordan elimination in
// place, without pivoting (the coarsest operator is a Galerkin product of
// the SPD level-0 operator with a full-rank prolongator, so it is SPD, and
// elimination without pivoting is stable on SPD matrices; a pivot that is
// not positive and finite reports the matrix as singular).  M (n x n,
// row-major) starts as A; for each panel K of GJB consecutive indices:
//   Q = (M_KK)^-1,
//   M_IJ -= M_IK Q M_KJ  (I, J outside K),
//   M_KJ  = Q M_KJ,  M_IK = -M_IK Q,  M_KK = Q,
// and after the last panel M = A^-1.  Each panel is two launches: one block
// per 32-column tile J inverts M_KK (every block the same way, in shared
// memory), forms the new row panel Q M_KJ and copies the old column panel
// M_JK aside; then one block per 32 x 32 tile of M applies the update.  The
// n^3 FP64 multiply-adds so run on every SM, in 2 n / GJB launches.  The
// launches run back to back with programmatic dependent launch: each kernel
// may be scheduled while its predecessor runs and waits for it (and its
// writes) before touching memory.
constexpr int GJB = 32;

__device__ __forceinline__ void gj_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
static void gj_launch(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args &&...args)
{
    prime_kernel((const void *)kernel);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GW_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Inverse of the bk x bk pivot block in shared memory (row stride GJB+1),
// in-place Gauss-Jordan without pivoting; 256 threads.  Returns false (for
// every thread) if a pivot is not positive and finite.
__device__ bool gj_invert_block(double (*a)[GJB + 1], double *col, int bk)
{
    const int tid = threadIdx.x;
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int p = 0; p < bk; ++p) {
        const double piv = a[p][p];
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (tid == 0) bad = 1;
            break;  // uniform: every thread read the same pivot
        }
        if (tid < bk) col[tid] = a[tid][p];
        __syncthreads();
        // row p scaled by 1/piv, with its diagonal entry replaced by 1/piv
        if (tid < bk) a[p][tid] = (tid == p ? 1.0 : a[p][tid]) / piv;
        __syncthreads();
        for (int t = tid; t < bk * bk; t += blockDim.x) {
            const int i = t / bk, j = t % bk;
            if (i != p) a[i][j] = (j == p ? 0.0 : a[i][j]) - col[i] * a[p][j];
        }
        __syncthreads();
    }
    __syncthreads();
    return bad == 0;
}

// One block per 32-index tile J: Q = (M_KK)^-1, Rn[:, J] = Q M_KJ, Cs[J, :]
// = M_JK (old values); block 0 also stores Q.
__global__ void __launch_bounds__(256) k_bgj_panel(int n, int k0, int bk, const double *__restrict__ M,
                                                   double *__restrict__ Q, double *__restrict__ Rn,
                                                   double *__restrict__ Cs, int *__restrict__ singular)
{
    __shared__ double a[GJB][GJB + 1], t[GJB][GJB + 1];
    __shared__ double col[GJB];
    const int tid = threadIdx.x, j0 = blockIdx.x * GJB, bj = min(GJB, n - j0);
    gj_enter();
    if (*(volatile const int *)singular) return;
    for (int e = tid; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        a[i][j] = i < bk && j < bk ? M[(size_t)(k0 + i) * n + k0 + j] : 0.0;
        t[i][j] = i < bk && j < bj ? M[(size_t)(k0 + i) * n + j0 + j] : 0.0;
    }
    __syncthreads();
    // old column panel rows of this tile
    for (int e = tid; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        if (i < bj && j < bk) Cs[(size_t)(j0 + i) * GJB + j] = M[(size_t)(j0 + i) * n + k0 + j];
    }
    if (!gj_invert_block(a, col, bk)) {
        if (tid == 0) atomicExch(singular, 1);
        return;
    }
    if (blockIdx.x == 0)
        for (int e = tid; e < GJB * GJB; e += blockDim.x) Q[e] = a[e / GJB][e % GJB];
    // Rn[:, J] = Q M_KJ, terms in ascending inner index
    for (int e = tid; e < bk * bj; e += blockDim.x) {
        const int i = e / bj, j = e % bj;
        double s = 0.0;
        for (int q = 0; q < bk; ++q) s = fma(a[i][q], t[q][j], s);
        Rn[(size_t)i * n + j0 + j] = s;
    }
}

// One block per 32 x 32 tile (I, J) of M: the panel update above.
__global__ void __launch_bounds__(256) k_bgj_update(int n, int k0, int bk, double *__restrict__ M,
                                                    const double *__restrict__ Q, const double *__restrict__ Rn,
                                                    const double *__restrict__ Cs, const int *__restrict__ singular)
{
    __shared__ double c[GJB][GJB + 1], r[GJB][GJB + 1];
    const int tid = threadIdx.x;
    const int nt = (n + GJB - 1) / GJB;
    const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
    const int i0 = ti * GJB, j0 = tj * GJB, bi = min(GJB, n - i0), bj = min(GJB, n - j0);
    const int kt = k0 / GJB;
    gj_enter();
    if (*(volatile const int *)singular) return;
    if (ti == kt && tj == kt) {
        for (int e = tid; e < bk * bk; e += blockDim.x)
            M[(size_t)(k0 + e / bk) * n + k0 + e % bk] = Q[(e / bk) * GJB + e % bk];
        return;
    }
    if (ti == kt) {
        for (int e = tid; e < bk * bj; e += blockDim.x)
            M[(size_t)(k0 + e / bj) * n + j0 + e % bj] = Rn[(size_t)(e / bj) * n + j0 + e % bj];
        return;
    }
    // c = old M_IK (bi x bk); r = Rn[:, J] (bk x bj), or Q for the tile in column K
    for (int e = tid; e < GJB * GJB; e += blockDim.x) {
        const int i = e / GJB, j = e % GJB;
        c[i][j] = i < bi && j < bk ? Cs[(size_t)(i0 + i) * GJB + j] : 0.0;
        r[i][j] = i < bk && j < bj ? (tj == kt ? Q[i * GJB + j] : Rn[(size_t)i * n + j0 + j]) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < bi * bj; e += blockDim.x) {
        const int i = e / bj, j = e % bj;
        double s = 0.0;
        for (int q = 0; q < bk; ++q) s = fma(c[i][q], r[q][j], s);
        double *m = M + (size_t)(i0 + i) * n + j0 + j;
        *m = tj == kt ? -s : *m - s;
    }
}

__global__ void k_gj_fill(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                          double *__restrict__ M)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        for (int e = rp[i]; e < rp[i + 1]; ++e) M[(size_t)i * n + ci[e]] = v[e];
    }
}

void setup_dense_inverse(const DCSR &A, DBuf<double> &Ainv, cudaStream_t st)
{
    const int n = A.nr;
    if (n > 4096) fail(GW_ERR_SETUP, "coarsest level has %d unknowns (more than 4096)", n);
    const int nt = (n + GJB - 1) / GJB;
    DBuf<double> Q((size_t)GJB * GJB), Rn((size_t)GJB * n), Cs((size_t)nt * GJB * GJB);
    DBuf<int> sing(1);
    Ainv.alloc((size_t)n * n);
    GW_CUDA(cudaMemsetAsync(Ainv.p, 0, Ainv.bytes(), st));
    GW_CUDA(cudaMemsetAsync(sing.p, 0, sizeof(int), st));
    gw_launch(k_gj_fill, nblk(n, 128), 128, 0, st, n, A.rp.p, A.ci.p, A.v.p, Ainv.p);
    GW_LAUNCH_CHECK();
    for (int k0 = 0; k0 < n; k0 += GJB) {
        const int bk = std::min(GJB, n - k0);
        gj_launch(k_bgj_panel, nt, 256, st, n, k0, bk, (const double *)Ainv.p, Q.p, Rn.p, Cs.p, (int *)sing.p);
        gj_launch(k_bgj_update, nt * nt, 256, st, n, k0, bk, Ainv.p, (const double *)Q.p, (const double *)Rn.p,
                  (const double *)Cs.p, (const int *)sing.p);
    }
    GW_LAUNCH_CHECK();
    if (read_int(sing.p, st)) fail(GW_ERR_SETUP, "coarsest-level matrix (%d unknowns) is singular", n);
}

// ------------------------------------------------- smoother data (per level) --
__global__ void k_gersh(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                        double *__restrict__ d, unsigned long long *__restrict__ rho_bits)
{
    unsigned long long best = 0;
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double s = 0.0, dd = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            s += fabs(v[e]);
            if (ci[e] == i) dd = v[e];
        }
        d[i] = dd;
        const double ratio = s / dd;
        if (ratio > 0.0 && isfinite(ratio)) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(ratio);
            best = b > best ? b : best;
        }
    }
    block_atomic_max(best, rho_bits);
}

double setup_gershgorin(const DCSR &A, DBuf<double> &diag, cudaStream_t st)
{
    diag.alloc((size_t)A.nr);
    DBuf<unsigned long long> rb(1);
    GW_CUDA(cudaMemsetAsync(rb.p, 0, sizeof(unsigned long long), st));
    gw_launch(k_gersh, nblk(A.nr, 256), 256, 0, st, A.nr, A.rp.p, A.ci.p, A.v.p, diag.p, rb.p);
    GW_LAUNCH_CHECK();
    unsigned long long bits = 0;
    GW_CUDA(cudaMemcpyAsync(&bits, rb.p, sizeof bits, cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    double r;
    memcpy(&r, &bits, sizeof r);
    return r;
}

__global__ void k_pow_start(int n, uint64_t seed, int level, double *__restrict__ v)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        const uint64_t h = smix64(seed ^ ((uint64_t)level << 48) ^ (uint64_t)(uint32_t)i ^ 0x00c0ffee00000000ULL);
        v[i] = (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    }
}

// w = D^-1 A v and per-block partial sums of w.w; G lanes a row
template <int G>
__global__ void __launch_bounds__(256) k_pow_step(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                  const double *__restrict__ a, const double *__restrict__ d,
                                                  const double *__restrict__ v, double *__restrict__ w,
                                                  double *__restrict__ part)
{
    __shared__ double sh[256];
    const int lane = threadIdx.x & (G - 1);
    double loc = 0.0;
    const long long groups = (long long)gridDim.x * (blockDim.x / G);
    // whole warps stay in the loop (the groups' shuffles need every lane)
    for (long long ii = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
         G == 1 ? ii < n : __any_sync(0xffffffffu, ii < n); ii += groups) {
        const int i = (int)ii;
        double s = 0.0;
        if (ii < n)
            for (int e = rp[i] + lane; e < rp[i + 1]; e += G) s += a[e] * v[ci[e]];
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off, G);
        if (lane == 0 && ii < n) {
            s /= d[i];
            w[i] = s;
            loc += s * s;
        }
    }
    sh[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// lambda_max(D^-1 A) by 10 power iterations from a hashed start vector:
// x_{k+1} = D^-1 A x_k without normalising (the spectral radius of D^-1 A is
// a few units at most, so ten steps stay far from overflow), and
// lambda = |x_10| / |x_9|, the same estimate as normalised iterations give.
// The ten steps run back to back; the host reads the two last norms once.
double setup_power_lambda(const DCSR &A, const double *diag, uint64_t seed, int level, cudaStream_t st)
{
    const int n = A.nr;
    const double per_row = n ? (double)A.nnz / n : 0.0;
    const int G = per_row <= 12.0 ? 1 : per_row <= 48.0 ? 8 : 32;
    const int g = nblk((long long)n * G, 256, 1024);
    DBuf<double> v((size_t)n), w((size_t)n), part((size_t)2 * g);
    gw_launch(k_pow_start, nblk(n, 256, 1024), 256, 0, st, n, seed, level, v.p);
    GW_LAUNCH_CHECK();
    for (int it = 0; it < 10; ++it) {
        double *pp = part.p + (size_t)(it & 1) * g;
        if (G == 1) gw_launch(k_pow_step<1>, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, diag, v.p, w.p, pp);
        else if (G == 8) gw_launch(k_pow_step<8>, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, diag, v.p, w.p, pp);
        else gw_launch(k_pow_step<32>, g, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, diag, v.p, w.p, pp);
        GW_LAUNCH_CHECK();
        std::swap(v, w);
    }
    // it = 8 wrote |x_9|^2 into the first half, it = 9 |x_10|^2 into the second
    std::vector<double> h((size_t)2 * g);
    GW_CUDA(cudaMemcpyAsync(h.data(), part.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    double s9 = 0.0, s10 = 0.0;
    for (int b = 0; b < g; ++b) {
        s9 += h[(size_t)b];
        s10 += h[(size_t)g + b];
    }
    return s9 > 0.0 ? sqrt(s10 / s9) : 0.0;
}

// ------------------------------------------------------- sliced ELL format --
// perm for rows sorted by descending length (ties by index) within windows of
// SELL_SORT_WINDOW rows: one block per window, rank by counting
__global__ void __launch_bounds__(SELL_SORT_WINDOW) k_sell_sort(int nr, const int *__restrict__ rp,
                                                                int *__restrict__ perm)
{
    __shared__ int len[SELL_SORT_WINDOW];
    const int w0 = blockIdx.x * SELL_SORT_WINDOW, t = threadIdx.x, r = w0 + t;
    const int m = min(SELL_SORT_WINDOW, nr - w0);
    len[t] = t < m ? rp[r + 1] - rp[r] : -1;
    __syncthreads();
    if (t < m) {
        int rank = 0;
        for (int u = 0; u < m; ++u) rank += (len[u] > len[t] || (len[u] == len[t] && u < t)) ? 1 : 0;
        perm[w0 + rank] = r;
    }
}

__global__ void k_sell_width(int nr, int nslices, int V, const int *__restrict__ rp, const int *__restrict__ perm,
                             int *__restrict__ width)
{
    GRID_STRIDE(s, nslices)
    {
        int w = 0;
        for (int l = 0; l < SELL_C; ++l) {
            const long long r = s * SELL_C + l;
            if (r < nr) {
                const int o = perm ? perm[r] : (int)r;
                w = max(w, rp[o + 1] - rp[o]);
            }
        }
        w = (w + V - 1) / V * V;
        width[s] = w * SELL_C;
    }
}

template <class T>
__global__ void k_sell_fill(int nr, int nc, int nslices, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ v, const int *__restrict__ perm, const int *__restrict__ sp,
                            int *__restrict__ sci, T *__restrict__ sv)
{
    constexpr int V = SellV<T>::V;
    GRID_STRIDE(rr, (long long)nslices * SELL_C)
    {
        const int r = (int)rr, s = r / SELL_C, lane = r % SELL_C;
        const int o = (perm && r < nr) ? perm[r] : r;
        const int base = sp[s], w = (sp[s + 1] - base) / SELL_C;
        const int b = r < nr ? rp[o] : 0, len = r < nr ? rp[o + 1] - b : 0;
        const int pad = o < nc ? o : 0;
        for (int k = 0; k < w; ++k) {
            const size_t o = (size_t)base + (size_t)(k / V) * SELL_C * V + (size_t)lane * V + (k % V);
            if (k < len) {
                sci[o] = ci[b + k];
                sv[o] = (T)v[b + k];
            } else {
                sci[o] = pad;
                sv[o] = (T)0;
            }
        }
    }
}

template <class T>
void to_sell(const DCSR &A, Sell<T> &S, cudaStream_t st, bool sorted)
{
    constexpr int V = SellV<T>::V;
    S.nr = A.nr;
    S.nc = A.nc;
    S.nnz = A.nnz;
    S.nslices = (A.nr + SELL_C - 1) / SELL_C;
    S.perm.release();
    if (sorted && A.nr > 0) {
        S.perm.alloc((size_t)A.nr);
        gw_launch(k_sell_sort, (A.nr + SELL_SORT_WINDOW - 1) / SELL_SORT_WINDOW, SELL_SORT_WINDOW, 0, st, A.nr, A.rp.p,
                                                                                                  S.perm.p);
        GW_LAUNCH_CHECK();
    }
    S.sp.alloc((size_t)S.nslices + 1);
    gw_launch(k_sell_width, nblk(S.nslices, 256), 256, 0, st, A.nr, S.nslices, V, A.rp.p, S.perm.p, S.sp.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(S.sp.p, S.sp.p, S.nslices, st);
    S.stored = read_int(S.sp.p + S.nslices, st);
    S.ci.alloc((size_t)S.stored);
    S.v.alloc((size_t)S.stored);
    gw_launch(k_sell_fill<T>, nblk((long long)S.nslices * SELL_C, 256), 256, 0, st, A.nr, A.nc, S.nslices, A.rp.p, A.ci.p,
                                                                          A.v.p, S.perm.p, S.sp.p, S.ci.p, S.v.p);
    GW_LAUNCH_CHECK();
}

template void to_sell<float>(const DCSR &, Sell<float> &, cudaStream_t, bool);
template void to_sell<double>(const DCSR &, Sell<double> &, cudaStream_t, bool);

// ----------------------------------------------- CSR and stencil formats --
template <class T>
__global__ void k_convert_vals(long long nnz, const double *__restrict__ v, T *__restrict__ o)
{
    GRID_STRIDE(e, nnz) o[e] = (T)v[e];
}

// split a 7-point grid operator into diagonal and +x/+y/+z couplings; counts
// entries that are not on the grid stencil
template <class T>
__global__ void k_to_stencil(int n, int nx, int sxy, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ v, T *__restrict__ d, T *__restrict__ ox, T *__restrict__ oy,
                             T *__restrict__ oz, int *__restrict__ bad)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double dd = 0.0, a = 0.0, b = 0.0, c = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const long long j = ci[e];
            if (j == i) dd = v[e];
            else if (j == (long long)i + sxy) c = v[e];
            else if (j == (long long)i + nx) b = v[e];
            else if (j == (long long)i + 1) a = v[e];
            else if (!(j == (long long)i - sxy || j == (long long)i - nx || j == (long long)i - 1)) atomicAdd(bad, 1);
        }
        d[i] = (T)dd;
        ox[i] = (T)a;
        oy[i] = (T)b;
        oz[i] = (T)c;
    }
}

// BF16 couplings and the corrected FP32 diagonal (see StenB)
__global__ void k_to_stencil_bf16(int n, int nx, int sxy, const int *__restrict__ rp, const int *__restrict__ ci,
                                  const double *__restrict__ v, float *__restrict__ d, __nv_bfloat16 *__restrict__ ox,
                                  __nv_bfloat16 *__restrict__ oy, __nv_bfloat16 *__restrict__ oz,
                                  int *__restrict__ bad)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double dd = 0.0, a = 0.0, b = 0.0, c = 0.0, corr = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const long long j = ci[e];
            const double x = v[e];
            if (j == i) {
                dd = x;
                continue;
            }
            if (j == (long long)i + sxy) c = x;
            else if (j == (long long)i + nx) b = x;
            else if (j == (long long)i + 1) a = x;
            else if (!(j == (long long)i - sxy || j == (long long)i - nx || j == (long long)i - 1)) atomicAdd(bad, 1);
            const double xr = (double)__bfloat162float(__double2bfloat16(x));
            corr += fabs(xr) - fabs(x);
        }
        d[i] = (float)(dd + corr);
        ox[i] = __double2bfloat16(a);
        oy[i] = __double2bfloat16(b);
        oz[i] = __double2bfloat16(c);
    }
}

// sqrt of the diagonal (FP32) for the scaled FP16 stencil
__global__ void k_sten_sd(int n, const int *__restrict__ rp, const int *__restrict__ ci, const double *__restrict__ v,
                          float *__restrict__ sd)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        double dd = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i) dd = v[e];
        sd[i] = (float)sqrt(dd);
    }
}

// scaled couplings in FP16 and the FP16 correction of the unit diagonal (see StenH)
__global__ void k_to_stencil_fp16(int n, int nx, int sxy, const int *__restrict__ rp, const int *__restrict__ ci,
                                  const double *__restrict__ v, const float *__restrict__ sd,
                                  __half *__restrict__ dd, __half *__restrict__ ox, __half *__restrict__ oy,
                                  __half *__restrict__ oz, int *__restrict__ bad)
{
    GRID_STRIDE(ii, n)
    {
        const int i = (int)ii;
        const double si = (double)sd[i];
        double a = 0.0, b = 0.0, c = 0.0, corr = 0.0;
        if (!(si > 0.0)) atomicAdd(bad, 1);
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const long long j = ci[e];
            if (j == i) continue;
            const double sj = (double)sd[j];
            const double x = v[e] / (si * sj);
            if (j == (long long)i + sxy) c = x;
            else if (j == (long long)i + nx) b = x;
            else if (j == (long long)i + 1) a = x;
            else if (!(j == (long long)i - sxy || j == (long long)i - nx || j == (long long)i - 1)) atomicAdd(bad, 1);
            const double xr = (double)__half2float(__double2half(x));
            corr += (fabs(xr) - fabs(x)) * sj / si;
        }
        dd[i] = __double2half(corr);
        ox[i] = __double2half(a);
        oy[i] = __double2half(b);
        oz[i] = __double2half(c);
    }
}

// Short rows (the prolongator) and rows of medium length on big levels as
// sliced ELL, one thread per row; long rows on small levels as CSR read by a
// whole warp, so the level still covers the GPU.
#ifndef GW_LONG_BIG_FMT
#define GW_LONG_BIG_FMT FMT_SELL  // long rows on levels of 65536 rows or more
#endif

int choose_fmt(const DCSR &A)
{
    const double avg = A.nr > 0 ? (double)A.nnz / A.nr : 0.0;
    if (avg <= 12.0) return FMT_SELL;
    if (A.nr >= 65536) return GW_LONG_BIG_FMT;
    return FMT_CSR32;
}

template <class T>
bool to_store(const DCSR &A, MatStore<T> &M, int fmt, int nx, int ny, int nz, cudaStream_t st)
{
    M.nr = A.nr;
    M.nc = A.nc;
    M.nnz = A.nnz;
    M.fmt = fmt;
    if (fmt == FMT_SELL_SORTED) {
        M.fmt = FMT_SELL;
        to_sell<T>(A, M.sell, st, true);
        return true;
    }
    if (fmt == FMT_STENH) {
        StenH &S = M.stenh;
        const int n = A.nr;
        if (sizeof(T) == 4) {
            S.n = n;
            S.nx = nx;
            S.ny = ny;
            S.nz = nz;
            S.sd.alloc((size_t)n);
            S.dd.alloc((size_t)n);
            S.ox.alloc((size_t)n);
            S.oy.alloc((size_t)n);
            S.oz.alloc((size_t)n);
            DBuf<int> bad(1);
            GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            gw_launch(k_sten_sd, nblk(n, 256), 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, S.sd.p);
            gw_launch(k_to_stencil_fp16, nblk(n, 256), 256, 0, st, n, nx, nx * ny, A.rp.p, A.ci.p, A.v.p,
                      (const float *)S.sd.p, S.dd.p, S.ox.p, S.oy.p, S.oz.p, bad.p);
            GW_LAUNCH_CHECK();
            if (read_int(bad.p, st) == 0) return true;
            S = StenH();
        }
        fmt = FMT_STEN;
        M.fmt = fmt;
    }
    if (fmt == FMT_STENB) {
        StenB &S = M.stenb;
        const int n = A.nr;
        if (sizeof(T) == 4) {
            S.n = n;
            S.nx = nx;
            S.ny = ny;
            S.nz = nz;
            S.d.alloc((size_t)n);
            S.ox.alloc((size_t)n);
            S.oy.alloc((size_t)n);
            S.oz.alloc((size_t)n);
            DBuf<int> bad(1);
            GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
            gw_launch(k_to_stencil_bf16, nblk(n, 256), 256, 0, st, n, nx, nx * ny, A.rp.p, A.ci.p, A.v.p, S.d.p, S.ox.p,
                                                            S.oy.p, S.oz.p, bad.p);
            GW_LAUNCH_CHECK();
            if (read_int(bad.p, st) == 0) return true;
            S.d.release();
            S.ox.release();
            S.oy.release();
            S.oz.release();
        }
        fmt = FMT_STEN;
        M.fmt = fmt;
    }
    if (fmt == FMT_STEN) {
        StenT<T> &S = M.sten;
        const int n = A.nr;
        S.n = n;
        S.nx = nx;
        S.ny = ny;
        S.nz = nz;
        S.d.alloc((size_t)n);
        S.ox.alloc((size_t)n);
        S.oy.alloc((size_t)n);
        S.oz.alloc((size_t)n);
        DBuf<int> bad(1);
        GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        gw_launch(k_to_stencil<T>, nblk(n, 256), 256, 0, st, n, nx, nx * ny, A.rp.p, A.ci.p, A.v.p, S.d.p, S.ox.p, S.oy.p,
                                                     S.oz.p, bad.p);
        GW_LAUNCH_CHECK();
        if (read_int(bad.p, st) == 0) return true;
        S.d.release();
        S.ox.release();
        S.oy.release();
        S.oz.release();
        fmt = choose_fmt(A);
        M.fmt = fmt;
    }
    if (fmt == FMT_SELL) {
        to_sell<T>(A, M.sell, st);
        return true;
    }
    CsrT<T> &C = M.csr;
    C.nr = A.nr;
    C.nc = A.nc;
    C.nnz = A.nnz;
    C.rp.alloc((size_t)A.nr + 1);
    C.ci.alloc((size_t)std::max(A.nnz, 1));
    C.v.alloc((size_t)std::max(A.nnz, 1));
    GW_CUDA(cudaMemcpyAsync(C.rp.p, A.rp.p, ((size_t)A.nr + 1) * sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (A.nnz) {
        GW_CUDA(cudaMemcpyAsync(C.ci.p, A.ci.p, (size_t)A.nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
        gw_launch(k_convert_vals<T>, nblk(A.nnz, 256), 256, 0, st, A.nnz, A.v.p, C.v.p);
        GW_LAUNCH_CHECK();
    }
    return true;
}

template bool to_store<float>(const DCSR &, MatStore<float> &, int, int, int, int, cudaStream_t);
template bool to_store<double>(const DCSR &, MatStore<double> &, int, int, int, int, cudaStream_t);

}  // namespace gw
