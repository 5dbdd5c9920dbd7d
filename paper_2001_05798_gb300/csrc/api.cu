// api.cu -- the C ABI of libgw and the construction of the hierarchy.
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include <memory>
#include <new>


#include "gw_internal.cuh"

struct gw_matrix_s {
    int dev = 0;
    int nx = 0, ny = 0, nz = 0;
    gw::DCSR A;
};

struct gw_hierarchy_s {
    std::unique_ptr<gw::Hier> h;
    gw_matrix base = nullptr;   // the matrix the caller set the hierarchy up from (C)
    gw::DCSR shifted;           // C + diag(s) while a transient shift is applied
    gw::DBuf<double> s_built;   // shift the coarse levels were built with (empty: none)
    gw::DBuf<double> s_now;     // shift now applied (empty: none)
    gw::DBuf<double> s_ref;     // shift the coarse operators were last formed with (empty: none)
};

namespace gw {

// ---------------------------------------------------------------- helpers --
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) GW_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// A read-only input that may live on the host: staged into device memory.
template <class T>
struct DevIn {
    const T *p = nullptr;
    DBuf<T> own;
    DevIn(const T *src, size_t n, cudaStream_t st)
    {
        if (!src) return;
        if (is_device_ptr(src)) {
            p = src;
        } else {
            own.alloc(n);
            GW_CUDA(cudaMemcpyAsync(own.p, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
            p = own.p;
        }
    }
};

Hier::~Hier()
{
    if (batch) batch_forget(*static_cast<Batch *>(batch), this);
    drop_graphs(*this);
    block_free(blk);
    if (cap) cudaStreamDestroy(cap);
    if (cap2) cudaStreamDestroy(cap2);
    if (ctl_host) host_free(ctl_host);
}

__global__ void k_make_dw(int n, const double *__restrict__ d, double scale, float *__restrict__ of,
                          double *__restrict__ od)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double w = scale / d[i];
        if (of) of[i] = (float)w;
        if (od) od[i] = w;
    }
}

template <class T>
static void alloc_vectors(CycLevel<T> &c, int n)
{
    c.n = n;
    c.x.alloc((size_t)n);
    c.b.alloc((size_t)n);
    c.r.alloc((size_t)n);
    c.t.alloc((size_t)n);
    c.d.alloc((size_t)n);
    c.d2.alloc((size_t)n);
}

static void cheb_coeffs(double lam, int degree, double &c0, double *c1, double *c2)
{
    const double a = lam / 30.0, b = 1.1 * lam;
    const double theta = (b + a) / 2.0, delta = (b - a) / 2.0, sigma = theta / delta;
    double rho = 1.0 / sigma;
    c0 = 1.0 / theta;
    for (int k = 1; k < degree && k < 8; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c1[k] = rn * rho;
        c2[k] = 2.0 * rn / delta;
        rho = rn;
    }
}

// Cycle storage of level k in the cycle precision: A_k (the 7-point stencil on
// level 0), P_k and R_k when given, the smoother's diagonal weights and the
// Chebyshev coefficients.  Returns the device bytes it holds.
// restrictions in sliced ELL are stored over length-sorted rows (padding of
// the 32-row slices 1.51 -> 1.11 at 128^3); their kernel writes through the
// row permutation
#ifndef GW_SORT_RESTRICTION
#define GW_SORT_RESTRICTION 1
#endif
static int sorted_sell(int fmt) { return GW_SORT_RESTRICTION && fmt == FMT_SELL ? FMT_SELL_SORTED : fmt; }

static long long store_level(Hier &H, int k, const DCSR &A, const DCSR *P, const DCSR *R, cudaStream_t st)
{
    const gw_amg_opts &o = H.o;
    const bool f64 = o.prec == GW_PREC_FP64;
    const int n = A.nr;
    long long bytes = 0;
    DBuf<double> diag;
    const double rhoJ = setup_gershgorin(A, diag, st);
    H.info[(size_t)k].jacobi_w = (4.0 / 3.0) / rhoJ;
    double scale = 1.0;
    double c0 = 0.0, c1[8] = {0}, c2[8] = {0};
    if (o.smoother == GW_SMOOTH_JACOBI) {
        scale = H.info[(size_t)k].jacobi_w;
    } else {
        const double lam = setup_power_lambda(A, diag.p, o.seed, k, st);
        H.info[(size_t)k].lambda_max = lam;
        cheb_coeffs(lam, o.degree, c0, c1, c2);
    }
    const int g = (int)std::min<long long>(((long long)n + 255) / 256, 152LL * 16);
    if (f64) {
        CycLevel<double> &c = H.cd[(size_t)k];
        to_store<double>(A, c.A, k == 0 ? FMT_STEN : choose_fmt(A), H.gnx, H.gny, H.gnz, st);
        if (P) to_store<double>(*P, c.P, choose_fmt(*P), 0, 0, 0, st);
        if (R) to_store<double>(*R, c.R, sorted_sell(choose_fmt(*R)), 0, 0, 0, st);
        c.dw.alloc((size_t)n);
        gw_launch(k_make_dw, std::max(g, 1), 256, 0, st, n, diag.p, scale, nullptr, c.dw.p);
        c.c0 = c0;
        memcpy(c.c1, c1, sizeof c1);
        memcpy(c.c2, c2, sizeof c2);
        bytes += (long long)(c.A.bytes() + c.P.bytes() + c.R.bytes() + c.dw.bytes());
    } else {
        CycLevel<float> &c = H.cf[(size_t)k];
        const bool fine16 = k == 0 && (o.half_storage & GW_HALF_FINE) != 0;
        const bool fineh = k == 0 && (o.half_storage & GW_HALF_FINE16) != 0;
        to_store<float>(A, c.A, k == 0 ? (fine16 ? FMT_STENB : fineh ? FMT_STENH : FMT_STEN) : choose_fmt(A),
                        H.gnx, H.gny, H.gnz,
                        st);
        if (k == 0) {
            H.A32 = MatStore<float>();
            if (c.A.fmt == FMT_STENB || c.A.fmt == FMT_STENH) {
                to_store<float>(A, H.A32, FMT_STEN, H.gnx, H.gny, H.gnz, st);
                bytes += (long long)H.A32.bytes();
            }
        }
        if (P && !(k == 0 && H.p0.n)) to_store<float>(*P, c.P, choose_fmt(*P), 0, 0, 0, st);
        if (k == 0 && H.p0.n) bytes += (long long)H.p0.bytes();
        if (R) to_store<float>(*R, c.R, sorted_sell(choose_fmt(*R)), 0, 0, 0, st);
        c.dw.alloc((size_t)n);
        gw_launch(k_make_dw, std::max(g, 1), 256, 0, st, n, diag.p, scale, c.dw.p, nullptr);
        c.c0 = c0;
        memcpy(c.c1, c1, sizeof c1);
        memcpy(c.c2, c2, sizeof c2);
        bytes += (long long)(c.A.bytes() + c.P.bytes() + c.R.bytes() + c.dw.bytes());
    }
    GW_LAUNCH_CHECK();
    GW_CUDA(cudaStreamSynchronize(st));
    return bytes;
}

// Level 0 becomes A (same grid and pattern); the coarse levels stay.  Used
// for the transient shift while the cached hierarchy remains valid.
void refresh_level0(Hier &H, const DCSR &A, cudaStream_t st)
{
    H.A0 = &A;
    store_level(H, 0, A, nullptr, nullptr, st);
    if (H.o.prec != GW_PREC_FP64) to_store<double>(A, H.A64, FMT_STEN, H.gnx, H.gny, H.gnz, st);
    drop_graphs(H);
    GW_CUDA(cudaStreamSynchronize(st));
}

void refresh_numeric(Hier &H, const DCSR &A, cudaStream_t st)
{
    H.A0 = &A;
    const int L = H.L;
    for (int l = 0; l + 1 < L; ++l) {
        const DCSR &Al = l == 0 ? A : H.A[(size_t)l];
        DCSR AP, Ac;
        setup_spgemm(Al, H.P[(size_t)l], AP, st);
        setup_spgemm(H.R[(size_t)l], AP, Ac, st);
        if (Ac.nnz != H.A[(size_t)l + 1].nnz) fail(GW_ERR_SETUP, "refresh: the pattern of level %d changed", l + 1);
        H.A[(size_t)l + 1] = std::move(Ac);
    }
    for (int l = 0; l + 1 < L; ++l) store_level(H, l, l == 0 ? A : H.A[(size_t)l], nullptr, nullptr, st);
    setup_dense_inverse(H.A[(size_t)L - 1], H.Ainv, st);
    if (H.o.prec != GW_PREC_FP64) to_store<double>(A, H.A64, FMT_STEN, H.gnx, H.gny, H.gnz, st);
    drop_graphs(H);
    GW_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------ hierarchy checks --
// Every setup scans the stored hierarchy for non-finite values (a coarse
// operator, a prolongator, the coarsest inverse), so that a bad input or a
// breakdown in the setup is reported there, not as a stalled solve.  With the
// environment variable GW_VALIDATE=1 it also checks every index array the
// cycle kernels gather through (CSR row pointers and columns of all levels,
// the sliced-ELL columns, the implicit level-0 transfer's aggregate and
// member lists) against its bounds.  The checks count violations on the
// device and report them as GW_ERR_SETUP; nothing asserts on the GPU.
__global__ void k_nonfinite(long long n, const double *__restrict__ v, int *__restrict__ bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicAdd(bad, 1);
}

__global__ void k_check_csr(int nr, int nc, long long nnz, const int *__restrict__ rp, const int *__restrict__ ci,
                            int *__restrict__ bad)
{
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < nr; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const int a = rp[i], b = rp[i + 1];
        if (a < 0 || b < a || b > nnz || (i == 0 && a != 0) || (i == nr - 1 && b != nnz)) {
            atomicAdd(bad, 1);
            continue;
        }
        for (int e = a; e < b; ++e)
            if (ci[e] < 0 || ci[e] >= nc || (e > a && ci[e] <= ci[e - 1])) atomicAdd(bad, 1);
    }
}

__global__ void k_check_range(long long n, const int *__restrict__ x, int lo, int hi, int *__restrict__ bad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (x[i] < lo || x[i] >= hi) atomicAdd(bad, 1);
}

static int grid_of(long long n) { return (int)std::max(1LL, std::min<long long>((n + 255) / 256, 152LL * 16)); }

static void check_hierarchy(Hier &H, cudaStream_t st)
{
    // non-finite scan: one counter per array, read back together
    const int L = H.L;
    DBuf<int> cnt((size_t)2 * L + 1);
    GW_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), st));
    for (int l = 1; l < L; ++l) {
        const DCSR &A = H.A[(size_t)l];
        gw_launch(k_nonfinite, grid_of(A.nnz), 256, 0, st, (long long)A.nnz, (const double *)A.v.p, cnt.p + l);
    }
    for (int l = 0; l + 1 < L; ++l) {
        const DCSR &P = H.P[(size_t)l];
        gw_launch(k_nonfinite, grid_of(P.nnz), 256, 0, st, (long long)P.nnz, (const double *)P.v.p, cnt.p + L + l);
    }
    const long long nc2 = (long long)H.info[(size_t)L - 1].n * H.info[(size_t)L - 1].n;
    gw_launch(k_nonfinite, grid_of(nc2), 256, 0, st, nc2, (const double *)H.Ainv.p, cnt.p + 2 * L);
    GW_LAUNCH_CHECK();
    std::vector<int> c((size_t)2 * L + 1);
    GW_CUDA(cudaMemcpyAsync(c.data(), cnt.p, cnt.bytes(), cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    for (int l = 1; l < L; ++l)
        if (c[(size_t)l]) fail(GW_ERR_SETUP, "setup: non-finite entries in the operator of level %d", l);
    for (int l = 0; l + 1 < L; ++l) {
        if (c[(size_t)L + l]) fail(GW_ERR_SETUP, "setup: non-finite entries in the prolongator of level %d", l);
        const gw_level_info &li = H.info[(size_t)l];
        if (!isfinite(li.lambda_max) || !isfinite(li.jacobi_w) || !isfinite(li.omega_p))
            fail(GW_ERR_SETUP, "setup: non-finite smoother or prolongator weights on level %d", l);
    }
    if (c[(size_t)2 * L]) fail(GW_ERR_SETUP, "setup: non-finite entries in the coarsest-level inverse");
    DBuf<int> bad(1);
    auto count = [&](auto launch) {
        GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        launch();
        GW_LAUNCH_CHECK();
        return read_int(bad.p, st);
    };
    static const bool validate = [] {
        const char *e = getenv("GW_VALIDATE");
        return e && e[0] == '1';
    }();
    if (!validate) return;
    auto csr = [&](const char *what, int l, int nr, int nc, long long nnz, const int *rp, const int *ci) {
        if (count([&] { gw_launch(k_check_csr, grid_of(nr), 256, 0, st, nr, nc, nnz, rp, ci, bad.p); }))
            fail(GW_ERR_SETUP, "validation: %s of level %d has row pointers or columns out of bounds", what, l);
    };
    auto range = [&](const char *what, int l, long long n, const int *x, int lo, int hi) {
        if (n > 0 && count([&] { gw_launch(k_check_range, grid_of(n), 256, 0, st, n, x, lo, hi, bad.p); }))
            fail(GW_ERR_SETUP, "validation: %s of level %d out of [%d, %d)", what, l, lo, hi);
    };
    for (int l = 0; l < H.L; ++l) {
        const DCSR &A = l == 0 ? *H.A0 : H.A[(size_t)l];
        csr("the operator", l, A.nr, A.nc, A.nnz, A.rp.p, A.ci.p);
        if (l + 1 < H.L) {
            const DCSR &P = H.P[(size_t)l], &R = H.R[(size_t)l];
            csr("the prolongator", l, P.nr, P.nc, P.nnz, P.rp.p, P.ci.p);
            csr("the restriction", l, R.nr, R.nc, R.nnz, R.rp.p, R.ci.p);
            range("the aggregate ids", l, H.info[(size_t)l].n, H.agg[(size_t)l].p, 0, H.info[(size_t)l].naggregates);
        }
    }
    // the cycle's own storage of the levels
    auto cyc = [&](auto &C) {
        for (int l = 1; l + 1 < H.L; ++l) {
            for (const auto *M : {&C[(size_t)l].A, &C[(size_t)l].P, &C[(size_t)l].R}) {
                if (M->fmt == FMT_SELL && M->sell.stored) {
                    range("a sliced-ELL column array", l, M->sell.stored, M->sell.ci.p, 0, std::max(1, M->nc));
                    if (M->sell.perm.p) range("a sliced-ELL row permutation", l, M->nr, M->sell.perm.p, 0, M->nr);
                } else if (M->fmt == FMT_CSR4 || M->fmt == FMT_CSR8 || M->fmt == FMT_CSR32) {
                    csr("a warp-CSR matrix", l, M->csr.nr, M->csr.nc, M->csr.nnz, M->csr.rp.p, M->csr.ci.p);
                }
            }
        }
    };
    if (H.o.prec == GW_PREC_FP64) cyc(H.cd);
    else cyc(H.cf);
    if (H.p0.n) {
        range("the implicit transfer's aggregate ids", 0, H.p0.n, H.p0.agg, 0, H.p0.nc);
        range("the implicit transfer's member lists", 0, H.p0.n, H.p0.mem.p, 0, H.p0.n);
        csr("the implicit transfer's member pointers", 0, H.p0.nc, H.p0.n, H.p0.n, H.p0.mptr.p, H.p0.mem.p);
    }
}

// Smoothed-aggregation setup (see setup.cu for the stages).  Levels are added
// while the level has more than n_coarse unknowns and fewer than max_levels
// levels exist; a level whose aggregation keeps more than 0.9 of its unknowns
// (or finds none) becomes the coarsest.  theta halves per level.
void build_hierarchy(Hier &H, cudaStream_t st)
{
    NvtxRange range("gw setup");
    const gw_amg_opts &o = H.o;
    int nsm = 0;
    GW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, H.dev));
    H.max_blocks = std::max(1, std::min(RED_MAX_BLOCKS, nsm * GW_BLOCKS_PER_SM));
    H.A.clear();
    H.A.emplace_back();  // placeholder for level 0 (the matrix handle's CSR)
    std::vector<DCSR> &R = H.R;
    R.clear();
    auto Al = [&](int l) -> const DCSR & { return l == 0 ? *H.A0 : H.A[(size_t)l]; };
    double th = o.theta;
    int l = 0;
    for (;;) {
        const DCSR &A = Al(l);
        gw_level_info li;
        memset(&li, 0, sizeof li);
        li.n = A.nr;
        li.nnz = A.nnz;
        H.info.push_back(li);
        H.agg.emplace_back();
        H.root.emplace_back();
        if (A.nr <= o.n_coarse || l + 1 >= o.max_levels) break;
        char nm[48];
        snprintf(nm, sizeof nm, "gw setup level %d", l);
        NvtxRange lrange(nm);
        DBuf<unsigned char> S;
        setup_strength(A, th * th, S, st);
        H.info[(size_t)l].mis_rounds = setup_mis2(A, S.p, o.seed, l, H.root[(size_t)l], o.mis_max_rounds, st);
        const int m = setup_aggregate(A, S.p, H.root[(size_t)l].p, o.seed, l, H.agg[(size_t)l], st);
        H.info[(size_t)l].naggregates = m;
        if (m == 0 || (double)m > 0.9 * (double)A.nr) {
            H.info[(size_t)l].naggregates = 0;
            break;
        }
        DCSR P, Rl, AP, Ac;
        double omega = 0.0, rho = 0.0;
        setup_smooth_p(A, S.p, H.agg[(size_t)l].p, m, P, &omega, &rho, st);
        if (l == 0 && o.prec != GW_PREC_FP64) setup_implicit_p(A, S.p, H.agg[0].p, m, omega, H.gnx, H.gny, H.gnz, H.p0, st);
        setup_transpose(P, Rl, st);
        setup_spgemm(A, P, AP, st);
        setup_spgemm(Rl, AP, Ac, st);
        H.info[(size_t)l].omega_p = omega;
        H.info[(size_t)l].nnz_p = P.nnz;
        H.P.push_back(std::move(P));
        R.push_back(std::move(Rl));
        H.A.push_back(std::move(Ac));
        ++l;
        th = th * 0.5;
    }
    H.L = l + 1;
    const int L = H.L;
    if (H.p0.n) H.p0.agg = H.agg[0].p;
    setup_dense_inverse(Al(L - 1), H.Ainv, st);
    H.info[(size_t)L - 1].bytes += (long long)H.Ainv.bytes();
    const bool f64 = o.prec == GW_PREC_FP64;
    if (f64) H.cd.resize((size_t)L);
    else H.cf.resize((size_t)L);
    for (int k = 0; k < L; ++k) {
        const DCSR &A = Al(k);
        const int n = A.nr;
        long long bytes = 0;
        if (k < L - 1) bytes += store_level(H, k, A, &H.P[(size_t)k], &R[(size_t)k], st);
        if (f64) {
            alloc_vectors(H.cd[(size_t)k], n);
            bytes += 6LL * n * 8;
        } else {
            alloc_vectors(H.cf[(size_t)k], n);
            bytes += 6LL * n * 4;
        }
        H.info[(size_t)k].bytes += bytes;
    }
    if (!f64) {
        to_store<double>(*H.A0, H.A64, FMT_STEN, H.gnx, H.gny, H.gnz, st);
        H.info[0].bytes += (long long)H.A64.bytes();
    }
    const int n = H.A0->nr;
    H.n = n;
    H.x.alloc((size_t)n);
    H.r.alloc((size_t)n);
    H.p.alloc((size_t)n);
    H.p2.alloc((size_t)n);
    H.q.alloc((size_t)n);
    H.z.alloc((size_t)n);
    H.b.alloc((size_t)n);
    if (!f64) {
        H.r.release();
        H.p.release();
        H.p2.release();
        H.q.release();
        H.z.release();
        H.xs32.alloc((size_t)n);
        H.r32.alloc((size_t)n);
        H.p32.alloc((size_t)n);
        H.p32b.alloc((size_t)n);
        H.q32.alloc((size_t)n);
        H.z32.alloc((size_t)n);
    }
    H.part.alloc(2 * (size_t)RED_MAX_BLOCKS);
    H.ctl.alloc(1);
    GW_CUDA(cudaMemsetAsync(H.ctl.p, 0, sizeof(Ctl), st));
    GW_CUDA(host_malloc((void **)&H.ctl_host, sizeof(Ctl)));
    memset(H.ctl_host, 0, sizeof(Ctl));
    H.info[0].bytes += f64 ? 7LL * n * 8 : 2LL * n * 8 + 6LL * n * 4;
    check_hierarchy(H, st);
    GW_CUDA(cudaStreamSynchronize(st));
}

}  // namespace gw

using namespace gw;

static std::unique_ptr<Hier> new_hier(gw_matrix A, const gw_amg_opts &o, const DCSR *A0, cudaStream_t st)
{
    std::unique_ptr<Hier> h(new Hier);
    h->dev = A->dev;
    h->o = o;
    h->A0 = A0;
    h->gnx = A->nx;
    h->gny = A->ny;
    h->gnz = A->nz;
    build_hierarchy(*h, st);
    if (h->L < 2) fail(GW_ERR_SETUP, "gw_amg_setup: the matrix is small enough for one level (n <= n_coarse)");
    return h;
}

// |s_i - s_built_i| >= delta * C_ii counts a row that breaks the reuse criterion
__global__ void k_reuse_check(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ v, const double *__restrict__ s,
                              const double *__restrict__ sb, double delta, int *__restrict__ bad)
{
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        double cii = 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i) cii = v[e];
        const double ds = (s ? s[i] : 0.0) - (sb ? sb[i] : 0.0);
        if (!(fabs(ds) < delta * cii)) atomicAdd(bad, 1);
    }
}

// The coarse operators formed with the shift s_ref stay while every
// |s_i - s_ref_i| <= gamma s_ref_i: their storage part P^T diag(s) P then
// stays within the factors 1 -/+ gamma of the one they hold (s_ref = 0 only
// for s = 0).
__global__ void k_coarse_check(int n, const double *__restrict__ s, const double *__restrict__ sr, double gamma,
                               int *__restrict__ bad)
{
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const double a = s ? s[i] : 0.0, r = sr ? sr[i] : 0.0;
        if (!(fabs(a - r) <= gamma * r) && !(a == 0.0 && r == 0.0)) atomicAdd(bad, 1);
    }
}

// A = C + diag(s) on a copy of C's pattern
__global__ void k_shift_diag(int n, const int *__restrict__ rp, const int *__restrict__ ci, double *__restrict__ v,
                             const double *__restrict__ s)
{
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        for (int e = rp[i]; e < rp[i + 1]; ++e)
            if (ci[e] == i) v[e] = v[e] + s[i];
    }
}

constexpr double SHIFT_COARSE_GAMMA = 0.25;

#define GW_API_BEGIN try {
#define GW_API_END                                    \
    }                                                 \
    catch (const gw::Error &e)                        \
    {                                                 \
        gw::set_last_error(e.msg.c_str());            \
        return e.code;                                \
    }                                                 \
    catch (const std::bad_alloc &)                    \
    {                                                 \
        gw::set_last_error("host allocation failed"); \
        return GW_ERR_OOM;                            \
    }                                                 \
    catch (...)                                       \
    {                                                 \
        gw::set_last_error("unexpected failure");     \
        return GW_ERR_CUDA;                           \
    }                                                 \
    return GW_OK;

extern "C" {

void gw_amg_opts_default(gw_amg_opts *o)
{
    if (!o) return;
    o->theta = 0.04;
    o->smoother = GW_SMOOTH_CHEBYSHEV;
    o->degree = 2;
    o->nu = 1;
    o->n_coarse = 1024;
    o->max_levels = 12;
    o->seed = 0x5EEDULL;
    o->prec = GW_PREC_MIXED32;
    o->delta = 0.1;
    o->half_storage = 0;
    o->mis_max_rounds = 200;
}

const char *gw_status_str(int s)
{
    switch (s) {
    case GW_OK: return "GW_OK";
    case GW_ERR_ARG: return "GW_ERR_ARG";
    case GW_ERR_CUDA: return "GW_ERR_CUDA";
    case GW_ERR_OOM: return "GW_ERR_OOM";
    case GW_ERR_SETUP: return "GW_ERR_SETUP";
    case GW_ERR_NOT_CONVERGED: return "GW_ERR_NOT_CONVERGED";
    case GW_ERR_BREAKDOWN: return "GW_ERR_BREAKDOWN";
    default: return "GW_UNKNOWN_STATUS";
    }
}

const char *gw_last_error(void) { return gw::last_error_cstr(); }

long long gw_device_allocations(void) { return gw::device_allocations(); }

int gw_assemble(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz, const gw_bc *bc,
                const double *q, gw_matrix *A_out, double *b_out, void *stream)
{
    GW_API_BEGIN
    if (!grid || !Kx || !bc || !A_out || !b_out) fail(GW_ERR_ARG, "gw_assemble: null argument");
    *A_out = nullptr;
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 1 || ny < 1 || nz < 1) fail(GW_ERR_ARG, "gw_assemble: grid sizes must be >= 1");
    const double dx = grid->dx, dy = grid->dy, dz = grid->dz;
    if (!(dx > 0.0) || !(dy > 0.0) || !(dz > 0.0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
        fail(GW_ERR_ARG, "gw_assemble: cell sizes must be positive and finite");
    const long long n64 = (long long)nx * ny * nz;
    if (n64 > 0x7fffffffLL / 8) fail(GW_ERR_ARG, "gw_assemble: %lld cells is too many", n64);
    int ndir = 0;
    for (int f = 0; f < 6; ++f) {
        if (bc->type[f] != GW_NOFLOW && bc->type[f] != GW_DIRICHLET) fail(GW_ERR_ARG, "gw_assemble: bad face type");
        if (bc->type[f] == GW_DIRICHLET) {
            if (!isfinite(bc->value[f])) fail(GW_ERR_ARG, "gw_assemble: head on face %d is not finite", f);
            ++ndir;
        }
    }
    if (ndir == 0) fail(GW_ERR_ARG, "gw_assemble: no Dirichlet face, the system is singular");
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    const size_t n = (size_t)n64;
    int dev = 0;
    GW_CUDA(cudaGetDevice(&dev));
    DevIn<double> kx(Kx, n, st), ky(Ky ? Ky : Kx, n, st), kz(Kz ? Kz : Kx, n, st), qq(q, n, st);
    const bool bdev = is_device_ptr(b_out);
    DBuf<double> btmp;
    double *bd = b_out;
    if (!bdev) {
        btmp.alloc(n);
        bd = btmp.p;
    }
    DBuf<int> flag(1);
    gw_matrix M = new gw_matrix_s;
    try {
        M->dev = dev;
        M->nx = nx;
        M->ny = ny;
        M->nz = nz;
        assemble_csr(nx, ny, nz, dx, dy, dz, kx.p, ky.p, kz.p, bc->type, bc->value, qq.p, M->A, bd, flag.p, st);
        if (!bdev) GW_CUDA(cudaMemcpyAsync(b_out, bd, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        GW_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        delete M;
        throw;
    }
    *A_out = M;
    GW_API_END
}

int gw_matrix_size(gw_matrix A, int *n, long long *nnz)
{
    GW_API_BEGIN
    if (!A) fail(GW_ERR_ARG, "gw_matrix_size: null matrix");
    if (n) *n = A->A.nr;
    if (nnz) *nnz = A->A.nnz;
    GW_API_END
}

int gw_matrix_export(gw_matrix A, int *rowptr, int *col, double *val, void *stream)
{
    GW_API_BEGIN
    if (!A) fail(GW_ERR_ARG, "gw_matrix_export: null matrix");
    DeviceGuard g(A->dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    if (rowptr) to_device(rowptr, A->A.rp.p, ((size_t)A->A.nr + 1) * sizeof(int), st);
    if (col) to_device(col, A->A.ci.p, (size_t)A->A.nnz * sizeof(int), st);
    if (val) to_device(val, A->A.v.p, (size_t)A->A.nnz * sizeof(double), st);
    GW_CUDA(cudaStreamSynchronize(st));
    GW_API_END
}

int gw_amg_setup(gw_matrix A, const gw_amg_opts *opts, gw_hierarchy *H_out, void *stream)
{
    GW_API_BEGIN
    if (!A || !H_out) fail(GW_ERR_ARG, "gw_amg_setup: null argument");
    *H_out = nullptr;
    gw_amg_opts o;
    gw_amg_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.theta >= 0.0) || !isfinite(o.theta)) fail(GW_ERR_ARG, "gw_amg_setup: theta must be >= 0");
    if (o.smoother != GW_SMOOTH_JACOBI && o.smoother != GW_SMOOTH_CHEBYSHEV) fail(GW_ERR_ARG, "gw_amg_setup: bad smoother");
    if (o.degree < 1 || o.degree > 8 || o.nu < 1 || o.nu > 8) fail(GW_ERR_ARG, "gw_amg_setup: degree and nu must be in 1..8");
    if (o.n_coarse < 1 || o.n_coarse > 4096) fail(GW_ERR_ARG, "gw_amg_setup: n_coarse must be in 1..4096");
    if (o.max_levels < 2 || o.max_levels > 16) fail(GW_ERR_ARG, "gw_amg_setup: max_levels must be in 2..16");
    if (o.mis_max_rounds < 0) fail(GW_ERR_ARG, "gw_amg_setup: mis_max_rounds must be >= 0");
    if (o.mis_max_rounds == 0) o.mis_max_rounds = 200;
    if (o.prec == GW_PREC_MIXEDBF16) {
        o.prec = GW_PREC_MIXED32;
        o.half_storage |= GW_HALF_FINE;
    }
    if (o.prec == GW_PREC_MIXED16) {
        o.prec = GW_PREC_MIXED32;
        o.half_storage |= GW_HALF_FINE16;
    }
    if (o.prec != GW_PREC_FP64 && o.prec != GW_PREC_MIXED32) fail(GW_ERR_ARG, "gw_amg_setup: bad precision");
    if (o.half_storage & ~(GW_HALF_FINE | GW_HALF_FINE16))
        fail(GW_ERR_ARG, "gw_amg_setup: bad half_storage bits");
    if ((o.half_storage & GW_HALF_FINE) && (o.half_storage & GW_HALF_FINE16))
        fail(GW_ERR_ARG, "gw_amg_setup: the fine stencil is stored either in BF16 or in FP16");
    if (o.prec == GW_PREC_FP64 && o.half_storage)
        fail(GW_ERR_ARG, "gw_amg_setup: half_storage belongs to the mixed form");
    if (!(o.delta > 0.0 && o.delta < 1.0)) fail(GW_ERR_ARG, "gw_amg_setup: delta must be in (0, 1)");
    DeviceGuard g(A->dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    gw_hierarchy h = new gw_hierarchy_s;
    try {
        h->base = A;
        h->h = new_hier(A, o, &A->A, st);
    } catch (...) {
        delete h;
        throw;
    }
    *H_out = h;
    GW_API_END
}

int gw_pcg_solve(gw_hierarchy H, const double *b, double *h, double tol, int maxit, int *iters, double *relres,
                 void *stream)
{
    int status = GW_OK;
    GW_API_BEGIN
    if (!H || !b || !h) fail(GW_ERR_ARG, "gw_pcg_solve: null argument");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_pcg_solve: the hierarchy's solve is in a batch");
    if (!(tol > 0.0) || !isfinite(tol) || maxit < 1) fail(GW_ERR_ARG, "gw_pcg_solve: need tol > 0 and maxit >= 1");
    Hier &hh = *H->h;
    DeviceGuard g(hh.dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    const size_t bytes = (size_t)hh.n * sizeof(double);
    GW_CUDA(cudaMemcpyAsync(hh.b.p, b, bytes, cudaMemcpyDefault, st));
    status = pcg_run(hh, tol, maxit, iters, relres, st);
    GW_CUDA(cudaMemcpyAsync(h, hh.x.p, bytes, cudaMemcpyDefault, st));
    GW_CUDA(cudaStreamSynchronize(st));
    if (status != GW_OK) {
        gw::set_last_error(status == GW_ERR_NOT_CONVERGED ? "gw_pcg_solve: maxit reached"
                           : status == GW_ERR_ARG          ? "gw_pcg_solve: the right-hand side has a non-finite entry"
                                                           : "gw_pcg_solve: CG breakdown");
        return status;
    }
    GW_API_END
}

int gw_hierarchy_prepare(gw_hierarchy H)
{
    GW_API_BEGIN
    if (!H) fail(GW_ERR_ARG, "gw_hierarchy_prepare: null hierarchy");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_hierarchy_prepare: the hierarchy's solve is in a batch");
    Hier &hh = *H->h;
    DeviceGuard g(hh.dev);
    pcg_prepare(hh);
    GW_API_END
}

int gw_pcg_solve_many(gw_hierarchy H, int k, const double *B, double *X, double tol, int maxit, int *iters,
                      double *relres, void *stream)
{
    int worst = GW_OK;
    GW_API_BEGIN
    if (!H || !B || !X || k < 1) fail(GW_ERR_ARG, "gw_pcg_solve_many: bad argument");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_pcg_solve_many: the hierarchy's solve is in a batch");
    if (!(tol > 0.0) || !isfinite(tol) || maxit < 1) fail(GW_ERR_ARG, "gw_pcg_solve_many: need tol > 0 and maxit >= 1");
    Hier &hh = *H->h;
    DeviceGuard g(hh.dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    const size_t n = (size_t)hh.n, bytes = n * sizeof(double);
    if (k > 1 && block_supported(hh)) {
        worst = block_solve(hh, k, B, X, tol, maxit, iters, relres, st);
        if (worst != GW_OK) {
            gw::set_last_error("gw_pcg_solve_many: a right-hand side did not converge");
            return worst;
        }
        return GW_OK;
    }
    for (int c = 0; c < k; ++c) {
        int it = 0;
        double rel = 0.0;
        GW_CUDA(cudaMemcpyAsync(hh.b.p, B + (size_t)c * n, bytes, cudaMemcpyDefault, st));
        const int status = pcg_run(hh, tol, maxit, &it, &rel, st);
        GW_CUDA(cudaMemcpyAsync(X + (size_t)c * n, hh.x.p, bytes, cudaMemcpyDefault, st));
        if (iters) iters[c] = it;
        if (relres) relres[c] = rel;
        if (status != GW_OK && worst == GW_OK) worst = status;
    }
    GW_CUDA(cudaStreamSynchronize(st));
    if (worst != GW_OK) {
        gw::set_last_error("gw_pcg_solve_many: a right-hand side did not converge");
        return worst;
    }
    GW_API_END
}

int gw_hierarchy_shift(gw_hierarchy H, const double *s, double delta, int *rebuilt, void *stream)
{
    GW_API_BEGIN
    if (!H || !H->base) fail(GW_ERR_ARG, "gw_hierarchy_shift: null hierarchy");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_hierarchy_shift: the hierarchy's solve is in a batch");
    if (!(delta > 0.0 && delta < 1.0)) fail(GW_ERR_ARG, "gw_hierarchy_shift: delta must be in (0, 1)");
    gw_matrix C = H->base;
    DeviceGuard g(C->dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    const int n = C->A.nr;
    const int gb = (int)std::min<long long>(((long long)n + 255) / 256, 152LL * 16);
    DBuf<double> snew;
    if (s) {
        snew.alloc((size_t)n);
        GW_CUDA(cudaMemcpyAsync(snew.p, s, (size_t)n * sizeof(double), cudaMemcpyDefault, st));
    }
    DBuf<int> bad(1);
    GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    gw_launch(k_reuse_check, gb, 256, 0, st, n, C->A.rp.p, C->A.ci.p, C->A.v.p, snew.p, H->s_built.p, delta, bad.p);
    GW_LAUNCH_CHECK();
    const bool reuse = read_int(bad.p, st) == 0;
    DCSR A;
    const DCSR *target = &C->A;
    if (s) {
        A.nr = A.nc = n;
        A.nnz = C->A.nnz;
        A.rp.alloc((size_t)n + 1);
        A.ci.alloc((size_t)A.nnz);
        A.v.alloc((size_t)A.nnz);
        GW_CUDA(cudaMemcpyAsync(A.rp.p, C->A.rp.p, A.rp.bytes(), cudaMemcpyDeviceToDevice, st));
        GW_CUDA(cudaMemcpyAsync(A.ci.p, C->A.ci.p, A.ci.bytes(), cudaMemcpyDeviceToDevice, st));
        GW_CUDA(cudaMemcpyAsync(A.v.p, C->A.v.p, A.v.bytes(), cudaMemcpyDeviceToDevice, st));
        gw_launch(k_shift_diag, gb, 256, 0, st, n, A.rp.p, A.ci.p, A.v.p, snew.p);
        GW_LAUNCH_CHECK();
    }
    if (reuse) {
        // keep the coarse operators if the shift stayed close to theirs,
        // else form them again on the kept aggregates and prolongators
        GW_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        gw_launch(k_coarse_check, gb, 256, 0, st, n, (const double *)snew.p, (const double *)H->s_ref.p,
                  SHIFT_COARSE_GAMMA, bad.p);
        GW_LAUNCH_CHECK();
        const bool keep_coarse = read_int(bad.p, st) == 0;
        if (s) {
            H->shifted = std::move(A);
            target = &H->shifted;
        }
        if (keep_coarse) {
            refresh_level0(*H->h, *target, st);
        } else {
            refresh_numeric(*H->h, *target, st);
            if (s) {
                H->s_ref.alloc((size_t)n);
                GW_CUDA(cudaMemcpyAsync(H->s_ref.p, snew.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            } else {
                H->s_ref.release();
            }
        }
        if (s) H->s_now = std::move(snew);
        else H->s_now.release();
        GW_CUDA(cudaStreamSynchronize(st));
        if (rebuilt) *rebuilt = keep_coarse ? 0 : 2;
    } else {
        const gw_amg_opts o = H->h->o;
        if (s) target = &A;
        std::unique_ptr<Hier> nh = new_hier(C, o, target, st);
        nh->prof_on = H->h->prof_on;
        H->h = std::move(nh);
        if (s) {
            H->shifted = std::move(A);
            H->h->A0 = &H->shifted;
            H->s_built.alloc((size_t)n);
            GW_CUDA(cudaMemcpyAsync(H->s_built.p, snew.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            H->s_ref.alloc((size_t)n);
            GW_CUDA(cudaMemcpyAsync(H->s_ref.p, snew.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            H->s_now = std::move(snew);
        } else {
            H->shifted = DCSR();
            H->s_built.release();
            H->s_ref.release();
            H->s_now.release();
        }
        GW_CUDA(cudaStreamSynchronize(st));
        if (rebuilt) *rebuilt = 1;
    }
    GW_API_END
}

int gw_vcycle(gw_hierarchy H, const double *r, double *z, void *stream)
{
    GW_API_BEGIN
    if (!H || !r || !z) fail(GW_ERR_ARG, "gw_vcycle: null argument");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_vcycle: the hierarchy's solve is in a batch");
    if (!is_device_ptr(r) || !is_device_ptr(z)) fail(GW_ERR_ARG, "gw_vcycle: r and z must be device pointers");
    DeviceGuard g(H->h->dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    vcycle_enqueue(*H->h, r, z, nullptr, false, st);
    GW_CUDA(cudaStreamSynchronize(st));
    GW_API_END
}

int gw_hierarchy_info(gw_hierarchy H, gw_level_info *out, int cap, int *nlevels)
{
    GW_API_BEGIN
    if (!H) fail(GW_ERR_ARG, "gw_hierarchy_info: null hierarchy");
    if (nlevels) *nlevels = H->h->L;
    for (int l = 0; out && l < cap && l < H->h->L; ++l) out[l] = H->h->info[(size_t)l];
    GW_API_END
}

int gw_hierarchy_export(gw_hierarchy H, int level, int *agg, unsigned char *root, int *a_rowptr, int *a_col,
                        double *a_val, int *p_rowptr, int *p_col, double *p_val, void *stream)
{
    GW_API_BEGIN
    if (!H) fail(GW_ERR_ARG, "gw_hierarchy_export: null hierarchy");
    Hier &hh = *H->h;
    if (level < 0 || level >= hh.L) fail(GW_ERR_ARG, "gw_hierarchy_export: level out of range");
    DeviceGuard g(hh.dev);
    cudaStream_t st = (cudaStream_t)stream;
    AllocStream alloc_scope(st);
    const DCSR &A = level == 0 ? *hh.A0 : hh.A[(size_t)level];
    const size_t n = (size_t)A.nr;
    if (agg && hh.agg[(size_t)level].p) to_device(agg, hh.agg[(size_t)level].p, n * sizeof(int), st);
    if (root && hh.root[(size_t)level].p) to_device(root, hh.root[(size_t)level].p, n, st);
    if (a_rowptr) to_device(a_rowptr, A.rp.p, (n + 1) * sizeof(int), st);
    if (a_col) to_device(a_col, A.ci.p, (size_t)A.nnz * sizeof(int), st);
    if (a_val) to_device(a_val, A.v.p, (size_t)A.nnz * sizeof(double), st);
    if (level < hh.L - 1) {
        const DCSR &P = hh.P[(size_t)level];
        if (p_rowptr) to_device(p_rowptr, P.rp.p, (n + 1) * sizeof(int), st);
        if (p_col) to_device(p_col, P.ci.p, (size_t)P.nnz * sizeof(int), st);
        if (p_val) to_device(p_val, P.v.p, (size_t)P.nnz * sizeof(double), st);
    }
    GW_CUDA(cudaStreamSynchronize(st));
    GW_API_END
}

int gw_profile_enable(gw_hierarchy H, int on)
{
    GW_API_BEGIN
    if (!H) fail(GW_ERR_ARG, "gw_profile_enable: null hierarchy");
    DeviceGuard g(H->h->dev);
    if ((bool)on != H->h->prof_on) {
        H->h->prof_on = on != 0;
        drop_graphs(*H->h);
    }
    GW_API_END
}

int gw_profile_read(gw_hierarchy H, gw_profile *out, int reset)
{
    GW_API_BEGIN
    if (!H || !out) fail(GW_ERR_ARG, "gw_profile_read: null argument");
    Hier &h = *H->h;
    memset(out, 0, sizeof *out);
    for (int k = 0; k < GW_PK_COUNT; ++k) {
        out->ms[k] = h.prof_ms[k];
        out->launches[k] = h.prof_cnt[k];
        out->bytes[k] = h.prof_b[k];
    }
    out->kernel_launches = h.launches;
    out->solves = h.solves;
    if (reset) {
        for (int k = 0; k < GW_PK_COUNT; ++k) {
            h.prof_ms[k] = 0.0;
            h.prof_cnt[k] = 0;
        }
        h.launches = 0;
        h.solves = 0;
    }
    GW_API_END
}

void gw_matrix_free(gw_matrix A)
{
    if (!A) return;
    try {
        DeviceGuard g(A->dev);
        delete A;
    } catch (...) {
    }
}

void gw_hierarchy_free(gw_hierarchy H)
{
    if (!H) return;
    try {
        DeviceGuard g(H->h->dev);
        delete H;
    } catch (...) {
    }
}

// ------------------------------------------------------------ batched solves --
struct gw_batch_s {
    gw::Batch *b = nullptr;
    int dev = 0;
};

int gw_batch_create(int max_slots, gw_batch *B_out)
{
    GW_API_BEGIN
    if (!B_out) fail(GW_ERR_ARG, "gw_batch_create: null argument");
    *B_out = nullptr;
    std::unique_ptr<gw_batch_s> B(new gw_batch_s);
    GW_CUDA(cudaGetDevice(&B->dev));
    B->b = gw::batch_create(max_slots);
    *B_out = B.release();
    GW_API_END
}

int gw_batch_add(gw_batch B, gw_hierarchy H, const double *b, double tol, int maxit, int *slot)
{
    GW_API_BEGIN
    if (!B || !H || !b) fail(GW_ERR_ARG, "gw_batch_add: null argument");
    if (!(tol > 0.0) || !isfinite(tol) || maxit < 1) fail(GW_ERR_ARG, "gw_batch_add: need tol > 0 and maxit >= 1");
    if (H->h->batch) fail(GW_ERR_ARG, "gw_batch_add: the hierarchy's solve is already in a batch");
    DeviceGuard g(B->dev);
    const int s = gw::batch_add(*B->b, *H->h, b, tol, maxit);
    if (slot) *slot = s;
    GW_API_END
}

int gw_batch_run(gw_batch B, int iterations, int *finished)
{
    GW_API_BEGIN
    if (!B || iterations < 0) fail(GW_ERR_ARG, "gw_batch_run: bad argument");
    DeviceGuard g(B->dev);
    const int f = gw::batch_run(*B->b, iterations);
    if (finished) *finished = f;
    GW_API_END
}

int gw_batch_state(gw_batch B, int slot, int *state)
{
    GW_API_BEGIN
    if (!B || !state) fail(GW_ERR_ARG, "gw_batch_state: null argument");
    *state = gw::batch_state(*B->b, slot);
    if (*state < 0) fail(GW_ERR_ARG, "gw_batch_state: no slot %d", slot);
    GW_API_END
}

int gw_batch_take(gw_batch B, int slot, double *h, int *iters, double *relres)
{
    int status = GW_OK;
    GW_API_BEGIN
    if (!B) fail(GW_ERR_ARG, "gw_batch_take: null batch");
    DeviceGuard g(B->dev);
    status = gw::batch_take(*B->b, slot, h, iters, relres);
    if (status != GW_OK) {
        gw::set_last_error(status == GW_ERR_NOT_CONVERGED ? "gw_batch_take: maxit reached"
                           : status == GW_ERR_ARG          ? "gw_batch_take: the right-hand side has a non-finite entry"
                                                           : "gw_batch_take: CG breakdown");
        return status;
    }
    GW_API_END
}

void gw_batch_free(gw_batch B)
{
    if (!B) return;
    try {
        DeviceGuard g(B->dev);
        gw::batch_free(B->b);
    } catch (...) {
    }
    delete B;
}

}  // extern "C"
