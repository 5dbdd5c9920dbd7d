// assemble.cu -- finite-volume assembly of the steady flow system C h = Q.
//
// Cell-centred 5/7-point finite volumes on a regular grid give an M-matrix
// (Benchmarking Examples section); Eq. 2 of the paper with zero storage is
// C h = Q.  Face transmissibilities are harmonic means of the two cells'
// conductivities times face area over centre distance; a Dirichlet head sits
// on the boundary face, half a cell from the centre.  Every product and sum
// is an explicitly rounded intrinsic in a fixed order, so the matrix is the
// same double for double as any implementation that follows that order.
#include <atomic>
#include <mutex>

#include "gw_internal.cuh"

namespace gw {

struct AsmGeom {
    int nx, ny, nz;
    double g[3];      // face area over centre distance per axis
    int bct[6];
    double bcv[6];
};

__device__ __forceinline__ double harm_T(double a, double b, double g)
{
    double t = __dmul_rn(2.0, a);
    t = __dmul_rn(t, b);
    double s = __dadd_rn(a, b);
    return __dmul_rn(__ddiv_rn(t, s), g);
}

__global__ void k_asm_validate(int n, const double *__restrict__ Kx, const double *__restrict__ Ky,
                               const double *__restrict__ Kz, const double *__restrict__ q, int *flag)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double a = Kx[i], b = Ky[i], c = Kz[i];
        bool bad = !(a > 0.0) || !isfinite(a) || !(b > 0.0) || !isfinite(b) || !(c > 0.0) || !isfinite(c);
        if (q && !isfinite(q[i])) bad = true;
        if (bad) atomicOr(flag, 1);
    }
}

__global__ void k_asm_rowcount(AsmGeom G, int *__restrict__ cnt)
{
    const long long n = (long long)G.nx * G.ny * G.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % G.nx), y = (int)((i / G.nx) % G.ny), z = (int)(i / ((long long)G.nx * G.ny));
        cnt[i] = 1 + (x > 0) + (x < G.nx - 1) + (y > 0) + (y < G.ny - 1) + (z > 0) + (z < G.nz - 1);
    }
}

__global__ void k_asm_fill(AsmGeom G, const double *__restrict__ Kx, const double *__restrict__ Ky,
                           const double *__restrict__ Kz, const double *__restrict__ q, const int *__restrict__ rp,
                           int *__restrict__ ci, double *__restrict__ v, double *__restrict__ b)
{
    const long long n = (long long)G.nx * G.ny * G.nz;
    const int sxy = G.nx * G.ny;
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const int x = i % G.nx, y = (i / G.nx) % G.ny, z = i / sxy;
        const double *K[3] = {Kx, Ky, Kz};
        const int crd[3] = {x, y, z}, dim[3] = {G.nx, G.ny, G.nz}, stride[3] = {1, G.nx, sxy};
        double T[6];
        int nb[6];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int f = 2 * d + s;
                const bool interior = s == 0 ? crd[d] > 0 : crd[d] < dim[d] - 1;
                if (interior) {
                    const int j = s == 0 ? i - stride[d] : i + stride[d];
                    const int lo = min(i, j), hi = max(i, j);
                    T[f] = harm_T(K[d][lo], K[d][hi], G.g[d]);
                    nb[f] = j;
                } else {
                    nb[f] = -1;
                    T[f] = G.bct[f] == GW_DIRICHLET ? __dmul_rn(__dmul_rn(2.0, K[d][i]), G.g[d]) : 0.0;
                }
            }
        }
        double diag = 0.0, rhs = q ? q[i] : 0.0;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (nb[f] >= 0) {
                diag = __dadd_rn(diag, T[f]);
            } else if (G.bct[f] == GW_DIRICHLET) {
                diag = __dadd_rn(diag, T[f]);
                rhs = __dadd_rn(rhs, __dmul_rn(T[f], G.bcv[f]));
            }
        }
        b[i] = rhs;
        int e = rp[i];
        // ascending columns: -z, -y, -x, i, +x, +y, +z
        const int order[7] = {4, 2, 0, -1, 1, 3, 5};
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const int f = order[k];
            if (f < 0) {
                ci[e] = i;
                v[e] = diag;
                ++e;
            } else if (nb[f] >= 0) {
                ci[e] = nb[f];
                v[e] = -T[f];
                ++e;
            }
        }
    }
}

void assemble_csr(int nx, int ny, int nz, double dx, double dy, double dz, const double *Kx, const double *Ky,
                  const double *Kz, const int *bct, const double *bcv, const double *q, DCSR &A, double *b,
                  int *dflag, cudaStream_t st)
{
    const int n = nx * ny * nz;
    AsmGeom G;
    G.nx = nx;
    G.ny = ny;
    G.nz = nz;
    G.g[0] = (dy * dz) / dx;
    G.g[1] = (dx * dz) / dy;
    G.g[2] = (dx * dy) / dz;
    for (int f = 0; f < 6; ++f) {
        G.bct[f] = bct[f];
        G.bcv[f] = bcv[f];
    }
    const int bs = 256;
    const int grid = (int)std::min<long long>((n + bs - 1) / bs, 152LL * 16);
    GW_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), st));
    gw_launch(k_asm_validate, grid, bs, 0, st, n, Kx, Ky, Kz, q, dflag);
    GW_LAUNCH_CHECK();
    if (read_int(dflag, st)) fail(GW_ERR_ARG, "gw_assemble: a conductivity is <= 0 or not finite, or q is not finite");
    A.nr = A.nc = n;
    A.rp.alloc((size_t)n + 1);
    gw_launch(k_asm_rowcount, grid, bs, 0, st, G, A.rp.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(A.rp.p, A.rp.p, n, st);
    A.nnz = read_int(A.rp.p + n, st);
    A.ci.alloc((size_t)A.nnz);
    A.v.alloc((size_t)A.nnz);
    gw_launch(k_asm_fill, grid, bs, 0, st, G, Kx, Ky, Kz, q, A.rp.p, A.ci.p, A.v.p, b);
    GW_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- adjoint --
// dJ/dlnK_i = lambda^T (dQ/dlnK_i - dC/dlnK_i h), with lnK scaling Kx, Ky, Kz of
// cell i together: an interior face with T = 2 K_i K_j/(K_i+K_j) g has
// dT/dlnK_i = T K_j/(K_i + K_j) and contributes -dT/dlnK_i (h_i - h_j)
// (lambda_i - lambda_j); a Dirichlet face (T_b = 2 K_i g, dT_b/dlnK_i = T_b)
// contributes -T_b (h_i - h_b) lambda_i.
__global__ void k_adj_grad(AsmGeom G, const double *__restrict__ Kx, const double *__restrict__ Ky,
                           const double *__restrict__ Kz, const double *__restrict__ h,
                           const double *__restrict__ lam, double *__restrict__ grad)
{
    const long long n = (long long)G.nx * G.ny * G.nz;
    const int sxy = G.nx * G.ny;
    for (long long ii = blockIdx.x * (long long)blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const int crd[3] = {i % G.nx, (i / G.nx) % G.ny, i / sxy}, dim[3] = {G.nx, G.ny, G.nz},
                  stride[3] = {1, G.nx, sxy};
        const double *K[3] = {Kx, Ky, Kz};
        const double hi = h[i], li = lam[i];
        double s = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double Ki = K[d][i];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * d + side;
                const bool interior = side == 0 ? crd[d] > 0 : crd[d] < dim[d] - 1;
                if (interior) {
                    const int j = side == 0 ? i - stride[d] : i + stride[d];
                    const double Kj = K[d][j];
                    const double T = harm_T(K[d][min(i, j)], K[d][max(i, j)], G.g[d]);
                    s += T * (Kj / (Ki + Kj)) * (hi - h[j]) * (li - lam[j]);
                } else if (G.bct[f] == GW_DIRICHLET) {
                    s += (2.0 * Ki) * G.g[d] * (hi - G.bcv[f]) * li;
                }
            }
        }
        grad[i] = -s;
    }
}

__global__ void k_zero(long long n, double *__restrict__ a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0.0;
}

// J = sum_k (h[obs_k] - hobs_k)^2 summed in k order by one block; dJ/dh
// scattered in k order by one thread (repeated cells add up)
__global__ void k_misfit(int nobs, const double *__restrict__ h, const int *__restrict__ obs,
                         const double *__restrict__ hobs, double *__restrict__ J, double *__restrict__ dJdh)
{
    __shared__ double sh[1024];
    double loc = 0.0;
    for (int k = threadIdx.x; k < nobs; k += blockDim.x) {
        const double r = h[obs[k]] - hobs[k];
        loc += r * r;
    }
    sh[threadIdx.x] = loc;
    __syncthreads();
    for (int off = blockDim.x >> 1; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *J = sh[0];
        if (dJdh)
            for (int k = 0; k < nobs; ++k) dJdh[obs[k]] += 2.0 * (h[obs[k]] - hobs[k]);
    }
}

// ------------------------------------------------------ Darcy face fluxes --
// Velocity on every face (staggered layout: face f = 0..n_d along axis d),
// positive along the axis: K_harm (h_a - h_b) / spacing between cells a < b
// (T / A_f with T of the assembly), 2 K (h_face - h) / spacing on Dirichlet
// faces, 0 on no-flow faces.  One thread per cell writes the lower face of
// each axis, and the upper one where the cell is last along that axis, so K
// and h are read once and every face array is written in row order.  One
// division per face: 2 K_a K_b (h_a - h_b) inv / (K_a + K_b), inv = 1/spacing.
struct FluxGeom {
    int n[3];
    double inv[3];    // 1 / spacing per axis
    int bct[6];
    double bcv[6];
};

__global__ void k_darcy(FluxGeom G, const double *__restrict__ Kx, const double *__restrict__ Ky,
                        const double *__restrict__ Kz, const double *__restrict__ h, double *__restrict__ vx,
                        double *__restrict__ vy, double *__restrict__ vz)
{
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const int ncell = nx * ny * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
        const int x = i % nx, yz = i / nx, y = yz % ny, z = yz / ny;
        const int c[3] = {x, y, z};
        const int stride[3] = {1, nx, nx * ny};
        const double *K[3] = {Kx, Ky, Kz};
        double *v[3] = {vx, vy, vz};
        const double hi = h[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double Ki = K[d][i];
            // face index of this cell's lower face along d
            const long long lo = d == 0 ? x + (long long)(nx + 1) * yz
                               : d == 1 ? x + (long long)nx * (y + (long long)(ny + 1) * z)
                                        : (long long)i;
            double out = 0.0;
            if (c[d] > 0) {
                const double Ka = K[d][i - stride[d]];
                out = (2.0 * Ka * Ki * (h[i - stride[d]] - hi) * G.inv[d]) / (Ka + Ki);
            } else if (G.bct[2 * d] == GW_DIRICHLET) {
                out = 2.0 * Ki * (G.bcv[2 * d] - hi) * G.inv[d];
            }
            v[d][lo] = out;
            if (c[d] == G.n[d] - 1) {
                const long long up = lo + (d == 0 ? 1 : d == 1 ? nx : (long long)nx * ny);
                v[d][up] = G.bct[2 * d + 1] == GW_DIRICHLET ? 2.0 * Ki * (hi - G.bcv[2 * d + 1]) * G.inv[d] : 0.0;
            }
        }
    }
}

}  // namespace gw

// ------------------------------------------- assembly without allocations --
// Some callers cannot allocate device memory at the point where they need
// the system assembled: a solver embedded in a host code that hands the
// library a fixed device pool, a caller inside a region where cudaMalloc
// would synchronise the device or is forbidden, or a process whose memory is
// budgeted up front.  gw_assemble_noalloc serves them: the caller passes the
// output arrays, and the only working memory the kernels need (the
// validation flag and the block totals of the row-pointer scan) lives in the
// fixed device array below, which every GPU that loads the library holds
// until the process exits.
namespace gw {

// 1 validation flag + block totals of a scan over at most NOALLOC_MAX_CELLS
// rows (2048 rows per block, two scan levels)
constexpr long long NOALLOC_MAX_CELLS = 1LL << 27;
constexpr size_t NOALLOC_SCRATCH_INTS = 1 + (size_t)(NOALLOC_MAX_CELLS / 2048) + 64 + 16;

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_SCRATCH_INTS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::atomic<int *> g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// The device address of the array: its name in host code is only a host-side
// stand-in, so it is looked up once per device with that device current.  The
// lookup can load this file's module, which would invalidate a graph capture
// running on another thread, so it waits at the library's capture gate.
static int *noalloc_scratch(int dev)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(GW_ERR_ARG, "gw_assemble_noalloc: device %d out of range", dev);
    int *p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (p) return p;
    auto gate = capture_gate();
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        fail(GW_ERR_CUDA, "gw_assemble_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
    return p;
}

}  // namespace gw

extern "C" int gw_assemble_noalloc(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz,
                                   const gw_bc *bc, const double *q, int *rowptr, int *col, double *val, double *b,
                                   void *stream)
{
    using namespace gw;
    try {
        if (!grid || !Kx || !bc || !rowptr || !col || !val || !b) fail(GW_ERR_ARG, "gw_assemble_noalloc: null argument");
        {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            GW_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
            if (cs != cudaStreamCaptureStatusNone)
                fail(GW_ERR_ARG, "gw_assemble_noalloc: the stream is being captured (the call synchronises it)");
        }
        const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
        if (nx < 1 || ny < 1 || nz < 1) fail(GW_ERR_ARG, "gw_assemble_noalloc: grid sizes must be >= 1");
        const double dx = grid->dx, dy = grid->dy, dz = grid->dz;
        if (!(dx > 0.0) || !(dy > 0.0) || !(dz > 0.0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz))
            fail(GW_ERR_ARG, "gw_assemble_noalloc: cell sizes must be positive and finite");
        const long long n64 = (long long)nx * ny * nz;
        if (n64 > NOALLOC_MAX_CELLS)
            fail(GW_ERR_ARG, "gw_assemble_noalloc: %lld cells exceeds the maximum of %lld", n64, NOALLOC_MAX_CELLS);
        int ndir = 0;
        for (int f = 0; f < 6; ++f) {
            if (bc->type[f] != GW_NOFLOW && bc->type[f] != GW_DIRICHLET)
                fail(GW_ERR_ARG, "gw_assemble_noalloc: bad face type");
            if (bc->type[f] == GW_DIRICHLET) {
                if (!isfinite(bc->value[f])) fail(GW_ERR_ARG, "gw_assemble_noalloc: head on face %d is not finite", f);
                ++ndir;
            }
        }
        if (ndir == 0) fail(GW_ERR_ARG, "gw_assemble_noalloc: no Dirichlet face, the system is singular");
        const double *ky = Ky ? Ky : Kx, *kz = Kz ? Kz : Kx;
        const void *ptrs[8] = {Kx, ky, kz, q, rowptr, col, val, b};
        for (int k = 0; k < 8; ++k)
            if (ptrs[k] && !is_device_ptr(ptrs[k]))
                fail(GW_ERR_ARG, "gw_assemble_noalloc: every array must be device memory (argument %d is not)", k);
        cudaStream_t st = (cudaStream_t)stream;
        int dev = 0;
        GW_CUDA(cudaGetDevice(&dev));
        int *scratch = noalloc_scratch(dev);
        const int n = (int)n64;
        AsmGeom G;
        G.nx = nx;
        G.ny = ny;
        G.nz = nz;
        G.g[0] = (dy * dz) / dx;
        G.g[1] = (dx * dz) / dy;
        G.g[2] = (dx * dy) / dz;
        for (int f = 0; f < 6; ++f) {
            G.bct[f] = bc->type[f];
            G.bcv[f] = bc->value[f];
        }
        const int bs = 256;
        const int grid_b = (int)std::min<long long>((n + bs - 1) / bs, 152LL * 16);
        int *flag = scratch;
        GW_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
        gw_launch(k_asm_validate, grid_b, bs, 0, st, n, Kx, ky, kz, q, flag);
        GW_LAUNCH_CHECK();
        if (read_int(flag, st))
            fail(GW_ERR_ARG, "gw_assemble_noalloc: a conductivity is <= 0 or not finite, or q is not finite");
        gw_launch(k_asm_rowcount, grid_b, bs, 0, st, G, rowptr);
        GW_LAUNCH_CHECK();
        if (!exclusive_scan_in(rowptr, rowptr, n, scratch + 1, NOALLOC_SCRATCH_INTS - 1, st))
            fail(GW_ERR_ARG, "gw_assemble_noalloc: grid too large for the scan workspace");
        gw_launch(k_asm_fill, grid_b, bs, 0, st, G, Kx, ky, kz, q, rowptr, col, val, b);
        GW_LAUNCH_CHECK();
        GW_CUDA(cudaStreamSynchronize(st));
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.code;
    } catch (...) {
        set_last_error("unexpected failure");
        return GW_ERR_CUDA;
    }
    return GW_OK;
}

extern "C" int gw_adjoint_gradient(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz,
                                   const gw_bc *bc, const double *h, const double *lambda, double *grad, void *stream)
{
    using namespace gw;
    try {
        if (!grid || !Kx || !bc || !h || !lambda || !grad) fail(GW_ERR_ARG, "gw_adjoint_gradient: null argument");
        const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
        if (nx < 1 || ny < 1 || nz < 1) fail(GW_ERR_ARG, "gw_adjoint_gradient: grid sizes must be >= 1");
        const long long n64 = (long long)nx * ny * nz;
        if (n64 > 0x7fffffffLL / 8) fail(GW_ERR_ARG, "gw_adjoint_gradient: too many cells");
        const double *ky = Ky ? Ky : Kx, *kz = Kz ? Kz : Kx;
        const void *ptrs[7] = {Kx, ky, kz, h, lambda, grad, nullptr};
        for (int k = 0; k < 6; ++k)
            if (!is_device_ptr(ptrs[k])) fail(GW_ERR_ARG, "gw_adjoint_gradient: arrays must be device memory");
        AsmGeom G;
        G.nx = nx;
        G.ny = ny;
        G.nz = nz;
        G.g[0] = (grid->dy * grid->dz) / grid->dx;
        G.g[1] = (grid->dx * grid->dz) / grid->dy;
        G.g[2] = (grid->dx * grid->dy) / grid->dz;
        for (int f = 0; f < 6; ++f) {
            G.bct[f] = bc->type[f];
            G.bcv[f] = bc->value[f];
        }
        cudaStream_t st = (cudaStream_t)stream;
        AllocStream alloc_scope(st);
        const int grid_b = (int)std::min<long long>((n64 + 255) / 256, 152LL * 16);
        gw_launch(k_adj_grad, grid_b, 256, 0, st, G, Kx, ky, kz, h, lambda, grad);
        GW_LAUNCH_CHECK();
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.code;
    } catch (...) {
        set_last_error("unexpected failure");
        return GW_ERR_CUDA;
    }
    return GW_OK;
}

extern "C" int gw_misfit(int n, const double *h, int nobs, const int *obs, const double *hobs, double *J,
                         double *dJdh, void *stream)
{
    using namespace gw;
    try {
        if (n < 1 || nobs < 0 || nobs > (1 << 24) || !h || !J || (nobs && (!obs || !hobs)))
            fail(GW_ERR_ARG, "gw_misfit: bad argument");
        cudaStream_t st = (cudaStream_t)stream;
        AllocStream alloc_scope(st);
        DBuf<double> jd(1);
        if (dJdh) {
            gw_launch(k_zero, (int)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, st, n, dJdh);
            GW_LAUNCH_CHECK();
        }
        gw_launch(k_misfit, 1, 1024, 0, st, nobs, h, obs, hobs, jd.p, dJdh);
        GW_LAUNCH_CHECK();
        GW_CUDA(cudaMemcpyAsync(J, jd.p, sizeof(double), cudaMemcpyDefault, st));
        GW_CUDA(cudaStreamSynchronize(st));
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.code;
    } catch (...) {
        set_last_error("unexpected failure");
        return GW_ERR_CUDA;
    }
    return GW_OK;
}

extern "C" int gw_darcy_flux(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz,
                             const gw_bc *bc, const double *h, double *vx, double *vy, double *vz, void *stream)
{
    using namespace gw;
    try {
        if (!grid || !Kx || !bc || !h || !vx || !vy || !vz) fail(GW_ERR_ARG, "gw_darcy_flux: null argument");
        const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
        if (nx < 1 || ny < 1 || nz < 1) fail(GW_ERR_ARG, "gw_darcy_flux: grid sizes must be >= 1");
        const double *K[3] = {Kx, Ky ? Ky : Kx, Kz ? Kz : Kx};
        double *v[3] = {vx, vy, vz};
        const void *ptrs[7] = {K[0], K[1], K[2], h, vx, vy, vz};
        for (int k = 0; k < 7; ++k)
            if (!is_device_ptr(ptrs[k])) fail(GW_ERR_ARG, "gw_darcy_flux: arrays must be device memory");
        const double sp[3] = {grid->dx, grid->dy, grid->dz};
        FluxGeom G;
        for (int d = 0; d < 3; ++d) {
            if (!(sp[d] > 0.0) || !isfinite(sp[d])) fail(GW_ERR_ARG, "gw_darcy_flux: spacings must be finite and > 0");
            G.inv[d] = 1.0 / sp[d];
        }
        G.n[0] = nx;
        G.n[1] = ny;
        G.n[2] = nz;
        for (int f = 0; f < 6; ++f) {
            G.bct[f] = bc->type[f];
            G.bcv[f] = bc->value[f];
        }
        if ((long long)nx * ny * nz > 0x7fffffffLL) fail(GW_ERR_ARG, "gw_darcy_flux: more than 2^31 - 1 cells");
        cudaStream_t st = (cudaStream_t)stream;
        AllocStream alloc_scope(st);
        const long long n = (long long)nx * ny * nz;
        const int gb = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
        gw_launch(k_darcy, gb, 256, 0, st, G, K[0], K[1], K[2], h, v[0], v[1], v[2]);
        GW_LAUNCH_CHECK();
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.code;
    } catch (...) {
        set_last_error("unexpected failure");
        return GW_ERR_CUDA;
    }
    return GW_OK;
}
