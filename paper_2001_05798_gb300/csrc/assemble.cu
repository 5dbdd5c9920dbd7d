// assemble.cu -- finite-volume assembly of the steady flow system C h = Q.
//
// Cell-centred 5/7-point finite volumes on a regular grid give an M-matrix
// (Benchmarking Examples section); Eq. 2 of the paper with zero storage is
// C h = Q.  Face transmissibilities are harmonic means of the two cells'
// conductivities times face area over centre distance; a Dirichlet head sits
// on the boundary face, half a cell from the centre.  Every product and sum
// is an explicitly rounded intrinsic in a fixed order, so the matrix is the
// same double for double as any implementation that follows that order.
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
    k_asm_validate<<<grid, bs, 0, st>>>(n, Kx, Ky, Kz, q, dflag);
    GW_LAUNCH_CHECK();
    if (read_int(dflag, st)) fail(GW_ERR_ARG, "gw_assemble: a conductivity is <= 0 or not finite, or q is not finite");
    A.nr = A.nc = n;
    A.rp.alloc((size_t)n + 1);
    k_asm_rowcount<<<grid, bs, 0, st>>>(G, A.rp.p);
    GW_LAUNCH_CHECK();
    exclusive_scan(A.rp.p, A.rp.p, n, st);
    A.nnz = read_int(A.rp.p + n, st);
    A.ci.alloc((size_t)A.nnz);
    A.v.alloc((size_t)A.nnz);
    k_asm_fill<<<grid, bs, 0, st>>>(G, Kx, Ky, Kz, q, A.rp.p, A.ci.p, A.v.p, b);
    GW_LAUNCH_CHECK();
}

}  // namespace gw
