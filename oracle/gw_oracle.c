/*
 * gw_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * AMG-preconditioned CG solve of the steady groundwater flow system C h = Q
 * (Sbai & Larabi, "On Solving Groundwater Flow and Transport Models with
 * Algebraic Multigrid Preconditioning", Eq. 2 with S = 0).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library; the two are written
 * separately from the same definitions so that a mistake in one shows up as
 * a disagreement with the other.
 *
 * What each part follows:
 *   assembly       -- cell-centred 5/7-point finite volumes giving an
 *                     M-matrix (Benchmarking Examples section); harmonic-mean
 *                     face transmissibilities, Dirichlet head on the
 *                     boundary face at half-cell distance.
 *   strength, MIS-2, aggregation, smoothed P, Galerkin RAP
 *                  -- the AMG setup phase (Introduction: nodal aggregation,
 *                     prolongation/restriction built automatically;
 *                     "CG/AMG/SA" smoothed aggregation, Results section).
 *   V-cycle        -- restrict, smooth, recurse, coarse direct solve,
 *                     interpolate, correct, smooth (Introduction).
 *   PCG            -- AMG as a preconditioner of conjugate gradients
 *                     (Introduction; convergence tolerance 1e-12 used as the
 *                     reference tolerance, Benchmarking Examples section).
 *
 * Every floating-point sum is written out in a fixed order and the file is
 * compiled with -ffp-contract=off, so that the setup stages reproduce the
 * same doubles as any implementation that follows the same order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SETUP 4
#define OR_ERR_NOT_CONVERGED 5
#define OR_ERR_BREAKDOWN 6

#define OR_NOFLOW 0
#define OR_DIRICHLET 1

#define OR_MAXL 16

/* ------------------------------------------------------------------ CSR -- */
typedef struct {
    int nr, nc, nnz;
    int *rp;     /* nr+1 */
    int *ci;     /* nnz, ascending within each row */
    double *v;   /* nnz */
} ocsr;

static ocsr *csr_new(int nr, int nc, int nnz)
{
    ocsr *m = (ocsr *)calloc(1, sizeof(ocsr));
    m->nr = nr; m->nc = nc; m->nnz = nnz;
    m->rp = (int *)calloc((size_t)nr + 1, sizeof(int));
    m->ci = (int *)malloc(((size_t)nnz + 1) * sizeof(int));
    m->v = (double *)malloc(((size_t)nnz + 1) * sizeof(double));
    return m;
}

void or_csr_free(ocsr *m)
{
    if (!m) return;
    free(m->rp); free(m->ci); free(m->v); free(m);
}

void or_csr_info(const ocsr *m, int *nr, int *nc, int *nnz)
{
    *nr = m->nr; *nc = m->nc; *nnz = m->nnz;
}

void or_csr_copy(const ocsr *m, int *rp, int *ci, double *v)
{
    if (rp) memcpy(rp, m->rp, ((size_t)m->nr + 1) * sizeof(int));
    if (ci) memcpy(ci, m->ci, (size_t)m->nnz * sizeof(int));
    if (v) memcpy(v, m->v, (size_t)m->nnz * sizeof(double));
}

ocsr *or_csr_from(int nr, int nc, const int *rp, const int *ci, const double *v)
{
    ocsr *m = csr_new(nr, nc, rp[nr]);
    memcpy(m->rp, rp, ((size_t)nr + 1) * sizeof(int));
    memcpy(m->ci, ci, (size_t)m->nnz * sizeof(int));
    memcpy(m->v, v, (size_t)m->nnz * sizeof(double));
    return m;
}

/* y = A x, row by row, ascending column order */
static void csr_spmv(const ocsr *A, const double *x, double *y)
{
    for (int i = 0; i < A->nr; ++i) {
        double s = 0.0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) s += A->v[e] * x[A->ci[e]];
        y[i] = s;
    }
}

void or_spmv(const ocsr *A, const double *x, double *y) { csr_spmv(A, x, y); }

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------- assembly -- */
/* harmonic mean of two conductivities, evaluated as (2*a*b)/(a+b) with the
 * product taken left to right; a is the conductivity of the lower-index cell */
static double harm(double a, double b)
{
    double t = 2.0 * a;
    t = t * b;
    double s = a + b;
    return t / s;
}

/* number of structural nonzeros of the 7-point operator on nx*ny*nz cells
 * (no rows eliminated): 7n - 2(ny nz + nx nz + nx ny) */
long long or_nnz7(int nx, int ny, int nz)
{
    long long n = (long long)nx * ny * nz;
    return n + 2LL * ((long long)(nx - 1) * ny * nz + (long long)nx * (ny - 1) * nz +
                      (long long)nx * ny * (nz - 1));
}

/*
 * Assemble the steady flow system C h = Q on a regular nx*ny*nz grid of
 * cells dx*dy*dz (nz = 1 gives the 2D 5-point operator).
 *   interior face f between cells i < j along axis d:
 *        T_f = harm(K_d[i], K_d[j]) * g_d,  g_x = dy dz / dx (etc.)
 *   Dirichlet boundary face of cell i:  T_b = (2 K_d[i]) * g_d
 *   a_ii = sum of T over the faces of i in the order -x,+x,-y,+y,-z,+z
 *   a_ij = -T_f
 *   b_i  = q_i + sum over Dirichlet faces (same order) of T_b * h_b
 * bct/bcv: type and head of faces -x,+x,-y,+y,-z,+z.
 * Returns a CSR handle (columns ascending), writes b; *status = 0 on success,
 * OR_ERR_ARG on a bad size, a non-positive or non-finite K, or no Dirichlet
 * face (singular pure-Neumann system).
 */
ocsr *or_assemble(int nx, int ny, int nz, double dx, double dy, double dz,
                  const double *Kx, const double *Ky, const double *Kz,
                  const int *bct, const double *bcv, const double *q,
                  double *b, int *status)
{
    *status = OR_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    if (!(dx > 0.0) || !(dy > 0.0) || !(dz > 0.0)) return NULL;
    long long n64 = (long long)nx * ny * nz;
    if (n64 > 0x7fffffffLL / 8) return NULL;
    int n = (int)n64;
    int ndir = 0;
    for (int f = 0; f < 6; ++f) {
        if (bct[f] != OR_NOFLOW && bct[f] != OR_DIRICHLET) return NULL;
        if (bct[f] == OR_DIRICHLET) {
            if (!isfinite(bcv[f])) return NULL;
            ++ndir;
        }
    }
    if (ndir == 0) return NULL;
    for (int i = 0; i < n; ++i) {
        if (!(Kx[i] > 0.0) || !isfinite(Kx[i])) return NULL;
        if (!(Ky[i] > 0.0) || !isfinite(Ky[i])) return NULL;
        if (!(Kz[i] > 0.0) || !isfinite(Kz[i])) return NULL;
        if (q && !isfinite(q[i])) return NULL;
    }
    const double g[3] = {(dy * dz) / dx, (dx * dz) / dy, (dx * dy) / dz};
    const double *K[3] = {Kx, Ky, Kz};
    const int dim[3] = {nx, ny, nz};
    const int stride[3] = {1, nx, nx * ny};
    long long nnz = or_nnz7(nx, ny, nz);
    ocsr *A = csr_new(n, n, (int)nnz);
    int e = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int i = x + nx * (y + ny * z);
                int crd[3] = {x, y, z};
                double T[6];      /* face transmissibility, 0 if no-flow */
                int nb[6];        /* neighbour index or -1 (boundary face) */
                for (int d = 0; d < 3; ++d) {
                    for (int s = 0; s < 2; ++s) {
                        int f = 2 * d + s;
                        int interior = s == 0 ? crd[d] > 0 : crd[d] < dim[d] - 1;
                        if (interior) {
                            int j = s == 0 ? i - stride[d] : i + stride[d];
                            int lo = i < j ? i : j, hi = i < j ? j : i;
                            T[f] = harm(K[d][lo], K[d][hi]) * g[d];
                            nb[f] = j;
                        } else {
                            nb[f] = -1;
                            T[f] = bct[f] == OR_DIRICHLET ? (2.0 * K[d][i]) * g[d] : 0.0;
                        }
                    }
                }
                double diag = 0.0, rhs = q ? q[i] : 0.0;
                for (int f = 0; f < 6; ++f) {
                    if (nb[f] >= 0) diag += T[f];
                    else if (bct[f] == OR_DIRICHLET) {
                        diag += T[f];
                        rhs += T[f] * bcv[f];
                    }
                }
                b[i] = rhs;
                /* columns ascending: -z, -y, -x, i, +x, +y, +z */
                A->rp[i] = e;
                const int order[7] = {4, 2, 0, -1, 1, 3, 5};
                for (int k = 0; k < 7; ++k) {
                    int f = order[k];
                    if (f < 0) { A->ci[e] = i; A->v[e] = diag; ++e; }
                    else if (nb[f] >= 0) { A->ci[e] = nb[f]; A->v[e] = -T[f]; ++e; }
                }
            }
    A->rp[n] = e;
    *status = OR_OK;
    return A;
}

/* ------------------------------------------------------------- strength -- */
static double csr_diag_of(const ocsr *A, int i)
{
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
        if (A->ci[e] == i) return A->v[e];
    return 0.0;
}

static int csr_find(const ocsr *A, int i, int j)
{
    int lo = A->rp[i], hi = A->rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (A->ci[mid] == j) return mid;
        if (A->ci[mid] < j) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * Symmetrised strength of connection (smoothed aggregation, Vanek, Mandel &
 * Brezina 1996): (i,j), i != j, is strong iff a_ij^2 > theta2 * (a_ii a_jj);
 * the graph used is S union S^T.  S[e] is set per CSR slot.
 */
void or_strength(const ocsr *A, double theta2, unsigned char *S)
{
    int n = A->nr;
    double *d = (double *)malloc((size_t)n * sizeof(double));
    unsigned char *raw = (unsigned char *)malloc((size_t)A->nnz + 1);
    for (int i = 0; i < n; ++i) d[i] = csr_diag_of(A, i);
    for (int i = 0; i < n; ++i)
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (j == i) { raw[e] = 0; continue; }
            double lhs = A->v[e] * A->v[e];
            double rhs = d[i] * d[j];
            rhs = theta2 * rhs;
            raw[e] = lhs > rhs;
        }
    for (int i = 0; i < n; ++i)
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            unsigned char s = raw[e];
            if (!s && j != i) {
                int t = csr_find(A, j, i);
                if (t >= 0) s = raw[t];
            }
            S[e] = s;
        }
    free(d); free(raw);
}

/* ---------------------------------------------------------------- MIS-2 -- */
/* SplitMix64 finaliser applied to x + golden gamma (Steele, Lea & Flood 2014) */
static uint64_t smix(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t or_key(uint64_t seed, int level, int i)
{
    return smix(seed ^ ((uint64_t)level << 48) ^ (uint64_t)(uint32_t)i);
}

typedef struct { uint64_t k; int i; } kidx;

static int kidx_desc(const void *a, const void *b)
{
    const kidx *x = (const kidx *)a, *y = (const kidx *)b;
    if (x->k != y->k) return x->k > y->k ? -1 : 1;
    if (x->i != y->i) return x->i > y->i ? -1 : 1;
    return 0;
}

/*
 * Distance-2 maximal independent set on the strength graph, by its
 * definition: visit the nodes in descending (key, index) and select a node
 * unless an already selected node lies within graph distance 2 (through any
 * intermediate node).  This is the lexicographically first MIS of S^2.
 */
void or_mis2(const ocsr *A, const unsigned char *S, uint64_t seed, int level, unsigned char *root)
{
    int n = A->nr;
    kidx *ord = (kidx *)malloc((size_t)n * sizeof(kidx));
    unsigned char *blk = (unsigned char *)calloc((size_t)n, 1);
    for (int i = 0; i < n; ++i) { ord[i].k = or_key(seed, level, i); ord[i].i = i; root[i] = 0; }
    qsort(ord, (size_t)n, sizeof(kidx), kidx_desc);
    for (int t = 0; t < n; ++t) {
        int r = ord[t].i;
        if (blk[r]) continue;
        root[r] = 1;
        blk[r] = 1;
        for (int e = A->rp[r]; e < A->rp[r + 1]; ++e) {
            if (!S[e]) continue;
            int j = A->ci[e];
            blk[j] = 1;
            for (int f = A->rp[j]; f < A->rp[j + 1]; ++f)
                if (S[f]) blk[A->ci[f]] = 1;
        }
    }
    free(ord); free(blk);
}

/*
 * Aggregates from the MIS-2 roots:
 *  1. roots numbered 0..m-1 in ascending node index;
 *  2. every strong neighbour of a root joins that root's aggregate;
 *  3. every node still unassigned joins the aggregate of the step-2 strong
 *     neighbour whose root has the largest (key, root index).
 * Returns m, or -1 if a node stays unassigned (a non-maximal root set).
 */
int or_aggregate(const ocsr *A, const unsigned char *S, const unsigned char *root,
                 uint64_t seed, int level, int *agg)
{
    int n = A->nr, m = 0;
    int *rootof = (int *)malloc((size_t)n * sizeof(int));
    int *agg2 = (int *)malloc((size_t)n * sizeof(int));
    for (int i = 0; i < n; ++i) {
        if (root[i]) { agg2[i] = m++; rootof[i] = i; }
        else { agg2[i] = -1; rootof[i] = -1; }
    }
    for (int i = 0; i < n; ++i) {
        if (root[i]) continue;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (S[e] && j != i && root[j]) {
                agg2[i] = agg2[j];
                rootof[i] = j;
                break;
            }
        }
    }
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        agg[i] = agg2[i];
        if (agg2[i] >= 0) continue;
        int best = -1;
        uint64_t bk = 0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (!S[e] || j == i || agg2[j] < 0) continue;
            int r = rootof[j];
            uint64_t k = or_key(seed, level, r);
            if (best < 0 || k > bk || (k == bk && r > best)) { best = r; bk = k; }
        }
        if (best < 0) { bad = 1; continue; }
        agg[i] = agg2[best];
    }
    free(rootof); free(agg2);
    return bad ? -1 : m;
}

/* ---------------------------------------------------- smoothed prolongator */
/*
 * Filtered matrix A_F: weak off-diagonals dropped and added to the diagonal
 * (a^F_ii = a_ii + sum of weak a_ij in ascending j).  rho = max over rows
 * with a strong neighbour of (sum_j |a^F_ij|, ascending j) / a^F_ii, a
 * Gershgorin bound of D_F^-1 A_F; omega = (4/3)/rho.
 * P = (I - omega D_F^-1 A_F) P_tent with P_tent(i, agg(i)) = 1:
 *   P(i,c) = [c == agg(i)] - s_i * sum_{j in {i} U S(i), agg(j) = c} a^F_ij,
 *   s_i = omega / a^F_ii, sums in ascending j; rows without a strong
 *   neighbour keep their P_tent row.  Columns ascending, no entry dropped.
 */
ocsr *or_smooth_p(const ocsr *A, const unsigned char *S, const int *agg, int nagg,
                  double *omega_out, double *rho_out)
{
    int n = A->nr;
    double *aF = (double *)malloc((size_t)n * sizeof(double));
    unsigned char *hs = (unsigned char *)calloc((size_t)n, 1);
    double rho = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = csr_diag_of(A, i);
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (j == i) continue;
            if (S[e]) hs[i] = 1; else d += A->v[e];
        }
        aF[i] = d;
    }
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) continue;
        double s = 0.0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (j == i) s += fabs(aF[i]);
            else if (S[e]) s += fabs(A->v[e]);
        }
        double ratio = s / aF[i];
        if (ratio > rho) rho = ratio;
    }
    double omega = rho > 0.0 ? (4.0 / 3.0) / rho : 0.0;
    *omega_out = omega;
    if (rho_out) *rho_out = rho;
    /* pattern: sorted unique aggregates of {i} U S(i) */
    int cap = A->nnz + n;
    ocsr *P = csr_new(n, nagg, cap);
    int *cols = (int *)malloc((size_t)(A->nnz + 1) * sizeof(int));
    int e0 = 0;
    for (int i = 0; i < n; ++i) {
        P->rp[i] = e0;
        if (!hs[i]) {
            P->ci[e0] = agg[i]; P->v[e0] = 1.0; ++e0;
            continue;
        }
        int nc = 0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
            int j = A->ci[e];
            if (j != i && !S[e]) continue;
            int c = agg[j], dup = 0;
            for (int t = 0; t < nc; ++t) if (cols[t] == c) { dup = 1; break; }
            if (!dup) cols[nc++] = c;
        }
        /* insertion sort of the (short) column list */
        for (int a = 1; a < nc; ++a) {
            int c = cols[a], t = a - 1;
            while (t >= 0 && cols[t] > c) { cols[t + 1] = cols[t]; --t; }
            cols[t + 1] = c;
        }
        double s = omega / aF[i];
        for (int t = 0; t < nc; ++t) {
            int c = cols[t];
            double acc = 0.0;
            for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) {
                int j = A->ci[e];
                if (j != i && !S[e]) continue;
                if (agg[j] != c) continue;
                acc += (j == i) ? aF[i] : A->v[e];
            }
            double delta = (c == agg[i]) ? 1.0 : 0.0;
            P->ci[e0] = c;
            P->v[e0] = delta - s * acc;
            ++e0;
        }
    }
    P->rp[n] = e0;
    P->nnz = e0;
    free(cols); free(aF); free(hs);
    return P;
}

/* ------------------------------------------------ transpose and SpGEMM -- */
/* R = P^T; each row of R lists its columns (rows of P) in ascending order */
ocsr *or_transpose(const ocsr *P)
{
    ocsr *R = csr_new(P->nc, P->nr, P->nnz);
    for (int e = 0; e < P->nnz; ++e) R->rp[P->ci[e] + 1]++;
    for (int c = 0; c < P->nc; ++c) R->rp[c + 1] += R->rp[c];
    int *pos = (int *)malloc(((size_t)P->nc + 1) * sizeof(int));
    memcpy(pos, R->rp, ((size_t)P->nc + 1) * sizeof(int));
    for (int i = 0; i < P->nr; ++i)
        for (int e = P->rp[i]; e < P->rp[i + 1]; ++e) {
            int c = P->ci[e], t = pos[c]++;
            R->ci[t] = i;
            R->v[t] = P->v[e];
        }
    free(pos);
    return R;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * C = L * Rm in the canonical order: C(i,c) = sum over L's row i in
 * ascending column k of L(i,k) * Rm(k,c), accumulated from 0.0.  The pattern
 * is structural (no numerically-zero entry dropped), columns ascending.
 * Used for A P and for P^T (A P).
 */
ocsr *or_spgemm(const ocsr *L, const ocsr *Rm)
{
    int nr = L->nr, nc = Rm->nc;
    int *mark = (int *)malloc((size_t)nc * sizeof(int));
    double *acc = (double *)malloc((size_t)nc * sizeof(double));
    int *list = (int *)malloc((size_t)nc * sizeof(int));
    for (int c = 0; c < nc; ++c) mark[c] = -1;
    size_t cap = (size_t)L->nnz * 4 + 16, used = 0;
    int *ci = (int *)malloc(cap * sizeof(int));
    double *v = (double *)malloc(cap * sizeof(double));
    int *rp = (int *)malloc(((size_t)nr + 1) * sizeof(int));
    for (int i = 0; i < nr; ++i) {
        int cnt = 0;
        for (int e = L->rp[i]; e < L->rp[i + 1]; ++e) {
            int k = L->ci[e];
            double lv = L->v[e];
            for (int f = Rm->rp[k]; f < Rm->rp[k + 1]; ++f) {
                int c = Rm->ci[f];
                if (mark[c] != i) { mark[c] = i; acc[c] = 0.0; list[cnt++] = c; }
                acc[c] += lv * Rm->v[f];
            }
        }
        qsort(list, (size_t)cnt, sizeof(int), cmp_int);
        if (used + (size_t)cnt > cap) {
            while (used + (size_t)cnt > cap) cap *= 2;
            ci = (int *)realloc(ci, cap * sizeof(int));
            v = (double *)realloc(v, cap * sizeof(double));
        }
        rp[i] = (int)used;
        for (int t = 0; t < cnt; ++t) { ci[used] = list[t]; v[used] = acc[list[t]]; ++used; }
    }
    rp[nr] = (int)used;
    ocsr *C = (ocsr *)calloc(1, sizeof(ocsr));
    C->nr = nr; C->nc = nc; C->nnz = (int)used;
    C->rp = rp; C->ci = ci; C->v = v;
    free(mark); free(acc); free(list);
    return C;
}

/* ------------------------------------------------------------- dense LU -- */
/* Doolittle LU with partial pivoting (first row of largest |a_ik|),
 * row-major, in place; piv[k] is the row swapped with row k. 0 or -1 */
int or_lu_factor(int n, double *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double t = fabs(a[(size_t)i * n + k]);
            if (t > best) { best = t; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        double piv_v = a[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double l = a[(size_t)i * n + k] / piv_v;
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
        }
    }
    return 0;
}

void or_lu_solve(int n, const double *lu, const int *piv, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int k = 0; k < n; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int j = 0; j < i; ++j) s -= lu[(size_t)i * n + j] * x[j];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int j = i + 1; j < n; ++j) s -= lu[(size_t)i * n + j] * x[j];
        x[i] = s / lu[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------ hierarchy -- */
typedef struct {
    int L;
    ocsr *A[OR_MAXL], *P[OR_MAXL], *R[OR_MAXL];
    unsigned char *S[OR_MAXL], *root[OR_MAXL];
    int *agg[OR_MAXL];
    int nagg[OR_MAXL];
    double theta2[OR_MAXL], omegaP[OR_MAXL], rhoP[OR_MAXL];
    double *dinv[OR_MAXL];
    double jw[OR_MAXL], rhoJ[OR_MAXL], lam[OR_MAXL];
    double cheb_c0[OR_MAXL], cheb_c1[OR_MAXL][8], cheb_c2[OR_MAXL][8];
    double *x[OR_MAXL], *b[OR_MAXL], *r[OR_MAXL], *t[OR_MAXL], *d[OR_MAXL];
    int nlu;
    double *lu;
    int *piv;
    int smoother, degree, nu;
    uint64_t seed;
    int status;
} ohier;

int or_h_status(const ohier *H) { return H->status; }
int or_h_nlevels(const ohier *H) { return H->L; }
ocsr *or_h_A(const ohier *H, int l) { return H->A[l]; }
ocsr *or_h_P(const ohier *H, int l) { return l < H->L - 1 ? H->P[l] : NULL; }
ocsr *or_h_R(const ohier *H, int l) { return l < H->L - 1 ? H->R[l] : NULL; }
int or_h_nagg(const ohier *H, int l) { return H->nagg[l]; }

void or_h_copy_level(const ohier *H, int l, int *agg, unsigned char *root, unsigned char *S)
{
    int n = H->A[l]->nr;
    if (agg && H->agg[l]) memcpy(agg, H->agg[l], (size_t)n * sizeof(int));
    if (root && H->root[l]) memcpy(root, H->root[l], (size_t)n);
    if (S && H->S[l]) memcpy(S, H->S[l], (size_t)H->A[l]->nnz);
}

/* out: theta2, omegaP, rhoP, jacobi weight, rhoJ, lambda_hat */
void or_h_scalars(const ohier *H, int l, double *out)
{
    out[0] = H->theta2[l]; out[1] = H->omegaP[l]; out[2] = H->rhoP[l];
    out[3] = H->jw[l]; out[4] = H->rhoJ[l]; out[5] = H->lam[l];
}

void or_h_free(ohier *H)
{
    if (!H) return;
    for (int l = 0; l < OR_MAXL; ++l) {
        or_csr_free(H->A[l]); or_csr_free(H->P[l]); or_csr_free(H->R[l]);
        free(H->S[l]); free(H->root[l]); free(H->agg[l]); free(H->dinv[l]);
        free(H->x[l]); free(H->b[l]); free(H->r[l]); free(H->t[l]); free(H->d[l]);
    }
    free(H->lu); free(H->piv); free(H);
}

/* uniform in [-1, 1) from the counter-based hash, for the power iteration */
static double start_val(uint64_t seed, int l, int i)
{
    uint64_t h = smix(seed ^ ((uint64_t)l << 48) ^ (uint64_t)(uint32_t)i ^ 0x00c0ffee00000000ULL);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* Jacobi data and Chebyshev interval for level l (not bit-compared) */
static void smoother_setup(ohier *H, int l)
{
    ocsr *A = H->A[l];
    int n = A->nr;
    H->dinv[l] = (double *)malloc((size_t)n * sizeof(double));
    double rho = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = csr_diag_of(A, i), s = 0.0;
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) s += fabs(A->v[e]);
        H->dinv[l][i] = 1.0 / d;
        double ratio = s / d;
        if (ratio > rho) rho = ratio;
    }
    H->rhoJ[l] = rho;
    H->jw[l] = (4.0 / 3.0) / rho;
    /* lambda_max(D^-1 A): 10 power iterations from a hashed start vector */
    double *v = (double *)malloc((size_t)n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) v[i] = start_val(H->seed, l, i);
    double nv = sqrt(dot(n, v, v));
    for (int i = 0; i < n; ++i) v[i] /= nv;
    double lam = 0.0;
    for (int it = 0; it < 10; ++it) {
        csr_spmv(A, v, w);
        for (int i = 0; i < n; ++i) w[i] *= H->dinv[l][i];
        lam = sqrt(dot(n, w, w));
        for (int i = 0; i < n; ++i) v[i] = w[i] / lam;
    }
    free(v); free(w);
    H->lam[l] = lam;
    /* Chebyshev on [lam/30, 1.1 lam] */
    double a = lam / 30.0, bb = 1.1 * lam;
    double theta = (bb + a) / 2.0, delta = (bb - a) / 2.0, sigma = theta / delta;
    double rho_c = 1.0 / sigma;
    H->cheb_c0[l] = 1.0 / theta;
    for (int k = 1; k < H->degree && k < 8; ++k) {
        double rn = 1.0 / (2.0 * sigma - rho_c);
        H->cheb_c1[l][k] = rn * rho_c;
        H->cheb_c2[l][k] = 2.0 * rn / delta;
        rho_c = rn;
    }
}

/*
 * Smoothed-aggregation setup.  Levels are added while the level has more
 * than n_coarse unknowns and fewer than max_levels levels exist; a level
 * whose aggregation keeps more than 0.9 of its unknowns (or finds none)
 * becomes the coarsest.  theta halves per level.  The coarsest level
 * (at most 4096 unknowns) is factored by dense LU.
 */
ohier *or_setup(const ocsr *A0, double theta0, int smoother, int degree, int nu,
                int n_coarse, int max_levels, uint64_t seed)
{
    ohier *H = (ohier *)calloc(1, sizeof(ohier));
    H->smoother = smoother; H->degree = degree < 1 ? 1 : degree; H->nu = nu < 1 ? 1 : nu;
    H->seed = seed;
    if (max_levels > OR_MAXL) max_levels = OR_MAXL;
    if (max_levels < 1) max_levels = 1;
    H->A[0] = or_csr_from(A0->nr, A0->nc, A0->rp, A0->ci, A0->v);
    int l = 0;
    double th = theta0;
    for (;;) {
        ocsr *A = H->A[l];
        int n = A->nr;
        H->theta2[l] = th * th;
        if (n <= n_coarse || l + 1 >= max_levels) break;
        H->S[l] = (unsigned char *)malloc((size_t)A->nnz + 1);
        or_strength(A, H->theta2[l], H->S[l]);
        H->root[l] = (unsigned char *)malloc((size_t)n);
        or_mis2(A, H->S[l], seed, l, H->root[l]);
        H->agg[l] = (int *)malloc((size_t)n * sizeof(int));
        int m = or_aggregate(A, H->S[l], H->root[l], seed, l, H->agg[l]);
        if (m < 0) { H->status = OR_ERR_SETUP; H->L = l + 1; return H; }
        H->nagg[l] = m;
        if (m == 0 || (double)m > 0.9 * (double)n) break;
        H->P[l] = or_smooth_p(A, H->S[l], H->agg[l], m, &H->omegaP[l], &H->rhoP[l]);
        H->R[l] = or_transpose(H->P[l]);
        ocsr *AP = or_spgemm(A, H->P[l]);
        H->A[l + 1] = or_spgemm(H->R[l], AP);
        or_csr_free(AP);
        ++l;
        th = th * 0.5;
    }
    H->L = l + 1;
    for (int k = 0; k < H->L; ++k) {
        int n = H->A[k]->nr;
        H->x[k] = (double *)calloc((size_t)n, sizeof(double));
        H->b[k] = (double *)calloc((size_t)n, sizeof(double));
        H->r[k] = (double *)calloc((size_t)n, sizeof(double));
        H->t[k] = (double *)calloc((size_t)n, sizeof(double));
        H->d[k] = (double *)calloc((size_t)n, sizeof(double));
        if (k < H->L - 1) smoother_setup(H, k);
    }
    ocsr *Ac = H->A[H->L - 1];
    int nc = Ac->nr;
    if (nc > 4096) { H->status = OR_ERR_SETUP; return H; }
    H->nlu = nc;
    H->lu = (double *)calloc((size_t)nc * nc, sizeof(double));
    H->piv = (int *)malloc((size_t)nc * sizeof(int));
    for (int i = 0; i < nc; ++i)
        for (int e = Ac->rp[i]; e < Ac->rp[i + 1]; ++e) H->lu[(size_t)i * nc + Ac->ci[e]] = Ac->v[e];
    if (or_lu_factor(nc, H->lu, H->piv) != 0) H->status = OR_ERR_SETUP;
    return H;
}

/* ------------------------------------------------------------- V-cycle -- */
/* one smoothing application on level l: x <- S(x) for A x = b.  x0zero says
 * x enters as zero (no residual product needed for the first step). */
static void smooth(ohier *H, int l, const double *b, double *x, int x0zero)
{
    ocsr *A = H->A[l];
    int n = A->nr;
    double *r = H->r[l], *d = H->d[l], *t = H->t[l], *dinv = H->dinv[l];
    if (H->smoother == 0) {
        for (int s = 0; s < H->nu; ++s) {
            if (x0zero && s == 0) {
                for (int i = 0; i < n; ++i) x[i] = H->jw[l] * (dinv[i] * b[i]);
                continue;
            }
            csr_spmv(A, x, t);
            for (int i = 0; i < n; ++i) x[i] = x[i] + H->jw[l] * (dinv[i] * (b[i] - t[i]));
        }
        return;
    }
    for (int s = 0; s < H->nu; ++s) {
        if (x0zero && s == 0) {
            for (int i = 0; i < n; ++i) r[i] = b[i];
        } else {
            csr_spmv(A, x, t);
            for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
        }
        for (int i = 0; i < n; ++i) d[i] = H->cheb_c0[l] * (dinv[i] * r[i]);
        for (int k = 1; k <= H->degree; ++k) {
            for (int i = 0; i < n; ++i) x[i] = x[i] + d[i];
            if (k == H->degree) break;
            csr_spmv(A, d, t);
            for (int i = 0; i < n; ++i) r[i] = r[i] - t[i];
            for (int i = 0; i < n; ++i)
                d[i] = H->cheb_c1[l][k] * d[i] + H->cheb_c2[l][k] * (dinv[i] * r[i]);
        }
    }
}

static void vcycle(ohier *H, int l, const double *b, double *x)
{
    if (l == H->L - 1) { or_lu_solve(H->nlu, H->lu, H->piv, b, x); return; }
    ocsr *A = H->A[l];
    int n = A->nr;
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    smooth(H, l, b, x, 1);
    double *r = H->r[l], *t = H->t[l];
    csr_spmv(A, x, t);
    for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    double *bc = H->b[l + 1], *xc = H->x[l + 1];
    csr_spmv(H->R[l], r, bc);
    vcycle(H, l + 1, bc, xc);
    csr_spmv(H->P[l], xc, t);
    for (int i = 0; i < n; ++i) x[i] = x[i] + t[i];
    smooth(H, l, b, x, 0);
}

/* one smoothing application on level l (x0zero: x enters as zero) */
void or_h_smooth(ohier *H, int l, const double *b, double *x, int x0zero)
{
    if (l < 0 || l >= H->L - 1) return;
    smooth(H, l, b, x, x0zero);
}

/* z = M^-1 r with one V-cycle from a zero initial guess */
void or_vcycle(ohier *H, const double *r, double *z) { vcycle(H, 0, r, z); }

/*
 * Preconditioned CG (Saad, Algorithm 9.1) from x0 = 0 on A = level-0 matrix.
 * Stops when the TRUE relative residual ||b - A x||_2 / ||b||_2 <= tol: when
 * the recursive residual passes the test the true one is computed; if it
 * fails, it replaces the recursive residual and the iteration continues.
 * Returns 0, OR_ERR_NOT_CONVERGED (x = last iterate) or OR_ERR_BREAKDOWN.
 */
int or_pcg(ohier *H, const double *b, double *x, double tol, int maxit, int *iters, double *relres)
{
    ocsr *A = H->A[0];
    int n = A->nr;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    int st = OR_ERR_NOT_CONVERGED, it = 0;
    double bn = sqrt(dot(n, b, b)), rel = 0.0;
    for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    if (bn == 0.0) { st = OR_OK; goto done; }
    or_vcycle(H, r, z);
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    rel = 1.0;
    while (it < maxit) {
        ++it;
        csr_spmv(A, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { st = OR_ERR_BREAKDOWN; break; }
        double alpha = rz / pq;
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rn = sqrt(dot(n, r, r));
        if (!isfinite(rn)) { st = OR_ERR_BREAKDOWN; break; }
        if (rn <= tol * bn) {
            csr_spmv(A, x, q);
            for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
            double tn = sqrt(dot(n, r, r));
            rel = tn / bn;
            if (tn <= tol * bn) { st = OR_OK; break; }
        }
        or_vcycle(H, r, z);
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (st != OR_OK) {
        csr_spmv(A, x, q);
        for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
        rel = sqrt(dot(n, r, r)) / bn;
    }
done:
    *iters = it;
    *relres = rel;
    free(r); free(z); free(p); free(q);
    return st;
}

/* plain CG without preconditioner, for tests of the preconditioner's effect */
int or_cg_plain(const ocsr *A, const double *b, double *x, double tol, int maxit, int *iters, double *relres)
{
    int n = A->nr;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; }
    double bn = sqrt(dot(n, b, b)), rr = dot(n, r, r);
    int it = 0, st = OR_ERR_NOT_CONVERGED;
    while (it < maxit && sqrt(rr) > tol * bn) {
        ++it;
        csr_spmv(A, p, q);
        double alpha = rr / dot(n, p, q);
        for (int i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        double rr2 = dot(n, r, r);
        double beta = rr2 / rr;
        rr = rr2;
        for (int i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    if (sqrt(rr) <= tol * bn) st = OR_OK;
    csr_spmv(A, x, q);
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
    *iters = it;
    *relres = bn > 0.0 ? sqrt(dot(n, r, r)) / bn : 0.0;
    free(r); free(p); free(q);
    return st;
}

/* ------------------------------------------------------------- adjoint -- */
/*
 * Gradient of an objective J(h) with respect to ln K (K scaling Kx, Ky, Kz of
 * a cell together), given the heads h of C h = Q and the adjoint state
 * lambda of C lambda = dJ/dh (C is symmetric, so the same operator serves).
 * Differentiating C(K) h = Q(K):
 *   dJ/dlnK_i = lambda^T (dQ/dlnK_i - dC/dlnK_i h).
 * An interior face between i and j with T = 2 K_i K_j/(K_i + K_j) g has
 * dT/dlnK_i = T K_j/(K_i + K_j) and enters rows i and j as T (h_i - h_j) and
 * T (h_j - h_i), giving -dT/dlnK_i (h_i - h_j)(lambda_i - lambda_j); a
 * Dirichlet face with T_b = 2 K_i g enters row i as T_b (h_i - h_b), giving
 * -T_b (h_i - h_b) lambda_i.  Faces are visited in the order -x,+x,-y,+y,-z,+z.
 */
void or_adjoint_grad(int nx, int ny, int nz, double dx, double dy, double dz, const double *Kx, const double *Ky,
                     const double *Kz, const int *bct, const double *bcv, const double *h, const double *lam,
                     double *grad)
{
    const double g[3] = {(dy * dz) / dx, (dx * dz) / dy, (dx * dy) / dz};
    const double *K[3] = {Kx, Ky, Kz};
    const int dim[3] = {nx, ny, nz};
    const int stride[3] = {1, nx, nx * ny};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int i = x + nx * (y + ny * z);
                int crd[3] = {x, y, z};
                double s = 0.0;
                for (int d = 0; d < 3; ++d)
                    for (int side = 0; side < 2; ++side) {
                        int f = 2 * d + side;
                        int interior = side == 0 ? crd[d] > 0 : crd[d] < dim[d] - 1;
                        if (interior) {
                            int j = side == 0 ? i - stride[d] : i + stride[d];
                            int lo = i < j ? i : j, hi = i < j ? j : i;
                            double T = harm(K[d][lo], K[d][hi]) * g[d];
                            double c = T * (K[d][j] / (K[d][i] + K[d][j]));
                            s += c * (h[i] - h[j]) * (lam[i] - lam[j]);
                        } else if (bct[f] == OR_DIRICHLET) {
                            double Tb = (2.0 * K[d][i]) * g[d];
                            s += Tb * (h[i] - bcv[f]) * lam[i];
                        }
                    }
                grad[i] = -s;
            }
}

/* J = sum_k (h[obs_k] - hobs_k)^2 and its gradient dJ/dh (zero off the
 * observation cells) */
double or_misfit(int n, const double *h, int nobs, const int *obs, const double *hobs, double *dJdh)
{
    double J = 0.0;
    if (dJdh)
        for (int i = 0; i < n; ++i) dJdh[i] = 0.0;
    for (int k = 0; k < nobs; ++k) {
        double r = h[obs[k]] - hobs[k];
        J += r * r;
        if (dJdh) dJdh[obs[k]] += 2.0 * r;
    }
    return J;
}

/* ---------------------------------------------------- transient shift -- */
/* C + diag(s): the implicit transient operator of Eq. 2, s_i = S_i V_i / dt */
ocsr *or_shift_csr(const ocsr *C, const double *s)
{
    ocsr *A = or_csr_from(C->nr, C->nc, C->rp, C->ci, C->v);
    for (int i = 0; i < A->nr; ++i)
        for (int e = A->rp[i]; e < A->rp[i + 1]; ++e)
            if (A->ci[e] == i) A->v[e] = A->v[e] + s[i];
    return A;
}

/* The cached hierarchy stays valid while the diagonal moved by less than
 * delta C_ii in every row: |s_i - s_built_i| < delta * C_ii (s_built = 0 gives
 * the criterion S_i V_i / dt < delta C_ii of the Discussion section). */
int or_reuse_ok(const ocsr *C, const double *s, const double *s_built, double delta)
{
    for (int i = 0; i < C->nr; ++i) {
        double cii = csr_diag_of(C, i);
        double ds = s[i] - (s_built ? s_built[i] : 0.0);
        if (!(fabs(ds) < delta * cii)) return 0;
    }
    return 1;
}

/* keep the coarse levels, replace the level-0 operator and redo its smoother data */
void or_h_refresh_level0(ohier *H, const ocsr *A)
{
    or_csr_free(H->A[0]);
    H->A[0] = or_csr_from(A->nr, A->nc, A->rp, A->ci, A->v);
    free(H->dinv[0]);
    H->dinv[0] = NULL;
    if (H->L > 1) smoother_setup(H, 0);
}

/*
 * Numeric refresh of a cached hierarchy (Discussion: the preconditioner is
 * reused while the storage term changes little): level 0 becomes A (C plus
 * the storage diagonal, the same pattern), the aggregates and the smoothed
 * prolongators P_l are kept, and every coarse operator is formed again by
 * its Galerkin definition A_{l+1} = P_l^T (A_l P_l) from the new A_l; then
 * the smoother data of every level and the coarsest LU are redone.  The
 * pattern of each A_{l+1} does not change (A_l + diag keeps the pattern of
 * A_l, whose diagonal is structural), so only values are replaced.
 */
void or_h_refresh_numeric(ohier *H, const ocsr *A)
{
    or_csr_free(H->A[0]);
    H->A[0] = or_csr_from(A->nr, A->nc, A->rp, A->ci, A->v);
    for (int l = 0; l + 1 < H->L; ++l) {
        ocsr *AP = or_spgemm(H->A[l], H->P[l]);
        ocsr *Ac = or_spgemm(H->R[l], AP);
        or_csr_free(AP);
        or_csr_free(H->A[l + 1]);
        H->A[l + 1] = Ac;
    }
    for (int k = 0; k + 1 < H->L; ++k) {
        free(H->dinv[k]);
        H->dinv[k] = NULL;
        smoother_setup(H, k);
    }
    ocsr *Ac = H->A[H->L - 1];
    int nc = Ac->nr;
    for (size_t i = 0; i < (size_t)nc * nc; ++i) H->lu[i] = 0.0;
    for (int i = 0; i < nc; ++i)
        for (int e = Ac->rp[i]; e < Ac->rp[i + 1]; ++e) H->lu[(size_t)i * nc + Ac->ci[e]] = Ac->v[e];
    if (or_lu_factor(nc, H->lu, H->piv) != 0) H->status = OR_ERR_SETUP;
}

/* ---------------------------------------------------- Darcy face fluxes -- */
/*
 * Darcy velocity on every face of the grid (staggered layout): vx has
 * (nx+1)*ny*nz entries, face xf = 0..nx of row (y, z) at xf + (nx+1)(y + ny z);
 * likewise vy ((ny+1) faces per column) and vz.  Positive along +x (+y, +z).
 * Interior face between cells a (lower) and b: T (h_a - h_b) / A_f with T the
 * face transmissibility of the assembly and A_f the face area; a Dirichlet
 * boundary face uses T_b and the face head; a no-flow face carries 0.
 * The velocities feed the advective transport problem (Eq. 1).
 */
void or_darcy_flux(int nx, int ny, int nz, double dx, double dy, double dz, const double *Kx, const double *Ky,
                   const double *Kz, const int *bct, const double *bcv, const double *h, double *vx, double *vy,
                   double *vz)
{
    const double g[3] = {(dy * dz) / dx, (dx * dz) / dy, (dx * dy) / dz};
    const double area[3] = {dy * dz, dx * dz, dx * dy};
    const double *K[3] = {Kx, Ky, Kz};
    const int dim[3] = {nx, ny, nz};
    double *v[3] = {vx, vy, vz};
    for (int d = 0; d < 3; ++d) {
        int fd[3] = {nx, ny, nz};
        fd[d] += 1;
        for (int z = 0; z < fd[2]; ++z)
            for (int y = 0; y < fd[1]; ++y)
                for (int x = 0; x < fd[0]; ++x) {
                    int c[3] = {x, y, z};
                    int f = c[d];
                    double out;
                    /* cells on either side */
                    int ca[3] = {x, y, z}, cb[3] = {x, y, z};
                    ca[d] = f - 1;
                    cb[d] = f;
                    int ia = ca[0] + nx * (ca[1] + ny * ca[2]);
                    int ib = cb[0] + nx * (cb[1] + ny * cb[2]);
                    if (f > 0 && f < dim[d]) {
                        double T = harm(K[d][ia], K[d][ib]) * g[d];
                        out = T * (h[ia] - h[ib]) / area[d];
                    } else if (f == 0) {
                        out = bct[2 * d] == OR_DIRICHLET ? (2.0 * K[d][ib]) * g[d] * (bcv[2 * d] - h[ib]) / area[d]
                                                         : 0.0;
                    } else {
                        out = bct[2 * d + 1] == OR_DIRICHLET
                                  ? (2.0 * K[d][ia]) * g[d] * (h[ia] - bcv[2 * d + 1]) / area[d]
                                  : 0.0;
                    }
                    v[d][x + fd[0] * (y + fd[1] * z)] = out;
                }
    }
}
