/*
 * gw.h -- C ABI of the GB300-native AMG-preconditioned CG solver for steady
 * groundwater flow (libgw.so, CUDA for sm_103a).
 *
 * The library solves C h = Q, the steady confined flow system (Sbai &
 * Larabi, Eq. 2 with zero storage), where C is the global conductance matrix
 * of a cell-centred 5/7-point finite-volume discretisation (an M-matrix;
 * Benchmarking Examples section) and Q holds the sources and the boundary
 * contributions.  The solver is conjugate gradients preconditioned by one
 * smoothed-aggregation algebraic-multigrid V-cycle per iteration
 * (Introduction: setup phase, V-cycle, AMG as a Krylov preconditioner).  The
 * hierarchy is built once and reused across right-hand sides, as the dual
 * delineation approach reuses one matrix for many solves (Introduction).
 * The ABI is plain C so that any language with a C foreign-function interface
 * (the paper names Fortran's iso_c_binding) can call it.
 *
 * Conventions for every entry point:
 *  - Return value: a gw_status (GW_OK = 0).  No call aborts and no C++
 *    exception crosses the ABI.  gw_last_error() gives a one-line reason for
 *    the last failure on the calling thread.
 *  - Arrays are plain pointers.  Unless stated otherwise an array may be in
 *    host memory or in device memory of the current CUDA device; the library
 *    looks the pointer up and copies host arrays in and out itself.  Arrays
 *    stay owned by the caller; handles own their device memory until freed.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it.  Calls that return host-visible
 *    results (gw_amg_setup, gw_pcg_solve, gw_hierarchy_info) synchronise it.
 *  - Cells are numbered i = x + nx*(y + ny*z); fields are nx*ny*nz doubles.
 *  - Everything runs on the GPU in hand-written kernels; there is no CPU
 *    fallback.  One GPU per handle: the device current at creation.
 *  - Results are bitwise reproducible run to run for the same inputs.
 */
#ifndef GW_H
#define GW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GW_OK = 0,
    GW_ERR_ARG = 1,           /* null pointer, bad size, K <= 0 or not finite, no Dirichlet face */
    GW_ERR_CUDA = 2,          /* a CUDA call failed (see gw_last_error) */
    GW_ERR_OOM = 3,           /* device allocation failed */
    GW_ERR_SETUP = 4,         /* setup could not build a hierarchy (round cap, coarsest level too big) */
    GW_ERR_NOT_CONVERGED = 5, /* maxit reached: h holds the last iterate, relres is set */
    GW_ERR_BREAKDOWN = 6      /* p^T A p <= 0 or a non-finite scalar in CG */
} gw_status;

/* Regular grid of nx*ny*nz cells of size dx*dy*dz; nz = 1 gives the 2D
 * 5-point operator. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
} gw_grid;

enum { GW_NOFLOW = 0, GW_DIRICHLET = 1 };

/* Boundary condition of the six domain faces in the order -x,+x,-y,+y,-z,+z:
 * GW_NOFLOW (zero flux) or GW_DIRICHLET (head value[f] on the face). */
typedef struct {
    int type[6];
    double value[6];
} gw_bc;

/* Arithmetic of the solve.  The coarsest level always uses the FP64 dense
 * inverse and dot products are always summed in FP64 across threads.
 * GW_PREC_FP64: the hierarchy, the V-cycle and every CG vector in FP64.
 * GW_PREC_MIXED32: the hierarchy and V-cycle in FP32, the CG recurrence in
 * FP32 against the FP32 level-0 operator, and the solution in FP64 by
 * reliable updates: when the FP32 residual has fallen by the factor delta
 * since the last update, or passes the stopping test, the FP32 correction is
 * added to the FP64 solution and the residual is recomputed as b - A h with
 * the FP64 operator in FP64 arithmetic; the solve stops only on that FP64
 * residual. */
typedef enum {
    GW_PREC_FP64 = 0,
    GW_PREC_MIXED32 = 1,
    GW_PREC_MIXED16 = 2,   /* GW_PREC_MIXED32 with GW_HALF_FINE16: FP16-stored scaled fine stencil */
    GW_PREC_MIXEDBF16 = 3  /* GW_PREC_MIXED32 with GW_HALF_FINE: BF16-stored fine stencil */
} gw_prec;

enum { GW_SMOOTH_JACOBI = 0, GW_SMOOTH_CHEBYSHEV = 1 };

/* Bits of gw_amg_opts.half_storage. */
enum { GW_HALF_FINE = 2, GW_HALF_FINE16 = 4 };

/* Setup and cycle options (gw_amg_opts_default fills the defaults). */
typedef struct {
    double theta;        /* strength threshold on level 0, halved per level (0.04) */
    int smoother;        /* GW_SMOOTH_CHEBYSHEV (default) or GW_SMOOTH_JACOBI (weight 4/3 over the Gershgorin bound) */
    int degree;          /* Chebyshev degree (2) */
    int nu;              /* pre- and post-smoothing applications per level (1) */
    int n_coarse;        /* stop coarsening at this many unknowns or fewer (1024) */
    int max_levels;      /* at most this many levels (12) */
    uint64_t seed;       /* seed of the MIS-2 priorities (0x5EED) */
    int prec;            /* gw_prec (GW_PREC_MIXED32) */
    double delta;        /* mixed form: reliable update when the FP32 residual fell by this factor (0.1) */
    int half_storage;    /* mixed form, bit mask (0):
                            GW_HALF_FINE: the V-cycle's level-0 stencil with BF16 couplings and an
                              FP32 diagonal corrected so that rows keep their sums (CG's own
                              products stay FP32);
                            GW_HALF_FINE16: the level-0 stencil scaled to D^-1/2 A D^-1/2, its
                              couplings in FP16, sqrt(a_ii) in FP32 and the unit diagonal's
                              row-sum correction in FP16 (not together with GW_HALF_FINE) */
    int mis_max_rounds;  /* parallel MIS-2 rounds allowed per level before the setup fails with
                            GW_ERR_SETUP (200; 0 means the default) */
} gw_amg_opts;

/* Per-level statistics in the columns of the paper's Table 1 (unknowns,
 * nonzeros, memory) plus what the GPU hierarchy adds. */
typedef struct {
    int n;                  /* unknowns */
    long long nnz;          /* structural nonzeros of A_l */
    long long nnz_p;        /* nonzeros of P_l (0 on the coarsest level) */
    long long bytes;        /* device bytes held for this level */
    int naggregates;        /* aggregates formed from this level (0 on the coarsest) */
    int mis_rounds;         /* parallel MIS-2 rounds used on this level */
    double omega_p;         /* prolongator smoothing weight (4/3)/rho_F */
    double jacobi_w;        /* Jacobi weight (4/3)/rho_Gershgorin(D^-1 A) */
    double lambda_max;      /* power-iteration estimate of lambda_max(D^-1 A) */
} gw_level_info;

typedef struct gw_matrix_s *gw_matrix;
typedef struct gw_hierarchy_s *gw_hierarchy;
typedef struct gw_batch_s *gw_batch;

/* Fills *opts with the defaults listed in gw_amg_opts. */
void gw_amg_opts_default(gw_amg_opts *opts);

/*
 * gw_assemble -- build C and Q (Eq. 2 with S = 0; 5/7-point finite volumes,
 * Benchmarking Examples section).  For an interior face between cells i < j
 * along axis d the transmissibility is T = (2 K_i K_j)/(K_i + K_j) * g_d with
 * g_x = dy dz / dx (and likewise for y, z) and K the conductivity along d;
 * a Dirichlet face of cell i has T_b = 2 K_i g_d (head at the face, half a
 * cell away).  Row i: a_ii = sum of T over the faces of i in the order
 * -x,+x,-y,+y,-z,+z, a_ij = -T, b_i = q_i + sum over its Dirichlet faces of
 * T_b h_b.  A is symmetric bitwise.
 *   grid, bc          host structs.
 *   Kx, Ky, Kz        conductivities, n doubles each (host or device); Ky and
 *                     Kz may be equal to Kx.
 *   q                 source per cell (n doubles, host or device) or NULL.
 *   A_out             receives a new matrix handle (CSR, FP64, columns
 *                     ascending; nnz = 7n - 2(ny nz + nx nz + nx ny) in 3D).
 *   b_out             n doubles (host or device), receives Q.
 * Errors: GW_ERR_ARG for a null pointer, a non-positive size or spacing, a
 * K <= 0 or non-finite value, a non-finite q or head, or no Dirichlet face
 * (the system would be singular).  Checked on the device before any output
 * is written; b_out is untouched on error.
 */
int gw_assemble(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz, const gw_bc *bc,
                const double *q, gw_matrix *A_out, double *b_out, void *stream);

/*
 * gw_assemble_noalloc -- the same assembly as gw_assemble (the same matrix
 * and right-hand side, double for double), for callers that cannot allocate
 * device memory at this point: the caller passes the output CSR arrays and
 * the library allocates nothing.  The paper has no counterpart; this entry
 * point exists for such callers only.
 *   Kx, Ky, Kz, q     as in gw_assemble, but device memory only (Ky, Kz may be
 *                     NULL or equal to Kx; q may be NULL).
 *   rowptr            n+1 ints, device: receives the row pointers.
 *   col, val          device arrays of at least 7n - 2(ny nz + nx nz + nx ny)
 *                     ints / doubles: receive columns (ascending) and values.
 *   b                 n doubles, device: receives Q.
 * Working memory: a fixed array of about 256 KB in device memory that the
 * library holds on every GPU that loads it, until the process exits; grids
 * of more than 2^27 cells are rejected with GW_ERR_ARG.  The first call on a
 * device looks up that array's device address.  Every call synchronises its
 * stream (it reads a validation flag back), so no call may be made on a
 * stream that is being captured: such a call returns GW_ERR_ARG.  With
 * stream NULL the call runs on the legacy default stream, which
 * synchronises with other blocking streams; pass a non-default stream when
 * other threads capture graphs.  All calls on a device share the array (the
 * call clears the part that must start at zero): calls that overlap on the
 * GPU race, so serialise them (one stream, or wait for the previous call,
 * which synchronises its stream before returning).
 * Errors: as gw_assemble, plus GW_ERR_ARG for a host pointer or a capturing
 * stream.
 */
int gw_assemble_noalloc(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz, const gw_bc *bc,
                        const double *q, int *rowptr, int *col, double *val, double *b, void *stream);

/*
 * gw_adjoint_gradient -- the face-flux product of the adjoint method: the
 * gradient of an objective J(h) with respect to ln K per cell (ln K scaling
 * Kx, Ky, Kz of the cell together), given the heads h of C h = Q and the
 * adjoint state lambda solving C lambda = dJ/dh (C is symmetric, so
 * gw_pcg_solve on the same hierarchy gives lambda).  Differentiating the
 * assembly of gw_assemble: an interior face with T = 2 K_i K_j/(K_i+K_j) g
 * contributes -T K_j/(K_i+K_j) (h_i - h_j)(lambda_i - lambda_j) to cell i, a
 * Dirichlet face with T_b = 2 K_i g contributes -T_b (h_i - h_b) lambda_i.
 * The paper's method does not need gradients; this serves sensitivity
 * analysis, which the paper names as the use of fast flow solves (Abstract).
 *   grid, Kx, Ky, Kz, bc  as passed to gw_assemble (arrays in device memory).
 *   h, lambda             n doubles, device.
 *   grad                  n doubles, device: receives dJ/dlnK.
 * Asynchronous on stream.  Errors: GW_ERR_ARG.
 */
int gw_adjoint_gradient(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz, const gw_bc *bc,
                        const double *h, const double *lambda, double *grad, void *stream);

/*
 * gw_misfit -- the head-misfit objective J = sum_k (h[obs_k] - hobs_k)^2 over
 * observation cells and, if dJdh is not NULL, its gradient dJ/dh (n doubles,
 * device; zero off the observation cells, repeated cells add up).  h, obs
 * (nobs ints), hobs (nobs doubles) in device memory; J is one double, host or
 * device.  Synchronises the stream.
 */
int gw_misfit(int n, const double *h, int nobs, const int *obs, const double *hobs, double *J, double *dJdh,
              void *stream);

/* Size of the matrix behind a handle. */
int gw_matrix_size(gw_matrix A, int *n, long long *nnz);

/* Copies the CSR arrays of A (rowptr n+1 ints, col nnz ints, val nnz doubles;
 * host or device; any may be NULL). */
int gw_matrix_export(gw_matrix A, int *rowptr, int *col, double *val, void *stream);

/*
 * gw_amg_setup -- the AMG setup phase (Introduction): strength graph,
 * deterministic parallel MIS-2 aggregation with hashed seeded priorities,
 * tentative prolongator, one damped-Jacobi smoothing of it, Galerkin coarse
 * operators A_{l+1} = P^T A_l P by a two-pass SpGEMM, and a dense inverse of
 * the (SPD) coarsest level by block Gauss-Jordan elimination without
 * pivoting; then the V-cycle storage in the chosen precision.  All of it
 * runs in CUDA kernels.  The aggregates and the P and A_{l+1} patterns and
 * values are the same as a serial FP64 implementation that sums in the
 * stated order (no fused multiply-add in these stages).
 * Environment, read once per process, for checks and tests: GW_VALIDATE=1
 * adds index validation of every level after the setup (GW_ERR_SETUP on a
 * bad index); GW_SETUP_FORMS=thread|warp forces one of the two row-parallel
 * forms of the SpGEMM and prolongator passes (the library otherwise picks
 * one per product; both give the same bits).
 *   A     assembled matrix; the hierarchy keeps a reference to it (freeing A
 *         before H is the caller's error).
 *   opts  host struct or NULL for the defaults.
 * Errors: GW_ERR_ARG (bad option), GW_ERR_OOM, GW_ERR_SETUP (MIS-2 round cap
 * reached, a node left unaggregated, coarsest level above 4096 unknowns or
 * with a pivot that is not positive), GW_ERR_CUDA.
 */
int gw_amg_setup(gw_matrix A, const gw_amg_opts *opts, gw_hierarchy *H_out, void *stream);

/*
 * gw_pcg_solve -- AMG-preconditioned conjugate gradients from h0 = 0
 * (Saad, Algorithm 9.1; AMG as a preconditioner, Introduction).  Stops when
 * the TRUE relative residual ||b - A h||_2 / ||b||_2 <= tol: when the
 * recursive residual passes the test the true one is computed in FP64 and,
 * if it fails, replaces the recursive residual.
 *   b       n doubles (host or device), right-hand side.
 *   h       n doubles (host or device), receives the heads.
 *   tol     > 0; maxit >= 1.
 *   iters   host int or NULL: iterations done.
 *   relres  host double or NULL: final true relative residual.
 * Returns GW_OK, GW_ERR_NOT_CONVERGED (h = last iterate), GW_ERR_BREAKDOWN,
 * GW_ERR_ARG or GW_ERR_CUDA.  Synchronises the stream.  Concurrent solves on
 * one hierarchy must be serialised by the caller (the hierarchy holds the
 * work vectors).
 */
int gw_pcg_solve(gw_hierarchy H, const double *b, double *h, double tol, int maxit, int *iters,
                 double *relres, void *stream);

/*
 * gw_hierarchy_shift -- the implicit transient form (Eq. 2): the hierarchy
 * set up from C now solves (C + diag(s)) h = b, s_i = S_i V_i / dt (s NULL:
 * back to C).  The cached aggregates and prolongators are reused while the
 * diagonal moved by less than delta C_ii in every row since they were built,
 * |s_i - s_built_i| < delta C_ii, the criterion of the Discussion section with
 * delta about 0.01.  Reused, the coarse operators formed with an earlier
 * shift s_ref are kept when every |s_i - s_ref_i| <= s_ref_i / 4 (their
 * storage part P^T diag(s) P then stays within a factor 3/4 to 5/4 of the one
 * they hold): only level 0 is refreshed and *rebuilt = 0.  Otherwise every
 * coarse operator is formed again as P^T A P of the shifted level above on the
 * kept prolongators (the same values as a setup would compute on those
 * prolongators), with its smoother data and the coarsest inverse, and
 * *rebuilt = 2.  When the criterion fails the whole hierarchy is set up again
 * for C + diag(s) and *rebuilt = 1.
 *   s       n doubles (host or device), s_i >= 0, or NULL.
 *   delta   in (0, 1).
 * Synchronises the stream.  Errors: GW_ERR_ARG, GW_ERR_OOM, GW_ERR_SETUP,
 * GW_ERR_CUDA (the hierarchy keeps its previous state on an error).
 */
int gw_hierarchy_shift(gw_hierarchy H, const double *s, double delta, int *rebuilt, void *stream);

/*
 * gw_hierarchy_prepare -- capture the CUDA graphs of gw_pcg_solve now; the
 * first solve does it otherwise.  Later solves only replay them.  A capture
 * is invalidated when another thread meanwhile starts work that synchronises
 * the device (cudaMalloc or cudaFree by other libraries, a kernel module
 * loaded on first use); a multi-threaded caller that runs such work
 * concurrently calls this while it holds that work off.  The library's own
 * allocations already wait for its captures.  Errors: GW_ERR_ARG,
 * GW_ERR_CUDA.
 */
int gw_hierarchy_prepare(gw_hierarchy H);

/*
 * gw_pcg_solve_many -- k right-hand sides on one hierarchy.  Systems that
 * share a matrix reuse its factorisation or preconditioner (Introduction,
 * on the dual delineation approach); here the shared matrix is the flow
 * operator C, e.g. well or boundary scenarios, or forward and adjoint
 * solves.  B and X are n x k, column-major
 * (column c at B + c*n), host or device; iters and relres receive k values
 * (host, may be NULL).  In the mixed form k >= 2
 * columns run in interleaved blocks of up to 8 that share every matrix read
 * of the V-cycle and of CG, each column with its own CG scalars, reliable
 * updates and stop; otherwise the columns are solved one after another.
 * Each column is solved to the true relative residual tol; the first call
 * of a block width captures its graphs and allocates its working vectors
 * (about 70 bytes per cell and column at width 8).  Returns GW_OK, or the
 * first failing status with every column solved as far as it went.
 * Errors: GW_ERR_ARG, GW_ERR_CUDA, GW_ERR_NOT_CONVERGED, GW_ERR_BREAKDOWN.
 */
int gw_pcg_solve_many(gw_hierarchy H, int k, const double *B, double *X, double tol, int maxit, int *iters,
                      double *relres, void *stream);

/*
 * gw_darcy_flux -- Darcy velocities on every face, from the heads: the
 * velocity field of the advective transport problem (Eq. 1).  Staggered
 * layout: vx has (nx+1)*ny*nz entries (face xf = 0..nx of row (y,z) at
 * xf + (nx+1)(y + ny z)), vy nx*(ny+1)*nz, vz nx*ny*(nz+1); positive along
 * +x, +y, +z.  An interior face carries T (h_a - h_b)/A_f (T as in
 * gw_assemble, a the lower cell, A_f the face area), a Dirichlet face uses
 * T_b and its head, a no-flow face 0.  All arrays device memory.
 * Asynchronous on stream.  Errors: GW_ERR_ARG.
 */
int gw_darcy_flux(const gw_grid *grid, const double *Kx, const double *Ky, const double *Kz, const gw_bc *bc,
                  const double *h, double *vx, double *vy, double *vz, void *stream);

/* Applies one V-cycle z = M^-1 r (from a zero initial guess) with the
 * hierarchy's precision; r and z are n doubles on the device. */
int gw_vcycle(gw_hierarchy H, const double *r, double *z, void *stream);

/* Table-1 statistics: fills out[0..min(cap, levels)-1] and *nlevels. */
int gw_hierarchy_info(gw_hierarchy H, gw_level_info *out, int cap, int *nlevels);

/*
 * Copies level l of the hierarchy for inspection: aggregate id per node
 * (n ints), MIS-2 root flag (n bytes), the FP64 CSR of A_l and of P_l.
 * Sizes from gw_hierarchy_info (P_l has n rows and naggregates columns).
 * Any pointer may be NULL; host or device memory.
 */
int gw_hierarchy_export(gw_hierarchy H, int level, int *agg, unsigned char *root, int *a_rowptr, int *a_col,
                        double *a_val, int *p_rowptr, int *p_col, double *p_val, void *stream);

/*
 * Benchmark instrumentation (no counterpart in the paper).  With profiling
 * on, the captured CG iteration graph records CUDA events around the
 * level-0 kernels of every iteration, one by one: the CG product q = A p
 * with its dot (GW_PK_SPMV), the x/r update (GW_PK_UPDATE), the first and the
 * following pre-smoothing kernels (GW_PK_PRE1, GW_PK_PRE2), the residual
 * (GW_PK_RESID), the restriction (GW_PK_RESTRICT), the interpolation and
 * correction (GW_PK_PROLONG), the first and the following post-smoothing
 * kernels (GW_PK_POST1, GW_PK_POST2; the last one yields z) and the direction
 * update (GW_PK_PUPDATE); and the coarser levels as groups: level 1 down to
 * the restriction to level 2 (GW_PK_L1DOWN), levels 2 and below with the
 * coarsest solve (GW_PK_DEEP), and the interpolation to level 1 with its
 * post-smoothing (GW_PK_L1UP).  Only iterations that ran to the end are
 * counted.  bytes[k] is the algorithmic traffic of one launch (or group) of
 * kind k: every array counted once, a gathered vector once, padding not
 * counted.  kernel_launches counts every kernel the solves launched (graph
 * kernel nodes included), profiling on or off.  Events between kernels
 * break the programmatic launch overlap, so profiled solves run slower.
 */
enum {
    GW_PK_SPMV = 0,
    GW_PK_UPDATE,
    GW_PK_PRE1,
    GW_PK_PRE2,
    GW_PK_RESID,
    GW_PK_RESTRICT,
    GW_PK_L1DOWN,
    GW_PK_DEEP,
    GW_PK_L1UP,
    GW_PK_PROLONG,
    GW_PK_POST1,
    GW_PK_POST2,
    GW_PK_PUPDATE,
    GW_PK_COUNT
};

typedef struct {
    double ms[GW_PK_COUNT];           /* summed device time per kind */
    long long launches[GW_PK_COUNT];  /* timed launches per kind */
    double bytes[GW_PK_COUNT];        /* algorithmic bytes of one launch */
    long long kernel_launches;        /* kernels launched by gw_pcg_solve */
    long long solves;                 /* gw_pcg_solve calls counted */
} gw_profile;

/* Turns the event instrumentation on or off (the iteration graph is
 * re-captured on the next solve). */
int gw_profile_enable(gw_hierarchy H, int on);

/* Copies the counters gathered since the last reset; reset != 0 clears them. */
int gw_profile_read(gw_hierarchy H, gw_profile *out, int reset);

/*
 * Free a handle.  Device memory goes back to the library's memory pool (in
 * stream order, without synchronising the device); the pool keeps it for
 * the next allocation.  Every call that uses a handle finishes its device
 * work before it returns, except gw_vcycle: let the work of a gw_vcycle
 * call finish before freeing its hierarchy.  A matrix must outlive the
 * hierarchies set up on it.
 */
void gw_matrix_free(gw_matrix A);
void gw_hierarchy_free(gw_hierarchy H);

/*
 * Batched solves -- many flow solves at once, as in the sensitivity-analysis
 * sweeps the paper names as the use of fast solves (Abstract), each with its
 * own resident hierarchy (grid size and conductivity field free per solve).
 * A batch keeps up to max_slots solves in flight.  Every launch of the batched
 * iteration runs one pass of the AMG-preconditioned CG iteration (the CG
 * product, the update, the reliable update, or one smoothing, residual,
 * restriction, coarse-solve or interpolation pass of one level) for every
 * solve that has it, over a device table of the slots' levels; the iteration
 * is one captured CUDA graph replayed by gw_batch_run.  A solve gives the same
 * result bit for bit alone or in any mix (its passes keep their own work
 * partition and reduction order), and the same iterates as gw_pcg_solve up to
 * the rounding of its reductions.  Solves join and leave between replays.
 * Supported hierarchies: the mixed form with FP32 storage (GW_PREC_MIXED32,
 * half_storage 0), Chebyshev smoothing of degree >= 2 with nu = 1 (the same
 * degree for every solve of a batch), 2 to 12 levels on a 7-point grid.
 * Calls on one batch must not overlap (one host thread drives it); the batch
 * runs on its own CUDA stream.
 *
 * gw_batch_create -- an empty batch of max_slots (1..256) slots on the
 *   current device.  Errors: GW_ERR_ARG, GW_ERR_OOM, GW_ERR_CUDA.
 * gw_batch_add -- starts the solve of C h = b on hierarchy H (b: n doubles,
 *   host or device; tol > 0 on the true relative residual, maxit >= 1) in a
 *   free slot, written to *slot; runs the solve's first V-cycle.  While the
 *   solve is in the batch, H may not be solved, shifted or prepared
 *   elsewhere (GW_ERR_ARG); freeing H removes its solve from the batch.
 *   Errors: GW_ERR_ARG (unsupported hierarchy, no free slot, bad argument),
 *   GW_ERR_OOM, GW_ERR_CUDA.
 * gw_batch_run -- replays the batched iteration up to `iterations` times,
 *   returning after the first replay in which some solve finished; *finished
 *   receives the number of finished solves waiting to be taken.
 * gw_batch_state -- *state = 0 (free slot), 1 (solve running) or 2 (finished).
 * gw_batch_take -- takes the finished solve of a slot: heads into h (n
 *   doubles, host or device, or NULL), iterations and true relative residual
 *   (host, may be NULL); frees the slot.  Returns the solve's status (GW_OK,
 *   GW_ERR_NOT_CONVERGED, GW_ERR_BREAKDOWN, or GW_ERR_ARG for a non-finite
 *   right-hand side) or GW_ERR_ARG when the slot holds no finished solve.
 * gw_batch_free -- frees the batch; solves not taken are abandoned.
 */
int gw_batch_create(int max_slots, gw_batch *B_out);
int gw_batch_add(gw_batch B, gw_hierarchy H, const double *b, double tol, int maxit, int *slot);
int gw_batch_run(gw_batch B, int iterations, int *finished);
int gw_batch_state(gw_batch B, int slot, int *state);
int gw_batch_take(gw_batch B, int slot, double *h, int *iters, double *relres);
void gw_batch_free(gw_batch B);

/* Static string naming a status code. */
const char *gw_status_str(int status);

/* One-line description of the last failure on the calling thread. */
const char *gw_last_error(void);

/*
 * gw_device_allocations -- the number of device allocations (from the
 * library's memory pool, or cudaMalloc outside a call that takes a stream)
 * the library has made in this process so far.  It
 * lets a caller check that a sequence of calls allocated nothing, for
 * example gw_assemble_noalloc.  Not part of the paper's method.
 */
long long gw_device_allocations(void);

#ifdef __cplusplus
}
#endif
#endif /* GW_H */
