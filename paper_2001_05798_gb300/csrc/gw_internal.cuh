// gw_internal.cuh -- internal types and helpers of libgw (CUDA, sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gw.h"

namespace gw {

// A named NVTX range for the lifetime of the object (setup levels, solves,
// batch replays); it costs nothing unless a profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ------------------------------------------------------------------ errors --
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const char *fmt, ...);
void set_last_error(const char *msg);
const char *last_error_cstr();

#define GW_CUDA(call)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            ::gw::fail(e_ == cudaErrorMemoryAllocation ? GW_ERR_OOM : GW_ERR_CUDA, "%s: %s (%s:%d)", \
                       #call, cudaGetErrorString(e_), __FILE__, __LINE__);                            \
    } while (0)

#define GW_LAUNCH_CHECK() GW_CUDA(cudaGetLastError())

// ------------------------------------------------- allocation vs capture --
// Device memory comes from a library-owned memory pool per device through
// stream-ordered allocation: a buffer is taken on the stream of the API call
// in progress on this thread (AllocStream, set by every entry point that takes
// a stream) and given back on the stream of the call that releases it, after
// that call's earlier work.  Buffers released outside any call (a handle
// freed) go back on a library stream of the device: every call that uses a
// handle's buffers has finished its device work when it returns, except
// gw_vcycle, whose work the caller lets finish before freeing the hierarchy.
// The pool keeps the memory it has, so that neither an allocation nor a free
// goes to the driver or synchronises the device once the pool has grown.
// Without an AllocStream (buffers made outside an API call) plain cudaMalloc
// and cudaFree are used.  cudaFree and cudaFreeHost synchronise the device,
// which invalidates a graph capture that another thread has in progress:
// every allocation and free of the library therefore waits while a capture
// is in progress, and a capture waits for allocations in flight.
cudaError_t dev_malloc(void **p, size_t bytes, int *pool_dev);
void dev_free(void *p, int pool_dev);
// the same on an explicit stream, for a buffer used and released within one
// stream's work
cudaError_t dev_malloc_on(void **p, size_t bytes, cudaStream_t st);
void dev_free_on(void *p, cudaStream_t st);
cudaError_t host_malloc(void **p, size_t bytes);
void host_free(void *p);
struct AllocStream {
    explicit AllocStream(cudaStream_t st);
    ~AllocStream();
    AllocStream(const AllocStream &) = delete;
    AllocStream &operator=(const AllocStream &) = delete;

  private:
    cudaStream_t prev_;
    bool prev_on_;
};
// Device allocations made by the library so far (from its pool or by
// cudaMalloc), for callers that must check that a call allocates nothing.
long long device_allocations();
// Outside this thread's own capture: waits until no other thread of the
// library captures, and keeps captures from starting while the returned
// lock is held (with lazy module loading, a module load or symbol lookup
// during another thread's capture invalidates that capture).
std::unique_lock<std::mutex> capture_gate();
struct CaptureScope {
    CaptureScope();
    ~CaptureScope();
    CaptureScope(const CaptureScope &) = delete;
    CaptureScope &operator=(const CaptureScope &) = delete;
};

// ---------------------------------------------------------- device buffers --
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    int pdev = -1;  // device of the pool it came from, -1 for cudaMalloc
    DBuf() = default;
    explicit DBuf(size_t n_) { alloc(n_); }
    void alloc(size_t n_)
    {
        release();
        if (n_) GW_CUDA(dev_malloc((void **)&p, n_ * sizeof(T), &pdev));
        n = n_;
    }
    void release()
    {
        if (p) dev_free(p, pdev);
        p = nullptr;
        n = 0;
        pdev = -1;
    }
    ~DBuf() { release(); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), pdev(o.pdev)
    {
        o.p = nullptr;
        o.n = 0;
        o.pdev = -1;
    }
    DBuf &operator=(DBuf &&o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            pdev = o.pdev;
            o.p = nullptr;
            o.n = 0;
            o.pdev = -1;
        }
        return *this;
    }
    size_t bytes() const { return n * sizeof(T); }
};

// FP64 CSR on the device, columns ascending within each row.
struct DCSR {
    int nr = 0, nc = 0, nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> v;
    size_t bytes() const { return rp.bytes() + ci.bytes() + v.bytes(); }
};

// Sliced ELL with slices of 32 rows.  Row r = 32*s + lane; slot k of that row
// lives at sp[s] + (k / V) * 32 * V + lane * V + (k % V), so one thread loads
// V consecutive slots of its row with one 16-byte (or 8-byte for indices of
// the FP64 form) load and a warp reads 32 * 16 contiguous bytes.  Padding
// slots hold column = row (or 0 for a rectangular matrix) and value 0.
constexpr int SELL_C = 32;

template <class T>
struct SellV;
template <>
struct SellV<float> {
    static constexpr int V = 4;
};
template <>
struct SellV<double> {
    static constexpr int V = 2;
};

template <class T>
struct Sell {
    int nr = 0, nc = 0, nslices = 0;
    long long stored = 0, nnz = 0;
    DBuf<int> sp;  // nslices + 1 slice offsets (elements)
    DBuf<int> ci;
    DBuf<T> v;
    DBuf<int> perm;  // rows sorted by length within windows: slot row r is row perm[r] (empty: r)
    size_t bytes() const { return sp.bytes() + ci.bytes() + v.bytes() + perm.bytes(); }
};

// CSR in the cycle's precision T (read by groups of 8 or 32 lanes per row).
template <class T>
struct CsrT {
    int nr = 0, nc = 0;
    long long nnz = 0;
    DBuf<int> rp, ci;
    DBuf<T> v;
    size_t bytes() const { return rp.bytes() + ci.bytes() + v.bytes(); }
};

// Index-free 7-point operator on an nx*ny*nz grid: the diagonal and the
// couplings to the +x, +y, +z neighbours (zero where there is none).  The
// coupling to a -x neighbour is ox[i-1] because the assembled operator is
// symmetric bit for bit.
template <class T>
struct StenT {
    int n = 0, nx = 0, ny = 0, nz = 0;
    DBuf<T> d, ox, oy, oz;
    size_t bytes() const { return d.bytes() + ox.bytes() + oy.bytes() + oz.bytes(); }
};

// The level-0 stencil with BF16 couplings (FP32 cycle only).  The diagonal
// is FP32 and absorbs the rounding of the couplings of its row,
// d_i = a_ii + sum_j (|bf16(a_ij)| - |a_ij|), so the stored operator keeps
// the row sums, the symmetry and the M-matrix signs of A.
struct StenB {
    int n = 0, nx = 0, ny = 0, nz = 0;
    DBuf<float> d;
    DBuf<__nv_bfloat16> ox, oy, oz;
    size_t bytes() const { return d.bytes() + ox.bytes() + oy.bytes() + oz.bytes(); }
};

// The level-0 stencil scaled to D^-1/2 A D^-1/2 (FP32 cycle only): sd_i =
// sqrt(a_ii) in FP32, the scaled +x/+y/+z couplings in FP16 (all in
// [-1, 0]), and the diagonal 1 + dd_i with dd_i in FP16 chosen so that the
// stored operator sd (C + diag(1 + dd)) sd keeps the row sums of A:
// dd_i = sum_j (|fp16(c_ij)| - |c_ij|) sd_j / sd_i.
struct StenH {
    int n = 0, nx = 0, ny = 0, nz = 0;
    DBuf<float> sd;
    DBuf<__half> dd, ox, oy, oz;
    size_t bytes() const { return sd.bytes() + dd.bytes() + ox.bytes() + oy.bytes() + oz.bytes(); }
};

enum { FMT_SELL = 0, FMT_CSR4 = 1, FMT_CSR8 = 2, FMT_CSR32 = 3, FMT_STEN = 4, FMT_STENB = 6,
       FMT_STENH = 8 };
// to_store request: sliced ELL over rows sorted by length within windows of
// SELL_SORT_WINDOW rows (stored as FMT_SELL with a row permutation); only
// for matrices read by the restriction, which writes its output row through it
constexpr int FMT_SELL_SORTED = 7;
constexpr int SELL_SORT_WINDOW = 256;

template <class T>
struct MatStore {
    int fmt = FMT_SELL;
    int nr = 0, nc = 0;
    long long nnz = 0;
    Sell<T> sell;
    CsrT<T> csr;
    StenT<T> sten;
    StenB stenb;
    StenH stenh;
    size_t bytes() const
    {
        return sell.bytes() + csr.bytes() + sten.bytes() + stenb.bytes() + stenh.bytes();
    }
};

int choose_fmt(const DCSR &A);
// fmt FMT_STEN needs the grid (nx, ny, nz); returns false if A is not a 7-point grid operator
template <class T>
bool to_store(const DCSR &A, MatStore<T> &M, int fmt, int nx, int ny, int nz, cudaStream_t st);

// ------------------------------------------------------------ CG control --
// Scalars of the CG recurrence live on the device so that an iteration needs
// no host round trip.
struct Ctl {
    double bnorm2, tol2;
    double rz, pq, alpha, beta, rr, rt2, relres, qz, rmax2, delta2;
    int it, maxit, done, status, check, flexible;
    unsigned int cnt[8];  // arrival counters of the last-block reductions
    // handle of the while node of the solve's graph (0 when the solve does
    // not run under one): the last kernel of the iteration sets it to 0 once
    // the solve is done
    unsigned long long cond;
};

constexpr int RED_MAX_BLOCKS = 4096;
#ifndef GW_BLOCKS_PER_SM
#define GW_BLOCKS_PER_SM 8  // grid cap of the cycle and CG kernels, per SM
#endif

// ------------------------------------------------------------ scan / misc --
void exclusive_scan(const int *in, int *out, int n, cudaStream_t st);  // out[n] = total
bool exclusive_scan_in(const int *in, int *out, int n, int *scratch, size_t cap, cudaStream_t st);
int read_int(const int *dptr, cudaStream_t st);
void to_device(void *dst, const void *src, size_t bytes, cudaStream_t st);
bool is_device_ptr(const void *p);
// Loads a kernel's code before its first launch outside a graph capture,
// waiting while another thread captures (with lazy module loading, a kernel
// loaded during a capture on another thread invalidates that capture).
void prime_kernel(const void *fn);

template <class... KArgs, class... Args>
inline void gw_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    prime_kernel((const void *)kernel);
    kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

// one wave of a kernel on the current device: resident blocks per SM (at
// block_size threads) times the SMs; cached per device and kernel
int kernel_wave(const void *fn, int block_size);

// -------------------------------------------------------------- assembly --
void assemble_csr(int nx, int ny, int nz, double dx, double dy, double dz, const double *Kx, const double *Ky,
                  const double *Kz, const int *bct, const double *bcv, const double *q, DCSR &A, double *b,
                  int *dflag, cudaStream_t st);

// The level-0 prolongator of the FP32 cycle applied from its definition,
// P = (I - omega D_F^-1 A_F) P_tent, instead of stored entries: on the 7-point
// grid (P e)_i = w_i e[agg_i] - s_i sum_j f_ij e[agg_j] over the six
// neighbours, with s_i = omega / (A_F)_ii, f_ij = a_ij for a strong coupling
// and 0 otherwise, and w_i = 1 - omega (w_i = 1, s_i = 0 for a row without
// strong couplings, whose row is the tentative one).  f is symmetric, so
// only the +x, +y, +z couplings are stored: 16 bytes a row plus agg, against
// about 63 bytes a row of padded sliced ELL at 128^3.
// Its transpose, the restriction, is applied the same way:
// (P^T r)_c = sum over the members j of aggregate c of u_j, with
// u_j = w_j r_j - sum_i f_ij s_i r_i over the six neighbours i of j; the
// member lists (ascending) are the rows of the tentative prolongator's
// transpose.
struct ImplP {
    int n = 0, nx = 0, sxy = 0, nc = 0;
    float w0 = 0.f;  // 1 - omega
    const int *agg = nullptr;
    DBuf<float> s, fx, fy, fz;
    DBuf<int> mptr, mem;  // members of aggregate c: mem[mptr[c] .. mptr[c+1])
    size_t bytes() const
    {
        return s.bytes() + fx.bytes() + fy.bytes() + fz.bytes() + mptr.bytes() + mem.bytes();
    }
};

// ----------------------------------------------------------------- setup --
struct LevelSetupOut {
    int nagg = 0, rounds = 0;
    double omega = 0, rho = 0;
};
void setup_strength(const DCSR &A, double theta2, DBuf<unsigned char> &S, cudaStream_t st);
int setup_mis2(const DCSR &A, const unsigned char *S, uint64_t seed, int level, DBuf<unsigned char> &root,
               int max_rounds, cudaStream_t st);  // returns rounds; GW_ERR_SETUP after max_rounds
int setup_aggregate(const DCSR &A, const unsigned char *S, const unsigned char *root, uint64_t seed, int level,
                    DBuf<int> &agg, cudaStream_t st);  // returns nagg
void setup_smooth_p(const DCSR &A, const unsigned char *S, const int *agg, int nagg, DCSR &P, double *omega,
                    double *rho, cudaStream_t st);
void setup_transpose(const DCSR &P, DCSR &R, cudaStream_t st);
// false (out.n = 0) when A is not a 7-point operator on the nx*ny*nz grid
bool setup_implicit_p(const DCSR &A, const unsigned char *S, const int *agg, int nagg, double omega, int nx, int ny,
                      int nz, ImplP &out, cudaStream_t st);
void setup_spgemm(const DCSR &L, const DCSR &Rm, DCSR &C, cudaStream_t st);
void setup_dense_inverse(const DCSR &A, DBuf<double> &Ainv, cudaStream_t st);
double setup_gershgorin(const DCSR &A, DBuf<double> &diag, cudaStream_t st);  // max_i sum|a_ij|/a_ii
double setup_power_lambda(const DCSR &A, const double *diag, uint64_t seed, int level, cudaStream_t st);

template <class T>
void to_sell(const DCSR &A, Sell<T> &S, cudaStream_t st, bool sorted = false);

// ---------------------------------------------------------------- cycle --
// Storage of one level of the V-cycle in the cycle's precision T.
template <class T>
struct CycLevel {
    int n = 0;
    MatStore<T> A, P, R;  // A_l, P_l (n x n_{l+1}), R_l = P_l^T
    DBuf<T> dw;          // Jacobi: w / a_ii; Chebyshev: 1 / a_ii
    DBuf<T> x, b, r, t, d, d2;
    double c0 = 0.0, c1[8] = {0}, c2[8] = {0};  // Chebyshev coefficients
};

struct BlockState;  // interleaved multi-right-hand-side solver state (block.cu)

struct Hier {
    int dev = 0;
    gw_amg_opts o{};
    const DCSR *A0 = nullptr;  // level-0 FP64 CSR (owned by the matrix handle)
    int L = 0;
    std::vector<DCSR> A;       // A[l] for l >= 1 (A[0] is *A0)
    std::vector<DCSR> P;       // P[l] for l < L-1
    std::vector<DCSR> R;       // R[l] = P[l]^T, kept for numeric refreshes
    std::vector<DBuf<int>> agg;
    std::vector<DBuf<unsigned char>> root;
    std::vector<gw_level_info> info;
    std::vector<CycLevel<float>> cf;
    std::vector<CycLevel<double>> cd;
    MatStore<double> A64;      // level-0 FP64 matrix of the outer CG (mixed precision)
    MatStore<float> A32;       // level-0 FP32 operator of the CG recurrence when the cycle's is BF16
    ImplP p0;                  // level-0 prolongator of the FP32 cycle (n = 0: stored P)
    int gnx = 0, gny = 0, gnz = 0;  // grid of the level-0 operator
    int max_blocks = 1216;     // one wave of 256-thread blocks (SMs x 8)
    DBuf<double> Ainv;         // dense inverse of the coarsest level, row-major
    // outer CG
    int n = 0;
    DBuf<double> x, r, p, p2, q, z, b, part;  // FP64 form (x, b also hold the mixed form's solution and rhs)
    DBuf<float> xs32, r32, p32, p32b, q32, z32;  // mixed form: FP32 recurrence (two direction buffers)
    DBuf<Ctl> ctl;
    Ctl *ctl_host = nullptr;   // pinned mirror of the control block
    cudaStream_t cap = nullptr, cap2 = nullptr;
    // gsolve: the whole solve (start + while node over one CG iteration);
    // ginit + gexec: the profiled form (start, then replays of GRAPH_ITERS
    // iterations polled by the host)
    cudaGraphExec_t gexec = nullptr, ginit = nullptr, gsolve = nullptr;
    unsigned long long cond = 0;  // the while node's conditional handle
    int graph_iters = 0;
    long long init_kernels = 0, iter_kernels = 0;
    // profiling of the level-0 kernels (events captured into the graph)
    struct Mark {
        int kind, iter;
        cudaEvent_t a, b;
        double bytes;
    };
    bool prof_on = false, prof_capture = false;
    int cap_iter = 0;
    double prof_bytes = 0.0;
    std::vector<Mark> marks;
    double prof_ms[GW_PK_COUNT] = {0}, prof_b[GW_PK_COUNT] = {0};
    long long prof_cnt[GW_PK_COUNT] = {0};
    long long launches = 0, solves = 0;
    BlockState *blk = nullptr;  // created by the first interleaved solve
    void *batch = nullptr;      // the batch that holds this hierarchy's solve (cycle.cu), if any
    ~Hier();
};

void drop_graphs(Hier &H);

// the FP32 level-0 operator of the mixed CG recurrence
inline const MatStore<float> &cg_op32(const Hier &H) { return H.A32.nr ? H.A32 : H.cf[0].A; }

void build_hierarchy(Hier &H, cudaStream_t st);
void refresh_level0(Hier &H, const DCSR &A, cudaStream_t st);
// level 0 becomes A and every coarse operator is formed again as
// P_l^T A_l P_l on the kept prolongators (same patterns), with the smoother
// data of every level and the coarsest inverse redone
void refresh_numeric(Hier &H, const DCSR &A, cudaStream_t st);
void vcycle_enqueue(Hier &H, const double *r, double *z, Ctl *ctl, bool dot, cudaStream_t st);
int pcg_run(Hier &H, double tol, int maxit, int *iters, double *relres, cudaStream_t st);
void pcg_prepare(Hier &H);  // capture the solver's graphs now

// k right-hand sides (column-major, leading dimension n, host or device)
// solved in interleaved blocks of up to 8 columns; mixed form only.
bool block_supported(const Hier &H);
int block_solve(Hier &H, int k, const double *B, double *X, double tol, int maxit, int *iters, double *relres,
                cudaStream_t st);
void block_drop_graphs(BlockState *s);

// Batched solves (cycle.cu): the same pass of several hierarchies' solves in
// one launch, one captured iteration graph replayed for all of them.
struct Batch;
Batch *batch_create(int max_slots);
void batch_free(Batch *B);
int batch_add(Batch &B, Hier &H, const double *b, double tol, int maxit);  // returns the slot
int batch_run(Batch &B, int iterations);                                   // finished solves waiting
int batch_state(const Batch &B, int slot);                                 // 0 free, 1 running, 2 finished
int batch_take(Batch &B, int slot, double *h, int *iters, double *relres);  // the solve's status
long long batch_kernel_launches(const Batch &B);
void batch_forget(Batch &B, Hier *H);
void block_free(BlockState *s);

}  // namespace gw
