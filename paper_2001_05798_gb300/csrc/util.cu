// util.cu -- error plumbing, device scan and small host helpers of libgw.
#include <stdarg.h>

#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>
#include <set>

#include "gw_internal.cuh"

namespace gw {

static thread_local std::string g_last_error;

void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

const char *last_error_cstr() { return g_last_error.c_str(); }

[[noreturn]] void fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    throw Error{code, std::string(buf)};
}

// ------------------------------------------------- allocation vs capture --
static std::mutex g_alloc_mu;
static std::condition_variable g_alloc_cv;
static int g_captures = 0;
static std::atomic<long long> g_device_allocs{0};

long long device_allocations() { return g_device_allocs.load(); }

cudaError_t dev_malloc(void **p, size_t bytes)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    g_device_allocs.fetch_add(1);
    return cudaMalloc(p, bytes);
}

void dev_free(void *p)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    cudaFree(p);
}

cudaError_t host_malloc(void **p, size_t bytes)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    return cudaMallocHost(p, bytes);
}

void host_free(void *p)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    cudaFreeHost(p);
}

// One capture at a time: the first use of a kernel in a capture loads its
// code (the occupancy query of launch sizing does), which invalidates a
// capture running on another thread; the capturing thread's own capture is
// not affected.
static std::mutex g_capture_mu;
static thread_local bool t_capturing = false;

CaptureScope::CaptureScope()
{
    g_capture_mu.lock();
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ++g_captures;
    }
    t_capturing = true;
}

std::unique_lock<std::mutex> capture_gate()
{
    std::unique_lock<std::mutex> lk(g_alloc_mu, std::defer_lock);
    if (!t_capturing) {
        lk.lock();
        g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    }
    return lk;
}

CaptureScope::~CaptureScope()
{
    t_capturing = false;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        --g_captures;
    }
    g_alloc_cv.notify_all();
    g_capture_mu.unlock();
}

// ------------------------------------------------------------------ scan --
// Exclusive prefix sum of n ints, three phases: per-block scan of 2048
// elements, scan of the block totals (recursively), add-back.
constexpr int SCAN_BS = 256, SCAN_IT = 8, SCAN_CHUNK = SCAN_BS * SCAN_IT;

__global__ void k_scan_block(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ bsum, int n)
{
    __shared__ int sh[SCAN_BS];
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * SCAN_CHUNK + (long long)tid * SCAN_IT;
    int v[SCAN_IT];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IT; ++k) {
        long long idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        s += v[k];
    }
    sh[tid] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_BS; off <<= 1) {
        int t = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += t;
        __syncthreads();
    }
    int excl = sh[tid] - s;
#pragma unroll
    for (int k = 0; k < SCAN_IT; ++k) {
        long long idx = base + k;
        if (idx < n) out[idx] = excl;
        excl += v[k];
    }
    if (tid == SCAN_BS - 1) bsum[blockIdx.x] = sh[tid];
}

__global__ void k_scan_add(int *__restrict__ out, const int *__restrict__ bsum, int n)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += bsum[idx / SCAN_CHUNK];
}

__global__ void k_set_at(int *dst, const int *src) { *dst = *src; }

void exclusive_scan(const int *in, int *out, int n, cudaStream_t st)
{
    if (n <= 0) {
        GW_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
        return;
    }
    int nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    int *bsum = nullptr;
    g_device_allocs.fetch_add(1);
    GW_CUDA(cudaMallocAsync((void **)&bsum, (size_t)(nb + 1) * sizeof(int), st));
    gw_launch(k_scan_block, nb, SCAN_BS, 0, st, in, out, bsum, n);
    GW_LAUNCH_CHECK();
    if (nb > 1) {
        exclusive_scan(bsum, bsum, nb, st);
        gw_launch(k_scan_add, (n + 255) / 256, 256, 0, st, out, bsum, n);
        GW_LAUNCH_CHECK();
        gw_launch(k_set_at, 1, 1, 0, st, out + n, bsum + nb);
    } else {
        gw_launch(k_set_at, 1, 1, 0, st, out + n, bsum);
    }
    GW_LAUNCH_CHECK();
    GW_CUDA(cudaFreeAsync(bsum, st));
}

// Same scan, with the block totals kept in caller-provided device memory of
// `cap` ints instead of an allocation; returns false if cap is too small.
bool exclusive_scan_in(const int *in, int *out, int n, int *scratch, size_t cap, cudaStream_t st)
{
    if (n <= 0) {
        GW_CUDA(cudaMemsetAsync(out, 0, sizeof(int), st));
        return true;
    }
    const int nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if ((size_t)nb + 1 > cap) return false;
    int *bsum = scratch;
    gw_launch(k_scan_block, nb, SCAN_BS, 0, st, in, out, bsum, n);
    GW_LAUNCH_CHECK();
    if (nb > 1) {
        if (!exclusive_scan_in(bsum, bsum, nb, scratch + nb + 1, cap - (size_t)nb - 1, st)) return false;
        gw_launch(k_scan_add, (n + 255) / 256, 256, 0, st, out, bsum, n);
        GW_LAUNCH_CHECK();
        gw_launch(k_set_at, 1, 1, 0, st, out + n, bsum + nb);
    } else {
        gw_launch(k_set_at, 1, 1, 0, st, out + n, bsum);
    }
    GW_LAUNCH_CHECK();
    return true;
}

int read_int(const int *dptr, cudaStream_t st)
{
    int v = 0;
    GW_CUDA(cudaMemcpyAsync(&v, dptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    GW_CUDA(cudaStreamSynchronize(st));
    return v;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void to_device(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    GW_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
}

void prime_kernel(const void *fn)
{
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> loaded;
    int dev = 0;
    GW_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_pair(dev, fn);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (loaded.count(key)) return;
    }
    auto gate = capture_gate();
    cudaFuncAttributes a;
    GW_CUDA(cudaFuncGetAttributes(&a, fn));
    std::lock_guard<std::mutex> lock(mu);
    loaded.insert(key);
}

int kernel_wave(const void *fn, int block_size)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cache;
    int dev = 0;
    GW_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_pair(dev, fn);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    // the query may load the kernel's code: outside a capture of this thread,
    // wait until no other thread captures (and keep captures from starting)
    auto gate = capture_gate();
    int nb = 0, sms = 0;
    GW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block_size, 0));
    GW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int w = std::max(1, nb) * std::max(1, sms);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = w;
    return w;
}

}  // namespace gw
