// util.cu -- error plumbing, device scan and small host helpers of libgw.
#include <stdarg.h>
#include <string.h>

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

static thread_local cudaStream_t t_alloc_stream = nullptr;
static thread_local bool t_alloc_on = false;

AllocStream::AllocStream(cudaStream_t st) : prev_(t_alloc_stream), prev_on_(t_alloc_on)
{
    t_alloc_stream = st;
    t_alloc_on = true;
}

AllocStream::~AllocStream()
{
    t_alloc_stream = prev_;
    t_alloc_on = prev_on_;
}

constexpr int POOL_DEVS = 64;
struct DevPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t free_st = nullptr;  // releases made outside any call
};
static DevPool g_pool[POOL_DEVS];

// with g_alloc_mu held
static DevPool &pool_of(int dev)
{
    DevPool &d = g_pool[dev];
    if (!d.pool) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        GW_CUDA(cudaMemPoolCreate(&d.pool, &props));
        unsigned long long keep = ~0ULL;
        GW_CUDA(cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep));
        GW_CUDA(cudaStreamCreateWithFlags(&d.free_st, cudaStreamNonBlocking));
    }
    return d;
}

static int current_pool_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= POOL_DEVS) return -1;
    return dev;
}

cudaError_t dev_malloc(void **p, size_t bytes, int *pool_dev)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    g_device_allocs.fetch_add(1);
    *pool_dev = -1;
    const int dev = t_alloc_on ? current_pool_device() : -1;
    if (dev < 0) return cudaMalloc(p, bytes);
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool_of(dev).pool, t_alloc_stream);
    if (e == cudaSuccess) *pool_dev = dev;
    return e;
}

void dev_free(void *p, int pool_dev)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    if (pool_dev < 0) {
        cudaFree(p);
        return;
    }
    cudaFreeAsync(p, t_alloc_on ? t_alloc_stream : pool_of(pool_dev).free_st);
}

cudaError_t dev_malloc_on(void **p, size_t bytes, cudaStream_t st)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    g_device_allocs.fetch_add(1);
    const int dev = current_pool_device();
    if (dev < 0) return cudaMallocAsync(p, bytes, st);
    return cudaMallocFromPoolAsync(p, bytes, pool_of(dev).pool, st);
}

void dev_free_on(void *p, cudaStream_t st)
{
    std::unique_lock<std::mutex> lk(g_alloc_mu);
    g_alloc_cv.wait(lk, [] { return g_captures == 0; });
    cudaFreeAsync(p, st);
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
    GW_CUDA(dev_malloc_on((void **)&bsum, (size_t)(nb + 1) * sizeof(int), st));
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
    dev_free_on(bsum, st);
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
