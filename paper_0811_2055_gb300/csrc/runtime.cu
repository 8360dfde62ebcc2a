// Host runtime of libgblod: error messages, allocation, launch accounting, the CUDA-event
// timing probe and small helpers shared by the build and render paths.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gb {

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }
const char *get_error() { return t_err.c_str(); }

// The library's own stream-ordered memory pool of the current device.  Its release threshold is
// unbounded: memory freed by the library stays mapped in the pool for its next allocations, so a
// build that frees its sort buffers and then allocates the sorted particle arrays (and a later build
// of the same size) reuses mapped memory.  Pools with the default threshold of zero unmap freed
// memory at every stream synchronisation, and the build synchronises once per octree level.
// gblod_trim_cache returns the cached memory to the device.
static cudaMemPool_t lib_pool()
{
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t mp = nullptr;
        GB_CUDA(cudaMemPoolCreate(&mp, &props));
        uint64_t keep = ~0ull;
        GB_CUDA(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep));
        pools[dev] = mp;
    }
    return pools[dev];
}

void *Allocator::get(size_t bytes, cudaStream_t s) const
{
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (has_hook) {
        p = hook.alloc(bytes, (void *)s, hook.ctx);
        if (!p) fail(GBLOD_ERR_OOM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
        return p;
    }
    cudaError_t e = pooled ? cudaMallocFromPoolAsync(&p, bytes, lib_pool(), s) : cudaMallocAsync(&p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        fail(GBLOD_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    check_cuda(e, pooled ? "cudaMallocFromPoolAsync" : "cudaMallocAsync");
    return p;
}

void trim_cache(uint64_t keep_bytes)
{
    GB_CUDA(cudaMemPoolTrimTo(lib_pool(), (size_t)keep_bytes));
}

void Allocator::put(void *p, size_t bytes, cudaStream_t s) const
{
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (has_hook) {
        hook.free(p, bytes, (void *)s, hook.ctx);
        return;
    }
    (void)cudaFreeAsync(p, s);
}

void *HostStage::get(size_t b)
{
    if (b > bytes) {
        if (p) cudaFreeHost(p);
        p = nullptr;
        size_t want = b < 4096 ? 4096 : b;
        GB_CUDA(cudaMallocHost(&p, want));
        bytes = want;
    }
    return p;
}

HostStage::~HostStage()
{
    if (p) cudaFreeHost(p);
}

// ------------------------------------------------------------------ launches and probe
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct Probe {
    std::mutex mu;
    int kid = GBLOD_K_ANY;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> done;
    cudaEvent_t open = nullptr;
    double total_ms = 0.0;
    uint64_t launches = 0;

    cudaEvent_t take()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        GB_CUDA(cudaEventCreate(&e));
        return e;
    }
};

static Probe &probe()
{
    static Probe *p = new Probe();
    return *p;
}

void probe_before(int kid, cudaStream_t s)
{
    Probe &P = probe();
    if (P.kid == GBLOD_K_ANY || kid != P.kid) return;
    std::lock_guard<std::mutex> g(P.mu);
    P.open = P.take();
    GB_CUDA(cudaEventRecord(P.open, s));
}

void probe_after(int kid, cudaStream_t s)
{
    Probe &P = probe();
    if (P.kid == GBLOD_K_ANY || kid != P.kid) return;
    std::lock_guard<std::mutex> g(P.mu);
    cudaEvent_t e = P.take();
    GB_CUDA(cudaEventRecord(e, s));
    P.done.emplace_back(P.open, e);
    P.open = nullptr;
}

static void probe_drain(Probe &P)
{
    for (auto &pr : P.done) {
        GB_CUDA(cudaEventSynchronize(pr.second));
        float ms = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        P.total_ms += ms;
        P.launches += 1;
        P.pool.push_back(pr.first);
        P.pool.push_back(pr.second);
    }
    P.done.clear();
}

int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        GB_CUDA(cudaGetDevice(&dev));
        GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int persistent_blocks(int per_sm) { return num_sms() * per_sm; }

} // namespace gb

extern "C" {

uint64_t gblod_launch_count(void) { return gb::g_launches.load(); }

gblod_status gblod_trim_cache(uint64_t keep_bytes)
{
    try {
        gb::trim_cache(keep_bytes);
        return GBLOD_OK;
    } catch (const gb::Error &e) {
        return e.st;
    }
}

gblod_status gblod_probe_enable(int32_t kernel)
{
    if (kernel < 0 || kernel >= GBLOD_K_COUNT_) {
        gb::set_error("gblod_probe_enable: unknown kernel id");
        return GBLOD_ERR_INVALID_ARG;
    }
    try {
        gb::Probe &P = gb::probe();
        std::lock_guard<std::mutex> g(P.mu);
        gb::probe_drain(P);
        P.kid = kernel;
        P.total_ms = 0.0;
        P.launches = 0;
        return GBLOD_OK;
    } catch (const gb::Error &e) {
        return e.st;
    }
}

gblod_status gblod_probe_read(double *total_ms, uint64_t *launches)
{
    try {
        gb::Probe &P = gb::probe();
        std::lock_guard<std::mutex> g(P.mu);
        gb::probe_drain(P);
        if (total_ms) *total_ms = P.total_ms;
        if (launches) *launches = P.launches;
        return GBLOD_OK;
    } catch (const gb::Error &e) {
        return e.st;
    }
}

const char *gblod_status_string(gblod_status s)
{
    switch (s) {
    case GBLOD_OK: return "ok";
    case GBLOD_ERR_INVALID_ARG: return "invalid argument";
    case GBLOD_ERR_RANGE: return "value out of range";
    case GBLOD_ERR_OOM: return "out of memory";
    case GBLOD_ERR_CUDA: return "CUDA error";
    case GBLOD_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case GBLOD_ERR_NOT_IMPLEMENTED: return "not implemented";
    case GBLOD_ERR_CAPACITY: return "reserved scratch too small for the batch";
    }
    return "unknown status";
}

const char *gblod_last_error(void) { return gb::get_error(); }

} // extern "C"
