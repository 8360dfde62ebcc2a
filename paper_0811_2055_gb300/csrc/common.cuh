// Shared internals of libgblod: allocation through the caller's hook, launch accounting and
// the timing probe, error plumbing, and small device helpers used by several kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <string>

#include "../../include/gblod.h"

namespace gb {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
const char *get_error();

struct Error {
    gblod_status st;
    Error(gblod_status s) : st(s) {}
};

inline void check_cuda(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        throw Error(GBLOD_ERR_CUDA);
    }
}
#define GB_CUDA(x) ::gb::check_cuda((x), #x)

inline void fail(gblod_status s, const std::string &msg)
{
    set_error(msg);
    throw Error(s);
}

// ------------------------------------------------------------------ memory
struct Allocator {
    gblod_allocator hook{};
    bool has_hook = false;
    bool pooled = true; // without a hook: the library's retaining pool (else cudaMallocAsync's default pool)
    explicit Allocator(const gblod_allocator *a = nullptr, bool use_pool = true) : pooled(use_pool)
    {
        if (a && a->alloc && a->free) {
            hook = *a;
            has_hook = true;
        }
    }
    void *get(size_t bytes, cudaStream_t s) const;
    void put(void *p, size_t bytes, cudaStream_t s) const;
};

// Grow-only device buffer.
template <class T> struct DBuf {
    T *p = nullptr;
    size_t cap = 0; // elements
    void ensure(const Allocator &A, size_t n, cudaStream_t s)
    {
        if (n <= cap) return;
        if (p) A.put(p, cap * sizeof(T), s);
        p = nullptr; // a failing allocation below leaves an empty buffer, not a released one
        cap = 0;
        size_t want = n + n / 4 + 64;
        p = static_cast<T *>(A.get(want * sizeof(T), s));
        cap = want;
    }
    void release(const Allocator &A, cudaStream_t s)
    {
        if (p) A.put(p, cap * sizeof(T), s);
        p = nullptr;
        cap = 0;
    }
};

// Exact-size device buffer freed on scope exit.
template <class T> struct Scratch {
    const Allocator *A = nullptr;
    cudaStream_t s = nullptr;
    T *p = nullptr;
    size_t n = 0;
    Scratch() = default;
    Scratch(const Allocator &a, size_t count, cudaStream_t st) : A(&a), s(st), n(count)
    {
        p = count ? static_cast<T *>(a.get(count * sizeof(T), st)) : nullptr;
    }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    Scratch(Scratch &&o) noexcept { *this = std::move(o); }
    Scratch &operator=(Scratch &&o) noexcept
    {
        reset();
        A = o.A; s = o.s; p = o.p; n = o.n;
        o.p = nullptr; o.n = 0;
        return *this;
    }
    ~Scratch() { reset(); }
    void reset()
    {
        if (p && A) A->put(p, n * sizeof(T), s);
        p = nullptr;
        n = 0;
    }
    T *release_ptr()
    {
        T *q = p;
        p = nullptr;
        n = 0;
        return q;
    }
};

// Pinned host staging for small read-backs.
struct HostStage {
    void *p = nullptr;
    size_t bytes = 0;
    void *get(size_t b);
    ~HostStage();
};

// ------------------------------------------------------------------ launches
void probe_before(int kid, cudaStream_t s);
void probe_after(int kid, cudaStream_t s);
void count_launch();

template <typename... KArgs, typename... Args>
inline void launch(int kid, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
    probe_before(kid, s);
    kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
    probe_after(kid, s);
    count_launch();
    GB_CUDA(cudaGetLastError());
}

int num_sms();
int persistent_blocks(int per_sm);
void trim_cache(uint64_t keep_bytes); // unmaps the library pool's cached memory beyond keep_bytes

// ------------------------------------------------------------------ scans (scan.cu)
// Exclusive prefix sums in place-free form: out[i] = sum_{k<i} in[k]; if total != nullptr the
// grand total is written there (device pointer).  `tmp` is grown as needed, to at most
// scan_temp_bytes(n, sizeof element): it is never grown when it already holds that many bytes.
constexpr size_t SCAN_TILE_ELEMS = 2048; // elements per scan block (256 threads x 8)
constexpr size_t scan_temp_bytes(size_t n, size_t elem)
{
    size_t need = 0, m = n;
    while (m > SCAN_TILE_ELEMS) {
        m = (m + SCAN_TILE_ELEMS - 1) / SCAN_TILE_ELEMS;
        need += 2 * m * elem + 512;
    }
    return need + 1024;
}
struct ScanTmp {
    DBuf<unsigned char> buf;
};
void scan_exclusive_u32(const Allocator &A, ScanTmp &t, const uint32_t *in, uint32_t *out, size_t n,
                        uint32_t *total, cudaStream_t s);
void scan_exclusive_u64(const Allocator &A, ScanTmp &t, const uint64_t *in, uint64_t *out, size_t n,
                        uint64_t *total, cudaStream_t s);

// 128-bit unsigned as two words (device arithmetic with explicit carries).
struct U128 {
    uint64_t lo, hi;
};
void scan_exclusive_u128(const Allocator &A, ScanTmp &t, const U128 *in, U128 *out, size_t n, U128 *total,
                         cudaStream_t s);

// ------------------------------------------------------------------ sort (sort.cu)
struct SortTmp {
    DBuf<unsigned char> buf;
    ScanTmp scan;
};
// Stable LSD radix sort of (keys, vals) ascending by bits [0, key_bits) of the key.  On return
// the sorted data is in (*keys, *vals), which point either to the input or to the alternate
// buffers.  Digits that are constant over all keys are skipped.
void radix_sort_pairs(const Allocator &A, SortTmp &t, uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                      uint32_t *vals_alt, size_t n, int key_bits, cudaStream_t s, HostStage &hs);

} // namespace gb

// ------------------------------------------------------------------ device helpers
namespace gbd {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ gb::U128 add128(gb::U128 a, gb::U128 b)
{
    gb::U128 r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
    return r;
}

__device__ __forceinline__ gb::U128 sub128(gb::U128 a, gb::U128 b)
{
    gb::U128 r;
    r.lo = a.lo - b.lo;
    r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
    return r;
}

} // namespace gbd
