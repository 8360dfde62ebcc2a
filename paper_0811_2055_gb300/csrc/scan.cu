// Device-wide exclusive prefix sums (reduce, scan the block totals, scan again with offsets).
// Used for tile offsets, node and chunk numbering, and the exact 128-bit mass prefix.
#include "common.cuh"

namespace gb {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
static_assert(SCAN_TILE == (int)SCAN_TILE_ELEMS, "scan_temp_bytes assumes this block size");

template <class T> struct Ops;

template <> struct Ops<uint32_t> {
    static __device__ __forceinline__ uint32_t zero() { return 0u; }
    static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) { return a + b; }
    static __device__ __forceinline__ uint32_t shfl_up(uint32_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
    static __device__ __forceinline__ uint32_t shfl(uint32_t v, int l) { return __shfl_sync(0xffffffffu, v, l); }
};

template <> struct Ops<uint64_t> {
    static __device__ __forceinline__ uint64_t zero() { return 0ull; }
    static __device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) { return a + b; }
    static __device__ __forceinline__ uint64_t shfl_up(uint64_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
    static __device__ __forceinline__ uint64_t shfl(uint64_t v, int l) { return __shfl_sync(0xffffffffu, v, l); }
};

template <> struct Ops<U128> {
    static __device__ __forceinline__ U128 zero() { return U128{0ull, 0ull}; }
    static __device__ __forceinline__ U128 add(U128 a, U128 b) { return gbd::add128(a, b); }
    static __device__ __forceinline__ U128 shfl_up(U128 v, int d)
    {
        return U128{__shfl_up_sync(0xffffffffu, v.lo, d), __shfl_up_sync(0xffffffffu, v.hi, d)};
    }
    static __device__ __forceinline__ U128 shfl(U128 v, int l)
    {
        return U128{__shfl_sync(0xffffffffu, v.lo, l), __shfl_sync(0xffffffffu, v.hi, l)};
    }
};

// Exclusive scan of one value per thread across the block; every thread receives the block
// total in `tot`.
template <class T> __device__ T block_exclusive(T v, T &tot)
{
    using O = Ops<T>;
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ T warp_ex[NW];
    __shared__ T total_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = O::shfl_up(incl, d);
        if (lane >= d) incl = O::add(incl, o);
    }
    if (lane == 31) warp_ex[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T wi = lane < NW ? warp_ex[lane] : O::zero();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = O::shfl_up(wi, d);
            if (lane >= d) wi = O::add(wi, o);
        }
        T wex = O::shfl_up(wi, 1);
        if (lane == 0) wex = O::zero();
        if (lane < NW) warp_ex[lane] = wex;
        if (lane == NW - 1) total_s = wi;
    }
    __syncthreads();
    T self_ex = O::shfl_up(incl, 1);
    if (lane == 0) self_ex = O::zero();
    T res = O::add(warp_ex[warp], self_ex);
    tot = total_s;
    __syncthreads();
    return res;
}

template <class T> __global__ void k_scan_reduce(const T *in, size_t n, T *partial)
{
    using O = Ops<T>;
    size_t base = (size_t)blockIdx.x * SCAN_TILE;
    T s = O::zero();
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        size_t i = base + (size_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s = O::add(s, in[i]);
    }
    T tot;
    (void)block_exclusive<T>(s, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_down(const T *in, T *out, size_t n, const T *offsets, T *total, unsigned nblocks)
{
    using O = Ops<T>;
    __shared__ T tile[SCAN_TILE];
    size_t base = (size_t)blockIdx.x * SCAN_TILE;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int j = k * SCAN_THREADS + threadIdx.x;
        size_t i = base + j;
        tile[j] = i < n ? in[i] : O::zero();
    }
    __syncthreads();
    T loc[SCAN_ITEMS];
    T run = O::zero();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        loc[k] = run;
        run = O::add(run, tile[threadIdx.x * SCAN_ITEMS + k]);
    }
    T tot;
    T ex = block_exclusive<T>(run, tot);
    T off = offsets ? offsets[blockIdx.x] : O::zero();
    ex = O::add(ex, off);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) tile[threadIdx.x * SCAN_ITEMS + k] = O::add(ex, loc[k]);
    __syncthreads();
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int j = k * SCAN_THREADS + threadIdx.x;
        size_t i = base + j;
        if (i < n) out[i] = tile[j];
    }
    if (total && blockIdx.x == nblocks - 1 && threadIdx.x == 0) *total = O::add(off, tot);
}

template <class T>
void scan_impl(const Allocator &A, ScanTmp &t, const T *in, T *out, size_t n, T *total, cudaStream_t s,
               size_t tmp_off)
{
    if (n == 0) {
        if (total) GB_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return;
    }
    size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        launch(GBLOD_K_SCAN, k_scan_down<T>, dim3(1), dim3(SCAN_THREADS), 0, s, in, out, n, (const T *)nullptr,
               total, 1u);
        return;
    }
    // temp layout: [partial nb][offsets nb] then the recursion's own space
    size_t need = tmp_off + 2 * nb * sizeof(T) + 256;
    if (t.buf.cap < need) fail(GBLOD_ERR_INVALID_ARG, "scan temp undersized");
    T *partial = reinterpret_cast<T *>(t.buf.p + ((tmp_off + 255) / 256) * 256);
    T *offs = partial + nb;
    size_t next_off = (size_t)((unsigned char *)(offs + nb) - t.buf.p);
    launch(GBLOD_K_SCAN, k_scan_reduce<T>, dim3((unsigned)nb), dim3(SCAN_THREADS), 0, s, in, n, partial);
    scan_impl<T>(A, t, partial, offs, nb, (T *)nullptr, s, next_off);
    launch(GBLOD_K_SCAN, k_scan_down<T>, dim3((unsigned)nb), dim3(SCAN_THREADS), 0, s, in, out, n,
           (const T *)offs, total, (unsigned)nb);
}

template <class T>
void scan_entry(const Allocator &A, ScanTmp &t, const T *in, T *out, size_t n, T *total, cudaStream_t s)
{
    // worst-case temp: sum over levels of 2 * ceil(n / TILE^k) * sizeof(T) plus alignment slack
    t.buf.ensure(A, scan_temp_bytes(n, sizeof(T)), s);
    scan_impl<T>(A, t, in, out, n, total, s, 0);
}

} // namespace

void scan_exclusive_u32(const Allocator &A, ScanTmp &t, const uint32_t *in, uint32_t *out, size_t n,
                        uint32_t *total, cudaStream_t s)
{
    scan_entry<uint32_t>(A, t, in, out, n, total, s);
}

void scan_exclusive_u64(const Allocator &A, ScanTmp &t, const uint64_t *in, uint64_t *out, size_t n,
                        uint64_t *total, cudaStream_t s)
{
    scan_entry<uint64_t>(A, t, in, out, n, total, s);
}

void scan_exclusive_u128(const Allocator &A, ScanTmp &t, const U128 *in, U128 *out, size_t n, U128 *total,
                         cudaStream_t s)
{
    scan_entry<U128>(A, t, in, out, n, total, s);
}

} // namespace gb
