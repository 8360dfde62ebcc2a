// A2: stable LSD radix sort of (64-bit key, 32-bit value) pairs, 8-bit digits.
//
// Each pass is reduce-then-scan with no inter-CTA waiting: an upsweep writes one 256-bin
// digit histogram per 4096-key tile (digit-major), a device scan turns them into global
// offsets, and the scatter kernel re-reads its tile, ranks every key stably inside the tile
// (warp-striped rounds of 32 keys; __match_any_sync finds equal digits in a round, per-warp
// running counters carry ranks across rounds, warps are ordered by a prefix over the tile)
// and writes it to its final place.  Digits that are the same for every key are skipped.
#include "common.cuh"

namespace gb {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS; // 4096 keys

__global__ void k_diff_or(const uint64_t *keys, size_t n, unsigned long long *out)
{
    const uint64_t k0 = keys[0];
    uint64_t acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc |= keys[i] ^ k0;
    for (int d = 16; d > 0; d >>= 1) acc |= __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicOr(out, (unsigned long long)acc);
}

__global__ void __launch_bounds__(RS_THREADS) k_upsweep(const uint64_t *keys, size_t n, int shift, uint32_t *hist,
                                                        uint32_t ntiles)
{
    __shared__ uint32_t wh[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wh[0][0])[i] = 0u;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * RS_TILE + (size_t)warp * (RS_ROUNDS * 32);
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * 32 + lane;
        if (i < n) atomicAdd(&wh[warp][(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t d = threadIdx.x, sum = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) sum += wh[w][d];
    hist[(size_t)d * ntiles + blockIdx.x] = sum;
}

// Scatter of one tile: keys are ranked stably inside the tile as above, placed in shared memory in
// the tile's digit order, and then written out by consecutive threads, so that each digit's run of
// keys (about 16 per tile and digit) goes to consecutive addresses (coalesced stores); values
// follow through the same buffer.
struct ScatterSmem {
    union {
        uint64_t k[RS_TILE];
        uint32_t v[RS_TILE];
    } buf;
    uint8_t dig[RS_TILE];
    uint32_t wh[RS_WARPS][256];
    uint32_t toff[256];
    uint32_t tstart[256]; // first tile-local position of each digit
    uint32_t wsum[RS_WARPS];
};
static_assert(sizeof(ScatterSmem) <= 48 * 1024, "static shared memory limit");

__global__ void __launch_bounds__(RS_THREADS)
    k_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
              uint32_t *__restrict__ vout, size_t n, int shift, const uint32_t *__restrict__ offs, uint32_t ntiles)
{
    __shared__ ScatterSmem sm;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&sm.wh[0][0])[i] = 0u;
    sm.toff[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();

    const uint32_t lt = gbd::lanemask_lt();
    const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
    const size_t base = tile0 + (size_t)warp * (RS_ROUNDS * 32);
    const uint32_t nt = (uint32_t)min((size_t)RS_TILE, n - tile0); // keys in this tile
    uint64_t k[RS_ROUNDS];
    uint32_t v[RS_ROUNDS];
    uint32_t rk[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? kin[i] : 0ull;
        v[r] = ok ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * 32 + lane;
        bool ok = i < n;
        uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
        uint32_t tag = ok ? d : (256u + (uint32_t)lane);
        uint32_t peers = __match_any_sync(0xffffffffu, tag);
        uint32_t before = __popc(peers & lt);
        uint32_t cur = ok ? sm.wh[warp][d] : 0u;
        rk[r] = cur + before;
        __syncwarp();
        if (ok && before == 0) sm.wh[warp][d] = cur + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t total; // this thread's digit: keys of the tile with digit threadIdx.x
    {
        uint32_t d = threadIdx.x, run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = sm.wh[w][d];
            sm.wh[w][d] = run;
            run += c;
        }
        total = run;
    }
    // exclusive scan of the digit totals over the block: each digit's first tile-local position
    {
        uint32_t incl = total;
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, dd);
            if (lane >= dd) incl += o;
        }
        if (lane == 31) sm.wsum[warp] = incl;
        __syncthreads();
        uint32_t woff = 0;
        for (int w = 0; w < warp; ++w) woff += sm.wsum[w];
        sm.tstart[threadIdx.x] = woff + incl - total;
    }
    __syncthreads();
    // keys in tile-local digit order
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
            const uint32_t L = sm.tstart[d] + sm.wh[warp][d] + rk[r];
            sm.buf.k[L] = k[r];
            sm.dig[L] = (uint8_t)d;
            rk[r] = L; // the element's tile-local position, for the values below
        }
    }
    __syncthreads();
    for (uint32_t L = threadIdx.x; L < nt; L += RS_THREADS) {
        const uint32_t d = sm.dig[L];
        kout[(size_t)sm.toff[d] + (L - sm.tstart[d])] = sm.buf.k[L];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        size_t i = base + (size_t)r * 32 + lane;
        if (i < n) sm.buf.v[rk[r]] = v[r];
    }
    __syncthreads();
    for (uint32_t L = threadIdx.x; L < nt; L += RS_THREADS) {
        const uint32_t d = sm.dig[L];
        vout[(size_t)sm.toff[d] + (L - sm.tstart[d])] = sm.buf.v[L];
    }
}

} // namespace

void radix_sort_pairs(const Allocator &A, SortTmp &t, uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                      uint32_t *vals_alt, size_t n, int key_bits, cudaStream_t s, HostStage &hs)
{
    if (n <= 1) return;
    if (n >= (1ull << 32)) fail(GBLOD_ERR_INVALID_ARG, "radix sort: n must be below 2^32");
    const uint32_t ntiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
    const size_t hist_n = (size_t)256 * ntiles;
    t.buf.ensure(A, hist_n * sizeof(uint32_t) + 256, s);
    uint32_t *hist = reinterpret_cast<uint32_t *>(t.buf.p);

    // which digits vary at all
    Scratch<unsigned long long> diff(A, 1, s);
    GB_CUDA(cudaMemsetAsync(diff.p, 0, sizeof(unsigned long long), s));
    launch(GBLOD_K_SORT_UPSWEEP, k_diff_or, dim3(persistent_blocks(4)), dim3(256), 0, s, (const uint64_t *)*keys, n,
           diff.p);
    auto *hdiff = static_cast<unsigned long long *>(hs.get(sizeof(unsigned long long)));
    GB_CUDA(cudaMemcpyAsync(hdiff, diff.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    const unsigned long long varying = *hdiff;

    uint64_t *kin = *keys, *kout = keys_alt;
    uint32_t *vin = *vals, *vout = vals_alt;
    for (int shift = 0; shift < key_bits; shift += 8) {
        if (((varying >> shift) & 255ull) == 0ull) continue;
        launch(GBLOD_K_SORT_UPSWEEP, k_upsweep, dim3(ntiles), dim3(RS_THREADS), 0, s, (const uint64_t *)kin, n, shift,
               hist, ntiles);
        scan_exclusive_u32(A, t.scan, hist, hist, hist_n, (uint32_t *)nullptr, s);
        launch(GBLOD_K_SORT_SCATTER, k_scatter, dim3(ntiles), dim3(RS_THREADS), 0, s, (const uint64_t *)kin,
               (const uint32_t *)vin, kout, vout, n, shift, (const uint32_t *)hist, ntiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    *keys = kin;
    *vals = vin;
}

} // namespace gb
