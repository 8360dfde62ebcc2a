// Issue-rate probes of the integer instruction mixes that the splat kernels execute, timed with CUDA
// events on the caller's stream.  They give the measured ceilings the benchmark reports its
// roofline fractions against: the splat kernels are bound by integer instruction issue, not by
// memory, and the integer ceiling is not one number (wide and high-word multiplies, table reads
// from shared memory and plain adds go to different pipes).
//
// Every probe runs a grid of (SMs x resident blocks) x 256 threads; each thread keeps independent
// chains so that dependency latency is hidden, reads its inputs from kernel arguments and shared
// memory (nothing can be folded at compile time) and writes its result to `sink`.
#include "common.cuh"

namespace gb {
namespace {

constexpr int MB_T = 256;

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    return x;
}

// 8 independent chains of (a ^ b) + c: two int32 ALU operations per step and chain
__global__ void __launch_bounds__(MB_T) k_mb_alu(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8], b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = mix32(seed + threadIdx.x * 8u + (uint32_t)k);
        b[k] = mix32(a[k] + 1u);
    }
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = (a[k] ^ b[k]) + b[(k + r) & 7];
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = s;
}

// 8 independent chains of a * m + c (one 32-bit multiply-add per step and chain)
__global__ void __launch_bounds__(MB_T) k_mb_imad(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8], m[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = mix32(seed + threadIdx.x * 8u + (uint32_t)k);
        m[k] = mix32(a[k]) | 1u;
    }
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = a[k] * m[k] + m[(k + r + 1) & 7];
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = s;
}

// 8 independent 64-bit accumulations of a 32 x 32 -> 64 product
__global__ void __launch_bounds__(MB_T) k_mb_imad_wide(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    unsigned long long acc[8];
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = mix32(seed + threadIdx.x * 8u + (uint32_t)k);
        acc[k] = x[k];
    }
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += (unsigned long long)x[k] * x[(k + r + 1) & 7];
        }
        x[i & 7] += 1u;
    }
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += acc[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = (uint32_t)(s ^ (s >> 32));
}

// 8 independent 32-bit accumulations of the high word of a 32 x 32 product
__global__ void __launch_bounds__(MB_T) k_mb_imad_hi(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t acc[8], x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        x[k] = mix32(seed + threadIdx.x * 8u + (uint32_t)k);
        acc[k] = x[k];
    }
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += __umulhi(x[k], x[(k + r + 1) & 7]);
        }
        x[i & 7] += 1u;
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += acc[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = s;
}

// one conflict-free shared-memory word load per step (lane-dependent addresses)
__global__ void __launch_bounds__(MB_T) k_mb_lds(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    __shared__ uint32_t t[1024];
    for (int i = threadIdx.x; i < 1024; i += MB_T) t[i] = mix32(seed + (uint32_t)i);
    __syncthreads();
    uint32_t s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = (uint32_t)k;
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k] += t[(((s[k] & 31u) ^ lane) + 32u * (uint32_t)((k + r) & 31)) & 1023u];
        }
    }
    uint32_t o = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) o += s[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = o;
}

// The radial rule's per-pixel body with every pixel inside the support: squared distance, table
// index as the high word of q S shifted by 5, shared table read, two-part amplitude accumulation.
// Four pixels (blocks) per lane and record, as in the splat kernel.
__global__ void __launch_bounds__(MB_T) k_mb_radial(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    __shared__ int32_t K[1024];
    __shared__ int4 rec[256];
    for (int i = threadIdx.x; i < 1024; i += MB_T) K[i] = (int32_t)(mix32(seed + (uint32_t)i) & 0xFFFFu);
    for (int i = threadIdx.x; i < 256; i += MB_T) {
        const uint32_t h = mix32(seed ^ (uint32_t)(i * 7919));
        rec[i] = make_int4((int)(h & 0xFFFFu), (int)(h >> 16), (int)(mix32(h) & 0x7FFFu), (int)(mix32(h + 1u)));
    }
    __syncthreads();
    const int pxv = (int)(threadIdx.x & 7u) * 256 + 128, pyv0 = (int)(threadIdx.x >> 3) * 256 + 128;
    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
    uint32_t lo[4] = {0u, 0u, 0u, 0u};
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll 2
        for (int j = 0; j < 8; ++j) {
            const int4 A = rec[(i * 8u + (uint32_t)j) & 255u];
            const uint32_t Wl = (uint32_t)A.w & 0xFFFFu;
            const int dx = pxv - A.x;
            const uint32_t dx2 = (uint32_t)(dx * dx);
            const int dy0 = pyv0 - A.y;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int dy = dy0 + k * 2048;
                const uint32_t q = dx2 + (uint32_t)(dy * dy);
                const uint32_t idx = __umulhi(q, (uint32_t)A.z) >> 5;
                const uint32_t kv = (uint32_t)K[idx];
                acc[k] += (unsigned long long)((uint32_t)A.w >> 16) * kv;
                lo[k] += (Wl * kv) >> 16;
            }
        }
    }
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) s += acc[k] + lo[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = (uint32_t)(s ^ (s >> 32));
}

// The separable rule's per-pixel body: per record the lane's column weight Kx (from its own
// table lookup), then for each of 16 rows acc += P_hi Kx and lo += hi32(P_lo Kx), P = (Wq K_y)
// of the row read from shared memory (the same address in every lane: a broadcast).
__global__ void __launch_bounds__(MB_T) k_mb_separable(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    __shared__ int32_t K[1024];
    __shared__ uint4 P[256 * 8]; // 256 records x 16 rows of (P_hi, P_lo)
    __shared__ int2 rec[256];
    for (int i = threadIdx.x; i < 1024; i += MB_T) K[i] = (int32_t)(mix32(seed + (uint32_t)i) & 0xFFFFu);
    for (int i = threadIdx.x; i < 256 * 8; i += MB_T) {
        const uint32_t h = mix32(seed ^ (uint32_t)(i * 104729));
        P[i] = make_uint4(h & 0xFFFFFFu, mix32(h), mix32(h + 3u) & 0xFFFFFFu, mix32(h + 5u));
    }
    for (int i = threadIdx.x; i < 256; i += MB_T) {
        const uint32_t h = mix32(seed ^ (uint32_t)(i * 7919));
        rec[i] = make_int2((int)(h & 0xFFFFu), (int)(mix32(h) & 0x7FFFu));
    }
    __syncthreads();
    const int pxv = (int)(threadIdx.x & 31u) * 256 + 128;
    unsigned long long acc[16];
    uint32_t lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        acc[k] = 0ull;
        lo[k] = 0u;
    }
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
        const uint32_t r = i & 255u;
        const int2 R = rec[r];
        const int dx = pxv - R.x;
        const uint32_t ix = __umulhi((uint32_t)(dx * dx), (uint32_t)R.y) >> 5;
        const uint32_t kx = ix < 1024u ? (uint32_t)K[ix] : 0u;
        const uint4 *Pr = &P[r * 8u];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint4 p = Pr[k];
            acc[2 * k] += (unsigned long long)p.x * kx;
            lo[2 * k] += __umulhi(p.y, kx);
            acc[2 * k + 1] += (unsigned long long)p.z * kx;
            lo[2 * k + 1] += __umulhi(p.w, kx);
        }
    }
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += acc[k] + lo[k];
    sink[blockIdx.x * MB_T + threadIdx.x] = (uint32_t)(s ^ (s >> 32));
}

} // namespace

// units of work of one launch per thread and outer iteration, by kind
static double mb_units_per_iter(int kind)
{
    switch (kind) {
    case GBLOD_MB_ALU: return 8.0 * 8.0 * 2.0;
    case GBLOD_MB_IMAD: return 8.0 * 8.0;
    case GBLOD_MB_IMAD_WIDE: return 8.0 * 8.0;
    case GBLOD_MB_IMAD_HI: return 8.0 * 8.0;
    case GBLOD_MB_LDS: return 8.0 * 8.0;
    case GBLOD_MB_RADIAL: return 8.0 * 4.0;
    case GBLOD_MB_SEPARABLE: return 16.0;
    default: return 0.0;
    }
}

void microbench(int kind, uint32_t iters, cudaStream_t s, double *ms, double *units)
{
    void (*k)(uint32_t, uint32_t, uint32_t *) = nullptr;
    switch (kind) {
    case GBLOD_MB_ALU: k = k_mb_alu; break;
    case GBLOD_MB_IMAD: k = k_mb_imad; break;
    case GBLOD_MB_IMAD_WIDE: k = k_mb_imad_wide; break;
    case GBLOD_MB_IMAD_HI: k = k_mb_imad_hi; break;
    case GBLOD_MB_LDS: k = k_mb_lds; break;
    case GBLOD_MB_RADIAL: k = k_mb_radial; break;
    case GBLOD_MB_SEPARABLE: k = k_mb_separable; break;
    default: fail(GBLOD_ERR_INVALID_ARG, "unknown microbenchmark kind");
    }
    if (iters == 0 || iters > (1u << 24)) fail(GBLOD_ERR_INVALID_ARG, "iters must be in 1..2^24");
    int per_sm = 0;
    GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, MB_T, 0));
    if (per_sm < 1) per_sm = 1;
    const unsigned grid = (unsigned)(num_sms() * per_sm);
    uint32_t *sink = nullptr;
    GB_CUDA(cudaMallocAsync(&sink, (size_t)grid * MB_T * 4, s));
    cudaEvent_t e0, e1;
    GB_CUDA(cudaEventCreate(&e0));
    GB_CUDA(cudaEventCreate(&e1));
    // one untimed launch (clocks up, code loaded), then the timed one
    k<<<grid, MB_T, 0, s>>>(iters / 4 + 1, 1u, sink);
    count_launch();
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaEventRecord(e0, s));
    k<<<grid, MB_T, 0, s>>>(iters, 2u, sink);
    count_launch();
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaEventRecord(e1, s));
    GB_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    GB_CUDA(cudaEventElapsedTime(&t, e0, e1));
    GB_CUDA(cudaEventDestroy(e0));
    GB_CUDA(cudaEventDestroy(e1));
    GB_CUDA(cudaFreeAsync(sink, s));
    GB_CUDA(cudaStreamSynchronize(s));
    *ms = (double)t;
    *units = (double)grid * MB_T * (double)iters * mb_units_per_iter(kind);
}

} // namespace gb

extern "C" gblod_status gblod_microbench(int32_t kind, uint32_t iters, void *stream, double *ms, double *units)
{
    try {
        if (!ms || !units) gb::fail(GBLOD_ERR_INVALID_ARG, "gblod_microbench: ms and units must not be NULL");
        if (kind < 0 || kind >= GBLOD_MB_COUNT_) gb::fail(GBLOD_ERR_INVALID_ARG, "gblod_microbench: unknown kind");
        double t = 0.0, u = 0.0;
        gb::microbench(kind, iters, (cudaStream_t)stream, &t, &u);
        *ms = t;
        *units = u;
        return GBLOD_OK;
    } catch (const gb::Error &e) {
        return e.st;
    }
}
