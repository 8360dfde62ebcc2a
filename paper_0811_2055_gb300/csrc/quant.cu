// 16-bit block codes of the stored points (storage paragraph): positions in 2 bytes per
// coordinate spanning the node's cell, weight and smoothing length coded linearly over the
// node's range.  One block per node codes its points and reduces the decoded bounds; a
// level-by-level pass (deepest first) then folds the children into each node's subtree bounds
// and writes the quantised node table.
#include <cmath>

#include "octree.cuh"

namespace gb {
namespace {

constexpr int QT = 256;

struct Red6 {
    float v[6];
};

// block-wide reduction of six floats: slots 0-2 take the minimum, 3-5 the maximum (finite
// inputs; the comparison keeps whichever equal value it saw first, as a strict compare does)
__device__ __forceinline__ Red6 block_minmax6(Red6 r, float *sm)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int d = 16; d > 0; d >>= 1)
        for (int k = 0; k < 6; ++k) {
            const float o = __shfl_xor_sync(0xffffffffu, r.v[k], d);
            r.v[k] = k < 3 ? (o < r.v[k] ? o : r.v[k]) : (o > r.v[k] ? o : r.v[k]);
        }
    if (lane == 0)
        for (int k = 0; k < 6; ++k) sm[wid * 6 + k] = r.v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < QT / 32; ++w)
            for (int k = 0; k < 6; ++k) {
                const float o = sm[w * 6 + k];
                r.v[k] = k < 3 ? (o < r.v[k] ? o : r.v[k]) : (o > r.v[k] ? o : r.v[k]);
            }
    __syncthreads();
    return r; // valid in thread 0
}

__device__ __forceinline__ uint32_t code_floor(float x, float lo, float step)
{
    const double d = __ddiv_rn(__dsub_rn((double)x, (double)lo), (double)step);
    if (!(d >= 0.0)) return 0u;
    if (d >= 65535.0) return 65535u;
    return (uint32_t)floor(d);
}

__device__ __forceinline__ uint32_t code_rne(float v, float lo, float step)
{
    if (!(step > 0.0f) || !isfinite(v)) return 0u;
    const double d = rint(__ddiv_rn(__dsub_rn((double)v, (double)lo), (double)step));
    if (!(d >= 0.0)) return 0u;
    if (d >= 65535.0) return 65535u;
    return (uint32_t)d;
}

// lower bound and step of a linear code from the finite range [mn, mx] (mn > mx: none finite)
__device__ __forceinline__ void lin_range(float mn, float mx, float &lo, float &step)
{
    if (!(mn <= mx)) {
        lo = 0.0f;
        step = 0.0f;
        return;
    }
    lo = __fadd_rn(mn, 0.0f);
    step = __double2float_rn(__ddiv_rn(__dsub_rn((double)mx, (double)mn), 65535.0));
}

__global__ void __launch_bounds__(QT) k_block_encode(size_t nn, const gblod_node *__restrict__ nodes,
                                                     const float4 *__restrict__ pts4, const float *__restrict__ hs,
                                                     double lo0, double lo1, double lo2, double side,
                                                     ushort4 *__restrict__ q4, uint16_t *__restrict__ qw,
                                                     float4 *__restrict__ qa, float *__restrict__ own)
{
    __shared__ float sm[(QT / 32) * 6];
    __shared__ float4 sA, sB;
    for (size_t i = blockIdx.x; i < nn; i += gridDim.x) {
        const gblod_node g = nodes[i];
        const uint64_t p0 = g.point_first;
        const uint32_t m = g.point_count;
        // ranges of the finite weights and smoothing lengths
        Red6 r;
        r.v[0] = r.v[1] = r.v[2] = INFINITY;
        r.v[3] = r.v[4] = r.v[5] = -INFINITY;
        for (uint32_t j = threadIdx.x; j < m; j += QT) {
            const float w = pts4[p0 + j].w, h = hs[p0 + j];
            if (isfinite(w)) {
                r.v[0] = w < r.v[0] ? w : r.v[0];
                r.v[3] = w > r.v[3] ? w : r.v[3];
            }
            if (isfinite(h)) {
                r.v[1] = h < r.v[1] ? h : r.v[1];
                r.v[4] = h > r.v[4] ? h : r.v[4];
            }
        }
        r = block_minmax6(r, sm);
        if (threadIdx.x == 0) {
            // the node's cell from its locational code
            const int d = g.depth;
            const uint64_t path = g.code ^ (1ull << (3 * d));
            uint32_t q[3] = {0u, 0u, 0u};
            for (int l = 0; l < d; ++l) {
                const uint32_t o = (uint32_t)((path >> (3 * (d - 1 - l))) & 7ull);
                q[0] = (q[0] << 1) | ((o >> 2) & 1u);
                q[1] = (q[1] << 1) | ((o >> 1) & 1u);
                q[2] = (q[2] << 1) | (o & 1u);
            }
            const double e = ldexp(side, -d);
            float4 A, B;
            A.x = __double2float_rn(__dadd_rn(lo0, __dmul_rn(e, (double)q[0])));
            A.y = __double2float_rn(__dadd_rn(lo1, __dmul_rn(e, (double)q[1])));
            A.z = __double2float_rn(__dadd_rn(lo2, __dmul_rn(e, (double)q[2])));
            A.w = __double2float_rn(ldexp(e, -16));
            lin_range(r.v[0], r.v[3], B.x, B.y);
            lin_range(r.v[1], r.v[4], B.z, B.w);
            sA = A;
            sB = B;
            qa[2 * i] = A;
            qa[2 * i + 1] = B;
        }
        __syncthreads();
        const float4 A = sA, B = sB;
        // code, decode, and reduce the decoded bounds and the largest decoded h
        Red6 b;
        b.v[0] = b.v[1] = b.v[2] = INFINITY;
        b.v[3] = b.v[4] = b.v[5] = -INFINITY;
        float hm = 0.0f;
        for (uint32_t j = threadIdx.x; j < m; j += QT) {
            const float4 p = pts4[p0 + j];
            const float h = hs[p0 + j];
            ushort4 c;
            c.x = (unsigned short)code_floor(p.x, A.x, A.w);
            c.y = (unsigned short)code_floor(p.y, A.y, A.w);
            c.z = (unsigned short)code_floor(p.z, A.z, A.w);
            c.w = (unsigned short)code_rne(h, B.z, B.w);
            const uint32_t cw = code_rne(p.w, B.x, B.y);
            q4[p0 + j] = c;
            qw[p0 + j] = (uint16_t)cw;
            float x, y, z, w, hd;
            block_decode(c, cw, A, B, x, y, z, w, hd);
            b.v[0] = x < b.v[0] ? x : b.v[0];
            b.v[1] = y < b.v[1] ? y : b.v[1];
            b.v[2] = z < b.v[2] ? z : b.v[2];
            b.v[3] = x > b.v[3] ? x : b.v[3];
            b.v[4] = y > b.v[4] ? y : b.v[4];
            b.v[5] = z > b.v[5] ? z : b.v[5];
            hm = hd > hm ? hd : hm;
        }
        b = block_minmax6(b, sm);
        for (int d = 16; d > 0; d >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, hm, d);
            hm = o > hm ? o : hm;
        }
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = hm;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < QT / 32; ++w) hm = sm[w] > hm ? sm[w] : hm;
            for (int k = 0; k < 6; ++k) own[7 * i + k] = b.v[k];
            own[7 * i + 6] = hm;
        }
        __syncthreads();
    }
}

// one level, deepest first: subtree bounds and h_cull of the decoded points
__global__ void k_block_bottom_up(uint64_t L, uint32_t nd, const gblod_node *__restrict__ nodes,
                                  const float *__restrict__ own, gblod_node *qnodes)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd) return;
    const uint64_t i = L + t;
    gblod_node g = nodes[i];
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = own[7 * i + a];
        mx[a] = own[7 * i + 3 + a];
    }
    float hm = own[7 * i + 6];
    if (g.flags & GBLOD_NODE_INTERNAL)
        for (uint32_t k = g.child_first; k < g.child_first + g.child_count; ++k) {
            const gblod_node &c = qnodes[k];
            for (int a = 0; a < 3; ++a) {
                mn[a] = c.bmin[a] < mn[a] ? c.bmin[a] : mn[a];
                mx[a] = c.bmax[a] > mx[a] ? c.bmax[a] : mx[a];
            }
            hm = c.h_cull > hm ? c.h_cull : hm;
        }
    for (int a = 0; a < 3; ++a) {
        g.bmin[a] = mn[a];
        g.bmax[a] = mx[a];
    }
    g.h_cull = hm;
    qnodes[i] = g;
}

} // namespace

void block_quantize(gblod_octree *o, uint32_t flags, cudaStream_t s)
{
    const Allocator &A = o->A;
    if (!o->has_block16) {
        if (!o->has_float) fail(GBLOD_ERR_INVALID_ARG, "octree holds neither fp32 points nor codes");
        const size_t nn = o->n_nodes, np = o->n_points;
        if (nn) {
            o->q4 = static_cast<ushort4 *>(A.get(np * sizeof(ushort4), s));
            o->qw = static_cast<uint16_t *>(A.get(np * sizeof(uint16_t), s));
            o->qa = static_cast<float4 *>(A.get(2 * nn * sizeof(float4), s));
            o->qnodes = static_cast<gblod_node *>(A.get(nn * sizeof(gblod_node), s));
            Scratch<float> own(A, 7 * nn, s);
            const unsigned G = (unsigned)std::min<size_t>(nn, (size_t)persistent_blocks(8));
            launch(GBLOD_K_BUILD_OTHER, k_block_encode, dim3(G), dim3(QT), 0, s, nn, (const gblod_node *)o->nodes,
                   (const float4 *)o->pts4, (const float *)o->hs, o->lo[0], o->lo[1], o->lo[2], o->side, o->q4,
                   o->qw, o->qa, own.p);
            for (int d = o->depth_max; d >= 0; --d) {
                const uint64_t L = o->level_first[d];
                const uint32_t n = (uint32_t)(o->level_first[d + 1] - L);
                launch(GBLOD_K_BUILD_OTHER, k_block_bottom_up, dim3((n + 255) / 256), dim3(256), 0, s, L, n,
                       (const gblod_node *)o->nodes, (const float *)own.p, o->qnodes);
            }
            GB_CUDA(cudaStreamSynchronize(s));
        }
        o->has_block16 = true;
        o->bytes += np * (sizeof(ushort4) + sizeof(uint16_t)) + nn * (2 * sizeof(float4) + sizeof(gblod_node));
    }
    if ((flags & GBLOD_QUANTIZE_DROP_FLOAT) && o->has_float) {
        GB_CUDA(cudaStreamSynchronize(s));
        A.put(o->pts4, o->n_points * sizeof(float4), o->stream);
        A.put(o->hs, o->n_points * sizeof(float), o->stream);
        o->pts4 = nullptr;
        o->hs = nullptr;
        o->has_float = false;
        o->bytes -= o->n_points * (sizeof(float4) + sizeof(float));
    }
}

} // namespace gb
