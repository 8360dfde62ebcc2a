// The device-resident octree and the build / selection entry points shared by the C ABI.
#pragma once

#include <vector>

#include "common.cuh"

struct gblod_octree {
    gb::Allocator A;
    cudaStream_t stream = nullptr; // stream the memory was allocated on
    uint64_t n = 0, n_nodes = 0, n_points = 0;
    int depth_max = 0;
    int equal_mass = 1;
    uint32_t n_max = 0;
    uint64_t seed = 0;
    double lo[3] = {0, 0, 0};
    double side = 1.0;
    gblod_node *nodes = nullptr; // n_nodes, breadth first
    float4 *pts4 = nullptr;      // n_points (x, y, z, weight)
    float *hs = nullptr;         // n_points
    uint32_t *pt_src = nullptr;  // n_points: sorted position each point copies
    uint64_t *skey = nullptr;    // n: sorted Morton keys
    uint32_t *sidx = nullptr;    // n: input index per sorted position
    std::vector<uint64_t> level_first; // host: first node index of every depth, plus the end
    size_t bytes = 0;
    // 16-bit block codes (gblod_octree_quantize); null until coded
    ushort4 *q4 = nullptr;      // n_points: position codes x, y, z and the h code
    uint16_t *qw = nullptr;     // n_points: weight code
    float4 *qa = nullptr;       // 2 per node: (qlo x, y, z, qstep), (w lo, w step, h lo, h step)
    gblod_node *qnodes = nullptr; // node table with bounds and h_cull of the decoded subtrees
    bool has_float = true, has_block16 = false;
};

namespace gb {

gblod_octree *build_octree(const float *xyz, const float *mass, const float *h, const uint32_t *ids, uint64_t n,
                           const gblod_build_params &p, const Allocator &A, cudaStream_t s);
void free_octree(gblod_octree *o);

// Codes every stored point (16-bit block codes); GBLOD_QUANTIZE_DROP_FLOAT frees the fp32 points.
void block_quantize(gblod_octree *o, uint32_t flags, cudaStream_t s);

// Decoding of the 16-bit block codes: one IEEE round-to-nearest per operation, no FMA.
__device__ __forceinline__ float block_decode_pos(uint32_t c, float lo, float step)
{
    return __fadd_rn(lo, __fmul_rn(__fadd_rn(__uint2float_rn(c), 0.5f), step));
}
__device__ __forceinline__ float block_decode_lin(uint32_t c, float lo, float step)
{
    return __fadd_rn(lo, __fmul_rn(__uint2float_rn(c), step));
}
__device__ __forceinline__ void block_decode(const ushort4 q, uint32_t cw, const float4 A, const float4 B, float &x,
                                             float &y, float &z, float &w, float &h)
{
    x = block_decode_pos(q.x, A.x, A.w);
    y = block_decode_pos(q.y, A.y, A.w);
    z = block_decode_pos(q.z, A.z, A.w);
    w = block_decode_lin(cw, B.x, B.y);
    h = block_decode_lin(q.w, B.z, B.w);
}

// Work arrays the subselection reads and writes (all device pointers).
struct SelectIn {
    const float4 *s4;        // sorted particles (x, y, z, mass)
    const float *sh;         // sorted smoothing lengths
    const uint32_t *sid;     // sorted ids
    const uint64_t *ncode;   // per node
    const uint32_t *nfirst;  // per node
    const uint32_t *ncount;  // per node
    const uint64_t *npfirst; // per node: first stored point
    const float *nw;         // per node: representative weight
    const float *ns;         // per node: smoothing-length scale
    unsigned int *nhmax;     // per node: float bits of the largest representative h (atomicMax)
    float4 *pts4;
    float *hs;
    uint32_t *pt_src;
    uint32_t n_max;
};

// A4 + A5 for every node whose index is listed in rep_nodes (device, n_rep entries).
void select_representatives(const Allocator &A, cudaStream_t s, HostStage &hs, ScanTmp &scan, const SelectIn &in,
                            const uint32_t *rep_nodes, uint32_t n_rep, uint32_t n_max, uint64_t seed,
                            int equal_mass);

} // namespace gb
