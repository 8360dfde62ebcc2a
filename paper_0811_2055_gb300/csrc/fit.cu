// Access to one node's stored points, for fitting its representatives (abstract: an LOD image
// "indistinguishable from a full rendering"): read the points and the member particles of a node,
// and write fitted points back.  The node's particle bounds and h_cull, and those of every
// ancestor, grow to cover the written points, so the view-frustum cull (which tests a node's
// bounds grown by the blob radius of its subtree's largest smoothing length) stays conservative.
#include "octree.cuh"

namespace gb {
namespace {

constexpr int FT = 256;

// a coordinate or smoothing length as it enters the bounds: -0 is stored as +0, so the bounds do
// not depend on which zero a reduction meets first
__device__ __forceinline__ float bound_value(float v) { return __fadd_rn(v, 0.0f); }

__global__ void __launch_bounds__(FT) k_union_bounds(gblod_node *__restrict__ nodes, uint32_t node,
                                                     const float4 *__restrict__ pts4, const float *__restrict__ hs,
                                                     uint32_t count)
{
    __shared__ float red[7][FT];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, hm = -INFINITY;
    for (uint32_t i = threadIdx.x; i < count; i += FT) {
        const float4 p = pts4[i];
        const float v[3] = {bound_value(p.x), bound_value(p.y), bound_value(p.z)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = v[a] < mn[a] ? v[a] : mn[a];
            mx[a] = v[a] > mx[a] ? v[a] : mx[a];
        }
        const float h = bound_value(hs[i]);
        hm = h > hm ? h : hm;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = mn[a];
        red[3 + a][threadIdx.x] = mx[a];
    }
    red[6][threadIdx.x] = hm;
    __syncthreads();
    for (int w = FT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float o = red[a][threadIdx.x + w], p = red[3 + a][threadIdx.x + w];
                red[a][threadIdx.x] = o < red[a][threadIdx.x] ? o : red[a][threadIdx.x];
                red[3 + a][threadIdx.x] = p > red[3 + a][threadIdx.x] ? p : red[3 + a][threadIdx.x];
            }
            const float q = red[6][threadIdx.x + w];
            red[6][threadIdx.x] = q > red[6][threadIdx.x] ? q : red[6][threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0 || count == 0) return;
    // the node and every ancestor (at most 22 of them)
    for (int32_t k = (int32_t)node; k >= 0; k = nodes[k].parent) {
        gblod_node &g = nodes[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g.bmin[a] = red[a][0] < g.bmin[a] ? red[a][0] : g.bmin[a];
            g.bmax[a] = red[3 + a][0] > g.bmax[a] ? red[3 + a][0] : g.bmax[a];
        }
        g.h_cull = red[6][0] > g.h_cull ? red[6][0] : g.h_cull;
    }
}

gblod_node read_node(const gblod_octree *o, uint32_t node, cudaStream_t s)
{
    if (node >= o->n_nodes) fail(GBLOD_ERR_INVALID_ARG, "node index out of range");
    gblod_node g;
    GB_CUDA(cudaMemcpyAsync(&g, o->nodes + node, sizeof(g), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return g;
}

void drop_block16(gblod_octree *o, cudaStream_t s)
{
    if (!o->has_block16) return;
    o->A.put(o->q4, o->n_points * sizeof(ushort4), s);
    o->A.put(o->qw, o->n_points * sizeof(uint16_t), s);
    o->A.put(o->qa, 2 * o->n_nodes * sizeof(float4), s);
    o->A.put(o->qnodes, o->n_nodes * sizeof(gblod_node), s);
    o->bytes -= o->n_points * (sizeof(ushort4) + sizeof(uint16_t)) + o->n_nodes * (2 * sizeof(float4) + sizeof(gblod_node));
    o->q4 = nullptr;
    o->qw = nullptr;
    o->qa = nullptr;
    o->qnodes = nullptr;
    o->has_block16 = false;
}

} // namespace
} // namespace gb

using namespace gb;

extern "C" {

gblod_status gblod_octree_node_points(const gblod_octree *o, uint32_t node, float *d_pts4, float *d_hs,
                                      uint32_t *count, void *stream)
{
    try {
        if (!o || !count) fail(GBLOD_ERR_INVALID_ARG, "octree and count must not be NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const gblod_node g = read_node(o, node, s);
        if ((d_pts4 || d_hs) && !o->has_float)
            fail(GBLOD_ERR_INVALID_ARG, "octree holds no fp32 points (dropped after quantisation)");
        if (d_pts4 && g.point_count)
            GB_CUDA(cudaMemcpyAsync(d_pts4, o->pts4 + g.point_first, (size_t)g.point_count * sizeof(float4),
                                    cudaMemcpyDeviceToDevice, s));
        if (d_hs && g.point_count)
            GB_CUDA(cudaMemcpyAsync(d_hs, o->hs + g.point_first, (size_t)g.point_count * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s));
        *count = g.point_count;
        return GBLOD_OK;
    } catch (const Error &e) {
        return e.st;
    }
}

gblod_status gblod_octree_node_members(const gblod_octree *o, uint32_t node, uint32_t *d_ids, uint32_t *count,
                                       void *stream)
{
    try {
        if (!o || !count) fail(GBLOD_ERR_INVALID_ARG, "octree and count must not be NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const gblod_node g = read_node(o, node, s);
        if (d_ids && g.seg_count)
            GB_CUDA(cudaMemcpyAsync(d_ids, o->sidx + g.seg_first, (size_t)g.seg_count * sizeof(uint32_t),
                                    cudaMemcpyDeviceToDevice, s));
        *count = g.seg_count;
        return GBLOD_OK;
    } catch (const Error &e) {
        return e.st;
    }
}

gblod_status gblod_octree_set_points(gblod_octree *o, uint32_t node, const float *d_pts4, const float *d_hs,
                                     uint32_t count, void *stream)
{
    try {
        if (!o || !d_pts4 || !d_hs) fail(GBLOD_ERR_INVALID_ARG, "octree and point arrays must not be NULL");
        if (!o->has_float) fail(GBLOD_ERR_INVALID_ARG, "octree holds no fp32 points (dropped after quantisation)");
        cudaStream_t s = (cudaStream_t)stream;
        const gblod_node g = read_node(o, node, s);
        if (count != g.point_count)
            fail(GBLOD_ERR_INVALID_ARG, "count must equal the node's stored point count (" +
                                            std::to_string(g.point_count) + ")");
        if (count == 0) return GBLOD_OK;
        GB_CUDA(cudaMemcpyAsync(o->pts4 + g.point_first, d_pts4, (size_t)count * sizeof(float4),
                                cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaMemcpyAsync(o->hs + g.point_first, d_hs, (size_t)count * sizeof(float), cudaMemcpyDeviceToDevice,
                                s));
        // written points copy no input particle
        GB_CUDA(cudaMemsetAsync(o->pt_src + g.point_first, 0xFF, (size_t)count * sizeof(uint32_t), s));
        launch(GBLOD_K_BUILD_OTHER, k_union_bounds, dim3(1), dim3(FT), 0, s, o->nodes, node,
               (const float4 *)(o->pts4 + g.point_first), (const float *)(o->hs + g.point_first), count);
        drop_block16(o, s);
        GB_CUDA(cudaStreamSynchronize(s));
        return GBLOD_OK;
    } catch (const Error &e) {
        return e.st;
    }
}

} // extern "C"
