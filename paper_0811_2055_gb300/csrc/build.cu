// Octree build on the device (octree paragraph of the paper): A1 Morton keys, A2 radix sort,
// A3 per-node counting level by level, then the node table, exact node masses, leaf blocks and
// the bottom-up cull data.  The subselection (A4/A5) lives in select.cu.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lodmath.cuh"
#include "octree.cuh"

namespace gb {
namespace {

constexpr uint32_t FL_LEAF = GBLOD_NODE_LEAF, FL_INTERNAL = GBLOD_NODE_INTERNAL, FL_LOSSY = GBLOD_NODE_LOSSY,
                   FL_REPS = GBLOD_NODE_REPS;

inline unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ------------------------------------------------------------------ A1 and input checks
__global__ void k_mass_check(const float *mass, size_t n, unsigned *minb, unsigned *maxb, unsigned *bad)
{
    unsigned lo = 0xFFFFFFFFu, hi = 0u, nbad = 0u;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float m = mass[i];
        if (!(m >= 0x1p-24f && m <= 0x1p+24f)) {
            nbad = 1u;
            continue;
        }
        const unsigned b = __float_as_uint(m);
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
        nbad |= __shfl_xor_sync(0xffffffffu, nbad, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(minb, lo);
        atomicMax(maxb, hi);
        if (nbad) atomicOr(bad, 1u);
    }
}

// pow2: the root cube starts at 0 and scale is a power of two in fp32 range (the fp32 product is exact)
__global__ void k_morton(const float *__restrict__ xyz, const uint32_t *__restrict__ order, size_t n, double lx,
                         double ly, double lz, double scale, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                         int pow2)
{
    const float sf = (float)scale;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t src = order ? (size_t)order[i] : i;
        const float x = xyz[3 * src], y = xyz[3 * src + 1], z = xyz[3 * src + 2];
        keys[i] = pow2 ? gbd::morton_key_pow2(x, y, z, sf) : gbd::morton_key(x, y, z, lx, ly, lz, scale);
        if (!order) vals[i] = (uint32_t)i;
    }
}

__global__ void k_id_keys(const uint32_t *ids, size_t n, uint64_t *keys, uint32_t *vals)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        keys[i] = ids[i];
        vals[i] = (uint32_t)i;
    }
}

// Particles in sorted order: s4 = (x, y, z, m), sh = h, sid = the caller's id (written only when
// the caller gave ids: otherwise it equals perm), mfix = the fixed-point mass (written only for
// unequal masses: with one mass m0 for all, a node's exact mass is its count times m0's, and the
// mass array is not read).
__global__ void k_gather_sorted(const float *__restrict__ xyz, const float *__restrict__ mass,
                                const float *__restrict__ h, const uint32_t *__restrict__ ids,
                                const uint32_t *__restrict__ perm, size_t n, float4 *__restrict__ s4,
                                float *__restrict__ sh, uint32_t *__restrict__ sid, U128 *__restrict__ mfix,
                                int equal_mass, float m0)
{
    // four independent elements per thread and iteration (each a coalesced sweep of the sorted
    // order), so that four random reads of the particle arrays are in flight at a time
    constexpr int GU = 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < n; j0 += stride * GU) {
        size_t i[GU];
        float x[GU], y[GU], z[GU], m[GU], hh[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const size_t j = j0 + u * stride;
            i[u] = j < n ? (size_t)perm[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            if (j0 + u * stride < n) {
                x[u] = xyz[3 * i[u]];
                y[u] = xyz[3 * i[u] + 1];
                z[u] = xyz[3 * i[u] + 2];
                m[u] = equal_mass ? m0 : mass[i[u]];
                hh[u] = h[i[u]];
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const size_t j = j0 + u * stride;
            if (j < n) {
                s4[j] = make_float4(x[u], y[u], z[u], m[u]);
                sh[j] = hh[u];
                if (sid) sid[j] = ids[i[u]];
                if (mfix) mfix[j] = gbd::mass_fixed(m[u]);
            }
        }
    }
}

// ------------------------------------------------------------------ A3 levels
__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t *a, uint32_t lo, uint32_t hi, uint64_t v)
{
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_child_counts(const uint64_t *__restrict__ skey, const uint64_t *__restrict__ code,
                               const uint32_t *__restrict__ first, const uint32_t *__restrict__ count, uint64_t L,
                               uint32_t nd, int d, uint32_t n_max, uint32_t *cc, uint32_t *cf, uint32_t *nz)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nd * 8) return;
    const uint64_t node = L + (t >> 3);
    const uint32_t o = (uint32_t)(t & 7);
    const uint32_t c = count[node];
    if (c > n_max && d < GBLOD_MAX_DEPTH) {
        const uint64_t pfx = code[node] ^ (1ull << (3 * d));
        const uint64_t cp = (pfx << 3) | o;
        const int sh = 60 - 3 * d;
        const uint32_t b = first[node], e = b + c;
        const uint32_t lo = lower_bound_u64(skey, b, e, cp << sh);
        const uint32_t hi = lower_bound_u64(skey, lo, e, (cp + 1) << sh);
        cc[t] = hi - lo;
        cf[t] = lo;
        nz[t] = hi > lo ? 1u : 0u;
    } else {
        cc[t] = 0u;
        cf[t] = 0u;
        nz[t] = 0u;
    }
}

struct NodeSoA {
    uint64_t *code;
    uint32_t *first, *count, *child_first, *child_count;
    int32_t *depth, *parent;
};

__global__ void k_emit_children(NodeSoA N, const uint32_t *__restrict__ cc, const uint32_t *__restrict__ cf,
                                const uint32_t *__restrict__ slot, uint64_t L, uint32_t nd, int d, uint64_t Lnext)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nd * 8) return;
    const uint64_t parent = L + (t >> 3);
    if (cc[t]) {
        const uint64_t j = Lnext + slot[t];
        N.code[j] = N.code[parent] * 8 + (t & 7);
        N.first[j] = cf[t];
        N.count[j] = cc[t];
        N.depth[j] = d + 1;
        N.parent[j] = (int32_t)parent;
        N.child_first[j] = 0u;
        N.child_count[j] = 0u;
    }
    if ((t & 7) == 0) {
        uint32_t k = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) k += cc[t + q] ? 1u : 0u;
        N.child_first[parent] = k ? (uint32_t)(Lnext + slot[t]) : 0u;
        N.child_count[parent] = k;
    }
}

// ------------------------------------------------------------------ node table
__global__ void k_node_classify(size_t nn, const uint32_t *count, const int32_t *depth, uint32_t n_max,
                                uint32_t *flags, uint64_t *pcount, uint32_t *isrep)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const uint32_t c = count[i];
    uint32_t f;
    if (c > n_max)
        f = depth[i] < GBLOD_MAX_DEPTH ? (FL_INTERNAL | FL_REPS) : (FL_LOSSY | FL_REPS);
    else
        f = FL_LEAF;
    flags[i] = f;
    pcount[i] = (f & FL_REPS) ? n_max : c;
    isrep[i] = (f & FL_REPS) ? 1u : 0u;
}

__global__ void k_compact_reps(size_t nn, const uint32_t *isrep, const uint32_t *pos, uint32_t *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nn && isrep[i]) out[pos[i]] = (uint32_t)i;
}

// Node mass from the exclusive prefix of mass * 2^47; representative weight and h scale.
// Exact node masses: prefix differences of the fixed-point masses, or (prefix null: one mass m0
// for every particle) count times m0's fixed-point value.
__global__ void k_node_mass(size_t nn, size_t n, const uint32_t *first, const uint32_t *count, const uint32_t *flags,
                            const U128 *prefix, const U128 *total, float m0, uint32_t n_max, uint64_t *mlo,
                            uint64_t *mhi, float *w, float *s)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    U128 M;
    if (prefix) {
        const size_t b = first[i], e = b + count[i];
        const U128 a = prefix[b];
        const U128 z = e < n ? prefix[e] : *total;
        M = gbd::sub128(z, a);
    } else {
        const U128 f = gbd::mass_fixed(m0); // < 2^71, times a count < 2^32
        M.lo = f.lo * count[i];
        M.hi = f.hi * count[i] + __umul64hi(f.lo, (uint64_t)count[i]);
    }
    mlo[i] = M.lo;
    mhi[i] = M.hi;
    if (flags[i] & FL_REPS) {
        const double Md =
            __dmul_rn(__dadd_rn(__dmul_rn(__ull2double_rn(M.hi), 0x1p64), __ull2double_rn(M.lo)), 0x1p-47);
        w[i] = __double2float_rn(__ddiv_rn(Md, (double)n_max));
        const double t = __ddiv_rn((double)count[i], (double)n_max);
        s[i] = __double2float_rn(gbd::cube_root_ge1(t));
    } else {
        w[i] = 0.0f;
        s[i] = 1.0f;
    }
}

// Leaves: copy the sorted particles into the node block; every non-internal node: particle
// bounds; leaves: largest h.  One block per node (grid-stride), NaN coordinates are skipped.
__global__ void k_leaf_nodes(size_t nn, const uint32_t *__restrict__ flags, const uint32_t *__restrict__ first,
                             const uint32_t *__restrict__ count, const uint64_t *__restrict__ pfirst,
                             const float4 *__restrict__ s4, const float *__restrict__ sh, float4 *__restrict__ pts4,
                             float *__restrict__ hs, uint32_t *__restrict__ pt_src, float *__restrict__ bmin,
                             float *__restrict__ bmax, unsigned *__restrict__ hmax_bits)
{
    __shared__ float red[7][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (size_t node = blockIdx.x; node < nn; node += gridDim.x) {
        const uint32_t f = flags[node];
        if (f & FL_INTERNAL) continue;
        const uint32_t b = first[node], c = count[node];
        const uint64_t pf = pfirst[node];
        float mn0 = INFINITY, mn1 = INFINITY, mn2 = INFINITY, mx0 = -INFINITY, mx1 = -INFINITY, mx2 = -INFINITY;
        float hm = 0.0f;
        const bool leaf = (f & FL_LEAF) != 0;
        for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
            const float4 p = s4[b + k];
            mn0 = fminf(mn0, p.x);
            mn1 = fminf(mn1, p.y);
            mn2 = fminf(mn2, p.z);
            mx0 = fmaxf(mx0, p.x);
            mx1 = fmaxf(mx1, p.y);
            mx2 = fmaxf(mx2, p.z);
            if (leaf) {
                const float h = sh[b + k];
                pts4[pf + k] = p;
                hs[pf + k] = h;
                pt_src[pf + k] = b + k;
                hm = h > hm ? h : hm;
            }
        }
        for (int d = 16; d > 0; d >>= 1) {
            mn0 = fminf(mn0, __shfl_xor_sync(0xffffffffu, mn0, d));
            mn1 = fminf(mn1, __shfl_xor_sync(0xffffffffu, mn1, d));
            mn2 = fminf(mn2, __shfl_xor_sync(0xffffffffu, mn2, d));
            mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, d));
            mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, d));
            mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, d));
            const float o = __shfl_xor_sync(0xffffffffu, hm, d);
            hm = o > hm ? o : hm;
        }
        if (lane == 0) {
            red[0][warp] = mn0; red[1][warp] = mn1; red[2][warp] = mn2;
            red[3][warp] = mx0; red[4][warp] = mx1; red[5][warp] = mx2;
            red[6][warp] = hm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w) {
                mn0 = fminf(mn0, red[0][w]); mn1 = fminf(mn1, red[1][w]); mn2 = fminf(mn2, red[2][w]);
                mx0 = fmaxf(mx0, red[3][w]); mx1 = fmaxf(mx1, red[4][w]); mx2 = fmaxf(mx2, red[5][w]);
                hm = red[6][w] > hm ? red[6][w] : hm;
            }
            bmin[3 * node] = mn0; bmin[3 * node + 1] = mn1; bmin[3 * node + 2] = mn2;
            bmax[3 * node] = mx0; bmax[3 * node + 1] = mx1; bmax[3 * node + 2] = mx2;
            if (leaf) hmax_bits[node] = __float_as_uint(hm);
        }
        __syncthreads();
    }
}

// One level, deepest first: cull radius and bounds of every node of the level.
__global__ void k_bottom_up(uint64_t L, uint32_t nd, const uint32_t *flags, const uint32_t *child_first,
                            const uint32_t *child_count, float *bmin, float *bmax, const unsigned *hmax_bits,
                            float *hcull)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd) return;
    const uint64_t i = L + t;
    float h = __uint_as_float(hmax_bits[i]);
    if (flags[i] & FL_INTERNAL) {
        float mn0 = INFINITY, mn1 = INFINITY, mn2 = INFINITY, mx0 = -INFINITY, mx1 = -INFINITY, mx2 = -INFINITY;
        const uint32_t k0 = child_first[i], kc = child_count[i];
        for (uint32_t k = k0; k < k0 + kc; ++k) {
            mn0 = fminf(mn0, bmin[3 * k]); mn1 = fminf(mn1, bmin[3 * k + 1]); mn2 = fminf(mn2, bmin[3 * k + 2]);
            mx0 = fmaxf(mx0, bmax[3 * k]); mx1 = fmaxf(mx1, bmax[3 * k + 1]); mx2 = fmaxf(mx2, bmax[3 * k + 2]);
            const float hc = hcull[k];
            h = hc > h ? hc : h;
        }
        bmin[3 * i] = mn0; bmin[3 * i + 1] = mn1; bmin[3 * i + 2] = mn2;
        bmax[3 * i] = mx0; bmax[3 * i + 1] = mx1; bmax[3 * i + 2] = mx2;
    }
    hcull[i] = h;
}

struct PackIn {
    const uint64_t *code, *pfirst, *mlo, *mhi;
    const uint32_t *first, *count, *child_first, *child_count, *flags;
    const int32_t *depth, *parent;
    const float *hcull, *w, *s, *bmin, *bmax;
    uint32_t n_max;
};

__global__ void k_pack_nodes(size_t nn, PackIn P, gblod_node *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    gblod_node g;
    g.code = P.code[i];
    g.seg_first = P.first[i];
    g.point_first = P.pfirst[i];
    g.mass_lo = P.mlo[i];
    g.mass_hi = P.mhi[i];
    g.seg_count = P.count[i];
    g.point_count = (P.flags[i] & FL_REPS) ? P.n_max : P.count[i];
    g.child_first = P.child_first[i];
    g.child_count = P.child_count[i];
    g.depth = P.depth[i];
    g.flags = (int32_t)P.flags[i];
    g.parent = P.parent[i];
    g.pad = 0;
    g.h_cull = P.hcull[i];
    g.w_rep = P.w[i];
    g.s_rep = P.s[i];
    g.pad2 = 0.0f;
    for (int a = 0; a < 3; ++a) {
        g.bmin[a] = P.bmin[3 * i + a];
        g.bmax[a] = P.bmax[3 * i + a];
    }
    out[i] = g;
}

// growable node arrays (structure of arrays), contents kept on growth
struct NodeStore {
    DBuf<uint64_t> code;
    DBuf<uint32_t> first, count, child_first, child_count;
    DBuf<int32_t> depth, parent;
    size_t cap = 0;

    template <class T> static void grow1(const Allocator &A, DBuf<T> &b, size_t used, size_t want, cudaStream_t s)
    {
        T *np = static_cast<T *>(A.get(want * sizeof(T), s));
        if (b.p && used) GB_CUDA(cudaMemcpyAsync(np, b.p, used * sizeof(T), cudaMemcpyDeviceToDevice, s));
        if (b.p) A.put(b.p, b.cap * sizeof(T), s);
        b.p = np;
        b.cap = want;
    }
    void reserve(const Allocator &A, size_t used, size_t need, cudaStream_t s)
    {
        if (need <= cap) return;
        size_t want = std::max(need, cap * 2);
        grow1(A, code, used, want, s);
        grow1(A, first, used, want, s);
        grow1(A, count, used, want, s);
        grow1(A, child_first, used, want, s);
        grow1(A, child_count, used, want, s);
        grow1(A, depth, used, want, s);
        grow1(A, parent, used, want, s);
        cap = want;
    }
    NodeSoA soa() { return NodeSoA{code.p, first.p, count.p, child_first.p, child_count.p, depth.p, parent.p}; }
    void release(const Allocator &A, cudaStream_t s)
    {
        code.release(A, s); first.release(A, s); count.release(A, s); child_first.release(A, s);
        child_count.release(A, s); depth.release(A, s); parent.release(A, s);
    }
};

__global__ void k_init_root(NodeSoA N, uint32_t n)
{
    N.code[0] = 1ull;
    N.first[0] = 0u;
    N.count[0] = n;
    N.depth[0] = 0;
    N.parent[0] = -1;
    N.child_first[0] = 0u;
    N.child_count[0] = 0u;
}

template <class T> T read1(const T *d, cudaStream_t s, HostStage &hs)
{
    T *h = static_cast<T *>(hs.get(sizeof(T)));
    GB_CUDA(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return *h;
}

} // namespace

void free_octree(gblod_octree *o)
{
    if (!o) return;
    cudaStream_t s = o->stream;
    o->A.put(o->nodes, o->n_nodes * sizeof(gblod_node), s);
    o->A.put(o->pts4, o->n_points * sizeof(float4), s);
    o->A.put(o->hs, o->n_points * sizeof(float), s);
    o->A.put(o->pt_src, o->n_points * sizeof(uint32_t), s);
    o->A.put(o->skey, o->n * sizeof(uint64_t), s);
    o->A.put(o->sidx, o->n * sizeof(uint32_t), s);
    o->A.put(o->q4, o->n_points * sizeof(ushort4), s);
    o->A.put(o->qw, o->n_points * sizeof(uint16_t), s);
    o->A.put(o->qa, 2 * o->n_nodes * sizeof(float4), s);
    o->A.put(o->qnodes, o->n_nodes * sizeof(gblod_node), s);
    delete o;
}

namespace {
struct BuildTemps {
    const Allocator &A;
    cudaStream_t s;
    ScanTmp scan;
    SortTmp sort;
    NodeStore N;
    DBuf<uint32_t> cc, cf, nz, slot;
    BuildTemps(const Allocator &a, cudaStream_t st) : A(a), s(st) {}
    ~BuildTemps()
    {
        N.release(A, s);
        cc.release(A, s); cf.release(A, s); nz.release(A, s); slot.release(A, s);
        scan.buf.release(A, s);
        sort.buf.release(A, s);
        sort.scan.buf.release(A, s);
    }
};
} // namespace

static gblod_octree *build_octree_impl(gblod_octree *o, const float *xyz, const float *mass, const float *h,
                                       const uint32_t *ids, uint64_t n, const gblod_build_params &p,
                                       const Allocator &A, cudaStream_t s);

gblod_octree *build_octree(const float *xyz, const float *mass, const float *h, const uint32_t *ids, uint64_t n,
                           const gblod_build_params &p, const Allocator &A, cudaStream_t s)
{
    gblod_octree *o = new gblod_octree();
    try {
        return build_octree_impl(o, xyz, mass, h, ids, n, p, A, s);
    } catch (...) {
        (void)cudaStreamSynchronize(s);
        free_octree(o);
        throw;
    }
}

static gblod_octree *build_octree_impl(gblod_octree *o, const float *xyz, const float *mass, const float *h,
                                       const uint32_t *ids, uint64_t n, const gblod_build_params &p,
                                       const Allocator &A, cudaStream_t s)
{
    HostStage hs;
    BuildTemps tmp(A, s);
    ScanTmp &scan = tmp.scan;
    SortTmp &sort = tmp.sort;
    o->A = A;
    o->stream = s;
    o->n = n;
    o->n_max = p.n_max;
    o->seed = p.seed;
    for (int a = 0; a < 3; ++a) o->lo[a] = p.root_lo[a];
    o->side = p.root_side;
    if (n == 0) {
        o->level_first = {0};
        return o;
    }
    const int T = 256;
    const unsigned G = (unsigned)persistent_blocks(8);
    float m0 = 0.0f; // the common mass when all are equal

    // masses: range and whether they are all equal
    {
        Scratch<unsigned> mm(A, 3, s);
        const unsigned init[3] = {0xFFFFFFFFu, 0u, 0u};
        GB_CUDA(cudaMemcpyAsync(mm.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
        launch(GBLOD_K_BUILD_OTHER, k_mass_check, dim3(G), dim3(T), 0, s, mass, (size_t)n, mm.p, mm.p + 1, mm.p + 2);
        unsigned *hm = static_cast<unsigned *>(hs.get(3 * sizeof(unsigned)));
        GB_CUDA(cudaMemcpyAsync(hm, mm.p, 3 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        if (hm[2]) fail(GBLOD_ERR_RANGE, "gblod_build_lod: every mass must be finite and in [2^-24, 2^24]");
        o->equal_mass = hm[0] == hm[1] ? 1 : 0;
        std::memcpy(&m0, &hm[0], sizeof(float));
    }

    // A1 + A2: keys in (key, id) order
    Scratch<uint64_t> keyA(A, n, s), keyB(A, n, s);
    Scratch<uint32_t> valA(A, n, s), valB(A, n, s);
    uint64_t *keys = keyA.p;
    uint32_t *vals = valA.p;
    const double scale = 2097152.0 / p.root_side;
    int sexp = 0;
    const int pow2 = p.root_lo[0] == 0.0 && p.root_lo[1] == 0.0 && p.root_lo[2] == 0.0 &&
                     std::frexp(scale, &sexp) == 0.5 && sexp > -120 && sexp < 120 ? 1 : 0;
    if (ids) {
        launch(GBLOD_K_BUILD_OTHER, k_id_keys, dim3(G), dim3(T), 0, s, ids, (size_t)n, keys, vals);
        radix_sort_pairs(A, sort, &keys, &vals, keys == keyA.p ? keyB.p : keyA.p, vals == valA.p ? valB.p : valA.p,
                         n, 32, s, hs);
        // vals = input indices in id order; keys in that order
        uint64_t *kdst = keys == keyA.p ? keyB.p : keyA.p;
        launch(GBLOD_K_MORTON, k_morton, dim3(G), dim3(T), 0, s, xyz, (const uint32_t *)vals, (size_t)n, p.root_lo[0],
               p.root_lo[1], p.root_lo[2], scale, kdst, (uint32_t *)nullptr, pow2);
        keys = kdst;
    } else {
        launch(GBLOD_K_MORTON, k_morton, dim3(G), dim3(T), 0, s, xyz, (const uint32_t *)nullptr, (size_t)n,
               p.root_lo[0], p.root_lo[1], p.root_lo[2], scale, keys, vals, pow2);
    }
    radix_sort_pairs(A, sort, &keys, &vals, keys == keyA.p ? keyB.p : keyA.p, vals == valA.p ? valB.p : valA.p, n, 63,
                     s, hs);
    // keep the sorted keys and permutation in the octree
    uint64_t *skey = keys;
    uint32_t *sidx = vals;
    if (skey == keyA.p) keyA.release_ptr(); else keyB.release_ptr();
    if (sidx == valA.p) valA.release_ptr(); else valB.release_ptr();
    o->skey = skey;
    o->sidx = sidx;
    keyA.reset(); keyB.reset(); valA.reset(); valB.reset();

    // sorted particle arrays and fixed-point masses (with no caller ids the sorted ids are sidx;
    // with equal masses no prefix of masses is needed)
    Scratch<float4> s4(A, n, s);
    Scratch<float> sh(A, n, s);
    Scratch<uint32_t> sid(A, ids ? n : 1, s);
    Scratch<U128> mpre(A, o->equal_mass ? 1 : n, s), mtot(A, 1, s);
    launch(GBLOD_K_BUILD_OTHER, k_gather_sorted, dim3(G), dim3(T), 0, s, xyz, mass, h, ids, (const uint32_t *)sidx,
           (size_t)n, s4.p, sh.p, ids ? sid.p : (uint32_t *)nullptr, o->equal_mass ? (U128 *)nullptr : mpre.p,
           o->equal_mass, m0);
    if (!o->equal_mass) scan_exclusive_u128(A, scan, mpre.p, mpre.p, n, mtot.p, s);
    const uint32_t *sorted_ids = ids ? sid.p : sidx;

    // A3: node table, one level at a time
    NodeStore &N = tmp.N;
    N.reserve(A, 0, 1024, s);
    launch(GBLOD_K_BUILD_OTHER, k_init_root, dim3(1), dim3(1), 0, s, N.soa(), (uint32_t)n);
    std::vector<uint64_t> level_first = {0, 1};
    DBuf<uint32_t> &cc = tmp.cc, &cf = tmp.cf, &nz = tmp.nz, &slot = tmp.slot;
    Scratch<uint32_t> total(A, 1, s);
    for (int d = 0; d < GBLOD_MAX_DEPTH; ++d) {
        const uint64_t L = level_first[d];
        const uint32_t nd = (uint32_t)(level_first[d + 1] - L);
        if (nd == 0) break;
        const size_t m = (size_t)nd * 8;
        cc.ensure(A, m, s); cf.ensure(A, m, s); nz.ensure(A, m, s); slot.ensure(A, m, s);
        launch(GBLOD_K_BUILD_OTHER, k_child_counts, dim3(blocks_for(m, T)), dim3(T), 0, s, (const uint64_t *)skey,
               (const uint64_t *)N.code.p, (const uint32_t *)N.first.p, (const uint32_t *)N.count.p, L, nd, d,
               p.n_max, cc.p, cf.p, nz.p);
        scan_exclusive_u32(A, scan, nz.p, slot.p, m, total.p, s);
        const uint32_t nnext = read1(total.p, s, hs);
        const uint64_t Lnext = level_first[d + 1];
        N.reserve(A, Lnext, Lnext + nnext, s);
        launch(GBLOD_K_BUILD_OTHER, k_emit_children, dim3(blocks_for(m, T)), dim3(T), 0, s, N.soa(),
               (const uint32_t *)cc.p, (const uint32_t *)cf.p, (const uint32_t *)slot.p, L, nd, d, Lnext);
        if (nnext == 0) break;
        level_first.push_back(Lnext + nnext);
    }
    cc.release(A, s); cf.release(A, s); nz.release(A, s); slot.release(A, s);
    const size_t nn = level_first.back();
    o->n_nodes = nn;
    o->depth_max = (int)level_first.size() - 2;
    o->level_first = level_first;

    // classify, number the stored points, masses and representative parameters
    Scratch<uint32_t> flags(A, nn, s), isrep(A, nn, s), reppos(A, nn, s);
    Scratch<uint64_t> pcount(A, nn, s), pfirst(A, nn, s), ptotal(A, 1, s), mlo(A, nn, s), mhi(A, nn, s);
    Scratch<float> w(A, nn, s), sc(A, nn, s), hcull(A, nn, s), bmin(A, 3 * nn, s), bmax(A, 3 * nn, s);
    Scratch<unsigned> hmax(A, nn, s);
    launch(GBLOD_K_BUILD_OTHER, k_node_classify, dim3(blocks_for(nn, T)), dim3(T), 0, s, nn,
           (const uint32_t *)N.count.p, (const int32_t *)N.depth.p, p.n_max, flags.p, pcount.p, isrep.p);
    scan_exclusive_u64(A, scan, pcount.p, pfirst.p, nn, ptotal.p, s);
    scan_exclusive_u32(A, scan, isrep.p, reppos.p, nn, total.p, s);
    const uint64_t npts = read1(ptotal.p, s, hs);
    const uint32_t n_rep = read1(total.p, s, hs);
    o->n_points = npts;
    launch(GBLOD_K_BUILD_OTHER, k_node_mass, dim3(blocks_for(nn, T)), dim3(T), 0, s, nn, (size_t)n,
           (const uint32_t *)N.first.p, (const uint32_t *)N.count.p, (const uint32_t *)flags.p,
           o->equal_mass ? (const U128 *)nullptr : (const U128 *)mpre.p, (const U128 *)mtot.p, m0, p.n_max, mlo.p,
           mhi.p, w.p, sc.p);
    mpre.reset();
    GB_CUDA(cudaMemsetAsync(hmax.p, 0, nn * sizeof(unsigned), s));

    o->pts4 = static_cast<float4 *>(A.get(npts * sizeof(float4), s));
    o->hs = static_cast<float *>(A.get(npts * sizeof(float), s));
    o->pt_src = static_cast<uint32_t *>(A.get(npts * sizeof(uint32_t), s));
    o->nodes = static_cast<gblod_node *>(A.get(nn * sizeof(gblod_node), s));

    // A4 + A5: representatives of every over-full node
    if (n_rep) {
        Scratch<uint32_t> reps(A, n_rep, s);
        launch(GBLOD_K_BUILD_OTHER, k_compact_reps, dim3(blocks_for(nn, T)), dim3(T), 0, s, nn,
               (const uint32_t *)isrep.p, (const uint32_t *)reppos.p, reps.p);
        SelectIn in{s4.p, sh.p, sorted_ids, N.code.p, N.first.p, N.count.p, pfirst.p, w.p, sc.p, hmax.p,
                    o->pts4, o->hs, o->pt_src, p.n_max};
        select_representatives(A, s, hs, scan, in, reps.p, n_rep, p.n_max, p.seed, o->equal_mass);
    }

    // leaves, bounds, cull radii
    launch(GBLOD_K_BUILD_OTHER, k_leaf_nodes, dim3((unsigned)std::min<size_t>(nn, 65535 * 4)), dim3(T), 0, s, nn,
           (const uint32_t *)flags.p, (const uint32_t *)N.first.p, (const uint32_t *)N.count.p,
           (const uint64_t *)pfirst.p, (const float4 *)s4.p, (const float *)sh.p, o->pts4, o->hs, o->pt_src, bmin.p,
           bmax.p, hmax.p);
    for (int d = o->depth_max; d >= 0; --d) {
        const uint64_t L = level_first[d];
        const uint32_t nd = (uint32_t)(level_first[d + 1] - L);
        launch(GBLOD_K_BUILD_OTHER, k_bottom_up, dim3(blocks_for(nd, T)), dim3(T), 0, s, L, nd,
               (const uint32_t *)flags.p, (const uint32_t *)N.child_first.p, (const uint32_t *)N.child_count.p,
               bmin.p, bmax.p, (const unsigned *)hmax.p, hcull.p);
    }
    PackIn P{N.code.p, pfirst.p, mlo.p, mhi.p, N.first.p, N.count.p, N.child_first.p, N.child_count.p, flags.p,
             N.depth.p, N.parent.p, hcull.p, w.p, sc.p, bmin.p, bmax.p, p.n_max};
    launch(GBLOD_K_BUILD_OTHER, k_pack_nodes, dim3(blocks_for(nn, T)), dim3(T), 0, s, nn, P, o->nodes);
    GB_CUDA(cudaStreamSynchronize(s));
    o->bytes = nn * sizeof(gblod_node) + npts * (sizeof(float4) + sizeof(float) + sizeof(uint32_t)) +
               n * (sizeof(uint64_t) + sizeof(uint32_t));
    return o;
}

} // namespace gb
