// Per-frame path: R1 view-dependent node selection (depth paragraph: near nodes deep, far
// nodes shallow), R2 projection and screen-tile binning, R3 tiled splatting of every point as a
// blob evaluated at every pixel it covers (GPU paragraph) into 64-bit fixed point, R4 log tone
// map.  The brute-force frame runs R2-R4 over the raw particle arrays.
//
// Determinism: the per-point arithmetic is fp32 with one round-to-nearest per operation in a
// fixed order, positions are quantised to 1/256 px, the kernel is a 1024-entry integer table
// and every pixel is an exact 64-bit integer sum, so the image does not depend on launch
// shape, tiling or the order in which splats are added.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <vector>

#include "lodmath.cuh"
#include "render.cuh"

namespace gb {

void check_image(const gblod_camera &c);
void check_format(const gblod_octree *o, const gblod_render_params &rp);

// integer kernel tables (Gaussian, cubic), filled once per device
__device__ int32_t g_ktab[2][1024];

namespace {

constexpr unsigned ST_RANGE = 1u;
constexpr int RT = 256;       // render block size
constexpr int CHUNK = 2048;   // points per block iteration in the projection kernels
constexpr uint32_t ITEM = 2048; // records per splat work item
constexpr float A_GAUSS = 0x1.499c68p+29f; // 2^32 / (2 pi (1 - e^-4.5))
constexpr float A_CUBIC = 0x1.d1a452p+30f; // 2^32 * 10 / (7 pi)
constexpr float B_GAUSS = 0x1.c71c72p+27f; // 2^31 / 9
constexpr float B_CUBIC = 0x1p+29f;        // 2^31 / 4

void kernel_table_host(int kernel, int32_t *K)
{
    const double qmax = kernel == GBLOD_KERNEL_CUBIC ? 4.0 : 9.0;
    for (int i = 0; i < 1024; ++i) {
        const double q = ((double)i + 0.5) * qmax / 1024.0;
        double f;
        if (kernel == GBLOD_KERNEL_CUBIC) {
            const double xi = std::sqrt(q);
            if (xi < 1.0) {
                const double a = 1.0 - 1.5 * q;
                const double b = 0.75 * (q * xi);
                f = a + b;
            } else {
                const double t = 2.0 - xi;
                f = 0.25 * ((t * t) * t);
            }
        } else {
            f = std::exp(-0.5 * q);
        }
        K[i] = (int32_t)std::nearbyint(65536.0 * f);
    }
}

void set_splat_smem_limits();

// once per device: the kernel tables, and the dynamic shared-memory limit of the splat kernels
// (a device setting, so it is made before any launch that a stream capture could record)
void ensure_tables()
{
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (done[dev]) return;
    static int32_t K[2][1024];
    kernel_table_host(GBLOD_KERNEL_GAUSSIAN, K[0]);
    kernel_table_host(GBLOD_KERNEL_CUBIC, K[1]);
    GB_CUDA(cudaMemcpyToSymbol(g_ktab, K, sizeof(K)));
    set_splat_smem_limits();
    done[dev] = 1;
}

struct Proj {
    float ex, ey, ez, rx, ry, rz, ux, uy, uz, fx, fy, fz;
    float F, CX, CY, ZN, smin, smax, A, B, Rk, Wf, Hf;
    int W, H, TW, TH, tiles_x, tiles_y, kernel;
};

Proj make_proj(const gblod_camera &c, const gblod_render_params &rp)
{
    Proj P;
    P.ex = (float)c.eye[0]; P.ey = (float)c.eye[1]; P.ez = (float)c.eye[2];
    P.rx = (float)c.right[0]; P.ry = (float)c.right[1]; P.rz = (float)c.right[2];
    P.ux = (float)c.up[0]; P.uy = (float)c.up[1]; P.uz = (float)c.up[2];
    P.fx = (float)c.fwd[0]; P.fy = (float)c.fwd[1]; P.fz = (float)c.fwd[2];
    P.F = (float)c.f_px;
    P.CX = (float)c.cx;
    P.CY = (float)c.cy;
    P.ZN = (float)c.z_near;
    P.smin = (float)rp.sigma_min_px;
    P.smax = (float)rp.sigma_max_px;
    const bool cubic = rp.kernel == GBLOD_KERNEL_CUBIC;
    P.A = cubic ? A_CUBIC : A_GAUSS;
    P.B = cubic ? B_CUBIC : B_GAUSS;
    P.Rk = cubic ? 2.0f : 3.0f;
    P.Wf = (float)c.width;
    P.Hf = (float)c.height;
    P.W = c.width;
    P.H = c.height;
    P.TW = rp.tile_w > 0 ? rp.tile_w : 64;
    P.TH = rp.tile_h > 0 ? rp.tile_h : 16;
    P.tiles_x = (P.W + P.TW - 1) / P.TW;
    P.tiles_y = (P.H + P.TH - 1) / P.TH;
    P.kernel = cubic ? 1 : 0;
    return P;
}

struct Splat {
    int32_t U, V;
    uint32_t S;
    float Wf; // amplitude before rounding; Wq = rne(Wf)
};

// R2 for one point.  Returns 1 drawn, 0 culled, -1 amplitude out of range.
__device__ __forceinline__ int project(const Proj &P, float x, float y, float z, float w, float h, Splat &s)
{
    const float dx = __fsub_rn(x, P.ex), dy = __fsub_rn(y, P.ey), dz = __fsub_rn(z, P.ez);
    const float xc = __fadd_rn(__fadd_rn(__fmul_rn(P.rx, dx), __fmul_rn(P.ry, dy)), __fmul_rn(P.rz, dz));
    const float yc = __fadd_rn(__fadd_rn(__fmul_rn(P.ux, dx), __fmul_rn(P.uy, dy)), __fmul_rn(P.uz, dz));
    const float zc = __fadd_rn(__fadd_rn(__fmul_rn(P.fx, dx), __fmul_rn(P.fy, dy)), __fmul_rn(P.fz, dz));
    if (!(zc > P.ZN)) return 0;
    const float iz = __fdiv_rn(1.0f, zc);
    const float u = __fadd_rn(P.CX, __fmul_rn(__fmul_rn(P.F, xc), iz));
    const float v = __fsub_rn(P.CY, __fmul_rn(__fmul_rn(P.F, yc), iz));
    const float sg = __fmul_rn(__fmul_rn(P.F, h), iz);
    const float sigma = sg >= P.smin ? (sg <= P.smax ? sg : P.smax) : P.smin;
    const float s2 = __fmul_rn(sigma, sigma);
    const float Wf = __fdiv_rn(__fmul_rn(w, P.A), s2);
    const float Sf = __fdiv_rn(P.B, s2);
    const float R = __fadd_rn(__fmul_rn(P.Rk, sigma), 2.0f);
    if (!(__fadd_rn(u, R) >= 0.0f && __fsub_rn(u, R) <= P.Wf && __fadd_rn(v, R) >= 0.0f &&
          __fsub_rn(v, R) <= P.Hf))
        return 0;
    if (!(Wf >= 0.0f && Wf < 0x1p48f)) return -1;
    s.U = __float2int_rn(__fmul_rn(u, 256.0f));
    s.V = __float2int_rn(__fmul_rn(v, 256.0f));
    s.S = __float2uint_rn(Sf);
    s.Wf = Wf;
    return 1;
}

// Pixel box (inclusive) that contains every pixel where the table index can be below 1024:
// q S < 2^47 needs |d| < sqrt(2^47 / S) in 1/256 px.
// Returns the bounding radius r (1/256 px) the box was cut from: every pixel of the box has |dx| <= r
// and |dy| <= r.
__device__ __forceinline__ int splat_box(int U, int V, uint32_t S, int W, int H, int &x0, int &x1, int &y0, int &y1)
{
    const float ql = __fdiv_rn(140737488355328.0f, __uint2float_rn(S));
    const int r = (int)sqrtf(ql) + 2;
    const int ax = U - 128 - r, bx = U - 128 + r, ay = V - 128 - r, by = V - 128 + r;
    x0 = -((-ax) >> 8);
    x1 = bx >> 8;
    y0 = -((-ay) >> 8);
    y1 = by >> 8;
    x0 = max(x0, 0);
    y0 = max(y0, 0);
    x1 = min(x1, W - 1);
    y1 = min(y1, H - 1);
    return r;
}

// Points whose pixel box is at most DIRECT_BOX pixels on a side are not binned: the scatter pass
// adds their contributions straight to the image, one 64-bit atomic per pixel inside the support.
// The image is a sum of integers, so it is the same whichever pass adds a contribution and in
// whatever order.  Small boxes are most of the drawn points (sigma at or near its minimum) but a
// small share of the pixel work, and each of their (tile, point) records would cost the splat
// kernel a staging slot, a list entry and a test of a 32-pixel block for a few pixels.  Measured
// on the mid fly-through: 8 is faster than 4 and 6.
constexpr int DIRECT_BOX = 8;

__device__ __forceinline__ bool direct_box(int x0, int x1, int y0, int y1)
{
    return x1 - x0 < DIRECT_BOX && y1 - y0 < DIRECT_BOX;
}

// Bounding radius (1/256 px) up to which a box's pixels all have q = dx^2 + dy^2 < 2^32 (2 r^2 <
// 2^32): dx^2 and dy^2 are then signed 32-bit products and the table index (q S) >> 37 is the high
// word of the 32 x 32 product q S shifted by 5.  Wider boxes (the visible sliver of a large blob
// centred off the image) take 64-bit distances.
constexpr int R_NARROW = 46340;

// One point's clipped pixel box for walk_boxes: n pixels (0: none) from origin xy = x0 | y0 << 16,
// meta = ceil(2^8 / bw) | bw << 9 | wide << 13 | kernel << 14 | Wl << 16 for box width bw <=
// DIRECT_BOX and the radial kernel's table (0 Gaussian, 1 cubic), and the rule's other operands U,
// V, S and Wh (Wq = Wh 2^16 + Wl).
struct BoxWalk {
    uint32_t n = 0, xy = 0, meta = 0;
    int U = 0, V = 0;
    uint32_t S = 0, Wh = 0;
};

__device__ __forceinline__ BoxWalk box_walk(int U, int V, uint32_t S, unsigned long long Wq, int r, int x0, int x1,
                                            int y0, int y1, int kernel = 0)
{
    BoxWalk b;
    const uint32_t bw = (uint32_t)(x1 - x0 + 1);
    b.n = bw * (uint32_t)(y1 - y0 + 1);
    b.xy = (uint32_t)x0 | ((uint32_t)y0 << 16);
    b.meta = ((256u + bw - 1u) / bw) | (bw << 9) | (r > R_NARROW ? 1u << 13 : 0u) | ((uint32_t)kernel << 14) |
             ((uint32_t)(Wq & 0xFFFFull) << 16);
    b.U = U;
    b.V = V;
    b.S = S;
    b.Wh = (uint32_t)(Wq >> 16);
    return b;
}

// The per-pixel rule over the boxes (at most DIRECT_BOX x DIRECT_BOX pixels) of a warp's points,
// one point per lane: the warp walks the concatenation of all lanes' box pixels (row-major within a
// box) 32 (point, pixel) pairs at a time, pair k on lane k mod 32.  Lanes stay busy whatever the box
// sizes, and neighbouring lanes take neighbouring pixels of one point instead of 32 points' pixels
// at the same offset (in dense regions often the same pixel).  The owner of pair k of a window: each
// lane whose box starts inside the window writes its lane number at its start offset in a per-warp
// table, one OR-reduction gives the mask of start offsets, and pair k belongs to the box with the
// last start at or before k (the highest set bit of the mask up to k), or, if none, to the box that
// owned the previous window's last pair (boxes are contiguous runs of pairs).  Row and column of pixel m of a box:
// m / bw = (m ceil(2^8 / bw)) >> 8, exact for m < 64 and bw <= 8.  tab(meta, idx) reads the table
// entry; add(tag, x, y, c) receives every nonzero contribution with the tag of the point's lane
// (TAGGED: the lane's `tag`, e.g. its view in a batch; else 0).  Returns this lane's pixel updates.
// Every lane of the warp calls it.
template <bool TAGGED, class Tab, class Add>
__device__ __forceinline__ unsigned walk_boxes(const BoxWalk &b, uint32_t tag, Tab tab, Add add)
{
    const int lane = threadIdx.x & 31;
    uint32_t incl = b.n;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - b.n;
    __shared__ uint8_t owner_at[RT / 32][32];
    uint8_t *own = owner_at[threadIdx.x >> 5];
    unsigned hits = 0;
    int carry = 0; // owner of the previous window's last pair
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t k = base + (uint32_t)lane;
        const bool starts = b.n && excl >= base && excl < base + 32u;
        if (starts) own[excl - base] = (uint8_t)lane;
        const uint32_t smask = __reduce_or_sync(0xffffffffu, starts ? 1u << (excl - base) : 0u);
        __syncwarp();
        const uint32_t upto = smask & (0xffffffffu >> (31 - lane)); // start offsets 0..lane
        const int src = upto ? (int)own[31 - __clz(upto)] : carry;
        carry = __shfl_sync(0xffffffffu, src, 31);
        __syncwarp(); // the table is rewritten in the next window
        const uint32_t m = k - __shfl_sync(0xffffffffu, excl, src);
        const uint32_t meta = __shfl_sync(0xffffffffu, b.meta, src), xy = __shfl_sync(0xffffffffu, b.xy, src);
        const int U = __shfl_sync(0xffffffffu, b.U, src), V = __shfl_sync(0xffffffffu, b.V, src);
        const uint32_t S = __shfl_sync(0xffffffffu, b.S, src), Wh = __shfl_sync(0xffffffffu, b.Wh, src);
        const uint32_t t = TAGGED ? __shfl_sync(0xffffffffu, tag, src) : 0u;
        if (k < total) {
            const uint32_t bw = (meta >> 9) & 15u;
            const uint32_t row = (m * (meta & 0x1FFu)) >> 8, col = m - row * bw;
            const int x = (int)(xy & 0xFFFFu) + (int)col, y = (int)(xy >> 16) + (int)row;
            uint32_t idx;
            if (!(meta & (1u << 13))) {
                const int dx = x * 256 + 128 - U, dy = y * 256 + 128 - V;
                idx = __umulhi((uint32_t)(dx * dx) + (uint32_t)(dy * dy), S) >> 5;
            } else {
                const long long dx = (long long)x * 256 + 128 - U, dy = (long long)y * 256 + 128 - V;
                const unsigned long long i64 = ((unsigned long long)(dx * dx + dy * dy) * S) >> 37;
                idx = i64 < 1024ull ? (uint32_t)i64 : 1024u;
            }
            if (idx < 1024u) {
                const uint32_t kv = (uint32_t)tab(meta, idx);
                const unsigned long long c = (unsigned long long)Wh * kv + (((meta >> 16) * kv) >> 16);
                if (c) add(t, x, y, c);
                ++hits;
            }
        }
    }
    return hits;
}

// Adds a warp's pixel updates to the frame counters (every lane of the warp calls it)
__device__ __forceinline__ void count_hits(unsigned hits, FrameStatsDev *stats)
{
    unsigned long long h64 = hits;
    for (int d = 16; d > 0; d >>= 1) h64 += __shfl_xor_sync(0xffffffffu, h64, d);
    if ((threadIdx.x & 31) == 0 && h64) {
        atomicAdd(&stats->pixel_updates, h64);
        atomicAdd(&stats->pixel_updates_total, h64);
    }
}

// ------------------------------------------------------------------ R1
struct Frustum {
    double n[5][3];
    double off[5];
    double E[3];
    double lo[3];
    double F, side, lam2, zn2, rk;
};

Frustum make_frustum(const gblod_camera &c, const gblod_render_params &rp, const gblod_octree *o)
{
    // host FP64, every product and sum rounded on its own (built with -ffp-contract=off)
    Frustum f;
    const double rk = rp.kernel == GBLOD_KERNEL_CUBIC ? 2.0 : 3.0;
    const double M = rk * rp.sigma_min_px + 2.0;
    const double F = c.f_px;
    const double cl = c.cx + M;
    const double cr = ((double)c.width + M) - c.cx;
    const double ct = c.cy + M;
    const double cb = ((double)c.height + M) - c.cy;
    for (int a = 0; a < 3; ++a) {
        f.n[0][a] = c.fwd[a];
        double t1, t2;
        t1 = F * c.right[a]; t2 = cl * c.fwd[a]; f.n[1][a] = t1 + t2;
        t1 = -(F * c.right[a]); t2 = cr * c.fwd[a]; f.n[2][a] = t1 + t2;
        t1 = -(F * c.up[a]); t2 = ct * c.fwd[a]; f.n[3][a] = t1 + t2;
        t1 = F * c.up[a]; t2 = cb * c.fwd[a]; f.n[4][a] = t1 + t2;
        f.E[a] = c.eye[a];
        f.lo[a] = o->lo[a];
    }
    f.off[0] = -c.z_near;
    f.off[1] = f.off[2] = f.off[3] = f.off[4] = 0.0;
    f.F = F;
    f.side = o->side;
    const double lam = rp.lambda_px < 0.0 ? std::sqrt((double)o->n_max) : rp.lambda_px;
    f.lam2 = lam * lam;
    f.zn2 = c.z_near * c.z_near;
    f.rk = rk;
    return f;
}

// 0 cull, 1 emit, 2 refine
__device__ __forceinline__ int classify(const gblod_node &g, const Frustum &fr)
{
    const double rho = __dmul_rn(fr.rk, (double)g.h_cull);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double s = fr.off[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double na = fr.n[k][a];
            const double pa = na > 0.0 ? __dsub_rn(__dadd_rn((double)g.bmax[a], rho), fr.E[a])
                                       : __dsub_rn(__dsub_rn((double)g.bmin[a], rho), fr.E[a]);
            s = __dadd_rn(s, __dmul_rn(na, pa));
        }
        if (s < 0.0) return 0;
    }
    if (!(g.flags & GBLOD_NODE_INTERNAL)) return 1;
    const int d = g.depth;
    const uint64_t pfx = g.code ^ (1ull << (3 * d));
    const uint32_t q[3] = {gbd::compact3(pfx >> 2), gbd::compact3(pfx >> 1), gbd::compact3(pfx)};
    const double e = ldexp(fr.side, -d);
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double blo = __dadd_rn(fr.lo[a], __dmul_rn(e, (double)q[a]));
        const double bhi = __dadd_rn(blo, e);
        const double E = fr.E[a];
        const double da = E < blo ? __dsub_rn(blo, E) : (E > bhi ? __dsub_rn(E, bhi) : 0.0);
        d2 = __dadd_rn(d2, __dmul_rn(da, da));
    }
    const double fe = __dmul_rn(fr.F, e);
    const double lhs = __dmul_rn(fe, fe);
    const double rhs = __dmul_rn(fr.lam2, d2 > fr.zn2 ? d2 : fr.zn2);
    return lhs > rhs ? 2 : 1;
}

__global__ void k_select_init(uint32_t *front, uint32_t *cnt)
{
    front[0] = 0u;
    cnt[0] = 1u;
}

// One level of the walk.  Emitted nodes are kept only if they belong to this part of a split frame
// (node index mod n_parts == part; n_parts = 1 keeps every one); refined nodes are walked either way.
__global__ void __launch_bounds__(RT) k_select_level(const gblod_node *__restrict__ nodes, Frustum fr,
                                                     const uint32_t *__restrict__ fin, const uint32_t *nin,
                                                     uint32_t *__restrict__ fout, uint32_t *nout,
                                                     uint32_t *__restrict__ sel, uint32_t *nsel, uint32_t part,
                                                     uint32_t n_parts)
{
    const uint32_t n = *nin;
    const uint32_t lt = gbd::lanemask_lt();
    const int lane = threadIdx.x & 31;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        int cls = 0;
        uint32_t node = 0, ccount = 0, cfirst = 0;
        if (i < n) {
            node = fin[i];
            const gblod_node g = nodes[node];
            cls = classify(g, fr);
            ccount = g.child_count;
            cfirst = g.child_first;
            if (cls == 1 && n_parts > 1 && node % n_parts != part) cls = 0;
        }
        // warp-aggregated appends
        const uint32_t em = __ballot_sync(0xffffffffu, cls == 1);
        if (em) {
            const int leader = __ffs(em) - 1;
            uint32_t b = 0;
            if (lane == leader) b = atomicAdd(nsel, (uint32_t)__popc(em));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (cls == 1) sel[b + __popc(em & lt)] = node;
        }
        uint32_t want = cls == 2 ? ccount : 0u, incl = want;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t b = 0;
            if (lane == 31) b = atomicAdd(nout, total);
            b = __shfl_sync(0xffffffffu, b, 31);
            const uint32_t at = b + incl - want;
            for (uint32_t k = 0; k < want; ++k) fout[at + k] = cfirst + k;
        }
    }
}

// exclusive prefix of the selected nodes' point counts; base[j] maps a flat index to a point
__global__ void __launch_bounds__(1024) k_sel_prefix(const gblod_node *__restrict__ nodes,
                                                     const uint32_t *__restrict__ sel, const uint32_t *nsel,
                                                     uint64_t *__restrict__ pfx, int64_t *__restrict__ base,
                                                     FrameStatsDev *stats)
{
    __shared__ unsigned long long wsum[32];
    const uint32_t n = *nsel;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long run = 0;
    for (uint32_t start = 0; start < n; start += 1024) {
        const uint32_t i = start + threadIdx.x;
        unsigned long long c = 0, pf = 0;
        if (i < n) {
            const gblod_node &g = nodes[sel[i]];
            c = g.point_count;
            pf = g.point_first;
        }
        unsigned long long incl = c;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        unsigned long long before = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            before += w < warp ? wsum[w] : 0ull;
            all += wsum[w];
        }
        const unsigned long long ex = run + before + incl - c;
        if (i < n) {
            pfx[i] = ex;
            base[i] = (int64_t)pf - (int64_t)ex;
        }
        run += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pfx[n] = run;
        stats->points = run;
        stats->nodes_selected = n;
    }
}

// ------------------------------------------------------------------ R2
struct SrcLOD {
    const float4 *pts4;
    const float *hs;
    const uint64_t *pfx;  // n_sel + 1 entries
    const int64_t *base;
    const uint32_t *nsel;
    const unsigned long long *total;
};

// selected nodes' 16-bit block codes (decoded on load)
struct SrcLODQ : SrcLOD {
    const ushort4 *q4;
    const uint16_t *qw;
    const float4 *qa;
    const uint32_t *sel; // node index per selected entry
};

struct SrcFlat {
    const float *xyz, *mass, *h;
    unsigned long long n;
};

__device__ __forceinline__ unsigned long long src_total(const SrcLOD &s) { return *s.total; }
__device__ __forceinline__ unsigned long long src_total(const SrcFlat &s) { return s.n; }

// per block iteration: locate the selected nodes covering [a, b)
__device__ __forceinline__ void src_range(const SrcLOD &s, unsigned long long a, unsigned long long b, uint32_t &j0,
                                          uint32_t &j1)
{
    __shared__ uint32_t sj[2];
    if (threadIdx.x < 2) {
        const unsigned long long v = threadIdx.x == 0 ? a : b - 1;
        uint32_t lo = 0, hi = *s.nsel; // largest j with pfx[j] <= v
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s.pfx[mid] <= v)
                lo = mid;
            else
                hi = mid;
        }
        sj[threadIdx.x] = lo;
    }
    __syncthreads();
    j0 = sj[0];
    j1 = sj[1];
    __syncthreads();
}
__device__ __forceinline__ void src_range(const SrcFlat &, unsigned long long, unsigned long long, uint32_t &j0,
                                          uint32_t &j1)
{
    j0 = j1 = 0;
}

__device__ __forceinline__ void src_load(const SrcLOD &s, unsigned long long e, uint32_t j0, uint32_t j1, float &x,
                                         float &y, float &z, float &w, float &h)
{
    uint32_t lo = j0, hi = j1 + 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.pfx[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    const unsigned long long p = (unsigned long long)((long long)e + s.base[lo]);
    const float4 q = s.pts4[p];
    x = q.x; y = q.y; z = q.z; w = q.w;
    h = s.hs[p];
}
__device__ __forceinline__ void src_load(const SrcLODQ &s, unsigned long long e, uint32_t j0, uint32_t j1, float &x,
                                         float &y, float &z, float &w, float &h)
{
    uint32_t lo = j0, hi = j1 + 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.pfx[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    const unsigned long long p = (unsigned long long)((long long)e + s.base[lo]);
    const uint32_t node = s.sel[lo];
    block_decode(s.q4[p], s.qw[p], s.qa[2 * node], s.qa[2 * node + 1], x, y, z, w, h);
}
__device__ __forceinline__ void src_load(const SrcFlat &s, unsigned long long e, uint32_t, uint32_t, float &x,
                                         float &y, float &z, float &w, float &h)
{
    x = s.xyz[3 * e];
    y = s.xyz[3 * e + 1];
    z = s.xyz[3 * e + 2];
    w = s.mass[e];
    h = s.h[e];
}

// Sum of drawn amplitudes as 128 bits per thread; one atomic pair per warp at the end (the sum
// must stay below 2^64, reading R-19)
struct AmpSum {
    unsigned long long lo = 0, hi = 0;
    __device__ __forceinline__ void add(unsigned long long v)
    {
        lo += v;
        hi += lo < v ? 1ull : 0ull;
    }
    __device__ __forceinline__ void flush(FrameStatsDev *stats)
    {
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long ol = __shfl_xor_sync(0xffffffffu, lo, d), oh = __shfl_xor_sync(0xffffffffu, hi, d);
            lo += ol;
            hi += oh + (lo < ol ? 1ull : 0ull);
        }
        if ((threadIdx.x & 31) == 0 && (lo | hi)) {
            const unsigned long long old = lo ? atomicAdd(&stats->amp_lo, lo) : 0ull;
            const unsigned long long carry = lo && old + lo < old ? 1ull : 0ull;
            if (hi + carry) atomicAdd(&stats->amp_hi, hi + carry);
        }
    }
};

// Warp-cooperative scatter of (splat, tile) records.  Lane l contributes n_l pairs: the tiles
// t00_l + row * tiles_x_l + col of its box, row < n_l / tw_l, col < tw_l (n_l = 0: none).  The warp
// walks the concatenation of all lanes' pairs 32 at a time, so one lane with many tiles does not
// hold the others idle; pairs of one round that share a tile reserve their slots from cursor[t]
// with one atomic (match_any) and write the source lane's record r (slots at or past rec_cap are
// dropped).
__device__ __forceinline__ void scatter_pairs(uint32_t n, uint32_t t00, int tw, int tiles_x, const uint4 r,
                                              uint32_t *__restrict__ cursor, uint4 *__restrict__ rec,
                                              unsigned long long rec_cap)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = gbd::lanemask_lt();
    uint32_t incl = n;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - n;
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t k = base + (uint32_t)lane;
        int src = 0; // the last lane whose pairs start at or before k
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t ex = __shfl_sync(0xffffffffu, excl, src + step);
            if (ex <= k) src += step;
        }
        const uint32_t m = k - __shfl_sync(0xffffffffu, excl, src);
        const uint32_t st00 = __shfl_sync(0xffffffffu, t00, src);
        const int stw = __shfl_sync(0xffffffffu, tw, src), stx = __shfl_sync(0xffffffffu, tiles_x, src);
        uint4 sr;
        sr.x = __shfl_sync(0xffffffffu, r.x, src);
        sr.y = __shfl_sync(0xffffffffu, r.y, src);
        sr.z = __shfl_sync(0xffffffffu, r.z, src);
        sr.w = __shfl_sync(0xffffffffu, r.w, src);
        const bool act = k < total;
        const uint32_t amask = __ballot_sync(0xffffffffu, act);
        if (act) {
            const uint32_t row = m / (uint32_t)stw, col = m - row * (uint32_t)stw;
            const uint32_t t = st00 + row * (uint32_t)stx + col;
            const uint32_t peers = __match_any_sync(amask, t);
            const int leader = __ffs(peers) - 1;
            uint32_t b = 0;
            if (lane == leader) b = atomicAdd(&cursor[t], (uint32_t)__popc(peers));
            b = __shfl_sync(peers, b, leader);
            const unsigned long long pos = (unsigned long long)b + __popc(peers & lt);
            if (pos < rec_cap) rec[pos] = sr;
        }
    }
}

template <class Src>
__global__ void __launch_bounds__(RT, 4) k_project_count(Src src, Proj P, unsigned long long e_lo,
                                                      unsigned long long e_hi, uint32_t *__restrict__ tile_cnt,
                                                      unsigned *status, FrameStatsDev *stats)
{
    const unsigned long long total = min(src_total(src), e_hi);
    const int lane = threadIdx.x & 31;
    unsigned long long splats = 0, pairs = 0;
    AmpSum amp;
    for (unsigned long long a = e_lo + (unsigned long long)blockIdx.x * CHUNK; a < total;
         a += (unsigned long long)gridDim.x * CHUNK) {
        const unsigned long long b = min(total, a + CHUNK);
        uint32_t j0, j1;
        src_range(src, a, b, j0, j1);
        for (unsigned long long e0 = a; e0 < b; e0 += RT) {
            const unsigned long long e = e0 + threadIdx.x;
            int res = 0;
            Splat s;
            if (e < b) {
                float x, y, z, w, h;
                src_load(src, e, j0, j1, x, y, z, w, h);
                res = project(P, x, y, z, w, h, s);
            }
            if (__any_sync(0xffffffffu, res < 0) && lane == 0) atomicOr(status, ST_RANGE);
            if (res == 1) {
                amp.add(__float2ull_rn(s.Wf));
                ++splats;
                int x0, x1, y0, y1;
                splat_box(s.U, s.V, s.S, P.W, P.H, x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1 && !direct_box(x0, x1, y0, y1)) {
                    const int tx0 = x0 / P.TW, tx1 = x1 / P.TW, ty0 = y0 / P.TH, ty1 = y1 / P.TH;
                    pairs += (unsigned long long)(tx1 - tx0 + 1) * (unsigned long long)(ty1 - ty0 + 1);
                    for (int ty = ty0; ty <= ty1; ++ty)
                        for (int tx = tx0; tx <= tx1; ++tx) {
                            const uint32_t t = (uint32_t)(ty * P.tiles_x + tx);
                            const uint32_t mask = __activemask();
                            const uint32_t peers = __match_any_sync(mask, t);
                            const int leader = __ffs(peers) - 1;
                            if (lane == leader) atomicAdd(&tile_cnt[t], (uint32_t)__popc(peers));
                        }
                }
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        splats += __shfl_xor_sync(0xffffffffu, splats, d);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, d);
    }
    if (lane == 0 && splats) atomicAdd(&stats->splats, splats);
    if (lane == 0 && pairs) atomicAdd(&stats->pairs, pairs);
    amp.flush(stats);
}

// Writes the (tile, point) records of the binned points and splats the points with small boxes
// into img; cstats (null: not counted) receives the pixel updates of the latter.
template <class Src>
__global__ void __launch_bounds__(RT, 4) k_project_scatter(Src src, Proj P, unsigned long long e_lo,
                                                           unsigned long long e_hi, uint32_t *__restrict__ cursor,
                                                           uint4 *__restrict__ rec, unsigned long long *img,
                                                           FrameStatsDev *cstats)
{
    const unsigned long long total = min(src_total(src), e_hi);
    const int32_t *K = g_ktab[P.kernel];
    unsigned hits = 0;
    for (unsigned long long a = e_lo + (unsigned long long)blockIdx.x * CHUNK; a < total;
         a += (unsigned long long)gridDim.x * CHUNK) {
        const unsigned long long b = min(total, a + CHUNK);
        uint32_t j0, j1;
        src_range(src, a, b, j0, j1);
        for (unsigned long long e0 = a; e0 < b; e0 += RT) {
            const unsigned long long e = e0 + threadIdx.x;
            int res = 0;
            Splat s;
            if (e < b) {
                float x, y, z, w, h;
                src_load(src, e, j0, j1, x, y, z, w, h);
                res = project(P, x, y, z, w, h, s);
            }
            uint32_t n = 0, t00 = 0;
            int tw = 1;
            uint4 r = make_uint4(0u, 0u, 0u, 0u);
            BoxWalk direct;
            if (res == 1) {
                int x0, x1, y0, y1;
                const int rad = splat_box(s.U, s.V, s.S, P.W, P.H, x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1) {
                    if (direct_box(x0, x1, y0, y1)) {
                        direct = box_walk(s.U, s.V, s.S, __float2ull_rn(s.Wf), rad, x0, x1, y0, y1);
                    } else {
                        r = make_uint4((uint32_t)s.U, (uint32_t)s.V, s.S, __float_as_uint(s.Wf));
                        const int tx0 = x0 / P.TW, tx1 = x1 / P.TW, ty0 = y0 / P.TH, ty1 = y1 / P.TH;
                        tw = tx1 - tx0 + 1;
                        n = (uint32_t)(tw * (ty1 - ty0 + 1));
                        t00 = (uint32_t)(ty0 * P.tiles_x + tx0);
                    }
                }
            }
            scatter_pairs(n, t00, tw, P.tiles_x, r, cursor, rec, ~0ull);
            hits += walk_boxes<false>(
                direct, 0u, [&](uint32_t, uint32_t i) { return K[i]; },
                [&](uint32_t, int x, int y, unsigned long long c) { atomicAdd(&img[(size_t)y * P.W + x], c); });
        }
    }
    if (cstats) count_hits(hits, cstats);
}

// Partitioned binning for point sources in no spatial order (the caller's particle arrays): the
// warp-level aggregation of the per-tile counters above finds few equal tiles in a warp there, so
// every (splat, tile) pair would be one global atomic on one of a few thousand counters.  Instead
// each CTA of the persistent grid counts its own points per tile in shared memory and writes one
// histogram, tile-major: hist[t * G + cta].  An exclusive scan of the histograms gives every CTA
// its own base in every tile, so the scatter pass places records with shared-memory atomics only,
// and the records of a tile keep the order of the CTAs.  Both passes walk the same chunks (the same
// grid G and chunk stride), so they see the same points.  Points whose pixel box is at most
// DIRECT_BOX on a side are binned too, into a second record stream (their own histograms, after the
// binned points' in the same scan), and splatted by k_splat_small into a shared-memory tile image:
// in no spatial order, adding them straight to the image would be one global atomic per pixel at
// random addresses.
constexpr uint32_t PART_MAX_TILES = 4096; // two shared-memory histograms: 32 KB
constexpr uint32_t ITEM_SMALL = 4096;     // small records per k_splat_small work item

template <class Src>
__global__ void __launch_bounds__(RT, 4) k_project_hist(Src src, Proj P, unsigned long long e_lo,
                                                     unsigned long long e_hi, uint32_t *__restrict__ hist,
                                                     unsigned *status, FrameStatsDev *stats)
{
    extern __shared__ uint32_t sh_cnt[]; // [ntiles] binned points, then [ntiles] small boxes
    const uint32_t ntiles = (uint32_t)(P.tiles_x * P.tiles_y);
    for (uint32_t t = threadIdx.x; t < 2 * ntiles; t += RT) sh_cnt[t] = 0u;
    __syncthreads();
    const unsigned long long total = min(src_total(src), e_hi);
    const int lane = threadIdx.x & 31;
    unsigned long long splats = 0, pairs = 0;
    AmpSum amp;
    for (unsigned long long a = e_lo + (unsigned long long)blockIdx.x * CHUNK; a < total;
         a += (unsigned long long)gridDim.x * CHUNK) {
        const unsigned long long b = min(total, a + CHUNK);
        uint32_t j0, j1;
        src_range(src, a, b, j0, j1);
        for (unsigned long long e0 = a; e0 < b; e0 += RT) {
            const unsigned long long e = e0 + threadIdx.x;
            int res = 0;
            Splat s;
            if (e < b) {
                float x, y, z, w, h;
                src_load(src, e, j0, j1, x, y, z, w, h);
                res = project(P, x, y, z, w, h, s);
            }
            if (__any_sync(0xffffffffu, res < 0) && lane == 0) atomicOr(status, ST_RANGE);
            if (res == 1) {
                amp.add(__float2ull_rn(s.Wf));
                ++splats;
                int x0, x1, y0, y1;
                splat_box(s.U, s.V, s.S, P.W, P.H, x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1) {
                    const bool small = direct_box(x0, x1, y0, y1);
                    uint32_t *cnt = small ? sh_cnt + ntiles : sh_cnt;
                    const int tx0 = x0 / P.TW, tx1 = x1 / P.TW, ty0 = y0 / P.TH, ty1 = y1 / P.TH;
                    if (!small) pairs += (unsigned long long)(tx1 - tx0 + 1) * (unsigned long long)(ty1 - ty0 + 1);
                    for (int ty = ty0; ty <= ty1; ++ty)
                        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&cnt[ty * P.tiles_x + tx], 1u);
                }
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        splats += __shfl_xor_sync(0xffffffffu, splats, d);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, d);
    }
    if (lane == 0 && splats) atomicAdd(&stats->splats, splats);
    if (lane == 0 && pairs) atomicAdd(&stats->pairs, pairs);
    amp.flush(stats);
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < 2 * ntiles; t += RT) hist[(size_t)t * gridDim.x + blockIdx.x] = sh_cnt[t];
}

// tile counts and offsets from the scanned (tile, CTA) histogram
__global__ void k_tiles_from_hist(uint32_t ntiles, uint32_t G, const uint32_t *__restrict__ off,
                                  const uint32_t *total, uint32_t *tile_cnt, uint32_t *tile_off)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t a = off[(size_t)t * G], b = t + 1 < ntiles ? off[(size_t)(t + 1) * G] : *total;
    tile_off[t] = a;
    tile_cnt[t] = b - a;
}

// Writes the (tile, point) records of the binned points at this CTA's bases and splats the points
// with small boxes into img (cstats, if not null, receives the latter's pixel updates).
template <class Src>
__global__ void __launch_bounds__(RT, 4) k_project_scatter_part(Src src, Proj P, unsigned long long e_lo,
                                                             unsigned long long e_hi, const uint32_t *__restrict__ off,
                                                             uint4 *__restrict__ rec, unsigned long long *img,
                                                             FrameStatsDev *cstats)
{
    extern __shared__ uint32_t sh_cur[]; // [ntiles] binned points, then [ntiles] small boxes
    const uint32_t ntiles = (uint32_t)(P.tiles_x * P.tiles_y);
    for (uint32_t t = threadIdx.x; t < 2 * ntiles; t += RT) sh_cur[t] = off[(size_t)t * gridDim.x + blockIdx.x];
    __syncthreads();
    const unsigned long long total = min(src_total(src), e_hi);
    for (unsigned long long a = e_lo + (unsigned long long)blockIdx.x * CHUNK; a < total;
         a += (unsigned long long)gridDim.x * CHUNK) {
        const unsigned long long b = min(total, a + CHUNK);
        uint32_t j0, j1;
        src_range(src, a, b, j0, j1);
        for (unsigned long long e0 = a; e0 < b; e0 += RT) {
            const unsigned long long e = e0 + threadIdx.x;
            int res = 0;
            Splat s;
            if (e < b) {
                float x, y, z, w, h;
                src_load(src, e, j0, j1, x, y, z, w, h);
                res = project(P, x, y, z, w, h, s);
            }
            if (res == 1) {
                int x0, x1, y0, y1;
                splat_box(s.U, s.V, s.S, P.W, P.H, x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1) {
                    uint32_t *cur = direct_box(x0, x1, y0, y1) ? sh_cur + ntiles : sh_cur;
                    const uint4 r = make_uint4((uint32_t)s.U, (uint32_t)s.V, s.S, __float_as_uint(s.Wf));
                    const int tx0 = x0 / P.TW, tx1 = x1 / P.TW, ty0 = y0 / P.TH, ty1 = y1 / P.TH;
                    for (int ty = ty0; ty <= ty1; ++ty)
                        for (int tx = tx0; tx <= tx1; ++tx) rec[atomicAdd(&cur[ty * P.tiles_x + tx], 1u)] = r;
                }
            }
        }
    }
    (void)img;
    (void)cstats;
}

__global__ void k_tile_items_n(uint32_t ntiles, const uint32_t *tile_cnt, uint32_t per_item, uint32_t *item_cnt)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) item_cnt[t] = (tile_cnt[t] + per_item - 1) / per_item;
}

__global__ void k_fill_items_n(uint32_t ntiles, const uint32_t *tile_cnt, const uint32_t *tile_off,
                               const uint32_t *item_off, uint32_t per_item, uint4 *items)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t c = tile_cnt[t], o = tile_off[t];
    uint32_t k = item_off[t];
    for (uint32_t s = 0; s < c; s += per_item, ++k) items[k] = make_uint4(t, o + s, o + min(c, s + per_item), 0u);
}

// Small-box records of one work item (a tile and up to ITEM_SMALL of its records): each warp takes
// 32 records at a time and walks their pixel boxes, clipped to the tile, with walk_boxes, adding the
// per-pixel rule's contributions to a shared tile image.  A contribution c < 2^49 is added as three
// fields, c = lo + mid 2^16 + hi 2^32 with lo, mid < 2^16, to 32-bit words by fire-and-forget
// 32-bit shared atomics (hi, rarely nonzero, only when it is): a pixel receives at most one
// contribution per record, so at most ITEM_SMALL = 2^12 per item, and no word can overflow
// (lo and mid sums < 2^28, hi sums < 2^29).  The lo and mid words have four copies, one per group
// of two warps, so that warps adding to the same pixel -- points pile up in dense halo cores --
// mostly meet only in the final sum; the fields are then recombined in 64 bits and added to the
// image once per pixel.  A box is small once clipped to the image, so its pixels can lie far from a
// centre outside the image (the visible sliver of a large blob): walk_boxes takes 64-bit distances
// for those.
static_assert(ITEM_SMALL <= (1u << 12), "32-bit field sums of the small-box tile image");
template <bool COUNT>
__global__ void __launch_bounds__(RT, 5) k_splat_small(const uint4 *__restrict__ rec, const uint4 *__restrict__ items,
                                                      Proj P, unsigned long long *__restrict__ img, FrameStatsDev *stats)
{
    __shared__ uint32_t tlo[4][1024], tmid[4][1024], thi[1024]; // TW x TH <= 1024 (checked on the host)
    __shared__ int32_t K[1024];
    for (int i = threadIdx.x; i < 1024; i += RT) {
        K[i] = g_ktab[P.kernel][i];
        thi[i] = 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            tlo[c][i] = 0u;
            tmid[c][i] = 0u;
        }
    }
    __syncthreads();
    uint32_t *lo = tlo[(threadIdx.x >> 6) & 3], *mid = tmid[(threadIdx.x >> 6) & 3];
    const uint4 it = items[blockIdx.x];
    const int tx = (int)(it.x % (uint32_t)P.tiles_x), ty = (int)(it.x / (uint32_t)P.tiles_x);
    const int X0 = tx * P.TW, Y0 = ty * P.TH;
    const int X1 = min(X0 + P.TW, P.W) - 1, Y1 = min(Y0 + P.TH, P.H) - 1;
    const int TW = P.TW;
    unsigned hits = 0;
    for (uint32_t base = it.y + (threadIdx.x & ~31u); base < it.z; base += RT) { // uniform per warp
        const uint32_t r = base + (threadIdx.x & 31u);
        BoxWalk b;
        if (r < it.z) {
            const uint4 R = rec[r];
            const int U = (int)R.x, V = (int)R.y;
            int x0, x1, y0, y1;
            const int rad = splat_box(U, V, R.z, P.W, P.H, x0, x1, y0, y1);
            x0 = max(x0, X0);
            x1 = min(x1, X1);
            y0 = max(y0, Y0);
            y1 = min(y1, Y1);
            if (x0 <= x1 && y0 <= y1)
                b = box_walk(U, V, R.z, __float2ull_rn(__uint_as_float(R.w)), rad, x0, x1, y0, y1);
        }
        hits += walk_boxes<false>(b, 0u, [&](uint32_t, uint32_t i) { return K[i]; },
                                  [&](uint32_t, int x, int y, unsigned long long c) {
            const int p = (y - Y0) * TW + (x - X0);
            atomicAdd(&lo[p], (uint32_t)c & 0xFFFFu);
            atomicAdd(&mid[p], ((uint32_t)c >> 16));
            const uint32_t h = (uint32_t)(c >> 32);
            if (h) atomicAdd(&thi[p], h);
        });
    }
    __syncthreads();
    const int tw = X1 - X0 + 1, th = Y1 - Y0 + 1;
    for (int i = threadIdx.x; i < tw * th; i += RT) {
        const int y = i / tw, x = i - y * tw, k = y * P.TW + x;
        const unsigned long long v =
            (unsigned long long)tlo[0][k] + tlo[1][k] + tlo[2][k] + tlo[3][k] +
            (((unsigned long long)tmid[0][k] + tmid[1][k] + tmid[2][k] + tmid[3][k]) << 16) +
            ((unsigned long long)thi[k] << 32);
        if (v) atomicAdd(&img[(size_t)(Y0 + y) * P.W + (X0 + x)], v);
    }
    if (COUNT) count_hits(hits, stats);
}

__global__ void k_tile_items(uint32_t ntiles, const uint32_t *tile_cnt, uint32_t *item_cnt)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) item_cnt[t] = (tile_cnt[t] + ITEM - 1) / ITEM;
}

__global__ void k_fill_items(uint32_t ntiles, const uint32_t *tile_cnt, const uint32_t *tile_off,
                             const uint32_t *item_off, uint4 *items)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t c = tile_cnt[t], o = tile_off[t];
    uint32_t k = item_off[t];
    for (uint32_t s = 0; s < c; s += ITEM, ++k) items[k] = make_uint4(t, o + s, o + min(c, s + ITEM), 0u);
}

// ------------------------------------------------------------------ R3
// One block per work item (a tile and up to ITEM of its records).  The tile is cut into 8 x 4
// pixel blocks, one lane per pixel; each warp owns up to SPLAT_SLOTS blocks of one block column
// (see strip_height).  Records are staged through shared memory STAGE at a time and listed per
// block column; each warp compacts, by ballot, its column's records whose support reaches one of
// its blocks, evaluates only those for its pixels and keeps the sums in registers.
// Exact integer shortcuts of the per-pixel rule, all identities:
//   (q S) >> 37 < 1024  <=>  q < QL = floor((2^47 - 1) / S) + 1     (one compare per miss)
//   floor(Wq K / 2^16)   =   Wh K + floor(Wl K / 2^16),  Wq = Wh 2^16 + Wl, Wl < 2^16
// Wh K goes to a 64-bit sum and floor(Wl K / 2^16) < 2^16 to a 32-bit one (at most ITEM = 2048
// records per block keeps it below 2^27).  Each pixel's sum is added to the image once.
constexpr int SPLAT_SLOTS = 4; // 8 warps x 4 blocks of 32 pixels: tiles up to 1024 pixels
static_assert(ITEM <= (1u << 15), "32-bit partial sums need at most 2^15 records per item");

constexpr int STAGE = 512; // records staged in shared memory at a time (record index: 9 bits)

struct SplatSmem {
    int32_t K[1024];
    uint4 raw[STAGE];             // records of the next stage, copied asynchronously
    int4 A[STAGE];                // U, V, S, Wh = Wq >> 16
    uint4 B[STAGE];               // QL low, Wl = Wq & 0xFFFF, QL high, unused
    uint16_t list[RT / 32][STAGE]; // per warp: record | touched blocks of its column << 9; small records
                                   // touching all four blocks from the front, other small ones from the back
    uint16_t large[RT / 32][STAGE]; // per warp: the same for records with QL > 2^30
    uint16_t cand[8][STAGE];       // per block column: records whose support may reach it
    uint32_t ncand[2][8];          // candidate counts, two sets used on alternate stages
};
// dynamic shared memory: four CTAs per SM fit in its 228 KB with the 1 KB each CTA reserves
static_assert(4 * (sizeof(SplatSmem) + 1024) <= 228 * 1024, "four splat CTAs per SM");

// 16-byte global -> shared copy that bypasses registers and L1 (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async16(uint32_t smem_addr, const uint4 *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A record is "small" when QL <= 2^30: every pixel of a block its support reaches then lies
// within 2^15 + 8 px of its centre on each axis (in 1/256 px), so dx^2 + dy^2 < 2^32 and the
// table index (q S) >> 37 is the high word of a 32 x 32 product shifted by 5.
constexpr unsigned long long QL_SMALL = 1ull << 30;

// Each warp owns up to SPLAT_SLOTS blocks of 8 x 4 pixels in one block column: with the tile's
// nbx x nby blocks, sh = the smallest count with nbx ceil(nby / sh) <= 8 warps, warp w takes column
// w % nbx and the block rows g, g + ng, g + 2 ng, ... (g = w / nbx, ng = ceil(nby / sh)), so the
// rows of a column are interleaved between its warps and their work stays balanced.
__host__ __device__ __forceinline__ int strip_height(int nbx, int nby)
{
    int sh = 1;
    while (sh < SPLAT_SLOTS && nbx * ((nby + sh - 1) / sh) > RT / 32) ++sh;
    return sh;
}

// Splats records [it.y, it.z) of tile `tile` (index inside the view) of view P into img; COUNT
// adds the pixel updates to `hits`.  Each
// lane owns one pixel column position of its warp's strip and one pixel in every block of it;
// a record's centre offset in x and its square are computed once per strip, not once per block.
template <bool COUNT>
__device__ __forceinline__ void splat_item(const uint4 *__restrict__ rec, const uint4 it, const uint32_t tile,
                                           const Proj &P, unsigned long long *__restrict__ img, SplatSmem &sm,
                                           unsigned &hits)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = gbd::lanemask_lt();
    const int tx = (int)(tile % (uint32_t)P.tiles_x), ty = (int)(tile / (uint32_t)P.tiles_x);
    const int X0 = tx * P.TW, Y0 = ty * P.TH;
    const int TWc = min(P.TW, P.W - X0), THc = min(P.TH, P.H - Y0); // tile clipped to the image
    const int nbx = (P.TW + 7) >> 3, nby = (P.TH + 3) >> 2;
    const int sh = strip_height(nbx, nby);
    const int ng = (nby + sh - 1) / sh;                    // row groups
    const int scol = warp % nbx, srow = warp / nbx;         // block column, first block row
    const bool active = warp < nbx * ng;                    // warp-uniform
    const int bx0 = scol * 8;
    const int pxl = bx0 + (lane & 7), pyl0 = srow * 4 + (lane >> 3);
    const int pxv = (X0 + pxl) * 256 + 128, pyv0 = (Y0 + pyl0) * 256 + 128;
    // blocks k of the strip that exist inside the clipped tile; their pixel-centre rectangles
    unsigned kvalid = 0;
#pragma unroll
    for (int k = 0; k < SPLAT_SLOTS; ++k)
        if (k < sh && srow + k * ng < nby && bx0 < TWc && (srow + k * ng) * 4 < THc) kvalid |= 1u << k;
    if (!active) kvalid = 0;
    const int cx0 = (X0 + bx0) * 256 + 128, cx1 = (X0 + min(bx0 + 7, TWc - 1)) * 256 + 128;
    unsigned long long acc[SPLAT_SLOTS];
    uint32_t acc_lo[SPLAT_SLOTS];
    unsigned hk[SPLAT_SLOTS];
#pragma unroll
    for (int k = 0; k < SPLAT_SLOTS; ++k) {
        acc[k] = 0ull;
        acc_lo[k] = 0u;
        hk[k] = 0u;
    }
    const int dstep = ng * 1024; // y offset between the warp's consecutive blocks, 1/256 px
    uint16_t *lst = sm.list[warp], *lrg = sm.large[warp];
    // records reach shared memory through `raw`, copied (cp.async) one stage ahead of their use
    const uint32_t raw_addr = (uint32_t)__cvta_generic_to_shared(&sm.raw[threadIdx.x]);
    for (int t = threadIdx.x; t < STAGE; t += RT)
        if (it.y + t < it.z) cp_async16(raw_addr + 16u * (uint32_t)(t - threadIdx.x), rec + it.y + t);
    cp_async_commit();
    if (threadIdx.x < 16) sm.ncand[threadIdx.x >> 3][threadIdx.x & 7] = 0u;
    int par = 0;
    for (uint32_t base = it.y; base < it.z; base += STAGE, par ^= 1) {
        cp_async_wait_all();
        __syncthreads();
        // the other set of counts was last read two stages ago: clear it for the next stage
        if (threadIdx.x < 8) sm.ncand[par ^ 1][threadIdx.x] = 0u;
        const int nb = (int)min((uint32_t)STAGE, it.z - base);
        for (int t = threadIdx.x; t < nb; t += RT) {
            const uint4 R = sm.raw[t];
            const unsigned long long Wq = __float2ull_rn(__uint_as_float(R.w));
            const unsigned long long QL = 140737488355327ull / (unsigned long long)R.z + 1ull;
            sm.A[t] = make_int4((int)R.x, (int)R.y, (int)R.z, (int)(uint32_t)(Wq >> 16));
            sm.B[t] = make_uint4((uint32_t)QL, (uint32_t)(Wq & 0xFFFFull), (uint32_t)(QL >> 32), 0u);
            // block columns whose pixel centres may lie inside the support (|x - U| < sqrt(QL),
            // rounded up): a superset of the columns the exact per-block test can accept
            const int rq = (int)sqrtf((float)QL) + 2;
            const int lx0 = ((int)R.x - 128 - rq) >> 8, lx1 = ((int)R.x - 128 + rq) >> 8; // floor
            const int c0 = max(0, lx0 - X0) >> 3, c1 = min(TWc - 1, lx1 - X0) >> 3;
            if (lx1 - X0 >= 0)
                for (int c = c0; c <= c1; ++c) sm.cand[c][atomicAdd(&sm.ncand[par][c], 1u)] = (uint16_t)t;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < STAGE; t += RT)
            if (base + STAGE + t < it.z)
                cp_async16(raw_addr + 16u * (uint32_t)(t - threadIdx.x), rec + base + STAGE + t);
        cp_async_commit();
        if (!kvalid) continue; // warp-uniform
        // records whose support reaches a pixel centre of a block of this strip: exact test
        // q_min < QL against each block's pixel-centre rectangle
        int nf = 0, np = 0, nl = 0;
        const int nc = (int)sm.ncand[par][scol];
        for (int j0 = 0; j0 < nc; j0 += 32) {
            const int j = j0 + lane < nc ? sm.cand[scol][j0 + lane] : 0;
            unsigned m = 0;
            bool small = false;
            if (j0 + lane < nc) {
                const int4 A = sm.A[j];
                const uint4 B = sm.B[j];
                const unsigned long long QL = ((unsigned long long)B.z << 32) | B.x;
                small = QL <= QL_SMALL;
                const long long ex = (long long)A.x - (long long)min(max(A.x, cx0), cx1);
                const unsigned long long ex2 = (unsigned long long)(ex * ex);
#pragma unroll
                for (int k = 0; k < SPLAT_SLOTS; ++k) {
                    if (!(kvalid >> k & 1u)) continue;
                    const int by = (srow + k * ng) * 4;
                    const int cy0 = (Y0 + by) * 256 + 128, cy1 = (Y0 + min(by + 3, THc - 1)) * 256 + 128;
                    const long long ey = (long long)A.y - (long long)min(max(A.y, cy0), cy1);
                    if (ex2 + (unsigned long long)(ey * ey) < QL) m |= 1u << k;
                }
            }
            const bool tf = m == 0xFu && small, tp = m && m != 0xFu && small, tl = m && !small;
            const uint32_t mf = __ballot_sync(0xffffffffu, tf), mp = __ballot_sync(0xffffffffu, tp),
                           ml = __ballot_sync(0xffffffffu, tl);
            const uint16_t e = (uint16_t)(j | (m << 9));
            if (tf) lst[nf + __popc(mf & lt)] = e;
            if (tp) lst[STAGE - 1 - (np + __popc(mp & lt))] = e;
            if (tl) lrg[nl + __popc(ml & lt)] = e;
            nf += __popc(mf);
            np += __popc(mp);
            nl += __popc(ml);
        }
        __syncwarp();
        // small records touching all four blocks: no per-block test, four independent chains
#pragma unroll 4
        for (int i = 0; i < nf; ++i) {
            const int j = lst[i] & 511;
            const int4 A = sm.A[j];
            const uint2 B = *reinterpret_cast<const uint2 *>(&sm.B[j]); // QL, Wl
            const int dx = pxv - A.x;
            const uint32_t dx2 = (uint32_t)(dx * dx);
            const int dy0 = pyv0 - A.y;
#pragma unroll
            for (int k = 0; k < SPLAT_SLOTS; ++k) {
                const int dy = dy0 + k * dstep;
                const uint32_t q = dx2 + (uint32_t)(dy * dy);
                if (q < B.x) {
                    const uint32_t idx = __umulhi(q, (uint32_t)A.z) >> 5;
                    const uint32_t kv = (uint32_t)sm.K[idx];
                    acc[k] += (unsigned long long)(uint32_t)A.w * kv;
                    acc_lo[k] += (B.y * kv) >> 16;
                    if (COUNT) ++hk[k];
                }
            }
        }
        // lanes whose pixel lies outside the tile compute too; their sums are never stored
#pragma unroll 2
        for (int i = STAGE - np; i < STAGE; ++i) {
            const uint32_t e = lst[i];
            const int j = e & 511;
            const int4 A = sm.A[j];
            const uint2 B = *reinterpret_cast<const uint2 *>(&sm.B[j]); // QL, Wl
            const int dx = pxv - A.x;
            const uint32_t dx2 = (uint32_t)(dx * dx);
            const int dy0 = pyv0 - A.y;
#pragma unroll
            for (int k = 0; k < SPLAT_SLOTS; ++k) {
                if (!(e >> (9 + k) & 1u)) continue; // warp-uniform
                const int dy = dy0 + k * dstep;
                const uint32_t q = dx2 + (uint32_t)(dy * dy);
                if (q < B.x) {
                    const uint32_t idx = __umulhi(q, (uint32_t)A.z) >> 5;
                    const uint32_t kv = (uint32_t)sm.K[idx];
                    acc[k] += (unsigned long long)(uint32_t)A.w * kv;
                    acc_lo[k] += (B.y * kv) >> 16;
                    if (COUNT) ++hk[k];
                }
            }
        }
        for (int i = 0; i < nl; ++i) {
            const uint32_t e = lrg[i];
            const int j = e & 511;
            const int4 A = sm.A[j];
            const uint4 B = sm.B[j];
            const unsigned long long QL = ((unsigned long long)B.z << 32) | B.x;
            const int dx = pxv - A.x;
            const long long dx2 = (long long)dx * dx;
            const int dy0 = pyv0 - A.y;
#pragma unroll
            for (int k = 0; k < SPLAT_SLOTS; ++k) {
                if (!(e >> (9 + k) & 1u)) continue;
                const int dy = dy0 + k * dstep;
                const unsigned long long q = (unsigned long long)(dx2 + (long long)dy * dy);
                if (q < QL) {
                    const uint32_t idx = (uint32_t)((q * (unsigned long long)(uint32_t)A.z) >> 37);
                    const uint32_t kv = (uint32_t)sm.K[idx];
                    acc[k] += (unsigned long long)(uint32_t)A.w * kv;
                    acc_lo[k] += (B.y * kv) >> 16;
                    if (COUNT) ++hk[k];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < SPLAT_SLOTS; ++k) {
        const int pyl = pyl0 + 4 * ng * k;
        if (!(kvalid >> k & 1u) || pxl >= TWc || pyl >= THc) continue;
        if (COUNT) hits += hk[k];
        const unsigned long long v = acc[k] + acc_lo[k];
        if (v) atomicAdd(&img[(size_t)(Y0 + pyl) * P.W + (X0 + pxl)], v);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(RT, 4) k_splat_tiles(const uint4 *__restrict__ rec, const uint4 *__restrict__ items,
                                                       Proj P, unsigned long long *__restrict__ img,
                                                       FrameStatsDev *stats)
{
    extern __shared__ __align__(16) unsigned char splat_smem[];
    SplatSmem &sm = *reinterpret_cast<SplatSmem *>(splat_smem);
    for (int i = threadIdx.x; i < 1024; i += RT) sm.K[i] = g_ktab[P.kernel][i];
    unsigned hits = 0;
    const uint4 it = items[blockIdx.x];
    splat_item<COUNT>(rec, it, it.x, P, img, sm, hits);
    if (COUNT) count_hits(hits, stats);
}

// ------------------------------------------------------------------ R4
__global__ void k_image_max(const unsigned long long *img, size_t n, unsigned long long *out)
{
    unsigned long long m = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = img[i] > m ? img[i] : m;
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// out = 0 if I <= lo, else min(255, rne(255 ln(I/lo) / ln(hi/lo))), I = acc 2^-32
__global__ void k_tonemap(const unsigned long long *img, size_t n, const unsigned long long *maxv, int auto_range,
                          double lo_acc_fixed, double hi_acc_fixed, uint8_t *out)
{
    __shared__ double s_lo;
    __shared__ float s_l2lo, s_scale;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        double hi = hi_acc_fixed, lo = lo_acc_fixed;
        if (auto_range) {
            hi = (double)*maxv;
            lo = hi * 1e-4;
        }
        s_ok = (hi > 0.0 && lo > 0.0 && hi > lo) ? 1 : 0;
        s_lo = lo;
        s_l2lo = s_ok ? (float)log2(lo) : 0.0f;
        s_scale = s_ok ? (float)(255.0 / log2(hi / lo)) : 0.0f;
    }
    __syncthreads();
    const double lo = s_lo;
    const float l2lo = s_l2lo, scale = s_scale;
    const int ok = s_ok;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long a = img[i];
        uint8_t o = 0;
        if (ok && (double)a > lo) {
            const float t = rintf((log2f((float)a) - l2lo) * scale);
            o = (uint8_t)(t > 255.0f ? 255.0f : (t < 0.0f ? 0.0f : t));
        }
        out[i] = o;
    }
}

__global__ void k_project_debug(const float4 *pts4, const float *h, size_t n, Proj P, long long *out)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 q = pts4[i];
        Splat s;
        const int r = project(P, q.x, q.y, q.z, q.w, h[i], s);
        out[5 * i + 0] = r;
        out[5 * i + 1] = r == 1 ? s.U : 0;
        out[5 * i + 2] = r == 1 ? s.V : 0;
        out[5 * i + 3] = r == 1 ? (long long)s.S : 0;
        out[5 * i + 4] = r == 1 ? (long long)__float2ull_rn(s.Wf) : 0;
    }
}

__global__ void k_morton_plain(const float *xyz, size_t n, double lx, double ly, double lz, double scale,
                               uint64_t *keys)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        keys[i] = gbd::morton_key(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lx, ly, lz, scale);
}

// ------------------------------------------------------------------ frame driver
// A frame is binned and splatted in one pass when its (tile, splat) records fit the record
// budget; otherwise the projected points are split into ranges whose records fit, each range is
// binned and splatted on its own, and the integer partial images add up to the same image.
constexpr unsigned long long RECORD_BUDGET_DEFAULT = 1ull << 28; // 4 GiB of records
constexpr unsigned long long RECORD_BUDGET_MAX = 1ull << 31;     // offsets stay 32-bit

struct PassCounts {
    unsigned long long pairs, points; // records of the pass (both streams when partitioned), points
    uint32_t items, small_items;      // splat work items, small-box work items (partitioned only)
};

// The caller's particle arrays are in no spatial order: they are binned by the partitioned passes
// (one shared-memory histogram per CTA) whenever the tile count fits shared memory.
template <class Src> constexpr bool unordered_source() { return false; }
template <> constexpr bool unordered_source<SrcFlat>() { return true; }

template <class Src> bool partitioned(const Proj &P)
{
    return unordered_source<Src>() && (uint32_t)(P.tiles_x * P.tiles_y) <= PART_MAX_TILES;
}

template <class Src>
PassCounts bin_count(gblod_renderer *r, const Src &src, const Proj &P, unsigned long long lo, unsigned long long hi,
                     FrameStatsDev *stats, cudaStream_t s)
{
    const Allocator &A = r->A;
    const uint32_t ntiles = (uint32_t)(P.tiles_x * P.tiles_y);
    const unsigned G = (unsigned)persistent_blocks(4);
    if (partitioned<Src>(P)) {
        const size_t nh = (size_t)ntiles * G;
        r->cta_hist.ensure(A, 2 * nh, s);
        r->cta_off.ensure(A, 2 * nh + 1, s);
        r->tile_cnt_s.ensure(A, ntiles, s);
        r->tile_off_s.ensure(A, ntiles + 1, s);
        r->item_cnt_s.ensure(A, ntiles, s);
        r->item_off_s.ensure(A, ntiles + 1, s);
        launch(GBLOD_K_PROJECT_COUNT, k_project_hist<Src>, dim3(G), dim3(RT), (size_t)ntiles * 8, s, src, P, lo, hi,
               r->cta_hist.p, r->status, stats);
        scan_exclusive_u32(A, r->scan, r->cta_hist.p, r->cta_off.p, 2 * nh, r->cta_off.p + 2 * nh, s);
        const dim3 tg((ntiles + 255) / 256);
        launch(GBLOD_K_RENDER_OTHER, k_tiles_from_hist, tg, dim3(256), 0, s, ntiles, G, (const uint32_t *)r->cta_off.p,
               (const uint32_t *)(r->cta_off.p + nh), r->tile_cnt.p, r->tile_off.p);
        launch(GBLOD_K_RENDER_OTHER, k_tiles_from_hist, tg, dim3(256), 0, s, ntiles, G,
               (const uint32_t *)(r->cta_off.p + nh), (const uint32_t *)(r->cta_off.p + 2 * nh), r->tile_cnt_s.p,
               r->tile_off_s.p);
        GB_CUDA(cudaMemcpyAsync(r->tile_off.p + ntiles, r->cta_off.p + nh, 4, cudaMemcpyDeviceToDevice, s));
        launch(GBLOD_K_RENDER_OTHER, k_tile_items_n, tg, dim3(256), 0, s, ntiles, (const uint32_t *)r->tile_cnt_s.p,
               ITEM_SMALL, r->item_cnt_s.p);
        scan_exclusive_u32(A, r->scan, r->item_cnt_s.p, r->item_off_s.p, ntiles, r->item_off_s.p + ntiles, s);
    } else {
        GB_CUDA(cudaMemsetAsync(r->tile_cnt.p, 0, (size_t)ntiles * 4, s));
        launch(GBLOD_K_PROJECT_COUNT, k_project_count<Src>, dim3(G), dim3(RT), 0, s, src, P, lo, hi, r->tile_cnt.p,
               r->status, stats);
        scan_exclusive_u32(A, r->scan, r->tile_cnt.p, r->tile_off.p, ntiles, r->tile_off.p + ntiles, s);
    }
    launch(GBLOD_K_RENDER_OTHER, k_tile_items, dim3((ntiles + 255) / 256), dim3(256), 0, s, ntiles,
           (const uint32_t *)r->tile_cnt.p, r->item_cnt.p);
    scan_exclusive_u32(A, r->scan, r->item_cnt.p, r->item_off.p, ntiles, r->item_off.p + ntiles, s);
    unsigned long long *h = static_cast<unsigned long long *>(r->hs.get(40));
    h[2] = h[3] = h[4] = 0;
    GB_CUDA(cudaMemcpyAsync(h, &stats->pairs, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(h + 1, &stats->points, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(h + 2, r->item_off.p + ntiles, 4, cudaMemcpyDeviceToHost, s));
    if (partitioned<Src>(P)) {
        const size_t nh = (size_t)ntiles * G;
        GB_CUDA(cudaMemcpyAsync(h + 3, r->item_off_s.p + ntiles, 4, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(h + 4, r->cta_off.p + 2 * nh, 4, cudaMemcpyDeviceToHost, s));
    }
    GB_CUDA(cudaStreamSynchronize(s));
    const bool part = partitioned<Src>(P);
    return PassCounts{part ? (h[4] & 0xFFFFFFFFull) : h[0], h[1], (uint32_t)(h[2] & 0xFFFFFFFFull),
                      (uint32_t)(h[3] & 0xFFFFFFFFull)};
}

template <class Src>
void bin_splat(gblod_renderer *r, const Src &src, const Proj &P, unsigned long long lo, unsigned long long hi,
               const PassCounts &pc, unsigned long long *img, cudaStream_t s)
{
    const Allocator &A = r->A;
    const uint32_t ntiles = (uint32_t)(P.tiles_x * P.tiles_y);
    r->records.ensure(A, pc.pairs, s);
    r->items.ensure(A, (size_t)pc.items + pc.small_items, s);
    if (partitioned<Src>(P)) {
        launch(GBLOD_K_PROJECT_SCATTER, k_project_scatter_part<Src>, dim3((unsigned)persistent_blocks(4)), dim3(RT),
               (size_t)ntiles * 8, s, src, P, lo, hi, (const uint32_t *)r->cta_off.p, r->records.p, img,
               r->count_updates ? r->stats : (FrameStatsDev *)nullptr);
        launch(GBLOD_K_RENDER_OTHER, k_fill_items_n, dim3((ntiles + 255) / 256), dim3(256), 0, s, ntiles,
               (const uint32_t *)r->tile_cnt_s.p, (const uint32_t *)r->tile_off_s.p, (const uint32_t *)r->item_off_s.p,
               ITEM_SMALL, r->items.p + pc.items);
        launch(GBLOD_K_SPLAT, r->count_updates ? k_splat_small<true> : k_splat_small<false>, dim3(pc.small_items),
               dim3(RT), 0, s, (const uint4 *)r->records.p, (const uint4 *)(r->items.p + pc.items), P, img, r->stats);
    } else {
        GB_CUDA(cudaMemcpyAsync(r->tile_cur.p, r->tile_off.p, (size_t)ntiles * 4, cudaMemcpyDeviceToDevice, s));
        launch(GBLOD_K_PROJECT_SCATTER, k_project_scatter<Src>, dim3((unsigned)persistent_blocks(4)), dim3(RT), 0, s,
               src, P, lo, hi, r->tile_cur.p, r->records.p, img,
               r->count_updates ? r->stats : (FrameStatsDev *)nullptr);
    }
    launch(GBLOD_K_RENDER_OTHER, k_fill_items, dim3((ntiles + 255) / 256), dim3(256), 0, s, ntiles,
           (const uint32_t *)r->tile_cnt.p, (const uint32_t *)r->tile_off.p, (const uint32_t *)r->item_off.p,
           r->items.p);
    launch(GBLOD_K_SPLAT, r->count_updates ? k_splat_tiles<true> : k_splat_tiles<false>, dim3(pc.items), dim3(RT),
           sizeof(SplatSmem), s, (const uint4 *)r->records.p, (const uint4 *)r->items.p, P, img, r->stats);
}

template <class Src>
void frame_common(gblod_renderer *r, const Src &src, const Proj &P, const gblod_render_params &rp, uint8_t *image,
                  uint64_t *accum, cudaStream_t s)
{
    const Allocator &A = r->A;
    const uint32_t ntiles = (uint32_t)(P.tiles_x * P.tiles_y);
    r->count_updates = (rp.flags & GBLOD_RENDER_COUNT_UPDATES) != 0;
    r->tile_cnt.ensure(A, ntiles, s);
    r->tile_off.ensure(A, ntiles + 1, s);
    r->tile_cur.ensure(A, ntiles, s);
    r->item_cnt.ensure(A, ntiles, s);
    r->item_off.ensure(A, ntiles + 1, s);
    r->pass_stats.ensure(A, 1, s);
    const size_t npix = (size_t)P.W * P.H;
    unsigned long long *img = reinterpret_cast<unsigned long long *>(accum);
    if (!img) {
        r->accum.ensure(A, npix, s);
        img = r->accum.p;
    }
    GB_CUDA(cudaMemsetAsync(img, 0, npix * 8, s));
    const unsigned long long RECORD_BUDGET =
        rp.record_budget ? std::min<unsigned long long>(rp.record_budget, RECORD_BUDGET_MAX) : RECORD_BUDGET_DEFAULT;
    // whole frame first; its counts also give the frame statistics
    const PassCounts all = bin_count(r, src, P, 0ull, ~0ull, r->stats, s);
    const unsigned long long tl[1] = {ntiles};
    GB_CUDA(cudaMemcpyAsync(&r->stats->tiles, tl, 8, cudaMemcpyHostToDevice, s));
    if (all.pairs <= RECORD_BUDGET) {
        bin_splat(r, src, P, 0ull, ~0ull, all, img, s);
    } else {
        // split the point range until every piece's records fit the budget (a single point
        // may exceed it; its records always fit the 2^31 maximum)
        const unsigned long long pieces =
            std::max(1ull, std::min(all.points, (all.pairs + RECORD_BUDGET - 1) / RECORD_BUDGET * 2));
        std::vector<std::pair<unsigned long long, unsigned long long>> todo;
        for (unsigned long long k = pieces; k-- > 0;) {
            const unsigned long long lo = all.points * k / pieces, hi = all.points * (k + 1) / pieces;
            if (hi > lo) todo.emplace_back(lo, hi);
        }
        while (!todo.empty()) {
            const auto [lo, hi] = todo.back();
            todo.pop_back();
            GB_CUDA(cudaMemsetAsync(r->pass_stats.p, 0, sizeof(FrameStatsDev), s));
            const PassCounts pc = bin_count(r, src, P, lo, hi, r->pass_stats.p, s);
            if (pc.pairs > RECORD_BUDGET && hi - lo > 1) {
                const unsigned long long mid = lo + (hi - lo) / 2;
                todo.emplace_back(mid, hi);
                todo.emplace_back(lo, mid);
                continue;
            }
            if (pc.pairs > RECORD_BUDGET_MAX) fail(GBLOD_ERR_RANGE, "one point needs more than 2^31 tile records");
            bin_splat(r, src, P, lo, hi, pc, img, s);
        }
    }
    if (image) {
        r->maxv.ensure(A, 1, s);
        double lo = 0.0, hi = 0.0;
        if (rp.tone_auto) {
            GB_CUDA(cudaMemsetAsync(r->maxv.p, 0, 8, s));
            launch(GBLOD_K_TONEMAP, k_image_max, dim3(persistent_blocks(2)), dim3(256), 0, s,
                   (const unsigned long long *)img, npix, r->maxv.p);
        } else {
            lo = std::ldexp(rp.tone_lo, 32);
            hi = std::ldexp(rp.tone_hi, 32);
        }
        launch(GBLOD_K_TONEMAP, k_tonemap, dim3(persistent_blocks(2)), dim3(256), 0, s,
               (const unsigned long long *)img, npix, (const unsigned long long *)r->maxv.p, rp.tone_auto ? 1 : 0,
               lo, hi, image);
    }
}


// ------------------------------------------------------------------ batched views (no host waits)
// Many views -- each with its own camera, resolution and octree -- rendered by one set of
// launches: R1 walks (view, node) pairs, the points of all selected nodes of all views form one
// flat index space, screen tiles of all views one global tile space, and persistent kernels read
// every data-dependent count from device memory.  Nothing waits on the host, so the sequence can
// be captured in a CUDA graph.  Scratch has a reserved capacity; a batch that needs more sets the
// sticky capacity bit of the renderer's status instead of growing it.
constexpr unsigned ST_CAPACITY = 4u;
constexpr int VIEWS_PER_CHUNK = 40;

struct ViewDev {
    Proj P;
    Frustum F;
    const gblod_node *nodes;
    const float4 *pts4;
    const float *hs;
    const ushort4 *q4;   // non-null: draw the 16-bit block codes
    const uint16_t *qw;
    const float4 *qa;
    unsigned long long *accum;
    uint8_t *image;
    unsigned long long pix_base;
    uint32_t tile_base, n_nodes;
    double lo_acc, hi_acc; // fixed tone range in accumulator units (unused when automatic)
};

struct ViewChunk {
    int first, n;
    ViewDev v[VIEWS_PER_CHUNK];
};
static_assert(sizeof(ViewChunk) < 30000, "kernel parameter block too large");

__global__ void k_set_views(ViewChunk c, ViewDev *dst)
{
    for (int i = threadIdx.x; i < c.n; i += blockDim.x) dst[c.first + i] = c.v[i];
}

__global__ void k_bzero(const ViewDev *__restrict__ views)
{
    const ViewDev &V = views[blockIdx.y];
    const size_t n = (size_t)V.P.W * V.P.H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        V.accum[i] = 0ull;
}

__global__ void k_bselect_init(const ViewDev *__restrict__ views, int n, unsigned long long *front, uint32_t *cnt)
{
    for (int v = threadIdx.x; v < n; v += blockDim.x)
        if (views[v].n_nodes) front[atomicAdd(cnt, 1u)] = (unsigned long long)v << 32;
}

__global__ void __launch_bounds__(RT) k_bselect_level(const ViewDev *__restrict__ views,
                                                      const unsigned long long *__restrict__ fin, const uint32_t *nin,
                                                      unsigned long long *__restrict__ fout, uint32_t *nout,
                                                      unsigned long long *__restrict__ sel, uint32_t *nsel)
{
    const uint32_t n = *nin;
    const uint32_t lt = gbd::lanemask_lt();
    const int lane = threadIdx.x & 31;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        int cls = 0;
        unsigned long long ent = 0;
        uint32_t ccount = 0, cfirst = 0;
        if (i < n) {
            ent = fin[i];
            const int v = (int)(ent >> 32);
            const gblod_node g = views[v].nodes[(uint32_t)ent];
            cls = classify(g, views[v].F);
            ccount = g.child_count;
            cfirst = g.child_first;
        }
        const uint32_t em = __ballot_sync(0xffffffffu, cls == 1);
        if (em) {
            const int leader = __ffs(em) - 1;
            uint32_t b = 0;
            if (lane == leader) b = atomicAdd(nsel, (uint32_t)__popc(em));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (cls == 1) sel[b + __popc(em & lt)] = ent;
        }
        uint32_t want = cls == 2 ? ccount : 0u, incl = want;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        if (total) {
            uint32_t b = 0;
            if (lane == 31) b = atomicAdd(nout, total);
            b = __shfl_sync(0xffffffffu, b, 31);
            const uint32_t at = b + incl - want;
            const unsigned long long hiv = ent & 0xFFFFFFFF00000000ull;
            for (uint32_t k = 0; k < want; ++k) fout[at + k] = hiv | (cfirst + k);
        }
    }
}

__global__ void k_bsel_counts(const ViewDev *__restrict__ views, const unsigned long long *__restrict__ sel,
                              const uint32_t *nsel, uint32_t cap, unsigned long long *counts)
{
    const uint32_t n = *nsel;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        unsigned long long c = 0;
        if (i < n) {
            const unsigned long long e = sel[i];
            c = views[e >> 32].nodes[(uint32_t)e].point_count;
        }
        counts[i] = c;
    }
}

__global__ void k_bsel_base(const ViewDev *__restrict__ views, const unsigned long long *__restrict__ sel,
                            const uint32_t *nsel, const unsigned long long *__restrict__ pfx, long long *base,
                            FrameStatsDev *stats)
{
    const uint32_t n = *nsel;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long e = sel[i];
        base[i] = (long long)views[e >> 32].nodes[(uint32_t)e].point_first - (long long)pfx[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) stats->nodes_selected = n;
}

struct SrcBatch {
    const ViewDev *views;
    const unsigned long long *sel;
    const unsigned long long *pfx;
    const long long *base;
    const uint32_t *nsel;
    const unsigned long long *total;
};

__device__ __forceinline__ void bsrc_range(const SrcBatch &s, unsigned long long a, unsigned long long b,
                                           uint32_t &j0, uint32_t &j1)
{
    __shared__ uint32_t sj[2];
    if (threadIdx.x < 2) {
        const unsigned long long v = threadIdx.x == 0 ? a : b - 1;
        uint32_t lo = 0, hi = *s.nsel;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s.pfx[mid] <= v) lo = mid; else hi = mid;
        }
        sj[threadIdx.x] = lo;
    }
    __syncthreads();
    j0 = sj[0];
    j1 = sj[1];
    __syncthreads();
}

// point e of the flat space: its view and its data
__device__ __forceinline__ int bsrc_load(const SrcBatch &s, unsigned long long e, uint32_t j0, uint32_t j1, float &x,
                                         float &y, float &z, float &w, float &h)
{
    uint32_t lo = j0, hi = j1 + 1;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s.pfx[mid] <= e) lo = mid; else hi = mid;
    }
    const unsigned long long ent = s.sel[lo];
    const int v = (int)(ent >> 32);
    const unsigned long long p = (unsigned long long)((long long)e + s.base[lo]);
    const ViewDev &V = s.views[v];
    if (V.q4) {
        const uint32_t node = (uint32_t)ent;
        block_decode(V.q4[p], V.qw[p], V.qa[2 * node], V.qa[2 * node + 1], x, y, z, w, h);
    } else {
        const float4 q = V.pts4[p];
        x = q.x; y = q.y; z = q.z; w = q.w;
        h = V.hs[p];
    }
    return v;
}

// Counting pass (SCATTER false) or record pass (true) over the flat point space of a batch; the
// record pass also splats the points with small boxes into their view's image, and counts their
// pixel updates when count_updates is set.
template <bool SCATTER>
__global__ void __launch_bounds__(RT) k_bproject(SrcBatch src, uint32_t *__restrict__ tile_cnt,
                                                 uint32_t *__restrict__ cursor, uint4 *__restrict__ rec,
                                                 unsigned long long rec_cap, unsigned *status, FrameStatsDev *stats,
                                                 int count_updates)
{
    const unsigned long long total = *src.total;
    unsigned hits = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = gbd::lanemask_lt();
    unsigned long long splats = 0, pairs = 0;
    AmpSum amp;
    __shared__ Proj sP[2];
    __shared__ int sV[2];
    for (unsigned long long a = (unsigned long long)blockIdx.x * CHUNK; a < total;
         a += (unsigned long long)gridDim.x * CHUNK) {
        const unsigned long long b = min(total, a + CHUNK);
        uint32_t j0, j1;
        bsrc_range(src, a, b, j0, j1);
        // the chunk's points belong to the views of its first and last nodes, or rarely in between
        if (threadIdx.x < 2) {
            const int vv = (int)(src.sel[threadIdx.x == 0 ? j0 : j1] >> 32);
            sV[threadIdx.x] = vv;
            sP[threadIdx.x] = src.views[vv].P;
        }
        __syncthreads();
        for (unsigned long long e0 = a; e0 < b; e0 += RT) {
            const unsigned long long e = e0 + threadIdx.x;
            int res = 0, v = 0;
            Splat s;
            if (e < b) {
                float x, y, z, w, h;
                v = bsrc_load(src, e, j0, j1, x, y, z, w, h);
                const Proj &Pv = v == sV[0] ? sP[0] : (v == sV[1] ? sP[1] : src.views[v].P);
                res = project(Pv, x, y, z, w, h, s);
            }
            if (!SCATTER) {
                if (__any_sync(0xffffffffu, res < 0) && lane == 0) atomicOr(status, ST_RANGE);
                if (res == 1) amp.add(__float2ull_rn(s.Wf));
            }
            uint32_t n = 0, t00 = 0;
            int tw = 1, tiles_x = 1;
            uint4 r = make_uint4(0u, 0u, 0u, 0u);
            BoxWalk direct;
            if (res == 1) {
                const Proj &P = v == sV[0] ? sP[0] : (v == sV[1] ? sP[1] : src.views[v].P);
                const uint32_t tb = src.views[v].tile_base;
                if (!SCATTER) ++splats;
                int x0, x1, y0, y1;
                const int rad = splat_box(s.U, s.V, s.S, P.W, P.H, x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1) {
                    if (direct_box(x0, x1, y0, y1)) {
                        if (SCATTER)
                            direct = box_walk(s.U, s.V, s.S, __float2ull_rn(s.Wf), rad, x0, x1, y0, y1, P.kernel);
                    } else {
                        const int tx0 = x0 / P.TW, tx1 = x1 / P.TW, ty0 = y0 / P.TH, ty1 = y1 / P.TH;
                        tw = tx1 - tx0 + 1;
                        n = (uint32_t)(tw * (ty1 - ty0 + 1));
                        t00 = tb + (uint32_t)(ty0 * P.tiles_x + tx0);
                        tiles_x = P.tiles_x;
                        if (!SCATTER) pairs += n;
                        r = make_uint4((uint32_t)s.U, (uint32_t)s.V, s.S, __float_as_uint(s.Wf));
                    }
                }
            }
            if (SCATTER) {
                scatter_pairs(n, t00, tw, tiles_x, r, cursor, rec, rec_cap);
                hits += walk_boxes<true>(
                    direct, (uint32_t)v, [&](uint32_t meta, uint32_t i) { return g_ktab[(meta >> 14) & 1u][i]; },
                    [&](uint32_t t, int x, int y, unsigned long long c) {
                        atomicAdd(&src.views[t].accum[(size_t)y * src.views[t].P.W + x], c);
                    });
            } else if (n) {
                // counting: fire-and-forget atomics, so the per-lane loop is cheaper than the
                // warp-cooperative walk
                for (uint32_t m = 0; m < n; ++m) {
                    const uint32_t row = m / (uint32_t)tw;
                    const uint32_t t = t00 + row * (uint32_t)tiles_x + (m - row * (uint32_t)tw);
                    const uint32_t peers = __match_any_sync(__activemask(), t);
                    if (lane == __ffs(peers) - 1) atomicAdd(&tile_cnt[t], (uint32_t)__popc(peers));
                }
            }
        }
        __syncthreads();
    }
    if (!SCATTER) {
        for (int d = 16; d > 0; d >>= 1) {
            splats += __shfl_xor_sync(0xffffffffu, splats, d);
            pairs += __shfl_xor_sync(0xffffffffu, pairs, d);
        }
        if (lane == 0 && splats) atomicAdd(&stats->splats, splats);
        if (lane == 0 && pairs) atomicAdd(&stats->pairs, pairs);
        amp.flush(stats);
    } else if (count_updates) {
        count_hits(hits, stats);
    }
}

// items of every tile of every view; a tile's view comes from the tile bases
__global__ void k_bfill_items(uint32_t ntiles, const ViewDev *__restrict__ views, int nviews,
                              const uint32_t *tile_cnt, const uint32_t *tile_off, const uint32_t *item_off,
                              uint4 *items, uint32_t items_cap, unsigned long long rec_cap,
                              const FrameStatsDev *stats, unsigned *status)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && (stats->pairs > rec_cap || item_off[ntiles] > items_cap)) atomicOr(status, ST_CAPACITY);
    if (t >= ntiles) return;
    int lo = 0, hi = nviews;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (views[mid].tile_base <= t) lo = mid; else hi = mid;
    }
    const uint32_t c = tile_cnt[t], o = tile_off[t], local = t - views[lo].tile_base;
    uint32_t k = item_off[t];
    for (uint32_t s = 0; s < c && k < items_cap; s += ITEM, ++k) {
        const uint32_t b = o + s, e = o + min(c, s + ITEM);
        // records beyond the capacity were never written: clip (the batch is flagged)
        const uint32_t bc = (uint32_t)min((unsigned long long)b, rec_cap), ec = (uint32_t)min((unsigned long long)e, rec_cap);
        items[k] = make_uint4(local, bc, ec, (uint32_t)lo);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(RT, 4) k_bsplat(const uint4 *__restrict__ rec, const uint4 *__restrict__ items,
                                                  const uint32_t *nitems_p, uint32_t items_cap,
                                                  const ViewDev *__restrict__ views, unsigned *next_item,
                                                  FrameStatsDev *stats)
{
    extern __shared__ __align__(16) unsigned char splat_smem[];
    SplatSmem &sm = *reinterpret_cast<SplatSmem *>(splat_smem);
    __shared__ Proj sP;
    __shared__ uint32_t s_item;
    int kernel_loaded = -1;
    unsigned hits = 0;
    const uint32_t nitems = min(*nitems_p, items_cap);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(next_item, 1u);
        __syncthreads();
        const uint32_t i = s_item;
        if (i >= nitems) break;
        const uint4 it = items[i];
        if (threadIdx.x == 0) sP = views[it.w].P;
        __syncthreads();
        const Proj P = sP;
        if (P.kernel != kernel_loaded) {
            for (int j = threadIdx.x; j < 1024; j += RT) sm.K[j] = g_ktab[P.kernel][j];
            kernel_loaded = P.kernel;
        }
        splat_item<COUNT>(rec, it, it.x, P, views[it.w].accum, sm, hits);
    }
    if (COUNT) count_hits(hits, stats);
}

// R4 over the views of a batch: blockIdx.y = view, grid-stride over that view's pixels
__global__ void k_bmax(const ViewDev *__restrict__ views, unsigned long long *maxv)
{
    const ViewDev &V = views[blockIdx.y];
    const size_t n = (size_t)V.P.W * V.P.H;
    unsigned long long m = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = V.accum[i] > m ? V.accum[i] : m;
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&maxv[blockIdx.y], m);
}
__global__ void k_btonemap(const ViewDev *__restrict__ views, const unsigned long long *maxv, int auto_range)
{
    const ViewDev &V = views[blockIdx.y];
    if (!V.image) return;
    __shared__ double s_lo;
    __shared__ float s_l2lo, s_scale;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        double hi = V.hi_acc, lo = V.lo_acc;
        if (auto_range) {
            hi = (double)maxv[blockIdx.y];
            lo = hi * 1e-4;
        }
        s_ok = (hi > 0.0 && lo > 0.0 && hi > lo) ? 1 : 0;
        s_lo = lo;
        s_l2lo = s_ok ? (float)log2(lo) : 0.0f;
        s_scale = s_ok ? (float)(255.0 / log2(hi / lo)) : 0.0f;
    }
    __syncthreads();
    const double lo = s_lo;
    const float l2lo = s_l2lo, scale = s_scale;
    const int ok = s_ok;
    const size_t n = (size_t)V.P.W * V.P.H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long a = V.accum[i];
        uint8_t o = 0;
        if (ok && (double)a > lo) {
            const float t = rintf((log2f((float)a) - l2lo) * scale);
            o = (uint8_t)(t > 255.0f ? 255.0f : (t < 0.0f ? 0.0f : t));
        }
        V.image[i] = o;
    }
}

struct BatchPlan {
    std::vector<ViewDev> host;
    uint32_t ntiles = 0, max_levels = 0;
    unsigned long long npix = 0;
    uint64_t nodes = 0;
};

BatchPlan plan_batch(const gblod_view *views, int n, const gblod_render_params &rp)
{
    if (n > 65535) fail(GBLOD_ERR_INVALID_ARG, "a batch holds at most 65535 views");
    BatchPlan b;
    b.host.resize(n);
    for (int v = 0; v < n; ++v) {
        const gblod_view &V = views[v];
        if (!V.octree) fail(GBLOD_ERR_INVALID_ARG, "batch view has no octree");
        if (!V.d_accum) fail(GBLOD_ERR_INVALID_ARG, "batch views need d_accum");
        check_image(V.camera);
        check_format(V.octree, rp);
        ViewDev &d = b.host[v];
        std::memset(&d, 0, sizeof(d));
        d.P = make_proj(V.camera, rp);
        d.F = make_frustum(V.camera, rp, V.octree);
        if (rp.point_format == GBLOD_POINTS_BLOCK16) {
            d.nodes = V.octree->qnodes;
            d.q4 = V.octree->q4;
            d.qw = V.octree->qw;
            d.qa = V.octree->qa;
        } else {
            d.nodes = V.octree->nodes;
            d.pts4 = V.octree->pts4;
            d.hs = V.octree->hs;
        }
        d.accum = reinterpret_cast<unsigned long long *>(V.d_accum);
        d.image = V.d_image;
        d.pix_base = b.npix;
        d.tile_base = b.ntiles;
        d.n_nodes = (uint32_t)V.octree->n_nodes;
        d.lo_acc = std::ldexp(rp.tone_lo, 32);
        d.hi_acc = std::ldexp(rp.tone_hi, 32);
        const unsigned long long tiles = (unsigned long long)d.P.tiles_x * d.P.tiles_y;
        if ((unsigned long long)b.ntiles + tiles > 0x7FFFFFFFull) fail(GBLOD_ERR_INVALID_ARG, "too many tiles in batch");
        b.ntiles += (uint32_t)tiles;
        b.npix += (unsigned long long)d.P.W * d.P.H;
        b.nodes += V.octree->n_nodes;
        b.max_levels = std::max<uint32_t>(b.max_levels, (uint32_t)V.octree->depth_max + 1);
    }
    if (b.nodes >= 0xFFFFFFFFull) fail(GBLOD_ERR_INVALID_ARG, "too many nodes in batch");
    return b;
}

// the splat kernels stage SplatSmem (above the 48 KB a launch may take without opting in)
void set_splat_smem_limits()
{
    const int bytes = (int)sizeof(SplatSmem);
    GB_CUDA(cudaFuncSetAttribute(k_splat_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GB_CUDA(cudaFuncSetAttribute(k_splat_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GB_CUDA(cudaFuncSetAttribute(k_bsplat<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GB_CUDA(cudaFuncSetAttribute(k_bsplat<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

} // namespace

void reserve_batch(gblod_renderer *r, const gblod_view *views, int n, const gblod_render_params &rp,
                   uint64_t record_capacity, cudaStream_t s)
{
    if (n < 1) fail(GBLOD_ERR_INVALID_ARG, "batch needs at least one view");
    const BatchPlan b = plan_batch(views, n, rp);
    const Allocator &A = r->A;
    const uint64_t rec_cap = record_capacity ? record_capacity : RECORD_BUDGET_DEFAULT;
    if (rec_cap > 0xFFFFFFFFull) fail(GBLOD_ERR_INVALID_ARG, "record capacity must stay below 2^32");
    r->b_views.ensure(A, (size_t)n * sizeof(ViewDev), s);
    r->b_frontA.ensure(A, b.nodes + 1, s);
    r->b_frontB.ensure(A, b.nodes + 1, s);
    r->b_sel.ensure(A, b.nodes + 1, s);
    r->b_counts.ensure(A, b.nodes + 1, s);
    r->b_pfx.ensure(A, b.nodes + 2, s);
    r->b_base.ensure(A, b.nodes + 1, s);
    r->lvl_cnt.ensure(A, b.max_levels + 3, s);
    r->tile_cnt.ensure(A, b.ntiles, s);
    r->tile_off.ensure(A, b.ntiles + 1, s);
    r->tile_cur.ensure(A, b.ntiles, s);
    r->item_cnt.ensure(A, b.ntiles, s);
    r->item_off.ensure(A, b.ntiles + 1, s);
    r->records.ensure(A, rec_cap, s);
    r->items.ensure(A, b.ntiles + rec_cap / ITEM + 1, s);
    r->maxv.ensure(A, n, s);
    // scan temp for the largest scans of this batch
    scan_exclusive_u64(A, r->scan, reinterpret_cast<const uint64_t *>(r->b_counts.p),
                       reinterpret_cast<uint64_t *>(r->b_pfx.p), b.nodes + 1, nullptr, s);
    scan_exclusive_u32(A, r->scan, r->tile_cnt.p, r->tile_off.p, b.ntiles, nullptr, s);
    r->b_rec_cap = rec_cap;
    GB_CUDA(cudaStreamSynchronize(s));
}

void render_batch(gblod_renderer *r, const gblod_view *views, int n, const gblod_render_params &rp, cudaStream_t s)
{
    if (n < 1) fail(GBLOD_ERR_INVALID_ARG, "batch needs at least one view");
    BatchPlan b = plan_batch(views, n, rp);
    const Allocator &A = r->A;
    // scratch must have been reserved (no allocation here, so the call can be graph-captured)
    const uint64_t items_cap = b.ntiles + r->b_rec_cap / ITEM + 1;
    if (r->b_views.cap < (size_t)n * sizeof(ViewDev) || r->b_frontA.cap < b.nodes + 1 || r->b_sel.cap < b.nodes + 1 ||
        r->b_pfx.cap < b.nodes + 2 || r->lvl_cnt.cap < b.max_levels + 3 || r->tile_cnt.cap < b.ntiles ||
        r->tile_off.cap < b.ntiles + 1 || r->item_off.cap < b.ntiles + 1 || r->records.cap < r->b_rec_cap ||
        r->items.cap < items_cap || r->maxv.cap < (size_t)n || r->b_rec_cap == 0)
        fail(GBLOD_ERR_INVALID_ARG, "gblod_render_batch: call gblod_renderer_reserve_batch for this batch first");
    r->last_stream = s;
    r->last_was_lod = false;
    ViewDev *dv = reinterpret_cast<ViewDev *>(r->b_views.p);
    for (int c0 = 0; c0 < n; c0 += VIEWS_PER_CHUNK) {
        ViewChunk ch;
        ch.first = c0;
        ch.n = std::min(VIEWS_PER_CHUNK, n - c0);
        for (int i = 0; i < ch.n; ++i) ch.v[i] = b.host[c0 + i];
        launch(GBLOD_K_RENDER_OTHER, k_set_views, dim3(1), dim3(64), 0, s, ch, dv);
    }
    const unsigned G = (unsigned)persistent_blocks(4);
    GB_CUDA(cudaMemsetAsync(r->stats, 0, offsetof(FrameStatsDev, pixel_updates_total), s));
    GB_CUDA(cudaMemsetAsync(r->lvl_cnt.p, 0, (size_t)(b.max_levels + 3) * 4, s));
    GB_CUDA(cudaMemsetAsync(r->tile_cnt.p, 0, (size_t)b.ntiles * 4, s));
    const dim3 GV((unsigned)std::max(1, (int)G / n), (unsigned)n); // (blocks per view, views)
    launch(GBLOD_K_RENDER_OTHER, k_bzero, GV, dim3(256), 0, s, (const ViewDev *)dv);
    // R1 over (view, node) pairs
    uint32_t *nsel = r->lvl_cnt.p + b.max_levels + 1;
    unsigned long long *fin = r->b_frontA.p, *fout = r->b_frontB.p;
    launch(GBLOD_K_SELECT_NODES, k_bselect_init, dim3(1), dim3(256), 0, s, (const ViewDev *)dv, n, fin, r->lvl_cnt.p);
    for (uint32_t d = 0; d < b.max_levels; ++d) {
        launch(GBLOD_K_SELECT_NODES, k_bselect_level, dim3((unsigned)persistent_blocks(2)), dim3(RT), 0, s,
               (const ViewDev *)dv, (const unsigned long long *)fin, (const uint32_t *)(r->lvl_cnt.p + d), fout,
               r->lvl_cnt.p + d + 1, r->b_sel.p, nsel);
        std::swap(fin, fout);
    }
    const uint32_t cap = (uint32_t)(b.nodes + 1);
    launch(GBLOD_K_SELECT_NODES, k_bsel_counts, dim3(G), dim3(256), 0, s, (const ViewDev *)dv,
           (const unsigned long long *)r->b_sel.p, (const uint32_t *)nsel, cap, r->b_counts.p);
    scan_exclusive_u64(A, r->scan, reinterpret_cast<const uint64_t *>(r->b_counts.p),
                       reinterpret_cast<uint64_t *>(r->b_pfx.p), cap, reinterpret_cast<uint64_t *>(&r->stats->points),
                       s);
    launch(GBLOD_K_SELECT_NODES, k_bsel_base, dim3(G), dim3(256), 0, s, (const ViewDev *)dv,
           (const unsigned long long *)r->b_sel.p, (const uint32_t *)nsel, (const unsigned long long *)r->b_pfx.p,
           r->b_base.p, r->stats);
    // R2: count, offsets, scatter
    const SrcBatch src{dv, r->b_sel.p, r->b_pfx.p, r->b_base.p, nsel, &r->stats->points};
    launch(GBLOD_K_PROJECT_COUNT, k_bproject<false>, dim3(G), dim3(RT), 0, s, src, r->tile_cnt.p,
           (uint32_t *)nullptr, (uint4 *)nullptr, 0ull, r->status, r->stats, 0);
    scan_exclusive_u32(A, r->scan, r->tile_cnt.p, r->tile_off.p, b.ntiles, r->tile_off.p + b.ntiles, s);
    launch(GBLOD_K_RENDER_OTHER, k_tile_items, dim3((b.ntiles + 255) / 256), dim3(256), 0, s, b.ntiles,
           (const uint32_t *)r->tile_cnt.p, r->item_cnt.p);
    scan_exclusive_u32(A, r->scan, r->item_cnt.p, r->item_off.p, b.ntiles, r->item_off.p + b.ntiles, s);
    GB_CUDA(cudaMemcpyAsync(r->tile_cur.p, r->tile_off.p, (size_t)b.ntiles * 4, cudaMemcpyDeviceToDevice, s));
    launch(GBLOD_K_PROJECT_SCATTER, k_bproject<true>, dim3(G), dim3(RT), 0, s, src, (uint32_t *)nullptr,
           r->tile_cur.p, r->records.p, (unsigned long long)r->b_rec_cap, r->status, r->stats,
           (rp.flags & GBLOD_RENDER_COUNT_UPDATES) ? 1 : 0);
    launch(GBLOD_K_RENDER_OTHER, k_bfill_items, dim3((b.ntiles + 255) / 256), dim3(256), 0, s, b.ntiles,
           (const ViewDev *)dv, n, (const uint32_t *)r->tile_cnt.p, (const uint32_t *)r->tile_off.p,
           (const uint32_t *)r->item_off.p, r->items.p, (uint32_t)items_cap, (unsigned long long)r->b_rec_cap,
           (const FrameStatsDev *)r->stats, r->status);
    // R3: persistent over the items of all views
    launch(GBLOD_K_SPLAT, (rp.flags & GBLOD_RENDER_COUNT_UPDATES) ? k_bsplat<true> : k_bsplat<false>, dim3(G), dim3(RT),
           sizeof(SplatSmem), s, (const uint4 *)r->records.p, (const uint4 *)r->items.p,
           (const uint32_t *)(r->item_off.p + b.ntiles), (uint32_t)items_cap, (const ViewDev *)dv,
           r->lvl_cnt.p + b.max_levels + 2, r->stats);
    // R4
    if (rp.tone_auto) {
        GB_CUDA(cudaMemsetAsync(r->maxv.p, 0, (size_t)n * 8, s));
        launch(GBLOD_K_TONEMAP, k_bmax, GV, dim3(256), 0, s, (const ViewDev *)dv, r->maxv.p);
    }
    launch(GBLOD_K_TONEMAP, k_btonemap, GV, dim3(256), 0, s, (const ViewDev *)dv,
           (const unsigned long long *)r->maxv.p, rp.tone_auto ? 1 : 0);
}

namespace {
} // namespace

void renderer_init(gblod_renderer *r, cudaStream_t s)
{
    ensure_tables();
    r->status = static_cast<unsigned *>(r->A.get(sizeof(unsigned), s));
    r->stats = static_cast<FrameStatsDev *>(r->A.get(sizeof(FrameStatsDev), s));
    GB_CUDA(cudaMemsetAsync(r->status, 0, sizeof(unsigned), s));
    GB_CUDA(cudaMemsetAsync(r->stats, 0, sizeof(FrameStatsDev), s));
    GB_CUDA(cudaStreamSynchronize(s));
}

void renderer_release(gblod_renderer *r)
{
    cudaStream_t s = r->last_stream;
    const Allocator &A = r->A;
    if (s) (void)cudaStreamSynchronize(s);
    A.put(r->status, sizeof(unsigned), s);
    A.put(r->stats, sizeof(FrameStatsDev), s);
    r->frontA.release(A, s); r->frontB.release(A, s); r->sel.release(A, s); r->lvl_cnt.release(A, s);
    r->sel_pfx.release(A, s); r->sel_base.release(A, s);
    r->tile_cnt.release(A, s); r->tile_off.release(A, s); r->tile_cur.release(A, s);
    r->cta_hist.release(A, s); r->cta_off.release(A, s);
    r->tile_cnt_s.release(A, s); r->tile_off_s.release(A, s); r->item_cnt_s.release(A, s); r->item_off_s.release(A, s);
    r->item_cnt.release(A, s); r->item_off.release(A, s);
    r->records.release(A, s); r->items.release(A, s); r->accum.release(A, s); r->maxv.release(A, s);
    r->pass_stats.release(A, s);
    r->b_views.release(A, s); r->b_frontA.release(A, s); r->b_frontB.release(A, s); r->b_sel.release(A, s);
    r->b_counts.release(A, s); r->b_pfx.release(A, s); r->b_base.release(A, s);
    r->d_cams.release(A, s); r->d_rec.release(A, s); r->d_cnt.release(A, s); r->d_off.release(A, s);
    r->d_cur.release(A, s); r->d_icnt.release(A, s); r->d_ioff.release(A, s); r->d_items.release(A, s);
    r->scan.buf.release(A, s);
}

void check_format(const gblod_octree *o, const gblod_render_params &rp)
{
    if (rp.point_format == GBLOD_POINTS_BLOCK16 ? !o->has_block16 : !o->has_float)
        fail(GBLOD_ERR_INVALID_ARG, rp.point_format == GBLOD_POINTS_BLOCK16
                                        ? "octree holds no 16-bit block codes (gblod_octree_quantize)"
                                        : "octree holds no fp32 points (dropped after quantisation)");
}

void check_image(const gblod_camera &c)
{
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
        fail(GBLOD_ERR_INVALID_ARG, "camera width/height must be in 1..16384");
}

void render_lod(gblod_renderer *r, const gblod_octree *o, const gblod_camera &cam, const gblod_render_params &rp,
                uint8_t *image, uint64_t *accum, cudaStream_t s, uint32_t part, uint32_t n_parts)
{
    check_image(cam);
    check_format(o, rp);
    r->last_stream = s;
    r->last_was_lod = true;
    const Allocator &A = r->A;
    const Proj P = make_proj(cam, rp);
    GB_CUDA(cudaMemsetAsync(r->stats, 0, offsetof(FrameStatsDev, pixel_updates_total), s));
    const uint64_t nn = o->n_nodes;
    const int levels = o->depth_max + 1;
    r->frontA.ensure(A, nn + 1, s);
    r->frontB.ensure(A, nn + 1, s);
    r->sel.ensure(A, nn + 1, s);
    r->lvl_cnt.ensure(A, levels + 2, s);
    r->sel_pfx.ensure(A, nn + 2, s);
    r->sel_base.ensure(A, nn + 1, s);
    GB_CUDA(cudaMemsetAsync(r->lvl_cnt.p, 0, (size_t)(levels + 2) * 4, s));
    uint32_t *nsel = r->lvl_cnt.p + levels + 1;
    const bool q = rp.point_format == GBLOD_POINTS_BLOCK16;
    const gblod_node *nodes = q ? o->qnodes : o->nodes;
    if (nn > 0) {
        const Frustum fr = make_frustum(cam, rp, o);
        launch(GBLOD_K_SELECT_NODES, k_select_init, dim3(1), dim3(1), 0, s, r->frontA.p, r->lvl_cnt.p);
        uint32_t *fin = r->frontA.p, *fout = r->frontB.p;
        const unsigned G = (unsigned)persistent_blocks(2);
        for (int d = 0; d < levels; ++d) {
            launch(GBLOD_K_SELECT_NODES, k_select_level, dim3(G), dim3(RT), 0, s, nodes, fr,
                   (const uint32_t *)fin, (const uint32_t *)(r->lvl_cnt.p + d), fout, r->lvl_cnt.p + d + 1,
                   r->sel.p, nsel, part, n_parts);
            std::swap(fin, fout);
        }
    }
    launch(GBLOD_K_SELECT_NODES, k_sel_prefix, dim3(1), dim3(1024), 0, s, nodes, (const uint32_t *)r->sel.p,
           (const uint32_t *)nsel, r->sel_pfx.p, r->sel_base.p, r->stats);
    SrcLOD src{o->pts4, o->hs, r->sel_pfx.p, r->sel_base.p, nsel, &r->stats->points};
    if (q) {
        SrcLODQ sq;
        static_cast<SrcLOD &>(sq) = src;
        sq.q4 = o->q4;
        sq.qw = o->qw;
        sq.qa = o->qa;
        sq.sel = r->sel.p;
        frame_common(r, sq, P, rp, image, accum, s);
    } else {
        frame_common(r, src, P, rp, image, accum, s);
    }
}

// R4 alone on a caller's accumulation image (e.g. the sum of the parts of a split frame).
void tonemap_image(gblod_renderer *r, const uint64_t *accum, int W, int H, const gblod_render_params &rp,
                   uint8_t *image, cudaStream_t s)
{
    const size_t npix = (size_t)W * H;
    r->maxv.ensure(r->A, 1, s);
    double lo = 0.0, hi = 0.0;
    if (rp.tone_auto) {
        GB_CUDA(cudaMemsetAsync(r->maxv.p, 0, 8, s));
        launch(GBLOD_K_TONEMAP, k_image_max, dim3(persistent_blocks(2)), dim3(256), 0, s,
               (const unsigned long long *)accum, npix, r->maxv.p);
    } else {
        lo = std::ldexp(rp.tone_lo, 32);
        hi = std::ldexp(rp.tone_hi, 32);
    }
    launch(GBLOD_K_TONEMAP, k_tonemap, dim3(persistent_blocks(2)), dim3(256), 0, s, (const unsigned long long *)accum,
           npix, (const unsigned long long *)r->maxv.p, rp.tone_auto ? 1 : 0, lo, hi, image);
}

void render_brute(gblod_renderer *r, const float *xyz, const float *mass, const float *h, uint64_t n,
                  const gblod_camera &cam, const gblod_render_params &rp, uint8_t *image, uint64_t *accum,
                  cudaStream_t s)
{
    check_image(cam);
    r->last_stream = s;
    r->last_was_lod = false;
    const Proj P = make_proj(cam, rp);
    GB_CUDA(cudaMemsetAsync(r->stats, 0, offsetof(FrameStatsDev, pixel_updates_total), s));
    const unsigned long long pts[1] = {n};
    GB_CUDA(cudaMemcpyAsync(&r->stats->points, pts, 8, cudaMemcpyHostToDevice, s));
    SrcFlat src{xyz, mass, h, n};
    frame_common(r, src, P, rp, image, accum, s);
}

void project_points(const float4 *pts4, const float *h, uint64_t n, const gblod_camera &cam,
                    const gblod_render_params &rp, int64_t *out, cudaStream_t s)
{
    const Proj P = make_proj(cam, rp);
    launch(GBLOD_K_RENDER_OTHER, k_project_debug, dim3(persistent_blocks(4)), dim3(256), 0, s, pts4, h, (size_t)n, P,
           reinterpret_cast<long long *>(out));
}

void morton_keys(const float *xyz, uint64_t n, const double lo[3], double side, uint64_t *keys, cudaStream_t s)
{
    launch(GBLOD_K_MORTON, k_morton_plain, dim3(persistent_blocks(4)), dim3(256), 0, s, xyz, (size_t)n, lo[0], lo[1],
           lo[2], 2097152.0 / side, keys);
}

} // namespace gb

// ------------------------------------------------------------------ fixed-scratch brute-force frame
// For callers that cannot allocate device memory: the scratch of a brute-force frame lives in one
// file-scope device array of fixed size, and nothing is allocated per call.  Host code must not
// pass g_noalloc_scratch itself to a kernel (in host code the name is only a stand-in for the
// device object); its device address is looked up with cudaGetSymbolAddress in the current device's
// context on every call.
namespace gb {
namespace {

constexpr size_t na_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_TILES = GBLOD_NOALLOC_MAX_TILES;
constexpr size_t NA_RECORDS = GBLOD_NOALLOC_MAX_RECORDS;
constexpr size_t NA_ITEMS = NA_TILES + NA_RECORDS / ITEM;
constexpr size_t NA_SCAN_BYTES = 65536;
constexpr size_t NA_OFF_RECORDS = 0;
constexpr size_t NA_OFF_ITEMS = NA_OFF_RECORDS + na_align(NA_RECORDS * sizeof(uint4));
constexpr size_t NA_OFF_TILE_CNT = NA_OFF_ITEMS + na_align(NA_ITEMS * sizeof(uint4));
constexpr size_t NA_OFF_TILE_OFF = NA_OFF_TILE_CNT + na_align(NA_TILES * 4);
constexpr size_t NA_OFF_TILE_CUR = NA_OFF_TILE_OFF + na_align((NA_TILES + 1) * 4);
constexpr size_t NA_OFF_ITEM_CNT = NA_OFF_TILE_CUR + na_align(NA_TILES * 4);
constexpr size_t NA_OFF_ITEM_OFF = NA_OFF_ITEM_CNT + na_align(NA_TILES * 4);
constexpr size_t NA_OFF_SCAN = NA_OFF_ITEM_OFF + na_align((NA_TILES + 1) * 4);
constexpr size_t NA_OFF_STATS = NA_OFF_SCAN + na_align(NA_SCAN_BYTES);
constexpr size_t NA_OFF_STATUS = NA_OFF_STATS + na_align(sizeof(FrameStatsDev));
constexpr size_t NA_OFF_MAXV = NA_OFF_STATUS + na_align(sizeof(unsigned));
constexpr size_t NA_BYTES = NA_OFF_MAXV + na_align(sizeof(unsigned long long));
static_assert(NA_BYTES == GBLOD_NOALLOC_SCRATCH_BYTES, "GBLOD_NOALLOC_SCRATCH_BYTES must match the layout");
// the two scans of NA_TILES counts find their temp space large enough and never allocate
static_assert(scan_temp_bytes(NA_TILES, sizeof(uint32_t)) <= NA_SCAN_BYTES, "scan temp exceeds its fixed region");

} // namespace
} // namespace gb

static __device__ __align__(256) unsigned char g_noalloc_scratch[gb::NA_BYTES];

namespace gb {
namespace {

// Device address of g_noalloc_scratch in the current device's context, looked up on every call
// (a lookup is cheap next to a frame, and a cached address would go stale if the context were
// torn down and created again).
unsigned char *noalloc_scratch()
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    check_cuda(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    if (!p) fail(GBLOD_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    return static_cast<unsigned char *>(p);
}

} // namespace

gblod_status render_brute_noalloc(const float *xyz, const float *mass, const float *h, uint64_t n,
                                  const gblod_camera &cam, const gblod_render_params &rp, uint8_t *image,
                                  uint64_t *accum, cudaStream_t s)
{
    check_image(cam);
    if (!accum) fail(GBLOD_ERR_INVALID_ARG, "gblod_render_bruteforce_noalloc needs d_accum (caller-owned output)");
    const Proj P = make_proj(cam, rp);
    const size_t ntiles = (size_t)P.tiles_x * P.tiles_y;
    if (ntiles > NA_TILES)
        fail(GBLOD_ERR_INVALID_ARG, "gblod_render_bruteforce_noalloc: " + std::to_string(ntiles) +
                                        " screen tiles exceed the fixed maximum of " + std::to_string(NA_TILES));
    ensure_tables();
    unsigned char *base = noalloc_scratch();
    uint4 *records = reinterpret_cast<uint4 *>(base + NA_OFF_RECORDS);
    uint4 *items = reinterpret_cast<uint4 *>(base + NA_OFF_ITEMS);
    uint32_t *tile_cnt = reinterpret_cast<uint32_t *>(base + NA_OFF_TILE_CNT);
    uint32_t *tile_off = reinterpret_cast<uint32_t *>(base + NA_OFF_TILE_OFF);
    uint32_t *tile_cur = reinterpret_cast<uint32_t *>(base + NA_OFF_TILE_CUR);
    uint32_t *item_cnt = reinterpret_cast<uint32_t *>(base + NA_OFF_ITEM_CNT);
    uint32_t *item_off = reinterpret_cast<uint32_t *>(base + NA_OFF_ITEM_OFF);
    FrameStatsDev *stats = reinterpret_cast<FrameStatsDev *>(base + NA_OFF_STATS);
    unsigned *status = reinterpret_cast<unsigned *>(base + NA_OFF_STATUS);
    unsigned long long *maxv = reinterpret_cast<unsigned long long *>(base + NA_OFF_MAXV);
    // the scan helper finds its temp space already large enough and never allocates
    const Allocator none;
    ScanTmp scan;
    scan.buf.p = base + NA_OFF_SCAN;
    scan.buf.cap = NA_SCAN_BYTES;

    // the array keeps the previous call's contents: clear everything that must start at zero
    GB_CUDA(cudaMemsetAsync(tile_cnt, 0, ntiles * 4, s));
    GB_CUDA(cudaMemsetAsync(stats, 0, sizeof(FrameStatsDev), s));
    GB_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
    const SrcFlat src{xyz, mass, h, n};
    const unsigned G = (unsigned)persistent_blocks(4);
    const uint32_t nt = (uint32_t)ntiles;
    launch(GBLOD_K_PROJECT_COUNT, k_project_count<SrcFlat>, dim3(G), dim3(RT), 0, s, src, P, 0ull, ~0ull, tile_cnt,
           status, stats);
    scan_exclusive_u32(none, scan, tile_cnt, tile_off, ntiles, tile_off + ntiles, s);
    launch(GBLOD_K_RENDER_OTHER, k_tile_items, dim3((nt + 255) / 256), dim3(256), 0, s, nt,
           (const uint32_t *)tile_cnt, item_cnt);
    scan_exclusive_u32(none, scan, item_cnt, item_off, ntiles, item_off + ntiles, s);
    if (scan.buf.p != base + NA_OFF_SCAN) fail(GBLOD_ERR_CUDA, "scan temp left the fixed scratch");

    // one read-back into host stack memory (no pinned staging buffer is allocated)
    uint32_t counts[2] = {0, 0};
    unsigned long long amp_hi = 0, pairs64 = 0;
    unsigned st_bits = 0;
    GB_CUDA(cudaMemcpyAsync(&pairs64, &stats->pairs, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&counts[0], tile_off + ntiles, 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&counts[1], item_off + ntiles, 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&amp_hi, &stats->amp_hi, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(&st_bits, status, 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    const uint32_t nitems = counts[1];
    if (pairs64 > NA_RECORDS || nitems > NA_ITEMS)
        fail(GBLOD_ERR_RANGE, "gblod_render_bruteforce_noalloc: the frame needs " + std::to_string(pairs64) +
                                  " (tile, splat) records, more than the fixed maximum of " +
                                  std::to_string(NA_RECORDS));
    const size_t npix = (size_t)P.W * P.H;
    unsigned long long *img = reinterpret_cast<unsigned long long *>(accum);
    GB_CUDA(cudaMemsetAsync(img, 0, npix * 8, s)); // before the scatter, which adds the small boxes
    GB_CUDA(cudaMemcpyAsync(tile_cur, tile_off, ntiles * 4, cudaMemcpyDeviceToDevice, s));
    launch(GBLOD_K_PROJECT_SCATTER, k_project_scatter<SrcFlat>, dim3(G), dim3(RT), 0, s, src, P, 0ull, ~0ull,
           tile_cur, records, img,
           (rp.flags & GBLOD_RENDER_COUNT_UPDATES) ? stats : (FrameStatsDev *)nullptr);
    launch(GBLOD_K_RENDER_OTHER, k_fill_items, dim3((nt + 255) / 256), dim3(256), 0, s, nt,
           (const uint32_t *)tile_cnt, (const uint32_t *)tile_off, (const uint32_t *)item_off, items);
    launch(GBLOD_K_SPLAT, (rp.flags & GBLOD_RENDER_COUNT_UPDATES) ? k_splat_tiles<true> : k_splat_tiles<false>,
           dim3(nitems), dim3(RT), sizeof(SplatSmem), s, (const uint4 *)records, (const uint4 *)items, P, img, stats);
    if (image) {
        double lo = 0.0, hi = 0.0;
        if (rp.tone_auto) {
            GB_CUDA(cudaMemsetAsync(maxv, 0, 8, s));
            launch(GBLOD_K_TONEMAP, k_image_max, dim3(persistent_blocks(2)), dim3(256), 0, s,
                   (const unsigned long long *)img, npix, maxv);
        } else {
            lo = std::ldexp(rp.tone_lo, 32);
            hi = std::ldexp(rp.tone_hi, 32);
        }
        launch(GBLOD_K_TONEMAP, k_tonemap, dim3(persistent_blocks(2)), dim3(256), 0, s,
               (const unsigned long long *)img, npix, (const unsigned long long *)maxv, rp.tone_auto ? 1 : 0, lo, hi,
               image);
    }
    return (st_bits & ST_RANGE) || amp_hi ? GBLOD_ERR_RANGE : GBLOD_OK;
}

} // namespace gb
