// Differentiable float splat: forward image and its adjoint with respect to the points'
// positions, weights and log smoothing lengths, for fitting a node's representatives to the
// full-data image (the paper's goal that the LOD image be indistinguishable from a full render).
//
// Reading (float path, not the exact integer path): fp32 projection as in the renderer,
// sigma = clamp(F exp(l) / zc, sigma_min, sigma_max), kernel
//   K(r) = (exp(-r^2 / 2 sigma^2) - exp(-4.5)) / (2 pi sigma^2 C'),  r < 3 sigma,  C' = 1 - 5.5 e^-4.5
// (unit integral, continuous at the support edge), I = sum_i w_i K_i, fp32 accumulation.
// The adjoint recomputes every per-pixel term tile by tile; nothing is stored per pixel.
#include <cmath>
#include <vector>

#include "render.cuh"

namespace gb {
namespace {

constexpr int DT = 16;           // 16 x 16 tiles, one thread per pixel
constexpr int DRT = DT * DT;     // 256 threads
constexpr uint32_t DITEM = 1024; // records per work item
constexpr float E45 = 0.011108996538242306f;   // exp(-4.5)
constexpr float INV_2PI_C = 0.16951204f;       // 1 / (2 pi (1 - 5.5 exp(-4.5)))

struct DCam {
    float ex, ey, ez, rx, ry, rz, ux, uy, uz, fx, fy, fz;
    float F, CX, CY, ZN, smin, smax;
    int W, H, tiles_x, tiles_y;
};

struct DRec {
    uint32_t idx;
    float u, v, s;
};
__device__ __forceinline__ DRec make_drec() { return DRec{0u, 0.f, 0.f, 1.f}; }

struct DProj {
    float u, v, s, xc, yc, zc;
    bool clamped;
};

__device__ __forceinline__ bool dproject(const DCam &c, const float *xyz, const float *logh, uint32_t i, DProj &o)
{
    const float dx = xyz[3 * i] - c.ex, dy = xyz[3 * i + 1] - c.ey, dz = xyz[3 * i + 2] - c.ez;
    o.xc = c.rx * dx + c.ry * dy + c.rz * dz;
    o.yc = c.ux * dx + c.uy * dy + c.uz * dz;
    o.zc = c.fx * dx + c.fy * dy + c.fz * dz;
    if (!(o.zc > c.ZN)) return false;
    const float iz = 1.0f / o.zc;
    o.u = c.CX + c.F * o.xc * iz;
    o.v = c.CY - c.F * o.yc * iz;
    const float s = c.F * expf(logh[i]) * iz;
    o.clamped = !(s >= c.smin && s <= c.smax);
    o.s = s >= c.smin ? (s <= c.smax ? s : c.smax) : c.smin;
    const float R = 3.0f * o.s + 1.0f;
    return o.u + R >= 0.0f && o.u - R <= (float)c.W && o.v + R >= 0.0f && o.v - R <= (float)c.H;
}

__device__ __forceinline__ void dtiles(const DCam &c, const DProj &o, int &tx0, int &tx1, int &ty0, int &ty1)
{
    const float R = 3.0f * o.s + 1.0f;
    const int x0 = max(0, (int)floorf(o.u - R - 0.5f)), x1 = min(c.W - 1, (int)ceilf(o.u + R - 0.5f));
    const int y0 = max(0, (int)floorf(o.v - R - 0.5f)), y1 = min(c.H - 1, (int)ceilf(o.v + R - 0.5f));
    tx0 = x0 / DT;
    tx1 = x1 / DT;
    ty0 = y0 / DT;
    ty1 = y1 / DT;
    if (x0 > x1 || y0 > y1) tx0 = 1, tx1 = 0;
}

// count (SCATTER = false) or write (SCATTER = true) the (tile, point) records of views [v0, v0 + nv)
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_dbin(const DCam *__restrict__ cams, int v0, int nv, const float *xyz,
                                             const float *logh, uint32_t n, uint32_t *cnt_or_cursor, DRec *rec)
{
    const DCam &c0 = cams[v0];
    const uint32_t ntiles = (uint32_t)(c0.tiles_x * c0.tiles_y);
    const unsigned long long total = (unsigned long long)nv * n;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = gbd::lanemask_lt();
    for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
         e - threadIdx.x < total; e += (unsigned long long)gridDim.x * blockDim.x) {
        DProj o;
        bool vis = false;
        int vl = 0;
        uint32_t i = 0;
        if (e < total) {
            vl = (int)(e / n);
            i = (uint32_t)(e % n);
            vis = dproject(cams[v0 + vl], xyz, logh, i, o);
        }
        if (vis) {
            int tx0, tx1, ty0, ty1;
            dtiles(cams[v0 + vl], o, tx0, tx1, ty0, ty1);
            const int tilesx = cams[v0 + vl].tiles_x;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    const uint32_t t = (uint32_t)vl * ntiles + (uint32_t)(ty * tilesx + tx);
                    const uint32_t mask = __activemask();
                    const uint32_t peers = __match_any_sync(mask, t);
                    const int leader = __ffs(peers) - 1;
                    if (!SCATTER) {
                        if (lane == leader) atomicAdd(&cnt_or_cursor[t], (uint32_t)__popc(peers));
                    } else {
                        uint32_t b = 0;
                        if (lane == leader) b = atomicAdd(&cnt_or_cursor[t], (uint32_t)__popc(peers));
                        b = __shfl_sync(peers, b, leader);
                        rec[b + __popc(peers & lt)] = DRec{i, o.u, o.v, o.s};
                    }
                }
        }
    }
}

__global__ void k_ditems(uint32_t ntiles_all, const uint32_t *cnt, uint32_t *icnt)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles_all) icnt[t] = (cnt[t] + DITEM - 1) / DITEM;
}

__global__ void k_dfill(uint32_t ntiles_all, const uint32_t *cnt, const uint32_t *off, const uint32_t *ioff,
                        uint4 *items)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles_all) return;
    uint32_t k = ioff[t];
    for (uint32_t s = 0; s < cnt[t]; s += DITEM, ++k) items[k] = make_uint4(t, off[t] + s, off[t] + min(cnt[t], s + DITEM), 0u);
}

// Forward, pixel-parallel: one thread per pixel of a 16 x 16 tile (warp w owns rows 2w and 2w + 1),
// the item's records staged in shared memory; each warp first compacts, by ballot, the staged records
// whose 3-sigma disc reaches its two rows, then sums only those (no atomics inside the tile).
__global__ void __launch_bounds__(DRT) k_dforward(const DCam *__restrict__ cams, int v0, const DRec *__restrict__ rec,
                                                  const uint4 *__restrict__ items, const float *__restrict__ w,
                                                  float *images)
{
    __shared__ float4 sR[DRT];
    __shared__ float sW[DRT];
    __shared__ uint8_t sL[DRT / 32][DRT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = gbd::lanemask_lt();
    const uint4 it = items[blockIdx.x];
    const DCam &c = cams[v0];
    const uint32_t ntiles = (uint32_t)(c.tiles_x * c.tiles_y);
    const uint32_t vl = it.x / ntiles, t = it.x % ntiles;
    const int px = (int)(t % c.tiles_x) * DT + (threadIdx.x % DT), py = (int)(t / c.tiles_x) * DT + (threadIdx.x / DT);
    const float fx = px + 0.5f, fy = py + 0.5f;
    // pixel-centre rows of this warp
    const float wy0 = (float)((int)(t / c.tiles_x) * DT + 2 * warp) + 0.5f, wy1 = wy0 + 1.0f;
    float acc = 0.0f;
    for (uint32_t b = it.y; b < it.z; b += DRT) {
        __syncthreads();
        if (b + threadIdx.x < it.z) {
            const DRec r = rec[b + threadIdx.x];
            sR[threadIdx.x] = make_float4(r.u, r.v, r.s, 0.0f);
            sW[threadIdx.x] = w[r.idx];
        }
        __syncthreads();
        const int nb = (int)min((uint32_t)DRT, it.z - b);
        int n = 0;
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int j = j0 + lane;
            bool touch = false;
            if (j < nb) {
                // a row reaches the disc iff its distance to the centre is below 3 sigma (the same
                // strict test as the per-pixel one, on the row nearest the centre)
                const float4 q = sR[j];
                const float dyn = q.y < wy0 ? wy0 - q.y : (q.y > wy1 ? q.y - wy1 : 0.0f);
                touch = dyn * dyn < 9.0f * (q.z * q.z);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, touch);
            if (touch) sL[warp][n + __popc(m & lt)] = (uint8_t)j;
            n += __popc(m);
        }
        __syncwarp();
        for (int i = 0; i < n; ++i) {
            const float4 q = sR[sL[warp][i]];
            const float dx = fx - q.x, dy = fy - q.y, r2 = dx * dx + dy * dy, s2 = q.z * q.z;
            if (r2 < 9.0f * s2) acc += sW[sL[warp][i]] * (expf(-r2 / (2.0f * s2)) - E45) * (INV_2PI_C / s2);
        }
    }
    if (px < c.W && py < c.H && acc != 0.0f)
        atomicAdd(&images[((size_t)(v0 + vl) * c.H + py) * c.W + px], acc);
}

// The partial derivatives of one record over the pixels (x, y) = (x0 + i % bw, y0 + i / bw) of its box
// for i = first, first + step, ...: the per-pixel terms are recomputed from (u, v, sigma).
__device__ __forceinline__ void dgrad_pixels(const DRec &r, float wi, float (*sg)[DT + 1], int X0, int Y0, int x0,
                                             int y0, int bw, int area, int first, int step, float &tw, float &tu,
                                             float &tv, float &ts)
{
    const float s = r.s, s2 = s * s;
    const float inv2s2 = 1.0f / (2.0f * s2), norm = INV_2PI_C / s2, e45 = E45 * (INV_2PI_C / s2);
    for (int i = first; i < area; i += step) {
        const int y = y0 + i / bw, x = x0 + i % bw;
        const float g = sg[y][x];
        const float dx = (float)(X0 + x) + 0.5f - r.u;
        const float dy = (float)(Y0 + y) + 0.5f - r.v;
        const float r2 = dx * dx + dy * dy;
        if (g != 0.0f && r2 < 9.0f * s2) {
            const float e = expf(-r2 * inv2s2) * norm;
            const float k = e - e45;
            const float gwv = g * wi;
            tw += g * k;
            tu += gwv * e * dx / s2;
            tv += gwv * e * dy / s2;
            ts += gwv * (e * r2 / (s2 * s) - 2.0f * k / s);
        }
    }
}

// chains a record's (w, u, v, sigma) derivatives to its position, weight and log smoothing length
__device__ __forceinline__ void dgrad_commit(const DCam &c, const float *xyz, const float *logh, uint32_t idx,
                                             float tw, float tu, float tv, float ts, float *gxyz, float *gw,
                                             float *glogh)
{
    if (tw == 0.f && tu == 0.f && tv == 0.f && ts == 0.f) return;
    DProj o;
    dproject(c, xyz, logh, idx, o);
    const float iz = 1.0f / o.zc;
    const float dxc = tu * c.F * iz;
    const float dyc = -tv * c.F * iz;
    const float ds_dz = o.clamped ? 0.0f : -o.s * iz;
    const float dzc = tu * (-c.F * o.xc * iz * iz) + tv * (c.F * o.yc * iz * iz) + ts * ds_dz;
    atomicAdd(&gxyz[3 * idx], c.rx * dxc + c.ux * dyc + c.fx * dzc);
    atomicAdd(&gxyz[3 * idx + 1], c.ry * dxc + c.uy * dyc + c.fy * dzc);
    atomicAdd(&gxyz[3 * idx + 2], c.rz * dxc + c.uz * dyc + c.fz * dzc);
    atomicAdd(&gw[idx], tw);
    if (!o.clamped) atomicAdd(&glogh[idx], ts * o.s);
}

// Adjoint: the tile's dL/dI values are staged in shared memory.  Each lane takes one record; a
// record whose box inside the tile is small is walked by its own lane with the partial derivatives
// in registers, a large one is walked by the whole warp (lanes over its pixels) and reduced with
// shuffles, so no lane is held up by a large record while the others idle.  Every per-pixel term is
// recomputed from (u, v, sigma); nothing per pixel is stored.
constexpr int DBIG = 64; // box pixels from which a record is walked by the warp
__global__ void __launch_bounds__(DRT) k_dbackward(const DCam *__restrict__ cams, int v0, const DRec *__restrict__ rec,
                                                   const uint4 *__restrict__ items, const float *__restrict__ xyz,
                                                   const float *__restrict__ w, const float *__restrict__ logh,
                                                   const float *__restrict__ grad_img, float *gxyz, float *gw,
                                                   float *glogh)
{
    __shared__ float sg[DT][DT + 1];
    const int lane = threadIdx.x & 31;
    const uint4 it = items[blockIdx.x];
    const DCam &c0 = cams[v0];
    const uint32_t ntiles = (uint32_t)(c0.tiles_x * c0.tiles_y);
    const uint32_t vl = it.x / ntiles, t = it.x % ntiles;
    const DCam &c = cams[v0 + vl];
    const int X0 = (int)(t % c.tiles_x) * DT, Y0 = (int)(t / c.tiles_x) * DT;
    {
        const int px = X0 + (threadIdx.x % DT), py = Y0 + (threadIdx.x / DT);
        sg[threadIdx.x / DT][threadIdx.x % DT] =
            px < c.W && py < c.H ? grad_img[((size_t)(v0 + vl) * c.H + py) * c.W + px] : 0.0f;
    }
    __syncthreads();
    const int xw = min(DT, c.W - X0), yh = min(DT, c.H - Y0); // tile clipped to the image
    for (uint32_t b0 = it.y + (threadIdx.x & ~31u); b0 < it.z; b0 += DRT) {
        const uint32_t b = b0 + lane;
        DRec r = make_drec();
        int x0 = 0, y0 = 0, bw = 0, area = 0;
        float wi = 0.0f;
        if (b < it.z) {
            r = rec[b];
            const float R = 3.0f * r.s;
            x0 = max(0, (int)floorf(r.u - R - 0.5f) - X0);
            const int x1 = min(xw - 1, (int)ceilf(r.u + R - 0.5f) - X0);
            y0 = max(0, (int)floorf(r.v - R - 0.5f) - Y0);
            const int y1 = min(yh - 1, (int)ceilf(r.v + R - 0.5f) - Y0);
            bw = max(0, x1 - x0 + 1);
            area = bw * max(0, y1 - y0 + 1);
            wi = w[r.idx];
        }
        const bool big = area >= DBIG;
        // small records: one lane each
        if (!big && area > 0) {
            float tw = 0.f, tu = 0.f, tv = 0.f, ts = 0.f;
            dgrad_pixels(r, wi, sg, X0, Y0, x0, y0, bw, area, 0, 1, tw, tu, tv, ts);
            dgrad_commit(c, xyz, logh, r.idx, tw, tu, tv, ts, gxyz, gw, glogh);
        }
        // large records: the whole warp, one after another
        uint32_t m = __ballot_sync(0xffffffffu, big);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            DRec q;
            q.idx = __shfl_sync(0xffffffffu, r.idx, src);
            q.u = __shfl_sync(0xffffffffu, r.u, src);
            q.v = __shfl_sync(0xffffffffu, r.v, src);
            q.s = __shfl_sync(0xffffffffu, r.s, src);
            const float qw = __shfl_sync(0xffffffffu, wi, src);
            const int qx0 = __shfl_sync(0xffffffffu, x0, src), qy0 = __shfl_sync(0xffffffffu, y0, src);
            const int qbw = __shfl_sync(0xffffffffu, bw, src), qarea = __shfl_sync(0xffffffffu, area, src);
            float tw = 0.f, tu = 0.f, tv = 0.f, ts = 0.f;
            dgrad_pixels(q, qw, sg, X0, Y0, qx0, qy0, qbw, qarea, lane, 32, tw, tu, tv, ts);
            for (int d = 16; d > 0; d >>= 1) {
                tw += __shfl_xor_sync(0xffffffffu, tw, d);
                tu += __shfl_xor_sync(0xffffffffu, tu, d);
                tv += __shfl_xor_sync(0xffffffffu, tv, d);
                ts += __shfl_xor_sync(0xffffffffu, ts, d);
            }
            if (lane == 0) dgrad_commit(c, xyz, logh, q.idx, tw, tu, tv, ts, gxyz, gw, glogh);
        }
    }
}

DCam make_dcam(const gblod_camera &c, const gblod_render_params &rp)
{
    DCam d;
    d.ex = (float)c.eye[0]; d.ey = (float)c.eye[1]; d.ez = (float)c.eye[2];
    d.rx = (float)c.right[0]; d.ry = (float)c.right[1]; d.rz = (float)c.right[2];
    d.ux = (float)c.up[0]; d.uy = (float)c.up[1]; d.uz = (float)c.up[2];
    d.fx = (float)c.fwd[0]; d.fy = (float)c.fwd[1]; d.fz = (float)c.fwd[2];
    d.F = (float)c.f_px; d.CX = (float)c.cx; d.CY = (float)c.cy; d.ZN = (float)c.z_near;
    d.smin = (float)rp.sigma_min_px;
    d.smax = (float)rp.sigma_max_px;
    d.W = c.width;
    d.H = c.height;
    d.tiles_x = (c.width + DT - 1) / DT;
    d.tiles_y = (c.height + DT - 1) / DT;
    return d;
}

} // namespace

// Runs forward (grad_img == nullptr) or backward over chunks of views whose records fit a budget.
void diff_pass(gblod_renderer *r, const float *xyz, const float *w, const float *logh, uint64_t n,
               const gblod_camera *cams, int nv, const gblod_render_params &rp, float *images, const float *grad_img,
               float *gxyz, float *gw, float *glogh, cudaStream_t s)
{
    if (n >= 0xFFFFFFFFull) fail(GBLOD_ERR_INVALID_ARG, "too many points");
    const int W = cams[0].width, H = cams[0].height;
    for (int v = 0; v < nv; ++v)
        if (cams[v].width != W || cams[v].height != H) fail(GBLOD_ERR_INVALID_ARG, "all views need one resolution");
    const Allocator &A = r->A;
    std::vector<DCam> hc(nv);
    for (int v = 0; v < nv; ++v) hc[v] = make_dcam(cams[v], rp);
    r->d_cams.ensure(A, (size_t)nv * sizeof(DCam), s);
    DCam *dc = reinterpret_cast<DCam *>(r->d_cams.p);
    GB_CUDA(cudaMemcpyAsync(dc, hc.data(), (size_t)nv * sizeof(DCam), cudaMemcpyHostToDevice, s));
    const size_t npix = (size_t)W * H;
    if (images) GB_CUDA(cudaMemsetAsync(images, 0, (size_t)nv * npix * sizeof(float), s));
    if (grad_img) {
        GB_CUDA(cudaMemsetAsync(gxyz, 0, n * 3 * sizeof(float), s));
        GB_CUDA(cudaMemsetAsync(gw, 0, n * sizeof(float), s));
        GB_CUDA(cudaMemsetAsync(glogh, 0, n * sizeof(float), s));
    }
    if (n == 0) return;
    const uint32_t ntiles = (uint32_t)(hc[0].tiles_x * hc[0].tiles_y);
    const unsigned G = (unsigned)persistent_blocks(4);
    // views per chunk: about 2^26 (view, point) pairs, so records stay near a few GB
    const int vchunk = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)nv, (1ull << 26) / std::max<uint64_t>(n, 1)));
    for (int v0 = 0; v0 < nv; v0 += vchunk) {
        const int cnv = std::min(vchunk, nv - v0);
        const uint32_t nt = ntiles * (uint32_t)cnv;
        r->d_cnt.ensure(A, nt, s);
        r->d_off.ensure(A, nt + 1, s);
        r->d_cur.ensure(A, nt, s);
        r->d_icnt.ensure(A, nt, s);
        r->d_ioff.ensure(A, nt + 1, s);
        GB_CUDA(cudaMemsetAsync(r->d_cnt.p, 0, (size_t)nt * 4, s));
        launch(GBLOD_K_RENDER_OTHER, k_dbin<false>, dim3(G), dim3(256), 0, s, (const DCam *)dc, v0, cnv, xyz, logh,
               (uint32_t)n, r->d_cnt.p, (DRec *)nullptr);
        scan_exclusive_u32(A, r->scan, r->d_cnt.p, r->d_off.p, nt, r->d_off.p + nt, s);
        launch(GBLOD_K_RENDER_OTHER, k_ditems, dim3((nt + 255) / 256), dim3(256), 0, s, nt, (const uint32_t *)r->d_cnt.p,
               r->d_icnt.p);
        scan_exclusive_u32(A, r->scan, r->d_icnt.p, r->d_ioff.p, nt, r->d_ioff.p + nt, s);
        uint32_t tot[2];
        GB_CUDA(cudaMemcpyAsync(&tot[0], r->d_off.p + nt, 4, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(&tot[1], r->d_ioff.p + nt, 4, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        r->d_rec.ensure(A, (size_t)tot[0] * sizeof(DRec), s);
        r->d_items.ensure(A, tot[1], s);
        GB_CUDA(cudaMemcpyAsync(r->d_cur.p, r->d_off.p, (size_t)nt * 4, cudaMemcpyDeviceToDevice, s));
        DRec *rec = reinterpret_cast<DRec *>(r->d_rec.p);
        launch(GBLOD_K_RENDER_OTHER, k_dbin<true>, dim3(G), dim3(256), 0, s, (const DCam *)dc, v0, cnv, xyz, logh,
               (uint32_t)n, r->d_cur.p, rec);
        launch(GBLOD_K_RENDER_OTHER, k_dfill, dim3((nt + 255) / 256), dim3(256), 0, s, nt, (const uint32_t *)r->d_cnt.p,
               (const uint32_t *)r->d_off.p, (const uint32_t *)r->d_ioff.p, r->d_items.p);
        if (!grad_img)
            launch(GBLOD_K_SPLAT, k_dforward, dim3(tot[1]), dim3(DRT), 0, s, (const DCam *)dc, v0, (const DRec *)rec,
                   (const uint4 *)r->d_items.p, w, images);
        else
            launch(GBLOD_K_SPLAT, k_dbackward, dim3(tot[1]), dim3(DRT), 0, s, (const DCam *)dc, v0, (const DRec *)rec,
                   (const uint4 *)r->d_items.p, xyz, w, logh, grad_img, gxyz, gw, glogh);
    }
}

} // namespace gb
