// The C ABI declared in include/gblod.h: host-side argument checks, then the device work.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "render.cuh"

using namespace gb;

namespace {

template <class F> gblod_status guarded(F &&f)
{
    try {
        f();
        return GBLOD_OK;
    } catch (const Error &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return GBLOD_ERR_OOM;
    } catch (...) {
        set_error("unexpected exception");
        return GBLOD_ERR_CUDA;
    }
}

bool finite3(const double v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

void check_camera(const gblod_camera *c)
{
    if (!c) fail(GBLOD_ERR_INVALID_ARG, "camera is NULL");
    if (!finite3(c->eye) || !finite3(c->right) || !finite3(c->up) || !finite3(c->fwd) || !std::isfinite(c->f_px) ||
        !std::isfinite(c->cx) || !std::isfinite(c->cy) || !std::isfinite(c->z_near))
        fail(GBLOD_ERR_INVALID_ARG, "camera fields must be finite");
    if (!(c->f_px > 0.0) || !(c->z_near >= 0.0)) fail(GBLOD_ERR_INVALID_ARG, "camera needs f_px > 0, z_near >= 0");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        fail(GBLOD_ERR_INVALID_ARG, "camera width/height must be in 1..16384");
}

gblod_render_params check_params(const gblod_render_params *p)
{
    if (!p) fail(GBLOD_ERR_INVALID_ARG, "render params are NULL");
    gblod_render_params q = *p;
    if (!(q.sigma_min_px > 0.0) || !(q.sigma_max_px >= q.sigma_min_px) || !std::isfinite(q.sigma_max_px))
        fail(GBLOD_ERR_INVALID_ARG, "need 0 < sigma_min_px <= sigma_max_px < inf");
    if ((float)q.sigma_max_px > 4096.0f) fail(GBLOD_ERR_INVALID_ARG, "sigma_max_px must be <= 4096");
    if (q.kernel != GBLOD_KERNEL_GAUSSIAN && q.kernel != GBLOD_KERNEL_CUBIC)
        fail(GBLOD_ERR_INVALID_ARG, "unknown kernel");
    if (std::isnan(q.lambda_px)) fail(GBLOD_ERR_INVALID_ARG, "lambda_px is NaN");
    if (q.tile_w == 0) q.tile_w = 64;
    if (q.tile_h == 0) q.tile_h = 16;
    if (q.tile_w < 1 || q.tile_h < 1 || q.tile_w > 64 || q.tile_h > 64 ||
        ((q.tile_w + 7) / 8) * ((q.tile_h + 15) / 16) > 8)
        fail(GBLOD_ERR_INVALID_ARG, "tile must be 1..64 x 1..64 with ceil(w/8) ceil(h/16) <= 8 (8 strips of 8 x 16 pixels)");
    if (!q.tone_auto && !(q.tone_hi > q.tone_lo && q.tone_lo > 0.0 && std::isfinite(q.tone_hi)))
        fail(GBLOD_ERR_INVALID_ARG, "fixed tone range needs 0 < tone_lo < tone_hi < inf");
    if (q.point_format != GBLOD_POINTS_FLOAT && q.point_format != GBLOD_POINTS_BLOCK16)
        fail(GBLOD_ERR_INVALID_ARG, "unknown point_format");
    if (q.flags & ~GBLOD_RENDER_COUNT_UPDATES) fail(GBLOD_ERR_INVALID_ARG, "unknown render flags");
    return q;
}

struct TuneEntry {
    int w, h;
    double ms;
};
std::map<std::string, TuneEntry> &tune_cache()
{
    static std::map<std::string, TuneEntry> m;
    return m;
}
std::mutex &tune_mutex()
{
    static std::mutex m;
    return m;
}

} // namespace

extern "C" {

gblod_status gblod_build_lod(const float *d_xyz, const float *d_mass, const float *d_h, const uint32_t *d_ids,
                             uint64_t n, const gblod_build_params *params, const gblod_allocator *alloc,
                             void *stream, gblod_octree **out)
{
    return guarded([&] {
        if (!out || !params) fail(GBLOD_ERR_INVALID_ARG, "out and params must not be NULL");
        if (n > 0 && (!d_xyz || !d_mass || !d_h)) fail(GBLOD_ERR_INVALID_ARG, "particle arrays must not be NULL");
        if (n >= 0xFFFFFFFFull) fail(GBLOD_ERR_INVALID_ARG, "n must be below 2^32 - 1");
        if (params->n_max < 1) fail(GBLOD_ERR_INVALID_ARG, "n_max must be >= 1");
        if (!finite3(params->root_lo) || !(params->root_side > 0.0) || !std::isfinite(params->root_side))
            fail(GBLOD_ERR_INVALID_ARG, "root cube must be finite with side > 0");
        Allocator A(alloc);
        *out = build_octree(d_xyz, d_mass, d_h, d_ids, n, *params, A, (cudaStream_t)stream);
    });
}

void gblod_octree_free(gblod_octree *octree)
{
    if (!octree) return;
    (void)cudaStreamSynchronize(octree->stream);
    free_octree(octree);
    (void)cudaGetLastError();
}

gblod_status gblod_octree_get_info(const gblod_octree *o, gblod_octree_info *out)
{
    if (!o || !out) {
        set_error("octree and out must not be NULL");
        return GBLOD_ERR_INVALID_ARG;
    }
    gblod_octree_info i;
    std::memset(&i, 0, sizeof(i));
    i.n_particles = o->n;
    i.n_nodes = o->n_nodes;
    i.n_points = o->n_points;
    i.device_bytes = o->bytes;
    i.depth_max = o->depth_max;
    i.equal_mass = o->equal_mass;
    i.n_max = o->n_max;
    i.formats = (o->has_float ? 1u : 0u) | (o->has_block16 ? 2u : 0u);
    *out = i;
    return GBLOD_OK;
}

gblod_status gblod_octree_export(const gblod_octree *o, gblod_node *h_nodes, float *h_pts4, float *h_hs,
                                 uint32_t *h_pt_src, uint64_t *h_skey, uint32_t *h_sidx)
{
    return guarded([&] {
        if (!o) fail(GBLOD_ERR_INVALID_ARG, "octree is NULL");
        cudaStream_t s = o->stream;
        if (h_nodes && o->n_nodes)
            GB_CUDA(cudaMemcpyAsync(h_nodes, o->nodes, o->n_nodes * sizeof(gblod_node), cudaMemcpyDeviceToHost, s));
        if ((h_pts4 || h_hs) && !o->has_float)
            fail(GBLOD_ERR_INVALID_ARG, "octree holds no fp32 points (dropped after quantisation)");
        if (h_pts4 && o->n_points)
            GB_CUDA(cudaMemcpyAsync(h_pts4, o->pts4, o->n_points * sizeof(float4), cudaMemcpyDeviceToHost, s));
        if (h_hs && o->n_points)
            GB_CUDA(cudaMemcpyAsync(h_hs, o->hs, o->n_points * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (h_pt_src && o->n_points)
            GB_CUDA(cudaMemcpyAsync(h_pt_src, o->pt_src, o->n_points * 4, cudaMemcpyDeviceToHost, s));
        if (h_skey && o->n) GB_CUDA(cudaMemcpyAsync(h_skey, o->skey, o->n * 8, cudaMemcpyDeviceToHost, s));
        if (h_sidx && o->n) GB_CUDA(cudaMemcpyAsync(h_sidx, o->sidx, o->n * 4, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
    });
}

gblod_status gblod_octree_quantize(gblod_octree *o, uint32_t flags, void *stream)
{
    return guarded([&] {
        if (!o) fail(GBLOD_ERR_INVALID_ARG, "octree is NULL");
        if (flags & ~GBLOD_QUANTIZE_DROP_FLOAT) fail(GBLOD_ERR_INVALID_ARG, "unknown quantize flags");
        block_quantize(o, flags, (cudaStream_t)stream);
    });
}

gblod_status gblod_octree_export_block16(const gblod_octree *o, uint16_t *h_codes, float *h_qa, gblod_node *h_qnodes)
{
    return guarded([&] {
        if (!o) fail(GBLOD_ERR_INVALID_ARG, "octree is NULL");
        if (!o->has_block16) fail(GBLOD_ERR_INVALID_ARG, "octree holds no 16-bit block codes");
        cudaStream_t s = o->stream;
        const size_t np = o->n_points, nn = o->n_nodes;
        if (h_codes && np) {
            std::vector<ushort4> q4(np);
            std::vector<uint16_t> qw(np);
            GB_CUDA(cudaMemcpyAsync(q4.data(), o->q4, np * sizeof(ushort4), cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaMemcpyAsync(qw.data(), o->qw, np * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
            for (size_t j = 0; j < np; ++j) {
                h_codes[5 * j] = q4[j].x;
                h_codes[5 * j + 1] = q4[j].y;
                h_codes[5 * j + 2] = q4[j].z;
                h_codes[5 * j + 3] = qw[j];
                h_codes[5 * j + 4] = q4[j].w;
            }
        }
        if (h_qa && nn) GB_CUDA(cudaMemcpyAsync(h_qa, o->qa, nn * 2 * sizeof(float4), cudaMemcpyDeviceToHost, s));
        if (h_qnodes && nn)
            GB_CUDA(cudaMemcpyAsync(h_qnodes, o->qnodes, nn * sizeof(gblod_node), cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
    });
}

gblod_status gblod_renderer_create(const gblod_allocator *alloc, gblod_renderer **out)
{
    return guarded([&] {
        if (!out) fail(GBLOD_ERR_INVALID_ARG, "out is NULL");
        gblod_renderer *r = new gblod_renderer();
        r->A = Allocator(alloc, false); // grow-only buffers: the default stream-ordered pool
        try {
            renderer_init(r, nullptr);
        } catch (...) {
            delete r;
            throw;
        }
        *out = r;
    });
}

void gblod_renderer_destroy(gblod_renderer *r)
{
    if (!r) return;
    try {
        renderer_release(r);
    } catch (...) {
    }
    delete r;
    (void)cudaGetLastError();
}

gblod_status gblod_render(gblod_renderer *r, const gblod_octree *octree, const gblod_camera *camera,
                          const gblod_render_params *params, uint8_t *d_image, uint64_t *d_accum, void *stream)
{
    return guarded([&] {
        if (!r || !octree) fail(GBLOD_ERR_INVALID_ARG, "renderer and octree must not be NULL");
        check_camera(camera);
        const gblod_render_params p = check_params(params);
        render_lod(r, octree, *camera, p, d_image, d_accum, (cudaStream_t)stream);
    });
}

gblod_status gblod_render_part(gblod_renderer *r, const gblod_octree *octree, const gblod_camera *camera,
                               const gblod_render_params *params, int32_t part, int32_t n_parts, uint64_t *d_accum,
                               void *stream)
{
    return guarded([&] {
        if (!r || !octree) fail(GBLOD_ERR_INVALID_ARG, "renderer and octree must not be NULL");
        if (!d_accum) fail(GBLOD_ERR_INVALID_ARG, "gblod_render_part needs d_accum (the partial image)");
        if (n_parts < 1 || part < 0 || part >= n_parts) fail(GBLOD_ERR_INVALID_ARG, "need 0 <= part < n_parts");
        check_camera(camera);
        const gblod_render_params p = check_params(params);
        render_lod(r, octree, *camera, p, nullptr, d_accum, (cudaStream_t)stream, (uint32_t)part, (uint32_t)n_parts);
    });
}

gblod_status gblod_tonemap(gblod_renderer *r, const uint64_t *d_accum, int32_t width, int32_t height,
                           const gblod_render_params *params, uint8_t *d_image, void *stream)
{
    return guarded([&] {
        if (!r || !d_accum || !d_image) fail(GBLOD_ERR_INVALID_ARG, "renderer, d_accum and d_image must not be NULL");
        if (width < 1 || height < 1 || width > 16384 || height > 16384)
            fail(GBLOD_ERR_INVALID_ARG, "width/height must be in 1..16384");
        const gblod_render_params p = check_params(params);
        tonemap_image(r, d_accum, width, height, p, d_image, (cudaStream_t)stream);
    });
}

gblod_status gblod_render_bruteforce(gblod_renderer *r, const float *d_xyz, const float *d_mass, const float *d_h,
                                     uint64_t n, const gblod_camera *camera, const gblod_render_params *params,
                                     uint8_t *d_image, uint64_t *d_accum, void *stream)
{
    return guarded([&] {
        if (!r) fail(GBLOD_ERR_INVALID_ARG, "renderer is NULL");
        if (n > 0 && (!d_xyz || !d_mass || !d_h)) fail(GBLOD_ERR_INVALID_ARG, "particle arrays must not be NULL");
        check_camera(camera);
        const gblod_render_params p = check_params(params);
        render_brute(r, d_xyz, d_mass, d_h, n, *camera, p, d_image, d_accum, (cudaStream_t)stream);
    });
}

gblod_status gblod_render_bruteforce_noalloc(const float *d_xyz, const float *d_mass, const float *d_h, uint64_t n,
                                             const gblod_camera *camera, const gblod_render_params *params,
                                             uint8_t *d_image, uint64_t *d_accum, void *stream)
{
    gblod_status out = GBLOD_OK;
    gblod_status st = guarded([&] {
        if (n > 0 && (!d_xyz || !d_mass || !d_h)) fail(GBLOD_ERR_INVALID_ARG, "particle arrays must not be NULL");
        check_camera(camera);
        const gblod_render_params p = check_params(params);
        out = render_brute_noalloc(d_xyz, d_mass, d_h, n, *camera, p, d_image, d_accum, (cudaStream_t)stream);
        if (out == GBLOD_ERR_RANGE) set_error("a drawn amplitude or the amplitude sum is out of fixed-point range");
    });
    return st != GBLOD_OK ? st : out;
}

gblod_status gblod_renderer_reserve_batch(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                          const gblod_render_params *params, uint64_t record_capacity, void *stream)
{
    return guarded([&] {
        if (!r || !views || n_views < 1) fail(GBLOD_ERR_INVALID_ARG, "renderer and at least one view needed");
        const gblod_render_params p = check_params(params);
        for (int i = 0; i < n_views; ++i) check_camera(&views[i].camera);
        reserve_batch(r, views, n_views, p, record_capacity, (cudaStream_t)stream);
    });
}

gblod_status gblod_render_batch(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                const gblod_render_params *params, void *stream)
{
    return guarded([&] {
        if (!r || !views || n_views < 1) fail(GBLOD_ERR_INVALID_ARG, "renderer and at least one view needed");
        const gblod_render_params p = check_params(params);
        for (int i = 0; i < n_views; ++i) check_camera(&views[i].camera);
        render_batch(r, views, n_views, p, (cudaStream_t)stream);
    });
}

gblod_status gblod_autotune_tiles(gblod_renderer *r, const gblod_view *views, int32_t n_views,
                                  gblod_render_params *params_inout, uint64_t record_capacity, void *stream,
                                  double *best_ms)
{
    return guarded([&] {
        if (!r || !views || n_views < 1 || !params_inout) fail(GBLOD_ERR_INVALID_ARG, "bad autotune arguments");
        gblod_render_params p = check_params(params_inout);
        for (int i = 0; i < n_views; ++i) check_camera(&views[i].camera);
        static const int cand[][2] = {{16, 16}, {32, 16}, {16, 32}, {32, 32}, {64, 16}};
        cudaStream_t s = (cudaStream_t)stream;
        // cache key: device, the views' resolutions, the batch's splat-count class and the parameters
        // that change the work; one render with the caller's tile measures the splat count
        reserve_batch(r, views, n_views, p, record_capacity, s);
        render_batch(r, views, n_views, p, s);
        unsigned long long splats = 0;
        GB_CUDA(cudaMemcpyAsync(&splats, &r->stats->splats, 8, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        {
            unsigned bits = 0; // this render only measures; an overflow here is not the caller's
            GB_CUDA(cudaMemcpy(&bits, r->status, 4, cudaMemcpyDeviceToHost));
            const unsigned keep = bits & ~4u;
            if (keep != bits) GB_CUDA(cudaMemcpy(r->status, &keep, 4, cudaMemcpyHostToDevice));
        }
        int dev = 0;
        GB_CUDA(cudaGetDevice(&dev));
        cudaDeviceProp prop;
        GB_CUDA(cudaGetDeviceProperties(&prop, dev));
        std::vector<long long> res;
        for (int i = 0; i < n_views; ++i) res.push_back((long long)views[i].camera.width << 20 | views[i].camera.height);
        std::sort(res.begin(), res.end());
        std::string key = std::to_string(dev) + ":" + prop.name + ":" + std::to_string(p.kernel) + ":" +
                          std::to_string(p.point_format) + ":" + std::to_string(record_capacity) + ":" +
                          std::to_string(63 - __builtin_clzll(splats | 1ull));
        for (long long v : res) key += ":" + std::to_string(v);
        {
            std::lock_guard<std::mutex> g(tune_mutex());
            auto it = tune_cache().find(key);
            if (it != tune_cache().end()) {
                params_inout->tile_w = p.tile_w = it->second.w;
                params_inout->tile_h = p.tile_h = it->second.h;
                reserve_batch(r, views, n_views, p, record_capacity, s);
                if (best_ms) *best_ms = it->second.ms;
                return;
            }
        }
        cudaEvent_t e0, e1;
        GB_CUDA(cudaEventCreate(&e0));
        GB_CUDA(cudaEventCreate(&e1));
        double best = -1.0;
        int bw = p.tile_w, bh = p.tile_h;
        for (const auto &c : cand) {
            p.tile_w = c[0];
            p.tile_h = c[1];
            reserve_batch(r, views, n_views, p, record_capacity, s);
            render_batch(r, views, n_views, p, s); // warm-up
            GB_CUDA(cudaEventRecord(e0, s));
            for (int k = 0; k < 3; ++k) render_batch(r, views, n_views, p, s);
            GB_CUDA(cudaEventRecord(e1, s));
            GB_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            GB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            // a candidate whose records overflow the capacity skipped work: not eligible
            unsigned bits = 0;
            GB_CUDA(cudaMemcpy(&bits, r->status, 4, cudaMemcpyDeviceToHost));
            if (bits & 4u) {
                const unsigned keep = bits & ~4u;
                GB_CUDA(cudaMemcpy(r->status, &keep, 4, cudaMemcpyHostToDevice));
                continue;
            }
            if (best < 0.0 || ms / 3.0 < best) {
                best = ms / 3.0;
                bw = c[0];
                bh = c[1];
            }
        }
        (void)cudaEventDestroy(e0);
        (void)cudaEventDestroy(e1);
        if (best < 0.0) fail(GBLOD_ERR_CAPACITY, "every tile candidate overflowed the record capacity");
        params_inout->tile_w = bw;
        params_inout->tile_h = bh;
        p.tile_w = bw;
        p.tile_h = bh;
        reserve_batch(r, views, n_views, p, record_capacity, s);
        if (best_ms) *best_ms = best;
        std::lock_guard<std::mutex> g(tune_mutex());
        tune_cache()[key] = TuneEntry{bw, bh, best};
    });
}

void gblod_autotune_cache_clear(void)
{
    std::lock_guard<std::mutex> g(tune_mutex());
    tune_cache().clear();
}

gblod_status gblod_diff_render(gblod_renderer *r, const float *d_xyz, const float *d_w, const float *d_logh,
                               uint64_t n, const gblod_camera *cams, int32_t n_views,
                               const gblod_render_params *params, float *d_images, void *stream)
{
    return guarded([&] {
        if (!r || !cams || n_views < 1 || !d_images) fail(GBLOD_ERR_INVALID_ARG, "bad arguments");
        if (n > 0 && (!d_xyz || !d_w || !d_logh)) fail(GBLOD_ERR_INVALID_ARG, "point arrays must not be NULL");
        const gblod_render_params p = check_params(params);
        for (int i = 0; i < n_views; ++i) check_camera(&cams[i]);
        diff_pass(r, d_xyz, d_w, d_logh, n, cams, n_views, p, d_images, nullptr, nullptr, nullptr, nullptr,
                  (cudaStream_t)stream);
    });
}

gblod_status gblod_diff_backward(gblod_renderer *r, const float *d_xyz, const float *d_w, const float *d_logh,
                                 uint64_t n, const gblod_camera *cams, int32_t n_views,
                                 const gblod_render_params *params, const float *d_grad_images, float *d_grad_xyz,
                                 float *d_grad_w, float *d_grad_logh, void *stream)
{
    return guarded([&] {
        if (!r || !cams || n_views < 1 || !d_grad_images) fail(GBLOD_ERR_INVALID_ARG, "bad arguments");
        if (n > 0 && (!d_xyz || !d_w || !d_logh || !d_grad_xyz || !d_grad_w || !d_grad_logh))
            fail(GBLOD_ERR_INVALID_ARG, "point and gradient arrays must not be NULL");
        const gblod_render_params p = check_params(params);
        for (int i = 0; i < n_views; ++i) check_camera(&cams[i]);
        diff_pass(r, d_xyz, d_w, d_logh, n, cams, n_views, p, nullptr, d_grad_images, d_grad_xyz, d_grad_w,
                  d_grad_logh, (cudaStream_t)stream);
    });
}

gblod_status gblod_renderer_status(gblod_renderer *r, void *stream, int reset)
{
    gblod_status out = GBLOD_OK;
    gblod_status st = guarded([&] {
        if (!r) fail(GBLOD_ERR_INVALID_ARG, "renderer is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        unsigned *h = static_cast<unsigned *>(r->hs.get(16));
        unsigned long long *amp = reinterpret_cast<unsigned long long *>(h + 2);
        GB_CUDA(cudaMemcpyAsync(h, r->status, 4, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaMemcpyAsync(amp, &r->stats->amp_hi, 8, cudaMemcpyDeviceToHost, s));
        GB_CUDA(cudaStreamSynchronize(s));
        unsigned bits = h[0];
        if (*amp) bits |= 1u;
        if (reset) GB_CUDA(cudaMemsetAsync(r->status, 0, 4, s));
        if (bits & 2u)
            out = GBLOD_ERR_DEVICE_TIMEOUT;
        else if (bits & 4u)
            out = GBLOD_ERR_CAPACITY;
        else if (bits & 1u)
            out = GBLOD_ERR_RANGE;
        if (reset) GB_CUDA(cudaStreamSynchronize(s));
    });
    return st != GBLOD_OK ? st : out;
}

gblod_status gblod_renderer_stats(gblod_renderer *r, void *stream, gblod_frame_stats *out)
{
    return guarded([&] {
        if (!r || !out) fail(GBLOD_ERR_INVALID_ARG, "renderer and out must not be NULL");
        FrameStatsDev *h = static_cast<FrameStatsDev *>(r->hs.get(sizeof(FrameStatsDev)));
        GB_CUDA(cudaMemcpyAsync(h, r->stats, sizeof(FrameStatsDev), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        GB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        out->nodes_selected = h->nodes_selected;
        out->points = h->points;
        out->splats = h->splats;
        out->pairs = h->pairs;
        out->tiles = h->tiles;
        out->amplitude_lo = h->amp_lo;
        out->amplitude_hi = h->amp_hi;
        out->pixel_updates = h->pixel_updates;
        out->pixel_updates_total = h->pixel_updates_total;
    });
}

gblod_status gblod_renderer_last_selection(gblod_renderer *r, void *stream, uint32_t *h_nodes, uint64_t cap,
                                           uint64_t *count)
{
    return guarded([&] {
        if (!r || !count) fail(GBLOD_ERR_INVALID_ARG, "renderer and count must not be NULL");
        if (!r->last_was_lod || !r->sel.p) {
            *count = 0;
            return;
        }
        FrameStatsDev *h = static_cast<FrameStatsDev *>(r->hs.get(sizeof(FrameStatsDev)));
        GB_CUDA(cudaMemcpyAsync(h, r->stats, sizeof(FrameStatsDev), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
        GB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        const uint64_t n = h->nodes_selected;
        *count = n;
        const uint64_t m = n < cap ? n : cap;
        if (h_nodes && m) {
            GB_CUDA(cudaMemcpyAsync(h_nodes, r->sel.p, m * 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
            GB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        }
    });
}

gblod_status gblod_morton_keys(const float *d_xyz, uint64_t n, const double root_lo[3], double root_side,
                               uint64_t *d_keys, void *stream)
{
    return guarded([&] {
        if (n > 0 && (!d_xyz || !d_keys)) fail(GBLOD_ERR_INVALID_ARG, "arrays must not be NULL");
        if (!root_lo || !finite3(root_lo) || !(root_side > 0.0) || !std::isfinite(root_side))
            fail(GBLOD_ERR_INVALID_ARG, "root cube must be finite with side > 0");
        if (n) morton_keys(d_xyz, n, root_lo, root_side, d_keys, (cudaStream_t)stream);
    });
}

gblod_status gblod_project(const float *d_pts4, const float *d_h, uint64_t n, const gblod_camera *camera,
                           const gblod_render_params *params, int64_t *d_out, void *stream)
{
    return guarded([&] {
        if (n > 0 && (!d_pts4 || !d_h || !d_out)) fail(GBLOD_ERR_INVALID_ARG, "arrays must not be NULL");
        check_camera(camera);
        const gblod_render_params p = check_params(params);
        if (n) project_points(reinterpret_cast<const float4 *>(d_pts4), d_h, n, *camera, p, d_out, (cudaStream_t)stream);
    });
}

} // extern "C"
