// Render workspace and the frame entry points shared by the C ABI.
#pragma once

#include "octree.cuh"

namespace gb {
struct FrameStatsDev {
    unsigned long long nodes_selected, points, splats, pairs, tiles, amp_lo, amp_hi, items;
    unsigned long long pixel_updates;       // (splat, pixel) contributions of the last frame
    unsigned long long pixel_updates_total; // since the renderer was created (never reset)
};
} // namespace gb

struct gblod_renderer {
    gb::Allocator A;
    gb::HostStage hs;
    gb::ScanTmp scan;
    unsigned *status = nullptr;             // sticky device status bits
    gb::FrameStatsDev *stats = nullptr;     // device counters of the last frame
    bool count_updates = false;             // this frame counts its pixel updates
    // R1
    gb::DBuf<uint32_t> frontA, frontB, sel, lvl_cnt;
    gb::DBuf<uint64_t> sel_pfx;
    gb::DBuf<int64_t> sel_base;
    // R2 / R3
    gb::DBuf<uint32_t> tile_cnt, tile_off, tile_cur, item_cnt, item_off;
    gb::DBuf<uint32_t> cta_hist, cta_off; // partitioned binning: (tile, CTA) counts and their offsets
    gb::DBuf<uint32_t> tile_cnt_s, tile_off_s, item_cnt_s, item_off_s; // its small-box record stream
    gb::DBuf<uint4> records, items;
    gb::DBuf<unsigned long long> accum, maxv;
    gb::DBuf<gb::FrameStatsDev> pass_stats; // counters of one range when a frame is split
    // batched views
    gb::DBuf<unsigned char> b_views; // per-view device constants (projection, frustum, pointers)
    gb::DBuf<unsigned long long> b_frontA, b_frontB, b_sel, b_counts, b_pfx;
    gb::DBuf<long long> b_base;
    uint64_t b_rec_cap = 0;
    // differentiable float splat
    gb::DBuf<unsigned char> d_cams, d_rec;
    gb::DBuf<uint32_t> d_cnt, d_off, d_cur, d_icnt, d_ioff;
    gb::DBuf<uint4> d_items;
    cudaStream_t last_stream = nullptr;
    bool last_was_lod = false;
};

namespace gb {
void renderer_init(gblod_renderer *r, cudaStream_t s);
void renderer_release(gblod_renderer *r);
void render_lod(gblod_renderer *r, const gblod_octree *o, const gblod_camera &cam, const gblod_render_params &rp,
                uint8_t *image, uint64_t *accum, cudaStream_t s, uint32_t part = 0, uint32_t n_parts = 1);
void tonemap_image(gblod_renderer *r, const uint64_t *accum, int W, int H, const gblod_render_params &rp,
                   uint8_t *image, cudaStream_t s);
void render_brute(gblod_renderer *r, const float *xyz, const float *mass, const float *h, uint64_t n,
                  const gblod_camera &cam, const gblod_render_params &rp, uint8_t *image, uint64_t *accum,
                  cudaStream_t s);
gblod_status render_brute_noalloc(const float *xyz, const float *mass, const float *h, uint64_t n,
                                  const gblod_camera &cam, const gblod_render_params &rp, uint8_t *image,
                                  uint64_t *accum, cudaStream_t s);
void reserve_batch(gblod_renderer *r, const gblod_view *views, int n, const gblod_render_params &rp,
                   uint64_t record_capacity, cudaStream_t s);
void render_batch(gblod_renderer *r, const gblod_view *views, int n, const gblod_render_params &rp, cudaStream_t s);
void diff_pass(gblod_renderer *r, const float *xyz, const float *w, const float *logh, uint64_t n,
               const gblod_camera *cams, int nv, const gblod_render_params &rp, float *images, const float *grad_img,
               float *gxyz, float *gw, float *glogh, cudaStream_t s);
void project_points(const float4 *pts4, const float *h, uint64_t n, const gblod_camera &cam,
                    const gblod_render_params &rp, int64_t *out, cudaStream_t s);
void morton_keys(const float *xyz, uint64_t n, const double lo[3], double side, uint64_t *keys, cudaStream_t s);
} // namespace gb
