// A4 + A5: density-weighted random subselection of every over-full node (octree paragraph:
// "simplified using a density-weighted random subselection ... until the same data is
// represented by only n points"), and the representatives' blocks.
//
// Every particle i of node c gets the key k_i = u_i (all masses equal) or the bits of
// E(u_i)/m_i (exponential race), u_i = Philox(seed; id_i, code_c); the node keeps the n_max
// smallest (k_i, id_i).  Per node this is a segmented radix select, all nodes at once:
//   hist     4096-element chunks histogram the top log2(B) key bits (B ~ count/1024 bins, at
//            most 4096: a shared-memory histogram per chunk)
//   find     per node, the bin b that holds rank n_max
//   mark     keys below bin b set their bit in a per-node bitmap (warp ballots, no atomics);
//            keys in bin b become candidates (k, id, position)
//   resolve  per node, 8-bit radix rounds over the candidates' remaining (k, id) bits decide
//            the last `need` members
//   count/write  a per-chunk popcount, a scan, and a stable compaction of the bitmap write
//            the representatives in ascending (Morton key, id) order.
// Keys are recomputed from the ids (counter-based generator) instead of being stored.
#include <algorithm>

#include "lodmath.cuh"
#include "octree.cuh"

namespace gb {
namespace {

constexpr int ST = 256;          // threads per selection block
constexpr uint32_t CH = 4096;    // elements per chunk (multiple of 32 * 8 warps)
constexpr int ROUNDS = CH / ST;  // 16 words of 32 per warp

struct Cand {
    uint64_t key;
    uint32_t id;
    uint32_t rel;
};

struct RepInfo {
    const uint32_t *nodes;     // node index per rep slot
    const uint32_t *chunk_off; // first chunk of each rep slot (n_rep + 1 entries)
    const uint32_t *hoff;      // first histogram bin of each rep slot
    const uint8_t *logb;       // log2 bins
    const uint64_t *woff;      // first bitmap word of each rep slot
};

__global__ void k_sel_setup(uint32_t n_rep, const uint32_t *nodes, const uint32_t *ncount, uint32_t *nchunks,
                            uint32_t *nbins, uint8_t *logb, uint64_t *nwords)
{
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rep) return;
    const uint32_t c = ncount[nodes[r]];
    nchunks[r] = (c + CH - 1) / CH;
    uint32_t want = (c + 1023) / 1024, lb = 0;
    while (lb < 12 && (1u << lb) < want) ++lb; // at most 4096 bins: the chunk histogram stays in shared memory
    logb[r] = (uint8_t)lb;
    nbins[r] = 1u << lb;
    nwords[r] = (c + 31) / 32;
}

__device__ __forceinline__ uint32_t find_slot(const uint32_t *chunk_off, uint32_t n_rep, uint32_t c)
{
    // largest r with chunk_off[r] <= c
    uint32_t lo = 0, hi = n_rep;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (chunk_off[mid] <= c)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t sel_key(const SelectIn &in, uint32_t j, uint64_t code, uint64_t seed,
                                            int equal_mass, uint32_t &id)
{
    id = in.sid[j];
    const uint64_t u = gbd::node_draw(seed, code, id);
    if (equal_mass) return u;
    const double k = __ddiv_rn(gbd::neg_log_unit(u), (double)in.s4[j].w);
    return (uint64_t)__double_as_longlong(k);
}

struct ChunkCtx {
    uint32_t r, node, first, count, start;
    uint64_t code;
    int logb;
};

__device__ __forceinline__ void load_chunk(ChunkCtx &C, const SelectIn &in, const RepInfo &R, uint32_t n_rep)
{
    __shared__ ChunkCtx sc;
    if (threadIdx.x == 0) {
        const uint32_t c = blockIdx.x;
        const uint32_t r = find_slot(R.chunk_off, n_rep, c);
        const uint32_t node = R.nodes[r];
        sc.r = r;
        sc.node = node;
        sc.first = in.nfirst[node];
        sc.count = in.ncount[node];
        sc.start = (c - R.chunk_off[r]) * CH;
        sc.code = in.ncode[node];
        sc.logb = R.logb[r];
    }
    __syncthreads();
    C = sc;
}

__global__ void __launch_bounds__(ST) k_sel_hist(SelectIn in, RepInfo R, uint32_t n_rep, uint64_t seed,
                                                 int equal_mass, uint32_t *hist)
{
    __shared__ uint32_t sh[4096];
    ChunkCtx C;
    load_chunk(C, in, R, n_rep);
    const int nb = 1 << C.logb; // <= 4096
    for (int i = threadIdx.x; i < nb; i += ST) sh[i] = 0u;
    __syncthreads();
    uint32_t *gh = hist + R.hoff[C.r];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < ROUNDS; ++k) {
        const uint32_t rel = C.start + (uint32_t)warp * (ROUNDS * 32) + (uint32_t)k * 32 + lane;
        if (rel < C.count) {
            uint32_t id;
            const uint64_t key = sel_key(in, C.first + rel, C.code, seed, equal_mass, id);
            const uint32_t d = C.logb ? (uint32_t)(key >> (64 - C.logb)) : 0u;
            atomicAdd(&sh[d], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += ST)
        if (sh[i]) atomicAdd(&gh[i], sh[i]);
}

// block exclusive scan of one u32 per thread; every thread gets the total
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t &tot)
{
    __shared__ uint32_t wsum[ST / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < ST / 32; ++w) {
        const uint32_t x = wsum[w];
        before += w < warp ? x : 0u;
        all += x;
    }
    __syncthreads();
    tot = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(ST) k_sel_find(RepInfo R, uint32_t n_max, const uint32_t *hist, uint32_t *tb,
                                                 uint32_t *need, uint64_t *ccount)
{
    const uint32_t r = blockIdx.x;
    const uint32_t nb = 1u << R.logb[r];
    const uint32_t *h = hist + R.hoff[r];
    uint32_t run = 0;
    for (uint32_t base = 0; base < nb; base += ST) {
        const uint32_t hv = base + threadIdx.x < nb ? h[base + threadIdx.x] : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_u32(hv, tot);
        const uint32_t cum = run + ex;
        if (cum < n_max && n_max <= cum + hv) {
            tb[r] = base + threadIdx.x;
            need[r] = n_max - cum;
            ccount[r] = hv;
        }
        run += tot;
    }
}

__global__ void __launch_bounds__(ST) k_sel_mark(SelectIn in, RepInfo R, uint32_t n_rep, uint64_t seed,
                                                 int equal_mass, const uint32_t *tb, const uint64_t *cand_off,
                                                 uint32_t *cursor, Cand *cand, uint32_t *bitmap)
{
    ChunkCtx C;
    load_chunk(C, in, R, n_rep);
    const uint32_t b = tb[C.r];
    uint32_t *words = bitmap + R.woff[C.r];
    Cand *cb = cand + cand_off[C.r];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = gbd::lanemask_lt();
    for (int k = 0; k < ROUNDS; ++k) {
        const uint32_t rel0 = C.start + (uint32_t)warp * (ROUNDS * 32) + (uint32_t)k * 32;
        if (rel0 >= C.count) break; // warp-uniform
        const uint32_t rel = rel0 + lane;
        const bool ok = rel < C.count;
        uint64_t key = 0;
        uint32_t id = 0, d = 0xFFFFFFFFu;
        if (ok) {
            key = sel_key(in, C.first + rel, C.code, seed, equal_mass, id);
            d = C.logb ? (uint32_t)(key >> (64 - C.logb)) : 0u;
        }
        const uint32_t below = __ballot_sync(0xffffffffu, ok && d < b);
        if (lane == 0) words[rel0 >> 5] = below;
        const uint32_t eq = __ballot_sync(0xffffffffu, ok && d == b);
        if (eq) {
            const int leader = __ffs(eq) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&cursor[C.r], (uint32_t)__popc(eq));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (ok && d == b) cb[base + __popc(eq & lt)] = Cand{key, id, rel};
        }
    }
}

// bits [sh, sh + nbits) of the 96-bit value (key << 32) | id
__device__ __forceinline__ uint32_t digit96(const Cand &c, int sh, int nbits)
{
    uint64_t v;
    if (sh >= 32)
        v = c.key >> (sh - 32);
    else
        v = (c.key << (32 - sh)) | (uint64_t)(c.id >> sh);
    return (uint32_t)(v & ((1ull << nbits) - 1ull));
}

__global__ void __launch_bounds__(ST) k_sel_resolve(RepInfo R, const uint32_t *need_in, const uint64_t *ccount,
                                                    const uint64_t *cand_off, uint64_t cand_total, Cand *cand,
                                                    uint32_t *bitmap)
{
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_b, s_cum, s_hb, s_cnt;
    const uint32_t r = blockIdx.x;
    uint32_t m = (uint32_t)ccount[r], need = need_in[r];
    Cand *A = cand + cand_off[r];
    Cand *B = cand + cand_total + cand_off[r];
    uint32_t *words = bitmap + R.woff[r];
    int top = 96 - R.logb[r];
    while (need < m && top > 0) {
        const int nbits = top < 8 ? top : 8;
        const int sh = top - nbits;
        for (int i = threadIdx.x; i < 256; i += ST) hist[i] = 0u;
        if (threadIdx.x == 0) s_cnt = 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += ST) atomicAdd(&hist[digit96(A[i], sh, nbits)], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t cum = 0, q = 0;
            for (; q < (1u << nbits); ++q) {
                if (cum + hist[q] >= need) break;
                cum += hist[q];
            }
            s_b = q;
            s_cum = cum;
            s_hb = hist[q];
        }
        __syncthreads();
        const uint32_t b = s_b;
        for (uint32_t i = threadIdx.x; i < m; i += ST) {
            const Cand c = A[i];
            const uint32_t d = digit96(c, sh, nbits);
            if (d < b)
                atomicOr(&words[c.rel >> 5], 1u << (c.rel & 31));
            else if (d == b)
                B[atomicAdd(&s_cnt, 1u)] = c;
        }
        __syncthreads();
        need -= s_cum;
        m = s_hb;
        Cand *t = A;
        A = B;
        B = t;
        top = sh;
        __syncthreads();
    }
    // the remaining candidates are all kept (need == m), or, only possible with duplicate ids,
    // the first `need` of them
    for (uint32_t i = threadIdx.x; i < m && i < need; i += ST) atomicOr(&words[A[i].rel >> 5], 1u << (A[i].rel & 31));
}

__global__ void __launch_bounds__(ST) k_sel_count(SelectIn in, RepInfo R, uint32_t n_rep, const uint32_t *bitmap,
                                                  uint32_t *chunk_sel)
{
    ChunkCtx C;
    load_chunk(C, in, R, n_rep);
    const uint32_t len = min(CH, C.count - C.start);
    const uint32_t nw = (len + 31) / 32;
    const uint32_t *words = bitmap + R.woff[C.r] + C.start / 32;
    uint32_t v = 0;
    for (uint32_t i = threadIdx.x; i < nw; i += ST) v += __popc(words[i]);
    uint32_t tot;
    (void)block_scan_u32(v, tot);
    if (threadIdx.x == 0) chunk_sel[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(ST) k_sel_write(SelectIn in, RepInfo R, uint32_t n_rep, const uint32_t *bitmap,
                                                  const uint32_t *chunk_pos)
{
    __shared__ uint32_t woff[ST / 32];
    ChunkCtx C;
    load_chunk(C, in, R, n_rep);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t len = min(CH, C.count - C.start);
    const uint32_t nw = (len + 31) / 32;
    const uint32_t *words = bitmap + R.woff[C.r] + C.start / 32;
    const uint32_t w0 = (uint32_t)warp * ROUNDS;
    uint32_t mine = 0;
    for (int q = lane; q < ROUNDS; q += 32)
        if (w0 + q < nw) mine += __popc(words[w0 + q]);
    for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
    if (lane == 0) woff[warp] = mine;
    __syncthreads();
    uint32_t base = chunk_pos[blockIdx.x] - chunk_pos[R.chunk_off[C.r]];
    for (int w = 0; w < warp; ++w) base += woff[w];
    const uint64_t pf = in.npfirst[C.node];
    const float wr = in.nw[C.node], sr = in.ns[C.node];
    const uint32_t lt = gbd::lanemask_lt();
    float hm = 0.0f;
    for (int q = 0; q < ROUNDS; ++q) {
        const uint32_t wi = w0 + q;
        if (wi >= nw) break;
        const uint32_t W = words[wi];
        const uint32_t rank = base + __popc(W & lt);
        if (((W >> lane) & 1u) && rank < in.n_max) {
            const uint64_t idx = pf + rank;
            const uint32_t j = C.first + C.start + wi * 32 + lane;
            const float4 p = in.s4[j];
            const float h = __fmul_rn(in.sh[j], sr);
            in.pts4[idx] = make_float4(p.x, p.y, p.z, wr);
            in.hs[idx] = h;
            in.pt_src[idx] = j;
            hm = h > hm ? h : hm;
        }
        base += __popc(W);
    }
    for (int d = 16; d > 0; d >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, hm, d);
        hm = o > hm ? o : hm;
    }
    if (lane == 0 && hm > 0.0f) atomicMax(&in.nhmax[C.node], __float_as_uint(hm));
}

template <class T> T readback(const T *d, cudaStream_t s, HostStage &hs)
{
    T *h = static_cast<T *>(hs.get(sizeof(T)));
    GB_CUDA(cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return *h;
}

} // namespace

void select_representatives(const Allocator &A, cudaStream_t s, HostStage &hs, ScanTmp &scan, const SelectIn &in,
                            const uint32_t *rep_nodes, uint32_t n_rep, uint32_t n_max, uint64_t seed,
                            int equal_mass)
{
    Scratch<uint32_t> nchunks(A, n_rep + 1, s), chunk_off(A, n_rep + 1, s), nbins(A, n_rep, s), hoff(A, n_rep, s);
    Scratch<uint64_t> nwords(A, n_rep, s), woff(A, n_rep, s);
    Scratch<uint8_t> logb(A, n_rep, s);
    Scratch<uint32_t> tot32(A, 2, s);
    Scratch<uint64_t> tot64(A, 1, s);
    launch(GBLOD_K_BUILD_OTHER, k_sel_setup, dim3((n_rep + 255) / 256), dim3(256), 0, s, n_rep, rep_nodes, in.ncount,
           nchunks.p, nbins.p, logb.p, nwords.p);
    scan_exclusive_u32(A, scan, nchunks.p, chunk_off.p, n_rep, chunk_off.p + n_rep, s);
    scan_exclusive_u32(A, scan, nbins.p, hoff.p, n_rep, tot32.p, s);
    scan_exclusive_u64(A, scan, nwords.p, woff.p, n_rep, tot64.p, s);
    uint32_t totals[2];
    GB_CUDA(cudaMemcpyAsync(static_cast<uint32_t *>(hs.get(16)), chunk_off.p + n_rep, 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(static_cast<uint32_t *>(hs.get(16)) + 1, tot32.p, 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    totals[0] = static_cast<uint32_t *>(hs.get(16))[0];
    totals[1] = static_cast<uint32_t *>(hs.get(16))[1];
    const uint64_t total_words = readback(tot64.p, s, hs);
    const uint32_t n_chunks = totals[0], n_bins = totals[1];

    RepInfo R{rep_nodes, chunk_off.p, hoff.p, logb.p, woff.p};
    Scratch<uint32_t> hist(A, n_bins, s), tb(A, n_rep, s), need(A, n_rep, s);
    Scratch<uint64_t> ccount(A, n_rep, s), cand_off(A, n_rep, s);
    Scratch<uint32_t> bitmap(A, total_words, s);
    GB_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)n_bins * 4, s));
    launch(GBLOD_K_SEL_HIST, k_sel_hist, dim3(n_chunks), dim3(ST), 0, s, in, R, n_rep, seed, equal_mass, hist.p);
    launch(GBLOD_K_BUILD_OTHER, k_sel_find, dim3(n_rep), dim3(ST), 0, s, R, n_max, (const uint32_t *)hist.p, tb.p,
           need.p, ccount.p);
    scan_exclusive_u64(A, scan, ccount.p, cand_off.p, n_rep, tot64.p, s);
    const uint64_t cand_total = readback(tot64.p, s, hs);
    Scratch<Cand> cand(A, 2 * (size_t)cand_total + 2, s);
    Scratch<uint32_t> cursor(A, n_rep, s);
    GB_CUDA(cudaMemsetAsync(cursor.p, 0, (size_t)n_rep * 4, s));
    launch(GBLOD_K_SEL_MARK, k_sel_mark, dim3(n_chunks), dim3(ST), 0, s, in, R, n_rep, seed, equal_mass,
           (const uint32_t *)tb.p, (const uint64_t *)cand_off.p, cursor.p, cand.p, bitmap.p);
    launch(GBLOD_K_BUILD_OTHER, k_sel_resolve, dim3(n_rep), dim3(ST), 0, s, R, (const uint32_t *)need.p,
           (const uint64_t *)ccount.p, (const uint64_t *)cand_off.p, cand_total, cand.p, bitmap.p);
    Scratch<uint32_t> chunk_sel(A, n_chunks, s), chunk_pos(A, n_chunks, s);
    launch(GBLOD_K_BUILD_OTHER, k_sel_count, dim3(n_chunks), dim3(ST), 0, s, in, R, n_rep, (const uint32_t *)bitmap.p,
           chunk_sel.p);
    scan_exclusive_u32(A, scan, chunk_sel.p, chunk_pos.p, n_chunks, tot32.p, s);
    launch(GBLOD_K_SEL_WRITE, k_sel_write, dim3(n_chunks), dim3(ST), 0, s, in, R, n_rep, (const uint32_t *)bitmap.p,
           (const uint32_t *)chunk_pos.p);
    const uint32_t kept = readback(tot32.p, s, hs); // modulo 2^32, like the positions it sums
    if (kept != (uint32_t)((uint64_t)n_rep * n_max))
        fail(GBLOD_ERR_CUDA, "subselection kept " + std::to_string(kept) + " points, expected " +
                                 std::to_string((uint64_t)n_rep * n_max));
}

} // namespace gb
