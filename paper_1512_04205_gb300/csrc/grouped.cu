// Grouped launches of a batch plan: the sketch and the subtract pass of every
// clip as one launch each, over a work list built here.
//
//   sketch     one CTA per (clip, frame chunk of <= 256 frames, 256-row pair
//              of C, range of `sketch_steps` 64-pixel K steps); FP32 partial
//              sums per range, then one fixed-order FP64 reduce over all clips
//   subtract   lambda^t tables (one warp per clip), then one CTA per range of
//              `subtract_tiles` consecutive 960-pixel tiles of one clip
//
// Tensor maps, descriptors, partial sums and tables live in one device
// allocation written once per work-item size, so the launches can be
// captured into a graph and replayed.
#include <algorithm>

#include "batch_internal.cuh"
#include "tc_common.cuh"

namespace cdmd {
namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int nc_bucket(int ncols) {
    if (ncols <= 4) return 4;
    if (ncols <= 8) return 8;
    if (ncols <= 10) return 10;
    return 12;
}

}  // namespace

void grouped_free(GroupedPlan* g) {
    if (g->dev) cudaFree(g->dev);
    *g = GroupedPlan();
}

cdmd_status grouped_build(GroupedPlan* g, const std::vector<GroupedClip>& clips, cdmd_bgmode mode, int sketch_steps,
                          int subtract_tiles, int num_sms, cudaStream_t stream) {
    (void)mode;
    int max_ncols = 0, max_n = 0;
    for (size_t i = 0; i < clips.size(); ++i) {
        const GroupedClip& c = clips[i];
        if (reinterpret_cast<uintptr_t>(c.D) % 16 != 0 || c.ldd % 16 != 0)
            return fail(CDMD_ERR_UNSUPPORTED, "grouped passes need 16-byte aligned clips (clip %zu)", i);
        if (c.m > 0x7fffffffLL - 2 * subtract_tile_pixels())
            return fail(CDMD_ERR_UNSUPPORTED, "grouped passes: clip %zu too large", i);
        max_ncols = std::max(max_ncols, c.ncols);
        max_n = std::max(max_n, c.n);
    }
    if (max_ncols > 12) return fail(CDMD_ERR_UNSUPPORTED, "grouped subtract covers up to 12 modes per clip");
    const int nc = nc_bucket(max_ncols);
    const int tile_px = subtract_tile_pixels();

    // ---- work-item sizes (0 = automatic: about two items per SM) ----
    int64_t pair_steps = 0, tiles_all = 0;
    for (const GroupedClip& c : clips) {
        pair_steps += static_cast<int64_t>((c.k + 255) / 256) * ((c.m + 63) / 64) * ((c.n + 255) / 256);
        tiles_all += (c.m + tile_px - 1) / tile_px;
    }
    if (sketch_steps <= 0)
        sketch_steps = static_cast<int>(std::max<int64_t>(64, (pair_steps + 2 * num_sms - 1) / (2 * num_sms)));
    if (subtract_tiles <= 0)
        subtract_tiles = static_cast<int>(std::max<int64_t>(1, (tiles_all + 2 * num_sms - 1) / (2 * num_sms)));

    // ---- sizes ----
    struct Chunk {
        int clip, t0, nf, splits;
        int64_t part_off;   // floats
    };
    std::vector<Chunk> chunks;
    int64_t part_floats = 0, nsk = 0;
    for (size_t i = 0; i < clips.size(); ++i) {
        const GroupedClip& c = clips[i];
        const int64_t steps = (c.m + 63) / 64;
        const int splits = static_cast<int>((steps + sketch_steps - 1) / sketch_steps);
        const int pairs = (c.k + 255) / 256;
        for (int t0 = 0; t0 < c.n; t0 += 256) {
            const int nf = std::min(256, c.n - t0);
            chunks.push_back({static_cast<int>(i), t0, nf, splits, part_floats});
            part_floats += static_cast<int64_t>(splits) * nf * c.k;
            nsk += static_cast<int64_t>(pairs) * splits;
        }
    }
    int64_t nsb = 0;
    for (const GroupedClip& c : clips) {
        const int64_t tiles = (c.m + tile_px - 1) / tile_px;
        nsb += (tiles + subtract_tiles - 1) / subtract_tiles;
    }
    if (nsk > 0x7fffffff || nsb > 0x7fffffff) return fail(CDMD_ERR_UNSUPPORTED, "grouped work list too long");
    size_t off = 0;
    const size_t o_tm_sk = off;
    off = align256(off + chunks.size() * sizeof(CUtensorMap));
    const size_t o_tm_sb = off;
    off = align256(off + clips.size() * sizeof(CUtensorMap));
    const size_t o_items = off;
    off = align256(off + nsk * sizeof(SketchItem));
    const size_t o_chunks = off;
    off = align256(off + chunks.size() * sizeof(ReduceChunk));
    const size_t o_prefix = off;
    off = align256(off + (chunks.size() + 1) * sizeof(int64_t));
    const size_t o_sbclips = off;
    off = align256(off + clips.size() * sizeof(SubtractClip));
    const size_t o_sbitems = off;
    off = align256(off + nsb * sizeof(SubtractItem));
    std::vector<size_t> o_table(clips.size());
    for (size_t i = 0; i < clips.size(); ++i) {
        o_table[i] = off;
        off = align256(off + subtract_table_bytes_nc(clips[i].n, nc));
    }
    const size_t o_part = off;
    off = align256(off + part_floats * sizeof(float));

    // ---- allocation (replaces any earlier plan) ----
    if (g->dev) {
        CDMD_CHECK_CUDA(cudaStreamSynchronize(stream));
        cudaFree(g->dev);
        g->dev = nullptr;
    }
    char* dev = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&dev), off) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(CDMD_ERR_NOMEM, "grouped plan: %zu bytes", off);
    }
    g->dev = dev;
    g->dev_bytes = off;

    // ---- descriptors on the host, then one copy per section ----
    std::vector<CUtensorMap> tm_sk(chunks.size()), tm_sb(clips.size());
    std::vector<SketchItem> items;
    items.reserve(nsk);
    std::vector<ReduceChunk> rchunks(chunks.size());
    std::vector<int64_t> prefix(chunks.size() + 1, 0);
    const CUtensorMap* dtm_sk = reinterpret_cast<const CUtensorMap*>(dev + o_tm_sk);
    const CUtensorMap* dtm_sb = reinterpret_cast<const CUtensorMap*>(dev + o_tm_sb);
    float* dpart = reinterpret_cast<float*>(dev + o_part);
    for (size_t q = 0; q < chunks.size(); ++q) {
        const Chunk& ch = chunks[q];
        const GroupedClip& c = clips[ch.clip];
        cdmd_status st = make_video_tmap(&tm_sk[q], c.D + static_cast<int64_t>(ch.t0) * c.ldd, c.m, ch.nf, c.ldd, 64,
                                         ch.nf);
        if (st != CDMD_OK) return st;
        const int64_t steps = (c.m + 63) / 64;
        const int pairs = (c.k + 255) / 256;
        const uint2 key = seed_key(c.seed);
        for (int sp = 0; sp < ch.splits; ++sp)
            for (int pr = 0; pr < pairs; ++pr) {
                SketchItem it{};
                it.tmap = dtm_sk + q;
                it.part = dpart + ch.part_off + static_cast<int64_t>(sp) * ch.nf * c.k;
                it.m = c.m;
                it.step0 = static_cast<int64_t>(sp) * sketch_steps;
                it.nsteps = std::min<int64_t>(sketch_steps, steps - it.step0);
                it.key = key;
                it.n = ch.nf;
                it.k = c.k;
                it.pair = pr;
                items.push_back(it);
            }
        rchunks[q] = ReduceChunk{dpart + ch.part_off, c.buf->DY + static_cast<int64_t>(ch.t0) * c.k,
                                 static_cast<int64_t>(ch.nf) * c.k, ch.splits, 0};
        prefix[q + 1] = prefix[q] + rchunks[q].elems;
    }
    std::vector<SubtractClip> sbc(clips.size());
    std::vector<SubtractItem> sbi;
    sbi.reserve(nsb);
    for (size_t i = 0; i < clips.size(); ++i) {
        const GroupedClip& c = clips[i];
        cdmd_status st = make_subtract_tmap(&tm_sb[i], c.D, c.m, c.n, c.ldd);
        if (st != CDMD_OK) return st;
        SubtractClip d{};
        d.tmap = dtm_sb + i;
        d.Phi = c.buf->Phi;
        d.table = dev + o_table[i];
        d.mask = c.mask;
        d.cols = c.lstsq ? nullptr : c.buf->sel;
        d.beta = c.buf->beta;
        d.lambda = c.buf->lambda;
        d.m = c.m;
        d.words_per_frame = (c.m + 31) / 32;
        d.n = c.n;
        d.ncols = c.ncols;
        d.r = c.r;
        sbc[i] = d;
        const int64_t tiles = (c.m + tile_px - 1) / tile_px;
        for (int64_t t0 = 0; t0 < tiles; t0 += subtract_tiles)
            sbi.push_back(SubtractItem{static_cast<int>(i), 0, t0, std::min<int64_t>(subtract_tiles, tiles - t0)});
    }
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tm_sk, tm_sk.data(), tm_sk.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tm_sb, tm_sb.data(), tm_sb.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_items, items.data(), items.size() * sizeof(SketchItem), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_chunks, rchunks.data(), rchunks.size() * sizeof(ReduceChunk),
                               cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_sbclips, sbc.data(), sbc.size() * sizeof(SubtractClip), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_sbitems, sbi.data(), sbi.size() * sizeof(SubtractItem), cudaMemcpyHostToDevice));

    g->built = true;
    g->sketch_steps = sketch_steps;
    g->subtract_tiles = subtract_tiles;
    g->sk_items = reinterpret_cast<const SketchItem*>(dev + o_items);
    g->sk_nitems = static_cast<int>(items.size());
    int max_nf = 0;
    for (const Chunk& ch : chunks) max_nf = std::max(max_nf, ch.nf);
    g->sk_smem = sketch_tc_smem_bytes(max_nf);
    g->rd_chunks = reinterpret_cast<const ReduceChunk*>(dev + o_chunks);
    g->rd_prefix = reinterpret_cast<const int64_t*>(dev + o_prefix);
    g->rd_nchunks = static_cast<int>(chunks.size());
    g->rd_total = prefix.back();
    g->sb_clips = reinterpret_cast<const SubtractClip*>(dev + o_sbclips);
    g->sb_nclips = static_cast<int>(clips.size());
    g->sb_items = reinterpret_cast<const SubtractItem*>(dev + o_sbitems);
    g->sb_nitems = static_cast<int>(sbi.size());
    g->sb_nc = nc;
    g->sb_max_n = max_n;
    return CDMD_OK;
}

cdmd_status grouped_sketch(const GroupedPlan* g, int* status, cudaStream_t stream) {
    return launch_sketch_grouped(g->sk_items, g->sk_nitems, g->sk_smem, g->rd_chunks, g->rd_prefix, g->rd_nchunks,
                                 g->rd_total, status, stream);
}

cdmd_status grouped_subtract(const GroupedPlan* g, cdmd_bgmode mode, float tau, int* status, cudaStream_t stream) {
    return launch_subtract_grouped(g->sb_clips, g->sb_nclips, g->sb_items, g->sb_nitems, g->sb_nc, g->sb_max_n, mode,
                                   tau, status, stream);
}

}  // namespace cdmd
