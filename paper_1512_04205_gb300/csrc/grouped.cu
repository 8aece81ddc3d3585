// Grouped launches of a batch plan: the sketch and the subtract pass of every
// clip as one launch each, over a work list built here.
//
//   sketch     one CTA per (frame chunk of <= 256 frames of one clip, or of
//              two consecutive clips that share C, row block of C, range of
//              `sketch_steps` 64-pixel K steps); FP32 partial sums per range,
//              then one fixed-order FP64 reduce over all clips
//   subtract   lambda^t tables (one warp per clip), then on the tensor cores
//              one CTA per range of consecutive 128-pixel tiles of a clip with
//              32 <= n <= 256 frames (about one item per SM), and in the
//              CUDA-core kernel one CTA per range of `subtract_tiles`
//              consecutive 960-pixel tiles of every other clip
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

    // ---- frame chunks, and units of one chunk or two chunks sharing C ----
    struct Chunk {
        int clip, t0, nf, splits;
        int64_t part_off;   // floats
    };
    struct Unit {
        int c0, c1;          // chunk indices (c1 < 0: one chunk)
    };
    std::vector<Chunk> chunks;
    for (size_t i = 0; i < clips.size(); ++i)
        for (int t0 = 0; t0 < clips[i].n; t0 += 256)
            chunks.push_back({static_cast<int>(i), t0, std::min(256, clips[i].n - t0), 0, 0});
    auto shares_c = [&](const Chunk& a, const Chunk& b) {
        const GroupedClip& ca = clips[a.clip];
        const GroupedClip& cb = clips[b.clip];
        return a.clip != b.clip && ca.m == cb.m && ca.k == cb.k && ca.seed == cb.seed &&
               sketch_tc_pair_fits(a.nf, b.nf);
    };
    std::vector<Unit> units;
    for (size_t q = 0; q < chunks.size();) {
        if (q + 1 < chunks.size() && shares_c(chunks[q], chunks[q + 1])) {
            units.push_back({static_cast<int>(q), static_cast<int>(q + 1)});
            q += 2;
        } else {
            units.push_back({static_cast<int>(q), -1});
            q += 1;
        }
    }
    auto unit_rowblks = [&](const Unit& u) {
        const int rows = u.c1 >= 0 ? 128 : 256;
        return (clips[chunks[u.c0].clip].k + rows - 1) / rows;
    };

    // ---- work-item sizes (0 = automatic: about two items per SM) ----
    int64_t unit_steps = 0, tiles_all = 0;
    for (const Unit& u : units)
        unit_steps += static_cast<int64_t>(unit_rowblks(u)) * ((clips[chunks[u.c0].clip].m + 63) / 64);
    for (const GroupedClip& c : clips) tiles_all += (c.m + tile_px - 1) / tile_px;
    if (sketch_steps <= 0)
        sketch_steps = static_cast<int>(std::max<int64_t>(64, (unit_steps + 2 * num_sms - 1) / (2 * num_sms)));
    if (subtract_tiles <= 0)
        subtract_tiles = static_cast<int>(std::max<int64_t>(1, (tiles_all + 2 * num_sms - 1) / (2 * num_sms)));

    // ---- sizes ----
    int64_t part_floats = 0, nsk = 0;
    for (Chunk& ch : chunks) {
        const GroupedClip& c = clips[ch.clip];
        const int64_t steps = (c.m + 63) / 64;
        ch.splits = static_cast<int>((steps + sketch_steps - 1) / sketch_steps);
        ch.part_off = part_floats;
        part_floats += static_cast<int64_t>(ch.splits) * ch.nf * c.k;
    }
    for (const Unit& u : units) nsk += static_cast<int64_t>(unit_rowblks(u)) * chunks[u.c0].splits;
    // the subtract of a clip runs on the tensor cores (mask only, MODULUS or
    // REAL, 32 <= n <= 256) or else in the CUDA-core kernel
    const int tc_px = subtract_tc_tile_pixels();
    std::vector<int> tc_slot(clips.size(), -1);
    int ntc_clips = 0, tc_max_n = 0, tc_max_ncols = 0;
    int64_t tc_tiles_all = 0;
    for (size_t i = 0; i < clips.size(); ++i) {
        const GroupedClip& c = clips[i];
        if (mode != CDMD_BG_STATIC && c.n >= 32 && c.n <= 256 && c.ncols <= 16 &&
            reinterpret_cast<uintptr_t>(c.buf->Phi) % 16 == 0 && reinterpret_cast<uintptr_t>(c.D) % 16 == 0 &&
            c.ldd % 16 == 0) {
            tc_slot[i] = ntc_clips++;
            tc_max_n = std::max(tc_max_n, c.n);
            tc_max_ncols = std::max(tc_max_ncols, c.ncols);
            tc_tiles_all += (c.m + tc_px - 1) / tc_px;
        }
    }
    // about one tensor-core item per SM
    const int64_t tc_item_tiles = std::max<int64_t>(8, (tc_tiles_all + num_sms - 1) / std::max(1, num_sms));
    int64_t nsb = 0, ntc = 0;
    for (size_t i = 0; i < clips.size(); ++i) {
        const GroupedClip& c = clips[i];
        if (tc_slot[i] >= 0) {
            ntc += ((c.m + tc_px - 1) / tc_px + tc_item_tiles - 1) / tc_item_tiles;
        } else {
            const int64_t tiles = (c.m + tile_px - 1) / tile_px;
            nsb += (tiles + subtract_tiles - 1) / subtract_tiles;
        }
    }
    if (nsk > 0x7fffffff || nsb > 0x7fffffff || ntc > 0x7fffffff)
        return fail(CDMD_ERR_UNSUPPORTED, "grouped work list too long");
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
    const size_t o_tm_tc = off;
    off = align256(off + ntc_clips * sizeof(CUtensorMap));
    const size_t o_tcclips = off;
    off = align256(off + ntc_clips * sizeof(SubTcClip));
    const size_t o_tcitems = off;
    off = align256(off + ntc * sizeof(SubtractItem));
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
        rchunks[q] = ReduceChunk{dpart + ch.part_off, c.buf->DY + static_cast<int64_t>(ch.t0) * c.k,
                                 static_cast<int64_t>(ch.nf) * c.k, ch.splits, 0};
        prefix[q + 1] = prefix[q] + rchunks[q].elems;
    }
    size_t max_smem = 0;
    for (const Unit& u : units) {
        const int nclips = u.c1 >= 0 ? 2 : 1;
        const int cq[2] = {u.c0, u.c1 >= 0 ? u.c1 : u.c0};
        const GroupedClip& c = clips[chunks[u.c0].clip];
        const int64_t steps = (c.m + 63) / 64;
        const int rowblks = unit_rowblks(u);
        max_smem = std::max(max_smem, sketch_tc_smem_bytes(nclips == 1 ? 2 : 1, nclips, chunks[cq[0]].nf,
                                                           nclips > 1 ? chunks[cq[1]].nf : 0));
        for (int sp = 0; sp < chunks[u.c0].splits; ++sp)
            for (int rb = 0; rb < rowblks; ++rb) {
                SketchItem it{};
                for (int g = 0; g < 2; ++g) {
                    const Chunk& ch = chunks[cq[g]];
                    it.tmap[g] = dtm_sk + cq[g];
                    it.part[g] = g < nclips ? dpart + ch.part_off + static_cast<int64_t>(sp) * ch.nf * c.k : nullptr;
                    it.n[g] = g < nclips ? ch.nf : 0;
                }
                it.m = c.m;
                it.step0 = static_cast<int64_t>(sp) * sketch_steps;
                it.nsteps = std::min<int64_t>(sketch_steps, steps - it.step0);
                it.key = seed_key(c.seed);
                it.nclips = nclips;
                it.mtiles = nclips == 1 ? 2 : 1;
                it.k = c.k;
                it.rowblk = rb;
                items.push_back(it);
            }
    }
    std::vector<SubtractClip> sbc(clips.size());
    std::vector<SubtractItem> sbi, tci;
    std::vector<CUtensorMap> tm_tc(ntc_clips);
    std::vector<SubTcClip> tcc(ntc_clips);
    const CUtensorMap* dtm_tc = reinterpret_cast<const CUtensorMap*>(dev + o_tm_tc);
    sbi.reserve(nsb);
    tci.reserve(ntc);
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
        if (tc_slot[i] >= 0) {
            const int q = tc_slot[i];
            st = make_subtract_tc_tmap(&tm_tc[q], c.D, c.m, c.n, c.ldd);
            if (st != CDMD_OK) return st;
            SubTcClip t{};
            t.tmap = dtm_tc + q;
            t.Phi = reinterpret_cast<const float2*>(c.buf->Phi);
            t.tb = subtract_tc_table(dev + o_table[i], c.n, nc);
            t.mask = c.mask;
            t.m = c.m;
            t.n = c.n;
            t.ncols = c.ncols;
            t.nc_pad = nc;
            tcc[q] = t;
            const int64_t tiles = (c.m + tc_px - 1) / tc_px;
            for (int64_t t0 = 0; t0 < tiles; t0 += tc_item_tiles)
                tci.push_back(SubtractItem{q, 0, t0, std::min<int64_t>(tc_item_tiles, tiles - t0)});
        } else {
            const int64_t tiles = (c.m + tile_px - 1) / tile_px;
            for (int64_t t0 = 0; t0 < tiles; t0 += subtract_tiles)
                sbi.push_back(SubtractItem{static_cast<int>(i), 0, t0, std::min<int64_t>(subtract_tiles, tiles - t0)});
        }
    }
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tm_sk, tm_sk.data(), tm_sk.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tm_sb, tm_sb.data(), tm_sb.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_items, items.data(), items.size() * sizeof(SketchItem), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_chunks, rchunks.data(), rchunks.size() * sizeof(ReduceChunk),
                               cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_prefix, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_sbclips, sbc.data(), sbc.size() * sizeof(SubtractClip), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_sbitems, sbi.data(), sbi.size() * sizeof(SubtractItem), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tm_tc, tm_tc.data(), tm_tc.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tcclips, tcc.data(), tcc.size() * sizeof(SubTcClip), cudaMemcpyHostToDevice));
    CDMD_CHECK_CUDA(cudaMemcpy(dev + o_tcitems, tci.data(), tci.size() * sizeof(SubtractItem), cudaMemcpyHostToDevice));

    g->built = true;
    g->sketch_steps = sketch_steps;
    g->subtract_tiles = subtract_tiles;
    g->sk_items = reinterpret_cast<const SketchItem*>(dev + o_items);
    g->sk_nitems = static_cast<int>(items.size());
    g->sk_smem = max_smem;
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
    g->tc_clips = reinterpret_cast<const SubTcClip*>(dev + o_tcclips);
    g->tc_items = reinterpret_cast<const SubtractItem*>(dev + o_tcitems);
    g->tc_nitems = static_cast<int>(tci.size());
    g->tc_max_n = tc_max_n;
    g->tc_max_ncols = tc_max_ncols;
    return CDMD_OK;
}

cdmd_status grouped_sketch(const GroupedPlan* g, int* status, cudaStream_t stream) {
    return launch_sketch_grouped(g->sk_items, g->sk_nitems, g->sk_smem, g->rd_chunks, g->rd_prefix, g->rd_nchunks,
                                 g->rd_total, status, stream);
}

cdmd_status grouped_subtract(const GroupedPlan* g, cdmd_bgmode mode, float tau, int* status, cudaStream_t stream) {
    // lambda^t tables of every clip, the CUDA-core items, then the tensor-core items
    cdmd_status st = launch_subtract_grouped(g->sb_clips, g->sb_nclips, g->sb_items, g->sb_nitems, g->sb_nc,
                                             g->sb_max_n, mode, tau, status, stream);
    if (st != CDMD_OK || g->tc_nitems == 0) return st;
    return launch_subtract_tc_grouped(g->tc_clips, g->tc_items, g->tc_nitems, g->tc_max_ncols, mode, tau, status,
                                      stream);
}

}  // namespace cdmd
