// Internal declarations of the batch plan and its grouped launches.
#pragma once

#include <cuda.h>

#include <vector>

#include "cdmd_internal.cuh"

namespace cdmd {

// One clip's results and intermediates inside a batch plan.
struct ClipBuffers {
    double* DY = nullptr;       // k x n
    double* sigma = nullptr;    // r
    double* lambda = nullptr;   // 2r
    double* G = nullptr;        // 2 (n-1) r
    double* beta = nullptr;     // 2r
    int32_t* sel = nullptr;     // K (+ padding)
    int32_t* nsel = nullptr;
    float* Phi = nullptr;       // m x ncols complex
};

// Device-side state of the grouped launches (descriptor arrays, tensor maps,
// partial sums and tables in one allocation), built once per plan and per
// work-item size.
struct SketchItem;
struct ReduceChunk;
struct SubtractClip;
struct SubtractItem;
struct SubTcClip;
struct GroupedPlan {
    bool built = false;
    int sketch_steps = 0;        // 64-pixel K steps per sketch work item
    int subtract_tiles = 0;      // pixel tiles per subtract work item
    void* dev = nullptr;
    size_t dev_bytes = 0;
    // sketch
    const SketchItem* sk_items = nullptr;
    int sk_nitems = 0;
    size_t sk_smem = 0;
    const ReduceChunk* rd_chunks = nullptr;
    const int64_t* rd_prefix = nullptr;
    int rd_nchunks = 0;
    int64_t rd_total = 0;
    // subtract
    const SubtractClip* sb_clips = nullptr;
    int sb_nclips = 0;
    const SubtractItem* sb_items = nullptr;
    int sb_nitems = 0;
    int sb_nc = 0;
    int sb_max_n = 0;
    // tensor-core subtract
    const SubTcClip* tc_clips = nullptr;
    const SubtractItem* tc_items = nullptr;
    int tc_nitems = 0;
    int tc_max_n = 0;
    int tc_max_ncols = 0;
};

struct GroupedClip {             // what the grouped launches need of a clip
    const uint8_t* D;
    int64_t m;
    int n;
    int64_t ldd;
    int k, r, ncols;
    int lstsq;                   // all r modes (no selection list)
    uint64_t seed;
    const ClipBuffers* buf;
    uint32_t* mask;
};

// ---- grouped sketch: one CTA per item ----------------------------------------
struct SketchItem {
    const CUtensorMap* tmap[2];  // frame chunk of each clip (box 64 pixels x n frames), global memory
    float* part[2];              // this item's split of each clip: [n][k] partial sums
    int64_t m;
    int64_t step0, nsteps;       // 64-pixel K steps
    uint2 key;
    int n[2];                    // frames of each clip (<= 256)
    int nclips;                  // clips sharing C (same m, k, seed): 1 or 2
    int mtiles;                  // 128-row tiles of C per CTA: 2 for one clip, 1 for two
    int k, rowblk;               // rows rowblk * 128 mtiles .. of C
};
struct ReduceChunk {             // DY[e] = sum over splits of part[s * elems + e]
    const float* part;
    double* DY;
    int64_t elems;
    int splits;
    int pad;
};
size_t sketch_tc_smem_bytes(int mtiles, int nclips, int n0, int n1);
bool sketch_tc_pair_fits(int n0, int n1);   // two clips of n0, n1 frames can share one CTA's C
cdmd_status launch_sketch_grouped(const SketchItem* items, int nitems, size_t smem, const ReduceChunk* chunks,
                                  const int64_t* prefix, int nchunks, int64_t total, int* status, cudaStream_t stream);

// ---- grouped subtract: lambda^t tables (one warp per clip), then one CTA per
// item of consecutive pixel tiles of one clip --------------------------------
struct SubtractClip {
    const CUtensorMap* tmap;     // box 192 pixels x 16 frames, global memory
    const float* Phi;            // m x ncols complex
    void* table;                 // lambda^t table of this clip (stride nc)
    uint32_t* mask;
    const int32_t* cols;         // selected modes (NULL: 0..ncols-1)
    const double* beta;
    const double* lambda;
    int64_t m;
    int64_t words_per_frame;
    int n, ncols, r;
    int pad;
};
struct SubtractItem {
    int clip;
    int pad;
    int64_t tile0, ntiles;
};
// Tensor-core subtract of one clip inside a grouped launch (mask only,
// MODULUS or REAL, 32 <= n <= 256, ncols <= 16, aligned video and Phi).
struct SubTcClip {
    const CUtensorMap* tmap;     // box 64 pixels x n frames, 64-byte swizzle, global memory
    const float2* Phi;           // m x ncols complex
    SubTcTable tb;               // amplitudes and lambda^t tables of the clip
    uint32_t* mask;
    int64_t m;
    int n, ncols, nc_pad;
    int pad;
};
size_t subtract_tc_smem(int n);
// Views of a table built by the (grouped) table kernel, column stride nc.
SubTcTable subtract_tc_table(void* table, int n, int nc);
int subtract_tc_tile_pixels();
cdmd_status make_subtract_tc_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd);
cdmd_status launch_subtract_tc_grouped(const SubTcClip* clips, const SubtractItem* items, int nitems, int max_ncols,
                                       cdmd_bgmode mode, float tau, int* status, cudaStream_t stream);

size_t subtract_table_bytes_nc(int n, int nc);
size_t subtract_tma_smem(int n, int nc);
int subtract_tile_pixels();
cdmd_status make_subtract_tmap(CUtensorMap* map, const uint8_t* D, int64_t m, int n, int64_t ldd);
cdmd_status launch_subtract_grouped(const SubtractClip* clips, int nclips, const SubtractItem* items, int nitems,
                                    int nc, int max_n, cdmd_bgmode mode, float tau, int* status, cudaStream_t stream);

// Build (or rebuild for new item sizes) the grouped launches' descriptors.
cdmd_status grouped_build(GroupedPlan* g, const std::vector<GroupedClip>& clips, cdmd_bgmode mode, int sketch_steps,
                          int subtract_tiles, int num_sms, cudaStream_t stream);
void grouped_free(GroupedPlan* g);
// The sketch of every clip (partials + fixed-order reduce into each DY).
cdmd_status grouped_sketch(const GroupedPlan* g, int* status, cudaStream_t stream);
// lambda^t tables, then background / threshold / mask of every clip.
cdmd_status grouped_subtract(const GroupedPlan* g, cdmd_bgmode mode, float tau, int* status, cudaStream_t stream);

}  // namespace cdmd
