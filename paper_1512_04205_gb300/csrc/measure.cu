// Gather-form measurement matrices (Section 3.3) and the gather sketch.
//
// SPARSE (very sparse random projections, entries +1 / 0 / -1 with
// probabilities 1/(2s), 1-1/s, 1/(2s)): entry (i, j) is non-zero iff word
// i%4 of Philox counter (j, i/4, 2, 0) is below floor(2^32/s); its sign is +1
// for an even word.  The matrix is built once as CSC by pixel (count, scan,
// fill) and applied in one streaming pass over D: a CTA owns a pixel range
// and a slab of frames, accumulates sign * pixel into an integer k x slab
// tile in shared memory (exact), and writes it as an int32 partial that the
// FP64 reduction sums.
//
// ROWSAMPLE (single-pixel measurements): Floyd's sampling of k distinct
// pixels from the same Philox definition, on the device: the k draws in
// parallel, then one thread walks them in order against a hash set (the
// algorithm is sequential: whether t is taken depends on the earlier picks),
// then a rank sort puts the picks in increasing order.  No host round trip,
// so the build can be captured in a CUDA graph.  The sketch is a plain gather
// of k rows of D.

#include "cdmd_internal.cuh"

namespace cdmd {
namespace {

constexpr uint32_t kStreamSparse = 2u;
constexpr uint32_t kStreamRowsample = 3u;
constexpr uint32_t kStreamSrftFreq = 6u;

// floor(2^32 * density) as a 64-bit integer: entry non-zero iff word < it.
__host__ __device__ inline uint64_t sparse_threshold(double density) {
    return static_cast<uint64_t>(4294967296.0 * density);
}

// nnz of pixel column j
__global__ void sparse_count_kernel(int64_t m, int k, uint2 key, uint64_t thr, int64_t* __restrict__ counts) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int64_t c = 0;
    for (int q = 0; 4 * q < k; ++q) {
        const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(q), kStreamSparse, 0u), key);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * q + e < k && static_cast<uint64_t>(ws[e]) < thr) ++c;
    }
    counts[j] = c;
}

// Exclusive scan of counts[0..m) into col_ptr[0..m], three phases.
constexpr int kScanBlock = 1024;

__global__ void scan_block_kernel(const int64_t* __restrict__ in, int64_t m, int64_t* __restrict__ out,
                                  int64_t* __restrict__ block_sums) {
    __shared__ int64_t s[kScanBlock];
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanBlock + threadIdx.x;
    s[threadIdx.x] = (i < m) ? in[i] : 0;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        const int64_t v = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < m) out[i] = s[threadIdx.x] - ((i < m) ? in[i] : 0);   // exclusive
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_sums_kernel(int64_t* block_sums, int64_t nblocks, int64_t* total) {
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t v = block_sums[b];
        block_sums[b] = run;
        run += v;
    }
    *total = run;
}

__global__ void scan_add_kernel(int64_t* __restrict__ out, int64_t m, const int64_t* __restrict__ block_sums,
                                const int64_t* __restrict__ total) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanBlock + threadIdx.x;
    if (i < m) out[i] += block_sums[blockIdx.x];
    if (i == 0) out[m] = *total;
}

__global__ void sparse_fill_kernel(int64_t m, int k, uint2 key, uint64_t thr, const int64_t* __restrict__ col_ptr,
                                   int64_t capacity, int32_t* __restrict__ row_idx, int* status) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int64_t pos = col_ptr[j];
    for (int q = 0; 4 * q < k; ++q) {
        const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(j), static_cast<uint32_t>(q), kStreamSparse, 0u), key);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (4 * q + e < k && static_cast<uint64_t>(ws[e]) < thr) {
                if (pos < capacity) {
                    const uint32_t sign = (ws[e] & 1u) ? 0x80000000u : 0u;
                    row_idx[pos] = static_cast<int32_t>(static_cast<uint32_t>(4 * q + e) | sign);
                } else {
                    record_status(status, CDMD_ERR_INVALID_ARG);
                }
                ++pos;
            }
        }
    }
}

// One pass over D: CTA (slab, split) accumulates sign * D[t, j] into an
// integer tile acc[i][t - t0] for its pixels.  A thread owns a pixel: it
// loads the slab's frames of that pixel (a warp reads one 32-byte sector per
// frame) and adds them into the rows of the pixel's non-zeros.  The tile's
// row stride is kSlab + 1 words, so the atomic adds of a warp (random rows,
// same frame) spread over the banks instead of meeting in two.
constexpr int kGatherThreads = 512;
constexpr size_t kGatherSmemMax = 232448;   // opt-in shared memory per CTA

template <int kSlab>
__global__ void __launch_bounds__(kGatherThreads)
sparse_sketch_kernel(const uint8_t* __restrict__ D, int64_t m, int n, int64_t ldd, int k,
                     const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                     int64_t pix_per_split, int32_t* __restrict__ part) {
    constexpr int kSlabStride = kSlab + 1;
    extern __shared__ int32_t acc[];   // [k][kSlabStride]
    const int t0 = blockIdx.x * kSlab;
    const int nt = min(kSlab, n - t0);
    for (int idx = threadIdx.x; idx < k * kSlabStride; idx += kGatherThreads) acc[idx] = 0;
    __syncthreads();
    const int64_t pbeg = static_cast<int64_t>(blockIdx.y) * pix_per_split;
    const int64_t pend = min(m, pbeg + pix_per_split);
    for (int64_t j = pbeg + threadIdx.x; j < pend; j += kGatherThreads) {
        const int64_t a = col_ptr[j], b = col_ptr[j + 1];
        if (a == b) continue;
        int32_t x[kSlab];
#pragma unroll
        for (int t = 0; t < kSlab; ++t) x[t] = (t < nt) ? static_cast<int32_t>(D[static_cast<int64_t>(t0 + t) * ldd + j]) : 0;
        for (int64_t e = a; e < b; ++e) {
            const uint32_t code = static_cast<uint32_t>(row_idx[e]);
            const int i = static_cast<int>(code & 0x7fffffffu);
            const bool neg = (code & 0x80000000u) != 0u;
            int32_t* row = acc + i * kSlabStride;
#pragma unroll
            for (int t = 0; t < kSlab; ++t)
                if (t < nt) atomicAdd(row + t, neg ? -x[t] : x[t]);
        }
    }
    __syncthreads();
    int32_t* dst = part + static_cast<int64_t>(blockIdx.y) * k * n;
    for (int idx = threadIdx.x; idx < k * nt; idx += kGatherThreads) {
        const int i = idx / nt, t = idx % nt;
        dst[static_cast<int64_t>(i) * n + t0 + t] = acc[i * kSlabStride + t];
    }
}

__global__ void sparse_reduce_kernel(const int32_t* __restrict__ part, int splits, int k, int n,
                                     double* __restrict__ DY) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(k) * n) return;
    const int i = static_cast<int>(idx / n), t = static_cast<int>(idx % n);
    int64_t s = 0;
    for (int sp = 0; sp < splits; ++sp) s += part[(static_cast<int64_t>(sp) * k + i) * n + t];
    DY[static_cast<int64_t>(t) * k + i] = static_cast<double>(s);
}

// DY[t*k + i] = D[t*ldd + rows[i]]
__global__ void rowsample_sketch_kernel(const uint8_t* __restrict__ D, int n, int64_t ldd, int k,
                                        const int64_t* __restrict__ rows, double* __restrict__ DY) {
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<int64_t>(k) * n) return;
    const int i = static_cast<int>(idx % k), t = static_cast<int>(idx / k);
    DY[idx] = static_cast<double>(D[static_cast<int64_t>(t) * ldd + rows[i]]);
}

// Floyd's sampling of k distinct integers in [0, m), step 1 (parallel): the
// draw of step t = m-k+i, v = floor(((w1 << 32) | w0) (t + 1) / 2^64) from
// words 0, 1 of Philox counter (t, 0, stream, 0) (stream 3: single-pixel rows;
// stream 6: the SRFT's kept frequencies); v is uniform in [0, t].
__global__ void rowsample_draw_kernel(int64_t m, int k, uint2 key, uint32_t stream_id, int64_t* __restrict__ draws) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int64_t t = m - k + i;
    const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(t), 0u, stream_id, 0u), key);
    const uint64_t u64 = (static_cast<uint64_t>(w.y) << 32) | w.x;
    draws[i] = static_cast<int64_t>(__umul64hi(u64, static_cast<uint64_t>(t + 1)));
}

// Open-addressing set of non-negative int64 keys (empty slot = -1), linear
// probing from a multiplicative hash; 2^bits slots, at least twice the keys.
__device__ __forceinline__ uint32_t set_slot(int64_t key, int bits) {
    return static_cast<uint32_t>((static_cast<uint64_t>(key) * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Floyd's sampling, step 2 (one CTA): clear the set, then thread 0 takes the
// draws in order: step t keeps v unless v is already taken, else t (t itself
// is never taken before step t: earlier draws are <= their own t < t).  The
// set lives in dynamic shared memory when `table` is NULL, else in `table`.
__global__ void rowsample_floyd_kernel(int64_t m, int k, const int64_t* __restrict__ draws, int64_t* table,
                                       int bits, int64_t* __restrict__ picks) {
    extern __shared__ int64_t smem_table[];
    int64_t* set = table != nullptr ? table : smem_table;
    const uint32_t slots = 1u << bits;
    for (uint32_t s = threadIdx.x; s < slots; s += blockDim.x) set[s] = -1;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const uint32_t mask = slots - 1u;
    for (int i = 0; i < k; ++i) {
        const int64_t t = m - k + i;
        const int64_t v = draws[i];
        uint32_t s = set_slot(v, bits);
        bool taken = false;
        for (;;) {                                  // ends: the set is at most half full
            const int64_t e = set[s];
            if (e == -1) break;
            if (e == v) { taken = true; break; }
            s = (s + 1u) & mask;
        }
        int64_t pick = v;
        if (taken) {
            pick = t;
            s = set_slot(t, bits);
            while (set[s] != -1) s = (s + 1u) & mask;
        }
        set[s] = pick;
        picks[i] = pick;
    }
}

// Floyd's sampling, step 3: rows[rank] = pick, rank = number of smaller picks
// (the picks are distinct), so rows come out in increasing order.
__global__ void rank_sort_kernel(const int64_t* __restrict__ picks, int k, int64_t* __restrict__ rows) {
    __shared__ int64_t tile[1024];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t mine = i < k ? picks[i] : 0;
    int rank = 0;
    for (int base = 0; base < k; base += 1024) {
        const int cnt = min(1024, k - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) tile[q] = picks[base + q];
        __syncthreads();
        for (int q = 0; q < cnt; ++q) rank += tile[q] < mine ? 1 : 0;
    }
    if (i < k) rows[rank] = mine;
}

}  // namespace

cdmd_status launch_measure_sparse_count(cdmd_ctx* ctx, int64_t m, int k, uint64_t seed, double density,
                                        int64_t* d_counts, cudaStream_t stream) {
    (void)ctx;
    sparse_count_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, stream>>>(
        m, k, seed_key(seed), sparse_threshold(density), d_counts);
    CDMD_CHECK_LAUNCH("sparse_count_kernel");
    return CDMD_OK;
}

cdmd_status launch_measure_build(cdmd_ctx* ctx, cdmd_measure* meas, cudaStream_t stream) {
    if (meas->ctype == CDMD_C_ROWSAMPLE || meas->ctype == CDMD_C_SRFT) {
        // ROWSAMPLE: k pixels of [0, m); SRFT: ceil(k/2) frequencies of [0, m)
        const bool srft = meas->ctype == CDMD_C_SRFT;
        const int64_t m = meas->m;
        const int k = srft ? (meas->k + 1) / 2 : meas->k;
        int bits = 1;
        while ((1ll << bits) < 2ll * k) ++bits;
        const size_t slots = static_cast<size_t>(1) << bits;
        constexpr size_t kSmemTable = static_cast<size_t>(96) << 10;   // set in shared memory up to 96 KB
        const bool in_smem = slots * sizeof(int64_t) <= kSmemTable;
        int64_t* scratch = nullptr;
        const size_t words = 2 * static_cast<size_t>(k) + (in_smem ? 0 : slots);
        cdmd_status st = ensure_buffer(ctx, BUF_SMALL, words * sizeof(int64_t), reinterpret_cast<void**>(&scratch));
        if (st != CDMD_OK) return st;
        int64_t* draws = scratch;
        int64_t* picks = draws + k;
        int64_t* table = in_smem ? nullptr : picks + k;
        rowsample_draw_kernel<<<static_cast<unsigned>((k + 255) / 256), 256, 0, stream>>>(
            m, k, seed_key(meas->seed), srft ? kStreamSrftFreq : kStreamRowsample, draws);
        CDMD_CHECK_LAUNCH("rowsample_draw_kernel");
        const size_t smem = in_smem ? slots * sizeof(int64_t) : 0;
        if (smem > 48 * 1024)
            CDMD_CHECK_CUDA(cudaFuncSetAttribute(rowsample_floyd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem)));
        rowsample_floyd_kernel<<<1, 1024, smem, stream>>>(m, k, draws, table, bits, picks);
        CDMD_CHECK_LAUNCH("rowsample_floyd_kernel");
        rank_sort_kernel<<<static_cast<unsigned>((k + 255) / 256), 256, 0, stream>>>(picks, k, meas->rows);
        CDMD_CHECK_LAUNCH("rank_sort_kernel");
        return CDMD_OK;
    }
    // SPARSE: count -> scan -> fill
    const int64_t m = meas->m;
    const int64_t nblocks = (m + kScanBlock - 1) / kScanBlock;
    int64_t* scratch = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SMALL, static_cast<size_t>(m + nblocks + 2) * sizeof(int64_t),
                                   reinterpret_cast<void**>(&scratch));
    if (st != CDMD_OK) return st;
    int64_t* counts = scratch;
    int64_t* bsums = counts + m;
    int64_t* total = bsums + nblocks;
    st = launch_measure_sparse_count(ctx, m, meas->k, meas->seed, meas->density, counts, stream);
    if (st != CDMD_OK) return st;
    scan_block_kernel<<<static_cast<unsigned>(nblocks), kScanBlock, 0, stream>>>(counts, m, meas->col_ptr, bsums);
    CDMD_CHECK_LAUNCH("scan_block_kernel");
    scan_sums_kernel<<<1, 32, 0, stream>>>(bsums, nblocks, total);
    CDMD_CHECK_LAUNCH("scan_sums_kernel");
    scan_add_kernel<<<static_cast<unsigned>(nblocks), kScanBlock, 0, stream>>>(meas->col_ptr, m, bsums, total);
    CDMD_CHECK_LAUNCH("scan_add_kernel");
    sparse_fill_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, stream>>>(
        m, meas->k, seed_key(meas->seed), sparse_threshold(meas->density), meas->col_ptr, meas->nnz_capacity,
        meas->row_idx, ctx->d_status);
    CDMD_CHECK_LAUNCH("sparse_fill_kernel");
    return CDMD_OK;
}

cdmd_status launch_sketch_gather(cdmd_ctx* ctx, const uint8_t* D, int64_t m, int n, int64_t ldd,
                                 const cdmd_measure* meas, double* DY, cudaStream_t stream) {
    const int k = meas->k;
    if (meas->ctype == CDMD_C_SRFT) return launch_sketch_srft(ctx, D, m, n, ldd, meas, DY, stream);
    if (meas->ctype == CDMD_C_ROWSAMPLE) {
        const int64_t tot = static_cast<int64_t>(k) * n;
        rowsample_sketch_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, stream>>>(D, n, ldd, k, meas->rows, DY);
        CDMD_CHECK_LAUNCH("rowsample_sketch_kernel");
        return CDMD_OK;
    }
    // frames per slab: 32 while the k x 33 integer tile fits, else 16
    const int slab = (static_cast<size_t>(k) * 33 * sizeof(int32_t) <= kGatherSmemMax) ? 32 : 16;
    const int slabs = (n + slab - 1) / slab;
    // about two CTAs per SM in total (the tile takes up to ~130 KB)
    int64_t splits = std::max<int64_t>(1, (2LL * ctx->num_sms + slabs - 1) / slabs);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, m / 4096));
    const int64_t pps = (m + splits - 1) / splits;
    splits = (m + pps - 1) / pps;
    int32_t* part = nullptr;
    cdmd_status st = ensure_buffer(ctx, BUF_SKETCH_PARTIAL, static_cast<size_t>(splits) * k * n * sizeof(int32_t),
                                   reinterpret_cast<void**>(&part));
    if (st != CDMD_OK) return st;
    const size_t smem = static_cast<size_t>(k) * (slab + 1) * sizeof(int32_t);
    const dim3 grid(slabs, static_cast<unsigned>(splits));
    if (slab == 32) {
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(sparse_sketch_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kGatherSmemMax)));
        sparse_sketch_kernel<32><<<grid, kGatherThreads, smem, stream>>>(D, m, n, ldd, k, meas->col_ptr, meas->row_idx,
                                                                          pps, part);
    } else {
        CDMD_CHECK_CUDA(cudaFuncSetAttribute(sparse_sketch_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kGatherSmemMax)));
        sparse_sketch_kernel<16><<<grid, kGatherThreads, smem, stream>>>(D, m, n, ldd, k, meas->col_ptr, meas->row_idx,
                                                                          pps, part);
    }
    CDMD_CHECK_LAUNCH("sparse_sketch_kernel");
    const int64_t tot = static_cast<int64_t>(k) * n;
    sparse_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, stream>>>(part, static_cast<int>(splits), k, n, DY);
    CDMD_CHECK_LAUNCH("sparse_reduce_kernel");
    return CDMD_OK;
}

}  // namespace cdmd
