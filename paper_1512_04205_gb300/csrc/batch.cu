// Batches of clips: one plan for many clips of uneven resolution and length.
//
// The paper cuts long videos into independent 200-frame batches (Section
// 4.1); here many such clips run through one plan.  The plan owns every
// per-clip buffer, a set of lanes (a stream and a context whose workspace
// serves the clips of that lane) and, when asked, a CUDA graph of the whole
// batch:
//
//   fork          the caller's stream -> every lane stream
//   per lane      its clips in order: sketch -> decompose -> lift -> subtract
//   join          every lane -> the caller's stream
//
// With CDMD_BATCH_GROUPED the clips are split into waves of about equal work
// and the sketch and subtract passes of each wave are one grouped launch
// each: the waves' sketches run back to back on the caller's stream; when
// wave w's sketch is done its clips' small solves and lifts run on the lanes,
// and when those are done its grouped subtract runs on a stream of its own.
// So the small solves of one wave overlap the sketch of the next.
//
// Clips are assigned to lanes longest-first (each to the least loaded lane,
// by k m n), so uneven clips balance.  The autotuner times candidate knobs
// on the batch itself (two runs each, the second timed with events) and
// keeps the fastest: the lane count, the SM cap of the lanes' full-data
// passes, the number of waves and the work-item sizes of the grouped
// launches.
#include <algorithm>
#include <vector>

#include "batch_internal.cuh"

struct cdmd_batch {
    int device = 0;
    std::vector<cdmd_clip> clips;
    cdmd_batch_params p{};
    // lanes
    int lanes_max = 0;
    int lanes = 0;
    int sm_limit = 0;
    std::vector<cdmd_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    std::vector<int> lane_of;
    // waves of the grouped passes
    static constexpr int kMaxWaves = 8;
    int waves = 1;
    std::vector<std::vector<int>> wave_clips;
    std::vector<cudaEvent_t> ev_wave_sketch;        // [kMaxWaves]
    std::vector<cudaEvent_t> ev_lane_wave;          // [lanes_max * kMaxWaves]
    cudaStream_t sub_stream = nullptr;
    cudaEvent_t ev_sub_done = nullptr;
    // per-clip buffers (one allocation)
    void* pool = nullptr;
    std::vector<cdmd::ClipBuffers> buf;
    // grouped passes, one plan per wave
    std::vector<cdmd::GroupedPlan> grouped;
    int sketch_steps = 0;
    int subtract_tiles = 0;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float run_ms = 0.0f;
};

namespace cdmd {
namespace {

int ncols_of(const cdmd_batch* b, const cdmd_clip& c) { return b->p.selector == CDMD_SEL_LSTSQ ? c.r : c.K; }

cdmd_status check_clip(const cdmd_batch* b, const cdmd_clip& c, int i) {
    CDMD_REQUIRE(c.D != nullptr && c.mask != nullptr, "clip %d: D or mask is NULL", i);
    CDMD_REQUIRE(c.m >= 1 && c.m <= 0x7fffffffLL, "clip %d: m out of range", i);
    CDMD_REQUIRE(c.n >= 2 && c.n <= 512, "clip %d: n must be in [2, 512]", i);
    CDMD_REQUIRE(c.ldd >= c.m, "clip %d: ldd < m", i);
    CDMD_REQUIRE(c.k >= 1, "clip %d: k must be >= 1", i);
    CDMD_REQUIRE(c.r >= 1 && c.r <= 32 && c.r <= c.k && c.r <= c.n - 1, "clip %d: r must be in [1, min(32, k, n-1)]",
                 i);
    CDMD_REQUIRE(c.K >= 1 && c.K <= c.r, "clip %d: K must be in [1, r]", i);
    if (b->p.prec == CDMD_PREC_BF16X2)
        CDMD_REQUIRE(reinterpret_cast<uintptr_t>(c.D) % 16 == 0 && c.ldd % 16 == 0,
                     "clip %d: BF16X2 needs a 16-byte aligned D and ldd %% 16 == 0", i);
    return CDMD_OK;
}

// Per-clip buffers, 256-byte aligned pieces of one pool.
size_t plan_buffers(cdmd_batch* b, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* q = base ? base + off : nullptr;
        off += (bytes + 255) & ~static_cast<size_t>(255);
        return q;
    };
    b->buf.resize(b->clips.size());
    for (size_t i = 0; i < b->clips.size(); ++i) {
        const cdmd_clip& c = b->clips[i];
        ClipBuffers& q = b->buf[i];
        q.DY = reinterpret_cast<double*>(take(sizeof(double) * c.k * static_cast<size_t>(c.n)));
        q.sigma = reinterpret_cast<double*>(take(sizeof(double) * c.r));
        q.lambda = reinterpret_cast<double*>(take(sizeof(double) * 2 * c.r));
        q.G = reinterpret_cast<double*>(take(sizeof(double) * 2 * static_cast<size_t>(c.n - 1) * c.r));
        q.beta = reinterpret_cast<double*>(take(sizeof(double) * 2 * c.r));
        q.sel = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (c.r + 4)));
        q.nsel = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 4));
        q.Phi = reinterpret_cast<float*>(take(sizeof(float) * 2 * static_cast<size_t>(c.m) * ncols_of(b, c)));
    }
    return off;
}

// Lanes by longest processing time first.
void assign_lanes(cdmd_batch* b) {
    const size_t nc = b->clips.size();
    std::vector<int> order(nc);
    for (size_t i = 0; i < nc; ++i) order[i] = static_cast<int>(i);
    auto cost = [&](int i) {
        const cdmd_clip& c = b->clips[i];
        return static_cast<double>(c.k) * static_cast<double>(c.m) * c.n;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
    std::vector<double> load(b->lanes, 0.0);
    b->lane_of.assign(nc, 0);
    for (int i : order) {
        const int l = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        b->lane_of[i] = l;
        load[l] += cost(i);
    }
    // waves of about equal work, each listing its clips longest first
    const int nw = std::max(1, std::min<int>(b->waves, static_cast<int>(nc)));
    std::vector<double> wl(nw, 0.0);
    b->wave_clips.assign(nw, std::vector<int>());
    for (int i : order) {
        const int w = static_cast<int>(std::min_element(wl.begin(), wl.end()) - wl.begin());
        b->wave_clips[w].push_back(i);
        wl[w] += cost(i);
    }
}

}  // namespace
}  // namespace cdmd

namespace cdmd {
namespace {

bool grouped(const cdmd_batch* b) { return (b->p.flags & CDMD_BATCH_GROUPED) != 0; }
// the grouped sketch is the tensor-core (BF16 hi+lo) kernel; FP32 batches
// sketch per clip
bool grouped_sketch_on(const cdmd_batch* b) { return grouped(b) && b->p.prec == CDMD_PREC_BF16X2; }

// The per-clip passes of clip i on its lane (skipping the passes the grouped
// launches do for every clip).
cdmd_status run_clip(cdmd_batch* b, int i) {
    const cdmd_clip& c = b->clips[i];
    const ClipBuffers& q = b->buf[i];
    const int l = b->lane_of[i];
    cdmd_ctx* ctx = b->ctx[l];
    void* s = b->streams[l];
    const int ncols = ncols_of(b, c);
    cdmd_status st;
    if (!grouped_sketch_on(b)) {
        st = cdmd_sketch(ctx, c.D, c.m, c.n, c.ldd, CDMD_C_GAUSSIAN, c.k, c.seed, b->p.prec, q.DY, s);
        if (st != CDMD_OK) return st;
    }
    st = cdmd_decompose(ctx, q.DY, c.k, c.n, c.r, c.K, b->p.selector, q.sigma, q.lambda, q.G, nullptr, q.beta, q.sel,
                        q.nsel, s);
    if (st != CDMD_OK) return st;
    const int32_t* cols = (b->p.selector == CDMD_SEL_LSTSQ) ? nullptr : q.sel;
    st = cdmd_lift(ctx, c.D, c.m, c.n, c.ldd, q.G, c.r, cols, ncols, b->p.prec, q.Phi, s);
    if (st != CDMD_OK) return st;
    if (!grouped(b))
        st = cdmd_subtract(ctx, c.D, c.m, c.n, c.ldd, q.Phi, ncols, cols, q.beta, q.lambda, c.r, b->p.tau,
                           b->p.bgmode, c.mask, nullptr, s);
    return st;
}

// One run of the whole batch on `stream` (eager, or recorded while capturing).
cdmd_status run_batch(cdmd_batch* b, cudaStream_t stream) {
    for (int l = 0; l < b->lanes; ++l) {
        cdmd_ctx* c = b->ctx[l];
        c->num_sms = b->sm_limit > 0 ? std::min(b->sm_limit, c->device_sms) : c->device_sms;
    }
    CDMD_CHECK_CUDA(cudaEventRecord(b->ev_fork, stream));
    for (int l = 0; l < b->lanes; ++l) CDMD_CHECK_CUDA(cudaStreamWaitEvent(b->streams[l], b->ev_fork, 0));
    if (!grouped(b)) {
        // every clip on its lane, longest first
        std::vector<int> order(b->clips.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
            const cdmd_clip &x = b->clips[a], &y = b->clips[c];
            return static_cast<double>(x.k) * x.m * x.n > static_cast<double>(y.k) * y.m * y.n;
        });
        for (int i : order) {
            cdmd_status st = run_clip(b, i);
            if (st != CDMD_OK) return st;
        }
    } else {
        const int nw = static_cast<int>(b->wave_clips.size());
        CDMD_CHECK_CUDA(cudaStreamWaitEvent(b->sub_stream, b->ev_fork, 0));
        // the waves' grouped sketches, back to back on the caller's stream
        for (int w = 0; w < nw; ++w) {
            if (grouped_sketch_on(b)) {
                cdmd_status st = grouped_sketch(&b->grouped[w], b->ctx[0]->d_status, stream);
                if (st != CDMD_OK) return st;
            }
            CDMD_CHECK_CUDA(cudaEventRecord(b->ev_wave_sketch[w], stream));
        }
        for (int w = 0; w < nw; ++w) {
            // small solves and lifts of wave w on the lanes, once its sketch is done
            for (int l = 0; l < b->lanes; ++l)
                CDMD_CHECK_CUDA(cudaStreamWaitEvent(b->streams[l], b->ev_wave_sketch[w], 0));
            for (int i : b->wave_clips[w]) {
                cdmd_status st = run_clip(b, i);
                if (st != CDMD_OK) return st;
            }
            // then its grouped subtract on the subtract stream
            for (int l = 0; l < b->lanes; ++l) {
                cudaEvent_t e = b->ev_lane_wave[static_cast<size_t>(l) * cdmd_batch::kMaxWaves + w];
                CDMD_CHECK_CUDA(cudaEventRecord(e, b->streams[l]));
                CDMD_CHECK_CUDA(cudaStreamWaitEvent(b->sub_stream, e, 0));
            }
            cdmd_status st = grouped_subtract(&b->grouped[w], b->p.bgmode, b->p.tau, b->ctx[0]->d_status,
                                              b->sub_stream);
            if (st != CDMD_OK) return st;
        }
        CDMD_CHECK_CUDA(cudaEventRecord(b->ev_sub_done, b->sub_stream));
        CDMD_CHECK_CUDA(cudaStreamWaitEvent(stream, b->ev_sub_done, 0));
    }
    for (int l = 0; l < b->lanes; ++l) {
        CDMD_CHECK_CUDA(cudaEventRecord(b->ev_join[l], b->streams[l]));
        CDMD_CHECK_CUDA(cudaStreamWaitEvent(stream, b->ev_join[l], 0));
    }
    return CDMD_OK;
}

std::vector<GroupedClip> grouped_clips(const cdmd_batch* b, int w) {
    const std::vector<int>& ids = b->wave_clips[w];
    std::vector<GroupedClip> g(ids.size());
    for (size_t q = 0; q < ids.size(); ++q) {
        const int i = ids[q];
        const cdmd_clip& c = b->clips[i];
        g[q] = GroupedClip{c.D,       c.m,       c.n, c.ldd, c.k, c.r, ncols_of(b, c),
                           b->p.selector == CDMD_SEL_LSTSQ ? 1 : 0, c.seed, &b->buf[i], c.mask};
    }
    return g;
}

// Configure lanes, SM cap, waves and grouped item sizes, then run once
// eagerly (sizes every workspace).
cdmd_status configure(cdmd_batch* b, int lanes, int sm_limit, int waves, int sketch_steps, int subtract_tiles,
                      cudaStream_t stream) {
    const bool rebuild = b->lanes != lanes || b->waves != waves || b->grouped.empty() ||
                         b->sketch_steps != sketch_steps || b->subtract_tiles != subtract_tiles ||
                         sketch_steps <= 0 || subtract_tiles <= 0;
    b->lanes = lanes;
    b->sm_limit = sm_limit;
    b->waves = waves;
    assign_lanes(b);
    if (grouped(b) && rebuild) {
        for (GroupedPlan& g : b->grouped) grouped_free(&g);
        b->grouped.assign(b->wave_clips.size(), GroupedPlan());
        for (size_t w = 0; w < b->wave_clips.size(); ++w) {
            cdmd_status st = grouped_build(&b->grouped[w], grouped_clips(b, static_cast<int>(w)), b->p.bgmode,
                                           sketch_steps, subtract_tiles, b->ctx[0]->device_sms, stream);
            if (st == CDMD_ERR_UNSUPPORTED) {
                // clips the grouped kernels do not cover: per-clip launches
                b->p.flags &= ~CDMD_BATCH_GROUPED;
                clear_error();
                break;
            } else if (st != CDMD_OK) {
                return st;
            }
        }
    }
    b->sketch_steps = grouped(b) ? b->grouped[0].sketch_steps : 0;
    b->subtract_tiles = grouped(b) ? b->grouped[0].subtract_tiles : 0;
    cdmd_status st = run_batch(b, stream);
    if (st != CDMD_OK) return st;
    CDMD_CHECK_CUDA(cudaStreamSynchronize(stream));
    return CDMD_OK;
}

// Milliseconds of one eager run (after one untimed run).
cdmd_status time_run(cdmd_batch* b, cudaStream_t stream, float* ms) {
    cudaEvent_t e0, e1;
    CDMD_CHECK_CUDA(cudaEventCreate(&e0));
    CDMD_CHECK_CUDA(cudaEventCreate(&e1));
    cdmd_status st = run_batch(b, stream);
    if (st == CDMD_OK) {
        cudaEventRecord(e0, stream);
        st = run_batch(b, stream);
        cudaEventRecord(e1, stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

cdmd_status autotune(cdmd_batch* b, cudaStream_t stream) {
    const int sms = b->ctx[0]->device_sms;
    struct Cand {
        int lanes, sm_limit, waves, sketch_steps, subtract_tiles;
    };
    float best = 1e30f;
    Cand pick = {b->lanes, b->sm_limit, b->waves, b->sketch_steps, b->subtract_tiles};
    auto trial = [&](const Cand& c, bool* better) -> cdmd_status {
        cdmd_status st = configure(b, c.lanes, c.sm_limit, c.waves, c.sketch_steps, c.subtract_tiles, stream);
        if (st != CDMD_OK) return st;
        float ms = 0.0f;
        st = time_run(b, stream, &ms);
        if (st != CDMD_OK) return st;
        *better = ms < best;
        if (*better) best = ms;
        return CDMD_OK;
    };
    // lanes and SM cap
    const int lane_opts[] = {2, 4, 8};
    const int cap_opts[] = {0, sms - 16, sms - 32};
    for (int lo : lane_opts) {
        if (lo > b->lanes_max) continue;
        for (int co : cap_opts) {
            const Cand c = {lo, co, b->waves, 0, 0};
            bool better = false;
            cdmd_status st = trial(c, &better);
            if (st != CDMD_OK) return st;
            if (better) pick = {c.lanes, c.sm_limit, c.waves, b->sketch_steps, b->subtract_tiles};
        }
    }
    if (grouped(b)) {
        // waves at the chosen lanes / cap
        const int wave_opts[] = {1, 2, 4, 8};
        for (int wo : wave_opts) {
            if (wo > static_cast<int>(b->clips.size())) continue;
            const Cand c = {pick.lanes, pick.sm_limit, wo, 0, 0};
            bool better = false;
            cdmd_status st = trial(c, &better);
            if (st != CDMD_OK) return st;
            if (better) pick = {c.lanes, c.sm_limit, wo, b->sketch_steps, b->subtract_tiles};
        }
        // work-item sizes of the grouped passes
        const int base_steps = pick.sketch_steps > 0 ? pick.sketch_steps : 1;
        const int step_opts[] = {base_steps / 2, base_steps, base_steps * 2};
        const int tile_opts[] = {1, 2, 4, 8};
        for (int so : step_opts) {
            if (so < 1) continue;
            for (int to : tile_opts) {
                const Cand c = {pick.lanes, pick.sm_limit, pick.waves, so, to};
                bool better = false;
                cdmd_status st = trial(c, &better);
                if (st != CDMD_OK) return st;
                if (better) pick = c;
            }
        }
    }
    b->run_ms = best;
    return configure(b, pick.lanes, pick.sm_limit, pick.waves, pick.sketch_steps, pick.subtract_tiles, stream);
}

void release(cdmd_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (GroupedPlan& g : b->grouped) grouped_free(&g);
    for (cudaEvent_t e : b->ev_join)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_wave_sketch)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_lane_wave)
        if (e) cudaEventDestroy(e);
    if (b->ev_sub_done) cudaEventDestroy(b->ev_sub_done);
    if (b->sub_stream) cudaStreamDestroy(b->sub_stream);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cdmd_ctx* c : b->ctx) cdmd_destroy(c);
    if (b->pool) cudaFree(b->pool);
}

}  // namespace
}  // namespace cdmd

using namespace cdmd;

extern "C" {

cdmd_status cdmd_batch_create(cdmd_batch** out, int device, const cdmd_clip* clips, int nclips,
                              const cdmd_batch_params* params, void* stream) {
    clear_error();
    CDMD_REQUIRE(out != nullptr && clips != nullptr && params != nullptr, "NULL argument");
    *out = nullptr;
    CDMD_REQUIRE(nclips >= 1, "nclips must be >= 1");
    CDMD_REQUIRE(params->prec == CDMD_PREC_FP32 || params->prec == CDMD_PREC_BF16X2, "unknown precision");
    CDMD_REQUIRE(params->selector != CDMD_SEL_MLP || params->selector_blob != nullptr,
                 "CDMD_SEL_MLP needs selector_blob");
    CDMD_REQUIRE(params->lanes >= 0 && params->lanes <= 64, "lanes must be in [0, 64]");
    cdmd_batch* b = new cdmd_batch();
    b->device = device;
    b->p = *params;
    b->clips.assign(clips, clips + nclips);
    for (int i = 0; i < nclips; ++i) {
        cdmd_status st = check_clip(b, b->clips[i], i);
        if (st != CDMD_OK) {
            delete b;
            return st;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    auto fail_out = [&](cdmd_status st) {
        release(b);
        delete b;
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
    b->lanes_max = params->lanes > 0 ? params->lanes : 8;
    for (int l = 0; l < b->lanes_max; ++l) {
        cdmd_ctx* c = nullptr;
        cdmd_status st = cdmd_create(&c, device);
        if (st != CDMD_OK) return fail_out(st);
        b->ctx.push_back(c);
        if (params->selector == CDMD_SEL_MLP) {
            st = cdmd_selector_load(c, params->selector_blob, stream);
            if (st != CDMD_OK) return fail_out(st);
        }
        cudaStream_t ls = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return fail_out(cuda_fail(cudaGetLastError(), "cdmd_batch_create: streams"));
        b->streams.push_back(ls);
        b->ev_join.push_back(ev);
    }
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_sub_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->sub_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail_out(cuda_fail(cudaGetLastError(), "cdmd_batch_create: events"));
    b->ev_wave_sketch.assign(cdmd_batch::kMaxWaves, nullptr);
    b->ev_lane_wave.assign(static_cast<size_t>(b->lanes_max) * cdmd_batch::kMaxWaves, nullptr);
    for (cudaEvent_t& e : b->ev_wave_sketch)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail_out(cuda_fail(cudaGetLastError(), "cdmd_batch_create: events"));
    for (cudaEvent_t& e : b->ev_lane_wave)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return fail_out(cuda_fail(cudaGetLastError(), "cdmd_batch_create: events"));
    const size_t bytes = plan_buffers(b, nullptr);
    if (cudaMalloc(&b->pool, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail_out(fail(CDMD_ERR_NOMEM, "cdmd_batch_create: %zu bytes of clip buffers", bytes));
    }
    plan_buffers(b, static_cast<char*>(b->pool));
    // default knobs, then (optionally) the autotuner, then the capture
    const int sms = b->ctx[0]->device_sms;
    cdmd_status st = configure(b, b->lanes_max, b->lanes_max > 1 ? sms - 16 : 0, grouped(b) ? 4 : 1, 0, 0, s);
    if (st != CDMD_OK) return fail_out(st);
    if (params->flags & CDMD_BATCH_AUTOTUNE) {
        st = autotune(b, s);
        if (st != CDMD_OK) return fail_out(st);
    }
    if (params->flags & CDMD_BATCH_GRAPH) {
        // capture on a stream of our own (the caller's may be the legacy
        // default stream, which cannot be captured); the graph then launches
        // into any stream
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
            return fail_out(cuda_fail(cudaGetLastError(), "cdmd_batch_create: capture stream"));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return fail_out(cuda_fail(e, "cudaStreamBeginCapture"));
        }
        st = run_batch(b, cs);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (st != CDMD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return fail_out(st);
        }
        if (e != cudaSuccess) return fail_out(cuda_fail(e, "cudaStreamEndCapture"));
        b->graph = graph;
        if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess)
            return fail_out(cuda_fail(cudaGetLastError(), "cudaGraphInstantiate"));
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return CDMD_OK;
}

cdmd_status cdmd_batch_run(cdmd_batch* b, void* stream) {
    clear_error();
    CDMD_REQUIRE(b != nullptr, "batch is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cdmd_status st = CDMD_OK;
    if (b->exec) {
        const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphLaunch");
    } else {
        st = run_batch(b, static_cast<cudaStream_t>(stream));
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return st;
}

cdmd_status cdmd_batch_status_sync(cdmd_batch* b, void* stream) {
    clear_error();
    CDMD_REQUIRE(b != nullptr, "batch is NULL");
    cdmd_status first = CDMD_OK;
    for (int l = 0; l < b->lanes_max; ++l) {
        const cdmd_status st = cdmd_status_sync(b->ctx[l], stream);
        if (first == CDMD_OK) first = st;
    }
    return first;
}

cdmd_status cdmd_batch_views(cdmd_batch* b, int clip, double** DY, double** lambda, double** beta, int32_t** sel,
                             float** Phi) {
    clear_error();
    CDMD_REQUIRE(b != nullptr, "batch is NULL");
    CDMD_REQUIRE(clip >= 0 && clip < static_cast<int>(b->clips.size()), "clip %d out of range", clip);
    const ClipBuffers& q = b->buf[clip];
    if (DY) *DY = q.DY;
    if (lambda) *lambda = q.lambda;
    if (beta) *beta = q.beta;
    if (sel) *sel = q.sel;
    if (Phi) *Phi = q.Phi;
    return CDMD_OK;
}

cdmd_status cdmd_batch_tuning(cdmd_batch* b, int32_t* lanes, int32_t* sm_limit, int32_t* waves,
                              int32_t* sketch_steps, int32_t* subtract_tiles, float* run_ms) {
    clear_error();
    CDMD_REQUIRE(b != nullptr, "batch is NULL");
    if (lanes) *lanes = b->lanes;
    if (sm_limit) *sm_limit = b->sm_limit;
    if (waves) *waves = grouped(b) ? static_cast<int32_t>(b->wave_clips.size()) : 0;
    if (sketch_steps) *sketch_steps = b->sketch_steps;
    if (subtract_tiles) *subtract_tiles = b->subtract_tiles;
    if (run_ms) *run_ms = b->run_ms;
    return CDMD_OK;
}

void cdmd_batch_destroy(cdmd_batch* b) {
    if (b == nullptr) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    release(b);
    delete b;
    if (prev >= 0) cudaSetDevice(prev);
}

cdmd_status cdmd_copy(void* dst, const void* src, size_t bytes, void* stream) {
    clear_error();
    CDMD_REQUIRE(bytes == 0 || (dst != nullptr && src != nullptr), "NULL argument");
    if (bytes == 0) return CDMD_OK;
    CDMD_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)));
    return CDMD_OK;
}

}  // extern "C"
