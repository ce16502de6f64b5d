// vi_server.cu -- continuous-batching render server (host side of vi_server_*).
//
// Requests (volume, TF, light, stack shape, camera, output) arrive at any time
// and are admitted in arrival order into a fixed set of render slots as slots
// and device memory free up.  Each slot is a context with its own CUDA stream:
// the frames of different requests run their sweeps and marches concurrently
// on the GPU, so small frames fill it together instead of one after another.
// Volumes are registered once and kept resident (pair bricks and brick ranges) up
// to a count and a byte budget; when room is needed an idle volume is evicted
// (by default the one whose GreedyDual credit -- reload cost plus an aging
// clock -- is lowest, or the least recently used one) and reloaded from the
// caller's host copy on its next request.  Each slot keeps its last attenuation stack for a later view of
// the same scene.  Optionally a request's device work after its uploads is
// captured and launched as one CUDA graph.  Completion is signalled by a stream
// host callback; every wait on the host side is bounded (VI_ETIMEOUT).
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vi_context.h"

namespace {

using Clock = std::chrono::steady_clock;

struct ServerVolume {
    VolumeRes res;
    size_t used = 0;  // device bytes of res
    const void* host = nullptr;
    int dtype = 0, nx = 0, ny = 0, nz = 0;
    bool resident = false;
    int pins = 0;           // slots rendering from it
    uint64_t last_use = 0;  // admission counter at last use
    double credit = 0;      // GreedyDual credit: the aging clock at last use + reload cost
    cudaEvent_t ready = nullptr;  // recorded after its last load; every reader's stream waits on it
};

struct Request {
    uint64_t ticket = 0;
    vi_request req{};
    std::vector<float> tf;
    int status = VI_REQ_QUEUED;
    int result = VI_OK;
    double t_submit = 0, t_start = 0, t_end = 0;
};

struct Slot {
    vi_server* server = nullptr;
    vi_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    Request* req = nullptr;
    int vol = -1;
    std::atomic<bool> gpu_done{false};  // set by the stream callback
    // The request whose attenuation stack the context holds (its build
    // succeeded and nothing has freed it since); null if none.
    bool has_stack = false;
    uint64_t stack_use = 0;  // admission counter when the kept stack last served a request
    vi_request stack_req{};
    std::vector<float> stack_tf;
    // Executable graphs of a request's device work, one per shape of it:
    // index 1 with a sweep, + 2 with a copy to host output.
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
    bool batched = false;         // the current request's march is in a batch
    int* batch_status = nullptr;  // page-locked: its frame's status word
};

bool same_bits(float a, float b) { return std::memcmp(&a, &b, sizeof(float)) == 0; }

// True if request r needs exactly the stack (and TF and light) slot sl holds.
bool stack_matches(const Slot* sl, const Request* r) {
    if (!sl->has_stack) return false;
    const vi_request &a = sl->stack_req, &b = r->req;
    const vi_build_opts &x = a.build, &y = b.build;
    bool eq = a.volume_id == b.volume_id && a.tf_entries == b.tf_entries &&
              same_bits(a.tf_vmin, b.tf_vmin) && same_bits(a.tf_vmax, b.tf_vmax) &&
              a.n_slices == b.n_slices && a.slice_res == b.slice_res && a.mode == b.mode &&
              x.format == y.format && same_bits(x.cone_half_angle_deg, y.cone_half_angle_deg) &&
              same_bits(x.shell_radius_vox, y.shell_radius_vox) &&
              x.opacity_correction == y.opacity_correction && same_bits(x.comp_n, y.comp_n) &&
              x.quantity == y.quantity && x.shell_count == y.shell_count;
    for (int i = 0; eq && i < 3; ++i)
        eq = same_bits(a.light_dir[i], b.light_dir[i]) &&
             same_bits(a.light_color[i], b.light_color[i]);
    return eq && sl->stack_tf.size() == r->tf.size() &&
           std::memcmp(sl->stack_tf.data(), r->tf.data(), r->tf.size() * sizeof(float)) == 0;
}

}  // namespace

struct vi_server {
    int device = 0;
    size_t budget = 0;
    int max_resident = 0;
    Clock::time_point t0;
    std::vector<ServerVolume*> vols;
    std::vector<Slot*> slots;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1, admissions = 0;
    vi_server_stats stats{};
    std::mutex mu;
    std::condition_variable wake;  // worker: new request or a finished slot
    std::condition_variable done;  // waiters: a request finished
    std::thread worker;
    bool stop = false;
    // Stream-ordered pool for every device buffer of the server (volumes and
    // slots): evictions and reloads reuse blocks without cudaMalloc / cudaFree.
    cudaMemPool_t pool = nullptr;
    bool graphs = false;  // launch each request's device work as one CUDA graph
    // Batched marches: the requests admitted in one scheduling pass are
    // marched together in persistent launches on batch_stream, each frame
    // waiting on the device for its slot's stack.
    bool batching = false;
    cudaStream_t batch_stream = nullptr;
    std::vector<Slot*> pending;  // admitted this pass, march not yet enqueued
    double batch_wait_ms = 10000.0;
    int eviction = VI_EVICT_COST;  // victim choice (vi_server_set_eviction)
    double gd_clock = 0;           // GreedyDual aging clock: the credit of the last victim
};

namespace {

double now_ms(const vi_server* s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

size_t bytes_in_use(const vi_server* s) {
    size_t b = 0;
    for (const ServerVolume* v : s->vols) b += v->used;
    for (const Slot* sl : s->slots) b += sl->ctx->used;
    return b;
}

// Runs on the driver's callback thread once a slot's frame is done.  It takes
// no lock (the worker may hold it across a synchronising CUDA call); a missed
// wake-up only delays the worker to its next bounded wait.
void CUDART_CB on_slot_done(void* p) {
    Slot* sl = static_cast<Slot*>(p);
    sl->gpu_done.store(true, std::memory_order_release);
    sl->server->wake.notify_one();
}

// Device bytes a request needs in a slot beyond what the slot holds now.
size_t slot_growth(const Slot* sl, const Request* r, const ServerVolume* v) {
    const vi_request& q = r->req;
    const int fmt = q.mode == VI_NONE ? 0 : q.build.format;
    const size_t esize = fmt == VI_F32 ? 4 : 2;
    vi_detail::StackLayout L;
    const size_t stack =
        q.mode == VI_NONE ||
                vi_detail::stack_layout(sl->ctx->device, q.n_slices, q.slice_res, esize, &L) != VI_OK
            ? 0
            : L.bytes;
    constexpr int B = 1 << vi::kBrickShift;
    const size_t bricks =
        (size_t)((v->nx + B - 1) / B) * ((v->ny + B - 1) / B) * ((v->nz + B - 1) / B);
    const size_t out = q.out_on_device ? 0 : (size_t)q.width * q.height * 16;
    const vi_ctx* c = sl->ctx;
    auto grow = [](size_t need, size_t cap) { return need > cap ? need - cap : 0; };
    return grow(stack, c->stack_cap) + grow(q.tf_entries * 16, c->tf_cap) +
           grow((q.tf_entries + 1) * 4, c->tfcnt_cap) + grow(bricks + 2 * bricks * vi::kCellsPerBrick * vi::kCellsPerBrick * vi::kCellsPerBrick,
                c->bflags_cap) +
           grow(out, c->out_cap) + grow(256, c->counter_cap);
}

// Frees an idle volume's buffers, ordered on `stream`: no device-wide
// synchronisation, and the pool hands the blocks to the next allocations.
void evict(vi_server* s, ServerVolume* v, cudaStream_t stream) {
    vi_detail::volume_release(&v->res, &v->used, stream);
    v->resident = false;
    ++s->stats.volume_evictions;
}

// Raw voxel bytes of a volume: what a reload copies from the host.
size_t raw_bytes(const ServerVolume* v) {
    return (size_t)v->nx * (size_t)v->ny * (size_t)v->nz * (v->dtype == VI_U16 ? 2 : 1);
}

// Reload cost of a volume, in MiB of raw voxels: its host-to-device copy and
// its pair-brick build both grow with it.
double reload_cost(const ServerVolume* v) { return (double)raw_bytes(v) / (1 << 20); }

// The idle resident volume to evict next (never `keep`), or null.
// VI_EVICT_LRU: the least recently used.  VI_EVICT_COST (GreedyDual, with the
// reload cost as the cost): the lowest credit, where a volume's credit is set
// at each use to the aging clock plus its reload cost and the clock rises to
// each victim's credit -- so a volume that is costly to reload stays resident
// over cheap ones until it has gone unused for long enough (ties: the least
// recently used).
ServerVolume* pick_victim(vi_server* s, int keep) {
    ServerVolume* victim = nullptr;
    for (int i = 0; i < (int)s->vols.size(); ++i) {
        ServerVolume* v = s->vols[i];
        if (i == keep || !v->resident || v->pins) continue;
        if (!victim) {
            victim = v;
        } else if (s->eviction == VI_EVICT_COST && v->credit != victim->credit) {
            if (v->credit < victim->credit) victim = v;
        } else if (v->last_use < victim->last_use) {
            victim = v;
        }
    }
    if (victim && s->eviction == VI_EVICT_COST && victim->credit > s->gd_clock)
        s->gd_clock = victim->credit;
    return victim;
}

// Makes room for `extra` bytes: first frees the stacks of idle slots other
// than `target`, then evicts idle volumes (pick_victim's order, never
// `keep`); true if the budget now allows it.
bool make_room(vi_server* s, size_t extra, const Slot* target, int keep) {
    if (!s->budget) return true;
    for (Slot* sl : s->slots) {
        if (bytes_in_use(s) + extra <= s->budget) return true;
        if (sl != target && !sl->req) {
            vi_detail::ctx_trim(sl->ctx);
            sl->has_stack = false;
        }
    }
    while (bytes_in_use(s) + extra > s->budget) {
        ServerVolume* victim = pick_victim(s, keep);
        if (!victim) return false;
        evict(s, victim, target->stream);
    }
    return true;
}

void finish(vi_server* s, Request* r, int status, int result) {
    r->status = status;
    r->result = result;
    r->t_end = now_ms(s);
    if (status == VI_REQ_DONE) ++s->stats.completed;
    else if (status == VI_REQ_FAILED) ++s->stats.failed;
    else if (status == VI_REQ_CANCELLED) ++s->stats.cancelled;
    s->done.notify_all();
}

// True if the request's output can be the target of a captured copy: device
// memory, or page-locked host memory (a copy to pageable memory is not).
bool output_capturable(const vi_request& q) {
    if (q.out_on_device) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q.out_rgba) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// Ends the capture begun on the slot's stream and, if the captured calls
// succeeded (rc), launches the graph: through the slot's executable graph
// for this shape of work, updated in place, or a new one when there is none
// or the update is refused.  Returns a vi_status.
int launch_captured(vi_server* s, Slot* sl, int rc, int shape) {
    sl->ctx->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(sl->stream, &g);
    if (!rc && (e != cudaSuccess || !g)) rc = VI_ECUDA;
    cudaGraphExec_t& x = sl->exec[shape];
    if (!rc && x) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(x, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    }
    if (!rc && !x) {
        if (cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
            ++s->stats.graph_instantiations;
        } else {
            x = nullptr;
            rc = VI_ECUDA;
        }
    }
    if (!rc) rc = cudaGraphLaunch(x, sl->stream) == cudaSuccess ? VI_OK : VI_ECUDA;
    if (!rc) ++s->stats.graph_launches;
    if (g) cudaGraphDestroy(g);
    if (rc) cudaGetLastError();
    return rc;
}

// Whether a request's march can join a batch (vi_render_batch's restrictions).
bool batchable(const vi_request& q) {
    return (q.mode == VI_NONE || q.build.format == VI_F32 || q.build.format == VI_F16) &&
           q.build.quantity == VI_TRANSMITTANCE && q.build.shell_count <= 1 &&
           q.render.slice_filter == VI_SLICE_NEAREST && q.width > 0 && q.height > 0;
}

// Enqueues a request's work on a slot; returns a vi_status.  With `reuse` the
// slot's kept stack (and TF and light) serve the request and no sweep runs.
// With graphs on, the sweep, the march, the output copy and the completion
// callback are captured and launched as one graph after the uploads.
int start(vi_server* s, Slot* sl, Request* r, bool reuse) {
    vi_detail::NvtxRange nvtx_range("vi_server request");
    const vi_request& q = r->req;
    ServerVolume* v = s->vols[q.volume_id];
    vi_ctx* c = sl->ctx;
    int rc = cudaStreamWaitEvent(sl->stream, v->ready, 0) == cudaSuccess ? VI_OK : VI_ECUDA;
    if (!rc) rc = vi_detail::ctx_bind_volume(c, &v->res, reuse);
    if (!reuse) {
        sl->has_stack = false;
        if (!rc)
            rc = vi_set_transfer_function(c, r->tf.data(), q.tf_entries, q.tf_vmin, q.tf_vmax);
        if (!rc) rc = vi_set_light(c, q.light_dir, q.light_color);
    }
    const bool sweep = !reuse && q.mode != VI_NONE;
    sl->batched = false;
    if (!rc && s->batching && batchable(q)) {
        // The sweep (or nothing) on the slot's stream, then the publication the
        // batch's frame waits for on the device; the march joins this pass's
        // batch (flush_batch).
        if (!reuse) {
            rc = vi_build_attenuation(c, q.n_slices, q.slice_res, q.mode, &q.build);
            if (!rc) {
                sl->has_stack = true;
                sl->stack_req = q;
                sl->stack_tf = r->tf;
            }
        }
        if (!rc) rc = vi_post_ready(c);
        if (!rc) {
            sl->batched = true;
            s->pending.push_back(sl);
        }
        return rc;
    }
    const bool graph = !rc && s->graphs && output_capturable(q);
    if (graph) {
        rc = vi_detail::ctx_reserve(c, sweep, q.n_slices, q.slice_res, q.build.format, q.width,
                                    q.height, q.out_on_device);
        if (rc) return rc;
        if (cudaStreamBeginCapture(sl->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return VI_ECUDA;
        }
        c->capturing = true;
    }
    if (!rc && !reuse) {
        rc = vi_build_attenuation(c, q.n_slices, q.slice_res, q.mode, &q.build);
        if (!rc) {
            sl->has_stack = true;
            sl->stack_req = q;
            sl->stack_tf = r->tf;
        }
    }
    if (!rc)
        rc = vi_detail::ctx_render_async(c, &q.camera, q.width, q.height, q.step_vox, q.out_rgba,
                                         q.out_on_device, &q.render);
    if (!rc && cudaLaunchHostFunc(sl->stream, on_slot_done, sl) != cudaSuccess) rc = VI_ECUDA;
    if (graph) rc = launch_captured(s, sl, rc, (sweep ? 1 : 0) + (q.out_on_device ? 0 : 2));
    return rc;
}

// Fails a slot's request that could not be enqueued.
void fail_slot(vi_server* s, Slot* sl, int rc) {
    sl->has_stack = false;
    cudaStreamSynchronize(sl->stream);
    vi_sync(sl->ctx);
    --s->vols[sl->vol]->pins;
    finish(s, sl->req, VI_REQ_FAILED, rc);
    sl->req = nullptr;
    sl->vol = -1;
    sl->batched = false;
}

// Enqueues the marches of the requests admitted in this pass as one batch on
// the batch stream, then their host-output copies and completion callbacks.
void flush_batch(vi_server* s) {
    if (s->pending.empty()) return;
    vi_detail::NvtxRange nvtx_range("vi_server batch");
    std::vector<Slot*> slots;
    std::vector<vi::BatchFrame> tab;
    std::vector<vi_ctx*> ctxs;
    std::vector<int*> dst;
    for (Slot* sl : s->pending) {
        const vi_request& q = sl->req->req;
        vi::BatchFrame b;
        const int rc = vi_detail::ctx_batch_frame(sl->ctx, &q.camera, q.width, q.height,
                                                  q.step_vox, q.out_rgba, q.out_on_device,
                                                  &q.render, &b);
        if (rc) {
            fail_slot(s, sl, rc);
            continue;
        }
        b.index = (int)tab.size();
        *sl->batch_status = VI_OK;
        tab.push_back(b);
        slots.push_back(sl);
        ctxs.push_back(sl->ctx);
        dst.push_back(sl->batch_status);
    }
    s->pending.clear();
    if (tab.empty()) return;
    cudaError_t e = vi_detail::enqueue_batch(ctxs.data(), tab.data(), (int)tab.size(),
                                             (unsigned long long)(s->batch_wait_ms * 1e6),
                                             dst.data(), s->batch_stream);
    for (size_t k = 0; k < slots.size(); ++k) {
        Slot* sl = slots[k];
        const vi_request& q = sl->req->req;
        if (e == cudaSuccess && !q.out_on_device)
            e = cudaMemcpyAsync(q.out_rgba, sl->ctx->out, (size_t)q.width * q.height * 16,
                                cudaMemcpyDeviceToHost, s->batch_stream);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s->batch_stream, on_slot_done, sl);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(s->batch_stream);
            fail_slot(s, sl, VI_ECUDA);
        }
    }
    ++s->stats.batches;
    s->stats.batched_frames += tab.size();
}

// One pass of the scheduler under the lock: retire finished slots, then admit
// queued requests in order while a slot and the memory budget allow.
void schedule(vi_server* s) {
    for (Slot* sl : s->slots) {
        if (!sl->req || !sl->gpu_done.load(std::memory_order_acquire)) continue;
        int rc = vi_sync(sl->ctx);
        if (!rc && sl->batched) rc = *sl->batch_status;  // VI_ETIMEOUT if its wait ran out
        sl->batched = false;
        finish(s, sl->req, rc ? VI_REQ_FAILED : VI_REQ_DONE, rc);
        --s->vols[sl->vol]->pins;
        sl->req = nullptr;
        sl->vol = -1;
        sl->gpu_done.store(false);
    }
    while (!s->queue.empty()) {
        Request* r = s->queue.front();
        // A free slot that holds the stack this request needs; else a free one
        // that holds no stack; else the free one whose stack was used longest
        // ago (the kept stacks are a least-recently-used cache).
        Slot* sl = nullptr;
        bool reuse = false;
        for (Slot* cand : s->slots) {
            if (cand->req) continue;
            if (stack_matches(cand, r)) {
                sl = cand;
                reuse = true;
                break;
            }
            if (!sl || (sl->has_stack && !cand->has_stack) ||
                (sl->has_stack == cand->has_stack && cand->stack_use < sl->stack_use))
                sl = cand;
        }
        if (!sl) break;
        const int vid = r->req.volume_id;
        ServerVolume* v = s->vols[vid];
        const size_t vol_need = v->resident ? 0 : vi_detail::volume_bytes(v->dtype, v->nx, v->ny,
                                                                           v->nz);
        const size_t need = vol_need + slot_growth(sl, r, v);
        bool busy = false;
        for (Slot* o : s->slots) busy = busy || o->req;
        if (!make_room(s, need, sl, vid)) {
            if (busy) break;  // wait for running frames to release memory
            s->queue.pop_front();
            finish(s, r, VI_REQ_FAILED, VI_ENOMEM);
            continue;
        }
        if (s->max_resident && !v->resident) {
            int resident = 0;
            for (ServerVolume* o : s->vols) resident += o->resident;
            while (resident >= s->max_resident) {
                ServerVolume* victim = pick_victim(s, vid);
                if (!victim) break;
                evict(s, victim, sl->stream);
                --resident;
            }
            if (resident >= s->max_resident) {
                if (busy) break;
                s->queue.pop_front();
                finish(s, r, VI_REQ_FAILED, VI_ENOMEM);
                continue;
            }
        }
        s->queue.pop_front();
        if (!v->resident) {
            vi_detail::NvtxRange nvtx_range("vi_server volume load");
            int rc = vi_detail::volume_load(&v->res, &v->used, 0, v->host, v->dtype, v->nx,
                                                  v->ny, v->nz, 0, sl->stream, nullptr);
            // Slots on other streams may read this volume next: they wait on
            // this event (pair bricks and brick ranges built) before they do.
            if (!rc && cudaEventRecord(v->ready, sl->stream) != cudaSuccess) rc = VI_ECUDA;
            if (rc) {
                vi_detail::volume_release(&v->res, &v->used, sl->stream);  // a partial load
                finish(s, r, VI_REQ_FAILED, rc);
                continue;
            }
            v->resident = true;
            ++s->stats.volume_loads;
            s->stats.volume_load_bytes += raw_bytes(v);
        }
        v->last_use = ++s->admissions;
        v->credit = s->gd_clock + reload_cost(v);
        sl->stack_use = s->admissions;
        ++v->pins;
        sl->req = r;
        sl->vol = vid;
        sl->gpu_done.store(false);
        r->status = VI_REQ_RUNNING;
        r->t_start = now_ms(s);
        const int rc = start(s, sl, r, reuse);
        if (!rc && reuse) ++s->stats.stack_reuses;
        if (rc) fail_slot(s, sl, rc);
        const size_t b = bytes_in_use(s);
        if (b > s->stats.peak_bytes) s->stats.peak_bytes = b;
    }
    flush_batch(s);
}

void worker_main(vi_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        schedule(s);
        bool busy = false;
        for (Slot* sl : s->slots) busy = busy || sl->req;
        if (s->stop && !busy) break;
        s->wake.wait_for(lk, std::chrono::milliseconds(2));
    }
}

bool finite3(const float v[3]) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

}  // namespace

extern "C" {

int vi_server_create(vi_server** out, int device, int slots, size_t memory_budget,
                     int max_resident_volumes) {
    if (!out) return VI_EINVAL;
    *out = nullptr;
    if (slots < 1 || slots > 64 || max_resident_volumes < 0) return VI_EINVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return VI_ECUDA;
    }
    if (device < 0 || device >= count) return VI_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return VI_ECUDA;
    vi_server* s = new (std::nothrow) vi_server();
    if (!s) return VI_ENOMEM;
    s->device = device;
    s->budget = memory_budget;
    s->max_resident = max_resident_volumes;
    s->t0 = Clock::now();
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaGetLastError();
        if (s->pool) cudaMemPoolDestroy(s->pool);
        delete s;
        return VI_ECUDA;
    }
    for (int i = 0; i < slots; ++i) {
        Slot* sl = new Slot();
        sl->server = s;
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
            vi_create(&sl->ctx, device, sl->stream) != VI_OK) {
            if (sl->stream) cudaStreamDestroy(sl->stream);
            delete sl;
            for (Slot* o : s->slots) {
                vi_destroy(o->ctx);
                cudaStreamDestroy(o->stream);
                delete o;
            }
            cudaMemPoolDestroy(s->pool);
            delete s;
            return VI_ECUDA;
        }
        sl->ctx->pool = s->pool;
        // Slots render concurrently: blocks of 256 threads let the marches of
        // several slots share SMs (one 1024-thread block needs a whole SM's
        // registers; with them the 8-slot capacity fell by about 15 %).
        sl->ctx->march_block = 256;
        s->slots.push_back(sl);
    }
    // With a budget, reserve it in the pool up front (allocated once, freed at
    // once, kept by the pool): later allocations carve from memory the pool
    // already holds instead of mapping more while requests are served.
    if (s->budget) {
        void* block = nullptr;
        cudaStream_t st = s->slots[0]->stream;
        if (cudaMallocFromPoolAsync(&block, s->budget, s->pool, st) == cudaSuccess) {
            cudaFreeAsync(block, st);
            cudaStreamSynchronize(st);
        }
        cudaGetLastError();  // a budget the device cannot hold is reserved on demand instead
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return VI_OK;
}

int vi_server_destroy(vi_server* s) {
    if (!s) return VI_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request* r : s->queue) finish(s, r, VI_REQ_CANCELLED, VI_OK);
        s->queue.clear();
    }
    s->wake.notify_all();
    s->worker.join();
    cudaSetDevice(s->device);
    // The completion callbacks touch the server: let every one of them return.
    for (Slot* sl : s->slots) cudaStreamSynchronize(sl->stream);
    if (s->batch_stream) {
        cudaStreamSynchronize(s->batch_stream);
        cudaStreamDestroy(s->batch_stream);
    }
    for (Slot* sl : s->slots) {
        if (sl->batch_status) cudaFreeHost(sl->batch_status);
        for (cudaGraphExec_t x : sl->exec)
            if (x) cudaGraphExecDestroy(x);
        vi_destroy(sl->ctx);
        cudaStreamDestroy(sl->stream);
        delete sl;
    }
    for (ServerVolume* v : s->vols) {
        vi_detail::volume_release(&v->res, &v->used, nullptr);
        cudaEventDestroy(v->ready);
        delete v;
    }
    cudaDeviceSynchronize();
    cudaMemPoolDestroy(s->pool);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
    return VI_OK;
}

int vi_server_add_volume(vi_server* s, const void* host_data, int dtype, int nx, int ny, int nz,
                         int* volume_id) {
    if (!s || !host_data || !volume_id) return VI_EINVAL;
    if (dtype != VI_U8 && dtype != VI_U16) return VI_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 65536 || ny > 65536 || nz > 65536) return VI_EINVAL;
    if (s->budget && vi_detail::volume_bytes(dtype, nx, ny, nz) > s->budget) return VI_ENOMEM;
    std::lock_guard<std::mutex> lk(s->mu);
    ServerVolume* v = new (std::nothrow) ServerVolume();
    if (!v) return VI_ENOMEM;
    if (cudaSetDevice(s->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&v->ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete v;
        return VI_ECUDA;
    }
    v->host = host_data;
    v->dtype = dtype;
    v->nx = nx;
    v->ny = ny;
    v->nz = nz;
    v->res.pool = s->pool;
    *volume_id = (int)s->vols.size();
    s->vols.push_back(v);
    return VI_OK;
}

int vi_server_submit(vi_server* s, const vi_request* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return VI_EINVAL;
    // Malformed requests are refused here; the ones that pass can still fail
    // later (memory, CUDA), which the ticket's result reports.
    if (!q->tf_rgba || q->tf_entries < 2 || q->tf_entries > 8192) return VI_EINVAL;
    if (!std::isfinite(q->tf_vmin) || !std::isfinite(q->tf_vmax) || !(q->tf_vmax > q->tf_vmin))
        return VI_EINVAL;
    for (int e = 0; e < 4 * q->tf_entries; ++e)
        if (!std::isfinite(q->tf_rgba[e])) return VI_EINVAL;
    for (int e = 0; e < q->tf_entries; ++e)
        if (!(q->tf_rgba[4 * e + 3] >= 0.0f && q->tf_rgba[4 * e + 3] <= 1.0f)) return VI_EINVAL;
    if (!finite3(q->light_dir) || !finite3(q->light_color)) return VI_EINVAL;
    if (q->light_dir[0] == 0.0f && q->light_dir[1] == 0.0f && q->light_dir[2] == 0.0f)
        return VI_EINVAL;
    if (q->n_slices < 1 || q->slice_res < 1 || q->mode < VI_NONE || q->mode > VI_CONE)
        return VI_EINVAL;
    if (q->build.format < VI_F32 || q->build.format > VI_UNORM16) return VI_EINVAL;
    if (q->build.quantity != VI_TRANSMITTANCE && q->build.quantity != VI_OPTICAL_DEPTH)
        return VI_EINVAL;
    if (q->build.quantity == VI_OPTICAL_DEPTH && q->build.format == VI_UNORM16) return VI_EINVAL;
    if (q->build.shell_count < 0 || q->build.shell_count > VI_MAX_SHELLS) return VI_EINVAL;
    if (q->render.slice_filter != VI_SLICE_NEAREST && q->render.slice_filter != VI_SLICE_LINEAR)
        return VI_EINVAL;
    if (q->width < 0 || q->height < 0 || (q->width * (long long)q->height > 0 && !q->out_rgba))
        return VI_EINVAL;
    if (q->out_on_device != VI_OUT_HOST && q->out_on_device != VI_OUT_DEVICE) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->volume_id < 0 || q->volume_id >= (int)s->vols.size()) return VI_EINVAL;
    if (s->stop) return VI_ESTATE;
    Request* r = new (std::nothrow) Request();
    if (!r) return VI_ENOMEM;
    r->req = *q;
    r->tf.assign(q->tf_rgba, q->tf_rgba + 4 * q->tf_entries);
    r->req.tf_rgba = r->tf.data();
    r->ticket = s->next_ticket++;
    r->t_submit = now_ms(s);
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    ++s->stats.submitted;
    *ticket = r->ticket;
    s->wake.notify_one();
    return VI_OK;
}

int vi_server_wait(vi_server* s, uint64_t ticket, double timeout_ms, int* status, int* result) {
    if (!s || !(timeout_ms >= 0.0)) return VI_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VI_EINVAL;
    Request* r = it->second;
    auto finished = [r] { return r->status >= VI_REQ_DONE; };
    const auto limit = std::chrono::duration<double, std::milli>(std::min(timeout_ms, 1e9));
    const bool ok = s->done.wait_for(lk, limit, finished);
    if (status) *status = r->status;
    if (result) *result = r->result;
    return ok ? VI_OK : VI_ETIMEOUT;
}

int vi_server_cancel(vi_server* s, uint64_t ticket) {
    if (!s) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VI_EINVAL;
    Request* r = it->second;
    if (r->status != VI_REQ_QUEUED) return VI_ESTATE;
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == r) {
            s->queue.erase(q);
            break;
        }
    finish(s, r, VI_REQ_CANCELLED, VI_OK);
    return VI_OK;
}

int vi_server_timing(vi_server* s, uint64_t ticket, double* submit_ms, double* start_ms,
                     double* end_ms) {
    if (!s) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VI_EINVAL;
    const Request* r = it->second;
    if (submit_ms) *submit_ms = r->t_submit;
    if (start_ms) *start_ms = r->t_start;
    if (end_ms) *end_ms = r->t_end;
    return VI_OK;
}

int vi_server_release(vi_server* s, uint64_t ticket) {
    if (!s) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return VI_EINVAL;
    if (it->second->status < VI_REQ_DONE) return VI_ESTATE;
    delete it->second;
    s->reqs.erase(it);
    return VI_OK;
}

int vi_server_set_batching(vi_server* s, int enabled, double wait_ms) {
    if (!s || !(wait_ms >= 0.0 && wait_ms <= 1e7)) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (enabled && !s->batch_stream) {
        if (cudaSetDevice(s->device) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s->batch_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s->batch_stream = nullptr;
            return VI_ECUDA;
        }
        for (Slot* sl : s->slots)
            if (!sl->batch_status &&
                cudaHostAlloc(reinterpret_cast<void**>(&sl->batch_status), sizeof(int),
                              cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                sl->batch_status = nullptr;
                return VI_ECUDA;
            }
    }
    s->batching = enabled != 0;
    s->batch_wait_ms = wait_ms;
    return VI_OK;
}

int vi_server_set_eviction(vi_server* s, int policy) {
    if (!s || (policy != VI_EVICT_LRU && policy != VI_EVICT_COST)) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->eviction = policy;
    return VI_OK;
}

int vi_server_set_graphs(vi_server* s, int enabled) {
    if (!s) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->graphs = enabled != 0;
    return VI_OK;
}

int vi_server_get_stats(vi_server* s, vi_server_stats* out) {
    if (!s || !out) return VI_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int)s->queue.size();
    out->running = 0;
    for (const Slot* sl : s->slots) out->running += sl->req != nullptr;
    out->resident_volumes = 0;
    for (const ServerVolume* v : s->vols) out->resident_volumes += v->resident;
    out->bytes_in_use = bytes_in_use(s);
    return VI_OK;
}

}  // extern "C"
