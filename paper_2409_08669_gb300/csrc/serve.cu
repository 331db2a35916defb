// Serving: continuous batching of render requests over resident scenes.
//
// A scheduler thread owns `max_slots` execution slots, each a frame workspace,
// in groups of `max_batch` slots.  A group renders one batch at a time: up to
// max_batch requests on the same scene, as one batched frame -- one
// Preprocess launch for all of its cameras (the scene is read once), each
// camera's depth sort, scan and tile sort on its own stream, and one Render
// launch per depth slice for all of them -- so different groups' batches run
// concurrently on the GPU.  Requests wait in a FIFO queue; whenever a group
// is free, the head is admitted together with later queued requests on the
// same scene, while the predicted device memory of everything in flight (pair
// buffers sized by each request's predicted Gaussian-tile pair count, plus
// per-Gaussian and per-pixel buffers) stays within the budget.  So a request
// arriving while others run starts as soon as a group and memory free up, and
// concurrent requests on one scene share launches.  Each (group, scene, batch
// size, resolutions) frame is captured once as a CUDA graph and replayed after
// one-thread kernels write the requests' cameras into the slots' device
// copies that the graph's kernels read.  With max_batch = 1 every slot is a
// group of one (frames of different requests overlap but never share a
// launch).  The predicted pair count per pixel is learned per scene from
// completed frames (running maximum over recent frames, plus a margin).
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>
#include <algorithm>

#include "adr_internal.cuh"

using namespace adr;

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Scene {
    const float *means, *scales, *rots, *opac, *sh;
    int64_t n;
    SetDev st;
    double pairs_per_pixel = -1.0;   // learned; < 0 = unknown
};

enum ReqState { kQueued, kRunning, kDone };

struct Request {
    uint64_t ticket = 0;
    int scene = 0;
    CamDev cam{};
    float* out = nullptr;
    double t_submit = 0, t_done = 0;
    int64_t pred_pairs = 0;
    size_t pred_bytes = 0;
    ReqState state = kQueued;
    adr_status result = ADR_OK;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
};

struct Slot {
    Workspace ws;
    FrameState fs;
    std::atomic<uint32_t> calls{0};
    cudaStream_t stream = nullptr;     // this camera's sort stages within a batch
    float* img = nullptr;              // slot-owned image the graph renders into
    uint32_t* host_words = nullptr;    // pinned: status word, pair count
};

// max_batch slots that render one batch at a time.
struct Group {
    std::vector<Slot*> slots;
    cudaStream_t stream = nullptr;     // the batch's launches
    cudaEvent_t done = nullptr;
    BatchStreams bs{};
    std::vector<Request*> reqs;        // the batch in flight (empty: free)
    // key: scene, batch size, then width and height of each camera
    std::map<std::vector<int>, GraphEntry> graphs;
};

}  // namespace

struct adr_server {
    adr_serve_config cfg{};
    std::vector<Scene> scenes;
    std::vector<Slot*> slots;
    std::vector<Group*> groups;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> requests;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t inflight_bytes = 0;
    int inflight = 0;
    // statistics
    std::vector<double> latencies;
    int max_inflight = 0;
    int64_t admitted_while_busy = 0, rejected = 0, capacity_errors = 0, graph_replays = 0;
    int64_t batches = 0, batched_frames = 0, largest_batch = 0;
    double t_first_submit = -1, t_last_done = 0;
    char error[256] = "";   // why the last failed launch failed
};

namespace {

size_t predicted_bytes(const adr_server* s, const Scene& sc, const CamDev& cam, int64_t* pairs_out) {
    const int64_t pixels = (int64_t)cam.width * cam.height;
    int64_t pairs;
    if (sc.pairs_per_pixel < 0) {
        pairs = s->cfg.slot_pair_capacity;                       // unknown scene: reserve a full slot
    } else {
        pairs = (int64_t)(sc.pairs_per_pixel * (double)pixels * 1.25) + 4096;
        pairs = std::min<int64_t>(pairs, s->cfg.slot_pair_capacity);
    }
    *pairs_out = pairs;
    return (size_t)pairs * 12 + (size_t)sc.n * 150 + (size_t)pixels * 32;
}

// Records why a launch failed (read by adr_serve_poll) and returns ADR_ERR_CUDA.
adr_status launch_failed(adr_server* s, const char* step, cudaError_t e) {
    snprintf(s->error, sizeof(s->error), "%s: %s", step, cudaGetErrorString(e));
    return ADR_ERR_CUDA;
}

#define SERVE_CUDA(step, call)                                  \
    do {                                                        \
        const cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return launch_failed(s, step, e_); \
    } while (0)

// The batch's cameras as pipeline items: slot b renders request b into its
// own image.
int batch_items(Group& g, std::vector<BatchItem>& items) {
    const int k = (int)g.reqs.size();
    items.resize(k);
    for (int b = 0; b < k; ++b) {
        Slot& sl = *g.slots[b];
        items[b] = BatchItem{&sl.ws, &sl.fs, &sl.calls, sl.img, nullptr, nullptr};
    }
    return k;
}

// Captures the batch's frame into a graph.  The graph reads the cameras and
// settings from the slots' device copies, which kernels launched before each
// replay write.
adr_status capture_batch(adr_server* s, Group& g, const Scene& sc, GraphEntry& ge) {
    cudaStream_t strm = g.stream;
    std::vector<BatchItem> items;
    const int k = batch_items(g, items);
    cudaGraph_t graph = nullptr;
    SERVE_CUDA("cudaStreamBeginCapture", cudaStreamBeginCapture(strm, cudaStreamCaptureModeThreadLocal));
    enqueue_frame_batch(items.data(), k, sc.means, sc.scales, sc.rots, sc.opac, sc.sh, strm, &g.bs,
                        /*set_params=*/false);
    const cudaError_t ec = cudaStreamEndCapture(strm, &graph);
    if (ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return launch_failed(s, "cudaStreamEndCapture", ec != cudaSuccess ? ec : cudaErrorUnknown);
    }
    const cudaError_t e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return launch_failed(s, "cudaGraphInstantiate", e);
    return ADR_OK;
}

adr_status run_batch(adr_server* s, Group& g) {
    const Scene& sc = s->scenes[g.reqs[0]->scene];
    const int k = (int)g.reqs.size();
    cudaStream_t strm = g.stream;
    for (int b = 0; b < k; ++b) {
        Slot& sl = *g.slots[b];
        fill_frame_state(sl.fs, sc.n, g.reqs[b]->cam, sc.st);
        SERVE_CUDA("clearing the status word", cudaMemsetAsync(sl.ws.status, 0, 16, strm));
    }
    if (s->cfg.use_graphs) {
        std::vector<int> key{g.reqs[0]->scene, k};
        for (int b = 0; b < k; ++b) {
            key.push_back(g.reqs[b]->cam.width);
            key.push_back(g.reqs[b]->cam.height);
        }
        auto it = g.graphs.find(key);
        if (it == g.graphs.end()) {
            GraphEntry ge;
            const adr_status st = capture_batch(s, g, sc, ge);
            if (st != ADR_OK) return st;
            it = g.graphs.emplace(key, ge).first;
        } else {
            for (int b = 0; b < k; ++b)   // the replay's preprocess stages
                count_stage(g.slots[b]->calls, g.slots[b]->ws, strm);
        }
        for (int b = 0; b < k; ++b)
            launch_set_frame_params(FrameParams{g.reqs[b]->cam, sc.st}, g.slots[b]->ws.d_fp, strm);
        SERVE_CUDA("camera launch", cudaGetLastError());
        SERVE_CUDA("cudaGraphLaunch", cudaGraphLaunch(it->second.exec, strm));
        s->graph_replays++;
    } else {
        std::vector<BatchItem> items;
        batch_items(g, items);
        enqueue_frame_batch(items.data(), k, sc.means, sc.scales, sc.rots, sc.opac, sc.sh, strm,
                            &g.bs, /*set_params=*/true);
        SERVE_CUDA("frame launch", cudaGetLastError());
    }
    for (int b = 0; b < k; ++b) {
        Slot& sl = *g.slots[b];
        Request& r = *g.reqs[b];
        const size_t img_bytes = (size_t)3 * r.cam.width * r.cam.height * sizeof(float);
        SERVE_CUDA("image copy", cudaMemcpyAsync(r.out, sl.img, img_bytes, cudaMemcpyDeviceToDevice, strm));
        SERVE_CUDA("status read", cudaMemcpyAsync(sl.host_words, sl.ws.status, 4,
                                                  cudaMemcpyDeviceToHost, strm));
        SERVE_CUDA("pair count read", cudaMemcpyAsync(sl.host_words + 1, sl.ws.counters + kCntPairs,
                                                      4, cudaMemcpyDeviceToHost, strm));
    }
    SERVE_CUDA("cudaEventRecord", cudaEventRecord(g.done, strm));
    s->batches++;
    s->batched_frames += k;
    s->largest_batch = std::max<int64_t>(s->largest_batch, k);
    return ADR_OK;
}

#undef SERVE_CUDA

void finish_request(adr_server* s, Request* r, uint32_t bits, uint32_t pairs, cudaError_t q) {
    r->t_done = now_ms();
    if (q != cudaSuccess) {
        r->result = ADR_ERR_CUDA;
        snprintf(s->error, sizeof(s->error), "frame: %s", cudaGetErrorString(q));
    } else {
        const StatusReport rep = status_from_bits(bits, (int64_t)pairs, s->cfg.slot_pair_capacity);
        r->result = rep.status;
        if (rep.status == ADR_ERR_CAPACITY) s->capacity_errors++;
        if (rep.status == ADR_ERR_CUDA) snprintf(s->error, sizeof(s->error), "%s", rep.message);
    }
    Scene& sc = s->scenes[r->scene];
    if (q == cudaSuccess && !(bits & kErrLookback)) {   // a skipped frame's pair count is not a measurement
        const double ppp = (double)pairs / ((double)r->cam.width * r->cam.height);
        sc.pairs_per_pixel = sc.pairs_per_pixel < 0 ? ppp
                                                    : std::max(ppp, 0.9 * sc.pairs_per_pixel + 0.1 * ppp);
    }
    r->state = kDone;
    s->latencies.push_back(r->t_done - r->t_submit);
    s->t_last_done = r->t_done;
    s->inflight_bytes -= r->pred_bytes;
    s->inflight--;
}

void scheduler(adr_server* s) {
    cudaSetDevice(s->cfg.device);
    std::unique_lock<std::mutex> lk(s->mu);
    const size_t B = (size_t)s->cfg.max_batch;
    while (!s->stop) {
        bool progressed = false;
        // Completions.
        for (Group* g : s->groups) {
            if (g->reqs.empty()) continue;
            const cudaError_t q = cudaEventQuery(g->done);
            if (q == cudaErrorNotReady) continue;
            for (size_t b = 0; b < g->reqs.size(); ++b)
                finish_request(s, g->reqs[b], g->slots[b]->host_words[0], g->slots[b]->host_words[1], q);
            g->reqs.clear();
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // Admissions: the FIFO head, plus (with batching) later queued
        // requests on the same scene, while a group is free and the memory
        // budget allows.
        while (!s->queue.empty()) {
            Group* free_group = nullptr;
            for (Group* g : s->groups)
                if (g->reqs.empty()) { free_group = g; break; }
            if (!free_group) break;
            auto fits = [&](Request* r) {
                r->pred_bytes = predicted_bytes(s, s->scenes[r->scene], r->cam, &r->pred_pairs);
                return s->inflight == 0 || s->inflight_bytes + r->pred_bytes <= (size_t)s->cfg.mem_budget_bytes;
            };
            auto admit = [&](Request* r) {
                if (s->inflight > 0) s->admitted_while_busy++;
                r->state = kRunning;
                free_group->reqs.push_back(r);
                s->inflight++;
                s->inflight_bytes += r->pred_bytes;
                s->max_inflight = std::max(s->max_inflight, s->inflight);
            };
            Request* head = s->queue.front();
            if (!fits(head)) break;                              // wait for memory to free up
            s->queue.pop_front();
            admit(head);
            for (auto it = s->queue.begin(); it != s->queue.end() && free_group->reqs.size() < B;) {
                if ((*it)->scene == head->scene && fits(*it)) {
                    admit(*it);
                    it = s->queue.erase(it);
                } else {
                    ++it;
                }
            }
            // cameras in a canonical order, so graphs are shared by equal batches
            std::stable_sort(free_group->reqs.begin(), free_group->reqs.end(), [](const Request* a, const Request* b) {
                return a->cam.width != b->cam.width ? a->cam.width < b->cam.width : a->cam.height < b->cam.height;
            });
            const adr_status st = run_batch(s, *free_group);
            if (st != ADR_OK) {   // launch failed: report and free the group
                for (Request* r : free_group->reqs) {
                    r->result = st;
                    r->state = kDone;
                    r->t_done = now_ms();
                    s->inflight--;
                    s->inflight_bytes -= r->pred_bytes;
                }
                free_group->reqs.clear();
                s->cv_done.notify_all();
            }
            progressed = true;
        }
        if (!progressed) {
            if (s->inflight == 0 && s->queue.empty())
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
}

void destroy_server(adr_server* s) {
    for (Group* g : s->groups) {
        if (g->stream) cudaStreamSynchronize(g->stream);
        for (auto& kv : g->graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (g->done) cudaEventDestroy(g->done);
        if (g->bs.fork) cudaEventDestroy(g->bs.fork);
        for (int b = 0; b < kMaxBatch; ++b)
            if (g->bs.join[b]) cudaEventDestroy(g->bs.join[b]);
        if (g->stream) cudaStreamDestroy(g->stream);
        delete g;
    }
    for (Slot* sl : s->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        free_workspace(sl->ws);
        if (sl->img) cudaFree(sl->img);
        if (sl->host_words) cudaFreeHost(sl->host_words);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
    }
    for (auto& kv : s->requests) delete kv.second;
    delete s;
}

}  // namespace

extern "C" {

adr_status adr_serve_create(adr_server** out, const adr_serve_config* cfg) {
    if (!out || !cfg) return report_error(ADR_ERR_INVALID, "adr_serve_create: NULL argument");
    *out = nullptr;
    if (cfg->max_slots < 1 || cfg->max_slots > 64 || cfg->max_batch < 1 ||
        cfg->max_batch > kMaxBatch || cfg->max_slots % cfg->max_batch != 0 ||
        cfg->slot_pair_capacity <= 0 ||
        cfg->slot_pair_capacity > (int64_t(1) << 30) || cfg->slot_max_gaussians <= 0 ||
        cfg->slot_max_gaussians > kMaxGaussians ||
        cfg->max_width <= 0 || cfg->max_height <= 0 || cfg->max_width > 4096 ||
        cfg->max_height > 4096 || cfg->mem_budget_bytes <= 0)
        return report_error(ADR_ERR_INVALID, "adr_serve_create: configuration out of range");
    if (cudaSetDevice(cfg->device) != cudaSuccess)
        return report_error(ADR_ERR_INVALID, "adr_serve_create: device not present");
    adr_server* s = new adr_server();
    s->cfg = *cfg;
    for (int i = 0; i < cfg->max_slots; ++i) {
        Slot* sl = new Slot();
        s->slots.push_back(sl);
        adr_status st = alloc_workspace(sl->ws, cfg->slot_max_gaussians, cfg->slot_pair_capacity,
                                        cfg->max_width, cfg->max_height, cfg->device);
        if (st != ADR_OK ||
            cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc((void**)&sl->img, (size_t)3 * cfg->max_width * cfg->max_height * sizeof(float)) != cudaSuccess ||
            cudaHostAlloc((void**)&sl->host_words, 16, cudaHostAllocDefault) != cudaSuccess) {
            (void)cudaGetLastError();   // an allocation error is not sticky: clear it
            destroy_server(s);
            return report_error(ADR_ERR_CUDA, "adr_serve_create: slot allocation failed");
        }
    }
    for (int gi = 0; gi < cfg->max_slots / cfg->max_batch; ++gi) {
        Group* g = new Group();
        s->groups.push_back(g);
        bool ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&g->bs.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int b = 0; b < cfg->max_batch; ++b) {
            Slot* sl = s->slots[gi * cfg->max_batch + b];
            g->slots.push_back(sl);
            g->bs.side[b] = sl->stream;
            ok = ok && cudaEventCreateWithFlags(&g->bs.join[b], cudaEventDisableTiming) == cudaSuccess;
        }
        if (!ok) {
            (void)cudaGetLastError();
            destroy_server(s);
            return report_error(ADR_ERR_CUDA, "adr_serve_create: group allocation failed");
        }
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return report_ok();
}

void adr_serve_destroy(adr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy_server(s);
}

adr_status adr_serve_add_scene(adr_server* s, const float* means, const float* scales,
                               const float* rots, const float* opac, const float* sh, int64_t n,
                               const adr_settings* settings, int32_t* scene_id) {
    if (!s || !scene_id) return report_error(ADR_ERR_INVALID, "adr_serve_add_scene: NULL argument");
    if (n <= 0 || n > s->cfg.slot_max_gaussians)
        return report_error(ADR_ERR_INVALID, "adr_serve_add_scene: n outside 1..slot_max_gaussians");
    if (!means || !scales || !rots || !opac || !sh || (uintptr_t)rots % 16 || (uintptr_t)sh % 16)
        return report_error(ADR_ERR_INVALID, "adr_serve_add_scene: bad parameter pointer");
    SetDev st;
    adr_status r = settings_to_dev(settings, st);
    if (r != ADR_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    Scene sc{means, scales, rots, opac, sh, n, st, -1.0};
    s->scenes.push_back(sc);
    *scene_id = (int32_t)s->scenes.size() - 1;
    return report_ok();
}

adr_status adr_serve_submit(adr_server* s, int32_t scene_id, const adr_camera* camera,
                            float* out_img, uint64_t* ticket) {
    if (!s || !ticket || !out_img) return report_error(ADR_ERR_INVALID, "adr_serve_submit: NULL argument");
    CamDev cam;
    adr_status r = camera_to_dev(camera, s->cfg.max_width, s->cfg.max_height, cam);
    if (r != ADR_OK) return r;
    std::lock_guard<std::mutex> lk(s->mu);
    if (scene_id < 0 || scene_id >= (int32_t)s->scenes.size())
        return report_error(ADR_ERR_INVALID, "adr_serve_submit: unknown scene");
    const Scene& sc = s->scenes[scene_id];
    const int64_t min_bytes = (int64_t)sc.n * 150 + (int64_t)cam.width * cam.height * 32 + 4096 * 12;
    if (min_bytes > s->cfg.mem_budget_bytes) {
        s->rejected++;
        return report_error(ADR_ERR_ADMISSION, "adr_serve_submit: request can never fit the memory budget");
    }
    Request* q = new Request();
    q->ticket = s->next_ticket++;
    q->scene = scene_id;
    q->cam = cam;
    q->out = out_img;
    q->t_submit = now_ms();
    if (s->t_first_submit < 0) s->t_first_submit = q->t_submit;
    s->requests[q->ticket] = q;
    s->queue.push_back(q);
    *ticket = q->ticket;
    s->cv_work.notify_all();
    return report_ok();
}

adr_status adr_serve_poll(adr_server* s, uint64_t ticket, int64_t timeout_us) {
    if (!s) return report_error(ADR_ERR_INVALID, "adr_serve_poll: NULL server");
    if (timeout_us < 0) return report_error(ADR_ERR_INVALID, "adr_serve_poll: negative timeout");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return report_error(ADR_ERR_INVALID, "adr_serve_poll: unknown ticket");
    Request* r = it->second;
    if (r->state != kDone && timeout_us != 0) {
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
        s->cv_done.wait_until(lk, deadline, [&] { return r->state == kDone; });
    }
    if (r->state != kDone) {
        if (timeout_us == 0) return ADR_PENDING;
        return report_error(ADR_ERR_TIMEOUT, "adr_serve_poll: request not finished before the timeout");
    }
    const adr_status res = r->result;
    s->requests.erase(it);
    delete r;
    if (res == ADR_ERR_CUDA) {
        char msg[320];
        snprintf(msg, sizeof(msg), "adr_serve_poll: the request failed (%s)", s->error);
        return report_error(res, msg);
    }
    if (res == ADR_ERR_TIMEOUT)
        return report_error(res, "adr_serve_poll: a device-side lookback wait gave up; the "
                                 "request's frame was skipped (ticket released)");
    if (res != ADR_OK) return report_error(res, "adr_serve_poll: the request failed on the device");
    return report_ok();
}

adr_status adr_serve_stats(adr_server* s, double* out, int32_t n) {
    if (!s || !out || n < 1) return report_error(ADR_ERR_INVALID, "adr_serve_stats: bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> lat = s->latencies;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        const size_t k = std::min(lat.size() - 1, (size_t)(p * (double)(lat.size() - 1) + 0.5));
        return lat[k];
    };
    double mean = 0;
    for (double v : lat) mean += v;
    mean = lat.empty() ? 0.0 : mean / (double)lat.size();
    const double span = s->t_last_done - s->t_first_submit;
    const double vals[13] = {(double)lat.size(), pct(0.5), pct(0.99), mean,
                             (double)s->max_inflight, (double)s->admitted_while_busy,
                             (double)s->rejected, span > 0 ? 1e3 * (double)lat.size() / span : 0.0,
                             (double)s->capacity_errors, (double)s->graph_replays,
                             (double)s->batches, (double)s->largest_batch,
                             s->batches ? (double)s->batched_frames / (double)s->batches : 0.0};
    for (int i = 0; i < n && i < 13; ++i) out[i] = vals[i];
    return report_ok();
}

adr_status adr_serve_reset_stats(adr_server* s) {
    if (!s) return report_error(ADR_ERR_INVALID, "adr_serve_reset_stats: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->latencies.clear();
    s->max_inflight = s->inflight;
    s->admitted_while_busy = s->rejected = s->capacity_errors = s->graph_replays = 0;
    s->batches = s->batched_frames = s->largest_batch = 0;
    s->t_first_submit = -1;
    s->t_last_done = 0;
    return report_ok();
}

}  // extern "C"
