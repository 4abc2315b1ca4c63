// Serving runtime behind the C ABI (dmas_server_*): a native thread admits
// frames against a device-memory budget, batches them per lane and launches
// them through dmas_beamform_batch_upload, so the path from a frame's arrival
// to its launch involves no interpreter lock and no thread hand-off beyond
// the submit call.  Built on the public ABI only (dmas.h).
//
// Lanes: the fast lane (frames with N*M*T <= fast_cost) runs batches of up to
// max_batch frames on fast_streams high-priority streams, one batch in flight
// per stream; the bulk lane runs one frame per batch on one low-priority
// stream with up to bulk_depth batches queued on it, so big frames execute
// first in, first out while the fast lane's kernels overtake them on the SMs.
//
// One thread does everything: it reaps finished batches (event queries),
// admits and launches what fits, and while batches are in flight waits at
// most kPollUs microseconds on its condition variable (a submit wakes it at
// once).  Device memory for a batch's frames and scratch comes from a pool of
// the server's own (cudaMallocFromPoolAsync / cudaFreeAsync on the lane's
// stream), so neither allocation nor release synchronises the device.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dmas.h"

namespace {

constexpr int kPollUs = 20;
constexpr int kMaxBatch = 64;
constexpr size_t kCopyPiece = (size_t)32 << 20;

double now_s() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Sensor {
    dmas_plan *plan;
    size_t frame_bytes, image_bytes, dev_bytes;
    bool fast;
};

struct Req {
    uint64_t ticket;
    int sensor;
    const float *h_frame;
    float *h_image;
    int keep;                  // hand the device image over in the completion
    float *d_image;            // allocated at launch
    double t_arrival, t_admitted;
};

// Images come from one pool per device that lives as long as the process, so
// an image handed over may outlive the server; freed memory stays in the pool.
cudaMemPool_t image_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&pools[device], &props) != cudaSuccess) {
            cudaGetLastError();
            pools[device] = nullptr;
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return pools[device];
}

struct Lane {
    std::vector<cudaStream_t> streams;
    int depth = 1;
    int max_batch = 1;
    std::deque<Req> queue;
    int in_flight = 0;
    int next = 0;
};

struct Batch {
    std::vector<Req> reqs;
    cudaEvent_t ev = nullptr;
    void *mem = nullptr;
    size_t reserved = 0;
    int lane = 0;
    cudaStream_t stream = nullptr;
};

}  // namespace

struct dmas_server {
    int device = 0;
    std::vector<Sensor> sensors;
    Lane lanes[2];  // 0: fast, 1: bulk
    size_t budget = 0, reserved = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<dmas_server_done> done;
    std::vector<Batch> inflight;
    std::vector<cudaEvent_t> events;  // free for reuse
    uint64_t next_ticket = 1;
    int pending = 0;  // queued or in flight
    bool closing = false;
    std::thread thread;

    void loop();
    void reap();
    bool launch(Batch &b);
    void finish(const Req &r, int status, int batch_size, double t);
};

// Completion record (lock held).
void dmas_server::finish(const Req &r, int status, int batch_size, double t) {
    dmas_server_done d;
    d.ticket = r.ticket;
    d.sensor = r.sensor;
    d.status = status;
    d.batch_size = batch_size;
    d.t_arrival = r.t_arrival;
    d.t_admitted = r.t_admitted;
    d.t_done = t;
    d.d_image = status == DMAS_OK && r.keep ? r.d_image : nullptr;
    done.push_back(d);
    --pending;
}

// Batches whose completion event has fired: record their frames' completion
// and release their memory and budget.
void dmas_server::reap() {
    std::lock_guard<std::mutex> lock(mu);
    bool any = false;
    for (size_t i = 0; i < inflight.size();) {
        Batch &b = inflight[i];
        const cudaError_t q = cudaEventQuery(b.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = now_s();
        const int status = q == cudaSuccess ? DMAS_OK : DMAS_ECUDA;
        if (q != cudaSuccess) cudaGetLastError();
        for (const Req &r : b.reqs) {
            if (status != DMAS_OK && r.keep && r.d_image) cudaFreeAsync(r.d_image, b.stream);
            finish(r, status, (int)b.reqs.size(), t);
        }
        cudaFreeAsync(b.mem, b.stream);
        events.push_back(b.ev);
        reserved -= b.reserved;
        lanes[b.lane].in_flight -= 1;
        inflight[i] = std::move(inflight.back());
        inflight.pop_back();
        any = true;
    }
    if (any) cv_done.notify_all();
}

// Enqueue one batch on its stream: frames and scratch from the pool, the
// uploads and the batch in one call, the optional copies to the host, the
// completion event.  false: nothing was enqueued (the caller completes the
// frames with an error).
bool dmas_server::launch(Batch &b) {
    const int n = (int)b.reqs.size();
    dmas_plan *plans[kMaxBatch];
    const float *h_frames[kMaxBatch];
    float *d_frames[kMaxBatch], *d_images[kMaxBatch];
    size_t off[kMaxBatch], frames_total = 0;
    for (int k = 0; k < n; ++k) {
        const Sensor &s = sensors[b.reqs[k].sensor];
        plans[k] = s.plan;
        h_frames[k] = b.reqs[k].h_frame;
        off[k] = frames_total;
        frames_total += round256(s.frame_bytes);
    }
    // the images, then the frames and scratch in one block
    cudaMemPool_t ipool = image_pool(device);
    int made = 0;
    bool ok = ipool != nullptr;
    for (; ok && made < n; ++made) {
        void *img = nullptr;
        ok = cudaMallocFromPoolAsync(&img, sensors[b.reqs[made].sensor].image_bytes, ipool,
                                     b.stream) == cudaSuccess;
        if (ok) b.reqs[made].d_image = d_images[made] = (float *)img;
        else --made;
    }
    const size_t ws = dmas_batch_workspace_bytes(n, plans);
    if (ok) ok = cudaMallocFromPoolAsync(&b.mem, frames_total + ws, pool, b.stream) == cudaSuccess;
    if (ok) {
        char *base = (char *)b.mem;
        for (int k = 0; k < n; ++k) d_frames[k] = (float *)(base + off[k]);
        ok = dmas_beamform_batch_upload(n, plans, h_frames, d_frames, d_images,
                                        base + frames_total, ws, b.stream, nullptr) == DMAS_OK;
    }
    if (ok && events.empty()) {
        cudaEvent_t e;
        ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (ok) events.push_back(e);
    }
    if (!ok) {
        cudaGetLastError();
        for (int k = 0; k < made; ++k) {
            cudaFreeAsync(b.reqs[k].d_image, b.stream);
            b.reqs[k].d_image = nullptr;
        }
        if (b.mem) cudaFreeAsync(b.mem, b.stream);
        b.mem = nullptr;
        return false;
    }
    // copies to the host in pieces of kCopyPiece bytes, so other streams'
    // copies interleave with a big image's; images not handed over are freed
    // after them
    for (int k = 0; k < n; ++k) {
        const Req &r = b.reqs[k];
        if (r.h_image) {
            const size_t bytes = sensors[r.sensor].image_bytes;
            for (size_t o = 0; o < bytes; o += kCopyPiece)
                cudaMemcpyAsync((char *)r.h_image + o, (const char *)r.d_image + o,
                                std::min(kCopyPiece, bytes - o), cudaMemcpyDeviceToHost,
                                b.stream);
        }
        if (!r.keep) cudaFreeAsync(r.d_image, b.stream);
    }
    b.ev = events.back();
    events.pop_back();
    cudaEventRecord(b.ev, b.stream);
    return true;
}

void dmas_server::loop() {
    cudaSetDevice(device);
    for (;;) {
        reap();
        Batch b;
        {
            std::unique_lock<std::mutex> lock(mu);
            int li = -1;
            for (int l = 0; l < 2 && li < 0; ++l) {
                Lane &ln = lanes[l];
                if (ln.queue.empty() || ln.in_flight >= ln.depth) continue;
                const size_t head = sensors[ln.queue.front().sensor].dev_bytes;
                if (head > budget || reserved + head <= budget) li = l;
            }
            if (li < 0) {
                if (closing && pending == 0) return;
                if (inflight.empty())
                    cv_work.wait_for(lock, std::chrono::milliseconds(50));
                else
                    cv_work.wait_for(lock, std::chrono::microseconds(kPollUs));
                continue;
            }
            Lane &ln = lanes[li];
            const double t = now_s();
            while (!ln.queue.empty() && (int)b.reqs.size() < ln.max_batch) {
                Req r = ln.queue.front();
                const size_t need = sensors[r.sensor].dev_bytes;
                if (need > budget) {  // can never fit
                    ln.queue.pop_front();
                    r.t_admitted = t;
                    finish(r, DMAS_ENOMEM, 1, t);
                    cv_done.notify_all();
                    continue;
                }
                if (reserved + need > budget) break;
                ln.queue.pop_front();
                r.t_admitted = t;
                reserved += need;
                b.reserved += need;
                b.reqs.push_back(r);
            }
            if (b.reqs.empty()) continue;
            b.lane = li;
            b.stream = ln.streams[ln.next];
            ln.next = (ln.next + 1) % (int)ln.streams.size();
            ln.in_flight += 1;
        }
        const bool ok = launch(b);
        std::lock_guard<std::mutex> lock(mu);
        if (ok) {
            inflight.push_back(std::move(b));
        } else {
            const double t = now_s();
            for (const Req &r : b.reqs) finish(r, DMAS_ECUDA, (int)b.reqs.size(), t);
            reserved -= b.reserved;
            lanes[b.lane].in_flight -= 1;
            cv_done.notify_all();
        }
    }
}

namespace {

void release_all(dmas_server *s) {
    for (int l = 0; l < 2; ++l)
        for (cudaStream_t st : s->lanes[l].streams)
            if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : s->events) cudaEventDestroy(e);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // namespace

extern "C" {

dmas_status dmas_server_create(const dmas_server_desc *d, dmas_server **out) {
    if (!out) return DMAS_EINVAL;
    *out = nullptr;
    if (!d || d->n_plans < 1 || !d->plans || d->fast_streams < 1 || d->max_batch < 1 ||
        d->max_batch > kMaxBatch || d->bulk_depth < 1 || d->budget_bytes == 0 ||
        !(d->fast_cost >= 0.0))
        return DMAS_EINVAL;
    for (int i = 0; i < d->n_plans; ++i)
        if (!d->plans[i]) return DMAS_EINVAL;
    dmas_server *s = new (std::nothrow) dmas_server;
    if (!s) return DMAS_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return DMAS_ECUDA;
    }
    try {
        for (int i = 0; i < d->n_plans; ++i) {
            dmas_plan_info info;
            if (dmas_plan_get_info(d->plans[i], &info) != DMAS_OK) {
                delete s;
                return DMAS_EINVAL;
            }
            Sensor sn;
            sn.plan = d->plans[i];
            sn.frame_bytes = (size_t)info.n_mics * info.n_samples * sizeof(float);
            sn.image_bytes = (size_t)info.n_dirs * info.n_samples * sizeof(float);
            sn.dev_bytes = sn.frame_bytes + sn.image_bytes + dmas_plan_workspace_bytes(d->plans[i]);
            sn.fast = (double)info.n_mics * info.n_dirs * info.n_samples <= d->fast_cost;
            s->sensors.push_back(sn);
        }
    } catch (const std::bad_alloc &) {
        delete s;
        return DMAS_ENOMEM;
    }
    s->budget = d->budget_bytes;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    s->lanes[0].depth = d->fast_streams;
    s->lanes[0].max_batch = d->max_batch;
    s->lanes[1].depth = d->bulk_depth;
    s->lanes[1].max_batch = 1;
    bool ok = true;
    for (int k = 0; k < d->fast_streams && ok; ++k) {
        cudaStream_t st = nullptr;
        ok = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi) == cudaSuccess;
        s->lanes[0].streams.push_back(st);
    }
    if (ok) {
        cudaStream_t st = nullptr;
        ok = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo) == cudaSuccess;
        s->lanes[1].streams.push_back(st);
    }
    if (ok) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        ok = cudaMemPoolCreate(&s->pool, &props) == cudaSuccess;
        if (ok) {
            // keep freed memory in the pool for the next batches
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (!ok) {
        cudaGetLastError();
        release_all(s);
        return DMAS_ECUDA;
    }
    // grow both pools now (twice every sensor's frame and scratch, and its
    // image, capped at the budget), so the first frames do not wait for the
    // pools to map memory
    {
        size_t frames = 0, images = 0;
        for (const Sensor &sn : s->sensors) {
            frames += round256(sn.frame_bytes) + (sn.dev_bytes - sn.frame_bytes - sn.image_bytes);
            images += round256(sn.image_bytes);
        }
        frames = std::min(2 * frames, s->budget);
        images = std::min(2 * images, s->budget);
        cudaStream_t st = s->lanes[1].streams[0];
        void *a = nullptr, *b = nullptr;
        if (cudaMallocFromPoolAsync(&a, frames, s->pool, st) == cudaSuccess) cudaFreeAsync(a, st);
        cudaMemPool_t ip = image_pool(s->device);
        if (ip && cudaMallocFromPoolAsync(&b, images, ip, st) == cudaSuccess) cudaFreeAsync(b, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
    }
    try {
        s->thread = std::thread([s] { s->loop(); });
    } catch (...) {
        release_all(s);
        return DMAS_ENOMEM;
    }
    *out = s;
    return DMAS_OK;
}

dmas_status dmas_server_submit(dmas_server *s, int sensor, const float *h_frame, float *h_image,
                               int keep_image, double t_arrival, uint64_t *ticket) {
    if (!s || !h_frame || !ticket || sensor < 0 || sensor >= (int)s->sensors.size())
        return DMAS_EINVAL;
    Req r;
    r.sensor = sensor;
    r.h_frame = h_frame;
    r.h_image = h_image;
    r.keep = keep_image != 0;
    r.d_image = nullptr;
    r.t_arrival = t_arrival;
    r.t_admitted = 0.0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->closing) return DMAS_EBUSY;
        r.ticket = s->next_ticket++;
        try {
            s->lanes[s->sensors[sensor].fast ? 0 : 1].queue.push_back(r);
        } catch (const std::bad_alloc &) {
            return DMAS_ENOMEM;
        }
        ++s->pending;
    }
    *ticket = r.ticket;
    s->cv_work.notify_one();
    return DMAS_OK;
}

dmas_status dmas_server_wait(dmas_server *s, double timeout_s, dmas_server_done *out) {
    if (!s || !out || !(timeout_s >= 0.0)) return DMAS_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty())
        s->cv_done.wait_for(lock, std::chrono::duration<double>(std::min(timeout_s, 3600.0)),
                            [s] { return !s->done.empty(); });
    if (s->done.empty()) return DMAS_ETIMEOUT;
    *out = s->done.front();
    s->done.pop_front();
    return DMAS_OK;
}

dmas_status dmas_server_image_free(float *d_image, void *stream) {
    if (!d_image) return DMAS_OK;
    if (cudaFreeAsync(d_image, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return DMAS_ECUDA;
    }
    return DMAS_OK;
}

int dmas_server_pending(dmas_server *s) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lock(s->mu);
    return s->pending;
}

dmas_status dmas_server_destroy(dmas_server *s) {
    if (!s) return DMAS_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->closing = true;
    }
    s->cv_work.notify_all();
    if (s->thread.joinable()) s->thread.join();
    cudaSetDevice(s->device);
    for (int l = 0; l < 2; ++l)
        for (cudaStream_t st : s->lanes[l].streams)
            if (st) cudaStreamSynchronize(st);
    release_all(s);
    return DMAS_OK;
}

}  // extern "C"
