/*
 * Serving form: a continuous-batching request loop on one GPU.
 *
 * Requests are subcube detection jobs of any shape, submitted from host
 * memory at any time.  A request is admitted as soon as a worker slot is free
 * and its device footprint fits the HBM budget: the footprint is that of the
 * context sf_detect_host runs it on (the cube, the mask and one x-filtered
 * scratch cube per distinct non-zero sigma_xy; where rows are not 16-byte
 * multiples, the scratch rows padded and one more scratch cube, the cube's
 * padded copy).  Admitted requests run
 * concurrently, one CUDA stream per worker, so their copies and kernels
 * overlap on the device; a request that arrives while others are on the GPU
 * is admitted as soon as a slot and memory free up (no batch boundary).
 * Contexts are kept per shape after use (their plans, compiled kernels and
 * device buffers stay resident) and counted against the budget; idle ones are
 * destroyed, least recently used first, when an admission needs the room.
 * A request larger than the whole budget completes at once with SF_EBUDGET.
 * A request still waiting for admission can be cancelled (it completes with
 * SF_ECANCELED); one already admitted runs to its end.
 *
 * The paper processes device-sized sections one after another, with copies
 * not overlapped (Sec. 3.1), and names overlapping input with processing as
 * future work (Sec. 6); this loop overlaps whole requests instead.
 */
#include "sf.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int64_t id;
    const void *h_cube;
    int64_t nx, ny, nz;
    uint32_t *h_mask;
    int64_t t_submit;
    int64_t t_done = 0;
    int64_t bytes;
    sf_status status = SF_OK;
};

using Shape = std::tuple<int64_t, int64_t, int64_t>;

struct Idle {
    Shape shape;
    sf_ctx *ctx;
    int64_t bytes;
};

}  // namespace

struct sf_server {
    sf_config proto{};
    std::vector<sf_filter_spec> filters;
    int64_t budget = 0;
    int n_xy = 0;
    size_t ebytes = 4;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::deque<Request *> done;
    std::list<Idle> idle;              /* front = most recently used */
    int64_t in_use = 0, idle_bytes = 0, peak = 0;
    int64_t next_id = 1;
    int64_t n_submitted = 0, n_admitted = 0, n_completed = 0, n_rejected = 0, n_evicted = 0,
            n_created = 0, n_cancelled = 0;
    int busy = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    int device = 0;
};

namespace {

int64_t footprint(const sf_server *s, int64_t nx, int64_t ny, int64_t nz)
{
    auto up = [](int64_t v) { return (v + 255) / 256 * 256; };
    const int64_t cube = up(nx * ny * nz * (int64_t)s->ebytes);
    const int64_t mask = up(nx * ny * ((nz + 31) / 32) * 4);
    /* the context's scratch: rows padded to 16 bytes, and a padded copy of
     * the cube, where nz * element size is not a multiple of 16 (sf_create) */
    const int64_t vec = 16 / (int64_t)s->ebytes;
    const int64_t zs = nz % vec != 0 ? (nz + vec - 1) / vec * vec : nz;
    const int64_t slot = up(nx * ny * zs * (int64_t)s->ebytes);
    return cube + slot * (s->n_xy + (zs != nz ? 1 : 0)) + mask + 4096;
}

/* make room for `need` bytes by destroying idle contexts (LRU); caller holds mu */
bool make_room(sf_server *s, int64_t need, std::vector<sf_ctx *> &doomed)
{
    while (s->in_use + s->idle_bytes + need > s->budget && !s->idle.empty()) {
        Idle &v = s->idle.back();
        doomed.push_back(v.ctx);
        s->idle_bytes -= v.bytes;
        ++s->n_evicted;
        s->idle.pop_back();
    }
    return s->in_use + s->idle_bytes + need <= s->budget;
}

void worker(sf_server *s, int slot)
{
    cudaSetDevice(s->device);
    cudaStream_t st = s->streams[slot];
    for (;;) {
        Request *r = nullptr;
        sf_ctx *ctx = nullptr;
        std::vector<sf_ctx *> doomed;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop && s->queue.empty()) return;
                if (!s->queue.empty()) {
                    Request *h = s->queue.front();
                    const Shape shape{h->nx, h->ny, h->nz};
                    /* an idle context of this shape is reused in place */
                    auto it = std::find_if(s->idle.begin(), s->idle.end(),
                                           [&](const Idle &v) { return v.shape == shape; });
                    if (it != s->idle.end()) {
                        ctx = it->ctx;
                        s->idle_bytes -= it->bytes;
                        s->idle.erase(it);
                        r = h;
                    } else if (make_room(s, h->bytes, doomed)) {
                        r = h;
                    }
                    if (r) {
                        s->queue.pop_front();
                        s->in_use += r->bytes;
                        s->peak = std::max(s->peak, s->in_use + s->idle_bytes);
                        ++s->n_admitted;
                        ++s->busy;
                        break;
                    }
                }
                s->cv_work.wait(lk);
            }
        }
        for (sf_ctx *d : doomed) sf_destroy(d);
        if (!ctx) {
            sf_config cfg = s->proto;
            cfg.nx = r->nx;
            cfg.ny = r->ny;
            cfg.nz = r->nz;
            cfg.filters = s->filters.data();
            r->status = sf_create(&cfg, &ctx);
            if (r->status == SF_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                ++s->n_created;
            }
        }
        if (r->status == SF_OK) r->status = sf_detect_host(ctx, r->h_cube, r->h_mask, st);
        r->t_done = now_ns();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->in_use -= r->bytes;
            --s->busy;
            if (ctx && r->status == SF_OK) {
                s->idle.push_front(Idle{Shape{r->nx, r->ny, r->nz}, ctx, r->bytes});
                s->idle_bytes += r->bytes;
                ctx = nullptr;
            }
            ++s->n_completed;
            s->done.push_back(r);
        }
        if (ctx) sf_destroy(ctx);
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

sf_status sf_server_create(const sf_config *proto, int64_t budget_bytes, int32_t max_inflight,
                           sf_server **out)
{
    if (!out) return SF_EINVAL;
    *out = nullptr;
    if (!proto || !proto->filters || proto->n_filters < 1 || budget_bytes <= 0 || max_inflight < 1 ||
        max_inflight > 64)
        return SF_EINVAL;
    int dev = proto->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return SF_ECUDA;
    sf_server *s = new sf_server();
    s->proto = *proto;
    s->filters.assign(proto->filters, proto->filters + proto->n_filters);
    s->proto.filters = nullptr;
    s->proto.device = dev;
    s->device = dev;
    s->budget = budget_bytes;
    s->ebytes = proto->storage == SF_F32 ? 4 : 2;
    std::vector<float> seen;
    for (const sf_filter_spec &f : s->filters)
        if (f.sigma_xy > 0.f && std::find(seen.begin(), seen.end(), f.sigma_xy) == seen.end()) seen.push_back(f.sigma_xy);
    s->n_xy = (int)seen.size();
    cudaSetDevice(dev);
    for (int i = 0; i < max_inflight; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return SF_ECUDA;
        }
        s->streams.push_back(st);
    }
    for (int i = 0; i < max_inflight; ++i) s->workers.emplace_back(worker, s, i);
    *out = s;
    return SF_OK;
}

sf_status sf_server_submit(sf_server *s, const void *h_cube, int64_t nx, int64_t ny, int64_t nz,
                           uint32_t *h_mask, int64_t *id)
{
    if (!s || !h_cube || !h_mask || nx < 1 || ny < 1 || nz < 1) return SF_EINVAL;
    Request *r = new Request{};
    r->h_cube = h_cube;
    r->nx = nx;
    r->ny = ny;
    r->nz = nz;
    r->h_mask = h_mask;
    r->t_submit = now_ns();
    r->bytes = footprint(s, nx, ny, nz);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        ++s->n_submitted;
        if (id) *id = r->id;
        if (r->bytes > s->budget) {
            /* can never fit: complete at once */
            r->status = SF_EBUDGET;
            r->t_done = r->t_submit;
            ++s->n_rejected;
            ++s->n_completed;
            s->done.push_back(r);
            s->cv_done.notify_all();
            return SF_OK;
        }
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    return SF_OK;
}

sf_status sf_server_cancel(sf_server *s, int64_t id)
{
    if (!s) return SF_EINVAL;
    Request *r = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const Request *q) { return q->id == id; });
        if (it == s->queue.end()) return SF_ESTATE;   /* admitted, done, or unknown */
        r = *it;
        s->queue.erase(it);
        r->status = SF_ECANCELED;
        r->t_done = now_ns();
        ++s->n_cancelled;
        ++s->n_completed;
        s->done.push_back(r);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return SF_OK;
}

sf_status sf_server_poll(sf_server *s, int64_t *ids, int32_t *statuses, int64_t *latency_ns,
                         int32_t cap, int32_t timeout_ms, int32_t *n)
{
    if (!s || !n || cap < 0 || (cap > 0 && (!ids || !statuses || !latency_ns))) return SF_EINVAL;
    *n = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->done.empty(); });
    while (*n < cap && !s->done.empty()) {
        Request *r = s->done.front();
        s->done.pop_front();
        ids[*n] = r->id;
        statuses[*n] = (int32_t)r->status;
        latency_ns[*n] = r->t_done - r->t_submit;
        ++*n;
        delete r;
    }
    return SF_OK;
}

sf_status sf_server_stats(sf_server *s, int64_t *out, int32_t cap)
{
    if (!s || !out || cap < 1) return SF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t v[] = {s->n_submitted, s->n_admitted, s->n_completed, s->n_rejected, s->in_use,
                         s->peak,        s->idle_bytes, s->n_evicted,   s->n_created,  s->busy,
                         (int64_t)s->queue.size(), s->budget, s->n_cancelled};
    const int32_t m = std::min<int32_t>(cap, (int32_t)(sizeof(v) / sizeof(v[0])));
    std::memcpy(out, v, sizeof(int64_t) * (size_t)m);
    return SF_OK;
}

sf_status sf_server_destroy(sf_server *s)
{
    if (!s) return SF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread &t : s->workers) t.join();
    for (Idle &v : s->idle) sf_destroy(v.ctx);
    for (Request *r : s->done) delete r;
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return SF_OK;
}

}  /* extern "C" */
