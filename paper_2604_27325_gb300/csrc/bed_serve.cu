// Native request loop: continuous batching of eigendecomposition requests on one GPU.
//
// Host code only (C++ threads and the CUDA runtime); the device work is the library's launches.
// Requests are admitted in arrival order while their memory fits: the pinned host result arena always,
// the device arena for what is staged there (inputs that are not page-locked, or everything when
// zero-copy is off). Everything admitted since the previous launch goes into one launch on a free
// stream slot (several launches overlap on the device). With zero-copy (the default) a launch reads
// page-locked inputs in place and writes eigenvalues, eigenvectors and flags straight into the
// result arena, so a request's latency holds no copy; its per-matrix addresses are handed to the
// kernels as descriptors in page-locked memory. The completion thread polls every in-flight launch
// and retires each as soon as it is done, whatever the order. In FIFO mode each request is one
// uniform-size launch on a single stream instead (the plain per-request baseline, same data path).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "bed_internal.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, capacity) elements with coalescing free blocks (host bookkeeping).
class Arena {
public:
    explicit Arena(int64_t cap) : cap_(cap) { free_[0] = cap; }
    int64_t alloc(int64_t size)
    {
        size = pad(size);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= size) {
                const int64_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > size) free_[off + size] = len - size;
                used_ += size;
                return off;
            }
        }
        return -1;
    }
    void release(int64_t off, int64_t size)
    {
        size = pad(size);
        used_ -= size;
        auto it = free_.emplace(off, size).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t capacity() const { return cap_; }
    int64_t used() const { return used_; }
    // 4-element (16-byte) granules keep every block 16-byte aligned
    static int64_t pad(int64_t x) { return (std::max<int64_t>(x, 1) + 3) / 4 * 4; }

private:
    int64_t cap_, used_ = 0;
    std::map<int64_t, int64_t> free_;
};

struct Request {
    int64_t id;
    const float* A;  // caller's host buffer
    int b, n;
    double t_submit = 0, t_admit = 0, t_done = 0;
    const float* A_in = nullptr;  // device-visible address of A when it is read in place (zero-copy)
    bool checked = false;         // A_in decided (at admission)
    int64_t a_off = -1;           // device input arena (staged input); the eigenvector arena uses it too
    int64_t w_off = -1;           // device eigenvalue arena (staged outputs)
    int64_t h_off = -1;           // pinned result arena: [V | W | info]
    int state = 0;                // 0 pending, 1 in flight, 2 done
    int32_t status = BED_OK;
    int64_t dev_elems() const { return int64_t(b) * n * n; }
    int64_t w_elems() const { return int64_t(b) * n; }
    int64_t host_elems() const { return int64_t(b) * (int64_t(n) * n + n + 1); }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    bed::MatDesc* desc_h = nullptr;  // page-locked descriptors of the launch's matrices
    int32_t* ns_h = nullptr;         // page-locked sizes
    const bed::MatDesc* desc_d = nullptr;  // their device-visible addresses
    const int32_t* ns_d = nullptr;
    int32_t* info_d = nullptr;       // flags of staged outputs
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool busy = false;
};

struct Launch {
    int slot;
    std::vector<Request*> reqs;
    double t_start, t_enqueued;  // host clock when launch() began and when its work was enqueued
};

}  // namespace

struct bed_server {
    bed_server_config cfg{};
    bed_params params{};
    bed_ragged_tuning tuning{};
    int device = 0;
    float* dev = nullptr;   // [A arena | V arena | W arena]
    float* host = nullptr;  // pinned results: per request [V | W | info]
    float* host_d = nullptr;  // device-visible address of `host`
    int64_t cap_av = 0, cap_w = 0;
    Arena* av = nullptr;
    Arena* w = nullptr;
    Arena* h = nullptr;
    std::vector<Slot> slots;
    std::deque<Request*> pending;
    std::deque<Launch> inflight;
    std::unordered_map<int64_t, Request*> reqs;
    std::mutex mu;
    std::condition_variable cv;
    bool running = true;
    int launching = 0;  // batches taken from `pending` whose launch is not yet in `inflight`
    int64_t next_id = 1;
    // statistics
    std::vector<double> lat;
    int64_t n_requests = 0, n_matrices = 0, n_launches = 0, peak_dev = 0;
    double max_admit_wait = 0, max_enqueue = 0, max_inflight = 0;  // where a request's time went, at worst
    double t_first = 0, t_last = 0;
    std::thread sched, done;
    int64_t dev_bytes_in_use() const { return 4 * (2 * av->used() + w->used()); }
};

namespace {

void fail_request(bed_server* s, Request* r, int32_t status)
{
    r->status = status;
    r->state = 2;
    r->t_done = now_s();
    (void)s;
}

// Releases the device arena space a request holds (host result space stays until bed_server_release).
void release_device(bed_server* s, Request* r)
{
    if (r->a_off >= 0) s->av->release(r->a_off, r->dev_elems());
    if (r->w_off >= 0) s->w->release(r->w_off, r->w_elems());
    r->a_off = r->w_off = -1;
}

void launch(bed_server* s, int si, std::vector<Request*>& batch)
{
    const double t_start = now_s();
    Slot& sl = s->slots[si];
    float* Ad = s->dev;
    float* Vd = s->dev + s->cap_av;
    float* Wd = s->dev + 2 * s->cap_av;
    const bool zc = s->cfg.zero_copy != 0;
    cudaError_t e = cudaSuccess;
    bed_status st = BED_OK;
    // inputs that are not read in place are copied into the device arena first
    for (Request* r : batch)
        if (e == cudaSuccess && !r->A_in)
            e = cudaMemcpyAsync(Ad + r->a_off, r->A, r->dev_elems() * sizeof(float), cudaMemcpyHostToDevice,
                                sl.stream);
    // addresses of every matrix: input in place or staged; outputs in the result arena (zero-copy) or
    // in the device arenas
    int64_t k = 0;
    for (Request* r : batch) {
        const float* a = r->A_in ? r->A_in : Ad + r->a_off;
        float* hv = s->host_d + r->h_off;
        float* hw = hv + r->dev_elems();
        int32_t* hi = reinterpret_cast<int32_t*>(hw + r->w_elems());
        for (int j = 0; j < r->b; ++j) {
            bed::MatDesc& d = sl.desc_h[k + j];
            d.A = a + int64_t(j) * r->n * r->n;
            d.V = zc ? hv + int64_t(j) * r->n * r->n : Vd + r->a_off + int64_t(j) * r->n * r->n;
            d.W = zc ? hw + int64_t(j) * r->n : Wd + r->w_off + int64_t(j) * r->n;
            d.info = zc ? hi + j : sl.info_d + k + j;
            sl.ns_h[k + j] = r->n;
        }
        k += r->b;
    }
    if (e == cudaSuccess) {
        if (s->cfg.mode == 0 && batch.size() > 1) {
            bed_params prm;
            bed::KParams kp;
            if (!bed::make_kparams(&s->params, &prm, &kp)) {
                st = BED_ERR_INVALID_ARG;
            } else {
                e = bed::launch_ragged_desc(sl.desc_d, sl.ns_d, k, s->tuning, kp, sl.ws, sl.stream);
            }
        } else {
            // one request: the uniform kernel on its contiguous matrices. In batching mode it takes the
            // team shape and leaf size the ragged kernel gives this n, so that a request's results do not
            // depend on whether it shared a launch (team types 0..4 have 256, 128, 64, 32 and 192 threads)
            Request* r = batch[0];
            const bed::MatDesc& d = sl.desc_h[0];
            bed_params p = s->params;
            if (s->cfg.mode == 0) {
                const int tt = s->tuning.team[r->n];
                p.threads_per_matrix = (tt == 4) ? 192 : (256 >> tt);
                p.leaf_size = s->tuning.leaf[r->n];
            }
            st = bed::eigh_common(d.A, d.W, d.V, d.info, r->b, r->n, &p, nullptr, sl.stream, true);
        }
    }
    if (!zc) {
        k = 0;
        for (Request* r : batch) {
            float* hv = s->host + r->h_off;
            float* hw = hv + r->dev_elems();
            int32_t* hi = reinterpret_cast<int32_t*>(hw + r->w_elems());
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hv, Vd + r->a_off, r->dev_elems() * sizeof(float), cudaMemcpyDeviceToHost,
                                    sl.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hw, Wd + r->w_off, r->w_elems() * sizeof(float), cudaMemcpyDeviceToHost,
                                    sl.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hi, sl.info_d + k, r->b * sizeof(int32_t), cudaMemcpyDeviceToHost, sl.stream);
            k += r->b;
        }
    }
    if (e == cudaSuccess && st == BED_OK) e = cudaEventRecord(sl.event, sl.stream);
    std::lock_guard<std::mutex> lock(s->mu);
    --s->launching;
    if (e != cudaSuccess || st != BED_OK) {
        // what was enqueued before the failure may still run: wait for it before the space is reused
        cudaStreamSynchronize(sl.stream);
        for (Request* r : batch) {
            fail_request(s, r, st != BED_OK ? st : BED_ERR_CUDA);
            release_device(s, r);
        }
        sl.busy = false;
        s->cv.notify_all();
        return;
    }
    const double t_enq = now_s();
    s->max_enqueue = std::max(s->max_enqueue, t_enq - t_start);
    s->inflight.push_back(Launch{si, batch, t_start, t_enq});
    ++s->n_launches;
    s->cv.notify_all();
}

void scheduler(bed_server* s)
{
    cudaSetDevice(s->device);
    const bool zc = s->cfg.zero_copy != 0;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv.wait(lock, [&] {
            const bool slot = std::any_of(s->slots.begin(), s->slots.end(), [](const Slot& x) { return !x.busy; });
            return !s->running || (!s->pending.empty() && slot);
        });
        if (!s->running && s->pending.empty()) return;
        if (s->pending.empty()) continue;
        int si = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (!s->slots[i].busy) {
                si = int(i);
                break;
            }
        if (si < 0) {  // shutting down with every slot busy: wait for the completion thread
            s->cv.wait_for(lock, std::chrono::microseconds(200));
            continue;
        }
        // admit from the head, in order, while everything fits
        std::vector<Request*> batch;
        int64_t count = 0;
        const int64_t cap = s->cfg.max_launch_matrices;
        while (!s->pending.empty()) {
            Request* r = s->pending.front();
            if (!batch.empty() && (s->cfg.mode != 0 || count + r->b > cap)) break;
            if (!r->checked) {  // in place only if the whole input is page-locked and mapped
                r->A_in = zc ? static_cast<const float*>(bed::mapped_range(r->A, r->dev_elems() * sizeof(float)))
                             : nullptr;
                r->checked = true;
            }
            const bool stage_in = !r->A_in, stage_out = !zc;
            int64_t a = -1, wo = -1;
            if (stage_in || stage_out) {
                a = s->av->alloc(r->dev_elems());
                if (a < 0) break;
            }
            if (stage_out) {
                wo = s->w->alloc(r->w_elems());
                if (wo < 0) {
                    s->av->release(a, r->dev_elems());
                    break;
                }
            }
            const int64_t ho = s->h->alloc(r->host_elems());
            if (ho < 0) {
                if (a >= 0) s->av->release(a, r->dev_elems());
                if (wo >= 0) s->w->release(wo, r->w_elems());
                break;
            }
            r->a_off = a;
            r->w_off = wo;
            r->h_off = ho;
            r->state = 1;
            r->t_admit = now_s();
            s->pending.pop_front();
            batch.push_back(r);
            count += r->b;
        }
        if (batch.empty()) {  // the head waits for memory that completions or releases will free
            if (!s->running && s->inflight.empty() && s->launching == 0) {
                // shutting down and nothing in flight can free memory any more: drop what cannot fit
                for (Request* r : s->pending) fail_request(s, r, BED_ERR_TOO_LARGE);
                s->pending.clear();
                s->cv.notify_all();
                continue;
            }
            s->cv.wait_for(lock, std::chrono::microseconds(200));
            continue;
        }
        s->peak_dev = std::max(s->peak_dev, s->dev_bytes_in_use());
        s->slots[si].busy = true;
        ++s->launching;
        lock.unlock();
        launch(s, si, batch);
        lock.lock();
    }
}

// Polls every in-flight launch (a copy of their events is taken under the lock, queried outside it) and
// retires each completed one at once, so that a short launch is not held behind a longer, older one.
void completer(bed_server* s)
{
    cudaSetDevice(s->device);
    std::vector<std::pair<int, cudaEvent_t>> evs;
    std::vector<std::pair<int, cudaError_t>> fin;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        s->cv.wait(lock, [&] {
            return !s->inflight.empty() || (!s->running && s->pending.empty() && s->launching == 0);
        });
        if (s->inflight.empty()) {
            if (!s->running && s->pending.empty() && s->launching == 0) return;
            continue;
        }
        evs.clear();
        for (const Launch& L : s->inflight) evs.emplace_back(L.slot, s->slots[L.slot].event);
        lock.unlock();
        fin.clear();
        for (const auto& x : evs) {
            const cudaError_t q = cudaEventQuery(x.second);
            if (q != cudaErrorNotReady) fin.emplace_back(x.first, q);
        }
        const double t = now_s();
        if (fin.empty()) std::this_thread::yield();  // launches in flight: keep polling
        lock.lock();
        for (const auto& f : fin) {
            auto it = std::find_if(s->inflight.begin(), s->inflight.end(),
                                   [&](const Launch& L) { return L.slot == f.first; });
            if (it == s->inflight.end()) continue;
            s->max_inflight = std::max(s->max_inflight, t - it->t_enqueued);
            for (Request* r : it->reqs) {
                s->max_admit_wait = std::max(s->max_admit_wait, r->t_admit - r->t_submit);
                release_device(s, r);
                r->state = 2;
                r->t_done = t;
                r->status = f.second == cudaSuccess ? BED_OK : BED_ERR_CUDA;
                s->lat.push_back(t - r->t_submit);
                ++s->n_requests;
                s->n_matrices += r->b;
                s->t_last = t;
            }
            s->slots[it->slot].busy = false;
            s->inflight.erase(it);
        }
        if (!fin.empty()) s->cv.notify_all();
    }
}

}  // namespace

extern "C" {

void bed_server_default_config(bed_server_config* c)
{
    if (!c) return;
    c->device_budget_bytes = size_t(4) << 30;
    c->host_result_bytes = size_t(2) << 30;
    c->streams = 3;
    c->max_launch_matrices = 16384;
    c->mode = 0;
    c->zero_copy = 1;
}

bed_status bed_server_create(const bed_server_config* cfg, const bed_params* p, const bed_ragged_tuning* t,
                             bed_server** out)
{
    if (!out) return BED_ERR_INVALID_ARG;
    *out = nullptr;
    bed_server_config c;
    bed_server_default_config(&c);
    if (cfg) c = *cfg;
    if (c.streams < 1 || c.streams > 16 || c.max_launch_matrices < 1 || c.max_launch_matrices > (1 << 24) ||
        (c.mode != 0 && c.mode != 1) || (c.zero_copy != 0 && c.zero_copy != 1) || c.device_budget_bytes < 4096 ||
        c.host_result_bytes < 4096)
        return BED_ERR_INVALID_ARG;
    {
        bed_params prm;
        bed::KParams kp;
        if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    }
    if (c.mode == 1) c.streams = 1;
    auto* s = new bed_server();
    s->cfg = c;
    bed_default_params(&s->params);
    if (p) s->params = *p;
    bed_ragged_default_tuning(&s->tuning);
    if (t) s->tuning = *t;
    cudaGetDevice(&s->device);
    // device budget in floats: 15/32 each for the input and eigenvector arenas, 1/16 for eigenvalues
    const int64_t units = int64_t(c.device_budget_bytes / 4);
    s->cap_av = units * 15 / 32 / 4 * 4;
    s->cap_w = (units - 2 * s->cap_av) / 4 * 4;
    cudaError_t e = cudaMalloc(&s->dev, size_t(2 * s->cap_av + s->cap_w) * sizeof(float));
    if (e == cudaSuccess) e = cudaHostAlloc(&s->host, c.host_result_bytes, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->host_d), s->host, 0);
    s->av = new Arena(s->cap_av);
    s->w = new Arena(s->cap_w);
    s->h = new Arena(int64_t(c.host_result_bytes / 4));
    const int m = c.max_launch_matrices;
    s->slots.resize(c.streams);
    for (auto& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.desc_h, m * sizeof(bed::MatDesc), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.ns_h, m * sizeof(int32_t), cudaHostAllocMapped);
        if (e == cudaSuccess)
            e = cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<bed::MatDesc**>(&sl.desc_d)), sl.desc_h, 0);
        if (e == cudaSuccess)
            e = cudaHostGetDevicePointer(reinterpret_cast<void**>(const_cast<int32_t**>(&sl.ns_d)), sl.ns_h, 0);
        if (e == cudaSuccess) e = cudaMalloc(&sl.info_d, m * sizeof(int32_t));
        sl.ws_bytes = bed_eigh_ragged_workspace_size(m);
        if (e == cudaSuccess) e = cudaMalloc(&sl.ws, sl.ws_bytes);
    }
    if (e != cudaSuccess) {
        s->running = false;
        bed_server_destroy(s);
        return bed::cuda_fail(e);
    }
    s->sched = std::thread(scheduler, s);
    s->done = std::thread(completer, s);
    *out = s;
    return BED_OK;
}

bed_status bed_server_submit(bed_server* s, const float* A_host, int32_t b, int32_t n, int64_t* request_id)
{
    if (!s || !A_host || !request_id || b < 1 || n < 1 || n > 64) return BED_ERR_INVALID_ARG;
    auto* r = new Request{};
    r->A = A_host;
    r->b = b;
    r->n = n;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    *request_id = r->id;
    // every launch's descriptor arrays hold max_launch_matrices entries, in both modes
    if (Arena::pad(r->dev_elems()) > s->av->capacity() || Arena::pad(r->w_elems()) > s->w->capacity() ||
        Arena::pad(r->host_elems()) > s->h->capacity() || r->b > s->cfg.max_launch_matrices) {
        fail_request(s, r, BED_ERR_TOO_LARGE);
        return BED_ERR_TOO_LARGE;
    }
    if (s->t_first == 0) s->t_first = r->t_submit;
    s->pending.push_back(r);
    s->cv.notify_all();
    return BED_OK;
}

bed_status bed_server_wait(bed_server* s, int64_t id, double timeout_s, const float** W, const float** V,
                           const int32_t** info)
{
    if (!s) return BED_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return BED_ERR_INVALID_ARG;
    Request* r = it->second;
    const bool ok = s->cv.wait_for(lock, std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s),
                                   [&] { return r->state == 2; });
    if (!ok) return BED_ERR_TIMEOUT;
    if (r->status != BED_OK) return static_cast<bed_status>(r->status);
    float* hv = s->host + r->h_off;
    if (V) *V = hv;
    if (W) *W = hv + r->dev_elems();
    if (info) *info = reinterpret_cast<const int32_t*>(hv + r->dev_elems() + r->w_elems());
    return BED_OK;
}

bed_status bed_server_release(bed_server* s, int64_t id)
{
    if (!s) return BED_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second->state != 2) return BED_ERR_INVALID_ARG;
    Request* r = it->second;
    if (r->h_off >= 0) s->h->release(r->h_off, r->host_elems());
    s->reqs.erase(it);
    delete r;
    s->cv.notify_all();
    return BED_OK;
}

bed_status bed_server_get_stats(bed_server* s, bed_server_stats* out)
{
    if (!s || !out) return BED_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof *out);
    out->requests = s->n_requests;
    out->matrices = s->n_matrices;
    out->launches = s->n_launches;
    out->peak_device_bytes = s->peak_dev;
    out->span_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, size_t(q * (v.size() - 1) + 0.5))]; };
        out->p50_s = pct(0.50);
        out->p99_s = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_s = sum / v.size();
        out->max_s = v.back();
    }
    out->max_admit_wait_s = s->max_admit_wait;
    out->max_enqueue_s = s->max_enqueue;
    out->max_inflight_s = s->max_inflight;
    return BED_OK;
}

bed_status bed_server_reset_stats(bed_server* s)
{
    if (!s) return BED_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->lat.clear();
    s->n_requests = s->n_matrices = s->n_launches = 0;
    s->peak_dev = s->dev_bytes_in_use();
    s->t_first = s->t_last = 0;
    s->max_admit_wait = s->max_enqueue = s->max_inflight = 0;
    return BED_OK;
}

void bed_server_destroy(bed_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->running = false;
        s->cv.notify_all();
    }
    if (s->sched.joinable()) s->sched.join();
    if (s->done.joinable()) s->done.join();
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.event) cudaEventDestroy(sl.event);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.desc_h);
        cudaFreeHost(sl.ns_h);
        cudaFree(sl.info_d);
        cudaFree(sl.ws);
    }
    for (auto& kv : s->reqs) delete kv.second;
    cudaFree(s->dev);
    cudaFreeHost(s->host);
    delete s->av;
    delete s->w;
    delete s->h;
    delete s;
}

}  // extern "C"
