// ntt_serve.cu -- request loop for convolution serving: requests of
// different power-of-two lengths arrive from host threads and are batched
// continuously (a new batch leaves as soon as a stream slot is free, while
// earlier batches still run) and convolved by the fused kernels through the
// resident plans of the library; per-request latency is recorded.  Requests
// whose buffers the GPU can address (page-locked host memory over the
// C2C link, or device memory) run in place: the kernels read and write them
// through the batch's descriptor list.  Others are admitted against a fixed
// device-memory pool, copied in, convolved and copied back.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"
#include "serve_pool.h"

namespace {

using ntt::Pool;

double now_us()
{
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t id = 0;
    const void *f = nullptr, *g = nullptr;
    void *h = nullptr;
    uint32_t N = 0;
    int L = 0;
    double t_submit = 0, t_done = 0;
    ntt_status status = NTT_OK;
    bool done = false;
    size_t off = 0, bytes = 0;          // pool block holding f, g, h on the device (staged)
    bool direct = false;                // the kernels address f, g, h themselves
    const void *fd = nullptr, *gd = nullptr;
    void *hd = nullptr;                 // device-side addresses of f, g, h (direct)
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Req *> reqs;
    void *descs_dev = nullptr;          // device descriptor list of this slot
    void *descs_host = nullptr;         // pinned staging for it
    void *scratch = nullptr;            // split-path scratch of this slot (split_words words)
    bool busy = false;
};

}  // namespace

struct ntt_server_s {
    uint64_t m = 0;
    int word = 64;
    ntt_server_config cfg{};
    void *pool_mem = nullptr;
    Pool pool;
    std::vector<Slot> slots;
    std::map<int, ntt_plan_t> plans;    // log2 N -> cached plan (library-owned)
    size_t split_words = 0;             // scratch words per slot for the split path
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> live;
    std::vector<double> lat_us;
    uint64_t next_id = 1, submitted = 0, completed = 0, rejected = 0, batches = 0, direct = 0;
    uint32_t inflight = 0, max_inflight = 0;
    bool stop = false;
    std::atomic<size_t> npending{0};    // pending.size(), readable without the lock
    std::atomic<bool> stopping{false};  // stop, readable without the lock
    ntt_status fatal = NTT_OK;
    std::thread worker;
    int device = 0;
};

// The address at which the kernels of `device` reach p: page-locked host
// memory (mapped into the unified address space), memory of that device, or
// managed memory; nullptr when they cannot (pageable memory, another GPU).
static const void *device_address(const void *p, int device)
{
    // The query needs the device's context bound to the calling thread (a
    // client thread may never have touched CUDA); the caller's current
    // device is restored afterwards.
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    cudaSetDevice(device);
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    switch (at.type) {
    case cudaMemoryTypeHost: return at.devicePointer;
    case cudaMemoryTypeDevice: return at.device == device ? at.devicePointer : nullptr;
    case cudaMemoryTypeManaged: return at.devicePointer;
    default: return nullptr;
    }
}

static ntt_status server_launch(ntt_server_t s, Slot &slot, std::vector<Req *> &batch)
{
    const size_t elt = s->word / 8;
    cudaStream_t st = slot.stream;
    unsigned char *base = (unsigned char *)s->pool_mem;
    // group by length: descriptors laid out class by class
    std::stable_sort(batch.begin(), batch.end(), [](const Req *a, const Req *b) { return a->L > b->L; });
    void **host = (void **)slot.descs_host;
    for (size_t i = 0; i < batch.size(); ++i) {
        Req *r = batch[i];
        if (r->direct) {
            host[3 * i + 0] = const_cast<void *>(r->fd);
            host[3 * i + 1] = const_cast<void *>(r->gd);
            host[3 * i + 2] = r->hd;
            continue;
        }
        unsigned char *d = base + r->off;
        const size_t seq = (size_t)r->N * elt;
        host[3 * i + 0] = d;
        host[3 * i + 1] = d + seq;
        host[3 * i + 2] = d + 2 * seq;
        if (cudaMemcpyAsync(d, r->f, seq, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d + seq, r->g, seq, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ntt_fail(NTT_ERR_CUDA, "server: input copy");
    }
    if (cudaMemcpyAsync(slot.descs_dev, slot.descs_host, batch.size() * 3 * sizeof(void *), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return ntt_fail(NTT_ERR_CUDA, "server: descriptor copy");
    for (size_t i = 0; i < batch.size();) {
        size_t j = i;
        while (j < batch.size() && batch[j]->L == batch[i]->L) ++j;
        ntt_plan_t p = s->plans[batch[i]->L];
        // pairs per scratch wave for this length (2 N words each)
        const uint32_t wave = (uint32_t)std::max<size_t>(1, s->split_words / ((size_t)2 << batch[i]->L));
        ntt_status e = ntt_conv_descs(p, (unsigned char *)slot.descs_dev + i * 3 * sizeof(void *), (long long)(j - i),
                                      slot.scratch, wave, st);
        if (e != NTT_OK) return e;
        i = j;
    }
    for (Req *r : batch) {
        if (r->direct) continue;
        const size_t seq = (size_t)r->N * elt;
        if (cudaMemcpyAsync(r->h, base + r->off + 2 * seq, seq, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ntt_fail(NTT_ERR_CUDA, "server: output copy");
    }
    if (cudaEventRecord(slot.done, st) != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "server: event");
    return NTT_OK;
}

// The server thread owns the slots: it queries their events and launches
// batches without the lock, and takes the lock only to finish completed
// batches and to take requests out of the queue, so submitting threads are
// never held up by GPU calls.  While work is on the GPU it polls with a
// yield (a timed sleep this short overshoots by tens of microseconds, which
// the requests would wait out); when idle it blocks until a submit.
static void server_loop(ntt_server_t s)
{
    cudaSetDevice(s->device);
    const size_t elt = s->word / 8;
    std::vector<size_t> ready;
    std::vector<size_t> to_launch;
    uint32_t busy = 0;                             // slots with a batch on the GPU (this thread's count)
    while (true) {
        ready.clear();
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (s->slots[i].busy && cudaEventQuery(s->slots[i].done) != cudaErrorNotReady) ready.push_back(i);
        const bool work = !ready.empty() || (s->npending.load(std::memory_order_acquire) > 0 && busy < s->slots.size()) ||
                          s->stopping.load();
        if (!work) {
            if (busy > 0) {
                std::this_thread::yield();
            } else {
                std::unique_lock<std::mutex> lk(s->mu);
                if (s->pending.empty() && !s->stop) s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            continue;
        }
        to_launch.clear();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            // completions
            for (size_t i : ready) {
                Slot &slot = s->slots[i];
                const cudaError_t q = cudaEventQuery(slot.done);
                const double t = now_us();
                for (Req *r : slot.reqs) {
                    r->status = q == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
                    r->t_done = t;
                    r->done = true;
                    if (r->direct) ++s->direct;
                    else s->pool.release(r->off, r->bytes);
                    s->lat_us.push_back(t - r->t_submit);
                    ++s->completed;
                }
                slot.reqs.clear();
                slot.busy = false;
                --s->inflight;
                --busy;
            }
            if (!ready.empty()) s->cv_done.notify_all();
            if (s->stop && s->pending.empty() && s->inflight == 0) break;
            // admission: one batch per free slot
            for (size_t i = 0; i < s->slots.size(); ++i) {
                Slot &slot = s->slots[i];
                if (slot.busy || s->pending.empty()) continue;
                std::vector<Req *> batch;
                while (!s->pending.empty() && batch.size() < s->cfg.max_batch) {
                    Req *r = s->pending.front();
                    if (!r->direct) {
                        const size_t need = 3 * (size_t)r->N * elt;
                        size_t off;
                        if (!s->pool.alloc(need, &off)) break;    // wait for memory to free up
                        r->off = off;
                        r->bytes = need;
                    }
                    batch.push_back(r);
                    s->pending.pop_front();
                    s->npending.fetch_sub(1, std::memory_order_relaxed);
                }
                if (batch.empty()) break;
                slot.reqs = std::move(batch);
                slot.busy = true;
                ++s->batches;
                ++s->inflight;
                ++busy;
                s->max_inflight = std::max(s->max_inflight, s->inflight);
                to_launch.push_back(i);
            }
        }
        // launches, outside the lock
        for (size_t i : to_launch) {
            Slot &slot = s->slots[i];
            ntt::Trace tr("server batch");
            const ntt_status e = server_launch(s, slot, slot.reqs);
            if (e == NTT_OK) continue;
            std::lock_guard<std::mutex> lk(s->mu);
            for (Req *r : slot.reqs) {
                r->status = e;
                r->done = true;
                if (!r->direct) s->pool.release(r->off, r->bytes);
            }
            slot.reqs.clear();
            slot.busy = false;
            --s->inflight;
            --busy;
            s->fatal = e;
            s->cv_done.notify_all();
        }
    }
}

extern "C" void ntt_server_destroy(ntt_server_t s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->stopping.store(true);
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot &slot : s->slots) {
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.done) cudaEventDestroy(slot.done);
        cudaFree(slot.descs_dev);
        cudaFreeHost(slot.descs_host);
        cudaFree(slot.scratch);
    }
    cudaFree(s->pool_mem);
    for (auto &kv : s->live) delete kv.second;
    delete s;
}

extern "C" ntt_status ntt_server_create(uint64_t m, const ntt_server_config *cfg, ntt_server_t *out)
{
    if (!out || !cfg || cfg->pool_bytes == 0 || cfg->streams == 0 || cfg->max_batch == 0 || cfg->max_log2N == 0)
        return ntt_fail(NTT_ERR_ARG, "ntt_server_create: invalid argument");
    *out = nullptr;
    ntt_server_s *s = new ntt_server_s();
    s->m = m;
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    auto bail = [&](ntt_status e) { ntt_server_destroy(s); return e; };
    // resident plans for every admissible length (twiddle tables stay on the device)
    size_t split_words = 0;
    for (uint32_t L = 0; L <= cfg->max_log2N; ++L) {
        ntt_plan_t p;
        ntt_status e = ntt_cached_plan(m, 1u << L, &p);
        if (e != NTT_OK) return bail(e);
        s->plans[(int)L] = p;
        ntt_plan_info_t info;
        ntt_plan_get_info(p, &info);
        s->word = (int)info.word_bits;
        if (info.four_step) {
            const uint32_t w = std::min<uint32_t>(info.wave, cfg->max_batch);
            split_words = std::max(split_words, (size_t)2 * w * ((size_t)1 << L));
        }
    }
    s->split_words = split_words;
    if (!ntt::dev_alloc(&s->pool_mem, cfg->pool_bytes)) return bail(ntt_fail(NTT_ERR_OOM, "server: pool"));
    s->pool.init(cfg->pool_bytes);
    s->slots.resize(cfg->streams);
    for (Slot &slot : s->slots) {
        if (cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess ||
            !ntt::dev_alloc(&slot.descs_dev, (size_t)cfg->max_batch * 3 * sizeof(void *)) ||
            cudaHostAlloc(&slot.descs_host, (size_t)cfg->max_batch * 3 * sizeof(void *), cudaHostAllocDefault) != cudaSuccess) {
            (void)cudaGetLastError();          // (see ntt::dev_alloc)
            return bail(ntt_fail(NTT_ERR_OOM, "server: slot resources"));
        }
        if (split_words) {
            if (!ntt::dev_alloc(&slot.scratch, split_words * (s->word / 8)))
                return bail(ntt_fail(NTT_ERR_OOM, "server: split scratch"));
        }
    }
    s->worker = std::thread(server_loop, s);
    *out = s;
    return NTT_OK;
}

extern "C" ntt_status ntt_server_submit(ntt_server_t s, const void *f, const void *g, void *h, uint32_t N, uint64_t *id)
{
    if (!s || !f || !g || !h || N == 0 || (N & (N - 1)) != 0) return ntt_fail(NTT_ERR_ARG, "ntt_server_submit: invalid argument");
    const int L = __builtin_ctz(N);
    if ((uint32_t)L > s->cfg.max_log2N) return ntt_fail(NTT_ERR_LENGTH, "ntt_server_submit: N above the server's maximum");
    const size_t need = Pool::round(3 * (size_t)N * (s->word / 8));
    Req *r = new Req();
    r->f = f; r->g = g; r->h = h; r->N = N; r->L = L;
    if (!(s->cfg.flags & NTT_SERVER_STAGE_ALL)) {
        const void *fd = device_address(f, s->device), *gd = device_address(g, s->device);
        void *hd = const_cast<void *>(device_address(h, s->device));
        if (fd && gd && hd) {
            r->direct = true;
            r->fd = fd; r->gd = gd; r->hd = hd;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    if (id) *id = r->id;
    r->t_submit = now_us();
    ++s->submitted;
    s->live[r->id] = r;
    if (!r->direct && need > s->pool.size()) {    // can never be admitted
        r->status = NTT_ERR_ADMISSION;
        r->done = true;
        ++s->rejected;
        return ntt_fail(NTT_ERR_ADMISSION, "ntt_server_submit: request needs %zu bytes, pool holds %zu", need, s->pool.size());
    }
    s->pending.push_back(r);
    s->npending.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_one();
    return NTT_OK;
}

extern "C" ntt_status ntt_server_wait(ntt_server_t s, uint64_t id, uint32_t timeout_ms)
{
    if (!s) return ntt_fail(NTT_ERR_ARG, "ntt_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(id);
    if (it == s->live.end()) return ntt_fail(NTT_ERR_ARG, "ntt_server_wait: unknown or already collected request");
    Req *r = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
        return ntt_fail(NTT_ERR_TIMEOUT, "ntt_server_wait: request %llu not done in %u ms", (unsigned long long)id, timeout_ms);
    const ntt_status st = r->status;
    s->live.erase(it);
    delete r;
    return st;
}

extern "C" ntt_status ntt_server_drain(ntt_server_t s, uint32_t timeout_ms)
{
    if (!s) return ntt_fail(NTT_ERR_ARG, "ntt_server_drain: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return s->pending.empty() && s->inflight == 0;
    });
    if (!ok) return ntt_fail(NTT_ERR_TIMEOUT, "ntt_server_drain: work still pending after %u ms", timeout_ms);
    return s->fatal;
}

extern "C" ntt_status ntt_server_get_stats(ntt_server_t s, ntt_server_stats *out)
{
    if (!s || !out) return ntt_fail(NTT_ERR_ARG, "ntt_server_get_stats: invalid argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->max_inflight_batches = s->max_inflight;
    out->pool_bytes = s->pool.size();
    out->peak_pool_bytes = s->pool.peak();
    out->direct = s->direct;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_us = sum / (double)v.size();
    }
    return NTT_OK;
}

extern "C" ntt_status ntt_server_reset_stats(ntt_server_t s)
{
    if (!s) return ntt_fail(NTT_ERR_ARG, "ntt_server_reset_stats: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_us.clear();
    s->submitted = s->completed = s->rejected = s->batches = s->direct = 0;
    s->max_inflight = 0;
    return NTT_OK;
}
