// ntt_batch.cu -- uneven batches: many convolutions of different
// power-of-two lengths modulo one prime, grouped by length, each length
// class run by its fused kernel (or the split path), the short ones inside one
// persistent launch on a forked stream, and optionally captured once into a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt_count.h"
#include "ntt_launch.h"



namespace {

std::mutex g_cache_mu;
std::map<std::pair<uint64_t, uint32_t>, ntt_plan_t> g_plan_cache;   // library-owned, live until exit

}  // namespace

ntt_status ntt_cached_plan(uint64_t m, uint32_t N, ntt_plan_t *out)
{
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_plan_cache.find({m, N});
    if (it != g_plan_cache.end()) {
        // a schedule tuned or loaded since the plan was made applies to it too
        ntt_schedule_t s;
        if (ntt_tuned_schedule(ntt_plan_word_bits(it->second), ntt_plan_log2(it->second), &s))
            ntt_plan_set_block(it->second, s.block);
        *out = it->second;
        return NTT_OK;
    }
    ntt_plan_t p = nullptr;
    ntt_status s = ntt_plan(m, N, &p);
    if (s != NTT_OK) return s;
    g_plan_cache[{m, N}] = p;
    *out = p;
    return NTT_OK;
}

struct BatchClass {
    int L = 0;
    ntt_plan_t plan = nullptr;       // cached, not owned
    size_t off = 0;                  // first descriptor of the class in the device list
    size_t count = 0;
    void *scratch = nullptr;         // split path: owned by the batch plan
    uint32_t wave = 0;
    double work = 0;                 // N log N count: classes launch largest work first
    int stream = 0;
};

struct ntt_batch_s {
    uint64_t m = 0;
    int word = 32;
    std::vector<BatchClass> classes;
    // whole-sequence lengths: one persistent launch over a work list
    void *items = nullptr;           // ntt::WorkItem[nitems]
    int nitems = 0;
    std::vector<ntt_plan_t> persist_plans;   // indexed by log2 N; null where absent
    int *counter = nullptr;
    size_t persist_smem = 0;
    int persist_grid = 0;
    int persist_lmax = 0;            // longest length among the items
    void *descs = nullptr;           // DevDesc<W>[count], grouped by class
    size_t count = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned kernel_nodes = 0;       // kernel launches one replay of gexec runs
    std::vector<ntt_conv_desc> host_descs;   // copy, for cache comparison
};

extern "C" void ntt_batch_destroy(ntt_batch_t b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &c : b->classes) cudaFree(c.scratch);
    cudaFree(b->descs);
    cudaFree(b->items);
    cudaFree(b->counter);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

extern "C" ntt_status ntt_batch_plan(uint64_t m, const ntt_conv_desc *descs, size_t count, ntt_batch_t *out)
{
    ntt::Trace tr("ntt_batch_plan");
    if (!out || !descs || count == 0) return ntt_fail(NTT_ERR_ARG, "ntt_batch_plan: invalid argument");
    *out = nullptr;
    std::map<uint32_t, std::vector<size_t>> by_len;
    for (size_t i = 0; i < count; ++i) {
        const ntt_conv_desc &d = descs[i];
        if (!d.f || !d.g || !d.h) return ntt_fail(NTT_ERR_ARG, "ntt_batch_plan: descriptor %zu has a NULL pointer", i);
        by_len[d.N].push_back(i);
    }
    ntt_batch_s *b = new ntt_batch_s();
    b->m = m;
    b->count = count;
    b->host_descs.assign(descs, descs + count);
    auto bail = [&](ntt_status s) { ntt_batch_destroy(b); return s; };

    // classes, largest work first
    for (auto &kv : by_len) {
        BatchClass c;
        ntt_status s = ntt_cached_plan(m, kv.first, &c.plan);
        if (s != NTT_OK) return bail(s);
        c.L = ntt_plan_log2(c.plan);
        c.count = kv.second.size();
        c.work = (double)c.count * (double)kv.first * (c.L + 1);
        b->classes.push_back(c);
    }
    b->word = ntt_plan_word_bits(b->classes[0].plan);
    std::sort(b->classes.begin(), b->classes.end(), [](const BatchClass &x, const BatchClass &y) { return x.work > y.work; });

    // device descriptor list grouped by class
    const size_t elt = b->word / 8;
    std::vector<unsigned char> host(count * 3 * sizeof(void *));
    size_t pos = 0;
    for (auto &c : b->classes) {
        c.off = pos;
        for (size_t i : by_len[1u << c.L]) {
            const void *ptrs[3] = {descs[i].f, descs[i].g, descs[i].h};
            memcpy(&host[pos * 3 * sizeof(void *)], ptrs, sizeof ptrs);
            ++pos;
        }
    }
    if (!ntt::dev_alloc(&b->descs, host.size())) return bail(ntt_fail(NTT_ERR_OOM, "ntt_batch_plan: descriptors"));
    if (cudaMemcpy(b->descs, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(ntt_fail(NTT_ERR_CUDA, "ntt_batch_plan: upload descriptors"));

    // split classes get their own scratch so that classes run concurrently
    for (auto &c : b->classes) {
        ntt_plan_info_t info;
        ntt_plan_get_info(c.plan, &info);
        if (info.four_step) {
            c.wave = std::min<uint32_t>(info.wave, (uint32_t)c.count);
            if (!ntt::dev_alloc(&c.scratch, 2 * (size_t)c.wave * ((size_t)1 << c.L) * elt))
                return bail(ntt_fail(NTT_ERR_OOM, "ntt_batch_plan: scratch"));
        }
    }

    // Short lengths become work items of a single persistent launch on
    // stream 0; each item covers two rounds of a block's rows in flight.
    // Longer lengths keep their own launches (stream assignment below).
    const int lrmax = b->word == 32 ? ntt::LRMax<uint32_t>::v : ntt::LRMax<uint64_t>::v;
    std::vector<ntt::WorkItem> items;
    b->persist_plans.assign(lrmax + 1, nullptr);
    size_t nsplit = 0;             // classes with their own launches
    for (auto &c : b->classes) {
        if (!ntt_persist_class(b->word, c.L)) { ++nsplit; continue; }
        b->persist_lmax = std::max(b->persist_lmax, c.L);
        c.stream = -1;                                   // runs inside the persistent launch
        const int ppb = b->word == 32 ? ntt::Launch<uint32_t>::pairs_per_block(c.L) : ntt::Launch<uint64_t>::pairs_per_block(c.L);
        const long long per = 2LL * ppb;
        for (long long i = 0; i < (long long)c.count; i += per)
            items.push_back(ntt::WorkItem{c.L, 0, (long long)c.off + i, std::min<long long>(per, (long long)c.count - i)});
        b->persist_plans[c.L] = c.plan;
        b->persist_smem = std::max(b->persist_smem, ntt_full_smem(b->word, c.L));
    }
    b->nitems = (int)items.size();
    if (b->nitems) {
        if (!ntt::dev_alloc(&b->items, items.size() * sizeof(ntt::WorkItem)) ||
            !ntt::dev_alloc(&b->counter, sizeof(int)))
            return bail(ntt_fail(NTT_ERR_OOM, "ntt_batch_plan: work list"));
        if (cudaMemcpy(b->items, items.data(), items.size() * sizeof(ntt::WorkItem), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(ntt_fail(NTT_ERR_CUDA, "ntt_batch_plan: upload work list"));
        b->persist_grid = std::min(ntt_num_sms(), b->nitems);
    }
    // Streams: the persistent launch on one, every class with launches of its
    // own on another, one after the other, largest work first.  Each of those
    // classes' kernels fills the GPU, so running two at once only makes them
    // interfere: measured on GB300 (10,000 uneven pairs, graph replay) 7.80 ms
    // with them spread over three streams by longest processing time, 7.44 ms
    // on one beside the persistent launch's, 7.47 ms with everything on one.
    if (nsplit == 0 && b->nitems == 0) return bail(ntt_fail(NTT_ERR_ARG, "ntt_batch_plan: empty batch"));
    const int K = (b->nitems && nsplit) ? 2 : 1;
    const int own = K - 1;                                   // stream of the own-launch classes
    for (auto &c : b->classes)
        if (c.stream != -1) c.stream = own;
    b->streams.resize(K);
    b->done.resize(K);
    for (int i = 0; i < K; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(ntt_fail(NTT_ERR_CUDA, "ntt_batch_plan: streams"));
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(ntt_fail(NTT_ERR_CUDA, "ntt_batch_plan: event"));
    *out = b;
    return NTT_OK;
}

extern "C" ntt_status ntt_batch_exec(ntt_batch_t b, ntt_stream_t stream)
{
    ntt::Trace tr("ntt_batch_exec");
    if (!b) return ntt_fail(NTT_ERR_ARG, "ntt_batch_exec: NULL batch");
    cudaStream_t user = (cudaStream_t)stream;
    if (cudaEventRecord(b->fork, user) != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec: record");
    for (auto s : b->streams)
        if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec: wait");
    if (b->nitems) {
        ntt_status s = ntt_launch_persistent(b->word, b->descs, b->items, b->nitems, b->counter, b->persist_plans.data(),
                                             b->persist_lmax, b->persist_grid, b->persist_smem, b->streams[0]);
        if (s != NTT_OK) return s;
    }
    for (auto &c : b->classes) {
        if (c.stream < 0) continue;                       // in the persistent launch
        cudaStream_t st = b->streams[c.stream];
        const unsigned char *d = (const unsigned char *)b->descs + c.off * 3 * sizeof(void *);
        ntt_status s = ntt_conv_descs(c.plan, d, (long long)c.count, c.scratch, c.wave, st);
        if (s != NTT_OK) return s;
    }
    for (size_t i = 0; i < b->streams.size(); ++i) {
        if (cudaEventRecord(b->done[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(user, b->done[i], 0) != cudaSuccess)
            return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec: join");
    }
    return NTT_OK;
}

extern "C" ntt_status ntt_batch_exec_graph(ntt_batch_t b, ntt_stream_t stream)
{
    ntt::Trace tr("ntt_batch_exec_graph");
    if (!b) return ntt_fail(NTT_ERR_ARG, "ntt_batch_exec_graph: NULL batch");
    cudaStream_t user = (cudaStream_t)stream;
    if (!b->gexec) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec_graph: stream");
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        ntt_status s = e == cudaSuccess ? ntt_batch_exec(b, (ntt_stream_t)cap) : NTT_ERR_CUDA;
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess || s != NTT_OK || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return s != NTT_OK ? s : ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec_graph: capture failed");
        }
        b->graph = g;
        if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess)
            return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec_graph: instantiate");
        // the captured launches were counted as issued but did not run:
        // take them back, and count the graph's kernel nodes per replay
        size_t n = 0;
        cudaGraphGetNodes(g, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        if (n) cudaGraphGetNodes(g, nodes.data(), &n);
        for (size_t i = 0; i < n; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->kernel_nodes;
        }
        ntt::launch_count.fetch_sub(b->kernel_nodes, std::memory_order_relaxed);
    }
    cudaError_t e = cudaGraphLaunch(b->gexec, user);
    if (e != cudaSuccess) return ntt_fail(NTT_ERR_CUDA, "ntt_batch_exec_graph: launch: %s", cudaGetErrorString(e));
    ntt::launch_count.fetch_add(b->kernel_nodes, std::memory_order_relaxed);
    return NTT_OK;
}

extern "C" ntt_status conv_batched(uint64_t m, const ntt_conv_desc *descs, size_t count, ntt_stream_t stream)
{
    if (!descs || count == 0) return ntt_fail(NTT_ERR_ARG, "conv_batched: invalid argument");
    static thread_local ntt_batch_t last = nullptr;
    bool same = last && last->m == m && last->count == count &&
                memcmp(last->host_descs.data(), descs, count * sizeof(ntt_conv_desc)) == 0;
    if (!same) {
        if (last) {
            // the previous batch plan may still be in use by queued work
            cudaDeviceSynchronize();
            ntt_batch_destroy(last);
            last = nullptr;
        }
        ntt_status s = ntt_batch_plan(m, descs, count, &last);
        if (s != NTT_OK) return s;
    }
    return ntt_batch_exec(last, stream);
}
