// ntt_tune.cu -- autotuner of the convolution schedule.  Per (GPU name,
// word size, log2 N) it measures and records:
//  - split path (N above one block): its form (the four-step twist, or
//    row-dependent twiddles) and how many pairs a scratch wave carries
//    (bigger waves fill the SMs with more rows and amortise the column
//    passes; smaller ones keep the scratch resident in L2);
//  - whole sequences: the fused kernel's threads per block (512, or 256:
//    half the rows and shared memory per block, so two blocks share an SM),
//    and for lengths above one warp's whether a batch plan runs them inside
//    its single persistent launch or as a launch of their own.
// The winners live in a process-wide table that ntt_plan and ntt_batch_plan
// consult, and can be saved to / loaded from a JSON file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt_launch.h"

namespace {

struct Entry {
    ntt_schedule_t s;
    double ms;
};

std::mutex g_mu;
std::map<std::tuple<std::string, int, int>, Entry> g_table;

std::string gpu_name()
{
    int dev = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    return p.name;
}

void record(int word, int L, const ntt_schedule_t &s, double ms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[std::make_tuple(gpu_name(), word, L)] = Entry{s, ms};
}

// Timing helper: the mean of `reps` calls of fn on st after one untimed call.
template <class F>
double time_ms(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, F fn)
{
    if (fn() != NTT_OK) return 1e30;
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps; ++i)
        if (fn() != NTT_OK) return 1e30;
    cudaEventRecord(e1, st);
    float ms = 0;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return 1e30;
    return ms / reps;
}

}  // namespace

bool ntt_tuned_schedule(int word_bits, int log2N, ntt_schedule_t *out)
{
    // NTT_SCHEDULE names a schedule file that the first plan of the process
    // loads (as ntt_autotune_load would), e.g. to run tests under a schedule
    static const bool from_env = [] {
        const char *path = getenv("NTT_SCHEDULE");
        return path && *path && ntt_autotune_load(path) == NTT_OK;
    }();
    (void)from_env;
    const std::string name = gpu_name();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(std::make_tuple(name, word_bits, log2N));
    if (it == g_table.end()) return false;
    *out = it->second.s;
    return true;
}

extern "C" ntt_status ntt_autotune(uint64_t m, uint32_t N, size_t batch, ntt_tune_result *out)
{
    if (!out || batch == 0) return ntt_fail(NTT_ERR_ARG, "ntt_autotune: invalid argument");
    memset(out, 0, sizeof *out);
    ntt_plan_t p = nullptr;
    ntt_status s = ntt_plan(m, N, &p);
    if (s != NTT_OK) return s;
    ntt_plan_info_t info;
    ntt_plan_get_info(p, &info);
    const int word = (int)info.word_bits, L = (int)info.log2N;
    const int rw = word == 32 ? ntt::Arith<uint32_t>::RB + 5 : ntt::Arith<uint64_t>::RB + 5;
    out->default_wave = out->wave = info.wave;
    out->default_twist = out->twist = info.twist;
    out->default_block = info.four_step ? 0u : (uint32_t)ntt_default_block(word, L);
    out->block = info.block;
    out->default_persist = (!info.four_step && L <= rw) ? 1u : 0u;
    out->persist = out->default_persist;
    const size_t elt = info.word_bits / 8;
    const size_t seq = (size_t)N * elt;
    void *f = nullptr, *g = nullptr, *h = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    auto cleanup = [&]() {
        cudaFree(f); cudaFree(g); cudaFree(h);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        ntt_plan_destroy(p);
    };
    if (!ntt::dev_alloc(&f, batch * seq) || !ntt::dev_alloc(&g, batch * seq) || !ntt::dev_alloc(&h, batch * seq)) {
        cleanup();
        return ntt_fail(NTT_ERR_OOM, "ntt_autotune: buffers");
    }
    cudaMemset(f, 0, batch * seq);
    cudaMemset(g, 0, batch * seq);
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // (split lengths keep the whole-sequence defaults in their entry)
    ntt_schedule_t best_s{info.wave, (int)info.twist, info.four_step ? ntt::BLOCK : (int)info.block,
                          (int)out->default_persist};
    double best = 1e30, dflt = 0;

    if (info.four_step) {
        std::vector<uint32_t> cand;
        for (uint32_t w = 1; w <= batch && w <= 4096; w *= 2) cand.push_back(w);
        if (info.wave <= batch) cand.push_back(info.wave);
        cand.push_back((uint32_t)std::min<size_t>(batch, 65536));
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        for (uint32_t w : cand) {
            void *scratch = nullptr;
            if (!ntt::dev_alloc(&scratch, 2 * (size_t)w * seq)) continue;   // too big: skip candidate
            for (int tw = 0; tw < 2; ++tw) {
                const double t = time_ms(st, e0, e1, 3, [&] {
                    return ntt_conv_with_scratch(p, f, g, h, (long long)batch, scratch, w, st, tw);
                });
                if (w == info.wave && tw == (int)info.twist) dflt = t;
                if (t < best) { best = t; best_s.wave = w; best_s.twist = tw; }
            }
            cudaFree(scratch);
        }
    } else {
        // threads per block of the fused kernel
        for (int blk : {ntt::BLOCK, ntt::BLOCK_HALF}) {
            if (!ntt_plan_set_block(p, blk)) continue;
            const double t = time_ms(st, e0, e1, 5, [&] { return conv_circular(p, f, g, h, batch, (ntt_stream_t)st); });
            if (blk == (int)out->default_block) dflt = t;
            if (t < best) { best = t; best_s.block = blk; }
        }
        // column/row lengths: inside a batch plan's persistent launch, or a
        // launch of their own (one-warp lengths always run inside it)
        if (L > rw) {
            std::vector<ntt_conv_desc> host(batch);
            for (size_t i = 0; i < batch; ++i)
                host[i] = ntt_conv_desc{(const char *)f + i * seq, (const char *)g + i * seq, (char *)h + i * seq, N, 0};
            const ntt_schedule_t keep = best_s;
            double tp[2] = {1e30, 1e30};
            for (int pm = 0; pm < 2; ++pm) {
                ntt_schedule_t trial = keep;
                trial.persist = pm;
                record(word, L, trial, 0.0);             // the batch plan reads the table
                ntt_batch_t b = nullptr;
                if (ntt_batch_plan(m, host.data(), batch, &b) != NTT_OK) {
                    (void)cudaGetLastError();
                    continue;
                }
                tp[pm] = time_ms(st, e0, e1, 5, [&] { return ntt_batch_exec(b, (ntt_stream_t)st); });
                cudaStreamSynchronize(st);
                ntt_batch_destroy(b);
            }
            out->own_launch_ms = tp[0] < 1e30 ? tp[0] : 0.0;
            out->persist_ms = tp[1] < 1e30 ? tp[1] : 0.0;
            best_s.persist = tp[1] < tp[0] ? 1 : 0;
        }
    }
    cleanup();
    if (best >= 1e30) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table.erase(std::make_tuple(gpu_name(), word, L));      // (a trial entry may be left)
        return ntt_fail(NTT_ERR_CUDA, "ntt_autotune: no candidate ran");
    }
    out->wave = info.four_step ? best_s.wave : 0u;
    out->twist = info.four_step ? (uint32_t)best_s.twist : 0u;
    out->block = info.four_step ? 0u : (uint32_t)best_s.block;
    out->persist = info.four_step ? 0u : (uint32_t)best_s.persist;
    out->ms = best;
    out->default_ms = dflt;
    record(word, L, best_s, best);
    return NTT_OK;
}

extern "C" ntt_status ntt_autotune_save(const char *path)
{
    if (!path) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_save: NULL path");
    FILE *fp = fopen(path, "w");
    if (!fp) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_save: cannot open %s", path);
    std::lock_guard<std::mutex> lk(g_mu);
    fprintf(fp, "{\"schedules\": [\n");
    size_t i = 0;
    for (auto &kv : g_table) {
        const ntt_schedule_t &s = kv.second.s;
        fprintf(fp,
                "  {\"gpu\": \"%s\", \"word_bits\": %d, \"log2N\": %d, \"wave\": %u, \"twist\": %d, \"block\": %d, "
                "\"persist\": %d, \"ms\": %.6f}%s\n",
                std::get<0>(kv.first).c_str(), std::get<1>(kv.first), std::get<2>(kv.first), s.wave, s.twist, s.block,
                s.persist, kv.second.ms, ++i < g_table.size() ? "," : "");
    }
    fprintf(fp, "]}\n");
    fclose(fp);
    return NTT_OK;
}

// Value of "key": <int> in a line, if present.
static bool json_int(const char *line, const char *key, long long *v)
{
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\": ", key);
    const char *q = strstr(line, pat);
    if (!q) return false;
    return sscanf(q + strlen(pat), "%lld", v) == 1;
}

extern "C" ntt_status ntt_autotune_load(const char *path)
{
    if (!path) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: NULL path");
    FILE *fp = fopen(path, "r");
    if (!fp) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: cannot open %s", path);
    char line[1024];
    int n = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    while (fgets(line, sizeof line, fp)) {
        const char *q = strstr(line, "{\"gpu\": \"");
        if (!q) continue;
        q += 9;
        const char *e = strchr(q, '"');
        if (!e || e - q >= 256) continue;
        const std::string gpu(q, (size_t)(e - q));
        long long word, L, wave = 0, twist = 1, block = ntt::BLOCK, persist = -1;
        double ms = 0;
        if (!json_int(line, "word_bits", &word) || !json_int(line, "log2N", &L)) continue;
        json_int(line, "wave", &wave);
        json_int(line, "twist", &twist);
        json_int(line, "block", &block);
        json_int(line, "persist", &persist);
        if (block == 0) block = ntt::BLOCK;          // (entries of split lengths may carry 0: no choice)
        if (const char *mq = strstr(line, "\"ms\": ")) sscanf(mq + 6, "%lf", &ms);
        if ((word != 32 && word != 64) || L < 0 || L > 31 || wave < 0 || wave > 0xffffffffll) continue;
        if ((twist != 0 && twist != 1) || (block != ntt::BLOCK && block != ntt::BLOCK_HALF)) continue;
        const int rw = word == 32 ? ntt::Arith<uint32_t>::RB + 5 : ntt::Arith<uint64_t>::RB + 5;
        if (persist < 0) persist = L <= rw ? 1 : 0;
        ntt_schedule_t s{(uint32_t)wave, (int)twist, (int)block, persist != 0 ? 1 : 0};
        g_table[std::make_tuple(gpu, (int)word, (int)L)] = Entry{s, ms};
        ++n;
    }
    fclose(fp);
    return n > 0 ? NTT_OK : ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: no schedule in %s", path);
}
