// ntt_tune.cu -- autotuner of the split path's schedule: its form (the
// four-step twist, or row-dependent twiddles) and how many pairs a scratch
// wave carries (bigger waves fill the SMs with more rows and amortise the
// column passes; smaller ones keep the scratch resident in L2).  The winner
// is kept per (GPU name, word size, log2 N) in a process-wide table that
// ntt_plan consults, and can be saved to / loaded from a JSON file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_internal.h"

namespace {

struct Entry {
    uint32_t wave;
    int twist;
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

}  // namespace

bool ntt_tuned_schedule(int word_bits, int log2N, uint32_t *wave, int *twist)
{
    const std::string name = gpu_name();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(std::make_tuple(name, word_bits, log2N));
    if (it == g_table.end()) return false;
    *wave = it->second.wave;
    *twist = it->second.twist;
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
    out->default_wave = info.wave;
    out->wave = info.wave;
    out->default_twist = info.twist;
    out->twist = info.twist;
    if (!info.four_step) {                       // one block per sequence: nothing to choose
        ntt_plan_destroy(p);
        return NTT_OK;
    }
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
    if (!ntt::dev_alloc(&f, batch * seq) || !ntt::dev_alloc(&g, batch * seq) ||
        !ntt::dev_alloc(&h, batch * seq)) {
        cleanup();
        return ntt_fail(NTT_ERR_OOM, "ntt_autotune: buffers");
    }
    cudaMemset(f, 0, batch * seq);
    cudaMemset(g, 0, batch * seq);
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<uint32_t> cand;
    for (uint32_t w = 1; w <= batch && w <= 4096; w *= 2) cand.push_back(w);
    if (info.wave <= batch) cand.push_back(info.wave);
    cand.push_back((uint32_t)std::min<size_t>(batch, 65536));
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    double best = 1e30, dflt = 0;
    uint32_t best_w = info.wave;
    int best_tw = (int)info.twist;
    for (uint32_t w : cand) {
        void *scratch = nullptr;
        if (!ntt::dev_alloc(&scratch, 2 * (size_t)w * seq)) continue;   // too big: skip candidate
        for (int tw = 0; tw < 2; ++tw) {
            ntt_status r = ntt_conv_with_scratch(p, f, g, h, (long long)batch, scratch, w, st, tw);
            float ms = 0;
            double t = 1e30;
            if (r == NTT_OK) {
                cudaEventRecord(e0, st);
                for (int i = 0; i < 3 && r == NTT_OK; ++i)
                    r = ntt_conv_with_scratch(p, f, g, h, (long long)batch, scratch, w, st, tw);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) == cudaSuccess && r == NTT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    t = ms / 3.0;
            }
            if (w == info.wave && tw == (int)info.twist) dflt = t;
            if (t < best) { best = t; best_w = w; best_tw = tw; }
        }
        cudaFree(scratch);
    }
    cleanup();
    if (best >= 1e30) return ntt_fail(NTT_ERR_CUDA, "ntt_autotune: no candidate ran");
    out->wave = best_w;
    out->twist = (uint32_t)best_tw;
    out->ms = best;
    out->default_ms = dflt;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_table[std::make_tuple(gpu_name(), (int)info.word_bits, (int)info.log2N)] = Entry{best_w, best_tw, best};
    }
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
        fprintf(fp, "  {\"gpu\": \"%s\", \"word_bits\": %d, \"log2N\": %d, \"wave\": %u, \"twist\": %d, \"ms\": %.6f}%s\n",
                std::get<0>(kv.first).c_str(), std::get<1>(kv.first), std::get<2>(kv.first), kv.second.wave,
                kv.second.twist, kv.second.ms, ++i < g_table.size() ? "," : "");
    }
    fprintf(fp, "]}\n");
    fclose(fp);
    return NTT_OK;
}

extern "C" ntt_status ntt_autotune_load(const char *path)
{
    if (!path) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: NULL path");
    FILE *fp = fopen(path, "r");
    if (!fp) return ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: cannot open %s", path);
    char line[512];
    int n = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    while (fgets(line, sizeof line, fp)) {
        char gpu[256];
        int word, log2N, twist;
        unsigned wave;
        double ms;
        const char *q = strstr(line, "{\"gpu\": \"");
        if (!q) continue;
        q += 9;
        const char *e = strchr(q, '"');
        if (!e || (size_t)(e - q) >= sizeof gpu) continue;
        memcpy(gpu, q, (size_t)(e - q));
        gpu[e - q] = 0;
        if (sscanf(e, "\", \"word_bits\": %d, \"log2N\": %d, \"wave\": %u, \"twist\": %d, \"ms\": %lf", &word, &log2N,
                   &wave, &twist, &ms) == 5 &&
            wave > 0 && (twist == 0 || twist == 1)) {
            g_table[std::make_tuple(std::string(gpu), word, log2N)] = Entry{wave, twist, ms};
            ++n;
        }
    }
    fclose(fp);
    return n > 0 ? NTT_OK : ntt_fail(NTT_ERR_ARG, "ntt_autotune_load: no schedule in %s", path);
}
