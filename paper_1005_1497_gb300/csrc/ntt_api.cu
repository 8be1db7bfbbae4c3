// ntt_api.cu -- C ABI of the library: plans (host number theory, twiddle
// tables), dispatch of the transforms and convolutions, batch plans and the
// host-buffer path.  Declared in include/ntt_gb300.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ntt_gb300.h"
#include "ntt_launch.h"
#include "nt_host.h"
#include "host_sched.h"
#include "ntt_internal.h"

using ntt::ColArgs;
using ntt::DevDesc;
using ntt::Launch;
using ntt::ModC;
using ntt::NttArgs;
using ntt::RowArgs;

// ------------------------------------------------------------------ errors

static thread_local char g_last_error[512] = "";

ntt_status ntt_fail(ntt_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

static ntt_status cuda_fail(cudaError_t e, const char *what)
{
    return ntt_fail(NTT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(expr, what)                              \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

extern "C" const char *ntt_status_str(ntt_status s)
{
    switch (s) {
    case NTT_OK: return "NTT_OK";
    case NTT_ERR_LENGTH: return "NTT_ERR_LENGTH";
    case NTT_ERR_MODULUS: return "NTT_ERR_MODULUS";
    case NTT_ERR_WORD: return "NTT_ERR_WORD";
    case NTT_ERR_RANGE: return "NTT_ERR_RANGE";
    case NTT_ERR_OOM: return "NTT_ERR_OOM";
    case NTT_ERR_CUDA: return "NTT_ERR_CUDA";
    case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT";
    case NTT_ERR_ARG: return "NTT_ERR_ARG";
    case NTT_ERR_ADMISSION: return "NTT_ERR_ADMISSION";
    }
    return "NTT_ERR_UNKNOWN";
}

extern "C" const char *ntt_last_error(void) { return g_last_error; }

namespace ntt {
std::atomic<unsigned long long> launch_count{0};
}

extern "C" uint64_t ntt_launch_count(void) { return ntt::launch_count.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------- plans

struct ntt_plan_s {
    uint64_t m = 0;
    uint32_t N = 0;
    int L = 0;
    int word = 32;
    uint64_t n_max = 0, omega = 0, n_inv = 0;
    void *tw = nullptr;               // (z_i, z'_i) pairs, i < max(1, N/2)
    ModC<uint32_t> c32{};
    ModC<uint64_t> c64{};
    bool split = false;
    int LR = 0;
    uint32_t wave = 0;                 // pairs per scratch wave (split path)
    bool twist = false;                // split path form: the four-step twist (else row-dependent twiddles)
    int block = ntt::BLOCK;            // whole sequences: threads per block of the fused kernel
    long long small_max = 0;           // whole one-warp lengths: batches up to this run one block per pair
    void *scratch = nullptr;           // 2 * wave * N words
    void *pw = nullptr;                // split path: (w^e, Shoup quotient), e < N (the twist)
    void *pd = nullptr;                // one column pass: the twist factor of element x, at x (the diagonal)
    void *pwl = nullptr;               // split path: (w^(s l), quotient) at s 32 + l, s < 2^(L - LR), l < 32
    int nsm = 1;
    int device = 0;
    unsigned long long *counter = nullptr;
    // host-buffer path
    void *stage = nullptr;
    size_t stage_pairs = 0;
    cudaStream_t hstream[3] = {};       // conv_circular_host: inbound copies, convolutions, outbound copies
    cudaEvent_t hevent[3 * 4] = {};     // per staging slot: inputs in, convolved, output out
};

template <typename W>
static void fill_modc(ModC<W> &c, uint64_t m, uint64_t ninv)
{
    const int B = (int)sizeof(W) * 8;
    c.m = (W)m;
    c.m2 = (W)(2 * m);
    c.mneg = (W)(0 - nt::inv_pow2(m, B));
    const uint64_t cN = nt::shl_mod(ninv, B, m);
    c.cN = (W)cN;
    c.cNp = (W)nt::shoup_quot(cN, m, B);
    c.onep = (W)nt::shoup_quot(1, m, B);
    c.ninv = (W)ninv;
    c.ninvp = (W)nt::shoup_quot(ninv, m, B);
}

static int num_sms()
{
    int dev = 0, n = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

extern "C" void ntt_plan_destroy(ntt_plan_t p)
{
    if (!p) return;
    cudaFree(p->tw);
    cudaFree(p->scratch);
    cudaFree(p->pw);
    cudaFree(p->pd);
    cudaFree(p->pwl);
    cudaFree(p->counter);
    cudaFree(p->stage);
    for (cudaStream_t st : p->hstream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : p->hevent)
        if (ev) cudaEventDestroy(ev);
    delete p;
}

extern "C" ntt_status ntt_plan(uint64_t m, uint32_t N, ntt_plan_t *out)
{
    ntt::Trace tr("ntt_plan");
    if (!out) return ntt_fail(NTT_ERR_ARG, "ntt_plan: out is NULL");
    *out = nullptr;
    if (m < 3 || !nt::is_prime(m)) return ntt_fail(NTT_ERR_MODULUS, "ntt_plan: m=%llu is not an odd prime", (unsigned long long)m);
    if (m >= (1ull << 57)) return ntt_fail(NTT_ERR_WORD, "ntt_plan: m=%llu needs more than 57 bits", (unsigned long long)m);
    const uint64_t nmax = nt::order_of_two_pow2(m);
    if (nmax == 0) return ntt_fail(NTT_ERR_MODULUS, "ntt_plan: ord_m(2) is not a power of two for m=%llu", (unsigned long long)m);
    if (N == 0 || (N & (N - 1)) != 0) return ntt_fail(NTT_ERR_LENGTH, "ntt_plan: N=%u is not a power of two", N);
    if (nmax % N != 0) return ntt_fail(NTT_ERR_LENGTH, "ntt_plan: N=%u does not divide ord_m(2)=%llu", N, (unsigned long long)nmax);
    const int word = m < (1ull << 25) ? 32 : 64;
    const int L = __builtin_ctz(N);
    const int lmax = word == 32 ? Launch<uint32_t>::LMAX : Launch<uint64_t>::LMAX;
    if (L > lmax) return ntt_fail(NTT_ERR_LENGTH, "ntt_plan: N=2^%d above the supported 2^%d for %d-bit words", L, lmax, word);

    auto p = std::unique_ptr<ntt_plan_s, void (*)(ntt_plan_t)>(new ntt_plan_s(), ntt_plan_destroy);
    p->m = m; p->N = N; p->L = L; p->word = word; p->n_max = nmax;
    p->omega = nt::pow_mod(2, nmax / N, m);
    p->n_inv = nt::pow_mod(N % m, m - 2, m);            // Fermat: N^(m-2) = N^-1 for prime m
    cudaGetDevice(&p->device);
    p->nsm = num_sms();
    const int lrmax = word == 32 ? Launch<uint32_t>::LRMAX : Launch<uint64_t>::LRMAX;
    p->split = L > lrmax;
    p->LR = p->split ? lrmax : L;
    if (!p->split) p->block = ntt_default_block(word, L);
    if (!p->split)                                      // one block per pair below this batch (host_sched.h)
        p->small_max = ntt::small_batch_max(L, (word == 32 ? ntt::Arith<uint32_t>::RB : ntt::Arith<uint64_t>::RB) + 5,
                                            word / 8, p->nsm);
    ntt_schedule_t sched;
    const bool tuned = ntt_tuned_schedule(word, L, &sched);
    if (!p->split && tuned) {
        const bool ok = word == 32 ? Launch<uint32_t>::block_ok(L, sched.block) : Launch<uint64_t>::block_ok(L, sched.block);
        if (ok) p->block = sched.block;
    }

    // Twiddles z_i = w^{brv_{L-1}(i)}, i < N/2, with w^e = 2^{e N_Max / N}
    // generated by doubling modulo m (shift and conditional subtraction).
    const size_t half = N > 1 ? N / 2 : 1;
    std::vector<uint64_t> pw2 = nt::powers_of_two_by_doubling(N > 1 ? (nmax / N) * half : 1, m);
    const int B = word;
    const size_t elt = word / 8;
    std::vector<unsigned char> host(2 * half * elt);
    for (size_t i = 0; i < half; ++i) {
        uint64_t z = 1;
        if (N > 1) {
            const uint64_t e = nt::bit_reverse(i, L - 1);
            z = pw2[e * (nmax / N)];
        }
        const uint64_t zp = nt::shoup_quot(z, m, B);
        if (word == 32) {
            uint32_t a[2] = {(uint32_t)z, (uint32_t)zp};
            memcpy(&host[2 * i * elt], a, sizeof a);
        } else {
            uint64_t a[2] = {z, zp};
            memcpy(&host[2 * i * elt], a, sizeof a);
        }
    }
    if (!ntt::dev_alloc(&p->tw, host.size())) return ntt_fail(NTT_ERR_OOM, "ntt_plan: twiddle table");
    CUDA_TRY(cudaMemcpy(p->tw, host.data(), host.size(), cudaMemcpyHostToDevice), "ntt_plan: upload twiddles");
    if (!ntt::dev_alloc(&p->counter, sizeof(unsigned long long))) return ntt_fail(NTT_ERR_OOM, "ntt_plan: counter");
    if (word == 32) fill_modc(p->c32, m, p->n_inv);
    else fill_modc(p->c64, m, p->n_inv);

    if (p->split) {
        // Pairs per wave: at least enough to fill every SM with rows several
        // times over, and as many as 256 MB of scratch (2 N words per pair)
        // holds -- fewer, longer launches; the autotuner chose such waves on
        // GB300 (64 pairs of 2^19 words, the whole of the uneven batch's
        // classes), where the scratch is a small part of the 280 GB.
        const uint64_t rows_per_pair = 1ull << (L - p->LR);
        const uint32_t tuned_wave = tuned ? sched.wave : 0u;      // autotuned schedule, if any
        const int tuned_twist = tuned ? sched.twist : -1;
        uint64_t wave = tuned_wave;
        if (wave == 0)
            wave = std::max<uint64_t>((uint64_t)p->nsm * 4 / rows_per_pair, (256ull << 20) / (2 * (uint64_t)N * elt));
        // Form: the twist, measured faster on GB300 at every length (u64 2^16
        // -23%, 2^18 -15%; u32 2^19 -1%, and the autotuner's choice for every
        // u32 class 2^15..2^19); the autotuner measures both.
        p->twist = tuned_twist >= 0 ? tuned_twist != 0 : true;
        if (const char *env = getenv("NTT_SPLIT_TWIST")) p->twist = atoi(env) != 0;   // explicit override
        if (wave < 1) wave = 1;
        p->wave = (uint32_t)wave;
        if (!ntt::dev_alloc(&p->scratch, 2 * wave * N * elt)) return ntt_fail(NTT_ERR_OOM, "ntt_plan: scratch");
        // powers w^e, e < N, for the twist between the column and row passes
        // (w^e = 2^{e N_Max / N}, again from the doubling sequence)
        std::vector<uint64_t> all = nt::powers_of_two_by_doubling((nmax / N) * (uint64_t)N, m);
        std::vector<unsigned char> tab(2 * (size_t)N * elt);
        for (size_t e = 0; e < N; ++e) {
            const uint64_t z = all[e * (nmax / N)], zp = nt::shoup_quot(z, m, B);
            if (word == 32) {
                uint32_t a[2] = {(uint32_t)z, (uint32_t)zp};
                memcpy(&tab[2 * e * elt], a, sizeof a);
            } else {
                uint64_t a[2] = {z, zp};
                memcpy(&tab[2 * e * elt], a, sizeof a);
            }
        }
        if (!ntt::dev_alloc(&p->pw, tab.size())) return ntt_fail(NTT_ERR_OOM, "ntt_plan: power table");
        CUDA_TRY(cudaMemcpy(p->pw, tab.data(), tab.size(), cudaMemcpyHostToDevice), "ntt_plan: upload powers");
        if (L - p->LR <= 5) {
            // one column pass: element x = t + k 2^LR (t < 2^LR, k < 2^(L-LR))
            // takes w^(brv(k) t), the same for every pair, so the factor is
            // stored at x and read in the data's own (coalesced) layout
            const int lc = L - p->LR;
            std::vector<unsigned char> dg(tab.size());
            for (size_t x = 0; x < N; ++x) {
                const size_t k = x >> p->LR, t = x & (((size_t)1 << p->LR) - 1);
                size_t sk = 0;
                for (int i = 0; i < lc; ++i) sk |= ((k >> i) & 1u) << (lc - 1 - i);
                const size_t e = (sk * t) % N;
                memcpy(&dg[2 * x * elt], &tab[2 * e * elt], 2 * elt);
            }
            if (!ntt::dev_alloc(&p->pd, dg.size())) return ntt_fail(NTT_ERR_OOM, "ntt_plan: twist diagonal");
            CUDA_TRY(cudaMemcpy(p->pd, dg.data(), dg.size(), cudaMemcpyHostToDevice), "ntt_plan: upload twist diagonal");
        }
        const size_t ns = (size_t)1 << (L - p->LR);
        std::vector<unsigned char> lt(2 * ns * 32 * elt);
        for (size_t sidx = 0; sidx < ns; ++sidx)
            for (size_t l = 0; l < 32; ++l) {
                const uint64_t e = (sidx * l) % N;
                const uint64_t z = all[e * (nmax / N)], zp = nt::shoup_quot(z, m, B);
                const size_t i = sidx * 32 + l;
                if (word == 32) {
                    uint32_t a[2] = {(uint32_t)z, (uint32_t)zp};
                    memcpy(&lt[2 * i * elt], a, sizeof a);
                } else {
                    uint64_t a[2] = {z, zp};
                    memcpy(&lt[2 * i * elt], a, sizeof a);
                }
            }
        if (!ntt::dev_alloc(&p->pwl, lt.size())) return ntt_fail(NTT_ERR_OOM, "ntt_plan: lane power table");
        CUDA_TRY(cudaMemcpy(p->pwl, lt.data(), lt.size(), cudaMemcpyHostToDevice), "ntt_plan: upload lane powers");
    }
    *out = p.release();
    return NTT_OK;
}

extern "C" ntt_status ntt_plan_get_info(ntt_plan_t p, ntt_plan_info_t *info)
{
    if (!p || !info) return ntt_fail(NTT_ERR_ARG, "ntt_plan_get_info: NULL argument");
    memset(info, 0, sizeof *info);
    info->m = p->m; info->N = p->N; info->log2N = (uint32_t)p->L; info->n_max = p->n_max;
    info->omega = p->omega; info->n_inv = p->n_inv; info->word_bits = (uint32_t)p->word;
    info->four_step = p->split ? 1u : 0u; info->wave = p->wave;
    info->twist = p->split && p->twist ? 1u : 0u;
    info->block = p->split ? 0u : (uint32_t)p->block;
    info->small_max = (uint32_t)std::min<long long>(p->small_max, 0xffffffffLL);
    return NTT_OK;
}

extern "C" int ntt_plan_word_bits(ntt_plan_t p) { return p ? p->word : 0; }

// ------------------------------------------------------------- dispatch

template <typename W> static const ModC<W> &modc(ntt_plan_t p);
template <> const ModC<uint32_t> &modc<uint32_t>(ntt_plan_t p) { return p->c32; }
template <> const ModC<uint64_t> &modc<uint64_t>(ntt_plan_t p) { return p->c64; }

// Persistent grid: as many blocks as the SMs hold at once (`per_sm` each),
// fewer when the rows run out.
static int row_grid(int nsm, long long rows, int per_block, int per_sm = 1)
{
    long long blocks = (rows + per_block - 1) / per_block;
    if (blocks > (long long)nsm * per_sm) blocks = (long long)nsm * per_sm;
    return (int)(blocks > 0 ? blocks : 1);
}

// Fused convolution of `batch` pairs; src/dst modes: 0 contiguous arrays,
// 1 descriptor list (descs, pair0 offsets into it).
template <typename W>
static cudaError_t conv_dispatch(ntt_plan_t p, const W *f, const W *g, W *h, const DevDesc<W> *descs,
                                 long long pair0, long long batch, W *scratch, uint32_t wave, cudaStream_t st,
                                 int twist = -1)
{
    const bool tw_form = twist < 0 ? p->twist : twist != 0;
    const ModC<W> &c = modc<W>(p);
    const W *tw = (const W *)p->tw;
    const int mode = descs ? 1 : 0;
    if (!p->split) {
        RowArgs<W> a{f, g, h, descs, batch, pair0, tw, c};
        if (mode == 0 && batch <= p->small_max)
            return Launch<W>::conv_small(p->L, a, (int)std::min<long long>(batch, (long long)p->nsm * Launch<W>::SMALL_PER_SM), st);
        const int grid = row_grid(p->nsm, batch, Launch<W>::pairs_per_block(p->L, p->block), ntt::BLOCK / p->block);
        return Launch<W>::conv_full(p->L, mode, a, grid, st, p->block);
    }
    const long long N = p->N;
    for (long long w0 = 0; w0 < batch; w0 += wave) {
        const long long np = std::min<long long>(wave, batch - w0);
        ColArgs<W> ca{f, g, descs, scratch, scratch + (size_t)wave * N, h, np, pair0 + w0, tw, c, (const W *)p->pw,
                      (const W *)p->pwl, (const W *)p->pd};
        cudaError_t e = Launch<W>::cols_fwd(p->L, 2, mode, tw_form, ca, st);
        if (e != cudaSuccess) return e;
        const long long rows = np << (p->L - p->LR);
        RowArgs<W> ra{scratch, scratch + (size_t)wave * N, scratch, nullptr, rows, 0, tw, c};
        e = Launch<W>::conv_rows_split(p->L, tw_form, ra, row_grid(p->nsm, rows, Launch<W>::pairs_per_block(p->LR)), st);
        if (e != cudaSuccess) return e;
        e = Launch<W>::cols_inv(p->L, mode, tw_form, ca, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename W>
static cudaError_t ntt_dispatch(ntt_plan_t p, const W *x, W *y, long long batch, bool inv, cudaStream_t st)
{
    const ModC<W> &c = modc<W>(p);
    const W *tw = (const W *)p->tw;
    if (!p->split) {
        NttArgs<W> a{x, y, batch, tw, c};
        return Launch<W>::ntt_full(p->L, inv, a, row_grid(p->nsm, batch, Launch<W>::rows_per_block(p->L)), st);
    }
    const long long N = p->N;
    W *scratch = (W *)p->scratch;
    const long long wave = (long long)p->wave * 2;     // one sequence per pair: twice the pairs fit
    for (long long w0 = 0; w0 < batch; w0 += wave) {
        const long long np = std::min<long long>(wave, batch - w0);
        // the plan's form: the twist (whole-row trees with the uniform table)
        // or row-dependent twiddles; both leave the same tree order
        const bool twisted = p->twist;
        ColArgs<W> ca{x, nullptr, nullptr, scratch, nullptr, nullptr, np, w0, tw, c, (const W *)p->pw,
                      (const W *)p->pwl, (const W *)p->pd};
        cudaError_t e = Launch<W>::cols_fwd(p->L, 1, 0, twisted, ca, st);
        if (e != cudaSuccess) return e;
        const long long rows = np << (p->L - p->LR);
        RowArgs<W> ra{scratch, nullptr, nullptr, nullptr, rows, 0, tw, c};
        const int grid = row_grid(p->nsm, rows, Launch<W>::rows_per_block(p->LR));
        e = twisted ? Launch<W>::rows_uni(ra, grid, st) : Launch<W>::rows_fwd(p->L, ra, grid, st);
        if (e != cudaSuccess) return e;
        e = Launch<W>::bitrev_out(p->L, inv, scratch, y + (size_t)w0 * N, np, c, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" ntt_status ntt_forward(ntt_plan_t p, const void *x, void *X, size_t batch, ntt_stream_t stream)
{
    ntt::Trace tr("ntt_forward");
    if (!p || !x || !X || batch == 0) return ntt_fail(NTT_ERR_ARG, "ntt_forward: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = p->word == 32 ? ntt_dispatch<uint32_t>(p, (const uint32_t *)x, (uint32_t *)X, (long long)batch, false, st)
                                  : ntt_dispatch<uint64_t>(p, (const uint64_t *)x, (uint64_t *)X, (long long)batch, false, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "ntt_forward");
}

extern "C" ntt_status ntt_inverse(ntt_plan_t p, const void *X, void *x, size_t batch, ntt_stream_t stream)
{
    ntt::Trace tr("ntt_inverse");
    if (!p || !x || !X || batch == 0) return ntt_fail(NTT_ERR_ARG, "ntt_inverse: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = p->word == 32 ? ntt_dispatch<uint32_t>(p, (const uint32_t *)X, (uint32_t *)x, (long long)batch, true, st)
                                  : ntt_dispatch<uint64_t>(p, (const uint64_t *)X, (uint64_t *)x, (long long)batch, true, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "ntt_inverse");
}

extern "C" ntt_status conv_circular(ntt_plan_t p, const void *f, const void *g, void *h, size_t batch,
                                    ntt_stream_t stream)
{
    ntt::Trace tr("conv_circular");
    if (!p || !f || !g || !h || batch == 0) return ntt_fail(NTT_ERR_ARG, "conv_circular: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = p->word == 32
        ? conv_dispatch<uint32_t>(p, (const uint32_t *)f, (const uint32_t *)g, (uint32_t *)h, nullptr, 0,
                                  (long long)batch, (uint32_t *)p->scratch, p->wave, st)
        : conv_dispatch<uint64_t>(p, (const uint64_t *)f, (const uint64_t *)g, (uint64_t *)h, nullptr, 0,
                                  (long long)batch, (uint64_t *)p->scratch, p->wave, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "conv_circular");
}

extern "C" ntt_status conv_circular_plain(ntt_plan_t p, const void *f, const void *g, void *h, size_t batch,
                                          void *work, ntt_stream_t stream)
{
    if (!p || !f || !g || !h || !work || batch == 0) return ntt_fail(NTT_ERR_ARG, "conv_circular_plain: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = p->nsm * 8;
    cudaError_t e = p->word == 32
        ? Launch<uint32_t>::plain(p->L, (const uint32_t *)f, (const uint32_t *)g, (uint32_t *)h, (uint32_t *)work,
                                  (long long)batch, (const uint32_t *)p->tw, p->c32, grid, st)
        : Launch<uint64_t>::plain(p->L, (const uint64_t *)f, (const uint64_t *)g, (uint64_t *)h, (uint64_t *)work,
                                  (long long)batch, (const uint64_t *)p->tw, p->c64, grid, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "conv_circular_plain");
}

extern "C" ntt_status ntt_check_range(ntt_plan_t p, const void *data, size_t count, uint64_t *bad,
                                      ntt_stream_t stream)
{
    if (!p || !data) return ntt_fail(NTT_ERR_ARG, "ntt_check_range: invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(p->counter, 0, sizeof(unsigned long long), st), "ntt_check_range: memset");
    cudaError_t e = p->word == 32
        ? Launch<uint32_t>::check_range((const uint32_t *)data, (long long)count, (uint32_t)p->m, p->counter, p->nsm * 4, st)
        : Launch<uint64_t>::check_range((const uint64_t *)data, (long long)count, p->m, p->counter, p->nsm * 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "ntt_check_range");
    unsigned long long h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, p->counter, sizeof h, cudaMemcpyDeviceToHost, st), "ntt_check_range: copy");
    CUDA_TRY(cudaStreamSynchronize(st), "ntt_check_range: sync");
    if (bad) *bad = h;
    return h ? ntt_fail(NTT_ERR_RANGE, "ntt_check_range: %llu words >= m", h) : NTT_OK;
}

// ------------------------------------------------------- host-buffer path

// The device address of page-locked host memory (mapped into the unified
// address space); nullptr for anything else.
static const void *host_device_address(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

extern "C" ntt_status conv_circular_host(ntt_plan_t p, const void *f, const void *g, void *h, size_t batch,
                                         ntt_stream_t stream)
{
    ntt::Trace tr("conv_circular_host");
    if (!p || !f || !g || !h || batch == 0) return ntt_fail(NTT_ERR_ARG, "conv_circular_host: invalid argument");
    const size_t elt = p->word / 8;
    const size_t seq = (size_t)p->N * elt;
    // Page-locked buffers can also be read and written in place by the
    // kernels over the C2C link.  By default a batch whose inputs and output
    // total at most DIRECT_MAX bytes goes that way whole (no copies to wait
    // for: measured on GB300, 1 x 2^10 end to end 33 -> 19 us, 256 x 2^14
    // 0.31 -> 0.25 ms; from about 192 MB on the staged copies are faster,
    // 1024 x 2^14 0.876 against 0.892 ms).  NTT_HOST_DIRECT (percent)
    // overrides that: its share of the pairs goes in place on its own stream
    // while the copy engines stage the rest.
    constexpr size_t DIRECT_MAX = (size_t)96 << 20;
    size_t ndirect = 0;
    const void *fd = host_device_address(f), *gd = host_device_address(g);
    void *hd = const_cast<void *>(host_device_address(h));
    if (fd && gd && hd && !p->split) {
        const char *env = getenv("NTT_HOST_DIRECT");
        const int pct = env ? std::max(0, std::min(100, atoi(env))) : (3 * batch * seq <= DIRECT_MAX ? 100 : 0);
        ndirect = batch * (size_t)pct / 100;
    }
    if (ndirect == batch) {
        ntt_status s = conv_circular(p, fd, gd, hd, batch, stream);
        if (s != NTT_OK) return s;
        CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "conv_circular_host: sync");
        return NTT_OK;
    }
    // Chunks of ~48 MB of input (~32 MB on the split path; host_sched.h)
    // through SLOTS staging slots, with one stream per engine: every inbound
    // copy on one stream (the busier direction of the link never waits for a
    // convolution), the convolutions on a second, the outbound copies on a
    // third; events order a chunk's steps and free its slot for the chunk
    // SLOTS later.  (Measured on GB300 over C2C: about 210 GB/s in and 190 GB/s
    // out alone, more with both directions at once; one copy/compute stream
    // per slot was slower; 4096 x 2^14 with the shrinking last chunks below:
    // 24 / 32 / 48 / 64 MB chunks 3.16 / 3.09 / 3.03 / 3.02-3.05 ms.)
    constexpr int SLOTS = 4;
    size_t chunk = ntt::host_chunk_pairs(seq, p->split, batch);
    if (!p->stage || p->stage_pairs < chunk) {
        cudaFree(p->stage);
        p->stage = nullptr;
        if (!ntt::dev_alloc(&p->stage, SLOTS * 3 * chunk * seq)) return ntt_fail(NTT_ERR_OOM, "conv_circular_host: staging");
        p->stage_pairs = chunk;
        for (cudaStream_t &st : p->hstream)
            if (!st) CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
        for (cudaEvent_t &ev : p->hevent)
            if (!ev) CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    }
    chunk = p->stage_pairs < chunk ? p->stage_pairs : chunk;
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s_in = p->hstream[0], s_cv = p->hstream[1], s_out = p->hstream[2];
    cudaEvent_t *in_done = p->hevent, *cv_done = p->hevent + SLOTS, *out_done = p->hevent + 2 * SLOTS;
    cudaEvent_t start;
    CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "event");
    CUDA_TRY(cudaEventRecord(start, user), "record");
    for (cudaStream_t st : p->hstream) CUDA_TRY(cudaStreamWaitEvent(st, start, 0), "wait");
    cudaEventDestroy(start);
    if (ndirect) {                                  // the in-place share, on the user stream
        ntt_status s = conv_circular(p, fd, gd, hd, ndirect, stream);
        if (s != NTT_OK) return s;
    }
    const unsigned char *fb = (const unsigned char *)f, *gb = (const unsigned char *)g;
    unsigned char *hb = (unsigned char *)h;
    // Chunk sizes: the last ones shrink for whole-sequence lengths.  The split
    // path keeps full chunks: a few pairs of 2^19 are too few rows for the GPU
    // (64 x 2^19 end to end 1.65 -> 2.13 ms with the shrinking chunks).
    const std::vector<size_t> sizes = ntt::host_chunk_sizes(batch - ndirect, chunk, !p->split);
    size_t b0 = ndirect;
    for (size_t i = 0; i < sizes.size(); b0 += sizes[i], ++i) {
        const size_t nb = sizes[i];
        const size_t slot = i % SLOTS;
        unsigned char *base = (unsigned char *)p->stage + slot * 3 * chunk * seq;
        void *df = base, *dg = base + chunk * seq, *dh = base + 2 * chunk * seq;
        if (i >= (size_t)SLOTS) CUDA_TRY(cudaStreamWaitEvent(s_in, out_done[slot], 0), "wait slot");
        CUDA_TRY(cudaMemcpyAsync(df, fb + b0 * seq, nb * seq, cudaMemcpyHostToDevice, s_in), "H2D f");
        CUDA_TRY(cudaMemcpyAsync(dg, gb + b0 * seq, nb * seq, cudaMemcpyHostToDevice, s_in), "H2D g");
        CUDA_TRY(cudaEventRecord(in_done[slot], s_in), "record");
        CUDA_TRY(cudaStreamWaitEvent(s_cv, in_done[slot], 0), "wait inputs");
        ntt_status s = conv_circular(p, df, dg, dh, nb, (ntt_stream_t)s_cv);
        if (s != NTT_OK) return s;
        CUDA_TRY(cudaEventRecord(cv_done[slot], s_cv), "record");
        CUDA_TRY(cudaStreamWaitEvent(s_out, cv_done[slot], 0), "wait convolution");
        CUDA_TRY(cudaMemcpyAsync(hb + b0 * seq, dh, nb * seq, cudaMemcpyDeviceToHost, s_out), "D2H h");
        CUDA_TRY(cudaEventRecord(out_done[slot], s_out), "record");
    }
    for (cudaStream_t st : p->hstream) {
        CUDA_TRY(cudaEventRecord(in_done[0], st), "record");     // (slot 0's events are free again here)
        CUDA_TRY(cudaStreamWaitEvent(user, in_done[0], 0), "wait");
    }
    CUDA_TRY(cudaStreamSynchronize(user), "conv_circular_host: sync");
    return NTT_OK;
}

int ntt_plan_log2(ntt_plan_t p) { return p ? p->L : -1; }

int ntt_plan_device(ntt_plan_t p) { return p ? p->device : -1; }

// Whole sequences: column/row lengths below the longest default to half
// blocks (two per SM; measured 4-16% faster on GB300 at 2^11..2^13 for 4096
// and 16384 pairs), one-warp lengths and the longest to full blocks (the
// one-warp lengths are within 4% either way at those batches); a tuned
// schedule overrides this.
int ntt_default_block(int word_bits, int L)
{
    const int rw = word_bits == 32 ? ntt::Arith<uint32_t>::RB + 5 : ntt::Arith<uint64_t>::RB + 5;
    const int lr = word_bits == 32 ? ntt::LRMax<uint32_t>::v : ntt::LRMax<uint64_t>::v;
    return (L > rw && L < lr) ? ntt::BLOCK_HALF : ntt::BLOCK;
}

bool ntt_plan_set_block(ntt_plan_t p, int block)
{
    if (!p || p->split) return false;
    const bool ok = p->word == 32 ? Launch<uint32_t>::block_ok(p->L, block) : Launch<uint64_t>::block_ok(p->L, block);
    if (ok) p->block = block;
    return ok;
}

ntt_status ntt_conv_descs(ntt_plan_t p, const void *descs, long long count, void *scratch, uint32_t wave,
                          cudaStream_t st)
{
    if (!p || !descs || count <= 0) return ntt_fail(NTT_ERR_ARG, "conv (descriptors): invalid argument");
    if (p->split && (!scratch || wave == 0)) return ntt_fail(NTT_ERR_ARG, "conv (descriptors): split path needs scratch");
    cudaError_t e = p->word == 32
        ? conv_dispatch<uint32_t>(p, nullptr, nullptr, nullptr, (const DevDesc<uint32_t> *)descs, 0, count,
                                  (uint32_t *)scratch, wave, st)
        : conv_dispatch<uint64_t>(p, nullptr, nullptr, nullptr, (const DevDesc<uint64_t> *)descs, 0, count,
                                  (uint64_t *)scratch, wave, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "conv (descriptors)");
}

ntt_status ntt_conv_with_scratch(ntt_plan_t p, const void *f, const void *g, void *h, long long batch,
                                 void *scratch, uint32_t wave, cudaStream_t st, int twist)
{
    if (!p || !f || !g || !h || batch <= 0) return ntt_fail(NTT_ERR_ARG, "conv (scratch): invalid argument");
    if (p->split && (!scratch || wave == 0)) return ntt_fail(NTT_ERR_ARG, "conv (scratch): split path needs scratch");
    cudaError_t e = p->word == 32
        ? conv_dispatch<uint32_t>(p, (const uint32_t *)f, (const uint32_t *)g, (uint32_t *)h, nullptr, 0, batch,
                                  (uint32_t *)scratch, wave, st, twist)
        : conv_dispatch<uint64_t>(p, (const uint64_t *)f, (const uint64_t *)g, (uint64_t *)h, nullptr, 0, batch,
                                  (uint64_t *)scratch, wave, st, twist);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "conv (scratch)");
}

// The exact convolution's fused launch for one prime (32-bit words, whole
// sequences): see Launch::conv_exact.
ntt_status ntt_launch_exact(ntt_plan_t p, bool garner, const void *f64, const void *g64, void *h, const void *exact_args,
                            long long np, cudaStream_t st)
{
    if (!p || p->word != 32 || p->split) return ntt_fail(NTT_ERR_ARG, "exact fused launch: not a whole-sequence 32-bit plan");
    RowArgs<uint32_t> a{(const uint32_t *)f64, (const uint32_t *)g64, (uint32_t *)h, nullptr, np, 0,
                        (const uint32_t *)p->tw, p->c32};
    const int grid = row_grid(p->nsm, np, Launch<uint32_t>::pairs_per_block(p->L));
    cudaError_t e = Launch<uint32_t>::conv_exact(p->L, garner, a, *(const ntt::ExactArgs *)exact_args, grid, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "exact fused launch");
}

// Whether a batch plan runs the whole-sequence length 2^L inside its one
// persistent launch: always for the one-warp lengths (their bodies share one
// kernel without spilling); for the column/row lengths when the autotuned
// schedule says so, or when NTT_PERSIST_LMAX (a log2 length) reaches L.
bool ntt_persist_class(int word_bits, int L)
{
    const int rw = word_bits == 32 ? ntt::Arith<uint32_t>::RB + 5 : ntt::Arith<uint64_t>::RB + 5;
    const int lr = word_bits == 32 ? ntt::LRMax<uint32_t>::v : ntt::LRMax<uint64_t>::v;
    if (L <= rw) return true;
    if (L > lr) return false;
    if (const char *e = getenv("NTT_PERSIST_LMAX"))
        if (atoi(e) >= L) return true;
    ntt_schedule_t s;
    return ntt_tuned_schedule(word_bits, L, &s) && s.persist != 0;
}

size_t ntt_full_smem(int word_bits, int log2N)
{
    return word_bits == 32 ? Launch<uint32_t>::conv_full_smem(log2N) : Launch<uint64_t>::conv_full_smem(log2N);
}

int ntt_num_sms() { return num_sms(); }

// One RowArgs per length: the batch's descriptor list, and the plan's
// twiddle table and constants (a null table marks an absent length).
template <typename W>
static void fill_persist_classes(ntt::PersistArgs<W> &a, const void *descs, const ntt_plan_t *plans)
{
    for (int L = 0; L <= ntt::LRMax<W>::v; ++L) {
        RowArgs<W> &r = a.cls[L];
        r = RowArgs<W>{};
        r.descs = (const DevDesc<W> *)descs;
        if (!plans[L]) continue;
        r.tw = (const W *)plans[L]->tw;
        if constexpr (sizeof(W) == 4) r.c = plans[L]->c32;
        else r.c = plans[L]->c64;
    }
}

ntt_status ntt_launch_persistent(int word_bits, const void *descs, const void *items, int nitems, int *counter,
                                 const ntt_plan_t *plans, int lmax, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        if (word_bits == 32) {
            ntt::PersistArgs<uint32_t> a{(const ntt::WorkItem *)items, nitems, counter, {}};
            fill_persist_classes(a, descs, plans);
            e = Launch<uint32_t>::conv_persistent(a, lmax, grid, smem, st);
        } else {
            ntt::PersistArgs<uint64_t> a{(const ntt::WorkItem *)items, nitems, counter, {}};
            fill_persist_classes(a, descs, plans);
            e = Launch<uint64_t>::conv_persistent(a, lmax, grid, smem, st);
        }
    }
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "persistent launch");
}
