/*
 * ntt_gb300.h -- C ABI of the GB300 (sm_103a) exact digital circular
 * convolution library.
 *
 * The library computes, exactly and modulo a prime m, the circular
 * convolution of two integer sequences of a power-of-two length N
 *
 *     h(j) = < sum_{k=0}^{N-1} f(k) * g(<j-k>_N) >_m           (Eq. 1)
 *
 * through the number-theoretic transform whose kernel is a power of two
 *
 *     X(u) = < sum_{t=0}^{N-1} x(t) * w^{ut} >_m,  w = 2^(N_Max/N)   (Eq. 2)
 *     x(t) = < N^-1 sum_{u=0}^{N-1} X(u) * w^{<-ut>_N} >_m            (Eq. 3)
 *
 * where N_Max = ord_m(2) is a power of two, i.e. m is a prime factor of a
 * Fermat number (Sec. III-A, Prop. 2; Table 1 lists 641, 2424833, 319489 and
 * 13631489, the last allowing every N <= 2^19).  <a>_m is the remainder in
 * [0, m) (Appendix A) and N^-1 the multiplicative inverse of N mod m.
 *
 * Conventions shared by every entry point
 *   - Words.  Sequences are arrays of unsigned words: uint32_t when
 *     m < 2^25, uint64_t when 2^25 <= m < 2^57 (ntt_plan_word_bits tells
 *     which).  Inputs must lie in [0, m); the fast paths do not check this
 *     and the result for other inputs is unspecified (ntt_check_range checks
 *     a buffer explicitly).  Every output is canonical, in [0, m).
 *   - Layout.  A batch of B sequences of length N is one contiguous
 *     row-major array [B][N]; element t of sequence b is at index b*N + t.
 *     Spectra (ntt_forward output, ntt_inverse input) are in natural order
 *     u = 0 .. N-1.
 *   - Memory.  Every data pointer named *_dev is a device pointer of the
 *     current CUDA device, owned by the caller, and must stay valid until the
 *     work queued on `stream` has completed.  Input and output may alias
 *     (in-place calls are allowed).  Pointers must be aligned to the word
 *     size.  Plans own their twiddle tables and scratch buffers (device
 *     memory allocated by ntt_plan, freed by ntt_plan_destroy).
 *   - Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls enqueue work and return without synchronising, except where a
 *     comment says otherwise; errors of the launch itself are returned,
 *     errors of the asynchronous work surface on the stream.
 *   - Errors.  Every call returns an ntt_status; nothing is thrown across the
 *     ABI.  ntt_last_error() gives a human-readable message for the last
 *     failure on the calling thread.
 */
#ifndef NTT_GB300_H
#define NTT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ntt_stream_t;         /* == cudaStream_t */
typedef struct ntt_plan_s *ntt_plan_t;            /* opaque, owned by the library */
typedef struct ntt_batch_s *ntt_batch_t;          /* opaque, owned by the library */

typedef enum {
    NTT_OK = 0,
    NTT_ERR_LENGTH = 1,    /* N not a power of two, or N does not divide ord_m(2), or N above the supported maximum */
    NTT_ERR_MODULUS = 2,   /* m not prime, or ord_m(2) not a power of two (m divides no Fermat number) */
    NTT_ERR_WORD = 3,      /* m too large for the supported word sizes (m >= 2^57) */
    NTT_ERR_RANGE = 4,     /* an input word is >= m (ntt_check_range only) */
    NTT_ERR_OOM = 5,       /* device or host allocation failed */
    NTT_ERR_CUDA = 6,      /* a CUDA runtime call failed; see ntt_last_error() */
    NTT_ERR_TIMEOUT = 7,   /* a bounded device-side wait expired */
    NTT_ERR_ARG = 8,       /* null pointer, zero count or otherwise invalid argument */
    NTT_ERR_ADMISSION = 9  /* a request does not fit the serving memory budget */
} ntt_status;

/* Human-readable name of a status code (static string, never NULL). */
const char *ntt_status_str(ntt_status s);

/* Message describing the last failure on the calling thread (static per
 * thread, overwritten by the next failure; "" if none). */
const char *ntt_last_error(void);

/* Kernel launches the library has issued in this process, counted on the
 * host as each launch is enqueued (all threads, all devices).  A replay by
 * ntt_batch_exec_graph counts the kernel nodes of its graph; launches that
 * a caller records into its own stream capture count once, at capture, and
 * replays of that graph are not seen.  The difference across a call is the
 * number of GPU kernels the call ran.  Never fails; needs no GPU. */
uint64_t ntt_launch_count(void);

/* ------------------------------------------------------------------ plans */

/* Create a plan for length N modulo m (Eq. 2/3 with w = 2^(ord_m(2)/N),
 * Sec. I; the multiplicative inverse of N mod m (Appendix A) as N^(m-2),
 * m prime).  Validates that m is prime and that ord_m(2) is a power of two
 * (Prop. 2), and that N is a power of two dividing ord_m(2) (Sec. I).
 * Supported lengths: 1 <= N <= 2^20 (the largest order of 2 among the
 * supported primes is 2^19 for 32-bit words and 2^20 for 64-bit words).
 * Builds the twiddle table {2^e mod m} on the host by doubling and uploads it
 * once to the current device; it stays resident.  Synchronous.
 * Lengths above one thread block (2^14 for 32-bit words, 2^13 for 64-bit)
 * use the plan's scratch: calls with such a plan must not overlap on the GPU
 * (issue them on one stream, or use one plan per stream); other plans have
 * no such restriction.
 * Errors: NTT_ERR_MODULUS, NTT_ERR_LENGTH, NTT_ERR_WORD, NTT_ERR_OOM,
 * NTT_ERR_CUDA, NTT_ERR_ARG (out == NULL). */
ntt_status ntt_plan(uint64_t m, uint32_t N, ntt_plan_t *out);

/* Release a plan and its device memory.  The caller must ensure no queued
 * work still uses it.  NULL is ignored. */
void ntt_plan_destroy(ntt_plan_t plan);

typedef struct {
    uint64_t m;          /* modulus */
    uint32_t N;          /* transform length */
    uint32_t log2N;
    uint64_t n_max;      /* ord_m(2) */
    uint64_t omega;      /* w = 2^(n_max/N) mod m */
    uint64_t n_inv;      /* N^-1 mod m */
    uint32_t word_bits;  /* 32 or 64 */
    uint32_t four_step;  /* 1 when N exceeds one thread block and the split path is used */
    uint32_t wave;       /* pairs per scratch wave of the split path (0 if unused) */
    uint32_t twist;      /* 1 when the split path (convolutions and natural-order transforms) uses
                            the four-step twist form, 0 for row-dependent twiddles */
    uint32_t block;      /* whole sequences: threads per block of the fused convolution kernel
                            (512, or 256 below the longest whole length); 0 on the split path */
    uint32_t small_max;  /* lengths of one warp's row (2^10 for 32-bit words, 2^9 for 64-bit):
                            conv_circular on contiguous pairs runs batches up to this size with one
                            thread block per pair instead of one warp per pair (too few pairs to fill
                            the GPU); 0 for longer lengths */
} ntt_plan_info_t;

/* Fill *info with the plan's parameters.  Errors: NTT_ERR_ARG. */
ntt_status ntt_plan_get_info(ntt_plan_t plan, ntt_plan_info_t *info);

/* 32 or 64 (the word type of every buffer used with this plan); 0 if plan is NULL. */
int ntt_plan_word_bits(ntt_plan_t plan);

/* ------------------------------------------------------------ transforms */

/* Forward transform of Eq. 2 on `batch` sequences: X_dev[b][u] =
 * < sum_t x_dev[b][t] * w^{ut} >_m, natural order.  Errors: NTT_ERR_ARG
 * (NULL pointer or batch == 0), NTT_ERR_CUDA. */
ntt_status ntt_forward(ntt_plan_t plan, const void *x_dev, void *X_dev, size_t batch, ntt_stream_t stream);

/* Inverse transform of Eq. 3 including the factor N^-1: x_dev[b][t] =
 * < N^-1 sum_u X_dev[b][u] * w^{<-ut>_N} >_m.  Errors as ntt_forward. */
ntt_status ntt_inverse(ntt_plan_t plan, const void *X_dev, void *x_dev, size_t batch, ntt_stream_t stream);

/* ---------------------------------------------------------- convolutions */

/* Circular convolution (Eq. 1) of `batch` pairs by the convolution theorem:
 * forward transforms of f and g, pointwise product <F(u) G(u)>_m, inverse
 * transform with N^-1 (Sec. I), fused on the device.  h_dev may alias f_dev
 * or g_dev.  Lengths above one thread block use the plan's scratch in waves.
 * Errors: NTT_ERR_ARG, NTT_ERR_CUDA. */
ntt_status conv_circular(ntt_plan_t plan, const void *f_dev, const void *g_dev, void *h_dev,
                         size_t batch, ntt_stream_t stream);

/* The same result computed in the plain form, one kernel launch per
 * butterfly stage over the whole batch (2 log2 N + 2 launches), with every
 * stage reading and writing device memory.  Kept as the comparison baseline
 * for the fused form.  work_dev must hold 2 * batch * N words of scratch
 * (caller-owned).  Errors: NTT_ERR_ARG, NTT_ERR_CUDA. */
ntt_status conv_circular_plain(ntt_plan_t plan, const void *f_dev, const void *g_dev, void *h_dev,
                               size_t batch, void *work_dev, ntt_stream_t stream);

/* conv_circular with the inputs and output in HOST memory (pageable or
 * page-locked).  The library copies f and g to the device, convolves and
 * copies h back in chunks of 32-48 MB of input, ordered after `stream`'s
 * earlier work, on three internal streams (inbound copies, convolutions,
 * outbound copies) so that those steps of different chunks overlap.  Device
 * staging memory (4 slots x 3 chunks, about 300 MB at most) is allocated on
 * first use and kept by the plan.  With page-locked buffers (cudaHostAlloc /
 * cudaHostRegister), which the GPU can address over the C2C link, and
 * whole-sequence lengths, a batch whose f, g and h total at most 96 MB is
 * instead read and written in place by the kernels (no copies: lower latency
 * for small batches; larger batches are faster through the copy pipeline).
 * The environment variable NTT_HOST_DIRECT=p (0..100) overrides that choice
 * and sends p percent of the pairs in place, the rest through the copies.
 * Returns after h_host is complete (synchronises `stream`).  Errors:
 * NTT_ERR_ARG, NTT_ERR_OOM, NTT_ERR_CUDA. */
ntt_status conv_circular_host(ntt_plan_t plan, const void *f_host, const void *g_host, void *h_host,
                              size_t batch, ntt_stream_t stream);

/* One convolution of an uneven batch: sequences f, g, h of length N (device
 * pointers, caller-owned). */
typedef struct {
    const void *f;
    const void *g;
    void *h;
    uint32_t N;
    uint32_t reserved;
} ntt_conv_desc;

/* Convolve `count` independent pairs of (possibly) different power-of-two
 * lengths modulo one prime m.  Equivalent to ntt_batch_plan + ntt_batch_exec
 * + ntt_batch_destroy, with the batch plan cached by the library for the
 * last (m, descriptor list) seen on this thread.  Errors as ntt_plan and
 * conv_circular. */
ntt_status conv_batched(uint64_t m, const ntt_conv_desc *descs, size_t count, ntt_stream_t stream);

/* Build a reusable execution plan for an uneven batch: groups the
 * descriptors by length, builds the per-length plans and device work lists,
 * picks each length's schedule (from the autotune table when one is loaded),
 * and allocates the scratch it needs.  Synchronous.  The descriptor array is
 * copied; the pointers it holds must stay valid while the batch plan is
 * executed. */
ntt_status ntt_batch_plan(uint64_t m, const ntt_conv_desc *descs, size_t count, ntt_batch_t *out);

/* Enqueue every convolution of the batch plan on `stream` (the persistent
 * launch of the short lengths and the other length classes' launches run on
 * two forked internal streams joined back into `stream`).  Capturable in a
 * CUDA graph. */
ntt_status ntt_batch_exec(ntt_batch_t batch, ntt_stream_t stream);

/* Capture ntt_batch_exec into a CUDA graph once (first call) and replay it on
 * `stream` (every call). */
ntt_status ntt_batch_exec_graph(ntt_batch_t batch, ntt_stream_t stream);

void ntt_batch_destroy(ntt_batch_t batch);

/* -------------------------------------------------------------- autotuning */

typedef struct {
    uint32_t wave;          /* split path: chosen pairs per scratch wave (0 for whole sequences) */
    uint32_t default_wave;  /* the heuristic choice (4 rows per SM, or 256 MB of scratch if more) */
    uint32_t twist;         /* split path: chosen form, 1 the four-step twist, 0 row-dependent twiddles */
    uint32_t default_twist; /* the heuristic form */
    double ms;              /* time of one convolution call over `batch` pairs with the choice */
    double default_ms;      /* the same with the heuristic schedule (0 if not measured) */
    uint32_t block;         /* whole sequences: chosen threads per block of the fused kernel */
    uint32_t default_block; /* the untuned choice: 256 for column/row lengths below the longest, else 512 */
    uint32_t persist;       /* whole sequences: 1 when a batch plan should run the length inside its
                               persistent launch, 0 as a launch of its own */
    uint32_t default_persist;  /* 1 for lengths that fit one warp, else 0 */
    double persist_ms;      /* a batch of `batch` pairs with the length in the persistent launch */
    double own_launch_ms;   /* the same batch with the length as its own launch (0 if not measured) */
} ntt_tune_result;

/* Time the candidate schedules of `batch` pairs of length N modulo m on the
 * current GPU and record the fastest for (GPU name, word size, log2 N);
 * plans and batch plans created afterwards use it.
 *  - Split path (N above one block): both forms (the four-step twist, or
 *    row-dependent twiddles) times the pairs per scratch wave (powers of
 *    two, the heuristic, all pairs).
 *  - Whole sequences: the fused kernel's threads per block (512, or 256 --
 *    half the rows and shared memory per block, two blocks per SM -- except
 *    at the longest whole length), and for lengths above one warp's
 *    (column/row lengths) whether a batch plan runs them inside its single
 *    persistent launch or as a launch of their own.
 * Synchronous; allocates its own buffers.  Errors: as ntt_plan,
 * NTT_ERR_OOM, NTT_ERR_CUDA. */
ntt_status ntt_autotune(uint64_t m, uint32_t N, size_t batch, ntt_tune_result *out);

/* Write / read the recorded schedules as JSON ({"schedules": [...]}, one
 * entry per GPU name, word size and log2 N, with the fields wave, twist,
 * block, persist and ms; entries without block / persist take the
 * defaults).  Loading adds to (and overrides) the recorded table.
 * Errors: NTT_ERR_ARG. */
ntt_status ntt_autotune_save(const char *path);
ntt_status ntt_autotune_load(const char *path);

/* ---------------------------------------------------------------- serving */

/* A convolution server: a background thread that admits requests of
 * different power-of-two lengths against a fixed device-memory pool and
 * batches them continuously.  A new batch (requests grouped by length, one
 * fused launch per length) leaves on a free stream slot as soon as pool
 * memory allows, while earlier batches are still on the GPU, so their copies
 * and kernels overlap.  Plans and twiddle tables of every length up to
 * 2^max_log2N stay resident.  Each request needs 3 N words of pool memory
 * (f, g, h) from admission until its result is back in host memory.  The
 * paper defines only the convolution; the server is the library's own. */
typedef struct ntt_server_s *ntt_server_t;

typedef struct {
    uint64_t pool_bytes;    /* device memory for in-flight requests */
    uint32_t streams;       /* batches in flight at once (stream slots) */
    uint32_t max_batch;     /* requests per batch at most */
    uint32_t max_log2N;     /* longest admissible length 2^max_log2N */
    uint32_t flags;         /* NTT_SERVER_STAGE_ALL: copy every request through the pool */
} ntt_server_config;

/* Requests whose three buffers the GPU can address (page-locked host memory,
 * device or managed memory) are "direct": the kernels read f, g and write h
 * in place through the batch's descriptor list, with no copies and no pool
 * memory.  Other requests (pageable memory), or all of them with this flag,
 * are staged: copied into a pool block, convolved, copied back. */
#define NTT_SERVER_STAGE_ALL 1u

typedef struct {
    uint64_t submitted, completed, rejected, batches;
    uint64_t pool_bytes, peak_pool_bytes;
    uint32_t max_inflight_batches, reserved;
    double p50_us, p99_us, mean_us, max_us;   /* submit -> result in host memory */
    uint64_t direct;        /* completed requests that ran in place (no pool, no copies) */
} ntt_server_stats;

/* Create a server for modulus m on the current device (allocates the pool,
 * per-slot streams, descriptor buffers and split-path scratch; builds the
 * plans).  Errors: as ntt_plan, NTT_ERR_ARG, NTT_ERR_OOM. */
ntt_status ntt_server_create(uint64_t m, const ntt_server_config *cfg, ntt_server_t *out);

/* Queue h = f (*) g of length N (Eq. 1).  f, g, h are pointers of N words
 * each -- host memory (page-locked memory runs direct, see above; pageable
 * memory is staged) or device memory -- that must stay valid until
 * ntt_server_wait returns for *id.  Thread-safe; returns at once.
 * Errors: NTT_ERR_ARG, NTT_ERR_LENGTH (N above 2^max_log2N),
 * NTT_ERR_ADMISSION (a staged request whose 3 N words exceed the whole pool;
 * *id is still set). */
ntt_status ntt_server_submit(ntt_server_t srv, const void *f_host, const void *g_host, void *h_host,
                             uint32_t N, uint64_t *id);

/* Block until request id has completed (its result is in h_host) or
 * timeout_ms elapses; then forget the request.  Returns the request's status,
 * or NTT_ERR_TIMEOUT (the request stays queryable). */
ntt_status ntt_server_wait(ntt_server_t srv, uint64_t id, uint32_t timeout_ms);

/* Block until no request is queued or on the GPU.  NTT_ERR_TIMEOUT on expiry. */
ntt_status ntt_server_drain(ntt_server_t srv, uint32_t timeout_ms);

/* Counters and latency percentiles since creation or the last reset. */
ntt_status ntt_server_get_stats(ntt_server_t srv, ntt_server_stats *out);
ntt_status ntt_server_reset_stats(ntt_server_t srv);

/* Stop the worker after all queued requests finish, and free the server. */
void ntt_server_destroy(ntt_server_t srv);

/* --------------------------------------------------- no-allocation variant */

/* Size in bytes of the library's static split-path scratch (per GPU). */
#define NTT_NOALLOC_SCRATCH_BYTES (16u << 20)

/* conv_circular for callers that cannot allocate device memory when they
 * convolve: programs whose device memory belongs to another allocator (a
 * framework pool that has reserved the GPU, a fixed memory map) and loops
 * that cannot afford cudaMalloc/cudaFree, which may synchronise the device.
 * The paper has no counterpart; this is an interface choice of the library.
 *
 * Same arguments, layout, ownership and result as conv_circular.  The call
 * allocates nothing: lengths that fit one thread block need no scratch, and
 * longer ones (the split path) use one static array of
 * NTT_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library
 * holds until the process exits.  The batch is processed in waves of
 * floor(16 MiB / (2 N word_bytes)) pairs; a length whose single pair needs
 * more than the array is rejected with NTT_ERR_ARG (no supported length
 * does today).  The plan must be created beforehand (ntt_plan allocates).
 *
 * The first call on a device is a set-up step: it looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, and
 * under CUDA's lazy module loading that lookup is what loads the array's
 * module and reserves its 16 MiB, which may synchronise the device.  Make
 * one call during initialisation (a batch of one pair is enough), and
 * before any stream capture; later calls only reuse the cached address.
 * The address, like every plan, does not survive cudaDeviceReset.  The
 * plan's device must be the current device (NTT_ERR_ARG otherwise).
 * All calls on a device share the one array and it keeps the last call's
 * contents; nothing in it needs clearing, but calls whose work overlaps on
 * the GPU (other streams, other threads) race on it and must be serialised
 * by the caller.
 * Errors: NTT_ERR_ARG, NTT_ERR_CUDA. */
ntt_status conv_circular_noalloc(ntt_plan_t plan, const void *f_dev, const void *g_dev, void *h_dev,
                                 size_t batch, ntt_stream_t stream);

/* ---------------------------------------------- exact integer convolution */

/* Exact (non-modular) circular convolution of signed 64-bit sequences,
 *     h(j) = sum_k f(k) g(<j-k>_N)   over the integers       (Eq. 1, no modulus)
 * -- the exact digital filtering of Sec. I -- from the modular convolutions
 * of several Rader primes (prime factors of Fermat numbers, Sec. III-A /
 * Table 1, whose multiplicative order of 2 the length N divides) and the
 * Chinese remainder theorem. */
#define NTT_EXACT_MAX_PRIMES 4

typedef struct ntt_exact_s *ntt_exact_t;          /* opaque, owned by the library */

typedef struct {
    uint32_t N;
    uint32_t bound_bits;            /* the caller's bound: every |h(j)| < 2^bound_bits */
    uint32_t nprimes;               /* primes used (<= NTT_EXACT_MAX_PRIMES) */
    uint32_t word_bits[NTT_EXACT_MAX_PRIMES];
    uint32_t reserved;
    uint64_t primes[NTT_EXACT_MAX_PRIMES];
    double capacity_bits;           /* log2 of the product M of the primes (> bound_bits + 1) */
    uint64_t wave;                  /* pairs per scratch wave */
} ntt_exact_info_t;

/* Plan exact convolutions of length N (a power of two) whose outputs all
 * satisfy |h(j)| < 2^bound_bits, 1 <= bound_bits <= 63 (e.g. bound_bits =
 * log2 N + bits(max|f|) + bits(max|g|)).  The plan takes the cheapest primes
 * (32-bit words first) whose product M reaches 2^(bound_bits + 1), creates
 * one modular plan per prime and owns device scratch for a wave of pairs
 * (at most 512 MiB of residues).
 * Errors: NTT_ERR_ARG (NULL out), NTT_ERR_LENGTH (N not a power of two, or
 * the primes that admit N cannot cover the bound), NTT_ERR_RANGE
 * (bound_bits outside 1..63), NTT_ERR_OOM, NTT_ERR_CUDA. */
ntt_status ntt_exact_plan(uint32_t N, uint32_t bound_bits, ntt_exact_t *out);

/* Fill *info.  Errors: NTT_ERR_ARG. */
ntt_status ntt_exact_get_info(ntt_exact_t plan, ntt_exact_info_t *info);

/* h_dev[b][j] = sum_k f_dev[b][k] g_dev[b][<j-k>_N] for b < batch: signed
 * 64-bit words, row-major [batch][N], device memory owned by the caller; h
 * may alias neither f nor g.  Exact whenever the plan's bound holds; an
 * output beyond it comes back as its residue modulo M in (-M/2, M/2].
 * Asynchronous on `stream`; a plan serves one call at a time.
 * Errors: NTT_ERR_ARG, NTT_ERR_CUDA. */
ntt_status conv_exact(ntt_exact_t plan, const int64_t *f_dev, const int64_t *g_dev, int64_t *h_dev, size_t batch,
                      ntt_stream_t stream);

/* Release the plan, its modular plans and its scratch.  NULL is a no-op. */
void ntt_exact_destroy(ntt_exact_t plan);

/* ------------------------------------------------- strict bit-shift form */

/* Circular convolution modulo a Rader prime m that divides F_4 = 2^16 + 1
 * (m = 65537, N <= 32) or F_5 = 2^32 + 1 (m = 641 or 6700417, N <= 64):
 * the regime where the transform of Eq. 2 / Eq. 3 is literally "bit-shifts,
 * additions and modulo" (Sec. I; Sec. III-A, Prop. 2), because every
 * twiddle 2^e has e < 2^t.
 *   mode NTT_SHIFT_STRICT: the transform runs modulo F_t; each twiddle is a
 *     shift followed by the multiply-free reduction lo - hi (2^(2^t) = -1),
 *     N^-1 is a shift; only the N pointwise products multiply; the result is
 *     reduced modulo m at the end.
 *   mode NTT_SHIFT_SHOUP: the same kernel with every twiddle applied as a
 *     Shoup product modulo m (the multiply form), for comparison.
 * f_dev, g_dev: uint32 residues in [0, m), row-major [batch][N]; h_dev:
 * uint32, canonical; device memory owned by the caller; h may not alias f
 * or g.  Identical results in both modes (and to conv_circular).
 * Errors: NTT_ERR_ARG, NTT_ERR_MODULUS (m not a prime factor of F_4 or F_5),
 * NTT_ERR_LENGTH (N not a power of two in 2..ord_m(2)), NTT_ERR_CUDA. */
#define NTT_SHIFT_STRICT 0
#define NTT_SHIFT_SHOUP 1
ntt_status conv_circular_shift(uint64_t m, uint32_t N, const uint32_t *f_dev, const uint32_t *g_dev, uint32_t *h_dev,
                               size_t batch, int mode, ntt_stream_t stream);

/* ----------------------------------------------------------------- checks */

/* Count the words of `count` words at data_dev (word size of the plan) that
 * are >= m; returns NTT_ERR_RANGE if any, NTT_OK otherwise.  Synchronous.
 * *bad (optional) receives the count. */
ntt_status ntt_check_range(ntt_plan_t plan, const void *data_dev, size_t count, uint64_t *bad, ntt_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* NTT_GB300_H */
