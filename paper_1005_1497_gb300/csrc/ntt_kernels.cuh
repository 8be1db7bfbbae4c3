// ntt_kernels.cuh -- kernels of the exact digital convolution, templated on
// the word type W (uint32_t / uint64_t) and on log2 N.
#pragma once

#include "ntt_core.cuh"

namespace ntt {

constexpr int BLOCK = 512;                 // threads of every row-kernel block

template <typename W> struct LRMax;        // longest row one block transforms
template <> struct LRMax<uint32_t> { static constexpr int v = 14; };
template <> struct LRMax<uint64_t> { static constexpr int v = 13; };

// One convolution of an uneven batch, as seen by the device.
template <typename W> struct DevDesc {
    const W *f;
    const W *g;
    W *h;
};

// Arguments of the row kernels.  For a whole-sequence launch (L == LR) row
// rho is pair pair0 + rho of the batch (contiguous arrays f, g, h or the
// descriptor list).  For the split path (L > LR) rho counts rows of the
// current wave inside the scratch arrays f (= F~, overwritten by H~) and g.
template <typename W> struct RowArgs {
    const W *f;
    const W *g;
    W *h;
    const DevDesc<W> *descs;
    long long nrows;
    long long pair0;
    const W *tw;
    ModC<W> c;
};

template <typename W, int L, int LR>
struct RowShape {
    using G = Geo<W, LR>;
    static constexpr int GPC = BLOCK / G::T;   // rows in flight per block
    static constexpr size_t smem(int ns) { return (size_t)GPC * ns * G::ROWP * sizeof(W); }
};

// Fused convolution rows: forward transforms of f and g, pointwise product
// with N^-1, transposed transform back, all in registers and shared memory.
template <typename W, int L, int LR, int SRC>
__global__ void __launch_bounds__(BLOCK, 1) k_conv_rows(RowArgs<W> a)
{
    using G = Geo<W, LR>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, LR>::GPC;
    constexpr bool FULL = (L == LR);
    constexpr uint32_t N = 1u << L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *S = reinterpret_cast<W *>(smem_raw) + (size_t)gid * 2 * G::ROWP;
    const uint32_t b0 = G::base(0, tau);
    constexpr int lo0 = G::lo(0);

    for (long long rho = (long long)blockIdx.x * GPC + gid; rho < a.nrows; rho += (long long)gridDim.x * GPC) {
        const W *fp, *gp;
        W *hp;
        uint32_t rowoff;
        if constexpr (FULL) {
            const long long pair = a.pair0 + rho;
            if constexpr (SRC == 1) {
                const DevDesc<W> d = a.descs[pair];
                fp = d.f; gp = d.g; hp = d.h;
            } else {
                fp = a.f + (size_t)pair * N; gp = a.g + (size_t)pair * N; hp = a.h + (size_t)pair * N;
            }
            rowoff = 0;
        } else {
            const long long pw = rho >> (L - LR);
            const uint32_t row = (uint32_t)rho & ((1u << (L - LR)) - 1u);
            const size_t off = (size_t)pw * N + ((size_t)row << LR);
            fp = a.f + off; gp = a.g + off; hp = a.h + off;
            rowoff = row << LR;
        }
        W v[2][R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            v[0][k] = fp[b0 + ((uint32_t)k << lo0)];
            v[1][k] = gp[b0 + ((uint32_t)k << lo0)];
        }
        fwd_all<W, L, LR, 0, 2>(v, rowoff, tau, S, gid, a.tw, a.c);
        W hv[R];
#pragma unroll
        for (int k = 0; k < R; ++k) hv[k] = pointwise(v[0][k], v[1][k], a.c);
        inv_all<W, L, LR, G::NPASS - 1>(hv, rowoff, tau, S, gid, a.tw, a.c);
        if constexpr (FULL) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const uint32_t x = b0 + ((uint32_t)k << lo0);
                hp[(N - x) & (N - 1u)] = csub<W>(hv[k], a.c.m);
            }
        } else {
#pragma unroll
            for (int k = 0; k < R; ++k) hp[b0 + ((uint32_t)k << lo0)] = hv[k];
        }
    }
}

// Natural-order forward transform (Eq. 2) or inverse transform (Eq. 3) of
// whole sequences (L <= LR_max).  The forward tree leaves X(brv(x)) at x; a
// shared-memory pass puts it back in natural order.  The inverse is
// N^-1 R F: same forward tree, output index <-u>_N, factor N^-1.
template <typename W> struct NttArgs {
    const W *x;
    W *y;
    long long batch;
    const W *tw;
    ModC<W> c;
};

template <typename W, int L, bool INV>
__global__ void __launch_bounds__(BLOCK, 1) k_ntt_rows(NttArgs<W> a)
{
    using G = Geo<W, L>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, L>::GPC;
    constexpr uint32_t N = 1u << L;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *S = reinterpret_cast<W *>(smem_raw) + (size_t)gid * G::ROWP;
    const uint32_t b0 = G::base(0, tau), bl = G::base(last, tau);
    constexpr int lo0 = G::lo(0), lol = G::lo(last);
    const W scale = INV ? a.c.ninv : (W)1;
    const W scalep = INV ? a.c.ninvp : a.c.onep;

    for (long long rho = (long long)blockIdx.x * GPC + gid; rho < a.batch; rho += (long long)gridDim.x * GPC) {
        const W *xp = a.x + (size_t)rho * N;
        W *yp = a.y + (size_t)rho * N;
        W v[1][R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[0][k] = xp[b0 + ((uint32_t)k << lo0)];
        fwd_all<W, L, L, 0, 1>(v, 0u, tau, S, gid, a.tw, a.c);
        group_sync<T>(gid);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t x = bl + ((uint32_t)k << lol);
            const uint32_t u = L == 0 ? 0u : (__brev(x) >> (32 - L));
            S[G::pad(u)] = v[0][k];
        }
        group_sync<T>(gid);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t u = b0 + ((uint32_t)k << lo0);
            W val = csub<W>(shoup<W>(S[G::pad(u)], scale, scalep, a.c.m), a.c.m);
            yp[INV ? ((N - u) & (N - 1u)) : u] = val;
        }
    }
}

// Split path for L > LR: "column" transforms of the top LC = L - LR index
// bits.  Element (c, k) of a sequence is x = c + k 2^LR (c < 2^LR, k < 2^LC);
// every level of the top bits has node index k >> (bits below), the same for
// all columns.  NS sequences per thread (f and g).
template <typename W> struct ColArgs {
    const W *src0;      // SRC == 0: contiguous batch base of sequence 0 (f)
    const W *src1;      // ... of sequence 1 (g)
    const DevDesc<W> *descs;   // SRC == 1
    W *dst0;            // scratch of the wave (F~), [pairs][N]
    W *dst1;            // scratch (G~)
    W *out;             // cols_inv, DST == 0: contiguous output base
    long long npairs;   // pairs in this wave
    long long pair0;    // first pair of the wave in the batch / descriptor list
    const W *tw;
    ModC<W> c;
};

template <typename W, int L, int LR, int J>
__device__ __forceinline__ void col_fwd_level(W (&v)[1 << (L - LR)], const W *__restrict__ tw, const ModC<W> &c)
{
    // J = register bit, element bit b = LR + J, global level L - 1 - b
    constexpr int RC = 1 << (L - LR);
    constexpr int dg = L - LR - 1 - J;
    if constexpr (dg == 0) {
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            if (k & (1 << J)) continue;
            ct_bfly_one<W>(v[k], v[k | (1 << J)], c);
        }
    } else {
        constexpr int CNT = RC >> (J + 1);
        W z[CNT], zp[CNT];
        load_tw<W, CNT>(tw, 0u, z, zp);
#pragma unroll
        for (int k = 0; k < RC; ++k) {
            if (k & (1 << J)) continue;
            ct_bfly<W>(v[k], v[k | (1 << J)], z[k >> (J + 1)], zp[k >> (J + 1)], c);
        }
    }
}

template <typename W, int L, int LR, int J>
__device__ __forceinline__ void col_fwd_levels(W (&v)[1 << (L - LR)], const W *__restrict__ tw, const ModC<W> &c)
{
    if constexpr (J >= 0) {
        col_fwd_level<W, L, LR, J>(v, tw, c);
        col_fwd_levels<W, L, LR, J - 1>(v, tw, c);
    }
}

template <typename W, int L, int LR, int J>
__device__ __forceinline__ void col_inv_levels(W (&v)[1 << (L - LR)], const W *__restrict__ tw, const ModC<W> &c)
{
    constexpr int RC = 1 << (L - LR);
    if constexpr (J < L - LR) {
        constexpr int dg = L - LR - 1 - J;
        if constexpr (dg == 0) {
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                if (k & (1 << J)) continue;
                gs_bfly_one<W>(v[k], v[k | (1 << J)], c);
            }
        } else {
            constexpr int CNT = RC >> (J + 1);
            W z[CNT], zp[CNT];
            load_tw<W, CNT>(tw, 0u, z, zp);
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                if (k & (1 << J)) continue;
                gs_bfly<W>(v[k], v[k | (1 << J)], z[k >> (J + 1)], zp[k >> (J + 1)], c);
            }
        }
        col_inv_levels<W, L, LR, J + 1>(v, tw, c);
    }
}

template <typename W, int L, int LR, int NS, int SRC>
__global__ void __launch_bounds__(256) k_cols_fwd(ColArgs<W> a)
{
    constexpr int RC = 1 << (L - LR);
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LR) return;
    const long long pw = idx >> LR;
    const uint32_t col = (uint32_t)idx & ((1u << LR) - 1u);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const W *src;
        if constexpr (SRC == 1) {
            const DevDesc<W> d = a.descs[a.pair0 + pw];
            src = s == 0 ? d.f : d.g;
        } else {
            src = (s == 0 ? a.src0 : a.src1) + (size_t)(a.pair0 + pw) * N;
        }
        W *dst = (s == 0 ? a.dst0 : a.dst1) + (size_t)pw * N;
        W v[RC];
#pragma unroll
        for (int k = 0; k < RC; ++k) v[k] = src[col + ((uint32_t)k << LR)];
        col_fwd_levels<W, L, LR, L - LR - 1>(v, a.tw, a.c);
#pragma unroll
        for (int k = 0; k < RC; ++k) dst[col + ((uint32_t)k << LR)] = v[k];
    }
}

// Transposed top levels of the split path, then the output stage: index
// <-x>_N, canonical residue.  DST 0: contiguous out; 1: descriptor h.
template <typename W, int L, int LR, int DST>
__global__ void __launch_bounds__(256) k_cols_inv(ColArgs<W> a)
{
    constexpr int RC = 1 << (L - LR);
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.npairs << LR) return;
    const long long pw = idx >> LR;
    const uint32_t col = (uint32_t)idx & ((1u << LR) - 1u);
    const W *src = a.dst0 + (size_t)pw * N;
    W *out;
    if constexpr (DST == 1) out = a.descs[a.pair0 + pw].h;
    else out = a.out + (size_t)(a.pair0 + pw) * N;
    W v[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) v[k] = src[col + ((uint32_t)k << LR)];
    col_inv_levels<W, L, LR, 0>(v, a.tw, a.c);
#pragma unroll
    for (int k = 0; k < RC; ++k) {
        const uint32_t x = col + ((uint32_t)k << LR);
        out[(N - x) & (N - 1u)] = csub<W>(v[k], a.c.m);
    }
}

// Forward row levels of the split path (single sequence, in place in scratch).
template <typename W, int L, int LR>
__global__ void __launch_bounds__(BLOCK, 1) k_rows_fwd(RowArgs<W> a)
{
    using G = Geo<W, LR>;
    constexpr int T = G::T, R = G::R, GPC = RowShape<W, L, LR>::GPC;
    constexpr uint32_t N = 1u << L;
    constexpr int last = G::NPASS - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gid = threadIdx.x / T;
    const uint32_t tau = threadIdx.x % T;
    W *S = reinterpret_cast<W *>(smem_raw) + (size_t)gid * G::ROWP;
    const uint32_t b0 = G::base(0, tau), bl = G::base(last, tau);
    for (long long rho = (long long)blockIdx.x * GPC + gid; rho < a.nrows; rho += (long long)gridDim.x * GPC) {
        const long long pw = rho >> (L - LR);
        const uint32_t row = (uint32_t)rho & ((1u << (L - LR)) - 1u);
        W *p = const_cast<W *>(a.f) + (size_t)pw * N + ((size_t)row << LR);
        W v[1][R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[0][k] = p[b0 + ((uint32_t)k << G::lo(0))];
        fwd_all<W, L, LR, 0, 1>(v, row << LR, tau, S, gid, a.tw, a.c);
#pragma unroll
        for (int k = 0; k < R; ++k) p[bl + ((uint32_t)k << G::lo(last))] = v[0][k];
    }
}

// Bit-reversal gather of a split-path spectrum: y[u] = X(u) from the tree
// order (X(brv(x)) at x); INV applies <-u>_N and N^-1.  Canonical outputs.
template <typename W, int L, bool INV>
__global__ void k_bitrev_out(const W *__restrict__ src, W *__restrict__ dst, long long batch, ModC<W> c)
{
    constexpr uint32_t N = 1u << L;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch << L) return;
    const long long b = idx >> L;
    const uint32_t t = (uint32_t)idx & (N - 1u);
    const uint32_t u = INV ? ((N - t) & (N - 1u)) : t;
    const uint32_t x = __brev(u) >> (32 - L);
    const W scale = INV ? c.ninv : (W)1;
    const W scalep = INV ? c.ninvp : c.onep;
    dst[idx] = csub<W>(shoup<W>(src[(size_t)b * N + x], scale, scalep, c.m), c.m);
}

// ---------------------------------------------------- plain per-stage form

// One forward tree level over the whole batch of f and g: work = [2][batch][N].
template <typename W>
__global__ void k_plain_fwd(const W *__restrict__ f, const W *__restrict__ g, W *work, long long batch,
                            int L, int d, const W *__restrict__ tw, ModC<W> c)
{
    const long long half = 1ll << (L - 1);
    const long long total = 2 * batch * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long s = i / (batch * half);
        const long long r = i - s * batch * half;
        const long long pair = r >> (L - 1);
        const uint32_t beta = (uint32_t)(r & (half - 1));
        const int sh = L - 1 - d;
        const uint32_t node = beta >> sh;
        const uint32_t i0 = (node << (sh + 1)) | (beta & ((1u << sh) - 1u));
        const uint32_t i1 = i0 + (1u << sh);
        W *dst = work + ((size_t)s * batch + pair) * ((size_t)half * 2);
        W x0, x1;
        if (d == 0) {
            const W *sp = (s == 0 ? f : g) + (size_t)pair * ((size_t)half * 2);
            x0 = sp[i0]; x1 = sp[i1];
            ct_bfly_one<W>(x0, x1, c);
        } else {
            x0 = dst[i0]; x1 = dst[i1];
            const W z = tw[2 * node], zp = tw[2 * node + 1];
            ct_bfly<W>(x0, x1, z, zp, c);
        }
        dst[i0] = x0; dst[i1] = x1;
    }
}

template <typename W>
__global__ void k_plain_pointwise(W *work, long long batch, int L, ModC<W> c)
{
    const long long n = batch << L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        work[i] = pointwise(work[i], work[n + i], c);
}

template <typename W>
__global__ void k_plain_inv(W *work, long long batch, int L, int d, const W *__restrict__ tw, ModC<W> c)
{
    const long long half = 1ll << (L - 1);
    const long long total = batch * half;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long pair = i >> (L - 1);
        const uint32_t beta = (uint32_t)(i & (half - 1));
        const int sh = L - 1 - d;
        const uint32_t node = beta >> sh;
        const uint32_t i0 = (node << (sh + 1)) | (beta & ((1u << sh) - 1u));
        const uint32_t i1 = i0 + (1u << sh);
        W *p = work + (size_t)pair * ((size_t)half * 2);
        W x0 = p[i0], x1 = p[i1];
        if (d == 0) gs_bfly_one<W>(x0, x1, c);
        else gs_bfly<W>(x0, x1, tw[2 * node], tw[2 * node + 1], c);
        p[i0] = x0; p[i1] = x1;
    }
}

template <typename W>
__global__ void k_plain_final(const W *__restrict__ work, W *h, long long batch, int L, ModC<W> c)
{
    const long long n = batch << L;
    const uint32_t N = 1u << L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long pair = i >> L;
        const uint32_t x = (uint32_t)i & (N - 1u);
        h[(size_t)pair * N + ((N - x) & (N - 1u))] = csub<W>(work[i], c.m);
    }
}

// Words >= m in data[0 .. n).
template <typename W>
__global__ void k_check_range(const W *__restrict__ data, long long n, W m, unsigned long long *bad)
{
    unsigned long long cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        cnt += data[i] >= m ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

}  // namespace ntt
