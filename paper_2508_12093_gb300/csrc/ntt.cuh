// ntt.cuh -- device building blocks of the limb NTT (see ntt.cu for the scheme).
//
// A pass runs M-point sub-transforms (M = 2^S) of an N-point negacyclic
// transform: the COLS pass the columns (stride C = N / M), the CHUNKS pass the
// contiguous chunks of M words. A thread holds E = 2^ceil(S/2) words; the
// long-distance stages act on words h + T k (T = M / E threads per
// sub-transform), then one shared-memory transpose, then the short-distance
// stages act on words E h + k. The cores below take the E words in registers
// (load layout) and return them in the store layout; kernels supply their own
// loads and stores, which is how the key-switching kernels fuse base
// conversion into the load and the key inner product into the store.
#pragma once
#include <type_traits>
#include <utility>

#include "ctx.cuh"

namespace ppst {

// launch on the context's stream (configuration and arguments as for <<<...>>>)
template <class... KArgs, class... Args>
inline void launch_on(Ctx &c, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    PPST_CUDA(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
}

template <int S, int SUB_ = 16>
struct PassShape {
    static constexpr int M = 1 << S;
    static constexpr int A = (S + 1) / 2;  // register stages before the transpose
    static constexpr int E = 1 << A;       // words per thread
    static constexpr int T = M / E;        // threads per sub-transform
    static constexpr int SUB = SUB_;       // sub-transforms per block (4, 8 or 16)
    static constexpr int THREADS = SUB * T;
    static constexpr int SMEM_WORDS = SUB * (M + M / E);  // padded transpose buffer
    static constexpr int MIN_BLOCKS = THREADS >= 256 ? 3 : (THREADS >= 128 ? 4 : 8);
};

// COLS passes keep row p of column `sub` at p SUB + sub (SUB = 16: a half-warp
// reads 16 columns of one row) or, for SUB < 16, at (p + p / E) SUB + sub: the
// pad every E rows keeps both transposes free of bank conflicts (a half-warp
// then touches 16 / SUB rows that are either consecutive or E apart)
template <int S, int SUB>
__device__ __forceinline__ int cols_smem(int p)
{
    typedef PassShape<S, SUB> P;
    return SUB == 16 ? p * 16 : (p + p / P::E) * SUB;
}

// forward lazy butterfly: X, Y in [0, 4q) -> [0, 4q)
__device__ __forceinline__ void bfly_fwd(uint64_t &X, uint64_t &Y, const Tw &w, uint64_t q, uint64_t q2)
{
    uint64_t x = X >= q2 ? X - q2 : X;
    uint64_t t = shoup(Y, w.w, w.s, q);
    X = x + t;
    Y = x - t + q2;
}

// inverse lazy butterfly: X, Y in [0, 2q) -> [0, 2q)
__device__ __forceinline__ void bfly_inv(uint64_t &X, uint64_t &Y, const Tw &w, uint64_t q, uint64_t q2)
{
    uint64_t s = X + Y;
    uint64_t d = X - Y + q2;
    X = s >= q2 ? s - q2 : s;
    Y = shoup(d, w.w, w.s, q);
}

__device__ __forceinline__ uint64_t reduce4q(uint64_t x, uint64_t q)
{
    uint64_t q2 = 2 * q;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

__device__ __forceinline__ Tw ldtw(const Tw *p)
{
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    return Tw{v.x, v.y};
}

// Storage order of the evaluation domain. The transform's natural output
// order is bit-reversed (word n holds a(psi^(2 brv(n) + 1))); within each chunk
// of M = 2^floor(logN/2) words, the word the CHUNKS pass computes at natural
// position E h + k is stored at h + T k, so that a thread's words are spread
// with stride T and every evaluation-domain access of the CHUNKS pass (keys,
// accumulators, outputs) is coalesced across the threads h.
__host__ __device__ __forceinline__ uint32_t eval_natural(uint32_t a, int logN)
{
    const int S = logN / 2, A = (S + 1) / 2;
    const uint32_t M = 1u << S, E = 1u << A, T = M / E;
    const uint32_t g = a >> S, r = a & (M - 1), h = r % T, k = r / T;
    return (g << S) + E * h + k;
}
__host__ __device__ __forceinline__ uint32_t eval_address(uint32_t n, int logN)
{
    const int S = logN / 2, A = (S + 1) / 2;
    const uint32_t M = 1u << S, E = 1u << A, T = M / E;
    const uint32_t g = n >> S, s = n & (M - 1), h = s / E, k = s % E;
    return (g << S) + h + T * k;
}

// thread coordinates of a pass: COLS -> (sub = column in block, h), CHUNKS -> (h, sub = chunk in block)
template <int S, bool COLS, int SUB = 16>
__device__ __forceinline__ void pass_coords(int &h, int &sub)
{
    typedef PassShape<S, SUB> P;
    if (COLS) {
        sub = threadIdx.x % P::SUB;
        h = threadIdx.x / P::SUB;
    } else {
        h = threadIdx.x % P::T;
        sub = threadIdx.x / P::T;
    }
}

// ---- forward, COLS pass: stages with m = 1 .. M/2 (distances in rows) ----
template <int S, int SUB = 16>
__device__ __forceinline__ void cols_fwd_core(uint64_t (&x)[PassShape<S>::E], uint64_t *sm, int h, int sub,
                                              const Tw *__restrict__ T, uint64_t q)
{
    typedef PassShape<S, SUB> P;
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int s = P::A - 1; s >= 0; s--) {
        const int d = P::T << s;
        const int mg = P::M / (2 * d);
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            bfly_fwd(x[k], x[k + (1 << s)], ldtw(T + mg + (k >> (s + 1))), q, q2);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) sm[cols_smem<S, SUB>(h + P::T * k) + sub] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = sm[cols_smem<S, SUB>(P::E * h + k) + sub];
#pragma unroll
    for (int d = P::T / 2; d >= 1; d >>= 1) {
        const int mg = P::M / (2 * d);
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            bfly_fwd(x[k], x[k + d], ldtw(T + mg + (P::E * h + k) / (2 * d)), q, q2);
        }
    }
}

// ---- forward, CHUNKS pass: stages with m = N/M .. N/2 on chunk g ----
template <int S>
__device__ __forceinline__ void chunks_fwd_core(uint64_t (&x)[PassShape<S>::E], uint64_t *sm, int h, int sub, int g,
                                                int N, const Tw *__restrict__ T, uint64_t q)
{
    typedef PassShape<S> P;
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int s = P::A - 1; s >= 0; s--) {
        const int d = P::T << s;
        const int mg = N / (2 * d);
        const int ib = g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            bfly_fwd(x[k], x[k + (1 << s)], ldtw(T + mg + ib + (k >> (s + 1))), q, q2);
        }
    }
    uint64_t *ssub = sm + sub * (P::M + P::M / P::E);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) {
        const int e = h + P::T * k;
        ssub[e + e / P::E] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = ssub[(P::E + 1) * h + k];
#pragma unroll
    for (int d = P::T / 2; d >= 1; d >>= 1) {
        const int mg = N / (2 * d);
        const int ib = g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            bfly_fwd(x[k], x[k + d], ldtw(T + mg + ib + (P::E * h + k) / (2 * d)), q, q2);
        }
    }
}

// ---- inverse, CHUNKS pass (first inverse pass): words E h + k in, h + T k out ----
template <int S>
__device__ __forceinline__ void chunks_inv_core(uint64_t (&x)[PassShape<S>::E], uint64_t *sm, int h, int sub, int g,
                                                int N, const Tw *__restrict__ T, uint64_t q)
{
    typedef PassShape<S> P;
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int d = 1; d <= P::T / 2; d <<= 1) {
        const int mg = N / (2 * d);
        const int ib = g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            bfly_inv(x[k], x[k + d], ldtw(T + mg + ib + (P::E * h + k) / (2 * d)), q, q2);
        }
    }
    uint64_t *ssub = sm + sub * (P::M + P::M / P::E);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) ssub[(P::E + 1) * h + k] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) {
        const int e = h + P::T * k;
        x[k] = ssub[e + e / P::E];
    }
#pragma unroll
    for (int s = 0; s < P::A; s++) {
        const int d = P::T << s;
        const int mg = N / (2 * d);
        const int ib = g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            bfly_inv(x[k], x[k + (1 << s)], ldtw(T + mg + ib + (k >> (s + 1))), q, q2);
        }
    }
}

// ---- inverse, COLS pass (last inverse pass): rows E h + k in, h + T k out ----
template <int S, int SUB = 16>
__device__ __forceinline__ void cols_inv_core(uint64_t (&x)[PassShape<S>::E], uint64_t *sm, int h, int sub,
                                              const Tw *__restrict__ T, uint64_t q)
{
    typedef PassShape<S, SUB> P;
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int d = 1; d <= P::T / 2; d <<= 1) {
        const int mg = P::M / (2 * d);
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            bfly_inv(x[k], x[k + d], ldtw(T + mg + (P::E * h + k) / (2 * d)), q, q2);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) sm[cols_smem<S, SUB>(P::E * h + k) + sub] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = sm[cols_smem<S, SUB>(h + P::T * k) + sub];
#pragma unroll
    for (int s = 0; s < P::A; s++) {
        const int d = P::T << s;
        const int mg = P::M / (2 * d);
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            bfly_inv(x[k], x[k + (1 << s)], ldtw(T + mg + (k >> (s + 1))), q, q2);
        }
    }
}

// ---------------------------------------------------------------------------
// 256-point passes with 8 words per thread (N = 2^15, 2^16): CHUNKS passes with one
// warp per chunk (the inner product, ModDown, the inverse transforms), COLS passes
// with SUB columns per block (ModUp, ModDown)
// ---------------------------------------------------------------------------
// XOR swizzle of a chunk's 256 words: the three layouts a warp uses (h + 32 k,
// 32 (h >> 2) + 4 k + (h & 3), 8 h + k) each touch 16 distinct 8-byte banks
// per half-warp
__device__ __forceinline__ int swz8(int p) { return p ^ ((p >> 4) & 7) ^ (((p >> 5) & 1) << 3); }

// where natural word p of a 256-word chunk is stored in the evaluation domain
// (the 16-word storage order of ntt.cuh: E h + k -> h + 16 k)
__device__ __forceinline__ int addr16(int p) { return (p >> 4) + ((p & 15) << 4); }

// The two exchanges by warp shuffles instead of shared memory (a variant the
// autotuner measures). A -> B swaps lane bits 2..4 with register bits 0..2
// (three butterfly-pattern rounds of shfl.xor 4, 8, 16); B -> C transposes, for
// each register parity, lane bits 0..1 with register bits 1..2 (rounds 1, 2).
// Each round sends the half of the registers the partner needs and keeps the rest.
__device__ __forceinline__ void xchg_ab_shfl(uint64_t (&x)[8], int h)
{
#pragma unroll
    for (int bit = 0; bit < 3; bit++) {
        const int s = 4 << bit, sv = 1 << bit;
        const bool up = h & s;
#pragma unroll
        for (int a = 0; a < 8; a++) {
            if (a & sv) continue;
            const uint64_t send = up ? x[a] : x[a | sv];
            const uint64_t recv = __shfl_xor_sync(0xffffffffu, send, s);
            if (up) x[a] = recv;
            else x[a | sv] = recv;
        }
    }
}

__device__ __forceinline__ void xchg_bc_shfl(uint64_t (&x)[8], int h)
{
    uint64_t y[8];
#pragma unroll
    for (int b = 0; b < 2; b++) {
        uint64_t m[4] = {x[b], x[2 + b], x[4 + b], x[6 + b]};
#pragma unroll
        for (int s = 1; s <= 2; s <<= 1) {
            const bool up = h & s;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                if (a & s) continue;
                const uint64_t send = up ? m[a] : m[a | s];
                const uint64_t recv = __shfl_xor_sync(0xffffffffu, send, s);
                if (up) m[a] = recv;
                else m[a | s] = recv;
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) y[r + 4 * b] = m[r];
    }
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = y[k];
}

// the three butterfly rounds of a 256-point forward pass with 8 words per thread:
// words h + 32 k in, 8 h + k out. tw(m, j) is the twiddle of group j of the
// stage with m groups (distance 128 / m); xab / xbc move the words from layout
// A (h + 32 k) to B (32 (h >> 2) + 4 k + (h & 3)) and from B to C (8 h + k).
template <class TwF, class XAB, class XBC>
__device__ __forceinline__ void fwd_rounds8(uint64_t (&x)[8], int h, TwF &&tw, XAB &&xab, XBC &&xbc, uint64_t q)
{
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int s = 2; s >= 0; s--) {  // distance 32 << s: m = 4 >> s groups, group k >> (s + 1)
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_fwd(x[k], x[k + (1 << s)], tw(4 >> s, k >> (s + 1)), q, q2);
        }
    }
    xab(x);
    const int hh = h >> 2;
#pragma unroll
    for (int s = 2; s >= 0; s--) {  // distance 4 << s: m = 32 >> s, group (hh << (2 - s)) | (k >> (s + 1))
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_fwd(x[k], x[k + (1 << s)], tw(32 >> s, (hh << (2 - s)) | (k >> (s + 1))), q, q2);
        }
    }
    xbc(x);
#pragma unroll
    for (int s = 1; s >= 0; s--) {  // distance 1 << s: m = 128 >> s, group (8 h + k) >> (s + 1)
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_fwd(x[k], x[k + (1 << s)], tw(128 >> s, (8 * h + k) >> (s + 1)), q, q2);
        }
    }
}

// forward CHUNKS pass of a chunk (one warp), 8 words per thread; the exchanges go
// through the warp's shared-memory buffer `ex` or (SHFL) through shuffles; tw(m, j)
// is psi^brv of m (N / 256 + g) + j for chunk g
template <bool SHFL, class TwF>
__device__ __forceinline__ void chunks_fwd_core8(uint64_t (&x)[8], uint64_t *ex, int h, TwF &&tw, uint64_t q)
{
    const int hh = h >> 2, hl = h & 3;
    auto xab = [&](uint64_t(&v)[8]) {
        if (SHFL) {
            xchg_ab_shfl(v, h);
            return;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) ex[swz8(h + 32 * k)] = v[k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = ex[swz8(32 * hh + 4 * k + hl)];
    };
    auto xbc = [&](uint64_t(&v)[8]) {
        if (SHFL) {
            xchg_bc_shfl(v, h);
            return;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) ex[swz8(32 * hh + 4 * k + hl)] = v[k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = ex[swz8(8 * h + k)];
    };
    fwd_rounds8(x, h, tw, xab, xbc, q);
}

// the three butterfly rounds of a 256-point inverse (Gentleman-Sande) pass with 8
// words per thread: words 8 h + k in (layout C), h + 32 k out (layout A), distances
// 1, 2 | 4, 8, 16 | 32, 64, 128; xcb / xba move the words from C to B and from B
// to A; tw(m, j) as for the forward rounds (inverse twiddles)
template <class TwF, class XCB, class XBA>
__device__ __forceinline__ void inv_rounds8(uint64_t (&x)[8], int h, TwF &&tw, XCB &&xcb, XBA &&xba, uint64_t q)
{
    const uint64_t q2 = 2 * q;
#pragma unroll
    for (int s = 0; s <= 1; s++) {  // distance 1 << s: m = 128 >> s, group (8 h + k) >> (s + 1)
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_inv(x[k], x[k + (1 << s)], tw(128 >> s, (8 * h + k) >> (s + 1)), q, q2);
        }
    }
    xcb(x);
    const int hh = h >> 2;
#pragma unroll
    for (int s = 0; s <= 2; s++) {  // distance 4 << s: m = 32 >> s, group (hh << (2 - s)) | (k >> (s + 1))
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_inv(x[k], x[k + (1 << s)], tw(32 >> s, (hh << (2 - s)) | (k >> (s + 1))), q, q2);
        }
    }
    xba(x);
#pragma unroll
    for (int s = 0; s <= 2; s++) {  // distance 32 << s: m = 4 >> s, group k >> (s + 1)
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if ((k >> s) & 1) continue;
            bfly_inv(x[k], x[k + (1 << s)], tw(4 >> s, k >> (s + 1)), q, q2);
        }
    }
}

// inverse CHUNKS pass of a chunk (one warp), 8 words per thread, exchanges through the
// warp's swizzled shared-memory buffer; tw(m, j) is psi^-brv of m (N / 256 + g) + j
template <class TwF>
__device__ __forceinline__ void chunks_inv_core8(uint64_t (&x)[8], uint64_t *ex, int h, TwF &&tw, uint64_t q)
{
    const int hh = h >> 2, hl = h & 3;
    auto xcb = [&](uint64_t(&v)[8]) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) ex[swz8(8 * h + k)] = v[k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = ex[swz8(32 * hh + 4 * k + hl)];
    };
    auto xba = [&](uint64_t(&v)[8]) {
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) ex[swz8(32 * hh + 4 * k + hl)] = v[k];
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = ex[swz8(h + 32 * k)];
    };
    inv_rounds8(x, h, tw, xcb, xba, q);
}

// forward COLS pass, 8 words per thread: SUB columns per block, column `sub` held by
// the 32 threads h; row p of column sub sits at (p SUB + sub) ^ (((p >> 3) & (16 / SUB - 1)) SUB)
// in the block's buffer (conflict-free for the three layouts, checked exhaustively);
// tw(m, j) is psi^brv of m + j (the first stages of the transform)
template <int SUB>
__device__ __forceinline__ int cols8_smem(int p, int sub)
{
    return (p * SUB + sub) ^ (((p >> 3) & (16 / SUB - 1)) * SUB);
}

template <int SUB, class TwF>
__device__ __forceinline__ void cols_fwd_core8(uint64_t (&x)[8], uint64_t *sm, int h, int sub, TwF &&tw, uint64_t q)
{
    const int hh = h >> 2, hl = h & 3;
    auto xab = [&](uint64_t(&v)[8]) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) sm[cols8_smem<SUB>(h + 32 * k, sub)] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = sm[cols8_smem<SUB>(32 * hh + 4 * k + hl, sub)];
    };
    auto xbc = [&](uint64_t(&v)[8]) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) sm[cols8_smem<SUB>(32 * hh + 4 * k + hl, sub)] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = sm[cols8_smem<SUB>(8 * h + k, sub)];
    };
    fwd_rounds8(x, h, tw, xab, xbc, q);
}

// calls f(std::integral_constant<int, sub>) for the sub-transforms per block of
// a pass of size 2^S: 16, 8 or 4 at S = 8 (N = 2^15, 2^16), 16 or 4 below
// (where 8 is rounded down to 4: fewer kernels to compile)
template <int S, class F>
void dispatch_sub(int sub, F &&f)
{
    if (sub == 16) f(std::integral_constant<int, 16>{});
    else if (S == 8 && sub == 8) f(std::integral_constant<int, S == 8 ? 8 : 4>{});
    else f(std::integral_constant<int, 4>{});
}

// calls f(std::integral_constant<int, s>) for the pass sizes of N = 2^10 .. 2^16
template <class F>
void dispatch_s(int s, F &&f)
{
    switch (s) {
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    default: throw_err(PPST_E_ARG, "unsupported ring degree for the NTT");
    }
}

inline int ntt_s_rows(int logN) { return (logN + 1) / 2; }  // COLS pass: log2 R
inline int ntt_s_chunk(int logN) { return logN / 2; }      // CHUNKS pass: log2 C

// sub-transforms per block of a pass over `rows` limbs: the largest of 16, 8, 4
// whose grid still has at least the context's minimum number of blocks (small
// grids, at low levels, spread over more SMs with smaller blocks)
inline int pass_sub(const Ctx &c, int S, int rows)
{
    const long per16 = (long)(c.N >> S) / 16 * rows;
    if (per16 >= (long)c.pass_min_blocks) return 16;
    if (2 * per16 >= (long)c.pass_min_blocks) return 8;
    return 4;
}

}  // namespace ppst
