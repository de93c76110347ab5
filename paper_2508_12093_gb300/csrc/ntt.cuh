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
