// ks.cuh -- definitions shared by the key-switching translation units (ks.cu:
// tensor, automorphism, ModUp and the inner product; ks_down.cu: ModDown and
// the rescale). The scheme is described at the top of ks.cu.
#pragma once
#include <atomic>

#include "bulk.cuh"
#include "ntt.cuh"

namespace ppst {

constexpr int BMAX = 16;

// per-item ciphertext pointers of a batched launch
struct ItemPtrs {
    const uint64_t *in0[BMAX];
    const uint64_t *in1[BMAX];
    uint64_t *out[BMAX];
};

// workspace slices of item `it`
struct Ws {
    size_t d2, ext, acc, conv, top;  // item strides in words
};
static inline Ws ws_strides(const Ctx &c)
{
    const size_t N = c.N, q = c.L + 1, e = c.ext_rows();
    return Ws{q * N, (size_t)c.dnum * e * N, 2 * e * N, 2 * q * N, 2 * N};
}

// ---------------------------------------------------------------------------
// 2. ModUp fused into the COLS pass
// ---------------------------------------------------------------------------
// sum_{i < A} src[i N + pos] f[i] mod q for the E words of this thread (A known at
// compile time: fully unrolled, all loads independent); A = 0: runtime count `a`
template <int A, int E, int T>
__device__ __forceinline__ void bconv_words(uint64_t (&x)[E], const uint64_t *__restrict__ src, const uint64_t *f,
                                            int a, int N, int C, int h, const PrimeC &pt)
{
    if (A > 0) {
        uint64_t fr[A > 0 ? A : 1];
#pragma unroll
        for (int i = 0; i < A; i++) fr[i] = f[i];
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t pos = (size_t)(h + T * k) * C;
            Acc4 acc{0, 0, 0, 0};
#pragma unroll
            for (int i = 0; i < A; i++) mac4(acc, src[(size_t)i * N + pos], fr[i]);
            x[k] = mont_redc(acc4_hi(acc), acc4_lo(acc), pt.q, pt.qinv);
        }
    } else {
#pragma unroll
        for (int k = 0; k < E; k++) {
            const size_t pos = (size_t)(h + T * k) * C;
            Acc4 acc{0, 0, 0, 0};
#pragma unroll 1
            for (int i = 0; i < a; i++) mac4(acc, src[(size_t)i * N + pos], f[i]);
            x[k] = mont_redc(acc4_hi(acc), acc4_lo(acc), pt.q, pt.qinv);
        }
    }
}

// calls f(std::integral_constant<int, a>) for the digit sizes with a compiled fast path, else f(0)
template <class F>
void dispatch_a(int a, F &&f)
{
    switch (a) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    default: f(std::integral_constant<int, 0>{}); break;
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
inline dim3 grid_s(const Ctx &c, int S, int sub, int rows) { return dim3((c.N >> S) / sub, rows); }

// runs f(S, SUB) for pass size s and the block shape pass_sub picks for `rows` limbs
template <class F>
void dispatch_pass(const Ctx &c, int s, int rows, F &&f)
{
    dispatch_s(s, [&](auto sv) {
        dispatch_sub<decltype(sv)::value>(pass_sub(c, decltype(sv)::value, rows), [&](auto bv) { f(sv, bv); });
    });
}


// ---------------------------------------------------------------------------
// 256-point CHUNKS pass with 8 words per thread (one warp per chunk), shared by
// the inner product (ks.cu) and ModDown's last pass (ks_down.cu)
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

// ModDown (+ rescale) of the accumulators of B items (ks_down.cu)
template <bool RESC>
void ks_moddown(Ctx &c, int level, int B, const ItemPtrs &ip);

}  // namespace ppst
