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


// ModDown (+ rescale) of the accumulators of B items (ks_down.cu)
template <bool RESC>
void ks_moddown(Ctx &c, int level, int B, const ItemPtrs &ip, bool first_pass_done);

}  // namespace ppst
