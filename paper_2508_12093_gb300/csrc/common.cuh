// common.cuh -- shared definitions of the GB300 RNS-CKKS library.
//
// 64-bit modular arithmetic on the device, written from the published methods:
//  * Shoup's multiplication by a constant w with precomputed w' = floor(w 2^64 / q)
//    (V. Shoup, NTL): x w - floor(x w' / 2^64) q lies in [0, 2q) for any x < 2^64;
//  * Montgomery reduction (P. Montgomery, 1985) in its signed form: for
//    T = hi 2^64 + lo < q 2^64, m = lo q^-1 mod 2^64, T 2^-64 = hi - mulhi(m, q)
//    (mod q), already in [0, q) after one conditional add;
//  * Harvey's lazy butterflies (D. Harvey, 2014) keep NTT values in [0, 4q).
// All primes are below 2^61, so 4q < 2^64.
#pragma once
#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

namespace ppst {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// per-prime constants (device copy lives in Ctx::d_pc)
// ---------------------------------------------------------------------------
struct PrimeC {
    uint64_t q;
    uint64_t qinv;      // q^-1 mod 2^64
    uint64_t r2;        // 2^128 mod q (to leave the Montgomery domain scaled by 2^-64)
    uint64_t ninv;      // N^-1 mod q
    uint64_t ninv_sh;   // Shoup companion of ninv
    uint64_t w64;       // floor(2^64 / q): Shoup companion of 1, reduces a 64-bit word
};

// a twiddle and its Shoup companion, loaded as one 16-byte word
struct __align__(16) Tw {
    uint64_t w, s;
};

__host__ __device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t q) { return x >= q ? x - q : x; }

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((u128)a * b) >> 64);
#endif
}

// x * w mod q in [0, 2q), w' = floor(w 2^64 / q)
__host__ __device__ __forceinline__ uint64_t shoup(uint64_t x, uint64_t w, uint64_t wsh, uint64_t q)
{
    return x * w - mulhi64(x, wsh) * q;
}

// (hi 2^64 + lo) 2^-64 mod q, fully reduced; requires hi < q
__host__ __device__ __forceinline__ uint64_t mont_redc(uint64_t hi, uint64_t lo, uint64_t q, uint64_t qinv)
{
    uint64_t m = lo * qinv;
    uint64_t mh = mulhi64(m, q);
    uint64_t r = hi - mh;
    return hi < mh ? r + q : r;
}

// the full 128-bit product a b = hi 2^64 + lo. On the device the four 32 x 32-bit
// partial products are summed with carry chains once, instead of computing
// the low and the high 64 bits separately (both need the cross terms).
__host__ __device__ __forceinline__ void mul128(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi)
{
#ifdef __CUDA_ARCH__
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    uint32_t w0, w1, w2, w3;
    asm("mul.lo.u32 %0, %4, %6;\n\t"
        "mul.hi.u32 %1, %4, %6;\n\t"
        "mul.lo.u32 %2, %5, %7;\n\t"
        "mul.hi.u32 %3, %5, %7;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    lo = ((uint64_t)w1 << 32) | w0;
    hi = ((uint64_t)w3 << 32) | w2;
#else
    lo = a * b;
    hi = mulhi64(a, b);
#endif
}

// a b 2^-64 mod q for a, b < q
__host__ __device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t q, uint64_t qinv)
{
    uint64_t lo, hi;
    mul128(a, b, lo, hi);
    return mont_redc(hi, lo, q, qinv);
}

// a b mod q for a, b < q (two Montgomery reductions)
__host__ __device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const PrimeC &p)
{
    return mont_mul(mont_mul(a, b, p.q, p.qinv), p.r2, p.q, p.qinv);
}

__host__ __device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) { return csub(a + b, q); }
__host__ __device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulate of a*b
struct Acc128 {
    uint64_t lo, hi;
};
// acc += a b (mod 2^128). On the device the four 32 x 32-bit partial products
// are accumulated straight into the four 32-bit words of acc with carry chains
// (schoolbook multiplication): no separate 64-bit high and low products, which
// would each recompute the cross terms. Operands enter as their 32-bit halves
// (the halves of a 64-bit register pair, so no moves are needed).
#define PPST_MAC4_ASM                                                                   \
    "mad.lo.cc.u32 %0, %4, %6, %0;\n\t"   /* + a0 b0 + a1 b1 2^64 */                  \
    "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"                                              \
    "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"                                              \
    "madc.hi.u32 %3, %5, %7, %3;\n\t"                                                 \
    "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"   /* + a0 b1 2^32 */                          \
    "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"                                              \
    "addc.u32 %3, %3, 0;\n\t"                                                         \
    "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"   /* + a1 b0 2^32 */                          \
    "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"                                              \
    "addc.u32 %3, %3, 0;"

__host__ __device__ __forceinline__ void mac(Acc128 &acc, uint64_t a, uint64_t b)
{
#ifdef __CUDA_ARCH__
    uint32_t w0 = (uint32_t)acc.lo, w1 = (uint32_t)(acc.lo >> 32), w2 = (uint32_t)acc.hi,
             w3 = (uint32_t)(acc.hi >> 32);
    asm(PPST_MAC4_ASM
        : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3)
        : "r"((uint32_t)a), "r"((uint32_t)(a >> 32)), "r"((uint32_t)b), "r"((uint32_t)(b >> 32)));
    acc.lo = ((uint64_t)w1 << 32) | w0;
    acc.hi = ((uint64_t)w3 << 32) | w2;
#else
    uint64_t l = a * b;
    uint64_t h = mulhi64(a, b);
    acc.lo += l;
    acc.hi += h + (acc.lo < l);
#endif
}

#ifdef __CUDACC__
// a 128-bit accumulator kept as four 32-bit words on the device, so that a
// chain of multiply-accumulates never repacks 64-bit halves between steps
struct Acc4 {
    uint32_t w0, w1, w2, w3;
};
__device__ __forceinline__ void mac4(Acc4 &a, uint64_t x, uint64_t y)
{
    asm(PPST_MAC4_ASM
        : "+r"(a.w0), "+r"(a.w1), "+r"(a.w2), "+r"(a.w3)
        : "r"((uint32_t)x), "r"((uint32_t)(x >> 32)), "r"((uint32_t)y), "r"((uint32_t)(y >> 32)));
}
__device__ __forceinline__ uint64_t acc4_lo(const Acc4 &a) { return ((uint64_t)a.w1 << 32) | a.w0; }
__device__ __forceinline__ uint64_t acc4_hi(const Acc4 &a) { return ((uint64_t)a.w3 << 32) | a.w2; }
#endif

// ---------------------------------------------------------------------------
// ChaCha20 block function (RFC 8439 Sec. 2.3), keyed by SplitMix64 of a seed.
// Used on the host (secret key) and in the sampling kernels.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t rotl32(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

#define PPST_QR(a, b, c, d)                 \
    a += b; d ^= a; d = rotl32(d, 16);      \
    c += d; b ^= c; b = rotl32(b, 12);      \
    a += b; d ^= a; d = rotl32(d, 8);       \
    c += d; b ^= c; b = rotl32(b, 7);

struct ChaChaKey {
    uint32_t k[8];
};

__host__ __device__ inline void chacha20_block(const ChaChaKey &key, uint32_t counter, uint32_t n0, uint32_t n1,
                                               uint32_t n2, uint32_t out[16])
{
    uint32_t x0 = 0x61707865u, x1 = 0x3320646eu, x2 = 0x79622d32u, x3 = 0x6b206574u;
    uint32_t x4 = key.k[0], x5 = key.k[1], x6 = key.k[2], x7 = key.k[3];
    uint32_t x8 = key.k[4], x9 = key.k[5], x10 = key.k[6], x11 = key.k[7];
    uint32_t x12 = counter, x13 = n0, x14 = n1, x15 = n2;
#pragma unroll 1
    for (int r = 0; r < 10; r++) {
        PPST_QR(x0, x4, x8, x12) PPST_QR(x1, x5, x9, x13) PPST_QR(x2, x6, x10, x14) PPST_QR(x3, x7, x11, x15)
        PPST_QR(x0, x5, x10, x15) PPST_QR(x1, x6, x11, x12) PPST_QR(x2, x7, x8, x13) PPST_QR(x3, x4, x9, x14)
    }
    out[0] = x0 + 0x61707865u; out[1] = x1 + 0x3320646eu; out[2] = x2 + 0x79622d32u; out[3] = x3 + 0x6b206574u;
    out[4] = x4 + key.k[0]; out[5] = x5 + key.k[1]; out[6] = x6 + key.k[2]; out[7] = x7 + key.k[3];
    out[8] = x8 + key.k[4]; out[9] = x9 + key.k[5]; out[10] = x10 + key.k[6]; out[11] = x11 + key.k[7];
    out[12] = x12 + counter; out[13] = x13 + n0; out[14] = x14 + n1; out[15] = x15 + n2;
}
#undef PPST_QR

// SplitMix64 (Steele, Lea, Flood 2014)
__host__ __device__ inline uint64_t splitmix64_next(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline ChaChaKey chacha_key_from_seed(uint64_t seed)
{
    ChaChaKey k;
    uint64_t s = seed;
    for (int i = 0; i < 4; i++) {
        uint64_t z = splitmix64_next(s);
        k.k[2 * i] = (uint32_t)z;
        k.k[2 * i + 1] = (uint32_t)(z >> 32);
    }
    return k;
}

// stream purposes (nonce word 0) -- one independent stream per use
enum Purpose : uint32_t {
    P_SECRET = 1, P_SWK_A = 2, P_SWK_E = 3, P_ENC_U = 4, P_ENC_E0 = 5, P_ENC_E1 = 6, P_PK_A = 7, P_PK_E = 8
};

// ---------------------------------------------------------------------------
// limb maps: which words and which prime a batched launch processes.
// Batch element b: poly = b / per_poly, i = b % per_poly;
//   words  base + poly * poly_stride + i * N;
//   prime  i < nq ? first_q + i : p_base + (i - nq).
// ---------------------------------------------------------------------------
struct LimbMap {
    uint64_t *base;
    size_t poly_stride;
    int per_poly, npoly, nq, first_q, p_base;
    __host__ __device__ int count() const { return per_poly * npoly; }
    __host__ __device__ uint64_t *ptr(int b, int N) const
    {
        return base + (size_t)(b / per_poly) * poly_stride + (size_t)(b % per_poly) * N;
    }
    __host__ __device__ int prime(int b) const
    {
        int i = b % per_poly;
        return i < nq ? first_q + i : p_base + (i - nq);
    }
};

// per-limb constant vectors passed by value (<= 64 limbs)
constexpr int MAXL = 64;
struct ConstVec {
    uint64_t c[MAXL];
    uint64_t sh[MAXL];
};

}  // namespace ppst
