// ks.cu -- fused, batched hybrid key switching (the HMult and rotation hot path).
//
// Key switching of d (level l, dnum digits of alpha primes, K special primes)
// is computed as three fused stages, none of which writes an evaluation-domain
// digit to HBM:
//   1. inverse NTT of d, its first pass fused into the tensor product (or the
//      automorphism), its final N^-1 carrying (Q_j / q_i)^-1 of the limb's
//      digit: the first factor of ModUp's base conversion comes for free;
//   2. k_modup_cols: for every digit j and target limb e outside it, the load
//      of the COLS transform pass computes the base conversion
//      sum_i y_i (Q_j / q_i) mod t_e on the fly (the digit's alpha limbs stay in
//      L2), then runs the pass;
//   3. k_inner_chunks: one block per (item, target limb e, 16 chunks) loops over
//      the digits, finishes the transform in registers (the digit's own limbs
//      are taken from d in the evaluation domain instead) and accumulates both
//      key polynomials; the twiddles of prime e are reused by every digit. The
//      8-word form (k_inner8) also runs ModDown's first inverse pass on the rows
//      ModDown takes to the coefficient domain (the P rows; in HMult the top
//      limb l too, after forming d_l + acc_l P^-1), so ModDown starts at their
//      COLS pass.
// ModDown (and, in HMult, the rescale after it) is fused the same way. For
// limb i < l of the HMult output:
//   out_i = (d_i + acc_i P^-1 - NTT(conv_i P^-1 + [top]_centred mod q_i)) q_l^-1
// which equals ModDown followed by rescale limb for limb (the transform is
// linear mod q_i), so one forward transform replaces two. `top` is limb l of
// the ModDown output in the coefficient domain:
//   top = INTT(d_l + acc_l P^-1) - conv_l P^-1.
// All values are exact residues: results are bit-identical to the unfused
// sequence (tensor, ModUp, NTT, inner product, ModDown, rescale).
//
// Batching: up to BMAX independent ciphertexts (same level, same key) go
// through each stage in one launch. The item is the fastest-varying block
// index of the inner-product kernel, so the blocks that read the same key
// tile run back to back and the tile is fetched from HBM once per batch.
#include "ks.cuh"

namespace ppst {

// ---------------------------------------------------------------------------
// 0. batched tensor / automorphism into the key-switch input buffers
// ---------------------------------------------------------------------------
// tensor (d0, d1 -> t[item]; d2 -> d2n[item] and, after the pass, d2[item]) and
// automorphism (sigma_g(c0) -> out[item].c0; sigma_g(c1) -> d2n[item], d2[item]),
// each fused with the first (CHUNKS) pass of the inverse transform of d2: a block
// owns SUB chunks of one limb, so each thread's E words (stored at h + T k,
// natural E h + k) are exactly what the inverse CHUNKS pass takes; d2 leaves in
// that pass's output layout for the COLS pass.
template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_tensor_ic(ItemPtrs ip, uint64_t *__restrict__ d2, uint64_t *__restrict__ d2n, const PrimeC *__restrict__ pc,
                const Tw *__restrict__ twi, int logN, int nl, size_t pstride, size_t d2_stride)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int it = blockIdx.y / nl, i = blockIdx.y - it * nl;
    const PrimeC p = pc[i];
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const size_t base = (size_t)i * N + (size_t)g * P::M + h;
    const uint64_t *a = ip.in0[it], *b = ip.in1[it];
    uint64_t *t = ip.out[it];
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) {
        const size_t off = base + P::T * k;
        const uint64_t x0 = a[off], x1 = a[pstride + off], y0 = b[off], y1 = b[pstride + off];
        t[off] = mul_mod(x0, y0, p);
        x[k] = mul_mod(x1, y1, p);
        d2n[it * d2_stride + off] = x[k];
        Acc128 acc{0, 0};
        mac(acc, x0, y1);
        mac(acc, x1, y0);
        t[pstride + off] = mont_mul(mont_redc(acc.hi, acc.lo, p.q, p.qinv), p.r2, p.q, p.qinv);
    }
    chunks_inv_core<S>(x, sm, h, sub, g, N, twi + (size_t)i * N, p.q);
    uint64_t *o = d2 + it * d2_stride + base;
#pragma unroll
    for (int k = 0; k < P::E; k++) o[P::T * k] = x[k];
}

// the tensor product with 8 words per thread (256-point chunks: N = 2^15, 2^16), one
// warp per chunk: the products at the storage addresses of natural words 8 h + k,
// then the first inverse pass of d2, which leaves in natural order (words h + 32 k)
template <int SUB>
__global__ void __launch_bounds__(32 * SUB, SUB == 8 ? 4 : 8)
    k_tensor_ic8(ItemPtrs ip, uint64_t *__restrict__ d2, uint64_t *__restrict__ d2n, const PrimeC *__restrict__ pc,
                 const Tw *__restrict__ twi, int logN, int nl, size_t pstride, size_t d2_stride)
{
    __shared__ uint64_t ex_all[SUB * 256];
    const int N = 1 << logN;
    const int it = blockIdx.y / nl, i = blockIdx.y - it * nl;
    const PrimeC p = pc[i];
    const int h = threadIdx.x & 31, sub = threadIdx.x >> 5;
    const int g = blockIdx.x * SUB + sub;
    const size_t base = (size_t)i * N + (size_t)g * 256;
    const uint64_t *a = ip.in0[it], *b = ip.in1[it];
    uint64_t *t = ip.out[it];
    uint64_t x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const size_t off = base + addr16(8 * h + k);
        const uint64_t x0 = a[off], x1 = a[pstride + off], y0 = b[off], y1 = b[pstride + off];
        t[off] = mul_mod(x0, y0, p);
        x[k] = mul_mod(x1, y1, p);
        d2n[it * d2_stride + off] = x[k];
        Acc128 acc{0, 0};
        mac(acc, x0, y1);
        mac(acc, x1, y0);
        t[pstride + off] = mont_mul(mont_redc(acc.hi, acc.lo, p.q, p.qinv), p.r2, p.q, p.qinv);
    }
    const Tw *T = twi + (size_t)i * N;
    const size_t tg = (size_t)(N >> 8) + g;
    chunks_inv_core8(x, ex_all + sub * 256, h, [&](int m, int j) { return ldtw(T + m * tg + j); }, p.q);
    uint64_t *o = d2 + it * d2_stride + base;
#pragma unroll
    for (int k = 0; k < 8; k++) o[h + 32 * k] = x[k];
}

// blockIdx.y = (item, poly, limb): poly 0 -> out[item].c0, poly 1 -> d2n and (after the pass) d2
template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_automorph_ic(ItemPtrs ip, uint64_t *__restrict__ d2, uint64_t *__restrict__ d2n, const PrimeC *__restrict__ pc,
                   const Tw *__restrict__ twi, int logN, int nl, uint64_t gal, size_t pstride, size_t d2_stride)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int row = blockIdx.y, it = row / (2 * nl), r2 = row - it * 2 * nl, poly = r2 / nl, i = r2 - poly * nl;
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    const size_t o = (size_t)i * N;
    const uint64_t *src = ip.in0[it] + (size_t)poly * pstride + o;
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) {
        // output address g M + h + T k holds natural word n = g M + E h + k; sigma_g moves
        // the evaluation at psi^(2 brv(n) + 1) from psi^(g (2 brv(n) + 1))
        const uint32_t n = (uint32_t)(g * P::M + P::E * h + k);
        const uint32_t bk = __brev(n) >> (32 - logN);
        const uint64_t e = ((2ull * bk + 1) * gal) & (2ull * N - 1);
        x[k] = src[eval_address(__brev((uint32_t)((e - 1) >> 1)) >> (32 - logN), logN)];
    }
    const size_t base = o + (size_t)g * P::M + h;
    if (poly == 0) {  // block-uniform
#pragma unroll
        for (int k = 0; k < P::E; k++) ip.out[it][base + P::T * k] = x[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < P::E; k++) d2n[it * d2_stride + base + P::T * k] = x[k];
    chunks_inv_core<S>(x, sm, h, sub, g, N, twi + (size_t)i * N, pc[i].q);
#pragma unroll
    for (int k = 0; k < P::E; k++) d2[it * d2_stride + base + P::T * k] = x[k];
}

// the automorphism with 8 words per thread (N = 2^15, 2^16), one warp per chunk: the
// Galois permutation into the storage addresses of natural words 8 h + k, then (poly 1)
// the first inverse pass, which leaves in natural order (words h + 32 k)
template <int SUB>
__global__ void __launch_bounds__(32 * SUB, SUB == 8 ? 4 : 8)
    k_automorph_ic8(ItemPtrs ip, uint64_t *__restrict__ d2, uint64_t *__restrict__ d2n,
                    const PrimeC *__restrict__ pc, const Tw *__restrict__ twi, int logN, int nl, uint64_t gal,
                    size_t pstride, size_t d2_stride)
{
    __shared__ uint64_t ex_all[SUB * 256];
    const int N = 1 << logN;
    const int row = blockIdx.y, it = row / (2 * nl), r2 = row - it * 2 * nl, poly = r2 / nl, i = r2 - poly * nl;
    const int h = threadIdx.x & 31, sub = threadIdx.x >> 5;
    const int g = blockIdx.x * SUB + sub;
    const size_t o = (size_t)i * N;
    const uint64_t *src = ip.in0[it] + (size_t)poly * pstride + o;
    uint64_t x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        // natural word n = 256 g + 8 h + k holds the evaluation at psi^(2 brv(n) + 1); sigma_g
        // moves it from psi^(g (2 brv(n) + 1))
        const uint32_t n = (uint32_t)(g * 256 + 8 * h + k);
        const uint32_t bk = __brev(n) >> (32 - logN);
        const uint64_t e = ((2ull * bk + 1) * gal) & (2ull * N - 1);
        x[k] = src[eval_address(__brev((uint32_t)((e - 1) >> 1)) >> (32 - logN), logN)];
    }
    const size_t base = o + (size_t)g * 256;
    if (poly == 0) {  // block-uniform
#pragma unroll
        for (int k = 0; k < 8; k++) ip.out[it][base + addr16(8 * h + k)] = x[k];
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) d2n[it * d2_stride + base + addr16(8 * h + k)] = x[k];
    const Tw *T = twi + (size_t)i * N;
    const size_t tg = (size_t)(N >> 8) + g;
    chunks_inv_core8(x, ex_all + sub * 256, h, [&](int m, int j) { return ldtw(T + m * tg + j); }, pc[i].q);
#pragma unroll
    for (int k = 0; k < 8; k++) d2[it * d2_stride + base + h + 32 * k] = x[k];
}

template <int S, int ALPHA, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, 2)
    k_modup_cols(const uint64_t *__restrict__ y, uint64_t *__restrict__ ext, const uint64_t *__restrict__ ks,
                 DigitOffs offs, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN, int level,
                 int alpha, int L, int K, int nd, size_t ext_stride, Ws ws)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int E_ext = level + 1 + K;
    const int per_item = nd * E_ext;
    const int it = blockIdx.y / per_item, rem = blockIdx.y - it * per_item;
    const int j = rem / E_ext, e = rem - j * E_ext;
    const int lo = j * alpha, hi = min(lo + alpha, level + 1), a = hi - lo;
    if (e >= lo && e < hi) return;  // a digit's own limbs come from d itself (block-uniform)
    const int t = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC pt = pc[t];
    __shared__ uint64_t f[16];
    if (threadIdx.x < a) f[threadIdx.x] = ks[offs.off[j] + 2 * a + (size_t)threadIdx.x * E_ext + e];
    __syncthreads();
    int h, sub;
    pass_coords<S, true, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t x[P::E];
    const uint64_t *yl = y + it * ws.d2 + (size_t)lo * N + g;
    if (ALPHA > 0 && a == ALPHA) bconv_words<ALPHA, P::E, P::T>(x, yl, f, a, N, C, h, pt);
    else bconv_words<0, P::E, P::T>(x, yl, f, a, N, C, h, pt);  // a partial last digit
    cols_fwd_core<S, SUB>(x, sm, h, sub, tw + (size_t)t * N, pt.q);
    uint64_t *out = ext + it * ws.ext + (size_t)j * ext_stride + (size_t)e * N;
#pragma unroll
    for (int k = 0; k < P::E; k++) out[(size_t)(P::E * h + k) * C + g] = x[k];
}

// the same pass with 8 words per thread (N = 2^15, 2^16: 256-row columns): SUB
// columns per block, column `sub` on the 32 threads h; three butterfly rounds with
// two block-wide exchanges through a swizzled shared-memory buffer
template <int ALPHA, int SUB>
__global__ void __launch_bounds__(32 * SUB, SUB == 8 ? 3 : 6)
    k_modup_cols8(const uint64_t *__restrict__ y, uint64_t *__restrict__ ext, const uint64_t *__restrict__ ks,
                  DigitOffs offs, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN, int level,
                  int alpha, int L, int K, int nd, size_t ext_stride, Ws ws)
{
    __shared__ uint64_t sm[SUB * 256];
    const int N = 1 << logN, C = N >> 8;
    const int E_ext = level + 1 + K;
    const int per_item = nd * E_ext;
    const int it = blockIdx.y / per_item, rem = blockIdx.y - it * per_item;
    const int j = rem / E_ext, e = rem - j * E_ext;
    const int lo = j * alpha, hi = min(lo + alpha, level + 1), a = hi - lo;
    if (e >= lo && e < hi) return;  // a digit's own limbs come from d itself (block-uniform)
    const int t = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC pt = pc[t];
    __shared__ uint64_t f[16];
    if (threadIdx.x < a) f[threadIdx.x] = ks[offs.off[j] + 2 * a + (size_t)threadIdx.x * E_ext + e];
    __syncthreads();
    const int sub = threadIdx.x % SUB, h = threadIdx.x / SUB;
    const int g = blockIdx.x * SUB + sub;
    uint64_t x[8];
    const uint64_t *yl = y + it * ws.d2 + (size_t)lo * N + g;
    if (ALPHA > 0 && a == ALPHA) bconv_words<ALPHA, 8, 32>(x, yl, f, a, N, C, h, pt);
    else bconv_words<0, 8, 32>(x, yl, f, a, N, C, h, pt);  // a partial last digit
    const Tw *T = tw + (size_t)t * N;
    cols_fwd_core8<SUB>(x, sm, h, sub, [&](int m, int jj) { return ldtw(T + m + jj); }, pt.q);
    uint64_t *out = ext + it * ws.ext + (size_t)j * ext_stride + (size_t)e * N;
#pragma unroll
    for (int k = 0; k < 8; k++) out[(size_t)(8 * h + k) * C + g] = x[k];
}

// ---------------------------------------------------------------------------
// 3. CHUNKS pass fused with the key inner product
// ---------------------------------------------------------------------------
// A block owns SUB consecutive chunks (one contiguous tile of SUB M words; SUB
// = 4, 8 or 16, chosen per context by the autotuner, 8 by default) of target
// limb e and loops over the digits. The digit tiles and the two key
// tiles of a digit are brought into shared memory by bulk asynchronous copies:
// digit j + 2 and the keys of digit j + 1 are in flight while digit j is
// transformed and accumulated, so the HBM latency is off the critical path.
template <int S, int SUB_>
struct InnerSmem {
    typedef PassShape<S> P;
    static constexpr int SUB = SUB_;             // chunks per block
    static constexpr int MIN_BLOCKS = 16 / SUB_; // blocks per SM the shared memory allows
    static constexpr int THREADS = SUB * P::T;
    static constexpr int TILE = SUB * P::M;      // words per tile
    static constexpr size_t X_OFF = 128;         // after the barriers: two digit tiles
    static constexpr size_t K_OFF = X_OFF + 2 * (size_t)TILE * 8;  // two key tiles
    static constexpr size_t T_OFF = K_OFF + 2 * (size_t)TILE * 8;  // transpose buffer
    static constexpr size_t BYTES = T_OFF + (size_t)SUB * (P::M + P::M / P::E) * 8;
};

template <int S, int SUB>
__global__ void __launch_bounds__(InnerSmem<S, SUB>::THREADS, InnerSmem<S, SUB>::MIN_BLOCKS)
    k_inner_chunks(const uint64_t *__restrict__ ext, const uint64_t *__restrict__ d2n, const uint64_t *__restrict__ key,
                   uint64_t *__restrict__ acc, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN,
                   int level, int alpha, int L, int K, int nd, size_t ext_stride, int B, Ws ws, int *err)
{
    typedef PassShape<S, SUB> P;
    typedef InnerSmem<S, SUB> SM;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // [0], [1]: digit stages; [2]: key stage
    uint64_t *xs = reinterpret_cast<uint64_t *>(smem + SM::X_OFF);
    uint64_t *ks = reinterpret_cast<uint64_t *>(smem + SM::K_OFF);
    uint64_t *sm = reinterpret_cast<uint64_t *>(smem + SM::T_OFF);
    constexpr uint32_t TB = SM::TILE * 8;
    const int N = 1 << logN;
    const int it = blockIdx.x % B, tile = blockIdx.x / B;
    const int e = (int)gridDim.y - 1 - (int)blockIdx.y;
    const int row = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC p = pc[row];
    const Tw *T = tw + (size_t)row * N;
    const size_t krow = (size_t)(L + 1 + K) * N;
    const size_t t0 = (size_t)tile * SM::TILE;
    const uint64_t *exte = ext + it * ws.ext + (size_t)e * N + t0;
    const uint64_t *d2ne = d2n + it * ws.d2 + (size_t)e * N + t0;
    const uint64_t *keye = key + (size_t)row * N + t0;
    // a digit's own limbs come from d in the evaluation domain (block-uniform)
    auto own = [&](int j) { return e >= j * alpha && e < min(j * alpha + alpha, level + 1); };
    auto load_digit = [&](int j) {
        mbar_arrive_expect_tx(&bar[j & 1], TB);
        bulk_g2s(xs + (j & 1) * SM::TILE, own(j) ? d2ne : exte + (size_t)j * ext_stride, TB, &bar[j & 1]);
    };
    auto load_keys = [&](int j) {
        mbar_arrive_expect_tx(&bar[2], 2 * TB);
        bulk_g2s(ks, keye + (size_t)j * 2 * krow, TB, &bar[2]);
        bulk_g2s(ks + SM::TILE, keye + (size_t)j * 2 * krow + krow, TB, &bar[2]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
        fence_proxy_async_smem();
        load_digit(0);
        if (nd > 1) load_digit(1);
        load_keys(0);
    }
    __syncthreads();
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = tile * SM::SUB + sub;
    const int w0 = sub * P::M + h;  // this thread's words of a tile: w0 + T k
    uint64_t a0[P::E], a1[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) a0[k] = a1[k] = 0;
    int j = 0;
    for (; j < nd; j++) {
        if (__syncthreads_or(!mbar_wait(&bar[j & 1], (j >> 1) & 1))) break;
        uint64_t x[P::E];
        const uint64_t *xt = xs + (j & 1) * SM::TILE + w0;
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = xt[P::T * k];
        if (!own(j)) {
            chunks_fwd_core<S>(x, sm, h, sub, g, N, T, p.q);
#pragma unroll
            for (int k = 0; k < P::E; k++) x[k] = reduce4q(x[k], p.q);
        }
        if (__syncthreads_or(!mbar_wait(&bar[2], j & 1))) break;
        const uint64_t *k0 = ks + w0, *k1 = k0 + SM::TILE;
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            a0[k] = add_mod(a0[k], mont_mul(x[k], k0[P::T * k], p.q, p.qinv), p.q);
            a1[k] = add_mod(a1[k], mont_mul(x[k], k1[P::T * k], p.q, p.qinv), p.q);
        }
        __syncthreads();  // digit stage j & 1 and the key stage are free again
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();  // the CTA's reads of those stages before the copies that refill them
            if (j + 2 < nd) load_digit(j + 2);
            if (j + 1 < nd) load_keys(j + 1);
        }
    }
    if (j < nd) {  // a copy did not arrive in time: report, drain what is in flight, give up
        if (threadIdx.x == 0) {
            *(volatile int *)err = 1;
            for (int d = j; d < min(j + 2, nd); d++) mbar_wait(&bar[d & 1], (d >> 1) & 1);
            mbar_wait(&bar[2], j & 1);
        }
        return;
    }
    uint64_t *o0 = acc + it * ws.acc + (size_t)e * N + t0 + w0, *o1 = o0 + krow;
#pragma unroll
    for (int k = 0; k < P::E; k++) {
        o0[P::T * k] = a0[k];
        o1[P::T * k] = a1[k];
    }
}

// ---------------------------------------------------------------------------
// 3'. the same stage with 8 words per thread (N = 2^15, 2^16: 256-point chunks)
// ---------------------------------------------------------------------------
// One warp per chunk (T = 32 threads x E = 8 words), three rounds of butterflies
// (distances 128..32, 16..4, 2..1) with two warp-local exchanges through a
// swizzled shared-memory buffer, so a thread holds half the registers of the
// 16-word form and more warps fit on an SM. LAZY: the products with the key are
// accumulated exactly in 128 bits over all digits and reduced once per word
// (sum x k 2^64 < nd q^2 < 2^128 for nd <= 64 digits and q < 2^61).
template <int SUB_>
struct Inner8Smem {
    static constexpr int M = 256, E = 8, T = 32;
    static constexpr int SUB = SUB_;              // chunks per block (one warp each)
    static constexpr int THREADS = SUB * T;
    static constexpr int TILE = SUB * M;
    static constexpr size_t X_OFF = 128;                              // two digit tiles
    static constexpr size_t K_OFF = X_OFF + 2 * (size_t)TILE * 8;    // two key tiles
    static constexpr size_t T_OFF = K_OFF + 2 * (size_t)TILE * 8;    // exchange buffers
    static constexpr size_t BYTES = T_OFF + (size_t)TILE * 8;
};

// Rows e >= inv_from of the accumulators are the ones ModDown takes to the
// coefficient domain (the P rows, and in HMult the top limb l after u = d_l +
// acc_l P^-1): they leave through the first (CHUNKS) inverse pass here, on the
// words already in registers, so ModDown runs only the COLS pass on them. The
// block rows are taken from the top, so the blocks with the longer epilogue start
// first. inv_from > level + K turns this off.
template <int SUB, bool LAZY, bool SHFL>
__global__ void __launch_bounds__(Inner8Smem<SUB>::THREADS, SUB == 8 ? 2 : 4)
    k_inner8(const uint64_t *__restrict__ ext, const uint64_t *__restrict__ d2n, const uint64_t *__restrict__ key,
             uint64_t *__restrict__ acc, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw,
             const Tw *__restrict__ twi, int logN, int level, int alpha, int L, int K, int nd, size_t ext_stride,
             int B, Ws ws, int inv_from, ItemPtrs dtop, Tw pinv, size_t pstride, int *err)
{
    typedef Inner8Smem<SUB> SM;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);  // [0], [1]: digit stages; [2]: key stage
    uint64_t *xs = reinterpret_cast<uint64_t *>(smem + SM::X_OFF);
    uint64_t *ks = reinterpret_cast<uint64_t *>(smem + SM::K_OFF);
    constexpr uint32_t TB = SM::TILE * 8;
    const int N = 1 << logN;
    const int it = blockIdx.x % B, tile = blockIdx.x / B;
    const int e = (int)gridDim.y - 1 - (int)blockIdx.y;
    const int row = e <= level ? e : L + 1 + (e - level - 1);
    const PrimeC p = pc[row];
    const Tw *T = tw + (size_t)row * N;
    const size_t krow = (size_t)(L + 1 + K) * N;
    const size_t t0 = (size_t)tile * SM::TILE;
    const uint64_t *exte = ext + it * ws.ext + (size_t)e * N + t0;
    const uint64_t *d2ne = d2n + it * ws.d2 + (size_t)e * N + t0;
    const uint64_t *keye = key + (size_t)row * N + t0;
    auto own = [&](int j) { return e >= j * alpha && e < min(j * alpha + alpha, level + 1); };
    auto load_digit = [&](int j) {
        mbar_arrive_expect_tx(&bar[j & 1], TB);
        bulk_g2s(xs + (j & 1) * SM::TILE, own(j) ? d2ne : exte + (size_t)j * ext_stride, TB, &bar[j & 1]);
    };
    auto load_keys = [&](int j) {
        mbar_arrive_expect_tx(&bar[2], 2 * TB);
        bulk_g2s(ks, keye + (size_t)j * 2 * krow, TB, &bar[2]);
        bulk_g2s(ks + SM::TILE, keye + (size_t)j * 2 * krow + krow, TB, &bar[2]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
        fence_proxy_async_smem();
        load_digit(0);
        if (nd > 1) load_digit(1);
        load_keys(0);
    }
    __syncthreads();
    const int h = threadIdx.x & 31, sub = threadIdx.x >> 5;
    const int g = tile * SUB + sub;
    uint64_t *ex = reinterpret_cast<uint64_t *>(smem + SM::T_OFF) + sub * SM::M;
    const size_t tg = (size_t)(N >> 8) + g;  // twiddle of group j of a stage with m groups: T[m tg + j]
    int ka[8];  // tile offsets (storage order) of this thread's output words 8 h + k
#pragma unroll
    for (int k = 0; k < 8; k++) ka[k] = sub * SM::M + addr16(8 * h + k);
    uint64_t a0[8], a1[8];  // running sums (not LAZY)
    Acc4 u0[8], u1[8];      // LAZY: exact 128-bit sums
#pragma unroll
    for (int k = 0; k < 8; k++) {
        a0[k] = a1[k] = 0;
        u0[k] = u1[k] = Acc4{0, 0, 0, 0};
    }
    int j = 0;
    for (; j < nd; j++) {
        if (__syncthreads_or(!mbar_wait(&bar[j & 1], (j >> 1) & 1))) break;
        uint64_t x[8];
        const uint64_t *xt = xs + (j & 1) * SM::TILE;
        if (own(j)) {  // already in the evaluation domain, storage order (block-uniform)
#pragma unroll
            for (int k = 0; k < 8; k++) x[k] = xt[ka[k]];
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) x[k] = xt[sub * SM::M + h + 32 * k];
            chunks_fwd_core8<SHFL>(x, ex, h, [&](int m, int jj) { return ldtw(T + m * tg + jj); }, p.q);
#pragma unroll
            for (int k = 0; k < 8; k++) x[k] = reduce4q(x[k], p.q);
        }
        if (__syncthreads_or(!mbar_wait(&bar[2], j & 1))) break;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint64_t k0 = ks[ka[k]], k1 = ks[SM::TILE + ka[k]];
            if (LAZY) {
                mac4(u0[k], x[k], k0);
                mac4(u1[k], x[k], k1);
            } else {
                a0[k] = add_mod(a0[k], mont_mul(x[k], k0, p.q, p.qinv), p.q);
                a1[k] = add_mod(a1[k], mont_mul(x[k], k1, p.q, p.qinv), p.q);
            }
        }
        __syncthreads();  // digit stage j & 1 and the key stage are free again
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();  // the CTA's reads of those stages before the copies that refill them
            if (j + 2 < nd) load_digit(j + 2);
            if (j + 1 < nd) load_keys(j + 1);
        }
    }
    if (j < nd) {  // a copy did not arrive in time: report, drain what is in flight, give up
        if (threadIdx.x == 0) {
            *(volatile int *)err = 1;
            for (int d = j; d < min(j + 2, nd); d++) mbar_wait(&bar[d & 1], (d >> 1) & 1);
            mbar_wait(&bar[2], j & 1);
        }
        return;
    }
    uint64_t *o0 = acc + it * ws.acc + (size_t)e * N + t0, *o1 = o0 + krow;
    if (LAZY) {
#pragma unroll
        for (int k = 0; k < 8; k++) {  // (hi mod q) 2^64 + lo, then one Montgomery reduction
            const uint64_t h0 = csub(shoup(acc4_hi(u0[k]), 1, p.w64, p.q), p.q);
            const uint64_t h1 = csub(shoup(acc4_hi(u1[k]), 1, p.w64, p.q), p.q);
            a0[k] = mont_redc(h0, acc4_lo(u0[k]), p.q, p.qinv);
            a1[k] = mont_redc(h1, acc4_lo(u1[k]), p.q, p.qinv);
        }
    }
    if (e < inv_from) {  // block-uniform
#pragma unroll
        for (int k = 0; k < 8; k++) {
            o0[ka[k]] = a0[k];
            o1[ka[k]] = a1[k];
        }
        return;
    }
    if (e == level) {  // HMult's top limb: u_k = d_k[l] + acc_k[l] P^-1 (evaluation domain)
        const uint64_t *d0 = dtop.in0[it] + (size_t)level * N + t0, *d1 = d0 + pstride;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            a0[k] = add_mod(d0[ka[k]], csub(shoup(a0[k], pinv.w, pinv.s, p.q), p.q), p.q);
            a1[k] = add_mod(d1[ka[k]], csub(shoup(a1[k], pinv.w, pinv.s, p.q), p.q), p.q);
        }
    }
    const Tw *TI = twi + (size_t)row * N;
    chunks_inv_core8(a0, ex, h, [&](int m, int jj) { return ldtw(TI + m * tg + jj); }, p.q);
    chunks_inv_core8(a1, ex, h, [&](int m, int jj) { return ldtw(TI + m * tg + jj); }, p.q);
#pragma unroll
    for (int k = 0; k < 8; k++) {  // the inverse pass's output order: word h + 32 k of the chunk
        o0[sub * SM::M + h + 32 * k] = a0[k];
        o1[sub * SM::M + h + 32 * k] = a1[k];
    }
}

// ---------------------------------------------------------------------------
// failure-detection self-test: one block waits on a barrier whose phase never
// completes (nothing is copied), gives up after limit_ns, records the timeout in
// the error word and returns, exactly as the pipelined kernels do
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(int *err, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar[1];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&bar[0], 16);  // 16 bytes announced, none will arrive
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait(&bar[0], 0, limit_ns)))
        if (threadIdx.x == 0) *(volatile int *)err = 1;
}

void wait_selftest(Ctx &c, uint32_t timeout_us)
{
    k_wait_selftest<<<1, 32, 0, c.stream>>>(c.d_err, (uint64_t)timeout_us * 1000);
    check_launch("k_wait_selftest");
}

// stages 1-3 for B items: d (limbs 0..level) of item b in the evaluation domain
// in ws_d2n[b] and (to be transformed) in ws_d2[b]; accumulators to ws_acc[b]
// d2 (every item) has been through the first inverse pass (k_tensor_ic / k_automorph_ic)
// Returns true when the inner product also ran ModDown's first inverse pass on
// its rows (the 8-word kernel): resc selects HMult's rows (the top limb l, whose
// u = d_l + acc_l P^-1 takes d from dtop.in0, and the P rows) or a rotation's (the
// P rows).
static bool ks_modup_inner(Ctx &c, int level, const Swk &key, int B, bool resc, const ItemPtrs &dtop)
{
    const Ws ws = ws_strides(c);
    const int nd = c.ndigits(level), E_ext = level + 1 + c.K;
    LimbMap md{c.ws_d2, ws.d2, level + 1, B, level + 1, 0, 0};
    ntt_inv_cols_mul(c, md, c.d_modup_outmul + c.modup_outmul_off[level]);
    DigitOffs offs;
    for (int j = 0; j < nd; j++) offs.off[j] = c.modup_off[level][j];
    const size_t es = c.ext_rows() * c.N;
    {
        uint64_t targets = 0;
        for (int j = 0; j < nd; j++) targets += E_ext - (std::min((j + 1) * c.alpha, level + 1) - j * c.alpha);
        ProfScope _ps(c, "modup_cols", (uint64_t)B * ((level + 1) + targets));  // limbs read once + written
        // 8 words per thread for grids that would leave SMs idle with 16 (below 3 x 152 blocks of the
        // 16-column form: low levels, few digits), 8 or 4 columns per block
        if (ntt_s_rows(c.logN) == 8 && c.modup_words == 8 && (long)(c.N >> 12) * targets * B < 456) {
            dispatch_a(c.alpha, [&](auto av) {
                constexpr int A = decltype(av)::value;
                auto launch8 = [&](auto bv) {
                    constexpr int SUB = decltype(bv)::value;
                    launch_on(c, k_modup_cols8<A, SUB>, grid_s(c, 8, SUB, B * nd * E_ext), 32 * SUB, 0, c.ws_d2,
                        c.ws_ext, c.d_ks, offs, c.d_pc, c.d_twf, c.logN, level, c.alpha, c.L, c.K, nd, es, ws);
                };
                if (pass_sub(c, 8, (int)targets * B) >= 16) launch8(std::integral_constant<int, 8>{});
                else launch8(std::integral_constant<int, 4>{});
            });
            check_launch("k_modup_cols8");
        } else
        dispatch_pass(c, ntt_s_rows(c.logN), (int)targets * B, [&](auto sv, auto bv) {
            constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
            dispatch_a(c.alpha, [&](auto av) {
                constexpr int A = decltype(av)::value;
                launch_on(c, k_modup_cols<S, A, SUB>, grid_s(c, S, SUB, B * nd * E_ext), PassShape<S, SUB>::THREADS,
                    0, c.ws_d2, c.ws_ext, c.d_ks, offs, c.d_pc, c.d_twf, c.logN, level, c.alpha, c.L, c.K, nd, es,
                    ws);
            });
        });
        check_launch("k_modup_cols");
    }
    // per target limb: the two key words of every digit, read once for the
    // batch (its items run back to back on the same key tile); per item and
    // target limb: one digit word per digit read, two accumulators written
    // method traffic: the switching key's limbs, once for the batch
    ProfScope _ps(c, "inner_chunks", (uint64_t)E_ext * 2 * nd + (uint64_t)B * E_ext * (nd + 2),
                  (uint64_t)E_ext * 2 * nd);
    auto launch = [&](auto sv, auto subv) {
        constexpr int S = decltype(sv)::value, SUB = decltype(subv)::value;
        typedef InnerSmem<S, SUB> SM;
        const dim3 grid(B * ((c.N >> S) / SUB), E_ext);
        static std::atomic<bool> attr_set{false};
        if (!attr_set.load()) {
            PPST_CUDA(cudaFuncSetAttribute(k_inner_chunks<S, SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SM::BYTES));
            attr_set = true;
        }
        launch_on(c, k_inner_chunks<S, SUB>, grid, SM::THREADS, SM::BYTES, c.ws_ext, c.ws_d2n, key.d, c.ws_acc,
            c.d_pc, c.d_twf, c.logN, level, c.alpha, c.L, c.K, nd, es, B, ws, c.d_err);
    };
    auto launch8s = [&](auto subv, auto lazyv, auto shflv) {
        constexpr int SUB = decltype(subv)::value;
        constexpr bool LAZY = decltype(lazyv)::value, SHFL = decltype(shflv)::value;
        typedef Inner8Smem<SUB> SM;
        const dim3 grid(B * (c.N / SM::TILE), E_ext);
        static std::atomic<bool> attr_set{false};
        if (!attr_set.load()) {
            PPST_CUDA(cudaFuncSetAttribute(k_inner8<SUB, LAZY, SHFL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SM::BYTES));
            attr_set = true;
        }
        const Tw pinv = c.md_const[(size_t)level * (c.L + 1) + level].pinv;
        launch_on(c, k_inner8<SUB, LAZY, SHFL>, grid, SM::THREADS, SM::BYTES, c.ws_ext, c.ws_d2n, key.d,
            c.ws_acc, c.d_pc, c.d_twf, c.d_twi, c.logN, level, c.alpha, c.L, c.K, nd, es, B, ws,
            resc ? level : level + 1, dtop, pinv, (size_t)(c.L + 1) * c.N, c.d_err);
    };
    auto launch8 = [&](auto subv, auto lazyv) {
        if (c.inner_shfl) launch8s(subv, lazyv, std::true_type{});
        else launch8s(subv, lazyv, std::false_type{});
    };
    bool fused = false;
    dispatch_s(ntt_s_chunk(c.logN), [&](auto sv) {
        constexpr int S = decltype(sv)::value;
        // the context's tile, halved (down to 4 chunks) while the grid would leave SMs idle
        int tile = c.inner_sub;
        while (tile > 4 && (long)B * ((c.N >> S) / tile) * E_ext < (long)c.pass_min_blocks) tile /= 2;
        if (S == 8 && c.inner_words == 8) {  // 8 words per thread: tiles of 4 or 8 chunks
            if (tile >= 8) {
                if (c.inner_lazy) launch8(std::integral_constant<int, 8>{}, std::true_type{});
                else launch8(std::integral_constant<int, 8>{}, std::false_type{});
            } else {
                if (c.inner_lazy) launch8(std::integral_constant<int, 4>{}, std::true_type{});
                else launch8(std::integral_constant<int, 4>{}, std::false_type{});
            }
            fused = true;
            return;
        }
        switch (tile) {
        case 4: launch(sv, std::integral_constant<int, 4>{}); break;
        case 16: launch(sv, std::integral_constant<int, 16>{}); break;
        default: launch(sv, std::integral_constant<int, 8>{}); break;
        }
    });
    check_launch("k_inner_chunks");
    return fused;
}

// HMult of B pairs (each pair at its own min level; all pairs share that level):
// tensor -> key switch of d2 -> add -> rescale, fused as above
std::vector<CtObj *> ev_hmult_batch(Ctx &c, const EvkObj &k, const std::vector<const CtObj *> &as,
                                    const std::vector<const CtObj *> &bs)
{
    const int B = (int)as.size();
    if (B < 1 || B > BMAX || bs.size() != as.size()) throw_err(PPST_E_ARG, "hmult batch: 1 to 16 pairs");
    const int lv = std::min(as[0]->level, bs[0]->level);
    for (int i = 0; i < B; i++)
        if (std::min(as[i]->level, bs[i]->level) != lv) throw_err(PPST_E_ARG, "hmult batch: pairs at different levels");
    if (lv < 1) throw_err(PPST_E_DEPTH, "hmult at level 0");
    if (!k.relin.d) throw_err(PPST_E_STATE, "no relinearisation key");
    ensure_workspace(c, B);
    const Ws ws = ws_strides(c);
    const size_t ps = (size_t)(c.L + 1) * c.N;
    std::vector<CtObj *> t(B, nullptr), o(B, nullptr);
    try {
        ItemPtrs ip{};
        for (int i = 0; i < B; i++) {
            t[i] = ct_new(c, lv, as[i]->scale * bs[i]->scale);
            ip.in0[i] = as[i]->d;
            ip.in1[i] = bs[i]->d;
            ip.out[i] = t[i]->d;
        }
        {
            ProfScope _ps(c, "tensor", (uint64_t)B * 7 * (lv + 1), (uint64_t)B * 4 * (lv + 1));  // reads a, b
            if (ntt_s_chunk(c.logN) == 8 && c.inv_words == 8) {  // 8 words per thread
                auto launch8 = [&](auto bv) {
                    constexpr int SUB = decltype(bv)::value;
                    launch_on(c, k_tensor_ic8<SUB>, dim3(c.N / (256 * SUB), B * (lv + 1)), 32 * SUB, 0, ip, c.ws_d2,
                        c.ws_d2n, c.d_pc, c.d_twi, c.logN, lv + 1, ps, ws.d2);
                };
                if (pass_sub(c, 8, B * (lv + 1)) >= 16) launch8(std::integral_constant<int, 8>{});
                else launch8(std::integral_constant<int, 4>{});
            } else
            dispatch_pass(c, ntt_s_chunk(c.logN), B * (lv + 1), [&](auto sv, auto bv) {
                constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
                launch_on(c, k_tensor_ic<S, SUB>, grid_s(c, S, SUB, B * (lv + 1)), PassShape<S, SUB>::THREADS, 0,
                    ip, c.ws_d2, c.ws_d2n, c.d_pc, c.d_twi, c.logN, lv + 1, ps, ws.d2);
            });
            check_launch("k_tensor_ic");
        }
        ItemPtrs op{};
        for (int i = 0; i < B; i++) {
            o[i] = ct_new(c, lv - 1, (as[i]->scale * bs[i]->scale) / (double)c.primes[lv]);
            op.in0[i] = t[i]->d;
            op.out[i] = o[i]->d;
        }
        const bool fused = ks_modup_inner(c, lv, k.relin, B, true, op);
        ks_moddown<true>(c, lv, B, op, fused);
    } catch (...) {
        for (CtObj *x : t) ct_free(x);
        for (CtObj *x : o) ct_free(x);
        throw;
    }
    for (CtObj *x : t) ct_free(x);
    return o;
}

CtObj *ev_hmult(Ctx &c, const EvkObj &k, const CtObj &a, const CtObj &b)
{
    return ev_hmult_batch(c, k, {&a}, {&b})[0];
}

// Rot(r) of B ciphertexts at one level: automorphism of (c0, c1), key switch of the rotated c1
std::vector<CtObj *> ev_rotate_batch(Ctx &c, const EvkObj &k, const std::vector<const CtObj *> &as, int r)
{
    const int B = (int)as.size();
    if (B < 1 || B > BMAX) throw_err(PPST_E_ARG, "rotate batch: 1 to 16 ciphertexts");
    const int lv = as[0]->level;
    for (const CtObj *a : as)
        if (a->level != lv) throw_err(PPST_E_ARG, "rotate batch: ciphertexts at different levels");
    const int rr = ((r % c.S) + c.S) % c.S;
    std::vector<CtObj *> o(B, nullptr);
    if (rr == 0) {
        for (int i = 0; i < B; i++) o[i] = ct_clone(*as[i]);
        return o;
    }
    auto it = k.rot.find(rr);
    if (it == k.rot.end()) throw_err(PPST_E_STATE, "no Galois key for rotation " + std::to_string(rr));
    ensure_workspace(c, B);
    const Ws ws = ws_strides(c);
    const size_t ps = (size_t)(c.L + 1) * c.N;
    try {
        ItemPtrs ip{};
        for (int i = 0; i < B; i++) {
            o[i] = ct_new(c, lv, as[i]->scale);
            ip.in0[i] = as[i]->d;
            ip.out[i] = o[i]->d;
        }
        {
            ProfScope _ps(c, "automorph", (uint64_t)B * 5 * (lv + 1), (uint64_t)B * 2 * (lv + 1));  // reads a
            if (ntt_s_chunk(c.logN) == 8 && c.inv_words == 8) {  // 8 words per thread
                auto launch8 = [&](auto bv) {
                    constexpr int SUB = decltype(bv)::value;
                    launch_on(c, k_automorph_ic8<SUB>, dim3(c.N / (256 * SUB), B * 2 * (lv + 1)), 32 * SUB, 0, ip,
                        c.ws_d2, c.ws_d2n, c.d_pc, c.d_twi, c.logN, lv + 1, galois_elt(c, rr), ps, ws.d2);
                };
                if (pass_sub(c, 8, B * (lv + 1)) >= 16) launch8(std::integral_constant<int, 8>{});
                else launch8(std::integral_constant<int, 4>{});
            } else
            dispatch_pass(c, ntt_s_chunk(c.logN), B * (lv + 1), [&](auto sv, auto bv) {
                constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
                launch_on(c, k_automorph_ic<S, SUB>, grid_s(c, S, SUB, B * 2 * (lv + 1)),
                    PassShape<S, SUB>::THREADS, 0, ip, c.ws_d2, c.ws_d2n, c.d_pc, c.d_twi, c.logN, lv + 1,
                    galois_elt(c, rr), ps, ws.d2);
            });
            check_launch("k_automorph_ic");
        }
        ItemPtrs op{};
        for (int i = 0; i < B; i++) {
            op.in0[i] = o[i]->d;  // sigma(c0), added to ModDown(acc_0) in place
            op.out[i] = o[i]->d;
        }
        const bool fused = ks_modup_inner(c, lv, it->second, B, false, op);
        ks_moddown<false>(c, lv, B, op, fused);
    } catch (...) {
        for (CtObj *x : o) ct_free(x);
        throw;
    }
    return o;
}

CtObj *ev_rotate(Ctx &c, const EvkObj &k, const CtObj &a, int r) { return ev_rotate_batch(c, k, {&a}, r)[0]; }

}  // namespace ppst
