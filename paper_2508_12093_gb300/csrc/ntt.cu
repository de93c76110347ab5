// ntt.cu -- limb-batched negacyclic NTT / inverse NTT for sm_103a.
//
// The transform evaluates a polynomial of Z_q[X]/(X^N + 1) at the odd powers
// of a primitive 2N-th root of unity psi: output word k holds
// a(psi^(2 brv(k) + 1)) (bit-reversed order). Forward: Cooley-Tukey with
// merged psi powers (stage with m groups of distance t = N/2m, group i uses
// psi^brv(m + i)); inverse: Gentleman-Sande with psi^-1 powers, then N^-1.
// Butterflies are Harvey's lazy ones (values in [0, 4q) forward, [0, 2q)
// inverse), twiddles are (w, floor(w 2^64 / q)) pairs for Shoup products.
//
// Two passes over HBM. N = R * C, R = 2^ceil(logN/2) rows, C = N / R:
//   COLS pass   the log2 R stages of distance >= C: every column
//               (c, c + C, c + 2C, ...) is an independent R-point transform;
//   CHUNKS pass the remaining stages, inside contiguous chunks of C words.
// A block runs SUB sub-transforms (SUB columns or chunks; 16 for large grids,
// 8 or 4 when few limbs would leave SMs idle); the per-thread register scheme
// is in ntt.cuh.
#include "ntt.cuh"

namespace ppst {

template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_ntt_fwd_cols(LimbMap map, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int b = blockIdx.y, p = map.prime(b);
    uint64_t *a = map.ptr(b, N);
    const uint64_t q = pc[p].q;
    int h, sub;
    pass_coords<S, true, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = a[(size_t)(h + P::T * k) * C + g];
    cols_fwd_core<S, SUB>(x, sm, h, sub, tw + (size_t)p * N, q);
#pragma unroll
    for (int k = 0; k < P::E; k++) a[(size_t)(P::E * h + k) * C + g] = x[k];
}

template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_ntt_fwd_chunks(LimbMap map, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int b = blockIdx.y, p = map.prime(b);
    const uint64_t q = pc[p].q;
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t *a = map.ptr(b, N) + (size_t)g * P::M;
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = a[h + P::T * k];
    chunks_fwd_core<S>(x, sm, h, sub, g, N, tw + (size_t)p * N, q);
    // natural word E h + k is stored at h + T k (see eval_address)
#pragma unroll
    for (int k = 0; k < P::E; k++) a[h + P::T * k] = reduce4q(x[k], q);
}

template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_ntt_inv_chunks(LimbMap map, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int b = blockIdx.y, p = map.prime(b);
    const uint64_t q = pc[p].q;
    int h, sub;
    pass_coords<S, false, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t *a = map.ptr(b, N) + (size_t)g * P::M;
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = a[h + P::T * k];  // natural word E h + k
    chunks_inv_core<S>(x, sm, h, sub, g, N, tw + (size_t)p * N, q);
#pragma unroll
    for (int k = 0; k < P::E; k++) a[h + P::T * k] = x[k];
}

// the first inverse pass with 8 words per thread (256-point chunks: N = 2^15, 2^16),
// one warp per chunk, SUB chunks per block: reads the evaluation domain's storage
// order, writes natural order (in place: a warp reads its whole chunk before any
// of its lanes writes)
template <int SUB>
__global__ void __launch_bounds__(32 * SUB, SUB == 8 ? 4 : 8)
    k_ntt_inv_chunks8(LimbMap map, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN)
{
    __shared__ uint64_t ex_all[SUB * 256];
    const int N = 1 << logN;
    const int b = blockIdx.y, p = map.prime(b);
    const uint64_t q = pc[p].q;
    const int h = threadIdx.x & 31, sub = threadIdx.x >> 5;
    const int g = blockIdx.x * SUB + sub;
    uint64_t *a = map.ptr(b, N) + (size_t)g * 256;
    uint64_t x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = a[addr16(8 * h + k)];
    const Tw *T = tw + (size_t)p * N;
    const size_t tg = (size_t)(N >> 8) + g;
    chunks_inv_core8(x, ex_all + sub * 256, h, [&](int m, int j) { return ldtw(T + m * tg + j); }, q);
#pragma unroll
    for (int k = 0; k < 8; k++) a[h + 32 * k] = x[k];
}

// last inverse pass; the result is multiplied by N^-1, or by outmul[i] for limb
// i of its polynomial (N^-1 times a constant of the caller's), and reduced to [0, q)
template <int S, int SUB>
__global__ void __launch_bounds__(PassShape<S, SUB>::THREADS, PassShape<S, SUB>::MIN_BLOCKS)
    k_ntt_inv_cols(LimbMap map, const PrimeC *__restrict__ pc, const Tw *__restrict__ tw, int logN,
                   const Tw *__restrict__ outmul)
{
    typedef PassShape<S, SUB> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN, C = N >> S;
    const int b = blockIdx.y, p = map.prime(b);
    uint64_t *a = map.ptr(b, N);
    const uint64_t q = pc[p].q;
    int h, sub;
    pass_coords<S, true, SUB>(h, sub);
    const int g = blockIdx.x * P::SUB + sub;
    uint64_t x[P::E];
#pragma unroll
    for (int k = 0; k < P::E; k++) x[k] = a[(size_t)(P::E * h + k) * C + g];
    cols_inv_core<S, SUB>(x, sm, h, sub, tw + (size_t)p * N, q);
    const Tw f = outmul ? outmul[b % map.per_poly] : Tw{pc[p].ninv, pc[p].ninv_sh};
#pragma unroll
    for (int k = 0; k < P::E; k++) a[(size_t)(h + P::T * k) * C + g] = csub(shoup(x[k], f.w, f.s, q), q);
}

template <int S, int SUB>
static dim3 pass_grid(const Ctx &c, const LimbMap &m)
{
    return dim3((c.N >> S) / SUB, m.count());
}

// runs f(S, SUB) with the pass size of `s` and the block shape pass_sub picks for m
template <class F>
static void dispatch_pass(const Ctx &c, int s, const LimbMap &m, F &&f)
{
    dispatch_s(s, [&](auto sv) {
        dispatch_sub<decltype(sv)::value>(pass_sub(c, decltype(sv)::value, m.count()), [&](auto bv) { f(sv, bv); });
    });
}

void ntt_fwd(Ctx &c, const LimbMap &m)
{
    if (m.count() == 0) return;
    {
        ProfScope _ps(c, "ntt_cols_fwd", (uint64_t)2 * m.count());
        dispatch_pass(c, ntt_s_rows(c.logN), m, [&](auto sv, auto bv) {
            constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
            launch_on(c, k_ntt_fwd_cols<S, SUB>, pass_grid<S, SUB>(c, m), PassShape<S, SUB>::THREADS, 0, m, c.d_pc,
                c.d_twf, c.logN);
        });
        check_launch("ntt_cols_fwd");
    }
    ProfScope _ps(c, "ntt_chunks_fwd", (uint64_t)2 * m.count());
    dispatch_pass(c, ntt_s_chunk(c.logN), m, [&](auto sv, auto bv) {
        constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
        launch_on(c, k_ntt_fwd_chunks<S, SUB>, pass_grid<S, SUB>(c, m), PassShape<S, SUB>::THREADS, 0, m, c.d_pc,
            c.d_twf, c.logN);
    });
    check_launch("ntt_chunks_fwd");
}

void ntt_inv_mul(Ctx &c, const LimbMap &m, const Tw *outmul)
{
    if (m.count() == 0) return;
    {
        ProfScope _ps(c, "ntt_chunks_inv", (uint64_t)2 * m.count());
        if (ntt_s_chunk(c.logN) == 8 && c.inv_words == 8) {  // 8 words per thread, 8 or 4 chunks per block
            auto launch8 = [&](auto bv) {
                constexpr int SUB = decltype(bv)::value;
                launch_on(c, k_ntt_inv_chunks8<SUB>, dim3(c.N / (256 * SUB), m.count()), 32 * SUB, 0, m, c.d_pc,
                    c.d_twi, c.logN);
            };
            if (pass_sub(c, 8, m.count()) >= 16) launch8(std::integral_constant<int, 8>{});
            else launch8(std::integral_constant<int, 4>{});
            check_launch("ntt_chunks_inv8");
        } else {
            dispatch_pass(c, ntt_s_chunk(c.logN), m, [&](auto sv, auto bv) {
                constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
                launch_on(c, k_ntt_inv_chunks<S, SUB>, pass_grid<S, SUB>(c, m), PassShape<S, SUB>::THREADS, 0, m,
                    c.d_pc, c.d_twi, c.logN);
            });
            check_launch("ntt_chunks_inv");
        }
    }
    ntt_inv_cols_mul(c, m, outmul);
}

void ntt_inv_cols_mul(Ctx &c, const LimbMap &m, const Tw *outmul)
{
    if (m.count() == 0) return;
    ProfScope _ps(c, "ntt_cols_inv", (uint64_t)2 * m.count());
    dispatch_pass(c, ntt_s_rows(c.logN), m, [&](auto sv, auto bv) {
        constexpr int S = decltype(sv)::value, SUB = decltype(bv)::value;
        launch_on(c, k_ntt_inv_cols<S, SUB>, pass_grid<S, SUB>(c, m), PassShape<S, SUB>::THREADS, 0, m, c.d_pc,
            c.d_twi, c.logN, outmul);
    });
    check_launch("ntt_cols_inv");
}

void ntt_inv(Ctx &c, const LimbMap &m) { ntt_inv_mul(c, m, nullptr); }

}  // namespace ppst
