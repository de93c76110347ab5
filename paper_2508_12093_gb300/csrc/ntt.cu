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
// Each pass runs M-point sub-transforms (M = R or C = 2^S). A thread holds
// E = 2^ceil(S/2) words in registers: first as x = h + T k (T = M/E threads
// per sub-transform), where the ceil(S/2) long-distance stages pair register
// k with k + 2^s; then, after one shared-memory transpose, as x = E h + k,
// where the short-distance stages again pair registers. A block runs 16
// sub-transforms (16 columns = 128-byte rows, or 16 chunks).
#include "ctx.cuh"

namespace ppst {

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

template <int S>
struct PassShape {
    static constexpr int M = 1 << S;
    static constexpr int A = (S + 1) / 2;  // register stages of round 1
    static constexpr int E = 1 << A;       // words per thread
    static constexpr int T = M / E;        // threads per sub-transform
    static constexpr int SUB = 16;         // sub-transforms per block
    static constexpr int THREADS = SUB * T;
    static constexpr int SMEM_WORDS = SUB * (M + M / E);  // padded transpose buffer
    static constexpr int MIN_BLOCKS = THREADS >= 256 ? 3 : 4;  // register cap for occupancy
};

// Round-1 stages (long distances) on x[k] = word h + T k of a sub-transform.
// Stage s (k-distance 2^s, word distance T 2^s, s = A-1 .. 0 forward):
// global m = mbase / (T 2^s), group i = ibase(s) + (k >> (s + 1)).
// For COLS: m_glob = R / (2 d) with d in rows, ibase = 0.
// For CHUNKS: m_glob = N / (2 d), ibase = g * (C / (2 d)).

// one pass of the forward transform
template <int S, bool COLS>
__global__ void __launch_bounds__(PassShape<S>::THREADS, PassShape<S>::MIN_BLOCKS) k_ntt_fwd_pass(LimbMap map, const PrimeC *__restrict__ pc,
                                                                        const Tw *__restrict__ tw, int logN)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int b = blockIdx.y;
    uint64_t *a = map.ptr(b, N);
    const int p = map.prime(b);
    const uint64_t q = pc[p].q, q2 = 2 * q;
    const Tw *T = tw + (size_t)p * N;
    const int tid = threadIdx.x;
    uint64_t x[P::E];
    int h, sub;
    if (COLS) {
        sub = tid % P::SUB;  // column within the block
        h = tid / P::SUB;
    } else {
        h = tid % P::T;
        sub = tid / P::T;    // chunk within the block
    }
    const int C = N >> S;   // COLS: number of columns; CHUNKS: not used
    const int g = blockIdx.x * P::SUB + sub;  // global column (COLS) or chunk (CHUNKS)
    // ---- load: word x = h + T k of sub-transform g
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = a[(size_t)(h + P::T * k) * C + g];
    } else {
        const uint64_t *src = a + (size_t)g * P::M;
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = src[h + P::T * k];
    }
    // ---- round 1: distances M/2 .. T
#pragma unroll
    for (int s = P::A - 1; s >= 0; s--) {
        const int d = P::T << s;                    // word (row) distance within the sub-transform
        const int mg = COLS ? (P::M / (2 * d)) : (N / (2 * d));
        const int ib = COLS ? 0 : g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            const Tw w = ldtw(T + mg + ib + (k >> (s + 1)));
            bfly_fwd(x[k], x[k + (1 << s)], w, q, q2);
        }
    }
    // ---- transpose through shared memory (padded one word per E)
    uint64_t *ssub = COLS ? sm : sm + sub * (P::M + P::M / P::E);
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) sm[(h + P::T * k) * P::SUB + sub] = x[k];
    } else {
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            const int e = h + P::T * k;
            ssub[e + e / P::E] = x[k];
        }
    }
    __syncthreads();
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = sm[(P::E * h + k) * P::SUB + sub];
    } else {
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = ssub[(P::E + 1) * h + k];
    }
    // ---- round 2: distances T/2 .. 1 on word E h + k
#pragma unroll
    for (int d = P::T / 2; d >= 1; d >>= 1) {
        const int mg = COLS ? (P::M / (2 * d)) : (N / (2 * d));
        const int ib = COLS ? 0 : g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            const Tw w = ldtw(T + mg + ib + (P::E * h + k) / (2 * d));
            bfly_fwd(x[k], x[k + d], w, q, q2);
        }
    }
    // ---- store word E h + k
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) a[(size_t)(P::E * h + k) * C + g] = x[k];
    } else {
        uint64_t *dst = a + (size_t)g * P::M + P::E * h;
#pragma unroll
        for (int k = 0; k < P::E; k += 2) {
            ulonglong2 v = make_ulonglong2(reduce4q(x[k], q), reduce4q(x[k + 1], q));
            *reinterpret_cast<ulonglong2 *>(dst + k) = v;
        }
    }
}

// one pass of the inverse transform (mirror image: short distances first)
template <int S, bool COLS>
__global__ void __launch_bounds__(PassShape<S>::THREADS, PassShape<S>::MIN_BLOCKS) k_ntt_inv_pass(LimbMap map, const PrimeC *__restrict__ pc,
                                                                        const Tw *__restrict__ tw, int logN)
{
    typedef PassShape<S> P;
    __shared__ uint64_t sm[P::SMEM_WORDS];
    const int N = 1 << logN;
    const int b = blockIdx.y;
    uint64_t *a = map.ptr(b, N);
    const int p = map.prime(b);
    const uint64_t q = pc[p].q, q2 = 2 * q;
    const Tw *T = tw + (size_t)p * N;
    const int tid = threadIdx.x;
    uint64_t x[P::E];
    int h, sub;
    if (COLS) {
        sub = tid % P::SUB;
        h = tid / P::SUB;
    } else {
        h = tid % P::T;
        sub = tid / P::T;
    }
    const int C = N >> S;
    const int g = blockIdx.x * P::SUB + sub;
    // ---- load word E h + k
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = a[(size_t)(P::E * h + k) * C + g];
    } else {
        const uint64_t *src = a + (size_t)g * P::M + P::E * h;
#pragma unroll
        for (int k = 0; k < P::E; k += 2) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src + k);
            x[k] = v.x;
            x[k + 1] = v.y;
        }
    }
    // ---- round 2 mirror: distances 1 .. T/2
#pragma unroll
    for (int d = 1; d <= P::T / 2; d <<= 1) {
        const int mg = COLS ? (P::M / (2 * d)) : (N / (2 * d));
        const int ib = COLS ? 0 : g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if (k & d) continue;
            const Tw w = ldtw(T + mg + ib + (P::E * h + k) / (2 * d));
            bfly_inv(x[k], x[k + d], w, q, q2);
        }
    }
    uint64_t *ssub = COLS ? sm : sm + sub * (P::M + P::M / P::E);
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) sm[(P::E * h + k) * P::SUB + sub] = x[k];
    } else {
#pragma unroll
        for (int k = 0; k < P::E; k++) ssub[(P::E + 1) * h + k] = x[k];
    }
    __syncthreads();
    if (COLS) {
#pragma unroll
        for (int k = 0; k < P::E; k++) x[k] = sm[(h + P::T * k) * P::SUB + sub];
    } else {
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            const int e = h + P::T * k;
            x[k] = ssub[e + e / P::E];
        }
    }
    // ---- round 1 mirror: distances T .. M/2 on word h + T k
#pragma unroll
    for (int s = 0; s < P::A; s++) {
        const int d = P::T << s;
        const int mg = COLS ? (P::M / (2 * d)) : (N / (2 * d));
        const int ib = COLS ? 0 : g * (P::M / (2 * d));
#pragma unroll
        for (int k = 0; k < P::E; k++) {
            if ((k >> s) & 1) continue;
            const Tw w = ldtw(T + mg + ib + (k >> (s + 1)));
            bfly_inv(x[k], x[k + (1 << s)], w, q, q2);
        }
    }
    // ---- store word h + T k (the COLS pass is the last one: times N^-1, to [0, q))
    if (COLS) {
        const uint64_t ni = pc[p].ninv, nish = pc[p].ninv_sh;
#pragma unroll
        for (int k = 0; k < P::E; k++) a[(size_t)(h + P::T * k) * C + g] = csub(shoup(x[k], ni, nish, q), q);
    } else {
        uint64_t *dst = a + (size_t)g * P::M;
#pragma unroll
        for (int k = 0; k < P::E; k++) dst[h + P::T * k] = x[k];
    }
}

template <int S, bool FWD, bool COLS>
static void launch_pass(Ctx &c, const LimbMap &m, const char *cls)
{
    typedef PassShape<S> P;
    const int subs = COLS ? (c.N >> S) : (c.N >> S);  // columns or chunks
    dim3 grid(subs / P::SUB, m.count());
    ProfScope _ps(c, cls, (uint64_t)m.count());
    if (FWD) k_ntt_fwd_pass<S, COLS><<<grid, P::THREADS, 0, c.stream>>>(m, c.d_pc, c.d_twf, c.logN);
    else k_ntt_inv_pass<S, COLS><<<grid, P::THREADS, 0, c.stream>>>(m, c.d_pc, c.d_twi, c.logN);
    check_launch(cls);
}

template <bool FWD, bool COLS>
static void pass_dispatch(Ctx &c, const LimbMap &m, int S, const char *cls)
{
    switch (S) {
    case 5: launch_pass<5, FWD, COLS>(c, m, cls); break;
    case 6: launch_pass<6, FWD, COLS>(c, m, cls); break;
    case 7: launch_pass<7, FWD, COLS>(c, m, cls); break;
    case 8: launch_pass<8, FWD, COLS>(c, m, cls); break;
    default: throw_err(PPST_E_ARG, "unsupported ring degree for the NTT");
    }
}

// rows R = 2^ceil(logN/2) (COLS pass), chunks of C = 2^floor(logN/2) words
void ntt_fwd(Ctx &c, const LimbMap &m)
{
    if (m.count() == 0) return;
    const int sR = (c.logN + 1) / 2, sC = c.logN / 2;
    pass_dispatch<true, true>(c, m, sR, "ntt_cols_fwd");
    pass_dispatch<true, false>(c, m, sC, "ntt_chunks_fwd");
}

void ntt_inv(Ctx &c, const LimbMap &m)
{
    if (m.count() == 0) return;
    const int sR = (c.logN + 1) / 2, sC = c.logN / 2;
    pass_dispatch<false, false>(c, m, sC, "ntt_chunks_inv");
    pass_dispatch<false, true>(c, m, sR, "ntt_cols_inv");
}

}  // namespace ppst
