// gb_cover_fast.cu -- two-phase form of the loop-inverted Goldbach cover.
//
// Same computation as the generic cover (gb_cover.cu): for p = 3, 5, 7, ... <= P
// in ascending order, every even n whose partner n - p is prime and that no
// smaller p covered gets p_min(n) = p (GoldbachGPU, arXiv 2603.02621, Sec.
// 2.3.1-2.3.2, in the bitwise form of Sec. 4.3).  Only the schedule differs.
//
// Phase A (k_cover_fast).  Most n are covered by one of the first few dozen
// primes, so the first KA odd primes are applied to every coverage word
// unconditionally, with the loop unrolled at compile time.  A lane owns one
// 32-bit word of C (32 even n).  With the halo chosen so that d_3 = (H - 4)/2
// is a multiple of 32, the partner bits of word w for the prime p start at bit
// 32(w + d_3/32) - (p-3)/2 of Q: the word offset and the shift of every step
// are compile-time constants, and the few Q words a lane needs sit in
// registers.  A step is then
//     s = funnel-shift of two window registers,  C |= s,  cum_k += popc(C)
// and the histogram of the first phase follows from the cumulative counts:
// #{n : p_min(n) = p_k} = cum_k - cum_{k-1}.
//
// Phase B, in the same kernel while the CTA's part of Q is still in L1.  After
// each round of the first phase, the warp takes the n left open one at a time:
// lane t probes the bit of Q at j + d_k for k = KA + t (32 consecutive primes
// per step, a few cache lines), and the lowest set bit of the ballot is the
// minimal prime.  Most open n are settled in one step.  An n still open after
// K primes goes to the retry pass (or counts as unresolved).
//
// The largest p_min of a segment, with its smallest n, comes from phase B (or
// the retry pass).  A segment where no n needed more than KA primes gets its
// maximum from the generic kernel run in max-only mode.
#include <utility>

#include "gb_internal.cuh"

namespace gb {

// k-th odd prime (k = 0 -> 3), evaluated at compile time
__host__ __device__ constexpr uint32_t odd_prime(int k)
{
    uint32_t c = 1;
    int n = -1;
    while (n < k) {
        c += 2;
        bool prime = true;
        for (uint32_t d = 3; d * d <= c; d += 2)
            if (c % d == 0) { prime = false; break; }
        if (prime) ++n;
    }
    return c;
}

// window registers needed for KA primes: R[t] = Q32[base - t], t <= (e+31)/32
__host__ __device__ constexpr int window_regs(int KA)
{
    return (int)(((odd_prime(KA - 1) - 3) / 2 + 31) / 32) + 1;
}

// cumulative counts are kept three per register (10-bit fields): a lane adds
// at most 32 per word and handles at most 31 words per CTA (32 * 31 < 2^10)
constexpr int kCumBits = 10;
constexpr uint32_t kCumMask = (1u << kCumBits) - 1;
constexpr int kMaxWordsPerLane = 31;
__host__ __device__ constexpr int cum_regs(int KA) { return (KA + 2) / 3; }

template <int K, int NR, int KH>
__device__ __forceinline__ void phase_a_step(const uint32_t (&R)[NR], uint32_t& C, uint32_t (&cum)[KH])
{
    constexpr uint32_t e = (odd_prime(K) - 3) / 2;    // bit distance from p = 3
    constexpr uint32_t c = (e + 31) / 32;
    constexpr uint32_t sh = 32 * c - e;
    static_assert(c < (uint32_t)NR, "window too small");
    uint32_t s;
    if constexpr (sh == 0) s = R[c];
    else s = __funnelshift_r(R[c], R[c - 1], sh);
    C |= s;
    if constexpr (K % 3 == 0) cum[K / 3] += __popc(C);
    else cum[K / 3] += __popc(C) << (kCumBits * (K % 3));
}

template <int NR, int KH, int... K>
__device__ __forceinline__ void phase_a(std::integer_sequence<int, K...>, const uint32_t (&R)[NR], uint32_t& C,
                                        uint32_t (&cum)[KH])
{
    (phase_a_step<K, NR, KH>(R, C, cum), ...);
}

// Second phase, warp-wide: the 32 lanes probe 32 consecutive primes for one
// open n at a time; their partner bits lie within a few words of Q, so a step
// costs one or two cache lines, and the first set bit of the ballot is p_min.
template <int NT, int KA>
__global__ void __launch_bounds__(NT, KA <= 64 ? 4 : 3) k_cover_fast(const CoverArgs a)
{
    constexpr int NW = NT / 32;
    constexpr int NR = window_regs(KA);
    constexpr int KH = cum_regs(KA);
    extern __shared__ uint32_t smem[];
    uint32_t* sd = smem;                                    // d_k for the K odd primes
    uint32_t* shist = sd + a.K;                             // K + 1 counters
    __shared__ unsigned long long smax;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // this CTA's words (32-bit words of C, 32 even n each), all in one segment
    const uint64_t wps = 2ull * a.words_per_seg;
    const uint32_t seg = blockIdx.x / a.chunks_per_seg;
    const uint32_t chunk = blockIdx.x % a.chunks_per_seg;
    const uint64_t seg_w0 = (uint64_t)seg * wps;
    const uint64_t w_begin = seg_w0 + (uint64_t)chunk * (2ull * a.cta_words);
    uint64_t w_end = w_begin + 2ull * a.cta_words;
    const uint64_t n_words32 = (a.n_count + 31) / 32;
    if (w_end > seg_w0 + wps) w_end = seg_w0 + wps;
    if (w_end > n_words32) w_end = n_words32;

    for (uint32_t k = threadIdx.x; k < a.K; k += NT) sd[k] = (a.H - a.primes[1 + k] - 1) >> 1;
    for (uint32_t k = threadIdx.x; k <= a.K; k += NT) shist[k] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();

    const uint32_t* Qc = reinterpret_cast<const uint32_t*>(a.Q) + w_begin;   // CTA-relative words
    const uint32_t D0w = ((a.H - 4) >> 1) >> 5;            // word offset of the p = 3 partner
    const uint32_t nw_cta = (uint32_t)(w_end > w_begin ? w_end - w_begin : 0);
    const uint64_t n_left = a.n_count - 32 * w_begin;       // n from the CTA's first n to the slab end
    const uint32_t n_rel_end = (uint32_t)(n_left < 32ull * nw_cta ? n_left : 32ull * nw_cta);
    const uint32_t j_cta = (uint32_t)(32 * (w_begin - seg_w0));   // segment-relative n of the CTA's first n

    uint32_t cum[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) cum[k] = 0;
    uint32_t init_pop = 0, nwords = 0, nsteps = 0;
    unsigned long long best = 0;                            // lane 0 only

    for (uint32_t wbase = 32 * warp; wbase < nw_cta; wbase += 32 * NW) {
        const uint32_t wrel = wbase + lane;
        const bool active = wrel < nw_cta;
        uint32_t C = 0xffffffffu;
        uint32_t R[NR];
        if (active) {
            C = 0;
            const uint32_t j0 = 32 * wrel;
            if (n_rel_end - j0 < 32) C = 0xffffffffu << (n_rel_end - j0);   // past the slab end
            if (a.has_n4 && w_begin + wrel == 0) {
                C |= 1u;                                     // n = 4 = 2 + 2
                atomicAdd(&shist[0], 1u);
            }
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = __ldg(Qc + wrel + D0w - t);
        } else {
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = 0;
        }
        init_pop += __popc(C);
        nwords += active;
        phase_a<NR, KH>(std::make_integer_sequence<int, KA>{}, R, C, cum);

        // second phase for the n this round left open, one n at a time
        const uint32_t m = ~C;
        unsigned lanes = __ballot_sync(0xffffffffu, m != 0);
        while (lanes) {
            const int src = __ffs(lanes) - 1;
            lanes &= lanes - 1;
            uint32_t mm = __shfl_sync(0xffffffffu, m, src);
            while (mm) {
                const uint32_t b = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint32_t rel = 32 * (wbase + (uint32_t)src) + b;   // CTA-relative n index
                uint32_t k = KA;
                for (;;) {
                    const uint32_t kt = k + (uint32_t)lane;
                    uint32_t bit = 0;
                    if (kt < a.K) {
                        const uint32_t i = rel + sd[kt];
                        bit = (__ldg(Qc + (i >> 5)) >> (i & 31)) & 1u;
                    }
                    const unsigned hb = __ballot_sync(0xffffffffu, bit);
                    ++nsteps;
                    if (hb) {
                        const uint32_t kk = k + (__ffs(hb) - 1);
                        if (lane == 0) {
                            atomicAdd(&shist[kk + 1], 1u);
                            const unsigned long long key =
                                ((unsigned long long)(kk + 2) << 32) | (0xffffffffull - (j_cta + rel));
                            if (key > best) best = key;
                        }
                        break;
                    }
                    k += 32;
                    if (k >= a.K) {
                        // open after every prime of this pass
                        if (lane == 0) {
                            const uint64_t jn = 32 * w_begin + rel;          // slab-relative n index
                            bool queued = false;
                            if (a.retry) {
                                const unsigned int slot = atomicAdd(a.retry_count, 1u);
                                if (slot < a.retry_cap) {
                                    a.retry[slot].w = jn >> 6;
                                    a.retry[slot].C = ~(1ull << (jn & 63));
                                    queued = true;
                                }
                            }
                            if (!queued) atomicAdd(&a.unresolved[seg], 1ull);
                        }
                        break;
                    }
                }
            }
        }
    }

    if (a.iters) {
        // first-phase word steps plus second-phase probes (32 per warp step)
        unsigned long long t = (unsigned long long)nwords * KA + (lane == 0 ? 32ull * nsteps : 0ull);
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(a.iters, t);
    }
    // first-phase histogram from the cumulative counts
    uint32_t prev = __reduce_add_sync(0xffffffffu, init_pop);
#pragma unroll
    for (int kk = 0; kk < KA; ++kk) {
        const uint32_t v = (cum[kk / 3] >> (kCumBits * (kk % 3))) & kCumMask;
        const uint32_t tot = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0 && tot != prev) atomicAdd(&shist[kk + 1], tot - prev);
        prev = tot;
    }
    if (lane == 0 && best) atomicMax(&smax, best);
    __syncthreads();
    uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    for (uint32_t kk = threadIdx.x; kk <= a.K; kk += NT)
        if (shist[kk]) atomicAdd(&hrow[kk], shist[kk]);
    if (threadIdx.x == 0 && smax) atomicMax(&a.maxkey[seg], smax);
}

int cover_fast_phase_primes(uint32_t K, uint64_t n_hi)
{
    // first-phase length by magnitude: the share of n still open after KA
    // primes grows with log n (about 0.6% after 64 primes near 1e10, 0.6%
    // after 128 near 4e18), and a second-phase probe costs several first-phase
    // steps' worth of work per n
    int want = n_hi < 1000000000ull ? 48 : n_hi < 100000000000ull ? 64 : n_hi < 100000000000000ull ? 96 : 128;
    const int opts[5] = {128, 96, 64, 48, 32};
    for (int o : opts)
        if (o <= want && (uint32_t)o <= K) return o;
    return 0;
}

template <int KA>
static cudaError_t launch_ka(const CoverArgs& a, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * a.K + 1) * 4;
    auto k = k_cover_fast<NT, KA>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cover_fast(const CoverArgs& a, int KA, cudaStream_t s)
{
    // 10-bit counters hold a lane's sum of at most 32 per word over its words
    // of a CTA
    if (2ull * a.cta_words > (unsigned long long)kMaxWordsPerLane * 256) return cudaErrorInvalidValue;
    switch (KA) {
    case 32: return launch_ka<32>(a, s);
    case 48: return launch_ka<48>(a, s);
    case 64: return launch_ka<64>(a, s);
    case 96: return launch_ka<96>(a, s);
    case 128: return launch_ka<128>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
