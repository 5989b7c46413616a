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
// #{n : p_min(n) = p_k} = cum_k - cum_{k-1}.  The n still open after KA primes
// (a few per thousand near 1e10) are appended to a slab-wide list.
//
// Phase B (k_cover_probe).  Each listed n probes the bit of Q at j + d_k for
// k = KA, KA+1, ... (four probes per step); the first set bit gives p_min.  One
// slab-wide list keeps every thread of the GPU busy; an n still open after K
// primes goes to the retry pass (or counts as unresolved).
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

// cumulative counts are kept two per register (16-bit halves): a lane adds at
// most 32 per word and handles fewer than 2^11 words per CTA
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
    if constexpr (K & 1) cum[K >> 1] += __popc(C) << 16;
    else cum[K >> 1] += __popc(C);
}

template <int NR, int KH, int... K>
__device__ __forceinline__ void phase_a(std::integer_sequence<int, K...>, const uint32_t (&R)[NR], uint32_t& C,
                                        uint32_t (&cum)[KH])
{
    (phase_a_step<K, NR, KH>(R, C, cum), ...);
}

template <int NT, int KA>
__global__ void __launch_bounds__(NT) k_cover_fast(const CoverArgs a, const OpenList open)
{
    constexpr int NW = NT / 32;
    constexpr int NR = window_regs(KA);
    constexpr int KH = KA / 2;
    __shared__ uint32_t shist[KA + 1];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // this CTA's words (32-bit words of C, 32 even n each)
    const uint64_t wps = 2ull * a.words_per_seg;
    const uint32_t seg = blockIdx.x / a.chunks_per_seg;
    const uint32_t chunk = blockIdx.x % a.chunks_per_seg;
    const uint64_t seg_w0 = (uint64_t)seg * wps;
    const uint64_t w_begin = seg_w0 + (uint64_t)chunk * (2ull * a.cta_words);
    uint64_t w_end = w_begin + 2ull * a.cta_words;
    const uint64_t n_words32 = (a.n_count + 31) / 32;
    if (w_end > seg_w0 + wps) w_end = seg_w0 + wps;
    if (w_end > n_words32) w_end = n_words32;

    for (int k = threadIdx.x; k <= KA; k += NT) shist[k] = 0;
    __syncthreads();

    const uint32_t* Qc = reinterpret_cast<const uint32_t*>(a.Q) + w_begin;   // CTA-relative words
    const uint32_t D0w = ((a.H - 4) >> 1) >> 5;            // word offset of the p = 3 partner
    const uint32_t nw_cta = (uint32_t)(w_end > w_begin ? w_end - w_begin : 0);
    const uint64_t n_left = a.n_count - 32 * w_begin;       // n from the CTA's first n to the slab end
    const uint32_t n_rel_end = (uint32_t)(n_left < 32ull * nw_cta ? n_left : 32ull * nw_cta);
    const uint32_t slab_n0 = (uint32_t)(32 * w_begin);      // slab-relative n of the CTA's first n

    uint32_t cum[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) cum[k] = 0;
    uint32_t init_pop = 0, nwords = 0;

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
                atomicAdd(&a.hist[(uint64_t)seg * a.hist_stride], 1u);
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

        // append the n still open
        uint32_t m = ~C;
        if (!__any_sync(0xffffffffu, m != 0)) continue;
        const uint32_t cnt = __popc(m);
        uint32_t pre = cnt;                                  // inclusive prefix over lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        uint32_t base = 0;
        if (lane == 31) base = atomicAdd(open.count, pre);
        base = __shfl_sync(0xffffffffu, base, 31);
        uint32_t pos = base + pre - cnt;
        const uint32_t j0 = slab_n0 + 32 * wrel;
        while (m) {
            const uint32_t b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < open.cap) open.n[pos] = j0 + b;
            ++pos;
        }
    }

    if (a.iters) {
        // first-phase word steps
        unsigned long long t = (unsigned long long)nwords * KA;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(a.iters, t);
    }
    // first-phase histogram from the cumulative counts
    uint32_t prev = __reduce_add_sync(0xffffffffu, init_pop);
#pragma unroll
    for (int k = 0; k < KA; ++k) {
        const uint32_t v = (k & 1) ? cum[k >> 1] >> 16 : cum[k >> 1] & 0xffffu;
        const uint32_t tot = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0 && tot != prev) atomicAdd(&shist[k + 1], tot - prev);
        prev = tot;
    }
    __syncthreads();
    uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    for (int k = 1 + threadIdx.x; k <= KA; k += NT)
        if (shist[k]) atomicAdd(&hrow[k], shist[k]);
}

// phase B: every thread walks the open list with a grid stride; one flat loop
// (probe up to four primes, or move to the next listed n) keeps lanes in step
__global__ void __launch_bounds__(256) k_cover_probe(const CoverArgs a, const OpenList open, uint32_t KA)
{
    const uint32_t total = min(*open.count, open.cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t* Q32 = reinterpret_cast<const uint32_t*>(a.Q);
    const uint32_t spn = 64 * a.words_per_seg;              // n per segment
    uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t j = 0, k = KA, nprobes = 0;
    if (e < total) j = open.n[e];
    while (e < total) {
        // probe k .. k+3; primes past K are never read
        uint32_t hit = 0;
        const uint32_t left = a.K - k;
        const uint32_t np = left < 4 ? left : 4u;
        for (uint32_t t = 0; t < np; ++t) {
            const uint32_t p = a.primes[1 + k + t];
            const uint64_t i = (uint64_t)j + ((a.H - p - 1) >> 1);
            hit |= ((__ldg(Q32 + (i >> 5)) >> (i & 31)) & 1u) << t;
        }
        nprobes += hit ? (uint32_t)__ffs(hit) : np;
        if (hit || left <= 4) {
            const uint32_t seg = j / spn;
            if (hit) {
                const uint32_t kk = k + (__ffs(hit) - 1);
                atomicAdd(&a.hist[(uint64_t)seg * a.hist_stride + kk + 1], 1u);
                const unsigned long long key =
                    ((unsigned long long)(kk + 2) << 32) | (0xffffffffull - (j - seg * spn));
                // keys only grow: a stale read can only cost an extra atomic
                if (key > *(volatile unsigned long long*)&a.maxkey[seg]) atomicMax(&a.maxkey[seg], key);
            } else {
                // open after every prime of this pass
                bool queued = false;
                if (a.retry) {
                    const unsigned int slot = atomicAdd(a.retry_count, 1u);
                    if (slot < a.retry_cap) {
                        a.retry[slot].w = j >> 6;
                        a.retry[slot].C = ~(1ull << (j & 63));
                        queued = true;
                    }
                }
                if (!queued) atomicAdd(&a.unresolved[seg], 1ull);
            }
            e += stride;
            k = KA;
            if (e < total) j = open.n[e];
        } else {
            k += 4;
        }
    }
    if (a.iters) {
        unsigned long long t = nprobes;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(a.iters, t);
    }
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
static cudaError_t launch_ka(const CoverArgs& a, const OpenList& open, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    k_cover_fast<NT, KA><<<grid, NT, 0, s>>>(a, open);
    return cudaGetLastError();
}

cudaError_t launch_cover_fast(const CoverArgs& a, const OpenList& open, int KA, cudaStream_t s)
{
    // 16-bit counters: a lane sums at most 32 per word over its words of a CTA
    if (2ull * a.cta_words > 2047ull * 256) return cudaErrorInvalidValue;
    switch (KA) {
    case 32: return launch_ka<32>(a, open, s);
    case 48: return launch_ka<48>(a, open, s);
    case 64: return launch_ka<64>(a, open, s);
    case 96: return launch_ka<96>(a, open, s);
    case 128: return launch_ka<128>(a, open, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cover_probe(const CoverArgs& a, const OpenList& open, int KA, cudaStream_t s)
{
    k_cover_probe<<<152 * 8, 256, 0, s>>>(a, open, (uint32_t)KA);
    return cudaGetLastError();
}

}  // namespace gb
