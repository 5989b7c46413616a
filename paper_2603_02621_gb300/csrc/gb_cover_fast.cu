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
// Phase B, in the same kernel while the warp's part of Q is still in L1.  The
// n still open after KA primes (a few per thousand near 1e10) are queued per
// warp in shared memory; each probes the bit of Q at j + d_k for k = KA,
// KA+1, ... (four probes per step), the first set bit giving p_min.  A lane
// keeps the n it is working on across drains and takes a new one from the
// queue when it finishes, and a drain stops once the queue is handed out.  The
// kernel is persistent: each warp takes chunks of coverage words from a global
// counter until none are left, carrying its unfinished n from chunk to chunk,
// so only its very last drain waits for its slowest n.  An n still open after
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
// at most 32 per word over the 16 words it takes in a chunk (512 < 2^10)
constexpr int kCumBits = 10;
constexpr uint32_t kCumMask = (1u << kCumBits) - 1;
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

constexpr int kQueueCap = 1024;      // queued n per warp (one round adds at most 1024)
constexpr int kQueueRun = 128;       // drain once this many n wait
constexpr uint32_t kChunkWords = 512;   // 32-bit coverage words per warp chunk (16 rounds)

// shared-memory layout (uint32 units): offsets table with 4 zero entries past
// K (the 4-wide probes may read them; their results are masked), then the
// 16-bit per-warp queues
__host__ __device__ constexpr uint32_t sd_len(uint32_t K) { return (K + 4 + 3) & ~3u; }

// Persistent kernel: each warp takes chunks of kChunkWords coverage words (all
// in one segment) from a global counter until none are left.
template <int NT, int KA>
__global__ void __launch_bounds__(NT, KA <= 64 ? 4 : 3) k_cover_fast(const CoverArgs a, unsigned int* chunk_ctr,
                                                                      uint32_t chunks_per_seg, uint32_t total_chunks)
{
    constexpr int NW = NT / 32;
    constexpr int NR = window_regs(KA);
    constexpr int KH = cum_regs(KA);
    extern __shared__ uint32_t smem[];
    uint32_t* sd = smem;                                    // d_k, K entries + 4 pad (0)
    uint16_t* queues = reinterpret_cast<uint16_t*>(sd + sd_len(a.K));   // NW * kQueueCap

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t* queue = queues + warp * kQueueCap;
    // queue entry: round << 10 | lane << 5 | bit: the n at chunk-relative index
    // 32 * (32 * round + lane) + bit

    for (uint32_t k = threadIdx.x; k < sd_len(a.K); k += NT) sd[k] = k < a.K ? (a.H - a.primes[1 + k] - 1) >> 1 : 0u;
    __syncthreads();

    const uint32_t* Q32 = reinterpret_cast<const uint32_t*>(a.Q);
    const uint32_t D0w = ((a.H - 4) >> 1) >> 5;            // word offset of the p = 3 partner
    const uint64_t wps = 2ull * a.words_per_seg;            // 32-bit words per segment
    const uint64_t spn = 32 * wps;                          // n per segment
    const uint64_t n_words32 = (a.n_count + 31) / 32;

    // phase-B state of each lane, parked in shared memory during the first
    // phase so that it takes no registers there (k = 0: no n held)
    __shared__ unsigned long long hold_n[NT];
    __shared__ uint32_t hold_k[NT];
    __shared__ uint32_t hold_probes[NT];
    hold_k[threadIdx.x] = 0;
    hold_probes[threadIdx.x] = 0;
    __syncwarp();

    uint32_t nwords = 0;
    int qn = 0;                                             // warp-uniform queue length
    uint64_t c_w0 = 0;                                      // first word of the current chunk

    // hand out the queued n; with final set, also finish every n in flight
    auto drain = [&](bool final) {
        __syncwarp();
        uint32_t k = hold_k[threadIdx.x];
        bool act = k != 0;
        uint64_t n = hold_n[threadIdx.x];
        uint32_t nprobes = hold_probes[threadIdx.x];
        uint32_t next = 0;
        for (;;) {
            const unsigned idle = __ballot_sync(0xffffffffu, !act);
            if (idle && next < (uint32_t)qn) {
                const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
                if (!act && next + rank < (uint32_t)qn) {
                    const uint32_t q = queue[next + rank];
                    act = true;
                    n = 32 * c_w0 + ((((q >> 10) * 32) + ((q >> 5) & 31)) << 5) + (q & 31);
                    k = KA;
                }
                next += __popc(idle);
            }
            if (!final && next >= (uint32_t)qn) break;      // queue handed out
            if (!__any_sync(0xffffffffu, act)) break;
            if (act) {
                uint32_t hit = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t i = n + sd[k + t];
                    hit |= ((__ldg(Q32 + (i >> 5)) >> (i & 31)) & 1u) << t;
                }
                const uint32_t left = a.K - k;
                if (left < 4) hit &= (1u << left) - 1u;
                nprobes += hit ? (uint32_t)__ffs(hit) : (left < 4 ? left : 4u);
                if (hit || left <= 4) {
                    const uint32_t seg = (uint32_t)(n / spn);
                    if (hit) {
                        const uint32_t kk = k + (__ffs(hit) - 1);
                        atomicAdd(&a.hist[(uint64_t)seg * a.hist_stride + kk + 1], 1u);
                        const unsigned long long key =
                            ((unsigned long long)(kk + 2) << 32) | (0xffffffffull - (uint32_t)(n - seg * spn));
                        // keys only grow: a stale read only costs an extra atomic
                        if (key > *(volatile unsigned long long*)&a.maxkey[seg]) atomicMax(&a.maxkey[seg], key);
                    } else {
                        // open after every prime of this pass
                        bool queued = false;
                        if (a.retry) {
                            const unsigned int slot = atomicAdd(a.retry_count, 1u);
                            if (slot < a.retry_cap) {
                                a.retry[slot].w = n >> 6;
                                a.retry[slot].C = ~(1ull << (n & 63));
                                queued = true;
                            }
                        }
                        if (!queued) atomicAdd(&a.unresolved[seg], 1ull);
                    }
                    act = false;
                } else {
                    k += 4;
                }
            }
        }
        hold_k[threadIdx.x] = act ? k : 0u;
        hold_n[threadIdx.x] = n;
        hold_probes[threadIdx.x] = nprobes;
        __syncwarp();
        qn = 0;
    };

    for (;;) {
        uint32_t chunk = 0;
        if (lane == 0) chunk = atomicAdd(chunk_ctr, 1u);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= total_chunks) break;
        const uint32_t seg = chunk / chunks_per_seg;
        const uint64_t seg_w0 = (uint64_t)seg * wps;
        const uint64_t w0 = seg_w0 + (uint64_t)(chunk % chunks_per_seg) * kChunkWords;
        uint64_t w1 = w0 + kChunkWords;
        if (w1 > seg_w0 + wps) w1 = seg_w0 + wps;
        if (w1 > n_words32) w1 = n_words32;
        if (w0 >= w1) continue;
        if (qn) drain(false);                                 // queue entries are chunk-relative
        c_w0 = w0;
        const uint32_t nw = (uint32_t)(w1 - w0);
        const uint64_t n_left = a.n_count - 32 * w0;
        const uint32_t n_rel_end = (uint32_t)(n_left < 32ull * nw ? n_left : 32ull * nw);
        const uint32_t* Qc = Q32 + w0;

        uint32_t cum[KH];
#pragma unroll
        for (int kk = 0; kk < KH; ++kk) cum[kk] = 0;
        uint32_t init_pop = 0;

        uint32_t round = 0;
        for (uint32_t wbase = 0; wbase < nw; wbase += 32, ++round) {
            const uint32_t wrel = wbase + lane;
            const bool active = wrel < nw;
            uint32_t C = 0xffffffffu;
            uint32_t R[NR];
            if (active) {
                C = 0;
                const uint32_t j0 = 32 * wrel;
                if (n_rel_end - j0 < 32) C = 0xffffffffu << (n_rel_end - j0);   // past the slab end
                if (a.has_n4 && w0 + wrel == 0) {
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

            // queue the n still open
            uint32_t m = ~C;
            if (!__any_sync(0xffffffffu, m != 0)) continue;
            const uint32_t cnt = __popc(m);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (qn + (int)total > kQueueCap) drain(false);
            uint32_t pos = qn + incl - cnt;
            const uint32_t tag = (round << 10) | ((uint32_t)lane << 5);
            while (m) {
                const uint32_t b = __ffs(m) - 1;
                m &= m - 1;
                queue[pos++] = (uint16_t)(tag | b);
            }
            qn += (int)total;
            if (qn >= kQueueRun) drain(false);
        }
        // first-phase histogram of the chunk from the cumulative counts
        uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
        uint32_t prev = __reduce_add_sync(0xffffffffu, init_pop);
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            const uint32_t v = (cum[kk / 3] >> (kCumBits * (kk % 3))) & kCumMask;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, v);
            if (lane == 0 && tot != prev) atomicAdd(&hrow[kk + 1], tot - prev);
            prev = tot;
        }
    }
    drain(true);

    if (a.iters) {
        // first-phase word steps plus second-phase probes
        unsigned long long t = (unsigned long long)nwords * KA + hold_probes[threadIdx.x];
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(a.iters, t);
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
static cudaError_t launch_ka(const CoverArgs& a, unsigned int* chunk_ctr, cudaStream_t s)
{
    constexpr int NT = 256;
    const uint64_t wps = 2ull * a.words_per_seg;
    const uint32_t chunks_per_seg = (uint32_t)((wps + kChunkWords - 1) / kChunkWords);
    const uint64_t total = (uint64_t)a.nseg * chunks_per_seg;
    if (total == 0) return cudaSuccess;
    if (total > 0xffffffffull) return cudaErrorInvalidValue;
    const size_t smem = (size_t)sd_len(a.K) * 4 + (size_t)(NT / 32) * kQueueCap * 2;
    auto k = k_cover_fast<NT, KA>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess) return e;
    // one resident wave of persistent CTAs (fewer if there are few chunks)
    uint64_t grid = (uint64_t)sms * (per_sm > 0 ? per_sm : 1);
    const uint64_t need = (total + (NT / 32) - 1) / (NT / 32);
    if (grid > need) grid = need;
    if ((e = cudaMemsetAsync(chunk_ctr, 0, sizeof(unsigned int), s)) != cudaSuccess) return e;
    k<<<(unsigned)grid, NT, smem, s>>>(a, chunk_ctr, chunks_per_seg, (uint32_t)total);
    return cudaGetLastError();
}

cudaError_t launch_cover_fast(const CoverArgs& a, unsigned int* chunk_ctr, int KA, cudaStream_t s)
{
    switch (KA) {
    case 32: return launch_ka<32>(a, chunk_ctr, s);
    case 48: return launch_ka<48>(a, chunk_ctr, s);
    case 64: return launch_ka<64>(a, chunk_ctr, s);
    case 96: return launch_ka<96>(a, chunk_ctr, s);
    case 128: return launch_ka<128>(a, chunk_ctr, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
