// gb_cover_fast.cu -- two-phase form of the loop-inverted Goldbach cover.
//
// Same computation as the generic cover (gb_cover.cu): for p = 3, 5, 7, ... <= P
// in ascending order, every even n whose partner n - p is prime and that no
// smaller p covered gets p_min(n) = p (GoldbachGPU, arXiv 2603.02621, Sec.
// 2.3.1-2.3.2, in the bitwise form of Sec. 4.3).  Only the schedule differs.
//
// Unrolled blocks.  Most n are covered by one of the first few dozen primes,
// so primes are applied in blocks of 64, unrolled at compile time.  A lane owns
// one 32-bit word of C (32 even n).  With the halo chosen so that
// d_3 = (H - 4)/2 is a multiple of 32, the partner bits of word w for the
// prime p start at bit 32(w + d_3/32) - (p-3)/2 of Q: the word offset and the
// shift of every step are compile-time constants, and the few Q words a lane
// needs sit in registers.  A step is then
//     s = funnel-shift of two window registers,  C |= s,  cum_k += popc(C)
// and the histogram follows from the cumulative counts:
// #{n : p_min(n) = p_k} = cum_k - cum_{k-1}.  The first block runs on every
// word of the CTA; the words it leaves open (about one in five near 1e10) are
// compacted in shared memory and the next block runs on those alone, so every
// lane of every step still works on an open word.
//
// Probing.  The few n open after the last block (about 1 in 10^5 near 1e10)
// are taken one at a time by a warp: lane t probes the bit of Q at j + d_k for
// k = k0 + t, and the lowest set bit of the ballot is p_min.  An n still open
// after K primes goes to the retry pass (or counts as unresolved).
//
// The largest p_min of a CTA's words, with its smallest n, comes from the
// probing when any n reached it; otherwise the last block that ran holds it,
// and that block is run once more over its input words, recording for each
// word the last step that set a bit.
#include <type_traits>
#include <utility>

#include "gb_internal.cuh"
#include "gb_sieve_tile.cuh"

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

// cumulative counts are kept three per register (10-bit fields): a lane adds
// at most 32 per word and handles at most 31 words per CTA in a block
// (32 * 31 < 2^10)
constexpr int kCumBits = 10;
constexpr uint32_t kCumMask = (1u << kCumBits) - 1;
__host__ __device__ constexpr int cum_regs(int KA) { return (KA + 2) / 3; }

// ---------------------------------------------------------------------------
// one unrolled block of 64 primes: indices K0 .. K0+63, window registers
// R[t] = Q32[base - C0 - t] with C0 = the first block step's word offset - 1
// ---------------------------------------------------------------------------
constexpr int kBlock = 64;

__host__ __device__ constexpr uint32_t step_e(int k) { return (odd_prime(k) - 3) / 2; }
__host__ __device__ constexpr int block_c0(int K0)
{
    return K0 == 0 ? 0 : (int)((step_e(K0) + 31) / 32) - 1;
}
__host__ __device__ constexpr int block_regs(int K0)
{
    return (int)((step_e(K0 + kBlock - 1) + 31) / 32) - block_c0(K0) + 1;
}

template <int K, int K0, int NR, int KH>
__device__ __forceinline__ void block_step(const uint32_t (&R)[NR], uint32_t& C, uint32_t (&cum)[KH])
{
    constexpr uint32_t e = step_e(K);
    constexpr int c = (int)((e + 31) / 32);
    constexpr uint32_t sh = 32 * c - e;
    constexpr int r = c - block_c0(K0);
    static_assert(r >= 0 && r < NR, "window too small");
    uint32_t s;
    if constexpr (sh == 0) s = R[r];
    else s = __funnelshift_r(R[r], R[r - 1], sh);
    C |= s;
    constexpr int j = K - K0;
    if constexpr (j % 3 == 0) cum[j / 3] += __popc(C);
    else cum[j / 3] += __popc(C) << (kCumBits * (j % 3));
}

template <int K0, int NR, int KH, int... J>
__device__ __forceinline__ void run_block(std::integer_sequence<int, J...>, const uint32_t (&R)[NR], uint32_t& C,
                                          uint32_t (&cum)[KH])
{
    (block_step<K0 + J, K0, NR, KH>(R, C, cum), ...);
}

// add one block's histogram (cumulative counts, warp-reduced) to shist
template <int K0, int KH>
__device__ __forceinline__ void flush_block(const uint32_t (&cum)[KH], uint32_t init_pop, uint32_t* shist, int lane)
{
    uint32_t prev = __reduce_add_sync(0xffffffffu, init_pop);
#pragma unroll
    for (int j = 0; j < kBlock; ++j) {
        const uint32_t v = (cum[j / 3] >> (kCumBits * (j % 3))) & kCumMask;
        const uint32_t tot = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0 && tot != prev) atomicAdd(&shist[K0 + j + 1], tot - prev);
        prev = tot;
    }
}

// ---------------------------------------------------------------------------
// block 0 on three consecutive words per lane.  The histogram needs, per step,
// popc(C0) + popc(C1) + popc(C2); a carry-save adder gives it with two
// popcounts: ones = C0 ^ C1 ^ C2, twos = majority(C0, C1, C2), and
// popc(C0) + popc(C1) + popc(C2) = popc(ones) + 2 popc(twos).
// Window: R[t] = Q32[w + 2 + d_3/32 - t] for the lane's first word w.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int block0_regs3() { return (int)((step_e(kBlock - 1) + 31) / 32) + 3; }

template <int K, int NR3, int KH>
__device__ __forceinline__ void step3(const uint32_t (&R)[NR3], uint32_t& C0, uint32_t& C1, uint32_t& C2,
                                      uint32_t (&cum)[KH])
{
    constexpr uint32_t e = step_e(K);
    constexpr int c = (int)((e + 31) / 32);
    constexpr uint32_t sh = 32 * c - e;
    static_assert(c + 2 < NR3, "window too small");
    uint32_t s0, s1, s2;
    if constexpr (sh == 0) {
        s0 = R[c + 2]; s1 = R[c + 1]; s2 = R[c];
    } else {
        s0 = __funnelshift_r(R[c + 2], R[c + 1], sh);
        s1 = __funnelshift_r(R[c + 1], R[c], sh);
        s2 = __funnelshift_r(R[c], R[c - 1], sh);
    }
    C0 |= s0;
    C1 |= s1;
    C2 |= s2;
    const uint32_t ones = C0 ^ C1 ^ C2;
    const uint32_t twos = (C0 & C1) | (C0 & C2) | (C1 & C2);
    const uint32_t t = __popc(ones) + 2 * __popc(twos);
    if constexpr (K % 3 == 0) cum[K / 3] += t;
    else cum[K / 3] += t << (kCumBits * (K % 3));
}

template <int NR3, int KH, int... J>
__device__ __forceinline__ void run_block0_3(std::integer_sequence<int, J...>, const uint32_t (&R)[NR3], uint32_t& C0,
                                             uint32_t& C1, uint32_t& C2, uint32_t (&cum)[KH])
{
    (step3<J, NR3, KH>(R, C0, C1, C2, cum), ...);
}


// Re-run block K0 over its input list recording, per word, the last step that
// set a bit and the lowest bit it set: the largest p_min among the list's
// words, with its smallest n.  Used when no n of the CTA outlived the blocks.
template <int K, int K0, int NR>
__device__ __forceinline__ void track_step(const uint32_t (&R)[NR], uint32_t& C, uint32_t& last, uint32_t& lastbits)
{
    constexpr uint32_t e = step_e(K);
    constexpr int c = (int)((e + 31) / 32);
    constexpr uint32_t sh = 32 * c - e;
    constexpr int r = c - block_c0(K0);
    uint32_t s;
    if constexpr (sh == 0) s = R[r];
    else s = __funnelshift_r(R[r], R[r - 1], sh);
    const uint32_t nw = s & ~C;
    C |= s;
    if (nw) { last = K + 1; lastbits = nw; }
}

template <int K0, int NR, int... J>
__device__ __forceinline__ void track_block_steps(std::integer_sequence<int, J...>, const uint32_t (&R)[NR],
                                                  uint32_t& C, uint32_t& last, uint32_t& lastbits)
{
    (track_step<K0 + J, K0, NR>(R, C, last, lastbits), ...);
}

// step of a tracked block: also records the last step that set a bit and the
// bits it set
template <int K, int K0, int NR, int KH>
__device__ __forceinline__ void block_step_tracked(const uint32_t (&R)[NR], uint32_t& C, uint32_t (&cum)[KH],
                                                   uint32_t& last, uint32_t& lastbits)
{
    constexpr uint32_t e = step_e(K);
    constexpr int c = (int)((e + 31) / 32);
    constexpr uint32_t sh = 32 * c - e;
    constexpr int r = c - block_c0(K0);
    static_assert(r >= 0 && r < NR, "window too small");
    uint32_t s;
    if constexpr (sh == 0) s = R[r];
    else s = __funnelshift_r(R[r], R[r - 1], sh);
    const uint32_t nw = s & ~C;
    C |= s;
    if (nw) { last = K + 1; lastbits = nw; }
    constexpr int j = K - K0;
    if constexpr (j % 3 == 0) cum[j / 3] += __popc(C);
    else cum[j / 3] += __popc(C) << (kCumBits * (j % 3));
}

template <int K0, int NR, int KH, int... J>
__device__ __forceinline__ void run_block_tracked(std::integer_sequence<int, J...>, const uint32_t (&R)[NR],
                                                  uint32_t& C, uint32_t (&cum)[KH], uint32_t& last,
                                                  uint32_t& lastbits)
{
    (block_step_tracked<K0 + J, K0, NR, KH>(R, C, cum, last, lastbits), ...);
}

// a word of the q window: read-only global load, or a shared-memory load when
// the window is a tile the same CTA has just sieved (fused kernel)
template <bool SQ>
__device__ __forceinline__ uint32_t ldq(const uint32_t* p)
{
    if constexpr (SQ) return *p;
    else return __ldg(p);
}

// block K0 on one word with tracking only (no histogram): the key of its
// largest p_min with the smallest n, 0 if the block set no bit
template <int K0, bool SQ>
__device__ __forceinline__ unsigned long long track_word(const uint32_t* Qc, uint32_t D0w, uint32_t wrel, uint32_t C,
                                                         uint32_t j_cta)
{
    constexpr int NR = block_regs(K0);
    constexpr int C0 = block_c0(K0);
    uint32_t R[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) R[t] = ldq<SQ>(Qc + wrel + D0w - C0 - t);
    uint32_t last = 0, lastbits = 0;
    track_block_steps<K0, NR>(std::make_integer_sequence<int, kBlock>{}, R, C, last, lastbits);
    if (!last) return 0;
    const uint32_t j = j_cta + 32 * wrel + (__ffs(lastbits) - 1);
    return ((unsigned long long)(last + 1) << 32) | (0xffffffffull - j);
}

// Later block K0 over a warp's list, batches of 32 words (one per lane),
// with per-word tracking of the last step that set a bit; words still open
// are compacted in place at the front of the list (writes never pass reads).
template <int K0, bool SQ>
__device__ __forceinline__ uint32_t later_block_warp(const uint32_t* Qc, uint32_t D0w, uint16_t* lw, uint32_t* lc,
                                                     uint32_t n_in, uint32_t* shist, uint32_t j_cta,
                                                     unsigned long long& best, uint32_t& nsteps)
{
    constexpr int NR = block_regs(K0);
    constexpr int KH = (kBlock + 2) / 3;
    constexpr int C0 = block_c0(K0);
    const int lane = threadIdx.x & 31;
    uint32_t cum[KH];
#pragma unroll
    for (int j = 0; j < KH; ++j) cum[j] = 0;
    uint32_t init_pop = 0, n_out = 0;
    for (uint32_t b = 0; b < n_in; b += 32) {
        const uint32_t e = b + lane;
        const bool active = e < n_in;
        uint32_t C = 0xffffffffu, wrel = 0;
        uint32_t R[NR];
        if (active) {
            wrel = lw[e];
            C = lc[e];
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = ldq<SQ>(Qc + wrel + D0w - C0 - t);
        } else {
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = 0;
        }
        __syncwarp();                                      // the batch is read before outputs land
        init_pop += __popc(C);
        nsteps += active ? kBlock : 0;
        uint32_t last = 0, lastbits = 0;
        run_block_tracked<K0, NR, KH>(std::make_integer_sequence<int, kBlock>{}, R, C, cum, last, lastbits);
        if (last) {
            const uint32_t j = j_cta + 32 * wrel + (__ffs(lastbits) - 1);
            const unsigned long long key = ((unsigned long long)(last + 1) << 32) | (0xffffffffull - j);
            if (key > best) best = key;
        }
        const bool open = C != 0xffffffffu;
        const unsigned m = __ballot_sync(0xffffffffu, open);
        if (open) {
            const uint32_t slot = n_out + __popc(m & ((1u << lane) - 1u));
            lw[slot] = (uint16_t)wrel;
            lc[slot] = C;
        }
        n_out += __popc(m);
        __syncwarp();
    }
    flush_block<K0, KH>(cum, init_pop, shist, lane);
    return n_out;
}

// Probing over a warp's list: the warp takes the open n one at a time, lane t
// probing the prime k + t; the lowest set bit of the ballot is p_min.
template <bool SQ>
__device__ __forceinline__ void probe_warp(const CoverArgs& a, const uint32_t* Qc, const uint16_t* lw,
                                           const uint32_t* lc, uint32_t n_in, uint32_t k_first, uint64_t w_begin,
                                           uint32_t j_cta, uint32_t seg, unsigned long long& best, uint32_t& nsteps)
{
    const int lane = threadIdx.x & 31;
    for (uint32_t e = 0; e < n_in; ++e) {
        const uint32_t wrel = lw[e];
        uint32_t mm = ~lc[e];
        while (mm) {
            const uint32_t b = __ffs(mm) - 1;
            mm &= mm - 1;
            const uint32_t rel = 32 * wrel + b;              // CTA-relative n index
            uint32_t k = k_first;
            for (;;) {
                const uint32_t kt = k + (uint32_t)lane;
                uint32_t bit = 0;
                if (kt < a.K) {
                    const uint32_t i = rel + ((a.H - __ldg(a.primes + 1 + kt) - 1) >> 1);
                    bit = (ldq<SQ>(Qc + (i >> 5)) >> (i & 31)) & 1u;
                }
                const unsigned hb = __ballot_sync(0xffffffffu, bit);
                if (lane == 0) nsteps += 32;
                if (hb) {
                    const uint32_t kk = k + (__ffs(hb) - 1);
                    if (lane == 0) {
                        atomicAdd(&a.hist[(uint64_t)seg * a.hist_stride + kk + 1], 1u);
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

// NB unrolled blocks of 64 primes (block 0 over every word, three words per
// lane; later blocks over the words still open, per warp), then per-n probing.
// One chunk of coverage words [w_begin, w_end) (32-bit words of the window
// a.Q, 32 even n each), all in segment (row) seg, whose first n has
// segment-relative index j_cta.  Called by every thread of the CTA; smem holds
// the per-warp lists; shist / smax are the CTA's shared counters.
template <int NT, int NB, bool SQ>
__device__ __forceinline__ void cover_chunk(const CoverArgs& a, const uint32_t* Qc, uint32_t seg, uint64_t w_begin,
                                            uint64_t w_end, uint32_t j_cta, uint32_t* smem, uint32_t* shist,
                                            unsigned long long& smax)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // a warp's list holds every word it takes in block 0
    const uint32_t cap = (2 * a.cta_words + 96 * NW - 1) / (96 * NW) * 96;
    uint32_t* lc = smem + (uint32_t)warp * cap;
    uint16_t* lw = reinterpret_cast<uint16_t*>(smem + NW * cap) + (uint32_t)warp * cap;

    __syncthreads();                                        // shared counters free (previous chunk)
    for (uint32_t k = threadIdx.x; k <= (uint32_t)(kBlock * NB); k += NT) shist[k] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();

    const uint32_t D0w = ((a.H - 4) >> 1) >> 5;            // word offset of the p = 3 partner
    const uint32_t nw_cta = (uint32_t)(w_end > w_begin ? w_end - w_begin : 0);
    const uint64_t n_left = a.n_count - 32 * w_begin;       // n from the CTA's first n to the window end
    const uint32_t n_rel_end = (uint32_t)(n_left < 32ull * nw_cta ? n_left : 32ull * nw_cta);

    uint32_t nsteps = 0, n_open = 0;
    // block 0 over every word of this warp, three consecutive words per lane
    {
        constexpr int NR3 = block0_regs3();
        constexpr int KH = (kBlock + 2) / 3;
        uint32_t cum[KH];
#pragma unroll
        for (int k = 0; k < KH; ++k) cum[k] = 0;
        uint32_t init_pop = 0;
        for (uint32_t wbase = 96 * warp; wbase < nw_cta; wbase += 96 * NW) {
            const uint32_t wl = wbase + 3 * (uint32_t)lane;           // the lane's first word
            uint32_t Cw[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const uint32_t w = wl + i;
                uint32_t C = 0xffffffffu;
                if (w < nw_cta) {
                    C = 0;
                    const uint32_t j0 = 32 * w;
                    if (n_rel_end - j0 < 32) C = 0xffffffffu << (n_rel_end - j0);   // past the slab end
                    if (a.has_n4 && w_begin + w == 0) {
                        C |= 1u;                                         // n = 4 = 2 + 2
                        atomicAdd(&shist[0], 1u);
                    }
                    nsteps += kBlock;
                }
                Cw[i] = C;
                init_pop += __popc(C);
            }
            uint32_t R[NR3];
            if (wl < nw_cta) {
                // the top word read, wl + 2, lies at most one word past the CTA's
                // last word: inside the q window, which runs past the slab
#pragma unroll
                for (int t = 0; t < NR3; ++t) R[t] = ldq<SQ>(Qc + wl + 2 + D0w - t);
            } else {
#pragma unroll
                for (int t = 0; t < NR3; ++t) R[t] = 0;
            }
            uint32_t C0 = Cw[0], C1 = Cw[1], C2 = Cw[2];
            run_block0_3<NR3, KH>(std::make_integer_sequence<int, kBlock>{}, R, C0, C1, C2, cum);
            Cw[0] = C0; Cw[1] = C1; Cw[2] = C2;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const bool open = Cw[i] != 0xffffffffu;
                const unsigned m = __ballot_sync(0xffffffffu, open);
                if (open) {
                    const uint32_t slot = n_open + __popc(m & ((1u << lane) - 1u));
                    lw[slot] = (uint16_t)(wl + i);
                    lc[slot] = Cw[i];
                }
                n_open += __popc(m);
            }
        }
        flush_block<0, KH>(cum, init_pop, shist, lane);
    }
    __syncwarp();
    unsigned long long best = 0;
    if constexpr (NB >= 2) n_open = later_block_warp<64, SQ>(Qc, D0w, lw, lc, n_open, shist, j_cta, best, nsteps);
    if constexpr (NB >= 3) n_open = later_block_warp<128, SQ>(Qc, D0w, lw, lc, n_open, shist, j_cta, best, nsteps);
    if constexpr (NB >= 4) n_open = later_block_warp<192, SQ>(Qc, D0w, lw, lc, n_open, shist, j_cta, best, nsteps);
    probe_warp<SQ>(a, Qc, lw, lc, n_open, (uint32_t)(kBlock * NB), w_begin, j_cta, seg, best, nsteps);

    // maximum: warp, CTA
    {
        const uint32_t khi = (uint32_t)(best >> 32);
        const uint32_t mhi = __reduce_max_sync(0xffffffffu, khi);
        const uint32_t klo = khi == mhi ? (uint32_t)best : 0u;
        const uint32_t mlo = __reduce_max_sync(0xffffffffu, klo);
        if (lane == 0 && mhi) atomicMax(&smax, ((unsigned long long)mhi << 32) | mlo);
    }
    __syncthreads();
    if (smax == 0) {
        // every n of the CTA was settled in block 0 (or stayed open): run block
        // 0 again over every word, recording each word's last covering step
        best = 0;
        for (uint32_t w = threadIdx.x; w < nw_cta; w += NT) {
            uint32_t C = 0;
            const uint32_t j0 = 32 * w;
            if (n_rel_end - j0 < 32) C = 0xffffffffu << (n_rel_end - j0);
            if (a.has_n4 && w_begin + w == 0) C |= 1u;
            const unsigned long long key = track_word<0, SQ>(Qc, D0w, (uint32_t)w, C, j_cta);
            if (key > best) best = key;
        }
        if (a.has_n4 && w_begin == 0 && threadIdx.x == 0) {
            // n = 4 (p_min 2, prime index 0) if nothing larger was found
            const unsigned long long k4 = (1ull << 32) | 0xffffffffull;
            if (k4 > best) best = k4;
        }
        const uint32_t khi = (uint32_t)(best >> 32);
        const uint32_t mhi = __reduce_max_sync(0xffffffffu, khi);
        const uint32_t klo = khi == mhi ? (uint32_t)best : 0u;
        const uint32_t mlo = __reduce_max_sync(0xffffffffu, klo);
        if (lane == 0 && mhi) atomicMax(&smax, ((unsigned long long)mhi << 32) | mlo);
        __syncthreads();
    }

    if (a.iters) {
        // unrolled word steps plus probes
        unsigned long long t = nsteps;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(a.iters, t);
    }
    uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    for (uint32_t kk = threadIdx.x; kk <= (uint32_t)(kBlock * NB); kk += NT)
        if (shist[kk]) atomicAdd(&hrow[kk], shist[kk]);
    if (threadIdx.x == 0 && smax) atomicMax(&a.maxkey[seg], smax);
}

template <int NT, int NB>
__global__ void __launch_bounds__(NT, 4) k_cover_fast(const CoverArgs a)
{
    extern __shared__ uint32_t smem[];                      // per warp: list C (32-bit), then words (16-bit)
    __shared__ uint32_t shist[kBlock * NB + 1];             // bins of the unrolled blocks' primes
    __shared__ unsigned long long smax;
    // this CTA's words, all in one segment
    const uint64_t wps = 2ull * a.words_per_seg;
    const uint32_t seg = blockIdx.x / a.chunks_per_seg;
    const uint32_t chunk = blockIdx.x % a.chunks_per_seg;
    const uint64_t seg_w0 = (uint64_t)seg * wps;
    const uint64_t w_begin = seg_w0 + (uint64_t)chunk * (2ull * a.cta_words);
    uint64_t w_end = w_begin + 2ull * a.cta_words;
    const uint64_t n_words32 = (a.n_count + 31) / 32;
    if (w_end > seg_w0 + wps) w_end = seg_w0 + wps;
    if (w_end > n_words32) w_end = n_words32;
    cover_chunk<NT, NB, false>(a, reinterpret_cast<const uint32_t*>(a.Q) + w_begin, seg, w_begin, w_end,
                               (uint32_t)(32 * (w_begin - seg_w0)), smem, shist, smax);
}

// Sieve and cover fused per CTA: the CTA sieves the q bits its chunk of
// coverage words reads into shared memory with the tile sieve and runs the
// block cover on them there; Q never goes through global memory.  The cover
// reads window words from w_begin + off_w (the partner offset of the largest
// prime of the pass, (H - P1 - 1) / 2 bits) to w_end + (H - 4) / 64 + 2, so
// the tile starts at word w_begin + off_w.
template <int NT, int NB>
__global__ void __launch_bounds__(NT, 2) k_seg_cover(const CoverArgs a, const SieveArgs sv, uint32_t off_w)
{
    extern __shared__ uint32_t smem[];                      // [lists | stamp tables | tile]
    __shared__ uint32_t shist[kBlock * NB + 1];
    __shared__ unsigned long long smax;
    constexpr int NW = NT / 32;
    const uint32_t cap = (2 * a.cta_words + 96 * NW - 1) / (96 * NW) * 96;
    uint32_t* lists = smem;
    uint32_t* wt = smem + (NW * cap * 6) / 4;
    uint32_t* tile = wt + ((kWheelWords + 3 + 3) & ~3u);    // 16-byte aligned
    const uint64_t wps = 2ull * a.words_per_seg;
    const uint32_t seg = blockIdx.x / a.chunks_per_seg;
    const uint32_t chunk = blockIdx.x % a.chunks_per_seg;
    const uint64_t seg_w0 = (uint64_t)seg * wps;
    const uint64_t w_begin = seg_w0 + (uint64_t)chunk * (2ull * a.cta_words);
    uint64_t w_end = w_begin + 2ull * a.cta_words;
    const uint64_t n_words32 = (a.n_count + 31) / 32;
    if (w_end > seg_w0 + wps) w_end = seg_w0 + wps;
    if (w_end > n_words32) w_end = n_words32;
    for (uint32_t i = threadIdx.x; i < kWheelWords; i += NT) wt[i] = sv.wheel[i];
    // tile word k is window word w_begin + off_w + k; the cover's Qc[k] is
    // window word w_begin + k and is only read at k >= off_w
    sieve_tile<NT>(sv, 32ull * (w_begin + off_w), wt, tile);
    cover_chunk<NT, NB, true>(a, tile - off_w, seg, w_begin, w_end, (uint32_t)(32 * (w_begin - seg_w0)), lists, shist,
                              smax);
}

template <int NB>
static cudaError_t launch_seg_nb(const CoverArgs& a, const SieveArgs& sv, uint32_t off_w, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    const uint32_t cap = (2 * a.cta_words + 96 * (NT / 32) - 1) / (96 * (NT / 32)) * 96;
    const size_t smem = (size_t)(NT / 32) * cap * 6 + ((kWheelWords + 3 + 3) & ~3u) * 4 + kFusedTileBits / 8;
    auto k = k_seg_cover<NT, NB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(a, sv, off_w);
    return cudaGetLastError();
}

uint32_t seg_cover_offset(uint32_t H, uint32_t P1)
{
    const uint32_t bits = P1 + 1 < H ? (H - P1 - 1) / 2 : 0;
    return bits >= 64 ? bits / 32 - 1 : 0;
}

cudaError_t launch_seg_cover(const CoverArgs& a, const SieveArgs& sv, int KA, uint32_t P1, cudaStream_t s)
{
    // the tile must hold the chunk's words and the partner halo read past
    // them, from the offset of the pass's largest prime on
    const uint32_t off_w = seg_cover_offset(a.H, P1);
    const uint64_t need_words = 2ull * a.cta_words + ((a.H - 4) >> 6) + 3 - off_w;
    if (need_words * 32 > kFusedTileBits || sv.tile_bits != kFusedTileBits || sv.out || sv.popcount)
        return cudaErrorInvalidValue;
    if (2ull * a.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    switch (KA) {
    case 64: return launch_seg_nb<1>(a, sv, off_w, s);
    case 128: return launch_seg_nb<2>(a, sv, off_w, s);
    case 192: return launch_seg_nb<3>(a, sv, off_w, s);
    case 256: return launch_seg_nb<4>(a, sv, off_w, s);
    default: return cudaErrorInvalidValue;
    }
}

// persistent: CTAs take (range, chunk) items from the queue until it is empty;
// row r of the histograms, keys and counts is range r
template <int NT, int NB>
__global__ void __launch_bounds__(NT, 4) k_cover_items(const CoverItemsArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t shist[kBlock * NB + 1];
    __shared__ unsigned long long smax;
    __shared__ uint32_t s_item;
    const uint32_t n_items = *a.n_items;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const uint32_t ri = a.item_range[item];
        const BatchRange r = a.ranges[ri];
        CoverArgs c = a.base;
        c.Q = a.Q + r.q_off;
        c.n_count = r.n;
        c.n_words = (r.n + 63) / 64;
        c.has_n4 = (r.lo == 4);
        const uint64_t w_begin = (uint64_t)a.item_chunk[item] * (2ull * c.cta_words);
        uint64_t w_end = w_begin + 2ull * c.cta_words;
        const uint64_t nw32 = (r.n + 31) / 32;
        if (w_end > nw32) w_end = nw32;
        cover_chunk<NT, NB, false>(c, reinterpret_cast<const uint32_t*>(c.Q) + w_begin, ri, w_begin, w_end,
                                   (uint32_t)(32 * w_begin), smem, shist, smax);
    }
}

template <int NB>
static cudaError_t launch_items_nb(const CoverItemsArgs& a, cudaStream_t s)
{
    constexpr int NT = 256;
    const uint32_t cap = (2 * a.base.cta_words + 96 * (NT / 32) - 1) / (96 * (NT / 32)) * 96;
    const size_t smem = (size_t)(NT / 32) * cap * 6;
    auto k = k_cover_items<NT, NB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess) return e;
    k<<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cover_items(const CoverItemsArgs& a, int KA, cudaStream_t s)
{
    if (2ull * a.base.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    switch (KA) {
    case 64: return launch_items_nb<1>(a, s);
    case 128: return launch_items_nb<2>(a, s);
    case 192: return launch_items_nb<3>(a, s);
    case 256: return launch_items_nb<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

int cover_fast_phase_primes(uint32_t K, uint64_t n_hi)
{
    // unrolled blocks of 64 primes, by magnitude: the share of n still open
    // after 64 primes is about 0.6% near 1e10, 1.5% near 1e12 and 6% near 4e18
    int nb = n_hi < 100000000000ull ? 2 : n_hi < 10000000000000000ull ? 3 : 4;
    while (nb > 0 && (uint32_t)(kBlock * nb) > K) --nb;
    return kBlock * nb;
}

template <int NB>
static cudaError_t launch_nb(const CoverArgs& a, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    // one list per warp holding every word it takes in block 0: 32-bit
    // coverage, 16-bit index
    const uint32_t cap = (2 * a.cta_words + 96 * (NT / 32) - 1) / (96 * (NT / 32)) * 96;
    const size_t smem = (size_t)(NT / 32) * cap * 6;
    auto k = k_cover_fast<NT, NB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cover_fast(const CoverArgs& a, int KA, cudaStream_t s)
{
    // 10-bit counters: in block 0 a lane adds at most 96 per step per round
    // (three words), at most 10 rounds of 768 words; later blocks add at most
    // 32 per listed word, at most 30 per lane
    if (2ull * a.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    switch (KA) {
    case 64: return launch_nb<1>(a, s);
    case 128: return launch_nb<2>(a, s);
    case 192: return launch_nb<3>(a, s);
    case 256: return launch_nb<4>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gb
