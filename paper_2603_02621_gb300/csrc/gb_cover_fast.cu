// gb_cover_fast.cu -- two-phase form of the loop-inverted Goldbach cover.
//
// Same computation as the generic cover (gb_cover.cu): for p = 3, 5, 7, ... <= P
// in ascending order, every even n whose partner n - p is prime and that no
// smaller p covered gets p_min(n) = p (GoldbachGPU, arXiv 2603.02621, Sec.
// 2.3.1-2.3.2, in the bitwise form of Sec. 4.3).  Only the schedule differs.
//
// Unrolled blocks.  Most n are covered by one of the first few dozen primes,
// so primes are applied in blocks unrolled at compile time.  A lane owns one
// 32-bit word of C (32 even n) at a time.  With the halo chosen so that
// d_3 = (H - 4)/2 is a multiple of 32, the partner bits of word w for the
// prime p start at bit 32(w + d_3/32) - (p-3)/2 of Q: the word offset and the
// shift of every step are compile-time constants, and the few Q words a lane
// needs sit in registers.  A step is then
//     s = funnel-shift of two window registers,  C |= s,  cum_k += popc(C)
// and the histogram follows from the cumulative counts:
// #{n : p_min(n) = p_k} = cum_k - cum_{k-1} (three counts per register, added
// by multiply-adds with the field weights).  Block 0 (L0 primes) runs on
// every word of the CTA, three consecutive words per lane sharing one window;
// the words it leaves open (about one in three after 48 primes near 1e10) go
// to per-warp lists in shared memory, and blocks of 32 primes run on the open
// words alone, each leaving a shorter list, so that every lane of every step
// still works on an open word.  The prefix KA = L0 + 32 x (later blocks).
//
// Probing.  The few n open after the last block (about 1 in 10^4 after 112
// primes near 1e10)
// are taken one at a time by a warp: lane t probes the bit of Q at j + d_k for
// k = k0 + t, and the lowest set bit of the ballot is p_min.  An n still open
// after K primes goes to the retry pass (or counts as unresolved).
//
// The largest p_min of a warp's words, with its smallest n, comes from the
// probing when any n reached it.  Otherwise it lies in the last block that set
// a bit (known from the histogram), and that block is run once more over its
// input words, recording per word the last step that set a bit and the bits it
// set.  A later block writes its output list above its input when there is
// room, so that the input is still there for this re-run; when there is not,
// the warp's words are re-run through every block up to that one.
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
// at most 32 per word and handles at most 30 listed words (or 10 rounds of
// three words) per CTA in a block (32 * 30 < 2^10)
constexpr int kCumBits = 10;
constexpr uint32_t kCumMask = (1u << kCumBits) - 1;

// schedule: block 0 of L0 primes, then at most kMaxLater blocks of kLater
constexpr int kLater = 32;
constexpr int kMaxLater = 6;
constexpr int kMaxPrefix = 64 + kLater * kMaxLater;

// a warp's list holds every word it takes in block 0 (ten rounds of 96 words
// at most: the 10-bit counters allow no more)
__host__ __device__ constexpr uint32_t list_cap(uint32_t cta_words, int NW)
{
    return (2 * cta_words + 96 * NW - 1) / (96 * NW) * 96;
}

__host__ __device__ constexpr uint32_t step_e(int k) { return (odd_prime(k) - 3) / 2; }
// window of a block of L primes from index K0: R[t] = Q32[base - C0 - t]
// with C0 = the first step's word offset - 1
__host__ __device__ constexpr int block_c0(int K0)
{
    return K0 == 0 ? 0 : (int)((step_e(K0) + 31) / 32) - 1;
}
__host__ __device__ constexpr int block_regs(int K0, int L)
{
    return (int)((step_e(K0 + L - 1) + 31) / 32) - block_c0(K0) + 1;
}

template <int K, int K0, int NR>
__device__ __forceinline__ uint32_t window_shift(const uint32_t (&R)[NR])
{
    constexpr uint32_t e = step_e(K);
    constexpr int c = (int)((e + 31) / 32);
    constexpr uint32_t sh = 32 * c - e;
    constexpr int r = c - block_c0(K0);
    static_assert(r >= 0 && r < NR, "window too small");
    if constexpr (sh == 0) return R[r];
    else return __funnelshift_r(R[r], R[r - 1], sh);
}

template <int K, int K0, int NR, int KH>
__device__ __forceinline__ void block_step(const uint32_t (&R)[NR], uint32_t& C, uint32_t (&cum)[KH],
                                           const uint32_t (&wt)[3])
{
    C |= window_shift<K, K0, NR>(R);
    constexpr int j = K - K0;
    cum[j / 3] = __popc(C) * wt[j % 3] + cum[j / 3];
}

template <int K0, int NR, int KH, int... J>
__device__ __forceinline__ void run_block(std::integer_sequence<int, J...>, const uint32_t (&R)[NR], uint32_t& C,
                                          uint32_t (&cum)[KH], const uint32_t (&wt)[3])
{
    (block_step<K0 + J, K0, NR, KH>(R, C, cum, wt), ...);
}

// add one block's histogram to shist; kmax becomes the largest bin (prime
// index + 1) the block added to, if any.  The lanes' cumulative counts are
// summed over the warp by a transposed butterfly: two counts per register as
// 16-bit fields (a lane's counts are at most 960, a warp's at most 30720), and
// at each of five shuffle stages a lane keeps half of its registers and sends
// the other half to its partner, so that lane l ends with the warp totals of
// the counts 2l and 2l + 1 (L / 2 = 32 registers, padded from 24 for L = 48)
// or, for L = 32, of the counts 2(l/2) and 2(l/2) + 1 (lanes l and l ^ 1
// alike).  The bins are the differences of consecutive totals.
template <int K0, int L, int KH>
__device__ __forceinline__ void flush_block(const uint32_t (&cum)[KH], uint32_t init_pop, uint32_t* shist, int lane,
                                            uint32_t& kmax)
{
    constexpr int NP = L / 2;                               // count pairs
    constexpr int NR = NP <= 16 ? 16 : 32;                  // registers, a power of two
    static_assert(L % 2 == 0 && NP <= NR, "block length");
    uint32_t P[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r < NP) {
            const uint32_t lo = (cum[(2 * r) / 3] >> (kCumBits * ((2 * r) % 3))) & kCumMask;
            const uint32_t hi = (cum[(2 * r + 1) / 3] >> (kCumBits * ((2 * r + 1) % 3))) & kCumMask;
            P[r] = lo | (hi << 16);
        } else {
            P[r] = 0;
        }
    }
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const unsigned o = 16u >> st;
        const int m = NR >> (st + 1);                       // registers kept after this stage
        if (m > 0) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int r = 0; r < (m > 0 ? m : 1); ++r) {
                const uint32_t send = up ? P[r] : P[r + m];
                const uint32_t keep = up ? P[r + m] : P[r];
                P[r] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        } else {
            P[0] += __shfl_xor_sync(0xffffffffu, P[0], o);
        }
    }
    const uint32_t pi = NR == 32 ? (uint32_t)lane : (uint32_t)lane >> 1;    // this lane's pair
    const uint32_t t_lo = P[0] & 0xffffu, t_hi = P[0] >> 16;
    const uint32_t before = __reduce_add_sync(0xffffffffu, init_pop);       // total before the block
    const uint32_t up_hi = __shfl_up_sync(0xffffffffu, t_hi, NR == 32 ? 1 : 2);
    const uint32_t prev = pi == 0 ? before : up_hi;
    uint32_t cand = 0;
    if (pi < (uint32_t)NP && (NR == 32 || (lane & 1) == 0)) {
        const uint32_t d_lo = t_lo - prev, d_hi = t_hi - t_lo;
        if (d_lo) atomicAdd(&shist[K0 + 2 * pi + 1], d_lo);
        if (d_hi) atomicAdd(&shist[K0 + 2 * pi + 2], d_hi);
        cand = d_hi ? K0 + 2 * pi + 2 : d_lo ? K0 + 2 * pi + 1 : 0;
    }
    const uint32_t top = __reduce_max_sync(0xffffffffu, cand);
    if (top) kmax = top;
}

// ---------------------------------------------------------------------------
// block 0 on three consecutive words per lane: one window serves the three
// words, so a step is three funnel shifts and three ORs, then the three
// words' popcounts added into the step's counter through a carry-save adder:
// popc(C0) + popc(C1) + popc(C2) = popc(x) + 2 popc(y) with x the sum bits and
// y the carry bits, two popcounts instead of three for two more logic ops
// (the popcounts bound the step: measured 8.15 against 9.19 ms for the cover
// of 2^34 even n near 5e11).
// Window: R[t] = Q32[w + 2 + d_3/32 - t] for the lane's first word w.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int block0_regs3(int L0) { return (int)((step_e(L0 - 1) + 31) / 32) + 3; }

// The counts reach the 10-bit fields by integer multiply-adds with the field
// weights 1, 2^10, 2^20 held as runtime values (not constants, which the
// compiler would turn into shifts): the multiply-adds run on the FMA pipe and
// leave the ALU pipe to the shifts and ORs, the popcounts run on the XU pipe.
template <int K, int NR3, int KH>
__device__ __forceinline__ void step3(const uint32_t (&R)[NR3], uint32_t& C0, uint32_t& C1, uint32_t& C2,
                                      uint32_t (&cum)[KH], const uint32_t (&wt)[3])
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
    const uint32_t w = wt[K % 3];
    const uint32_t x = C0 ^ C1 ^ C2;                        // sum bits
    const uint32_t y = (C0 & C1) | (C2 & (C0 | C1));        // carry bits (majority)
    const uint32_t py = __popc(y);
    cum[K / 3] = __popc(x) * w + cum[K / 3];
    cum[K / 3] = py * w + cum[K / 3];                       // twice: weight 2
    cum[K / 3] = py * w + cum[K / 3];
}

template <int NR3, int KH, int... J>
__device__ __forceinline__ void run_block0_3(std::integer_sequence<int, J...>, const uint32_t (&R)[NR3], uint32_t& C0,
                                             uint32_t& C1, uint32_t& C2, uint32_t (&cum)[KH], const uint32_t (&wt)[3])
{
    (step3<J, NR3, KH>(R, C0, C1, C2, cum, wt), ...);
}

// ---------------------------------------------------------------------------
// tracked steps: record the last step that set a bit and the bits it set
// ---------------------------------------------------------------------------
template <int K, int K0, int NR>
__device__ __forceinline__ void track_step(const uint32_t (&R)[NR], uint32_t& C, uint32_t& last, uint32_t& lastbits)
{
    const uint32_t s = window_shift<K, K0, NR>(R);
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

// a word of the q window: read-only global load, or a shared-memory load when
// the window is a tile the same CTA has just sieved (fused kernel)
template <bool SQ>
__device__ __forceinline__ uint32_t ldq(const uint32_t* p)
{
    if constexpr (SQ) return *p;
    else return __ldg(p);
}

// block (K0, L) on one word, tracked; C is updated.  The key of the word's
// largest p_min within the block with its smallest n, 0 if the block set no bit
template <int K0, int L, bool SQ>
__device__ __forceinline__ unsigned long long track_word(const uint32_t* Qc, uint32_t D0w, uint32_t wrel, uint32_t& C,
                                                         uint32_t j_cta)
{
    constexpr int NR = block_regs(K0, L);
    constexpr int C0 = block_c0(K0);
    uint32_t R[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) R[t] = ldq<SQ>(Qc + wrel + D0w - C0 - t);
    uint32_t last = 0, lastbits = 0;
    track_block_steps<K0, NR>(std::make_integer_sequence<int, L>{}, R, C, last, lastbits);
    if (!last) return 0;
    const uint32_t j = j_cta + 32 * wrel + (__ffs(lastbits) - 1);
    return ((unsigned long long)(last + 1) << 32) | (0xffffffffull - j);
}

// Later block K0 (kLater primes) over a warp's list [iw, ic) of n_in words, in
// batches of 32 words (one per lane); the words still open go to [ow, oc),
// which is either above the input or the input itself (then writes never pass
// reads: each batch is read before its outputs land).
template <int K0, bool SQ>
__device__ __forceinline__ uint32_t later_block_warp(const uint32_t* Qc, uint32_t D0w, const uint16_t* iw,
                                                     const uint32_t* ic, uint32_t n_in, uint16_t* ow, uint32_t* oc,
                                                     uint32_t* shist, uint32_t& nsteps, uint32_t& kmax,
                                                     const uint32_t (&wt)[3])
{
    constexpr int L = kLater;
    constexpr int NR = block_regs(K0, L);
    constexpr int KH = (L + 2) / 3;
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
            wrel = iw[e];
            C = ic[e];
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = ldq<SQ>(Qc + wrel + D0w - C0 - t);
        } else {
#pragma unroll
            for (int t = 0; t < NR; ++t) R[t] = 0;
        }
        __syncwarp();                                      // the batch is read before outputs land
        init_pop += __popc(C);
        nsteps += active ? L : 0;
        run_block<K0, NR, KH>(std::make_integer_sequence<int, L>{}, R, C, cum, wt);
        const bool open = C != 0xffffffffu;
        const unsigned m = __ballot_sync(0xffffffffu, open);
        if (open) {
            const uint32_t slot = n_out + __popc(m & ((1u << lane) - 1u));
            ow[slot] = (uint16_t)wrel;
            oc[slot] = C;
        }
        n_out += __popc(m);
    }
    __syncwarp();
    flush_block<K0, L, KH>(cum, init_pop, shist, lane, kmax);
    return n_out;
}

// later block b (1 .. kMaxLater) of a schedule with block 0 of L0 primes
template <int L0, bool SQ, int B = 1>
__device__ __forceinline__ uint32_t later_block_at(int b, const uint32_t* Qc, uint32_t D0w, const uint16_t* iw,
                                                   const uint32_t* ic, uint32_t n_in, uint16_t* ow, uint32_t* oc,
                                                   uint32_t* shist, uint32_t& nsteps, uint32_t& kmax,
                                                   const uint32_t (&wt)[3])
{
    if constexpr (B > kMaxLater) {
        return n_in;
    } else {
        if (b == B)
            return later_block_warp<L0 + kLater * (B - 1), SQ>(Qc, D0w, iw, ic, n_in, ow, oc, shist, nsteps, kmax,
                                                                  wt);
        return later_block_at<L0, SQ, B + 1>(b, Qc, D0w, iw, ic, n_in, ow, oc, shist, nsteps, kmax, wt);
    }
}

// later block b, tracked, on one word (C updated)
template <int L0, bool SQ, int B = 1>
__device__ __forceinline__ unsigned long long track_word_at(int b, const uint32_t* Qc, uint32_t D0w, uint32_t wrel,
                                                            uint32_t& C, uint32_t j_cta)
{
    if constexpr (B > kMaxLater) {
        return 0;
    } else {
        if (b == B) return track_word<L0 + kLater * (B - 1), kLater, SQ>(Qc, D0w, wrel, C, j_cta);
        return track_word_at<L0, SQ, B + 1>(b, Qc, D0w, wrel, C, j_cta);
    }
}

__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long key)
{
    const uint32_t khi = (uint32_t)(key >> 32);
    const uint32_t mhi = __reduce_max_sync(0xffffffffu, khi);
    const uint32_t klo = khi == mhi ? (uint32_t)key : 0u;
    const uint32_t mlo = __reduce_max_sync(0xffffffffu, klo);
    return ((unsigned long long)mhi << 32) | mlo;
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

// Block 0 of L0 primes over every word (three words per lane), up to
// kMaxLater blocks of 32 over the words still open (a.n_later of them), then
// per-n probing.  One chunk of coverage words [w_begin, w_end) (32-bit words
// of the window a.Q, 32 even n each), all in segment (row) seg, whose first n
// has segment-relative index j_cta.  Called by every thread of the CTA; smem
// holds the per-warp lists; shist / smax are the CTA's shared counters.
template <int NT, int L0, bool SQ>
__device__ __forceinline__ void cover_chunk(const CoverArgs& a, const uint32_t* Qc, uint32_t seg, uint64_t w_begin,
                                            uint64_t w_end, uint32_t j_cta, uint32_t* smem, uint32_t* shist,
                                            unsigned long long& smax)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t cap = list_cap(a.cta_words, NW);
    uint32_t* lc = smem + (uint32_t)warp * cap;
    uint16_t* lw = reinterpret_cast<uint16_t*>(smem + NW * cap) + (uint32_t)warp * cap;
    const int n_later = (int)a.n_later;
    const uint32_t prefix = (uint32_t)(L0 + kLater * n_later);
    const uint32_t wt[3] = {a.cum_wt[0], a.cum_wt[1], a.cum_wt[2]};   // 1, 2^10, 2^20

    __syncthreads();                                        // shared counters free (previous chunk)
    for (uint32_t k = threadIdx.x; k <= prefix; k += NT) shist[k] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();

    const uint32_t D0w = ((a.H - 4) >> 1) >> 5;            // word offset of the p = 3 partner
    const uint32_t nw_cta = (uint32_t)(w_end > w_begin ? w_end - w_begin : 0);
    const uint64_t n_left = a.n_count - 32 * w_begin;       // n from the CTA's first n to the window end
    const uint32_t n_rel_end = (uint32_t)(n_left < 32ull * nw_cta ? n_left : 32ull * nw_cta);
    // a word's coverage before the first prime: the lanes past the slab end,
    // and n = 4 (= 2 + 2)
    auto init_c = [&](uint32_t w) -> uint32_t {
        uint32_t C = 0;
        const uint32_t j0 = 32 * w;
        if (n_rel_end - j0 < 32) C = 0xffffffffu << (n_rel_end - j0);
        if (a.has_n4 && w_begin + w == 0) C |= 1u;
        return C;
    };

    uint32_t nsteps = 0, n_open = 0, kmax = 0;
    // block 0 over every word of this warp, three consecutive words per lane
    {
        constexpr int NR3 = block0_regs3(L0);
        constexpr int KH = (L0 + 2) / 3;
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
                    C = init_c(w);
                    if (a.has_n4 && w_begin + w == 0) atomicAdd(&shist[0], 1u);
                    nsteps += L0;
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
            run_block0_3<NR3, KH>(std::make_integer_sequence<int, L0>{}, R, C0, C1, C2, cum, wt);
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
        flush_block<0, L0, KH>(cum, init_pop, shist, lane, kmax);
    }
    __syncwarp();

    // later blocks; tb = the last block that set a bit, with its input list
    int tb = 0;
    uint32_t t_off = 0, t_n = 0;
    bool t_kept = false;
    uint32_t in_off = 0, n_cur = n_open;
    int b_run = 0;
    for (int b = 1; b <= n_later && n_cur > 0; ++b) {
        const bool stack = in_off + 2 * n_cur <= cap;
        const uint32_t out_off = stack ? in_off + n_cur : in_off;
        const uint32_t kprev = kmax;
        const uint32_t n_next = later_block_at<L0, SQ>(b, Qc, D0w, lw + in_off, lc + in_off, n_cur,
                                                          lw + out_off, lc + out_off, shist, nsteps, kmax, wt);
        if (kmax != kprev) {
            tb = b;
            t_off = in_off;
            t_n = n_cur;
            t_kept = stack;
        }
        in_off = out_off;
        n_cur = n_next;
        b_run = b;
    }
    unsigned long long best = 0;
    probe_warp<SQ>(a, Qc, lw + in_off, lc + in_off, n_cur, (uint32_t)(L0 + kLater * b_run), w_begin, j_cta, seg,
                   best, nsteps);

    // the warp's largest p_min with its smallest n
    unsigned long long wbest = warp_max_key(best);
    if (wbest == 0 && kmax > 0) {
        best = 0;
        if (tb > 0 && t_kept) {
            // block tb once more over its input list
            for (uint32_t e = lane; e < t_n; e += 32) {
                uint32_t C = lc[t_off + e];
                const unsigned long long key = track_word_at<L0, SQ>(tb, Qc, D0w, lw[t_off + e], C, j_cta);
                if (key > best) best = key;
            }
        } else {
            // the warp's words through blocks 0 .. tb
            for (uint32_t wbase = 96 * warp; wbase < nw_cta; wbase += 96 * NW) {
                for (uint32_t w = wbase + lane; w < wbase + 96 && w < nw_cta; w += 32) {
                    uint32_t C = init_c(w);
                    unsigned long long key = track_word<0, L0, SQ>(Qc, D0w, w, C, j_cta);
                    for (int b = 1; b <= tb; ++b) {
                        const unsigned long long k2 = track_word_at<L0, SQ>(b, Qc, D0w, w, C, j_cta);
                        if (k2 > key) key = k2;
                    }
                    if (key > best) best = key;
                }
            }
        }
        wbest = warp_max_key(best);
    }
    if (lane == 0 && wbest) atomicMax(&smax, wbest);
    __syncthreads();
    if (threadIdx.x == 0 && smax == 0 && a.has_n4 && w_begin == 0)
        smax = (1ull << 32) | 0xffffffffull;               // only n = 4 (p_min 2, prime index 0)

    if (a.iters) {
        // unrolled word steps plus probes
        unsigned long long t = nsteps;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t) atomicAdd(a.iters, t);
    }
    uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    for (uint32_t kk = threadIdx.x; kk <= prefix; kk += NT)
        if (shist[kk]) atomicAdd(&hrow[kk], shist[kk]);
    if (threadIdx.x == 0 && smax) atomicMax(&a.maxkey[seg], smax);
}

// KA = L0 + 32 x (later blocks): L0 = 48 when KA = 16 (mod 32), else 64
static bool split_prefix(int KA, int& L0, int& n_later)
{
    if (KA < 48 || KA > kMaxPrefix || KA % 16 != 0) return false;
    L0 = KA % 32 == 16 ? 48 : 64;
    n_later = (KA - L0) / kLater;
    return n_later <= kMaxLater;
}

template <int NT, int L0>
__global__ void __launch_bounds__(NT, 4) k_cover_fast(const CoverArgs a)
{
    extern __shared__ uint32_t smem[];                      // per warp: list C (32-bit), then words (16-bit)
    __shared__ uint32_t shist[kMaxPrefix + 1];              // bins of the unrolled blocks' primes
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
    cover_chunk<NT, L0, false>(a, reinterpret_cast<const uint32_t*>(a.Q) + w_begin, seg, w_begin, w_end,
                                  (uint32_t)(32 * (w_begin - seg_w0)), smem, shist, smax);
}

// Sieve and cover fused per CTA: the CTA sieves the q bits its chunk of
// coverage words reads into shared memory with the tile sieve and runs the
// block cover on them there; Q never goes through global memory.  The cover
// reads window words from w_begin + off_w (the partner offset of the largest
// prime of the pass, (H - P1 - 1) / 2 bits) to w_end + (H - 4) / 64 + 2, so
// the tile starts at word w_begin + off_w.
template <int NT, int L0>
__global__ void __launch_bounds__(NT, 2) k_seg_cover(const CoverArgs a, const SieveArgs sv, uint32_t off_w)
{
    extern __shared__ uint32_t smem[];                      // [lists | stamp tables | tile]
    __shared__ uint32_t shist[kMaxPrefix + 1];
    __shared__ unsigned long long smax;
    constexpr int NW = NT / 32;
    const uint32_t cap = list_cap(a.cta_words, NW);
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
    cover_chunk<NT, L0, true>(a, tile - off_w, seg, w_begin, w_end, (uint32_t)(32 * (w_begin - seg_w0)), lists, shist,
                              smax);
}

template <int L0>
static cudaError_t launch_seg_l0(const CoverArgs& a, const SieveArgs& sv, uint32_t off_w, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    const uint32_t cap = list_cap(a.cta_words, NT / 32);
    const size_t smem = (size_t)(NT / 32) * cap * 6 + ((kWheelWords + 3 + 3) & ~3u) * 4 + kFusedTileBits / 8;
    auto k = k_seg_cover<NT, L0>;
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

cudaError_t launch_seg_cover(const CoverArgs& a0, const SieveArgs& sv, int KA, uint32_t P1, cudaStream_t s)
{
    // the tile must hold the chunk's words and the partner halo read past
    // them, from the offset of the pass's largest prime on
    const uint32_t off_w = seg_cover_offset(a0.H, P1);
    const uint64_t need_words = 2ull * a0.cta_words + ((a0.H - 4) >> 6) + 3 - off_w;
    if (need_words * 32 > kFusedTileBits || sv.tile_bits != kFusedTileBits || sv.out || sv.popcount)
        return cudaErrorInvalidValue;
    if (2ull * a0.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    int L0 = 0, nl = 0;
    if (!split_prefix(KA, L0, nl) || (uint32_t)KA > a0.K) return cudaErrorInvalidValue;
    CoverArgs a = a0;
    a.n_later = (uint32_t)nl;
    a.cum_wt[0] = 1; a.cum_wt[1] = 1u << kCumBits; a.cum_wt[2] = 1u << (2 * kCumBits);
    return L0 == 48 ? launch_seg_l0<48>(a, sv, off_w, s) : launch_seg_l0<64>(a, sv, off_w, s);
}

// persistent: CTAs take (range, chunk) items from the queue until it is empty;
// row r of the histograms, keys and counts is range r
template <int NT, int L0>
__global__ void __launch_bounds__(NT, 4) k_cover_items(const CoverItemsArgs a)
{
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t shist[kMaxPrefix + 1];
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
        cover_chunk<NT, L0, false>(c, reinterpret_cast<const uint32_t*>(c.Q) + w_begin, ri, w_begin, w_end,
                                   (uint32_t)(32 * w_begin), smem, shist, smax);
    }
}

template <int L0>
static cudaError_t launch_items_l0(const CoverItemsArgs& a, cudaStream_t s)
{
    constexpr int NT = 256;
    const uint32_t cap = list_cap(a.base.cta_words, NT / 32);
    const size_t smem = (size_t)(NT / 32) * cap * 6;
    auto k = k_cover_items<NT, L0>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess) return e;
    k<<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cover_items(const CoverItemsArgs& a0, int KA, cudaStream_t s)
{
    if (2ull * a0.base.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    int L0 = 0, nl = 0;
    if (!split_prefix(KA, L0, nl) || (uint32_t)KA > a0.base.K) return cudaErrorInvalidValue;
    CoverItemsArgs a = a0;
    a.base.n_later = (uint32_t)nl;
    a.base.cum_wt[0] = 1; a.base.cum_wt[1] = 1u << kCumBits; a.base.cum_wt[2] = 1u << (2 * kCumBits);
    return L0 == 48 ? launch_items_l0<48>(a, s) : launch_items_l0<64>(a, s);
}

bool cover_prefix_valid(int KA)
{
    int L0 = 0, nl = 0;
    return split_prefix(KA, L0, nl);
}

int cover_fast_phase_primes(uint32_t K, uint64_t n_hi)
{
    // by magnitude (cover of 2^34 even n timed for KA = 112 .. 240 near 1e10,
    // 1e11, 5e11, 1e13, 1e15 and 4e18): 48 + 3 x 32 primes below 1e14, 48 +
    // 4 x 32 below 1e17, 48 + 6 x 32 above; the share of 32-n words still
    // open after 48 primes is about 0.31 near 1e10, after 80 about 0.05, after
    // 112 about 0.003
    int ka = n_hi < 100000000000000ull ? 144 : n_hi < 100000000000000000ull ? 176 : 240;
    while (ka >= 48 && (uint32_t)ka > K) ka -= 32;
    if (ka < 48 && K >= 48) ka = 48;                        // the shortest schedule, block 0 alone
    return ka >= 48 ? ka : 0;
}

template <int L0>
static cudaError_t launch_l0(const CoverArgs& a, cudaStream_t s)
{
    constexpr int NT = 256;
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    // one list per warp holding every word it takes in a sub-chunk: 32-bit
    // coverage, 16-bit CTA-relative index
    const uint32_t cap = list_cap(a.cta_words, NT / 32);
    const size_t smem = (size_t)(NT / 32) * cap * 6;
    auto k = k_cover_fast<NT, L0>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cover_fast(const CoverArgs& a0, int KA, cudaStream_t s)
{
    // 10-bit counters: in block 0 a lane adds at most 96 per step per round
    // (three words), at most 10 rounds of 768 words; later blocks add at most
    // 32 per listed word, at most 30 per lane
    if (2ull * a0.cta_words > 10ull * 768) return cudaErrorInvalidValue;
    int L0 = 0, nl = 0;
    if (!split_prefix(KA, L0, nl) || (uint32_t)KA > a0.K) return cudaErrorInvalidValue;
    CoverArgs a = a0;
    a.n_later = (uint32_t)nl;
    a.cum_wt[0] = 1; a.cum_wt[1] = 1u << kCumBits; a.cum_wt[2] = 1u << (2 * kCumBits);
    return L0 == 48 ? launch_l0<48>(a, s) : launch_l0<64>(a, s);
}

}  // namespace gb
