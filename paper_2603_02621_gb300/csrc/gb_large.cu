// gb_large.cu -- the sieving primes from the slice limit (2^20) up to sqrt of
// the window's first number, for windows of several L2-sized chunks
// (GoldbachGPU, arXiv 2603.02621, Sec. 2.3.1: a segmented sieve of [A, B]
// with the primes to sqrt(B); the large primes carried from segment to
// segment by their next multiple, as in the cache-efficient segmented sieves
// the paper cites).
//
// The window is struck one chunk of 2^L bits at a time (L2-resident words,
// global atomic AND).  Each prime is started once per window, not once per
// chunk:
//
//   * primes below half a chunk ("dense": at least two hits per chunk) keep
//     their next multiple in a per-prime word (offset in the current chunk,
//     29 bits, and wheel position, 3 bits), read and rewritten by every
//     chunk;
//   * larger primes ("sparse": at most a few hits per chunk, most chunks
//     none) are filed in a ring of per-chunk buckets, keyed by the chunk of
//     their next multiple; a chunk takes its own bucket, strikes each prime's
//     multiples in the chunk, and files the prime again under the chunk of its
//     next multiple.  An entry holds the prime itself (no lookup by index),
//     its wheel position and its offset in the target chunk.
//
// Every bucket is split into one column per CTA of a fixed grid: CTA g takes
// the sparse primes of its share at the start, and from then on only ever
// reads and writes column g, so its bucket counts live in shared memory for
// the length of a launch and no two CTAs append to the same count.
//
// Wheel mod 30: a multiple m p with m divisible by 3 or 5 is also a multiple
// of 3 or 5 and is cleared by the stamp; only m coprime to 30 is struck (8 of
// every 15 odd m).  The coprime residues of m mod 30 are 1, 7, 11, 13, 17,
// 19, 23, 29; from one to the next the bit index (m p - B) / 2 advances by p
// times the half gaps 3, 2, 1, 2, 1, 2, 3, 1.
//
// A bucket column that is full when an entry arrives cannot lose it: the
// prime's remaining multiples in the window are struck at once (clearing bits
// of chunks not yet visited is harmless, the strikes only clear composite
// bits), and the event is counted.
#include "gb_internal.cuh"

namespace gb {

namespace {

constexpr int kThreads = 256;

// half gap from wheel position w to w + 1, four bits per position
constexpr uint32_t kHalfGaps = 0x13212123u;
__device__ __forceinline__ uint32_t half_gap(uint32_t w) { return (kHalfGaps >> (4 * w)) & 0xfu; }

// inverse of p mod 30 for p mod 30 coprime to 30 (0 elsewhere)
__constant__ uint8_t kInv30[30] = {0, 1, 0, 0, 0, 0, 0, 13, 0, 0, 0, 11, 0, 7, 0,
                                   0, 0, 23, 0, 19, 0, 0, 0, 17, 0, 0, 0, 0, 0, 29};
// for an odd residue r of m mod 30: the wheel position of the first coprime
// residue >= r (low nibble) and half the distance to it (high nibble)
__constant__ uint8_t kNext30[30] = {0, 0x00, 0, 0x21, 0, 0x11, 0, 0x01, 0, 0x12, 0, 0x02, 0, 0x03, 0,
                                    0x14, 0, 0x04, 0, 0x05, 0, 0x16, 0, 0x06, 0, 0x27, 0, 0x17, 0, 0x07};

__device__ __forceinline__ void strike_bit(const BucketLargeArgs& a, uint64_t bit)
{
    if (!GB_DCHECK(bit < a.nbits, kDbgCarryStrike)) return;
    atomicAnd(a.out + (bit >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, (uint32_t)bit));
}

// every remaining multiple of p from window bit g on (wheel position w)
__device__ __forceinline__ uint32_t strike_rest(const BucketLargeArgs& a, uint64_t g, uint32_t p, uint32_t w)
{
    uint32_t n = 0;
    for (; g < a.nbits; ++n) {
        strike_bit(a, g);
        g += (uint64_t)p * half_gap(w);
        w = (w + 1) & 7u;
    }
    return n;
}

// this CTA's column counts of every bucket, in shared memory (the drained
// bucket's count starts over)
__device__ __forceinline__ void load_counts(const BucketLargeArgs& a, uint32_t* s_cnt, uint32_t drained)
{
    for (uint32_t t = threadIdx.x; t <= a.ring_mask; t += blockDim.x)
        s_cnt[t] = t == drained ? 0u : a.ring_cnt[(uint64_t)t * a.grid + blockIdx.x];
    __syncthreads();
}

__device__ __forceinline__ void store_counts(const BucketLargeArgs& a, const uint32_t* s_cnt)
{
    __syncthreads();
    for (uint32_t t = threadIdx.x; t <= a.ring_mask; t += blockDim.x)
        a.ring_cnt[(uint64_t)t * a.grid + blockIdx.x] = s_cnt[t];
}

// File the entry (p, w, offset o in chunk t) in this CTA's column of chunk
// t's bucket; called by every lane of the warp (valid marks the lanes with an
// entry).  Lanes filing into the same bucket share one shared-memory atomic.
__device__ __forceinline__ uint32_t file_entry(const BucketLargeArgs& a, uint32_t* s_cnt, bool valid, uint32_t t,
                                               uint32_t p, uint32_t w, uint32_t o)
{
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return 0;
    const int lane = threadIdx.x & 31;
    const uint32_t slot = t & a.ring_mask;
    const unsigned peers = __match_any_sync(act, slot);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(s_cnt + slot, (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t pos = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (pos < a.cap) {
        const uint64_t at = ((uint64_t)slot * a.grid + blockIdx.x) * a.cap + pos;
        if (GB_DCHECK(at < (uint64_t)(a.ring_mask + 1) * a.grid * a.cap && o < (1u << a.chunk_log2), kDbgCarryRing))
            a.ring[at] = ((uint64_t)p << 32) | ((uint64_t)w << 28) | o;
        return 0;
    }
    atomicAdd(a.spills, 1u);
    return strike_rest(a, ((uint64_t)t << a.chunk_log2) + o, p, w);
}

__device__ __forceinline__ void add_strikes(const BucketLargeArgs& a, unsigned long long n)
{
    if (!a.strikes) return;
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(a.strikes, n);
}

}  // namespace

// First multiple of each prime in the window (every prime has p^2 <= B, so
// the first odd multiple >= B is at least p^2), moved up to a coprime m.
__global__ void __launch_bounds__(kThreads) k_large_start(const BucketLargeArgs a)
{
    __shared__ uint32_t s_cnt[kCarryMaxRing];
    __shared__ uint8_t s_inv[30], s_next[30];             // the tables, where lanes may read different entries
    if (threadIdx.x < 30) {
        s_inv[threadIdx.x] = kInv30[threadIdx.x];
        s_next[threadIdx.x] = kNext30[threadIdx.x];
    }
    load_counts(a, s_cnt, 0xffffffffu);                   // (ends with a barrier)
    const uint32_t n = a.n_dense + a.n_sparse;
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long nstrike = 0;
    for (uint32_t k0 = blockIdx.x * blockDim.x; k0 < n; k0 += stride) {
        const uint32_t k = k0 + threadIdx.x;
        bool sparse = false;
        uint32_t p = 0, w = 0, o = 0, t = 0;
        if (k < n) {
            p = a.primes[k];
            const uint64_t i0 = first_odd_multiple(a.B, p, a.recip[k]);        // < p
            // m0 = (B + 2 i0) / p is odd; its residue mod 30 from (B + 2 i0) mod 30
            const uint32_t r = (a.B_mod30 + 2u * (uint32_t)(i0 % 15u)) % 30u;
            const uint32_t mr = (r * (uint32_t)s_inv[p % 30u]) % 30u;
            const uint32_t nx = s_next[mr];
            w = nx & 0xfu;
            const uint64_t i = i0 + (uint64_t)p * (nx >> 4);                 // < 3p
            if (k < a.n_dense) {
                // offset below 3p < 1.5 chunks: 29 bits; beyond the window it never strikes
                a.dstate[k] = (uint32_t)i | (w << 29);
            } else {
                t = (uint32_t)(i >> a.chunk_log2);
                o = (uint32_t)(i & ((1ull << a.chunk_log2) - 1));
                sparse = i < a.nbits;
            }
        }
        nstrike += file_entry(a, s_cnt, sparse, t, p, w, o);
    }
    store_counts(a, s_cnt);
    add_strikes(a, nstrike);
}

// Chunk c of the window: the dense primes, then this CTA's column of the
// bucket of chunk c.
__global__ void __launch_bounds__(kThreads) k_large_chunk(const BucketLargeArgs a, uint32_t c)
{
    __shared__ uint32_t s_cnt[kCarryMaxRing];
    // the previous chunk's bucket is drained: its counts start over for chunk
    // c - 1 + R (no entry of this launch can reach that far)
    load_counts(a, s_cnt, c > 0 ? (c - 1) & a.ring_mask : 0xffffffffu);
    const uint32_t C = 1u << a.chunk_log2;
    const uint64_t base = (uint64_t)c << a.chunk_log2;
    const uint64_t rest = a.nbits - base;
    const uint32_t span = rest < C ? (uint32_t)rest : C;
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long nstrike = 0;

    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_dense; k += stride) {
        const uint32_t st = a.dstate[k];
        const uint32_t p = a.primes[k];                                     // p < C / 2
        uint32_t off = st & 0x1fffffffu, w = st >> 29;
        while (off < span) {                                                // off + 3p < 2^30
            strike_bit(a, base + off);
            off += p * half_gap(w);
            w = (w + 1) & 7u;
            ++nstrike;
        }
        a.dstate[k] = (off - C) | (w << 29);                                // < 3p after a full chunk
    }

    const uint32_t slot = c & a.ring_mask;
    const uint32_t cnt = s_cnt[slot];
    const uint32_t n = cnt < a.cap ? cnt : a.cap;
    const uint64_t* bucket = a.ring + ((uint64_t)slot * a.grid + blockIdx.x) * a.cap;
    for (uint32_t e0 = 0; e0 < n; e0 += blockDim.x) {
        const uint32_t e = e0 + threadIdx.x;
        bool again = false;
        uint32_t p = 0, w = 0, t = 0, o = 0;
        if (e < n) {
            const uint64_t ent = bucket[e];
            p = (uint32_t)(ent >> 32);
            w = (uint32_t)(ent >> 28) & 7u;
            uint64_t off = ent & ((1ull << 28) - 1);
            while (off < span) {
                strike_bit(a, base + off);
                off += (uint64_t)p * half_gap(w);
                w = (w + 1) & 7u;
                ++nstrike;
            }
            // next multiple: in a later chunk (off >= span = C), or past the window
            again = base + off < a.nbits;
            t = c + (uint32_t)(off >> a.chunk_log2);
            o = (uint32_t)(off & (C - 1));
        }
        nstrike += file_entry(a, s_cnt, again, t, p, w, o);
    }
    store_counts(a, s_cnt);
    add_strikes(a, nstrike);
}

uint32_t carry_grid() { return device_sms() * 8; }

cudaError_t launch_large_start(const BucketLargeArgs& a, cudaStream_t s)
{
    const uint32_t n = a.n_dense + a.n_sparse;
    if (n == 0) return cudaSuccess;
    if (!a.primes || !a.recip || !a.out || (a.n_dense && !a.dstate) || !a.ring_cnt || !a.spills ||
        (a.n_sparse && (!a.ring || !a.cap)) || a.chunk_log2 > 28 || a.B <= 0 || a.ring_mask + 1 > kCarryMaxRing ||
        a.grid == 0)
        return cudaErrorInvalidValue;
    k_large_start<<<a.grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_large_chunk(const BucketLargeArgs& a, uint32_t c, cudaStream_t s)
{
    if (c >= a.nchunks || a.grid == 0 || a.ring_mask + 1 > kCarryMaxRing) return cudaErrorInvalidValue;
    k_large_chunk<<<a.grid, kThreads, 0, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace gb
