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
//     their next multiple in a per-prime word (offset in the current chunk)
//     and byte (wheel position), read and rewritten by every chunk;
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
// Wheel mod 210: a multiple m p with m divisible by 3, 5 or 7 is also a
// multiple of 3, 5 or 7 and is cleared by the stamp; only m coprime to 210 is
// struck (48 of every 105 odd m).  From one coprime residue of m mod 210 to
// the next the bit index (m p - B) / 2 advances by p times half the gap (1 to
// 5); the tables below (built at compile time) give those half gaps, the
// inverse of p mod 210 and, for an odd residue, the next coprime one.  Sparse
// entries hold p / 2 (p odd, below 2^31), so the carried primes stop at 2^31.
//
// A bucket column that is full when an entry arrives cannot lose it: the
// prime's remaining multiples in the window are struck at once (clearing bits
// of chunks not yet visited is harmless, the strikes only clear composite
// bits), and the event is counted.
#include "gb_internal.cuh"

namespace gb {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kWheelPos = 48;          // residues mod 210 coprime to 210

constexpr bool coprime210(int r) { return r % 2 != 0 && r % 3 != 0 && r % 5 != 0 && r % 7 != 0; }

struct Wheel210 {
    uint8_t hgap[kWheelPos];    // half gap from wheel position w to w + 1 (position 47 -> 0: 209 -> 211)
    uint8_t inv[210];           // p^-1 mod 210 for p coprime to 210 (0 elsewhere)
    uint16_t next[210];         // odd r: position of the first coprime residue >= r | half the distance << 6
};

constexpr Wheel210 make_wheel210()
{
    Wheel210 t{};
    int res[kWheelPos + 1] = {};
    int n = 0;
    for (int r = 1; r < 210; ++r)
        if (coprime210(r)) res[n++] = r;
    res[kWheelPos] = 211;                   // 1 + 210: the first residue of the next period
    for (int w = 0; w < (int)kWheelPos; ++w) t.hgap[w] = (uint8_t)((res[w + 1] - res[w]) / 2);
    for (int p = 1; p < 210; ++p)
        if (coprime210(p))
            for (int u = 1; u < 210; ++u)
                if (p * u % 210 == 1) t.inv[p] = (uint8_t)u;
    for (int r = 1; r < 210; r += 2) {
        int w = 0;
        while (res[w] < r) ++w;             // res[48] = 211 >= every r
        t.next[r] = (uint16_t)((w % (int)kWheelPos) | (((res[w] - r) / 2) << 6));
    }
    return t;
}
__constant__ Wheel210 kWheel210 = make_wheel210();

// the wheel tables in shared memory (lanes read different entries)
struct WheelShared {
    uint8_t hgap[kWheelPos];
    uint8_t inv[210];
    uint16_t next[210];
};
__device__ __forceinline__ void load_wheel(WheelShared& ws)
{
    for (uint32_t t = threadIdx.x; t < 210; t += blockDim.x) {
        ws.inv[t] = kWheel210.inv[t];
        ws.next[t] = kWheel210.next[t];
        if (t < kWheelPos) ws.hgap[t] = kWheel210.hgap[t];
    }
}

// a sparse entry: p / 2 (p odd, < 2^31) << 34 | wheel position << 28 | offset in the chunk (< 2^28)
__device__ __forceinline__ uint64_t make_entry(uint32_t p, uint32_t w, uint32_t o)
{
    return ((uint64_t)(p >> 1) << 34) | ((uint64_t)w << 28) | o;
}

__device__ __forceinline__ void strike_bit(const BucketLargeArgs& a, uint64_t bit)
{
    if (!GB_DCHECK(bit < a.nbits, kDbgCarryStrike)) return;
    atomicAnd(a.out + (bit >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, (uint32_t)bit));
}

// every remaining multiple of p from window bit g on (wheel position w)
__device__ __forceinline__ uint32_t strike_rest(const BucketLargeArgs& a, const uint8_t* hgap, uint64_t g, uint32_t p,
                                                uint32_t w)
{
    uint32_t n = 0;
    for (; g < a.nbits; ++n) {
        strike_bit(a, g);
        g += (uint64_t)p * hgap[w];
        w = w + 1 == kWheelPos ? 0u : w + 1;
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
__device__ __forceinline__ uint32_t file_entry(const BucketLargeArgs& a, uint32_t* s_cnt, const uint8_t* hgap,
                                               bool valid, uint32_t t, uint32_t p, uint32_t w, uint32_t o)
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
            a.ring[at] = make_entry(p, w, o);
        return 0;
    }
    atomicAdd(a.spills, 1u);
    return strike_rest(a, hgap, ((uint64_t)t << a.chunk_log2) + o, p, w);
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
    __shared__ WheelShared ws;
    load_wheel(ws);
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
            // m0 = (B + 2 i0) / p is odd; its residue mod 210 from (B + 2 i0) mod 210
            const uint32_t r = (a.B_mod210 + 2u * (uint32_t)(i0 % 105u)) % 210u;
            const uint32_t mr = (r * (uint32_t)ws.inv[p % 210u]) % 210u;
            const uint32_t nx = ws.next[mr];
            w = nx & 63u;
            const uint64_t i = i0 + (uint64_t)p * (nx >> 6);                 // < 5p
            if (k < a.n_dense) {
                // below 5p < 2.5 chunks; beyond the window it never strikes
                a.dstate[k] = (uint32_t)i;
                a.dpos[k] = (uint8_t)w;
            } else {
                t = (uint32_t)(i >> a.chunk_log2);
                o = (uint32_t)(i & ((1ull << a.chunk_log2) - 1));
                sparse = i < a.nbits;
            }
        }
        nstrike += file_entry(a, s_cnt, ws.hgap, sparse, t, p, w, o);
    }
    store_counts(a, s_cnt);
    add_strikes(a, nstrike);
}

// Chunk c of the window: the dense primes, then this CTA's column of the
// bucket of chunk c.
__global__ void __launch_bounds__(kThreads) k_large_chunk(const BucketLargeArgs a, uint32_t c)
{
    __shared__ uint32_t s_cnt[kCarryMaxRing];
    __shared__ uint8_t s_hg[kWheelPos];
    if (threadIdx.x < kWheelPos) s_hg[threadIdx.x] = kWheel210.hgap[threadIdx.x];
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
        uint32_t off = a.dstate[k], w = a.dpos[k];
        const uint32_t p = a.primes[k];                                     // p < C / 2
        while (off < span) {                                                // off + 5p < 2^31
            strike_bit(a, base + off);
            off += p * s_hg[w];
            w = w + 1 == kWheelPos ? 0u : w + 1;
            ++nstrike;
        }
        a.dstate[k] = off - C;                                              // < 5p after a full chunk
        a.dpos[k] = (uint8_t)w;
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
            p = ((uint32_t)(ent >> 34) << 1) | 1u;
            w = (uint32_t)(ent >> 28) & 63u;
            uint64_t off = ent & ((1ull << 28) - 1);
            while (off < span) {
                strike_bit(a, base + off);
                off += (uint64_t)p * s_hg[w];
                w = w + 1 == kWheelPos ? 0u : w + 1;
                ++nstrike;
            }
            // next multiple: in a later chunk (off >= span = C), or past the window
            again = base + off < a.nbits;
            t = c + (uint32_t)(off >> a.chunk_log2);
            o = (uint32_t)(off & (C - 1));
        }
        nstrike += file_entry(a, s_cnt, s_hg, again, t, p, w, o);
    }
    store_counts(a, s_cnt);
    add_strikes(a, nstrike);
}

uint32_t carry_grid() { return device_sms() * 8; }

cudaError_t launch_large_start(const BucketLargeArgs& a, cudaStream_t s)
{
    const uint32_t n = a.n_dense + a.n_sparse;
    if (n == 0) return cudaSuccess;
    if (!a.primes || !a.recip || !a.out || (a.n_dense && (!a.dstate || !a.dpos)) || !a.ring_cnt || !a.spills ||
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
