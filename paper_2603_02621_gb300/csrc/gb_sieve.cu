// gb_sieve.cu -- segmented sieve of Eratosthenes on the GPU, odd-only bitset.
//
// GoldbachGPU (arXiv 2603.02621) sieves each segment on the CPU and copies the
// bitset to the device (Sec. 2.3.1); Sec. 4.4 names that CPU sieve as the cost
// that dominates and Sec. 4.5 lists a GPU segmented sieve as future work.  Here
// every sieve runs on the device:
//
//   * the bit layout is the dense odd-only bitset of Sec. 2.2 (one bit per odd
//     number, 64-bit words, little-endian bit order), with bit 0 at a chosen odd
//     base instead of 3;
//   * one CTA owns one tile of the window in shared memory: the primes 3..43
//     are stamped from four periodic patterns, primes 47 <= p strike their
//     odd multiples from max(p^2, tile start) with shared-memory atomicAnd
//     (one warp per small prime, one thread per larger prime), and the
//     finished tile is stored with coalesced writes;
//   * the first multiple of p in a tile comes from a Barrett remainder with a
//     per-prime reciprocal, so no 64-bit division runs in the hot loop.
#include <atomic>

#include "gb_internal.cuh"
#include "gb_sieve_tile.cuh"

namespace gb {

uint32_t device_sms()
{
    constexpr int kMaxDev = 64;
    static std::atomic<uint32_t> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < kMaxDev) {
        const uint32_t c = cache[dev].load(std::memory_order_relaxed);
        if (c) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < kMaxDev) cache[dev].store((uint32_t)sms, std::memory_order_relaxed);
    return (uint32_t)sms;
}

// ---------------------------------------------------------------------------
// stamp tables: in table t, bit x (x = 0 .. 32*words-1) is 1 iff no prime of
// the table divides 2x + 1, i.e. x mod p != (p-1)/2 for each of its primes
// ---------------------------------------------------------------------------
__global__ void k_wheel_tables(uint32_t* wheel)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t P[14] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 0};
    const uint32_t first[5] = {0, 5, 7, 10, 13};                 // primes of table i: P[first[i] .. first[i+1])
    const uint32_t base[5] = {0, kWheelW1, kWheelW1 + kWheelW2, kWheelW1 + kWheelW2 + kWheelW3, kWheelWords};
    if (t >= kWheelWords) return;
    int tab = 0;
    while (t >= base[tab + 1]) ++tab;
    const uint32_t wi = t - base[tab];
    uint32_t v = 0;
    for (uint32_t b = 0; b < 32; ++b) {
        const uint32_t x = 32 * wi + b;
        bool keep = true;
        for (uint32_t k = first[tab]; k < first[tab + 1]; ++k) keep &= (x % P[k]) != (P[k] - 1) / 2;
        v |= (uint32_t)keep << b;
    }
    wheel[t] = v;
}

cudaError_t launch_wheel_tables(uint32_t* wheel, cudaStream_t s)
{
    k_wheel_tables<<<(kWheelWords + 255) / 256, 256, 0, s>>>(wheel);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// seed sieve: the odd numbers 1 .. 65535 (1024 words), plain Eratosthenes in
// one CTA; provides the primes < 2^16 that sieve every base up to 2^32.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_seed_sieve(uint32_t* out)
{
    __shared__ uint32_t sm[1024];
    sm[threadIdx.x] = 0xffffffffu;
    __syncthreads();
    if (threadIdx.x == 0) sm[0] &= ~1u;          // 1 is not prime
    __syncthreads();
    for (uint32_t p = 3; p * p < 65536u; p += 2) {
        uint32_t bp = (p - 1) / 2;
        bool prime = (sm[bp >> 5] >> (bp & 31)) & 1u;
        __syncthreads();                          // everyone read before strikes
        if (prime) {
            // odd multiples p*p, p*p + 2p, ... -> indices (p*p-1)/2 + k*p
            for (uint32_t i = (p * p - 1) / 2 + threadIdx.x * p; i < 32768u; i += 1024u * p)
                atomicAnd(&sm[i >> 5], ~(1u << (i & 31)));
        }
        __syncthreads();
    }
    out[threadIdx.x] = sm[threadIdx.x];
}

cudaError_t launch_seed_sieve(uint32_t* words, cudaStream_t s)
{
    k_seed_sieve<<<1, 1024, 0, s>>>(words);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tile sieve
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) k_sieve(const SieveArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t* wt = smem;                              // stamp tables (kWheelWords + 3 pad)
    uint32_t* sm = smem + kWheelWords + 3;            // tile words (16B aligned)
    for (uint32_t i = threadIdx.x; i < kWheelWords; i += NT) wt[i] = a.wheel[i];
    sieve_tile<NT>(a, (uint64_t)blockIdx.x * a.tile_bits, wt, sm);
}

// persistent: CTAs take (range, tile) items from the queue until it is empty
template <int NT>
__global__ void __launch_bounds__(NT) k_sieve_items(const SieveItemsArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t* wt = smem;                              // stamp tables (kWheelWords + 3 pad)
    uint32_t* sm = smem + kWheelWords + 3;            // tile words (16B aligned)
    __shared__ uint32_t s_item;
    for (uint32_t i = threadIdx.x; i < kWheelWords; i += NT) wt[i] = a.base.wheel[i];
    const uint32_t n_items = *a.n_items;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();                              // everyone has read s_item
        if (item >= n_items) break;
        const BatchRange r = a.ranges[a.item_range[item]];
        SieveArgs t = a.base;
        t.B = r.B;
        t.nbits = r.nbits;
        t.out = a.Q + 2 * r.q_off;
        t.popcount = nullptr;
        sieve_tile<NT>(t, (uint64_t)a.item_tile[item] * t.tile_bits, wt, sm);
    }
}

template <int NT>
static cudaError_t launch_sieve_items_nt(const SieveItemsArgs& a, cudaStream_t s)
{
    const size_t smem = (kWheelWords + 3) * 4 + (size_t)a.base.tile_bits / 8;
    auto k = k_sieve_items<NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem)) != cudaSuccess) return e;
    k<<<(unsigned)(device_sms() * (per_sm > 0 ? per_sm : 1)), NT, smem, s>>>(a);
    return cudaGetLastError();
}

// persistent grid: as many CTAs of `threads` (128, 256 or 512) as fit on the device
cudaError_t launch_sieve_items(const SieveItemsArgs& a, int threads, cudaStream_t s)
{
    switch (threads) {
    case 128: return launch_sieve_items_nt<128>(a, s);
    case 512: return launch_sieve_items_nt<512>(a, s);
    default: return launch_sieve_items_nt<256>(a, s);
    }
}

cudaError_t launch_sieve(const SieveArgs& a, int threads, cudaStream_t s)
{
    if (a.nbits == 0) return cudaSuccess;
    const uint64_t tiles = (a.nbits + a.tile_bits - 1) / a.tile_bits;
    const size_t smem = (kWheelWords + 3) * 4 + (size_t)a.tile_bits / 8;
    switch (threads) {
    case 128: {
        auto k = k_sieve<128>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)tiles, 128, smem, s>>>(a);
        break;
    }
    case 512: {
        auto k = k_sieve<512>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)tiles, 512, smem, s>>>(a);
        break;
    }
    case 1024: {
        auto k = k_sieve<1024>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)tiles, 1024, smem, s>>>(a);
        break;
    }
    default: {
        auto k = k_sieve<256>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)tiles, 256, smem, s>>>(a);
        break;
    }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// primes larger than a tile: each hits a tile at most once, so the tile kernel
// would spend a Barrett start per (tile, prime) for at most one strike.  Here
// one thread takes one prime for a whole chunk of the window (one Barrett
// start per chunk) and clears its multiples in global memory with atomic AND;
// a chunk of 2^28 bits (32 MB) keeps the struck words resident in L2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_large(const LargeArgs a)
{
    const int64_t b = a.B + 2 * (int64_t)a.bit_lo;          // number of the chunk's first bit
    const int64_t last = a.B + 2 * (int64_t)(a.bit_hi - 1);
    const uint64_t span = a.bit_hi - a.bit_lo;
    unsigned long long nstrike = 0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_primes; k += gridDim.x * blockDim.x) {
        const uint32_t p = a.primes[k];
        const uint64_t pp = (uint64_t)p * p;
        if ((int64_t)pp > last) continue;
        uint64_t i = first_odd_multiple(b, p, a.recip[k]);
        if ((int64_t)pp > b) {
            const uint64_t isq = ((uint64_t)((int64_t)pp - b)) >> 1;
            if (isq > i) i = isq;
        }
        for (; i < span; i += p) {
            const uint64_t bit = a.bit_lo + i;
            if (GB_DCHECK(bit < a.bit_hi, kDbgLargeStrike))
                atomicAnd(a.out + (bit >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, (uint32_t)bit));
            ++nstrike;
        }
    }
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if ((threadIdx.x & 31) == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
}

cudaError_t launch_large(const LargeArgs& a, cudaStream_t s)
{
    if (a.n_primes == 0 || a.bit_hi <= a.bit_lo) return cudaSuccess;
    const uint32_t cap = device_sms() * 64u;
    const uint32_t grid = (a.n_primes + 255) / 256 < cap ? (a.n_primes + 255) / 256 : cap;
    k_large<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Primes between the tile split and a few slices (kMidSliceBits): each CTA loads one
// slice of the window (already sieved by the smaller primes) into shared
// memory, strikes every such prime in it (one start per prime and slice), and
// stores it back -- shared-memory atomics instead of one L2 request per strike.
//
// The start is the index of the prime's first odd multiple in the slice.  By
// default it is a Barrett reduction of the slice's 64-bit first number.  With
// a residue table (RES) the slice s, whose first number is b_s = B + 2 s S,
// takes (-b_s) mod p = ((-B) mod p - s (2 S mod p)) mod p: a product below
// 2^33 (s < 2^13, p < 2^20) reduced by one 32-bit multiply-high with
// floor(2^33 / p), whose quotient is at most two short (two conditional
// subtractions), in place of the 64 x 64-bit product of the Barrett step.
// slice primes below this take the mod-30 wheel (their strikes per slice,
// 1.75 * 2^20 / p, outnumber the wheel's start cost)
#ifndef GB_MID_WHEEL_BELOW
#define GB_MID_WHEEL_BELOW (1u << 16)
#endif
constexpr uint32_t kMidWheelBelow = GB_MID_WHEEL_BELOW;

// nw words from src to dst by the whole CTA: 16-byte vectors, several in
// flight per thread, when both are 16-byte aligned (the slice is one CTA per
// SM: its load and store are not hidden behind another CTA's strikes)
__device__ __forceinline__ void copy_slice(uint32_t* dst, const uint32_t* src, uint32_t nw)
{
    uint32_t w0 = 0;
    if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
        const uint32_t nv = nw / 4;
        uint4* dv = reinterpret_cast<uint4*>(dst);
        const uint4* sv = reinterpret_cast<const uint4*>(src);
#pragma unroll 7
        for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) dv[v] = sv[v];
        w0 = 4 * nv;
    }
    for (uint32_t w = w0 + threadIdx.x; w < nw; w += blockDim.x) dst[w] = src[w];
}

template <bool RES>
__device__ __forceinline__ void mid_slice(int64_t B, uint64_t nbits, uint32_t* words, uint64_t t0,
                                          const uint32_t* primes, const uint64_t* recip, const uint4* res,
                                          uint32_t n_primes, uint32_t* slice, unsigned long long& nstrike)
{
    const uint64_t rem = nbits - t0;
    const uint32_t nb = rem < kMidSliceBits ? (uint32_t)rem : kMidSliceBits;
    const uint32_t nw = (nb + 31) / 32;
    uint32_t* q = words + t0 / 32;
    __syncthreads();                                          // slice free
    copy_slice(slice, q, nw);
    __syncthreads();
    const int64_t b = B + 2 * (int64_t)t0;
    const int64_t last = B + 2 * (int64_t)(t0 + nb - 1);
    const uint32_t sidx = (uint32_t)(t0 / kMidSliceBits);    // the slice's index (RES: < 2^13)
    const uint32_t bmod30 = pmod_u32(b, 30);
    // four primes per thread at a time (k, k + T, k + 2T, k + 3T): their loads
    // and starts are independent, so their latencies overlap
    constexpr int U = 4;
    const uint32_t T = blockDim.x;
    for (uint32_t k0 = threadIdx.x; k0 < n_primes; k0 += U * T) {
        uint32_t p[U], i[U];
        uint64_t m[U];
        uint4 rs[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t k = k0 + u * T;
            if constexpr (RES) {
                rs[u] = k < n_primes ? res[k] : make_uint4(0u, 0u, 0u, 0u);
                p[u] = rs[u].x;
            } else {
                p[u] = k < n_primes ? primes[k] : 0u;
                m[u] = k < n_primes ? recip[k] : 0ull;
            }
        }
        if ((int64_t)((uint64_t)p[0] * p[0]) > last) break;  // ascending primes
#pragma unroll
        for (int u = 0; u < U; ++u) {
            i[u] = nb;                                        // no strike
            const uint64_t pp = (uint64_t)p[u] * p[u];
            if (p[u] && (int64_t)pp <= last) {
                uint32_t s;
                if constexpr (RES) {
                    const uint64_t t = (uint64_t)sidx * rs[u].z;                    // < 2^33
                    const uint32_t qt = __umulhi((uint32_t)(t >> 1), rs[u].w);      // floor(t / p) - {0, 1, 2}
                    uint32_t r = (uint32_t)t - qt * p[u];                          // < 3p
                    if (r >= p[u]) r -= p[u];
                    if (r >= p[u]) r -= p[u];
                    const uint32_t x = rs[u].y >= r ? rs[u].y - r : rs[u].y + (p[u] - r);   // (-b) mod p
                    s = (x & 1u) ? (x + p[u]) >> 1 : x >> 1;                       // x + p < 2^21
                } else {
                    s = first_odd_multiple(b, p[u], m[u]);
                }
                if ((int64_t)pp > b) {
                    const uint64_t isq = ((uint64_t)((int64_t)pp - b)) >> 1;
                    if (isq > s) s = (uint32_t)isq;           // isq < nb here
                }
                i[u] = s;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t j = i[u];
            if (p[u] < kMidWheelBelow) {
                // the mod-30 wheel of the tile sieve (only m p with m coprime to
                // 15), for primes with enough strikes per slice to pay for its start
                if (j < nb) {
                    const uint32_t pm = p[u] % 30u;
                    const uint32_t inv = pm * pm % 30u * pm % 30u;                  // p^-1 mod 30
                    const uint32_t jr = (bmod30 + 2u * (j % 15u)) % 30u * inv % 30u >> 1;
                    const uint32_t pos = (uint32_t)(kNextPos30 >> (3 * jr)) & 7u;
                    j += p[u] * ((kNextHalf30 >> (2 * jr)) & 3u);                 // j + 3p < 2^22
                    uint32_t g = __funnelshift_r(kHalfGaps30, kHalfGaps30, 4 * pos);
                    for (; j < nb; g = __funnelshift_r(g, g, 4)) {
                        if (GB_DCHECK(j < kMidSliceBits, kDbgMidStrike))
                            atomicAnd(slice + (j >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, j));
                        j += p[u] * (g & 15u);
                        ++nstrike;
                    }
                }
            } else {
                for (; j < nb; j += p[u]) {                   // p < 2^31, j < 2^21: no wrap
                    if (GB_DCHECK(j < kMidSliceBits, kDbgMidStrike))
                        atomicAnd(slice + (j >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, j));
                    ++nstrike;
                }
            }
        }
    }
    __syncthreads();
    copy_slice(q, slice, nw);
}

// the residue table of one window for the slice starts (see mid_slice)
__global__ void __launch_bounds__(256) k_mid_residues(const LargeArgs a)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n_primes) return;
    const uint32_t p = a.primes[k];
    a.res[k] = make_uint4(p, neg_mod(a.B, p, a.recip[k]), (uint32_t)((2ull * kMidSliceBits) % p),
                          (uint32_t)((1ull << 33) / p));
}

template <bool RES>
__global__ void __launch_bounds__(1024) k_mid(const LargeArgs a, uint64_t nbits)
{
    extern __shared__ uint32_t slice[];
    unsigned long long nstrike = 0;
    mid_slice<RES>(a.B, nbits, a.out, (uint64_t)blockIdx.x * kMidSliceBits, a.primes, a.recip, a.res, a.n_primes,
                   slice, nstrike);
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if ((threadIdx.x & 31) == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
}

// batched: persistent CTAs take (range, slice) items from a device queue
__global__ void __launch_bounds__(1024) k_mid_items(const MidItemsArgs a)
{
    extern __shared__ uint32_t slice[];
    __shared__ uint32_t s_item;
    const uint32_t n_items = *a.n_items;
    unsigned long long nstrike = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const BatchRange r = a.ranges[a.item_range[item]];
        mid_slice<false>(r.B, r.nbits, a.Q + 2 * r.q_off, (uint64_t)a.item_slice[item] * kMidSliceBits, a.primes,
                         a.recip, nullptr, a.n_primes, slice, nstrike);
    }
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if ((threadIdx.x & 31) == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
}

cudaError_t launch_mid_items(const MidItemsArgs& a, cudaStream_t s)
{
    if (a.n_primes == 0) return cudaSuccess;
    if (!a.primes || !a.recip || !a.Q || !a.ranges || !a.item_range || !a.item_slice || !a.n_items || !a.head)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)kMidSliceBits / 8;
    cudaError_t e = cudaFuncSetAttribute(k_mid_items, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    k_mid_items<<<(unsigned)sms, 1024, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mid(const LargeArgs& a, uint64_t nbits, cudaStream_t s)
{
    if (a.n_primes == 0 || nbits == 0) return cudaSuccess;
    if (!a.primes || !a.recip || !a.out) return cudaErrorInvalidValue;
    const uint64_t slices = (nbits + kMidSliceBits - 1) / kMidSliceBits;
    if (slices > 0x7fffffffull) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kMidSliceBits / 8;
    if (a.res) {
        // residue starts: fewer than 2^13 slices and primes below 2^20
        if (slices > kMidResSlices) return cudaErrorInvalidValue;
        k_mid_residues<<<(a.n_primes + 255) / 256, 256, 0, s>>>(a);
        cudaError_t e = cudaFuncSetAttribute(k_mid<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_mid<true><<<(unsigned)slices, 1024, smem, s>>>(a, nbits);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(k_mid<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mid<false><<<(unsigned)slices, 1024, smem, s>>>(a, nbits);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_popcount(const uint32_t* w, uint64_t n, unsigned long long* count)
{
    unsigned long long c = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        c += __popc(w[i]);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_popcount(const uint32_t* words, uint64_t n, unsigned long long* count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256;
    const uint64_t cap = (uint64_t)device_sms() * 16;
    k_popcount<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(words, n, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// compaction: bitset -> ascending prime list (after a leading 2) + reciprocals
// ---------------------------------------------------------------------------
constexpr uint32_t kCompactChunk = 8192;   // words per CTA
constexpr int kCompactNT = 256;            // 32 words per thread

uint64_t compact_chunks(uint64_t nwords) { return (nwords + kCompactChunk - 1) / kCompactChunk; }

__global__ void __launch_bounds__(kCompactNT) k_compact_count(const uint32_t* words, uint64_t nwords,
                                                              uint32_t* counts)
{
    const uint64_t base = (uint64_t)blockIdx.x * kCompactChunk;
    uint32_t c = 0;
    for (uint32_t i = threadIdx.x; i < kCompactChunk; i += kCompactNT)
        if (base + i < nwords) c += __popc(words[base + i]);
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ uint32_t ws[kCompactNT / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kCompactNT / 32; ++i) t += ws[i];
        counts[blockIdx.x] = t;
    }
}

// single CTA: exclusive scan of counts in place (sequential per thread slice)
__global__ void __launch_bounds__(1024) k_compact_scan(uint32_t* counts, uint32_t n)
{
    __shared__ uint32_t part[1024];
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(n, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < 1024; ++i) { uint32_t v = part[i]; part[i] = run; run += v; }
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (uint32_t i = lo; i < hi; ++i) { uint32_t v = counts[i]; counts[i] = run; run += v; }
}

__global__ void __launch_bounds__(kCompactNT) k_compact_write(const CompactArgs a)
{
    constexpr uint32_t per = kCompactChunk / kCompactNT;   // 32 consecutive words
    const uint64_t base = (uint64_t)blockIdx.x * kCompactChunk + threadIdx.x * per;
    uint32_t c = 0;
    for (uint32_t i = 0; i < per; ++i)
        if (base + i < a.nwords) c += __popc(a.words[base + i]);
    // block exclusive scan of c
    __shared__ uint32_t sc[kCompactNT];
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < kCompactNT; o <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)o ? sc[threadIdx.x - o] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t pos = 1ull + a.counts[blockIdx.x] + sc[threadIdx.x] - c;   // slot 0 holds 2
    for (uint32_t i = 0; i < per; ++i) {
        if (base + i >= a.nwords) break;
        uint32_t v = a.words[base + i];
        while (v) {
            uint32_t bit = __ffs(v) - 1;
            v &= v - 1;
            uint64_t num = (uint64_t)(a.B + 2 * (int64_t)((base + i) * 32 + bit));
            uint32_t p = (uint32_t)num;
            a.primes[pos] = p;
            a.recip[pos] = 0xffffffffffffffffull / p;
            ++pos;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.primes[0] = 2;
        a.recip[0] = 0xffffffffffffffffull / 2;
    }
}

cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s)
{
    const uint64_t nchunks = compact_chunks(a.nwords);
    k_compact_count<<<(unsigned)nchunks, kCompactNT, 0, s>>>(a.words, a.nwords, a.counts);
    k_compact_scan<<<1, 1024, 0, s>>>(a.counts, (uint32_t)nchunks);
    k_compact_write<<<(unsigned)nchunks, kCompactNT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
