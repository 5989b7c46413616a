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
//   * one CTA owns one tile of the window in shared memory: the wheel primes
//     3..19 are stamped from two periodic patterns, primes 23 <= p strike
//     their odd multiples from max(p^2, tile start) with shared-memory
//     atomicAnd (one warp per small prime, one thread per larger prime), and the
//     finished tile is stored with coalesced writes;
//   * the first multiple of p in a tile comes from a Barrett remainder with a
//     per-prime reciprocal, so no 64-bit division runs in the hot loop.
#include "gb_internal.cuh"

namespace gb {

// ---------------------------------------------------------------------------
// wheel tables: bit x (x = 0 .. 32*words-1) is 1 iff no prime of the table
// divides 2x + 1, i.e. x mod p != (p-1)/2 for each p.
// ---------------------------------------------------------------------------
__global__ void k_wheel_tables(uint32_t* w1, uint32_t* w2)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t P1[5] = {3, 5, 7, 11, 13};
    const uint32_t P2[2] = {17, 19};
    if (t < kWheelW1) {
        uint32_t v = 0;
        for (uint32_t b = 0; b < 32; ++b) {
            uint32_t x = 32 * t + b;
            bool keep = true;
            for (int k = 0; k < 5; ++k) keep &= (x % P1[k]) != (P1[k] - 1) / 2;
            v |= (uint32_t)keep << b;
        }
        w1[t] = v;
    }
    if (t < kWheelW2) {
        uint32_t v = 0;
        for (uint32_t b = 0; b < 32; ++b) {
            uint32_t x = 32 * t + b;
            bool keep = true;
            for (int k = 0; k < 2; ++k) keep &= (x % P2[k]) != (P2[k] - 1) / 2;
            v |= (uint32_t)keep << b;
        }
        w2[t] = v;
    }
}

cudaError_t launch_wheel_tables(uint32_t* w1, uint32_t* w2, cudaStream_t s)
{
    k_wheel_tables<<<(kWheelW1 + 255) / 256, 256, 0, s>>>(w1, w2);
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
__device__ __forceinline__ uint32_t pmod_u32(int64_t x, uint32_t M)
{
    int64_t r = x % (int64_t)M;
    return (uint32_t)(r < 0 ? r + M : r);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_sieve(const SieveArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t* w1 = smem;                              // kWheelW1
    uint32_t* w2 = smem + kWheelW1;                   // kWheelW2 (+3 pad)
    uint32_t* sm = smem + kWheelW1 + kWheelW2 + 3;    // tile words (16B aligned)

    const uint64_t t0 = (uint64_t)blockIdx.x * a.tile_bits;
    const uint64_t rem = a.nbits - t0;
    const uint32_t nb = rem < a.tile_bits ? (uint32_t)rem : a.tile_bits;
    const uint32_t nw = ((nb + 63) / 64) * 2;         // whole 64-bit words
    const int64_t b = a.B + 2 * (int64_t)t0;          // number of the tile's bit 0

    for (uint32_t i = threadIdx.x; i < kWheelW1; i += NT) w1[i] = a.wheel1[i];
    for (uint32_t i = threadIdx.x; i < kWheelW2; i += NT) w2[i] = a.wheel2[i];
    __syncthreads();

    // 1. wheel stamp for 3..19, fix-ups for numbers <= 19 and below 2
    {
        const int64_t x0 = (b - 1) / 2;               // b = 2 x0 + 1 (exact: b odd)
        const uint32_t u1 = pmod_u32(x0, kWheelM1);
        const uint32_t u2 = pmod_u32(x0, kWheelM2);
        for (uint32_t w = threadIdx.x; w < nw; w += NT) {
            uint32_t a1 = (u1 + 32u * w) % kWheelM1;
            uint32_t a2 = (u2 + 32u * w) % kWheelM2;
            uint32_t v = __funnelshift_r(w1[a1 >> 5], w1[(a1 >> 5) + 1], a1 & 31)
                       & __funnelshift_r(w2[a2 >> 5], w2[(a2 >> 5) + 1], a2 & 31);
            const int64_t v0 = b + 64 * (int64_t)w;   // number of this word's bit 0
            if (v0 <= 19) {
                // the wheel primes themselves are prime; numbers < 2 are not
                for (uint32_t k = 0; k < 32; ++k) {
                    int64_t num = v0 + 2 * (int64_t)k;
                    if (num < 2) v &= ~(1u << k);
                    else if (num == 3 || num == 5 || num == 7 || num == 11 ||
                             num == 13 || num == 17 || num == 19) v |= 1u << k;
                }
            }
            sm[w] = v;
        }
    }
    __syncthreads();

    // 2. strikes of the primes 23 <= p with p^2 <= the tile's last number
    const int64_t last = b + 2 * (int64_t)(nb - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long nstrike = 0;
    for (uint32_t k = warp; k < a.n_warp; k += NT / 32) {
        const uint32_t p = a.primes[k];
        const uint64_t pp = (uint64_t)p * p;
        if ((int64_t)pp > last) break;               // ascending: the rest too
        uint32_t i0 = first_odd_multiple(b, p, a.recip[k]);
        if ((int64_t)pp > b) {
            uint32_t isq = (uint32_t)(((int64_t)pp - b) >> 1);
            if (isq > i0) i0 = isq;                  // same residue class mod p
        }
        const uint32_t step = 32u * p;
        for (uint32_t i = i0 + (uint32_t)lane * p; i < nb; i += step)
            atomicAnd(&sm[i >> 5], ~(1u << (i & 31)));
        if (a.strikes && lane == 0 && i0 < nb) nstrike += (nb - 1 - i0) / p + 1;
    }
    for (uint32_t k = a.n_warp + threadIdx.x; k < a.n_primes; k += NT) {
        const uint32_t p = a.primes[k];
        const uint64_t pp = (uint64_t)p * p;
        if ((int64_t)pp > last) break;
        uint32_t i = first_odd_multiple(b, p, a.recip[k]);
        if ((int64_t)pp > b) {
            uint32_t isq = (uint32_t)(((int64_t)pp - b) >> 1);
            if (isq > i) i = isq;
        }
        if (a.strikes && i < nb) nstrike += (nb - 1 - i) / p + 1;
        // i < 2^20 and p < 3.1e9 (p^2 < 2^63): i + p cannot wrap
        for (; i < nb; i += p) atomicAnd(&sm[i >> 5], ~(1u << (i & 31)));
    }
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if (lane == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
    __syncthreads();

    // 3. clear bits past the window end, store, count
    uint32_t cnt = 0;
    uint32_t* dst = a.out ? a.out + t0 / 32 : nullptr;
    for (uint32_t w = threadIdx.x; w < nw; w += NT) {
        uint32_t v = sm[w];
        const uint32_t bit0 = 32u * w;
        if (bit0 >= nb) v = 0;
        else if (nb - bit0 < 32) v &= (1u << (nb - bit0)) - 1u;
        cnt += __popc(v);
        if (dst) dst[w] = v;
    }
    if (a.popcount) {
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(a.popcount, (unsigned long long)cnt);
    }
}

cudaError_t launch_sieve(const SieveArgs& a, int threads, cudaStream_t s)
{
    if (a.nbits == 0) return cudaSuccess;
    const uint64_t tiles = (a.nbits + a.tile_bits - 1) / a.tile_bits;
    const size_t smem = (kWheelW1 + kWheelW2 + 3) * 4 + (size_t)a.tile_bits / 8;
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
