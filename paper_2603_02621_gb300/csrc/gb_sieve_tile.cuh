// gb_sieve_tile.cuh -- the segment sieve of one shared-memory tile, shared by
// the per-window kernel (gb_sieve.cu) and the batched kernels (gb_batch.cu).
#pragma once

#include "gb_internal.cuh"

namespace gb {

__device__ __forceinline__ uint32_t pmod_u32(int64_t x, uint32_t M)
{
    int64_t r = x % (int64_t)M;
    return (uint32_t)(r < 0 ? r + M : r);
}

// clear bit i of the tile: word i/32 at byte offset (i >> 3) & ~3, mask
// ~(1 << (i & 31)) as a rotate of 0xfffffffe (the funnel shift takes i mod 32)
// (tile_bits: the tile's size, for the bounds check of a debug build)
__device__ __forceinline__ void strike(uint32_t* sm, uint32_t i, uint32_t tile_bits)
{
    if (!GB_DCHECK(i < tile_bits, kDbgTileStrike)) return;
    atomicAnd(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(sm) + ((i >> 3) & ~3u)),
              __funnelshift_l(0xfffffffeu, 0xfffffffeu, i));
}

// clear the bits of mask in tile word w (tile_words: the tile's size in words)
__device__ __forceinline__ void strike_word(const uint32_t* sm, uint32_t* w, uint32_t mask, uint32_t tile_words)
{
    if (!GB_DCHECK((uint32_t)(w - sm) < tile_words, kDbgTileStrike)) return;
    atomicAnd(w, mask);
}

// warp-struck primes below this start each lane at a strike chosen so that the
// lanes' words fall in distinct shared-memory banks
#ifndef GB_ROTATE_BELOW
#define GB_ROTATE_BELOW 128
#endif
constexpr uint32_t kRotateBelow = GB_ROTATE_BELOW;

// Wheel mod 30 for the one-thread primes: the stamp has cleared the multiples
// of 3 and 5, so only m p with m coprime to 30 is struck (8 of every 15 odd m).
// Positions 0..7 are the coprime residues 1, 7, 11, 13, 17, 19, 23, 29; nibble
// w of kHalfGaps30 is half the gap from position w to the next (the bit index
// (m p - b) / 2 then grows by p times it).  For an odd residue m = 2j + 1 of
// the first multiple, kNextPos30 (3 bits at 3j) is the position of the first
// coprime residue >= m and kNextHalf30 (2 bits at 2j) half the distance to it.
constexpr uint32_t kHalfGaps30 = 0x13212123u;
constexpr uint64_t kNextPos30 = 0x1ffdac8d2248ull;
constexpr uint32_t kNextHalf30 = 0x6104118u;

// one stamp table read at pattern offset a (a < period): 32 bits from bit a
__device__ __forceinline__ uint32_t stamp_word(const uint32_t* tab, uint32_t a)
{
    return __funnelshift_r(tab[a >> 5], tab[(a >> 5) + 1], a & 31);
}

// One tile of a window: bits [t0, t0 + tile_bits) of the window a.B, a.nbits,
// sieved in shared memory (sm: tile_bits / 32 words; wt: the stamp tables
// already loaded) and stored to a.out (word t0 / 32 on).  Called by every
// thread of the CTA; begins with a barrier, so consecutive calls may reuse sm.
template <int NT>
__device__ __forceinline__ void sieve_tile(const SieveArgs& a, uint64_t t0, const uint32_t* wt, uint32_t* sm)
{
    constexpr int NW = NT / 32;
    const uint32_t* w1 = wt;
    const uint32_t* w2 = w1 + kWheelW1;
    const uint32_t* w3 = w2 + kWheelW2;
    const uint32_t* w4 = w3 + kWheelW3;

    const uint64_t rem = a.nbits - t0;
    const uint32_t nb = rem < a.tile_bits ? (uint32_t)rem : a.tile_bits;
    const uint32_t nw = ((nb + 63) / 64) * 2;         // whole 64-bit words
    const int64_t b = a.B + 2 * (int64_t)t0;          // number of the tile's bit 0

    __syncthreads();                                  // sm free, wt loaded

    // 1. stamp of 3..43, fix-ups for numbers <= 43 and below 2
    {
        const int64_t x0 = (b - 1) / 2;               // b = 2 x0 + 1 (exact: b odd)
        const uint32_t step = 32u * NT;               // pattern advance per loop trip
        uint32_t a1 = (pmod_u32(x0, kWheelM1) + 32u * threadIdx.x) % kWheelM1;
        uint32_t a2 = (pmod_u32(x0, kWheelM2) + 32u * threadIdx.x) % kWheelM2;
        uint32_t a3 = (pmod_u32(x0, kWheelM3) + 32u * threadIdx.x) % kWheelM3;
        uint32_t a4 = (pmod_u32(x0, kWheelM4) + 32u * threadIdx.x) % kWheelM4;
        const uint32_t s1 = step % kWheelM1, s2 = step % kWheelM2, s3 = step % kWheelM3, s4 = step % kWheelM4;
        for (uint32_t w = threadIdx.x; w < nw; w += NT) {
            uint32_t v = stamp_word(w1, a1) & stamp_word(w2, a2) & stamp_word(w3, a3) & stamp_word(w4, a4);
            const int64_t v0 = b + 64 * (int64_t)w;   // number of this word's bit 0
            if (v0 <= 43) {
                // the stamped primes themselves are prime; numbers < 2 are not
                for (uint32_t k = 0; k < 32; ++k) {
                    const int64_t num = v0 + 2 * (int64_t)k;
                    if (num < 2) {
                        v &= ~(1u << k);
                    } else if (num <= 43) {
                        const bool pr = num == 3 || num == 5 || num == 7 || num == 11 || num == 13 ||
                                        num == 17 || num == 19 || num == 23 || num == 29 || num == 31 ||
                                        num == 37 || num == 41 || num == 43;
                        if (pr) v |= 1u << k;
                    }
                }
            }
            sm[w] = v;
            a1 += s1; if (a1 >= kWheelM1) a1 -= kWheelM1;
            a2 += s2; if (a2 >= kWheelM2) a2 -= kWheelM2;
            a3 += s3; if (a3 >= kWheelM3) a3 -= kWheelM3;
            a4 += s4; if (a4 >= kWheelM4) a4 -= kWheelM4;
        }
    }
    __syncthreads();

    // 2. strikes of the primes 47 <= p with p^2 <= the tile's last number
    const int64_t last = b + 2 * (int64_t)(nb - 1);
    const uint32_t tw = a.tile_bits / 32;             // tile words (bounds of a debug build)
    (void)tw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long nstrike = 0;
    // 2a. small primes, one warp each: warp w takes the primes w, w + NW, ...;
    // 32 of them at a time, each lane computing one prime's first index
    for (uint32_t k0 = warp; k0 < a.n_warp; k0 += 32 * NW) {
        const uint32_t k = k0 + (uint32_t)lane * NW;
        uint32_t p = 0, i0 = nb;
        if (k < a.n_warp) {
            p = a.primes[k];
            const uint64_t pp = (uint64_t)p * p;
            if ((int64_t)pp <= last) {
                i0 = first_odd_multiple(b, p, a.recip[k]);
                if ((int64_t)pp > b) {
                    const uint32_t isq = (uint32_t)(((int64_t)pp - b) >> 1);
                    if (isq > i0) i0 = isq;              // same residue class mod p
                }
            }
        }
        if (a.strikes && i0 < nb) nstrike += (nb - 1 - i0) / p + 1;
        unsigned pending = __ballot_sync(0xffffffffu, i0 < nb);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1;
            const uint32_t q = __shfl_sync(0xffffffffu, p, src);
            const uint32_t j0 = __shfl_sync(0xffffffffu, i0, src);
            // lane l strikes j0 + l q + 32 q t: the step is q whole words, so
            // the bit in the word, hence the mask, is fixed per lane
            const uint32_t i = j0 + (uint32_t)lane * q;           // < 2^20 + 2^15: no wrap
            if (i < nb) {
                const uint32_t mask = __funnelshift_l(0xfffffffeu, 0xfffffffeu, i);
                const uint32_t w0 = i >> 5;                       // the lane's first word
                const uint32_t end = (nb - (i & 31u) + 31u) >> 5; // words whose bit i&31 is < nb
                // For small q a lane's words are many (t up to 2^18 / 32 q) and
                // the 32 lanes' first words share banks (they lie q/32 words
                // apart).  Lane l then starts at its strike t = rot with
                // w0 + rot q = l (mod 32), rot = (l - w0) q^-1 mod 32, runs to the
                // tile end, and strikes t = rot - 1 down to 0 after: at every step
                // the lanes' words are then in 32 distinct banks (each lane's
                // bank moves by the same q or -q per step).
                uint32_t rot = 0;
                if (q < kRotateBelow) {
                    const uint32_t qinv = q * (2u - q * q);       // q^-1 mod 64 (q odd)
                    rot = (((uint32_t)lane - w0) * qinv) & 31u;
                    if (w0 + rot * q >= end) rot = 0;             // a short (last) tile: no rotation
                }
                uint32_t x = w0 + rot * q;
                for (; x + 3 * q < end; x += 4 * q) {
                    strike_word(sm, sm + x, mask, tw);
                    strike_word(sm, sm + x + q, mask, tw);
                    strike_word(sm, sm + x + 2 * q, mask, tw);
                    strike_word(sm, sm + x + 3 * q, mask, tw);
                }
                for (; x < end; x += q) strike_word(sm, sm + x, mask, tw);
                uint32_t n = rot;                                 // then t = rot - 1, ..., 0
                for (; n >= 4; n -= 4) {
                    strike_word(sm, sm + w0 + (n - 1) * q, mask, tw);
                    strike_word(sm, sm + w0 + (n - 2) * q, mask, tw);
                    strike_word(sm, sm + w0 + (n - 3) * q, mask, tw);
                    strike_word(sm, sm + w0 + (n - 4) * q, mask, tw);
                }
                for (; n > 0; --n) strike_word(sm, sm + w0 + (n - 1) * q, mask, tw);
            }
        }
    }
    // 2b. larger primes, one thread each; four at a time per thread (k, k +
    // NT, k + 2 NT, k + 3 NT), so that their loads and Barrett starts overlap.
    // Below 2^20 they step through the mod-30 wheel: fewer strikes, hence
    // fewer of the shared-memory wavefronts the kernel is bound by.
    constexpr int U = 4;
    const uint32_t bmod30 = pmod_u32(b, 30);
    for (uint32_t k0 = a.n_warp + threadIdx.x; k0 < a.n_primes; k0 += U * NT) {
        uint32_t p[U], s[U];
        uint64_t m[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t k = k0 + u * NT;
            p[u] = k < a.n_primes ? a.primes[k] : 0u;
            m[u] = k < a.n_primes ? a.recip[k] : 0ull;
        }
        if ((int64_t)((uint64_t)p[0] * p[0]) > last) break;    // ascending primes
#pragma unroll
        for (int u = 0; u < U; ++u) {
            s[u] = nb;                                          // no strike
            const uint64_t pp = (uint64_t)p[u] * p[u];
            if (p[u] && (int64_t)pp <= last) {
                uint32_t i = first_odd_multiple(b, p[u], m[u]);
                if ((int64_t)pp > b) {
                    const uint32_t isq = (uint32_t)(((int64_t)pp - b) >> 1);
                    if (isq > i) i = isq;
                }
                s[u] = i;
                if (a.strikes && i < nb && p[u] >= (1u << 20)) nstrike += (nb - 1 - i) / p[u] + 1;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t i = s[u];
            if (p[u] < (1u << 20)) {
                if (i < nb) {
                    // m = (b + 2i) / p: m p = b + 2i (mod 30), m = (b + 2i) p^-1 with
                    // p^-1 = p^3 (mod 30) (the units mod 30 have exponent 4)
                    const uint32_t pm = p[u] % 30u;
                    const uint32_t inv = pm * pm % 30u * pm % 30u;
                    const uint32_t j = (bmod30 + 2u * (i % 15u)) % 30u * inv % 30u >> 1;
                    const uint32_t pos = (uint32_t)(kNextPos30 >> (3 * j)) & 7u;
                    i += p[u] * ((kNextHalf30 >> (2 * j)) & 3u);     // i + 3p < 2^22: no wrap
                    uint32_t g = __funnelshift_r(kHalfGaps30, kHalfGaps30, 4 * pos);
                    if (a.strikes) {
                        for (; i < nb; g = __funnelshift_r(g, g, 4)) {
                            strike(sm, i, a.tile_bits);
                            i += p[u] * (g & 15u);
                            ++nstrike;
                        }
                    } else {
                        for (; i < nb; g = __funnelshift_r(g, g, 4)) {
                            strike(sm, i, a.tile_bits);
                            i += p[u] * (g & 15u);
                        }
                    }
                }
            } else {
                // i < 2^20 and p < 3.1e9 (p^2 < 2^63): i + p cannot wrap
                for (; i < nb; i += p[u]) strike(sm, i, a.tile_bits);
            }
        }
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

}  // namespace gb
