// gb_query.cu -- single-n queries: the minimal Goldbach prime p_min(n) of an
// arbitrary even n < 2^63 (GoldbachGPU, arXiv 2603.02621, Sec. 2.4: the
// single-number check, here returning the minimal p and run on the GPU).
//
// One CTA per query.  Candidates p are the odd primes in ascending order, in
// windows of 2 * kQueryBits consecutive integers.  For each window the CTA
// first sieves the partners q = n - p in shared memory by the filter primes
// f <= kFilterMax (bit t <-> p = pl + 2t is cleared when f | q and q != f);
// then 128 candidate primes at a time are looked up in the window and the
// survivors get a deterministic Miller-Rabin test on q (bases the first 12
// primes: no composite below 3.3e24 passes them all; Sorenson and Webster,
// Math. Comp. 2017).  The CTA minimum over the lanes that found a prime
// partner is p_min; the windows stop at the first hit or at p > P.
#include "gb_internal.cuh"

namespace gb {

namespace {

constexpr uint32_t kQueryBits = 2048;      // window: 4096 consecutive integers of p
constexpr uint32_t kFilterMax = 2048;      // filter primes f <= 2048 (q with no factor <= 2048 and q < 2048^2 is prime)
constexpr int kQueryThreads = 128;

// Montgomery multiplication modulo an odd N < 2^63 (Montgomery, Math. Comp.
// 1985): for a, b < N returns a b R^-1 mod N with R = 2^64; ninv = -N^-1 mod
// 2^64.  a b + m N is divisible by R with m = (a b mod R) ninv mod R; its low
// word a b + m N (mod R) is 0, so the carry out of the low word is (lo != 0).
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t N, uint64_t ninv)
{
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t m = lo * ninv;
    const uint64_t t = hi + __umul64hi(m, N) + (lo != 0 ? 1ull : 0ull);   // < 2N < 2^64
    return t >= N ? t - N : t;
}

// strong probable-prime test of odd q > 37 to the bases 2, 3, 5, ..., 37
__device__ bool mr_prime(uint64_t q)
{
    // -q^-1 mod 2^64 by Newton's iteration x <- x (2 - q x): q is its own
    // inverse mod 8 (3 bits), each step doubles the correct bits
    uint64_t x = q;
#pragma unroll
    for (int i = 0; i < 5; ++i) x *= 2 - q * x;
    const uint64_t ninv = 0 - x;
    const uint64_t one = (0 - q) % q;                 // R mod q
    uint64_t r2 = one;                                // R^2 mod q by 64 doublings
    for (int i = 0; i < 64; ++i) {
        r2 <<= 1;                                     // r2 < q < 2^63: no overflow
        if (r2 >= q) r2 -= q;
    }
    const uint64_t minus_one = q - one;               // Montgomery form of q - 1
    uint64_t d = q - 1;
    int s = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++s;
    }
    const uint32_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int b = 0; b < 12; ++b) {
        const uint64_t a = mont_mul(bases[b], r2, q, ninv);     // a R mod q
        // a^d by left-to-right binary exponentiation
        uint64_t y = one;
        for (int bit = 63 - __clzll((long long)d); bit >= 0; --bit) {
            y = mont_mul(y, y, q, ninv);
            if ((d >> bit) & 1) y = mont_mul(y, a, q, ninv);
        }
        if (y == one || y == minus_one) continue;
        bool witness = true;
        for (int i = 1; i < s; ++i) {
            y = mont_mul(y, y, q, ninv);
            if (y == minus_one) {
                witness = false;
                break;
            }
        }
        if (witness) return false;
    }
    return true;
}

// q odd, q >= 3, with no prime factor <= kFilterMax other than itself
__device__ bool partner_prime(uint64_t q)
{
    if (q < (uint64_t)kFilterMax * kFilterMax) return true;
    return mr_prime(q);
}

}  // namespace

__global__ void __launch_bounds__(kQueryThreads) k_query(const QueryArgs a)
{
    __shared__ uint32_t win[kQueryBits / 32];
    __shared__ uint32_t s_best;
    const uint32_t tid = threadIdx.x;
    for (uint32_t qi = blockIdx.x; qi < a.count; qi += gridDim.x) {
        const uint64_t n = a.n[qi];
        if ((n & 1) || n < 4 || n >= (1ull << 63)) {           // not a valid query: no work, flagged
            if (tid == 0) {
                a.out[qi] = 0;
                atomicAdd(a.bad, 1u);
            }
            continue;
        }
        uint32_t best = 0xffffffffu;
        if (n == 4) best = 2;                                   // 4 = 2 + 2, the only even prime partner
        uint32_t k = 1;                                         // next candidate: primes[k]
        uint64_t pl = 3;                                        // window's first p
        while (best == 0xffffffffu && k <= a.K && pl + 3 <= n) {
            const uint64_t ph = pl + 2 * kQueryBits;
            // pre-sieve of the partners: bit t <-> p = pl + 2t, q = n - pl - 2t
            for (uint32_t w = tid; w < kQueryBits / 32; w += kQueryThreads) win[w] = 0xffffffffu;
            if (tid == 0) s_best = 0xffffffffu;
            __syncthreads();
            const uint64_t top = n - pl;                        // q of bit 0 (pl <= n - 3)
            for (uint32_t j = 1 + tid; j <= a.n_filter; j += kQueryThreads) {
                const uint32_t f = a.primes[j];
                const uint32_t r = barrett_mod(top, f, a.recip[j]);
                // 2t = r (mod f)
                uint32_t t = (r & 1u) ? (r + f) >> 1 : r >> 1;
                for (; t < kQueryBits; t += f)
                    if (top - 2ull * t != f) atomicAnd(&win[t >> 5], ~(1u << (t & 31)));
            }
            __syncthreads();
            // candidates of this window, 128 at a time, ascending
            for (;;) {
                const uint32_t kk = k + tid;
                const uint32_t p = kk <= a.K ? a.primes[kk] : 0xffffffffu;
                const bool in = p < ph;
                if (in && (uint64_t)p + 3 <= n) {
                    const uint32_t t = (uint32_t)((p - pl) >> 1);
                    if (((win[t >> 5] >> (t & 31)) & 1u) && partner_prime(n - p)) atomicMin(&s_best, p);
                }
                const int n_in = __syncthreads_count(in);
                best = s_best;
                k += (uint32_t)n_in;
                if (best != 0xffffffffu || n_in < kQueryThreads) break;
            }
            pl = ph;
            __syncthreads();                                    // window reused by the next round
        }
        if (tid == 0) a.out[qi] = best == 0xffffffffu ? 0u : best;
        __syncthreads();
    }
}

cudaError_t launch_query(const QueryArgs& a, cudaStream_t s)
{
    if (a.count == 0) return cudaSuccess;
    if (!a.n || !a.primes || !a.recip || !a.out || !a.bad) return cudaErrorInvalidValue;
    const uint32_t cap = device_sms() * 16u;
    const uint32_t grid = a.count < cap ? a.count : cap;
    k_query<<<grid, kQueryThreads, 0, s>>>(a);
    return cudaGetLastError();
}

uint32_t query_filter_max() { return kFilterMax; }

}  // namespace gb
