// gb_cover.cu -- the loop-inverted Goldbach cover and its retry pass.
//
// Sec. 2.3.1 of GoldbachGPU (arXiv 2603.02621) inverts the verification loop:
// iterate over the primes p and mark every even n whose partner q = n - p is
// prime.  Sec. 4.3 names the bitwise form of that marking as future work: hold
// the "verified" set as a bitset and replace per-n lookups by word-wide AND/OR
// operations.  This file is that form.
//
// Layout.  A slab holds the even n = A0 + 2j, j = 0 .. n_count-1, 64 per word
// of the coverage bitset C (word w <-> j = 64w .. 64w+63).  The q window Q holds
// the odd numbers B + 2i with B = A0 - H + 1 (H even, larger than every p).  For
// the prime p the partner of n = A0 + 2j sits at bit
//     i = j + (H - p - 1) / 2,
// so for each p, C word w takes the 64 bits of Q starting at bit 64w + d_p with
// d_p = (H - p - 1)/2: a funnel shift of Q words w + d_p/64 and the next one.
//
// For p = 3, 5, 7, ... <= P in ascending order (Sec. 2.3.2: the first hit is the
// minimal Goldbach prime p_min(n)):
//     s   = shifted Q bits            new = s & ~C
//     each bit of new: p_min(n) = p   hist[index(p)] += popc(new)
//     C  |= new
// A warp owns 32 consecutive words and stops as soon as all 32 are full
// (__all_sync), so the work per n is set by the p_min values actually met, not
// by the bound P (Sec. 2.3.4 counts O(S * pi(P)) per segment for the per-n
// form).  The last prime that set a bit in a word, with the lowest such bit,
// gives the word's largest p_min and the smallest n attaining it; a warp and
// then a CTA reduce those to one 64-bit key per segment.
//
// n = 4 is the one even n whose p_min is 2 (4 = 2 + 2); the odd-only window
// cannot represent q = 2, so it is set directly.  Words still not full after
// the first pass go to a retry list; the retry pass continues them with the
// primes P1 < p <= P2 (Sec. 2.3.3's exhaustive fallback, run on the GPU).
#include "gb_internal.cuh"

namespace gb {

__device__ __forceinline__ uint64_t shr_cat(uint64_t lo, uint64_t hi, uint32_t r)
{
    // bits r .. r+63 of the 128-bit value hi:lo
    return r ? (lo >> r) | (hi << (64 - r)) : lo;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_cover(const CoverArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t* sd = smem;                       // d_k for the K odd primes
    uint32_t* shist = smem + a.K;              // K + 1 counters (index 0 = p 2)
    __shared__ unsigned long long smax;

    const uint32_t seg = blockIdx.x / a.chunks_per_seg;
    const uint32_t chunk = blockIdx.x % a.chunks_per_seg;
    const uint64_t seg_w0 = (uint64_t)seg * a.words_per_seg;
    const uint64_t w_begin = seg_w0 + (uint64_t)chunk * a.cta_words;
    uint64_t w_end = w_begin + a.cta_words;
    if (w_end > seg_w0 + a.words_per_seg) w_end = seg_w0 + a.words_per_seg;
    if (w_end > a.n_words) w_end = a.n_words;

    // max-only mode: only segments that no other pass gave a maximum
    if (a.max_only && a.maxkey_check[seg] != 0) return;
    const bool full = !a.max_only;

    for (uint32_t k = threadIdx.x; k < a.K; k += NT) sd[k] = (a.H - a.primes[1 + k] - 1) >> 1;
    for (uint32_t k = threadIdx.x; k <= a.K; k += NT) shist[k] = 0;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long best = 0;
    uint32_t* const pmin = full ? a.pmin : nullptr;

    for (uint64_t wb = w_begin + 32 * warp; wb < w_end; wb += 32 * (NT / 32)) {
        const uint64_t w = wb + lane;
        const bool active = w < w_end;
        uint64_t C = ~0ull;
        if (active) {
            C = 0;
            const uint64_t j0 = 64 * w;
            if (a.n_count - j0 < 64) C = ~0ull << (a.n_count - j0);   // past the slab end
        }
        uint32_t last_pidx1 = 0;      // 1 + prime index of the last prime that set a bit
        uint64_t last_new = 0;
        if (a.has_n4 && w == 0) {
            C |= 1ull;                // n = 4 = 2 + 2
            last_pidx1 = 1;
            last_new = 1ull;
            atomicAdd(&shist[0], 1u);
            if (pmin) pmin[0] = 2;
        }
        const uint64_t* q = a.Q + w;
        for (uint32_t k = 0; k < a.K; ++k) {
            if (__all_sync(0xffffffffu, C == ~0ull)) break;
            const uint32_t d = sd[k];
            uint64_t nw = 0;
            if (active) {
                const uint64_t lo = __ldg(q + (d >> 6));
                const uint64_t hi = __ldg(q + (d >> 6) + 1);
                nw = shr_cat(lo, hi, d & 63) & ~C;
                C |= nw;
            }
            const uint32_t c = __popcll(nw);
            if (nw) {
                last_pidx1 = k + 2;
                last_new = nw;
                if (pmin) {
                    const uint32_t p = a.primes[1 + k];
                    uint64_t m = nw;
                    while (m) {
                        const uint32_t bit = __ffsll(m) - 1;
                        m &= m - 1;
                        pmin[64 * w + bit] = p;
                    }
                }
            }
            const uint32_t tot = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0 && tot) atomicAdd(&shist[k + 1], tot);
        }
        if (full && active && C != ~0ull) {
            bool queued = false;
            if (a.retry) {
                const unsigned int slot = atomicAdd(a.retry_count, 1u);
                if (slot < a.retry_cap) {
                    a.retry[slot].w = w;
                    a.retry[slot].C = C;
                    queued = true;
                }
            }
            if (!queued) atomicAdd(&a.unresolved[seg], (unsigned long long)__popcll(~C));
        }
        if (last_pidx1) {
            const uint64_t j = 64 * (w - seg_w0) + (__ffsll(last_new) - 1);
            const unsigned long long key = ((unsigned long long)last_pidx1 << 32) | (0xffffffffull - j);
            if (key > best) best = key;
        }
        if (full && a.iters) {
            // primes applied until the word filled (all K when it did not)
            uint32_t it = active ? (C == ~0ull ? (last_pidx1 > 1 ? last_pidx1 - 1 : 0) : a.K) : 0;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, it);
            if (lane == 0 && tot) atomicAdd(a.iters, (unsigned long long)tot);
        }
    }
    // warp max of the 64-bit key, then CTA, then segment
    const uint32_t khi = (uint32_t)(best >> 32);
    const uint32_t mhi = __reduce_max_sync(0xffffffffu, khi);
    const uint32_t klo = khi == mhi ? (uint32_t)best : 0u;
    const uint32_t mlo = __reduce_max_sync(0xffffffffu, klo);
    if (lane == 0 && mhi) atomicMax(&smax, ((unsigned long long)mhi << 32) | mlo);
    __syncthreads();
    uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    if (full)
        for (uint32_t k = threadIdx.x; k <= a.K; k += NT)
            if (shist[k]) atomicAdd(&hrow[k], shist[k]);
    if (threadIdx.x == 0 && smax) atomicMax(&a.maxkey[seg], smax);
}

cudaError_t launch_cover(const CoverArgs& a, int threads, cudaStream_t s)
{
    const unsigned grid = a.nseg * a.chunks_per_seg;
    if (grid == 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * a.K + 1) * 4;
    switch (threads) {
    case 128: {
        auto k = k_cover<128>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, 128, smem, s>>>(a);
        break;
    }
    case 512: {
        auto k = k_cover<512>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, 512, smem, s>>>(a);
        break;
    }
    default: {
        auto k = k_cover<256>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, 256, smem, s>>>(a);
        break;
    }
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// retry pass: one thread per queued word, primes P1 < p <= P2 in order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_retry(const RetryArgs a)
{
    const unsigned int n = min(*a.count, a.cap);
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint64_t w = a.items[t].w;
        uint64_t C = a.items[t].C;
        const uint32_t seg = (uint32_t)(w / a.words_per_seg);
        uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
        uint32_t last_pidx1 = 0;
        uint64_t last_new = 0;
        for (uint32_t k = a.K1 + 1; k <= a.K2 && C != ~0ull; ++k) {
            const uint32_t p = a.primes[k];
            const uint32_t d = (a.H - p - 1) >> 1;
            const uint64_t* q = a.Q + w + (d >> 6);
            const uint64_t nw = shr_cat(q[0], q[1], d & 63) & ~C;
            if (nw) {
                C |= nw;
                atomicAdd(&hrow[k], (uint32_t)__popcll(nw));
                last_pidx1 = k + 1;
                last_new = nw;
                if (a.pmin) {
                    uint64_t m = nw;
                    while (m) {
                        const uint32_t bit = __ffsll(m) - 1;
                        m &= m - 1;
                        a.pmin[64 * w + bit] = p;
                    }
                }
            }
        }
        if (C != ~0ull) atomicAdd(&a.unresolved[seg], (unsigned long long)__popcll(~C));
        if (last_pidx1) {
            const uint64_t j = 64 * (w - (uint64_t)seg * a.words_per_seg) + (__ffsll(last_new) - 1);
            atomicMax(&a.maxkey[seg], ((unsigned long long)last_pidx1 << 32) | (0xffffffffull - j));
        }
    }
}

cudaError_t launch_retry(const RetryArgs& a, cudaStream_t s)
{
    k_retry<<<2 * device_sms(), 128, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-segment reduction: key -> (p, j), uint64 histogram rows, merged histogram
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_reduce(const ReduceArgs a)
{
    const uint32_t seg = blockIdx.x;
    unsigned long long key = a.maxkey[seg];
    if (a.maxkey2 && a.maxkey2[seg] > key) key = a.maxkey2[seg];
    const uint32_t pidx1 = (uint32_t)(key >> 32);
    const uint32_t hl = pidx1;                      // entries >= hl are all zero
    const uint32_t* hrow = a.hist + (uint64_t)seg * a.hist_stride;
    const bool row = a.rows && seg < a.nrows;
    for (uint32_t k = threadIdx.x; k < hl; k += 256) {
        const uint32_t v = hrow[k];
        if (v) atomicAdd(&a.merged[k], (unsigned long long)v);
        if (row && k < a.row_stride) a.rows[(uint64_t)seg * a.row_stride + k] = v;
    }
    if (row)
        for (uint32_t k = hl + threadIdx.x; k < a.row_stride; k += 256)
            a.rows[(uint64_t)seg * a.row_stride + k] = 0;
    if (threadIdx.x == 0) {
        SegSummary s;
        s.unresolved = a.unresolved[seg];
        s.hist_len = hl;
        s.max_pmin = pidx1 ? a.primes[pidx1 - 1] : 0u;
        s.max_j = pidx1 ? (0xffffffffull - (key & 0xffffffffull)) : 0ull;
        a.summary[seg] = s;
    }
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s)
{
    if (a.nseg == 0) return cudaSuccess;
    k_reduce<<<a.nseg, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// range totals: unresolved sum, largest p_min with the smallest n (segments
// ascend, so among equal maxima the lowest segment wins), public records
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_finalize(const FinalizeArgs a)
{
    unsigned long long unres = 0, best = 0;        // best: p << 32 | (0xffffffff - seg)
    for (uint32_t k = threadIdx.x; k < a.nseg; k += 1024) {
        const SegSummary g = a.summary[k];
        unres += g.unresolved;
        if (g.max_pmin) {
            const unsigned long long key = ((unsigned long long)g.max_pmin << 32) | (0xffffffffull - k);
            if (key > best) best = key;
        }
        if (a.records && k < a.nrecords) {
            SegRecord r;
            r.lo = a.lo + 2 * (uint64_t)k * a.S;
            r.hi = r.lo + 2 * a.S < a.hi ? r.lo + 2 * a.S : a.hi;
            r.n_checked = (r.hi - r.lo) / 2;
            r.unresolved = g.unresolved;
            r.max_pmin = g.max_pmin;
            r.max_pmin_n = g.max_pmin ? r.lo + 2 * g.max_j : 0;
            r.hist_len = g.hist_len;
            a.records[k] = r;
        }
    }
    __shared__ unsigned long long s_unres, s_best;
    if (threadIdx.x == 0) { s_unres = 0; s_best = 0; }
    __syncthreads();
    atomicAdd(&s_unres, unres);
    atomicMax(&s_best, best);
    __syncthreads();
    if (threadIdx.x == 0) {
        RangeTotals t{};
        t.unresolved = s_unres;
        if (s_best) {
            const uint32_t k = 0xffffffffu - (uint32_t)(s_best & 0xffffffffull);
            const SegSummary g = a.summary[k];
            t.max_pmin = g.max_pmin;
            t.max_pmin_n = a.lo + 2 * (uint64_t)k * a.S + 2 * g.max_j;
            t.hist_len = g.hist_len;
        }
        *a.totals = t;
    }
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s)
{
    k_finalize<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
