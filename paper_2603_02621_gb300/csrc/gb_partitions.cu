// gb_partitions.cu -- Goldbach partition counts r(n): the number of prime
// pairs p <= q with p + q = n (GoldbachGPU, arXiv 2603.02621, Sec. 4.5: the
// counting of all representations named as future work).
//
// With P the odd-only prime bitset of [1, M) (bit i <-> 2i + 1) and
// m = (n - 2) / 2, the odd pairs are the i <= m / 2 with P[i] and P[m - i]:
// r(n) = popcount over i <= m/2 of P[i] & P[m - i] (n = 4 = 2 + 2 is added
// apart).  P[m - i] is read from the bit-reversed copy Rev (Rev[k] =
// P[Mp - 1 - k], Mp = 32 * words), where it is bit s + i with s = Mp - 1 - m:
// one funnel shift per 32-bit word aligns 32 partners at once, so a word
// step is a funnel shift, an AND and a popcount for 32 pairs.  A warp takes 32
// consecutive n (one per lane) and a run of words; runs of the same n-block
// add into the counts with one atomic per lane.
#include "gb_internal.cuh"

namespace gb {

__global__ void __launch_bounds__(256) k_reverse_bits(const uint32_t* P, uint32_t* rev, uint64_t words)
{
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= words; v += (uint64_t)gridDim.x * blockDim.x)
        rev[v] = v < words ? __brev(P[words - 1 - v]) : 0u;          // one zero word past the end
}

__global__ void __launch_bounds__(256) k_partitions(const PartitionArgs a)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp_id = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t item = warp_id;
    if (item >= (uint64_t)a.n_blocks * a.runs) return;
    const uint64_t blk = item / a.runs, run = item - blk * a.runs;
    const uint64_t j = blk * 32 + lane;                              // n index in the range
    const bool valid = j < a.count;
    const uint64_t n = a.lo + 2 * j;
    const uint64_t m = valid ? (n - 2) / 2 : 0;
    const uint64_t imax = m / 2;                                     // i <= m / 2
    const uint64_t s = (uint64_t)a.words * 32 - 1 - m;              // Rev bit of P[m]
    const uint64_t w0 = run * a.run_words;
    uint64_t w1 = w0 + a.run_words;
    const uint64_t wlast = imax / 32;                                // this lane's last word
    uint32_t cnt = 0;
    if (valid && n >= 6) {
        if (w1 > wlast + 1) w1 = wlast + 1;
        const uint32_t sh = (uint32_t)(s & 31);
        const uint64_t sw = s >> 5;
        for (uint64_t w = w0; w < w1; ++w) {
            const uint32_t pw = __ldg(a.P + w);
            const uint32_t lo_w = __ldg(a.rev + sw + w), hi_w = __ldg(a.rev + sw + w + 1);
            uint32_t x = pw & __funnelshift_r(lo_w, hi_w, sh);
            if (w == wlast) {
                const uint32_t b = (uint32_t)(imax & 31);            // bits 0..b of the last word
                x &= b == 31 ? 0xffffffffu : ((2u << b) - 1u);
            }
            cnt += __popc(x);
        }
    }
    if (run == 0 && valid && n == 4) cnt += 1;                       // 4 = 2 + 2
    if (valid && cnt) atomicAdd(a.counts + j, cnt);
}

cudaError_t launch_reverse_bits(const uint32_t* P, uint32_t* rev, uint64_t words, cudaStream_t s)
{
    if (!P || !rev) return cudaErrorInvalidValue;
    const uint64_t blocks = (words + 1 + 255) / 256;
    const uint64_t cap = (uint64_t)device_sms() * 32;
    k_reverse_bits<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(P, rev, words);
    return cudaGetLastError();
}

cudaError_t launch_partitions(const PartitionArgs& a, cudaStream_t s)
{
    const uint64_t warps = (uint64_t)a.n_blocks * a.runs;
    if (warps == 0) return cudaSuccess;
    if (!a.P || !a.rev || !a.counts || a.runs == 0) return cudaErrorInvalidValue;
    const uint64_t blocks = (warps + 7) / 8;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    k_partitions<<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
