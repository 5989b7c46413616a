// gb_batch.cu -- kernels of the batched mode: many ranges of uneven length and
// offset verified in one pass (GoldbachGPU, arXiv 2603.02621: the segment
// loop of Sec. 2.3, here over many independent ranges at once).
//
// The batch lays every range's q window end to end in one buffer.  The tile
// sieve and the block cover run as persistent kernels over (range, tile) and
// (range, chunk) items (gb_sieve.cu, gb_cover_fast.cu); this file holds the
// large-prime strikes over groups of ranges and the per-range reduction.
#include "gb_internal.cuh"

namespace gb {

// primes above the tile size: persistent CTAs take (group, block of 256
// primes) items in group-major order, so the CTAs work on one or two groups at
// a time and the struck words stay in L2; one thread per prime, over the
// pieces of the group in descending order of their prime counts, stopping at
// the first piece its prime does not reach (p^2 beyond the piece's end).
__global__ void __launch_bounds__(256) k_large_batch(const LargeBatchArgs a)
{
    __shared__ uint32_t s_item;
    const uint32_t n_items = *a.n_items;
    unsigned long long nstrike = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const uint32_t g = item / a.nblk;
        const uint32_t k = (item - g * a.nblk) * 256 + threadIdx.x;
        const uint32_t g0 = a.groups[g], g1 = a.groups[g + 1];
        if (g0 == g1 || k >= a.pieces[g0].n_primes) continue;
        const uint32_t p = a.primes[k];
        const uint64_t m = a.recip[k];
        const uint64_t pp = (uint64_t)p * p;
        for (uint32_t pi = g0; pi < g1; ++pi) {
            const LargePiece pc = a.pieces[pi];
            if (k >= pc.n_primes) break;                                   // and every later piece
            const BatchRange r = a.ranges[pc.range];
            const int64_t b = r.B + 2 * (int64_t)pc.bit_lo;               // number at the piece's first bit
            const int64_t last = r.B + 2 * (int64_t)(pc.bit_hi - 1);
            if ((int64_t)pp > last) continue;
            uint64_t i = first_odd_multiple(b, p, m);
            if ((int64_t)pp > b) {
                const uint64_t isq = ((uint64_t)((int64_t)pp - b)) >> 1;
                if (isq > i) i = isq;
            }
            uint32_t* q = a.Q + 2 * r.q_off;
            for (uint64_t bit = pc.bit_lo + i; bit < pc.bit_hi; bit += p) {
                atomicAnd(q + (bit >> 5), __funnelshift_l(0xfffffffeu, 0xfffffffeu, (uint32_t)bit));
                ++nstrike;
            }
        }
    }
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if ((threadIdx.x & 31) == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
}

cudaError_t launch_large_batch(const LargeBatchArgs& a, cudaStream_t s)
{
    if (a.n_primes == 0) return cudaSuccess;
    if (!a.ranges || !a.pieces || !a.groups || a.nblk == 0 || !a.n_items || !a.head || !a.primes || !a.recip || !a.Q)
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large_batch, 256, 0)) != cudaSuccess) return e;
    k_large_batch<<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// per range: key -> (p, n), uint64 histogram row, record; one CTA per range
__global__ void __launch_bounds__(256) k_reduce_batch(const ReduceBatchArgs a)
{
    const uint32_t ri = blockIdx.x;
    if (ri >= *a.count) return;
    const BatchRange r = a.ranges[ri];
    const unsigned long long key = a.maxkey[ri];
    const uint32_t pidx1 = (uint32_t)(key >> 32);
    const uint32_t* hrow = a.hist + (uint64_t)ri * a.hist_stride;
    if (a.rows) {
        uint64_t* orow = a.rows + (uint64_t)ri * a.row_stride;
        for (uint32_t k = threadIdx.x; k < a.row_stride; k += 256)
            orow[k] = (k < pidx1 && k < a.hist_stride) ? hrow[k] : 0ull;
    }
    if (threadIdx.x == 0) {
        SegRecord rec;
        rec.lo = r.lo;
        rec.hi = r.lo + 2 * r.n;
        rec.n_checked = r.n;
        rec.unresolved = a.unresolved[ri];
        rec.max_pmin = pidx1 ? a.primes[pidx1 - 1] : 0u;
        rec.max_pmin_n = pidx1 ? r.lo + 2 * (0xffffffffull - (key & 0xffffffffull)) : 0ull;
        rec.hist_len = pidx1;
        a.records[ri] = rec;
    }
}

cudaError_t launch_reduce_batch(const ReduceBatchArgs& a, uint32_t grid, cudaStream_t s)
{
    if (grid == 0) return cudaSuccess;
    k_reduce_batch<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
