// gb_bucket.cu -- bucket sieve for the primes above the tile split
// (GoldbachGPU, arXiv 2603.02621, Sec. 2.3.1: a segmented sieve of [A, B]
// with the primes to sqrt(B); the large primes binned into per-tile hit lists
// as in the cache-efficient segmented sieves the paper cites).
//
// A chunk of the q window (at most 2^30 bits) is cut into bucket tiles of
// 2^20 bits.  Fill: persistent CTAs take blocks of 256 consecutive large
// primes (CTA c gets blocks c, c + G, c + 2G, ...: every CTA sees primes of
// every size, so its share of the hits is the mean plus at most one block's);
// each thread walks its prime's hits in the chunk (one Barrett start per prime
// and piece) and stages each hit's 20-bit offset in shared memory, in a small
// buffer per bucket tile, up to 16 hits per round.  A bucket whose buffer
// reaches half full is flushed by one warp to the CTA's own list for that
// tile in global memory: coalesced stores, no atomics.  Apply: one CTA per bucket tile loads the tile's q words into
// shared memory, clears the bit of every entry of every CTA's list with a
// shared-memory atomic AND, and stores the words back.
//
// Per hit: one shared atomic and store when staged, one coalesced 4-byte
// global store when flushed, one 4-byte global load and one shared atomic
// when applied -- instead of one global atomic per hit.
#include "gb_internal.cuh"

namespace gb {

namespace {

constexpr int kFillThreads = 256;
constexpr int kFillWarps = kFillThreads / 32;
constexpr uint32_t kStage = 16;            // staged entries per bucket tile
constexpr uint32_t kFlushAt = kStage / 2;  // a bucket reaching this is flushed after the round
constexpr uint32_t kPerRound = 16;         // hits a thread stages per round
constexpr uint32_t kFlushList = kPerRound * kFillThreads;   // at most one listing per staged hit
constexpr int kApplyThreads = 1024;

struct Cursor {
    uint32_t piece;                        // current piece (n_pieces: exhausted)
    uint64_t i;                            // next hit, piece-relative bit
    uint64_t pos;                          // chunk bit of the piece's first bit
    uint64_t len;                          // piece bits
};

__device__ __forceinline__ BucketPiece piece_at(const BucketFillArgs& a, uint32_t k)
{
    return a.pieces ? a.pieces[k] : a.single;
}

// first hit of p at or after piece c.piece (p^2 and the first odd multiple)
__device__ __forceinline__ void seek(const BucketFillArgs& a, uint32_t npieces, uint32_t p, uint64_t m,
                                     uint64_t pp, Cursor& c)
{
    for (; c.piece < npieces; ++c.piece) {
        const BucketPiece pc = piece_at(a, c.piece);
        const int64_t b = pc.B + 2 * (int64_t)pc.r_lo;              // number at the piece's first bit
        const int64_t last = pc.B + 2 * (int64_t)(pc.r_hi - 1);
        if ((int64_t)pp > last) continue;
        uint64_t j = first_odd_multiple(b, p, m);
        if ((int64_t)pp > b) {
            const uint64_t isq = ((uint64_t)((int64_t)pp - b)) >> 1;
            if (isq > j) j = isq;
        }
        if (j < pc.r_hi - pc.r_lo) {
            c.i = j;
            c.pos = pc.pos;
            c.len = pc.r_hi - pc.r_lo;
            return;
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kFillThreads) k_bucket_fill(const BucketFillArgs a)
{
    extern __shared__ uint32_t smem[];
    uint32_t* stage = smem;                                  // [K][kStage]
    uint32_t* cnt = stage + (size_t)a.K * kStage;            // [K] staged entries (may overshoot kStage)
    uint32_t* gcnt = cnt + a.K;                              // [K] entries in this CTA's global lists
    uint32_t* flist = gcnt + a.K;                            // [kFlushList] buckets to flush this round
    __shared__ uint32_t n_flush;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = threadIdx.x; t < a.K; t += kFillThreads) {
        cnt[t] = 0;
        gcnt[t] = 0;
    }
    if (threadIdx.x == 0) n_flush = 0;
    __syncthreads();

    uint32_t* lists = a.lists + (size_t)blockIdx.x * a.K * a.cap;
    const uint32_t npieces = a.pieces ? a.n_pieces : 1u;
    const uint64_t per_step = (uint64_t)kFillThreads * gridDim.x;   // primes per step, whole grid
    const uint64_t steps = (a.n_primes + per_step - 1) / per_step;
    unsigned long long nstrike = 0;
    bool ovf = false;

    for (uint64_t st = 0; st < steps; ++st) {
        // a block of kFillThreads consecutive primes per CTA: similar sizes,
        // so the threads of a step have similar hit counts
        const uint64_t k = (st * gridDim.x + blockIdx.x) * kFillThreads + threadIdx.x;
        Cursor c{npieces, 0, 0, 0};
        uint32_t p = 0;
        uint64_t m = 0;
        if (k < a.n_primes) {
            p = a.primes[k];
            m = a.recip[k];
            c.piece = 0;
            seek(a, npieces, p, m, (uint64_t)p * p, c);
        }
        bool active = c.piece < npieces;
        while (__syncthreads_or(active)) {
            // up to kPerRound hits per thread; stop at a full buffer (retried
            // after the flush)
            for (uint32_t r = 0; r < kPerRound && active; ++r) {
                const uint64_t cb = c.pos + c.i;                      // chunk bit
                const uint32_t t = (uint32_t)(cb >> kBucketTileLog2);
                const uint32_t slot = atomicAdd(&cnt[t], 1u);
                if (slot >= kStage) break;
                stage[t * kStage + slot] = (uint32_t)cb & ((1u << kBucketTileLog2) - 1u);
                if (slot == kFlushAt - 1) flist[atomicAdd(&n_flush, 1u)] = t;
                ++nstrike;
                c.i += p;
                if (c.i >= c.len) {
                    ++c.piece;
                    seek(a, npieces, p, m, (uint64_t)p * p, c);
                    active = c.piece < npieces;
                }
            }
            __syncthreads();
            // every bucket holding >= kFlushAt entries crossed kFlushAt this
            // round (earlier crossings were flushed), so it is listed
            // (two buckets per warp step: one per half-warp)
            const uint32_t nf = n_flush;
            const uint32_t h = (uint32_t)lane >> 4, hl = (uint32_t)lane & 15u;
            for (uint32_t f = 2 * warp + h; f < nf; f += 2 * kFillWarps) {
                const uint32_t t = flist[f];
                const uint32_t cc = min(cnt[t], kStage);
                const uint32_t g = gcnt[t];
                if (hl < cc) {
                    if (g + hl < a.cap) lists[(size_t)t * a.cap + g + hl] = stage[t * kStage + hl];
                    else ovf = true;
                }
                __syncwarp(0xffffu << (16 * h));
                if (hl == 0) {
                    gcnt[t] = g + cc;
                    cnt[t] = 0;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) n_flush = 0;
        }
    }
    // the rest of every buffer
    __syncthreads();
    for (uint32_t t = warp; t < a.K; t += kFillWarps) {
        const uint32_t cc = min(cnt[t], kStage);
        const uint32_t g = gcnt[t];
        if ((uint32_t)lane < cc) {
            if (g + lane < a.cap) lists[(size_t)t * a.cap + g + lane] = stage[t * kStage + lane];
            else ovf = true;
        }
        __syncwarp();
        if (lane == 0) gcnt[t] = g + cc;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < a.K; t += kFillThreads)
        a.counts[(size_t)blockIdx.x * a.K + t] = min(gcnt[t], a.cap);
    if (ovf) atomicOr(a.overflow, 1u);
    if (a.strikes) {
        for (int o = 16; o; o >>= 1) nstrike += __shfl_xor_sync(0xffffffffu, nstrike, o);
        if (lane == 0 && nstrike) atomicAdd(a.strikes, nstrike);
    }
}

__global__ void __launch_bounds__(kApplyThreads) k_bucket_apply(const BucketApplyArgs a)
{
    extern __shared__ uint32_t tile[];                      // 2^15 words
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kApplyThreads / 32;
    for (uint32_t t = blockIdx.x; t < a.K; t += gridDim.x) {
        const uint64_t bit0 = (uint64_t)t << kBucketTileLog2;
        const uint64_t nbits = a.span - bit0 < (1ull << kBucketTileLog2) ? a.span - bit0 : (1ull << kBucketTileLog2);
        const uint32_t nw = (uint32_t)((nbits + 31) / 32);
        uint32_t* q = a.q + bit0 / 32;
        for (uint32_t w = threadIdx.x; w < nw; w += kApplyThreads) tile[w] = q[w];
        __syncthreads();
        for (uint32_t g = warp; g < a.G; g += NW) {
            const uint32_t c = a.counts[(size_t)g * a.K + t];
            const uint32_t* L = a.lists + ((size_t)g * a.K + t) * a.cap;
            for (uint32_t e = lane; e < c; e += 32) {
                const uint32_t off = L[e];
                atomicAnd(&tile[off >> 5], __funnelshift_l(0xfffffffeu, 0xfffffffeu, off));
            }
        }
        __syncthreads();
        for (uint32_t w = threadIdx.x; w < nw; w += kApplyThreads) q[w] = tile[w];
        __syncthreads();
    }
}

uint32_t bucket_fill_grid()
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t smem = bucket_fill_smem(kMaxBuckets);
    if (cudaFuncSetAttribute(k_bucket_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bucket_fill, kFillThreads, smem) != cudaSuccess)
        return 0;
    return (uint32_t)(sms * (per_sm > 0 ? per_sm : 1));
}

size_t bucket_fill_smem(uint32_t K) { return ((size_t)K * (kStage + 2) + kFlushList) * 4; }

cudaError_t launch_bucket_fill(const BucketFillArgs& a, uint32_t grid, cudaStream_t s)
{
    if (a.n_primes == 0 || a.K == 0) return cudaSuccess;
    if (a.K > kMaxBuckets || !a.primes || !a.recip || !a.lists || !a.counts || !a.overflow) return cudaErrorInvalidValue;
    const size_t smem = bucket_fill_smem(kMaxBuckets);
    cudaError_t e = cudaFuncSetAttribute(k_bucket_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bucket_fill<<<grid, kFillThreads, bucket_fill_smem(a.K), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bucket_apply(const BucketApplyArgs& a, cudaStream_t s)
{
    if (a.K == 0 || a.span == 0) return cudaSuccess;
    if (!a.lists || !a.counts || !a.q) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(1u << kBucketTileLog2) / 8;
    cudaError_t e = cudaFuncSetAttribute(k_bucket_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const uint32_t grid = a.K < (uint32_t)sms ? a.K : (uint32_t)sms;
    k_bucket_apply<<<grid, kApplyThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gb
