// gb_api.cu -- runtime and C ABI of libgb (declared in include/gb.h).
//
// The runtime owns the device arenas of a context and plans the work of a call:
//   gb_init          seed sieve (primes < 2^16) -> base sieve of [1, L] on the GPU
//                    -> compaction to the ascending prime list with Barrett
//                    reciprocals; L = max(base_limit, p1, p2)
//   gb_verify_range  the range is cut into segments of S even n (the unit of
//                    output) and slabs of whole segments (the unit of residency);
//                    per slab: segment sieve of the q window -> cover (p <= P1) ->
//                    retry (P1 < p <= P2) -> per-segment reduction; one copy of the
//                    results to the host at the end.
// Sec. 2.3 of GoldbachGPU (arXiv 2603.02621) describes the segment loop and its
// two phases; the structure above keeps them and moves the sieve to the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <memory>
#include <vector>

#include "gb.h"
#include "gb_internal.cuh"

namespace {

enum { kProfSieve = 0, kProfCover = 1, kProfRetry = 2, kProfReduce = 3, kProfLarge = 4 };

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

#define GB_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(GB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
// a kernel launch of a verification call, counted for the profile
#define GB_LAUNCH(expr)       \
    do {                      \
        GB_CUDA(expr);        \
        ctx->kernels += 1;    \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes)
    {
        if (bytes <= cap) return GB_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 8 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        cap = want;
        return GB_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    // take ownership of other's allocation (other is left empty)
    void take(DevBuf& other)
    {
        if (&other == this) return;
        release();
        p = other.p;
        cap = other.cap;
        other.p = nullptr;
        other.cap = 0;
    }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// grow-only pinned host buffer (staging of batch descriptors and results)
struct HostBuf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes)
    {
        if (bytes <= cap) return GB_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = bytes + bytes / 8 + 4096;
        const cudaError_t e = cudaMallocHost(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GB_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        }
        cap = want;
        return GB_OK;
    }
    HostBuf() = default;
    HostBuf(const HostBuf&) = delete;
    HostBuf& operator=(const HostBuf&) = delete;
    ~HostBuf()
    {
        if (p) cudaFreeHost(p);
    }
};

uint64_t isqrt_u64(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        uint64_t t = r | (1ull << b);
        if (t * t <= x) r = t;
    }
    return r;
}

}  // namespace

// base primes: built once by gb_init, shared with the contexts made from it
// by gb_init_shared (freed with the last of them)
struct BasePrimes {
    std::vector<uint32_t> h_primes;   // [2, 3, 5, ...] <= L
    DevBuf primes, recip;             // device copies
    DevBuf wheel;                     // pre-sieve stamp tables
};

struct gb_ctx {
    gb_config cfg{};
    cudaStream_t stream = nullptr;
    uint64_t L = 0;                   // primes are known up to L
    std::shared_ptr<BasePrimes> base = std::make_shared<BasePrimes>();
    DevBuf q;                         // slab q window
    DevBuf hist, maxkey, maxkey2, unres, retry, retry_count, summary, rows, merged, pmin, counter, totals, records;
    DevBuf work;                      // profiling work counters: [0] sieve strikes, [1] cover iterations
    // batched mode
    DevBuf bq, bhist, bkeys, bunres, bdesc, brecords, brows;
    DevBuf qn, qout;                  // single-n queries: inputs, outputs + invalid-n counter
    DevBuf part_p, part_rev, part_out;  // partition counts: prime bits, reversed bits, counts
    HostBuf hstage;
    bool batch_graph = true;          // batch kernels as one CUDA graph (GB_BATCH_GRAPH=0: plain launches)
    // bucket sieve of the primes >= 2^20 (GB_LARGE=bucket); by default they
    // are struck by global atomics, measured faster on GB300
    bool bucket_large = false;
    bool fused = false;               // sieve and block cover fused per CTA (GB_FUSED=1)
    uint32_t mid_limit = 1u << 20;    // primes from the split below this: per 2^20-bit slice (GB_MID_LOG2; 0 = off)
    uint32_t fill_grid = 0;           // persistent fill CTAs
    uint32_t bcap = 0;                // entries per (CTA, bucket tile) list
    uint64_t bucket_overflows = 0;    // chunks redone by the atomic kernel
    DevBuf blists, bcounts, bflags;

    // size the bucket lists for large primes [nsmall, np) and zero nchunks overflow flags
    int bucket_setup(uint64_t nsmall, uint64_t np, uint32_t nchunks)
    {
        if (!fill_grid) {
            fill_grid = gb::bucket_fill_grid();
            if (!fill_grid) return fail(GB_ECUDA, "bucket fill occupancy");
        }
        // hits per tile ~ 2^20 * sum 1/p over the large primes (Mertens:
        // ln ln p_last - ln ln p_first), shared by the fill CTAs; a CTA's
        // share is at most its first block of 256 primes plus the mean
        const double p0 = (double)base->h_primes[nsmall], p1 = (double)base->h_primes[np - 1];
        const double T = (double)(1u << gb::kBucketTileLog2);
        const double sinv = std::log(std::log(p1)) - std::log(std::log(p0)) + 1.0 / p0;
        const double mean = T * sinv / fill_grid;
        const double wmax = 256.0 * (T / p0 + 1.0);
        double c = mean + wmax + 8.0 * std::sqrt(mean + wmax) + 64.0;
        bcap = ((uint32_t)c + 31u) & ~31u;
        int rc;
        const size_t lists = (size_t)fill_grid * gb::kMaxBuckets * bcap * 4;
        if ((rc = blists.ensure(lists)) || (rc = bcounts.ensure((size_t)fill_grid * gb::kMaxBuckets * 4)) ||
            (rc = bflags.ensure((size_t)nchunks * 4)))
            return rc;
        GB_CUDA(cudaMemsetAsync(bflags.p, 0, (size_t)nchunks * 4, stream));
        return GB_OK;
    }
    bool capturing = false;           // cap_stream is being captured (profiling events become graph nodes)
    cudaStream_t cap_stream = nullptr;  // private stream the batch graph is captured on
    cudaGraphExec_t bgraph = nullptr;
    uint64_t work_strikes = 0, work_iters = 0, work_large = 0;
    int warp_split = 0;               // sieving primes below this strike one warp each
    bool generic_cover = false;       // force the generic cover kernel (GB_COVER=generic)
    uint64_t large_chunk_bits = 1ull << 28;   // large-prime strikes per L2-resident chunk of the window

    // per-kernel device time (CUDA events on the context's stream around each launch)
    bool profiling = false;
    double prof_ms[GB_PROF_KINDS] = {};
    uint64_t prof_launches[GB_PROF_KINDS] = {};
    uint64_t prof_units[GB_PROF_KINDS] = {};
    uint64_t kernels = 0;             // kernels launched by verification calls since profiling was enabled
    struct Pending { cudaEvent_t a, b; int kind; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int cur_kind = -1;
    cudaEvent_t cur_a = nullptr;

    cudaEvent_t take_event()
    {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void prof_begin(int kind, uint64_t units)
    {
        if (!profiling) return;
        cur_kind = kind;
        cur_a = take_event();
        cudaEventRecordWithFlags(cur_a, capturing ? cap_stream : stream,
                                 capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        prof_launches[kind] += 1;
        prof_units[kind] += units;
    }
    void prof_end()
    {
        if (!profiling || cur_kind < 0) return;
        cudaEvent_t b = take_event();
        cudaEventRecordWithFlags(b, capturing ? cap_stream : stream,
                                 capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        pending.push_back({cur_a, b, cur_kind});
        cur_kind = -1;
    }
    unsigned long long* work_ptr(int i) { return profiling && work.p ? work.as<unsigned long long>() + i : nullptr; }
    int prof_collect()
    {
        if (work.p) {
            unsigned long long w[3] = {0, 0, 0};
            cudaError_t e = cudaMemcpy(w, work.p, sizeof w, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemset(work.p, 0, sizeof w);
            if (e != cudaSuccess) return fail(GB_ECUDA, std::string("profile counters: ") + cudaGetErrorString(e));
            work_strikes += w[0];
            work_iters += w[1];
            work_large += w[2];
        }
        for (const Pending& p : pending) {
            cudaError_t e = cudaEventSynchronize(p.b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
            if (e != cudaSuccess) return fail(GB_ECUDA, std::string("profile events: ") + cudaGetErrorString(e));
            prof_ms[p.kind] += ms;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        return GB_OK;
    }
    ~gb_ctx()
    {
        if (bgraph) cudaGraphExecDestroy(bgraph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (const Pending& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }

    // number of primes <= x (x <= L)
    uint64_t pi(uint64_t x) const
    {
        return (uint64_t)(std::upper_bound(base->h_primes.begin(), base->h_primes.end(), (uint32_t)std::min<uint64_t>(x, 0xffffffffull)) - base->h_primes.begin());
    }
};

namespace {

int fill_defaults(gb_config& c)
{
    if (c.seg_len == 0) c.seg_len = 1u << 24;
    if (c.base_limit == 0) c.base_limit = 1u << 16;
    if (c.tile_bits == 0) c.tile_bits = 1u << 18;
    if (c.cta_threads == 0) c.cta_threads = 256;
    if (c.bucket_split == 0) c.bucket_split = c.tile_bits;
    if (c.p1 == 0) c.p1 = 1u << 15;
    if (c.slab_bits == 0) c.slab_bits = 1ull << 33;
    if (c.seg_len % 2048 || c.seg_len > (1u << 30))
        return fail(GB_EINVAL, "seg_len must be a multiple of 2048 and <= 2^30");
    if (c.tile_bits % 8192 || c.tile_bits > (1u << 20))
        return fail(GB_EINVAL, "tile_bits must be a multiple of 8192 and <= 2^20");
    if (c.cta_threads != 128 && c.cta_threads != 256 && c.cta_threads != 512)
        return fail(GB_EINVAL, "cta_threads must be 128, 256 or 512");
    if (c.base_limit > (1ull << 32)) return fail(GB_EINVAL, "base_limit must be <= 2^32");
    if (c.p1 < 2 || c.p1 > (1u << 24) || c.p2 > (1u << 24))
        return fail(GB_EINVAL, "p1 must be in [2, 2^24] and p2 <= 2^24");
    if (c.cover_prefix != 0 && c.cover_prefix != 1 && c.cover_prefix != 64 && c.cover_prefix != 128 &&
        c.cover_prefix != 192 && c.cover_prefix != 256)
        return fail(GB_EINVAL, "cover_prefix must be 0, 1, 64, 128, 192 or 256");
    if (c.slab_bits < c.seg_len) c.slab_bits = c.seg_len;
    return GB_OK;
}

// sieve the odd numbers B + 2i, i < nbits, into out (device words) or count only
// tile-sieve arguments for the window (B, nbits): the primes below the split
// (from 47 on; 3..43 are stamped); *np and *nsmall receive the count of
// primes <= sqrt(last number) and of those below the split
int tile_sieve_args(gb_ctx* ctx, int64_t B, uint64_t nbits, gb::SieveArgs& a, uint64_t& np, uint64_t& nsmall)
{
    const int64_t last = B + 2 * (int64_t)(nbits - 1);
    const uint64_t r = last > 0 ? isqrt_u64((uint64_t)last) : 0;
    if (r > ctx->L) return fail(GB_EINVAL, "window beyond base_limit^2");
    np = ctx->pi(r);                                // primes <= sqrt(last)
    nsmall = std::min<uint64_t>(np, std::max<uint64_t>(ctx->pi(ctx->cfg.bucket_split - 1), gb::kFirstStrikeIdx));
    a = gb::SieveArgs{};
    a.B = B;
    a.nbits = nbits;
    a.tile_bits = ctx->cfg.tile_bits;
    a.primes = ctx->base->primes.as<uint32_t>() + gb::kFirstStrikeIdx;
    a.recip = ctx->base->recip.as<uint64_t>() + gb::kFirstStrikeIdx;
    const uint64_t nstrike = nsmall > gb::kFirstStrikeIdx ? nsmall - gb::kFirstStrikeIdx : 0;
    const uint64_t nwarp = std::min<uint64_t>(nstrike, ctx->pi((uint64_t)ctx->warp_split - 1) > gb::kFirstStrikeIdx
                                                            ? ctx->pi((uint64_t)ctx->warp_split - 1) - gb::kFirstStrikeIdx : 0);
    a.n_warp = (uint32_t)nwarp;
    a.n_primes = (uint32_t)nstrike;
    a.wheel = ctx->base->wheel.as<uint32_t>();
    a.strikes = ctx->work_ptr(0);
    return GB_OK;
}

int run_sieve(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out, unsigned long long* popc)
{
    if (nbits == 0) return GB_OK;
    // primes from bucket_split on are struck by the large-prime kernel, chunk
    // by chunk, into the output words (the tile kernel only counts bits when
    // there are none)
    gb::SieveArgs a{};
    uint64_t np = 0, nsmall = 0;
    int rc0 = tile_sieve_args(ctx, B, nbits, a, np, nsmall);
    if (rc0) return rc0;
    const bool large = np > nsmall && out;
    if (np > nsmall && !out) return fail(GB_EINVAL, "internal: large primes need an output buffer");
    a.out = out;
    a.popcount = large ? nullptr : popc;
    ctx->prof_begin(kProfSieve, nbits);
    GB_LAUNCH(gb::launch_sieve(a, (int)ctx->cfg.cta_threads, ctx->stream));
    ctx->prof_end();
    if (large) {
        ctx->prof_begin(kProfLarge, nbits);
        gb::LargeArgs la{};
        la.B = B;
        la.primes = ctx->base->primes.as<uint32_t>() + nsmall;
        la.recip = ctx->base->recip.as<uint64_t>() + nsmall;
        la.n_primes = (uint32_t)(np - nsmall);
        la.out = out;
        la.strikes = ctx->work_ptr(2);
        // primes below mid_limit: per 2^20-bit slice in shared memory
        uint64_t nmid = nsmall;
        if (ctx->mid_limit > ctx->cfg.bucket_split) {
            nmid = std::min<uint64_t>(np, std::max<uint64_t>(nsmall, ctx->pi(ctx->mid_limit - 1)));
            if (nmid > nsmall) {
                gb::LargeArgs ma = la;
                ma.n_primes = (uint32_t)(nmid - nsmall);
                GB_LAUNCH(gb::launch_mid(ma, nbits, ctx->stream));
            }
            la.primes = ctx->base->primes.as<uint32_t>() + nmid;
            la.recip = ctx->base->recip.as<uint64_t>() + nmid;
            la.n_primes = (uint32_t)(np - nmid);
        }
        // primes of at least a bucket tile (2^20) go to the bucket sieve; those
        // between the split and a bucket tile hit a tile several times and
        // keep the atomic kernel
        const uint64_t nbucket_lo = ctx->bucket_large ? std::max<uint64_t>(nmid, ctx->pi((1u << gb::kBucketTileLog2) - 1)) : np;
        if (nbucket_lo < np) {
            // bucket sieve, chunk by chunk of at most 2^30 bits; a chunk whose
            // lists overflowed is struck again by the atomic kernel below
            const uint64_t chunk = (uint64_t)gb::kMaxBuckets << gb::kBucketTileLog2;
            const uint32_t nchunks = (uint32_t)((nbits + chunk - 1) / chunk);
            int rc = ctx->bucket_setup(nbucket_lo, np, nchunks);
            if (rc) return rc;
            gb::BucketFillArgs fa{};
            fa.primes = ctx->base->primes.as<uint32_t>() + nbucket_lo;
            fa.recip = ctx->base->recip.as<uint64_t>() + nbucket_lo;
            fa.n_primes = (uint32_t)(np - nbucket_lo);
            fa.lists = ctx->blists.as<uint32_t>();
            fa.counts = ctx->bcounts.as<uint32_t>();
            fa.cap = ctx->bcap;
            fa.strikes = ctx->work_ptr(2);
            gb::BucketApplyArgs aa{};
            aa.lists = fa.lists;
            aa.counts = fa.counts;
            aa.G = ctx->fill_grid;
            aa.cap = ctx->bcap;
            for (uint32_t c = 0; c < nchunks; ++c) {
                const uint64_t c0 = (uint64_t)c * chunk, span = std::min(nbits - c0, chunk);
                fa.single = gb::BucketPiece{B, c0, c0 + span, 0};
                fa.K = aa.K = (uint32_t)((span + (1u << gb::kBucketTileLog2) - 1) >> gb::kBucketTileLog2);
                fa.overflow = ctx->bflags.as<unsigned int>() + c;
                aa.q = out + c0 / 32;
                aa.span = span;
                GB_LAUNCH(gb::launch_bucket_fill(fa, ctx->fill_grid, ctx->stream));
                GB_LAUNCH(gb::launch_bucket_apply(aa, ctx->stream));
            }
            std::vector<unsigned int> flags(nchunks);
            GB_CUDA(cudaMemcpyAsync(flags.data(), ctx->bflags.p, nchunks * 4, cudaMemcpyDeviceToHost, ctx->stream));
            GB_CUDA(cudaStreamSynchronize(ctx->stream));
            for (uint32_t c = 0; c < nchunks; ++c) {
                if (!flags[c]) continue;
                gb::LargeArgs lb = la;
                lb.primes = fa.primes;
                lb.recip = fa.recip;
                lb.n_primes = fa.n_primes;
                lb.bit_lo = (uint64_t)c * chunk;
                lb.bit_hi = std::min(nbits, lb.bit_lo + chunk);
                lb.strikes = nullptr;
                ctx->bucket_overflows += 1;
                GB_LAUNCH(gb::launch_large(lb, ctx->stream));
            }
        }
        if (nbucket_lo > nmid) {
            la.n_primes = (uint32_t)(nbucket_lo - nmid);
            const uint64_t chunk = ctx->large_chunk_bits;
            for (uint64_t c0 = 0; c0 < nbits; c0 += chunk) {
                la.bit_lo = c0;
                la.bit_hi = std::min(nbits, c0 + chunk);
                GB_LAUNCH(gb::launch_large(la, ctx->stream));
            }
        }
        if (popc) GB_LAUNCH(gb::launch_popcount(out, ((nbits + 63) / 64) * 2, popc, ctx->stream));
        ctx->prof_end();
    }
    return GB_OK;
}

int build_primes(gb_ctx* ctx)
{
    cudaStream_t s = ctx->stream;
    int rc;
    if ((rc = ctx->base->wheel.ensure(gb::kWheelWords * 4))) return rc;
    GB_CUDA(gb::launch_wheel_tables(ctx->base->wheel.as<uint32_t>(), s));

    // seed: odd numbers 1 .. 65535
    DevBuf seedbits, counts, seedp, seedr;
    const uint64_t seed_words = 1024;
    if ((rc = seedbits.ensure(seed_words * 4)) || (rc = counts.ensure(gb::compact_chunks(seed_words) * 4)) ||
        (rc = seedp.ensure(8192 * 4)) || (rc = seedr.ensure(8192 * 8)))
        return rc;
    GB_CUDA(gb::launch_seed_sieve(seedbits.as<uint32_t>(), s));
    gb::CompactArgs ca{seedbits.as<uint32_t>(), seed_words, 1, counts.as<uint32_t>(), seedp.as<uint32_t>(),
                       seedr.as<uint64_t>()};
    GB_CUDA(gb::launch_compact(ca, s));
    std::vector<uint32_t> seedw(seed_words);
    GB_CUDA(cudaMemcpyAsync(seedw.data(), seedbits.p, seed_words * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    size_t nseed = 1;                                 // the prime 2
    for (uint32_t v : seedw) nseed += (size_t)__builtin_popcount(v);
    std::vector<uint32_t> seed(nseed);
    GB_CUDA(cudaMemcpyAsync(seed.data(), seedp.p, nseed * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    seedbits.release();

    if (ctx->L <= 65535) {
        // the seed list already holds every prime <= L
        ctx->base->h_primes.assign(seed.begin(), seed.end());
        ctx->base->h_primes.resize(std::upper_bound(seed.begin(), seed.end(), (uint32_t)ctx->L) - seed.begin());
        const size_t n = ctx->base->h_primes.size();
        if ((rc = ctx->base->primes.ensure(n * 4)) || (rc = ctx->base->recip.ensure(n * 8))) return rc;
        GB_CUDA(cudaMemcpyAsync(ctx->base->primes.p, seedp.p, n * 4, cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaMemcpyAsync(ctx->base->recip.p, seedr.p, n * 8, cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaStreamSynchronize(s));
        return GB_OK;
    }

    // base sieve of the odd numbers 1 .. L with the seed primes
    ctx->base->h_primes = seed;                            // primes < 2^16 serve as sieving primes
    ctx->base->primes.take(seedp);
    ctx->base->recip.take(seedr);
    const uint64_t nbits = (ctx->L + 1) / 2;
    const uint64_t nwords = ((nbits + 63) / 64) * 2;
    DevBuf bits, popc;
    if ((rc = bits.ensure(nwords * 4)) || (rc = popc.ensure(8)) || (rc = counts.ensure(gb::compact_chunks(nwords) * 4)))
        return rc;
    GB_CUDA(cudaMemsetAsync(popc.p, 0, 8, s));
    if ((rc = run_sieve(ctx, 1, nbits, bits.as<uint32_t>(), popc.as<unsigned long long>()))) return rc;
    unsigned long long nodd = 0;
    GB_CUDA(cudaMemcpyAsync(&nodd, popc.p, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    const uint64_t n = nodd + 1;
    DevBuf np, nr;
    if ((rc = np.ensure(n * 4)) || (rc = nr.ensure(n * 8))) return rc;
    gb::CompactArgs cb{bits.as<uint32_t>(), nwords, 1, counts.as<uint32_t>(), np.as<uint32_t>(), nr.as<uint64_t>()};
    GB_CUDA(gb::launch_compact(cb, s));
    ctx->base->h_primes.resize(n);
    GB_CUDA(cudaMemcpyAsync(ctx->base->h_primes.data(), np.p, n * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    ctx->base->primes.take(np);
    ctx->base->recip.take(nr);
    return GB_OK;
}

}  // namespace

// accessors for entry points in other translation units
namespace gb {
int ctx_view(const gb_ctx* ctx, CtxView* v)
{
    if (!ctx || !v) return fail(GB_EINVAL, "NULL argument");
    v->device = ctx->cfg.device;
    v->stream = ctx->stream;
    v->L = ctx->L;
    v->seg_len = ctx->cfg.seg_len;
    v->p1 = ctx->cfg.p1;
    v->p2 = ctx->cfg.p2;
    v->cta_threads = ctx->cfg.cta_threads;
    v->tile_bits = ctx->cfg.tile_bits;
    v->bucket_split = ctx->cfg.bucket_split;
    v->warp_split = (uint32_t)ctx->warp_split;
    v->primes = ctx->base->primes.as<uint32_t>();
    v->recip = ctx->base->recip.as<uint64_t>();
    v->wheel = ctx->base->wheel.as<uint32_t>();
    v->generic_cover = ctx->generic_cover;
    v->ka_override = (int)ctx->cfg.cover_prefix;
    v->large_chunk_bits = ctx->large_chunk_bits;
    return GB_OK;
}
uint64_t ctx_pi(const gb_ctx* ctx, uint64_t x) { return ctx->pi(x); }
int ctx_sieve(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out) { return run_sieve(ctx, B, nbits, out, nullptr); }
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace gb

namespace {

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

const char* gb_strerror(int code)
{
    switch (code) {
    case GB_OK: return "GB_OK";
    case GB_EINVAL: return "GB_EINVAL: invalid argument";
    case GB_ENOMEM: return "GB_ENOMEM: out of memory";
    case GB_ECUDA: return "GB_ECUDA: CUDA error";
    case GB_ETIMEOUT: return "GB_ETIMEOUT: bounded device wait gave up";
    case GB_EBUSY: return "GB_EBUSY: context busy";
    case GB_ERANGE: return "GB_ERANGE: output buffer too small";
    default: return "unknown gb error";
    }
}

const char* gb_last_error(void) { return g_last_error.c_str(); }

uint64_t gb_bitset_bytes(uint64_t N)
{
    if (N < 3) return 0;
    const uint64_t odd = (N - 1) / 2;               // odd numbers 3 .. N
    return ((odd + 63) / 64) * 8;
}

int gb_init(gb_ctx** out, const gb_config* cfg)
{
    if (!out) return fail(GB_EINVAL, "out is NULL");
    *out = nullptr;
    gb_config c{};
    if (cfg) c = *cfg;
    int rc = fill_defaults(c);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return fail(GB_EINVAL, "no such CUDA device");
    }
    GB_CUDA(cudaSetDevice(c.device));
    gb_ctx* ctx = new gb_ctx();
    ctx->cfg = c;
    ctx->stream = static_cast<cudaStream_t>(c.stream);
    ctx->L = std::max<uint64_t>({c.base_limit, c.p1, c.p2});
    // one warp per sieving prime below 2^10 (at least 32 strikes per lane in a
    // 2^18-bit tile); one thread per larger prime (bank-spread strikes)
    ctx->warp_split = (int)std::min<uint32_t>(1024, c.tile_bits / 64);
    if (const char* e = getenv("GB_WARP_SPLIT")) ctx->warp_split = atoi(e);
    if (const char* e = getenv("GB_COVER")) ctx->generic_cover = std::string(e) == "generic";
    if (const char* e = getenv("GB_BATCH_GRAPH")) ctx->batch_graph = atoi(e) != 0;
    if (const char* e = getenv("GB_LARGE")) ctx->bucket_large = std::string(e) == "bucket";
    if (const char* e = getenv("GB_FUSED")) ctx->fused = atoi(e) != 0;
    if (const char* e = getenv("GB_MID_LOG2")) {
        const int v = atoi(e);
        ctx->mid_limit = (v >= 16 && v <= 31) ? (1u << v) : 0u;
    }
    if (const char* e = getenv("GB_LARGE_CHUNK_LOG2")) {
        const int v = atoi(e);
        if (v >= 16 && v <= 40) ctx->large_chunk_bits = 1ull << v;
    }
    if (const char* e = getenv("GB_KA")) {
        const int v = atoi(e);
        if ((v == 64 || v == 128 || v == 192 || v == 256) && ctx->cfg.cover_prefix == 0) ctx->cfg.cover_prefix = v;
    }
    rc = build_primes(ctx);
    if (rc) {
        gb_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return GB_OK;
}

int gb_init_shared(gb_ctx** out, const gb_ctx* parent, void* stream)
{
    if (!out || !parent) return fail(GB_EINVAL, "NULL argument");
    *out = nullptr;
    GB_CUDA(cudaSetDevice(parent->cfg.device));
    if (parent->stream) GB_CUDA(cudaStreamSynchronize(parent->stream));
    else GB_CUDA(cudaDeviceSynchronize());
    gb_ctx* ctx = new gb_ctx();
    ctx->cfg = parent->cfg;
    ctx->cfg.stream = stream;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->L = parent->L;
    ctx->base = parent->base;
    ctx->warp_split = parent->warp_split;
    ctx->generic_cover = parent->generic_cover;
    ctx->batch_graph = parent->batch_graph;
    ctx->large_chunk_bits = parent->large_chunk_bits;
    ctx->bucket_large = parent->bucket_large;
    ctx->fused = parent->fused;
    ctx->mid_limit = parent->mid_limit;
    *out = ctx;
    return GB_OK;
}

void gb_destroy(gb_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->cfg.device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    // the base primes are shared with the contexts made by gb_init_shared:
    // they are freed with the last context holding them (delete below)
    DevBuf* bufs[] = {&ctx->q, &ctx->hist,
                      &ctx->maxkey, &ctx->maxkey2, &ctx->unres, &ctx->retry, &ctx->retry_count, &ctx->summary,
                      &ctx->rows, &ctx->merged, &ctx->pmin, &ctx->counter, &ctx->totals, &ctx->records, &ctx->work,
                      &ctx->bq, &ctx->bhist, &ctx->bkeys, &ctx->bunres, &ctx->bdesc, &ctx->brecords, &ctx->brows,
                      &ctx->qn, &ctx->qout, &ctx->blists, &ctx->bcounts, &ctx->bflags,
                      &ctx->part_p, &ctx->part_rev, &ctx->part_out};
    for (DevBuf* b : bufs) b->release();
    delete ctx;
}

int gb_get_config(const gb_ctx* ctx, gb_config* out)
{
    if (!ctx || !out) return fail(GB_EINVAL, "NULL argument");
    *out = ctx->cfg;
    return GB_OK;
}

int gb_set_config(gb_ctx* ctx, const gb_config* cfg)
{
    if (!ctx || !cfg) return fail(GB_EINVAL, "NULL argument");
    gb_config c = *cfg;
    int rc = fill_defaults(c);
    if (rc) return rc;
    if (c.device != ctx->cfg.device || c.base_limit != ctx->cfg.base_limit || c.stream != ctx->cfg.stream)
        return fail(GB_EINVAL, "device, base_limit and stream are fixed at gb_init");
    if (std::max(c.p1, c.p2) > ctx->L) return fail(GB_EINVAL, "p1/p2 above the context's base primes");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    if (ctx->stream) GB_CUDA(cudaStreamSynchronize(ctx->stream));
    else GB_CUDA(cudaDeviceSynchronize());
    ctx->cfg = c;
    if (!getenv("GB_WARP_SPLIT")) ctx->warp_split = (int)std::min<uint32_t>(1024, c.tile_bits / 64);
    return GB_OK;
}

int gb_sieve_segment(gb_ctx* ctx, int64_t A_odd, uint64_t n_bits, uint64_t* q_bits, uint64_t* popcount)
{
    if (!ctx || (!q_bits && n_bits)) return fail(GB_EINVAL, "NULL argument");
    if ((A_odd & 1) == 0) return fail(GB_EINVAL, "A_odd must be odd");
    if (n_bits > (1ull << 40)) return fail(GB_EINVAL, "n_bits too large");
    if (A_odd > (int64_t)(1ull << 62) || A_odd < -(int64_t)(1ull << 62))
        return fail(GB_EINVAL, "A_odd out of range");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->counter.ensure(8);
    if (rc) return rc;
    GB_CUDA(cudaMemsetAsync(ctx->counter.p, 0, 8, ctx->stream));
    rc = run_sieve(ctx, A_odd, n_bits, reinterpret_cast<uint32_t*>(q_bits),
                   ctx->counter.as<unsigned long long>());
    if (rc) return rc;
    unsigned long long c = 0;
    GB_CUDA(cudaMemcpyAsync(&c, ctx->counter.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    if (popcount) *popcount = c;
    return GB_OK;
}

int gb_prime_pi(gb_ctx* ctx, uint64_t x, uint64_t* count)
{
    if (!ctx || !count) return fail(GB_EINVAL, "NULL argument");
    *count = 0;
    if (x < 2) return GB_OK;
    if (isqrt_u64(x) > ctx->L) return fail(GB_EINVAL, "x beyond base_limit^2");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->counter.ensure(8);
    if (rc) return rc;
    GB_CUDA(cudaMemsetAsync(ctx->counter.p, 0, 8, ctx->stream));
    const uint64_t total = (x - 1) / 2;             // odd numbers 3 .. x
    const uint64_t chunk = ctx->cfg.slab_bits;
    // primes from bucket_split on strike into a buffer, so sieve into the slab buffer
    const bool need_buf = ctx->pi(isqrt_u64(x)) > ctx->pi(ctx->cfg.bucket_split - 1);
    if (need_buf && (rc = ctx->q.ensure(((std::min(chunk, total) + 63) / 64) * 8))) return rc;
    for (uint64_t done = 0; done < total; done += chunk) {
        const uint64_t nb = std::min(chunk, total - done);
        rc = run_sieve(ctx, 3 + 2 * (int64_t)done, nb, need_buf ? ctx->q.as<uint32_t>() : nullptr,
                       ctx->counter.as<unsigned long long>());
        if (rc) return rc;
    }
    unsigned long long c = 0;
    GB_CUDA(cudaMemcpyAsync(&c, ctx->counter.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    *count = c + 1;                                 // + the prime 2
    return GB_OK;
}

int gb_verify_range(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t P, gb_range_result* out)
{
    if (!ctx || !out) return fail(GB_EINVAL, "NULL argument");
    if ((lo & 1) || (hi & 1) || lo < 4 || hi <= lo) return fail(GB_EINVAL, "range must be even, lo >= 4, hi > lo");
    if (hi > (1ull << 63)) return fail(GB_EINVAL, "hi beyond 2^63");
    const gb_config& cfg = ctx->cfg;
    const uint32_t P1 = P ? P : cfg.p1;
    if (P1 < 2 || P1 > (1u << 24) || P1 > ctx->L) return fail(GB_EINVAL, "P out of range (2 .. min(2^24, base list))");
    const bool retry = cfg.p2 > P1;
    const uint32_t Pf = retry ? cfg.p2 : P1;
    const uint32_t K1 = (uint32_t)(ctx->pi(P1) - 1);      // odd primes <= P1
    const uint32_t Kf = (uint32_t)(ctx->pi(Pf) - 1);
    // halo: larger than every p of both passes, and H = 4 (mod 64) so that the
    // partner bits of p = 3 start on a 32-bit word boundary (two-phase cover)
    const uint32_t H = 64 * ((Pf + 1 - 4 + 63) / 64) + 4;
    const uint64_t S = cfg.seg_len;
    const uint64_t n_total = (hi - lo) / 2;
    const uint64_t nseg = (n_total + S - 1) / S;
    if (nseg > 0xffffffffull) return fail(GB_EINVAL, "too many segments");
    const uint64_t last_num = hi + 2 * 1024 + H;          // generous bound of the sieve window
    if (isqrt_u64(last_num) > ctx->L) return fail(GB_EINVAL, "hi beyond base_limit^2");
    const uint32_t hist_stride = Kf + 1;
    const uint64_t spb = std::max<uint64_t>(1, cfg.slab_bits / S);   // segments per slab
    GB_CUDA(cudaSetDevice(cfg.device));
    cudaStream_t s = ctx->stream;

    // where each output goes: caller device buffers are written in place,
    // host buffers through device staging and one copy at the end
    const bool want_rows = out->seg_hist && out->seg_hist_stride;
    const uint32_t row_stride = want_rows ? out->seg_hist_stride : 0;
    const uint64_t rows_n = want_rows ? (out->seg_cap ? std::min<uint64_t>(out->seg_cap, nseg) : nseg) : 0;
    const bool rows_dev = want_rows && is_device_ptr(out->seg_hist);
    const bool segs_dev = out->segs && is_device_ptr(out->segs);
    const bool pmin_dev = out->pmin && is_device_ptr(out->pmin);
    int rc;
    if ((rc = ctx->summary.ensure(nseg * sizeof(gb::SegSummary))) ||
        (rc = ctx->merged.ensure((size_t)hist_stride * 8)) ||
        (rc = ctx->totals.ensure(sizeof(gb::RangeTotals))) ||
        (want_rows && !rows_dev && (rc = ctx->rows.ensure(std::max<uint64_t>(1, nseg * row_stride) * 8))) ||
        (out->segs && !segs_dev && (rc = ctx->records.ensure(nseg * sizeof(gb::SegRecord)))))
        return rc;
    GB_CUDA(cudaMemsetAsync(ctx->merged.p, 0, (size_t)hist_stride * 8, s));
    uint64_t* rows_base = want_rows ? (rows_dev ? out->seg_hist : ctx->rows.as<uint64_t>()) : nullptr;

    // per-slab buffers
    const uint64_t slab_n = std::min<uint64_t>(spb * S, n_total);
    const uint64_t slab_words = (slab_n + 63) / 64;
    const uint64_t slab_segs = std::min<uint64_t>(spb, nseg);
    const uint64_t q_words = slab_words + H / 128 + 2;
    const uint32_t retry_cap = (uint32_t)std::min<uint64_t>(slab_words, 1u << 21);
    if ((rc = ctx->q.ensure(q_words * 8)) ||
        (rc = ctx->hist.ensure(slab_segs * hist_stride * 4)) ||
        (rc = ctx->maxkey.ensure(slab_segs * 8)) || (rc = ctx->maxkey2.ensure(slab_segs * 8)) ||
        (rc = ctx->unres.ensure(slab_segs * 8)) ||
        (retry && (rc = ctx->retry.ensure((size_t)retry_cap * sizeof(gb::RetryItem)))) ||
        (rc = ctx->retry_count.ensure(16)) ||
        (out->pmin && !pmin_dev && (rc = ctx->pmin.ensure(slab_n * 4))))
        return rc;

    unsigned int overflow_total = 0;
    for (uint64_t s0 = 0; s0 < nseg; s0 += spb) {
        const uint64_t ns = std::min<uint64_t>(spb, nseg - s0);
        const uint64_t A0 = lo + 2 * s0 * S;
        const uint64_t n_count = std::min<uint64_t>(ns * S, n_total - s0 * S);
        const uint64_t n_words = (n_count + 63) / 64;
        const uint64_t qw = n_words + H / 128 + 2;
        const int64_t B = (int64_t)A0 - (int64_t)H + 1;

        GB_CUDA(cudaMemsetAsync(ctx->hist.p, 0, ns * hist_stride * 4, s));
        GB_CUDA(cudaMemsetAsync(ctx->maxkey.p, 0, ns * 8, s));
        GB_CUDA(cudaMemsetAsync(ctx->maxkey2.p, 0, ns * 8, s));
        GB_CUDA(cudaMemsetAsync(ctx->unres.p, 0, ns * 8, s));
        GB_CUDA(cudaMemsetAsync(ctx->retry_count.p, 0, 16, s));
        uint32_t* pm = nullptr;
        if (out->pmin) {
            pm = pmin_dev ? out->pmin + (s0 * S) : ctx->pmin.as<uint32_t>();
            GB_CUDA(cudaMemsetAsync(pm, 0, n_count * 4, s));
        }

        gb::CoverArgs ca{};
        ca.Q = ctx->q.as<uint64_t>();
        ca.H = H;
        ca.n_count = n_count;
        ca.n_words = n_words;
        ca.words_per_seg = (uint32_t)(S / 64);
        ca.cta_words = std::min<uint32_t>(2048, (uint32_t)(S / 64));
        ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
        ca.nseg = (uint32_t)ns;
        ca.primes = ctx->base->primes.as<uint32_t>();
        ca.K = K1;
        ca.hist_stride = hist_stride;
        ca.hist = ctx->hist.as<uint32_t>();
        ca.maxkey = ctx->maxkey.as<unsigned long long>();
        ca.unresolved = ctx->unres.as<unsigned long long>();
        ca.pmin = pm;
        ca.retry = retry ? ctx->retry.as<gb::RetryItem>() : nullptr;
        ca.retry_count = retry ? ctx->retry_count.as<unsigned int>() : nullptr;
        ca.retry_cap = retry_cap;
        ca.has_n4 = (A0 == 4);
        ca.iters = ctx->work_ptr(1);
        // two-phase kernel unless a p_min array is wanted (the generic kernel
        // writes it) or the pass has too few primes for its first phase
        int KA = (pm || ctx->generic_cover || cfg.cover_prefix == 1) ? 0 : gb::cover_fast_phase_primes(K1, A0 + 2 * n_count);
        if (KA && cfg.cover_prefix > 1 && cfg.cover_prefix <= K1) KA = (int)cfg.cover_prefix;
        if (KA) {
            // block cover: 7680 32-bit words per CTA (ten rounds of 96 words per
            // warp, the most its 10-bit counters allow)
            ca.cta_words = std::min<uint32_t>(3840, (uint32_t)(S / 64));
            ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
        }
        // fused sieve + cover (GB_FUSED=1): block cover, no large primes, the
        // chunk plus its partner halo within one shared-memory tile
        bool fused = false;
        gb::SieveArgs fsv{};
        const uint32_t P1max = ctx->base->h_primes[K1];           // largest prime of the first pass
        if (ctx->fused && KA &&
            (2ull * ca.cta_words + (H - 4) / 64 + 3 - gb::seg_cover_offset(H, P1max)) * 32 <= gb::kFusedTileBits) {
            uint64_t np = 0, nsmall = 0;
            if ((rc = tile_sieve_args(ctx, B, qw * 64, fsv, np, nsmall))) return rc;
            fused = np <= nsmall;
            fsv.tile_bits = gb::kFusedTileBits;
        }
        bool q_in_hbm = false;
        if (!fused) {
            if ((rc = run_sieve(ctx, B, qw * 64, ctx->q.as<uint32_t>(), nullptr))) return rc;
            q_in_hbm = true;
        }
        ctx->prof_begin(kProfCover, n_count);
        if (fused) GB_LAUNCH(gb::launch_seg_cover(ca, fsv, KA, P1max, s));
        else if (KA) GB_LAUNCH(gb::launch_cover_fast(ca, KA, s));
        else GB_LAUNCH(gb::launch_cover(ca, (int)cfg.cta_threads, s));
        ctx->prof_end();

        if (retry && fused) {
            // the retry pass reads Q from global memory: sieve the slab there
            // only if some word was left open
            unsigned int cnt = 0;
            GB_CUDA(cudaMemcpyAsync(&cnt, ctx->retry_count.p, 4, cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
            if (cnt) {
                if ((rc = run_sieve(ctx, B, qw * 64, ctx->q.as<uint32_t>(), nullptr))) return rc;
                q_in_hbm = true;
            }
        }
        if (retry && q_in_hbm) {
            gb::RetryArgs ra{};
            ra.Q = ca.Q;
            ra.H = H;
            ra.words_per_seg = ca.words_per_seg;
            ra.primes = ca.primes;
            ra.K1 = K1;
            ra.K2 = Kf;
            ra.hist_stride = hist_stride;
            ra.hist = ca.hist;
            ra.maxkey = ca.maxkey;
            ra.unresolved = ca.unresolved;
            ra.pmin = pm;
            ra.items = ca.retry;
            ra.count = ca.retry_count;
            ra.cap = retry_cap;
            ctx->prof_begin(kProfRetry, n_count);
            GB_LAUNCH(gb::launch_retry(ra, s));
            ctx->prof_end();
        }

        gb::ReduceArgs rd{};
        rd.nseg = (uint32_t)ns;
        rd.maxkey2 = nullptr;
        rd.hist_stride = hist_stride;
        rd.hist = ca.hist;
        rd.maxkey = ca.maxkey;
        rd.unresolved = ca.unresolved;
        rd.primes = ca.primes;
        rd.summary = ctx->summary.as<gb::SegSummary>() + s0;
        rd.rows = (want_rows && s0 < rows_n) ? rows_base + s0 * row_stride : nullptr;
        rd.row_stride = row_stride;
        rd.nrows = (uint32_t)(want_rows ? std::min<uint64_t>(ns, rows_n > s0 ? rows_n - s0 : 0) : 0);
        rd.merged = ctx->merged.as<unsigned long long>();
        ctx->prof_begin(kProfReduce, ns);
        GB_LAUNCH(gb::launch_reduce(rd, s));
        ctx->prof_end();

        if (retry) {
            unsigned int cnt = 0;
            GB_CUDA(cudaMemcpyAsync(&cnt, ctx->retry_count.p, 4, cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
            if (cnt > retry_cap) overflow_total += cnt - retry_cap;
        }
        if (out->pmin && !pmin_dev)
            GB_CUDA(cudaMemcpyAsync(out->pmin + s0 * S, pm, n_count * 4, cudaMemcpyDeviceToHost, s));
    }
    if (overflow_total) {
        // the retry list could not hold every word left open: redo in one pass to Pf
        gb_range_result again = *out;
        const uint32_t saved_p2 = ctx->cfg.p2;
        ctx->cfg.p2 = 0;
        rc = gb_verify_range(ctx, lo, hi, Pf, &again);
        ctx->cfg.p2 = saved_p2;
        if (rc && rc != GB_ERANGE) return rc;
        again.p_final = Pf;
        *out = again;
        return rc;
    }

    gb::FinalizeArgs fa{};
    fa.lo = lo;
    fa.hi = hi;
    fa.S = S;
    fa.nseg = (uint32_t)nseg;
    fa.summary = ctx->summary.as<gb::SegSummary>();
    fa.records = out->segs ? (segs_dev ? reinterpret_cast<gb::SegRecord*>(out->segs) : ctx->records.as<gb::SegRecord>())
                           : nullptr;
    fa.nrecords = (uint32_t)(out->segs ? std::min<uint64_t>(out->seg_cap, nseg) : 0);
    fa.totals = ctx->totals.as<gb::RangeTotals>();
    ctx->prof_begin(kProfReduce, nseg);
    GB_LAUNCH(gb::launch_finalize(fa, s));
    ctx->prof_end();

    gb::RangeTotals tot{};
    GB_CUDA(cudaMemcpyAsync(&tot, ctx->totals.p, sizeof tot, cudaMemcpyDeviceToHost, s));
    const uint32_t nh = out->hist ? std::min<uint32_t>(out->hist_cap, hist_stride) : 0;
    if (nh) GB_CUDA(cudaMemcpyAsync(out->hist, ctx->merged.p, (size_t)nh * 8, cudaMemcpyDeviceToHost, s));
    const uint64_t nrec = out->segs ? std::min<uint64_t>(out->seg_cap, nseg) : 0;
    if (nrec && !segs_dev)
        GB_CUDA(cudaMemcpyAsync(out->segs, ctx->records.p, nrec * sizeof(gb::SegRecord), cudaMemcpyDeviceToHost, s));
    if (rows_n && !rows_dev)
        GB_CUDA(cudaMemcpyAsync(out->seg_hist, ctx->rows.p, rows_n * row_stride * 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (out->hist) for (uint32_t i = nh; i < out->hist_cap; ++i) out->hist[i] = 0;

    out->n_checked = n_total;
    out->n_segments = (uint32_t)nseg;
    out->p_final = Pf;
    out->unresolved = tot.unresolved;
    out->max_pmin = tot.max_pmin;
    out->max_pmin_n = tot.max_pmin_n;
    out->hist_len = tot.hist_len;

    // a segment histogram longer than the caller's row stride was truncated
    bool erange = (out->segs && out->seg_cap < nseg) || (want_rows && rows_n < nseg) ||
                  (out->hist && out->hist_cap < out->hist_len);
    if (want_rows && !erange && row_stride < hist_stride) {
        if (out->segs && !segs_dev) {
            for (uint64_t k = 0; k < nrec && !erange; ++k) erange = out->segs[k].hist_len > row_stride;
        } else {
            erange = tot.hist_len > row_stride;            // the longest row is the range maximum's
        }
    }
    if (erange) return fail(GB_ERANGE, "an output buffer was too small; what fit was written");
    return GB_OK;
}

int gb_verify_batch(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, uint32_t P,
                    gb_segment_result* results, uint64_t* hist, uint32_t hist_stride)
{
    if (!ctx || (count && (!lo || !hi || !results))) return fail(GB_EINVAL, "NULL argument");
    if (count == 0) return GB_OK;
    if (count > (1u << 24)) return fail(GB_EINVAL, "count above 2^24");
    const gb_config& cfg = ctx->cfg;
    const uint32_t P1 = P ? P : cfg.p1;
    if (P1 < 2 || P1 > (1u << 24) || P1 > ctx->L) return fail(GB_EINVAL, "P out of range (2 .. min(2^24, base list))");
    const uint32_t K1 = (uint32_t)(ctx->pi(P1) - 1);
    const uint32_t H = 64 * ((P1 + 1 - 4 + 63) / 64) + 4;     // first-pass halo
    const uint32_t hs = K1 + 1;                               // device histogram row
    const uint32_t T = cfg.tile_bits;
    const uint32_t cw = 3840;                                 // block-cover CTA chunk (64-bit words)
    GB_CUDA(cudaSetDevice(cfg.device));
    cudaStream_t s = ctx->stream;

    // per-range windows and work items
    uint64_t qwords = 0, n_sieve = 0, n_cover = 0, hi_max = 0, last_max = 0;
    for (uint32_t i = 0; i < count; ++i) {
        if ((lo[i] & 1) || (hi[i] & 1) || lo[i] < 4 || hi[i] <= lo[i] || hi[i] > (1ull << 63))
            return fail(GB_EINVAL, "range must be even, lo >= 4, hi > lo");
        const uint64_t n = (hi[i] - lo[i]) / 2;
        if (n > (1ull << 32)) return fail(GB_EINVAL, "a batch range holds at most 2^32 even n");
        const uint64_t qw = (n + 63) / 64 + H / 128 + 2;
        qwords += qw;
        n_sieve += (64 * qw + T - 1) / T;
        n_cover += (((n + 31) / 32) + 2ull * cw - 1) / (2ull * cw);
        hi_max = std::max(hi_max, hi[i]);
        last_max = std::max(last_max, lo[i] - H + 1 + 2 * (64 * qw - 1));   // window's last number
    }
    if (isqrt_u64(last_max) > ctx->L) return fail(GB_EINVAL, "hi beyond base_limit^2");
    if (n_sieve > 0xffffffffull || n_cover > 0xffffffffull) return fail(GB_EINVAL, "batch too large");

    // large primes: np primes <= sqrt of the batch's last number; those below
    // the split strike per tile, those below the mid limit per 2^20-bit slice
    // of each window in shared memory, the rest per window piece by atomics
    const uint64_t np = ctx->pi(isqrt_u64(last_max));
    const uint64_t nsmall = std::min<uint64_t>(np, std::max<uint64_t>(ctx->pi(cfg.bucket_split - 1), gb::kFirstStrikeIdx));
    const uint64_t nmid = ctx->mid_limit > cfg.bucket_split
                              ? std::min<uint64_t>(np, std::max<uint64_t>(nsmall, ctx->pi(ctx->mid_limit - 1)))
                              : nsmall;
    uint64_t n_mid = 0;
    if (nmid > nsmall)
        for (uint32_t i = 0; i < count; ++i) {
            const uint64_t qw = (hi[i] - lo[i]) / 2 / 64 + 1 + H / 128 + 2;
            n_mid += (64 * qw + (1ull << gb::kMidSliceLog2) - 1) >> gb::kMidSliceLog2;
        }
    if (n_mid > 0xffffffffull) return fail(GB_EINVAL, "batch too large");
    // window pieces of at most one L2-sized chunk, grouped up to a chunk;
    // within a group by their prime counts, descending
    std::vector<gb::LargePiece> pieces;
    std::vector<uint32_t> groups;
    uint32_t nblk = 0;
    if (np > nmid) {
        const uint64_t chunk = ctx->large_chunk_bits;
        uint64_t acc = 0;
        uint32_t most = 0;
        groups.push_back(0);
        for (uint32_t i = 0; i < count; ++i) {
            const uint64_t nb = 64 * ((hi[i] - lo[i]) / 2 / 64 + (((hi[i] - lo[i]) / 2) % 64 ? 1 : 0) + H / 128 + 2);
            const int64_t Bi = (int64_t)lo[i] - (int64_t)H + 1;
            for (uint64_t b0 = 0; b0 < nb; b0 += chunk) {
                const uint64_t b1 = std::min(nb, b0 + chunk);
                const int64_t lastn = Bi + 2 * (int64_t)(b1 - 1);
                const uint64_t npc = lastn > 0 ? ctx->pi(isqrt_u64((uint64_t)lastn)) : 0;
                const uint32_t nl = npc > nmid ? (uint32_t)(npc - nmid) : 0u;
                if (!nl) continue;
                if (acc && acc + (b1 - b0) > chunk) {
                    groups.push_back((uint32_t)pieces.size());
                    acc = 0;
                }
                pieces.push_back(gb::LargePiece{i, nl, b0, b1});
                acc += b1 - b0;
                most = std::max(most, nl);
            }
        }
        groups.push_back((uint32_t)pieces.size());
        for (size_t g = 0; g + 1 < groups.size(); ++g)
            std::stable_sort(pieces.begin() + groups[g], pieces.begin() + groups[g + 1],
                             [](const gb::LargePiece& x, const gb::LargePiece& y) { return x.n_primes > y.n_primes; });
        nblk = (most + 255) / 256;
    }
    const uint64_t n_pieces = pieces.size();
    const uint32_t n_groups = groups.empty() ? 0u : (uint32_t)groups.size() - 1;
    const uint64_t n_large_items = (uint64_t)n_groups * nblk;
    if (n_large_items > 0xffffffffull) return fail(GB_EINVAL, "batch too large");

    // device buffers
    const size_t desc_ranges = (size_t)count * sizeof(gb::BatchRange) + n_pieces * sizeof(gb::LargePiece);
    const size_t desc_bytes = desc_ranges + (size_t)(2 * n_sieve + 2 * n_cover + 2 * n_mid) * 4 +
                              (size_t)(n_groups + 1) * 4 + 64;
    const bool want_rows = hist && hist_stride;
    const bool res_dev = is_device_ptr(results);
    const bool rows_dev = want_rows && is_device_ptr(hist);
    int rc;
    if ((rc = ctx->bq.ensure(qwords * 8)) || (rc = ctx->bhist.ensure((size_t)count * hs * 4)) ||
        (rc = ctx->bkeys.ensure((size_t)count * 8)) || (rc = ctx->bunres.ensure((size_t)count * 8)) ||
        (rc = ctx->bdesc.ensure(desc_bytes)) || (rc = ctx->hstage.ensure(desc_bytes)) ||
        (!res_dev && (rc = ctx->brecords.ensure((size_t)count * sizeof(gb::SegRecord)))) ||
        (want_rows && !rows_dev && (rc = ctx->brows.ensure((size_t)count * hist_stride * 8))) ||
        (rc = ctx->counter.ensure(16)))
        return rc;

    // descriptors, staged in pinned memory: ranges | pieces | sieve items |
    // cover items | piece groups | mid items | counts
    unsigned char* hs_p = static_cast<unsigned char*>(ctx->hstage.p);
    gb::BatchRange* hr = reinterpret_cast<gb::BatchRange*>(hs_p);
    gb::LargePiece* hpc = reinterpret_cast<gb::LargePiece*>(hs_p + (size_t)count * sizeof(gb::BatchRange));
    std::memcpy(hpc, pieces.data(), n_pieces * sizeof(gb::LargePiece));
    uint32_t* s_range = reinterpret_cast<uint32_t*>(hs_p + desc_ranges);
    uint32_t* s_tile = s_range + n_sieve;
    uint32_t* c_range = s_tile + n_sieve;
    uint32_t* c_chunk = c_range + n_cover;
    uint32_t* g_first = c_chunk + n_cover;
    uint32_t* m_range = g_first + n_groups + 1;
    uint32_t* m_slice = m_range + n_mid;
    // [0] sieve items, [1] cover items, [2] ranges, [3] large-prime items, [4] mid items
    uint32_t* counts = m_slice + n_mid;
    {
        uint64_t off = 0, si = 0, ci = 0, mi = 0;
        for (uint32_t i = 0; i < count; ++i) {
            const uint64_t n = (hi[i] - lo[i]) / 2;
            const uint64_t qw = (n + 63) / 64 + H / 128 + 2;
            hr[i].lo = lo[i];
            hr[i].n = n;
            hr[i].B = (int64_t)lo[i] - (int64_t)H + 1;
            hr[i].nbits = 64 * qw;
            hr[i].q_off = off;
            off += qw;
            const uint64_t tiles = (64 * qw + T - 1) / T;
            for (uint64_t t = 0; t < tiles; ++t) { s_range[si] = i; s_tile[si] = (uint32_t)t; ++si; }
            const uint64_t chunks = (((n + 31) / 32) + 2ull * cw - 1) / (2ull * cw);
            for (uint64_t c = 0; c < chunks; ++c) { c_range[ci] = i; c_chunk[ci] = (uint32_t)c; ++ci; }
            if (n_mid) {
                const uint64_t slices = (64 * qw + (1ull << gb::kMidSliceLog2) - 1) >> gb::kMidSliceLog2;
                for (uint64_t t = 0; t < slices; ++t) { m_range[mi] = i; m_slice[mi] = (uint32_t)t; ++mi; }
            }
        }
        counts[0] = (uint32_t)n_sieve;
        counts[1] = (uint32_t)n_cover;
        counts[2] = count;
        for (uint32_t g = 0; g < n_groups + (n_groups ? 1u : 0u); ++g) g_first[g] = groups[g];
        counts[3] = (uint32_t)n_large_items;
        counts[4] = (uint32_t)mi;
    }
    unsigned char* dd = static_cast<unsigned char*>(ctx->bdesc.p);
    const size_t used = reinterpret_cast<unsigned char*>(counts + 5) - hs_p;
    GB_CUDA(cudaMemcpyAsync(dd, hs_p, used, cudaMemcpyHostToDevice, s));
    const gb::BatchRange* d_ranges = reinterpret_cast<const gb::BatchRange*>(dd);
    const gb::LargePiece* d_pieces = reinterpret_cast<const gb::LargePiece*>(dd + (size_t)count * sizeof(gb::BatchRange));
    const uint32_t* d_s_range = reinterpret_cast<const uint32_t*>(dd + desc_ranges);
    const uint32_t* d_s_tile = d_s_range + n_sieve;
    const uint32_t* d_c_range = d_s_tile + n_sieve;
    const uint32_t* d_c_chunk = d_c_range + n_cover;
    const uint32_t* d_groups = d_c_chunk + n_cover;
    const uint32_t* d_m_range = d_groups + n_groups + 1;
    const uint32_t* d_m_slice = d_m_range + n_mid;
    const uint32_t* d_counts = d_m_slice + n_mid;

    unsigned int* heads = ctx->counter.as<unsigned int>();
    GB_CUDA(cudaMemsetAsync(heads, 0, 16, s));
    GB_CUDA(cudaMemsetAsync(ctx->bhist.p, 0, (size_t)count * hs * 4, s));
    GB_CUDA(cudaMemsetAsync(ctx->bkeys.p, 0, (size_t)count * 8, s));
    GB_CUDA(cudaMemsetAsync(ctx->bunres.p, 0, (size_t)count * 8, s));

    // block-cover length (unrolled primes) for the batch's largest n
    int KA = ctx->generic_cover ? 0 : gb::cover_fast_phase_primes(K1, hi_max);
    if (KA && cfg.cover_prefix > 1 && cfg.cover_prefix <= K1) KA = (int)cfg.cover_prefix;
    if (!KA) return fail(GB_EINVAL, "gb_verify_batch needs P >= the 64th odd prime (313)");

    // the kernels of the batch, captured as one CUDA graph (re-used by update
    // while the sequence keeps its shape) or launched one by one
    // (captured on a private stream -- the caller's may be the legacy default
    // stream, which cannot be captured -- and launched on the caller's)
    const bool graph = ctx->batch_graph;
    cudaStream_t ls = s;
    if (graph) {
        if (!ctx->cap_stream) GB_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        ls = ctx->cap_stream;
        GB_CUDA(cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
    }
    gb::SegRecord* d_records = res_dev ? reinterpret_cast<gb::SegRecord*>(results) : ctx->brecords.as<gb::SegRecord>();
    int lrc = GB_OK;
    auto launches = [&]() -> int {
        // sieve: tile part (persistent, item queue), then the large primes
        gb::SieveItemsArgs sa{};
        sa.base.tile_bits = T;
        sa.base.primes = ctx->base->primes.as<uint32_t>() + gb::kFirstStrikeIdx;
        sa.base.recip = ctx->base->recip.as<uint64_t>() + gb::kFirstStrikeIdx;
        const uint64_t nstrike = nsmall > gb::kFirstStrikeIdx ? nsmall - gb::kFirstStrikeIdx : 0;
        const uint64_t nwarp_all = ctx->pi((uint64_t)ctx->warp_split - 1);
        sa.base.n_warp = (uint32_t)std::min<uint64_t>(nstrike, nwarp_all > gb::kFirstStrikeIdx ? nwarp_all - gb::kFirstStrikeIdx : 0);
        sa.base.n_primes = (uint32_t)nstrike;
        sa.base.wheel = ctx->base->wheel.as<uint32_t>();
        sa.base.strikes = ctx->work_ptr(0);
        sa.ranges = d_ranges;
        sa.item_range = d_s_range;
        sa.item_tile = d_s_tile;
        sa.n_items = d_counts + 0;
        sa.head = heads + 0;
        sa.Q = ctx->bq.as<uint32_t>();
        ctx->prof_begin(kProfSieve, qwords * 64);
        GB_LAUNCH(gb::launch_sieve_items(sa, (int)cfg.cta_threads, ls));
        {
            gb::LargeBatchArgs la{};
            la.ranges = d_ranges;
            la.pieces = d_pieces;
            la.groups = d_groups;
            la.nblk = nblk;
            la.n_items = d_counts + 3;
            la.head = heads + 2;
            la.primes = ctx->base->primes.as<uint32_t>() + nmid;
            la.recip = ctx->base->recip.as<uint64_t>() + nmid;
            la.n_primes = (uint32_t)(np - nmid);
            la.Q = ctx->bq.as<uint32_t>();
            la.strikes = ctx->work_ptr(2);
            ctx->prof_end();
            ctx->prof_begin(kProfLarge, qwords * 64);
            if (nmid > nsmall) {
                gb::MidItemsArgs ma{};
                ma.ranges = d_ranges;
                ma.item_range = d_m_range;
                ma.item_slice = d_m_slice;
                ma.n_items = d_counts + 4;
                ma.head = heads + 3;
                ma.primes = ctx->base->primes.as<uint32_t>() + nsmall;
                ma.recip = ctx->base->recip.as<uint64_t>() + nsmall;
                ma.n_primes = (uint32_t)(nmid - nsmall);
                ma.Q = ctx->bq.as<uint32_t>();
                ma.strikes = ctx->work_ptr(2);
                GB_LAUNCH(gb::launch_mid_items(ma, ls));
            }
            if (n_pieces) GB_LAUNCH(gb::launch_large_batch(la, ls));
        }
        ctx->prof_end();

        // cover: persistent, item queue; row r = range r; no retry here (open
        // ranges are redone below)
        gb::CoverItemsArgs cv{};
        cv.base.H = H;
        cv.base.cta_words = cw;
        cv.base.primes = ctx->base->primes.as<uint32_t>();
        cv.base.K = K1;
        cv.base.hist_stride = hs;
        cv.base.hist = ctx->bhist.as<uint32_t>();
        cv.base.maxkey = ctx->bkeys.as<unsigned long long>();
        cv.base.unresolved = ctx->bunres.as<unsigned long long>();
        cv.base.iters = ctx->work_ptr(1);
        cv.ranges = d_ranges;
        cv.item_range = d_c_range;
        cv.item_chunk = d_c_chunk;
        cv.n_items = d_counts + 1;
        cv.head = heads + 1;
        cv.Q = ctx->bq.as<uint64_t>();
        ctx->prof_begin(kProfCover, qwords * 64);
        GB_LAUNCH(gb::launch_cover_items(cv, KA, ls));
        ctx->prof_end();

        gb::ReduceBatchArgs ra{};
        ra.ranges = d_ranges;
        ra.count = d_counts + 2;
        ra.hist = ctx->bhist.as<uint32_t>();
        ra.hist_stride = hs;
        ra.maxkey = ctx->bkeys.as<unsigned long long>();
        ra.unresolved = ctx->bunres.as<unsigned long long>();
        ra.primes = ctx->base->primes.as<uint32_t>();
        ra.records = d_records;
        ra.rows = want_rows ? (rows_dev ? hist : ctx->brows.as<uint64_t>()) : nullptr;
        ra.row_stride = want_rows ? hist_stride : 0;
        ctx->prof_begin(kProfReduce, count);
        GB_LAUNCH(gb::launch_reduce_batch(ra, count, ls));
        ctx->prof_end();
        return GB_OK;
    };
    lrc = launches();
    if (graph) {
        ctx->capturing = false;
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ls, &g);
        if (lrc) {
            if (g) cudaGraphDestroy(g);
            return lrc;
        }
        if (ce != cudaSuccess) return fail(GB_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
        bool updated = false;
        if (ctx->bgraph) {
            cudaGraphExecUpdateResultInfo info{};
            updated = cudaGraphExecUpdate(ctx->bgraph, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(ctx->bgraph);
                ctx->bgraph = nullptr;
            }
        }
        cudaError_t ie = cudaSuccess;
        if (!updated) ie = cudaGraphInstantiate(&ctx->bgraph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            ctx->bgraph = nullptr;
            return fail(GB_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
        }
        GB_CUDA(cudaGraphLaunch(ctx->bgraph, s));
    } else if (lrc) {
        return lrc;
    }

    // results to the caller; ranges with open n are redone with the retry pass
    std::vector<gb::SegRecord> rec(count);
    GB_CUDA(cudaMemcpyAsync(rec.data(), d_records, (size_t)count * sizeof(gb::SegRecord), cudaMemcpyDeviceToHost, s));
    if (want_rows && !rows_dev)
        GB_CUDA(cudaMemcpyAsync(hist, ctx->brows.p, (size_t)count * hist_stride * 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    int status = GB_OK;
    for (uint32_t i = 0; i < count; ++i) {
        gb::SegRecord& r = rec[i];
        if (r.unresolved && cfg.p2 > P1) {
            // the range's totals and histogram from the plain path (retry pass included)
            gb_range_result one{};
            std::vector<uint64_t> row(want_rows ? hist_stride : 0);
            if (want_rows) {
                one.hist = row.data();
                one.hist_cap = hist_stride;
            }
            rc = gb_verify_range(ctx, r.lo, r.hi, P1, &one);
            if (rc && rc != GB_ERANGE) return rc;
            r.unresolved = one.unresolved;
            r.max_pmin = one.max_pmin;
            r.max_pmin_n = one.max_pmin_n;
            r.hist_len = one.hist_len;
            if (res_dev)
                GB_CUDA(cudaMemcpy(reinterpret_cast<gb::SegRecord*>(results) + i, &r, sizeof r, cudaMemcpyHostToDevice));
            if (want_rows) {
                if (rows_dev)
                    GB_CUDA(cudaMemcpy(hist + (uint64_t)i * hist_stride, row.data(), (size_t)hist_stride * 8,
                                       cudaMemcpyHostToDevice));
                else
                    std::memcpy(hist + (uint64_t)i * hist_stride, row.data(), (size_t)hist_stride * 8);
            }
        }
        if (want_rows && r.hist_len > hist_stride) status = GB_ERANGE;
    }
    if (!res_dev) std::memcpy(results, rec.data(), (size_t)count * sizeof(gb::SegRecord));
    if (status == GB_ERANGE) return fail(GB_ERANGE, "a histogram row was longer than hist_stride");
    return GB_OK;
}

int gb_query_batch(gb_ctx* ctx, const uint64_t* n, uint32_t count, uint32_t P, uint32_t* p_min)
{
    if (!ctx || (count && (!n || !p_min))) return fail(GB_EINVAL, "NULL argument");
    if (count == 0) return GB_OK;
    const gb_config& cfg = ctx->cfg;
    const uint32_t Pq = P ? P : std::max(cfg.p1, cfg.p2);
    if (Pq < 3 || Pq > ctx->L) return fail(GB_EINVAL, "P must be in [3, base primes]");
    if (ctx->L < gb::query_filter_max()) return fail(GB_EINVAL, "queries need base primes to 2048");
    GB_CUDA(cudaSetDevice(cfg.device));
    cudaStream_t s = ctx->stream;
    const bool n_dev = is_device_ptr(n), out_dev = is_device_ptr(p_min);
    if (!n_dev)
        for (uint32_t i = 0; i < count; ++i)
            if ((n[i] & 1) || n[i] < 4 || n[i] >= (1ull << 63)) return fail(GB_EINVAL, "n must be even, 4 <= n < 2^63");
    int rc;
    if ((!n_dev && (rc = ctx->qn.ensure((size_t)count * 8))) || (rc = ctx->qout.ensure((size_t)count * 4 + 16)))
        return rc;
    const uint64_t* d_n = n;
    if (!n_dev) {
        GB_CUDA(cudaMemcpyAsync(ctx->qn.p, n, (size_t)count * 8, cudaMemcpyHostToDevice, s));
        d_n = ctx->qn.as<uint64_t>();
    }
    unsigned int* bad = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(ctx->qout.p) + (size_t)count * 4);
    GB_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    gb::QueryArgs qa{};
    qa.n = d_n;
    qa.count = count;
    qa.primes = ctx->base->primes.as<uint32_t>();
    qa.recip = ctx->base->recip.as<uint64_t>();
    qa.n_filter = (uint32_t)(ctx->pi(gb::query_filter_max()) - 1);
    qa.K = (uint32_t)(ctx->pi(Pq) - 1);
    qa.out = out_dev ? p_min : ctx->qout.as<uint32_t>();
    qa.bad = bad;
    GB_LAUNCH(gb::launch_query(qa, s));
    unsigned int h_bad = 0;
    GB_CUDA(cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, s));
    if (!out_dev) GB_CUDA(cudaMemcpyAsync(p_min, qa.out, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (h_bad) return fail(GB_EINVAL, "n must be even, 4 <= n < 2^63 (device input)");
    return GB_OK;
}

int gb_partitions(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t* counts)
{
    if (!ctx || (hi > lo && !counts)) return fail(GB_EINVAL, "NULL argument");
    if ((lo & 1) || (hi & 1) || lo < 4 || hi < lo) return fail(GB_EINVAL, "range must be even, lo >= 4, hi >= lo");
    if (hi > (1ull << 34)) return fail(GB_EINVAL, "partition counts need hi <= 2^34");
    const uint64_t count = (hi - lo) / 2;
    if (count == 0) return GB_OK;
    if (count > (1ull << 28)) return fail(GB_EINVAL, "at most 2^28 even n per call");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    cudaStream_t s = ctx->stream;
    // P covers the odd numbers 1 .. the largest m = (hi - 4) / 2 index
    const uint64_t mmax = (hi - 4) / 2;
    const uint64_t words = ((mmax + 1 + 63) / 64) * 2;                  // whole 64-bit words
    const bool out_dev = is_device_ptr(counts);
    int rc;
    if ((rc = ctx->part_p.ensure(words * 4)) || (rc = ctx->part_rev.ensure((words + 1) * 4)) ||
        (!out_dev && (rc = ctx->part_out.ensure(count * 4))))
        return rc;
    if ((rc = run_sieve(ctx, 1, words * 32, ctx->part_p.as<uint32_t>(), nullptr))) return rc;
    GB_LAUNCH(gb::launch_reverse_bits(ctx->part_p.as<uint32_t>(), ctx->part_rev.as<uint32_t>(), words, s));
    uint32_t* d_out = out_dev ? counts : ctx->part_out.as<uint32_t>();
    GB_CUDA(cudaMemsetAsync(d_out, 0, count * 4, s));
    gb::PartitionArgs pa{};
    pa.P = ctx->part_p.as<uint32_t>();
    pa.rev = ctx->part_rev.as<uint32_t>();
    pa.words = words;
    pa.lo = lo;
    pa.count = count;
    pa.n_blocks = (count + 31) / 32;
    pa.run_words = 4096;
    pa.counts = d_out;
    const uint64_t need = ((hi - 4) / 2) / 2 / 32 + 1;                  // words of the largest n
    pa.runs = (need + pa.run_words - 1) / pa.run_words;
    GB_LAUNCH(gb::launch_partitions(pa, s));
    if (!out_dev) GB_CUDA(cudaMemcpyAsync(counts, d_out, count * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GB_OK;
}

int gb_query(gb_ctx* ctx, uint64_t n, uint32_t* p_min)
{
    if (!ctx || !p_min) return fail(GB_EINVAL, "NULL argument");
    return gb_query_batch(ctx, &n, 1, 0, p_min);
}

int gb_profile_enable(gb_ctx* ctx, int enable)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->prof_collect();
    if (rc) return rc;
    for (int k = 0; k < GB_PROF_KINDS; ++k) { ctx->prof_ms[k] = 0; ctx->prof_launches[k] = 0; ctx->prof_units[k] = 0; }
    ctx->work_strikes = ctx->work_iters = ctx->work_large = 0;
    ctx->kernels = 0;
    if (enable && !ctx->work.p) {
        if ((rc = ctx->work.ensure(24))) return rc;
        GB_CUDA(cudaMemset(ctx->work.p, 0, 24));
    }
    ctx->profiling = enable != 0;
    return GB_OK;
}

int gb_profile_read(gb_ctx* ctx, double* ms, uint64_t* launches, uint64_t* units)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->prof_collect();
    if (rc) return rc;
    for (int k = 0; k < GB_PROF_KINDS; ++k) {
        if (ms) ms[k] = ctx->prof_ms[k];
        if (launches) launches[k] = ctx->prof_launches[k];
        if (units) units[k] = ctx->prof_units[k];
    }
    return GB_OK;
}

int gb_profile_kernels(gb_ctx* ctx, uint64_t* kernels)
{
    if (!ctx || !kernels) return fail(GB_EINVAL, "NULL argument");
    *kernels = ctx->kernels;
    return GB_OK;
}

int gb_profile_work(gb_ctx* ctx, uint64_t* sieve_strikes, uint64_t* cover_iterations, uint64_t* large_strikes)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->prof_collect();
    if (rc) return rc;
    if (sieve_strikes) *sieve_strikes = ctx->work_strikes;
    if (cover_iterations) *cover_iterations = ctx->work_iters;
    if (large_strikes) *large_strikes = ctx->work_large;
    return GB_OK;
}

}  // extern "C"
