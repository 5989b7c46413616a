// gb_api.cu -- the runtime core of libgb (include/gb.h): error reporting,
// configuration, the context's lifetime and base primes, the sieve driver,
// gb_sieve_segment / gb_prime_pi and the profiling counters.
//
//   gb_init      seed sieve (primes < 2^16) -> base sieve of [1, L] on the GPU
//                -> compaction to the ascending prime list with Barrett
//                reciprocals; L = max(base_limit, p1, p2)
//   run_sieve    a q window: tile sieve of the primes below the split, then
//                the primes above it by 224 KB slices in shared memory (to
//                the mid limit) and by L2-resident chunks or bucket lists
//
// The verification entry points are in gb_verify.cu (gb_verify_range),
// gb_batch_host.cu (gb_verify_batch), gb_query_host.cu (gb_query,
// gb_partitions), gb_noalloc.cu, gb_tune.cu and gb_server.cu.
#include "gb_runtime.cuh"

thread_local std::string g_last_error;
std::atomic<uint64_t> g_alloc_count{0}, g_alloc_bytes{0};

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int fill_defaults(gb_config& c)
{
    if (c.seg_len == 0) c.seg_len = 1u << 24;
    if (c.base_limit == 0) c.base_limit = 1u << 16;
    if (c.tile_bits == 0) c.tile_bits = 1u << 18;
    if (c.cta_threads == 0) c.cta_threads = 256;
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
    if (c.cover_prefix > 1 && !gb::cover_prefix_valid((int)c.cover_prefix))
        return fail(GB_EINVAL, "cover_prefix must be 0, 1 or a multiple of 16 in [48, 256]");
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
    nsmall = std::min<uint64_t>(np, std::max<uint64_t>(ctx->pi(ctx->split(r) - 1), gb::kFirstStrikeIdx));
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

// The base primes [k0, k1) (from the slice limit on, every p^2 <= B) over the
// window (B, nbits), struck chunk by chunk of 2^clog2 bits with each prime
// started once and carried (gb_large.cu): the primes below half a chunk in
// per-prime words, the larger ones in a ring of per-chunk buckets.  A bucket
// holds at most the primes with a multiple m p (m coprime to 210) in one
// chunk: C (48/105) sum 1/p, which Mertens' theorem puts at
// C (48/105) (ln ln p_hi - ln ln p_lo); an entry that still finds its bucket
// full is struck through to the window's end by the kernel itself.
static int carry_large(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out, uint64_t k0, uint64_t k1,
                       uint32_t clog2)
{
    const uint64_t C = 1ull << clog2;
    const uint64_t kd = std::min<uint64_t>(k1, std::max<uint64_t>(k0, ctx->pi(C / 2 - 1)));
    gb::BucketLargeArgs a{};
    a.B = B;
    a.nbits = nbits;
    a.chunk_log2 = clog2;
    a.nchunks = (uint32_t)((nbits + C - 1) >> clog2);
    a.B_mod210 = (uint32_t)(B % 210);
    a.primes = ctx->base->primes.as<uint32_t>() + k0;
    a.recip = ctx->base->recip.as<uint64_t>() + k0;
    a.n_dense = (uint32_t)(kd - k0);
    a.n_sparse = (uint32_t)(k1 - kd);
    uint32_t R = 1;
    a.grid = gb::carry_grid();
    if (a.n_sparse) {
        const double p_lo = (double)ctx->base->h_primes[kd], p_hi = (double)ctx->base->h_primes[k1 - 1];
        // an entry moves at most 1 + 5 p / C chunks ahead (half gaps of the
        // wheel up to 5); the bucket being drained and the one drained before
        // it must stay out of reach
        const uint64_t adv = 1 + ((5ull * ctx->base->h_primes[k1 - 1]) >> clog2);
        while (R < adv + 2) R <<= 1;
        if (R > gb::kCarryMaxRing) return fail(GB_EINVAL, "internal: carried primes reach too many chunks ahead");
        // each CTA's column holds its share (1 / grid) of a bucket
        const double M = (double)C * (48.0 / 105.0) *
                         (std::log(std::log(p_hi)) - std::log(std::log(p_lo)) + 1.0 / p_lo) / a.grid;
        a.cap = (uint32_t)std::min(2.0e9, 1.15 * M + 8.0 * std::sqrt(M) + 64.0);
        if (ctx->carry_cap) a.cap = ctx->carry_cap;           // (test switch: small columns spill)
    }
    const size_t ncnt = (size_t)R * a.grid;
    int rc;
    if ((a.n_dense && ((rc = ctx->cstate.ensure((size_t)a.n_dense * 4)) || (rc = ctx->cpos.ensure(a.n_dense)))) ||
        (a.n_sparse && (rc = ctx->cring.ensure(ncnt * a.cap * 8))) || (rc = ctx->ccnt.ensure((ncnt + 1) * 4)))
        return rc;
    a.dstate = ctx->cstate.as<uint32_t>();
    a.dpos = ctx->cpos.as<uint8_t>();
    a.ring = ctx->cring.as<uint64_t>();
    a.ring_cnt = ctx->ccnt.as<uint32_t>();
    a.ring_mask = R - 1;
    a.spills = ctx->ccnt.as<unsigned int>() + ncnt;
    a.out = out;
    a.strikes = ctx->work_ptr(2);
    GB_CUDA(cudaMemsetAsync(ctx->ccnt.p, 0, (ncnt + 1) * 4, ctx->stream));
    GB_LAUNCH(gb::launch_large_start(a, ctx->stream));
    for (uint32_t c = 0; c < a.nchunks; ++c) GB_LAUNCH(gb::launch_large_chunk(a, c, ctx->stream));
    return GB_OK;
}

int run_sieve(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out, unsigned long long* popc, bool may_alloc)
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
        // primes below mid_limit: per shared-memory slice of the window
        uint64_t nmid = nsmall;
        const int64_t last = B + 2 * (int64_t)(nbits - 1);
        if (ctx->mid_limit > ctx->split(isqrt_u64((uint64_t)last))) {
            nmid = std::min<uint64_t>(np, std::max<uint64_t>(nsmall, ctx->pi(ctx->mid_limit - 1)));
            if (nmid > nsmall) {
                gb::LargeArgs ma = la;
                ma.n_primes = (uint32_t)(nmid - nsmall);
                // starts from a residue table of the window (16 bytes per
                // prime, sized once for every prime below the slice limit)
                // where the slices and primes allow it
                const uint64_t slices = (nbits + gb::kMidSliceBits - 1) / gb::kMidSliceBits;
                if (may_alloc && slices <= gb::kMidResSlices && ctx->base->h_primes[nmid - 1] < (1u << 20)) {
                    const uint64_t cap = ctx->pi(std::min<uint64_t>(ctx->mid_limit, 1u << 20) - 1);
                    int rc = ctx->mres.ensure((size_t)std::max<uint64_t>(cap, nmid) * 16);
                    if (rc) return rc;
                    ma.res = ctx->mres.as<uint4>();
                    ctx->kernels += 1;                      // the table's kernel
                }
                GB_LAUNCH(gb::launch_mid(ma, nbits, ctx->stream));
            }
            la.primes = ctx->base->primes.as<uint32_t>() + nmid;
            la.recip = ctx->base->recip.as<uint64_t>() + nmid;
            la.n_primes = (uint32_t)(np - nmid);
        }
        // primes of at least a bucket tile (2^20) go to the bucket sieve; those
        // between the split and a bucket tile hit a tile several times and
        // keep the atomic kernel
        // (never for a caller that must not allocate: the lists are sized on use)
        const uint64_t nbucket_lo = ctx->bucket_large && may_alloc
                                        ? std::max<uint64_t>(nmid, ctx->pi((1u << gb::kBucketTileLog2) - 1)) : np;
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
            GB_CUDA(ctx->copy(flags.data(), ctx->bflags.p, nchunks * 4, cudaMemcpyDeviceToHost, ctx->stream));
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
        // the primes with p^2 <= B, over a window of two chunks or more: started
        // once, carried from chunk to chunk; the rest restart in every chunk
        uint64_t natomic = nmid;
        const uint32_t clog2 = 28;
        if (nbucket_lo > nmid && ctx->carry_large && may_alloc && B > 0 && (nbits >> clog2) >= 2) {
            // (carried primes below 2^31: a bucket entry holds p / 2 in 30 bits)
            const uint64_t kb1 = std::min<uint64_t>(std::min<uint64_t>(nbucket_lo, ctx->pi(0x7fffffffu)),
                                                    std::max<uint64_t>(nmid, ctx->pi(isqrt_u64((uint64_t)B))));
            if (kb1 > nmid) {
                int rc = carry_large(ctx, B, nbits, out, nmid, kb1, clog2);
                if (rc) return rc;
                natomic = kb1;
            }
        }
        if (nbucket_lo > natomic) {
            la.primes = ctx->base->primes.as<uint32_t>() + natomic;
            la.recip = ctx->base->recip.as<uint64_t>() + natomic;
            la.n_primes = (uint32_t)(nbucket_lo - natomic);
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
    GB_CUDA(ctx->copy(seedw.data(), seedbits.p, seed_words * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    size_t nseed = 1;                                 // the prime 2
    for (uint32_t v : seedw) nseed += (size_t)__builtin_popcount(v);
    std::vector<uint32_t> seed(nseed);
    GB_CUDA(ctx->copy(seed.data(), seedp.p, nseed * 4, cudaMemcpyDeviceToHost, s));
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
    GB_CUDA(ctx->copy(&nodd, popc.p, 8, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    const uint64_t n = nodd + 1;
    DevBuf np, nr;
    if ((rc = np.ensure(n * 4)) || (rc = nr.ensure(n * 8))) return rc;
    gb::CompactArgs cb{bits.as<uint32_t>(), nwords, 1, counts.as<uint32_t>(), np.as<uint32_t>(), nr.as<uint64_t>()};
    GB_CUDA(gb::launch_compact(cb, s));
    ctx->base->h_primes.resize(n);
    GB_CUDA(ctx->copy(ctx->base->h_primes.data(), np.p, n * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    ctx->base->primes.take(np);
    ctx->base->recip.take(nr);
    return GB_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// accessors for entry points in other translation units
namespace gb {
// readers of the debug words of the translation units built with GB_DEBUG
// (registered while the library loads; a function-local list, so the order in
// which the units initialise does not matter)
static std::vector<uint32_t (*)(bool)>& debug_readers()
{
    static std::vector<uint32_t (*)(bool)> r;
    return r;
}
int debug_register(uint32_t (*reader)(bool reset))
{
    debug_readers().push_back(reader);
    return (int)debug_readers().size();
}
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
int ctx_sieve_noalloc(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out)
{
    return run_sieve(ctx, B, nbits, out, nullptr, false);
}
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace gb

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
    case GB_ECANCELED: return "GB_ECANCELED: request cancelled before it ran";
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
    gb::fault_from_env();
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
    // one warp per prime below 512 (larger primes: one thread each, through
    // the mod-30 wheel; measured faster from 512 on than warps without it)
    ctx->warp_split = (int)std::min<uint32_t>(512, c.tile_bits / 64);
    if (const char* e = getenv("GB_WARP_SPLIT")) ctx->warp_split = atoi(e);
    if (const char* e = getenv("GB_COVER")) ctx->generic_cover = std::string(e) == "generic";
    if (const char* e = getenv("GB_BATCH_GRAPH")) ctx->batch_graph = atoi(e) != 0;
    if (const char* e = getenv("GB_LARGE")) {
        ctx->bucket_large = std::string(e) == "bucket";
        ctx->carry_large = std::string(e) != "atomic";
    }
    if (const char* e = getenv("GB_FUSED")) ctx->fused = atoi(e) != 0;
    if (const char* e = getenv("GB_MID_LOG2")) {
        const int v = atoi(e);
        ctx->mid_limit = (v >= 16 && v <= 31) ? (1u << v) : 0u;
    }
    if (const char* e = getenv("GB_CARRY_CAP")) ctx->carry_cap = (uint32_t)std::strtoul(e, nullptr, 10);
    if (const char* e = getenv("GB_LARGE_CHUNK_LOG2")) {
        const int v = atoi(e);
        if (v >= 16 && v <= 40) ctx->large_chunk_bits = 1ull << v;
    }
    if (const char* e = getenv("GB_KA")) {
        const int v = atoi(e);
        if (gb::cover_prefix_valid(v) && ctx->cfg.cover_prefix == 0) ctx->cfg.cover_prefix = v;
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
    ctx->carry_large = parent->carry_large;
    ctx->carry_cap = parent->carry_cap;
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
                      &ctx->cstate, &ctx->cring, &ctx->ccnt,
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
    if (!getenv("GB_WARP_SPLIT")) ctx->warp_split = (int)std::min<uint32_t>(512, c.tile_bits / 64);
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
    GB_CUDA(ctx->copy(&c, ctx->counter.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
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
    const bool need_buf = ctx->pi(isqrt_u64(x)) > ctx->pi(ctx->split(isqrt_u64(x)) - 1);
    if (need_buf && (rc = ctx->q.ensure(((std::min(chunk, total) + 63) / 64) * 8))) return rc;
    for (uint64_t done = 0; done < total; done += chunk) {
        const uint64_t nb = std::min(chunk, total - done);
        rc = run_sieve(ctx, 3 + 2 * (int64_t)done, nb, need_buf ? ctx->q.as<uint32_t>() : nullptr,
                       ctx->counter.as<unsigned long long>());
        if (rc) return rc;
    }
    unsigned long long c = 0;
    GB_CUDA(ctx->copy(&c, ctx->counter.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    *count = c + 1;                                 // + the prime 2
    return GB_OK;
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
    ctx->copied_h2d = ctx->copied_d2h = 0;
    ctx->count_work = enable != 0 && enable != GB_PROFILE_EVENTS;
    if (ctx->count_work && !ctx->work.p) {
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

int gb_profile_copies(gb_ctx* ctx, uint64_t* h2d_bytes, uint64_t* d2h_bytes)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    if (h2d_bytes) *h2d_bytes = ctx->copied_h2d;
    if (d2h_bytes) *d2h_bytes = ctx->copied_d2h;
    return GB_OK;
}

uint32_t gb_debug_word(int reset)
{
    uint32_t first = 0;
    for (auto reader : gb::debug_readers()) {
        const uint32_t v = reader(reset != 0);
        if (v && !first) first = v;
    }
    return first;
}

int gb_debug_build(void)
{
#ifdef GB_DEBUG
    return 1;
#else
    return 0;
#endif
}

void gb_alloc_stats(uint64_t* count, uint64_t* bytes)
{
    if (count) *count = g_alloc_count.load();
    if (bytes) *bytes = g_alloc_bytes.load();
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
