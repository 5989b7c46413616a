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
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gb.h"
#include "gb_internal.cuh"

namespace {

enum { kProfSieve = 0, kProfCover = 1, kProfRetry = 2, kProfReduce = 3 };

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

struct gb_ctx {
    gb_config cfg{};
    cudaStream_t stream = nullptr;
    uint64_t L = 0;                   // primes are known up to L
    std::vector<uint32_t> h_primes;   // [2, 3, 5, ...] <= L
    DevBuf primes, recip;             // device copies
    DevBuf wheel;                     // pre-sieve stamp tables
    DevBuf q;                         // slab q window
    DevBuf hist, maxkey, maxkey2, unres, retry, retry_count, summary, rows, merged, pmin, counter, totals, records;
    DevBuf work;                      // profiling work counters: [0] sieve strikes, [1] cover iterations
    uint64_t work_strikes = 0, work_iters = 0;
    int warp_split = 0;               // sieving primes below this strike one warp each
    bool generic_cover = false;       // force the generic cover kernel (GB_COVER=generic)
    uint64_t large_chunk_bits = 1ull << 30;   // large-prime strikes per L2-sized chunk of the window
    int ka_override = 0;              // first-phase length of the two-phase cover (GB_KA)

    // per-kernel device time (CUDA events on the context's stream around each launch)
    bool profiling = false;
    double prof_ms[GB_PROF_KINDS] = {};
    uint64_t prof_launches[GB_PROF_KINDS] = {};
    uint64_t prof_units[GB_PROF_KINDS] = {};
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
        cudaEventRecord(cur_a, stream);
        prof_launches[kind] += 1;
        prof_units[kind] += units;
    }
    void prof_end()
    {
        if (!profiling || cur_kind < 0) return;
        cudaEvent_t b = take_event();
        cudaEventRecord(b, stream);
        pending.push_back({cur_a, b, cur_kind});
        cur_kind = -1;
    }
    unsigned long long* work_ptr(int i) { return profiling && work.p ? work.as<unsigned long long>() + i : nullptr; }
    int prof_collect()
    {
        if (work.p) {
            unsigned long long w[2] = {0, 0};
            cudaError_t e = cudaMemcpy(w, work.p, sizeof w, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemset(work.p, 0, sizeof w);
            if (e != cudaSuccess) return fail(GB_ECUDA, std::string("profile counters: ") + cudaGetErrorString(e));
            work_strikes += w[0];
            work_iters += w[1];
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
        for (const Pending& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }

    // number of primes <= x (x <= L)
    uint64_t pi(uint64_t x) const
    {
        return (uint64_t)(std::upper_bound(h_primes.begin(), h_primes.end(), (uint32_t)std::min<uint64_t>(x, 0xffffffffull)) - h_primes.begin());
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
    if (c.slab_bits < c.seg_len) c.slab_bits = c.seg_len;
    return GB_OK;
}

// sieve the odd numbers B + 2i, i < nbits, into out (device words) or count only
int run_sieve(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out, unsigned long long* popc)
{
    if (nbits == 0) return GB_OK;
    const int64_t last = B + 2 * (int64_t)(nbits - 1);
    const uint64_t r = last > 0 ? isqrt_u64((uint64_t)last) : 0;
    if (r > ctx->L) return fail(GB_EINVAL, "window beyond base_limit^2");
    const uint64_t np = ctx->pi(r);                 // primes <= sqrt(last)
    // primes from bucket_split on are struck by the large-prime kernel, chunk
    // by chunk, into the output words (the tile kernel only counts bits when
    // there are none)
    const uint64_t nsmall = std::min<uint64_t>(np, std::max<uint64_t>(ctx->pi(ctx->cfg.bucket_split - 1), gb::kFirstStrikeIdx));
    const bool large = np > nsmall && out;
    if (np > nsmall && !out) return fail(GB_EINVAL, "internal: large primes need an output buffer");
    gb::SieveArgs a{};
    a.B = B;
    a.nbits = nbits;
    a.tile_bits = ctx->cfg.tile_bits;
    a.primes = ctx->primes.as<uint32_t>() + gb::kFirstStrikeIdx;
    a.recip = ctx->recip.as<uint64_t>() + gb::kFirstStrikeIdx;
    const uint64_t nstrike = nsmall > gb::kFirstStrikeIdx ? nsmall - gb::kFirstStrikeIdx : 0;
    const uint64_t nwarp = std::min<uint64_t>(nstrike, ctx->pi((uint64_t)ctx->warp_split - 1) > gb::kFirstStrikeIdx
                                                            ? ctx->pi((uint64_t)ctx->warp_split - 1) - gb::kFirstStrikeIdx : 0);
    a.n_warp = (uint32_t)nwarp;
    a.n_primes = (uint32_t)nstrike;
    a.wheel = ctx->wheel.as<uint32_t>();
    a.out = out;
    a.popcount = large ? nullptr : popc;
    a.strikes = ctx->work_ptr(0);
    GB_CUDA(gb::launch_sieve(a, (int)ctx->cfg.cta_threads, ctx->stream));
    if (large) {
        gb::LargeArgs la{};
        la.B = B;
        la.primes = ctx->primes.as<uint32_t>() + nsmall;
        la.recip = ctx->recip.as<uint64_t>() + nsmall;
        la.n_primes = (uint32_t)(np - nsmall);
        la.out = out;
        la.strikes = ctx->work_ptr(0);
        const uint64_t chunk = ctx->large_chunk_bits;
        for (uint64_t c0 = 0; c0 < nbits; c0 += chunk) {
            la.bit_lo = c0;
            la.bit_hi = std::min(nbits, c0 + chunk);
            GB_CUDA(gb::launch_large(la, ctx->stream));
        }
        if (popc) GB_CUDA(gb::launch_popcount(out, ((nbits + 63) / 64) * 2, popc, ctx->stream));
    }
    return GB_OK;
}

int build_primes(gb_ctx* ctx)
{
    cudaStream_t s = ctx->stream;
    int rc;
    if ((rc = ctx->wheel.ensure(gb::kWheelWords * 4))) return rc;
    GB_CUDA(gb::launch_wheel_tables(ctx->wheel.as<uint32_t>(), s));

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
        ctx->h_primes.assign(seed.begin(), seed.end());
        ctx->h_primes.resize(std::upper_bound(seed.begin(), seed.end(), (uint32_t)ctx->L) - seed.begin());
        const size_t n = ctx->h_primes.size();
        if ((rc = ctx->primes.ensure(n * 4)) || (rc = ctx->recip.ensure(n * 8))) return rc;
        GB_CUDA(cudaMemcpyAsync(ctx->primes.p, seedp.p, n * 4, cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaMemcpyAsync(ctx->recip.p, seedr.p, n * 8, cudaMemcpyDeviceToDevice, s));
        GB_CUDA(cudaStreamSynchronize(s));
        return GB_OK;
    }

    // base sieve of the odd numbers 1 .. L with the seed primes
    ctx->h_primes = seed;                            // primes < 2^16 serve as sieving primes
    ctx->primes.take(seedp);
    ctx->recip.take(seedr);
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
    ctx->h_primes.resize(n);
    GB_CUDA(cudaMemcpyAsync(ctx->h_primes.data(), np.p, n * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    ctx->primes.take(np);
    ctx->recip.take(nr);
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
    v->primes = ctx->primes.as<uint32_t>();
    v->generic_cover = ctx->generic_cover;
    v->ka_override = ctx->ka_override;
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
    if (const char* e = getenv("GB_LARGE_CHUNK_LOG2")) {
        const int v = atoi(e);
        if (v >= 16 && v <= 40) ctx->large_chunk_bits = 1ull << v;
    }
    if (const char* e = getenv("GB_KA")) {
        const int v = atoi(e);
        if (v == 64 || v == 128 || v == 192 || v == 256) ctx->ka_override = v;
    }
    rc = build_primes(ctx);
    if (rc) {
        gb_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return GB_OK;
}

void gb_destroy(gb_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->cfg.device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    DevBuf* bufs[] = {&ctx->primes, &ctx->recip, &ctx->wheel, &ctx->q, &ctx->hist,
                      &ctx->maxkey, &ctx->maxkey2, &ctx->unres, &ctx->retry, &ctx->retry_count, &ctx->summary,
                      &ctx->rows, &ctx->merged, &ctx->pmin, &ctx->counter, &ctx->totals, &ctx->records, &ctx->work};
    for (DevBuf* b : bufs) b->release();
    delete ctx;
}

int gb_get_config(const gb_ctx* ctx, gb_config* out)
{
    if (!ctx || !out) return fail(GB_EINVAL, "NULL argument");
    *out = ctx->cfg;
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
    ctx->prof_begin(kProfSieve, n_bits);
    rc = run_sieve(ctx, A_odd, n_bits, reinterpret_cast<uint32_t*>(q_bits),
                   ctx->counter.as<unsigned long long>());
    ctx->prof_end();
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

        ctx->prof_begin(kProfSieve, qw * 64);
        if ((rc = run_sieve(ctx, B, qw * 64, ctx->q.as<uint32_t>(), nullptr))) return rc;
        ctx->prof_end();

        gb::CoverArgs ca{};
        ca.Q = ctx->q.as<uint64_t>();
        ca.H = H;
        ca.n_count = n_count;
        ca.n_words = n_words;
        ca.words_per_seg = (uint32_t)(S / 64);
        ca.cta_words = std::min<uint32_t>(2048, (uint32_t)(S / 64));
        ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
        ca.nseg = (uint32_t)ns;
        ca.primes = ctx->primes.as<uint32_t>();
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
        int KA = (pm || ctx->generic_cover) ? 0 : gb::cover_fast_phase_primes(K1, A0 + 2 * n_count);
        if (KA && ctx->ka_override && (uint32_t)ctx->ka_override <= K1) KA = ctx->ka_override;
        if (KA) {
            // block cover: 7680 32-bit words per CTA (ten rounds of 96 words per
            // warp, the most its 10-bit counters allow)
            ca.cta_words = std::min<uint32_t>(3840, (uint32_t)(S / 64));
            ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
        }
        ctx->prof_begin(kProfCover, n_count);
        if (KA) GB_CUDA(gb::launch_cover_fast(ca, KA, s));
        else GB_CUDA(gb::launch_cover(ca, (int)cfg.cta_threads, s));
        ctx->prof_end();

        if (retry) {
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
            GB_CUDA(gb::launch_retry(ra, s));
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
        GB_CUDA(gb::launch_reduce(rd, s));
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
    GB_CUDA(gb::launch_finalize(fa, s));
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

int gb_profile_enable(gb_ctx* ctx, int enable)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->prof_collect();
    if (rc) return rc;
    for (int k = 0; k < GB_PROF_KINDS; ++k) { ctx->prof_ms[k] = 0; ctx->prof_launches[k] = 0; ctx->prof_units[k] = 0; }
    ctx->work_strikes = ctx->work_iters = 0;
    if (enable && !ctx->work.p) {
        if ((rc = ctx->work.ensure(16))) return rc;
        GB_CUDA(cudaMemset(ctx->work.p, 0, 16));
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

int gb_profile_work(gb_ctx* ctx, uint64_t* sieve_strikes, uint64_t* cover_iterations)
{
    if (!ctx) return fail(GB_EINVAL, "NULL argument");
    GB_CUDA(cudaSetDevice(ctx->cfg.device));
    int rc = ctx->prof_collect();
    if (rc) return rc;
    if (sieve_strikes) *sieve_strikes = ctx->work_strikes;
    if (cover_iterations) *cover_iterations = ctx->work_iters;
    return GB_OK;
}

}  // extern "C"
