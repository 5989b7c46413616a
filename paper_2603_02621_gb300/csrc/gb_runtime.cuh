// gb_runtime.cuh -- the runtime's private declarations, shared by the
// translation units that implement the C ABI of include/gb.h: error
// reporting, the device and pinned host arenas, the context (gb_ctx) with its
// shared base primes, and the sieve driver.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gb.h"
#include "gb_internal.cuh"

enum { kProfSieve = 0, kProfCover = 1, kProfRetry = 2, kProfReduce = 3, kProfLarge = 4 };

// an NVTX range over a scope (host timeline of a profiler such as Nsight
// Systems: which call, slab and phase issued the launches; free when no tool
// is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// record msg as the calling thread's last error (gb_last_error) and return code
int fail(int code, const std::string& msg);

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

// allocations made by the library in this process (gb_alloc_stats)
extern std::atomic<uint64_t> g_alloc_count, g_alloc_bytes;

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes)
    {
        if (bytes <= cap) return GB_OK;
        if (gb::fault_hit(GB_FAULT_ALLOC)) return fail(GB_ENOMEM, "cudaMalloc: injected failure (GB_FAULT alloc)");
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = bytes + bytes / 8 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        g_alloc_count.fetch_add(1);
        g_alloc_bytes.fetch_add(want);
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
        if (gb::fault_hit(GB_FAULT_ALLOC)) return fail(GB_ENOMEM, "cudaMallocHost: injected failure (GB_FAULT alloc)");
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        const size_t want = bytes + bytes / 8 + 4096;
        const cudaError_t e = cudaMallocHost(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GB_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
        }
        g_alloc_count.fetch_add(1);
        g_alloc_bytes.fetch_add(want);
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

inline uint64_t isqrt_u64(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        uint64_t t = r | (1ull << b);
        if (t * t <= x) r = t;
    }
    return r;
}

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
    // bucket sieve of the primes >= 2^20 (GB_LARGE=bucket): per-tile hit
    // lists applied in shared memory; by default they are struck by global
    // atomics, measured faster on GB300
    bool bucket_large = false;
    // primes from mid_limit to sqrt(B) carried from chunk to chunk (gb_large.cu)
    // for windows of at least two chunks (GB_LARGE=atomic: restarted per chunk)
    bool carry_large = true;
    DevBuf cstate, cpos, cring, ccnt; // dense next-multiple offsets and wheel positions; bucket ring; bucket counts + spill count
    uint32_t carry_cap = 0;           // entries per bucket column (GB_CARRY_CAP, a test switch; 0 = sized by estimate)
    bool fused = false;               // sieve and block cover fused per CTA (GB_FUSED=1)
    uint32_t mid_limit = 1u << 20;    // primes from the split below this: per shared-memory slice (GB_MID_LOG2; 0 = off)
    DevBuf mres;                      // residue table of the slice starts (LargeArgs::res)
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
    // bytes copied between host and device memory by verification calls
    // (gb_profile_copies), reset by gb_profile_enable
    uint64_t copied_h2d = 0, copied_d2h = 0;
    cudaError_t copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s)
    {
        if (kind == cudaMemcpyHostToDevice) copied_h2d += bytes;
        else if (kind == cudaMemcpyDeviceToHost) copied_d2h += bytes;
        return cudaMemcpyAsync(dst, src, bytes, kind, s);
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
    // every phase is also an NVTX range named after its kind (a range left
    // open by an error return is closed by the next phase)
    bool nvtx_open = false;
    void prof_begin(int kind, uint64_t units)
    {
        static const char* const kNvtx[GB_PROF_KINDS] = {"gb/sieve", "gb/cover", "gb/retry", "gb/reduce",
                                                         "gb/large-primes"};
        if (nvtx_open) nvtxRangePop();
        nvtxRangePushA(kNvtx[kind]);
        nvtx_open = true;
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
        if (nvtx_open) nvtxRangePop();
        nvtx_open = false;
        if (!profiling || cur_kind < 0) return;
        cudaEvent_t b = take_event();
        cudaEventRecordWithFlags(b, capturing ? cap_stream : stream,
                                 capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        pending.push_back({cur_a, b, cur_kind});
        cur_kind = -1;
    }
    bool count_work = false;          // the kernels count their work (gb_profile_enable 1, not GB_PROFILE_EVENTS)
    unsigned long long* work_ptr(int i)
    {
        return profiling && count_work && work.p ? work.as<unsigned long long>() + i : nullptr;
    }
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
    // tile / large-prime split for a window whose sieving primes reach r: the
    // configured one, else by magnitude -- when primes reach 2^18 the ones
    // above 2^13 go faster to the 224 KB shared-memory slices (residue starts,
    // a wheel below 2^16) than through the tile sieve (measured on 2^34 even
    // n near 5e11 with the wheels in place: 2^13 15.33 ms per step, 2^14
    // 15.43, 2^15 15.78)
    uint32_t split(uint64_t r) const
    {
        if (cfg.bucket_split) return cfg.bucket_split;
        return r >= (1u << 18) ? std::min<uint32_t>(1u << 13, cfg.tile_bits) : cfg.tile_bits;
    }
};

// context configuration defaults and checks (gb_init, gb_set_config)
int fill_defaults(gb_config& c);
// tile-sieve arguments for the window (B, nbits); np / nsmall: primes <= sqrt
// of the last number and those below the split
int tile_sieve_args(gb_ctx* ctx, int64_t B, uint64_t nbits, gb::SieveArgs& a, uint64_t& np, uint64_t& nsmall);
// sieve of the window (B, nbits) into out (32-bit words; may be NULL when no
// prime is above the split), popcount optional; may_alloc false keeps to the
// kernels that need no buffer beyond out (no bucket lists)
int run_sieve(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out, unsigned long long* popc,
              bool may_alloc = true);
// base primes of a new context
int build_primes(gb_ctx* ctx);
// true for device (or managed) memory
bool is_device_ptr(const void* p);
