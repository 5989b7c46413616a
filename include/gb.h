/*
 * gb.h -- C ABI of libgb, a GB300 (sm_103a) implementation of the segmented
 * double sieve and the loop-inverted Goldbach cover of GoldbachGPU
 * (arXiv 2603.02621).
 *
 * The method (Sec. 2.3.1): instead of searching, for each even n, a prime p
 * with n - p prime, iterate over the primes p and mark every even n whose
 * partner q = n - p is prime.  The primality of every odd q in a window is
 * held as an odd-only bitset (Sec. 2.2: one bit per odd number), produced
 * here on the GPU by a segmented sieve of Eratosthenes (the GPU sieve that
 * Sec. 4.5 names as future work).  The marking is the word-parallel form
 * Sec. 4.3 names as future work: for p = 3, 5, 7, ... <= P in ascending order,
 * a shifted copy of the q-bitset is OR-ed into a coverage bitset C over the
 * even n, and the first p that sets an n's bit is that n's minimal Goldbach
 * prime p_min(n) (Sec. 2.3.2).  n with no p <= P1 go to a second GPU pass up
 * to P2 (replacing the CPU fallback of Sec. 2.3.3).
 *
 * Conventions (all entry points):
 *   - return 0 (GB_OK) on success, a GB_E* code otherwise; gb_strerror()
 *     names the code and gb_last_error() gives the last message of the
 *     calling thread;
 *   - ranges are half-open [lo, hi) over EVEN n; lo must be even and >= 4,
 *     hi even and > lo.  "[4, N]" inclusive is [4, N + 2);
 *   - prime index: the i-th prime with p_0 = 2, p_1 = 3, p_2 = 5, ...
 *   - every buffer is owned by the caller; the library owns its device
 *     arenas.  Pointers documented "host or device" are classified with
 *     cudaPointerGetAttributes; host memory may be pageable or pinned;
 *   - an n with no p <= the bound is DATA (counted as unresolved), not an
 *     error;
 *   - a context is bound to one device and one stream; calls on one
 *     context must not overlap (not thread-safe per context).
 */
#ifndef GB_H
#define GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK        0
#define GB_EINVAL    1  /* bad argument: odd/short range, lo >= hi, hi beyond base_limit^2, P > p2, bad config */
#define GB_ENOMEM    2  /* device or host allocation failed (or admission refused) */
#define GB_ECUDA     3  /* a CUDA runtime call failed; gb_last_error() has the CUDA message */
#define GB_ETIMEOUT  4  /* a bounded device wait gave up */
#define GB_EBUSY     5  /* the context is in use */
#define GB_ERANGE    6  /* an output buffer is too small; everything that fit was written */
#define GB_ECANCELED 7  /* a server request was cancelled before it ran */

typedef struct gb_ctx gb_ctx;

/* Context configuration.  Zero fields take the defaults given. */
typedef struct gb_config {
    int32_t  device;        /* CUDA device ordinal */
    uint32_t seg_len;       /* S: even n per segment (equal to the odd q per
                               segment).  Multiple of 2048; 0 = 2^24.  Segments
                               are the unit of the per-segment outputs. */
    uint64_t base_limit;    /* base primes are sieved to this bound at init;
                               every range needs hi <= base_limit^2 (and
                               base_limit >= the primes it needs, Sec. 2.3.1:
                               a segmented sieve of [A, B] needs primes to
                               sqrt(B)); 0 = 2^16; at most 2^32 */
    uint32_t tile_bits;     /* segment-sieve tile (odd numbers per CTA tile),
                               multiple of 8192, <= 2^20; 0 = 2^18 */
    uint32_t cta_threads;   /* threads per segment-sieve CTA: 128, 256 or
                               512; 0 = 256 */
    uint32_t bucket_split;  /* sieving primes >= this are struck by the
                               large-prime passes (per 2^20-bit shared-memory
                               slice below 2^20, else one start per L2-sized
                               chunk of the window, global atomic AND)
                               instead of per tile in shared memory; 0 = by
                               magnitude: 2^16 (at most tile_bits) when the
                               window's sieving primes reach 2^18, else
                               tile_bits */
    uint32_t p1;            /* first-pass bound P1 (p <= P1); 0 = 2^15 */
    uint32_t p2;            /* retry-pass bound P2; 0 or <= p1 = no retry pass;
                               <= 2^24 */
    uint32_t cover_prefix;  /* primes of the cover's unrolled phase, a
                               multiple of 16 in [48, 256]: a first block of
                               48 (prefix = 16 mod 32) or 64 primes over every
                               word, blocks of 32 over the words still open,
                               then per-n probing; 0 = chosen by the magnitude
                               of n; 1 = the generic cover (one 64-n word per
                               lane, primes looped until the word is full),
                               whose work counter is the algorithmic count.
                               Outputs do not depend on it (the batched mode
                               treats 1 as 0). */
    uint64_t slab_bits;     /* most q-bits sieved and kept resident at once
                               (a slab is a run of whole segments); 0 = 2^33 */
    void*    stream;        /* cudaStream_t for all work; NULL = the legacy
                               default stream */
} gb_config;

/* Largest hi of a range: the sieve window runs past hi by the halo (< 2^25)
 * and must stay below 2^63. */
#define GB_MAX_HI ((1ull << 63) - (1ull << 26))

/* Per-segment output (Sec. 2.3.2): the segment holds the even n in [lo, hi). */
typedef struct gb_segment_result {
    uint64_t lo, hi;
    uint64_t n_checked;     /* (hi - lo) / 2 */
    uint64_t unresolved;    /* n with no prime p <= the final bound */
    uint64_t max_pmin_n;    /* smallest n attaining max_pmin (0 if none) */
    uint32_t max_pmin;      /* largest p_min found in the segment (0 if none) */
    uint32_t hist_len;      /* 1 + prime index of max_pmin: entries of this
                               segment's histogram row that can be nonzero */
} gb_segment_result;

/* Output of gb_verify_range: totals over the range plus optional detail. */
typedef struct gb_range_result {
    /* --- written by the library --- */
    uint64_t n_checked;     /* (hi - lo) / 2 */
    uint64_t unresolved;    /* n with no prime p <= the final bound */
    uint64_t max_pmin_n;    /* smallest n attaining max_pmin (0 if none) */
    uint32_t max_pmin;      /* largest p_min over the range (0 if none) */
    uint32_t hist_len;      /* 1 + prime index of max_pmin */
    uint32_t n_segments;    /* number of segments of seg_len even n */
    uint32_t p_final;       /* largest bound used (P2 if a retry pass ran, else P) */
    /* --- optional caller buffers (NULL = skip) --- */
    uint64_t* hist;         /* host: hist[i] = #n whose p_min is the i-th
                               prime, summed over the range; hist_cap entries;
                               entries from hist_len on are written as 0 */
    uint32_t  hist_cap;
    uint32_t* pmin;         /* host or device: pmin[(n - lo)/2] = p_min(n), 0 if
                               unresolved; n_checked entries */
    gb_segment_result* segs;/* host or device: one record per segment, the
                               first min(seg_cap, n_segments) are written
                               (GB_ERANGE if seg_cap < n_segments) */
    uint32_t  seg_cap;
    uint64_t* seg_hist;     /* host or device: row k (seg_hist_stride entries)
                               is segment k's histogram, rows for the first
                               seg_cap segments (seg_cap 0: all n_segments
                               rows); GB_ERANGE if a segment's hist_len exceeds
                               the stride (the row is truncated) */
    uint32_t  seg_hist_stride;
    uint32_t  reserved;
} gb_range_result;

/* Create a context: select the device, sieve the base primes to
 * cfg->base_limit on the GPU (the base sieve of Sec. 2.3.1), build the
 * cover's prime tables to max(p1, p2).  cfg may be NULL (all defaults). */
int gb_init(gb_ctx** out, const gb_config* cfg);

/* Release every device resource of the context (NULL is a no-op). */
/* A second context on the same device that shares parent's base primes (no
 * second base sieve, no second copy in device or host memory) but has its own
 * stream (cudaStream_t, NULL = legacy default stream), its own device arenas
 * and a copy of parent's tunable configuration: contexts made this way run
 * their calls concurrently, one host thread each.  The shared primes live
 * until the last context using them is destroyed. */
int gb_init_shared(gb_ctx** out, const gb_ctx* parent, void* stream);

void gb_destroy(gb_ctx* ctx);

/* The configuration in effect, defaults filled in. */
int gb_get_config(const gb_ctx* ctx, gb_config* out);

/* Change the tunable fields of a context's configuration (seg_len, tile_bits,
 * cta_threads, bucket_split, p1, p2, cover_prefix, slab_bits; 0 = default as
 * in gb_init).  device, base_limit and stream must equal the context's
 * (GB_EINVAL otherwise); p1 and p2 must not exceed the base primes.  Waits
 * for the context's stream.  Outputs of later calls do not depend on the
 * tunables, except that per-segment outputs follow seg_len and the first-pass
 * histogram length follows p1. */
int gb_set_config(gb_ctx* ctx, const gb_config* cfg);

/* Autotuner (segment length, sieve tile, CTA size, tile / large-prime split, P):
 * verifies the sample workload [lo[i], hi[i]) i < count under candidate
 * settings, one parameter at a time (coordinate descent over tile_bits,
 * bucket_split, p1, cover_prefix, cta_threads and, for GB_TUNE_PLAIN,
 * seg_len), each timed with CUDA events on the context's stream as the
 * best of reps runs after a warm-up run; keeps the fastest setting in the
 * context and returns it in *out (optional) with its time in *best_ms
 * (optional).  mode GB_TUNE_PLAIN times gb_verify_range on each range,
 * GB_TUNE_BATCH one gb_verify_batch over all of them.  reps 0 = 2. */
#define GB_TUNE_PLAIN 0
#define GB_TUNE_BATCH 1
int gb_autotune(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, int mode, uint32_t reps,
                gb_config* out, double* best_ms);
/* Autotune cache.  When the environment variable GB_TUNE_CACHE names a file,
 * gb_autotune first looks up the key "<GPU name>|<SM count>|<mode>|<count>|
 * <hash of the sample's bounds>|<base_limit>|<p2>|<slab_bits>" there: on a
 * hit it applies the stored setting without timing anything (best_ms is the
 * stored time); otherwise it searches and appends one line
 * "<key>\t<tile_bits> <bucket_split> <p1> <cover_prefix> <seg_len>
 * <cta_threads> <best ms>".  The last line of a key wins; damaged lines are
 * skipped.  Host-only helpers over that file format: lookup returns GB_OK and
 * fills those fields of *cfg (the rest untouched), GB_ERANGE when the key is
 * absent or the file cannot be read; store appends (GB_EINVAL if the file
 * cannot be written or the key holds a tab or newline). */
int gb_tune_cache_lookup(const char* path, const char* key, gb_config* cfg, double* best_ms);
int gb_tune_cache_store(const char* path, const char* key, const gb_config* cfg, double best_ms);

/* Sieve one window of odd numbers (Sec. 2.2 layout, Sec. 2.3.1 segment sieve):
 * bit i (bit i%64 of word i/64, little-endian bit order) of q_bits is 1 iff the
 * odd number A_odd + 2i is prime, for 0 <= i < n_bits; bits from n_bits to the
 * end of the last word are 0.  A_odd is odd and may be <= 1 (numbers below 2
 * are not prime).  q_bits: DEVICE pointer, ceil(n_bits/64) uint64 words,
 * 16-byte aligned.  popcount (host, may be NULL): number of 1 bits.
 * GB_EINVAL if A_odd is even or A_odd + 2(n_bits-1) > base_limit^2. */
int gb_sieve_segment(gb_ctx* ctx, int64_t A_odd, uint64_t n_bits,
                     uint64_t* q_bits, uint64_t* popcount);

/* pi(x): number of primes <= x, counted from GPU-sieved bitsets (x <=
 * base_limit^2). */
int gb_prime_pi(gb_ctx* ctx, uint64_t x, uint64_t* count);

/* Exhaustive verification of every even n in [lo, hi) (Sec. 2.3, Table 4):
 * p_min(n) for all n with p <= P (P = 0: the context's p1), then, if the
 * context has p2 > P, a second GPU pass over the n still unresolved with
 * P < p <= p2 (Sec. 2.3.3's fallback, moved to the GPU).  Results are exact
 * integers.  Requires hi <= base_limit^2 and P <= 2^24. */
int gb_verify_range(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t P,
                    gb_range_result* out);

/* Batched verification: count independent ranges [lo[i], hi[i]) verified in
 * one pass of persistent kernels (the segment loop of Sec. 2.3 over many
 * ranges at once; the work queue and the per-range windows let thousands of
 * ranges of uneven length share the GPU).  Each range gets the outputs
 * gb_verify_range would give it: one record in
 * results[i] (lo, hi, n_checked, unresolved, max_pmin with its smallest n,
 * hist_len) and, if hist is given, row i (hist_stride entries) of its p_min
 * histogram.  P as in gb_verify_range (0: the context's p1); a range with n
 * still open after P is redone by gb_verify_range, retry pass included, so
 * the results equal calling gb_verify_range on each range.  lo/hi: host
 * arrays; results and hist: host or device.  Each range needs
 * hi - lo <= 2 * 2^32 and hi <= base_limit^2; count <= 2^24.  GB_ERANGE if a
 * range's hist_len exceeds hist_stride (the row is truncated). */
int gb_verify_batch(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, uint32_t P,
                    gb_segment_result* results, uint64_t* hist, uint32_t hist_stride);

/* Single-n query (Sec. 2.4, the single-number check; here the minimal p):
 * *p_min = the smallest prime p <= P with n - p prime, 0 if there is none,
 * for even n with 4 <= n < 2^63 (GB_EINVAL otherwise).  P is the context's
 * larger bound max(p1, p2).  Computed on the GPU: a window pre-sieve of the
 * partners n - p by the primes <= 2048, then a deterministic Miller-Rabin test
 * (bases 2..37) of each surviving partner, in ascending p.  Synchronous. */
int gb_query(gb_ctx* ctx, uint64_t n, uint32_t* p_min);

/* count queries at once (one CTA per n): n and p_min are host or device
 * arrays of count entries; P as for gb_verify_range's bound (0: the context's
 * max(p1, p2)), at most the base primes.  Any invalid n gives GB_EINVAL (its
 * p_min is 0; the others are still computed).  Synchronous. */
int gb_query_batch(gb_ctx* ctx, const uint64_t* n, uint32_t count, uint32_t P, uint32_t* p_min);

/* ---------------------------------------------------------------- serving
 * A request loop with continuous batching.  The server owns lanes + 1
 * contexts made from ctx by gb_init_shared (shared base primes, one stream
 * each), each driven by a host thread.  Ranges enter a FIFO queue: a free
 * range lane (lanes of them) admits the ranges at its head that fit in the
 * free part of the device-memory budget (at most max_batch; a range larger
 * than the whole budget runs alone) and runs them as one gb_verify_batch
 * call; ranges that arrive meanwhile are admitted by the next free lane, so
 * their work overlaps on the GPU.  Single-n queries enter a queue of their
 * own, served by the extra lane on a stream of the highest priority: every
 * queued query (at most max_batch) as one gb_query_batch call, so a query
 * never waits behind ranges on the host.  Results do not depend on the
 * batching.  ctx must outlive the server and must not be used while the
 * server runs. */
#define GB_REQ_RANGE 0   /* verify every even n in [lo, hi) (at most 2^32 n) */
#define GB_REQ_QUERY 1   /* p_min(n) for n = lo */
typedef struct gb_request {
    uint32_t kind;
    uint32_t reserved;
    uint64_t lo, hi;
} gb_request;
typedef struct gb_response {
    int32_t status;             /* GB_OK or the error of the call that served it */
    uint32_t p_min;             /* GB_REQ_QUERY: p_min(n), 0 if none <= P */
    gb_segment_result range;    /* GB_REQ_RANGE: the range's record */
    double t_submit_us;         /* host steady clock, microseconds since the */
    double t_start_us;          /* server was created: submitted, its batch */
    double t_done_us;           /* started, its batch finished */
} gb_response;
typedef struct gb_server gb_server;
/* lanes (range lanes) 1..16; hbm_budget_bytes 0 = half of the device memory free at
 * creation (cudaMemGetInfo); max_batch 0 = 256 */
int gb_server_create(gb_server** out, gb_ctx* ctx, uint32_t lanes, uint64_t hbm_budget_bytes, uint32_t max_batch);
/* queue a request (GB_EINVAL if it is malformed or beyond base_limit^2;
 * GB_EBUSY if the server is stopping or refuses it at admission) */
int gb_server_submit(gb_server* srv, const gb_request* req, uint64_t* ticket);
/* cancel a request still waiting in its queue: its response carries status
 * GB_ECANCELED and can be collected with gb_server_wait.  GB_EBUSY if it is
 * no longer queued (taken by a lane, which runs it to the end, or finished),
 * GB_EINVAL for a ticket that was never issued. */
int gb_server_cancel(gb_server* srv, uint64_t ticket);
/* wait for a ticket's response (each ticket can be collected once);
 * GB_ETIMEOUT if it is not done within timeout_ms */
int gb_server_wait(gb_server* srv, uint64_t ticket, gb_response* out, uint32_t timeout_ms);
int gb_server_stats(gb_server* srv, uint64_t* submitted, uint64_t* completed, uint64_t* batches,
                    uint64_t* in_flight_max_bytes);
/* finishes every queued request, then stops the lanes */
void gb_server_destroy(gb_server* srv);

/* Goldbach partition counts (Sec. 4.5, future work there): counts[j] = r(n)
 * for n = lo + 2j in [lo, hi), r(n) = the number of prime pairs p <= q with
 * p + q = n (r(4) = 1, r(100) = 6).  Computed on the GPU from the odd-only
 * prime bitset of [1, hi) and its bit-reversed copy: for each n, popcount of
 * the AND of the bitset with the reversed one shifted to n, over p <= n/2
 * (about n/128 word steps per n).  lo even >= 4, hi even, hi <= 2^34 and
 * hi <= base_limit^2, at most 2^28 n per call; counts host or device.
 * Synchronous. */
int gb_partitions(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t* counts);

/* gb_verify_range without memory allocation (the paper has no counterpart:
 * this is a calling convention of this library).  Some callers must not call
 * cudaMalloc while they run -- it can synchronize the device and stall every
 * stream, which a latency-bound request loop sharing the GPU cannot afford,
 * and a caller working inside a memory budget granted up front may not
 * allocate at all.  gb_verify_range may grow the context's device arenas on
 * a call; this entry point never allocates: its per-call scratch is one
 * file-scope device array of GB_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.
 *
 * Same arguments, outputs and results as gb_verify_range, with these limits
 * (beyond them: GB_ERANGE, nothing computed):
 *   - at most GB_NOALLOC_MAX_N even n, all in one segment (n <= seg_len);
 *   - final bound max(P, p2) at most GB_NOALLOC_MAX_P;
 *   - seg_hist_stride at most GB_NOALLOC_MAX_STRIDE;
 *   - out->pmin, if given, must be device memory (GB_EINVAL otherwise).
 * The large sieving primes always take the kernels that strike in place,
 * whatever GB_LARGE asks for (the bucket lists are arenas sized on use).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not keep using the library
 * across a cudaDeviceReset of that device (the kept address would be stale).
 * All calls share the one array: each clears what must start at zero, and
 * calls whose work overlaps on the GPU (other streams, other threads) race. */
#define GB_NOALLOC_SCRATCH_BYTES (4u << 20)
#define GB_NOALLOC_MAX_N         (1u << 22)
#define GB_NOALLOC_MAX_P         (1u << 20)
#define GB_NOALLOC_MAX_STRIDE    (1u << 17)
int gb_verify_range_noalloc(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t P,
                            gb_range_result* out);

/* Per-kernel device time, measured with CUDA events recorded on the
 * context's stream around every launch while profiling is enabled.  Kinds:
 * 0 segment sieve, tile part (units: q bits sieved), 1 cover (units: even n;
 * batched mode: q bits), 2 retry pass (units: even n of the slabs it ran on),
 * 3 reductions and the max-only pass (units: segments), 4 segment sieve,
 * primes above the tile split (units: q bits).  gb_profile_enable resets the
 * counters.  enable: 0 off; 1 (or any other nonzero value) event times and
 * the kernels' work counters (gb_profile_work); GB_PROFILE_EVENTS event
 * times alone, so that the timed kernels are exactly the ones that run with
 * profiling off (the work counters cost the strike loops an add per strike). */
#define GB_PROF_KINDS 5
#define GB_PROFILE_EVENTS 2
int gb_profile_enable(gb_ctx* ctx, int enable);
int gb_profile_read(gb_ctx* ctx, double* ms, uint64_t* launches, uint64_t* units);

/* Work counted by the kernels while profiling is enabled: bits struck by the
 * segment sieve's tile part (every strike of a prime >= 47 below the tile
 * split, duplicates included; primes 3..43 are stamped from patterns); the
 * cover's steps: for the two-phase kernel, first-phase (32-bit word, prime)
 * steps plus second-phase (n, prime) probes; for the generic kernel, the sum
 * over 64-n words of the number of primes applied until the word filled (the
 * bound's count for a word left open); and the bits struck by the primes
 * above the tile split. */
int gb_profile_work(gb_ctx* ctx, uint64_t* sieve_strikes, uint64_t* cover_iterations, uint64_t* large_strikes);

/* Kernels launched by verification calls of this context since the last
 * gb_profile_enable (counted whether or not profiling is on). */
int gb_profile_kernels(gb_ctx* ctx, uint64_t* kernels);

/* Debug builds (the library compiled with -DGB_DEBUG, libgb_debug.so): the
 * kernels check their shared- and global-memory strikes and bucket writes
 * against the bounds of their buffers; a failed check records its site
 * (1 tile strike, 2 slice strike, 3 large-prime strike, 4 carried strike,
 * 5 bucket entry) in a device word and skips the access instead of trapping.
 * gb_debug_word returns the first recorded site, 0 if none (always 0 in a
 * release build), and clears the words if reset is nonzero.  It synchronizes
 * with the device.  gb_debug_build is 1 in a debug build, 0 otherwise. */
uint32_t gb_debug_word(int reset);
int gb_debug_build(void);

/* Host-side fault injection, for tests of the error paths (the paper has no
 * counterpart).  Every fault is made on the host, none on the GPU: spec
 * "kind@n[,kind@n...]" makes the n-th event of that kind from now on fail,
 * with kind
 *   alloc   a device or pinned-host allocation of the library: the call that
 *           needed it returns GB_ENOMEM without calling the allocator (the
 *           context stays usable);
 *   submit  gb_server_submit: refused at admission with GB_EBUSY;
 *   cancel  gb_server_submit: the request is queued, then cancelled at once
 *           as by gb_server_cancel (its response carries GB_ECANCELED).
 * NULL or "" clears every fault.  The GB_FAULT environment variable, if set,
 * is applied at the first gb_init of the process.  GB_EINVAL for a malformed
 * spec (the faults in force do not change). */
#define GB_FAULT_ALLOC  0
#define GB_FAULT_SUBMIT 1
#define GB_FAULT_CANCEL 2
int gb_fault_set(const char* spec);
/* count one event of the kind against the spec in force: 1 if it is the one
 * that fails (the check the library makes at each allocation and submit) */
int gb_fault_tick(int kind);

/* Bytes copied between host and device memory by the calls of this context
 * since the last gb_profile_enable (every cudaMemcpyAsync the library issues
 * for the caller: inputs and staged descriptors to the device, results and
 * the counters the host reads back to the host; counted whether or not
 * profiling is on).  Either pointer may be NULL. */
int gb_profile_copies(gb_ctx* ctx, uint64_t* h2d_bytes, uint64_t* d2h_bytes);

/* Device (cudaMalloc) and pinned host (cudaMallocHost) allocations the
 * library has made in this process so far, and their total bytes: a call
 * allocated nothing iff the count is the same before and after it.  Either
 * pointer may be NULL. */
void gb_alloc_stats(uint64_t* count, uint64_t* bytes);

/* Bytes of the odd-only dense bitset for the odd numbers 3..N (Sec. 2.2):
 * ceil(#odd in [3, N] / 64) 64-bit words.  Host-only helper. */
uint64_t gb_bitset_bytes(uint64_t N);

/* Name of a GB_* code. */
const char* gb_strerror(int code);

/* Last error message of the calling thread ("" if none). */
const char* gb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GB_H */
