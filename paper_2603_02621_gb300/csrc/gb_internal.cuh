// gb_internal.cuh -- device helpers and kernel launchers shared by the
// translation units of libgb (segment sieve, Goldbach cover, runtime).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

typedef struct gb_ctx gb_ctx;

namespace gb {

// ---------------------------------------------------------------------------
// Pre-sieve patterns for the primes 3..43 (stamp of the segment sieve).
// Odd number v = 2x + 1 is divisible by the odd prime p iff x = (p-1)/2 mod p.
// Four periodic patterns over x: {3,5,7,11,13} (period 15015), {17,19} (323),
// {23,29,31} (20677) and {37,41,43} (65231); a tile word is the AND of the four,
// each read at x mod its period.
// ---------------------------------------------------------------------------
constexpr uint32_t kWheelM1 = 15015u;       // 3*5*7*11*13
constexpr uint32_t kWheelM2 = 323u;         // 17*19
constexpr uint32_t kWheelM3 = 20677u;       // 23*29*31
constexpr uint32_t kWheelM4 = 65231u;       // 37*41*43
constexpr uint32_t kWheelW1 = 472u;         // uint32 words holding bits [0, M1 + 64)
constexpr uint32_t kWheelW2 = 13u;          // uint32 words holding bits [0, M2 + 64)
constexpr uint32_t kWheelW3 = 650u;         // uint32 words holding bits [0, M3 + 64)
constexpr uint32_t kWheelW4 = 2042u;        // uint32 words holding bits [0, M4 + 64)
constexpr uint32_t kWheelWords = kWheelW1 + kWheelW2 + kWheelW3 + kWheelW4;   // 3177, +3 pad
constexpr uint32_t kStampedPrimes = 14u;    // 3 .. 43 come from the stamp
constexpr uint32_t kFirstStrikeIdx = 14u;   // index of 47 in 2,3,5,7,...,43,47,...

// Debug builds (-DGB_DEBUG): device-side bounds checks.  GB_DCHECK(cond,
// site) is cond; when it is false the check records the first failing site
// (a kDbg* code) in a device word of its translation unit and the caller
// skips the access -- no trap, the context stays usable.  gb_debug_word reads
// (and may clear) the words of every translation unit.  Release builds:
// always true, no code.
enum {
    kDbgTileStrike = 1, kDbgMidStrike = 2, kDbgLargeStrike = 3, kDbgCarryStrike = 4, kDbgCarryRing = 5,
};
#ifdef GB_DEBUG
int debug_register(uint32_t (*reader)(bool reset));
namespace {
__device__ unsigned int g_debug_word = 0;
uint32_t debug_read_tu(bool reset)
{
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_debug_word, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_debug_word, &z, sizeof z);
    }
    return v;
}
const int g_debug_registered = debug_register(debug_read_tu);
}  // namespace
#define GB_DCHECK(cond, site) ((cond) || (atomicCAS(&::gb::g_debug_word, 0u, (unsigned)(site)), false))
#else
#define GB_DCHECK(cond, site) true
#endif

// Host-side fault injection (gb_fault.cu): fault_hit counts one event of the
// kind (GB_FAULT_ALLOC, _SUBMIT, _CANCEL) and is true for the one the spec in
// force makes fail; fault_from_env applies GB_FAULT once per process.
bool fault_hit(int kind);
void fault_from_env();

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// looked up once per device ordinal); grids of persistent or grid-stride
// kernels are sized as multiples of it.  1 if the query fails.
uint32_t device_sms();

// Barrett reduction (P. Barrett, CRYPTO '86): with m = floor((2^64-1)/p), the
// quotient estimate hi64(x*m) is at most 2 below floor(x/p); two conditional
// subtractions finish the remainder.  p < 2^32, any 64-bit x.
__device__ __forceinline__ uint32_t barrett_mod(uint64_t x, uint32_t p, uint64_t m)
{
    uint64_t q = __umul64hi(x, m);
    uint64_t r = x - q * (uint64_t)p;
    if (r >= p) r -= p;
    if (r >= p) r -= p;
    return (uint32_t)r;
}

// (-b) mod p in [0, p), b any signed 64-bit value
__device__ __forceinline__ uint32_t neg_mod(int64_t b, uint32_t p, uint64_t m)
{
    if (b <= 0) return barrett_mod((uint64_t)(-b), p, m);
    uint32_t t = barrett_mod((uint64_t)b, p, m);
    return t ? p - t : 0u;
}

// Index i >= 0 of the first odd multiple of p in the odd-number sequence
// b, b+2, b+4, ... (b odd): 2i = -b (mod p), i < p.
__device__ __forceinline__ uint32_t first_odd_multiple(int64_t b, uint32_t p, uint64_t m)
{
    uint32_t r = neg_mod(b, p, m);
    return (r & 1u) ? (uint32_t)(((uint64_t)r + p) >> 1) : (r >> 1);
}

// ---------------------------------------------------------------------------
// Segment sieve
// ---------------------------------------------------------------------------
struct SieveArgs {
    int64_t  B;                 // odd number of bit 0
    uint64_t nbits;             // bits produced (a multiple of 64 is written per tile)
    uint32_t tile_bits;         // bits per CTA tile (multiple of 8192)
    const uint32_t* primes;     // sieving primes, ascending, starting at 23
    const uint64_t* recip;      // Barrett reciprocals of the same primes
    uint32_t n_warp;            // primes [0, n_warp): one warp strikes each
    uint32_t n_primes;          // primes [n_warp, n_primes): one thread each
    const uint32_t* wheel;      // the four stamp tables, kWheelWords words
    uint32_t* out;              // bit i -> word i/32, bit i%32 (NULL: count only)
    unsigned long long* popcount;   // optional total of 1 bits
    unsigned long long* strikes;    // optional: number of bits struck (work count)
};

// Strikes of the primes larger than a tile: one thread per prime, every odd
// multiple (>= p^2) in the bit range [bit_lo, bit_hi) of the window starting at
// the odd number B, cleared in place with global atomic AND.  Launched per
// chunk of the window small enough to stay in L2.
struct LargeArgs {
    int64_t  B;                 // odd number of bit 0 of the window
    uint64_t bit_lo, bit_hi;    // chunk of the window to strike
    const uint32_t* primes;     // the large primes
    const uint64_t* recip;      // their Barrett reciprocals
    uint32_t n_primes;
    uint32_t* out;              // window words
    unsigned long long* strikes;    // optional work count
    // optional (slices only): per prime {p, (-B) mod p, (2 kMidSliceBits) mod p,
    // floor(2^33 / p)}, filled by launch_mid before the slices run; needs fewer
    // than kMidResSlices slices and primes below 2^20 (NULL: a Barrett
    // reduction per prime and slice)
    uint4* res;
};
cudaError_t launch_large(const LargeArgs& a, cudaStream_t s);
// the same primes struck per slice of the window in shared memory (one
// Barrett start per prime and slice): for primes up to a few slices, whose
// strikes are dense enough to pay for the starts (LargeArgs: bit_lo / bit_hi
// unused, the whole window).  A slice is 224 KB of shared memory, nearly all
// an SM has, so that the starts -- most of the kernel's instructions -- are
// as few as they can be.
constexpr uint32_t kMidSliceBits = 7u << 18;
// slices per window for the residue starts (slice index x (2 kMidSliceBits mod p) < 2^33)
constexpr uint32_t kMidResSlices = 1u << 13;
cudaError_t launch_mid(const LargeArgs& a, uint64_t nbits, cudaStream_t s);
// Primes from the slice limit to sqrt(B) over a window of several chunks of
// 2^chunk_log2 bits (gb_large.cu): each prime started once per window and
// carried from chunk to chunk -- per-prime next-multiple words for the primes
// below half a chunk, a ring of per-chunk buckets for the larger ones -- with
// the multiples m p, m coprime to 210, struck by global atomic AND.
struct BucketLargeArgs {
    int64_t  B;                 // odd number of bit 0 of the window, with p^2 <= B for every prime
    uint64_t nbits;             // window bits
    uint32_t chunk_log2;        // chunk bits 2^chunk_log2 (<= 2^28)
    uint32_t nchunks;           // ceil(nbits / chunk)
    uint32_t B_mod210;          // B mod 210
    const uint32_t* primes;     // [0, n_dense): below half a chunk; then n_sparse larger ones, all below 2^31
    const uint64_t* recip;      // their Barrett reciprocals
    uint32_t n_dense, n_sparse;
    uint32_t* dstate;           // [n_dense]: next multiple's offset in the current chunk
    uint8_t* dpos;              // [n_dense]: its wheel position (0 .. 47, mod 210)
    uint64_t* ring;             // [R][grid][cap] entries: p / 2 << 34 | wheel position << 28 | offset in the chunk
    uint32_t* ring_cnt;         // [R][grid] entries per bucket column (zeroed before the start kernel)
    uint32_t ring_mask;         // R - 1; R > 1 + 5 max(p) / chunk + 1, R <= kCarryMaxRing
    uint32_t grid;              // CTAs of every launch (carry_grid()): one bucket column each
    uint32_t cap;               // entries per bucket column
    uint32_t* out;              // window words
    unsigned long long* strikes;    // optional work count
    unsigned int* spills;       // entries that found their column full (struck through to the window end)
};
constexpr uint32_t kCarryMaxRing = 64;
uint32_t carry_grid();
cudaError_t launch_large_start(const BucketLargeArgs& a, cudaStream_t s);
cudaError_t launch_large_chunk(const BucketLargeArgs& a, uint32_t c, cudaStream_t s);
// population count of n 32-bit words, added to *count
cudaError_t launch_popcount(const uint32_t* words, uint64_t n, unsigned long long* count, cudaStream_t s);

cudaError_t launch_wheel_tables(uint32_t* wheel /*kWheelWords*/, cudaStream_t s);
cudaError_t launch_seed_sieve(uint32_t* words /*1024*/, cudaStream_t s);
cudaError_t launch_sieve(const SieveArgs& a, int threads, cudaStream_t s);

// Compaction of an odd-only bitset (bit i <-> number B + 2i) into the list of
// its primes, ascending, written after a leading 2; plus Barrett reciprocals.
struct CompactArgs {
    const uint32_t* words;
    uint64_t nwords;
    int64_t  B;
    uint32_t* counts;           // scratch: one per chunk
    uint32_t* primes;           // out: [2, odd primes...]
    uint64_t* recip;            // out: floor((2^64-1)/p) per entry of primes
};
uint64_t compact_chunks(uint64_t nwords);
cudaError_t launch_compact(const CompactArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Goldbach cover
// ---------------------------------------------------------------------------
struct RetryItem {
    uint64_t w;                 // slab word index (64 even n per word)
    uint64_t C;                 // coverage bits after the first pass
};

struct CoverArgs {
    const uint64_t* Q;          // q window: bit i <-> odd number A0 - H + 1 + 2i
    uint32_t H;                 // halo, even, > every p of the pass
    uint64_t n_count;           // even n in the slab
    uint64_t n_words;           // ceil(n_count / 64)
    uint32_t words_per_seg;     // S / 64
    uint32_t cta_words;         // words per CTA (multiple of 32)
    uint32_t chunks_per_seg;    // ceil(words_per_seg / cta_words)
    uint32_t nseg;              // segments in the slab
    const uint32_t* primes;     // [2, 3, 5, ...]
    uint32_t K;                 // odd primes used: primes[1 .. K]
    uint32_t hist_stride;       // per-segment histogram row length
    uint32_t* hist;             // [nseg][hist_stride], prime-index histogram
    unsigned long long* maxkey; // [nseg]: (pidx+1) << 32 | (0xffffffff - j)
    unsigned long long* unresolved; // [nseg]
    uint32_t* pmin;             // optional, slab-relative n index
    RetryItem* retry;           // optional: words left with zero bits go here
    unsigned int* retry_count;
    uint32_t retry_cap;
    int has_n4;                 // slab starts at n = 4 (p_min(4) = 2)
    unsigned long long* iters;  // optional: sum over words of the primes applied
                                // until the word filled (work count)
    // generic kernel only: "max only" mode recomputes the segment maximum of
    // segments whose key in maxkey_check is still 0 and writes it to maxkey
    int max_only;
    const unsigned long long* maxkey_check;
    // block cover only (set by the launcher): blocks of 32 primes after block 0
    uint32_t n_later;
    uint32_t cum_wt[3];         // 1, 2^10, 2^20: weights of the packed 10-bit counters
};
cudaError_t launch_cover(const CoverArgs& a, int threads, cudaStream_t s);

// Block cover (k_cover_fast): unrolled blocks, the first (48 or 64 primes)
// over every 32-bit coverage word, each later one (32 primes) over the words
// still open; then, in the same kernel, each n still open probes the primes
// KA+1 .. K in order (KA = 48 or 64 + 32 x later blocks, at most 256; 48 when
// KA = 16 mod 32).  Needs K >= KA, H = 4 (mod 64) and no p_min array.
int cover_fast_phase_primes(uint32_t K, uint64_t n_hi);   // KA for K primes near n_hi (0: none)
bool cover_prefix_valid(int KA);
cudaError_t launch_cover_fast(const CoverArgs& a, int KA, cudaStream_t s);

// Sieve and block cover fused per CTA (k_seg_cover): the window is sieved
// tile by tile into shared memory (sv.out and sv.popcount null, sv.tile_bits
// == kFusedTileBits, no primes above the split) and covered there.
constexpr uint32_t kFusedTileBits = (1u << 18) + 8192;
uint32_t seg_cover_offset(uint32_t H, uint32_t P1);     // first window word the cover reads, per chunk
cudaError_t launch_seg_cover(const CoverArgs& a, const SieveArgs& sv, int KA, uint32_t P1, cudaStream_t s);

struct RetryArgs {
    const uint64_t* Q;
    uint32_t H;
    uint32_t words_per_seg;
    const uint32_t* primes;
    uint32_t K1, K2;            // odd-prime indices (1-based in primes[]) K1 < k <= K2
    uint32_t hist_stride;
    uint32_t* hist;
    unsigned long long* maxkey;
    unsigned long long* unresolved;
    uint32_t* pmin;
    const RetryItem* items;
    const unsigned int* count;
    uint32_t cap;
};
cudaError_t launch_retry(const RetryArgs& a, cudaStream_t s);

// Per-segment summary written by the reduce kernel (device layout, also the
// staging layout copied to the host).
struct SegSummary {
    uint64_t unresolved;
    uint64_t max_j;             // segment-relative n index of max_pmin
    uint32_t max_pmin;
    uint32_t hist_len;
};

struct ReduceArgs {
    uint32_t nseg;
    uint32_t hist_stride;
    const uint32_t* hist;
    const unsigned long long* maxkey;
    const unsigned long long* maxkey2;  // optional second key per segment (max-only pass)
    const unsigned long long* unresolved;
    const uint32_t* primes;
    SegSummary* summary;        // [nseg]
    uint64_t* rows;             // optional [nrows][row_stride] uint64 copy
    uint32_t row_stride;
    uint32_t nrows;             // rows written (<= nseg)
    unsigned long long* merged; // [hist_stride] running sum over segments
};
cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s);

// Totals over all segments of a range (device), and the public per-segment
// records (gb_segment_result layout) written where the caller wants them.
struct RangeTotals {
    unsigned long long unresolved;
    unsigned long long max_pmin_n;
    uint32_t max_pmin;
    uint32_t hist_len;
};

struct SegRecord {              // identical layout to gb_segment_result
    uint64_t lo, hi, n_checked, unresolved, max_pmin_n;
    uint32_t max_pmin, hist_len;
};

struct FinalizeArgs {
    uint64_t lo, hi, S;
    uint32_t nseg;
    const SegSummary* summary;
    SegRecord* records;         // optional
    uint32_t nrecords;          // records written (<= nseg)
    RangeTotals* totals;
};
cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched mode: many ranges in one pass of persistent kernels.  Each range has
// its own q window inside one batch buffer; the work is split into items that
// persistent CTAs take from device queues (atomic heads).
// ---------------------------------------------------------------------------
struct BatchRange {
    uint64_t lo;                // first even n
    uint64_t n;                 // even n in the range
    int64_t  B;                 // odd number of bit 0 of its q window
    uint64_t nbits;             // q window bits
    uint64_t q_off;             // 64-bit word offset of the window in the batch buffer
};

// persistent sieve over (range, tile) items; the tile part of the primes only
struct SieveItemsArgs {
    SieveArgs base;             // tile_bits, primes, recip, n_warp, n_primes, wheel, strikes
    const BatchRange* ranges;
    const uint32_t* item_range; // per item: range index
    const uint32_t* item_tile;  // per item: tile index within the range's window
    const uint32_t* n_items;    // device count
    unsigned int* head;         // queue head
    uint32_t* Q;                // batch buffer (32-bit words)
};
cudaError_t launch_sieve_items(const SieveItemsArgs& a, int threads, cudaStream_t s);

// persistent block cover over (range, chunk) items; row r = range r
struct CoverItemsArgs {
    CoverArgs base;             // H, cta_words, primes, K, hist_stride, hist, maxkey, unresolved
    const BatchRange* ranges;
    const uint32_t* item_range;
    const uint32_t* item_chunk;
    const uint32_t* n_items;
    unsigned int* head;
    const uint64_t* Q;          // batch buffer
};
cudaError_t launch_cover_items(const CoverItemsArgs& a, int KA, cudaStream_t s);

// primes from the split below the mid limit over (range, shared-memory slice)
// items of a batch, in shared memory
struct MidItemsArgs {
    const BatchRange* ranges;
    const uint32_t* item_range;
    const uint32_t* item_slice;
    const uint32_t* n_items;    // device
    unsigned int* head;         // device queue head (zeroed)
    const uint32_t* primes;
    const uint64_t* recip;
    uint32_t n_primes;
    uint32_t* Q;                // batch buffer (32-bit words)
    unsigned long long* strikes;
};
cudaError_t launch_mid_items(const MidItemsArgs& a, cudaStream_t s);

// large primes over groups of window pieces (a group's pieces together fit in
// L2; a long window is cut into several pieces): items (group, block of 256
// primes), group-major, from a device queue; a thread stops at the first
// piece of its group that its prime does not reach
// a run of one range's window bits, at most an L2-sized chunk
struct LargePiece {
    uint32_t range;
    uint32_t n_primes;          // large primes with p^2 <= the piece's last number
    uint64_t bit_lo, bit_hi;
};
struct LargeBatchArgs {
    const BatchRange* ranges;
    const LargePiece* pieces;   // grouped; within a group by n_primes, descending
    const uint32_t* groups;     // device: first piece of each group, then the count
    uint32_t nblk;              // blocks of 256 primes per group (the most any piece needs)
    const uint32_t* n_items;    // device: groups x nblk
    unsigned int* head;         // device queue head (zeroed)
    const uint32_t* primes;     // the large primes
    const uint64_t* recip;
    uint32_t n_primes;
    uint32_t* Q;                // batch buffer (32-bit words)
    unsigned long long* strikes;
};
cudaError_t launch_large_batch(const LargeBatchArgs& a, cudaStream_t s);

struct ReduceBatchArgs {
    const BatchRange* ranges;
    const uint32_t* count;      // device: ranges in the batch
    const uint32_t* hist;       // [range][hist_stride]
    uint32_t hist_stride;
    const unsigned long long* maxkey;
    const unsigned long long* unresolved;
    const uint32_t* primes;
    SegRecord* records;         // [range]
    uint64_t* rows;             // optional [range][row_stride]
    uint32_t row_stride;
};
cudaError_t launch_reduce_batch(const ReduceBatchArgs& a, uint32_t grid, cudaStream_t s);

// Bucket sieve for the primes above the tile split (gb_bucket.cu): a chunk
// of at most kMaxBuckets bucket tiles of 2^kBucketTileLog2 bits; pieces are
// runs of window bits with their own number base (one piece for a plain
// window, one per range of a batch group)
constexpr uint32_t kBucketTileLog2 = 20;
constexpr uint32_t kMaxBuckets = 1024;
struct BucketPiece {
    int64_t B;                  // odd number of the window's bit 0
    uint64_t r_lo, r_hi;        // window bits [r_lo, r_hi) in this chunk
    uint64_t pos;               // chunk bit of window bit r_lo
};
struct BucketFillArgs {
    const BucketPiece* pieces;  // device array, or nullptr: the one piece `single`
    uint32_t n_pieces;
    BucketPiece single;
    uint32_t K;                 // bucket tiles in the chunk (<= kMaxBuckets)
    const uint32_t* primes;     // the large primes
    const uint64_t* recip;
    uint32_t n_primes;
    uint32_t* lists;            // [grid][K][cap] 20-bit offsets
    uint32_t* counts;           // [grid][K]
    uint32_t cap;
    unsigned int* overflow;     // set if a list overflowed (entries dropped)
    unsigned long long* strikes;
};
struct BucketApplyArgs {
    const uint32_t* lists;
    const uint32_t* counts;
    uint32_t G, K, cap;
    uint32_t* q;                // 32-bit word of the chunk's bit 0
    uint64_t span;              // chunk bits
};
uint32_t bucket_fill_grid();    // persistent fill CTAs on this device (0 on error)
size_t bucket_fill_smem(uint32_t K);
cudaError_t launch_bucket_fill(const BucketFillArgs& a, uint32_t grid, cudaStream_t s);
cudaError_t launch_bucket_apply(const BucketApplyArgs& a, cudaStream_t s);

// Goldbach partition counts (gb_partitions.cu)
struct PartitionArgs {
    const uint32_t* P;          // odd-only prime bits of [1, 64 * words / 2 ...): bit i <-> 2i + 1
    const uint32_t* rev;        // bit-reversed P, words + 1 entries (last one zero)
    uint64_t words;             // 32-bit words of P
    uint64_t lo;                // first even n
    uint64_t count;             // even n in the range
    uint64_t n_blocks;          // ceil(count / 32)
    uint64_t runs;              // word runs per n-block
    uint64_t run_words;         // words per run
    uint32_t* counts;           // [count], zeroed; r(n) added
};
cudaError_t launch_reverse_bits(const uint32_t* P, uint32_t* rev, uint64_t words, cudaStream_t s);
cudaError_t launch_partitions(const PartitionArgs& a, cudaStream_t s);

// Single-n queries (gb_query.cu): one CTA per n, p_min over primes[1..K]
struct QueryArgs {
    const uint64_t* n;          // device: even n, 4 <= n < 2^63
    uint32_t count;
    const uint32_t* primes;     // [2, 3, 5, ...]
    const uint64_t* recip;
    uint32_t n_filter;          // pre-sieve primes primes[1..n_filter] (all odd primes <= query_filter_max())
    uint32_t K;                 // candidates primes[1..K] (p <= P)
    uint32_t* out;              // device: p_min, 0 if no p <= P
    unsigned int* bad;          // device: count of invalid n (their out is 0)
};
cudaError_t launch_query(const QueryArgs& a, cudaStream_t s);
uint32_t query_filter_max();

// Read-only view of a context for entry points defined outside gb_api.cu.
struct CtxView {
    int device;
    cudaStream_t stream;
    uint64_t L;                 // primes known up to L
    uint32_t seg_len, p1, p2, cta_threads, tile_bits, bucket_split, warp_split;
    const uint32_t* primes;     // device [2, 3, 5, ...]
    const uint64_t* recip;      // device Barrett reciprocals
    const uint32_t* wheel;      // device stamp tables
    bool generic_cover;
    int ka_override;
    uint64_t large_chunk_bits;
};
int ctx_view(const gb_ctx* ctx, CtxView* v);
uint64_t ctx_pi(const gb_ctx* ctx, uint64_t x);            // primes <= x (x <= L)
// segment sieve of the odd numbers B + 2i, i < nbits, into out (device
// words), with no device allocation: the large primes take the kernels that
// strike in place (never the bucket lists, which are sized on first use)
int ctx_sieve_noalloc(gb_ctx* ctx, int64_t B, uint64_t nbits, uint32_t* out);
int set_error(int code, const char* msg);                 // records gb_last_error()

}  // namespace gb
