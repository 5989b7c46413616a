// gb_noalloc.cu -- gb_verify_range_noalloc: exhaustive verification of a small
// range with no memory allocation in the call.
//
// Who needs it: code that must not call cudaMalloc while it runs.  cudaMalloc
// can synchronize the device and stall every stream, which a latency-bound
// request loop or a caller sharing the GPU with time-critical work cannot
// afford; some callers (for example ones working inside a fixed memory budget
// granted up front, or running where a failed allocation cannot be handled)
// may not allocate at all.  gb_verify_range grows the context's device arenas
// on first use and so may allocate; this entry point instead takes its
// per-call scratch from one file-scope device array of fixed size.
//
// That array is a static __device__ object: every GPU that loads the library
// holds it (GB_NOALLOC_SCRATCH_BYTES) until the process exits.  Its host-side
// name is only a stand-in for the device object, so host code passes the
// address that cudaGetSymbolAddress returns for the current device, looked up
// once per device on the first call there.  All calls share the array: each
// call clears the parts that must start at zero, and two calls whose work
// overlaps on the GPU (different streams, or different threads without
// ordering) race on it.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "gb.h"
#include "gb_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (looked up once)
int scratch_address(int device, unsigned char** out)
{
    if (device < 0 || device >= kMaxDevices) return gb::set_error(GB_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return gb::set_error(GB_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
        }
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[device]);
    return GB_OK;
}

bool on_device(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// bump carve-out of the scratch array, 256-byte aligned pieces
struct Carve {
    unsigned char* base;
    size_t used = 0;
    void* take(size_t bytes)
    {
        void* p = base + used;
        used += (bytes + 255) & ~size_t(255);
        return p;
    }
};

uint64_t isqrt64(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        const uint64_t t = r | (1ull << b);
        if (t * t <= x) r = t;
    }
    return r;
}

#define NA_CUDA(call)                                                                             \
    do {                                                                                          \
        const cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                                    \
            return gb::set_error(GB_ECUDA, (std::string(#call) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

}  // namespace

extern "C" int gb_verify_range_noalloc(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t P, gb_range_result* out)
{
    if (!ctx || !out) return gb::set_error(GB_EINVAL, "NULL argument");
    if ((lo & 1) || (hi & 1) || lo < 4 || hi <= lo) return gb::set_error(GB_EINVAL, "range must be even, lo >= 4, hi > lo");
    if (hi > GB_MAX_HI) return gb::set_error(GB_EINVAL, "hi beyond 2^63 - 2^26");
    gb::CtxView v{};
    int rc = gb::ctx_view(ctx, &v);
    if (rc) return rc;
    const uint64_t n_total = (hi - lo) / 2;
    if (n_total > GB_NOALLOC_MAX_N)
        return gb::set_error(GB_ERANGE, "gb_verify_range_noalloc: more than GB_NOALLOC_MAX_N even n");
    if (n_total > v.seg_len)
        return gb::set_error(GB_ERANGE, "gb_verify_range_noalloc: the range must fit in one segment (seg_len)");
    const uint32_t P1 = P ? P : v.p1;
    if (P1 < 2 || P1 > (1u << 24) || P1 > v.L) return gb::set_error(GB_EINVAL, "P out of range");
    const bool retry = v.p2 > P1;
    const uint32_t Pf = retry ? v.p2 : P1;
    if (Pf > GB_NOALLOC_MAX_P) return gb::set_error(GB_ERANGE, "gb_verify_range_noalloc: bound above GB_NOALLOC_MAX_P");
    if (out->pmin && !on_device(out->pmin))
        return gb::set_error(GB_EINVAL, "gb_verify_range_noalloc: pmin must be device memory (or NULL)");
    const bool want_rows = out->seg_hist && out->seg_hist_stride;
    if (want_rows && out->seg_hist_stride > GB_NOALLOC_MAX_STRIDE)
        return gb::set_error(GB_ERANGE, "gb_verify_range_noalloc: seg_hist_stride above GB_NOALLOC_MAX_STRIDE");
    const uint32_t K1 = (uint32_t)(gb::ctx_pi(ctx, P1) - 1);
    const uint32_t Kf = (uint32_t)(gb::ctx_pi(ctx, Pf) - 1);
    const uint32_t H = 64 * ((Pf + 1 - 4 + 63) / 64) + 4;   // as gb_verify_range
    const uint64_t S = v.seg_len;
    const uint32_t hist_stride = Kf + 1;
    if (isqrt64(hi + 2 * 1024 + H) > v.L) return gb::set_error(GB_EINVAL, "hi beyond base_limit^2");

    NA_CUDA(cudaSetDevice(v.device));
    unsigned char* base = nullptr;
    if ((rc = scratch_address(v.device, &base))) return rc;
    cudaStream_t s = v.stream;

    // carve the scratch array
    const uint64_t n_words = (n_total + 63) / 64;
    const uint64_t qw = n_words + H / 128 + 2;
    const bool rows_dev = want_rows && on_device(out->seg_hist);
    const bool segs_dev = out->segs && on_device(out->segs);
    Carve c{base};
    uint64_t* Q = static_cast<uint64_t*>(c.take(qw * 8));
    uint32_t* hist = static_cast<uint32_t*>(c.take((size_t)hist_stride * 4));
    unsigned long long* small = static_cast<unsigned long long*>(c.take(8 * 8));
    unsigned long long* maxkey = small + 0;
    unsigned long long* unres = small + 1;
    unsigned int* counters = reinterpret_cast<unsigned int*>(small + 2);   // [0] retry items
    gb::RetryItem* items = static_cast<gb::RetryItem*>(c.take(n_words * sizeof(gb::RetryItem)));
    gb::SegSummary* summary = static_cast<gb::SegSummary*>(c.take(sizeof(gb::SegSummary)));
    gb::SegRecord* records = static_cast<gb::SegRecord*>(c.take(sizeof(gb::SegRecord)));
    gb::RangeTotals* totals = static_cast<gb::RangeTotals*>(c.take(sizeof(gb::RangeTotals)));
    unsigned long long* merged = static_cast<unsigned long long*>(c.take((size_t)hist_stride * 8));
    uint64_t* rows = want_rows && !rows_dev ? static_cast<uint64_t*>(c.take((size_t)out->seg_hist_stride * 8)) : nullptr;
    if (c.used > GB_NOALLOC_SCRATCH_BYTES)
        return gb::set_error(GB_ERANGE, "gb_verify_range_noalloc: request does not fit the scratch array");

    // what must start at zero
    NA_CUDA(cudaMemsetAsync(hist, 0, (size_t)hist_stride * 4, s));
    NA_CUDA(cudaMemsetAsync(small, 0, 8 * 8, s));
    NA_CUDA(cudaMemsetAsync(merged, 0, (size_t)hist_stride * 8, s));
    if (out->pmin) NA_CUDA(cudaMemsetAsync(out->pmin, 0, n_total * 4, s));

    // q window and cover: the same kernels and the same choices as gb_verify_range
    const int64_t B = (int64_t)lo - (int64_t)H + 1;
    if ((rc = gb::ctx_sieve_noalloc(ctx, B, qw * 64, reinterpret_cast<uint32_t*>(Q)))) return rc;
    gb::CoverArgs ca{};
    ca.Q = Q;
    ca.H = H;
    ca.n_count = n_total;
    ca.n_words = n_words;
    ca.words_per_seg = (uint32_t)(S / 64);
    ca.cta_words = (uint32_t)std::min<uint64_t>(2048, S / 64);
    ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
    ca.nseg = 1;
    ca.primes = v.primes;
    ca.K = K1;
    ca.hist_stride = hist_stride;
    ca.hist = hist;
    ca.maxkey = maxkey;
    ca.unresolved = unres;
    ca.pmin = out->pmin;
    ca.retry = retry ? items : nullptr;
    ca.retry_count = counters;
    ca.retry_cap = (uint32_t)n_words;
    ca.has_n4 = (lo == 4);
    int KA = (out->pmin || v.generic_cover || v.ka_override == 1) ? 0 : gb::cover_fast_phase_primes(K1, hi);
    if (KA && v.ka_override > 1 && (uint32_t)v.ka_override <= K1) KA = v.ka_override;
    if (KA) {
        ca.cta_words = (uint32_t)std::min<uint64_t>(3840, S / 64);
        ca.chunks_per_seg = (uint32_t)((S / 64 + ca.cta_words - 1) / ca.cta_words);
        NA_CUDA(gb::launch_cover_fast(ca, KA, s));
    } else {
        NA_CUDA(gb::launch_cover(ca, (int)v.cta_threads, s));
    }
    if (retry) {
        gb::RetryArgs ra{};
        ra.Q = Q;
        ra.H = H;
        ra.words_per_seg = ca.words_per_seg;
        ra.primes = v.primes;
        ra.K1 = K1;
        ra.K2 = Kf;
        ra.hist_stride = hist_stride;
        ra.hist = hist;
        ra.maxkey = maxkey;
        ra.unresolved = unres;
        ra.pmin = out->pmin;
        ra.items = items;
        ra.count = counters;
        ra.cap = (uint32_t)n_words;                          // one item per word at most: never full
        NA_CUDA(gb::launch_retry(ra, s));
    }
    const uint32_t row_stride = want_rows ? out->seg_hist_stride : 0;
    gb::ReduceArgs rd{};
    rd.nseg = 1;
    rd.hist_stride = hist_stride;
    rd.hist = hist;
    rd.maxkey = maxkey;
    rd.maxkey2 = nullptr;
    rd.unresolved = unres;
    rd.primes = v.primes;
    rd.summary = summary;
    rd.rows = want_rows ? (rows_dev ? out->seg_hist : rows) : nullptr;
    rd.row_stride = row_stride;
    rd.nrows = want_rows ? 1u : 0u;
    rd.merged = merged;
    NA_CUDA(gb::launch_reduce(rd, s));
    gb::FinalizeArgs fa{};
    fa.lo = lo;
    fa.hi = hi;
    fa.S = S;
    fa.nseg = 1;
    fa.summary = summary;
    fa.records = out->segs ? (segs_dev ? reinterpret_cast<gb::SegRecord*>(out->segs) : records) : nullptr;
    fa.nrecords = out->segs && out->seg_cap ? 1u : 0u;
    fa.totals = totals;
    NA_CUDA(gb::launch_finalize(fa, s));

    gb::RangeTotals tot{};
    NA_CUDA(cudaMemcpyAsync(&tot, totals, sizeof tot, cudaMemcpyDeviceToHost, s));
    const uint32_t nh = out->hist ? std::min<uint32_t>(out->hist_cap, hist_stride) : 0;
    if (nh) NA_CUDA(cudaMemcpyAsync(out->hist, merged, (size_t)nh * 8, cudaMemcpyDeviceToHost, s));
    if (out->segs && out->seg_cap && !segs_dev)
        NA_CUDA(cudaMemcpyAsync(out->segs, records, sizeof(gb::SegRecord), cudaMemcpyDeviceToHost, s));
    if (want_rows && !rows_dev)
        NA_CUDA(cudaMemcpyAsync(out->seg_hist, rows, (size_t)row_stride * 8, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (out->hist)
        for (uint32_t i = nh; i < out->hist_cap; ++i) out->hist[i] = 0;
    out->n_checked = n_total;
    out->n_segments = 1;
    out->p_final = Pf;
    out->unresolved = tot.unresolved;
    out->max_pmin = tot.max_pmin;
    out->max_pmin_n = tot.max_pmin_n;
    out->hist_len = tot.hist_len;
    const bool erange = (out->segs && out->seg_cap < 1) || (out->hist && out->hist_cap < out->hist_len) ||
                        (want_rows && row_stride < tot.hist_len);
    if (erange) return gb::set_error(GB_ERANGE, "an output buffer was too small; what fit was written");
    return GB_OK;
}
