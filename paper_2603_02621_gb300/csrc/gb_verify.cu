// gb_verify.cu -- gb_verify_range: exhaustive verification of a range of
// even n (GoldbachGPU, arXiv 2603.02621, Sec. 2.3): the range is cut into
// segments of S even n (the unit of output) and slabs of whole segments (the
// unit of residency); per slab: segment sieve of the q window -> cover
// (p <= P1) -> retry (P1 < p <= P2) -> per-segment reduction; one copy of the
// results to the host at the end.
#include "gb_runtime.cuh"

extern "C" {

int gb_verify_range(gb_ctx* ctx, uint64_t lo, uint64_t hi, uint32_t P, gb_range_result* out)
{
    if (!ctx || !out) return fail(GB_EINVAL, "NULL argument");
    NvtxRange call_range("gb_verify_range");
    if ((lo & 1) || (hi & 1) || lo < 4 || hi <= lo) return fail(GB_EINVAL, "range must be even, lo >= 4, hi > lo");
    if (hi > GB_MAX_HI) return fail(GB_EINVAL, "hi beyond 2^63 - 2^26");
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
            GB_CUDA(ctx->copy(&cnt, ctx->retry_count.p, 4, cudaMemcpyDeviceToHost, s));
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
            GB_CUDA(ctx->copy(&cnt, ctx->retry_count.p, 4, cudaMemcpyDeviceToHost, s));
            GB_CUDA(cudaStreamSynchronize(s));
            if (cnt > retry_cap) overflow_total += cnt - retry_cap;
        }
        if (out->pmin && !pmin_dev)
            GB_CUDA(ctx->copy(out->pmin + s0 * S, pm, n_count * 4, cudaMemcpyDeviceToHost, s));
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
    GB_CUDA(ctx->copy(&tot, ctx->totals.p, sizeof tot, cudaMemcpyDeviceToHost, s));
    const uint32_t nh = out->hist ? std::min<uint32_t>(out->hist_cap, hist_stride) : 0;
    if (nh) GB_CUDA(ctx->copy(out->hist, ctx->merged.p, (size_t)nh * 8, cudaMemcpyDeviceToHost, s));
    const uint64_t nrec = out->segs ? std::min<uint64_t>(out->seg_cap, nseg) : 0;
    if (nrec && !segs_dev)
        GB_CUDA(ctx->copy(out->segs, ctx->records.p, nrec * sizeof(gb::SegRecord), cudaMemcpyDeviceToHost, s));
    if (rows_n && !rows_dev)
        GB_CUDA(ctx->copy(out->seg_hist, ctx->rows.p, rows_n * row_stride * 8, cudaMemcpyDeviceToHost, s));
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

}  // extern "C"
