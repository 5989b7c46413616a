// gb_batch_host.cu -- gb_verify_batch: many ranges of uneven length and
// offset in one pass (the segment loop of GoldbachGPU, arXiv 2603.02621,
// Sec. 2.3, over many ranges at once): descriptors and work items built on
// the host, the batch's kernels (gb_batch.cu, k_sieve_items, k_cover_items)
// captured as one CUDA graph.
#include "gb_runtime.cuh"

extern "C" {

int gb_verify_batch(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, uint32_t P,
                    gb_segment_result* results, uint64_t* hist, uint32_t hist_stride)
{
    if (!ctx || (count && (!lo || !hi || !results))) return fail(GB_EINVAL, "NULL argument");
    if (count == 0) return GB_OK;
    NvtxRange call_range("gb_verify_batch");
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
        if ((lo[i] & 1) || (hi[i] & 1) || lo[i] < 4 || hi[i] <= lo[i] || hi[i] > GB_MAX_HI)
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
    // the split strike per tile, those below the mid limit per 224 KB slice
    // of each window in shared memory, the rest per window piece by atomics
    const uint64_t np = ctx->pi(isqrt_u64(last_max));
    const uint32_t split = ctx->split(isqrt_u64(last_max));
    const uint64_t nsmall = std::min<uint64_t>(np, std::max<uint64_t>(ctx->pi(split - 1), gb::kFirstStrikeIdx));
    const uint64_t nmid = ctx->mid_limit > split
                              ? std::min<uint64_t>(np, std::max<uint64_t>(nsmall, ctx->pi(ctx->mid_limit - 1)))
                              : nsmall;
    uint64_t n_mid = 0;
    if (nmid > nsmall)
        for (uint32_t i = 0; i < count; ++i) {
            const uint64_t qw = (hi[i] - lo[i]) / 2 / 64 + 1 + H / 128 + 2;
            n_mid += (64 * qw + gb::kMidSliceBits - 1) / gb::kMidSliceBits;
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
                const uint64_t slices = (64 * qw + gb::kMidSliceBits - 1) / gb::kMidSliceBits;
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
    GB_CUDA(ctx->copy(dd, hs_p, used, cudaMemcpyHostToDevice, s));
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
    if (!KA) return fail(GB_EINVAL, "gb_verify_batch needs P >= the 48th odd prime (227)");

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
    GB_CUDA(ctx->copy(rec.data(), d_records, (size_t)count * sizeof(gb::SegRecord), cudaMemcpyDeviceToHost, s));
    if (want_rows && !rows_dev)
        GB_CUDA(ctx->copy(hist, ctx->brows.p, (size_t)count * hist_stride * 8, cudaMemcpyDeviceToHost, s));
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
                GB_CUDA(ctx->copy(reinterpret_cast<gb::SegRecord*>(results) + i, &r, sizeof r, cudaMemcpyHostToDevice, s));
            if (want_rows) {
                if (rows_dev)
                    GB_CUDA(ctx->copy(hist + (uint64_t)i * hist_stride, row.data(), (size_t)hist_stride * 8,
                                      cudaMemcpyHostToDevice, s));
                else
                    std::memcpy(hist + (uint64_t)i * hist_stride, row.data(), (size_t)hist_stride * 8);
            }
            if (res_dev || (want_rows && rows_dev)) GB_CUDA(cudaStreamSynchronize(s));   // r and row are reused
        }
        if (want_rows && r.hist_len > hist_stride) status = GB_ERANGE;
    }
    if (!res_dev) std::memcpy(results, rec.data(), (size_t)count * sizeof(gb::SegRecord));
    if (status == GB_ERANGE) return fail(GB_ERANGE, "a histogram row was longer than hist_stride");
    return GB_OK;
}

}  // extern "C"
