// gb_query_host.cu -- gb_query / gb_query_batch (GoldbachGPU, arXiv
// 2603.02621, Sec. 2.4) and gb_partitions (Sec. 4.5): argument checks,
// staging and the launches of the kernels in gb_query.cu and
// gb_partitions.cu.
#include "gb_runtime.cuh"

extern "C" {

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
        GB_CUDA(ctx->copy(ctx->qn.p, n, (size_t)count * 8, cudaMemcpyHostToDevice, s));
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
    GB_CUDA(ctx->copy(&h_bad, bad, 4, cudaMemcpyDeviceToHost, s));
    if (!out_dev) GB_CUDA(ctx->copy(p_min, qa.out, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
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
    if (!out_dev) GB_CUDA(ctx->copy(counts, d_out, count * 4, cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    return GB_OK;
}


int gb_query(gb_ctx* ctx, uint64_t n, uint32_t* p_min)
{
    if (!ctx || !p_min) return fail(GB_EINVAL, "NULL argument");
    return gb_query_batch(ctx, &n, 1, 0, p_min);
}

}  // extern "C"
