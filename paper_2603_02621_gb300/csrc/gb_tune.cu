// gb_tune.cu -- autotuner: picks the segment length, sieve tile, CTA size, the
// tile / large-prime split, the first-pass bound P and the cover's unrolled
// prefix for a sample workload by timing the real entry points (GoldbachGPU,
// arXiv 2603.02621: the segment length and P1 are the knobs of Sec. 2.3 and
// Sec. 2.4; the others are this implementation's).
//
// Coordinate descent: each parameter in turn (the sieve tile jointly with the
// split) is set to each of its candidates, the others held at the best so far; a candidate is timed as the best of
// `reps` runs after one warm-up run (which also sizes the arenas).  Outputs do
// not depend on any of these settings, so the search never changes a result.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "gb.h"

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer()
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// run the sample once under the context's current configuration
int run_sample(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, int mode,
               std::vector<gb_segment_result>& recs)
{
    if (mode == GB_TUNE_BATCH) return gb_verify_batch(ctx, lo, hi, count, 0, recs.data(), nullptr, 0);
    for (uint32_t i = 0; i < count; ++i) {
        gb_range_result r{};
        const int rc = gb_verify_range(ctx, lo[i], hi[i], 0, &r);
        if (rc) return rc;
    }
    return GB_OK;
}

// best-of-reps time of the sample under cfg; < 0 if the setting is rejected
double time_setting(gb_ctx* ctx, const gb_config& cfg, const uint64_t* lo, const uint64_t* hi, uint32_t count,
                    int mode, uint32_t reps, std::vector<gb_segment_result>& recs, Timer& t, int* err)
{
    *err = GB_OK;
    if (gb_set_config(ctx, &cfg) != GB_OK) return -1.0;
    cudaStream_t s = static_cast<cudaStream_t>(cfg.stream);
    int rc = run_sample(ctx, lo, hi, count, mode, recs);   // warm-up, arenas
    if (rc) {
        *err = rc;
        return -1.0;
    }
    double best = -1.0;
    for (uint32_t k = 0; k < reps; ++k) {
        cudaEventRecord(t.a, s);
        rc = run_sample(ctx, lo, hi, count, mode, recs);
        cudaEventRecord(t.b, s);
        if (rc) {
            *err = rc;
            return -1.0;
        }
        if (cudaEventSynchronize(t.b) != cudaSuccess) {
            *err = GB_ECUDA;
            return -1.0;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        if (best < 0 || ms < best) best = ms;
    }
    return best;
}

// key of a tuning result: the GPU (name and SM count), the mode, the
// settings that are not tuned (base primes, P2, slab) and the sample itself
// (count and an FNV-1a hash of its bounds)
std::string tune_key(const gb_config& c, int mode, const uint64_t* lo, const uint64_t* hi, uint32_t count)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, c.device) != cudaSuccess) {
        cudaGetLastError();
        std::snprintf(prop.name, sizeof prop.name, "unknown");
    }
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (uint32_t i = 0; i < count; ++i) {
        mix(lo[i]);
        mix(hi[i]);
    }
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == '|' || ch == '\t' || ch == '\n') ch = '_';
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s|%d|%d|%u|%016llx|%llu|%u|%llu", name.c_str(), prop.multiProcessorCount, mode,
                  count, (unsigned long long)h, (unsigned long long)c.base_limit, c.p2,
                  (unsigned long long)c.slab_bits);
    return buf;
}

}  // namespace

extern "C" int gb_tune_cache_lookup(const char* path, const char* key, gb_config* cfg, double* best_ms)
{
    if (!path || !key || !cfg) return GB_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return GB_ERANGE;
    char line[1024];
    int found = GB_ERANGE;
    const size_t klen = std::strlen(key);
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, key, klen) != 0 || line[klen] != '\t') continue;
        unsigned tile = 0, split = 0, p1 = 0, prefix = 0, seg = 0, cta = 0;
        double ms = 0;
        if (std::sscanf(line + klen + 1, "%u %u %u %u %u %u %lf", &tile, &split, &p1, &prefix, &seg, &cta, &ms) != 7)
            continue;                                      // a damaged line is skipped
        cfg->tile_bits = tile;
        cfg->bucket_split = split;
        cfg->p1 = p1;
        cfg->cover_prefix = prefix;
        cfg->seg_len = seg;
        cfg->cta_threads = cta;
        if (best_ms) *best_ms = ms;
        found = GB_OK;                                     // the last entry for a key wins
    }
    std::fclose(f);
    return found;
}

extern "C" int gb_tune_cache_store(const char* path, const char* key, const gb_config* cfg, double best_ms)
{
    if (!path || !key || !cfg || std::strchr(key, '\t') || std::strchr(key, '\n')) return GB_EINVAL;
    FILE* f = std::fopen(path, "a");
    if (!f) return GB_EINVAL;
    const int n = std::fprintf(f, "%s\t%u %u %u %u %u %u %.6f\n", key, cfg->tile_bits, cfg->bucket_split, cfg->p1,
                               cfg->cover_prefix, cfg->seg_len, cfg->cta_threads, best_ms);
    const int rc = std::fclose(f);
    return (n > 0 && rc == 0) ? GB_OK : GB_EINVAL;
}

extern "C" int gb_autotune(gb_ctx* ctx, const uint64_t* lo, const uint64_t* hi, uint32_t count, int mode,
                           uint32_t reps, gb_config* out, double* best_ms)
{
    if (!ctx || !lo || !hi || count == 0) return GB_EINVAL;
    if (mode != GB_TUNE_PLAIN && mode != GB_TUNE_BATCH) return GB_EINVAL;
    if (reps == 0) reps = 2;
    gb_config best{};
    int rc = gb_get_config(ctx, &best);
    if (rc) return rc;
    const gb_config start = best;
    // a result for this GPU, mode, setting and sample in the cache file
    const char* cache = std::getenv("GB_TUNE_CACHE");
    std::string key;
    if (cache && *cache) {
        key = tune_key(best, mode, lo, hi, count);
        gb_config hitc = best;
        double ms = 0;
        if (gb_tune_cache_lookup(cache, key.c_str(), &hitc, &ms) == GB_OK && gb_set_config(ctx, &hitc) == GB_OK) {
            if (out) *out = hitc;
            if (best_ms) *best_ms = ms;
            return GB_OK;
        }
    }
    std::vector<gb_segment_result> recs(mode == GB_TUNE_BATCH ? count : 0);
    Timer t;
    int err = GB_OK;
    double best_t = time_setting(ctx, best, lo, hi, count, mode, reps, recs, t, &err);
    if (best_t < 0) {
        gb_set_config(ctx, &start);
        return err ? err : GB_EINVAL;
    }

    uint64_t longest = 0;
    for (uint32_t i = 0; i < count; ++i) longest = std::max(longest, (hi[i] - lo[i]) / 2);

    // candidates of one parameter, given the best setting so far
    using Apply = std::function<bool(gb_config&, uint32_t)>;
    struct Param {
        std::vector<uint32_t> values;
        Apply apply;
    };
    std::vector<Param> params;
    // tile and tile / large-prime split together: value = log2(tile) * 16 +
    // log2(split / tile) + 4 (split from tile / 16 to 16 tiles; at least 2^10)
    {
        std::vector<uint32_t> ts;
        for (uint32_t lt = 16; lt <= 20; ++lt)
            for (uint32_t m = 0; m <= 8; ++m) ts.push_back(lt * 16 + m);
        params.push_back({ts, [](gb_config& c, uint32_t v) {
                              const uint32_t lt = v / 16, m = v % 16;
                              c.tile_bits = 1u << lt;
                              const uint64_t split = (1ull << lt) << m >> 4;
                              if (split < (1u << 10)) return false;
                              c.bucket_split = (uint32_t)std::min<uint64_t>(split, 0xffffffffull);
                              return true;
                          }});
    }
    params.push_back({{1u << 11, 1u << 12, 1u << 13, 1u << 14, 1u << 15}, [](gb_config& c, uint32_t v) {
                          if (c.p2 && v >= c.p2) return false;
                          c.p1 = v;
                          return true;
                      }});
    params.push_back({{80, 112, 144, 176, 208, 240}, [](gb_config& c, uint32_t v) {
                          c.cover_prefix = v;
                          return true;
                      }});
    if (mode == GB_TUNE_PLAIN) {
        params.push_back({{1u << 22, 1u << 23, 1u << 24, 1u << 25, 1u << 26, 1u << 27},
                          [longest](gb_config& c, uint32_t v) {
                              if (v > 2 * std::max<uint64_t>(longest, 1u << 22)) return false;
                              c.seg_len = v;
                              return true;
                          }});
    }
    // the tile sieve's CTA size (plain and persistent batched launches alike)
    params.push_back({{128, 256, 512}, [](gb_config& c, uint32_t v) {
                          c.cta_threads = v;
                          return true;
                      }});

    for (const Param& p : params) {
        for (uint32_t v : p.values) {
            gb_config c = best;
            if (!p.apply(c, v)) continue;
            if (std::memcmp(&c, &best, sizeof c) == 0) continue;
            const double ms = time_setting(ctx, c, lo, hi, count, mode, reps, recs, t, &err);
            if (err && err != GB_EINVAL) {
                gb_set_config(ctx, &start);
                return err;
            }
            if (ms >= 0 && ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
    }
    rc = gb_set_config(ctx, &best);
    if (rc) return rc;
    if (!key.empty()) gb_tune_cache_store(cache, key.c_str(), &best, best_t);   // a cache that cannot be written is skipped
    if (out) *out = best;
    if (best_ms) *best_ms = best_t;
    return GB_OK;
}
