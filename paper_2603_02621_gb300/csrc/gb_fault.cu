// gb_fault.cu -- host-side fault injection (testing aid; the paper has no
// counterpart).  A fault is made on the host, never on the GPU: an
// allocation that reports failure without calling cudaMalloc, a request the
// server refuses at admission, a queued request cancelled before it runs.
// Nothing here launches a kernel or touches device memory.
//
// Spec: "kind@n[,kind@n...]" -- the n-th event of that kind from the time the
// spec is set fails (n >= 1); kinds: alloc, submit, cancel.  Set by
// gb_fault_set, or by the GB_FAULT environment variable at the first gb_init.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "gb.h"
#include "gb_internal.cuh"

namespace {

constexpr int kKinds = 3;
const char* const kNames[kKinds] = {"alloc", "submit", "cancel"};
std::atomic<uint64_t> g_seen[kKinds];       // events of each kind since the spec was set
std::atomic<uint64_t> g_when[kKinds];       // the event number that fails (0 = none)
std::once_flag g_env_once;

int parse(const char* spec, uint64_t when[kKinds])
{
    for (int k = 0; k < kKinds; ++k) when[k] = 0;
    if (!spec) return GB_OK;
    std::string s(spec);
    size_t pos = 0;
    while (pos < s.size()) {
        size_t end = s.find(',', pos);
        if (end == std::string::npos) end = s.size();
        const std::string item = s.substr(pos, end - pos);
        pos = end + 1;
        if (item.empty()) continue;
        const size_t at = item.find('@');
        if (at == std::string::npos) return GB_EINVAL;
        const std::string name = item.substr(0, at), num = item.substr(at + 1);
        int k = -1;
        for (int i = 0; i < kKinds; ++i)
            if (name == kNames[i]) k = i;
        if (k < 0 || num.empty() || num.size() > 18 || num.find_first_not_of("0123456789") != std::string::npos)
            return GB_EINVAL;
        const uint64_t n = std::strtoull(num.c_str(), nullptr, 10);
        if (n == 0) return GB_EINVAL;
        when[k] = n;
    }
    return GB_OK;
}

int apply(const char* spec)
{
    uint64_t when[kKinds];
    const int rc = parse(spec, when);
    if (rc) return gb::set_error(rc, "GB_FAULT: expected kind@n[,kind@n...], kind alloc, submit or cancel, n >= 1");
    for (int k = 0; k < kKinds; ++k) {
        g_seen[k].store(0);
        g_when[k].store(when[k]);
    }
    return GB_OK;
}

}  // namespace

namespace gb {

void fault_from_env()
{
    std::call_once(g_env_once, [] {
        if (const char* e = getenv("GB_FAULT")) apply(e);
    });
}

bool fault_hit(int kind)
{
    if (kind < 0 || kind >= kKinds) return false;
    const uint64_t w = g_when[kind].load(std::memory_order_relaxed);
    if (!w) return false;
    return g_seen[kind].fetch_add(1) + 1 == w;
}

}  // namespace gb

extern "C" int gb_fault_set(const char* spec)
{
    std::call_once(g_env_once, [] {});              // an explicit spec wins over the environment
    return apply(spec && *spec ? spec : nullptr);
}

extern "C" int gb_fault_tick(int kind)
{
    return gb::fault_hit(kind) ? 1 : 0;
}
