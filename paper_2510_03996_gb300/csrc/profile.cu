// profile.cu -- launch-level timing with CUDA events on the context's stream.
// While a profile is open, every kernel launch site records an event named
// after the kernel; the time between consecutive events is that launch's
// device time (the stream runs them in order).  Events are pooled and reused.
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace fheon {
namespace {
struct Prof {
    std::mutex mu;
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<const char *> names;
};
Prof &prof()
{
    static Prof *p = new Prof(); // never destroyed: events outlive static teardown order
    return *p;
}
} // namespace

void prof_mark(cudaStream_t st, const char *name)
{
    Prof &P = prof();
    if (!P.on) return;
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.on || st != P.st) return;
    if (P.used == P.pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        P.pool.push_back(e);
    }
    cudaEventRecord(P.pool[P.used++], st);
    P.names.push_back(name);
}
} // namespace fheon

using namespace fheon;

extern "C" {

int fheon_profile_begin(fheon_ctx *ctx)
{
    if (!ctx) return FHEON_ERR_ARG;
    Prof &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    P.on = true;
    P.st = ctx->stream;
    P.used = 0;
    P.names.clear();
    if (P.pool.empty()) {
        cudaEvent_t e;
        FHEON_CUDA(ctx, cudaEventCreate(&e));
        P.pool.push_back(e);
    }
    FHEON_CUDA(ctx, cudaEventRecord(P.pool[P.used++], ctx->stream));
    P.names.push_back("start");
    return FHEON_OK;
}

int fheon_profile_end(fheon_ctx *ctx, char *out, size_t cap)
{
    if (!ctx || !out || cap == 0) return FHEON_ERR_ARG;
    Prof &P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    P.on = false;
    FHEON_CUDA(ctx, cudaStreamSynchronize(P.st));
    std::map<std::string, std::pair<long, double>> agg;
    for (size_t i = 1; i < P.used; i++) {
        float ms = 0;
        FHEON_CUDA(ctx, cudaEventElapsedTime(&ms, P.pool[i - 1], P.pool[i]));
        auto &a = agg[P.names[i]];
        a.first += 1;
        a.second += ms;
    }
    std::string s = "{";
    for (auto &kv : agg) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s\"%s\": [%ld, %.6f]", s.size() > 1 ? ", " : "", kv.first.c_str(), kv.second.first,
                 kv.second.second);
        s += buf;
    }
    s += "}";
    if (s.size() + 1 > cap) return fail(ctx, FHEON_ERR_ARG, "profile buffer too small (%zu bytes needed)", s.size() + 1);
    memcpy(out, s.c_str(), s.size() + 1);
    return FHEON_OK;
}

} // extern "C"
