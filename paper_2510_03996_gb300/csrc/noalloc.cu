// noalloc.cu -- a rotation entry point that allocates no device memory.
//
// fheon_rotate draws its key-switching workspace from the allocator hook.
// Some callers cannot allocate at the moment they rotate: a serving process
// whose device memory is carved up once at start-up and must not grow, a
// latency-critical path that cannot afford cudaMalloc/cudaFree (cudaFree
// synchronises the whole device), or code that runs inside a stream capture,
// where allocation calls are not allowed.  fheon_rotate_noalloc serves them:
// the same rotation kernels, with the workspace taken from the fixed array
// below instead of the allocator.
//
// The array is a file-scope __device__ variable, so every GPU that loads this
// library reserves FHEON_NOALLOC_SCRATCH_BYTES (32 MiB) for it until the
// process exits.  All calls share it: two calls that overlap on the GPU (for
// instance on two streams) race on it.  Every workspace word a rotation reads
// was written earlier in the same rotation, so nothing has to be cleared
// between calls even though the array keeps the previous call's contents.
#include <mutex>

#include "internal.h"

#define FHEON_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned long long g_noalloc_scratch[FHEON_NOALLOC_SCRATCH_BYTES / 8];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
int scratch_address(fheon_ctx *ctx, unsigned long long **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fheon::cuda_fail(ctx, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fheon::fail(ctx, FHEON_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fheon::cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned long long *>(g_scratch_addr[dev]);
    return FHEON_OK;
}
} // namespace

extern "C" int fheon_rotate_noalloc(fheon_ctx *ctx, const fheon_ct *in, int32_t step, fheon_ct *out)
{
    if (!ctx || !in || !out) return FHEON_ERR_ARG;
    if (out == in) return fheon::fail(ctx, FHEON_ERR_ARG, "fheon_rotate_noalloc: output must not alias the input");
    const u32 l = in->level;
    const size_t need = ctx->ks_ws_limbs(l) * ctx->limb_bytes();
    if (need > FHEON_NOALLOC_SCRATCH_BYTES)
        return fheon::fail(ctx, FHEON_ERR_ARG,
                           "fheon_rotate_noalloc: level %u at N=%u needs %zu bytes of scratch, more than the fixed "
                           "%llu-byte array; use fheon_rotate",
                           l, ctx->N, need, (unsigned long long)FHEON_NOALLOC_SCRATCH_BYTES);
    if (!out->c.p || out->cap < l)
        return fheon::fail(ctx, FHEON_ERR_ARG,
                           "fheon_rotate_noalloc: output holds %u limbs per component, needs %u (create it with "
                           "fheon_ct_create at level >= %u)",
                           out->cap, l, l);
    const u64 g = fheon_galois_elt(ctx, step);
    auto it = ctx->keys.find(g);
    if (it == ctx->keys.end()) return fheon::fail(ctx, FHEON_ERR_NO_KEY, "no rotation key for step %d", step);
    unsigned long long *scratch = nullptr;
    int rc = scratch_address(ctx, &scratch);
    if (rc) return rc;
    out->level = l;
    out->scale = in->scale;
    return fheon::keyswitch_rotate(ctx, in->c0(), in->c1(ctx->N), l, g, it->second.mem.as<u64>(), scratch, out->c0());
}
