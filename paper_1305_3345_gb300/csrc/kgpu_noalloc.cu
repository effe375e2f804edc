// kgpu_submit_noalloc: the batched path without any allocation.
//
// Some callers cannot allocate memory when they need the service: an OS-level
// caller on a page-writeback or memory-reclaim path (the kind of caller this
// service is built for) may be asked to encrypt pages precisely because memory
// is short, and an allocation there can block on the reclaim it is serving or
// fail outright; other callers run under a fixed memory budget that must not
// grow after start-up.  This entry point runs the same persistent batch kernel
// as kgpu_submit, but its scratch -- the work counter, the per-request status
// words and the device copy of the descriptors -- lives in one fixed array of
// device memory that is part of the library image (every GPU that loads the
// library holds it until the process exits), and the host side packs the
// descriptors into a fixed host array.  It calls no cudaMalloc, cudaFree or
// other allocating routine, and no host heap allocation either.
#include <cuda_runtime.h>

#include <mutex>

#include "kgpu_ctx.h"

using namespace kgpu;
using namespace kgpu::hostutil;

namespace {

constexpr size_t kCounterOff = 0;
constexpr size_t kStatusOff = 256;
constexpr size_t kBatchOff = kStatusOff + ((KGPU_NOALLOC_MAX_REQUESTS * sizeof(int) + 255) / 256) * 256;
static_assert(kBatchOff + batch_bytes(KGPU_NOALLOC_MAX_REQUESTS) <= KGPU_NOALLOC_SCRATCH_BYTES,
              "the fixed scratch must hold the largest batch");

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol, never a device address: the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KGPU_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Host staging for the packed batch (pageable; cudaMemcpyAsync has copied it
// out by the time it returns, so one array serves every call in turn).
std::mutex g_pack_mu;
alignas(256) unsigned char g_pack[batch_bytes(KGPU_NOALLOC_MAX_REQUESTS)];

// Validated allocation ranges for one call, in a fixed array.
struct FixedRangeCache {
    uintptr_t lo[16] = {}, hi[16] = {};
    int n = 0, next = 0;
    int check(const kgpu_ctx* ctx, const void* p, size_t len) {
        uintptr_t a = (uintptr_t)p, e = a + len;
        if (!p || e < a) return KGPU_EFAULT;
        for (int i = 0; i < n; i++)
            if (a >= lo[i] && e <= hi[i]) return KGPU_OK;
        uintptr_t base = 0;
        size_t size = 0;
        int rc = device_allocation(ctx, p, &base, &size);
        if (rc) return rc;
        int slot = n < 16 ? n++ : (next++ & 15);
        lo[slot] = base;
        hi[slot] = base + size;
        return e <= base + size ? KGPU_OK : KGPU_EFAULT;
    }
};

// Device address of the scratch on ctx's device; set up on the first call for
// that device, with the device current.
int scratch_on(const kgpu_ctx* ctx, unsigned char** out) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return KGPU_ENODEV;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[ctx->device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return KGPU_EIO;
        }
        g_scratch_dev[ctx->device] = ptr;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[ctx->device]);
    return KGPU_OK;
}

}  // namespace

extern "C" int kgpu_submit_noalloc(kgpu_ctx* ctx, const kgpu_request* reqs, size_t n, kgpu_stream stream,
                                   int* req_status) {
    if (!ctx || (n && !reqs)) return KGPU_EINVAL;
    if (n > KGPU_NOALLOC_MAX_REQUESTS) return KGPU_E2BIG;
    if (n == 0) return KGPU_OK;
    DeviceGuard g(ctx->device);
    unsigned char* scratch = nullptr;
    int rc = scratch_on(ctx, &scratch);
    if (rc) return rc;

    kgpu_tuning t;
    {
        std::lock_guard<std::mutex> lk(ctx->batch_mu);
        t = ctx->tune;
    }
    const uint32_t threads = t.threads ? t.threads : 1024;
    const uint32_t tile_chunks = t.tile_chunks ? t.tile_chunks : 32;
    const uint32_t ctas = t.ctas ? t.ctas : (uint32_t)ctx->num_sms;

    std::lock_guard<std::mutex> lk(g_pack_mu);
    FixedRangeCache cache;
    ReqDesc* descs = reinterpret_cast<ReqDesc*>(g_pack + batch_desc_offset());
    uint64_t* prefix = reinterpret_cast<uint64_t*>(g_pack + batch_prefix_offset((uint32_t)n));
    uint32_t* order = reinterpret_cast<uint32_t*>(g_pack + batch_order_offset((uint32_t)n));
    int first = KGPU_OK;
    for (size_t i = 0; i < n; i++) {
        int r = make_desc(ctx, reqs[i], cache, tile_chunks, &descs[i]);
        if (req_status) req_status[i] = r;
        if (r && !first) first = r;
    }
    if (first) return first;
    const uint64_t tiles = order_batch(descs, (uint32_t)n, [](uint32_t) { return false; },
                                       2 * (uint64_t)ctas * (threads / 32), prefix, order);
    BatchHeader* h = reinterpret_cast<BatchHeader*>(g_pack);
    h->total_tiles = tiles;
    h->nreq = (uint32_t)n;
    h->tag = 0;

    cudaStream_t s = (cudaStream_t)stream;
    BatchArgs a{};
    a.buf = scratch + kBatchOff;
    a.keys = ctx->d_keys;
    a.max_keys = ctx->cfg.max_keys;
    a.next_tile = reinterpret_cast<unsigned long long*>(scratch + kCounterOff);
    a.status = reinterpret_cast<int*>(scratch + kStatusOff);
    // the counter and the status words must start at zero on every call
    if (cudaMemcpyAsync(scratch + kBatchOff, g_pack, batch_bytes((uint32_t)n), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(scratch, 0, kStatusOff + n * sizeof(int), s) != cudaSuccess ||
        launch_batch(a, (int)threads, (int)ctas, s) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    return KGPU_OK;
}
