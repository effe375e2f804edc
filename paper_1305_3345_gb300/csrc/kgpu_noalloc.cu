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

// Layout of the fixed scratch: the work counter, the per-request status
// words, the device copy of the packed batch, then the staging areas of
// kStageWarps warps for CBC encryption of registered host pages.
constexpr size_t kCounterOff = 0;
constexpr size_t kStatusOff = 256;
constexpr size_t kBatchOff = kStatusOff + ((KGPU_NOALLOC_MAX_REQUESTS * sizeof(int) + 255) / 256) * 256;
constexpr size_t kStageOff = 45056;
constexpr uint32_t kStageWarps = KGPU_NOALLOC_STAGE_WARPS;
static_assert(kBatchOff + batch_bytes(KGPU_NOALLOC_MAX_REQUESTS) <= kStageOff,
              "the fixed scratch must hold the largest batch");
static_assert(kStageOff % 256 == 0 && kStageOff + kStageWarps * kStageWarpBytes <= KGPU_NOALLOC_SCRATCH_BYTES,
              "the fixed scratch must hold the staging areas");

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol, never a device address: the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KGPU_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Host staging for the packed batch, in pageable memory.  This relies on the
// CUDA runtime's documented behaviour for an asynchronous copy from pageable
// host memory to device memory: the call returns once the source has been
// copied into the runtime's own staging memory, and only the DMA to the
// device may still be pending.  Under that assumption the array can be
// refilled as soon as the copy call returns, so one array serves every call in
// turn under g_pack_mu.  (A stream being captured into a graph breaks the
// assumption -- the graph would keep this address -- so such calls are
// refused.)
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
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        // a capturing stream (or, for the legacy stream, a capture elsewhere)
        cudaGetLastError();
        return KGPU_EINVAL;
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_on(ctx, &scratch);
    if (rc) return rc;

    // batch_mu is held from validation to the event record, so a key deletion
    // or a host unregistration either sees this batch's event or runs wholly
    // before its validation
    std::lock_guard<std::mutex> blk(ctx->batch_mu);
    const kgpu_tuning t = ctx->tune;
    uint32_t threads = t.threads ? t.threads : kBatchDefaultThreads;
    const uint32_t tile_chunks = t.tile_chunks ? t.tile_chunks : kBatchDefaultTileChunks;
    const uint32_t ctas = t.ctas ? t.ctas : (uint32_t)ctx->num_sms;
    // CBC encryption of host pages is staged only in the 512-thread kernel
    if (threads > 512 && needs_staging(reqs, n)) threads = 512;

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

    BatchArgs a{};
    a.buf = scratch + kBatchOff;
    a.keys = ctx->d_keys;
    a.max_keys = ctx->cfg.max_keys;
    a.next_tile = reinterpret_cast<unsigned long long*>(scratch + kCounterOff);
    a.status = reinterpret_cast<int*>(scratch + kStatusOff);
    // the first kStageWarps warps of the launch stage host-page CBC
    // encryption; the others run it one lane per page (same bytes, slower)
    a.scratch = reinterpret_cast<uint4*>(scratch + kStageOff);
    a.scratch_warps = kStageWarps;
    // the counter and the status words must start at zero on every call
    if (cudaMemcpyAsync(scratch + kBatchOff, g_pack, batch_bytes((uint32_t)n), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(scratch, 0, kStatusOff + n * sizeof(int), s) != cudaSuccess ||
        launch_batch(a, (int)threads, (int)ctas, s) != cudaSuccess ||
        cudaEventRecord(ctx->noalloc_done, s) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    ctx->noalloc_issued = true;
    return KGPU_OK;
}
