// Context layout and host-side helpers shared by the C-ABI translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <utility>
#include <map>
#include <vector>

#include "kgpu_internal.h"

namespace kgpu {

// One slot of the batch ring (kgpu_submit): the paper's statically allocated,
// rotating pinned buffers (section 3.2), here four of them.  Each slot owns its
// pinned staging area, its device copy, a status array and an instantiated
// CUDA graph {copy in, reset counter and status, persistent kernel, copy
// status out}.
struct BatchSlot {
    uint64_t gen = 0;            // generation of the last ticket issued on this slot
    bool issued = false;
    cudaEvent_t done = nullptr;  // recorded after the graph
    uint8_t* h_buf = nullptr;    // pinned: header | descriptors | tile prefix
    uint8_t* d_buf = nullptr;
    size_t cap = 0;              // bytes of h_buf / d_buf
    int* d_status = nullptr;
    int* h_status = nullptr;     // pinned
    size_t status_cap = 0;       // entries
    unsigned long long* d_fin = nullptr;   // per request: tiles finished
    unsigned long long* h_done = nullptr;  // pinned, mapped: per-request completion words
    unsigned long long* d_done = nullptr;  // the device's view of h_done
    uint32_t tag = 0;                      // completion tag of the slot's current batch
    int pollers = 0;                       // kgpu_poll / kgpu_poll_each calls holding the slot
    unsigned long long* d_counter = nullptr;
    uint4* d_scratch = nullptr;  // per-warp staging for CBC encryption of host pages
    uint32_t scratch_warps = 0;
    uint32_t nreq = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_copy = nullptr, n_status_clear = nullptr, n_fin_clear = nullptr, n_kernel = nullptr,
                    n_status_out = nullptr;
    int graph_threads = 0, graph_grid = 0;
    BatchArgs args{};
};

constexpr int kBatchSlots = 4;

// A batch whose slot was reused by a later submission: it had completed (the
// submission waited for it), and this is what its polls still report.
struct RetiredBatch {
    uint32_t n = 0;                                // requests
    std::vector<std::pair<uint32_t, int>> failed;  // (request, KGPU_E* status) of the failed ones
};
constexpr size_t kRetiredKept = 4096;  // the newest retired batches are kept

// Serving state (kgpu_serve_*): the mapped host ring, the device counters and
// the host's bookkeeping of what is in flight.
struct ServeState {
    bool started = false;
    // Calls reading the ring's mapped words outside serve_mu (kgpu_serve_poll,
    // kgpu_replay_serve): kgpu_serve_stop frees the ring only once none is
    // left, and after it sets `stopping` they return instead of waiting.
    int readers = 0;
    bool stopping = false;
    bool closing = false;  // a kgpu_serve_stop is under way: further stops wait for it, submits are refused
    bool running = false;  // a kernel instance was launched and has not been seen to exit
    cudaStream_t stream = nullptr;
    cudaEvent_t kdone = nullptr;
    uint8_t* host_mem = nullptr;  // pinned, mapped: hdr | slots | done_seq | status | stamps
    uint8_t* dev_mem = nullptr;   // ServeDev | claim | fin
    ServeHostHdr* hdr = nullptr;
    ServeSlot* slots = nullptr;
    unsigned long long* done_seq = nullptr;
    int* status = nullptr;
    // the device's %globaltimer stamps of each slot's request: [0] dispatcher
    // took it, [1] tiles published, [2] first tile started, [3] completed
    static constexpr int kStamps = 4;
    unsigned long long* stamp[kStamps] = {};
    ServeArgs args{};
    uint32_t nslots = 0;
    uint64_t tile_ring = 0;  // entries of the device tile ring
    uint32_t tile_chunks = 8;
    uint64_t admit_bytes = 0;
    uint64_t next_seq = 0;
    uint64_t inflight_bytes = 0;
    std::vector<uint8_t> slot_busy;
    std::vector<uint64_t> slot_seq, slot_len;
    std::vector<uint64_t> outstanding;  // seqs published and not yet seen complete
    // slot_gen[s]: the seq staged in slot s, UINT64_MAX while stage() clears
    // the slot's mapped status and stamps -- a sequence lock that lets readers
    // without serve_mu tell whether what they read is still their request's.
    std::vector<uint64_t> slot_gen;
    // What the device reported for the last request each slot retired, copied
    // by reap -- always before the slot is staged again -- so a late reader
    // still finds it.  ret_seq[s] is the record's sequence lock (UINT64_MAX
    // while reap rewrites it).
    std::vector<uint64_t> ret_seq, ret_stamp[kStamps];
    std::vector<int> ret_status;
    std::map<uint64_t, int> failed;  // seq -> KGPU_E* of failed requests (the newest kFailedKept)
    uint64_t submitted = 0, completed = 0, busy_refusals = 0, launches = 0;
    uint64_t last_alive_check = 0;  // ns; publish re-checks the kernel at most every 20 us
    uint64_t last_publish_ns = 0;   // host time of the newest ring-head store
    unsigned last_exit = 0;
};

// A served request's completion callback, waiting for the request to complete.
struct ServeCallback {
    uint64_t seq = 0;
    kgpu_done_fn fn = nullptr;
    void* arg = nullptr;
};

// A host range registered with kgpu_host_register: [base, end) is page-locked
// and mapped for the context's device, where it is seen at base + dev_off.
struct HostRange {
    uintptr_t base = 0, end = 0;
    intptr_t dev_off = 0;
    bool owned = false;  // the library page-locked it and unlocks it again
};

}  // namespace kgpu

struct kgpu_ctx {
    int device = 0;
    int num_sms = 0;
    kgpu_config cfg{};
    std::mutex mu;
    std::vector<kgpu::HostKey> keys;
    kgpu::DevKey* d_keys = nullptr;
    uint32_t key_gen = 0;         // generation stamped on the last key set (under mu)
    cudaStream_t key_stream = nullptr;  // private non-blocking stream for key-table writes

    // host-resident pipeline (kgpu_aes_xts_crypt_host): three device staging
    // buffers on three streams -- one chunk being copied in, one transformed,
    // one copied out (the GPU-side triple buffering of the paper's section 3.2)
    static constexpr int kStages = 3;
    std::mutex host_mu;
    cudaStream_t hs[kStages] = {};
    uint8_t* staging[kStages] = {};
    size_t staging_bytes = 0;

    // batched submission (kgpu_submit / kgpu_poll)
    std::mutex batch_mu;
    kgpu::BatchSlot slots[kgpu::kBatchSlots];
    std::map<uint64_t, kgpu::RetiredBatch> retired;  // by ticket; guarded by batch_mu
    uint64_t next_ticket = 0;
    kgpu_tuning tune{};
    // the newest kgpu_submit_noalloc batch: recorded on the caller's stream
    // after its launch (guarded by batch_mu), waited on by batches_quiesce
    cudaEvent_t noalloc_done = nullptr;
    bool noalloc_issued = false;

    // kgpu_crypt: the measured crossover and the stream of its GPU leg's batches
    std::mutex dispatch_mu;
    kgpu_crossover xover{};
    cudaStream_t crypt_stream = nullptr;

    // serving loop (kgpu_serve_*)
    std::mutex serve_mu;
    kgpu::ServeState serve;

    // completion callbacks of served requests (kgpu_serve_submit_cb): one
    // thread per ring, started by the first such submit and joined before the
    // ring is freed.  cb_mu is taken after serve_mu, never before it.
    std::mutex cb_mu;
    std::condition_variable cb_cv;
    std::vector<kgpu::ServeCallback> cb_pending;  // under cb_mu
    bool cb_stop = false;                         // under cb_mu: deliver what is left and exit
    std::thread cb_thread;                        // started and joined under serve_mu

    // registered host ranges, sorted by base and disjoint
    std::mutex hreg_mu;
    std::vector<kgpu::HostRange> hreg;
};


namespace kgpu {
namespace hostutil {

constexpr int kVersion = (0 << 16) | 3;

// Makes ctx's device current for the scope (and binds its primary context to
// the calling thread, which the driver-API range check needs on threads that
// have made no CUDA call yet); restores the previous device afterwards.
class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
};

inline int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return KGPU_OK;
    if (e == cudaErrorMemoryAllocation) return KGPU_ENOMEM;
    return KGPU_EIO;
}

// cuMemGetAddressRange through the runtime's driver entry-point table, so the
// library has no link-time dependency on libcuda (it loads on GPU-less hosts).
typedef CUresult (*AddressRangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);

inline AddressRangeFn address_range_fn() {
    static AddressRangeFn fn = []() -> AddressRangeFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<AddressRangeFn>(f);
    }();
    return fn;
}

// The device allocation containing p: it must be device (or managed) memory of
// ctx's device.  [base, base + size) is the whole allocation.
inline int device_allocation(const kgpu_ctx* ctx, const void* p, uintptr_t* base, size_t* size) {
    if (!p) return KGPU_EFAULT;
    DeviceGuard g(ctx->device);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EFAULT;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return KGPU_EFAULT;
    if (a.type == cudaMemoryTypeDevice && a.device != ctx->device) return KGPU_EFAULT;
    CUdeviceptr b = 0;
    size_t sz = 0;
    AddressRangeFn range = address_range_fn();
    if (!range || range(&b, &sz, (CUdeviceptr)p) != CUDA_SUCCESS) return KGPU_EFAULT;
    *base = (uintptr_t)b;
    *size = sz;
    return KGPU_OK;
}

// [p, p + len) must lie inside one device allocation of ctx's device.
inline int check_device_range(const kgpu_ctx* ctx, const void* p, size_t len) {
    uintptr_t base = 0;
    size_t size = 0;
    int rc = device_allocation(ctx, p, &base, &size);
    if (rc) return rc;
    uintptr_t end = (uintptr_t)p + len;
    if (end < (uintptr_t)p || end > base + size) return KGPU_EFAULT;
    return KGPU_OK;
}

inline int check_host_ptr(const void* p) {
    if (!p) return KGPU_EFAULT;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EFAULT;
    }
    if (a.type == cudaMemoryTypeDevice) return KGPU_EFAULT;
    return KGPU_OK;
}

// src == dst, or disjoint; 16-byte aligned.
inline int check_pair(const void* src, const void* dst, size_t len) {
    uintptr_t s = (uintptr_t)src, d = (uintptr_t)dst;
    if ((s | d) & 15) return KGPU_EINVAL;
    if (s != d && s < d + len && d < s + len) return KGPU_EINVAL;
    return KGPU_OK;
}

inline int get_key(kgpu_ctx* ctx, kgpu_key h, bool want_xts, HostKey* out) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (h == 0 || h > ctx->keys.size()) return KGPU_ENOENT;
    const HostKey& k = ctx->keys[h - 1];
    if (!k.live || k.xts != want_xts) return KGPU_ENOENT;
    *out = k;
    return KGPU_OK;
}

// stealing: data units that are not a multiple of 16 bytes (at least 16) are
// allowed and end with ciphertext stealing.
inline int xts_args(kgpu_ctx* ctx, int dir, size_t len, size_t du, uint64_t first_sector, bool stealing = false) {
    if (!ctx) return KGPU_EINVAL;
    if (dir != KGPU_ENCRYPT && dir != KGPU_DECRYPT) return KGPU_EINVAL;
    if (du < 16 || (du % 16 && !stealing) || len % du) return KGPU_EINVAL;
    if (du / 16 > 0xFFFFFFFFull) return KGPU_EINVAL;
    uint64_t units = len / du;
    if (units && first_sector + (units - 1) < first_sector) return KGPU_EINVAL;  // 64-bit unit numbers
    return KGPU_OK;
}

inline void fill_bulk(BulkParams* p, const HostKey& k, int dir, const void* src, void* dst, size_t len, size_t du,
               uint64_t first_sector) {
    std::memset(p, 0, sizeof(*p));
    p->src = static_cast<const uint4*>(src);
    p->dst = static_cast<uint4*>(dst);
    p->nblocks = len / 16;
    p->bps = (uint32_t)(du / 16);
    p->first_sector = first_sector;
    std::memcpy(p->rk, dir == KGPU_ENCRYPT ? k.enc : k.dec, sizeof(p->rk));
    std::memcpy(p->tk, k.twk, sizeof(p->tk));
}


// Validated allocation ranges, built afresh for every call so that a range is
// never trusted after the caller could have freed it.
struct RangeCache {
    std::vector<std::pair<uintptr_t, uintptr_t>> r;
    int check(const kgpu_ctx* ctx, const void* p, size_t len) {
        uintptr_t a = (uintptr_t)p, e = a + len;
        if (!p || e < a) return KGPU_EFAULT;
        for (auto& x : r)
            if (a >= x.first && e <= x.second) return KGPU_OK;
        uintptr_t base = 0;
        size_t size = 0;
        int rc = device_allocation(ctx, p, &base, &size);
        if (rc) return rc;
        r.emplace_back(base, base + size);
        return e <= base + size ? KGPU_OK : KGPU_EFAULT;
    }
};

// [p, p + len) must lie inside one registered host range; *dev receives the
// address the device sees for p.  Takes a lock and allocates nothing.
inline int host_translate(kgpu_ctx* ctx, const void* p, size_t len, uintptr_t* dev) {
    uintptr_t a = (uintptr_t)p, e = a + len;
    if (!p || e < a) return KGPU_EFAULT;
    std::lock_guard<std::mutex> g(ctx->hreg_mu);
    auto it = std::upper_bound(ctx->hreg.begin(), ctx->hreg.end(), a,
                               [](uintptr_t x, const HostRange& r) { return x < r.base; });
    if (it == ctx->hreg.begin()) return KGPU_EFAULT;
    --it;
    if (a < it->base || e > it->end) return KGPU_EFAULT;
    *dev = (uintptr_t)((intptr_t)a + it->dev_off);
    return KGPU_OK;
}

// The device-visible address of a request buffer: device memory checked
// through the cache, or registered host memory when `host` is set.
template <class Cache>
int resolve_buffer(kgpu_ctx* ctx, Cache& rc, const void* p, size_t len, bool host, uintptr_t* dev) {
    if (host) return host_translate(ctx, p, len, dev);
    int r = rc.check(ctx, p, len);
    if (!r) *dev = (uintptr_t)p;
    return r;
}

constexpr uint32_t kReqFlagsAll = KGPU_REQ_SRC_HOST | KGPU_REQ_DST_HOST | KGPU_REQ_IVS_HOST;

// Work units per tile for a tile of tile_chunks 512-byte chunks: XTS/ECB
// count 32-block chunks; CBC decryption whole pages of about the same bytes;
// CBC encryption 32 pages, one chain per lane.
inline void set_tile_units(ReqDesc& d, uint32_t tile_chunks) {
    if (d.mode == KGPU_MODE_COPY) {
        d.tile_units = 1;  // the caller's unit_size is the tile
    } else if (d.mode == KGPU_MODE_CBC_ENC) {
        d.tile_units = 32;
    } else if (d.mode == KGPU_MODE_CBC_DEC) {
        uint64_t ppt = (uint64_t)tile_chunks * 32 / d.unit_blocks;
        d.tile_units = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(ppt, 1u << 30));
    } else {
        d.tile_units = std::max<uint32_t>(1, tile_chunks);
    }
}

// Validate one request and write its device descriptor (tile size in 512-B
// chunks for XTS/ECB; CBC tiles derive from it).  Cache: anything with
// int check(const kgpu_ctx*, const void*, size_t) -- RangeCache, or a
// fixed-capacity cache where the caller must not allocate.
// Whether a batch holds CBC encryption of registered host pages (run through
// the per-warp staging of the 512-thread batch kernel).
inline bool needs_staging(const kgpu_request* reqs, size_t n) {
    for (size_t i = 0; i < n; i++)
        if (reqs[i].mode == KGPU_MODE_CBC_ENC && (reqs[i].flags & (KGPU_REQ_SRC_HOST | KGPU_REQ_DST_HOST)))
            return true;
    return false;
}

template <class Cache>
int make_desc(kgpu_ctx* ctx, const kgpu_request& q, Cache& rc, uint32_t tile_chunks, ReqDesc* d) {
    std::memset(d, 0, sizeof(*d));
    if (q.flags & ~kReqFlagsAll) return KGPU_EINVAL;
    const bool cbc = q.mode == KGPU_MODE_CBC_DEC || q.mode == KGPU_MODE_CBC_ENC;
    const bool xts = q.mode == KGPU_MODE_XTS;
    const bool copy = q.mode == KGPU_MODE_COPY;
    if (!xts && !cbc && !copy && q.mode != KGPU_MODE_ECB) return KGPU_EINVAL;
    if ((xts || q.mode == KGPU_MODE_ECB) && q.dir != KGPU_ENCRYPT && q.dir != KGPU_DECRYPT) return KGPU_EINVAL;
    uint64_t unit = q.mode == KGPU_MODE_ECB ? 16 : q.unit_size;
    if (unit == 0 || unit % 16 || q.len % unit || unit / 16 > 0xFFFFFFFFull) return KGPU_EINVAL;
    if (xts) {
        uint64_t units = q.len / unit;
        if (units && q.sector + (units - 1) < q.sector) return KGPU_EINVAL;
    }
    if (!copy) {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (q.key == 0 || q.key > ctx->keys.size()) return KGPU_ENOENT;
        const HostKey& k = ctx->keys[q.key - 1];
        if (!k.live || k.xts != xts) return KGPU_ENOENT;
    }
    uintptr_t src = (uintptr_t)q.src, dst = (uintptr_t)q.dst, ivs = (uintptr_t)q.ivs;
    if (q.len) {
        int r = check_pair(q.src, q.dst, q.len);
        if (r) return r;
        if ((r = resolve_buffer(ctx, rc, q.src, q.len, q.flags & KGPU_REQ_SRC_HOST, &src)) ||
            (r = resolve_buffer(ctx, rc, q.dst, q.len, q.flags & KGPU_REQ_DST_HOST, &dst)))
            return r;
        // in place means the same bytes, wherever they are seen from
        if ((src == dst) != (q.src == q.dst)) return KGPU_EINVAL;
        if (cbc) {
            uint64_t npages = q.len / unit;
            if ((uintptr_t)q.ivs & 15) return KGPU_EINVAL;
            if ((r = resolve_buffer(ctx, rc, q.ivs, npages * 16, q.flags & KGPU_REQ_IVS_HOST, &ivs))) return r;
            uintptr_t iv0 = ivs, iv1 = iv0 + npages * 16;
            if (iv0 < dst + q.len && dst < iv1) return KGPU_EINVAL;
        }
        if (src != dst && src < dst + q.len && dst < src + q.len) return KGPU_EINVAL;
    }
    d->src = reinterpret_cast<const uint4*>(src);
    d->dst = reinterpret_cast<uint4*>(dst);
    d->ivs = reinterpret_cast<const uint4*>(ivs);
    d->nblocks = q.len / 16;
    d->first_sector = q.sector;
    d->unit_blocks = (uint32_t)(unit / 16);
    d->key = copy ? 0u : q.key - 1;
    d->mode = q.mode;
    d->dir = cbc ? (q.mode == KGPU_MODE_CBC_DEC ? 1u : 0u) : copy ? 0u : q.dir;
    d->flags = ((q.flags & KGPU_REQ_SRC_HOST) ? kDescSrcHost : 0u) | ((q.flags & KGPU_REQ_DST_HOST) ? kDescDstHost : 0u);
    set_tile_units(*d, tile_chunks);
    return KGPU_OK;
}


// Run order and tile prefix of a packed batch (descs already written; codes[i]
// nonzero marks request i refused, which contributes no tiles).
//
// A request's latency inside a batch is the time until its last tile is done,
// and tiles are handed out in run order, so requests run smallest first (the
// shortest-processing-time rule, which minimises the mean completion time):
// the many small requests of a mixed batch finish early instead of wherever
// the caller happened to put them.  Where a request sits does not move the
// batch's end as long as the last tiles handed out are short: XTS, ECB and
// CBC-decryption tiles are all about one tile of work, but a CBC-encryption
// tile is 32 serial chains of a page's blocks, several times longer, and one
// handed out last runs alone at the end.  So every CBC-encryption request
// runs before the tail reserve, the largest other requests holding their
// last reserve_tiles tiles (two per resident warp: enough short work to keep
// every warp busy while the long tiles finish).  Ties keep submission order.
// Allocation-free.  Returns the total tile count.
template <class Codes>
uint64_t order_batch(const ReqDesc* descs, uint32_t n, const Codes& codes, uint64_t reserve_tiles, uint64_t* prefix,
                     uint32_t* order) {
    auto tiles_of = [&](uint32_t i) -> uint64_t {
        return codes(i) ? 0 : (request_units(descs[i]) + descs[i].tile_units - 1) / descs[i].tile_units;
    };
    auto cbc_enc = [&](uint32_t i) { return descs[i].mode == KGPU_MODE_CBC_ENC; };
    // 1. fewest tiles first, ties in submission order.  prefix[0, n) holds
    // each request's tiles meanwhile.  Tile counts are usually small, and
    // then a counting sort (stable by construction) does it in one pass;
    // otherwise an in-place comparison sort on (tiles, index).
    constexpr uint32_t kBuckets = 1024;
    uint64_t max_tiles = 0;
    for (uint32_t i = 0; i < n; i++) {
        prefix[i] = tiles_of(i);
        max_tiles = std::max(max_tiles, prefix[i]);
    }
    if (max_tiles < kBuckets) {
        uint32_t start[kBuckets + 1] = {};
        for (uint32_t i = 0; i < n; i++) start[prefix[i] + 1]++;
        for (uint32_t b = 0; b < kBuckets; b++) start[b + 1] += start[b];
        for (uint32_t i = 0; i < n; i++) order[start[prefix[i]]++] = i;
    } else {  // a request of 1,024 tiles or more
        for (uint32_t i = 0; i < n; i++) order[i] = i;
        std::sort(order, order + n,
                  [&](uint32_t a, uint32_t b) { return prefix[a] != prefix[b] ? prefix[a] < prefix[b] : a < b; });
    }
    // 2. the tail reserve order[r, n): its CBC-encryption requests move in
    // front of the rest, both groups keeping their order
    uint32_t r = n;
    for (uint64_t held = 0; r > 0 && held < reserve_tiles; --r)
        if (!cbc_enc(order[r - 1])) held += prefix[order[r - 1]];
    uint32_t w = r;
    for (uint32_t j = r; j < n; j++)  // prefix[r, n) is free from here: the staging area
        prefix[j] = order[j];
    for (uint32_t j = r; j < n; j++)
        if (cbc_enc((uint32_t)prefix[j])) order[w++] = (uint32_t)prefix[j];
    for (uint32_t j = r; j < n; j++)
        if (!cbc_enc((uint32_t)prefix[j])) order[w++] = (uint32_t)prefix[j];
    // 3. exclusive prefix of tiles in run order
    uint64_t tiles = 0;
    for (uint32_t j = 0; j < n; j++) {
        prefix[j] = tiles;
        tiles += tiles_of(order[j]);
    }
    prefix[n] = tiles;
    return tiles;
}

void destroy_batch_slots(kgpu_ctx* ctx);  // kgpu_batch_api.cu
int destroy_serve(kgpu_ctx* ctx);         // kgpu_serve_api.cu; KGPU_EINVAL on the completion thread
// Wait until every request published to the serving ring so far has completed
// (no-op when serving is off).  kgpu_serve_api.cu.
int serve_quiesce(kgpu_ctx* ctx, int64_t timeout_ns);
// Wait for every issued batch slot.  kgpu_batch_api.cu.
int batches_quiesce(kgpu_ctx* ctx);

}  // namespace hostutil
}  // namespace kgpu
