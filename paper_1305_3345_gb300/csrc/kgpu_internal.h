// Internal declarations shared by the library's translation units: kernel
// parameter blocks, device descriptor formats and launch helpers.  Not part of
// the public C ABI (that is include/kgpu.h).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "kgpu.h"
#include "kgpu_bulk.h"

namespace kgpu {

// Key schedules as the unified (batched / serving) kernels read them from the
// device key table.  "u-frame" layout, 60 words each:
//   words 0..3            round 0 (whitening)
//   words 4r..4r+3        middle round r (1 <= r < Nr), each word rotated right
//                         by 16 bits (the kernels fold the rotation of the
//                         T2/T3 half of the round into the key)
//   words 56..59          final round Nr (fixed slot whatever Nr is)
// Decryption schedules are also stored in the state order (0, 3, 2, 1), which
// turns the inverse cipher into the same round shape as the forward one.
struct DevKey {
    uint32_t encu[kMaxRoundKeyWords];
    uint32_t decu[kMaxRoundKeyWords];
    uint32_t twku[kMaxRoundKeyWords];  // XTS tweak key (forward cipher)
    uint32_t nr;                       // 10, 12 or 14
    uint32_t flags;                    // kKeyLive | kKeyXts
    uint32_t gen;                      // context-wide setkey count when this key was set (never 0)
    uint32_t pad;
};
constexpr uint32_t kKeyLive = 1u;
constexpr uint32_t kKeyXts = 2u;

struct HostKey {
    bool live = false;
    bool xts = false;
    int nr = 0;
    uint32_t enc[kMaxRoundKeyWords];
    uint32_t dec[kMaxRoundKeyWords];
    uint32_t twk[kMaxRoundKeyWords];
};

// One request of a batch or of the serving ring, as the device sees it.
struct ReqDesc {
    const uint4* src;
    uint4* dst;
    const uint4* ivs;       // CBC: one IV per page
    uint64_t nblocks;       // len / 16
    uint64_t first_sector;  // XTS: number of the first data unit
    uint32_t unit_blocks;   // XTS data unit / CBC page, in 16-byte blocks
    uint32_t key;           // key-table slot
    uint32_t mode;          // KGPU_MODE_*
    uint32_t dir;           // KGPU_ENCRYPT / KGPU_DECRYPT (XTS, ECB)
    uint32_t tile_units;    // work units (32-block chunks or pages) per tile
    uint32_t flags;         // kDesc* below
};
static_assert(sizeof(ReqDesc) == 64, "descriptor layout");
constexpr uint32_t kDescSrcHost = 1u;  // source in registered host memory
constexpr uint32_t kDescDstHost = 2u;  // destination in registered host memory
constexpr uint32_t kDescQuad = 4u;     // CBC encryption, four lanes per page: tiles of kQuadPages pages
constexpr uint32_t kQuadPages = 8;

// Per-warp device scratch of the unified kernels: CBC encryption of
// host-resident pages moves 8 blocks of each of a warp's 32 pages through it
// at a time (32 x 8 x 16 B).
constexpr uint32_t kStageBlocks = 8;
constexpr size_t kStageWarpBytes = 32 * kStageBlocks * 16;

// Work units of a request: XTS/ECB count 32-block chunks, CBC counts pages,
// COPY counts its unit_size tiles.
__host__ __device__ inline uint64_t request_units(const ReqDesc& d) {
    if (d.mode == KGPU_MODE_CBC_DEC || d.mode == KGPU_MODE_CBC_ENC || d.mode == KGPU_MODE_COPY)
        return d.nblocks / d.unit_blocks;
    return (d.nblocks + 31) / 32;
}

// Header of a batch as copied to the device: the descriptors follow, then the
// exclusive prefix of tiles per request in run order (nreq + 1 entries), then
// the run order.
struct BatchHeader {
    uint64_t total_tiles;
    uint32_t nreq;
    uint32_t tag;  // low 32 bits of the batch's ticket, in its completion words
};

// Byte layout of a batch on the device: header, descriptors, tile prefix, run order.
__host__ __device__ constexpr size_t batch_desc_offset() { return sizeof(BatchHeader); }
__host__ __device__ constexpr size_t batch_prefix_offset(uint32_t nreq) {
    return sizeof(BatchHeader) + (size_t)nreq * sizeof(ReqDesc);
}
// The run order follows the prefix: order[k] is the index of the k-th request
// whose tiles are handed out (the prefix counts tiles in run order).
__host__ __device__ constexpr size_t batch_order_offset(uint32_t nreq) {
    return batch_prefix_offset(nreq) + ((size_t)nreq + 1) * sizeof(uint64_t);
}
__host__ __device__ constexpr size_t batch_bytes(uint32_t nreq) {
    return batch_order_offset(nreq) + ((size_t)nreq * sizeof(uint32_t) + 7) / 8 * 8;
}

// Arguments of the unified batch kernel (fixed per staging slot, so a captured
// graph never needs new kernel parameters; the request count is in the header).
struct BatchArgs {
    const uint8_t* buf;  // BatchHeader | ReqDesc[nreq] | uint64_t tile_start[nreq + 1]
    const DevKey* keys;
    uint32_t max_keys;
    uint32_t scratch_warps;         // warps (by global index) that have a scratch area
    unsigned long long* next_tile;  // work counter (zero before launch)
    int* status;                    // per request: 0, or a negative KGPU_E* set by the kernel
    uint4* scratch;                 // kStageWarpBytes per warp, or null
    unsigned long long* fin;        // per request: tiles finished (zero before launch), or null
    unsigned long long* done;       // per request, host-mapped: tag << 32 | status once complete
};

// ---------------------------------------------------------------------------
// Serving ring.  Descriptors, the published count and the completion words
// live in pinned host memory mapped into the device address space (the
// paper's message passing through pinned memory, section 3.1); the claim and
// finish counters live in device memory.
// ---------------------------------------------------------------------------
struct ServeSlot {
    ReqDesc d;
    unsigned long long ntiles;  // tiles of this request
    unsigned long long seq;     // request number (slot = seq & mask)
    unsigned long long pos0;    // device copy only: tile-ring position of its first tile
    unsigned long long t_disp;  // device copy only: %globaltimer when the dispatcher took it
    unsigned long long t_pub;   // device copy only: %globaltimer when its tiles were published
    unsigned long long pad[3];
};
static_assert(sizeof(ServeSlot) == 128, "slot layout");

// The host's words and the kernel's words sit on lines of their own: the
// dispatcher polls `head` while it stores its heartbeat, and one shared line
// would move between the host's cache and the device at every store.
struct ServeHostHdr {
    alignas(128) unsigned long long head;  // requests published (host writes, release)
    unsigned int stop;                     // host asks the kernel to exit
    unsigned int pad0;
    alignas(128) unsigned long long exit_code;  // kernel writes why it exited (kServeExit*)
    unsigned long long heartbeat;               // dispatcher's last %globaltimer
};
static_assert(sizeof(ServeHostHdr) == 256, "ring header: two 128-byte lines");
constexpr unsigned kServeExitStop = 1, kServeExitIdle = 2, kServeExitLifetime = 3;

// Each counter sits on its own 128-byte line: idle workers poll tile_head
// while busy ones update the others, and one shared line would serialise them.
struct ServeDev {
    alignas(128) unsigned long long tile_head;   // tiles published to the tile ring (dispatcher, release)
    alignas(128) unsigned long long tile_next;   // tiles claimed by workers (atomicAdd)
    alignas(128) unsigned long long tile_done;   // tiles finished
    alignas(128) unsigned long long mirrored;    // requests copied to device memory and enumerated
    alignas(128) unsigned long long done_count;  // requests completed
    alignas(128) unsigned int stop;              // 0 run, else a kServeExit* reason
};

struct ServeArgs {
    const ServeSlot* slots;           // [S], mapped host: descriptors as the host wrote them
    ServeHostHdr* hh;                 // mapped host
    unsigned long long* done_seq;     // [S], mapped host: seq + 1 once complete
    int* status;                      // [S], mapped host
    unsigned long long* t_start;      // [S], mapped host: %globaltimer when its first tile starts
    unsigned long long* t_done;       // [S], mapped host: %globaltimer at completion
    unsigned long long* t_disp;       // [S], mapped host: %globaltimer when the dispatcher took it
    unsigned long long* t_pub;        // [S], mapped host: %globaltimer when its tiles were published
    ServeDev* dev;
    ServeSlot* dslots;                // [S], device copy of the descriptors
    unsigned long long* fin;          // [S], device: tiles finished per request
    unsigned long long* tiles;        // [T], device tile ring: (slot << 32) | tile
    unsigned long long* mbox;         // [grid * 16], one 128-B line per CTA: published
                                      // tile count, bit 63 = stop (polled by that CTA only)
    const DevKey* keys;
    uint32_t max_keys;
    uint32_t slot_mask;               // S - 1
    unsigned long long tile_mask;     // T - 1
    uint32_t tile_bits;               // log2(T)
    uint32_t scratch_warps;           // warps (by global index) that have a scratch area
    unsigned long long idle_ns;       // exit after this long with nothing to do
    unsigned long long lifetime_ns;   // exit at a tile boundary after this long
    uint4* scratch;                   // kStageWarpBytes per warp, or null
};
constexpr int kServeThreads = 512;  // threads per CTA of the serving kernel
constexpr unsigned long long kMboxStop = 1ull << 63;
constexpr int kMboxStride = 16;  // words between two CTAs' mailboxes (128 B)

// Largest tile count of one served request (a request must fit the tile ring).
inline uint64_t serve_max_tiles(uint64_t tile_ring) { return tile_ring / 2; }

// Launch entry points of the unified kernels (kgpu_unified.cu).  They return
// a cudaError_t from the launch.
cudaError_t launch_batch(const BatchArgs& a, int threads, int grid, cudaStream_t s);
// The empty service as one plain launch: warp w copies unit w (unit_blocks
// blocks); 32 threads per unit, in CTAs of up to 1024 threads.
cudaError_t launch_copy(const uint4* src, uint4* dst, uint64_t nblocks, uint32_t unit_blocks, int num_sms,
                        cudaStream_t s);
const void* batch_kernel_fn(int threads);  // for CUDA-graph kernel nodes
cudaError_t launch_serve(const ServeArgs& a, int threads, int grid, cudaStream_t s);
cudaError_t launch_serve_reset(ServeDev* dev, unsigned long long* mbox, int ctas,
                               cudaStream_t s);  // before each (re)launch
cudaError_t upload_unified_tables(const uint32_t* te0, const uint32_t* td0, const uint32_t* sb4,
                                  const uint32_t* isb4);
cudaError_t configure_batch_kernels();  // unified kernels: opt-in to large dynamic shared memory

// Unified-kernel shared memory: three table regions plus one 512-B key slot
// per warp (data schedule, then the XTS tweak schedule, 240 B each).
inline size_t unified_smem_bytes(int threads) { return 3 * kRegionBytes + (size_t)(threads / 32) * 512; }
// The 512-thread batch kernel adds, after the key slots, a pool of staging
// areas its warps share for CBC encryption of device pages (32 pages x 4
// blocks, 64-byte rows), then the pool's free mask.  A warp that finds no free
// area runs its tile without one.
constexpr uint32_t kPoolBlocks = 4;
constexpr size_t kPoolRow = kPoolBlocks * 16;
constexpr size_t kPoolAreaBytes = 32 * kPoolRow;
constexpr uint32_t kPoolAreas = 13;
constexpr int kPoolThreads = 512;  // the batch-kernel variant that has the pool
inline size_t batch_smem_bytes(int threads) {
    return unified_smem_bytes(threads) + (threads == kPoolThreads ? kPoolAreas * kPoolAreaBytes + 16 : 0);
}
static_assert(3 * kRegionBytes + (kPoolThreads / 32) * 512 + kPoolAreas * kPoolAreaBytes + 16 <= 232448,
              "the staging pool exceeds the 227-KB shared-memory limit");
// Launch shape of a batch when the caller has set none (kgpu_submit,
// kgpu_submit_noalloc): the 512-thread kernel, with two blocks per lane and
// the staging pool, and 16-KiB XTS/ECB tiles.  On the mixed batches, with the
// same tiles: 634 against 598-601 GB/s for 1,024 threads on 10,000 requests,
// 586 against 510-531 GB/s on 1,000.
constexpr uint32_t kBatchDefaultThreads = 512;
constexpr uint32_t kBatchDefaultTileChunks = 32;
// The serving kernel adds, after the key slots, a staging area per warp for
// four-lane CBC encryption of host pages: 8 pages x 8 blocks, rows padded to
// 144 bytes so that both the whole-line copies and the column reads are free
// of bank conflicts.
constexpr size_t kServeStageRow = 144;
constexpr size_t kServeStageWarpBytes = 8 * kServeStageRow;
inline size_t serve_smem_bytes() {
    return unified_smem_bytes(kServeThreads) + (size_t)(kServeThreads / 32) * kServeStageWarpBytes;
}

}  // namespace kgpu
