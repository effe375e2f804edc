// Parameter blocks and launch entry points of the bulk kernels (kgpu_bulk.cu):
// one kernel per mode, direction and key size, for the per-call transforms.
// Kept apart from the batched and serving formats so that the bulk kernels'
// sources are exactly aes_device.cuh, kgpu_bulk.cu and this header.
#pragma once
#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace kgpu {

constexpr int kMaxRoundKeyWords = 60;  // AES-256: 4 * (14 + 1)

// Shared-memory footprint of the table layouts (see aes_device.cuh).
constexpr size_t kRegionBytes = 65536;
constexpr size_t kSmemEnc = 2 * kRegionBytes;  // regions A, B
constexpr size_t kSmemDec = 3 * kRegionBytes;  // regions A, B, C

// Threads per CTA of the bulk kernels (one CTA per SM).
constexpr int kBulkThreads = 1024;

// Staged CBC encryption: up to 20 warps per CTA (96 registers a thread), each
// with a 32-page x 8-block staging area (4608 B) after the two table regions.
// The launch picks the warp count for the page count (cbc_enc_staged_warps).
constexpr int kCbcEncStagedMaxWarps = 20;
constexpr int kCbcEncStagedThreads = kCbcEncStagedMaxWarps * 32;
constexpr size_t kStageWarpSmem = 4608;
constexpr size_t kSmemEncStaged = kSmemEnc + kCbcEncStagedMaxWarps * kStageWarpSmem;
static_assert(kSmemEncStaged <= 232448, "staged CBC encryption exceeds the 227-KB shared-memory limit");

// Warps per CTA of the staged CBC-encryption launch for `groups` groups of 32
// pages on num_sms SMs (one CTA per SM).
int cbc_enc_staged_warps(uint64_t groups, int num_sms);

// CBC encryption staged by the tensor-memory-access engine: each warp moves 8
// blocks of its 32 pages at a time as one 2-D tile (32 pages x 128 B, 128-byte
// swizzle) into a 4-KiB buffer after the table regions, with an mbarrier per
// warp after the buffers.
constexpr size_t kTmaWarpBytes = 4096;
constexpr size_t kSmemEncTma = kSmemEnc + kCbcEncStagedMaxWarps * (kTmaWarpBytes + 8);
static_assert(kSmemEncTma <= 232448, "TMA-staged CBC encryption exceeds the 227-KB shared-memory limit");

// Where dynamic shared memory starts in a CTA's shared window (the reserved
// system area comes first); the kernels fold it into their load offsets.
constexpr int kSmemReservedBytes = 1024;

// Parameters of the bulk XTS / ECB kernels (passed by value, read from the
// constant bank).
struct BulkParams {
    const uint4* src;
    uint4* dst;
    uint64_t nblocks;       // 16-byte blocks in the buffer
    uint32_t bps;           // blocks per data unit (XTS)
    uint32_t pad0;
    uint64_t first_sector;  // number of the first data unit (XTS)
    uint32_t rk[kMaxRoundKeyWords];  // data key schedule (encryption or decryption order)
    uint32_t tk[kMaxRoundKeyWords];  // tweak key schedule (always encryption)
};

// Parameters of the CBC kernels.
struct CbcParams {
    const uint4* src;
    uint4* dst;
    const uint4* ivs;       // one per page
    uint64_t npages;
    uint32_t bpp;           // blocks per page
    uint32_t pad0;
    uint32_t rk[kMaxRoundKeyWords];
};

// Parameters of the TMA-staged CBC encryption: the source and destination as
// 2-D tensors of 32-bit words (page words x pages, page stride bpp * 16 bytes)
// read and written in 32 x 32 boxes.
struct CbcTmaParams {
    CUtensorMap src_map;
    CUtensorMap dst_map;
    const uint4* ivs;  // one per page
    uint64_t npages;
    uint32_t bpp;      // blocks per page, a multiple of 8
    uint32_t pad0;
    uint32_t rk[kMaxRoundKeyWords];
};

// XTS with ciphertext stealing: data units of du bytes, du >= 16 and not a
// multiple of 16 (IEEE 1619-2007 5.3.2 / 5.4.2).  Unit u starts at byte u * du.
struct CtsParams {
    const uint8_t* src;
    uint8_t* dst;
    uint64_t units;
    uint64_t du;
    uint64_t first_sector;
    uint32_t rk[kMaxRoundKeyWords];
    uint32_t tk[kMaxRoundKeyWords];
};

cudaError_t launch_xts(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s);
cudaError_t launch_xts_cts(const CtsParams& p, int nr, int dir, int num_sms, cudaStream_t s);
cudaError_t launch_ecb(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s);
cudaError_t launch_cbc_dec(const CbcParams& p, int nr, int num_sms, cudaStream_t s);
cudaError_t launch_cbc_enc(const CbcParams& p, int nr, int num_sms, cudaStream_t s);
cudaError_t upload_tables(const uint32_t* te0, const uint32_t* td0, const uint32_t* isb4);
// Bounded waits of the bulk kernels that ran out on the current device (a
// process-wide count; 0 unless a tensor copy never completed).
cudaError_t bulk_wait_timeouts(unsigned int* out);
cudaError_t configure_kernels();  // opt-in to large dynamic shared memory

}  // namespace kgpu
