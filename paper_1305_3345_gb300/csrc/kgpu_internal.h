// Internal declarations shared by the library's translation units: kernel
// parameter blocks, launch helpers and the context layout.  Not part of the
// public C ABI (that is include/kgpu.h).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "kgpu.h"

namespace kgpu {

constexpr int kMaxRoundKeyWords = 60;  // AES-256: 4 * (14 + 1)

// Shared-memory footprint of the table layouts (see aes_device.cuh).
constexpr size_t kSmemEnc = 2 * 65536;  // regions A, B
constexpr size_t kSmemDec = 3 * 65536;  // regions A, B, C

constexpr int kBulkThreads = 1024;

// Where dynamic shared memory starts in a CTA's shared window (the reserved
// system area comes first); the kernels fold it into their load offsets.
constexpr int kSmemReservedBytes = 1024;  // threads per CTA of the bulk kernels (one CTA per SM)

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

// One device-side key record (batched and serving kernels read keys from HBM).
struct DevKey {
    uint32_t enc[kMaxRoundKeyWords];
    uint32_t dec[kMaxRoundKeyWords];
    uint32_t twk[kMaxRoundKeyWords];  // XTS tweak key (encryption order)
    uint32_t nr;                      // 10, 12 or 14
    uint32_t flags;                   // bit 0: XTS key, bit 1: live
    uint32_t pad[2];
};

struct HostKey {
    bool live = false;
    bool xts = false;
    int nr = 0;
    uint32_t enc[kMaxRoundKeyWords];
    uint32_t dec[kMaxRoundKeyWords];
    uint32_t twk[kMaxRoundKeyWords];
};

// Launch entry points implemented in the kernel translation units.  They
// return a cudaError_t from the launch.
cudaError_t launch_xts(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s);
cudaError_t launch_ecb(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s);
cudaError_t launch_cbc_dec(const CbcParams& p, int nr, int num_sms, cudaStream_t s);
cudaError_t launch_cbc_enc(const CbcParams& p, int nr, int num_sms, cudaStream_t s);
cudaError_t upload_tables(const uint32_t* te0, const uint32_t* td0, const uint32_t* isb4);
cudaError_t configure_kernels();  // opt-in to large dynamic shared memory

}  // namespace kgpu
