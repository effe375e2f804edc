// Parameter block and launch entry points of the bitsliced kernels
// (kgpu_bitslice.cu), kept apart so that the bitsliced kernels' sources are
// exactly aes_device.cuh, sbox_circuit.cuh, kgpu_bitslice.cu and this header.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace kgpu {

// Bitsliced kernels (kgpu_bitslice.cu): 32 blocks per thread as 128 bit-planes.
constexpr int kBsThreads = 384;  // 168 registers: 12 warps per SM (see the kernel's comment)
struct BsParams {
    const uint4* src;
    uint4* dst;
    uint4* tw;              // XTS: one tweak E_K2(unit) per data unit of the call
    uint64_t nblocks;       // 16-byte blocks (main kernel)
    uint64_t units;         // data units (tweak pre-pass)
    uint64_t first_sector;  // number of the first data unit
    uint32_t bps;           // blocks per data unit
    uint32_t pad;
    uint32_t rkm[128 * 15]; // round-key plane masks (0 or ~0), (Nr + 1) x 128
};
cudaError_t launch_bitsliced(const BsParams& p, int nr, bool tweak, int num_sms, cudaStream_t s);
cudaError_t launch_bitsliced_tweaks(const BsParams& p, int nr, int num_sms, cudaStream_t s);

}  // namespace kgpu
