// Context layout and host-side helpers shared by the C-ABI translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <utility>
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
    unsigned long long* d_counter = nullptr;
    uint32_t nreq = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_copy = nullptr, n_status_clear = nullptr, n_kernel = nullptr, n_status_out = nullptr;
    int graph_threads = 0, graph_grid = 0;
    BatchArgs args{};
};

constexpr int kBatchSlots = 4;

}  // namespace kgpu

struct kgpu_ctx {
    int device = 0;
    int num_sms = 0;
    kgpu_config cfg{};
    std::mutex mu;
    std::vector<kgpu::HostKey> keys;
    kgpu::DevKey* d_keys = nullptr;

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
    uint64_t next_ticket = 0;
    kgpu_tuning tune{};
};


namespace kgpu {
namespace hostutil {

constexpr int kVersion = (0 << 16) | 3;

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
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

inline int xts_args(kgpu_ctx* ctx, int dir, size_t len, size_t du, uint64_t first_sector) {
    if (!ctx) return KGPU_EINVAL;
    if (dir != KGPU_ENCRYPT && dir != KGPU_DECRYPT) return KGPU_EINVAL;
    if (du == 0 || du % 16 || len % du) return KGPU_EINVAL;
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


void destroy_batch_slots(kgpu_ctx* ctx);  // kgpu_batch_api.cu

}  // namespace hostutil
}  // namespace kgpu
