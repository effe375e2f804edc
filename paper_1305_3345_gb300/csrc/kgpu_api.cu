// C-ABI entry points (include/kgpu.h): context, key table, argument checks and
// the synchronous-looking host-resident pipeline.  Every transform itself runs
// in the CUDA kernels of kgpu_bulk.cu; this file only validates and launches.
#include <cuda.h>
#include <cuda_runtime.h>
#include <unistd.h>

#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "aes_tables_host.h"
#include "kgpu_bitslice.h"
#include "kgpu_ctx.h"

using namespace kgpu;
using namespace kgpu::hostutil;


extern "C" {

int kgpu_version(void) { return kVersion; }

const char* kgpu_strerror(int code) {
    switch (code) {
        case KGPU_OK: return "success";
        case KGPU_EIO: return "CUDA launch or runtime failure";
        case KGPU_E2BIG: return "too many requests for the fixed scratch area";
        case KGPU_ENOMEM: return "out of memory or table full";
        case KGPU_EFAULT: return "pointer not inside a usable allocation";
        case KGPU_EBUSY: return "busy: queue full or admission refused";
        case KGPU_ENODEV: return "no usable sm_103 CUDA device";
        case KGPU_EINVAL: return "invalid argument";
        case KGPU_ENOENT: return "unknown key or ticket";
        case KGPU_ETIMEDOUT: return "bounded wait timed out";
        case KGPU_ENOSYS: return "host AES library (libcrypto 3) not available";
        default: return "unknown error";
    }
}

int kgpu_init(kgpu_ctx** out, int device, const kgpu_config* cfg) {
    if (!out) return KGPU_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return KGPU_ENODEV;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return KGPU_ENODEV;
    if (prop.major != 10 || prop.minor != 3) return KGPU_ENODEV;  // built for sm_103a only
    int reserved = -1;
    if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess ||
        reserved != kSmemReservedBytes)
        return KGPU_ENODEV;  // the kernels' shared-memory offsets assume this layout
    kgpu_ctx* ctx = new (std::nothrow) kgpu_ctx();
    if (!ctx) return KGPU_ENOMEM;
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    if (cfg) ctx->cfg = *cfg;
    if (!ctx->cfg.max_keys) ctx->cfg.max_keys = 4096;
    if (!ctx->cfg.ring_slots) ctx->cfg.ring_slots = 4096;
    if (!ctx->cfg.admit_bytes) ctx->cfg.admit_bytes = 8ull << 30;
    if (!ctx->cfg.idle_timeout_ns) ctx->cfg.idle_timeout_ns = 2000000000ull;
    if (ctx->cfg.max_keys > (1u << 20) || (ctx->cfg.ring_slots & (ctx->cfg.ring_slots - 1)) ||
        ctx->cfg.host_dispatch > 1) {
        delete ctx;
        return KGPU_EINVAL;
    }

    DeviceGuard g(device);
    host::Tables t;
    host::make_tables(&t);
    int rc = from_cuda(configure_kernels());
    if (rc == KGPU_OK) rc = from_cuda(configure_batch_kernels());
    if (rc == KGPU_OK) rc = from_cuda(upload_tables(t.te0, t.td0, t.isb4));
    if (rc == KGPU_OK) rc = from_cuda(upload_unified_tables(t.te0, t.td0, t.sb4, t.isb4));
    if (rc == KGPU_OK) rc = from_cuda(cudaMalloc(&ctx->d_keys, sizeof(DevKey) * ctx->cfg.max_keys));
    if (rc == KGPU_OK) rc = from_cuda(cudaMemset(ctx->d_keys, 0, sizeof(DevKey) * ctx->cfg.max_keys));
    if (rc == KGPU_OK) rc = from_cuda(cudaStreamCreateWithFlags(&ctx->key_stream, cudaStreamNonBlocking));
    if (rc == KGPU_OK) rc = from_cuda(cudaEventCreateWithFlags(&ctx->noalloc_done, cudaEventDisableTiming));
    if (rc == KGPU_OK) rc = from_cuda(cudaStreamCreateWithFlags(&ctx->crypt_stream, cudaStreamNonBlocking));
    if (rc != KGPU_OK) {
        cudaGetLastError();
        kgpu_destroy(ctx);
        return rc;
    }
    ctx->keys.reserve(64);
    // the paper's start-up calibration of the CPU/GPU crossover (section 4)
    if (ctx->cfg.host_dispatch && (rc = kgpu_calibrate_dispatch(ctx, nullptr, 0, nullptr, nullptr)) != KGPU_OK) {
        kgpu_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return KGPU_OK;
}

int kgpu_destroy(kgpu_ctx* ctx) {
    if (!ctx) return KGPU_OK;
    if (int rc = destroy_serve(ctx)) return rc;  // called from a completion callback
    {
        DeviceGuard g(ctx->device);
        for (int i = 0; i < kgpu_ctx::kStages; i++) {
            if (ctx->hs[i]) {
                cudaStreamSynchronize(ctx->hs[i]);
                cudaStreamDestroy(ctx->hs[i]);
            }
            if (ctx->staging[i]) cudaFree(ctx->staging[i]);
        }
        destroy_batch_slots(ctx);
        if (ctx->noalloc_done) {
            cudaEventSynchronize(ctx->noalloc_done);
            cudaEventDestroy(ctx->noalloc_done);
        }
        if (ctx->key_stream) cudaStreamDestroy(ctx->key_stream);
        if (ctx->crypt_stream) cudaStreamDestroy(ctx->crypt_stream);
        if (ctx->d_keys) cudaFree(ctx->d_keys);
        for (const HostRange& r : ctx->hreg)
            if (r.owned) cudaHostUnregister(reinterpret_cast<void*>(r.base));
    }
    delete ctx;
    return KGPU_OK;
}

int kgpu_aes_setkey(kgpu_ctx* ctx, const uint8_t* key, size_t key_len, int xts, kgpu_key* out) {
    if (!ctx || !key || !out || (xts != 0 && xts != 1)) return KGPU_EINVAL;
    HostKey hk;
    hk.live = true;
    hk.xts = xts == 1;
    std::memset(hk.enc, 0, sizeof(hk.enc));
    std::memset(hk.dec, 0, sizeof(hk.dec));
    std::memset(hk.twk, 0, sizeof(hk.twk));
    size_t half = key_len;
    if (hk.xts) {
        // IEEE 1619 defines XTS-AES-128 and XTS-AES-256 only
        if (key_len != 32 && key_len != 64) return KGPU_EINVAL;
        half = key_len / 2;
        if (std::memcmp(key, key + half, half) == 0) return KGPU_EINVAL;
    }
    hk.nr = host::expand_key(key, half, hk.enc);
    if (!hk.nr) return KGPU_EINVAL;
    host::decrypt_schedule(hk.enc, hk.nr, hk.dec);
    if (hk.xts && host::expand_key(key + half, half, hk.twk) != hk.nr) return KGPU_EINVAL;

    DevKey dk;
    std::memset(&dk, 0, sizeof(dk));
    host::to_uframe(hk.enc, hk.nr, false, dk.encu);
    host::to_uframe(hk.dec, hk.nr, true, dk.decu);
    if (hk.xts) host::to_uframe(hk.twk, hk.nr, false, dk.twku);
    dk.nr = (uint32_t)hk.nr;
    dk.flags = kKeyLive | (hk.xts ? kKeyXts : 0u);

    std::lock_guard<std::mutex> lk(ctx->mu);
    size_t slot = ctx->keys.size();
    for (size_t i = 0; i < ctx->keys.size(); i++) {
        if (!ctx->keys[i].live) {
            slot = i;
            break;
        }
    }
    if (slot >= ctx->cfg.max_keys) return KGPU_ENOMEM;
    // A running serving kernel keeps the last schedule each warp loaded,
    // tagged with slot, direction and this generation: a new key in a freed
    // slot carries a generation no warp has seen (0 is never issued).
    if (++ctx->key_gen == 0) ++ctx->key_gen;
    dk.gen = ctx->key_gen;
    DeviceGuard g(ctx->device);
    if (cudaMemcpyAsync(ctx->d_keys + slot, &dk, sizeof(dk), cudaMemcpyHostToDevice, ctx->key_stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->key_stream) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    if (slot == ctx->keys.size()) ctx->keys.push_back(hk);
    else ctx->keys[slot] = hk;
    *out = (kgpu_key)(slot + 1);
    std::memset(&dk, 0, sizeof(dk));
    return KGPU_OK;
}

int kgpu_aes_delkey(kgpu_ctx* ctx, kgpu_key key) {
    if (!ctx) return KGPU_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (key == 0 || key > ctx->keys.size() || !ctx->keys[key - 1].live) return KGPU_ENOENT;
    }
    // Work that reads the device key record must finish first: batches in
    // flight and requests already published to the serving ring.  Launches of
    // the per-call entry points carry their schedule in the launch itself.
    int rc = batches_quiesce(ctx);
    if (!rc) rc = serve_quiesce(ctx, 60000000000ll);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->keys[key - 1].live) return KGPU_ENOENT;
    DeviceGuard g(ctx->device);
    DevKey zero;
    std::memset(&zero, 0, sizeof(zero));
    if (cudaMemcpyAsync(ctx->d_keys + (key - 1), &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->key_stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->key_stream) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    std::memset(&ctx->keys[key - 1], 0, sizeof(HostKey));
    ctx->keys[key - 1].live = false;
    return KGPU_OK;
}

namespace {

// Every OS page of [a, e) must be page-locked host memory mapped for the
// current device, all at one device-address offset (*off).
int pinned_offset(uintptr_t a, uintptr_t e, intptr_t* off) {
    long ps = sysconf(_SC_PAGESIZE);
    const uintptr_t page = ps > 0 ? (uintptr_t)ps : 4096;
    bool first = true;
    for (uintptr_t p = a;;) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, reinterpret_cast<void*>(p)) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_EFAULT;
        }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer) return KGPU_EFAULT;
        const intptr_t o = (intptr_t)at.devicePointer - (intptr_t)p;
        if (first)
            *off = o;
        else if (o != *off)
            return KGPU_EFAULT;
        first = false;
        if (p == e - 1) break;
        const uintptr_t next = (p / page + 1) * page;
        p = next < e ? next : e - 1;
    }
    return KGPU_OK;
}

}  // namespace

int kgpu_host_register(kgpu_ctx* ctx, void* ptr, size_t len, uint32_t flags) {
    if (!ctx || !ptr || !len || (flags != KGPU_HOSTREG_PIN && flags != KGPU_HOSTREG_PINNED)) return KGPU_EINVAL;
    const uintptr_t a = (uintptr_t)ptr, e = a + len;
    if (e < a) return KGPU_EINVAL;
    DeviceGuard g(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->hreg_mu);
    // the first range ending after a; ranges are disjoint, so sorted by end too
    auto it = std::lower_bound(ctx->hreg.begin(), ctx->hreg.end(), a,
                               [](const HostRange& r, uintptr_t x) { return r.end <= x; });
    if (it != ctx->hreg.end() && it->base < e) return KGPU_EINVAL;
    HostRange r;
    r.base = a;
    r.end = e;
    if (flags == KGPU_HOSTREG_PIN) {
        cudaError_t err = cudaHostRegister(ptr, len, cudaHostRegisterMapped | cudaHostRegisterPortable);
        if (err != cudaSuccess) {
            cudaGetLastError();
            if (err == cudaErrorHostMemoryAlreadyRegistered) return KGPU_EINVAL;
            return err == cudaErrorMemoryAllocation ? KGPU_ENOMEM : KGPU_EIO;
        }
        void* dp = nullptr;
        if (cudaHostGetDevicePointer(&dp, ptr, 0) != cudaSuccess || !dp) {
            cudaGetLastError();
            cudaHostUnregister(ptr);
            return KGPU_EIO;
        }
        r.dev_off = (intptr_t)dp - (intptr_t)a;
        r.owned = true;
    } else {
        int rc = pinned_offset(a, e, &r.dev_off);
        if (rc) return rc;
    }
    ctx->hreg.insert(it, r);
    return KGPU_OK;
}

int kgpu_host_unregister(kgpu_ctx* ctx, void* ptr) {
    if (!ctx || !ptr) return KGPU_EINVAL;
    auto find = [&]() {
        return std::find_if(ctx->hreg.begin(), ctx->hreg.end(),
                            [&](const HostRange& r) { return r.base == (uintptr_t)ptr; });
    };
    {
        std::lock_guard<std::mutex> lk(ctx->hreg_mu);
        if (find() == ctx->hreg.end()) return KGPU_ENOENT;
    }
    // batches in flight, requests on the serving ring and a host-buffer call
    // (it holds host_mu throughout) may still read or write the range
    int rc = batches_quiesce(ctx);
    if (!rc) rc = serve_quiesce(ctx, 60000000000ll);
    if (rc) return rc;
    HostRange r;
    {
        std::lock_guard<std::mutex> hk(ctx->host_mu);
        std::lock_guard<std::mutex> lk(ctx->hreg_mu);
        auto it = find();
        if (it == ctx->hreg.end()) return KGPU_ENOENT;
        r = *it;
        ctx->hreg.erase(it);
    }
    if (r.owned) {
        DeviceGuard g(ctx->device);
        if (cudaHostUnregister(ptr) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_EIO;
        }
    }
    return KGPU_OK;
}

int kgpu_aes_xts_crypt(kgpu_ctx* ctx, kgpu_key key, int dir, const void* src, void* dst, size_t len,
                       size_t du_size, uint64_t first_sector, kgpu_stream stream) {
    int rc = xts_args(ctx, dir, len, du_size, first_sector, true);
    if (rc) return rc;
    HostKey k;
    if ((rc = get_key(ctx, key, true, &k))) return rc;
    if (len == 0) return KGPU_OK;
    if ((rc = check_pair(src, dst, len))) return rc;
    if ((rc = check_device_range(ctx, src, len)) || (rc = check_device_range(ctx, dst, len))) return rc;
    if (du_size % 16) {  // data units ending in a partial block: ciphertext stealing
        CtsParams c;
        std::memset(&c, 0, sizeof(c));
        c.src = static_cast<const uint8_t*>(src);
        c.dst = static_cast<uint8_t*>(dst);
        c.units = len / du_size;
        c.du = du_size;
        c.first_sector = first_sector;
        std::memcpy(c.rk, dir == KGPU_ENCRYPT ? k.enc : k.dec, sizeof(c.rk));
        std::memcpy(c.tk, k.twk, sizeof(c.tk));
        DeviceGuard g(ctx->device);
        return from_cuda(launch_xts_cts(c, k.nr, dir, ctx->num_sms, (cudaStream_t)stream));
    }
    BulkParams p;
    fill_bulk(&p, k, dir, src, dst, len, du_size, first_sector);
    DeviceGuard g(ctx->device);
    return from_cuda(launch_xts(p, k.nr, dir, ctx->num_sms, (cudaStream_t)stream));
}

int kgpu_aes_ecb_crypt(kgpu_ctx* ctx, kgpu_key key, int dir, const void* src, void* dst, size_t len,
                       kgpu_stream stream) {
    if (!ctx || (dir != KGPU_ENCRYPT && dir != KGPU_DECRYPT) || len % 16) return KGPU_EINVAL;
    HostKey k;
    int rc = get_key(ctx, key, false, &k);
    if (rc) return rc;
    if (len == 0) return KGPU_OK;
    if ((rc = check_pair(src, dst, len))) return rc;
    if ((rc = check_device_range(ctx, src, len)) || (rc = check_device_range(ctx, dst, len))) return rc;
    BulkParams p;
    fill_bulk(&p, k, dir, src, dst, len, 16, 0);
    DeviceGuard g(ctx->device);
    return from_cuda(launch_ecb(p, k.nr, dir, ctx->num_sms, (cudaStream_t)stream));
}

static int cbc_common(kgpu_ctx* ctx, kgpu_key key, bool enc, const void* src, void* dst, size_t len,
                      size_t page, const uint8_t* ivs, kgpu_stream stream) {
    if (!ctx || page == 0 || page % 16 || len % page || page / 16 > 0xFFFFFFFFull) return KGPU_EINVAL;
    HostKey k;
    int rc = get_key(ctx, key, false, &k);
    if (rc) return rc;
    if (len == 0) return KGPU_OK;
    if ((rc = check_pair(src, dst, len))) return rc;
    if ((uintptr_t)ivs & 15) return KGPU_EINVAL;
    size_t npages = len / page;
    if ((rc = check_device_range(ctx, src, len)) || (rc = check_device_range(ctx, dst, len)) ||
        (rc = check_device_range(ctx, ivs, npages * 16)))
        return rc;
    // the IVs must not be overwritten while pages are being processed
    uintptr_t iv0 = (uintptr_t)ivs, iv1 = iv0 + npages * 16, d0 = (uintptr_t)dst;
    if (iv0 < d0 + len && d0 < iv1) return KGPU_EINVAL;
    CbcParams p;
    std::memset(&p, 0, sizeof(p));
    p.src = static_cast<const uint4*>(src);
    p.dst = static_cast<uint4*>(dst);
    p.ivs = reinterpret_cast<const uint4*>(ivs);
    p.npages = npages;
    p.bpp = (uint32_t)(page / 16);
    std::memcpy(p.rk, enc ? k.enc : k.dec, sizeof(p.rk));
    DeviceGuard g(ctx->device);
    cudaError_t e = enc ? launch_cbc_enc(p, k.nr, ctx->num_sms, (cudaStream_t)stream)
                        : launch_cbc_dec(p, k.nr, ctx->num_sms, (cudaStream_t)stream);
    return from_cuda(e);
}

namespace {

// Plane masks of a schedule (little-endian column words): plane 32w + k of
// round r is all ones when bit k of word w of round key r is set.
void fill_plane_masks(uint32_t* rkm, const uint32_t* sched, int nr) {
    for (int r = 0; r <= nr; r++)
        for (int w = 0; w < 4; w++)
            for (int k = 0; k < 32; k++) rkm[128 * r + 32 * w + k] = ((sched[4 * r + w] >> k) & 1u) ? ~0u : 0u;
}

}  // namespace

int kgpu_aes_xts_crypt_bitsliced(kgpu_ctx* ctx, kgpu_key key, int dir, const void* src, void* dst, size_t len,
                                 size_t du_size, uint64_t first_sector, kgpu_stream stream) {
    int rc = xts_args(ctx, dir, len, du_size, first_sector);
    if (rc) return rc;
    if (dir != KGPU_ENCRYPT) return KGPU_EINVAL;
    HostKey k;
    if ((rc = get_key(ctx, key, true, &k))) return rc;
    if (len == 0) return KGPU_OK;
    if ((rc = check_pair(src, dst, len))) return rc;
    if ((rc = check_device_range(ctx, src, len)) || (rc = check_device_range(ctx, dst, len))) return rc;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t units = len / du_size;
    void* tw = nullptr;
    if (cudaMallocAsync(&tw, units * 16, s) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_ENOMEM;
    }
    static thread_local BsParams p;  // 7.7 KB: kept off the stack
    std::memset(&p, 0, sizeof(p));
    p.src = static_cast<const uint4*>(src);
    p.dst = static_cast<uint4*>(dst);
    p.tw = static_cast<uint4*>(tw);
    p.nblocks = len / 16;
    p.units = units;
    p.first_sector = first_sector;
    p.bps = (uint32_t)(du_size / 16);
    fill_plane_masks(p.rkm, k.twk, k.nr);
    cudaError_t e = launch_bitsliced_tweaks(p, k.nr, ctx->num_sms, s);
    if (e == cudaSuccess) {
        fill_plane_masks(p.rkm, k.enc, k.nr);
        e = launch_bitsliced(p, k.nr, true, ctx->num_sms, s);
    }
    cudaError_t f = cudaFreeAsync(tw, s);
    if (e != cudaSuccess || f != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    return KGPU_OK;
}

int kgpu_aes_cbc_decrypt(kgpu_ctx* ctx, kgpu_key key, const void* src, void* dst, size_t len, size_t page_size,
                         const uint8_t* ivs, kgpu_stream stream) {
    return cbc_common(ctx, key, false, src, dst, len, page_size, ivs, stream);
}

int kgpu_aes_cbc_encrypt_pages(kgpu_ctx* ctx, kgpu_key key, const void* src, void* dst, size_t len,
                               size_t page_size, const uint8_t* ivs, kgpu_stream stream) {
    return cbc_common(ctx, key, true, src, dst, len, page_size, ivs, stream);
}

int kgpu_bulk_wait_timeouts(kgpu_ctx* ctx, uint32_t* count) {
    if (!ctx || !count) return KGPU_EINVAL;
    DeviceGuard g(ctx->device);
    unsigned int v = 0;
    if (bulk_wait_timeouts(&v) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    *count = v;
    return KGPU_OK;
}

int kgpu_aes_xts_crypt_host(kgpu_ctx* ctx, kgpu_key key, int dir, const void* src, void* dst, size_t len,
                            size_t du_size, uint64_t first_sector, size_t chunk_bytes) {
    int rc = xts_args(ctx, dir, len, du_size, first_sector);
    if (rc) return rc;
    HostKey k;
    if ((rc = get_key(ctx, key, true, &k))) return rc;
    if (len == 0) return KGPU_OK;
    if ((rc = check_pair(src, dst, len))) return rc;
    if ((rc = check_host_ptr(src)) || (rc = check_host_ptr(dst))) return rc;
    size_t chunk = chunk_bytes ? chunk_bytes : (4u << 20);
    if (chunk < du_size) chunk = du_size;
    chunk -= chunk % du_size;
    if (chunk > len) chunk = len;

    // held for the whole call: kgpu_host_unregister takes it before it unpins
    std::lock_guard<std::mutex> lk(ctx->host_mu);
    DeviceGuard g(ctx->device);
    for (int i = 0; i < kgpu_ctx::kStages; i++) {
        if (!ctx->hs[i] && cudaStreamCreateWithFlags(&ctx->hs[i], cudaStreamNonBlocking) != cudaSuccess)
            return KGPU_EIO;
    }
    // Both buffers in registered ranges: the kernel works on the host pages in
    // place over the coherent link, at the link's speed in both directions at
    // once, with no staging and no pipeline fill or drain.
    uintptr_t hsrc = 0, hdst = 0;
    if (host_translate(ctx, src, len, &hsrc) == KGPU_OK && host_translate(ctx, dst, len, &hdst) == KGPU_OK) {
        BulkParams p;
        fill_bulk(&p, k, dir, reinterpret_cast<const void*>(hsrc), reinterpret_cast<void*>(hdst), len, du_size,
                  first_sector);
        cudaError_t e = launch_xts(p, k.nr, dir, ctx->num_sms, ctx->hs[0]);
        cudaError_t e2 = cudaStreamSynchronize(ctx->hs[0]);
        return from_cuda(e != cudaSuccess ? e : e2);
    }
    if (ctx->staging_bytes < chunk) {
        for (int i = 0; i < kgpu_ctx::kStages; i++) {
            cudaStreamSynchronize(ctx->hs[i]);
            if (ctx->staging[i]) cudaFree(ctx->staging[i]);
            ctx->staging[i] = nullptr;
        }
        ctx->staging_bytes = 0;
        for (int i = 0; i < kgpu_ctx::kStages; i++) {
            if (cudaMalloc(&ctx->staging[i], chunk) != cudaSuccess) {
                cudaGetLastError();
                return KGPU_ENOMEM;
            }
        }
        ctx->staging_bytes = chunk;
    }
    const uint8_t* s = static_cast<const uint8_t*>(src);
    uint8_t* d = static_cast<uint8_t*>(dst);
    cudaError_t e = cudaSuccess;
    size_t idx = 0;
    for (size_t off = 0; off < len && e == cudaSuccess; off += chunk, idx++) {
        int st = (int)(idx % kgpu_ctx::kStages);
        size_t n = len - off < chunk ? len - off : chunk;
        cudaStream_t hs = ctx->hs[st];
        // In-order streams: this H2D waits for the D2H that last used the buffer.
        e = cudaMemcpyAsync(ctx->staging[st], s + off, n, cudaMemcpyHostToDevice, hs);
        if (e != cudaSuccess) break;
        BulkParams p;
        fill_bulk(&p, k, dir, ctx->staging[st], ctx->staging[st], n, du_size, first_sector + off / du_size);
        e = launch_xts(p, k.nr, dir, ctx->num_sms, hs);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(d + off, ctx->staging[st], n, cudaMemcpyDeviceToHost, hs);
    }
    for (int i = 0; i < kgpu_ctx::kStages; i++) {
        cudaError_t e2 = cudaStreamSynchronize(ctx->hs[i]);
        if (e == cudaSuccess) e = e2;
    }
    return from_cuda(e);
}

}  // extern "C"
