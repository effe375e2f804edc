// kgpu_crypt: one request at a time, on the GPU or -- below a measured
// crossover, for requests whose pages are in host memory -- on the host.
//
// The paper measures its GPU AES against the kernel's CPU AES and finds the
// GPU behind below a request size of two pages, because every GPU request
// pays a fixed launch-and-copy cost; it proposes measuring that crossover at
// start-up and sending smaller requests to the CPU (section 4).  This file is
// that dispatcher.  The GPU leg is the library's own (the serving ring, or one
// launch of the mode's kernel).  The host leg is a separate cipher implementation that the
// library does not contain: OpenSSL's libcrypto (version 3, AES-NI or the
// Arm cryptography extensions), loaded with dlopen at first use so that the
// library has no link-time dependency on it.  The host leg only ever touches
// registered host memory; device-resident requests always take the GPU leg.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "kgpu_ctx.h"

using namespace kgpu;
using namespace kgpu::hostutil;

namespace {

// ---------------------------------------------------------------- libcrypto

// The few EVP calls the host leg makes, resolved from libcrypto.so.3.
struct Evp {
    void* (*ctx_new)();
    void (*ctx_free)(void*);
    void* (*fetch)(void*, const char*, const char*);
    int (*init)(void*, const void*, void*, const unsigned char*, const unsigned char*, int);
    int (*set_padding)(void*, int);
    int (*update)(void*, unsigned char*, int*, const unsigned char*, int);
    // fetched ciphers: [0] AES-128, [1] AES-192, [2] AES-256
    const void* xts[3];
    const void* cbc[3];
    const void* ecb[3];
    bool ok = false;
};

const Evp& evp() {
    static Evp e;
    static std::once_flag once;
    std::call_once(once, [] {
        void* h = dlopen("libcrypto.so.3", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        auto sym = [h](const char* n) { return dlsym(h, n); };
        e.ctx_new = reinterpret_cast<void* (*)()>(sym("EVP_CIPHER_CTX_new"));
        e.ctx_free = reinterpret_cast<void (*)(void*)>(sym("EVP_CIPHER_CTX_free"));
        e.fetch = reinterpret_cast<void* (*)(void*, const char*, const char*)>(sym("EVP_CIPHER_fetch"));
        e.init = reinterpret_cast<int (*)(void*, const void*, void*, const unsigned char*, const unsigned char*,
                                          int)>(sym("EVP_CipherInit_ex"));
        e.set_padding = reinterpret_cast<int (*)(void*, int)>(sym("EVP_CIPHER_CTX_set_padding"));
        e.update = reinterpret_cast<int (*)(void*, unsigned char*, int*, const unsigned char*, int)>(
            sym("EVP_CipherUpdate"));
        if (!e.ctx_new || !e.ctx_free || !e.fetch || !e.init || !e.set_padding || !e.update) return;
        static const char* kXts[3] = {"AES-128-XTS", nullptr, "AES-256-XTS"};
        static const char* kCbc[3] = {"AES-128-CBC", "AES-192-CBC", "AES-256-CBC"};
        static const char* kEcb[3] = {"AES-128-ECB", "AES-192-ECB", "AES-256-ECB"};
        for (int i = 0; i < 3; i++) {
            e.xts[i] = kXts[i] ? e.fetch(nullptr, kXts[i], nullptr) : nullptr;
            e.cbc[i] = e.fetch(nullptr, kCbc[i], nullptr);
            e.ecb[i] = e.fetch(nullptr, kEcb[i], nullptr);
            if ((kXts[i] && !e.xts[i]) || !e.cbc[i] || !e.ecb[i]) return;
        }
        e.ok = true;
    });
    return e;
}

// One cipher context per thread, kept for the thread's lifetime.
struct ThreadCtx {
    void* c = nullptr;
    ~ThreadCtx() {
        if (c) evp().ctx_free(c);
    }
};

// The raw key bytes, recovered from the first Nk words of a FIPS-197 5.2
// schedule (those words are the key itself, little-endian in the schedule).
void raw_key(const uint32_t* sched, int nr, unsigned char* out) {
    const int nk = nr - 6;
    for (int i = 0; i < nk; i++)
        for (int j = 0; j < 4; j++) out[4 * i + j] = (unsigned char)(sched[i] >> (8 * j));
}

// The host leg: the request's pages are host memory (q.src, q.dst, q.ivs are
// the caller's own addresses).  Returns KGPU_OK or KGPU_E*.
int host_leg(const HostKey& k, const kgpu_request& q) {
    const Evp& e = evp();
    if (!e.ok) return KGPU_ENOSYS;
    // OpenSSL takes an XTS data unit in one call and, as IEEE 1619 does, at
    // most 2^20 blocks to a unit
    if (q.mode == KGPU_MODE_XTS && q.unit_size > (16u << 20)) return KGPU_EINVAL;
    thread_local ThreadCtx tc;
    if (!tc.c && !(tc.c = e.ctx_new())) return KGPU_ENOMEM;
    void* c = tc.c;
    const int ki = k.nr == 10 ? 0 : k.nr == 12 ? 1 : 2;
    unsigned char key[64];
    const int nk = k.nr - 6;
    raw_key(k.enc, k.nr, key);
    const auto* src = static_cast<const unsigned char*>(q.src);
    auto* dst = static_cast<unsigned char*>(q.dst);
    int rc = KGPU_OK, outl = 0;
    if (q.mode == KGPU_MODE_XTS) {
        raw_key(k.twk, k.nr, key + 4 * nk);  // XTS key = Key1 || Key2
        const int enc = q.dir == KGPU_ENCRYPT;
        if (!e.xts[ki] || e.init(c, e.xts[ki], nullptr, key, nullptr, enc) != 1) rc = KGPU_EIO;
        const uint64_t units = q.len / q.unit_size;
        for (uint64_t u = 0; u < units && !rc; u++) {
            unsigned char iv[16] = {};
            const uint64_t s = q.sector + u;  // IEEE 1619: the unit number, 128-bit little-endian
            for (int j = 0; j < 8; j++) iv[j] = (unsigned char)(s >> (8 * j));
            if (e.init(c, nullptr, nullptr, nullptr, iv, enc) != 1 ||
                e.update(c, dst + u * q.unit_size, &outl, src + u * q.unit_size, (int)q.unit_size) != 1)
                rc = KGPU_EIO;
        }
    } else if (q.mode == KGPU_MODE_CBC_DEC || q.mode == KGPU_MODE_CBC_ENC) {
        const int enc = q.mode == KGPU_MODE_CBC_ENC;
        if (e.init(c, e.cbc[ki], nullptr, key, nullptr, enc) != 1 || e.set_padding(c, 0) != 1) rc = KGPU_EIO;
        const uint64_t pages = q.len / q.unit_size;
        for (uint64_t p = 0; p < pages && !rc; p++) {
            if (e.init(c, nullptr, nullptr, nullptr, q.ivs + 16 * p, enc) != 1) rc = KGPU_EIO;
            // the chain carries across calls, so a long page goes in pieces
            for (uint64_t off = 0; off < q.unit_size && !rc;) {
                const int n = (int)std::min<uint64_t>(q.unit_size - off, 1u << 30);
                const uint64_t at = p * q.unit_size + off;
                if (e.update(c, dst + at, &outl, src + at, n) != 1) rc = KGPU_EIO;
                off += (uint64_t)n;
            }
        }
    } else if (q.mode == KGPU_MODE_ECB) {
        if (e.init(c, e.ecb[ki], nullptr, key, nullptr, q.dir == KGPU_ENCRYPT) != 1 || e.set_padding(c, 0) != 1)
            rc = KGPU_EIO;
        for (uint64_t off = 0; off < q.len && !rc;) {
            const int n = (int)std::min<uint64_t>(q.len - off, 1u << 30);
            if (e.update(c, dst + off, &outl, src + off, n) != 1) rc = KGPU_EIO;
            off += (uint64_t)n;
        }
    } else if (q.mode == KGPU_MODE_COPY) {
        if (dst != src) std::memmove(dst, src, q.len);
    } else {
        rc = KGPU_EINVAL;
    }
    std::memset(key, 0, sizeof(key));
    return rc;
}

// Every buffer of the request is registered host memory (the host leg's
// precondition).
bool host_resident(const kgpu_request& q) {
    const bool cbc = q.mode == KGPU_MODE_CBC_DEC || q.mode == KGPU_MODE_CBC_ENC;
    const uint32_t need = KGPU_REQ_SRC_HOST | KGPU_REQ_DST_HOST | (cbc ? KGPU_REQ_IVS_HOST : 0u);
    return (q.flags & need) == need;
}

bool serving(kgpu_ctx* ctx) {
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    return ctx->serve.started;
}

uint64_t mono_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// One plain launch of the mode's kernel for request d (pointers as the device
// sees them: device memory, or registered host memory through its mapping).
cudaError_t launch_one(const kgpu_ctx* ctx, const ReqDesc& d, const HostKey& k, cudaStream_t s) {
    if (d.mode == KGPU_MODE_COPY) return launch_copy(d.src, d.dst, d.nblocks, d.unit_blocks, ctx->num_sms, s);
    if (d.mode == KGPU_MODE_XTS || d.mode == KGPU_MODE_ECB) {
        BulkParams p;
        fill_bulk(&p, k, (int)d.dir, d.src, d.dst, d.nblocks * 16, (size_t)d.unit_blocks * 16, d.first_sector);
        return d.mode == KGPU_MODE_XTS ? launch_xts(p, k.nr, (int)d.dir, ctx->num_sms, s)
                                       : launch_ecb(p, k.nr, (int)d.dir, ctx->num_sms, s);
    }
    CbcParams p;
    std::memset(&p, 0, sizeof(p));
    p.src = d.src;
    p.dst = d.dst;
    p.ivs = d.ivs;
    p.npages = d.nblocks / d.unit_blocks;
    p.bpp = d.unit_blocks;
    const bool enc = d.mode == KGPU_MODE_CBC_ENC;
    std::memcpy(p.rk, enc ? k.enc : k.dec, sizeof(p.rk));
    return enc ? launch_cbc_enc(p, k.nr, ctx->num_sms, s) : launch_cbc_dec(p, k.nr, ctx->num_sms, s);
}

// The GPU leg: the serving ring if it runs, else one launch of the mode's
// kernel waited for on an event of its own (the paper's launch, copy and wait,
// with the pages read in place).
int gpu_leg(kgpu_ctx* ctx, const kgpu_request& q, const ReqDesc& d, int64_t timeout_ns) {
    const uint64_t t0 = mono_ns();
    auto left = [&]() -> int64_t {
        if (timeout_ns < 0) return -1;
        const uint64_t el = mono_ns() - t0;
        return el >= (uint64_t)timeout_ns ? 0 : (int64_t)((uint64_t)timeout_ns - el);
    };
    if (serving(ctx)) {
        kgpu_ticket t = 0;
        int rc;
        // a full ring or the byte cap: retry until the request is admitted
        while ((rc = kgpu_serve_submit(ctx, &q, &t)) == KGPU_EBUSY) {
            if (timeout_ns >= 0 && left() == 0) return KGPU_ETIMEDOUT;
            std::this_thread::yield();
        }
        if (rc == KGPU_OK) {
            // the request holds the caller's pages until it completes, and
            // the caller has no ticket to wait on later: wait for it
            int st = 0;
            rc = kgpu_serve_poll(ctx, t, -1, &st, nullptr);
            return rc ? rc : st;
        }
        if (serving(ctx)) return rc;  // refused on its own merits
        // the ring stopped between the check and the submit: a launch instead
    }
    HostKey k;
    if (d.mode != KGPU_MODE_COPY) {
        std::lock_guard<std::mutex> g(ctx->mu);
        k = ctx->keys[d.key];
        if (!k.live) return KGPU_ENOENT;
    }
    DeviceGuard g(ctx->device);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    cudaError_t e = launch_one(ctx, d, k, ctx->crypt_stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev, ctx->crypt_stream);
    // the launch reads and writes the caller's pages: wait until it is done,
    // spinning for the first 200 us, then sleeping between checks
    const uint64_t spin_until = mono_ns() + 200000;
    if (e == cudaSuccess) {
        while ((e = cudaEventQuery(ev)) == cudaErrorNotReady)
            if (mono_ns() > spin_until) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    return KGPU_OK;
}

int crypt(kgpu_ctx* ctx, const kgpu_request& q, uint32_t dispatch, int64_t timeout_ns, uint32_t* ran_on) {
    // validation as for a batch (keys, lengths, registered ranges, overlap)
    ReqDesc d;
    RangeCache cache;
    int rc = make_desc(ctx, q, cache, 32, &d);
    if (rc) return rc;
    bool host = false;
    if (dispatch == KGPU_DISPATCH_HOST) {
        if (!host_resident(q)) return KGPU_EINVAL;
        host = true;
    } else if (dispatch == KGPU_DISPATCH_AUTO && ctx->cfg.host_dispatch && host_resident(q) &&
               q.mode <= KGPU_MODE_ECB) {
        std::lock_guard<std::mutex> lk(ctx->dispatch_mu);
        if (ctx->xover.valid) {
            int nr = 10;
            std::lock_guard<std::mutex> g(ctx->mu);
            nr = ctx->keys[q.key - 1].nr;
            host = q.len < ctx->xover.bytes[q.mode][nr == 10 ? 0 : 1];
        }
    } else if (dispatch != KGPU_DISPATCH_AUTO && dispatch != KGPU_DISPATCH_GPU) {
        return KGPU_EINVAL;
    }
    if (ran_on) *ran_on = host ? KGPU_DISPATCH_HOST : KGPU_DISPATCH_GPU;
    if (!host) {
        if (!(q.flags & (KGPU_REQ_SRC_HOST | KGPU_REQ_DST_HOST | KGPU_REQ_IVS_HOST)))
            return gpu_leg(ctx, q, d, timeout_ns);
        // host pages on the GPU: host_mu is held until the request is done,
        // so kgpu_host_unregister (which drops a range only under it) cannot
        // unpin them meanwhile; validated again under it
        std::lock_guard<std::mutex> hold(ctx->host_mu);
        RangeCache again;
        if ((rc = make_desc(ctx, q, again, 32, &d))) return rc;
        return gpu_leg(ctx, q, d, timeout_ns);
    }
    HostKey k;
    if (q.mode != KGPU_MODE_COPY) {
        std::lock_guard<std::mutex> g(ctx->mu);
        k = ctx->keys[q.key - 1];
        if (!k.live) return KGPU_ENOENT;
    }
    return host_leg(k, q);
}

}  // namespace

extern "C" {

int kgpu_crypt(kgpu_ctx* ctx, const kgpu_request* req, uint32_t dispatch, int64_t timeout_ns, uint32_t* ran_on) {
    if (!ctx || !req || req->len == 0) return KGPU_EINVAL;
    return crypt(ctx, *req, dispatch, timeout_ns, ran_on);
}

int kgpu_get_crossover(kgpu_ctx* ctx, kgpu_crossover* out) {
    if (!ctx || !out) return KGPU_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->dispatch_mu);
    *out = ctx->xover;
    return KGPU_OK;
}

int kgpu_calibrate_dispatch(kgpu_ctx* ctx, kgpu_dispatch_point* points, size_t max_points, size_t* npoints,
                            kgpu_crossover* out) {
    if (!ctx) return KGPU_EINVAL;
    if (npoints) *npoints = 0;
    if (!evp().ok) return KGPU_ENOSYS;
    constexpr uint64_t kMin = 4096, kMax = 4u << 20, kPage = 4096;
    constexpr int kModes = 4;
    const uint32_t form = serving(ctx) ? KGPU_DISPATCH_FORM_RING : KGPU_DISPATCH_FORM_LAUNCH;

    // pinned, mapped host buffers (input, output, IVs), registered with the context
    unsigned char *in = nullptr, *outb = nullptr, *ivs = nullptr;
    const size_t iv_bytes = kMax / kPage * 16;
    int rc = KGPU_OK;
    {
        DeviceGuard g(ctx->device);
        if (cudaHostAlloc(&in, kMax, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
            cudaHostAlloc(&outb, kMax, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
            cudaHostAlloc(&ivs, iv_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            rc = KGPU_ENOMEM;
        }
    }
    // inputs and keys need only be fixed bytes: this measures time, not output
    if (!rc) {
        for (size_t i = 0; i < kMax; i++) in[i] = (unsigned char)(i * 131u + 7u);
        for (size_t i = 0; i < iv_bytes; i++) ivs[i] = (unsigned char)(i * 29u + 3u);
    }
    bool reg_in = false, reg_out = false, reg_iv = false;
    if (!rc) rc = kgpu_host_register(ctx, in, kMax, KGPU_HOSTREG_PINNED), reg_in = !rc;
    if (!rc) rc = kgpu_host_register(ctx, outb, kMax, KGPU_HOSTREG_PINNED), reg_out = !rc;
    if (!rc) rc = kgpu_host_register(ctx, ivs, iv_bytes, KGPU_HOSTREG_PINNED), reg_iv = !rc;
    kgpu_key keys[2][2] = {};  // [0: single, 1: XTS][0: AES-128, 1: AES-256]
    for (int x = 0; x < 2 && !rc; x++)
        for (int b = 0; b < 2 && !rc; b++) {
            unsigned char kb[64];
            const size_t len = (size_t)(b ? 32 : 16) * (x ? 2 : 1);
            for (size_t i = 0; i < len; i++) kb[i] = (unsigned char)(i * 37u + 11u * (unsigned)(x + 2 * b) + 1u);
            rc = kgpu_aes_setkey(ctx, kb, len, x, &keys[x][b]);
        }

    kgpu_crossover xo{};
    xo.form = form;
    size_t np = 0;
    for (int m = 0; m < kModes && !rc; m++) {
        for (int b = 0; b < 2 && !rc; b++) {
            uint64_t host_ns[16] = {}, gpu_ns[16] = {}, sizes[16] = {};
            int ns = 0;
            for (uint64_t size = kMin; size <= kMax && !rc; size *= 2, ns++) {
                kgpu_request q;
                std::memset(&q, 0, sizeof(q));
                q.mode = (uint32_t)m;
                q.dir = KGPU_ENCRYPT;
                q.key = keys[m == KGPU_MODE_XTS ? 1 : 0][b];
                q.src = in;
                q.dst = outb;
                q.len = size;
                q.unit_size = kPage;
                q.ivs = ivs;
                q.flags = KGPU_REQ_SRC_HOST | KGPU_REQ_DST_HOST | KGPU_REQ_IVS_HOST;
                // repetitions: about 2 MiB of each leg per point, 5 to 41
                const int reps = (int)std::max<uint64_t>(5, std::min<uint64_t>(41, (2u << 20) / size)) | 1;
                std::vector<uint64_t> th(reps), tg(reps);
                for (int r = -1; r < reps && !rc; r++) {  // r = -1: warm-up of both legs
                    uint64_t a = mono_ns();
                    rc = crypt(ctx, q, KGPU_DISPATCH_HOST, -1, nullptr);
                    uint64_t b2 = mono_ns();
                    if (!rc) rc = crypt(ctx, q, KGPU_DISPATCH_GPU, 10000000000ll, nullptr);
                    uint64_t c2 = mono_ns();
                    if (r >= 0) {
                        th[r] = b2 - a;
                        tg[r] = c2 - b2;
                    }
                }
                if (rc) break;
                std::nth_element(th.begin(), th.begin() + reps / 2, th.end());
                std::nth_element(tg.begin(), tg.begin() + reps / 2, tg.end());
                sizes[ns] = size;
                host_ns[ns] = th[reps / 2];
                gpu_ns[ns] = tg[reps / 2];
                if (points && np < max_points) points[np] = {(uint32_t)m, b ? 256u : 128u, size, host_ns[ns], gpu_ns[ns]};
                np++;
            }
            if (rc) break;
            // the smallest size from which the GPU leg is faster at every
            // larger measured size; 2x the largest if the host leg always wins
            uint64_t cross = 2 * kMax;
            for (int i = ns - 1; i >= 0 && gpu_ns[i] < host_ns[i]; i--) cross = sizes[i];
            xo.bytes[m][b] = cross;
        }
    }
    for (int x = 0; x < 2; x++)
        for (int b = 0; b < 2; b++)
            if (keys[x][b]) kgpu_aes_delkey(ctx, keys[x][b]);
    if (reg_in) kgpu_host_unregister(ctx, in);
    if (reg_out) kgpu_host_unregister(ctx, outb);
    if (reg_iv) kgpu_host_unregister(ctx, ivs);
    {
        DeviceGuard g(ctx->device);
        if (in) cudaFreeHost(in);
        if (outb) cudaFreeHost(outb);
        if (ivs) cudaFreeHost(ivs);
    }
    if (npoints) *npoints = std::min(np, max_points);
    if (rc) return rc;
    xo.valid = 1;
    {
        std::lock_guard<std::mutex> lk(ctx->dispatch_mu);
        ctx->xover = xo;
    }
    if (out) *out = xo;
    return KGPU_OK;
}

}  // extern "C"
