// Batched submission (kgpu_submit / kgpu_poll), launch-shape tuning and the
// autotuner.  Requests are validated and packed on the host; everything they
// ask for is computed by the persistent kernel in kgpu_unified.cu.
#include <cuda_runtime.h>

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

kgpu_tuning default_tuning(const kgpu_ctx* ctx) {
    kgpu_tuning t{};
    t.threads = kBatchDefaultThreads;
    t.tile_chunks = kBatchDefaultTileChunks;
    t.ctas = (uint32_t)ctx->num_sms;
    return t;
}

kgpu_tuning effective(const kgpu_ctx* ctx) {
    kgpu_tuning t = ctx->tune;
    kgpu_tuning d = default_tuning(ctx);
    if (!t.threads) t.threads = d.threads;
    if (!t.tile_chunks) t.tile_chunks = d.tile_chunks;
    if (!t.ctas) t.ctas = d.ctas;
    return t;
}

int tuning_ok(const kgpu_tuning* t) {
    if (t->threads && t->threads != 512 && t->threads != 1024) return KGPU_EINVAL;
    if (t->tile_chunks > (1u << 20)) return KGPU_EINVAL;
    if (t->ctas > 4096) return KGPU_EINVAL;
    return KGPU_OK;
}

// Validate all requests and pack header | descriptors | tile prefix into buf
// (which must hold batch_bytes(n)).  Returns the first error, with every
// request's own code in req_status when given.
int pack_batch(kgpu_ctx* ctx, const kgpu_request* reqs, size_t n, uint32_t tile_chunks, uint64_t warps, uint8_t* buf,
               int* req_status) {
    RangeCache rc;
    int first = KGPU_OK;
    ReqDesc* descs = reinterpret_cast<ReqDesc*>(buf + batch_desc_offset());
    uint64_t* prefix = reinterpret_cast<uint64_t*>(buf + batch_prefix_offset((uint32_t)n));
    uint32_t* order = reinterpret_cast<uint32_t*>(buf + batch_order_offset((uint32_t)n));
    for (size_t i = 0; i < n; i++) {
        int r = make_desc(ctx, reqs[i], rc, tile_chunks, &descs[i]);
        if (req_status) req_status[i] = r;
        if (r && !first) first = r;
        if (r) descs[i].nblocks = 0;  // refused: no tiles
    }
    const uint64_t tiles = order_batch(descs, (uint32_t)n, [&](uint32_t i) { return descs[i].nblocks == 0; },
                                       2 * warps, prefix, order);
    BatchHeader* h = reinterpret_cast<BatchHeader*>(buf);
    h->total_tiles = tiles;
    h->nreq = (uint32_t)n;
    h->tag = 0;
    return first;
}

void free_slot(kgpu::BatchSlot& s) {
    if (s.done) cudaEventSynchronize(s.done);
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    if (s.h_buf) cudaFreeHost(s.h_buf);
    if (s.d_buf) cudaFree(s.d_buf);
    if (s.h_status) cudaFreeHost(s.h_status);
    if (s.d_status) cudaFree(s.d_status);
    if (s.d_fin) cudaFree(s.d_fin);
    if (s.h_done) cudaFreeHost(s.h_done);
    if (s.d_counter) cudaFree(s.d_counter);
    if (s.d_scratch) cudaFree(s.d_scratch);
    if (s.done) cudaEventDestroy(s.done);
    uint64_t gen = s.gen;
    s = kgpu::BatchSlot();
    s.gen = gen;
}

// Keep what polls of the slot's finished batch report once the slot is
// reused: its request count and the failed requests' codes.  Caller holds
// batch_mu; the batch has completed.
void retire(kgpu_ctx* ctx, const kgpu::BatchSlot& s) {
    kgpu::RetiredBatch r;
    r.n = s.nreq;
    for (uint32_t i = 0; i < s.nreq; i++)
        if (s.h_status[i]) r.failed.emplace_back(i, s.h_status[i]);
    ctx->retired[s.gen] = std::move(r);
    while (ctx->retired.size() > kgpu::kRetiredKept) ctx->retired.erase(ctx->retired.begin());
}

int retired_status(const kgpu::RetiredBatch& r, int* req_status) {
    if (req_status) {
        std::memset(req_status, 0, r.n * sizeof(int));
        for (const auto& f : r.failed) req_status[f.first] = f.second;
    }
    return KGPU_OK;
}

// Grow the slot's buffers to hold n requests and (re)build its graph when the
// buffers or the launch shape changed.
int prepare_slot(kgpu_ctx* ctx, kgpu::BatchSlot& s, size_t n, const kgpu_tuning& t) {
    size_t need = batch_bytes((uint32_t)n);
    bool rebuild = !s.exec || s.graph_threads != (int)t.threads || s.graph_grid != (int)t.ctas;
    if (!s.done && cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) return KGPU_EIO;
    if (!s.d_counter && cudaMalloc(&s.d_counter, 16) != cudaSuccess) return KGPU_ENOMEM;
    // staging scratch for every warp of the launch (at most 32 warps per SM;
    // warps beyond it run host-page CBC encryption unstaged)
    const uint32_t want_warps =
        (uint32_t)std::min<uint64_t>((uint64_t)t.ctas * (t.threads / 32), (uint64_t)ctx->num_sms * 32);
    if (s.scratch_warps < want_warps) {
        if (s.d_scratch) cudaFree(s.d_scratch);
        s.d_scratch = nullptr;
        s.scratch_warps = 0;
        if (cudaMalloc(&s.d_scratch, (size_t)want_warps * kStageWarpBytes) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_ENOMEM;
        }
        s.scratch_warps = want_warps;
        rebuild = true;
    }
    if (s.cap < need || s.status_cap < n) {
        size_t cap = std::max(need, s.cap * 2);
        size_t scap = std::max(n, s.status_cap * 2);
        if (s.exec) cudaGraphExecDestroy(s.exec);
        if (s.graph) cudaGraphDestroy(s.graph);
        s.exec = nullptr;
        s.graph = nullptr;
        if (s.h_buf) cudaFreeHost(s.h_buf);
        if (s.d_buf) cudaFree(s.d_buf);
        if (s.h_status) cudaFreeHost(s.h_status);
        if (s.d_status) cudaFree(s.d_status);
        if (s.d_fin) cudaFree(s.d_fin);
        if (s.h_done) cudaFreeHost(s.h_done);
        s.h_buf = nullptr;
        s.d_buf = nullptr;
        s.h_status = nullptr;
        s.d_status = nullptr;
        s.d_fin = nullptr;
        s.h_done = nullptr;
        s.d_done = nullptr;
        s.cap = s.status_cap = 0;
        if (cudaHostAlloc(&s.h_buf, cap, cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&s.d_buf, cap) != cudaSuccess ||
            cudaHostAlloc(&s.h_status, scap * sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&s.d_status, scap * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&s.d_fin, scap * sizeof(unsigned long long)) != cudaSuccess ||
            cudaHostAlloc(&s.h_done, scap * sizeof(unsigned long long), cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess ||
            cudaHostGetDevicePointer(reinterpret_cast<void**>(&s.d_done), s.h_done, 0) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_ENOMEM;
        }
        std::memset(s.h_done, 0, scap * sizeof(unsigned long long));
        s.cap = cap;
        s.status_cap = scap;
        rebuild = true;
    }
    if (!rebuild) return KGPU_OK;
    if (s.exec) cudaGraphExecDestroy(s.exec);
    if (s.graph) cudaGraphDestroy(s.graph);
    s.exec = nullptr;
    s.graph = nullptr;

    s.args = BatchArgs{};
    s.args.buf = s.d_buf;
    s.args.keys = ctx->d_keys;
    s.args.max_keys = ctx->cfg.max_keys;
    s.args.next_tile = s.d_counter;
    s.args.status = s.d_status;
    s.args.scratch = s.d_scratch;
    s.args.scratch_warps = s.scratch_warps;
    s.args.fin = s.d_fin;
    s.args.done = s.d_done;

    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return KGPU_EIO;
    cudaGraphNode_t n_ctr = nullptr;
    bool ok = cudaGraphAddMemcpyNode1D(&s.n_copy, g, nullptr, 0, s.d_buf, s.h_buf, s.cap,
                                       cudaMemcpyHostToDevice) == cudaSuccess;
    cudaMemsetParams mp{};
    mp.dst = s.d_counter;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    ok = ok && cudaGraphAddMemsetNode(&n_ctr, g, nullptr, 0, &mp) == cudaSuccess;
    mp.dst = s.d_status;
    mp.width = s.status_cap;
    ok = ok && cudaGraphAddMemsetNode(&s.n_status_clear, g, nullptr, 0, &mp) == cudaSuccess;
    mp.dst = s.d_fin;
    mp.width = 2 * s.status_cap;
    ok = ok && cudaGraphAddMemsetNode(&s.n_fin_clear, g, nullptr, 0, &mp) == cudaSuccess;
    cudaKernelNodeParams kp{};
    void* kargs[] = {&s.args};
    kp.func = const_cast<void*>(batch_kernel_fn((int)t.threads));
    kp.gridDim = dim3(t.ctas);
    kp.blockDim = dim3(t.threads);
    kp.sharedMemBytes = (unsigned)batch_smem_bytes((int)t.threads);
    kp.kernelParams = kargs;
    cudaGraphNode_t deps[4] = {s.n_copy, n_ctr, s.n_status_clear, s.n_fin_clear};
    ok = ok && kp.func && cudaGraphAddKernelNode(&s.n_kernel, g, deps, 4, &kp) == cudaSuccess;
    ok = ok && cudaGraphAddMemcpyNode1D(&s.n_status_out, g, &s.n_kernel, 1, s.h_status, s.d_status,
                                        s.status_cap * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaGraphInstantiate(&s.exec, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        s.exec = nullptr;
        return KGPU_EIO;
    }
    s.graph = g;
    s.graph_threads = (int)t.threads;
    s.graph_grid = (int)t.ctas;
    return KGPU_OK;
}

int launch_slot(kgpu::BatchSlot& s, size_t n, cudaStream_t stream) {
    const size_t bytes = batch_bytes((uint32_t)n);
    bool ok = cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.n_copy, s.d_buf, s.h_buf, bytes,
                                                 cudaMemcpyHostToDevice) == cudaSuccess;
    cudaMemsetParams mp{};
    mp.dst = s.d_status;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = n;
    mp.height = 1;
    ok = ok && cudaGraphExecMemsetNodeSetParams(s.exec, s.n_status_clear, &mp) == cudaSuccess;
    mp.dst = s.d_fin;
    mp.width = 2 * n;
    ok = ok && cudaGraphExecMemsetNodeSetParams(s.exec, s.n_fin_clear, &mp) == cudaSuccess;
    ok = ok && cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.n_status_out, s.h_status, s.d_status, n * sizeof(int),
                                                  cudaMemcpyDeviceToHost) == cudaSuccess;
    ok = ok && cudaGraphLaunch(s.exec, stream) == cudaSuccess;
    ok = ok && cudaEventRecord(s.done, stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    return KGPU_OK;
}

}  // namespace

namespace kgpu {
namespace hostutil {

int batches_quiesce(kgpu_ctx* ctx) {
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    DeviceGuard g(ctx->device);
    for (auto& s : ctx->slots) {
        if (s.issued && s.done && cudaEventSynchronize(s.done) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_EIO;
        }
    }
    // allocation-free batches: every one issued before this call is ordered
    // before the newest on its stream, or was synchronised by its caller
    if (ctx->noalloc_issued && cudaEventSynchronize(ctx->noalloc_done) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    return KGPU_OK;
}

void destroy_batch_slots(kgpu_ctx* ctx) {
    for (auto& s : ctx->slots) free_slot(s);
}

}  // namespace hostutil
}  // namespace kgpu

extern "C" {

int kgpu_set_tuning(kgpu_ctx* ctx, const kgpu_tuning* t) {
    if (!ctx || !t) return KGPU_EINVAL;
    int rc = tuning_ok(t);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    ctx->tune = *t;
    return KGPU_OK;
}

int kgpu_get_tuning(kgpu_ctx* ctx, kgpu_tuning* t) {
    if (!ctx || !t) return KGPU_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    *t = effective(ctx);
    return KGPU_OK;
}

int kgpu_submit(kgpu_ctx* ctx, const kgpu_request* reqs, size_t n, kgpu_stream stream, kgpu_ticket* out,
                int* req_status) {
    if (!ctx || !out || (n && !reqs) || n > (1u << 24)) return KGPU_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    DeviceGuard g(ctx->device);
    kgpu_tuning t = effective(ctx);
    // CBC encryption of host pages is staged only in the 512-thread kernel
    if (t.threads > 512 && needs_staging(reqs, n)) t.threads = 512;
    const uint64_t ticket = ++ctx->next_ticket;
    kgpu::BatchSlot& s = ctx->slots[ticket % kBatchSlots];
    // a batch someone waits on (kgpu_poll, kgpu_poll_each) keeps its slot
    if (s.pollers > 0) {
        --ctx->next_ticket;
        return KGPU_EBUSY;
    }
    // rotate: the slot's previous batch must have finished before its
    // staging buffers are refilled; its polls keep working from the record
    if (s.issued) {
        if (cudaEventSynchronize(s.done) != cudaSuccess) {
            cudaGetLastError();
            return KGPU_EIO;
        }
        retire(ctx, s);
    }
    s.issued = false;
    int rc = prepare_slot(ctx, s, n ? n : 1, t);
    if (rc) return rc;
    rc = pack_batch(ctx, reqs, n, t.tile_chunks, (uint64_t)t.ctas * (t.threads / 32), s.h_buf, req_status);
    if (rc) return rc;
    s.nreq = (uint32_t)n;
    s.gen = ticket;
    s.tag = (uint32_t)(ticket % 0xFFFFFFFFull) + 1u;  // never 0, the value of a fresh word
    reinterpret_cast<BatchHeader*>(s.h_buf)->tag = s.tag;
    if (n) {
        if ((rc = launch_slot(s, n, (cudaStream_t)stream))) return rc;
    } else if (cudaEventRecord(s.done, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    s.issued = true;
    *out = ticket;
    return KGPU_OK;
}

int kgpu_poll_each(kgpu_ctx* ctx, kgpu_ticket ticket, int64_t timeout_ns, int* req_status, uint64_t* done_ns) {
    if (!ctx || !done_ns) return KGPU_EINVAL;
    const unsigned long long* words;
    uint32_t n, tag;
    std::vector<uint8_t> empty;  // requests with no tiles (len 0) complete at once
    {
        std::lock_guard<std::mutex> lk(ctx->batch_mu);
        kgpu::BatchSlot& s = ctx->slots[ticket % kBatchSlots];
        if (ticket == 0 || ticket > ctx->next_ticket) return KGPU_ENOENT;
        if (s.gen != ticket || !s.issued) {  // complete, slot since reused: times unknown
            auto it = ctx->retired.find(ticket);
            if (it == ctx->retired.end()) return KGPU_ENOENT;
            for (uint32_t i = 0; i < it->second.n; i++) done_ns[i] = 0;
            return retired_status(it->second, req_status);
        }
        words = s.h_done;
        n = s.nreq;
        tag = s.tag;
        s.pollers++;
        const ReqDesc* descs = reinterpret_cast<const ReqDesc*>(s.h_buf + batch_desc_offset());
        empty.resize(n);
        for (uint32_t i = 0; i < n; i++) empty[i] = descs[i].nblocks == 0;
    }
    auto now = []() {
        return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now().time_since_epoch())
            .count();
    };
    const uint64_t t0 = now();
    const uint64_t deadline = timeout_ns < 0 ? UINT64_MAX : t0 + (uint64_t)timeout_ns;
    std::vector<uint32_t> pending;
    pending.reserve(n);
    for (uint32_t i = 0; i < n; i++) {
        done_ns[i] = 0;
        if (empty[i]) done_ns[i] = t0;
        else pending.push_back(i);
    }
    int rc = KGPU_OK;
    std::vector<uint32_t> found;
    found.reserve(n);
    while (!pending.empty()) {
        size_t keep = 0;
        found.clear();
        for (uint32_t i : pending) {
            const unsigned long long v = __atomic_load_n(&words[i], __ATOMIC_ACQUIRE);
            if ((uint32_t)(v >> 32) == tag) found.push_back(i);
            else pending[keep++] = i;
        }
        // completions are stamped with the time after the scan that saw them:
        // late by at most the scan, never early
        const uint64_t t = now();
        for (uint32_t i : found) done_ns[i] = t;
        pending.resize(keep);
        if (!pending.empty() && t >= deadline) {
            rc = KGPU_ETIMEDOUT;
            break;
        }
    }
    // every request is complete; the status copy ends the batch's graph
    if (!rc) rc = kgpu_poll(ctx, ticket, -1, req_status);
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    ctx->slots[ticket % kBatchSlots].pollers--;
    return rc;
}

int kgpu_poll(kgpu_ctx* ctx, kgpu_ticket ticket, int64_t timeout_ns, int* req_status) {
    if (!ctx) return KGPU_EINVAL;
    cudaEvent_t ev;
    {
        std::lock_guard<std::mutex> lk(ctx->batch_mu);
        kgpu::BatchSlot& s = ctx->slots[ticket % kBatchSlots];
        if (ticket == 0 || ticket > ctx->next_ticket) return KGPU_ENOENT;
        if (s.gen != ticket || !s.issued) {  // complete, slot since reused
            auto it = ctx->retired.find(ticket);
            return it == ctx->retired.end() ? KGPU_ENOENT : retired_status(it->second, req_status);
        }
        ev = s.done;
        s.pollers++;  // the slot is not reused while this call waits on it
    }
    DeviceGuard g(ctx->device);
    cudaError_t e;
    if (timeout_ns < 0) {
        e = cudaEventSynchronize(ev);
    } else {
        // spin for the first 200 us (a short batch is done well within it,
        // and a sleep costs tens of microseconds of timer slack), then sleep
        // between checks
        const auto start = std::chrono::steady_clock::now();
        const auto deadline = start + std::chrono::nanoseconds(timeout_ns);
        for (;;) {
            e = cudaEventQuery(ev);
            const auto now = std::chrono::steady_clock::now();
            if (e != cudaErrorNotReady || now >= deadline) break;
            if (now - start > std::chrono::microseconds(200))
                std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    kgpu::BatchSlot& s = ctx->slots[ticket % kBatchSlots];
    s.pollers--;
    if (e == cudaErrorNotReady) return KGPU_ETIMEDOUT;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    if (req_status && s.nreq) std::memcpy(req_status, s.h_status, s.nreq * sizeof(int));
    return KGPU_OK;
}

int kgpu_autotune(kgpu_ctx* ctx, const kgpu_request* reqs, size_t n, kgpu_stream stream, uint32_t iters,
                  kgpu_tuning* best, float* best_ms) {
    if (!ctx || !reqs || !n || !best || n > (1u << 24)) return KGPU_EINVAL;
    for (size_t i = 0; i < n; i++)
        if (reqs[i].src == reqs[i].dst && reqs[i].len) return KGPU_EINVAL;
    if (iters == 0) iters = 3;
    std::lock_guard<std::mutex> lk(ctx->batch_mu);
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t thread_opts[] = {1024, 512};
    const uint32_t tile_opts[] = {8, 16, 32, 64, 128};
    size_t bytes = batch_bytes((uint32_t)n);
    std::vector<uint8_t> hbuf(bytes);
    uint8_t* dbuf = nullptr;
    unsigned long long* ctr = nullptr;
    int* status = nullptr;
    uint4* scratch = nullptr;
    const uint32_t scratch_warps = (uint32_t)ctx->num_sms * 32;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = KGPU_OK;
    if (cudaMalloc(&dbuf, bytes) != cudaSuccess || cudaMalloc(&ctr, 16) != cudaSuccess ||
        cudaMalloc(&scratch, (size_t)scratch_warps * kStageWarpBytes) != cudaSuccess ||
        cudaMalloc(&status, n * sizeof(int)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        rc = KGPU_ENOMEM;
    }
    kgpu_tuning chosen = effective(ctx);
    float chosen_ms = -1.f;
    for (uint32_t tc : tile_opts) {
        if (rc) break;
        for (uint32_t th : thread_opts) {
            // the run order's tail reserve depends on the warp count
            rc = pack_batch(ctx, reqs, n, tc, (uint64_t)ctx->num_sms * (th / 32), hbuf.data(), nullptr);
            if (rc) break;
            if (cudaMemcpy(dbuf, hbuf.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = KGPU_EIO;
                break;
            }
            BatchArgs a{};
            a.buf = dbuf;
            a.keys = ctx->d_keys;
            a.max_keys = ctx->cfg.max_keys;
            a.next_tile = ctr;
            a.status = status;
            a.scratch = scratch;
            a.scratch_warps = scratch_warps;
            float total = 0.f;
            bool ok = true;
            for (uint32_t it = 0; it <= iters && ok; it++) {
                ok = cudaMemsetAsync(ctr, 0, 16, st) == cudaSuccess;
                ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
                ok = ok && launch_batch(a, (int)th, ctx->num_sms, st) == cudaSuccess;
                ok = ok && cudaEventRecord(e1, st) == cudaSuccess;
                ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0.f;
                ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                if (it) total += ms;  // the first run is the warm-up
            }
            if (!ok) {
                cudaGetLastError();
                rc = KGPU_EIO;
                break;
            }
            float mean = total / iters;
            if (chosen_ms < 0 || mean < chosen_ms) {
                chosen_ms = mean;
                chosen.threads = th;
                chosen.tile_chunks = tc;
                chosen.ctas = (uint32_t)ctx->num_sms;
            }
        }
    }
    if (dbuf) cudaFree(dbuf);
    if (ctr) cudaFree(ctr);
    if (status) cudaFree(status);
    if (scratch) cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    ctx->tune = chosen;
    *best = chosen;
    if (best_ms) *best_ms = chosen_ms;
    return KGPU_OK;
}

}  // extern "C"
