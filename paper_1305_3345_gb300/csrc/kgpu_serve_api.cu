// Serving loop host side (kgpu_serve_*) and the trace-replay load generators
// (kgpu_replay_*).  The host validates requests, writes descriptors into the
// mapped ring and publishes them; the persistent kernel in kgpu_unified.cu
// does all the work and publishes completions back into the ring.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "kgpu_ctx.h"

using namespace kgpu;
using namespace kgpu::hostutil;

namespace {

// Words per request of kgpu_replay_serve_stages: published, dispatcher took
// it, tiles published, first tile started, completed, seen by the host.
constexpr size_t kStageWords = 6;

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// Wait for a trace's arrival time.  A sleeping thread may wake as late as the
// kernel's timer slack (50 us by default on Linux) after its timeout, so the
// load generators sleep only while they are far ahead and spin the rest.
void wait_until(uint64_t target) {
    for (uint64_t t = now_ns(); t < target; t = now_ns())
        if (target - t > 200000) std::this_thread::sleep_for(std::chrono::microseconds(20));
}

template <class T>
T load_acquire(const T* p) {
    return __atomic_load_n(p, __ATOMIC_ACQUIRE);
}

template <class T>
void store_release(T* p, T v) {
    __atomic_store_n(p, v, __ATOMIC_RELEASE);
}

void cpu_relax() { std::this_thread::yield(); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void serve_free(ServeState& st) {
    if (st.stream) {
        cudaStreamSynchronize(st.stream);
        cudaStreamDestroy(st.stream);
    }
    if (st.kdone) cudaEventDestroy(st.kdone);
    if (st.host_mem) cudaFreeHost(st.host_mem);
    if (st.dev_mem) cudaFree(st.dev_mem);
    st = ServeState();
}

int serve_alloc(kgpu_ctx* ctx, ServeState& st, const kgpu_serve_config* cfg) {
    kgpu_serve_config c{};
    if (cfg) c = *cfg;
    uint32_t S = c.ring_slots ? c.ring_slots : ctx->cfg.ring_slots;
    if (S < 2 || (S & (S - 1)) || S > (1u << 20)) return KGPU_EINVAL;
    st.nslots = S;
    // 1-KiB tiles when the ring keeps up: a lone request's pages spread over
    // more warps, each running its tile in one two-block step (one-at-a-time
    // 4-KiB XTS round trip p50: 2-KiB tiles 13.1 us, 1 KiB 11.4, 512 B 11.3;
    // XTS p50 at 100k requests/s 15.1, 13.6, 14.2 us); under backlog stage()
    // switches to 32-KiB tiles
    st.tile_chunks = c.tile_chunks ? c.tile_chunks : 2;
    if (st.tile_chunks > (1u << 20)) return KGPU_EINVAL;
    st.admit_bytes = c.admit_bytes ? c.admit_bytes : ctx->cfg.admit_bytes;
    const uint64_t idle = c.idle_timeout_ns ? c.idle_timeout_ns : ctx->cfg.idle_timeout_ns;
    const uint64_t life = c.lifetime_ns ? c.lifetime_ns : 30000000000ull;

    const size_t o_slots = sizeof(ServeHostHdr);
    const size_t o_done = o_slots + (size_t)S * sizeof(ServeSlot);
    const size_t o_status = o_done + (size_t)S * 8;
    const size_t o_stamps = align_up(o_status + (size_t)S * 4, 128);  // kStamps arrays of S words
    const size_t host_bytes = o_stamps + (size_t)ServeState::kStamps * S * 8;
    // tile ring: room for every tile admission allows in flight, plus slack
    uint64_t want = st.admit_bytes / ((uint64_t)st.tile_chunks * 512) + 2ull * S;
    uint64_t T = 1ull << 16;
    while (T < want && T < (1ull << 24)) T <<= 1;
    st.tile_ring = T;
    const size_t d_slots = sizeof(ServeDev), d_fin = d_slots + (size_t)S * sizeof(ServeSlot);
    const size_t d_tiles = d_fin + (size_t)S * 8;
    const size_t d_mbox = d_tiles + (size_t)T * 8;
    const size_t d_scratch = align_up(d_mbox + (size_t)ctx->num_sms * kMboxStride * 8, 256);
    const uint32_t scratch_warps = (uint32_t)ctx->num_sms * (kServeThreads / 32);
    const size_t dev_bytes = d_scratch + (size_t)scratch_warps * kStageWarpBytes;

    if (cudaHostAlloc(&st.host_mem, host_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaMalloc(&st.dev_mem, dev_bytes) != cudaSuccess ||
        cudaMemset(st.dev_mem, 0, dev_bytes) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&st.kdone, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        serve_free(st);
        return KGPU_ENOMEM;
    }
    std::memset(st.host_mem, 0, host_bytes);
    uint8_t* dmap = nullptr;
    if (cudaHostGetDevicePointer((void**)&dmap, st.host_mem, 0) != cudaSuccess) {
        cudaGetLastError();
        serve_free(st);
        return KGPU_EIO;
    }
    st.hdr = reinterpret_cast<ServeHostHdr*>(st.host_mem);
    st.slots = reinterpret_cast<ServeSlot*>(st.host_mem + o_slots);
    st.done_seq = reinterpret_cast<unsigned long long*>(st.host_mem + o_done);
    st.status = reinterpret_cast<int*>(st.host_mem + o_status);
    for (int k = 0; k < ServeState::kStamps; k++)
        st.stamp[k] = reinterpret_cast<unsigned long long*>(st.host_mem + o_stamps + (size_t)k * S * 8);

    ServeArgs& a = st.args;
    a = ServeArgs{};
    a.slots = reinterpret_cast<const ServeSlot*>(dmap + o_slots);
    a.hh = reinterpret_cast<ServeHostHdr*>(dmap);
    a.done_seq = reinterpret_cast<unsigned long long*>(dmap + o_done);
    a.status = reinterpret_cast<int*>(dmap + o_status);
    a.t_disp = reinterpret_cast<unsigned long long*>(dmap + o_stamps);
    a.t_pub = reinterpret_cast<unsigned long long*>(dmap + o_stamps + (size_t)S * 8);
    a.t_start = reinterpret_cast<unsigned long long*>(dmap + o_stamps + (size_t)2 * S * 8);
    a.t_done = reinterpret_cast<unsigned long long*>(dmap + o_stamps + (size_t)3 * S * 8);
    a.dev = reinterpret_cast<ServeDev*>(st.dev_mem);
    a.dslots = reinterpret_cast<ServeSlot*>(st.dev_mem + d_slots);
    a.fin = reinterpret_cast<unsigned long long*>(st.dev_mem + d_fin);
    a.tiles = reinterpret_cast<unsigned long long*>(st.dev_mem + d_tiles);
    a.tile_mask = T - 1;
    a.mbox = reinterpret_cast<unsigned long long*>(st.dev_mem + d_mbox);
    a.scratch = reinterpret_cast<uint4*>(st.dev_mem + d_scratch);
    a.scratch_warps = scratch_warps;
    a.tile_bits = 0;
    while ((1ull << a.tile_bits) < T) a.tile_bits++;
    a.keys = ctx->d_keys;
    a.max_keys = ctx->cfg.max_keys;
    a.slot_mask = S - 1;
    a.idle_ns = idle;
    a.lifetime_ns = life;

    st.slot_busy.assign(S, 0);
    st.slot_seq.assign(S, 0);
    st.slot_len.assign(S, 0);
    st.slot_gen.assign(S, UINT64_MAX);
    st.ret_seq.assign(S, UINT64_MAX);
    for (auto& r : st.ret_stamp) r.assign(S, 0);
    st.ret_status.assign(S, 0);
    st.failed.clear();
    st.outstanding.clear();
    st.outstanding.reserve(S);
    st.started = true;
    return KGPU_OK;
}

// (Re)launch the serving kernel if no instance is running.  Caller holds serve_mu.
int ensure_running(kgpu_ctx* ctx, ServeState& st) {
    if (st.running) {
        cudaError_t e = cudaEventQuery(st.kdone);
        if (e == cudaErrorNotReady) return KGPU_OK;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return KGPU_EIO;
        }
        st.running = false;
        st.last_exit = (unsigned)load_acquire(&st.hdr->exit_code);
    }
    store_release(&st.hdr->stop, 0u);
    store_release(&st.hdr->exit_code, 0ull);
    DeviceGuard g(ctx->device);
    if (launch_serve_reset(reinterpret_cast<ServeDev*>(st.dev_mem), st.args.mbox, ctx->num_sms, st.stream) !=
            cudaSuccess ||
        launch_serve(st.args, kServeThreads, ctx->num_sms, st.stream) != cudaSuccess ||
        cudaEventRecord(st.kdone, st.stream) != cudaSuccess) {
        cudaGetLastError();
        return KGPU_EIO;
    }
    st.running = true;
    st.launches++;
    return KGPU_OK;
}

// Retire every outstanding request whose completion the device has published.
// Failed requests whose codes are kept for kgpu_serve_poll after their slot
// has been reused.
constexpr size_t kFailedKept = 4096;

// Retire every outstanding request the device has completed.  The slot's
// status and stamps are the request's own here: the device wrote them before
// its completion word, and the slot is not staged again before this runs.
void reap(ServeState& st) {
    size_t w = 0;
    for (size_t i = 0; i < st.outstanding.size(); i++) {
        const uint64_t seq = st.outstanding[i];
        const uint32_t s = (uint32_t)(seq & (st.nslots - 1));
        if (load_acquire(&st.done_seq[s]) >= seq + 1) {
            const int code = load_acquire(&st.status[s]);
            __atomic_store_n(&st.ret_seq[s], UINT64_MAX, __ATOMIC_RELAXED);
            __atomic_thread_fence(__ATOMIC_RELEASE);
            __atomic_store_n(&st.ret_status[s], code, __ATOMIC_RELAXED);
            for (int k = 0; k < ServeState::kStamps; k++)
                __atomic_store_n(&st.ret_stamp[k][s], (uint64_t)load_acquire(&st.stamp[k][s]), __ATOMIC_RELAXED);
            __atomic_store_n(&st.ret_seq[s], seq, __ATOMIC_RELEASE);
            if (code) {
                st.failed[seq] = code;
                if (st.failed.size() > kFailedKept) st.failed.erase(st.failed.begin());
            }
            st.slot_busy[s] = 0;
            st.inflight_bytes -= st.slot_len[s];
            st.completed++;
        } else {
            st.outstanding[w++] = seq;
        }
    }
    st.outstanding.resize(w);
}

// The device's status and stamps for request seq, which the caller has seen
// complete (done_seq of its slot >= seq + 1, acquire), without serve_mu: from
// the slot's mapped words while the slot still holds seq, else from reap's
// record of it.  false when the slot has since retired a later request too.
// stamps: ServeState::kStamps words (dispatcher took it, tiles published,
// first tile started, completed).
bool read_completed(const ServeState& st, uint64_t seq, int* status, uint64_t* stamps) {
    const uint32_t s = (uint32_t)(seq & (st.nslots - 1));
    uint64_t v[ServeState::kStamps];
    if (__atomic_load_n(&st.slot_gen[s], __ATOMIC_ACQUIRE) == seq) {
        const int c = load_acquire(&st.status[s]);
        for (int k = 0; k < ServeState::kStamps; k++) v[k] = load_acquire(&st.stamp[k][s]);
        __atomic_thread_fence(__ATOMIC_ACQUIRE);
        if (__atomic_load_n(&st.slot_gen[s], __ATOMIC_RELAXED) == seq) {
            *status = c;
            for (int k = 0; k < ServeState::kStamps; k++) stamps[k] = v[k];
            return true;
        }
    }
    if (__atomic_load_n(&st.ret_seq[s], __ATOMIC_ACQUIRE) == seq) {
        const int c = __atomic_load_n(&st.ret_status[s], __ATOMIC_RELAXED);
        for (int k = 0; k < ServeState::kStamps; k++) v[k] = __atomic_load_n(&st.ret_stamp[k][s], __ATOMIC_RELAXED);
        __atomic_thread_fence(__ATOMIC_ACQUIRE);
        if (__atomic_load_n(&st.ret_seq[s], __ATOMIC_RELAXED) == seq) {
            *status = c;
            for (int k = 0; k < ServeState::kStamps; k++) stamps[k] = v[k];
            return true;
        }
    }
    return false;
}

// Leaves the readers count of a call that read the ring outside serve_mu.
struct ReaderGuard {
    kgpu_ctx* ctx;
    explicit ReaderGuard(kgpu_ctx* c) : ctx(c) {}
    ~ReaderGuard() {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        ctx->serve.readers--;
    }
    ReaderGuard(const ReaderGuard&) = delete;
    ReaderGuard& operator=(const ReaderGuard&) = delete;
};

// Publish a validated descriptor.  Caller holds serve_mu.
// Tile size of requests staged while the ring is backed up (512-byte chunks).
constexpr uint32_t kBacklogTileChunks = 64;  // 32 KiB

// Write one request into the next ring slot, without making it visible to
// the device yet (commit does that).  Caller holds serve_mu.
//
// Under backlog -- the request published a quarter of the ring ago is still
// running -- a new request waits behind the queue whatever its tile size, so
// it gets 32-KiB tiles: per tile the workers claim a position, reload a key
// schedule and (for XTS) run a 32-unit tweak batch, and on small tiles those
// costs cap the ring's throughput.  A ring that keeps up keeps the configured
// (default 2-KiB) tiles and their lower latency, and runs CBC encryption four
// lanes to a page (twice the chain speed, a quarter of the pages per warp;
// host pages through the warp's scratch area, whole lines at a time).  The
// check is one load of a completion word, whatever the number of requests in
// flight.
bool backlogged(const ServeState& st) {
    const uint64_t q = st.nslots / 4;
    if (st.next_seq < q) return false;
    const uint64_t seq = st.next_seq - q;
    return load_acquire(&st.done_seq[seq & (st.nslots - 1)]) < seq + 1;
}

int stage(ServeState& st, const ReqDesc& dreq, uint64_t* seq_out) {
    ReqDesc d = dreq;
    if (backlogged(st)) {
        set_tile_units(d, std::max<uint32_t>(st.tile_chunks, kBacklogTileChunks));
    } else if (d.mode == KGPU_MODE_CBC_ENC &&
               (!(d.flags & (kDescSrcHost | kDescDstHost)) || d.unit_blocks % kStageBlocks == 0)) {
        // a CBC-encryption request's latency is its chain time: while the ring
        // keeps up, four lanes share each page's chain (8 pages a warp); host
        // pages take the staged form of it, which needs whole 128-byte lines
        d.flags |= kDescQuad;
        d.tile_units = kQuadPages;
    }
    const uint64_t len = d.nblocks * 16;
    const uint64_t units = request_units(d);
    const uint64_t nt = (units + d.tile_units - 1) / d.tile_units;
    if (nt == 0 || nt > serve_max_tiles(st.tile_ring)) return KGPU_EINVAL;
    const uint64_t seq = st.next_seq;
    const uint32_t s = (uint32_t)(seq & (st.nslots - 1));
    auto refused = [&]() {
        return st.slot_busy[s] || (st.inflight_bytes > 0 && st.inflight_bytes + len > st.admit_bytes);
    };
    if (refused()) {
        reap(st);
        if (refused()) {
            st.busy_refusals++;
            return KGPU_EBUSY;
        }
    }
    ServeSlot& sl = st.slots[s];
    sl.d = d;
    sl.ntiles = nt;
    sl.seq = seq;
    // clear the slot's mapped words inside the generation's sequence lock
    __atomic_store_n(&st.slot_gen[s], UINT64_MAX, __ATOMIC_RELAXED);
    __atomic_thread_fence(__ATOMIC_RELEASE);
    __atomic_store_n(&st.status[s], 0, __ATOMIC_RELAXED);
    for (int k = 0; k < ServeState::kStamps; k++) __atomic_store_n(&st.stamp[k][s], 0ull, __ATOMIC_RELAXED);
    __atomic_store_n(&st.slot_gen[s], seq, __ATOMIC_RELEASE);
    st.slot_busy[s] = 1;
    st.slot_seq[s] = seq;
    st.slot_len[s] = len;
    st.inflight_bytes += len;
    st.outstanding.push_back(seq);
    st.next_seq++;
    st.submitted++;
    *seq_out = seq;
    return KGPU_OK;
}

// Publish every staged request with one release store of the ring head (the
// device's dispatcher polls that word over the host link, so one store per
// burst instead of one per request), then make sure a kernel is running.
int commit(kgpu_ctx* ctx, ServeState& st) {
    store_release(&st.hdr->head, (unsigned long long)st.next_seq);
    const uint64_t t = now_ns();
    st.last_publish_ns = t;
    if (!st.running || t - st.last_alive_check > 20000) {
        st.last_alive_check = t;
        return ensure_running(ctx, st);
    }
    return KGPU_OK;
}

int publish(kgpu_ctx* ctx, ServeState& st, const ReqDesc& d, uint64_t* seq_out) {
    int r = stage(st, d, seq_out);
    return r ? r : commit(ctx, st);
}

// The completion thread of kgpu_serve_submit_cb.  It scans the registered
// callbacks for requests whose completion the device has published and runs
// them one at a time, holding no lock.  Between scans it yields; after 200 us
// without a completion it sleeps 20 us at a time.  While callbacks wait it
// also relaunches the kernel if that exited with work pending, as a poll
// would.  Told to stop (once the ring's kernel has stopped), it runs what is
// left -- completed requests with their status, the rest with KGPU_ENOENT --
// and exits.  The ring's mapped words stay valid meanwhile: the ring is freed
// only after this thread has been joined.
void callback_loop(kgpu_ctx* ctx) {
    ServeState& st = ctx->serve;
    std::vector<ServeCallback> ready;
    uint64_t last_progress = now_ns(), last_check = last_progress;
    bool failing = false;  // the kernel could not be relaunched: what waits now gets KGPU_EIO
    for (;;) {
        bool stop = false;
        {
            std::unique_lock<std::mutex> lk(ctx->cb_mu);
            ctx->cb_cv.wait(lk, [&] { return !ctx->cb_pending.empty() || ctx->cb_stop; });
            stop = ctx->cb_stop;
            if (stop && ctx->cb_pending.empty()) return;
            size_t w = 0;
            for (size_t i = 0; i < ctx->cb_pending.size(); i++) {
                const ServeCallback& e = ctx->cb_pending[i];
                const uint32_t s = (uint32_t)(e.seq & (st.nslots - 1));
                if (stop || failing || load_acquire(&st.done_seq[s]) >= e.seq + 1) ready.push_back(e);
                else ctx->cb_pending[w++] = e;
            }
            ctx->cb_pending.resize(w);
        }
        failing = false;
        for (const ServeCallback& e : ready) {
            const uint32_t s = (uint32_t)(e.seq & (st.nslots - 1));
            // an incomplete request was taken only because the ring stopped
            // or the kernel could not be relaunched
            int code = stop ? KGPU_ENOENT : KGPU_EIO;
            if (load_acquire(&st.done_seq[s]) >= e.seq + 1) {
                uint64_t v[ServeState::kStamps] = {};
                if (!read_completed(st, e.seq, &code, v)) {  // slot since reused: failures are kept by ticket
                    std::lock_guard<std::mutex> lk(ctx->serve_mu);
                    auto f = st.failed.find(e.seq);
                    code = f != st.failed.end() ? f->second : 0;
                }
            }
            e.fn(e.arg, (kgpu_ticket)(e.seq + 1), code);
        }
        const uint64_t t = now_ns();
        if (!ready.empty()) last_progress = t;
        ready.clear();
        if (stop) continue;
        if (t - last_check > 50000) {
            last_check = t;
            std::lock_guard<std::mutex> lk(ctx->serve_mu);
            if (!st.closing) {
                reap(st);
                if (!st.outstanding.empty() && ensure_running(ctx, st)) failing = true;
            }
        }
        if (t - last_progress > 200000) std::this_thread::sleep_for(std::chrono::microseconds(20));
        else cpu_relax();
    }
}

bool on_callback_thread(const kgpu_ctx* ctx) {
    return ctx->cb_thread.joinable() && ctx->cb_thread.get_id() == std::this_thread::get_id();
}

// Join the completion thread (serve_mu held on entry and on return, released
// meanwhile, since callbacks may take it): it runs every callback still
// registered and exits.  The ring's kernel must have stopped.
void stop_callbacks(kgpu_ctx* ctx, std::unique_lock<std::mutex>& lk) {
    if (!ctx->cb_thread.joinable()) return;
    {
        std::lock_guard<std::mutex> g(ctx->cb_mu);
        ctx->cb_stop = true;
    }
    ctx->cb_cv.notify_all();
    std::thread t = std::move(ctx->cb_thread);
    lk.unlock();
    t.join();
    lk.lock();
    std::lock_guard<std::mutex> g(ctx->cb_mu);
    ctx->cb_stop = false;
    ctx->cb_pending.clear();
}

}  // namespace

namespace kgpu {
namespace hostutil {

int serve_quiesce(kgpu_ctx* ctx, int64_t timeout_ns) {
    std::unique_lock<std::mutex> lk(ctx->serve_mu);
    ServeState& st = ctx->serve;
    if (!st.started) return KGPU_OK;
    const uint64_t upto = st.next_seq, t0 = now_ns();
    for (;;) {
        reap(st);
        bool pending = false;
        for (uint64_t seq : st.outstanding) pending |= seq < upto;
        if (!pending) return KGPU_OK;
        if (timeout_ns >= 0 && now_ns() - t0 >= (uint64_t)timeout_ns) return KGPU_ETIMEDOUT;
        if (ensure_running(ctx, st)) return KGPU_EIO;
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
        if (!st.started) return KGPU_OK;
    }
}

int destroy_serve(kgpu_ctx* ctx) {
    std::unique_lock<std::mutex> lk(ctx->serve_mu);
    if (on_callback_thread(ctx)) return KGPU_EINVAL;
    ServeState& st = ctx->serve;
    if (!st.started) return KGPU_OK;
    st.closing = st.stopping = true;  // callbacks still to run see the ring going away
    store_release(&st.hdr->stop, 1u);
    if (st.stream) {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(st.stream);
    }
    stop_callbacks(ctx, lk);
    serve_free(st);
    return KGPU_OK;
}

}  // namespace hostutil
}  // namespace kgpu

extern "C" {

int kgpu_serve_start(kgpu_ctx* ctx, const kgpu_serve_config* cfg) {
    if (!ctx) return KGPU_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    if (ctx->serve.started) return KGPU_EBUSY;
    DeviceGuard g(ctx->device);
    int rc = serve_alloc(ctx, ctx->serve, cfg);
    if (rc) return rc;
    rc = ensure_running(ctx, ctx->serve);
    if (rc) serve_free(ctx->serve);
    return rc;
}

int kgpu_serve_submit(kgpu_ctx* ctx, const kgpu_request* req, kgpu_ticket* ticket) {
    if (!ctx || !req || !ticket) return KGPU_EINVAL;
    if (req->len == 0) return KGPU_EINVAL;
    ReqDesc d;
    RangeCache rc;
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    ServeState& st = ctx->serve;
    if (!st.started || st.closing) return KGPU_EINVAL;
    int r = make_desc(ctx, *req, rc, st.tile_chunks, &d);
    if (r) return r;
    uint64_t seq = 0;
    r = publish(ctx, st, d, &seq);
    if (r == KGPU_OK || r == KGPU_EIO) *ticket = seq + 1;
    return r;
}

int kgpu_serve_submit_cb(kgpu_ctx* ctx, const kgpu_request* req, kgpu_done_fn fn, void* arg, kgpu_ticket* ticket) {
    if (!ctx || !req || !fn || !ticket) return KGPU_EINVAL;
    if (req->len == 0) return KGPU_EINVAL;
    ReqDesc d;
    RangeCache rc;
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    ServeState& st = ctx->serve;
    if (!st.started || st.closing) return KGPU_EINVAL;
    int r = make_desc(ctx, *req, rc, st.tile_chunks, &d);
    if (r) return r;
    if (!ctx->cb_thread.joinable()) {
        try {
            ctx->cb_thread = std::thread(callback_loop, ctx);
        } catch (...) {
            return KGPU_ENOMEM;
        }
    }
    uint64_t seq = 0;
    r = publish(ctx, st, d, &seq);
    if (r != KGPU_OK && r != KGPU_EIO) return r;
    *ticket = seq + 1;
    {
        std::lock_guard<std::mutex> g(ctx->cb_mu);
        ctx->cb_pending.push_back(ServeCallback{seq, fn, arg});
    }
    ctx->cb_cv.notify_one();
    return r;
}

int kgpu_serve_submit_many(kgpu_ctx* ctx, const kgpu_request* reqs, size_t n, kgpu_ticket* tickets,
                           size_t* accepted) {
    if (!ctx || !accepted || (n && (!reqs || !tickets))) return KGPU_EINVAL;
    *accepted = 0;
    if (n == 0) return KGPU_OK;
    std::vector<ReqDesc> descs(n);
    RangeCache rc;
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    ServeState& st = ctx->serve;
    if (!st.started || st.closing) return KGPU_EINVAL;
    for (size_t i = 0; i < n; i++) {  // all or nothing on validation
        if (reqs[i].len == 0) return KGPU_EINVAL;
        int r = make_desc(ctx, reqs[i], rc, st.tile_chunks, &descs[i]);
        if (r) return r;
    }
    size_t k = 0;
    int r = KGPU_OK;
    for (; k < n; k++) {
        uint64_t seq = 0;
        if ((r = stage(st, descs[k], &seq))) break;
        tickets[k] = seq + 1;
    }
    *accepted = k;
    if (k) {
        const int c = commit(ctx, st);
        if (c) return c;
    }
    return r;
}

int kgpu_serve_poll(kgpu_ctx* ctx, kgpu_ticket ticket, int64_t timeout_ns, int* status, uint64_t* stamps) {
    if (!ctx) return KGPU_EINVAL;
    ServeState& st = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        if (!st.started || st.stopping || ticket == 0 || ticket > st.next_seq) return KGPU_ENOENT;
        st.readers++;
    }
    ReaderGuard reader(ctx);
    const uint64_t seq = ticket - 1;
    const uint32_t s = (uint32_t)(seq & (st.nslots - 1));
    const uint64_t t0 = now_ns();
    uint64_t last_check = t0;
    for (;;) {
        const unsigned long long d = load_acquire(&st.done_seq[s]);
        if (d >= seq + 1) {
            int code = 0;
            uint64_t v[ServeState::kStamps] = {};
            if (!read_completed(st, seq, &code, v)) {
                // its slot has retired a later request too: stamps are gone,
                // a failure code is kept by ticket
                std::lock_guard<std::mutex> lk(ctx->serve_mu);
                auto f = st.failed.find(seq);
                code = f != st.failed.end() ? f->second : 0;
                for (auto& x : v) x = 0;
            }
            if (status) *status = code;
            if (stamps) {
                stamps[0] = v[2];
                stamps[1] = v[3];
            }
            return KGPU_OK;
        }
        const uint64_t t = now_ns();
        if (timeout_ns == 0 || t - last_check > 50000) {
            std::lock_guard<std::mutex> lk(ctx->serve_mu);
            if (!st.started || st.stopping) return KGPU_ENOENT;
            reap(st);
            if (!st.outstanding.empty()) {
                int rc = ensure_running(ctx, st);
                if (rc) return rc;
            }
            last_check = t;
        }
        if (timeout_ns == 0 || (timeout_ns > 0 && t - t0 >= (uint64_t)timeout_ns)) return KGPU_ETIMEDOUT;
        cpu_relax();
    }
}

int kgpu_serve_stop(kgpu_ctx* ctx, int64_t drain_timeout_ns) {
    if (!ctx) return KGPU_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->serve_mu);
    if (on_callback_thread(ctx)) return KGPU_EINVAL;  // it would wait for itself
    ServeState& st = ctx->serve;
    if (!st.started) return KGPU_OK;
    if (st.closing) {  // another thread is stopping this ring: wait until it is gone
        while (st.started && st.closing) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
        return KGPU_OK;
    }
    st.closing = true;
    const uint64_t t0 = now_ns();
    int rc = KGPU_OK;
    for (;;) {
        reap(st);
        if (st.outstanding.empty()) break;
        if (drain_timeout_ns >= 0 && now_ns() - t0 >= (uint64_t)drain_timeout_ns) {
            rc = KGPU_ETIMEDOUT;
            break;
        }
        if (ensure_running(ctx, st)) {
            rc = KGPU_EIO;
            break;
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
    }
    store_release(&st.hdr->stop, 1u);
    DeviceGuard g(ctx->device);
    if (cudaEventSynchronize(st.kdone) != cudaSuccess) {
        cudaGetLastError();
        if (!rc) rc = KGPU_EIO;
    }
    // calls still reading the ring see `stopping` within 50 us and leave
    st.stopping = true;
    while (st.readers > 0) {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
    }
    stop_callbacks(ctx, lk);  // the kernel has stopped: what is left runs now
    serve_free(st);
    return rc;
}

int kgpu_serve_get_stats(kgpu_ctx* ctx, kgpu_serve_stats* out) {
    if (!ctx || !out) return KGPU_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    ServeState& st = ctx->serve;
    std::memset(out, 0, sizeof(*out));
    if (!st.started) return KGPU_OK;
    reap(st);
    if (st.running && cudaEventQuery(st.kdone) == cudaSuccess) {
        st.running = false;
        st.last_exit = (unsigned)load_acquire(&st.hdr->exit_code);
    }
    cudaGetLastError();
    out->submitted = st.submitted;
    out->completed = st.completed;
    out->busy_refusals = st.busy_refusals;
    out->launches = st.launches;
    out->inflight_bytes = st.inflight_bytes;
    out->running = st.running ? 1u : 0u;
    out->last_exit = st.last_exit;
    return KGPU_OK;
}

// Host monotonic time minus the device's %globaltimer, estimated from the
// dispatcher's heartbeat word (the timer's value, written every 16th idle
// poll): a load that sees a new value v ended at host time t >= the store's
// visibility >= v + offset, so t - v bounds the offset from above, and the
// smallest such bound over about 2 ms of samples is the estimate.  That is
// the true offset plus the shortest device-to-host store latency, so device
// times converted with it come out late by that latency (under a
// microsecond over NVLink-C2C).  (The host time must be taken after the
// load: one taken before it is no bound if the thread stalls in between.)
// Needs a running, idle serving kernel; 0 if the word did not move.  *at:
// the host time the estimate stands for (the middle of the samples).
static int64_t heartbeat_offset(const ServeState& st, uint64_t* at) {
    const unsigned long long* hb = &st.hdr->heartbeat;
    unsigned long long last = load_acquire(hb);
    int64_t best = INT64_MAX;
    const uint64_t begin = now_ns(), end = begin + 2000000;
    for (uint64_t t = begin; t < end;) {
        const unsigned long long v = load_acquire(hb);
        t = now_ns();
        if (v != last) {
            last = v;
            best = std::min<int64_t>(best, (int64_t)t - (int64_t)v);
        }
    }
    *at = begin + 1000000;
    return best == INT64_MAX ? 0 : best;
}

static int replay_serve_impl(kgpu_ctx* ctx, const kgpu_request* reqs, const uint64_t* arrival_ns, size_t n,
                             int64_t timeout_ns, uint64_t* latency_ns, uint64_t* wall_ns, uint64_t* detail,
                             int64_t* stages, int64_t* offset_out) {
    if (!ctx || !reqs || !arrival_ns || !latency_ns || !n) return KGPU_EINVAL;
    std::vector<ReqDesc> descs(n);
    uint32_t tile_chunks;
    uint32_t nslots;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        if (!ctx->serve.started || ctx->serve.stopping) return KGPU_EINVAL;
        tile_chunks = ctx->serve.tile_chunks;
        nslots = ctx->serve.nslots;
        ctx->serve.readers++;
    }
    ReaderGuard reader(ctx);
    {
        RangeCache rc;
        for (size_t i = 0; i < n; i++) {
            if (reqs[i].len == 0) return KGPU_EINVAL;
            int r = make_desc(ctx, reqs[i], rc, tile_chunks, &descs[i]);
            if (r) return r;
            if (i && arrival_ns[i] < arrival_ns[i - 1]) return KGPU_EINVAL;
        }
    }
    ServeState& st = ctx->serve;
    // the offset is estimated before and after the run and interpolated per
    // request, in case the two clocks run at slightly different rates
    int64_t off0 = 0;
    uint64_t at0 = 0;
    if (stages) {
        {
            std::lock_guard<std::mutex> lk(ctx->serve_mu);
            if (st.stopping || ensure_running(ctx, st)) return KGPU_EIO;
        }
        off0 = heartbeat_offset(st, &at0);
    }
    std::unique_ptr<std::atomic<uint64_t>[]> seq_of(new std::atomic<uint64_t>[n]);
    for (size_t i = 0; i < n; i++) {
        seq_of[i].store(UINT64_MAX, std::memory_order_relaxed);
        latency_ns[i] = UINT64_MAX;
    }
    std::atomic<size_t> produced{0};
    std::atomic<bool> abort{false};
    std::atomic<int> error{0};
    const uint64_t t0 = now_ns();
    const uint64_t deadline = timeout_ns > 0 ? t0 + (uint64_t)timeout_ns : UINT64_MAX;
    uint64_t last_done = t0;

    std::thread consumer([&]() {
        std::vector<size_t> pending;
        size_t seen = 0, done = 0;
        uint64_t last_check = now_ns();
        while (done < n) {
            const size_t p = produced.load(std::memory_order_acquire);
            while (seen < p) pending.push_back(seen++);
            size_t w = 0;
            const uint64_t t = now_ns();
            for (size_t k = 0; k < pending.size(); k++) {
                const size_t i = pending[k];
                const uint64_t seq = seq_of[i].load(std::memory_order_acquire);
                const uint32_t slot = (uint32_t)(seq & (nslots - 1));
                if (load_acquire(&st.done_seq[slot]) >= seq + 1) {
                    // the time after the completion was seen: one taken at the
                    // start of the scan would read early if the thread
                    // stalled during it
                    const uint64_t tc = now_ns();
                    latency_ns[i] = tc - (t0 + arrival_ns[i]);
                    if (detail || stages) {  // 0s once the slot has retired a later request too
                        int code = 0;
                        uint64_t v[ServeState::kStamps] = {};
                        if (!read_completed(st, seq, &code, v))
                            for (auto& x : v) x = 0;
                        if (detail) {
                            detail[3 * i + 1] = v[2];
                            detail[3 * i + 2] = v[3];
                        }
                        if (stages) {  // raw device stamps for now, converted after the run
                            for (int k = 0; k < ServeState::kStamps; k++) stages[kStageWords * i + 1 + k] = (int64_t)v[k];
                            stages[kStageWords * i + 5] = (int64_t)(tc - (t0 + arrival_ns[i]));
                        }
                    }
                    last_done = std::max(last_done, tc);
                    done++;
                } else {
                    pending[w++] = i;
                }
            }
            pending.resize(w);
            if (t - last_check > 100000) {  // relaunch the kernel if it exited with work pending
                // While the producer still publishes it checks the kernel itself,
                // and holds the mutex most of the time when the ring is full: do
                // not queue behind it, or completions go unseen meanwhile.
                std::unique_lock<std::mutex> lk(ctx->serve_mu, std::defer_lock);
                if (produced.load(std::memory_order_acquire) < n ? lk.try_lock() : (lk.lock(), true)) {
                    if (st.stopping) error.store(KGPU_ENOENT);
                    else if (!pending.empty() && ensure_running(ctx, st)) error.store(KGPU_EIO);
                    last_check = t;
                }
            }
            if (abort.load() || error.load() || t > deadline) break;
        }
    });

    // Producer: at each step, every request whose arrival time has passed is
    // staged and the burst is committed with one head update, as a caller
    // with several pages ready at once would do through kgpu_serve_submit_many.
    int rc = KGPU_OK;
    for (size_t i = 0; i < n && !rc;) {
        wait_until(t0 + arrival_ns[i]);
        size_t j = i;
        int r = KGPU_OK;
        {
            std::lock_guard<std::mutex> lk(ctx->serve_mu);
            const uint64_t t = now_ns();
            for (; j < n && j - i < 256 && t0 + arrival_ns[j] <= t; j++) {
                uint64_t seq = 0;
                r = stage(st, descs[j], &seq);
                if (r) break;
                if (detail) detail[3 * j] = t - (t0 + arrival_ns[j]);
                seq_of[j].store(seq, std::memory_order_release);
            }
            if (j > i) {
                const int c = commit(ctx, st);
                if (c) r = c;
                if (stages) {
                    const uint64_t tc = st.last_publish_ns;
                    for (size_t q = i; q < j; q++) stages[kStageWords * q] = (int64_t)(tc - (t0 + arrival_ns[q]));
                }
            }
        }
        if (j > i) produced.store(j, std::memory_order_release);
        if (r && r != KGPU_EBUSY) {
            rc = r;
        } else if (j == i) {  // refused: the ring or the byte cap is full
            if (now_ns() > deadline) rc = KGPU_ETIMEDOUT;
            else cpu_relax();
        }
        i = j;
        if (error.load()) rc = error.load();
    }
    if (rc) abort.store(true);
    consumer.join();
    if (!rc && error.load()) rc = error.load();
    if (!rc) {
        for (size_t i = 0; i < n; i++)
            if (latency_ns[i] == UINT64_MAX) rc = KGPU_ETIMEDOUT;
    }
    if (wall_ns) *wall_ns = last_done - t0;
    if (stages) {
        // device stamps to nanoseconds since each request's arrival, on the
        // host clock; a lost stamp (0) becomes INT64_MIN
        uint64_t at1 = 0;
        const int64_t off1 = rc ? off0 : heartbeat_offset(st, &at1);
        if (offset_out) {
            offset_out[0] = off0;
            offset_out[1] = off1;
        }
        const double slope = at1 > at0 ? (double)(off1 - off0) / (double)(at1 - at0) : 0.0;
        for (size_t i = 0; i < n; i++) {
            const int64_t arr = (int64_t)(t0 + arrival_ns[i]);
            const int64_t off = off0 + (int64_t)(slope * (double)(arr - (int64_t)at0));
            for (int k = 1; k <= ServeState::kStamps; k++) {
                int64_t& x = stages[kStageWords * i + k];
                x = x ? x + off - arr : INT64_MIN;
            }
        }
    }
    std::lock_guard<std::mutex> lk(ctx->serve_mu);
    reap(st);
    return rc;
}

int kgpu_replay_serve(kgpu_ctx* ctx, const kgpu_request* reqs, const uint64_t* arrival_ns, size_t n,
                      int64_t timeout_ns, uint64_t* latency_ns, uint64_t* wall_ns, uint64_t* detail) {
    return replay_serve_impl(ctx, reqs, arrival_ns, n, timeout_ns, latency_ns, wall_ns, detail, nullptr, nullptr);
}

int kgpu_replay_serve_stages(kgpu_ctx* ctx, const kgpu_request* reqs, const uint64_t* arrival_ns, size_t n,
                             int64_t timeout_ns, uint64_t* latency_ns, uint64_t* wall_ns, int64_t* stages,
                             int64_t* clock_offset_ns) {
    if (!stages) return KGPU_EINVAL;
    for (size_t i = 0; i < kStageWords * n; i++) stages[i] = 0;
    return replay_serve_impl(ctx, reqs, arrival_ns, n, timeout_ns, latency_ns, wall_ns, nullptr, stages,
                             clock_offset_ns);
}

int kgpu_replay_launches(kgpu_ctx* ctx, const kgpu_request* reqs, const uint64_t* arrival_ns, size_t n,
                         uint32_t nstreams, int64_t timeout_ns, uint64_t* latency_ns, uint64_t* wall_ns) {
    if (!ctx || !reqs || !arrival_ns || !latency_ns || !n || nstreams == 0 || nstreams > 256) return KGPU_EINVAL;
    {
        std::lock_guard<std::mutex> lk(ctx->serve_mu);
        if (ctx->serve.started) return KGPU_EBUSY;  // the serving kernel holds every SM
    }
    std::vector<ReqDesc> descs(n);
    std::vector<HostKey> keys;
    {
        RangeCache rc;
        for (size_t i = 0; i < n; i++) {
            if (reqs[i].len == 0) return KGPU_EINVAL;
            int r = make_desc(ctx, reqs[i], rc, 32, &descs[i]);
            if (r) return r;
            if (i && arrival_ns[i] < arrival_ns[i - 1]) return KGPU_EINVAL;
        }
        std::lock_guard<std::mutex> lk(ctx->mu);
        keys = ctx->keys;
    }
    DeviceGuard g(ctx->device);
    std::vector<cudaStream_t> streams(nstreams, nullptr);
    const size_t P = std::min<size_t>(n, 8192);
    std::vector<cudaEvent_t> events(P, nullptr);
    int rc = KGPU_OK;
    for (auto& s : streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = KGPU_EIO;
    for (auto& e : events)
        if (!rc && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = KGPU_EIO;
    for (size_t i = 0; i < n; i++) latency_ns[i] = UINT64_MAX;
    std::unique_ptr<std::atomic<uint8_t>[]> fin(new std::atomic<uint8_t>[n]);
    for (size_t i = 0; i < n; i++) fin[i].store(0);
    std::atomic<size_t> issued{0};
    std::atomic<bool> abort{false};
    const uint64_t t0 = now_ns();
    const uint64_t deadline = timeout_ns > 0 ? t0 + (uint64_t)timeout_ns : UINT64_MAX;
    uint64_t last_done = t0;

    std::thread consumer([&]() {
        std::vector<size_t> next(nstreams);
        for (uint32_t k = 0; k < nstreams; k++) next[k] = k;
        size_t done = 0;
        while (done < n && !abort.load()) {
            const size_t iss = issued.load(std::memory_order_acquire);
            for (uint32_t k = 0; k < nstreams; k++) {
                while (next[k] < iss) {
                    cudaError_t e = cudaEventQuery(events[next[k] % P]);
                    if (e == cudaErrorNotReady) break;
                    const uint64_t t = now_ns();
                    latency_ns[next[k]] = t - (t0 + arrival_ns[next[k]]);
                    last_done = t;
                    fin[next[k]].store(1, std::memory_order_release);
                    next[k] += nstreams;
                    done++;
                }
            }
            if (now_ns() > deadline) break;
        }
    });

    for (size_t i = 0; i < n && !rc; i++) {
        wait_until(t0 + arrival_ns[i]);
        if (i >= P) {  // the event slot is free once request i - P is seen complete
            while (!fin[i - P].load(std::memory_order_acquire)) {
                if (now_ns() > deadline) {
                    rc = KGPU_ETIMEDOUT;
                    break;
                }
                cpu_relax();
            }
            if (rc) break;
        }
        const ReqDesc& d = descs[i];
        cudaStream_t s = streams[i % nstreams];
        cudaError_t e;
        if (d.mode == KGPU_MODE_COPY) {
            e = launch_copy(d.src, d.dst, d.nblocks, d.unit_blocks, ctx->num_sms, s);
        } else if (d.mode == KGPU_MODE_XTS || d.mode == KGPU_MODE_ECB) {
            const HostKey& k = keys[d.key];
            BulkParams p;
            fill_bulk(&p, k, (int)d.dir, d.src, d.dst, d.nblocks * 16, (size_t)d.unit_blocks * 16, d.first_sector);
            e = d.mode == KGPU_MODE_XTS ? launch_xts(p, k.nr, (int)d.dir, ctx->num_sms, s)
                                        : launch_ecb(p, k.nr, (int)d.dir, ctx->num_sms, s);
        } else {
            const HostKey& k = keys[d.key];
            CbcParams p;
            std::memset(&p, 0, sizeof(p));
            p.src = d.src;
            p.dst = d.dst;
            p.ivs = d.ivs;
            p.npages = d.nblocks / d.unit_blocks;
            p.bpp = d.unit_blocks;
            const bool enc = d.mode == KGPU_MODE_CBC_ENC;
            std::memcpy(p.rk, enc ? k.enc : k.dec, sizeof(p.rk));
            e = enc ? launch_cbc_enc(p, k.nr, ctx->num_sms, s) : launch_cbc_dec(p, k.nr, ctx->num_sms, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(events[i % P], s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = KGPU_EIO;
            break;
        }
        issued.store(i + 1, std::memory_order_release);
    }
    if (rc) abort.store(true);
    consumer.join();
    for (auto& s : streams)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    for (auto& e : events)
        if (e) cudaEventDestroy(e);
    if (!rc) {
        for (size_t i = 0; i < n; i++)
            if (latency_ns[i] == UINT64_MAX) rc = KGPU_ETIMEDOUT;
    }
    if (wall_ns) *wall_ns = last_done - t0;
    return rc;
}

}  // extern "C"
