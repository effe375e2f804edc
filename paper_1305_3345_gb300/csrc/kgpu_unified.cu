// Unified persistent kernels: one CTA serves any mode (XTS, ECB, CBC decrypt,
// CBC encrypt), either direction and any key size, so that thousands of uneven
// requests with mixed keys and modes run in one launch (the batched form of
// the paper's many-small-requests workload, section 3.1) and in the serving
// loop.
//
// Work is cut into tiles (a run of 32-block chunks of one XTS/ECB request, a
// run of whole pages of one CBC-decrypt request, or up to 32 pages of one
// CBC-encrypt request -- one chain per lane).  Warps pull tile indices from a
// global counter, map them to their request by binary search over the tile
// prefix, load that request's key schedule into registers when it changes,
// and run the tile.
#include <cuda_runtime.h>

#include "aes_device.cuh"
#include "kgpu_internal.h"

namespace kgpu {

using namespace dev;

static_assert(kSmemBase == (uint32_t)kSmemReservedBytes, "table offsets assume the reserved shared area");

__device__ uint32_t g_u_te0[256];
__device__ uint32_t g_u_td0[256];
__device__ uint32_t g_u_sb4[256];
__device__ uint32_t g_u_isb4[256];

namespace {

// Regions A = Te0|Te1, B = Td0|Td1, C = S4|IS4, each row replicated per lane.
__device__ __forceinline__ void fill_unified(char* smem) {
    uint32_t* w = reinterpret_cast<uint32_t*>(smem);
    for (uint32_t i = threadIdx.x; i < 3 * 16384; i += blockDim.x) {
        uint32_t region = i >> 14, x = (i >> 6) & 255u, half = (i >> 5) & 1u;
        uint32_t v;
        if (region == 0) v = g_u_te0[x];
        else if (region == 1) v = g_u_td0[x];
        else v = half ? g_u_isb4[x] : g_u_sb4[x];
        if (region < 2 && half) v = rotl8(v);
        w[i] = v;
    }
}

__device__ __forceinline__ void xor4(uint4& v, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    v.x ^= a;
    v.y ^= b;
    v.z ^= c;
    v.w ^= d;
}

struct WarpKeys {
    RegKey data;          // schedule of the data cipher (encu or decu)
    const uint32_t* twk;  // this warp's shared slot holding the tweak schedule
    int nr;
};

// XTS (TWEAK) or ECB over the 32-block chunks [c0, c1) of one request.
template <bool TWEAK>
__device__ __forceinline__ void tile_blocks(const ReqDesc& d, uint64_t c0, uint64_t c1, int dir,
                                            const WarpKeys& K) {
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, dir);
    const UniLanes LE = uni_lanes(lane, 0);
    const SmemKey TK{K.twk};
    uint64_t blk = (c0 << 5) + lane;
    const uint32_t bps = d.unit_blocks;
    uint64_t base = 0;
    uint32_t srel = 0, j = 0;
    uint32_t z0 = 0, z1 = 0, z2 = 0, z3 = 0, t0 = 0, t1 = 0, t2 = 0, t3 = 0;

    auto tweak_batch = [&]() {
        uint64_t unit = d.first_sector + base + lane;
        z0 = (uint32_t)unit;
        z1 = (uint32_t)(unit >> 32);
        z2 = 0;
        z3 = 0;
        cipher_u(z0, z1, z2, z3, TK, K.nr, LE);
    };
    if (TWEAK) {
        base = (c0 << 5) / bps;
        uint64_t sabs = blk / bps;
        srel = (uint32_t)(sabs - base);
        j = (uint32_t)(blk - sabs * bps);
        tweak_batch();
        t0 = __shfl_sync(0xffffffffu, z0, srel);
        t1 = __shfl_sync(0xffffffffu, z1, srel);
        t2 = __shfl_sync(0xffffffffu, z2, srel);
        t3 = __shfl_sync(0xffffffffu, z3, srel);
        gf128_mul_xpow(t0, t1, t2, t3, j);
    }
    for (uint64_t c = c0; c < c1; ++c) {
        const bool valid = blk < d.nblocks;
        uint4 v = valid ? d.src[blk] : make_uint4(0, 0, 0, 0);
        if (TWEAK) xor4(v, t0, t1, t2, t3);
        cipher_block(v, K.data, K.nr, L, dir);
        if (TWEAK) xor4(v, t0, t1, t2, t3);
        if (valid) d.dst[blk] = v;
        blk += 32;
        if (TWEAK && c + 1 < c1) {
            j += 32;
            bool crossed = false;
            if (j >= bps) {
                uint32_t ns = j / bps;
                srel += ns;
                j -= ns * bps;
                crossed = true;
            }
            if (__any_sync(0xffffffffu, srel >= 32)) {
                uint32_t adv = __shfl_sync(0xffffffffu, srel, 0);
                base += adv;
                srel -= adv;
                tweak_batch();
            }
            if (__any_sync(0xffffffffu, crossed)) {
                uint32_t u0 = __shfl_sync(0xffffffffu, z0, srel & 31);
                uint32_t u1 = __shfl_sync(0xffffffffu, z1, srel & 31);
                uint32_t u2 = __shfl_sync(0xffffffffu, z2, srel & 31);
                uint32_t u3 = __shfl_sync(0xffffffffu, z3, srel & 31);
                if (crossed) {
                    t0 = u0;
                    t1 = u1;
                    t2 = u2;
                    t3 = u3;
                    gf128_mul_xk(t0, t1, t2, t3, j);
                }
            }
            if (!crossed) gf128_mul_x32(t0, t1, t2, t3);
        }
    }
}

// CBC decryption of pages [p0, p1) of one request (see cbc_dec_kernel).
__device__ __forceinline__ void tile_cbc_dec(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 1);
    const uint32_t bpp = d.unit_blocks;
    const uint64_t bend = p1 * bpp;
    uint64_t blk = p0 * bpp + lane;
    uint64_t page = p0 + lane / bpp;
    uint32_t j = lane % bpp;
    uint32_t carry0 = 0, carry1 = 0, carry2 = 0, carry3 = 0;
    for (uint64_t b = p0 * bpp; b < bend; b += 32) {
        const bool valid = blk < bend;
        const uint4 c = valid ? d.src[blk] : make_uint4(0, 0, 0, 0);
        // lane i takes lane i-1's block; lane 0 keeps lane 31's of the last step
        const uint32_t src_lane = (lane + 31) & 31;
        uint4 prev;
        prev.x = __shfl_sync(0xffffffffu, c.x, src_lane);
        prev.y = __shfl_sync(0xffffffffu, c.y, src_lane);
        prev.z = __shfl_sync(0xffffffffu, c.z, src_lane);
        prev.w = __shfl_sync(0xffffffffu, c.w, src_lane);
        if (lane == 0) {
            uint4 cur = prev;
            prev = make_uint4(carry0, carry1, carry2, carry3);
            carry0 = cur.x;
            carry1 = cur.y;
            carry2 = cur.z;
            carry3 = cur.w;
        }
        if (valid && j == 0) prev = d.ivs[page];
        uint4 v = c;
        cipher_block(v, K.data, K.nr, L, 1);
        xor4(v, prev.x, prev.y, prev.z, prev.w);
        if (valid) d.dst[blk] = v;
        blk += 32;
        j += 32;
        if (j >= bpp) {
            uint32_t ns = j / bpp;
            page += ns;
            j -= ns * bpp;
        }
    }
}

// CBC encryption of pages [p0, p1), p1 - p0 <= 32: one chain per lane.
__device__ __forceinline__ void tile_cbc_enc(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 0);
    const uint64_t page = p0 + lane;
    if (page >= p1) return;
    const uint32_t bpp = d.unit_blocks;
    const uint4* in = d.src + page * bpp;
    uint4* out = d.dst + page * bpp;
    uint4 x = d.ivs[page];
    uint4 nxt = in[0];
    for (uint32_t i = 0; i < bpp; ++i) {
        const uint4 cur = nxt;
        if (i + 1 < bpp) nxt = in[i + 1];
        xor4(x, cur.x, cur.y, cur.z, cur.w);
        cipher_block(x, K.data, K.nr, L, 0);
        out[i] = x;
    }
}

// Tile t of the batch -> (request, first unit, end unit).
__device__ __forceinline__ uint32_t find_request(const uint64_t* tile_start, uint32_t nreq, uint64_t t) {
    uint32_t lo = 0, hi = nreq;  // tile_start[lo] <= t < tile_start[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (tile_start[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Runs one tile of request d; returns 0 or a KGPU_E* status for the request.
__device__ __forceinline__ int run_tile(const ReqDesc& d, uint64_t tile_in_req, const DevKey* keys, uint32_t max_keys,
                                     WarpKeys& K, uint32_t& cur_sel) {
    const uint32_t lane = lane_id();
    if (d.key >= max_keys) return KGPU_ENOENT;
    const DevKey& dk = keys[d.key];
    const bool is_xts = d.mode == KGPU_MODE_XTS;
    const uint32_t flags = dk.flags;
    if (!(flags & kKeyLive) || ((flags & kKeyXts) != 0) != is_xts) return KGPU_ENOENT;
    const int dir = (d.mode == KGPU_MODE_CBC_DEC) ? 1 : (d.mode == KGPU_MODE_CBC_ENC) ? 0 : (int)d.dir;
    const uint32_t sel = d.key * 2u + (uint32_t)dir;
    if (sel != cur_sel) {
        K.data.load(dir ? dk.decu : dk.encu);
        K.nr = (int)dk.nr;
        if (is_xts) {
            uint32_t* slot = const_cast<uint32_t*>(K.twk);
            slot[lane] = dk.twku[lane];
            slot[lane + 32] = lane + 32 < 60 ? dk.twku[lane + 32] : 0u;
            __syncwarp();
        }
        cur_sel = sel;
    }
    const uint64_t units = request_units(d);
    const uint64_t u0 = tile_in_req * d.tile_units;
    uint64_t u1 = u0 + d.tile_units;
    if (u1 > units) u1 = units;
    switch (d.mode) {
        case KGPU_MODE_XTS: tile_blocks<true>(d, u0, u1, dir, K); break;
        case KGPU_MODE_ECB: tile_blocks<false>(d, u0, u1, dir, K); break;
        case KGPU_MODE_CBC_DEC: tile_cbc_dec(d, u0, u1, K); break;
        case KGPU_MODE_CBC_ENC: tile_cbc_enc(d, u0, u1, K); break;
        default: return KGPU_EINVAL;
    }
    return 0;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) batch_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    fill_unified(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    WarpKeys K;
    K.twk = reinterpret_cast<const uint32_t*>(smem + 3 * kRegion + warp * 256);
    K.nr = 0;
    uint32_t cur_sel = 0xffffffffu;

    const BatchHeader* hdr = reinterpret_cast<const BatchHeader*>(a.buf);
    const uint64_t total = hdr->total_tiles;
    const uint32_t nreq = hdr->nreq;
    const ReqDesc* reqs = reinterpret_cast<const ReqDesc*>(a.buf + batch_desc_offset());
    const uint64_t* tile_start = reinterpret_cast<const uint64_t*>(a.buf + batch_prefix_offset(nreq));
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(a.next_tile, 1ull);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < total) {
        const uint64_t t = next;
        if (lane == 0) next = atomicAdd(a.next_tile, 1ull);  // fetched while this tile runs
        const uint32_t i = find_request(tile_start, nreq, t);
        const ReqDesc d = reqs[i];
        const int st = run_tile(d, t - tile_start[i], a.keys, a.max_keys, K, cur_sel);
        if (st && lane == 0) a.status[i] = st;
        next = __shfl_sync(0xffffffffu, next, 0);
    }
}


// ---------------------------------------------------------------------------
// Serving kernel: the paper's Non-Stop Kernel (section 3.1) -- launched once,
// fed through pinned host memory -- with every wait bounded.
//
// CTA 0 / warp 0 is the dispatcher: it polls the host-written request count
// with system-scope acquire loads and mirrors it into device memory, so the
// thousands of worker warps poll L2 instead of the host link.  Workers walk
// the published requests in order; a request's tiles are claimed one at a time
// with compare-and-swap on a per-slot word tagged with the request number (so
// a warp that is late never touches the slot's next occupant), and the warp
// that finishes the last tile publishes the completion to the host.  Requests
// that arrive while others run are picked up as warps move past the ones that
// are fully claimed: continuous batching at tile granularity.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_vol(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ unsigned int ld_vol32(const unsigned int* p) {
    return *reinterpret_cast<const volatile unsigned int*>(p);
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr long long kNoTile = -1, kRetry = -2;

// Claim the next tile of request r (nt tiles) from its slot word.
__device__ long long claim_tile(unsigned long long* w, unsigned long long r, unsigned long long nt) {
    const unsigned long long mask = (1ull << kServeTagShift) - 1;
    unsigned long long old = ld_vol(w);
    for (int i = 0; i < 256; i++) {
        const unsigned long long tag = old >> kServeTagShift;
        if (tag > r) return kNoTile;  // r is retired and its slot reused
        unsigned long long want, k;
        if (tag < r) {                // slot still tagged with its previous occupant
            k = 0;
            want = (r << kServeTagShift) | 1ull;
        } else {
            k = old & mask;
            if (k >= nt) return kNoTile;
            want = old + 1;
        }
        const unsigned long long prev = atomicCAS(w, old, want);
        if (prev == old) return (long long)k;
        old = prev;
        __nanosleep(32);
    }
    return kRetry;
}

// Count one finished tile of request r; returns the finished count.
__device__ unsigned long long finish_tile(unsigned long long* w, unsigned long long r) {
    const unsigned long long mask = (1ull << kServeTagShift) - 1;
    unsigned long long old = ld_vol(w);
    for (int i = 0; i < 4096; i++) {
        if ((old >> kServeTagShift) == r) return (atomicAdd(w, 1ull) & mask) + 1;  // tag is stable now
        const unsigned long long prev = atomicCAS(w, old, (r << kServeTagShift) | 1ull);
        if (prev == old) return 1;
        old = prev;
    }
    return 0;  // unreachable in practice: the finish word only moves forward to r
}

__device__ void serve_dispatcher(const ServeArgs& a, unsigned long long t0) {
    if (lane_id() != 0) return;
    unsigned long long last = ld_vol(&a.dev->head);
    unsigned long long idle_since = t0, backoff = 64;
    unsigned int reason = 0;
    for (;;) {
        const unsigned long long now = gtimer();
        const unsigned long long h = ld_acquire_sys(&a.hh->head);
        if (h != last) {
            st_release_gpu(&a.dev->head, h);
            last = h;
            idle_since = now;
            backoff = 64;
        }
        if (ld_vol32(&a.hh->stop)) {
            reason = kServeExitStop;
            break;
        }
        const unsigned long long done = ld_vol(&a.dev->done_count);
        if (done != last) idle_since = now;  // requests outstanding: not idle
        if (now - idle_since > a.idle_ns && ld_acquire_sys(&a.hh->head) == last) {
            reason = kServeExitIdle;
            break;
        }
        if (now - t0 > a.lifetime_ns) {
            reason = kServeExitLifetime;
            break;
        }
        a.hh->heartbeat = now;
        __nanosleep((unsigned)backoff);
        if (backoff < 512) backoff <<= 1;
    }
    atomicExch(&a.dev->stop, reason);
    a.hh->exit_code = reason;
    __threadfence_system();
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) serve_kernel(const __grid_constant__ ServeArgs a) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    fill_unified(smem);
    __syncthreads();

    const unsigned long long t0 = gtimer();
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    if (blockIdx.x == 0 && warp == 0) {
        serve_dispatcher(a, t0);
        return;
    }
    WarpKeys K;
    K.twk = reinterpret_cast<const uint32_t*>(smem + 3 * kRegion + warp * 256);
    K.nr = 0;
    uint32_t cur_sel = 0xffffffffu;
    unsigned long long r = ld_vol(&a.dev->cursor);
    unsigned long long idle0 = 0;
    unsigned int backoff = 32;
    // workers give up on their own, later than the dispatcher's idle limit,
    // should it ever stop answering
    const unsigned long long own_idle = a.idle_ns + 1000000000ull;

    for (;;) {
        unsigned long long h = 0, now = 0;
        unsigned int stop = 0;
        if (lane == 0) {
            h = ld_acquire_gpu(&a.dev->head);
            stop = ld_vol32(&a.dev->stop);
            now = gtimer();
        }
        h = __shfl_sync(0xffffffffu, h, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        now = __shfl_sync(0xffffffffu, now, 0);
        if (stop || now - t0 > a.lifetime_ns) break;  // at a tile boundary: nothing held
        if (r >= h) {
            if (!idle0) idle0 = now;
            else if (now - idle0 > own_idle) break;
            __nanosleep(backoff);
            if (backoff < 1024) backoff <<= 1;
            unsigned long long c = lane == 0 ? ld_vol(&a.dev->cursor) : 0;
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c > r) r = c;
            continue;
        }
        idle0 = 0;
        backoff = 32;
        const uint32_t s = (uint32_t)(r & a.slot_mask);
        long long k = 0;
        unsigned long long nt = 0;
        if (lane == 0) {
            const unsigned long long seq = ld_vol(&a.slots[s].seq);
            nt = ld_vol(&a.slots[s].ntiles);
            k = seq != r ? kNoTile : claim_tile(&a.claim[s], r, nt);
        }
        k = __shfl_sync(0xffffffffu, k, 0);
        nt = __shfl_sync(0xffffffffu, nt, 0);
        if (k == kRetry) {
            __nanosleep(128);
            continue;
        }
        if (k == kNoTile) {
            if (lane == 0) atomicMax(&a.dev->cursor, r + 1);
            r++;
            continue;
        }
        const ReqDesc d = a.slots[s].d;
        if (k == 0 && lane == 0) a.t_start[s] = gtimer();
        const int st = run_tile(d, (uint64_t)k, a.keys, a.max_keys, K, cur_sel);
        if (st && lane == 0) *reinterpret_cast<volatile int*>(&a.status[s]) = st;
        __syncwarp();
        __threadfence();  // this tile's output is visible before it is counted
        if (lane == 0 && finish_tile(&a.fin[s], r) == nt) {
            a.t_done[s] = gtimer();
            __threadfence_system();
            st_release_sys(&a.done_seq[s], r + 1);
            atomicAdd(&a.dev->done_count, 1ull);
        }
    }
}

}  // namespace

cudaError_t upload_unified_tables(const uint32_t* te0, const uint32_t* td0, const uint32_t* sb4,
                                  const uint32_t* isb4) {
    cudaError_t e = cudaMemcpyToSymbol(g_u_te0, te0, 1024);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_u_td0, td0, 1024);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_u_sb4, sb4, 1024);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_u_isb4, isb4, 1024);
    return e;
}

cudaError_t configure_batch_kernels() {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)unified_smem_bytes(512));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unified_smem_bytes(512));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)unified_smem_bytes(256));
    return e;
}

const void* batch_kernel_fn(int threads) {
    if (threads == 512) return reinterpret_cast<const void*>(batch_kernel<512>);
    if (threads == 256) return reinterpret_cast<const void*>(batch_kernel<256>);
    return nullptr;
}

cudaError_t launch_serve(const ServeArgs& a, int threads, int grid, cudaStream_t s) {
    if (threads != 512) return cudaErrorInvalidValue;
    serve_kernel<512><<<grid, 512, unified_smem_bytes(512), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& a, int threads, int grid, cudaStream_t s) {
    if (threads == 512) batch_kernel<512><<<grid, 512, unified_smem_bytes(512), s>>>(a);
    else if (threads == 256) batch_kernel<256><<<grid, 256, unified_smem_bytes(256), s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace kgpu
