// Bulk device-resident kernels: XTS (IEEE 1619), ECB, CBC decrypt (parallel
// over blocks) and CBC encrypt (parallel over pages).
//
// All share one structure: one CTA per SM fills its replicated lookup tables
// into shared memory once (see aes_device.cuh).  For XTS, ECB and CBC
// decryption 1024 threads then walk their own contiguous ranges of the buffer
// 32 blocks (512 B) at a time, one 16-byte block per lane, so each warp-wide
// load and store is a fully coalesced 512-byte transaction; the work is split
// evenly over warps with the warp index interleaved across CTAs, so every SM
// gets the same share.  CBC encryption runs one page's chain per lane, 32
// pages per warp, with the warp count set by the page count, and moves the
// pages through shared memory in whole lines (register-staged, or as tensor
// tiles for large launches).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "aes_device.cuh"
#include "kgpu_bulk.h"

namespace kgpu {

using namespace dev;

static_assert(kSmemBase == (uint32_t)kSmemReservedBytes, "table offsets assume the reserved shared area");

// Cipher constants, uploaded once per device by upload_tables().
__device__ uint32_t g_te0[256];
__device__ uint32_t g_td0[256];
__device__ uint32_t g_isb4[256];

namespace {

// Regions A/B <- T0..T3 built from base[] by byte rotation.
__device__ __forceinline__ void fill_round_tables(uint32_t* w, const uint32_t* base) {
    for (uint32_t i = threadIdx.x; i < 2 * 16384; i += blockDim.x) {
        uint32_t x = (i >> 6) & 255u;
        uint32_t k = ((i >> 14) << 1) | ((i >> 5) & 1u);
        uint32_t v = base[x];
        w[i] = __funnelshift_l(v, v, 8 * k);
    }
}

__device__ __forceinline__ void fill_enc(char* smem) {
    fill_round_tables(reinterpret_cast<uint32_t*>(smem), g_te0);
}

// Regions A/B <- Td0..Td3; region C <- InvS (first half) | Te0 (second half).
__device__ __forceinline__ void fill_dec(char* smem) {
    uint32_t* w = reinterpret_cast<uint32_t*>(smem);
    fill_round_tables(w, g_td0);
    for (uint32_t i = threadIdx.x; i < 16384; i += blockDim.x) {
        uint32_t x = (i >> 6) & 255u;
        w[32768 + i] = (i & 32u) ? g_te0[x] : g_isb4[x];
    }
}

__device__ __forceinline__ void xor4(uint4& v, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    v.x ^= a;
    v.y ^= b;
    v.z ^= c;
    v.w ^= d;
}

// Even split of n items over the warps of the grid: [begin, end) for this warp.
__device__ __forceinline__ void warp_range(uint64_t n, uint64_t& begin, uint64_t& end) {
    const uint64_t W = total_warps(), wg = interleaved_warp();
    begin = n * wg / W;
    end = n * (wg + 1) / W;
}

// ---------------------------------------------------------------------------
// XTS (and ECB when TWEAK is false).
//
// Tweaks: a warp keeps E_K2 of 32 consecutive data units in its lanes (lane i
// holds the unit `base + i`, one AES per lane, computed together).  A lane
// moving to block j of a new unit takes that unit's E_K2 by shuffle and
// multiplies by alpha^j in closed form (j < 32 there); a lane staying in its
// unit steps its tweak by alpha^32.  So the tweak costs one extra AES per
// data unit and a few shifts per block -- never a sequential chain.
// ---------------------------------------------------------------------------
template <int NR, int DIR, bool TWEAK>
__global__ void __launch_bounds__(kBulkThreads, 1) bulk_kernel(const __grid_constant__ BulkParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;  // uniform over the CTA; refused at init
    if (DIR == 0) fill_enc(smem);
    else fill_dec(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const Rep1<2> IS{lane * 4u};
    const Rep1<2> TE{lane * 4u + 128u};
    const ParamKey K{p.rk};
    const ParamKey TK{p.tk};

    uint64_t c0, c1;
    warp_range((p.nblocks + 31) >> 5, c0, c1);
    if (c0 >= c1) return;

    uint64_t blk = (c0 << 5) + lane;
    const uint32_t bps = p.bps;
    uint64_t base = 0;
    uint32_t srel = 0, j = 0;
    uint32_t z0 = 0, z1 = 0, z2 = 0, z3 = 0;  // E_K2(unit base + lane)
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0;  // tweak of this lane's block

    auto tweak_batch = [&]() {
        uint64_t unit = p.first_sector + base + lane;
        z0 = (uint32_t)unit;
        z1 = (uint32_t)(unit >> 32);
        z2 = 0;
        z3 = 0;
        if (DIR == 0) encrypt_block<NR>(z0, z1, z2, z3, T, TK);
        else encrypt_block<NR>(z0, z1, z2, z3, TE, TK);
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

    // the next chunk is fetched while this one is enciphered
    uint4 nxt = blk < p.nblocks ? p.src[blk] : make_uint4(0, 0, 0, 0);
    for (uint64_t c = c0; c < c1; ++c) {
        const bool valid = blk < p.nblocks;
        uint4 v = nxt;
        if (c + 1 < c1 && blk + 32 < p.nblocks) nxt = p.src[blk + 32];
        if (TWEAK) xor4(v, t0, t1, t2, t3);
        if (DIR == 0) encrypt_block<NR>(v.x, v.y, v.z, v.w, T, K);
        else decrypt_block<NR>(v.x, v.y, v.z, v.w, T, IS, K);
        if (TWEAK) xor4(v, t0, t1, t2, t3);
        if (valid) p.dst[blk] = v;
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

// ---------------------------------------------------------------------------
// CBC decryption, one block per lane.  P_i = D(C_i) ^ C_{i-1}: C_{i-1} comes
// from the neighbouring lane by shuffle (lane 0 takes lane 31's block of the
// previous step), and from the page IV at the first block of a page.  Warps
// own whole pages and every block is read and written by the same lane, so
// in-place decryption needs no synchronisation.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(kBulkThreads, 1) cbc_dec_kernel(const __grid_constant__ CbcParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    fill_dec(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const Rep1<2> IS{lane * 4u};
    const ParamKey K{p.rk};

    uint64_t u0, u1;
    warp_range(p.npages, u0, u1);
    if (u0 >= u1) return;

    const uint32_t bpp = p.bpp;
    const uint64_t bend = u1 * bpp;
    uint64_t blk = u0 * bpp + lane;
    uint64_t page = u0 + lane / bpp;
    uint32_t j = lane % bpp;
    uint4 carry = make_uint4(0, 0, 0, 0);
    uint4 nxt = blk < bend ? p.src[blk] : make_uint4(0, 0, 0, 0);

    for (uint64_t b = u0 * bpp; b < bend; b += 32) {
        const bool valid = blk < bend;
        const uint4 c = nxt;
        if (blk + 32 < bend) nxt = p.src[blk + 32];  // prefetch the next step
        // one rotation gives lane i the block of lane i-1; lane 0 receives
        // lane 31's, which it keeps for the next step and replaces by the
        // one it kept from the previous step
        const uint32_t from = (lane + 31) & 31;
        uint4 prev;
        prev.x = __shfl_sync(0xffffffffu, c.x, from);
        prev.y = __shfl_sync(0xffffffffu, c.y, from);
        prev.z = __shfl_sync(0xffffffffu, c.z, from);
        prev.w = __shfl_sync(0xffffffffu, c.w, from);
        if (lane == 0) {
            const uint4 last = prev;
            prev = carry;
            carry = last;
        }
        if (valid && j == 0) prev = p.ivs[page];
        uint4 v = c;
        decrypt_block<NR>(v.x, v.y, v.z, v.w, T, IS, K);
        xor4(v, prev.x, prev.y, prev.z, prev.w);
        if (valid) p.dst[blk] = v;
        blk += 32;
        j += 32;
        if (j >= bpp) {
            uint32_t ns = j / bpp;
            page += ns;
            j -= ns * bpp;
        }
    }
}

// ---------------------------------------------------------------------------
// CBC encryption, one page per lane: C_i = E(P_i ^ C_{i-1}) is a sequential
// chain inside a page, so parallelism comes from pages.  Warps take groups of
// 32 pages; the next plaintext block is fetched while the current one is
// encrypted.
// ---------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(kBulkThreads, 1) cbc_enc_kernel(const __grid_constant__ CbcParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    fill_enc(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const ParamKey K{p.rk};
    const uint32_t bpp = p.bpp;
    const uint64_t ngroups = (p.npages + 31) >> 5;

    for (uint64_t g = interleaved_warp(); g < ngroups; g += total_warps()) {
        // lanes without a page step along with the others, loads and stores
        // predicated off, so the warp stays converged through the chain
        const uint64_t page = (g << 5) + lane;
        const bool valid = page < p.npages;
        const uint4* in = p.src + (valid ? page : 0) * bpp;
        uint4* out = p.dst + (valid ? page : 0) * bpp;
        const uint4 z = make_uint4(0, 0, 0, 0);
        uint4 x = valid ? p.ivs[page] : z;
        // the chain is sequential, so plaintext is fetched four blocks ahead
        uint4 q0 = valid ? in[0] : z;
        uint4 q1 = valid && bpp > 1 ? in[1] : z;
        uint4 q2 = valid && bpp > 2 ? in[2] : z;
        uint4 q3 = valid && bpp > 3 ? in[3] : z;
        for (uint32_t i = 0; i < bpp; ++i) {
            const uint4 cur = q0;
            q0 = q1;
            q1 = q2;
            q2 = q3;
            if (valid && i + 4 < bpp) q3 = in[i + 4];
            xor4(x, cur.x, cur.y, cur.z, cur.w);
            encrypt_block<NR>(x.x, x.y, x.z, x.w, T, K);
            if (valid) out[i] = x;
        }
    }
}


// ---------------------------------------------------------------------------
// CBC encryption, staged.  The chains are the same (one page per lane), but a
// lane's loads and stores at 4-KiB strides would touch 32 cache lines per
// warp instruction; instead each warp moves 8 blocks of each of its 32 pages at
// a time between global memory and a padded shared-memory area with
// coalesced accesses (four 128-B lines per instruction), and the lanes read
// and write their own chains there.  Used when a page is a multiple of 8
// blocks (128 B).  The next 8 blocks are fetched into registers while the
// current ones are enciphered.
// ---------------------------------------------------------------------------
constexpr int kStageBlocks = 8;
constexpr int kStageRow = kStageBlocks * 16 + 16;  // one page's 8 blocks, padded against bank conflicts
constexpr int kStageWarpBytes = 32 * kStageRow;
static_assert(kStageWarpBytes == kStageWarpSmem, "staging area size");

template <int NR>
__global__ void __launch_bounds__(kCbcEncStagedThreads, 1) cbc_enc_staged_kernel(const __grid_constant__ CbcParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    fill_enc(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const ParamKey K{p.rk};
    const uint32_t bpp = p.bpp;
    const uint32_t nchunks = bpp / kStageBlocks;
    char* stage = smem + kSmemEnc + warp * kStageWarpBytes;
    char* own = stage + lane * kStageRow;            // this lane's chain
    const uint32_t cp_page = lane >> 3, cp_blk = lane & 7;  // coalesced copy position
    const uint64_t ngroups = (p.npages + 31) >> 5;

    for (uint64_t g = interleaved_warp(); g < ngroups; g += total_warps()) {
        const uint64_t page = (g << 5) + lane;
        const bool valid = page < p.npages;
        uint4 x = valid ? p.ivs[page] : make_uint4(0, 0, 0, 0);
        uint4 R[4 * 2];
        auto fetch = [&](uint32_t c) {
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint64_t pg = (g << 5) + q * 4 + cp_page;
                R[q] = pg < p.npages ? p.src[pg * bpp + c * kStageBlocks + cp_blk] : make_uint4(0, 0, 0, 0);
            }
        };
        fetch(0);
        for (uint32_t c = 0; c < nchunks; ++c) {
            __syncwarp();  // the previous chunk's ciphertext has been written out
#pragma unroll
            for (int q = 0; q < 8; q++)
                *reinterpret_cast<uint4*>(stage + (q * 4 + cp_page) * kStageRow + cp_blk * 16) = R[q];
            __syncwarp();
            if (c + 1 < nchunks) fetch(c + 1);
#pragma unroll 1
            for (int i = 0; i < kStageBlocks; i++) {
                const uint4 pt = *reinterpret_cast<const uint4*>(own + i * 16);
                xor4(x, pt.x, pt.y, pt.z, pt.w);
                encrypt_block<NR>(x.x, x.y, x.z, x.w, T, K);
                *reinterpret_cast<uint4*>(own + i * 16) = x;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint64_t pg = (g << 5) + q * 4 + cp_page;
                if (pg < p.npages)
                    p.dst[pg * bpp + c * kStageBlocks + cp_blk] =
                        *reinterpret_cast<const uint4*>(stage + (q * 4 + cp_page) * kStageRow + cp_blk * 16);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// CBC encryption, staged by the tensor-memory-access engine.  The chains are
// the same (one page per lane).  Lane 0 brings each 8-block chunk of the
// warp's 32 pages in as one 2-D tile, 32 rows of 128 B, with 128-byte
// swizzle: 16-byte piece i of row r lands at piece i ^ (r % 8), so that the
// lanes' 16-byte reads of their own rows fall on distinct banks.  The lanes
// encipher their rows in place, and lane 0 writes the tile back with one
// tensor store, waits until the store has read the buffer, and brings in the
// next chunk.  Neither copy passes through registers or the load/store
// pipe.  Rows past the last page are filled with zeros on the way in and
// clipped on the way out.  Every wait on the tile's mbarrier is bounded; a
// wait that runs out is counted in g_bulk_wait_timeouts, the warp waits once
// more (bounded) for its copy in flight and leaves its remaining pages
// untouched.
// ---------------------------------------------------------------------------
__device__ unsigned int g_bulk_wait_timeouts;

__device__ __forceinline__ bool tile_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); i++) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tile_load(uint32_t sbuf, uint64_t map, int x, int y, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)kTmaWarpBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(sbuf),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tile_store(uint64_t map, int x, int y, uint32_t sbuf) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
                 "r"(x), "r"(y), "r"(sbuf)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tile_stores_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tile_stores_done() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int NR>
__global__ void __launch_bounds__(kCbcEncStagedThreads, 1) cbc_enc_tma_kernel(const __grid_constant__ CbcTmaParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    // kSmemBase + kSmemEnc + warp * 4096: 1024-byte aligned in the shared
    // window, as the 128-byte swizzle wants
    char* buf = smem + kSmemEnc + warp * kTmaWarpBytes;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(buf);
    const uint32_t bar =
        (uint32_t)__cvta_generic_to_shared(smem + kSmemEnc + kCbcEncStagedMaxWarps * kTmaWarpBytes + warp * 8);
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tensor copies see it initialised
    }
    fill_enc(smem);
    __syncthreads();

    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const ParamKey K{p.rk};
    const uint32_t nchunks = p.bpp / kStageBlocks;
    const uint64_t ngroups = (p.npages + 31) >> 5;
    const uint64_t src_map = reinterpret_cast<uint64_t>(&p.src_map);
    const uint64_t dst_map = reinterpret_cast<uint64_t>(&p.dst_map);
    char* own = buf + lane * 128;  // this lane's row
    uint32_t parity = 0;
    bool ok = true;
    for (uint64_t g = interleaved_warp(); ok && g < ngroups; g += total_warps()) {
        const uint64_t page = (g << 5) + lane;
        uint4 x = page < p.npages ? p.ivs[page] : make_uint4(0, 0, 0, 0);
        const int y = (int)(g << 5);
        if (lane == 0) {
            tile_stores_read();  // the previous group's last store has read the buffer
            tile_load(sbuf, src_map, 0, y, bar);
        }
        for (uint32_t c = 0; c < nchunks; ++c) {
            ok = __all_sync(0xffffffffu, tile_wait(bar, parity));
            if (!ok) break;
            parity ^= 1;
#pragma unroll 1
            for (int i = 0; i < kStageBlocks; i++) {
                uint4* blk = reinterpret_cast<uint4*>(own + ((i ^ (lane & 7)) << 4));
                const uint4 pt = *blk;
                xor4(x, pt.x, pt.y, pt.z, pt.w);
                encrypt_block<NR>(x.x, x.y, x.z, x.w, T, K);
                *blk = x;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tensor store sees the rows
            __syncwarp();
            if (lane == 0) {
                tile_store(dst_map, (int)(c * 32), y, sbuf);
                if (c + 1 < nchunks) {
                    tile_stores_read();
                    tile_load(sbuf, src_map, (int)((c + 1) * 32), y, bar);
                }
            }
        }
    }
    if (!ok && lane == 0) {
        atomicAdd(&g_bulk_wait_timeouts, 1u);
        tile_wait(bar, parity);  // the load still in flight, bounded
    }
    if (lane == 0) tile_stores_done();
}

// ---------------------------------------------------------------------------
// XTS with ciphertext stealing (IEEE 1619-2007 5.3.2 encryption, 5.4.2
// decryption) for data units of du bytes, du >= 16 and not a multiple of 16:
// m full blocks and a final partial block of b bytes.  One warp per data unit:
// full blocks 0..m-2 go to the lanes (block j with T * alpha^j), then lane 0
// runs the stealing pair, the last full block and the partial block, which
// depend on each other:
//   encryption: CC = enc(P_{m-1}, T a^{m-1});  C_m = CC[0..b);
//               C_{m-1} = enc(P_m || CC[b..16), T a^m)
//   decryption: PP = dec(C_{m-1}, T a^m);  P_m = PP[0..b);
//               P_{m-1} = dec(C_m || PP[b..16), T a^{m-1})
// Unit starts are only as aligned as u * du, so the unit's blocks move through
// 16-, 4- or 1-byte accesses as its start allows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 load_block(const uint8_t* q, uint32_t align) {
    if (align == 16) return *reinterpret_cast<const uint4*>(q);
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (align == 4) {
            w[i] = reinterpret_cast<const uint32_t*>(q)[i];
        } else {
            w[i] = (uint32_t)q[4 * i] | (uint32_t)q[4 * i + 1] << 8 | (uint32_t)q[4 * i + 2] << 16 |
                   (uint32_t)q[4 * i + 3] << 24;
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void store_block(uint8_t* q, const uint4& v, uint32_t align) {
    if (align == 16) {
        *reinterpret_cast<uint4*>(q) = v;
        return;
    }
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (align == 4) {
            reinterpret_cast<uint32_t*>(q)[i] = w[i];
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) q[4 * i + k] = (uint8_t)(w[i] >> (8 * k));
        }
    }
}

template <int NR, int DIR>
__global__ void __launch_bounds__(kBulkThreads, 1) xts_cts_kernel(const __grid_constant__ CtsParams p) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    if (DIR == 0) fill_enc(smem);
    else fill_dec(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const Rep4 T{lane * 4u, lane * 4u + 128u};
    const Rep1<2> IS{lane * 4u};
    const Rep1<2> TE{lane * 4u + 128u};
    const ParamKey K{p.rk};
    const ParamKey TK{p.tk};
    const uint64_t m = p.du / 16;
    const uint32_t b = (uint32_t)(p.du % 16);

    auto block = [&](uint4& v, uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3) {
        xor4(v, t0, t1, t2, t3);
        if (DIR == 0) encrypt_block<NR>(v.x, v.y, v.z, v.w, T, K);
        else decrypt_block<NR>(v.x, v.y, v.z, v.w, T, IS, K);
        xor4(v, t0, t1, t2, t3);
    };

    for (uint64_t u = interleaved_warp(); u < p.units; u += total_warps()) {
        const uint8_t* in = p.src + u * p.du;
        uint8_t* out = p.dst + u * p.du;
        const uint32_t off = (uint32_t)((uintptr_t)in & 15u);
        const uint32_t align = off == 0 ? 16u : (off & 3u) == 0 ? 4u : 1u;
        // E_K2(unit number) on every lane
        const uint64_t unit = p.first_sector + u;
        uint32_t z0 = (uint32_t)unit, z1 = (uint32_t)(unit >> 32), z2 = 0, z3 = 0;
        if (DIR == 0) encrypt_block<NR>(z0, z1, z2, z3, T, TK);
        else encrypt_block<NR>(z0, z1, z2, z3, TE, TK);
        // blocks 0..m-2, lane-strided
        uint32_t t0 = z0, t1 = z1, t2 = z2, t3 = z3;
        gf128_mul_xk(t0, t1, t2, t3, lane);
        for (uint64_t j = lane; j + 1 < m; j += 32) {
            uint4 v = load_block(in + 16 * j, align);
            block(v, t0, t1, t2, t3);
            store_block(out + 16 * j, v, align);
            gf128_mul_x32(t0, t1, t2, t3);
        }
        // the stealing pair: tweaks T a^{m-1} (a*) and T a^m (c*)
        if (lane == 0) {
            uint32_t a0 = z0, a1 = z1, a2 = z2, a3 = z3;
            gf128_mul_xpow(a0, a1, a2, a3, (uint32_t)(m - 1));
            uint32_t c0 = a0, c1 = a1, c2 = a2, c3 = a3;
            gf128_mul_xk(c0, c1, c2, c3, 1);
            uint4 x = load_block(in + 16 * (m - 1), align);
            const uint8_t* tail = in + 16 * m;
            // both inputs are read before anything is written (in-place calls)
            uint32_t yw[4] = {0, 0, 0, 0};
            if (DIR == 0) block(x, a0, a1, a2, a3);  // CC
            else block(x, c0, c1, c2, c3);           // PP
            const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const uint32_t byte = (uint32_t)k < b ? (uint32_t)tail[k] : (xw[k >> 2] >> (8 * (k & 3))) & 0xffu;
                yw[k >> 2] |= byte << (8 * (k & 3));
            }
            uint4 y = make_uint4(yw[0], yw[1], yw[2], yw[3]);
            if (DIR == 0) block(y, c0, c1, c2, c3);  // C_{m-1}
            else block(y, a0, a1, a2, a3);           // P_{m-1}
            store_block(out + 16 * (m - 1), y, align);
#pragma unroll
            for (int k = 0; k < 16; k++)
                if ((uint32_t)k < b) out[16 * m + k] = (uint8_t)(xw[k >> 2] >> (8 * (k & 3)));
        }
    }
}

template <class P>
using KernelFn = void (*)(P);

inline int grid_for(uint64_t warp_items, int num_sms) {
    // warp_items: how many warp-sized work items exist; at least one per warp.
    uint64_t ctas = (warp_items + (kBulkThreads / 32) - 1) / (kBulkThreads / 32);
    if (ctas < 1) ctas = 1;
    if (ctas > (uint64_t)num_sms) ctas = num_sms;
    return (int)ctas;
}

template <int NR>
KernelFn<BulkParams> pick_bulk(int dir, bool tweak) {
    if (tweak) return dir == 0 ? bulk_kernel<NR, 0, true> : bulk_kernel<NR, 1, true>;
    return dir == 0 ? bulk_kernel<NR, 0, false> : bulk_kernel<NR, 1, false>;
}

KernelFn<BulkParams> bulk_fn(int nr, int dir, bool tweak) {
    switch (nr) {
        case 10: return pick_bulk<10>(dir, tweak);
        case 12: return pick_bulk<12>(dir, tweak);
        case 14: return pick_bulk<14>(dir, tweak);
        default: return nullptr;
    }
}

KernelFn<CtsParams> cts_fn(int nr, int dir) {
    switch (nr) {
        case 10: return dir ? xts_cts_kernel<10, 1> : xts_cts_kernel<10, 0>;
        case 12: return dir ? xts_cts_kernel<12, 1> : xts_cts_kernel<12, 0>;
        case 14: return dir ? xts_cts_kernel<14, 1> : xts_cts_kernel<14, 0>;
        default: return nullptr;
    }
}

KernelFn<CbcParams> cbc_enc_staged_fn(int nr) {
    switch (nr) {
        case 10: return cbc_enc_staged_kernel<10>;
        case 12: return cbc_enc_staged_kernel<12>;
        case 14: return cbc_enc_staged_kernel<14>;
        default: return nullptr;
    }
}

KernelFn<CbcTmaParams> cbc_enc_tma_fn(int nr) {
    switch (nr) {
        case 10: return cbc_enc_tma_kernel<10>;
        case 12: return cbc_enc_tma_kernel<12>;
        case 14: return cbc_enc_tma_kernel<14>;
        default: return nullptr;
    }
}

// cuTensorMapEncodeTiled, found through the runtime (no link against the
// driver library); null if the driver does not provide it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// The pages [0, npages) of bpp blocks at base as a 2-D tensor of 32-bit words
// read and written in boxes of 32 words (one 8-block chunk) x 32 pages.
bool page_tile_map(CUtensorMap* m, const void* base, uint64_t npages, uint32_t bpp) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || npages > 0x7fffffffull) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)bpp * 4, (cuuint64_t)npages};
    const cuuint64_t stride[1] = {(cuuint64_t)bpp * 16};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estride[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base), dim, stride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

KernelFn<CbcParams> cbc_fn(int nr, bool enc) {
    switch (nr) {
        case 10: return enc ? cbc_enc_kernel<10> : cbc_dec_kernel<10>;
        case 12: return enc ? cbc_enc_kernel<12> : cbc_dec_kernel<12>;
        case 14: return enc ? cbc_enc_kernel<14> : cbc_dec_kernel<14>;
        default: return nullptr;
    }
}

}  // namespace

cudaError_t bulk_wait_timeouts(unsigned int* out) {
    return cudaMemcpyFromSymbol(out, g_bulk_wait_timeouts, sizeof(unsigned int));
}

cudaError_t configure_kernels() {
    for (int nr : {10, 12, 14}) {
        for (int dir = 0; dir < 2; dir++) {
            for (bool tw : {false, true}) {
                cudaError_t e = cudaFuncSetAttribute(bulk_fn(nr, dir, tw), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)(dir == 0 ? kSmemEnc : kSmemDec));
                if (e != cudaSuccess) return e;
            }
        }
        cudaError_t e = cudaFuncSetAttribute(cbc_fn(nr, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemEnc);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(cbc_fn(nr, false), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemDec);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(cbc_enc_staged_fn(nr), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemEncStaged);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(cbc_enc_tma_fn(nr), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemEncTma);
        if (e != cudaSuccess) return e;
        for (int dir = 0; dir < 2; dir++) {
            e = cudaFuncSetAttribute(cts_fn(nr, dir), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(dir == 0 ? kSmemEnc : kSmemDec));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t upload_tables(const uint32_t* te0, const uint32_t* td0, const uint32_t* isb4) {
    cudaError_t e = cudaMemcpyToSymbol(g_te0, te0, 1024);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_td0, td0, 1024);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_isb4, isb4, 1024);
    return e;
}

static cudaError_t launch_bulk(const BulkParams& p, int nr, int dir, bool tweak, int num_sms, cudaStream_t s) {
    auto fn = bulk_fn(nr, dir, tweak);
    if (!fn) return cudaErrorInvalidValue;
    int grid = grid_for((p.nblocks + 31) / 32, num_sms);
    fn<<<grid, kBulkThreads, dir == 0 ? kSmemEnc : kSmemDec, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_xts(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s) {
    return launch_bulk(p, nr, dir, true, num_sms, s);
}

cudaError_t launch_ecb(const BulkParams& p, int nr, int dir, int num_sms, cudaStream_t s) {
    return launch_bulk(p, nr, dir, false, num_sms, s);
}

cudaError_t launch_cbc_dec(const CbcParams& p, int nr, int num_sms, cudaStream_t s) {
    auto fn = cbc_fn(nr, false);
    if (!fn) return cudaErrorInvalidValue;
    int grid = grid_for(p.npages, num_sms);
    fn<<<grid, kBulkThreads, kSmemDec, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_xts_cts(const CtsParams& p, int nr, int dir, int num_sms, cudaStream_t s) {
    auto fn = cts_fn(nr, dir);
    if (!fn) return cudaErrorInvalidValue;
    const uint64_t warps = kBulkThreads / 32;
    const uint64_t ctas = (p.units + warps - 1) / warps;
    const int grid = (int)(ctas < (uint64_t)num_sms ? (ctas ? ctas : 1) : num_sms);
    fn<<<grid, kBulkThreads, dir == 0 ? kSmemEnc : kSmemDec, s>>>(p);
    return cudaGetLastError();
}

// A group (32 whole-page chains, one warp) is one long serial job, so the
// groups run in waves of warps x SMs, and a last wave that fills only part of
// the warps leaves the SMs' lookup path under-used for a whole chain's time.
// With 16 warps an SM's shared-memory path is kept busy (ncu: 91% of the
// kernel's own lookup bound, the rest being the tail), so a wave of w warps
// per SM costs about max(w, 16) chain-times of lookups.  Pick the warp count
// with the lowest total over the waves (ties: more warps).  1 GiB of 4-KiB
// pages is 8,192 groups: 16 warps take 3.37 waves (the fourth on 37% of the
// warps), 18 take 2.99.  (At 21 warps the register cap drops to 80 and the
// kernel spills.)
int cbc_enc_staged_warps(uint64_t groups, int num_sms) {
    constexpr int kSat = 16;
    const uint64_t sms = (uint64_t)(num_sms > 0 ? num_sms : 1);
    if (groups < kSat * sms) {  // one wave; extra warps only speed the table fill
        const uint64_t w = (groups + sms - 1) / sms;
        return (int)(w < 8 ? 8 : w);
    }
    int best = kCbcEncStagedMaxWarps;
    uint64_t best_cost = UINT64_MAX;
    for (int w = kCbcEncStagedMaxWarps; w >= kSat; --w) {
        const uint64_t per_wave = (uint64_t)w * sms;
        const uint64_t full = groups / per_wave, rest = groups % per_wave;
        const uint64_t last = (rest + sms - 1) / sms;  // warps per SM in the last wave
        const uint64_t cost = full * (uint64_t)w + (rest ? (last > kSat ? last : kSat) : 0);
        if (cost < best_cost) {
            best_cost = cost;
            best = w;
        }
    }
    return best;
}

// The last pair of tensor maps made, for calls that repeat on the same buffers
// (encoding one costs microseconds of host time).
struct TileMapCache {
    std::mutex mu;
    bool valid = false;
    const void* src = nullptr;
    const void* dst = nullptr;
    uint64_t npages = 0;
    uint32_t bpp = 0;
    CUtensorMap src_map, dst_map;
};

bool page_tile_maps(CbcTmaParams* t, const CbcParams& p) {
    static TileMapCache c;
    std::lock_guard<std::mutex> lk(c.mu);
    if (!(c.valid && c.src == p.src && c.dst == p.dst && c.npages == p.npages && c.bpp == p.bpp)) {
        c.valid = page_tile_map(&c.src_map, p.src, p.npages, p.bpp) && page_tile_map(&c.dst_map, p.dst, p.npages, p.bpp);
        if (!c.valid) return false;
        c.src = p.src;
        c.dst = p.dst;
        c.npages = p.npages;
        c.bpp = p.bpp;
    }
    t->src_map = c.src_map;
    t->dst_map = c.dst_map;
    return true;
}

cudaError_t launch_cbc_enc(const CbcParams& p, int nr, int num_sms, cudaStream_t s) {
    // The tensor tiles take a seventh of the staging traffic off the
    // shared-memory path, which pays once that path is the bound: from 12
    // groups of 32 pages per SM (measured at 4-KiB pages: 8 groups per SM
    // 227 us staged through registers against 232 us in tiles, 16 groups
    // 389 against 355 us).  Below that a launch is a chain's latency either
    // way, and the tiles' two tensor maps would only add host time.
    const uint64_t groups = (p.npages + 31) / 32;
    if (p.bpp % kStageBlocks == 0 && groups >= 12ull * (uint64_t)(num_sms > 0 ? num_sms : 1)) {
        CbcTmaParams t;
        std::memset(&t, 0, sizeof(t));
        auto fn = cbc_enc_tma_fn(nr);
        if (fn && page_tile_maps(&t, p)) {
            t.ivs = p.ivs;
            t.npages = p.npages;
            t.bpp = p.bpp;
            std::memcpy(t.rk, p.rk, sizeof(t.rk));
            const int grid = num_sms;
            const int warps = cbc_enc_staged_warps(groups, num_sms);
            fn<<<grid, warps * 32, kSmemEncTma, s>>>(t);
            return cudaGetLastError();
        }
    }
    if (p.bpp % kStageBlocks == 0) {
        auto fn = cbc_enc_staged_fn(nr);
        if (!fn) return cudaErrorInvalidValue;
        const int grid = (int)(groups < (uint64_t)num_sms ? (groups ? groups : 1) : num_sms);
        const int warps = cbc_enc_staged_warps(groups, num_sms);
        fn<<<grid, warps * 32, kSmemEnc + warps * kStageWarpSmem, s>>>(p);
        return cudaGetLastError();
    }
    auto fn = cbc_fn(nr, true);
    if (!fn) return cudaErrorInvalidValue;
    // a 32-page group is a heavy work item (32 chains of whole pages): give
    // every SM work as soon as there are as many groups as SMs
    const int grid = (int)(groups < (uint64_t)num_sms ? (groups ? groups : 1) : num_sms);
    fn<<<grid, kBulkThreads, kSmemEnc, s>>>(p);
    return cudaGetLastError();
}

}  // namespace kgpu
