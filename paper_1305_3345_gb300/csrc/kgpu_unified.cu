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
// prefix, copy that request's key schedule into the warp's key slot in shared
// memory when it changes (each round then reads its key with one broadcast
// load), and run the tile.  The 512-thread batch kernel also holds a pool of
// shared staging areas that CBC-encryption tiles of device pages move their
// pages through.
#include <cuda_runtime.h>

#include <algorithm>

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

// This warp's key slots in shared memory (512 B per warp after the tables):
// the data schedule at +0 and the XTS tweak schedule at +256.
struct WarpKeys {
    uint32_t* slot;       // generic pointer to the slot
    uint32_t data_saddr;  // shared-window addresses for the round-key loads
    uint32_t twk_saddr;
    uint32_t stage_saddr;  // serving kernel: this warp's staging rows in shared memory, else 0
    int nr;
};

__device__ __forceinline__ WarpKeys warp_keys(char* smem, uint32_t warp) {
    WarpKeys K;
    K.slot = reinterpret_cast<uint32_t*>(smem + 3 * kRegion + warp * 512);
    K.data_saddr = (uint32_t)__cvta_generic_to_shared(K.slot);
    K.twk_saddr = K.data_saddr + 256;
    K.stage_saddr = 0;
    K.nr = 0;
    return K;
}

// XTS (TWEAK) or ECB over the 32-block chunks [c0, c1) of one request.
template <bool TWEAK>
__device__ __forceinline__ void tile_blocks(const ReqDesc& d, uint64_t c0, uint64_t c1, int dir,
                                            const WarpKeys& K) {
    __syncwarp();  // lanes must run each step together (shuffles below)
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, dir);
    const UniLanes LE = uni_lanes(lane, 0);
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
        cipher_u(z0, z1, z2, z3, K.twk_saddr, K.nr, LE);
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
    // the next chunk is fetched while this one is enciphered (one warp runs a
    // tile alone, so the load latency would otherwise add to every step)
    uint4 nxt = (c0 < c1 && blk < d.nblocks) ? d.src[blk] : make_uint4(0, 0, 0, 0);
    for (uint64_t c = c0; c < c1; ++c) {
        const bool valid = blk < d.nblocks;
        uint4 v = nxt;
        if (c + 1 < c1 && blk + 32 < d.nblocks) nxt = d.src[blk + 32];
        if (TWEAK) xor4(v, t0, t1, t2, t3);
        cipher_block(v, K.data_saddr, K.nr, L, dir);
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

// Two blocks per lane through the unified cipher at once (u-frame state and
// key): one round-key broadcast serves both, and the warp keeps twice the
// independent lookups in flight.  Used by the 512-thread batch kernel, which
// has the registers for it.
__device__ __forceinline__ void cipher_u2(uint32_t& a0, uint32_t& a1, uint32_t& a2, uint32_t& a3, uint32_t& b0,
                                          uint32_t& b1, uint32_t& b2, uint32_t& b3, uint32_t key_saddr, int nr,
                                          const UniLanes& L) {
    uint4 k = round_key(key_saddr, 0);
    a0 ^= k.x, a1 ^= k.y, a2 ^= k.z, a3 ^= k.w;
    b0 ^= k.x, b1 ^= k.y, b2 ^= k.z, b3 ^= k.w;
#pragma unroll 1
    for (int r = 1; r < nr; r++) {
        k = round_key(key_saddr, r);
        const uint32_t s0 = uni_col(a0, a1, a2, a3, k.x, L), u0 = uni_col(b0, b1, b2, b3, k.x, L);
        const uint32_t s1 = uni_col(a1, a2, a3, a0, k.y, L), u1 = uni_col(b1, b2, b3, b0, k.y, L);
        const uint32_t s2 = uni_col(a2, a3, a0, a1, k.z, L), u2 = uni_col(b2, b3, b0, b1, k.z, L);
        const uint32_t s3 = uni_col(a3, a0, a1, a2, k.w, L), u3 = uni_col(b3, b0, b1, b2, k.w, L);
        a0 = s0, a1 = s1, a2 = s2, a3 = s3;
        b0 = u0, b1 = u1, b2 = u2, b3 = u3;
    }
    k = round_key(key_saddr, 14);  // the final round key sits in words 56..59
#define KGPU_FIN(P, x) lds_tab<kSmemBase>(row_addr<P>(x, L.f))
    const uint32_t o0 = merge_bytes(KGPU_FIN(0, a0), KGPU_FIN(1, a1), KGPU_FIN(2, a2), KGPU_FIN(3, a3)) ^ k.x;
    const uint32_t q0 = merge_bytes(KGPU_FIN(0, b0), KGPU_FIN(1, b1), KGPU_FIN(2, b2), KGPU_FIN(3, b3)) ^ k.x;
    const uint32_t o1 = merge_bytes(KGPU_FIN(0, a1), KGPU_FIN(1, a2), KGPU_FIN(2, a3), KGPU_FIN(3, a0)) ^ k.y;
    const uint32_t q1 = merge_bytes(KGPU_FIN(0, b1), KGPU_FIN(1, b2), KGPU_FIN(2, b3), KGPU_FIN(3, b0)) ^ k.y;
    const uint32_t o2 = merge_bytes(KGPU_FIN(0, a2), KGPU_FIN(1, a3), KGPU_FIN(2, a0), KGPU_FIN(3, a1)) ^ k.z;
    const uint32_t q2 = merge_bytes(KGPU_FIN(0, b2), KGPU_FIN(1, b3), KGPU_FIN(2, b0), KGPU_FIN(3, b1)) ^ k.z;
    const uint32_t o3 = merge_bytes(KGPU_FIN(0, a3), KGPU_FIN(1, a0), KGPU_FIN(2, a1), KGPU_FIN(3, a2)) ^ k.w;
    const uint32_t q3 = merge_bytes(KGPU_FIN(0, b3), KGPU_FIN(1, b0), KGPU_FIN(2, b1), KGPU_FIN(3, b2)) ^ k.w;
#undef KGPU_FIN
    a0 = o0, a1 = o1, a2 = o2, a3 = o3;
    b0 = q0, b1 = q1, b2 = q2, b3 = q3;
}

// Two blocks in natural column order in direction dir (see cipher_block).
__device__ __forceinline__ void cipher_block2(uint4& a, uint4& b, uint32_t key_saddr, int nr, const UniLanes& L,
                                              int dir) {
    if (dir) {
        uint32_t t = a.y;
        a.y = a.w, a.w = t;
        t = b.y;
        b.y = b.w, b.w = t;
    }
    cipher_u2(a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, key_saddr, nr, L);
    if (dir) {
        uint32_t t = a.y;
        a.y = a.w, a.w = t;
        t = b.y;
        b.y = b.w, b.w = t;
    }
}

// tile_blocks with two 32-block chunks per step: a lane takes block b of
// chunk c and block b of chunk c + 1, whose tweak is the same lane's tweak
// moved on by one chunk.
template <bool TWEAK>
__device__ __forceinline__ void tile_blocks2(const ReqDesc& d, uint64_t c0, uint64_t c1, int dir,
                                             const WarpKeys& K) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, dir);
    const UniLanes LE = uni_lanes(lane, 0);
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
        cipher_u(z0, z1, z2, z3, K.twk_saddr, K.nr, LE);
    };
    // the lane's block and tweak moved on by one chunk (every lane together:
    // the tweak batch and the shuffles are warp-wide)
    auto advance = [&]() {
        blk += 32;
        if (!TWEAK) return;
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
    const uint4 zz = make_uint4(0, 0, 0, 0);
    // the next step's two chunks are fetched while this step's are enciphered
    uint4 na = (c0 < c1 && blk < d.nblocks) ? d.src[blk] : zz;
    uint4 nb = (c0 + 1 < c1 && blk + 32 < d.nblocks) ? d.src[blk + 32] : zz;
    for (uint64_t c = c0; c < c1; c += 2) {
        const bool two = c + 1 < c1;
        uint4 va = na, vb = nb;
        const uint64_t ba = blk;
        const uint32_t a0 = t0, a1 = t1, a2 = t2, a3 = t3;
        if (two) advance();
        if (c + 2 < c1 && ba + 64 < d.nblocks) na = d.src[ba + 64];
        if (c + 3 < c1 && ba + 96 < d.nblocks) nb = d.src[ba + 96];
        if (TWEAK) {
            xor4(va, a0, a1, a2, a3);
            xor4(vb, t0, t1, t2, t3);
        }
        cipher_block2(va, vb, K.data_saddr, K.nr, L, dir);
        if (TWEAK) {
            xor4(va, a0, a1, a2, a3);
            xor4(vb, t0, t1, t2, t3);
        }
        if (ba < d.nblocks) d.dst[ba] = va;
        if (two && ba + 32 < d.nblocks) d.dst[ba + 32] = vb;
        if (c + 2 < c1) advance();
    }
}

// tile_cbc_dec with two 32-block steps at once: a lane takes block b of this
// step's first half and block b of its second half.
__device__ __forceinline__ void tile_cbc_dec2(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 1);
    const uint32_t bpp = d.unit_blocks;
    const uint64_t bend = p1 * bpp;
    uint64_t blk = p0 * bpp + lane;
    uint64_t pa = p0 + lane / bpp, pb = p0 + (lane + 32) / bpp;
    uint32_t ja = lane % bpp, jb = (lane + 32) % bpp;
    auto step = [&](uint64_t& page, uint32_t& j) {
        j += 64;
        if (j >= bpp) {
            uint32_t ns = j / bpp;
            page += ns;
            j -= ns * bpp;
        }
    };
    uint4 carry = make_uint4(0, 0, 0, 0);
    const uint4 zz = make_uint4(0, 0, 0, 0);
    uint4 na = blk < bend ? d.src[blk] : zz;
    uint4 nb = blk + 32 < bend ? d.src[blk + 32] : zz;
    const uint32_t src_lane = (lane + 31) & 31;
    for (uint64_t b = p0 * bpp; b < bend; b += 64) {
        const uint4 ca = na, cb = nb;
        if (blk + 64 < bend) na = d.src[blk + 64];  // prefetch the next step
        if (blk + 96 < bend) nb = d.src[blk + 96];
        // lane i takes lane i-1's block in each half; lane 0 of the second
        // half takes lane 31 of the first, lane 0 of the first the last step's
        uint4 xa, xb;
        xa.x = __shfl_sync(0xffffffffu, ca.x, src_lane);
        xa.y = __shfl_sync(0xffffffffu, ca.y, src_lane);
        xa.z = __shfl_sync(0xffffffffu, ca.z, src_lane);
        xa.w = __shfl_sync(0xffffffffu, ca.w, src_lane);
        xb.x = __shfl_sync(0xffffffffu, cb.x, src_lane);
        xb.y = __shfl_sync(0xffffffffu, cb.y, src_lane);
        xb.z = __shfl_sync(0xffffffffu, cb.z, src_lane);
        xb.w = __shfl_sync(0xffffffffu, cb.w, src_lane);
        uint4 prev_a = xa, prev_b = xb;
        if (lane == 0) {
            prev_a = carry;
            prev_b = xa;  // lane 31 of the first half
            carry = xb;   // lane 31 of the second half
        }
        if (blk < bend && ja == 0) prev_a = d.ivs[pa];
        if (blk + 32 < bend && jb == 0) prev_b = d.ivs[pb];
        uint4 va = ca, vb = cb;
        cipher_block2(va, vb, K.data_saddr, K.nr, L, 1);
        xor4(va, prev_a.x, prev_a.y, prev_a.z, prev_a.w);
        xor4(vb, prev_b.x, prev_b.y, prev_b.z, prev_b.w);
        if (blk < bend) d.dst[blk] = va;
        if (blk + 32 < bend) d.dst[blk + 32] = vb;
        blk += 64;
        step(pa, ja);
        step(pb, jb);
    }
}

// CBC decryption of pages [p0, p1) of one request (see cbc_dec_kernel).
__device__ __forceinline__ void tile_cbc_dec(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 1);
    const uint32_t bpp = d.unit_blocks;
    const uint64_t bend = p1 * bpp;
    uint64_t blk = p0 * bpp + lane;
    uint64_t page = p0 + lane / bpp;
    uint32_t j = lane % bpp;
    uint32_t carry0 = 0, carry1 = 0, carry2 = 0, carry3 = 0;
    uint4 nxt = blk < bend ? d.src[blk] : make_uint4(0, 0, 0, 0);
    for (uint64_t b = p0 * bpp; b < bend; b += 32) {
        const bool valid = blk < bend;
        const uint4 c = nxt;
        if (blk + 32 < bend) nxt = d.src[blk + 32];  // prefetch the next step
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
        cipher_block(v, K.data_saddr, K.nr, L, 1);
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
// Lanes without a page keep stepping with the others (their loads and stores
// are predicated off), so the warp runs every chain in one converged pass.
__device__ __forceinline__ void tile_cbc_enc(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 0);
    const uint64_t page = p0 + lane;
    const bool valid = page < p1;
    const uint32_t bpp = d.unit_blocks;
    const uint4* in = d.src + (valid ? page : p0) * bpp;
    uint4* out = d.dst + (valid ? page : p0) * bpp;
    const uint4 z = make_uint4(0, 0, 0, 0);
    uint4 x = valid ? d.ivs[page] : z;
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
        cipher_block(x, K.data_saddr, K.nr, L, 0);
        if (valid) out[i] = x;
    }
}

// CBC encryption of pages [p0, p1) (at most kQuadPages), four lanes per page:
// lane 4q + c holds column c of page q's chain state, so one chain advances
// about twice as fast as with a lane per page, for a quarter of the pages per
// warp -- the form for a lightly loaded device, where a request's latency is
// its chain time.  Each round a lane fetches the three other columns of its
// state from its quad (three independent shuffles), looks up its own column
// (the two-table round of uni_col) and reads its own round-key word from the
// warp's key slot (the quad's four words share one wavefront).  Lanes without
// a page step along with predicated-off memory accesses.
// One block of a four-lane chain: x is this lane's column of the block to
// encipher (plaintext xor chain value), key the shared address of its column
// of round 0 (words 4r + col of the schedule).
template <int NR>
__device__ __forceinline__ uint32_t quad_encrypt(uint32_t x, uint32_t s1, uint32_t s2, uint32_t s3,
                                                 const UniLanes& L, uint32_t key) {
    auto key_word = [&](int r) {
        uint32_t v;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(key + 16u * (uint32_t)r));
        return v;
    };
    x ^= key_word(0);
#pragma unroll
    for (int r = 1; r < NR; r++) {
        const uint32_t a1 = __shfl_sync(0xffffffffu, x, s1);
        const uint32_t a2 = __shfl_sync(0xffffffffu, x, s2);
        const uint32_t a3 = __shfl_sync(0xffffffffu, x, s3);
        x = uni_col(x, a1, a2, a3, key_word(r), L);
    }
    const uint32_t a1 = __shfl_sync(0xffffffffu, x, s1);
    const uint32_t a2 = __shfl_sync(0xffffffffu, x, s2);
    const uint32_t a3 = __shfl_sync(0xffffffffu, x, s3);
#define KGPU_FIN(P, v) lds_tab<kSmemBase>(row_addr<P>(v, L.f))
    return merge_bytes(KGPU_FIN(0, x), KGPU_FIN(1, a1), KGPU_FIN(2, a2), KGPU_FIN(3, a3)) ^ key_word(14);
#undef KGPU_FIN
}

template <int NR>
__device__ __forceinline__ void quad_chains(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    const uint32_t lane = lane_id();
    const uint32_t c = lane & 3u, base = lane & ~3u;
    const UniLanes L = uni_lanes(lane, 0);
    const uint64_t page = p0 + (lane >> 2);
    const bool valid = page < p1;
    const uint32_t bpp = d.unit_blocks;
    const uint32_t* in = reinterpret_cast<const uint32_t*>(d.src + (valid ? page : p0) * bpp) + c;
    uint32_t* out = reinterpret_cast<uint32_t*>(d.dst + (valid ? page : p0) * bpp) + c;
    const uint32_t key = K.data_saddr + 4u * c;  // word 4r + c of the schedule: round r, this column
    const uint32_t s1 = base | ((c + 1) & 3u), s2 = base | ((c + 2) & 3u), s3 = base | ((c + 3) & 3u);
    uint32_t x = valid ? reinterpret_cast<const uint32_t*>(d.ivs + page)[c] : 0u;
    // the chain is sequential, so plaintext is fetched four blocks ahead
    uint32_t q0 = valid ? in[0] : 0u;
    uint32_t q1 = valid && bpp > 1 ? in[4] : 0u;
    uint32_t q2 = valid && bpp > 2 ? in[8] : 0u;
    uint32_t q3 = valid && bpp > 3 ? in[12] : 0u;
    for (uint32_t i = 0; i < bpp; ++i) {
        const uint32_t cur = q0;
        q0 = q1;
        q1 = q2;
        q2 = q3;
        if (valid && i + 4 < bpp) q3 = in[4 * (i + 4)];
        x = quad_encrypt<NR>(x ^ cur, s1, s2, s3, L, key);
        if (valid) out[4 * i] = x;
    }
}

// Four-lane chains over pages in registered host memory: the warp moves 8
// blocks (one 128-byte line) of each of its 8 pages at a time between the
// buffers and its staging rows in shared memory with whole-line accesses -- a
// four-lane load straight from the pages would move a whole line over the
// link for 16 useful bytes -- and the quads run their chains on the staged
// copy.  The next chunk's lines are loaded from the host while the current
// chunk is enciphered.  sbuf: shared-window address of the warp's 8 rows of
// kServeStageRow bytes (the 16-byte pad per row spreads both the copies'
// 16-byte accesses and the quads' column reads over all banks).  Pages must
// hold a multiple of 8 blocks.
__device__ __forceinline__ void sts128(uint32_t a, const uint4& v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
                 : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

template <int NR>
__device__ __forceinline__ void quad_chains_staged(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K,
                                                   uint32_t sbuf) {
    const uint32_t lane = lane_id();
    const uint32_t c = lane & 3u, base = lane & ~3u, qp = lane >> 2;
    const UniLanes L = uni_lanes(lane, 0);
    const bool valid = p0 + qp < p1;
    const uint32_t bpp = d.unit_blocks;
    const uint32_t key = K.data_saddr + 4u * c;
    const uint32_t s1 = base | ((c + 1) & 3u), s2 = base | ((c + 2) & 3u), s3 = base | ((c + 3) & 3u);
    uint32_t x = valid ? reinterpret_cast<const uint32_t*>(d.ivs + p0 + qp)[c] : 0u;
    // copy positions: lanes 8p..8p+7 move page p's line (pages 0-3, then 4-7)
    const uint32_t cp_blk = lane & 7u, cp_pg0 = lane >> 3, cp_pg1 = cp_pg0 + 4;
    const bool ok0 = p0 + cp_pg0 < p1, ok1 = p0 + cp_pg1 < p1;
    const uint32_t cp0 = sbuf + cp_pg0 * (uint32_t)kServeStageRow + cp_blk * 16u;
    const uint32_t cp1 = sbuf + cp_pg1 * (uint32_t)kServeStageRow + cp_blk * 16u;
    const uint32_t col = sbuf + qp * (uint32_t)kServeStageRow + c * 4u;  // this lane's column of its page
    const uint4 z = make_uint4(0, 0, 0, 0);
    auto fetch = [&](uint32_t chunk, uint4& v0, uint4& v1) {
        v0 = ok0 ? d.src[(p0 + cp_pg0) * bpp + chunk + cp_blk] : z;
        v1 = ok1 ? d.src[(p0 + cp_pg1) * bpp + chunk + cp_blk] : z;
    };
    uint4 n0, n1;
    fetch(0, n0, n1);
    for (uint32_t ch = 0; ch < bpp; ch += kStageBlocks) {
        sts128(cp0, n0);
        sts128(cp1, n1);
        __syncwarp();
        if (ch + kStageBlocks < bpp) fetch(ch + kStageBlocks, n0, n1);  // in flight meanwhile
#pragma unroll 1
        for (uint32_t i = 0; i < kStageBlocks; i++) {
            x = quad_encrypt<NR>(x ^ lds32(col + 16u * i), s1, s2, s3, L, key);
            sts32(col + 16u * i, x);
        }
        __syncwarp();
        const uint4 o0 = lds128(cp0), o1 = lds128(cp1);
        if (ok0) d.dst[(p0 + cp_pg0) * bpp + ch + cp_blk] = o0;
        if (ok1) d.dst[(p0 + cp_pg1) * bpp + ch + cp_blk] = o1;
        __syncwarp();  // the rows are refilled next
    }
}

// The rounds are unrolled per key size: a lone chain is latency-bound, and a
// loop's branch would sit on its critical path every round.
__device__ __forceinline__ void tile_cbc_enc_quad(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K) {
    __syncwarp();
    switch (K.nr) {
        case 10: quad_chains<10>(d, p0, p1, K); break;
        case 12: quad_chains<12>(d, p0, p1, K); break;
        default: quad_chains<14>(d, p0, p1, K); break;
    }
}

__device__ __forceinline__ void tile_cbc_enc_quad_staged(const ReqDesc& d, uint64_t p0, uint64_t p1,
                                                         const WarpKeys& K, uint32_t sbuf) {
    __syncwarp();
    switch (K.nr) {
        case 10: quad_chains_staged<10>(d, p0, p1, K, sbuf); break;
        case 12: quad_chains_staged<12>(d, p0, p1, K, sbuf); break;
        default: quad_chains_staged<14>(d, p0, p1, K, sbuf); break;
    }
}

// CBC encryption of pages in registered host memory.  Over the host link a
// load moves a whole 128-byte line, so the one-lane-per-page accesses above
// would carry 16 useful bytes of every 128.  Here the warp moves 8 blocks
// (128 B) of each of its 32 pages at a time between the buffers and its
// 4-KiB scratch area in device memory, every instruction covering four whole
// lines, and the lanes run their chains on the scratch copy.  Scratch layout:
// [page of the tile][block of the chunk].  Pages must hold a multiple of 8
// blocks.  __syncwarp orders the lanes' scratch accesses (it is a memory
// barrier among the warp's threads).
__device__ __forceinline__ void tile_cbc_enc_staged(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K,
                                                    uint4* stage) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 0);
    const uint32_t bpp = d.unit_blocks;
    const uint4 z = make_uint4(0, 0, 0, 0);
    uint4 x = p0 + lane < p1 ? d.ivs[p0 + lane] : z;
    const uint32_t cp_page = lane >> 3, cp_blk = lane & (kStageBlocks - 1);  // copy position
    uint4* own = stage + lane * kStageBlocks;
    for (uint32_t c = 0; c < bpp; c += kStageBlocks) {
        // copy in, four instructions' worth of loads in flight at a time (the
        // register budget of the 1024-thread kernel)
#pragma unroll
        for (int h = 0; h < 8; h += 4) {
            uint4 v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint64_t pg = p0 + (h + q) * 4 + cp_page;
                v[q] = pg < p1 ? d.src[pg * bpp + c + cp_blk] : z;
            }
#pragma unroll
            for (int q = 0; q < 4; q++) stage[((h + q) * 4 + cp_page) * kStageBlocks + cp_blk] = v[q];
        }
        __syncwarp();
        // the scratch copy is near (L1/L2): two blocks ahead hide its latency
        uint4 q0 = own[0], q1 = own[1];
#pragma unroll 1
        for (uint32_t i = 0; i < kStageBlocks; ++i) {
            const uint4 cur = q0;
            q0 = q1;
            if (i + 2 < kStageBlocks) q1 = own[i + 2];
            xor4(x, cur.x, cur.y, cur.z, cur.w);
            cipher_block(x, K.data_saddr, K.nr, L, 0);
            own[i] = x;
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 8; h += 4) {
            uint4 v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] = stage[((h + q) * 4 + cp_page) * kStageBlocks + cp_blk];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint64_t pg = p0 + (h + q) * 4 + cp_page;
                if (pg < p1) d.dst[pg * bpp + c + cp_blk] = v[q];
            }
        }
    }
}

// CBC encryption of device pages through an area of the batch kernel's
// shared staging pool.  One lane runs one page's chain; a lane's own loads and
// stores would be 4 KiB from its neighbours', 32 lines per warp instruction.
// Instead the warp moves 4 blocks of each of its (up to) 32 pages at a time
// between global memory and the area -- every instruction covering 8 pages'
// 64 contiguous bytes -- and the lanes run their chains on the area's rows.
// Rows are 64 B with 16-byte piece i of row r stored at piece i ^ ((r/2) % 4),
// so that both the copies (two rows per 128 bytes of banks) and a lane's reads
// and writes of its own row are free of bank conflicts.  The next 4 blocks are
// loaded into registers while the current ones are enciphered.  Pages must
// hold a multiple of 4 blocks.
__device__ __forceinline__ uint32_t pool_piece(uint32_t row, uint32_t i) {
    return row * (uint32_t)kPoolRow + ((i ^ ((row >> 1) & 3u)) << 4);
}

__device__ __forceinline__ void tile_cbc_enc_pooled(const ReqDesc& d, uint64_t p0, uint64_t p1, const WarpKeys& K,
                                                    char* area) {
    __syncwarp();
    const uint32_t lane = lane_id();
    const UniLanes L = uni_lanes(lane, 0);
    const uint32_t bpp = d.unit_blocks;
    const uint4 z = make_uint4(0, 0, 0, 0);
    uint4 x = p0 + lane < p1 ? d.ivs[p0 + lane] : z;
    const uint32_t cp_page = lane >> 2, cp_blk = lane & (kPoolBlocks - 1);  // copy position
    uint4 R[4];
    auto fetch = [&](uint32_t c) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint64_t pg = p0 + q * 8 + cp_page;
            R[q] = pg < p1 ? d.src[pg * bpp + c + cp_blk] : z;
        }
    };
    fetch(0);
    for (uint32_t c = 0; c < bpp; c += kPoolBlocks) {
#pragma unroll
        for (int q = 0; q < 4; q++) *reinterpret_cast<uint4*>(area + pool_piece(q * 8 + cp_page, cp_blk)) = R[q];
        __syncwarp();
        if (c + kPoolBlocks < bpp) fetch(c + kPoolBlocks);
#pragma unroll 1
        for (uint32_t i = 0; i < kPoolBlocks; i++) {
            uint4* blk = reinterpret_cast<uint4*>(area + pool_piece(lane, i));
            const uint4 pt = *blk;
            xor4(x, pt.x, pt.y, pt.z, pt.w);
            cipher_block(x, K.data_saddr, K.nr, L, 0);
            *blk = x;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint64_t pg = p0 + q * 8 + cp_page;
            const uint4 v = *reinterpret_cast<const uint4*>(area + pool_piece(q * 8 + cp_page, cp_blk));
            if (pg < p1) d.dst[pg * bpp + c + cp_blk] = v;
        }
        __syncwarp();  // the rows are refilled next
    }
}

// Take a free area of the pool (warp-uniform result; -1 when all are in
// use) and give it back.  The mask lives after the areas.
__device__ __forceinline__ int pool_take(uint32_t* mask) {
    int a = -1;
    if (lane_id() == 0) {
        for (uint32_t tries = 0; tries < kPoolAreas; tries++) {
            const uint32_t m = *reinterpret_cast<volatile uint32_t*>(mask);
            const uint32_t free = ~m & ((1u << kPoolAreas) - 1u);
            if (!free) break;
            const uint32_t bit = free & (0u - free);
            if (!(atomicOr(mask, bit) & bit)) {
                a = __ffs(bit) - 1;
                break;
            }
        }
    }
    return __shfl_sync(0xffffffffu, a, 0);
}

__device__ __forceinline__ void pool_give(uint32_t* mask, int a) {
    __syncwarp();
    if (lane_id() == 0) {
        __threadfence_block();  // the warp's accesses to the area come first
        atomicAnd(mask, ~(1u << a));
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
// stage: this warp's scratch area, or null.  QUAD: compile the four-lanes-per-
// page CBC encryption in (only the serving kernel's descriptors ask for it,
// and it would cost the batch kernels registers).  TWO: XTS, ECB and CBC
// decryption two blocks per lane at a time (the 512-thread batch kernel,
// where throughput counts and the registers are there).
// The empty service (KGPU_MODE_COPY): units [u0, u1) of unit_blocks blocks
// each are copied through unchanged, one 16-byte access per lane per step.
__device__ __forceinline__ void tile_copy(const ReqDesc& d, uint64_t u0, uint64_t u1) {
    const uint64_t b1 = u1 * d.unit_blocks;
    for (uint64_t b = u0 * d.unit_blocks + lane_id(); b < b1; b += 32) d.dst[b] = d.src[b];
}

// RESIDENT: the kernel outlives key changes (the serving kernel), so the
// schedule a warp keeps is tagged with the key's generation as well, and the
// key record is read from L2 (ld.global.cg): the host rewrites it with a
// copy while the kernel runs, and a line this SM's L1 kept from the slot's
// previous key must not be taken for it.  A batch never sees a key change,
// since deleting a key waits for the batches in flight.
template <class T>
__device__ __forceinline__ T key_word(const T* p, bool l2_only) {
    return l2_only ? __ldcg(p) : *p;
}

template <bool QUAD, bool TWO = false, bool RESIDENT = false>
__device__ __forceinline__ int run_tile(const ReqDesc& d, uint64_t tile_in_req, const DevKey* keys, uint32_t max_keys,
                                     WarpKeys& K, uint32_t& cur_sel, uint32_t& cur_gen, uint4* stage,
                                     char* pool = nullptr) {
    const uint32_t lane = lane_id();
    if (d.mode == KGPU_MODE_COPY) {
        const uint64_t u0 = tile_in_req * d.tile_units, units = request_units(d);
        tile_copy(d, u0, u0 + d.tile_units < units ? u0 + d.tile_units : units);
        return 0;
    }
    if (d.key >= max_keys) return KGPU_ENOENT;
    const DevKey& dk = keys[d.key];
    const bool is_xts = d.mode == KGPU_MODE_XTS;
    const uint32_t flags = key_word(&dk.flags, RESIDENT);
    if (!(flags & kKeyLive) || ((flags & kKeyXts) != 0) != is_xts) return KGPU_ENOENT;
    const int dir = (d.mode == KGPU_MODE_CBC_DEC) ? 1 : (d.mode == KGPU_MODE_CBC_ENC) ? 0 : (int)d.dir;
    const uint32_t sel = d.key * 2u + (uint32_t)dir;
    const uint32_t gen = RESIDENT ? key_word(&dk.gen, true) : 0u;
    if (sel != cur_sel || gen != cur_gen) {
        const uint32_t* sched = dir ? dk.decu : dk.encu;
        __syncwarp();  // every lane is done with the previous key
        K.slot[lane] = key_word(&sched[lane], RESIDENT);
        if (lane < 28) K.slot[32 + lane] = key_word(&sched[32 + lane], RESIDENT);
        if (is_xts) {
            K.slot[64 + lane] = key_word(&dk.twku[lane], RESIDENT);
            if (lane < 28) K.slot[96 + lane] = key_word(&dk.twku[32 + lane], RESIDENT);
        }
        K.nr = (int)key_word(&dk.nr, RESIDENT);
        __syncwarp();
        cur_sel = sel;
        cur_gen = gen;
    }
    const uint64_t units = request_units(d);
    const uint64_t u0 = tile_in_req * d.tile_units;
    uint64_t u1 = u0 + d.tile_units;
    if (u1 > units) u1 = units;
    switch (d.mode) {
        case KGPU_MODE_XTS:
            if (TWO) tile_blocks2<true>(d, u0, u1, dir, K);
            else tile_blocks<true>(d, u0, u1, dir, K);
            break;
        case KGPU_MODE_ECB:
            if (TWO) tile_blocks2<false>(d, u0, u1, dir, K);
            else tile_blocks<false>(d, u0, u1, dir, K);
            break;
        case KGPU_MODE_CBC_DEC:
            if (TWO) tile_cbc_dec2(d, u0, u1, K);
            else tile_cbc_dec(d, u0, u1, K);
            break;
        case KGPU_MODE_CBC_ENC:
            if (stage && (d.flags & (kDescSrcHost | kDescDstHost)) && d.unit_blocks % kStageBlocks == 0) {
                if (QUAD && (d.flags & kDescQuad) && K.stage_saddr)
                    tile_cbc_enc_quad_staged(d, u0, u1, K, K.stage_saddr);
                else tile_cbc_enc_staged(d, u0, u1, K, stage);
            } else if (QUAD && (d.flags & kDescQuad)) {
                tile_cbc_enc_quad(d, u0, u1, K);
            } else if (pool && !(d.flags & (kDescSrcHost | kDescDstHost)) && d.unit_blocks % kPoolBlocks == 0) {
                uint32_t* mask = reinterpret_cast<uint32_t*>(pool + kPoolAreas * kPoolAreaBytes);
                const int a = pool_take(mask);
                if (a >= 0) {
                    tile_cbc_enc_pooled(d, u0, u1, K, pool + a * kPoolAreaBytes);
                    pool_give(mask, a);
                } else {
                    tile_cbc_enc(d, u0, u1, K);
                }
            } else {
                tile_cbc_enc(d, u0, u1, K);
            }
            break;
        default: return KGPU_EINVAL;
    }
    return 0;
}

// Memory-order helpers (PTX scopes: gpu = this device, sys = with the host).
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
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) batch_kernel(const __grid_constant__ BatchArgs a) {
    extern __shared__ __align__(128) char smem[];
    if (!smem_layout_ok(smem)) return;
    // the 512-thread variant's staging pool for CBC encryption of device pages
    char* pool = THREADS == kPoolThreads ? smem + 3 * kRegion + (THREADS / 32) * 512 : nullptr;
    if (pool && threadIdx.x == 0) *reinterpret_cast<uint32_t*>(pool + kPoolAreas * kPoolAreaBytes) = 0u;
    fill_unified(smem);
    __syncthreads();

    const uint32_t lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    WarpKeys K = warp_keys(smem, warp);
    uint32_t cur_sel = 0xffffffffu, cur_gen = 0;
    // Staged CBC encryption of host pages is compiled into the 512-thread
    // variant only: the 1024-thread variant has 64 registers per thread, and
    // the staged path would make it spill (the host side runs batches that
    // need staging with 512 threads).
    uint4* stage = nullptr;
    if constexpr (THREADS <= 512) {
        const uint32_t gw = blockIdx.x * (THREADS / 32) + warp;
        if (a.scratch && gw < a.scratch_warps) stage = a.scratch + (size_t)gw * (kStageWarpBytes / 16);
    }

    const BatchHeader* hdr = reinterpret_cast<const BatchHeader*>(a.buf);
    const uint64_t total = hdr->total_tiles;
    const uint32_t nreq = hdr->nreq;
    const ReqDesc* reqs = reinterpret_cast<const ReqDesc*>(a.buf + batch_desc_offset());
    const uint64_t* tile_start = reinterpret_cast<const uint64_t*>(a.buf + batch_prefix_offset(nreq));
    const uint32_t* order = reinterpret_cast<const uint32_t*>(a.buf + batch_order_offset(nreq));
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(a.next_tile, 1ull);
    next = __shfl_sync(0xffffffffu, next, 0);
    while (next < total) {
        const uint64_t t = next;
        if (lane == 0) next = atomicAdd(a.next_tile, 1ull);  // fetched while this tile runs
        const uint32_t k = find_request(tile_start, nreq, t);
        const uint32_t i = order[k];
        const ReqDesc d = reqs[i];
        const int st = run_tile<false, (THREADS <= 512)>(d, t - tile_start[k], a.keys, a.max_keys, K, cur_sel, cur_gen, stage,
                                                           pool);
        if (st && lane == 0) a.status[i] = st;
        if (a.fin) {
            // per-request completion: the warp that finishes a request's last
            // tile publishes (tag << 32 | status) to the host-mapped word,
            // after an acq_rel count that orders every warp's tile writes
            // before it (the same protocol as the serving ring)
            __syncwarp();
            unsigned long long f = 0;
            if (lane == 0) f = atom_add_acq_rel_gpu(&a.fin[i], 1ull) + 1;
            f = __shfl_sync(0xffffffffu, f, 0);
            if (lane == 0 && f == tile_start[k + 1] - tile_start[k]) {
                const unsigned int code = (unsigned int)*reinterpret_cast<volatile int*>(&a.status[i]);
                st_release_sys(&a.done[i], (unsigned long long)hdr->tag << 32 | code);
            }
        }
        next = __shfl_sync(0xffffffffu, next, 0);
    }
}


// ---------------------------------------------------------------------------
// Serving kernel: the paper's Non-Stop Kernel (section 3.1) -- launched once,
// fed through pinned host memory -- with every wait bounded.
//
// CTA 0 / warp 0 is the dispatcher.  It polls the host-written request count
// with system-scope acquire loads; for each new request it copies the
// descriptor into device memory, clears the request's finish counter and
// appends one entry per tile to a tile ring in device memory, then publishes
// the new ring head with a release store.  Worker warps take ring positions
// with one atomicAdd each (no retries, no contention loops), wait until their
// position is published, run that tile and count it finished; the warp that
// finishes a request's last tile publishes the completion to the host.  New
// requests are appended behind whatever is running: continuous batching at
// tile granularity.
//
// Exits: the host's stop flag, an idle period, or the lifetime limit make the
// dispatcher stop publishing and raise the device stop word; workers then
// finish any published position they hold and leave.  Positions claimed but
// never published are handed back by serve_reset_kernel before a relaunch.
// ---------------------------------------------------------------------------


__device__ void serve_dispatcher(const ServeArgs& a, unsigned long long t0) {
    const uint32_t lane = lane_id();
    unsigned long long m = ld_vol(&a.dev->mirrored);   // requests enumerated so far
    unsigned long long pub = ld_vol(&a.dev->tile_head);
    unsigned long long idle_since = t0;
    unsigned int backoff = 64, reason = 0, idle_polls = 0;
    const unsigned long long ring = a.tile_mask + 1;
    for (;;) {
        unsigned long long h = 0, now = 0;
        unsigned int stop = 0;
        if (lane == 0) {
            h = ld_acquire_sys(&a.hh->head);
            stop = *reinterpret_cast<volatile unsigned int*>(&a.hh->stop);
            now = gtimer();
        }
        h = __shfl_sync(0xffffffffu, h, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        now = __shfl_sync(0xffffffffu, now, 0);
        if (stop) {
            reason = kServeExitStop;
            break;
        }
        if (m < h) {
            // copy up to 32 new descriptors to device memory, one per lane
            // (the loads over the host link and the finished-tile count are
            // issued together: the request's own latency waits on them)
            const unsigned cnt = (unsigned)(h - m < 32 ? h - m : 32);
            const unsigned long long done_tiles = ld_vol(&a.dev->tile_done);
            unsigned long long nt = 0;
            if (lane < cnt) {
                const uint32_t s = (uint32_t)((m + lane) & a.slot_mask);
                const uint4* from = reinterpret_cast<const uint4*>(&a.slots[s]);
                uint4* to = reinterpret_cast<uint4*>(&a.dslots[s]);
                uint4 v[5];
#pragma unroll
                for (int q = 0; q < 5; q++) v[q] = from[q];  // ReqDesc, ntiles, seq
#pragma unroll
                for (int q = 0; q < 5; q++) to[q] = v[q];
                nt = (unsigned long long)v[4].y << 32 | v[4].x;  // ntiles
                a.dslots[s].t_disp = now;
                a.fin[s] = 0;
            }
            // enumerate their tiles, in order, as long as the ring has room;
            // each entry carries the high bits of its position as a tag
            unsigned taken = 0;
            for (unsigned i = 0; i < cnt; i++) {
                const unsigned long long n_i = __shfl_sync(0xffffffffu, nt, i);
                if (pub + n_i - done_tiles > ring) break;
                const unsigned long long s = (m + i) & a.slot_mask;
                if (lane == i) a.dslots[s].pos0 = pub;
                for (unsigned long long k = lane; k < n_i; k += 32) {
                    const unsigned long long pos = pub + k;
                    a.tiles[pos & a.tile_mask] = (((pos >> a.tile_bits) & 0xfffull) << 52) | (s << 32) | k;
                }
                pub += n_i;
                taken++;
            }
            if (lane < taken) a.dslots[(m + lane) & a.slot_mask].t_pub = gtimer();
            __syncwarp();
            __threadfence();
            if (taken && lane == 0) {
                a.dev->mirrored = m + taken;
                st_release_gpu(&a.dev->tile_head, pub);
            }
            if (taken) {
                // tell every CTA through its own mailbox line: the workers
                // poll only there, so no address is polled by the whole GPU
                __syncwarp();
                for (uint32_t c = lane; c < gridDim.x; c += 32)
                    *reinterpret_cast<volatile unsigned long long*>(&a.mbox[c * kMboxStride]) = pub;
            }
            m += taken;
            idle_since = now;
            backoff = 64;
            if (taken) continue;
        }
        const unsigned long long done = ld_vol(&a.dev->done_count);
        if (done != m || m != h) idle_since = now;  // work outstanding: not idle
        if (now - idle_since > a.idle_ns) {
            reason = kServeExitIdle;
            break;
        }
        if (now - t0 > a.lifetime_ns) {
            reason = kServeExitLifetime;
            break;
        }
        // the heartbeat (the host's clock-offset reference) every 16th idle
        // poll: a store over the link just before new work would make that
        // work's fence wait for it.  A system-scope release, so that it is
        // sent on at once (a plain store may wait in the cache, and the host
        // would then bound the offset too high).
        if (lane == 0 && (++idle_polls & 15) == 0) st_release_sys(&a.hh->heartbeat, now);
        __nanosleep(backoff);
        if (backoff < 128) backoff <<= 1;
    }
    if (lane == 0) {
        st_release_gpu32(&a.dev->stop, reason);
        a.hh->exit_code = reason;
        __threadfence_system();
    }
    __syncwarp();
    for (uint32_t c = lane; c < gridDim.x; c += 32)
        *reinterpret_cast<volatile unsigned long long*>(&a.mbox[c * kMboxStride]) = pub | kMboxStop;
}

// Before each launch: positions claimed but never published are handed back,
// and every CTA's mailbox restarts at the published count.
__global__ void serve_reset_kernel(ServeDev* dev, unsigned long long* mbox, int ctas) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (dev->tile_next > dev->tile_head) dev->tile_next = dev->tile_head;
        dev->stop = 0;
    }
    __syncthreads();
    const unsigned long long head = dev->tile_head;
    for (int c = threadIdx.x; c < ctas; c += blockDim.x) mbox[c * kMboxStride] = head;
    __threadfence();
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
    WarpKeys K = warp_keys(smem, warp);
    K.stage_saddr = (uint32_t)__cvta_generic_to_shared(smem + 3 * kRegion + (THREADS / 32) * 512 +
                                                       warp * kServeStageWarpBytes);
    uint32_t cur_sel = 0xffffffffu, cur_gen = 0;
    const uint32_t gw = blockIdx.x * (THREADS / 32) + warp;
    uint4* stage = a.scratch && gw < a.scratch_warps ? a.scratch + (size_t)gw * (kStageWarpBytes / 16) : nullptr;
    // a worker gives up on its own only if the dispatcher stopped answering
    const unsigned long long own_idle = a.idle_ns + 2000000000ull;

    // The loop keeps the warp's control flow uniform: lane-0-only work (the
    // claim and the finish count) is immediately followed by a shuffle of its
    // result, and the polling, stamps and status stores run on every lane.  A
    // lane that branched off alone could otherwise leave the warp split into
    // groups that then run the whole tile one after the other.
    for (;;) {
        unsigned long long T = 0;
        if (lane == 0) T = atomicAdd(&a.dev->tile_next, 1ull);
        T = __shfl_sync(0xffffffffu, T, 0);
        // wait until position T is published (bounded: stop bit, own limit).
        // The mailbox holds the published count: the dispatcher writes it
        // after a fence that follows its tile-ring and descriptor writes, and
        // the acquire load here orders this warp's reads of them after it.
        int go = 0;
        unsigned int backoff = 32;
        const unsigned long long w0 = gtimer();
        const unsigned long long* box = &a.mbox[blockIdx.x * kMboxStride];
        for (;;) {
            // every lane reads the same word of this CTA's mailbox line
            const unsigned long long v = __shfl_sync(0xffffffffu, ld_acquire_gpu(box), 0);
            if (T < (v & ~kMboxStop)) {
                go = 1;
                break;
            }
            if (v & kMboxStop) break;
            const unsigned long long now = __shfl_sync(0xffffffffu, gtimer(), 0);
            if (now - w0 > own_idle) break;
            __nanosleep(backoff);
            if (backoff < 256) backoff <<= 1;
        }
        if (!go) break;

        const unsigned long long e = a.tiles[T & a.tile_mask];
        uint32_t s = (uint32_t)(e >> 32) & 0xfffffu;
        uint64_t k = (uint32_t)e;
        if ((e >> 52) != ((T >> a.tile_bits) & 0xfffull)) {
            // the ring wrapped over this entry before it was read (only when
            // many later tiles finished meanwhile): find the request that owns
            // position T from the device copies of the in-flight descriptors
            uint32_t found = 0xffffffffu;
            for (uint32_t i = lane; i <= a.slot_mask; i += 32) {
                const unsigned long long p0 = a.dslots[i].pos0, n = a.dslots[i].ntiles;
                const unsigned long long fin = ld_vol(&a.fin[i]);
                if (n && fin < n && T >= p0 && T < p0 + n) found = i;
            }
            for (int off = 16; off; off >>= 1) found = min(found, __shfl_xor_sync(0xffffffffu, found, off));
            if (found == 0xffffffffu) continue;  // cannot happen: its request is still in flight
            s = found;
            k = T - a.dslots[s].pos0;
        }
        const ReqDesc d = a.dslots[s].d;
        const unsigned long long nt = a.dslots[s].ntiles;
        const unsigned long long seq = a.dslots[s].seq;
        const unsigned long long t_first = __shfl_sync(0xffffffffu, gtimer(), 0);
        if (k == 0) a.t_start[s] = t_first;  // same value from every lane
        const int st = run_tile<true, true, true>(d, k, a.keys, a.max_keys, K, cur_sel, cur_gen, stage);
        if (st) *reinterpret_cast<volatile int*>(&a.status[s]) = st;
        // Publication: the warp barrier orders every lane's stores before
        // lane 0, lane 0's acq_rel increment releases them at GPU scope, the
        // last increment of a request acquires all of its tiles' stores, and
        // the system-scope release store hands them to the host.
        __syncwarp();
        unsigned long long f = 0;
        if (lane == 0) f = atom_add_acq_rel_gpu(&a.fin[s], 1ull) + 1;
        f = __shfl_sync(0xffffffffu, f, 0);
        if (f == nt) {
            const unsigned long long t_end = __shfl_sync(0xffffffffu, gtimer(), 0);
            if (lane == 0) {
                a.t_done[s] = t_end;
                a.t_disp[s] = a.dslots[s].t_disp;
                a.t_pub[s] = a.dslots[s].t_pub;
                st_release_sys(&a.done_seq[s], seq + 1);
                atomicAdd(&a.dev->done_count, 1ull);
            }
            __syncwarp();
        }
        if (lane == 0) atomicAdd(&a.dev->tile_done, 1ull);
        __syncwarp();
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
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_smem_bytes(1024));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch_smem_bytes(512));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(serve_kernel<kServeThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)serve_smem_bytes());
    return e;
}

const void* batch_kernel_fn(int threads) {
    if (threads == 1024) return reinterpret_cast<const void*>(batch_kernel<1024>);
    if (threads == 512) return reinterpret_cast<const void*>(batch_kernel<512>);
    return nullptr;
}

cudaError_t launch_serve_reset(ServeDev* dev, unsigned long long* mbox, int ctas, cudaStream_t s) {
    serve_reset_kernel<<<1, 256, 0, s>>>(dev, mbox, ctas);
    return cudaGetLastError();
}

cudaError_t launch_serve(const ServeArgs& a, int threads, int grid, cudaStream_t s) {
    if (threads != kServeThreads) return cudaErrorInvalidValue;
    serve_kernel<kServeThreads><<<grid, kServeThreads, serve_smem_bytes(), s>>>(a);
    return cudaGetLastError();
}

// The empty service as a plain launch: warp w (of the whole grid) copies
// units w, w + warps, ...
__global__ void __launch_bounds__(1024) copy_kernel(const uint4* src, uint4* dst, uint64_t units,
                                                    uint32_t unit_blocks) {
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < units; w += warps) {
        const uint64_t b1 = (w + 1) * unit_blocks;
        for (uint64_t b = w * unit_blocks + (threadIdx.x & 31); b < b1; b += 32) dst[b] = src[b];
    }
}

cudaError_t launch_copy(const uint4* src, uint4* dst, uint64_t nblocks, uint32_t unit_blocks, int num_sms,
                        cudaStream_t s) {
    if (!unit_blocks || nblocks % unit_blocks) return cudaErrorInvalidValue;
    const uint64_t units = nblocks / unit_blocks;
    if (!units) return cudaSuccess;
    // 32 threads per unit: one CTA of up to 1024 threads, else CTAs of 1024
    // (at most 32 per SM; larger requests loop)
    const int threads = units * 32 <= 1024 ? (int)(units * 32) : 1024;
    const uint64_t ctas = (units * 32 + threads - 1) / threads;
    const int grid = (int)std::min<uint64_t>(ctas, (uint64_t)num_sms * 32);
    copy_kernel<<<grid, threads, 0, s>>>(src, dst, units, unit_blocks);
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& a, int threads, int grid, cudaStream_t s) {
    if (threads == 1024) batch_kernel<1024><<<grid, 1024, batch_smem_bytes(1024), s>>>(a);
    else if (threads == 512) batch_kernel<512><<<grid, 512, batch_smem_bytes(512), s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace kgpu
