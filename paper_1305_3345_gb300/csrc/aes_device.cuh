// Device-side AES building blocks for sm_103a (FIPS-197 Cipher and the
// equivalent inverse cipher of section 5.3.5, written as 32-bit table rounds),
// plus GF(2^128) tweak arithmetic for XTS (IEEE 1619 section 5.2).
//
// Shared-memory table layout.  Every lookup is a random byte index, so tables
// are replicated once per lane: lane l only ever reads column l of a row, which
// always sits in bank l -- every warp-wide lookup is bank-conflict free.
//
//   region A  [  0K,  64K): 256 rows x 256 B, row x = T0[x] (32 copies) | T1[x] (32 copies)
//   region B  [ 64K, 128K): T2 | T3
//   region C  [128K, 192K): F[x] (32 copies) | E0[x] (32 copies)
//
// Byte address of table k, index x, lane l inside a region pair:
//   x*256 + (k&1)*128 + l*4 + (k>>1)*64K
// which one PRMT builds from the state word: the index byte goes to byte 1 and
// the lane offset (l*4 or l*4+128, both < 256) to byte 0.
//
// Encryption kernels put Te0..Te3 in A/B; decryption kernels put Td0..Td3 in
// A/B, the inverse S-box (replicated into 4 bytes) in C's first half and the
// forward Te0 in C's second half (for the XTS tweak, which is always an
// encryption).
#pragma once
#include <cstdint>

namespace kgpu {
namespace dev {

constexpr uint32_t kRegion = 65536;
constexpr int kMaxKeyWords = 60;

__device__ __forceinline__ uint32_t rotl8(uint32_t v) { return __byte_perm(v, v, 0x2103); }
__device__ __forceinline__ uint32_t rotl16(uint32_t v) { return __byte_perm(v, v, 0x1032); }
__device__ __forceinline__ uint32_t rotl24(uint32_t v) { return __byte_perm(v, v, 0x0321); }

template <int K>
__device__ __forceinline__ uint32_t rotl_bytes(uint32_t v) {
    if constexpr (K == 0) return v;
    else if constexpr (K == 1) return rotl8(v);
    else if constexpr (K == 2) return rotl16(v);
    else return rotl24(v);
}

// Shared-window address where a kernel's dynamic shared memory begins when the
// kernel declares no static shared memory: the per-CTA reserved system area
// (cudaDevAttrReservedSharedMemoryPerBlock, 1 KiB on sm_100/sm_103) comes
// first.  The library checks this at context creation and every kernel checks
// it again before touching shared memory; folding it into the load's
// immediate offset saves one add per lookup.
constexpr uint32_t kSmemBase = 1024;

// Shared address (relative to the table base) of byte P of state word s in a
// 256-B-row replicated table: one PRMT.  lo = lane*4 (first half of the row)
// or lane*4 + 128 (second half) in its byte 0, byte 1 zero, and optionally a
// region index in byte 2; the index byte lands in byte 1 and lo's bytes 0, 2
// and 3 pass through.
template <int P>
__device__ __forceinline__ uint32_t row_addr(uint32_t s, uint32_t lo) {
    return __byte_perm(s, lo, 0x7604u | (P << 4));
}

// 32-bit shared load at table offset a + OFF (OFF includes kSmemBase and the
// region), as a single LDS with an immediate offset.
template <uint32_t OFF>
__device__ __forceinline__ uint32_t lds_tab(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
    return v;
}

// Four replicated round tables in regions A/B.
struct Rep4 {
    uint32_t lo0, lo1;
    template <int K, int P>
    __device__ __forceinline__ uint32_t t(uint32_t s) const {
        return lds_tab<kSmemBase + (K >> 1) * kRegion>(row_addr<P>(s, (K & 1) ? lo1 : lo0));
    }
};

// One replicated table (row 0) in region REGION, half selected by lo; rows
// 1..3 by byte rotation.
template <int REGION>
struct Rep1 {
    uint32_t lo;
    template <int K, int P>
    __device__ __forceinline__ uint32_t t(uint32_t s) const {
        return rotl_bytes<K>(lds_tab<kSmemBase + REGION * kRegion>(row_addr<P>(s, lo)));
    }
};

// True when this CTA's dynamic shared memory starts where the tables assume.
__device__ __forceinline__ bool smem_layout_ok(const void* dyn_smem) {
    return (uint32_t)__cvta_generic_to_shared(dyn_smem) == kSmemBase;
}

// Byte r of the result from v_r (r = 0..3).
__device__ __forceinline__ uint32_t merge_bytes(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    return __byte_perm(__byte_perm(v0, v1, 0x3250), __byte_perm(v2, v3, 0x7210), 0x7610);
}

// Round keys held in kernel-parameter space; indices are compile-time after
// unrolling, so each word is a constant-bank operand.
struct ParamKey {
    const uint32_t* rk;
    __device__ __forceinline__ uint32_t w(int i) const { return rk[i]; }
};

// FIPS-197 Cipher on the column words (s0..s3).  Rounds 1..NR-1 are
// SubBytes+ShiftRows+MixColumns as four table lookups per column; the final
// round takes S(x) from the byte of table (r+3)%4 that holds it unscaled.
template <int NR, class Tab, class Key>
__device__ __forceinline__ void encrypt_block(uint32_t& s0, uint32_t& s1, uint32_t& s2, uint32_t& s3,
                                              const Tab& T, const Key& k) {
    s0 ^= k.w(0);
    s1 ^= k.w(1);
    s2 ^= k.w(2);
    s3 ^= k.w(3);
#pragma unroll
    for (int r = 1; r < NR; r++) {
        uint32_t t0 = T.template t<0, 0>(s0) ^ T.template t<1, 1>(s1) ^ T.template t<2, 2>(s2) ^
                      T.template t<3, 3>(s3) ^ k.w(4 * r + 0);
        uint32_t t1 = T.template t<0, 0>(s1) ^ T.template t<1, 1>(s2) ^ T.template t<2, 2>(s3) ^
                      T.template t<3, 3>(s0) ^ k.w(4 * r + 1);
        uint32_t t2 = T.template t<0, 0>(s2) ^ T.template t<1, 1>(s3) ^ T.template t<2, 2>(s0) ^
                      T.template t<3, 3>(s1) ^ k.w(4 * r + 2);
        uint32_t t3 = T.template t<0, 0>(s3) ^ T.template t<1, 1>(s0) ^ T.template t<2, 2>(s1) ^
                      T.template t<3, 3>(s2) ^ k.w(4 * r + 3);
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    uint32_t o0 = merge_bytes(T.template t<3, 0>(s0), T.template t<0, 1>(s1), T.template t<1, 2>(s2),
                              T.template t<2, 3>(s3)) ^ k.w(4 * NR + 0);
    uint32_t o1 = merge_bytes(T.template t<3, 0>(s1), T.template t<0, 1>(s2), T.template t<1, 2>(s3),
                              T.template t<2, 3>(s0)) ^ k.w(4 * NR + 1);
    uint32_t o2 = merge_bytes(T.template t<3, 0>(s2), T.template t<0, 1>(s3), T.template t<1, 2>(s0),
                              T.template t<2, 3>(s1)) ^ k.w(4 * NR + 2);
    uint32_t o3 = merge_bytes(T.template t<3, 0>(s3), T.template t<0, 1>(s0), T.template t<1, 2>(s1),
                              T.template t<2, 3>(s2)) ^ k.w(4 * NR + 3);
    s0 = o0;
    s1 = o1;
    s2 = o2;
    s3 = o3;
}

// FIPS-197 5.3.5 equivalent inverse cipher with the InvMixColumns-adjusted
// schedule: InvShiftRows takes row r of output column c from column c - r.
// IS is the replicated inverse S-box (InvS(x) in all four bytes), same layout.
template <int NR, class Tab, class ISTab, class Key>
__device__ __forceinline__ void decrypt_block(uint32_t& s0, uint32_t& s1, uint32_t& s2, uint32_t& s3,
                                              const Tab& T, const ISTab& IS, const Key& k) {
    s0 ^= k.w(0);
    s1 ^= k.w(1);
    s2 ^= k.w(2);
    s3 ^= k.w(3);
#pragma unroll
    for (int r = 1; r < NR; r++) {
        uint32_t t0 = T.template t<0, 0>(s0) ^ T.template t<1, 1>(s3) ^ T.template t<2, 2>(s2) ^
                      T.template t<3, 3>(s1) ^ k.w(4 * r + 0);
        uint32_t t1 = T.template t<0, 0>(s1) ^ T.template t<1, 1>(s0) ^ T.template t<2, 2>(s3) ^
                      T.template t<3, 3>(s2) ^ k.w(4 * r + 1);
        uint32_t t2 = T.template t<0, 0>(s2) ^ T.template t<1, 1>(s1) ^ T.template t<2, 2>(s0) ^
                      T.template t<3, 3>(s3) ^ k.w(4 * r + 2);
        uint32_t t3 = T.template t<0, 0>(s3) ^ T.template t<1, 1>(s2) ^ T.template t<2, 2>(s1) ^
                      T.template t<3, 3>(s0) ^ k.w(4 * r + 3);
        s0 = t0;
        s1 = t1;
        s2 = t2;
        s3 = t3;
    }
    uint32_t o0 = merge_bytes(IS.template t<0, 0>(s0), IS.template t<0, 1>(s3), IS.template t<0, 2>(s2), IS.template t<0, 3>(s1)) ^ k.w(4 * NR + 0);
    uint32_t o1 = merge_bytes(IS.template t<0, 0>(s1), IS.template t<0, 1>(s0), IS.template t<0, 2>(s3), IS.template t<0, 3>(s2)) ^ k.w(4 * NR + 1);
    uint32_t o2 = merge_bytes(IS.template t<0, 0>(s2), IS.template t<0, 1>(s1), IS.template t<0, 2>(s0), IS.template t<0, 3>(s3)) ^ k.w(4 * NR + 2);
    uint32_t o3 = merge_bytes(IS.template t<0, 0>(s3), IS.template t<0, 1>(s2), IS.template t<0, 2>(s1), IS.template t<0, 3>(s0)) ^ k.w(4 * NR + 3);
    s0 = o0;
    s1 = o1;
    s2 = o2;
    s3 = o3;
}

// ---------------------------------------------------------------------------
// GF(2^128) tweak arithmetic (IEEE 1619 5.2).  The tweak is the 16-byte block
// read as a little-endian 128-bit polynomial, i.e. the four words w0..w3 with
// w0 least significant; alpha = x and the modulus is x^128 + x^7 + x^2 + x + 1.
// ---------------------------------------------------------------------------

// T <- T * x^k for 0 <= k <= 32, in closed form: shift the 128-bit value left by
// k and fold the (at most 32) bits that leave the top back in as h*(x^7+x^2+x+1),
// which has degree < 39 and so never needs a second reduction.
__device__ __forceinline__ void gf128_mul_xk(uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3, uint32_t k) {
    uint32_t h = __funnelshift_lc(w3, 0u, k);
    w3 = __funnelshift_lc(w2, w3, k);
    w2 = __funnelshift_lc(w1, w2, k);
    w1 = __funnelshift_lc(w0, w1, k);
    w0 = __funnelshift_lc(0u, w0, k);
    w0 ^= h ^ (h << 1) ^ (h << 2) ^ (h << 7);
    w1 ^= (h >> 31) ^ (h >> 30) ^ (h >> 25);
}

// T <- T * x^32: the fixed step between the blocks one lane handles in a warp
// that walks 32 consecutive blocks per iteration.
__device__ __forceinline__ void gf128_mul_x32(uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3) {
    uint32_t h = w3;
    w3 = w2;
    w2 = w1;
    w1 = w0 ^ (h >> 31) ^ (h >> 30) ^ (h >> 25);
    w0 = h ^ (h << 1) ^ (h << 2) ^ (h << 7);
}

// T <- T * x^j for any j (only used once per warp, at the start of its range).
__device__ __forceinline__ void gf128_mul_xpow(uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3, uint32_t j) {
    while (j > 32) {
        gf128_mul_x32(w0, w1, w2, w3);
        j -= 32;
    }
    gf128_mul_xk(w0, w1, w2, w3, j);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Warp index interleaved across CTAs (warp-in-CTA major), so that when a
// range of work is split over warps, each SM receives an equal share.
__device__ __forceinline__ uint32_t interleaved_warp() {
    return (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
}

__device__ __forceinline__ uint32_t total_warps() { return (blockDim.x >> 5) * gridDim.x; }

// ---------------------------------------------------------------------------
// Unified two-table cipher (batched and serving kernels, which must serve any
// mode, direction and key size from one CTA).
//
// Layout: region A = Te0 | Te1, region B = Td0 | Td1, region C = S4 | IS4
// (S(x) / InvS(x) in all four bytes), each replicated per lane as above.  The
// region index travels in byte 2 of the lane-offset registers, so one code path
// serves both directions.  Rows 2 and 3 are rows 0 and 1 rotated by 16 bits,
// and rotation commutes with xor, so per column
//     T2[c] ^ T3[d] ^ k  =  rotl16(T0[c] ^ T1[d] ^ rotr16(k))
// -- one PRMT, with rotr16(k) prepared on the host (u-frame key layout).
// The inverse cipher is run on the state permuted to (s0, s3, s2, s1): in that
// order InvShiftRows has exactly ShiftRows' shape, so the round code is shared.
// ---------------------------------------------------------------------------

// Lane-offset registers of the unified layout for one direction.
struct UniLanes {
    uint32_t r0;  // lane*4 | region << 16: row 0 table (Te0 or Td0)
    uint32_t r1;  // r0 + 128: row 1 table (Te1 or Td1)
    uint32_t f;   // lane*4 (+128 for InvS) | 2 << 16: final-round S-box
};

__device__ __forceinline__ UniLanes uni_lanes(uint32_t lane, int dir) {
    uint32_t base = lane * 4u | (uint32_t)dir << 16;
    return UniLanes{base, base + 128u, (lane * 4u + (dir ? 128u : 0u)) | (2u << 16)};
}

__device__ __forceinline__ uint32_t uni_col(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t kr,
                                            const UniLanes& L) {
    uint32_t hi = lds_tab<kSmemBase>(row_addr<2>(c, L.r0)) ^ lds_tab<kSmemBase>(row_addr<3>(d, L.r1)) ^ kr;
    return lds_tab<kSmemBase>(row_addr<0>(a, L.r0)) ^ lds_tab<kSmemBase>(row_addr<1>(b, L.r1)) ^ rotl16(hi);
}

// Round key r (16 bytes, four words) from a 16-byte-aligned key slot in
// shared memory: one broadcast LDS.128.
__device__ __forceinline__ uint4 round_key(uint32_t slot_saddr, int r) {
    uint4 k;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(k.x), "=r"(k.y), "=r"(k.z), "=r"(k.w)
                 : "r"(slot_saddr + 16u * (uint32_t)r));
    return k;
}

// One block through the cipher of the unified layout (u-frame state and key).
// The round count is a run-time value and the rounds are a real loop with the
// round key read from shared memory: the body is one round, which keeps the
// kernels that serve every mode small enough to stay in the instruction cache.
__device__ __forceinline__ void cipher_u(uint32_t& u0, uint32_t& u1, uint32_t& u2, uint32_t& u3,
                                         uint32_t key_saddr, int nr, const UniLanes& L) {
    uint4 k = round_key(key_saddr, 0);
    u0 ^= k.x;
    u1 ^= k.y;
    u2 ^= k.z;
    u3 ^= k.w;
#pragma unroll 1
    for (int r = 1; r < nr; r++) {
        k = round_key(key_saddr, r);
        const uint32_t t0 = uni_col(u0, u1, u2, u3, k.x, L);
        const uint32_t t1 = uni_col(u1, u2, u3, u0, k.y, L);
        const uint32_t t2 = uni_col(u2, u3, u0, u1, k.z, L);
        const uint32_t t3 = uni_col(u3, u0, u1, u2, k.w, L);
        u0 = t0;
        u1 = t1;
        u2 = t2;
        u3 = t3;
    }
    k = round_key(key_saddr, 14);  // the final round key sits in words 56..59
#define KGPU_FIN(P, x) lds_tab<kSmemBase>(row_addr<P>(x, L.f))
    const uint32_t o0 = merge_bytes(KGPU_FIN(0, u0), KGPU_FIN(1, u1), KGPU_FIN(2, u2), KGPU_FIN(3, u3)) ^ k.x;
    const uint32_t o1 = merge_bytes(KGPU_FIN(0, u1), KGPU_FIN(1, u2), KGPU_FIN(2, u3), KGPU_FIN(3, u0)) ^ k.y;
    const uint32_t o2 = merge_bytes(KGPU_FIN(0, u2), KGPU_FIN(1, u3), KGPU_FIN(2, u0), KGPU_FIN(3, u1)) ^ k.z;
    const uint32_t o3 = merge_bytes(KGPU_FIN(0, u3), KGPU_FIN(1, u0), KGPU_FIN(2, u1), KGPU_FIN(3, u2)) ^ k.w;
#undef KGPU_FIN
    u0 = o0;
    u1 = o1;
    u2 = o2;
    u3 = o3;
}

// Block in natural column order through the unified cipher in direction dir.
__device__ __forceinline__ void cipher_block(uint4& v, uint32_t key_saddr, int nr, const UniLanes& L, int dir) {
    if (dir) {
        uint32_t t = v.y;
        v.y = v.w;
        v.w = t;
    }
    cipher_u(v.x, v.y, v.z, v.w, key_saddr, nr, L);
    if (dir) {
        uint32_t t = v.y;
        v.y = v.w;
        v.w = t;
    }
}

}  // namespace dev
}  // namespace kgpu
