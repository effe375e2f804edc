// Bitsliced AES (FIPS-197) on the ALU: the comparison variant of the table
// kernels.  Each thread enciphers 32 blocks at once, held as 128 bit-planes
// (plane 8p+b holds bit b of state byte p of all 32 blocks, one block per bit
// position), so SubBytes is a Boolean circuit evaluated on 32-bit words
// (sbox_circuit.cuh), ShiftRows is a renaming of planes and MixColumns and
// AddRoundKey are XORs of planes.  No table lookups: the work runs on the ALU
// pipe (LOP3), not the shared-memory path the table kernels are bound by.
//
// Occupancy: the state alone is 128 registers; left to itself the compiler
// uses 254 and the SM holds 8 warps, too few to hide the ALU's fixed latencies
// and the instruction fetch over a ~2,500-instruction round.  At 384 threads
// per CTA it fits 168 registers and spills a few hundred bytes to local
// memory -- traffic on the LSU path, which this kernel otherwise leaves idle
// -- and 12 warps run 18-20% faster (measured: 256 -> 167 GB/s,
// 384 -> 197-201, 512 with 128 registers -> 130).
//
// Data layout: a warp owns a span of 1024 consecutive blocks; lane l takes
// blocks l, l+32, ..., l+992, so each of its 32 loads and stores is one
// coalesced 512-byte warp access.  A 32x32 bit transpose per state word turns
// the 32 loaded blocks into planes and back.
//
// XTS (IEEE 1619): the data-unit tweaks E_K2(unit) come from a bitsliced
// pre-pass (bs_tweak_kernel) into a caller-side buffer; the main kernel
// multiplies them by alpha^j in closed form as it walks each lane's blocks
// (j advances by 32 between a lane's consecutive blocks).
#include <cuda_runtime.h>

#include "aes_device.cuh"
#include "kgpu_bitslice.h"
#include "sbox_circuit.cuh"

namespace kgpu {

using namespace dev;

namespace {

constexpr int kBsSpan = 1024;  // blocks per warp iteration (32 lanes x 32 blocks)

// In-place 32x32 bit transpose: afterwards bit t of a[k] is the former bit k of
// a[t].  Five rounds of block swaps (16, 8, 4, 2, 1); the 16- and 8-bit rounds
// are byte permutes.
__device__ __forceinline__ void transpose32(uint32_t* a) {
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t lo = a[i], hi = a[i + 16];
        a[i] = __byte_perm(lo, hi, 0x5410);
        a[i + 16] = __byte_perm(lo, hi, 0x7632);
    }
#pragma unroll
    for (int g = 0; g < 32; g += 16) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint32_t lo = a[g + i], hi = a[g + i + 8];
            a[g + i] = __byte_perm(lo, hi, 0x6240);
            a[g + i + 8] = __byte_perm(lo, hi, 0x7351);
        }
    }
#pragma unroll
    for (int s = 4; s >= 1; s >>= 1) {
        const uint32_t m = s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            if (i & s) continue;
            const uint32_t t = ((a[i] >> s) ^ a[i + s]) & m;
            a[i + s] ^= t;
            a[i] ^= t << s;
        }
    }
}

// One S-box circuit, called 16 times a round rather than inlined 16 times: the
// round body shrinks by ~1,500 instructions, which eases the instruction fetch
// stalls that top this kernel's profile (measured +4%, for 16 argument moves
// per call).
struct Byte8 {
    uint32_t x0, x1, x2, x3, x4, x5, x6, x7;
};

__device__ __noinline__ Byte8 sbox_call(Byte8 b) {
    sbox_circuit(b.x0, b.x1, b.x2, b.x3, b.x4, b.x5, b.x6, b.x7);
    return b;
}

__device__ __forceinline__ void sub_bytes(uint32_t (&S)[128]) {
#pragma unroll
    for (int p = 0; p < 16; p++) {
        Byte8 b{S[8 * p + 0], S[8 * p + 1], S[8 * p + 2], S[8 * p + 3],
                S[8 * p + 4], S[8 * p + 5], S[8 * p + 6], S[8 * p + 7]};
        b = sbox_call(b);
        S[8 * p + 0] = b.x0;
        S[8 * p + 1] = b.x1;
        S[8 * p + 2] = b.x2;
        S[8 * p + 3] = b.x3;
        S[8 * p + 4] = b.x4;
        S[8 * p + 5] = b.x5;
        S[8 * p + 6] = b.x6;
        S[8 * p + 7] = b.x7;
    }
}

// ShiftRows, then MixColumns (when MIX), then AddRoundKey with the plane masks
// k[0..127] (each 0 or ~0).  Output byte r + 4c takes input byte
// r + 4((c + r) mod 4); per column, with a_r those four bytes,
//   out_r = a_r ^ t ^ xtime(a_r ^ a_{r+1}),  t = a_0 ^ a_1 ^ a_2 ^ a_3,
// which is 2a_r ^ 3a_{r+1} ^ a_{r+2} ^ a_{r+3}.  xtime on planes: bit b takes
// bit b-1, and bits 1, 3, 4 also take bit 7 (x^8 = x^4 + x^3 + x + 1).
template <bool MIX>
__device__ __forceinline__ void shift_mix_key(uint32_t (&S)[128], const uint32_t* k) {
    uint32_t N[128];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int src[4] = {0 + 4 * ((c + 0) & 3), 1 + 4 * ((c + 1) & 3), 2 + 4 * ((c + 2) & 3),
                            3 + 4 * ((c + 3) & 3)};
        if (!MIX) {
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int b = 0; b < 8; b++) N[8 * (r + 4 * c) + b] = S[8 * src[r] + b] ^ k[8 * (r + 4 * c) + b];
            continue;
        }
        uint32_t t[8];
#pragma unroll
        for (int b = 0; b < 8; b++)
            t[b] = S[8 * src[0] + b] ^ S[8 * src[1] + b] ^ S[8 * src[2] + b] ^ S[8 * src[3] + b];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            uint32_t u[8];
#pragma unroll
            for (int b = 0; b < 8; b++) u[b] = S[8 * src[r] + b] ^ S[8 * src[(r + 1) & 3] + b];
            uint32_t x2[8];
            x2[0] = u[7];
            x2[1] = u[0] ^ u[7];
            x2[2] = u[1];
            x2[3] = u[2] ^ u[7];
            x2[4] = u[3] ^ u[7];
            x2[5] = u[4];
            x2[6] = u[5];
            x2[7] = u[6];
#pragma unroll
            for (int b = 0; b < 8; b++)
                N[8 * (r + 4 * c) + b] = S[8 * src[r] + b] ^ t[b] ^ x2[b] ^ k[8 * (r + 4 * c) + b];
        }
    }
#pragma unroll
    for (int i = 0; i < 128; i++) S[i] = N[i];
}

// The forward cipher on planes; km holds (NR + 1) x 128 round-key masks in
// shared memory.  The round loop is not unrolled: one round is ~2,000
// instructions, and 14 unrolled rounds would not fit the instruction cache.
// The final round (no MixColumns) stays inside the loop behind a uniform
// branch: as a separate copy after the loop, its state assignment differed
// from the loop's and the kernel spilled ~0.9 KB per thread.
template <int NR>
__device__ __forceinline__ void bs_encrypt(uint32_t (&S)[128], const uint32_t* km) {
#pragma unroll
    for (int i = 0; i < 128; i++) S[i] ^= km[i];
#pragma unroll 1
    for (int r = 1; r <= NR; r++) {
        sub_bytes(S);
        if (r < NR)
            shift_mix_key<true>(S, km + 128 * r);
        else
            shift_mix_key<false>(S, km + 128 * r);
    }
}

template <int NR>
__device__ __forceinline__ void load_masks(uint32_t* km, const uint32_t* rkm) {
    for (int i = threadIdx.x; i < 128 * (NR + 1); i += blockDim.x) km[i] = rkm[i];
    __syncthreads();
}

// XTS tweak of one lane's current block: unit s (relative to the call's first
// unit), position j in the unit, value E_K2(unit) * alpha^j.
struct TweakWalk {
    uint32_t t0, t1, t2, t3;
    uint64_t s;
    uint32_t j;

    __device__ __forceinline__ void load(const uint4* tw) {
        const uint4 v = tw[s];
        t0 = v.x;
        t1 = v.y;
        t2 = v.z;
        t3 = v.w;
        gf128_mul_xpow(t0, t1, t2, t3, j);
    }
    __device__ __forceinline__ void start(const uint4* tw, uint64_t n, uint32_t bps) {
        s = n / bps;
        j = (uint32_t)(n - s * bps);
        load(tw);
    }
    // to the lane's next block, 32 blocks further on
    __device__ __forceinline__ void step(const uint4* tw, uint32_t bps) {
        j += 32;
        if (j < bps) {
            gf128_mul_x32(t0, t1, t2, t3);
            return;
        }
        s += j / bps;
        j %= bps;
        load(tw);
    }
};

template <int NR, bool TWEAK>
__global__ void __launch_bounds__(kBsThreads, 1) bs_kernel(const __grid_constant__ BsParams p) {
    __shared__ uint32_t km[128 * (NR + 1)];
    load_masks<NR>(km, p.rkm);
    const uint32_t lane = lane_id();
    const uint64_t spans = (p.nblocks + kBsSpan - 1) / kBsSpan;
    for (uint64_t sp = interleaved_warp(); sp < spans; sp += total_warps()) {
        const uint64_t base = sp * kBsSpan + lane;
        uint32_t S[128];
        TweakWalk w;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const uint64_t n = base + 32u * i;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (n < p.nblocks) {
                v = p.src[n];
                if (TWEAK) {
                    if (i == 0) w.start(p.tw, n, p.bps);
                    else w.step(p.tw, p.bps);
                    v.x ^= w.t0;
                    v.y ^= w.t1;
                    v.z ^= w.t2;
                    v.w ^= w.t3;
                }
            }
            S[i] = v.x;
            S[32 + i] = v.y;
            S[64 + i] = v.z;
            S[96 + i] = v.w;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) transpose32(S + 32 * q);
        bs_encrypt<NR>(S, km);
#pragma unroll
        for (int q = 0; q < 4; q++) transpose32(S + 32 * q);
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const uint64_t n = base + 32u * i;
            if (n < p.nblocks) {
                uint4 v = make_uint4(S[i], S[32 + i], S[64 + i], S[96 + i]);
                if (TWEAK) {
                    if (i == 0) w.start(p.tw, n, p.bps);
                    else w.step(p.tw, p.bps);
                    v.x ^= w.t0;
                    v.y ^= w.t1;
                    v.z ^= w.t2;
                    v.w ^= w.t3;
                }
                p.dst[n] = v;
            }
        }
    }
}

// XTS pre-pass: tw[u] = E_K2(LE128(first_sector + u)) for u < units, with the
// tweak key's masks in p.rkm.
template <int NR>
__global__ void __launch_bounds__(kBsThreads, 1) bs_tweak_kernel(const __grid_constant__ BsParams p) {
    __shared__ uint32_t km[128 * (NR + 1)];
    load_masks<NR>(km, p.rkm);
    const uint32_t lane = lane_id();
    const uint64_t spans = (p.units + kBsSpan - 1) / kBsSpan;
    for (uint64_t sp = interleaved_warp(); sp < spans; sp += total_warps()) {
        const uint64_t base = sp * kBsSpan + lane;
        uint32_t S[128];
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const uint64_t sector = p.first_sector + base + 32u * i;  // 128-bit little-endian, high half zero
            S[i] = (uint32_t)sector;
            S[32 + i] = (uint32_t)(sector >> 32);
            S[64 + i] = 0;
            S[96 + i] = 0;
        }
#pragma unroll
        for (int q = 0; q < 4; q++) transpose32(S + 32 * q);
        bs_encrypt<NR>(S, km);
#pragma unroll
        for (int q = 0; q < 4; q++) transpose32(S + 32 * q);
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const uint64_t u = base + 32u * i;
            if (u < p.units) p.tw[u] = make_uint4(S[i], S[32 + i], S[64 + i], S[96 + i]);
        }
    }
}

template <class F>
F pick(int nr, F f10, F f12, F f14) {
    return nr == 10 ? f10 : nr == 12 ? f12 : nr == 14 ? f14 : nullptr;
}

}  // namespace

cudaError_t launch_bitsliced(const BsParams& p, int nr, bool tweak, int num_sms, cudaStream_t s) {
    using Fn = void (*)(BsParams);
    Fn fn = tweak ? pick<Fn>(nr, bs_kernel<10, true>, bs_kernel<12, true>, bs_kernel<14, true>)
                  : pick<Fn>(nr, bs_kernel<10, false>, bs_kernel<12, false>, bs_kernel<14, false>);
    if (!fn) return cudaErrorInvalidValue;
    const uint64_t spans = (p.nblocks + kBsSpan - 1) / kBsSpan;
    const uint64_t ctas = (spans + kBsThreads / 32 - 1) / (kBsThreads / 32);
    const int grid = (int)(ctas < (uint64_t)num_sms ? (ctas ? ctas : 1) : num_sms);
    fn<<<grid, kBsThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_bitsliced_tweaks(const BsParams& p, int nr, int num_sms, cudaStream_t s) {
    using Fn = void (*)(BsParams);
    Fn fn = pick<Fn>(nr, bs_tweak_kernel<10>, bs_tweak_kernel<12>, bs_tweak_kernel<14>);
    if (!fn) return cudaErrorInvalidValue;
    const uint64_t spans = (p.units + kBsSpan - 1) / kBsSpan;
    const uint64_t ctas = (spans + kBsThreads / 32 - 1) / (kBsThreads / 32);
    const int grid = (int)(ctas < (uint64_t)num_sms ? (ctas ? ctas : 1) : num_sms);
    fn<<<grid, kBsThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace kgpu
