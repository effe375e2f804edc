// Host-side AES constants for the GPU library: S-box, inverse S-box, the
// round lookup tables and the key schedules (FIPS-197 sections 5.1.1, 5.2 and
// 5.3.5).  Everything is derived at start-up from GF(2^8) arithmetic -- nothing
// is typed in.  The field inverse is taken from discrete logarithms to the
// generator {03}; the affine map is written in its rotate form
//   S(a) = b ^ rotl8(b,1) ^ rotl8(b,2) ^ rotl8(b,3) ^ rotl8(b,4) ^ 0x63,  b = inv(a).
//
// Word convention used by the kernels: a 16-byte block is four little-endian
// 32-bit words; word c is column c of the FIPS-197 state with row r in bits
// 8r..8r+7.  Round-key words use the same convention.
#pragma once
#include <cstdint>
#include <cstring>

namespace kgpu {
namespace host {

inline uint8_t xt(uint8_t a) { return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1b : 0)); }

struct Field {
    uint8_t exp[512];
    uint8_t log[256];
    uint8_t sbox[256], isbox[256];
    Field() {
        uint8_t g = 1;
        for (int i = 0; i < 255; i++) {
            exp[i] = g;
            exp[i + 255] = g;
            log[g] = (uint8_t)i;
            g = (uint8_t)(g ^ xt(g));  // g *= {03}
        }
        exp[510] = exp[0];
        exp[511] = exp[1];
        log[0] = 0;
        for (int a = 0; a < 256; a++) {
            uint8_t b = a ? exp[255 - log[a]] : 0;
            auto rl = [](uint8_t v, int k) { return (uint8_t)((v << k) | (v >> (8 - k))); };
            uint8_t s = (uint8_t)(b ^ rl(b, 1) ^ rl(b, 2) ^ rl(b, 3) ^ rl(b, 4) ^ 0x63);
            sbox[a] = s;
            isbox[s] = (uint8_t)a;
        }
    }
    uint8_t mul(uint8_t a, uint8_t b) const {
        if (!a || !b) return 0;
        return exp[log[a] + log[b]];
    }
};

inline const Field& field() {
    static const Field f;
    return f;
}

// Round-table words.  te0[x] is the MixColumns image of the column (S(x),0,0,0):
// bytes ({02}S, S, S, {03}S).  td0[x] likewise for InvMixColumns of InvS(x):
// bytes ({0e}I, {09}I, {0d}I, {0b}I).  Tables for rows 1..3 are byte rotations.
// sb4 / isb4 replicate S(x) / InvS(x) into all four bytes (final rounds).
struct Tables {
    uint32_t te0[256], td0[256], sb4[256], isb4[256];
};

inline void make_tables(Tables* t) {
    const Field& f = field();
    for (int x = 0; x < 256; x++) {
        uint8_t s = f.sbox[x], i = f.isbox[x];
        t->te0[x] = (uint32_t)f.mul(2, s) | (uint32_t)s << 8 | (uint32_t)s << 16 | (uint32_t)f.mul(3, s) << 24;
        t->td0[x] = (uint32_t)f.mul(14, i) | (uint32_t)f.mul(9, i) << 8 | (uint32_t)f.mul(13, i) << 16 |
                    (uint32_t)f.mul(11, i) << 24;
        t->sb4[x] = 0x01010101u * s;
        t->isb4[x] = 0x01010101u * i;
    }
}

inline uint32_t sub_word(uint32_t w) {
    const Field& f = field();
    return (uint32_t)f.sbox[w & 0xff] | (uint32_t)f.sbox[(w >> 8) & 0xff] << 8 |
           (uint32_t)f.sbox[(w >> 16) & 0xff] << 16 | (uint32_t)f.sbox[w >> 24] << 24;
}

inline uint32_t inv_mix_word(uint32_t w) {
    const Field& f = field();
    uint8_t a0 = w & 0xff, a1 = (w >> 8) & 0xff, a2 = (w >> 16) & 0xff, a3 = w >> 24;
    uint8_t b0 = f.mul(14, a0) ^ f.mul(11, a1) ^ f.mul(13, a2) ^ f.mul(9, a3);
    uint8_t b1 = f.mul(9, a0) ^ f.mul(14, a1) ^ f.mul(11, a2) ^ f.mul(13, a3);
    uint8_t b2 = f.mul(13, a0) ^ f.mul(9, a1) ^ f.mul(14, a2) ^ f.mul(11, a3);
    uint8_t b3 = f.mul(11, a0) ^ f.mul(13, a1) ^ f.mul(9, a2) ^ f.mul(14, a3);
    return (uint32_t)b0 | (uint32_t)b1 << 8 | (uint32_t)b2 << 16 | (uint32_t)b3 << 24;
}

// FIPS-197 5.2 KeyExpansion into little-endian column words.  Returns Nr, or 0
// for an unsupported key length.  enc must hold 4*(Nr+1) <= 60 words.
inline int expand_key(const uint8_t* key, size_t len, uint32_t* enc) {
    int nk = (len == 16) ? 4 : (len == 24) ? 6 : (len == 32) ? 8 : 0;
    if (!nk) return 0;
    int nr = nk + 6;
    for (int i = 0; i < nk; i++) {
        enc[i] = (uint32_t)key[4 * i] | (uint32_t)key[4 * i + 1] << 8 | (uint32_t)key[4 * i + 2] << 16 |
                 (uint32_t)key[4 * i + 3] << 24;
    }
    uint8_t rc = 1;
    for (int i = nk; i < 4 * (nr + 1); i++) {
        uint32_t t = enc[i - 1];
        if (i % nk == 0) {
            t = sub_word((t >> 8) | (t << 24)) ^ rc;  // RotWord, SubWord, Rcon
            rc = xt(rc);
        } else if (nk == 8 && i % nk == 4) {
            t = sub_word(t);
        }
        enc[i] = enc[i - nk] ^ t;
    }
    return nr;
}

// FIPS-197 5.3.5 equivalent inverse cipher schedule: round keys in reverse
// order, InvMixColumns applied to those of rounds 1..Nr-1.
inline void decrypt_schedule(const uint32_t* enc, int nr, uint32_t* dec) {
    for (int r = 0; r <= nr; r++) {
        for (int c = 0; c < 4; c++) {
            uint32_t w = enc[4 * (nr - r) + c];
            dec[4 * r + c] = (r == 0 || r == nr) ? w : inv_mix_word(w);
        }
    }
}

}  // namespace host
}  // namespace kgpu

namespace kgpu {
namespace host {

// Unified-kernel ("u-frame") copy of a schedule: see DevKey in
// kgpu_internal.h.  perm_dec = true stores each round's words in the state
// order (0, 3, 2, 1) used for the inverse cipher.
inline void to_uframe(const uint32_t* sched, int nr, bool perm_dec, uint32_t* out) {
    for (int i = 0; i < 60; i++) out[i] = 0;
    for (int r = 0; r <= nr; r++) {
        for (int c = 0; c < 4; c++) {
            uint32_t w = sched[4 * r + (perm_dec ? (4 - c) % 4 : c)];
            if (r == 0) {
                out[c] = w;
            } else if (r == nr) {
                out[56 + c] = w;
            } else {
                out[4 * r + c] = (w >> 16) | (w << 16);
            }
        }
    }
}

}  // namespace host
}  // namespace kgpu
