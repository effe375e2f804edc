/*
 * aes_oracle.c -- TEST INFRASTRUCTURE, NOT THE PRODUCT.
 *
 * A plain, slow, obviously-correct CPU restatement of what the GPU page-crypto
 * service computes.  Only the test-suite, the smoke check and the bench's CPU
 * baseline leg may load it; the CUDA library never links or calls it, and it
 * shares no code, table or helper with the CUDA library.
 *
 * What it follows:
 *  - The paper's GPU AES service (section 3.3, "Example: A GPU AES
 *    Implementation") runs AES in ECB mode over page-sized buffers; the paper
 *    motivates per-page encryption for encrypted file systems there.  The paper
 *    does not restate AES itself, so the cipher below is written from its
 *    defining standard, FIPS-197 (sections named per function).
 *  - The page modes come from their standards: XTS from IEEE 1619-2007 section 5
 *    (= NIST SP 800-38E), CBC from NIST SP 800-38A section 6.2.
 *
 * Everything is byte-oriented exactly as the standards state it: the state is a
 * 4x4 byte array s[r][c], SubBytes uses an S-box computed at start-up from the
 * GF(2^8) inverse and the affine map (never typed in), MixColumns multiplies in
 * GF(2^8) by shift-and-xor, and the XTS tweak is advanced by sequential
 * multiplication by alpha on its 16-byte little-endian form.  No T-tables, no
 * word tricks, no closed-form tweak powers.
 *
 * Parallelism: independent data units / pages are spread over POSIX threads;
 * each unit is processed by the sequential definition.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-22)

/* ---------------------------------------------------------------------------
 * GF(2^8) with the AES modulus m(x) = x^8 + x^4 + x^3 + x + 1 (FIPS-197 4.2).
 * ------------------------------------------------------------------------- */

/* FIPS-197 4.2.1: multiplication by x, reducing by m(x) when bit 7 overflows. */
static uint8_t xtime(uint8_t a) {
    uint8_t hi = (uint8_t)(a & 0x80);
    uint8_t r = (uint8_t)(a << 1);
    if (hi) r ^= 0x1b;
    return r;
}

/* FIPS-197 4.2: a*b as a sum of a*x^i over the set bits i of b. */
uint8_t oracle_gf_mul(uint8_t a, uint8_t b) {
    uint8_t acc = 0;
    uint8_t p = a; /* a * x^i */
    for (int i = 0; i < 8; i++) {
        if (b & (1u << i)) acc ^= p;
        p = xtime(p);
    }
    return acc;
}

/* FIPS-197 5.1.1: multiplicative inverse in GF(2^8), with 0 mapped to 0.
 * Found by exhaustive search, the most literal reading of the definition. */
uint8_t oracle_gf_inv(uint8_t a) {
    if (a == 0) return 0;
    for (int b = 1; b < 256; b++)
        if (oracle_gf_mul(a, (uint8_t)b) == 1) return (uint8_t)b;
    return 0; /* unreachable: every nonzero element has an inverse */
}

static uint8_t SBOX[256];
static uint8_t INV_SBOX[256];
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

/* FIPS-197 5.1.1: S(a) = affine map of inv(a): bit i of the result is
 *   b_i ^ b_{(i+4) mod 8} ^ b_{(i+5) mod 8} ^ b_{(i+6) mod 8} ^ b_{(i+7) mod 8} ^ c_i
 * with c = 0x63. InvS is the inverse permutation of S. */
static void build_sbox(void) {
    for (int a = 0; a < 256; a++) {
        uint8_t b = oracle_gf_inv((uint8_t)a);
        uint8_t s = 0;
        for (int i = 0; i < 8; i++) {
            int bit = ((b >> i) & 1) ^ ((b >> ((i + 4) % 8)) & 1) ^ ((b >> ((i + 5) % 8)) & 1) ^
                      ((b >> ((i + 6) % 8)) & 1) ^ ((b >> ((i + 7) % 8)) & 1) ^ ((0x63 >> i) & 1);
            s |= (uint8_t)(bit << i);
        }
        SBOX[a] = s;
    }
    for (int a = 0; a < 256; a++) INV_SBOX[SBOX[a]] = (uint8_t)a;
}

static void init_once(void) { pthread_once(&g_once, build_sbox); }

void oracle_sbox(uint8_t out[256]) { init_once(); memcpy(out, SBOX, 256); }
void oracle_inv_sbox(uint8_t out[256]) { init_once(); memcpy(out, INV_SBOX, 256); }

/* ---------------------------------------------------------------------------
 * Key expansion (FIPS-197 5.2).
 * ------------------------------------------------------------------------- */

typedef struct {
    int nr;            /* number of rounds: 10, 12 or 14 */
    uint8_t w[60][4];  /* 4 * (nr + 1) words, each as 4 bytes */
} ExpandedKey;

/* key_len in bytes: 16, 24 or 32. Returns 0 or OR_EINVAL. */
static int key_expansion(const uint8_t *key, int key_len, ExpandedKey *ek) {
    init_once();
    int nk;
    if (key_len == 16) nk = 4;
    else if (key_len == 24) nk = 6;
    else if (key_len == 32) nk = 8;
    else return OR_EINVAL;
    int nr = nk + 6;
    ek->nr = nr;
    int total = 4 * (nr + 1);
    for (int i = 0; i < nk; i++)
        for (int k = 0; k < 4; k++) ek->w[i][k] = key[4 * i + k];
    uint8_t rcon = 0x01; /* Rcon[i/Nk] = [x^(i/Nk - 1), 0, 0, 0] */
    for (int i = nk; i < total; i++) {
        uint8_t temp[4];
        memcpy(temp, ek->w[i - 1], 4);
        if (i % nk == 0) {
            /* RotWord then SubWord, then xor Rcon */
            uint8_t t0 = temp[0];
            temp[0] = temp[1];
            temp[1] = temp[2];
            temp[2] = temp[3];
            temp[3] = t0;
            for (int k = 0; k < 4; k++) temp[k] = SBOX[temp[k]];
            temp[0] ^= rcon;
            rcon = xtime(rcon);
        } else if (nk > 6 && i % nk == 4) {
            for (int k = 0; k < 4; k++) temp[k] = SBOX[temp[k]];
        }
        for (int k = 0; k < 4; k++) ek->w[i][k] = (uint8_t)(ek->w[i - nk][k] ^ temp[k]);
    }
    return OR_OK;
}

/* Exposed for tests: writes 16 * (nr + 1) bytes, returns nr or OR_EINVAL. */
int oracle_key_expansion(const uint8_t *key, int key_len, uint8_t *out) {
    ExpandedKey ek;
    int rc = key_expansion(key, key_len, &ek);
    if (rc) return rc;
    memcpy(out, ek.w, (size_t)16 * (ek.nr + 1));
    return ek.nr;
}

/* ---------------------------------------------------------------------------
 * Cipher and InvCipher (FIPS-197 5.1 and 5.3) on the state s[r][c].
 * ------------------------------------------------------------------------- */

typedef uint8_t State[4][4];

static void load_state(State s, const uint8_t in[16]) {
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) s[r][c] = in[r + 4 * c]; /* 3.4 */
}

static void store_state(uint8_t out[16], State s) {
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) out[r + 4 * c] = s[r][c];
}

static void add_round_key(State s, const ExpandedKey *ek, int round) { /* 5.1.4 */
    for (int c = 0; c < 4; c++)
        for (int r = 0; r < 4; r++) s[r][c] ^= ek->w[4 * round + c][r];
}

static void sub_bytes(State s) { /* 5.1.1 */
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) s[r][c] = SBOX[s[r][c]];
}

static void inv_sub_bytes(State s) { /* 5.3.2 */
    for (int r = 0; r < 4; r++)
        for (int c = 0; c < 4; c++) s[r][c] = INV_SBOX[s[r][c]];
}

static void shift_rows(State s) { /* 5.1.2: s'[r][c] = s[r][(c + r) mod 4] */
    for (int r = 1; r < 4; r++) {
        uint8_t row[4];
        for (int c = 0; c < 4; c++) row[c] = s[r][(c + r) % 4];
        for (int c = 0; c < 4; c++) s[r][c] = row[c];
    }
}

static void inv_shift_rows(State s) { /* 5.3.1: s'[r][(c + r) mod 4] = s[r][c] */
    for (int r = 1; r < 4; r++) {
        uint8_t row[4];
        for (int c = 0; c < 4; c++) row[(c + r) % 4] = s[r][c];
        for (int c = 0; c < 4; c++) s[r][c] = row[c];
    }
}

/* 5.1.3: each column times the fixed polynomial {03}x^3 + {01}x^2 + {01}x + {02}. */
void oracle_mix_column(uint8_t col[4]) {
    uint8_t a0 = col[0], a1 = col[1], a2 = col[2], a3 = col[3];
    col[0] = (uint8_t)(oracle_gf_mul(2, a0) ^ oracle_gf_mul(3, a1) ^ a2 ^ a3);
    col[1] = (uint8_t)(a0 ^ oracle_gf_mul(2, a1) ^ oracle_gf_mul(3, a2) ^ a3);
    col[2] = (uint8_t)(a0 ^ a1 ^ oracle_gf_mul(2, a2) ^ oracle_gf_mul(3, a3));
    col[3] = (uint8_t)(oracle_gf_mul(3, a0) ^ a1 ^ a2 ^ oracle_gf_mul(2, a3));
}

/* 5.3.3: each column times {0b}x^3 + {0d}x^2 + {09}x + {0e}. */
void oracle_inv_mix_column(uint8_t col[4]) {
    uint8_t a0 = col[0], a1 = col[1], a2 = col[2], a3 = col[3];
    col[0] = (uint8_t)(oracle_gf_mul(0x0e, a0) ^ oracle_gf_mul(0x0b, a1) ^ oracle_gf_mul(0x0d, a2) ^
                       oracle_gf_mul(0x09, a3));
    col[1] = (uint8_t)(oracle_gf_mul(0x09, a0) ^ oracle_gf_mul(0x0e, a1) ^ oracle_gf_mul(0x0b, a2) ^
                       oracle_gf_mul(0x0d, a3));
    col[2] = (uint8_t)(oracle_gf_mul(0x0d, a0) ^ oracle_gf_mul(0x09, a1) ^ oracle_gf_mul(0x0e, a2) ^
                       oracle_gf_mul(0x0b, a3));
    col[3] = (uint8_t)(oracle_gf_mul(0x0b, a0) ^ oracle_gf_mul(0x0d, a1) ^ oracle_gf_mul(0x09, a2) ^
                       oracle_gf_mul(0x0e, a3));
}

static void mix_columns(State s) {
    for (int c = 0; c < 4; c++) {
        uint8_t col[4] = {s[0][c], s[1][c], s[2][c], s[3][c]};
        oracle_mix_column(col);
        for (int r = 0; r < 4; r++) s[r][c] = col[r];
    }
}

static void inv_mix_columns(State s) {
    for (int c = 0; c < 4; c++) {
        uint8_t col[4] = {s[0][c], s[1][c], s[2][c], s[3][c]};
        oracle_inv_mix_column(col);
        for (int r = 0; r < 4; r++) s[r][c] = col[r];
    }
}

/* FIPS-197 5.1, Figure 5 */
static void cipher(const uint8_t in[16], uint8_t out[16], const ExpandedKey *ek) {
    State s;
    load_state(s, in);
    add_round_key(s, ek, 0);
    for (int round = 1; round < ek->nr; round++) {
        sub_bytes(s);
        shift_rows(s);
        mix_columns(s);
        add_round_key(s, ek, round);
    }
    sub_bytes(s);
    shift_rows(s);
    add_round_key(s, ek, ek->nr);
    store_state(out, s);
}

/* FIPS-197 5.3, Figure 12 (the straightforward inverse cipher) */
static void inv_cipher(const uint8_t in[16], uint8_t out[16], const ExpandedKey *ek) {
    State s;
    load_state(s, in);
    add_round_key(s, ek, ek->nr);
    for (int round = ek->nr - 1; round >= 1; round--) {
        inv_shift_rows(s);
        inv_sub_bytes(s);
        add_round_key(s, ek, round);
        inv_mix_columns(s);
    }
    inv_shift_rows(s);
    inv_sub_bytes(s);
    add_round_key(s, ek, 0);
    store_state(out, s);
}

/* Single-block entry points for tests: dir 0 = Cipher, 1 = InvCipher. */
int oracle_block(const uint8_t *key, int key_len, int dir, const uint8_t in[16], uint8_t out[16]) {
    ExpandedKey ek;
    int rc = key_expansion(key, key_len, &ek);
    if (rc) return rc;
    if (dir == 0) cipher(in, out, &ek);
    else inv_cipher(in, out, &ek);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Parallel driver: run fn(unit) for unit in [0, n) on nthreads POSIX threads.
 * ------------------------------------------------------------------------- */

typedef void (*unit_fn)(void *ctx, size_t unit);

typedef struct {
    unit_fn fn;
    void *ctx;
    size_t begin, end;
} Span;

static void *span_main(void *arg) {
    Span *sp = (Span *)arg;
    for (size_t u = sp->begin; u < sp->end; u++) sp->fn(sp->ctx, u);
    return NULL;
}

static void parallel_units(size_t n, unit_fn fn, void *ctx, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > n) nthreads = (int)(n ? n : 1);
    if (nthreads == 1) {
        for (size_t u = 0; u < n; u++) fn(ctx, u);
        return;
    }
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    Span *sp = (Span *)calloc((size_t)nthreads, sizeof(Span));
    for (int t = 0; t < nthreads; t++) {
        sp[t].fn = fn;
        sp[t].ctx = ctx;
        sp[t].begin = n * (size_t)t / (size_t)nthreads;
        sp[t].end = n * (size_t)(t + 1) / (size_t)nthreads;
        pthread_create(&th[t], NULL, span_main, &sp[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    free(sp);
}

/* ---------------------------------------------------------------------------
 * XTS-AES (IEEE 1619-2007 section 5; NIST SP 800-38E).
 * ------------------------------------------------------------------------- */

/* IEEE 1619 5.2: multiply the tweak by alpha (the primitive element x) in
 * GF(2^128) mod x^128 + x^7 + x^2 + x + 1, with the 16 bytes read as a
 * little-endian polynomial: shift left one bit across the bytes, carrying the
 * top bit of byte k into byte k + 1, and fold the bit shifted out of byte 15
 * back in as 0x87 on byte 0. */
void oracle_xts_mul_alpha(uint8_t t[16]) {
    int carry = 0;
    for (int k = 0; k < 16; k++) {
        int next = (t[k] >> 7) & 1;
        t[k] = (uint8_t)((t[k] << 1) | carry);
        carry = next;
    }
    if (carry) t[0] ^= 0x87;
}

typedef struct {
    ExpandedKey k1, k2;
    int dir;
    const uint8_t *src;
    uint8_t *dst;
    size_t du;
    uint64_t first_sector;
} XtsJob;

/* IEEE 1619 5.3.1 / 5.4.1 on one 16-byte block with tweak value t:
 * out = E_K1(in ^ t) ^ t (or D_K1 for decryption). */
static void xts_block(const XtsJob *jb, int dir, const uint8_t in[16], uint8_t out[16], const uint8_t t[16]) {
    uint8_t pp[16], cc[16];
    for (int k = 0; k < 16; k++) pp[k] = (uint8_t)(in[k] ^ t[k]);
    if (dir == 0) cipher(pp, cc, &jb->k1);
    else inv_cipher(pp, cc, &jb->k1);
    for (int k = 0; k < 16; k++) out[k] = (uint8_t)(cc[k] ^ t[k]);
}

/* IEEE 1619 5.3 / 5.4 for data unit u: T = E_K2(i) with i the data-unit
 * number as a 128-bit little-endian value; block j uses T * alpha^j.  A unit
 * of m full blocks and a final partial block of b bytes (0 < b < 16) ends with
 * ciphertext stealing (5.3.2 encryption, 5.4.2 decryption):
 *   encryption: CC = enc(P_{m-1}, T a^{m-1}); C_m = the first b bytes of CC;
 *               C_{m-1} = enc(P_m || the last 16-b bytes of CC, T a^m);
 *   decryption: PP = dec(C_{m-1}, T a^m); P_m = the first b bytes of PP;
 *               P_{m-1} = dec(C_m || the last 16-b bytes of PP, T a^{m-1}). */
static void xts_unit(void *ctx, size_t u) {
    XtsJob *jb = (XtsJob *)ctx;
    uint64_t sector = jb->first_sector + (uint64_t)u;
    uint8_t ival[16] = {0};
    for (int k = 0; k < 8; k++) ival[k] = (uint8_t)(sector >> (8 * k));
    uint8_t t[16];
    cipher(ival, t, &jb->k2);
    const size_t m = jb->du / 16, b = jb->du % 16;
    const uint8_t *in = jb->src + u * jb->du;
    uint8_t *out = jb->dst + u * jb->du;
    /* the blocks before the stealing pair (all of them when b == 0) */
    const size_t plain = b ? m - 1 : m;
    for (size_t j = 0; j < plain; j++) {
        xts_block(jb, jb->dir, in + 16 * j, out + 16 * j, t);
        oracle_xts_mul_alpha(t);
    }
    if (!b) return;
    uint8_t t_last[16], last[16], tail[16], x[16], y[16];
    memcpy(t_last, t, 16); /* T a^{m-1} */
    oracle_xts_mul_alpha(t_last);
    /* now t = T a^{m-1}, t_last = T a^m; read both inputs before writing */
    memcpy(last, in + 16 * (m - 1), 16);
    memcpy(tail, in + 16 * m, b);
    if (jb->dir == 0) {
        xts_block(jb, 0, last, x, t);             /* CC */
        memcpy(y, tail, b);                        /* PP = P_m || CC[b..16) */
        memcpy(y + b, x + b, 16 - b);
        xts_block(jb, 0, y, out + 16 * (m - 1), t_last);
        memcpy(out + 16 * m, x, b);                /* C_m = CC[0..b) */
    } else {
        xts_block(jb, 1, last, x, t_last);        /* PP */
        memcpy(y, tail, b);                        /* CC = C_m || PP[b..16) */
        memcpy(y + b, x + b, 16 - b);
        xts_block(jb, 1, y, out + 16 * (m - 1), t);
        memcpy(out + 16 * m, x, b);                /* P_m = PP[0..b) */
    }
}

/* key = Key1 || Key2 (key_len 32 or 64 bytes), dir 0 encrypt / 1 decrypt.
 * len must be a multiple of du and du at least 16 bytes; a du that is not a
 * multiple of 16 ends every unit with ciphertext stealing.  Key1 == Key2 is
 * rejected, as IEEE 1619-2018 requires. */
int oracle_xts(const uint8_t *key, int key_len, int dir, const uint8_t *src, uint8_t *dst,
               size_t len, size_t du, uint64_t first_sector, int nthreads) {
    if (key_len != 32 && key_len != 64) return OR_EINVAL;
    if (du < 16 || len % du) return OR_EINVAL;
    if (dir != 0 && dir != 1) return OR_EINVAL;
    int half = key_len / 2;
    if (memcmp(key, key + half, (size_t)half) == 0) return OR_EINVAL;
    XtsJob jb;
    if (key_expansion(key, half, &jb.k1) || key_expansion(key + half, half, &jb.k2)) return OR_EINVAL;
    jb.dir = dir;
    jb.src = src;
    jb.dst = dst;
    jb.du = du;
    jb.first_sector = first_sector;
    parallel_units(len / du, xts_unit, &jb, nthreads);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * CBC (NIST SP 800-38A 6.2), one independent chain per page.
 * ------------------------------------------------------------------------- */

typedef struct {
    ExpandedKey k;
    int dir;
    const uint8_t *src;
    uint8_t *dst;
    size_t page;
    const uint8_t *ivs;
} CbcJob;

static void cbc_page(void *ctx, size_t p) {
    CbcJob *jb = (CbcJob *)ctx;
    const uint8_t *in = jb->src + p * jb->page;
    uint8_t *out = jb->dst + p * jb->page;
    uint8_t prev[16]; /* C_{j-1}, starting from the page's IV */
    memcpy(prev, jb->ivs + 16 * p, 16);
    size_t nblk = jb->page / 16;
    for (size_t j = 0; j < nblk; j++) {
        uint8_t x[16], y[16];
        if (jb->dir == 0) {
            /* C_j = CIPH_K(P_j xor C_{j-1}) */
            for (int k = 0; k < 16; k++) x[k] = (uint8_t)(in[16 * j + k] ^ prev[k]);
            cipher(x, y, &jb->k);
            memcpy(out + 16 * j, y, 16);
            memcpy(prev, y, 16);
        } else {
            /* P_j = CIPH_K^-1(C_j) xor C_{j-1}; C_j is saved first so that the
             * page may be decrypted in place. */
            uint8_t c[16];
            memcpy(c, in + 16 * j, 16);
            inv_cipher(c, y, &jb->k);
            for (int k = 0; k < 16; k++) out[16 * j + k] = (uint8_t)(y[k] ^ prev[k]);
            memcpy(prev, c, 16);
        }
    }
}

/* dir 0 encrypt / 1 decrypt; key_len 16, 24 or 32; ivs holds len/page 16-byte IVs. */
int oracle_cbc(const uint8_t *key, int key_len, int dir, const uint8_t *src, uint8_t *dst, size_t len,
               size_t page, const uint8_t *ivs, int nthreads) {
    if (page == 0 || page % 16 || len % page) return OR_EINVAL;
    if (dir != 0 && dir != 1) return OR_EINVAL;
    CbcJob jb;
    if (key_expansion(key, key_len, &jb.k)) return OR_EINVAL;
    jb.dir = dir;
    jb.src = src;
    jb.dst = dst;
    jb.page = page;
    jb.ivs = ivs;
    parallel_units(len / page, cbc_page, &jb, nthreads);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * ECB (NIST SP 800-38A 6.1): the mode of the paper's own GPU service (3.3).
 * ------------------------------------------------------------------------- */

typedef struct {
    ExpandedKey k;
    int dir;
    const uint8_t *src;
    uint8_t *dst;
} EcbJob;

static void ecb_block(void *ctx, size_t b) {
    EcbJob *jb = (EcbJob *)ctx;
    uint8_t x[16], y[16];
    memcpy(x, jb->src + 16 * b, 16);
    if (jb->dir == 0) cipher(x, y, &jb->k);
    else inv_cipher(x, y, &jb->k);
    memcpy(jb->dst + 16 * b, y, 16);
}

int oracle_ecb(const uint8_t *key, int key_len, int dir, const uint8_t *src, uint8_t *dst, size_t len,
               int nthreads) {
    if (len % 16) return OR_EINVAL;
    if (dir != 0 && dir != 1) return OR_EINVAL;
    EcbJob jb;
    if (key_expansion(key, key_len, &jb.k)) return OR_EINVAL;
    jb.dir = dir;
    jb.src = src;
    jb.dst = dst;
    parallel_units(len / 16, ecb_block, &jb, nthreads);
    return OR_OK;
}
