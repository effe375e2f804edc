/*
 * The library used from C alone, with no Python and no PyTorch: what an
 * operating-system-side caller would write.  Reads a 64-byte XTS key, a
 * 16-byte CBC key, page IVs and plaintext from files, then
 *   1. encrypts the plaintext with AES-256-XTS (4096-byte data units, first
 *      unit 5) through kgpu_aes_xts_crypt on device memory;
 *   2. encrypts it with AES-128-CBC (4096-byte pages) as one batched request
 *      through kgpu_submit / kgpu_poll;
 *   3. checks that a misaligned call is refused with KGPU_EINVAL;
 *   4. decrypts the XTS ciphertext again through the serving ring as a request
 *      with a completion callback, blocking on a condition variable until the
 *      callback has run (the paper's request model, section 3.2), and checks
 *      that the plaintext came back;
 * and writes both ciphertexts to files for the test to compare.
 * usage: c_api_example key64 key16 ivs plain out_xts out_cbc
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <cuda_runtime.h>

#include "kgpu.h"

static unsigned char *slurp(const char *path, size_t *len) {
    FILE *f = fopen(path, "rb");
    if (!f) return NULL;
    fseek(f, 0, SEEK_END);
    long n = ftell(f);
    fseek(f, 0, SEEK_SET);
    unsigned char *p = malloc(n > 0 ? (size_t)n : 1);
    if (p && fread(p, 1, (size_t)n, f) != (size_t)n) {
        free(p);
        p = NULL;
    }
    fclose(f);
    *len = (size_t)n;
    return p;
}

static int spill(const char *path, const void *p, size_t len) {
    FILE *f = fopen(path, "wb");
    if (!f) return -1;
    size_t w = fwrite(p, 1, len, f);
    fclose(f);
    return w == len ? 0 : -1;
}

#define CHECK(call)                                                                  \
    do {                                                                             \
        int rc_ = (call);                                                            \
        if (rc_) {                                                                   \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, kgpu_strerror(rc_)); \
            return 1;                                                                \
        }                                                                            \
    } while (0)

/* what the completion callback hands to the thread that waits for it */
struct done {
    pthread_mutex_t mu;
    pthread_cond_t cv;
    int calls, status;
    kgpu_ticket ticket;
};

static void on_done(void *arg, kgpu_ticket ticket, int status) {
    struct done *d = arg;
    pthread_mutex_lock(&d->mu);
    d->calls++;
    d->status = status;
    d->ticket = ticket;
    pthread_cond_signal(&d->cv);
    pthread_mutex_unlock(&d->mu);
}

int main(int argc, char **argv) {
    if (argc != 7) return 2;
    size_t nk64, nk16, niv, n;
    unsigned char *k64 = slurp(argv[1], &nk64), *k16 = slurp(argv[2], &nk16);
    unsigned char *ivs = slurp(argv[3], &niv), *plain = slurp(argv[4], &n);
    if (!k64 || !k16 || !ivs || !plain || nk64 != 64 || nk16 != 16 || n % 4096 || niv != n / 4096 * 16) return 2;

    kgpu_ctx *ctx;
    CHECK(kgpu_init(&ctx, 0, NULL));
    kgpu_key kx, kc;
    CHECK(kgpu_aes_setkey(ctx, k64, 64, 1, &kx));
    CHECK(kgpu_aes_setkey(ctx, k16, 16, 0, &kc));

    void *d_in, *d_out, *d_ivs;
    if (cudaMalloc(&d_in, n) || cudaMalloc(&d_out, 2 * n) || cudaMalloc(&d_ivs, niv)) return 3;
    if (cudaMemcpy(d_in, plain, n, cudaMemcpyHostToDevice) || cudaMemcpy(d_ivs, ivs, niv, cudaMemcpyHostToDevice))
        return 3;

    /* 1. per-call XTS on the default stream */
    CHECK(kgpu_aes_xts_crypt(ctx, kx, KGPU_ENCRYPT, d_in, d_out, n, 4096, 5, 0));

    /* 2. CBC encryption as a batched request */
    kgpu_request r;
    memset(&r, 0, sizeof(r));
    r.mode = KGPU_MODE_CBC_ENC;
    r.key = kc;
    r.src = d_in;
    r.dst = (char *)d_out + n;
    r.len = n;
    r.unit_size = 4096;
    r.ivs = d_ivs;
    kgpu_ticket t;
    int st = -1;
    CHECK(kgpu_submit(ctx, &r, 1, 0, &t, NULL));
    CHECK(kgpu_poll(ctx, t, -1, &st));
    if (st != 0) return 4;

    /* 3. a refused call launches nothing */
    if (kgpu_aes_xts_crypt(ctx, kx, KGPU_ENCRYPT, (char *)d_in + 8, d_out, 4096, 4096, 0, 0) != KGPU_EINVAL) return 5;

    /* 4. back through the serving ring, waiting for the completion callback */
    void *d_back;
    if (cudaMalloc(&d_back, n) || cudaDeviceSynchronize()) return 3;
    CHECK(kgpu_serve_start(ctx, NULL));
    kgpu_request q;
    memset(&q, 0, sizeof(q));
    q.mode = KGPU_MODE_XTS;
    q.dir = KGPU_DECRYPT;
    q.key = kx;
    q.src = d_out;
    q.dst = d_back;
    q.len = n;
    q.unit_size = 4096;
    q.sector = 5;
    struct done dn = {PTHREAD_MUTEX_INITIALIZER, PTHREAD_COND_INITIALIZER, 0, -1, 0};
    kgpu_ticket tq;
    CHECK(kgpu_serve_submit_cb(ctx, &q, on_done, &dn, &tq));
    struct timespec until;
    clock_gettime(CLOCK_REALTIME, &until);
    until.tv_sec += 30;
    pthread_mutex_lock(&dn.mu);
    while (dn.calls == 0 && pthread_cond_timedwait(&dn.cv, &dn.mu, &until) == 0) {
    }
    const int calls = dn.calls, status = dn.status;
    const kgpu_ticket seen = dn.ticket;
    pthread_mutex_unlock(&dn.mu);
    CHECK(kgpu_serve_stop(ctx, -1));
    if (calls != 1 || dn.calls != 1 || status != 0 || seen != tq) return 7;
    unsigned char *back = malloc(n);
    if (!back || cudaMemcpy(back, d_back, n, cudaMemcpyDeviceToHost)) return 3;
    if (memcmp(back, plain, n) != 0) return 8;
    free(back);
    cudaFree(d_back);

    unsigned char *out = malloc(2 * n);
    if (!out || cudaMemcpy(out, d_out, 2 * n, cudaMemcpyDeviceToHost)) return 3;
    if (spill(argv[5], out, n) || spill(argv[6], out + n, n)) return 6;

    CHECK(kgpu_aes_delkey(ctx, kx));
    CHECK(kgpu_aes_delkey(ctx, kc));
    cudaFree(d_in);
    cudaFree(d_out);
    cudaFree(d_ivs);
    CHECK(kgpu_destroy(ctx));
    free(out);
    free(plain);
    free(ivs);
    free(k64);
    free(k16);
    printf("c_api_example ok\n");
    return 0;
}
