/*
 * kgpu.h -- C ABI of the GB300 page-crypto service.
 *
 * The service follows the request model of "Augmenting Operating Systems With
 * the GPU" (section 3.2, the GLinux architecture): a caller hands the GPU
 * page-sized buffers together with a key and the sector or IV numbering, and
 * gets the transformed pages back, either by waiting on its own CUDA stream or
 * through a submit/poll ticket (the paper's request queue / response queue with
 * blocking or busy-waiting).  The cipher service itself is the paper's GPU AES
 * (section 3.3), extended from ECB to the page modes that encrypted storage
 * uses: XTS (IEEE 1619-2007 / NIST SP 800-38E) and CBC (NIST SP 800-38A).
 *
 * Conventions for every call:
 *  - Return value: 0 (KGPU_OK) or a negative errno-style code (KGPU_E*).
 *    Nothing is launched when a call returns an error.
 *  - Buffers are caller-owned; the library never frees caller memory.  Unless a
 *    call says otherwise, src/dst/ivs are DEVICE pointers (cudaMalloc, the
 *    PyTorch caching allocator, or managed memory) and must lie wholly inside
 *    one device allocation; this is checked, and a failure is KGPU_EFAULT.
 *  - src and dst must be 16-byte aligned.  src == dst (in place) is allowed
 *    for every mode; any other overlap is KGPU_EINVAL.
 *  - Lengths are in bytes and must be whole data units / pages; the unit size
 *    must be a nonzero multiple of 16, except the XTS data unit of
 *    kgpu_aes_xts_crypt, which may be any size from 16 bytes (a unit ending in
 *    a partial block uses ciphertext stealing).  There is no padding.
 *    len == 0 is a no-op.
 *  - Device work is asynchronous on the caller's stream (0 = legacy default
 *    stream).  A launch failure is reported as KGPU_EIO; an asynchronous fault
 *    surfaces from the next synchronising CUDA call on that stream.
 *  - A context is bound to one device.  Calls on one context may come from
 *    several host threads; key handles are shared by all of them.
 */
#ifndef KGPU_H
#define KGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default) /* the library is built with hidden visibility */
#endif

typedef struct kgpu_ctx kgpu_ctx;  /* opaque, library-owned */
typedef uint32_t kgpu_key;         /* handle into the context's key table */
typedef uint64_t kgpu_ticket;      /* handle of a submitted batch */
typedef struct CUstream_st *kgpu_stream; /* a cudaStream_t */

enum {
    KGPU_OK = 0,
    KGPU_EIO = -5,         /* CUDA launch or runtime failure */
    KGPU_E2BIG = -7,       /* more requests than a fixed-size area holds */
    KGPU_ENOMEM = -12,     /* allocation failed or a table is full */
    KGPU_EFAULT = -14,     /* a pointer is not (wholly) inside a usable allocation */
    KGPU_EBUSY = -16,      /* queue full / admission refused: retry later */
    KGPU_ENODEV = -19,     /* no such CUDA device, or not an sm_103 part */
    KGPU_EINVAL = -22,     /* malformed argument (length, alignment, key, mode) */
    KGPU_ENOENT = -2,      /* unknown key handle or ticket */
    KGPU_ENOSYS = -38,     /* the host AES library (OpenSSL libcrypto 3) could not be loaded */
    KGPU_ETIMEDOUT = -110  /* a bounded wait ran out */
};

enum { KGPU_ENCRYPT = 0, KGPU_DECRYPT = 1 };

enum {
    KGPU_MODE_XTS = 0,     /* XTS, direction from kgpu_request.dir */
    KGPU_MODE_CBC_DEC = 1, /* CBC decryption, parallel over blocks */
    KGPU_MODE_CBC_ENC = 2, /* CBC encryption, parallel over pages */
    KGPU_MODE_ECB = 3,     /* ECB, the paper's own service mode (section 3.3) */
    KGPU_MODE_COPY = 4     /* the empty service: dst receives src unchanged, no key
                              (the paper's round-trip measurement of its Non-Stop
                              Kernel with a service that does no work, section 3.1);
                              unit_size = bytes per tile, one warp per tile, so a
                              request of len bytes occupies 32 * len / unit_size
                              threads */
};

/* Library version, (major << 16) | minor. */
int kgpu_version(void);

/* Short English description of a KGPU_* code (static storage). */
const char *kgpu_strerror(int code);

/* Optional configuration; zero fields take defaults. */
typedef struct kgpu_config {
    uint32_t max_keys;            /* key-table capacity (default 4096) */
    uint32_t ring_slots;          /* serving ring capacity (default 4096, power of two) */
    uint64_t admit_bytes;         /* serving: cap on bytes in flight (default 8 GiB) */
    uint64_t idle_timeout_ns;     /* serving kernel exits after this long with no work (default 2 s) */
    uint32_t host_dispatch;       /* 1: measure the CPU/GPU crossover at kgpu_init and let kgpu_crypt
                                     run small host-resident requests on the host (default 0: off) */
    uint32_t reserved[7];
} kgpu_config;

/*
 * Create a context on CUDA device `device` (uploads the cipher tables and
 * allocates the device key table).  cfg may be NULL.  The context owns no
 * caller memory.  Errors: KGPU_ENODEV, KGPU_ENOMEM, KGPU_EIO, KGPU_EINVAL.
 */
int kgpu_init(kgpu_ctx **ctx, int device, const kgpu_config *cfg);

/* Stop the serving kernel if one runs, wait for the context's own work and
 * free everything the context allocated.  NULL is accepted.  Completion
 * callbacks still waiting run first, with KGPU_ENOENT for requests the
 * stopped kernel left unfinished (no drain).  Called from a completion
 * callback: KGPU_EINVAL, and the context stays as it was. */
int kgpu_destroy(kgpu_ctx *ctx);

/*
 * Register a key (the paper's pre-loaded service state, section 3.1).  The key
 * schedule is expanded on the host (FIPS-197 section 5.2) and stored in the
 * context, both for launch-time use and in the device key table read by the
 * batched and serving kernels.
 *   xts = 0: a single AES key of 16, 24 or 32 bytes (CBC, ECB).
 *   xts = 1: Key1 || Key2 of 32 or 64 bytes (XTS data key, then tweak key;
 *            IEEE 1619 defines XTS-AES-128 and XTS-AES-256 only);
 *            Key1 == Key2 is rejected (IEEE 1619-2018 requires them distinct).
 * The key bytes are copied; the caller may wipe its buffer after the call.
 * Errors: KGPU_EINVAL (length, duplicated halves), KGPU_ENOMEM (table full).
 */
int kgpu_aes_setkey(kgpu_ctx *ctx, const uint8_t *key, size_t key_len, int xts, kgpu_key *out);

/*
 * Forget a key.  Work already submitted with it completes first: batches of
 * kgpu_submit and kgpu_submit_noalloc, and requests published to the serving
 * ring.  (Per-call transforms carry their key schedule in the launch.)  The
 * handle may be reused by a later kgpu_aes_setkey.
 */
int kgpu_aes_delkey(kgpu_ctx *ctx, kgpu_key key);

/*
 * XTS-AES over len / du_size data units (IEEE 1619 section 5.3 / 5.4):
 * unit u is numbered first_sector + u, its tweak is E_Key2(number) with the
 * number as a 128-bit little-endian value, and block j of the unit is
 * processed with tweak * alpha^j in GF(2^128).  dir: KGPU_ENCRYPT / DECRYPT.
 * du_size: at least 16 bytes (512 and 4096 are the usual sectors).  A
 * du_size that is not a multiple of 16 ends every unit with a partial block,
 * handled by ciphertext stealing (IEEE 1619 5.3.2 / 5.4.2): the last full
 * block and the partial block are processed together, so every unit keeps its
 * length.  (Only this per-call entry point takes such units; the batched,
 * serving, host-pipeline and bitsliced forms require multiples of 16.)
 * src, dst: device pointers, len bytes each, 16-byte aligned; len a multiple
 * of du_size.  Async on `stream`.
 * Errors: KGPU_EINVAL, KGPU_ENOENT (not an XTS key), KGPU_EFAULT, KGPU_EIO.
 */
int kgpu_aes_xts_crypt(kgpu_ctx *ctx, kgpu_key key, int dir, const void *src, void *dst, size_t len,
                       size_t du_size, uint64_t first_sector, kgpu_stream stream);

/*
 * XTS-AES encryption by the bitsliced cipher: the comparison variant of
 * kgpu_aes_xts_crypt, with the same arguments, layout and result bytes.  Each
 * thread enciphers 32 blocks at once as 128 bit-planes, with the S-box as a
 * Boolean circuit of AND/XOR gates on 32-bit words (FIPS-197 5.1.1 through
 * composite-field inversion) and ShiftRows, MixColumns and AddRoundKey as plane
 * renamings and XORs: no table lookups, so the work runs on the ALU instead of
 * the shared-memory path.  The data-unit tweaks E_K2(unit) are computed by a
 * bitsliced pre-pass into a temporary device buffer of 16 bytes per data unit,
 * allocated and freed in stream order on `stream`.
 * dir must be KGPU_ENCRYPT (decryption runs only on the table path):
 * KGPU_EINVAL otherwise.  Other errors as kgpu_aes_xts_crypt, plus
 * KGPU_ENOMEM if the tweak buffer cannot be allocated.
 */
int kgpu_aes_xts_crypt_bitsliced(kgpu_ctx *ctx, kgpu_key key, int dir, const void *src, void *dst, size_t len,
                                 size_t du_size, uint64_t first_sector, kgpu_stream stream);

/*
 * CBC decryption, one chain per page (NIST SP 800-38A 6.2):
 *   P_0 = D_K(C_0) ^ IV_page,  P_i = D_K(C_i) ^ C_{i-1}.
 * Every block is independent given C_{i-1}, so the kernel runs one block per
 * thread.  ivs: DEVICE pointer to len / page_size IVs of 16 bytes.
 * page_size: nonzero multiple of 16 (4096 for file pages).
 */
int kgpu_aes_cbc_decrypt(kgpu_ctx *ctx, kgpu_key key, const void *src, void *dst, size_t len,
                         size_t page_size, const uint8_t *ivs, kgpu_stream stream);

/*
 * CBC encryption, one chain per page: C_0 = E_K(P_0 ^ IV_page),
 * C_i = E_K(P_i ^ C_{i-1}).  Sequential inside a page, parallel across pages
 * (one thread per page).  Arguments as kgpu_aes_cbc_decrypt.  Pages of a
 * multiple of 128 bytes move in and out in 2-D tiles by the tensor-memory-
 * access engine; the waits for those copies are bounded, and one that ran out
 * (never expected) leaves the rest of that warp's pages unwritten and is
 * counted by kgpu_bulk_wait_timeouts.
 */
int kgpu_aes_cbc_encrypt_pages(kgpu_ctx *ctx, kgpu_key key, const void *src, void *dst, size_t len,
                               size_t page_size, const uint8_t *ivs, kgpu_stream stream);

/*
 * Bounded waits of the bulk kernels that ran out on the context's device, as
 * a count for the whole process (the kernels' counter is per device, not per
 * context): 0 unless a tensor copy never completed.  Synchronous: copies the
 * counter from the device.  Errors: KGPU_EINVAL (NULL argument), KGPU_EIO.
 */
int kgpu_bulk_wait_timeouts(kgpu_ctx *ctx, uint32_t *count);

/*
 * ECB over len / 16 independent blocks: the mode of the paper's own GPU AES
 * service (section 3.3).  key: a single (non-XTS) key.
 */
int kgpu_aes_ecb_crypt(kgpu_ctx *ctx, kgpu_key key, int dir, const void *src, void *dst, size_t len,
                       kgpu_stream stream);

/*
 * XTS over HOST-resident pages, the paper's pinned-buffer pipeline (section
 * 3.1, "Data Copy Overhead", and the buffer rotation of section 3.2): the
 * buffer is cut into chunk_bytes pieces (a multiple of du_size; 0 = 4 MiB),
 * and each piece is copied host-to-device, transformed and copied back on one
 * of three library-owned streams (one chunk in, one transformed, one out), so
 * copies overlap compute.  src and dst are
 * HOST pointers (pinned memory gives full link speed; pageable memory works
 * but is slower); src == dst is allowed.  Blocks until dst holds the result.
 * Device staging buffers are owned by the context and reused across calls.
 * When both [src, src + len) and [dst, dst + len) lie inside ranges
 * registered with kgpu_host_register, there is no staging and no copy: the
 * kernel reads and writes the host pages in place over the host link, and
 * chunk_bytes is ignored.  kgpu_host_unregister waits for such a call.
 */
int kgpu_aes_xts_crypt_host(kgpu_ctx *ctx, kgpu_key key, int dir, const void *src, void *dst, size_t len,
                            size_t du_size, uint64_t first_sector, size_t chunk_bytes);

/* ------------------------------------------------------------------------
 * Batched submission: the paper's service-request protocol (section 3.2:
 * build a request, place it in the request queue, then wait by blocking or
 * by busy-waiting on the response queue), with many requests per submission.
 * ---------------------------------------------------------------------- */

/*
 * Registered host memory.  A GB300's GPU reaches page-locked host memory
 * coherently over its NVLink-C2C link, so the batched and serving kernels can
 * read a request's input pages from host memory and write its output pages
 * back there directly, with no staging copy (the role of the paper's
 * helper-driven copies in and out of pinned buffers, section 3.2).  A host
 * range must be registered first, so that the library only ever hands the GPU
 * host addresses it knows to be mapped for it.
 *
 * kgpu_host_register: ptr/len is the range (any alignment; requests inside it
 * still need 16-byte aligned pointers).  flags:
 *   KGPU_HOSTREG_PIN     the library page-locks and maps the range
 *                        (cudaHostRegister) and unlocks it again on
 *                        kgpu_host_unregister or kgpu_destroy;
 *   KGPU_HOSTREG_PINNED  the caller has page-locked it already (cudaHostAlloc,
 *                        cudaHostRegister, a framework's pinned allocator);
 *                        every page of the range is checked to be pinned and
 *                        mapped for this context's device, with one
 *                        device-address offset for the whole range.
 * Errors: KGPU_EINVAL (NULL, empty, wrapping, unknown flag, or overlapping a
 * range already registered), KGPU_EFAULT (PINNED and some page is not pinned
 * and mapped), KGPU_ENOMEM / KGPU_EIO (PIN and the runtime refused).
 * Registration is per context; the caller keeps ownership of the memory.
 *
 * kgpu_host_unregister: ptr is the start of a registered range (else
 * KGPU_ENOENT).  Waits for batches submitted with kgpu_submit or
 * kgpu_submit_noalloc, for requests published to the serving ring, and for
 * kgpu_aes_xts_crypt_host and kgpu_crypt calls running on host pages, then
 * forgets the range.
 */
#define KGPU_HOSTREG_PIN 0u
#define KGPU_HOSTREG_PINNED 1u
int kgpu_host_register(kgpu_ctx *ctx, void *ptr, size_t len, uint32_t flags);
int kgpu_host_unregister(kgpu_ctx *ctx, void *ptr);

/* kgpu_request.flags: which pointers of the request lie in registered host
 * memory (each must then fall inside one range registered with
 * kgpu_host_register, else KGPU_EFAULT); the others are device memory of the
 * context's GPU.  Any other bit set: KGPU_EINVAL. */
#define KGPU_REQ_SRC_HOST 0x1u
#define KGPU_REQ_DST_HOST 0x2u
#define KGPU_REQ_IVS_HOST 0x4u

/* One request of a batch.  Pointers are DEVICE pointers unless flags mark
 * them as registered host memory. */
typedef struct kgpu_request {
    uint32_t mode;       /* KGPU_MODE_* */
    uint32_t dir;        /* KGPU_ENCRYPT / KGPU_DECRYPT for XTS and ECB; ignored for CBC */
    kgpu_key key;        /* an XTS key for KGPU_MODE_XTS, a single key for CBC and ECB,
                            ignored for KGPU_MODE_COPY */
    uint32_t flags;      /* KGPU_REQ_* bits, or 0 */
    const void *src;     /* 16-byte aligned */
    void *dst;           /* == src (in place) or disjoint from it */
    uint64_t len;        /* bytes: a multiple of unit_size (ECB: of 16) */
    uint64_t unit_size;  /* XTS data-unit size / CBC page size / COPY bytes per warp-tile;
                            ignored for ECB */
    uint64_t sector;     /* XTS: number of the first data unit */
    const uint8_t *ivs;  /* CBC: len / unit_size IVs of 16 bytes, not overlapping dst */
} kgpu_request;

/* Launch shape of the persistent batch kernel (see kgpu_autotune). */
typedef struct kgpu_tuning {
    uint32_t threads;      /* threads per CTA: 512 or 1024 (default 512); a batch holding
                              CBC encryption of host pages runs with 512, the kernel
                              that stages those pages through whole-line copies */
    uint32_t tile_chunks;  /* work per XTS/ECB tile in 512-byte chunks (default 32 = 16 KiB);
                              CBC-decrypt tiles hold the same bytes in whole pages,
                              CBC-encrypt tiles hold up to 32 pages (one chain per lane) */
    uint32_t ctas;         /* CTAs of the persistent kernel (default 0 = one per SM) */
    uint32_t reserved;
} kgpu_tuning;

/*
 * Submit n requests as ONE launch of a persistent kernel on `stream`: warps
 * pull fixed-size tiles of the requests from a shared counter, whatever their
 * mode, key or size.  The requests are validated first; if any is malformed
 * nothing is launched, KGPU_EINVAL/KGPU_ENOENT/KGPU_EFAULT is returned and,
 * when req_status is non-NULL, req_status[i] holds each request's own code.
 * The descriptors are copied into one of four rotating pinned staging slots
 * (the paper's four static pinned buffers, section 3.2) and the submission is
 * replayed as a CUDA graph {copy in, clear, kernel, copy status out}.  When
 * all four slots hold unfinished batches, submit blocks until the oldest ends;
 * when the slot it would reuse is being waited on by a kgpu_poll or
 * kgpu_poll_each call, it returns KGPU_EBUSY (retry).  Reusing a slot does not
 * end its batch's ticket (see kgpu_poll).
 * *out receives a ticket for kgpu_poll.  n == 0 gives a ticket that is
 * already complete.  Requests of one batch run concurrently and in no fixed
 * order: no request may write bytes that another request of the same batch
 * reads or writes.
 */
int kgpu_submit(kgpu_ctx *ctx, const kgpu_request *reqs, size_t n, kgpu_stream stream, kgpu_ticket *out,
                int *req_status);

/*
 * Wait for a ticket (the response queue).  timeout_ns == 0: check once
 * (busy-wait by calling again); < 0: block until complete; > 0: wait at most
 * that long.  Returns KGPU_OK when the batch is complete (req_status, if not
 * NULL, receives each request's status: 0, or KGPU_ENOENT if its key was
 * deleted before it ran), KGPU_ETIMEDOUT if it is still running, and
 * KGPU_ENOENT for a ticket never issued.  A ticket whose slot a later
 * submission has reused was complete by then (the submission waited for it):
 * its poll returns KGPU_OK and its statuses from a record the library keeps
 * of the newest 4096 such batches; older ones give KGPU_ENOENT.  Safe to call
 * from several threads; while a call waits, its slot is not reused.
 */
int kgpu_poll(kgpu_ctx *ctx, kgpu_ticket ticket, int64_t timeout_ns, int *req_status);

/*
 * Wait for a ticket request by request: each request of the batch publishes
 * its own completion as the warp that finishes its last tile writes a
 * completion word in pinned host memory (after the request's output is in
 * place), so small requests are done long before the batch ends.  Polls those
 * words until every request is complete and writes, for each request i,
 * done_ns[i] = the host's CLOCK_MONOTONIC time (ns) at which its completion
 * was first seen (requests of zero length: the call's start).  Then behaves
 * as kgpu_poll(..., -1, req_status).  done_ns: n entries, caller-owned.
 * timeout_ns < 0: no limit; otherwise KGPU_ETIMEDOUT after that long with
 * some requests still running (done_ns[i] = 0 for those).  While a call waits
 * on a ticket, a kgpu_submit that would reuse its staging slot returns
 * KGPU_EBUSY instead.  A ticket whose slot had already been reused is
 * complete: KGPU_OK, with done_ns[i] = 0 for every request (the times were
 * not kept) and the statuses as kgpu_poll gives them.  Errors: KGPU_EINVAL,
 * KGPU_ENOENT (as kgpu_poll), KGPU_EIO.
 */
int kgpu_poll_each(kgpu_ctx *ctx, kgpu_ticket ticket, int64_t timeout_ns, int *req_status, uint64_t *done_ns);

/* Set / read the batch kernel's launch shape (validated: KGPU_EINVAL). */
int kgpu_set_tuning(kgpu_ctx *ctx, const kgpu_tuning *t);
int kgpu_get_tuning(kgpu_ctx *ctx, kgpu_tuning *t);

/*
 * Autotuner: runs the given batch (iters timed repetitions per candidate,
 * after one warm-up) under each candidate launch shape -- threads per CTA x
 * tile size -- times each with CUDA events on `stream`, keeps the fastest in
 * the context and returns it in *best (and its mean time in *best_ms if not
 * NULL).  The batch is executed many times, so every request must be out of
 * place (src != dst); in-place requests are rejected with KGPU_EINVAL.
 * Blocks until done.
 */
int kgpu_autotune(kgpu_ctx *ctx, const kgpu_request *reqs, size_t n, kgpu_stream stream, uint32_t iters,
                  kgpu_tuning *best, float *best_ms);

/* ------------------------------------------------------------------------
 * Serving loop: the paper's Non-Stop Kernel (section 3.1) -- a kernel that
 * is launched once and receives requests as messages in pinned memory while
 * it runs -- rebuilt with continuous batching and bounded waits.  Requests are
 * published one by one into a ring of descriptors in pinned host memory that
 * the device reads directly; a persistent kernel (one CTA per SM) claims them
 * in tiles as they arrive, so requests that arrive while others are running
 * are admitted as slots and memory free up and run alongside them.  While it
 * runs the kernel occupies every SM: other kernels of the process wait.
 * ---------------------------------------------------------------------- */

typedef struct kgpu_serve_config {
    uint32_t ring_slots;       /* ring capacity, power of two (0: the context's ring_slots) */
    uint32_t tile_chunks;      /* XTS/ECB tile in 512-byte chunks (0: 2, i.e. 1 KiB); requests
                                  published while the ring is backed up (the request
                                  published a quarter of the ring earlier still running)
                                  use at least 64 (32 KiB) for throughput */
    uint64_t admit_bytes;      /* cap on bytes in flight (0: the context's admit_bytes) */
    uint64_t idle_timeout_ns;  /* the kernel exits after this long with nothing to do
                                  (0: the context's idle_timeout_ns); it is relaunched
                                  by the next submit or poll */
    uint64_t lifetime_ns;      /* the kernel exits at a tile boundary after this long and is
                                  relaunched (0: 30 s), so no launch runs unbounded */
    uint32_t reserved[4];
} kgpu_serve_config;

typedef struct kgpu_serve_stats {
    uint64_t submitted;       /* requests accepted */
    uint64_t completed;       /* requests seen complete by the host */
    uint64_t busy_refusals;   /* submits refused with KGPU_EBUSY */
    uint64_t launches;        /* kernel launches (first launch + relaunches) */
    uint64_t inflight_bytes;  /* bytes of requests accepted and not yet seen complete */
    uint32_t running;         /* 1 while a kernel instance is believed to run */
    uint32_t last_exit;       /* why the last instance exited: 1 stop, 2 idle, 3 lifetime */
} kgpu_serve_stats;

/* Allocate the ring and launch the serving kernel on a library-owned stream.
 * cfg may be NULL.  KGPU_EBUSY if serving already runs on this context. */
int kgpu_serve_start(kgpu_ctx *ctx, const kgpu_serve_config *cfg);

/*
 * Publish one request (kgpu_request as for kgpu_submit; len must be > 0).
 * Returns KGPU_EBUSY -- nothing published, retry later -- when its ring slot is
 * still in use or when admitting it would put more than admit_bytes in flight
 * (a request larger than the cap is admitted when nothing else is in flight).
 * *ticket identifies the request for kgpu_serve_poll.
 */
int kgpu_serve_submit(kgpu_ctx *ctx, const kgpu_request *req, kgpu_ticket *ticket);

/*
 * Publish several requests at once (a writeback of many pages, say): all n
 * are validated first (any malformed one: its code is returned and nothing is
 * published); then they are placed on the ring in order, as long as slots and
 * the byte cap allow, and made visible to the device with one update of the
 * ring head.  *accepted receives how many were published; tickets[0..accepted)
 * their tickets.  Returns KGPU_OK when all were, KGPU_EBUSY when the ring or
 * the cap stopped the rest (retry those), KGPU_EINVAL when serving is not
 * started.
 */
int kgpu_serve_submit_many(kgpu_ctx *ctx, const kgpu_request *reqs, size_t n, kgpu_ticket *tickets,
                           size_t *accepted);

/*
 * Wait for a served request.  timeout_ns: 0 = check once, < 0 = wait until
 * done, > 0 = wait at most that long.  KGPU_OK when complete (*status, if not
 * NULL: 0 or the request's KGPU_E* code -- codes of the newest 4096 failed
 * requests are kept after their slots are reused; stamps, if not NULL: the
 * device's %globaltimer at its first tile and at its completion, 0 when the
 * slot has since retired a later request), KGPU_ETIMEDOUT while pending,
 * KGPU_ENOENT for a ticket
 * that was never issued.  Relaunches the kernel if it exited with work pending.
 */
int kgpu_serve_poll(kgpu_ctx *ctx, kgpu_ticket ticket, int64_t timeout_ns, int *status, uint64_t *stamps);

/*
 * Completion callbacks (section 3.2: a service request may carry one, and its
 * caller then blocks until the callback has run instead of busy-waiting on the
 * response queue).  fn(arg, ticket, status) receives the request's ticket and
 * what kgpu_serve_poll would report as its status: 0 or the request's KGPU_E*
 * code; KGPU_ENOENT if the ring was stopped (drain limit reached) or the
 * context destroyed before the request completed; KGPU_EIO if the serving
 * kernel could not be relaunched while the request waited.
 */
typedef void (*kgpu_done_fn)(void *arg, kgpu_ticket ticket, int status);

/*
 * kgpu_serve_submit with a completion callback (fn must not be NULL).  For a
 * request that is published -- KGPU_OK, or KGPU_EIO, for which
 * kgpu_serve_submit also hands out a ticket -- fn is called exactly once; on
 * any other return it is never called.  Callbacks run on the context's
 * completion thread, started by the first such submit on a ring: one at a time,
 * in the order the thread sees the completions (within tens of microseconds of
 * the device's completion store), so a slow callback delays the rest.  A
 * callback may submit, poll and set or delete keys; kgpu_serve_stop and
 * kgpu_destroy called from a callback return KGPU_EINVAL, since both wait for
 * the completion thread.  kgpu_serve_stop and kgpu_destroy return only after
 * every callback of the ring has returned, so arg may be released then.  The
 * ticket can still be polled.  Other errors as kgpu_serve_submit; KGPU_ENOMEM
 * if the completion thread cannot be started.
 */
int kgpu_serve_submit_cb(kgpu_ctx *ctx, const kgpu_request *req, kgpu_done_fn fn, void *arg,
                         kgpu_ticket *ticket);

/* Wait (at most drain_timeout_ns; < 0: no limit) for every published request
 * to complete, stop the kernel and free the ring.  KGPU_ETIMEDOUT if requests
 * were still pending at the limit (the kernel is stopped all the same).  Safe
 * against other threads: submissions made once a stop has begun are refused
 * (KGPU_EINVAL); kgpu_serve_poll and kgpu_replay_serve calls still running
 * when the ring is drained return KGPU_ENOENT within about 50 us, and the ring
 * is freed only after they have; a second concurrent stop waits for the first.
 * Completion callbacks still waiting run before it returns (KGPU_ENOENT for
 * requests the stopped kernel left unfinished).  KGPU_EINVAL when called from
 * a completion callback. */
int kgpu_serve_stop(kgpu_ctx *ctx, int64_t drain_timeout_ns);

int kgpu_serve_get_stats(kgpu_ctx *ctx, kgpu_serve_stats *out);

/*
 * Trace replay for measurements (open-loop load generation): request i is
 * issued at arrival_ns[i] after the call starts -- through the serving ring
 * (kgpu_replay_serve; serving must be started) or as its own kernel launch on
 * one of nstreams streams (kgpu_replay_launches, the per-request baseline) --
 * and latency_ns[i] receives the time from its arrival to the host seeing it
 * complete, so queueing behind a busy GPU counts.  *wall_ns receives the time
 * from the start to the last completion.  All requests are validated before
 * the first is issued.  KGPU_ETIMEDOUT if not all completed within timeout_ns
 * (their latency is then UINT64_MAX).  kgpu_replay_serve can also fill
 * detail[3 * i ...] (if not NULL) with: the time request i waited on the host
 * before it was published (ns, admission and ring limits included), and the
 * device's %globaltimer when its first tile started and when it completed
 * (both 0 if the host saw the completion only after its slot had retired a
 * later request too).
 */
int kgpu_replay_serve(kgpu_ctx *ctx, const kgpu_request *reqs, const uint64_t *arrival_ns, size_t n,
                      int64_t timeout_ns, uint64_t *latency_ns, uint64_t *wall_ns, uint64_t *detail);
int kgpu_replay_launches(kgpu_ctx *ctx, const kgpu_request *reqs, const uint64_t *arrival_ns, size_t n,
                         uint32_t nstreams, int64_t timeout_ns, uint64_t *latency_ns, uint64_t *wall_ns);

/*
 * kgpu_replay_serve, also splitting each request's latency by stage of the
 * request path (the paper's message passing between the host and a resident
 * kernel, section 3.1).  stages[6 * i ...] receives, in nanoseconds since
 * request i's arrival on the host clock: [0] the host published it (the ring
 * head store), [1] the device's dispatcher took it, [2] its tiles were
 * published to the workers, [3] its first tile started, [4] it completed on
 * the device, [5] the host saw it complete (= latency_ns[i]).  Entries 1-4
 * are device %globaltimer stamps moved to the host clock by an offset
 * estimated from the dispatcher's heartbeat before and after the run and
 * interpolated between the two (in case the clocks' rates differ);
 * clock_offset_ns, if not NULL, receives the two estimates (host time =
 * device time + offset).  Each estimate includes the shortest device-to-host
 * store latency, so those entries read late by that much (under a
 * microsecond).  A stamp lost to a slot that retired a later request before
 * the host looked is INT64_MIN.  Starts the serving kernel first if it is
 * not running.
 */
int kgpu_replay_serve_stages(kgpu_ctx *ctx, const kgpu_request *reqs, const uint64_t *arrival_ns, size_t n,
                             int64_t timeout_ns, uint64_t *latency_ns, uint64_t *wall_ns, int64_t *stages,
                             int64_t *clock_offset_ns);

/* ------------------------------------------------------------------------
 * One request at a time, with CPU/GPU dispatch by a measured crossover.
 *
 * The paper finds its GPU AES slower than the CPU's below a request size of
 * two pages, because a GPU request pays a fixed launch-and-copy cost, and
 * proposes measuring that crossover when the system starts and sending
 * smaller requests to the CPU (section 4).  kgpu_crypt is that dispatcher for
 * one request, in the paper's request model (section 3.2: build a request,
 * submit it, wait for it).  The host leg is AES-NI through OpenSSL's
 * libcrypto (version 3, loaded at run time); it is a separate implementation,
 * used only for requests whose every buffer is registered host memory, and
 * only when a context was created with kgpu_config.host_dispatch = 1 (or when
 * the caller forces it).
 * ---------------------------------------------------------------------- */

#define KGPU_DISPATCH_AUTO 0u /* host leg if enabled and len < the crossover, else GPU */
#define KGPU_DISPATCH_GPU 1u  /* always the GPU leg */
#define KGPU_DISPATCH_HOST 2u /* always the host leg (host-resident requests only) */

/*
 * Run one request (kgpu_request, any mode) and wait for it.  The GPU leg is
 * the serving ring when kgpu_serve_start has started it, otherwise one launch
 * of the mode's kernel on a stream of the context (the pages are read and
 * written in place, device memory or registered host memory alike).  The host
 * leg runs the request in the calling thread; it needs src and dst flagged
 * KGPU_REQ_SRC_HOST / KGPU_REQ_DST_HOST (and KGPU_REQ_IVS_HOST for CBC), else
 * KGPU_EINVAL.  With KGPU_DISPATCH_AUTO the host leg is taken when the context
 * was created with host_dispatch = 1, the request is host-resident in that
 * sense, and its length is below the measured crossover for its mode and key
 * size (AES-128 / AES-192 and AES-256 measured as AES-128 and AES-256).
 * Validation as kgpu_submit.  timeout_ns bounds the wait for admission to a
 * full serving ring (KGPU_ETIMEDOUT, nothing queued; < 0 waits without
 * limit); once the GPU has the request the call returns when it completes,
 * since it holds the caller's pages until then.  *ran_on (if not NULL)
 * receives KGPU_DISPATCH_GPU or KGPU_DISPATCH_HOST.  Returns the request's
 * status: 0, or a negative KGPU_E* code (KGPU_ENOSYS if the host leg was
 * forced and libcrypto is not available).
 */
int kgpu_crypt(kgpu_ctx *ctx, const kgpu_request *req, uint32_t dispatch, int64_t timeout_ns, uint32_t *ran_on);

/* Where kgpu_crypt's host leg stops: requests shorter than bytes[mode][k]
 * (mode KGPU_MODE_XTS..KGPU_MODE_ECB; k = 0 for AES-128, 1 for AES-256) run on
 * the host.  form: the GPU leg that was measured (KGPU_DISPATCH_FORM_*). */
#define KGPU_DISPATCH_FORM_LAUNCH 1u
#define KGPU_DISPATCH_FORM_RING 2u
typedef struct kgpu_crossover {
    uint64_t bytes[4][2];
    uint32_t form;
    uint32_t valid; /* 1 once measured */
} kgpu_crossover;

/* One measured point of the calibration: both legs' median time for one
 * request of `bytes` bytes, in registered pinned host memory. */
typedef struct kgpu_dispatch_point {
    uint32_t mode;     /* KGPU_MODE_XTS..KGPU_MODE_ECB */
    uint32_t key_bits; /* 128 or 256 */
    uint64_t bytes;
    uint64_t host_ns;
    uint64_t gpu_ns;
} kgpu_dispatch_point;

/*
 * Measure the crossover now: for XTS, CBC decryption, CBC encryption and
 * ECB, with AES-128 and AES-256 keys, and request sizes of 4 KiB to 4 MiB
 * (powers of two) in registered pinned host memory, time kgpu_crypt's host
 * leg and its GPU leg (the serving ring if it runs, else one launch) and
 * record, per mode and key size, the smallest size from which the GPU leg is
 * faster at every larger measured size (4 KiB if it is faster everywhere;
 * 8 MiB if the host leg is faster everywhere).  The context's table is
 * replaced, so call it again after kgpu_serve_start to route against the
 * ring.  points (if not NULL) receives up to max_points measured points and
 * *npoints their number (88 for the full sweep).  Allocates and frees its
 * own buffers and keys.  Takes about a second.  Errors: KGPU_ENOSYS (no
 * libcrypto), KGPU_ENOMEM, KGPU_EIO.
 */
int kgpu_calibrate_dispatch(kgpu_ctx *ctx, kgpu_dispatch_point *points, size_t max_points, size_t *npoints,
                            kgpu_crossover *out);

/* The context's current crossover table (valid = 0 before any calibration). */
int kgpu_get_crossover(kgpu_ctx *ctx, kgpu_crossover *out);

/* ------------------------------------------------------------------------
 * Allocation-free batched submission.  No counterpart in the paper.
 * ---------------------------------------------------------------------- */

#define KGPU_NOALLOC_MAX_REQUESTS 512
#define KGPU_NOALLOC_STAGE_WARPS 16
#define KGPU_NOALLOC_SCRATCH_BYTES 110592

/*
 * kgpu_submit for callers that cannot allocate memory when they call: for
 * example an OS-level caller on a page-writeback or memory-reclaim path, which
 * may need pages encrypted precisely because memory is short and whose
 * allocation could block on the very reclaim it serves, or a deployment whose
 * memory budget is fixed at start-up.  It runs the same persistent batch
 * kernel, but its scratch (work counter, per-request status words, device copy
 * of the descriptors, and KGPU_NOALLOC_STAGE_WARPS warps' 4-KiB staging areas
 * for CBC encryption of registered host pages) is one fixed array of
 * KGPU_NOALLOC_SCRATCH_BYTES of device memory inside the library image, which
 * every GPU that loads the library holds until the process exits; the
 * descriptors are packed in a fixed host array.  The call makes no
 * cudaMalloc/cudaFree or other allocating call.
 *
 * Arguments as kgpu_submit, without a ticket: the work is queued on `stream`
 * and the caller synchronises on that stream.  At most
 * KGPU_NOALLOC_MAX_REQUESTS requests per call: more is KGPU_E2BIG, with
 * nothing launched.  Validation as kgpu_submit (req_status, if not NULL,
 * receives each request's validation code).  kgpu_aes_delkey and
 * kgpu_host_unregister wait for batches queued here before they remove a key
 * or a range, as they do for kgpu_submit.  Batches run the launch shape set
 * with kgpu_set_tuning, else 512 threads and 16-KiB tiles, as kgpu_submit's
 * do.  A batch holding CBC encryption of host pages always runs the
 * 512-thread kernel, whose first
 * KGPU_NOALLOC_STAGE_WARPS warps stage those pages; the other warps run them
 * one lane per page (the same bytes, more link transfers).  The counter and
 * status words are cleared on every call, but every call shares the one
 * array: calls whose work overlaps on the GPU (on different streams, or from
 * different threads without ordering) race and corrupt each other -- order
 * them on one stream or synchronise in between.  A stream that is being
 * captured into a CUDA graph is refused (KGPU_EINVAL): the descriptors are
 * copied from a host array that the next call overwrites.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current).
 */
int kgpu_submit_noalloc(kgpu_ctx *ctx, const kgpu_request *reqs, size_t n, kgpu_stream stream, int *req_status);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* KGPU_H */
