/*
 * tdes.h -- C ABI of the GB300 (sm_103a) 3DES-EDE3 library libtdes_gb300.so.
 *
 * The operation is the one defined in "Bit-level Parallelization of 3DES
 * Encryption on GPU" (Altinok, Peker, Temizel), Sec. III:
 *   - key generation (Sec. III-A): PC-1, two 28-bit halves rotated left
 *     cumulatively by shift_keys, PC-2 -> 16 round keys per base key, for
 *     each of the three base keys;
 *   - DES (Sec. III-B): initial_perm, 16 rounds of expansion, round-key XOR,
 *     eight S-boxes, the per permutation and XOR into the left half, then the
 *     halves combined and final_perm; decryption reverses the round keys;
 *   - 3DES-EDE3 (Sec. III-B, the two equations):
 *       C = E_K3(D_K2(E_K1(P))),   P = D_K1(E_K2(D_K3(C))).
 * The paper encrypts files of independent 64-bit blocks in ECB mode (Sec. V);
 * CTR and CBC are the usual block-cipher modes built on the same cipher.
 *
 * Conventions shared by every call:
 *   - A block is 8 bytes, big-endian: bit 1 of the paper's numbering is the
 *     most significant bit of the first byte.  Keys use the same order; the
 *     parity bits (bit 8 of every byte) are ignored, as PC-1 drops them.
 *   - Data pointers are owned by the caller and must be addressable by the
 *     GPU with the same pointer: device memory of the device that was current
 *     when the key schedule was made, or page-locked host memory mapped into
 *     the device address space (cudaHostAlloc on a unified-address system;
 *     the kernels then read and write it over the host link, e.g.
 *     NVLink-C2C).  Single-message calls and server requests refuse other
 *     pointers with TDES_EINVAL; batch plans, which may hold millions of
 *     descriptors, trust the caller.  Pointers must be 8-byte aligned;
 *     16-byte aligned buffers take the fastest load path.
 *     `nbytes` must be a multiple of 8 (the paper's input consists of whole
 *     64-bit blocks); 0 is a valid empty call; one call takes less than
 *     2^31 tiles of 8 KiB (16 TiB), far above any GPU's memory.  in == out (in place) is
 *     allowed; any other overlap of the two ranges returns TDES_EINVAL.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) unless stated otherwise; the caller synchronises.
 *   - Every call returns TDES_OK (0) or a negative status and never aborts.
 *     tdes_last_error() gives a message for the last failure of the calling
 *     host thread.
 */
#ifndef TDES_GB300_H
#define TDES_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tdes_stream_t; /* same type as cudaStream_t */
typedef struct tdes_ks tdes_ks_t;          /* opaque, library-owned key schedule */

#define TDES_OK 0
#define TDES_EINVAL (-1)    /* bad argument: size, alignment, overlap, NULL, counter range */
#define TDES_ENOMEM (-2)    /* device allocation failed */
#define TDES_EBUSY (-3)     /* resource limit reached; retry later */
#define TDES_ETIMEDOUT (-4) /* a bounded wait ran out */
#define TDES_ECUDA (-5)     /* a CUDA runtime call failed; see tdes_last_error() */

/* Key schedule (Sec. III-A) for the triple K1, K2, K3 (8 bytes each).
 * Runs the key-schedule kernel on the current device and waits for it
 * (synchronous).  *out receives a handle holding, in device memory, the
 * round-constant tables of the bitsliced kernels for encryption and for
 * decryption (the decryption table is the round keys in reverse order,
 * Sec. III-B) and the six-bit round-key groups of the scalar path.  Weak
 * keys are accepted.  Free with tdes_key_free().
 *
 * A triple whose middle key equals one of its neighbours in the 56 bits the
 * key schedule uses (parity bits ignored) reduces EDE3 to one DES pass:
 * K1 = K2 gives DES under K3 (E_K3(D_K1(E_K1(x))) = E_K3(x)), K2 = K3 gives
 * DES under K1, and K1 = K2 = K3 gives DES under K (Sec. III-B).  Such a
 * triple gets a single-DES schedule: the same results, 16 rounds per block
 * instead of 48 (tdes_key_schedule_stages() reports 1). */
int tdes_key_schedule(const uint8_t k1[8], const uint8_t k2[8], const uint8_t k3[8],
                      tdes_ks_t **out);

/* Two-key 3DES: EDE3 under (k1, k2, k1).  Same as tdes_key_schedule(k1, k2,
 * k1, out). */
int tdes_key_schedule_2key(const uint8_t k1[8], const uint8_t k2[8], tdes_ks_t **out);

/* Single DES (Sec. III-A and the DES rounds of Sec. III-B) under the 8-byte
 * key k: the data calls below then compute DES_k with one 16-round pass per
 * block -- the result EDE3 gives under (k, k, k). */
int tdes_des_key_schedule(const uint8_t k[8], tdes_ks_t **out);

/* DES passes per block that data calls with this schedule run: 3 (EDE3) or
 * 1 (single DES).  TDES_EINVAL for NULL. */
int tdes_key_schedule_stages(const tdes_ks_t *ks);

/* Releases a key schedule (NULL is ignored).  The caller must ensure no
 * kernel that uses it is still running. */
void tdes_key_free(tdes_ks_t *ks);

/* ECB (the paper's mode, Sec. V): every 8-byte block of in[0, nbytes) is
 * encrypted (resp. decrypted) independently with EDE3 into out. */
int tdes_ecb_encrypt(const tdes_ks_t *ks, const void *in, void *out, size_t nbytes,
                     tdes_stream_t stream);
int tdes_ecb_decrypt(const tdes_ks_t *ks, const void *in, void *out, size_t nbytes,
                     tdes_stream_t stream);

/* CTR: out_i = in_i XOR E(nonce || ctr0 + i) for block i, where the counter
 * block is the 32-bit nonce followed by the 32-bit counter, both big-endian.
 * Encryption and decryption are the same call.  The counter never wraps:
 * ctr0 + nbytes/8 > 2^32 returns TDES_EINVAL. */
int tdes_ctr_crypt(const tdes_ks_t *ks, uint32_t nonce, uint32_t ctr0, const void *in,
                   void *out, size_t nbytes, tdes_stream_t stream);

/* CBC decryption: out_i = D(in_i) XOR in_{i-1}, with in_{-1} = iv (the
 * 64-bit IV serialised big-endian).  Parallel over blocks.  In place
 * (in == out) first snapshots the ciphertext block before every 8 KiB tile
 * into a stream-ordered temporary of 8 bytes per tile (cudaMallocAsync on
 * `stream`, freed on the same stream); TDES_ENOMEM if that fails. */
int tdes_cbc_decrypt(const tdes_ks_t *ks, uint64_t iv, const void *in, void *out,
                     size_t nbytes, tdes_stream_t stream);

/* CBC encryption: out_i = E(in_i XOR out_{i-1}), out_{-1} = iv.  Each block
 * depends on the previous one, so one warp walks the whole message (each
 * lane one bit of the round function; latency about 48 dependent rounds per
 * block, 16 for a single-DES schedule); batch many messages to get
 * throughput. */
int tdes_cbc_encrypt(const tdes_ks_t *ks, uint64_t iv, const void *in, void *out,
                     size_t nbytes, tdes_stream_t stream);

/* Allocation-free CBC decryption.  The paper has no counterpart: this is a
 * deployment variant of tdes_cbc_decrypt for callers that must not have the
 * library allocate device memory -- for example a server that reserves the
 * GPU's memory for its own pool at start-up and cannot let a request fail on
 * an allocation, or a host framework that gives its plugins pre-sized
 * buffers and forbids allocation on the hot path.  Same arguments and result
 * as tdes_cbc_decrypt.  An in-place call (in == out) saves the ciphertext
 * block before each 8 KiB tile in a fixed scratch array compiled into the
 * library (8 bytes per tile, TDES_NOALLOC_MAX_TILES tiles = 1 MiB of device
 * memory, held on every device that loads the library until the process
 * exits); in-place calls larger than TDES_NOALLOC_MAX_BYTES return
 * TDES_EINVAL.  Out-of-place calls use no scratch and have no size limit
 * beyond the 2^31 tiles of every call.
 * The call never calls cudaMalloc, cudaFree or any allocating routine.
 * The first in-place call of more than one tile on each device looks up the
 * scratch array's device address (cudaGetSymbolAddress) with that device
 * current, and looks it up again after the device's context changes (e.g.
 * after cudaDeviceReset); make that first call before any stream capture.
 * The size checks come before any device query, so an oversized call is
 * refused without touching the device.  All calls share the one array: two in-place
 * calls that overlap in time on the GPU (different streams, no ordering
 * between them) race on it and may return wrong plaintext.  Nothing in the
 * array needs clearing: each call writes every entry it reads first. */
#define TDES_NOALLOC_MAX_TILES 131072
#define TDES_NOALLOC_MAX_BYTES ((uint64_t)TDES_NOALLOC_MAX_TILES * 8192u)
int tdes_cbc_decrypt_noalloc(const tdes_ks_t *ks, uint64_t iv, const void *in, void *out,
                             size_t nbytes, tdes_stream_t stream);

/* Host-buffer ECB: encrypts (decrypt == 0) or decrypts host memory
 * host_in[0, nbytes) into host_out, streaming it through the caller's device
 * buffer dev_buf of dev_bytes bytes (16-byte aligned, at least 4 x 32 KiB,
 * used as 4 to 16 rotating parts of about 32 MiB): host-to-device copies,
 * the kernel and device-to-host copies of successive chunks overlap on
 * internal streams.  Host buffers should be pinned (cudaHostAlloc /
 * page-locked) for full copy speed.  Synchronous: returns when host_out is
 * complete.  in == out is allowed. */
int tdes_ecb_crypt_host(const tdes_ks_t *ks, int decrypt, const void *host_in, void *host_out,
                        size_t nbytes, void *dev_buf, size_t dev_bytes);

/* ------------------------------------------------------------------------
 * Batches: many messages, each with its own key triple and mode, in one
 * persistent launch.  Not in the paper (which encrypts one file under one
 * key triple in ECB, Sec. V); the cipher of every message is the same EDE3.
 * ------------------------------------------------------------------------ */

#define TDES_MODE_ECB_ENCRYPT 0u
#define TDES_MODE_ECB_DECRYPT 1u
#define TDES_MODE_CTR 2u          /* counter blocks: iv_or_ctr + i on the low 32 bits */
#define TDES_MODE_CBC_DECRYPT 3u
#define TDES_MODE_CBC_ENCRYPT 4u

typedef struct tdes_keytable tdes_keytable_t; /* opaque: device-resident key schedules */
typedef struct tdes_batch tdes_batch_t;       /* opaque: a planned batch */

/* One message of a batch.  in/out: device pointers, 8-byte aligned, equal
 * (in place) or disjoint; nbytes a multiple of 8 (0 = nothing to do).
 * iv_or_ctr: the CBC IV, or for CTR the first counter block
 * (nonce << 32 | ctr0; block i uses nonce || ctr0 + i, which must not pass
 * 2^32).  Messages of one batch must not overlap each other. */
typedef struct {
    uint32_t mode;      /* TDES_MODE_* */
    uint32_t key_index; /* key triple in the key table */
    uint64_t iv_or_ctr;
    const void *in;
    void *out;
    uint64_t nbytes;
} tdes_desc_t;

typedef struct {
    uint32_t n_cbc_enc_messages; /* serial chains, one GPU lane or warp each */
    uint64_t n_tiles;            /* bitsliced 1024-block tiles of large messages */
    uint32_t n_small_items;      /* warp items of small (<= 32-block) messages, one block
                                    per lane (batches with few small messages) */
    int warps_per_cta;
    int ctas_per_sm;
    uint64_t bytes_per_mode[5];  /* payload bytes, indexed by TDES_MODE_* */
    uint64_t n_mixed_tiles;      /* bitsliced tiles of small messages under up to 32 keys
                                    (batches with 8192 or more small-message blocks) */
    uint32_t n_direct_messages;  /* messages of 64 MiB or more (ECB, CTR, out-of-place CBC
                                    decryption) run by the single-key kernels */
    int tiles_per_claim;         /* tiles a warp claims at once (the automatic choice resolved) */
    int round_form;              /* TDES_ROUNDS_PER_PASS or TDES_ROUNDS_COMPACT */
    int tuned;                   /* 1: the shape came from the autotuner's cache at planning */
} tdes_batch_info_t;

/* Launch shape of a batch's kernels, i.e. what the autotuner searches.  A
 * shape changes how the work is spread over the GPU, never the result. */
#define TDES_ROUNDS_PER_PASS 0 /* the 48 rounds as three loops, one per DES pass */
#define TDES_ROUNDS_COMPACT 1  /* one loop body for all three passes (a third of the code) */
typedef struct {
    int warps_per_cta;   /* 1..8; each warp owns a 13 KB shared-memory slice */
    int ctas_per_sm;     /* resident CTAs per SM in the persistent grid; <= 0: as many as fit
                            (the grid is SMs x this) */
    int tiles_per_claim; /* 1024-block tiles a warp takes from the work counter per claim,
                            i.e. blocks per warp claim / 1024; 0: automatic (1, or 4 when
                            the batch has over 256 tiles per warp); at most 1024 */
    int round_form;      /* TDES_ROUNDS_PER_PASS or TDES_ROUNDS_COMPACT */
} tdes_launch_shape_t;

/* Key schedules (Sec. III-A) of `count` triples (keys: count x 24 bytes,
 * K1||K2||K3 each) computed by the key-schedule kernels and kept in device
 * memory (28225 bytes per triple: the bitsliced tables of both directions,
 * their one-bit-per-word copies for tiles that mix keys, and the scalar
 * round-key groups) on the current device.  Synchronous.  The raw keys are
 * not kept.  Free with tdes_keytable_free(). */
int tdes_keytable_create(const uint8_t *keys, uint32_t count, tdes_keytable_t **out);
void tdes_keytable_free(tdes_keytable_t *kt);

/* Validates `count` descriptors and lays the batch out in device memory
 * (synchronous; the plan can be launched many times).  per_desc_status
 * (nullable, count entries) receives TDES_OK or TDES_EINVAL per descriptor:
 * bad mode, key index, size, alignment, overlap or CTR counter range.
 * Rejected descriptors are skipped; the call still returns TDES_OK with the
 * plan of the valid ones (tdes_last_error() then counts the rejections).
 * Messages are classified: CBC encryption (serial chains), large messages
 * (more than 32 blocks: bitsliced tiles) and small ones (scalar blocks).
 * Messages of 64 MiB or more in ECB, CTR or out-of-place CBC decryption run
 * through the single-key kernels, launched ahead of the batch kernels in
 * the same launch (and the same CUDA graph). */
int tdes_batch_plan(const tdes_keytable_t *kt, const tdes_desc_t *descs, uint32_t count,
                    int *per_desc_status, tdes_batch_t **out);

/* Launch shape of the persistent kernel: warps per CTA (1..8; each warp owns
 * a 13 KB shared-memory slice) and CTAs per SM (<= 0: as many as fit); the
 * shape's other fields are kept. */
int tdes_batch_configure(tdes_batch_t *b, int warps_per_cta, int ctas_per_sm);

/* Sets (TDES_EINVAL outside the ranges of tdes_launch_shape_t) or reads a
 * plan's whole launch shape.  A plan starts in the shape the autotuner's
 * cache holds for its workload class (see tdes_batch_autotune), else in the
 * default shape: 8 warps per CTA, as many CTAs as fit, automatic tiles per
 * claim, TDES_ROUNDS_COMPACT.  Setting a shape drops the plan's captured
 * graph, which tdes_batch_launch_graph then captures again. */
int tdes_batch_set_shape(tdes_batch_t *b, const tdes_launch_shape_t *shape);
int tdes_batch_get_shape(const tdes_batch_t *b, tdes_launch_shape_t *shape);

/* Runs the whole batch on `stream`: one persistent launch whose warps claim
 * work items from an atomic counter (preceded by a small snapshot launch
 * when a large message is CBC-decrypted in place).  Asynchronous.  Two
 * launches of one plan must not run at the same time (they share its claim
 * counter and snapshot buffer): queue them on one stream or order them with
 * events.  tdes_batch_submit_plan does this itself within a context. */
int tdes_batch_launch(tdes_batch_t *b, tdes_stream_t stream);

/* The same work as one CUDA graph: captured on first use (and after
 * tdes_batch_configure), replayed by later calls.  Asynchronous. */
int tdes_batch_launch_graph(tdes_batch_t *b, tdes_stream_t stream);

int tdes_batch_info(const tdes_batch_t *b, tdes_batch_info_t *info);

/* Frees a plan; no launch of it may still be running. */
void tdes_batch_free(tdes_batch_t *b);

/* ------------------------------------------------------------------------
 * Autotuner.  Not in the paper: it picks the launch shape (warps per CTA,
 * CTAs per SM, i.e. grid size, tiles per claim, i.e. blocks per warp claim,
 * and the round loop's form) of the batch kernels by timing them, and keeps
 * the winner in a cache file keyed by workload class, which every later plan
 * (tdes_batch_plan, tdes_batch_submit) and server (tdes_server_config_default)
 * reads.  The class is the GPU's SM count, the share of the payload in each
 * kind of work (bitsliced tiles, mixed-key tiles, one-block-per-lane items,
 * CBC-encryption chains, graded 0..3) and the floor of log2 of the payload.
 * The cache file is TDES_AUTOTUNE_CACHE when that environment variable is
 * set, else $XDG_CACHE_HOME/tdes_gb300/autotune.jsonl, else
 * $HOME/.cache/tdes_gb300/autotune.jsonl: JSON lines, the last line of a
 * class winning.
 * ------------------------------------------------------------------------ */

typedef struct {
    char key[64];                  /* workload class */
    tdes_launch_shape_t best;      /* the shape chosen */
    tdes_launch_shape_t baseline;  /* the default shape */
    double best_ms, baseline_ms;   /* median device time per launch (CUDA events on `stream`);
                                      from the cache when from_cache is 1 */
    uint32_t candidates;           /* shapes timed (0 when taken from the cache) */
    int from_cache;
} tdes_autotune_result_t;

#define TDES_TUNE_FORCE 1u    /* time the candidates even if the cache has the class */
#define TDES_TUNE_NO_STORE 2u /* leave the cache file unchanged */

/* Tunes the launch shape of plan b: a coordinate search, timing `reps`
 * launches (after one warm-up launch) of each candidate on `stream` with
 * CUDA events -- (warps per CTA, CTAs per SM) over 4 and 8 warps and the
 * fitting CTA counts, then tiles per claim over 0, 1, 2, 4 and 8, then the
 * round form -- and a final alternating re-timing of the best against the
 * default shape, which is kept unless the best is faster.  The plan is left
 * in the chosen shape and, unless TDES_TUNE_NO_STORE, the choice is appended
 * to the cache.  If the cache already has b's class and TDES_TUNE_FORCE is
 * not set, that shape is applied without timing.  Synchronous (waits for
 * the device).  The plan's whole work runs (reps + 1) times per candidate:
 * every output is rewritten each time, so messages processed in place are
 * transformed again and again -- tune on a plan whose outputs are scratch,
 * or out of place with inputs left intact. */
int tdes_batch_autotune(tdes_batch_t *b, unsigned flags, int reps, tdes_stream_t stream,
                        tdes_autotune_result_t *res);

/* Path of the cache file in use (valid until the next call on this thread). */
const char *tdes_autotune_cache_path(void);

/* ------------------------------------------------------------------------
 * Batch contexts: submit, poll, wait.  The paper states the problem as
 * plaintext of 64-bit blocks, three 64-bit keys and a mode (Sec. IV-B,
 * IV-C); a batch is many such problems at once, each message with its own
 * key triple (an index into the context's key table) and mode, and a ticket
 * tells the caller when its batch is done without blocking on the device.
 * ------------------------------------------------------------------------ */

typedef struct tdes_ctx tdes_ctx_t; /* opaque */

typedef struct {
    uint32_t streams; /* batches in flight at once, each on its own stream (1..16) */
} tdes_ctx_config_t;

/* Defaults: 2 streams. */
void tdes_ctx_config_default(tdes_ctx_config_t *cfg);

/* A context on the current device over key table kt (which must outlive
 * it), owning its streams.  TDES_EINVAL if kt lives on another device. */
int tdes_ctx_create(const tdes_keytable_t *kt, const tdes_ctx_config_t *cfg, tdes_ctx_t **out);

/* Waits for every batch the context queued, then frees it and its tickets. */
void tdes_ctx_destroy(tdes_ctx_t *ctx);

/* Plans `count` descriptors as tdes_batch_plan does (rejected descriptors
 * are skipped and reported by tdes_batch_poll), queues the batch's work on
 * one of the context's streams -- a stream with nothing in flight if there
 * is one -- and returns without waiting for the device.  The plan is copied
 * into stream-ordered device memory (cudaMallocAsync) that returns to the
 * pool when the batch's kernels are done; the launch shape is the
 * autotuner's for the batch's class if the cache has one.  The context's
 * streams are non-blocking: they do not wait for work the caller queued
 * elsewhere (the legacy default stream included), so inputs must be ready
 * before the call.  Buffers must stay valid, and must not be touched by
 * other work, until the ticket completes.
 * *ticket identifies the batch (tickets increase by one per submission).
 * TDES_EINVAL for NULL arguments or a context of another device;
 * TDES_ENOMEM / TDES_ECUDA if queueing failed (no ticket is issued). */
int tdes_batch_submit(tdes_ctx_t *ctx, const tdes_desc_t *descs, uint32_t count,
                      uint64_t *ticket);

/* The same for a batch planned by tdes_batch_plan (it must use the
 * context's key table): its CUDA graph is replayed on a context stream.
 * A plan submitted again while its previous ticket is pending is queued on
 * that ticket's stream, behind it, so the two runs never overlap.
 * The plan must not be freed or reconfigured before the ticket completes. */
int tdes_batch_submit_plan(tdes_ctx_t *ctx, tdes_batch_t *b, uint64_t *ticket);

/* Non-blocking.  Returns 1 while the batch is pending (also for a ticket not
 * issued yet), and once it is done TDES_OK if every descriptor ran, else the
 * first rejected descriptor's status (TDES_EINVAL), or TDES_ECUDA if the
 * batch failed on the device.  per_desc_status (nullable; as many entries as
 * the batch had descriptors) receives per descriptor: 0 done, 1 pending, or
 * < 0 (TDES_EINVAL: rejected at submission and skipped; TDES_ECUDA).
 * TDES_EINVAL for a released ticket. */
int tdes_batch_poll(tdes_ctx_t *ctx, uint64_t ticket, int *per_desc_status);

/* Waits at most timeout_ns for a ticket, sleeping between polls (from 2 us
 * doubling up to 1 ms); returns tdes_batch_poll's final status or
 * TDES_ETIMEDOUT.  Never hangs. */
int tdes_batch_wait(tdes_ctx_t *ctx, uint64_t ticket, uint64_t timeout_ns);

/* Forgets a completed ticket (its per-descriptor statuses); TDES_EBUSY
 * while it is pending.  Tickets are otherwise kept until tdes_ctx_destroy. */
int tdes_batch_release(tdes_ctx_t *ctx, uint64_t ticket);

/* ------------------------------------------------------------------------
 * Uniform messages: n_msgs messages of msg_bytes each, back to back (message
 * i is bytes [i * msg_bytes, (i + 1) * msg_bytes) of in and of out), each
 * under its own key triple and mode, planned and run on the device.  Not in
 * the paper (one file under one triple in ECB, Sec. V); every message gets
 * the same EDE3 (Sec. III-B) in the mode of TDES_MODE_*, as in a batch.
 * Meant for very many small messages, where host-side descriptors
 * (tdes_batch_plan) would not fit: messages are sorted by (key, mode class)
 * on the device, full groups run in single-key bitsliced tiles, the rest in
 * tiles that mix 32 keys, and CBC encryption runs 1024 (or 32 x 32) chains
 * per tile, one bitsliced pass per block position.
 * ------------------------------------------------------------------------ */

#define TDES_UNIFORM_MAX_MSGS (1ull << 31)

/* Device scratch the call needs for n_msgs messages of msg_bytes under the
 * key table kt: 4 to 8 bytes per message (more for longer messages, whose
 * slices hold fewer messages), about 100 bytes per key triple and 25 MB
 * (1.42 GB for 2^28 messages of 64 bytes under 65536 triples).
 * TDES_EINVAL for a msg_bytes that is not a multiple of 8 in [8, 256] or
 * n_msgs > TDES_UNIFORM_MAX_MSGS. */
int tdes_uniform_scratch_bytes(const tdes_keytable_t *kt, uint64_t n_msgs, uint64_t msg_bytes,
                               size_t *bytes);

/* Encrypts or decrypts every message, asynchronously on `stream`; no host
 * synchronisation and no allocation, so the call can be captured in a CUDA
 * graph.  Device arrays of n_msgs entries: key_index (index into kt, 4-byte
 * aligned), mode (TDES_MODE_*, one byte each), iv_or_ctr (8-byte aligned;
 * CBC IV, or for CTR nonce << 32 | ctr0 as in tdes_desc_t).  in / out:
 * device pointers, 8-byte aligned, equal (in place) or disjoint.  scratch:
 * device memory of at least tdes_uniform_scratch_bytes(), 256-byte aligned,
 * owned by the caller and not shared with a concurrent call; its contents
 * need no initialisation.  Messages with a key index >= the table's count,
 * a mode > TDES_MODE_CBC_ENCRYPT or a CTR counter that would pass 2^32 are
 * skipped (their output bytes are not written); their number is written to
 * *skipped (device memory, 8-byte aligned, nullable) by the end of the
 * call's work.  Returns TDES_EINVAL for bad arguments before any work is
 * queued. */
int tdes_uniform_crypt(const tdes_keytable_t *kt, const uint32_t *key_index, const uint8_t *mode,
                       const uint64_t *iv_or_ctr, const void *in, void *out, uint64_t msg_bytes,
                       uint64_t n_msgs, void *scratch, size_t scratch_bytes,
                       uint64_t *skipped, tdes_stream_t stream);

typedef struct {
    uint64_t skipped;          /* messages skipped (see tdes_uniform_crypt) */
    uint32_t key_tiles;        /* single-key tiles of ECB / CTR / CBC-decrypt messages */
    uint32_t mixed_slices;     /* mixed-key slices of such messages (32 per tile) */
    uint32_t chain_key_tiles;  /* single-key tiles of 1024 CBC-encryption chains */
    uint32_t chain_slices;     /* mixed-key slices of up to 32 CBC-encryption chains */
} tdes_uniform_info_t;

/* The plan of the last call that used `scratch`, read back synchronously
 * (waits for the device). */
int tdes_uniform_info(const void *scratch, tdes_uniform_info_t *info);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of individual requests.  Not in the paper.
 * ------------------------------------------------------------------------ */

typedef struct tdes_server tdes_server_t; /* opaque */

typedef struct {
    uint64_t budget_bytes;   /* HBM admission budget: input + output bytes of the requests
                                admitted and not yet complete (in place counts once) */
    uint32_t slots;          /* batches in flight at once, each on its own stream */
    uint32_t max_batch;      /* requests per batch at most */
    int warps_per_cta;       /* persistent-kernel shape, 1..8 */
    int reserve_ctas_per_sm; /* with slots > 1: CTAs per SM a batch leaves for the next one */
    uint32_t ring_entries;   /* completion records kept; older tickets read as complete */
    uint64_t stage_bytes;    /* device staging per slot for requests in host memory (default
                                0: none).  A request whose buffers are pinned host memory and
                                that has at least stage_min_bytes is copied in, processed and
                                copied out on its batch's stream, so the copies of one batch
                                overlap the kernels of the others; smaller ones, and any that
                                do not fit the slot's staging, are read and written by the
                                kernels over the host link (which gave the higher closed-loop
                                throughput on a GB300) */
    uint64_t stage_min_bytes;
    int round_form;          /* TDES_ROUNDS_PER_PASS or TDES_ROUNDS_COMPACT (batch kernel's rounds) */
} tdes_server_config_t;

/* Defaults: 8 GiB budget, 4 slots, 16384 requests per batch, 4 warps per CTA,
 * 1 CTA per SM reserved, 2^21 completion records, TDES_ROUNDS_PER_PASS --
 * except that slots, warps per CTA, reserved CTAs and the round form come
 * from the autotune cache when it has an entry for the current device's SM
 * count (tdes_server_autotune). */
void tdes_server_config_default(tdes_server_config_t *cfg);

/* Starts a server on the current device over a key table (which must
 * outlive it).  A dispatcher thread admits queued requests in arrival order
 * while the admitted bytes stay within the budget, plans each admitted group
 * into one persistent batch launch on a free slot, and records completions;
 * requests arriving while batches run go into the next free slot.  A batch
 * completes as a whole, so a CBC-encryption request of more than 512 blocks
 * (one serial chain, about a microsecond per block) is batched alone and
 * holds up no other request.  For 200 us after its last progress (a batch
 * dispatched or completed) the dispatcher polls without sleeping; after that
 * it sleeps until a submission when nothing is in flight, and otherwise
 * polls in naps (5 us doubling to 100 us, ended early by a submission). */
int tdes_server_create(const tdes_keytable_t *kt, const tdes_server_config_t *cfg,
                       tdes_server_t **out);

/* Queues one request (same rules as a batch descriptor; device buffers must
 * stay valid until it completes).  Never blocks: *ticket identifies it.
 * TDES_EINVAL for a bad descriptor or one larger than the whole budget. */
int tdes_server_submit(tdes_server_t *s, const tdes_desc_t *req, uint64_t *ticket);

/* 0 complete, 1 pending, < 0 the request failed. */
int tdes_server_poll(tdes_server_t *s, uint64_t ticket);

/* Waits (bounded) for a ticket: its status, or TDES_ETIMEDOUT; never hangs.
 * The thread sleeps until the dispatcher signals a completion (at most 1 ms
 * per sleep).  A ticket not issued yet reads as pending. */
int tdes_server_wait(tdes_server_t *s, uint64_t ticket, uint64_t timeout_ns);

/* A group of `count` (>= 1) requests under one ticket.  Every descriptor is
 * checked as by tdes_server_submit first; if any is refused the call
 * returns TDES_EINVAL and queues none.  The requests are then admitted and
 * batched like single submissions (they may run in different batches).
 * *ticket identifies the group (its requests hold tickets ticket ..
 * ticket + count - 1, usable with tdes_server_poll). */
int tdes_server_submit_group(tdes_server_t *s, const tdes_desc_t *reqs, uint32_t count,
                             uint64_t *ticket);

/* 0 when every request of the group is complete, 1 while any is pending,
 * < 0 the first failed request's status.  per_desc_status (nullable, count
 * entries) receives each request's tdes_server_poll result. */
int tdes_server_poll_group(tdes_server_t *s, uint64_t ticket, uint32_t count,
                           int *per_desc_status);

/* Waits (bounded) for a whole group: its tdes_server_poll_group result, or
 * TDES_ETIMEDOUT; never hangs. */
int tdes_server_wait_group(tdes_server_t *s, uint64_t ticket, uint32_t count,
                           uint64_t timeout_ns);

/* Finishes every queued and running request, then stops the server. */
void tdes_server_destroy(tdes_server_t *s);

/* Open-loop load generator for a server.  Draws n_requests requests from a
 * seeded SplitMix64 stream: with probability small_frac a size uniform in
 * [small_min, small_max], else log-uniform in [large_min, large_max] (both
 * rounded down to multiples of 8); mode ECB-encrypt / CTR / CBC-decrypt with
 * mode_probs; key index uniform below n_keys; input at a random 16-byte
 * aligned offset of in_pool; output in a ring over out_pool whose regions
 * are reused only after their previous request completed.  Arrivals are
 * Poisson at offered_gbps of payload (<= 0: all at once, i.e. saturation).
 * Latency = completion time seen by the dispatcher - scheduled arrival. */
typedef struct {
    uint64_t n_requests;
    double offered_gbps;
    uint64_t seed;
    double small_frac;
    uint32_t small_min, small_max;
    uint64_t large_min, large_max;
    double mode_probs[3];
    uint32_t n_keys;
    const void *in_pool;
    uint64_t in_pool_bytes;
    void *out_pool;
    uint64_t out_pool_bytes;
} tdes_loadtest_config_t;

typedef struct {
    double p50_ms, p90_ms, p99_ms, p999_ms, mean_ms, max_ms;
    double small_p50_ms, small_p99_ms, large_p50_ms, large_p99_ms;
    double gbps;          /* payload bytes / (last completion - start) */
    double offered_gbps;
    double duration_s;
    uint64_t requests, bytes, batches;
    uint32_t max_slots_busy;     /* tdes_server_stats over this run */
    uint32_t max_device_overlap;
    double device_overlap_frac;  /* device_overlap_ms / device_busy_ms */
} tdes_loadtest_result_t;

int tdes_serve_loadtest(tdes_server_t *s, const tdes_loadtest_config_t *cfg,
                        tdes_loadtest_result_t *res);

/* Overlap of a server's batches.  A batch is "in flight" from its dispatch
 * to the dispatcher's noticing its completion event, and "on the device"
 * from the start of its first kernel's first CTA to the end of its last
 * kernel's last warp: times the kernels read from the GPU's global timer
 * and write to a ring of the last 2^20 batches (no per-batch host work). */
typedef struct {
    uint64_t batches;            /* batches completed (and timed) since the last reset */
    uint32_t max_slots_busy;     /* most batches in flight at once */
    uint32_t max_device_overlap; /* most batches on the device at one instant */
    double device_busy_ms;       /* time with at least one batch on the device */
    double device_overlap_ms;    /* time with two or more batches on the device */
    double batch_ms_sum;         /* sum of the batches' times on the device */
    uint64_t untimed_batches;    /* batches that failed, or whose times the ring lost */
} tdes_server_stats_t;

/* Statistics since the server started or since the last call with reset != 0
 * (which clears them after reading).  tdes_serve_loadtest resets them when
 * it starts. */
int tdes_server_stats(tdes_server_t *s, int reset, tdes_server_stats_t *out);

/* Autotuner of the server's shape (warps per CTA, CTAs per SM each batch
 * leaves free for the next, slots, round form) for the request mix of `load`
 * (its offered_gbps is ignored).  A shape's score is its p99 latency at one
 * offered load for all candidates, 95% of the built-in default's closed-loop
 * throughput, among the shapes that keep at least 97% of that throughput
 * closed-loop; each figure is the median of three tdes_serve_loadtest runs
 * on a fresh server.  Coordinate search over warps 2, 4, 8, reserved CTAs 1,
 * 2 (at least one CTA per SM stays free so that a new batch can start while
 * others run), slots 2, 4, 8 and the two round forms, then the best against
 * the built-in default (4 warps, 1 reserved CTA, 4 slots, per-pass rounds),
 * alternating, kept only if better.  "Better" on p99 means lower by more than
 * 3%, so that shapes within run-to-run spread of each other do not replace
 * one another.  Unless TDES_TUNE_NO_STORE, the choice is
 * appended to the autotune cache, from which tdes_server_config_default takes
 * it on this kind of GPU.  If the cache already has it and TDES_TUNE_FORCE is
 * not set, nothing is timed.  The load tests write into load->out_pool. */
typedef struct {
    char key[64];
    tdes_server_config_t best;     /* the default configuration with the tuned fields */
    tdes_server_config_t baseline; /* the built-in default */
    double best_gbps, baseline_gbps; /* closed-loop throughput */
    uint32_t candidates;
    int from_cache;
    double best_p99_ms, baseline_p99_ms; /* p99 at load_gbps (0 when from the cache) */
    double load_gbps;
} tdes_server_autotune_result_t;

int tdes_server_autotune(const tdes_keytable_t *kt, const tdes_loadtest_config_t *load,
                         unsigned flags, tdes_server_autotune_result_t *res);

/* Number of LOP3 instructions the eight generated S-box circuits take per
 * round, i.e. per 32 blocks per round (the circuit size fixed at build time). */
int tdes_sbox_gate_count(void);

/* Small calls.  ECB, CTR and CBC-decryption calls of at most this many
 * blocks run one block per GPU thread (the scalar round: latency of 48
 * dependent rounds, 16 for single DES) instead of bitsliced tiles of 1024
 * blocks (latency of a whole tile, however few blocks it holds).  In-place
 * CBC decryption takes that path only up to 1024 blocks.  Results are
 * identical either way.  Process-wide; the default, TDES_SMALL_CUTOFF_DEFAULT,
 * is about where the two paths take equally long on GB300.  0 sends every
 * call to the bitsliced kernels.  Returns the previous value. */
#define TDES_SMALL_CUTOFF_DEFAULT 196608u
uint64_t tdes_set_small_cutoff(uint64_t nblocks);

/* Short English text of a status code. */
const char *tdes_strerror(int status);

/* Message of the last failure on the calling host thread ("" if none). */
const char *tdes_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TDES_GB300_H */
