/*
 * tdes_oracle.c -- plain, slow, single-threaded CPU oracle for 3DES-EDE3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library under paper_2007_10752_gb300/) never calls it, and the
 * two share no code, headers or tables.
 *
 * It follows "Bit-level Parallelization of 3DES Encryption on GPU"
 * (Altinok, Peker, Temizel) step by step:
 *   - key generation, Sec. III-A (PC-1, 28/28 split, cumulative left
 *     rotations by shift_keys, PC-2), run once per base key;
 *   - DES encryption, Sec. III-B (initial_perm, 16 rounds of exp_d /
 *     round-key XOR / S-boxes / per / XOR into the left half / swap, then
 *     the halves combined and final_perm);
 *   - decryption = the same steps with the round keys in reverse order
 *     (Sec. III-B, paragraph after the encryption steps);
 *   - 3DES-EDE3: C = E_K3(D_K2(E_K1(P))), P = D_K1(E_K2(D_K3(C)))
 *     (Sec. III-B, the two 3DES equations).
 * Like the paper's memory design (Sec. IV-C) every bit is held in its own
 * byte, and every table is indexed 1-based exactly as printed in the
 * appendix ("the 57th bit of the original key becomes the 1st bit").
 *
 * Readings taken where the paper is silent or garbled:
 *   - bit 1 of a 64-bit block or key is the most significant bit of its
 *     first byte (blocks are big-endian byte strings);
 *   - the S-box row is 2*b1 + b6 and the column b2b3b4b5, both counted
 *     from 0 (the worked example in Sec. III-B prints "row 2" for outer
 *     bits 01; we read it as the second row, index 1);
 *   - after round 16 the halves are combined as R16 || L16 (the last swap
 *     is undone), which is the only order for which decryption with
 *     reversed round keys inverts encryption;
 *   - modes other than ECB are not in the paper (it uses ECB only,
 *     Sec. V); CTR and CBC follow the usual definitions:
 *       CTR: O_i = P_i XOR E(nonce32 || ctr32), ctr32 = ctr0 + i, both
 *            32-bit halves big-endian; the counter never wraps;
 *       CBC: C_i = E(P_i XOR C_{i-1}),  P_i = D(C_i) XOR C_{i-1},
 *            C_{-1} = IV (64-bit, serialised big-endian).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <pthread.h>

#include "tdes_oracle.h"

/* ---- Appendix A tables, transcribed as printed (1-indexed entries) ---- */

static const unsigned char pc_1[56] = {
    57, 49, 41, 33, 25, 17, 9,  1,  58, 50, 42, 34, 26, 18,
    10, 2,  59, 51, 43, 35, 27, 19, 11, 3,  60, 52, 44, 36,
    63, 55, 47, 39, 31, 23, 15, 7,  62, 54, 46, 38, 30, 22,
    14, 6,  61, 53, 45, 37, 29, 21, 13, 5,  28, 20, 12, 4};

static const int shift_keys[16] = {1, 1, 2, 2, 2, 2, 2, 2,
                                   1, 2, 2, 2, 2, 2, 2, 1};

static const unsigned char pc_2[48] = {
    14, 17, 11, 24, 1,  5,  3,  28, 15, 6,  21, 10,
    23, 19, 12, 4,  26, 8,  16, 7,  27, 20, 13, 2,
    41, 52, 31, 37, 47, 55, 30, 40, 51, 45, 33, 48,
    44, 49, 39, 56, 34, 53, 46, 42, 50, 36, 29, 32};

static const unsigned char initial_perm[64] = {
    58, 50, 42, 34, 26, 18, 10, 2, 60, 52, 44, 36, 28, 20, 12, 4,
    62, 54, 46, 38, 30, 22, 14, 6, 64, 56, 48, 40, 32, 24, 16, 8,
    57, 49, 41, 33, 25, 17, 9,  1, 59, 51, 43, 35, 27, 19, 11, 3,
    61, 53, 45, 37, 29, 21, 13, 5, 63, 55, 47, 39, 31, 23, 15, 7};

static const unsigned char exp_d[48] = {
    32, 1,  2,  3,  4,  5,  4,  5,  6,  7,  8,  9,
    8,  9,  10, 11, 12, 13, 12, 13, 14, 15, 16, 17,
    16, 17, 18, 19, 20, 21, 20, 21, 22, 23, 24, 25,
    24, 25, 26, 27, 28, 29, 28, 29, 30, 31, 32, 1};

static const unsigned char s[8][4][16] = {
    {{14, 4, 13, 1, 2, 15, 11, 8, 3, 10, 6, 12, 5, 9, 0, 7},
     {0, 15, 7, 4, 14, 2, 13, 1, 10, 6, 12, 11, 9, 5, 3, 8},
     {4, 1, 14, 8, 13, 6, 2, 11, 15, 12, 9, 7, 3, 10, 5, 0},
     {15, 12, 8, 2, 4, 9, 1, 7, 5, 11, 3, 14, 10, 0, 6, 13}},
    {{15, 1, 8, 14, 6, 11, 3, 4, 9, 7, 2, 13, 12, 0, 5, 10},
     {3, 13, 4, 7, 15, 2, 8, 14, 12, 0, 1, 10, 6, 9, 11, 5},
     {0, 14, 7, 11, 10, 4, 13, 1, 5, 8, 12, 6, 9, 3, 2, 15},
     {13, 8, 10, 1, 3, 15, 4, 2, 11, 6, 7, 12, 0, 5, 14, 9}},
    {{10, 0, 9, 14, 6, 3, 15, 5, 1, 13, 12, 7, 11, 4, 2, 8},
     {13, 7, 0, 9, 3, 4, 6, 10, 2, 8, 5, 14, 12, 11, 15, 1},
     {13, 6, 4, 9, 8, 15, 3, 0, 11, 1, 2, 12, 5, 10, 14, 7},
     {1, 10, 13, 0, 6, 9, 8, 7, 4, 15, 14, 3, 11, 5, 2, 12}},
    {{7, 13, 14, 3, 0, 6, 9, 10, 1, 2, 8, 5, 11, 12, 4, 15},
     {13, 8, 11, 5, 6, 15, 0, 3, 4, 7, 2, 12, 1, 10, 14, 9},
     {10, 6, 9, 0, 12, 11, 7, 13, 15, 1, 3, 14, 5, 2, 8, 4},
     {3, 15, 0, 6, 10, 1, 13, 8, 9, 4, 5, 11, 12, 7, 2, 14}},
    {{2, 12, 4, 1, 7, 10, 11, 6, 8, 5, 3, 15, 13, 0, 14, 9},
     {14, 11, 2, 12, 4, 7, 13, 1, 5, 0, 15, 10, 3, 9, 8, 6},
     {4, 2, 1, 11, 10, 13, 7, 8, 15, 9, 12, 5, 6, 3, 0, 14},
     {11, 8, 12, 7, 1, 14, 2, 13, 6, 15, 0, 9, 10, 4, 5, 3}},
    {{12, 1, 10, 15, 9, 2, 6, 8, 0, 13, 3, 4, 14, 7, 5, 11},
     {10, 15, 4, 2, 7, 12, 9, 5, 6, 1, 13, 14, 0, 11, 3, 8},
     {9, 14, 15, 5, 2, 8, 12, 3, 7, 0, 4, 10, 1, 13, 11, 6},
     {4, 3, 2, 12, 9, 5, 15, 10, 11, 14, 1, 7, 6, 0, 8, 13}},
    {{4, 11, 2, 14, 15, 0, 8, 13, 3, 12, 9, 7, 5, 10, 6, 1},
     {13, 0, 11, 7, 4, 9, 1, 10, 14, 3, 5, 12, 2, 15, 8, 6},
     {1, 4, 11, 13, 12, 3, 7, 14, 10, 15, 6, 8, 0, 5, 9, 2},
     {6, 11, 13, 8, 1, 4, 10, 7, 9, 5, 0, 15, 14, 2, 3, 12}},
    {{13, 2, 8, 4, 6, 15, 11, 1, 10, 9, 3, 14, 5, 0, 12, 7},
     {1, 15, 13, 8, 10, 3, 7, 4, 12, 5, 6, 11, 0, 14, 9, 2},
     {7, 11, 4, 1, 9, 12, 14, 2, 0, 6, 10, 13, 15, 3, 5, 8},
     {2, 1, 14, 7, 4, 10, 8, 13, 15, 12, 9, 0, 3, 5, 6, 11}}};

static const unsigned char per[32] = {16, 7,  20, 21, 29, 12, 28, 17,
                                      1,  15, 23, 26, 5,  18, 31, 10,
                                      2,  8,  24, 14, 32, 27, 3,  9,
                                      19, 13, 30, 6,  22, 11, 4,  25};

static const unsigned char final_perm[64] = {
    40, 8, 48, 16, 56, 24, 64, 32, 39, 7, 47, 15, 55, 23, 63, 31,
    38, 6, 46, 14, 54, 22, 62, 30, 37, 5, 45, 13, 53, 21, 61, 29,
    36, 4, 44, 12, 52, 20, 60, 28, 35, 3, 43, 11, 51, 19, 59, 27,
    34, 2, 42, 10, 50, 18, 58, 26, 33, 1, 41, 9,  49, 17, 57, 25};

/* ---- byte <-> one-byte-per-bit conversion (bit 1 = MSB of byte 0) ---- */

static void unpack_bits(const uint8_t bytes[8], uint8_t bits[65]) {
    bits[0] = 0; /* unused: arrays are 1-indexed like the tables */
    for (int i = 1; i <= 64; ++i) {
        int byte = (i - 1) / 8;
        int shift = 7 - (i - 1) % 8;
        bits[i] = (uint8_t)((bytes[byte] >> shift) & 1u);
    }
}

static void pack_bits(const uint8_t bits[65], uint8_t bytes[8]) {
    for (int b = 0; b < 8; ++b) bytes[b] = 0;
    for (int i = 1; i <= 64; ++i) {
        int byte = (i - 1) / 8;
        int shift = 7 - (i - 1) % 8;
        bytes[byte] |= (uint8_t)(bits[i] << shift);
    }
}

/* ---- Sec. III-A: key generation for one base key ---- */

void oracle_des_round_keys(const uint8_t key[8], uint8_t round_key[16][48]) {
    uint8_t kbits[65];
    unpack_bits(key, kbits);

    /* PC-1: 64 -> 56 bits; bit i of the result is key bit pc_1[i]. */
    uint8_t c[29], d[29]; /* 1-indexed 28-bit halves */
    for (int i = 1; i <= 28; ++i) c[i] = kbits[pc_1[i - 1]];
    for (int i = 1; i <= 28; ++i) d[i] = kbits[pc_1[28 + i - 1]];

    for (int r = 0; r < 16; ++r) {
        /* circular left shift of each half by shift_keys[r], cumulative */
        for (int t = 0; t < shift_keys[r]; ++t) {
            uint8_t c1 = c[1], d1 = d[1];
            for (int i = 1; i < 28; ++i) {
                c[i] = c[i + 1];
                d[i] = d[i + 1];
            }
            c[28] = c1;
            d[28] = d1;
        }
        /* PC-2 over the combined 56 bits C||D */
        uint8_t cd[57];
        for (int i = 1; i <= 28; ++i) {
            cd[i] = c[i];
            cd[28 + i] = d[i];
        }
        for (int j = 0; j < 48; ++j) round_key[r][j] = cd[pc_2[j]];
    }
}

/* ---- Sec. III-B: the S-box step for one 6-bit group ----
 * b[1..6] are the group's bits in order; the outer bits b1,b6 pick the row
 * and the middle bits b2..b5 the column. */
static int sbox_lookup(int g, const uint8_t b[7]) {
    int row = 2 * b[1] + b[6];
    int col = 8 * b[2] + 4 * b[3] + 2 * b[4] + b[5];
    return s[g][row][col];
}

int oracle_sbox(int g, int six) {
    uint8_t b[7];
    b[0] = 0;
    for (int i = 1; i <= 6; ++i) b[i] = (uint8_t)((six >> (6 - i)) & 1);
    return sbox_lookup(g & 7, b);
}

/* ---- Sec. III-B: one DES pass over one 64-bit block ---- */

static void des_block(const uint8_t round_key[16][48], int decrypt,
                      const uint8_t in[8], uint8_t out[8]) {
    uint8_t x[65], m[65];
    unpack_bits(in, x);
    for (int j = 1; j <= 64; ++j) m[j] = x[initial_perm[j - 1]];

    uint8_t left[33], right[33];
    for (int j = 1; j <= 32; ++j) {
        left[j] = m[j];
        right[j] = m[32 + j];
    }

    for (int r = 0; r < 16; ++r) {
        const uint8_t *k = round_key[decrypt ? 15 - r : r];

        uint8_t er[49]; /* expansion of the right half, XOR round key */
        for (int j = 1; j <= 48; ++j) er[j] = (uint8_t)(right[exp_d[j - 1]] ^ k[j - 1]);

        uint8_t sb[33]; /* eight 6 -> 4 substitutions */
        for (int g = 0; g < 8; ++g) {
            int v = sbox_lookup(g, &er[6 * g]); /* its b[1]..b[6] = er[6g+1..6g+6] */
            for (int t = 0; t < 4; ++t) sb[4 * g + 1 + t] = (uint8_t)((v >> (3 - t)) & 1);
        }

        uint8_t f[33];
        for (int j = 1; j <= 32; ++j) f[j] = sb[per[j - 1]];

        for (int j = 1; j <= 32; ++j) {
            uint8_t new_right = (uint8_t)(left[j] ^ f[j]);
            left[j] = right[j];
            right[j] = new_right;
        }
    }

    uint8_t pre[65]; /* halves combined as R16 || L16 */
    for (int j = 1; j <= 32; ++j) {
        pre[j] = right[j];
        pre[32 + j] = left[j];
    }
    uint8_t y[65];
    y[0] = 0;
    for (int j = 1; j <= 64; ++j) y[j] = pre[final_perm[j - 1]];
    pack_bits(y, out);
}

void oracle_des_block(const uint8_t key[8], int decrypt, const uint8_t in[8],
                      uint8_t out[8]) {
    uint8_t rk[16][48];
    oracle_des_round_keys(key, rk);
    des_block(rk, decrypt, in, out);
}

/* ---- Sec. III-B, 3DES equations ---- */

/* The block cipher the modes below run: EDE3 under three keys, or a single
 * DES pass under the first key (passes == 1). */
typedef struct {
    int passes;
    uint8_t rk[3][16][48];
} tdes_keys;

static void tdes_expand(const uint8_t keys[24], tdes_keys *k) {
    k->passes = 3;
    for (int i = 0; i < 3; ++i) oracle_des_round_keys(keys + 8 * i, k->rk[i]);
}

static void des_expand(const uint8_t key[8], tdes_keys *k) {
    k->passes = 1;
    oracle_des_round_keys(key, k->rk[0]);
}

static void tdes_block(const tdes_keys *k, int decrypt, const uint8_t in[8], uint8_t out[8]) {
    uint8_t a[8], b[8];
    if (k->passes == 1) { /* single DES */
        des_block(k->rk[0], decrypt, in, out);
    } else if (!decrypt) { /* E_K3(D_K2(E_K1(P))) */
        des_block(k->rk[0], 0, in, a);
        des_block(k->rk[1], 1, a, b);
        des_block(k->rk[2], 0, b, out);
    } else { /* D_K1(E_K2(D_K3(C))) */
        des_block(k->rk[2], 1, in, a);
        des_block(k->rk[1], 0, a, b);
        des_block(k->rk[0], 1, b, out);
    }
}

void oracle_tdes_block(const uint8_t keys[24], int decrypt, const uint8_t in[8],
                       uint8_t out[8]) {
    tdes_keys k;
    tdes_expand(keys, &k);
    tdes_block(&k, decrypt, in, out);
}

/* ---- modes over whole buffers of 8-byte blocks ---- */

static void be64_store(uint64_t v, uint8_t out[8]) {
    for (int i = 0; i < 8; ++i) out[i] = (uint8_t)(v >> (56 - 8 * i));
}

static void ecb_range(const tdes_keys *k, int decrypt, const uint8_t *in, uint8_t *out,
                      uint64_t first, uint64_t end) {
    for (uint64_t i = first; i < end; ++i) tdes_block(k, decrypt, in + 8 * i, out + 8 * i);
}

void oracle_tdes_ecb(const uint8_t keys[24], int decrypt, const uint8_t *in, uint8_t *out,
                     uint64_t nblocks) {
    tdes_keys k;
    tdes_expand(keys, &k);
    ecb_range(&k, decrypt, in, out, 0, nblocks);
}

void oracle_des_ecb(const uint8_t key[8], int decrypt, const uint8_t *in, uint8_t *out,
                    uint64_t nblocks) {
    tdes_keys k;
    des_expand(key, &k);
    ecb_range(&k, decrypt, in, out, 0, nblocks);
}

static void ctr_range(const tdes_keys *k, uint32_t nonce, uint32_t ctr0, const uint8_t *in,
                      uint8_t *out, uint64_t first, uint64_t end) {
    for (uint64_t i = first; i < end; ++i) {
        uint8_t cb[8], ks[8];
        uint64_t counter = ((uint64_t)nonce << 32) | (uint32_t)(ctr0 + (uint32_t)i);
        be64_store(counter, cb);
        tdes_block(k, 0, cb, ks);
        for (int t = 0; t < 8; ++t) out[8 * i + t] = (uint8_t)(in[8 * i + t] ^ ks[t]);
    }
}

int oracle_tdes_ctr(const uint8_t keys[24], uint32_t nonce, uint32_t ctr0, const uint8_t *in,
                    uint8_t *out, uint64_t nblocks) {
    if ((uint64_t)ctr0 + nblocks > ((uint64_t)1 << 32)) return -1; /* counter would wrap */
    tdes_keys k;
    tdes_expand(keys, &k);
    ctr_range(&k, nonce, ctr0, in, out, 0, nblocks);
    return 0;
}

int oracle_des_ctr(const uint8_t key[8], uint32_t nonce, uint32_t ctr0, const uint8_t *in,
                   uint8_t *out, uint64_t nblocks) {
    if ((uint64_t)ctr0 + nblocks > ((uint64_t)1 << 32)) return -1; /* counter would wrap */
    tdes_keys k;
    des_expand(key, &k);
    ctr_range(&k, nonce, ctr0, in, out, 0, nblocks);
    return 0;
}

static void cbc_encrypt(const tdes_keys *k, uint64_t iv, const uint8_t *in, uint8_t *out,
                        uint64_t nblocks) {
    uint8_t prev[8];
    be64_store(iv, prev);
    for (uint64_t i = 0; i < nblocks; ++i) {
        uint8_t x[8];
        for (int t = 0; t < 8; ++t) x[t] = (uint8_t)(in[8 * i + t] ^ prev[t]);
        tdes_block(k, 0, x, out + 8 * i);
        memcpy(prev, out + 8 * i, 8);
    }
}

static void cbc_decrypt(const tdes_keys *k, uint64_t iv, const uint8_t *in, uint8_t *out,
                        uint64_t nblocks) {
    uint8_t prev[8];
    be64_store(iv, prev);
    for (uint64_t i = 0; i < nblocks; ++i) {
        uint8_t cur[8], y[8];
        memcpy(cur, in + 8 * i, 8); /* copy first so that in == out works */
        tdes_block(k, 1, cur, y);
        for (int t = 0; t < 8; ++t) out[8 * i + t] = (uint8_t)(y[t] ^ prev[t]);
        memcpy(prev, cur, 8);
    }
}

void oracle_tdes_cbc_encrypt(const uint8_t keys[24], uint64_t iv, const uint8_t *in,
                             uint8_t *out, uint64_t nblocks) {
    tdes_keys k;
    tdes_expand(keys, &k);
    cbc_encrypt(&k, iv, in, out, nblocks);
}

void oracle_tdes_cbc_decrypt(const uint8_t keys[24], uint64_t iv, const uint8_t *in,
                             uint8_t *out, uint64_t nblocks) {
    tdes_keys k;
    tdes_expand(keys, &k);
    cbc_decrypt(&k, iv, in, out, nblocks);
}

void oracle_des_cbc_encrypt(const uint8_t key[8], uint64_t iv, const uint8_t *in, uint8_t *out,
                            uint64_t nblocks) {
    tdes_keys k;
    des_expand(key, &k);
    cbc_encrypt(&k, iv, in, out, nblocks);
}

void oracle_des_cbc_decrypt(const uint8_t key[8], uint64_t iv, const uint8_t *in, uint8_t *out,
                            uint64_t nblocks) {
    tdes_keys k;
    des_expand(key, &k);
    cbc_decrypt(&k, iv, in, out, nblocks);
}

/* ---- multi-threaded ECB/CTR for the CPU timing baseline only ----
 * The same per-block code, with the blocks split into contiguous ranges,
 * one per thread (the paper's CPU baseline parallelises the loop over
 * blocks with an OpenMP parallel-for, Sec. V). */

typedef struct {
    const tdes_keys *k;
    int mode; /* 0 ecb-enc, 1 ecb-dec, 2 ctr */
    uint32_t nonce, ctr0;
    const uint8_t *in;
    uint8_t *out;
    uint64_t first, end;
} mt_job;

static void *mt_worker(void *arg) {
    mt_job *j = (mt_job *)arg;
    if (j->mode == 2)
        ctr_range(j->k, j->nonce, j->ctr0, j->in, j->out, j->first, j->end);
    else
        ecb_range(j->k, j->mode, j->in, j->out, j->first, j->end);
    return NULL;
}

int oracle_tdes_parallel(const uint8_t keys[24], int mode, uint32_t nonce, uint32_t ctr0,
                         const uint8_t *in, uint8_t *out, uint64_t nblocks, int nthreads) {
    if (nthreads < 1 || nthreads > 1024 || mode < 0 || mode > 2) return -1;
    if (mode == 2 && (uint64_t)ctr0 + nblocks > ((uint64_t)1 << 32)) return -1;
    tdes_keys k;
    tdes_expand(keys, &k);
    pthread_t tid[1024];
    mt_job jobs[1024];
    uint64_t per_thread = (nblocks + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t first = per_thread * (uint64_t)t;
        uint64_t end = first + per_thread;
        if (first >= nblocks) break;
        if (end > nblocks) end = nblocks;
        jobs[t] = (mt_job){&k, mode, nonce, ctr0, in, out, first, end};
        if (pthread_create(&tid[t], NULL, mt_worker, &jobs[t]) != 0) {
            mt_worker(&jobs[t]); /* run inline if a thread cannot start */
            tid[t] = 0;
            jobs[t].k = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (jobs[t].k != NULL) pthread_join(tid[t], NULL);
    return 0;
}

/* ---- many messages, each under its own triple and mode (batch checks) ---- */

typedef struct {
    const uint8_t *keys;
    const uint32_t *key_index;
    const uint8_t *mode;
    const uint64_t *iv;
    const uint64_t *offset, *nblocks;
    const uint8_t *in;
    uint8_t *out;
    uint64_t first, end;
} msg_job;

static void *msg_worker(void *arg) {
    msg_job *j = (msg_job *)arg;
    for (uint64_t i = j->first; i < j->end; ++i) {
        const uint8_t *k = j->keys + 24 * (uint64_t)j->key_index[i];
        const uint8_t *in = j->in + j->offset[i];
        uint8_t *out = j->out + j->offset[i];
        const uint64_t nb = j->nblocks[i], iv = j->iv[i];
        switch (j->mode[i]) {
        case 0: oracle_tdes_ecb(k, 0, in, out, nb); break;
        case 1: oracle_tdes_ecb(k, 1, in, out, nb); break;
        case 2: oracle_tdes_ctr(k, (uint32_t)(iv >> 32), (uint32_t)iv, in, out, nb); break;
        case 3: oracle_tdes_cbc_decrypt(k, iv, in, out, nb); break;
        default: oracle_tdes_cbc_encrypt(k, iv, in, out, nb); break;
        }
    }
    return NULL;
}

int oracle_tdes_messages(const uint8_t *keys, uint32_t n_keys, const uint32_t *key_index,
                         const uint8_t *mode, const uint64_t *iv_or_ctr, const uint64_t *offset,
                         const uint64_t *nblocks, const uint8_t *in, uint8_t *out, uint64_t n,
                         int nthreads) {
    if (nthreads < 1 || nthreads > 1024) return -1;
    for (uint64_t i = 0; i < n; ++i) {
        if (key_index[i] >= n_keys || mode[i] > 4) return -1;
        if (mode[i] == 2 && (iv_or_ctr[i] & 0xFFFFFFFFull) + nblocks[i] > ((uint64_t)1 << 32))
            return -1;
    }
    pthread_t tid[1024];
    msg_job jobs[1024];
    const uint64_t per_thread = (n + (uint64_t)nthreads - 1) / (uint64_t)nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t first = per_thread * (uint64_t)t, end = first + per_thread;
        if (first >= n) break;
        if (end > n) end = n;
        jobs[t] = (msg_job){keys, key_index, mode, iv_or_ctr, offset, nblocks, in, out, first, end};
        if (pthread_create(&tid[t], NULL, msg_worker, &jobs[t]) != 0) {
            msg_worker(&jobs[t]); /* run inline if a thread cannot start */
            jobs[t].keys = NULL;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (jobs[t].keys != NULL) pthread_join(tid[t], NULL);
    return 0;
}
