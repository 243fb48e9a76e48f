/*
 * tdes_oracle.h -- CPU oracle for 3DES-EDE3 (test infrastructure only).
 *
 * Plain, slow, single-threaded reference of the method in "Bit-level
 * Parallelization of 3DES Encryption on GPU", Sec. III: one byte per bit,
 * 1-indexed appendix tables.  Only tests, the smoke check and the CPU
 * baseline of the benchmark use it; the CUDA library shares nothing with it.
 * Two helpers at the end split work over host threads (the CPU baseline's
 * timing, and checks of whole batches); each thread runs the same code.
 *
 * Byte conventions: blocks and keys are 8-byte big-endian strings (bit 1 =
 * MSB of byte 0).  A key triple is 24 bytes K1||K2||K3.  Buffers hold
 * nblocks * 8 bytes.  in == out is allowed everywhere.
 */
#ifndef TDES_ORACLE_H
#define TDES_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Sec. III-A: the 16 round keys of one base key, one byte per bit. */
void oracle_des_round_keys(const uint8_t key[8], uint8_t round_key[16][48]);

/* Sec. III-B S-box step: S-box g (0..7) of the 6-bit group `six`, whose
 * most significant bit is the group's first bit b1.  Returns 0..15. */
int oracle_sbox(int g, int six);

/* Sec. III-B: single DES on one block (decrypt != 0: round keys reversed). */
void oracle_des_block(const uint8_t key[8], int decrypt, const uint8_t in[8], uint8_t out[8]);

/* Sec. III-B, 3DES equations: EDE3 on one block. */
void oracle_tdes_block(const uint8_t keys[24], int decrypt, const uint8_t in[8], uint8_t out[8]);

/* Modes over a buffer of nblocks 8-byte blocks. */
void oracle_tdes_ecb(const uint8_t keys[24], int decrypt, const uint8_t *in, uint8_t *out,
                     uint64_t nblocks);
/* Returns -1 (and writes nothing) when ctr0 + nblocks > 2^32. */
int oracle_tdes_ctr(const uint8_t keys[24], uint32_t nonce, uint32_t ctr0, const uint8_t *in,
                    uint8_t *out, uint64_t nblocks);
void oracle_tdes_cbc_encrypt(const uint8_t keys[24], uint64_t iv, const uint8_t *in,
                             uint8_t *out, uint64_t nblocks);
void oracle_tdes_cbc_decrypt(const uint8_t keys[24], uint64_t iv, const uint8_t *in,
                             uint8_t *out, uint64_t nblocks);

/* The same modes over single DES under one 8-byte key (Sec. III-B: one
 * pass of 16 rounds; EDE3 under (K, K, K) gives the same result). */
void oracle_des_ecb(const uint8_t key[8], int decrypt, const uint8_t *in, uint8_t *out,
                    uint64_t nblocks);
int oracle_des_ctr(const uint8_t key[8], uint32_t nonce, uint32_t ctr0, const uint8_t *in,
                   uint8_t *out, uint64_t nblocks);
void oracle_des_cbc_encrypt(const uint8_t key[8], uint64_t iv, const uint8_t *in, uint8_t *out,
                            uint64_t nblocks);
void oracle_des_cbc_decrypt(const uint8_t key[8], uint64_t iv, const uint8_t *in, uint8_t *out,
                            uint64_t nblocks);

/* ECB (mode 0 encrypt, 1 decrypt) or CTR (mode 2) split over nthreads host
 * threads; used only to time the CPU baseline.  Returns 0 or -1. */
int oracle_tdes_parallel(const uint8_t keys[24], int mode, uint32_t nonce, uint32_t ctr0,
                         const uint8_t *in, uint8_t *out, uint64_t nblocks, int nthreads);

/* Many independent messages, each under its own triple and mode, for
 * checking whole batches: message i is the nblocks[i] blocks at byte offset
 * offset[i] of in, written at the same offset of out, under the triple
 * keys[24 * key_index[i] ..] (n_keys triples) in mode[i]: 0 ECB encrypt,
 * 1 ECB decrypt, 2 CTR (iv_or_ctr[i] = nonce << 32 | ctr0), 3 CBC decrypt,
 * 4 CBC encrypt (iv_or_ctr[i] = IV).  Each message is computed by the mode
 * functions above; messages are split into contiguous ranges over nthreads
 * host threads.  Returns -1 and writes nothing if any message has a key
 * index >= n_keys, a mode > 4 or a CTR counter that would pass 2^32. */
int oracle_tdes_messages(const uint8_t *keys, uint32_t n_keys, const uint32_t *key_index,
                         const uint8_t *mode, const uint64_t *iv_or_ctr, const uint64_t *offset,
                         const uint64_t *nblocks, const uint8_t *in, uint8_t *out, uint64_t n,
                         int nthreads);

#ifdef __cplusplus
}
#endif
#endif
