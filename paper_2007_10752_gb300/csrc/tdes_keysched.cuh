// tdes_keysched.cuh -- key schedule as a gather of key bits.
//
// "Bit-level Parallelization of 3DES Encryption on GPU", Sec. III-A: each
// 48-bit round key is PC-2 of the two 28-bit halves of PC-1(K), rotated left
// cumulatively by shift_keys.  Rotations and both permutations only move
// bits, so every round-key bit is one fixed bit of K; the generator composes
// the three steps at build time into per-word recipes.  The kernel then
// needs only a gather: one thread per word of the per-key tables.
#pragma once
#include <cstdint>

#include "tdes_bitslice.cuh"
#include "generated/tdes_generated_scalar.cuh"

#define TDES_SUBKEY_WORDS (48 * 8)  // 48 rounds x 8 six-bit groups (bytes)

// Key bit b (b = 64*key + bit - 1, bit 1 = MSB of the key's first byte).
TDES_HD uint32_t tdes_key_bit(const uint8_t* __restrict__ keys, unsigned b) {
    return (keys[b >> 3] >> (7u - (b & 7u))) & 1u;
}

// One word of the bitsliced round-constant table: -(bit a XOR bit b), OR 1
// for the multiplier words.
TDES_HD uint32_t tdes_table_word(const uint8_t* __restrict__ keys, const uint8_t* __restrict__ rec) {
    uint32_t x = 0;
    if (rec[1] != 255) x ^= tdes_key_bit(keys, rec[1]);
    if (rec[2] != 255) x ^= tdes_key_bit(keys, rec[2]);
    uint32_t w = 0u - x;
    return rec[0] ? (w | 1u) : w;
}

// One six-bit round-key group of the scalar path: round r, S-box g.
TDES_HD uint8_t tdes_subkey_chunk(const uint8_t* __restrict__ keys, const uint8_t* __restrict__ bits48) {
    uint32_t c = 0;
    for (int u = 0; u < 6; ++u) c = (c << 1) | tdes_key_bit(keys, bits48[u]);
    return (uint8_t)c;
}
