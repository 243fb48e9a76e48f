// GENERATED by paper_2007_10752_gb300/gen/emit_cuda.py -- do not edit.
// Round of the bitsliced path for tables with a different key per bit
// position (from the S-box circuits in gen/sbox_lop3.json).
#pragma once
#include <cstdint>

// Needs TDES_HD and lop3<LUT>(a, b, c) from tdes_bitslice.cuh.

// The same round for tables whose masks differ from bit to bit (one key
// per bit position: tiles of small messages under many keys).  The
// multiply-add form of a masked XOR holds only for all-0 or all-1 masks,
// so the doubled expansion inputs take a plain XOR; the multipliers are
// not read.
TDES_HD void tdes_round_mixed(uint32_t (&T)[32], const uint32_t (&S)[32],
                              const uint32_t* __restrict__ k) {
    {  // S-box 1
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 4);
    const uint32_t x0 = S[31] ^ kd.x;  // second copy
    const uint32_t x1 = S[0] ^ kd.y;
    const uint32_t x2 = S[1];
    const uint32_t x3 = S[2];
    const uint32_t x4 = S[3];
    const uint32_t x5 = S[4];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 0);
    const uint32_t s0_0 = lop3<0xe8>(x2, x4, x5);
    const uint32_t s0_1 = lop3<0xa3>(x3, x2, s0_0);
    const uint32_t s0_2 = lop3<0x86>(x1, x3, s0_1);
    const uint32_t s0_3 = lop3<0x96>(x4, x5, s0_2);
    const uint32_t s0_4 = lop3<0x97>(x1, x2, s0_3);
    const uint32_t s0_5 = lop3<0x3a>(s0_1, s0_2, s0_4);
    const uint32_t s0_6 = lop3<0x8c>(x1, s0_1, s0_3);
    const uint32_t s0_7 = lop3<0x6c>(x5, s0_5, s0_6);
    const uint32_t s0_8 = lop3<0xac>(x0, s0_3, s0_7);
    T[8] = lop3<0x96>(T[8], s0_8, kc.x);
    const uint32_t s0_9 = lop3<0x29>(x0, x3, x5);
    const uint32_t s0_10 = lop3<0xba>(s0_0, s0_1, s0_9);
    const uint32_t s0_11 = lop3<0x9e>(x2, s0_3, s0_10);
    const uint32_t s0_12 = lop3<0x4b>(x0, x3, x5);
    const uint32_t s0_13 = lop3<0x1e>(s0_1, s0_8, s0_12);
    const uint32_t s0_14 = lop3<0x1a>(s0_7, s0_10, s0_13);
    const uint32_t s0_15 = lop3<0xac>(x1, s0_11, s0_14);
    T[16] = lop3<0x96>(T[16], s0_15, kc.y);
    const uint32_t s0_16 = lop3<0x4a>(x3, x5, s0_3);
    const uint32_t s0_17 = lop3<0xb6>(s0_2, s0_4, s0_16);
    const uint32_t s0_18 = lop3<0x4e>(x3, s0_2, s0_13);
    const uint32_t s0_19 = lop3<0x6b>(x4, s0_14, s0_18);
    const uint32_t s0_20 = lop3<0x6c>(x0, s0_17, s0_19);
    T[22] = lop3<0x96>(T[22], s0_20, kc.z);
    const uint32_t s0_21 = lop3<0x79>(x2, s0_13, s0_19);
    const uint32_t s0_22 = lop3<0x3a>(x3, s0_1, s0_21);
    const uint32_t s0_23 = lop3<0x72>(x1, x3, x4);
    const uint32_t s0_24 = lop3<0x1e>(x2, s0_13, s0_23);
    const uint32_t s0_25 = lop3<0xac>(x5, s0_22, s0_24);
    const uint32_t s0_26 = lop3<0x96>(x0, x1, s0_25);
    T[30] = lop3<0x96>(T[30], s0_26, kc.w);
    }
    {  // S-box 2
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 12);
    const uint32_t x0 = S[3] ^ kd.x;  // second copy
    const uint32_t x1 = S[4] ^ kd.y;
    const uint32_t x2 = S[5];
    const uint32_t x3 = S[6];
    const uint32_t x4 = S[7];
    const uint32_t x5 = S[8];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 8);
    const uint32_t s1_0 = lop3<0xe7>(x0, x1, x5);
    const uint32_t s1_1 = lop3<0x2a>(x0, x4, s1_0);
    const uint32_t s1_2 = lop3<0x7d>(x0, x1, x5);
    const uint32_t s1_3 = lop3<0x2b>(x1, x4, s1_2);
    const uint32_t s1_4 = lop3<0x6c>(x3, s1_1, s1_3);
    const uint32_t s1_5 = lop3<0x81>(x0, x4, x5);
    const uint32_t s1_6 = lop3<0xb1>(s1_0, s1_3, s1_5);
    const uint32_t s1_7 = lop3<0x6c>(x2, s1_4, s1_6);
    T[17] = lop3<0x96>(T[17], s1_7, kc.w);
    const uint32_t s1_8 = lop3<0x81>(x1, s1_1, s1_7);
    const uint32_t s1_9 = lop3<0x86>(x0, x4, s1_8);
    const uint32_t s1_10 = lop3<0x96>(x1, x2, s1_9);
    const uint32_t s1_11 = lop3<0x68>(s1_1, s1_2, s1_10);
    const uint32_t s1_12 = lop3<0xd4>(x1, x4, s1_5);
    const uint32_t s1_13 = lop3<0x6c>(x3, s1_11, s1_12);
    T[12] = lop3<0x96>(T[12], s1_13, kc.x);
    const uint32_t s1_14 = lop3<0x9c>(s1_0, s1_7, s1_13);
    const uint32_t s1_15 = lop3<0x5a>(x1, x5, s1_14);
    const uint32_t s1_16 = lop3<0xb8>(s1_7, s1_10, s1_13);
    const uint32_t s1_17 = lop3<0x76>(x0, x5, s1_16);
    const uint32_t s1_18 = lop3<0x6c>(x4, s1_15, s1_17);
    T[27] = lop3<0x96>(T[27], s1_18, kc.y);
    const uint32_t s1_19 = lop3<0x79>(s1_4, s1_12, s1_17);
    const uint32_t s1_20 = lop3<0xa2>(s1_7, s1_13, s1_19);
    const uint32_t s1_21 = lop3<0x56>(x2, s1_11, s1_14);
    const uint32_t s1_22 = lop3<0x92>(s1_4, s1_12, s1_21);
    const uint32_t s1_23 = lop3<0x6c>(x0, s1_20, s1_22);
    const uint32_t s1_24 = lop3<0x4a>(s1_9, s1_17, s1_23);
    T[1] = lop3<0x96>(T[1], s1_24, kc.z);
    }
    {  // S-box 3
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 20);
    const uint32_t x0 = S[7] ^ kd.x;  // second copy
    const uint32_t x1 = S[8] ^ kd.y;
    const uint32_t x2 = S[9];
    const uint32_t x3 = S[10];
    const uint32_t x4 = S[11];
    const uint32_t x5 = S[12];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 16);
    const uint32_t s2_0 = lop3<0xe4>(x2, x3, x4);
    const uint32_t s2_1 = lop3<0x96>(x5, x1, s2_0);
    const uint32_t s2_2 = lop3<0xab>(x1, x2, x4);
    const uint32_t s2_3 = lop3<0xe6>(x1, x2, s2_0);
    const uint32_t s2_4 = lop3<0xac>(x5, s2_2, s2_3);
    const uint32_t s2_5 = lop3<0xe6>(x3, x4, s2_4);
    const uint32_t s2_6 = lop3<0x6c>(x0, s2_1, s2_5);
    T[5] = lop3<0x96>(T[5], s2_6, kc.w);
    const uint32_t s2_7 = lop3<0x38>(x0, s2_1, s2_2);
    const uint32_t s2_8 = lop3<0xa5>(x0, x1, s2_1);
    const uint32_t s2_9 = lop3<0x24>(x2, s2_7, s2_8);
    const uint32_t s2_10 = lop3<0x36>(x0, x5, s2_0);
    const uint32_t s2_11 = lop3<0xbe>(x4, s2_1, s2_10);
    const uint32_t s2_12 = lop3<0x6c>(x3, s2_9, s2_11);
    T[15] = lop3<0x96>(T[15], s2_12, kc.y);
    const uint32_t s2_13 = lop3<0x35>(s2_0, s2_4, s2_6);
    const uint32_t s2_14 = lop3<0xb6>(x0, x2, s2_13);
    const uint32_t s2_15 = lop3<0x96>(x5, x4, s2_14);
    const uint32_t s2_16 = lop3<0x79>(x0, x1, s2_14);
    const uint32_t s2_17 = lop3<0x9b>(x1, x2, s2_16);
    const uint32_t s2_18 = lop3<0x6c>(x3, s2_15, s2_17);
    T[23] = lop3<0x96>(T[23], s2_18, kc.x);
    const uint32_t s2_19 = lop3<0x61>(x3, s2_2, s2_15);
    const uint32_t s2_20 = lop3<0x1e>(s2_7, s2_18, s2_19);
    const uint32_t s2_21 = lop3<0x69>(s2_3, s2_10, s2_12);
    const uint32_t s2_22 = lop3<0x9e>(x5, s2_19, s2_21);
    const uint32_t s2_23 = lop3<0x6c>(x1, s2_20, s2_22);
    T[29] = lop3<0x96>(T[29], s2_23, kc.z);
    }
    {  // S-box 4
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 28);
    const uint32_t x0 = S[11] ^ kd.x;  // second copy
    const uint32_t x1 = S[12] ^ kd.y;
    const uint32_t x2 = S[13];
    const uint32_t x3 = S[14];
    const uint32_t x4 = S[15];
    const uint32_t x5 = S[16];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 24);
    const uint32_t s3_0 = lop3<0x41>(x0, x1, x2);
    const uint32_t s3_1 = lop3<0xb6>(x1, x3, s3_0);
    const uint32_t s3_2 = lop3<0x6a>(x0, x2, x3);
    const uint32_t s3_3 = lop3<0xae>(x0, x1, s3_2);
    const uint32_t s3_4 = lop3<0x6c>(x4, s3_1, s3_3);
    const uint32_t s3_5 = lop3<0x6d>(x1, x2, x4);
    const uint32_t s3_6 = lop3<0x92>(x3, x1, s3_5);
    const uint32_t s3_7 = lop3<0x1a>(x2, s3_2, s3_6);
    const uint32_t s3_8 = lop3<0x9e>(x4, s3_0, s3_7);
    const uint32_t s3_9 = lop3<0xac>(x5, s3_4, s3_8);
    T[0] = lop3<0x96>(T[0], s3_9, kc.w);
    const uint32_t s3_10 = lop3<0x69>(x2, x4, s3_4);
    const uint32_t s3_11 = lop3<0xeb>(x1, x3, s3_10);
    const uint32_t s3_12 = lop3<0x92>(x0, s3_6, s3_11);
    const uint32_t s3_13 = lop3<0x56>(x4, s3_1, s3_2);
    const uint32_t s3_14 = lop3<0xc7>(x2, s3_4, s3_8);
    const uint32_t s3_15 = lop3<0x6c>(x1, s3_13, s3_14);
    const uint32_t s3_16 = lop3<0xac>(x5, s3_12, s3_15);
    T[25] = lop3<0x96>(T[25], s3_16, kc.x);
    const uint32_t s3_17 = lop3<0x3a>(x5, s3_4, s3_8);
    T[9] = lop3<0x96>(T[9], s3_17, kc.z);
    const uint32_t s3_18 = lop3<0x3a>(x5, s3_12, s3_15);
    T[19] = lop3<0x96>(T[19], s3_18, kc.y);
    }
    {  // S-box 5
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 36);
    const uint32_t x0 = S[15] ^ kd.x;  // second copy
    const uint32_t x1 = S[16] ^ kd.y;
    const uint32_t x2 = S[17];
    const uint32_t x3 = S[18];
    const uint32_t x4 = S[19];
    const uint32_t x5 = S[20];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 32);
    const uint32_t s4_0 = lop3<0x81>(x0, x3, x5);
    const uint32_t s4_1 = lop3<0xb6>(x2, x5, s4_0);
    const uint32_t s4_2 = lop3<0x9e>(x0, x2, x5);
    const uint32_t s4_3 = lop3<0x6c>(x3, s4_2, x5);
    const uint32_t s4_4 = lop3<0xac>(x4, s4_1, s4_3);
    const uint32_t s4_5 = lop3<0x90>(x2, x4, s4_1);
    const uint32_t s4_6 = lop3<0xb6>(x0, x3, s4_5);
    const uint32_t s4_7 = lop3<0x2a>(x4, s4_3, s4_6);
    const uint32_t s4_8 = lop3<0xac>(x1, s4_4, s4_7);
    T[24] = lop3<0x96>(T[24], s4_8, kc.z);
    const uint32_t s4_9 = lop3<0xed>(x0, x2, x5);
    const uint32_t s4_10 = lop3<0x92>(s4_4, s4_6, s4_9);
    const uint32_t s4_11 = lop3<0xba>(s4_1, s4_8, s4_10);
    const uint32_t s4_12 = lop3<0x65>(x2, x3, s4_2);
    const uint32_t s4_13 = lop3<0xb8>(x0, x4, s4_12);
    const uint32_t s4_14 = lop3<0x63>(s4_9, s4_11, s4_13);
    const uint32_t s4_15 = lop3<0xac>(x1, s4_11, s4_14);
    T[7] = lop3<0x96>(T[7], s4_15, kc.x);
    const uint32_t s4_16 = lop3<0xa9>(x0, x4, s4_7);
    const uint32_t s4_17 = lop3<0xc6>(x2, s4_12, s4_16);
    const uint32_t s4_18 = lop3<0x3a>(s4_5, s4_13, s4_17);
    const uint32_t s4_19 = lop3<0xed>(x0, x3, s4_1);
    const uint32_t s4_20 = lop3<0x6c>(x1, s4_18, s4_19);
    T[13] = lop3<0x96>(T[13], s4_20, kc.y);
    const uint32_t s4_21 = lop3<0x93>(s4_2, s4_8, s4_11);
    const uint32_t s4_22 = lop3<0xb6>(x1, s4_17, s4_21);
    const uint32_t s4_23 = lop3<0xa6>(x4, x1, s4_22);
    const uint32_t s4_24 = lop3<0x6a>(x1, s4_1, s4_16);
    const uint32_t s4_25 = lop3<0x82>(x3, s4_20, s4_24);
    const uint32_t s4_26 = lop3<0x6c>(x5, s4_23, s4_25);
    T[2] = lop3<0x96>(T[2], s4_26, kc.w);
    }
    {  // S-box 6
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 44);
    const uint32_t x0 = S[19] ^ kd.x;  // second copy
    const uint32_t x1 = S[20] ^ kd.y;
    const uint32_t x2 = S[21];
    const uint32_t x3 = S[22];
    const uint32_t x4 = S[23];
    const uint32_t x5 = S[24];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 40);
    const uint32_t s5_0 = lop3<0x59>(x1, x2, x3);
    const uint32_t s5_1 = lop3<0x96>(x4, x0, s5_0);
    const uint32_t s5_2 = lop3<0xab>(x2, x4, s5_1);
    const uint32_t s5_3 = lop3<0xad>(x0, x2, s5_2);
    const uint32_t s5_4 = lop3<0x9b>(x1, s5_0, s5_3);
    const uint32_t s5_5 = lop3<0x6c>(x5, s5_2, s5_4);
    const uint32_t s5_6 = lop3<0x96>(x1, x2, s5_5);
    T[3] = lop3<0x96>(T[3], s5_6, kc.x);
    const uint32_t s5_7 = lop3<0x75>(x1, x2, x5);
    const uint32_t s5_8 = lop3<0x6c>(x4, s5_7, x2);
    const uint32_t s5_9 = lop3<0x63>(x0, s5_1, s5_8);
    const uint32_t s5_10 = lop3<0x51>(x0, x1, x4);
    const uint32_t s5_11 = lop3<0xac>(x5, s5_6, s5_10);
    const uint32_t s5_12 = lop3<0x6c>(x3, s5_9, s5_11);
    T[18] = lop3<0x96>(T[18], s5_12, kc.w);
    const uint32_t s5_13 = lop3<0x65>(x1, x3, x5);
    const uint32_t s5_14 = lop3<0x7a>(s5_4, s5_9, s5_13);
    const uint32_t s5_15 = lop3<0xa8>(s5_8, s5_9, s5_14);
    const uint32_t s5_16 = lop3<0x56>(x5, s5_4, s5_6);
    const uint32_t s5_17 = lop3<0x4b>(s5_1, s5_7, s5_16);
    const uint32_t s5_18 = lop3<0xac>(x0, s5_15, s5_17);
    T[28] = lop3<0x96>(T[28], s5_18, kc.y);
    const uint32_t s5_19 = lop3<0x26>(x0, s5_8, s5_12);
    const uint32_t s5_20 = lop3<0x7a>(s5_1, s5_6, s5_19);
    const uint32_t s5_21 = lop3<0x28>(x2, x3, s5_2);
    const uint32_t s5_22 = lop3<0x26>(s5_6, s5_12, s5_21);
    const uint32_t s5_23 = lop3<0x58>(s5_13, s5_17, s5_22);
    const uint32_t s5_24 = lop3<0xac>(x1, s5_20, s5_23);
    T[10] = lop3<0x96>(T[10], s5_24, kc.z);
    }
    {  // S-box 7
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 52);
    const uint32_t x0 = S[23] ^ kd.x;  // second copy
    const uint32_t x1 = S[24] ^ kd.y;
    const uint32_t x2 = S[25];
    const uint32_t x3 = S[26];
    const uint32_t x4 = S[27];
    const uint32_t x5 = S[28];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 48);
    const uint32_t s6_0 = lop3<0x24>(x0, x2, x5);
    const uint32_t s6_1 = lop3<0xb6>(x3, x0, s6_0);
    const uint32_t s6_2 = lop3<0x98>(x0, x1, s6_1);
    const uint32_t s6_3 = lop3<0x96>(x5, x2, s6_2);
    const uint32_t s6_4 = lop3<0x90>(x0, x1, x5);
    const uint32_t s6_5 = lop3<0xd8>(s6_0, s6_3, s6_4);
    const uint32_t s6_6 = lop3<0x5b>(x3, x0, s6_5);
    const uint32_t s6_7 = lop3<0x6c>(x4, s6_3, s6_6);
    T[31] = lop3<0x96>(T[31], s6_7, kc.x);
    const uint32_t s6_8 = lop3<0x6f>(x1, s6_0, s6_3);
    const uint32_t s6_9 = lop3<0x78>(x4, s6_6, s6_8);
    const uint32_t s6_10 = lop3<0xb4>(x1, x4, s6_9);
    const uint32_t s6_11 = lop3<0xda>(x5, s6_3, s6_10);
    const uint32_t s6_12 = lop3<0xba>(s6_1, s6_7, s6_11);
    const uint32_t s6_13 = lop3<0x6c>(x3, s6_9, s6_12);
    T[11] = lop3<0x96>(T[11], s6_13, kc.y);
    const uint32_t s6_14 = lop3<0x9c>(x1, x2, s6_7);
    const uint32_t s6_15 = lop3<0x9e>(x0, x1, s6_14);
    const uint32_t s6_16 = lop3<0xe8>(x0, s6_2, s6_9);
    const uint32_t s6_17 = lop3<0x3a>(x4, s6_15, s6_16);
    const uint32_t s6_18 = lop3<0xac>(x3, s6_15, s6_17);
    const uint32_t s6_19 = lop3<0x96>(x5, x4, s6_18);
    T[6] = lop3<0x96>(T[6], s6_19, kc.w);
    const uint32_t s6_20 = lop3<0x1c>(x3, s6_7, s6_13);
    const uint32_t s6_21 = lop3<0x4e>(x0, s6_17, s6_20);
    const uint32_t s6_22 = lop3<0x9c>(x3, s6_0, s6_20);
    const uint32_t s6_23 = lop3<0xac>(x5, s6_21, s6_22);
    const uint32_t s6_24 = lop3<0x7a>(x1, s6_10, s6_23);
    T[21] = lop3<0x96>(T[21], s6_24, kc.z);
    }
    {  // S-box 8
    const uint4 kd = *reinterpret_cast<const uint4*>(k + 60);
    const uint32_t x0 = S[27] ^ kd.x;  // second copy
    const uint32_t x1 = S[28] ^ kd.y;
    const uint32_t x2 = S[29];
    const uint32_t x3 = S[30];
    const uint32_t x4 = S[31];
    const uint32_t x5 = S[0];
    const uint4 kc = *reinterpret_cast<const uint4*>(k + 56);
    const uint32_t s7_0 = lop3<0x39>(x0, x1, x4);
    const uint32_t s7_1 = lop3<0xd6>(x0, x1, x4);
    const uint32_t s7_2 = lop3<0xac>(x2, s7_0, s7_1);
    const uint32_t s7_3 = lop3<0x9d>(x0, x1, x4);
    const uint32_t s7_4 = lop3<0x6c>(x3, s7_2, s7_3);
    const uint32_t s7_5 = lop3<0x19>(x4, s7_2, s7_3);
    const uint32_t s7_6 = lop3<0x68>(x3, s7_1, s7_5);
    const uint32_t s7_7 = lop3<0xea>(x1, x3, s7_6);
    const uint32_t s7_8 = lop3<0x6c>(x5, s7_4, s7_7);
    T[20] = lop3<0x96>(T[20], s7_8, kc.w);
    const uint32_t s7_9 = lop3<0xcb>(x2, x4, x5);
    const uint32_t s7_10 = lop3<0xa3>(x0, s7_6, s7_9);
    const uint32_t s7_11 = lop3<0x96>(x5, x1, s7_10);
    const uint32_t s7_12 = lop3<0xac>(x0, x1, x5);
    const uint32_t s7_13 = lop3<0xea>(x2, s7_0, s7_12);
    const uint32_t s7_14 = lop3<0x6c>(x3, s7_11, s7_13);
    T[26] = lop3<0x96>(T[26], s7_14, kc.y);
    const uint32_t s7_15 = lop3<0x72>(x2, x3, x4);
    const uint32_t s7_16 = lop3<0x9e>(x4, x5, s7_4);
    const uint32_t s7_17 = lop3<0x6c>(x0, s7_15, s7_16);
    const uint32_t s7_18 = lop3<0x49>(x0, x5, s7_8);
    const uint32_t s7_19 = lop3<0xe9>(x3, s7_9, s7_18);
    const uint32_t s7_20 = lop3<0x6c>(x1, s7_17, s7_19);
    T[14] = lop3<0x96>(T[14], s7_20, kc.z);
    const uint32_t s7_21 = lop3<0xbd>(x1, x3, s7_15);
    const uint32_t s7_22 = lop3<0x92>(s7_14, s7_20, s7_21);
    const uint32_t s7_23 = lop3<0x36>(x5, s7_4, s7_22);
    const uint32_t s7_24 = lop3<0x9a>(x1, x5, s7_23);
    T[4] = lop3<0x96>(T[4], s7_24, kc.x);
    }
}

