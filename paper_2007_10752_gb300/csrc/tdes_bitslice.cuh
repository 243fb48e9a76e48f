// tdes_bitslice.cuh -- bitsliced 3DES-EDE3 core shared by every kernel.
//
// A thread holds 32 independent 64-bit blocks.  After a 32x32 bit-matrix
// transpose of their two 32-bit words, word A_w[c] holds one bit position of
// all 32 blocks ("bit-plane"), so one 32-bit logic instruction advances 32
// blocks at once.  The initial and final permutations and the expansion and
// permutation inside the round are then only renames of planes, and the
// S-boxes are circuits of LOP3 instructions (3-input lookup tables).
//
// What is computed is "Bit-level Parallelization of 3DES Encryption on GPU",
// Sec. III-B: IP, 16 rounds per DES pass, FP, and the EDE3 composition
// E_K3(D_K2(E_K1(P))) (decryption: D_K1(E_K2(D_K3(C)))).  Between the three
// DES passes FP and IP cancel, so the 48 rounds run back to back on the
// planes and only the half that takes the next XOR changes.
//
// Everything here is __host__ __device__ so that the same code can be run on
// the host by the generator's self-check; the kernels are the product.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define TDES_HD __host__ __device__ __forceinline__

template <int LUT>
TDES_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
#else
    uint32_t r = 0;
    for (int i = 0; i < 8; ++i)
        if ((LUT >> i) & 1) r |= ((i & 4) ? a : ~a) & ((i & 2) ? b : ~b) & ((i & 1) ? c : ~c);
    return r;
#endif
}

TDES_HD uint32_t byte_perm(uint32_t a, uint32_t b, uint32_t sel) {
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, sel);
#else
    uint64_t v = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xFF) << (8 * i);
    return r;
#endif
}

#include "generated/tdes_generated.cuh"

// In-place 32x32 bit-matrix transpose: afterwards bit s of A[c] is the old
// bit c of A[s].  Five stages each exchange one bit of the row index with
// the same bit of the column index; the 16- and 8-bit stages are byte
// permutes, the 4-, 2- and 1-bit stages a shift plus a LOP3 select per word.
TDES_HD void transpose32(uint32_t (&A)[32]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t a = A[i], b = A[i + 16];
        A[i] = byte_perm(a, b, 0x5410);
        A[i + 16] = byte_perm(a, b, 0x7632);
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i & 8) continue;
        const uint32_t a = A[i], b = A[i + 8];
        A[i] = byte_perm(a, b, 0x6240);
        A[i + 8] = byte_perm(a, b, 0x7351);
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i & 4) continue;
        const uint32_t a = A[i], b = A[i + 4];
        A[i] = lop3<0xe4>(a, b << 4, 0x0F0F0F0Fu);  // (a & m) | ((b << 4) & ~m)
        A[i + 4] = lop3<0xe4>(a >> 4, b, 0x0F0F0F0Fu);  // ((a >> 4) & m) | (b & ~m)
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i & 2) continue;
        const uint32_t a = A[i], b = A[i + 2];
        A[i] = lop3<0xe4>(a, b << 2, 0x33333333u);
        A[i + 2] = lop3<0xe4>(a >> 2, b, 0x33333333u);
    }
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
        const uint32_t a = A[i], b = A[i + 1];
        A[i] = lop3<0xe4>(a, b << 1, 0x55555555u);
        A[i + 1] = lop3<0xe4>(a >> 1, b, 0x55555555u);
    }
}
// lop3<0xe4>(x, y, m) = m ? x : y  (0xE4 = (0xAA & 0xF0) | (~0xAA & 0xCC)).

TDES_HD void xor_planes(uint32_t (&H)[32], const uint32_t* __restrict__ k) {
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(k + i);
        H[i] ^= v.x;
        H[i + 1] ^= v.y;
        H[i + 2] ^= v.z;
        H[i + 3] ^= v.w;
    }
}

// The 48 rounds of EDE3 on keyed planes.  tab is the per-key round-constant
// table (TDES_TABLE_WORDS words, encryption or decryption order) built by
// the key-schedule kernel.
// Each key-mask pass (prologue, the two re-keyings, epilogue) touches only the
// half whose stored key bits change there; the generator checks that the
// other half's constants are zero and says which half it is (TDES_*_HALF_R).
#define TDES_KEY_PASS(NAME, BASE)                           \
    do {                                                    \
        if (NAME##_HALF_R) xor_planes(Rh, tab + (BASE) + 32); \
        else xor_planes(Lh, tab + (BASE));                  \
    } while (0)

//
// STAGES = 1 runs a single DES pass (16 rounds) on a single-DES table
// (TDES1_TABLE_WORDS words: prologue, 16 rounds, epilogue).  The first
// pass of EDE3 targets the halves in the same order, so tdes_fp applies.
template <int STAGES = 3>
TDES_HD void tdes_rounds(uint32_t (&Lh)[32], uint32_t (&Rh)[32], const uint32_t* __restrict__ tab) {
    static_assert(STAGES == 1 || STAGES == 3, "one DES pass or EDE3");
    if constexpr (STAGES == 1) {
        TDES_KEY_PASS(TDES1_PRO, TDES_TABLE_PRO);
    } else {
        TDES_KEY_PASS(TDES_PRO, TDES_TABLE_PRO);
    }
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {  // first DES pass: rounds 0..15
        tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it));
        tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it + 1));
    }
    if constexpr (STAGES == 1) {
        TDES_KEY_PASS(TDES1_EPI, TDES1_TABLE_EPI);
    } else {
        TDES_KEY_PASS(TDES_REKEY16, TDES_TABLE_REKEY16);
#pragma unroll 1
        for (int it = 0; it < 8; ++it) {  // second pass: the XOR target repeats at its start
            tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (16 + 2 * it));
            tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (17 + 2 * it));
        }
        TDES_KEY_PASS(TDES_REKEY32, TDES_TABLE_REKEY32);
#pragma unroll 1
        for (int it = 0; it < 8; ++it) {  // third pass
            tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (32 + 2 * it));
            tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (33 + 2 * it));
        }
        TDES_KEY_PASS(TDES_EPI, TDES_TABLE_EPI);
    }
}

// The same with the pass count chosen at run time (the batch kernel, whose
// key tables mix EDE3 and single-DES schedules): the prologue and epilogue
// of the two table layouts touch the same halves, so the one-pass case only
// skips the re-keyings and the last two passes and takes its own epilogue.
static_assert(TDES_PRO_HALF_R == TDES1_PRO_HALF_R && TDES_EPI_HALF_R == TDES1_EPI_HALF_R,
              "runtime pass count assumes matching prologue and epilogue halves");
TDES_HD void tdes_rounds_rt(uint32_t (&Lh)[32], uint32_t (&Rh)[32], const uint32_t* __restrict__ tab,
                            bool one_pass) {
    TDES_KEY_PASS(TDES_PRO, TDES_TABLE_PRO);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it));
        tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it + 1));
    }
    if (one_pass) {
        TDES_KEY_PASS(TDES_EPI, TDES1_TABLE_EPI);
        return;
    }
    TDES_KEY_PASS(TDES_REKEY16, TDES_TABLE_REKEY16);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (16 + 2 * it));
        tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (17 + 2 * it));
    }
    TDES_KEY_PASS(TDES_REKEY32, TDES_TABLE_REKEY32);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (32 + 2 * it));
        tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (33 + 2 * it));
    }
    TDES_KEY_PASS(TDES_EPI, TDES_TABLE_EPI);
}

// 32 blocks: A0[s], A1[s] are the first and second little-endian 32-bit
// words of block s on entry and of its result on return.
template <int STAGES = 3>
TDES_HD void tdes_process32(uint32_t (&A0)[32], uint32_t (&A1)[32], const uint32_t* __restrict__ tab) {
    transpose32(A0);
    transpose32(A1);
    uint32_t Lh[32], Rh[32];
    tdes_ip(A0, A1, Lh, Rh);
    tdes_rounds<STAGES>(Lh, Rh, tab);
    tdes_fp(Lh, Rh, A0, A1);
    transpose32(A0);
    transpose32(A1);
}

TDES_HD void tdes_process32_rt(uint32_t (&A0)[32], uint32_t (&A1)[32],
                               const uint32_t* __restrict__ tab, bool one_pass) {
    transpose32(A0);
    transpose32(A1);
    uint32_t Lh[32], Rh[32];
    tdes_ip(A0, A1, Lh, Rh);
    tdes_rounds_rt(Lh, Rh, tab, one_pass);
    tdes_fp(Lh, Rh, A0, A1);
    transpose32(A0);
    transpose32(A1);
}
