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
    if (STAGES == 1) {
        TDES_KEY_PASS(TDES1_PRO, TDES_TABLE_PRO);
    } else {
        TDES_KEY_PASS(TDES_PRO, TDES_TABLE_PRO);
    }
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {  // first DES pass: rounds 0..15
        tdes_round(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it));
        tdes_round(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it + 1));
    }
    if (STAGES == 1) {
        TDES_KEY_PASS(TDES1_EPI, TDES1_TABLE_EPI);
        return;
    }
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

// ---------------------------------------------------------------- scalar path
// One block at a time (serial CBC encryption).  A block is a 64-bit value
// with bit 1 at position 63 (big-endian bytes); a half has bit 1 at 31.

TDES_HD uint32_t rotr32(uint32_t x, int n) { return (x >> n) | (x << ((32 - n) & 31)); }

TDES_HD uint64_t permute64(uint64_t v, const uint8_t* __restrict__ src) {
    uint64_t r = 0;
    for (int j = 0; j < 64; ++j) r |= ((v >> (63 - src[j])) & 1ull) << (63 - j);
    return r;
}

// One Feistel round of the scalar path.  The expansion windows of S-boxes
// 1, 7, 5, 3 are the four bytes of rotr(R, 27) and those of S-boxes 2, 8, 6, 4
// the four bytes of rotr(R, 23) (six bits each, first bit most significant),
// so two rotates and two XORs with the round's key words ke/ko form all eight
// S-box inputs; sp[64g + x] is S-box g followed by the permutation.  Each
// six-bit index is extracted already scaled by 4 (a byte offset into sp).
TDES_HD uint32_t sp_at(const uint32_t* __restrict__ sp, int g, uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(sp + 64 * g) +
                                               byte_off);
}

TDES_HD uint32_t tdes_f_scalar(uint32_t R, uint32_t ke, uint32_t ko,
                               const uint32_t* __restrict__ sp) {
    const uint32_t we = rotr32(R, 27) ^ ke;
    const uint32_t wo = rotr32(R, 23) ^ ko;
    const uint32_t a = sp_at(sp, 0, (we << 2) & 0xFCu) ^ sp_at(sp, 6, (we >> 6) & 0xFCu) ^
                       sp_at(sp, 4, (we >> 14) & 0xFCu);
    const uint32_t b = sp_at(sp, 2, (we >> 22) & 0xFCu) ^ sp_at(sp, 1, (wo << 2) & 0xFCu) ^
                       sp_at(sp, 7, (wo >> 6) & 0xFCu);
    const uint32_t c = sp_at(sp, 5, (wo >> 14) & 0xFCu) ^ sp_at(sp, 3, (wo >> 22) & 0xFCu);
    return a ^ b ^ c;
}

// sp: 8 x 64 S-box/permutation words; keys: 48 rounds x (ke, ko) words (the
// round-key groups in the byte order of the expansion windows); ip/fp: the
// permutations as 0-based source bits.
TDES_HD uint64_t tdes_block_scalar(uint64_t v, const uint32_t* __restrict__ sp,
                                   const uint32_t* __restrict__ keys,
                                   const uint8_t* __restrict__ ip, const uint8_t* __restrict__ fp) {
    v = permute64(v, ip);
    uint32_t L = (uint32_t)(v >> 32), R = (uint32_t)v;
    for (int r = 0; r < 48; ++r) {
        const uint32_t t = L ^ tdes_f_scalar(R, keys[2 * r], keys[2 * r + 1], sp);
        L = R;
        R = t;
        if ((r & 15) == 15) {  // end of a DES pass: undo the last swap (R16 || L16)
            const uint32_t u = L;
            L = R;
            R = u;
        }
    }
    return permute64(((uint64_t)L << 32) | R, fp);
}

// Permutation of a 64-bit block by 16 nibble tables (tab[n][v]: the output
// bits contributed by value v in input nibble n); 16 independent lookups.
TDES_HD uint64_t permute64_nib(uint64_t v, const uint64_t* __restrict__ tab) {
    uint64_t r = 0;
#pragma unroll
    for (int n = 0; n < 16; ++n) r |= tab[16 * n + (uint32_t)((v >> (60 - 4 * n)) & 15u)];
    return r;
}

// The same EDE3 block as tdes_block_scalar with the permutations by nibble
// tables (ipn/fpn: 16 x 16 words each) instead of bit loops.  The 16 rounds
// of a DES pass are unrolled by two so that the halves alternate in place,
// and each round's key words are loaded one round ahead, off the chain of
// dependent operations that sets the latency of a block.  rounds = 16 runs
// single DES on the first 16 rounds' key words.
TDES_HD uint64_t tdes_block_scalar_nib(uint64_t v, const uint32_t* __restrict__ sp,
                                       const uint32_t* __restrict__ keys,
                                       const uint64_t* __restrict__ ipn,
                                       const uint64_t* __restrict__ fpn, int rounds = 48) {
    v = permute64_nib(v, ipn);
    uint32_t L = (uint32_t)(v >> 32), R = (uint32_t)v;
    uint32_t ke = keys[0], ko = keys[1];
    for (int r = 0; r < rounds; r += 2) {
        const uint32_t ke1 = keys[2 * r + 2], ko1 = keys[2 * r + 3];
        L ^= tdes_f_scalar(R, ke, ko, sp);
        const int rn = r + 2 < rounds ? r + 2 : r;  // the last prefetch rereads the last pair
        ke = keys[2 * rn];
        ko = keys[2 * rn + 1];
        R ^= tdes_f_scalar(L, ke1, ko1, sp);
        if ((r & 15) == 14) {  // end of a DES pass: R16 || L16 continues as the next L0 || R0
            const uint32_t u = L;
            L = R;
            R = u;
        }
    }
    return permute64_nib(((uint64_t)L << 32) | R, fpn);
}

#ifdef __CUDACC__
// Warp-cooperative EDE3 block for one serial chain per warp: lane l holds
// the constants of half bit i = 32 - l (TDES_LANE_SBOX_INIT) and computes that
// bit of the round function from its S-box output mask; one ballot gathers the
// 32 bits, so a round is rotate, XOR, shift and ballot instead of eight table
// lookups and their XOR tree.  IP and FP are two ballots each.  Every lane
// returns the same value.  keys: the chain's 384-byte round-key words (the
// scalar layout), in shared memory.
struct LaneConsts {
    uint32_t mlo, mhi, rot, keypos;
    uint32_t ip_hi, ip_lo, fp_hi, fp_lo;
};

__device__ __forceinline__ uint32_t lane_bit(uint64_t v, uint32_t src) {
    return (uint32_t)(v >> (63u - src)) & 1u;
}

// rounds = 16 runs single DES on the first 16 rounds' key words.
__device__ __forceinline__ uint64_t tdes_block_warp(uint64_t v, const LaneConsts& c,
                                                    const uint8_t* __restrict__ keys,
                                                    int rounds = 48) {
    uint32_t L = __ballot_sync(0xFFFFFFFFu, lane_bit(v, c.ip_hi));
    uint32_t R = __ballot_sync(0xFFFFFFFFu, lane_bit(v, c.ip_lo));
    uint32_t k = keys[c.keypos];
#pragma unroll 2
    for (int r = 0; r < rounds; ++r) {
        const uint32_t kn = keys[8 * (r + 1 < rounds ? r + 1 : r) + c.keypos];
        const uint32_t x = ((rotr32(R, (int)c.rot) & 63u) ^ k);
        const uint32_t w = (x & 32u) ? c.mhi : c.mlo;
        const uint32_t f = __ballot_sync(0xFFFFFFFFu, (w >> (x & 31u)) & 1u);
        const uint32_t t = L ^ f;
        L = R;
        R = t;
        if ((r & 15) == 15) {  // end of a DES pass: R16 || L16 continues as L0 || R0
            const uint32_t u = L;
            L = R;
            R = u;
        }
        k = kn;
    }
    const uint64_t pre = ((uint64_t)L << 32) | R;
    const uint32_t hi = __ballot_sync(0xFFFFFFFFu, lane_bit(pre, c.fp_hi));
    const uint32_t lo = __ballot_sync(0xFFFFFFFFu, lane_bit(pre, c.fp_lo));
    return ((uint64_t)hi << 32) | lo;
}
#endif

TDES_HD uint64_t bswap64(uint64_t x) {
    x = ((x & 0x00FF00FF00FF00FFull) << 8) | ((x >> 8) & 0x00FF00FF00FF00FFull);
    x = ((x & 0x0000FFFF0000FFFFull) << 16) | ((x >> 16) & 0x0000FFFF0000FFFFull);
    return (x << 32) | (x >> 32);
}
