// tdes_mixed.cuh -- bitsliced EDE3 on tiles whose 32 bit positions carry
// different keys (small messages of a batch under many key triples).
//
// In a tile of the single-key kernels every round-constant word is all 0 or
// all 1: one key for all 32 blocks of a lane.  Here bit s of every word
// belongs to "slice" s, and slice s has its own key, so a table word is the
// 32 slices' key bits side by side.  The rounds are those of
// tdes_bitslice.cuh ("Bit-level Parallelization of 3DES Encryption on GPU",
// Sec. III-B) with the doubled expansion inputs XORed plainly
// (tdes_round_mixed); the table is built per tile from the key table's
// bit-packed copies by 32x32 bit transposes across the lanes of a warp.
#pragma once
#include "tdes_bitslice.cuh"
#include "generated/tdes_generated_mixed.cuh"

#ifdef __CUDACC__
// Lane i holds row i of a 32x32 bit matrix (bit j = M[i][j]); returns column
// `lane` (bit i = M[i][lane]).  Each step swaps the off-diagonal blocks of
// width w between lanes i and i ^ w: the partner's word rotated left by w
// (by 32 - w in the lane of the pair whose bit w is set) has the block this
// lane takes in place, and one select under a per-lane mask merges it with
// the block this lane keeps.  Three operations a step (shuffle, rotate,
// select) where the two-branch form took about eight.
__device__ __forceinline__ uint32_t transpose_lanes32(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t hi = w == 16 ? 0xFFFF0000u
                          : w == 8  ? 0xFF00FF00u
                          : w == 4  ? 0xF0F0F0F0u
                          : w == 2  ? 0xCCCCCCCCu
                                    : 0xAAAAAAAAu;
        const bool upper = (lane & w) != 0;
        const uint32_t keep = upper ? hi : ~hi;  // this lane's own block
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, w);
        const uint32_t r = __funnelshift_l(y, y, upper ? 32 - w : w);
        x = (x & keep) | (r & ~keep);
    }
    return x;
}
#endif

// The 48 rounds of EDE3 on a table of per-slice masks (TDES_TABLE_WORDS
// words, the three-pass layout).
TDES_HD void tdes_rounds_mixed(uint32_t (&Lh)[32], uint32_t (&Rh)[32],
                               const uint32_t* __restrict__ tab) {
    TDES_KEY_PASS(TDES_PRO, TDES_TABLE_PRO);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round_mixed(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it));
        tdes_round_mixed(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (2 * it + 1));
    }
    TDES_KEY_PASS(TDES_REKEY16, TDES_TABLE_REKEY16);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round_mixed(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (16 + 2 * it));
        tdes_round_mixed(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (17 + 2 * it));
    }
    TDES_KEY_PASS(TDES_REKEY32, TDES_TABLE_REKEY32);
#pragma unroll 1
    for (int it = 0; it < 8; ++it) {
        tdes_round_mixed(Lh, Rh, tab + TDES_TABLE_ROUND0 + 64 * (32 + 2 * it));
        tdes_round_mixed(Rh, Lh, tab + TDES_TABLE_ROUND0 + 64 * (33 + 2 * it));
    }
    TDES_KEY_PASS(TDES_EPI, TDES_TABLE_EPI);
}

TDES_HD void tdes_process32_mixed(uint32_t (&A0)[32], uint32_t (&A1)[32],
                                  const uint32_t* __restrict__ tab) {
    transpose32(A0);
    transpose32(A1);
    uint32_t Lh[32], Rh[32];
    tdes_ip(A0, A1, Lh, Rh);
    tdes_rounds_mixed(Lh, Rh, tab);
    tdes_fp(Lh, Rh, A0, A1);
    transpose32(A0);
    transpose32(A1);
}
