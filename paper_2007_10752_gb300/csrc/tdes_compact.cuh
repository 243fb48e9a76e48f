// tdes_compact.cuh -- the 48 EDE3 rounds (Sec. III-B) with one copy of the
// round code for all three DES passes.
//
// tdes_rounds_rt and tdes_rounds_mixed spell the three passes out as three
// loops, because the second pass starts on the other half (the last swap of
// each DES pass is undone, so the XOR target repeats at a pass boundary).
// Here the halves' names are exchanged around the second pass instead (64
// register moves per tile), so the three passes run one loop body.  In
// kernels with much code outside the rounds, a third of the round code
// keeps the instruction cache from thrashing when warps sit in different
// passes: the uniform-message tiles measured 93 -> 75 ms on 2^28 messages,
// and the batch kernel 3.78 -> 3.60 ms on the 4096-message batch's parallel
// modes (its default form; the three-loop form stays selectable).  The
// single-key kernels keep the three-loop form, which measured faster there.
#pragma once
#include "tdes_mixed.cuh"

TDES_HD void swap_halves(uint32_t (&Lh)[32], uint32_t (&Rh)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const uint32_t t = Lh[i];
        Lh[i] = Rh[i];
        Rh[i] = t;
    }
}

// MIXED: per-slice table words (tdes_round_mixed); otherwise a single-key
// table, three passes or (one_pass) a single-DES table of one pass.
template <bool MIXED>
TDES_HD void tdes_rounds_compact(uint32_t (&Lh)[32], uint32_t (&Rh)[32],
                                 const uint32_t* __restrict__ tab, bool one_pass) {
    TDES_KEY_PASS(TDES_PRO, TDES_TABLE_PRO);
    const int passes = (!MIXED && one_pass) ? 1 : 3;
#pragma unroll 1
    for (int pass = 0; pass < passes; ++pass) {
        if (pass == 1) {
            TDES_KEY_PASS(TDES_REKEY16, TDES_TABLE_REKEY16);
            swap_halves(Lh, Rh);
        } else if (pass == 2) {
            swap_halves(Lh, Rh);
            TDES_KEY_PASS(TDES_REKEY32, TDES_TABLE_REKEY32);
        }
#pragma unroll 1
        for (int it = 0; it < 8; ++it) {
            const uint32_t* k = tab + TDES_TABLE_ROUND0 + 64 * (16 * pass + 2 * it);
            if (MIXED) {
                tdes_round_mixed(Lh, Rh, k);
                tdes_round_mixed(Rh, Lh, k + 64);
            } else {
                tdes_round(Lh, Rh, k);
                tdes_round(Rh, Lh, k + 64);
            }
        }
    }
    if (!MIXED && one_pass) {
        TDES_KEY_PASS(TDES_EPI, TDES1_TABLE_EPI);
        return;
    }
    TDES_KEY_PASS(TDES_EPI, TDES_TABLE_EPI);
}

template <bool MIXED>
TDES_HD void tdes_process32_compact(uint32_t (&A0)[32], uint32_t (&A1)[32],
                                    const uint32_t* __restrict__ tab, bool one_pass) {
    transpose32(A0);
    transpose32(A1);
    uint32_t Lh[32], Rh[32];
    tdes_ip(A0, A1, Lh, Rh);
    tdes_rounds_compact<MIXED>(Lh, Rh, tab, one_pass);
    tdes_fp(Lh, Rh, A0, A1);
    transpose32(A0);
    transpose32(A1);
}
