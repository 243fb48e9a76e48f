// tdes_scalar.cuh -- one-block-at-a-time 3DES paths: the scalar round (one
// block per thread; small calls, small batch messages, short CBC chains) and
// the warp-cooperative round (one serial CBC-encryption chain per warp).
//
// Both compute the same EDE3 block as the bitsliced core of
// tdes_bitslice.cuh ("Bit-level Parallelization of 3DES Encryption on GPU",
// Sec. III-B), one 64-bit block at a time, with the expansion windows read
// out of rotated halves and the S-boxes and permutation as lookups.  ROUNDS
// is 48 (EDE3) or 16 (single DES, on the first 16 rounds' key words).
#pragma once
#include "tdes_bitslice.cuh"
#include "generated/tdes_generated_scalar.cuh"

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
// dependent operations that sets the latency of a block.
template <int ROUNDS = 48>
TDES_HD uint64_t tdes_block_scalar_nib(uint64_t v, const uint32_t* __restrict__ sp,
                                       const uint32_t* __restrict__ keys,
                                       const uint64_t* __restrict__ ipn,
                                       const uint64_t* __restrict__ fpn) {
    constexpr int rounds = ROUNDS;
    v = permute64_nib(v, ipn);
    uint32_t L = (uint32_t)(v >> 32), R = (uint32_t)v;
    uint32_t ke = keys[0], ko = keys[1];
#pragma unroll
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

template <int ROUNDS = 48>
__device__ __forceinline__ uint64_t tdes_block_warp(uint64_t v, const LaneConsts& c,
                                                    const uint8_t* __restrict__ keys) {
    constexpr int rounds = ROUNDS;
    uint32_t L = __ballot_sync(0xFFFFFFFFu, lane_bit(v, c.ip_hi));
    uint32_t R = __ballot_sync(0xFFFFFFFFu, lane_bit(v, c.ip_lo));
    uint32_t k = keys[c.keypos];
    // The S-box input is x = (rotr(R, rot) & 63) ^ k and the lane's bit is
    // bit (x & 31) of mhi or mlo as x's bit 5 says.  That bit 5 is R's bit
    // (rot + 5) XOR k's bit 5, so the key part of the choice is made before
    // R is known (m0, m1), and the in-word index is a rotate amount (only
    // its low 5 bits count): R -> {bit test, select} || {rotate, XOR} ->
    // rotate -> ballot.
    // Lane j's F bit is bit j of the new R once XORed with bit j of L, so
    // each lane XORs its own bit of L (Lb, taken from R a round ahead, off
    // the dependent path) into its vote and the ballot is the new R.
    const uint32_t b5 = 1u << ((c.rot + 5u) & 31u);
    uint32_t lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    uint32_t Lb = (L >> lane) & 1u;
#pragma unroll
    for (int r = 0; r < rounds; ++r) {
        const uint32_t kn = keys[8 * (r + 1 < rounds ? r + 1 : r) + c.keypos];
        const uint32_t m0 = (k & 32u) ? c.mhi : c.mlo;
        const uint32_t m1 = (k & 32u) ? c.mlo : c.mhi;
        const uint32_t w = (R & b5) ? m1 : m0;
        const uint32_t sh = __funnelshift_r(R, R, c.rot) ^ k;
        const uint32_t Rb = (R >> lane) & 1u;
        const uint32_t t = __ballot_sync(0xFFFFFFFFu, (__funnelshift_r(w, w, sh) ^ Lb) & 1u);
        L = R;
        Lb = Rb;
        R = t;
        if ((r & 15) == 15) {  // end of a DES pass: R16 || L16 continues as L0 || R0
            const uint32_t u = L;
            L = R;
            R = u;
            Lb = (L >> lane) & 1u;
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

#ifdef __CUDACC__
// One CBC-encryption chain walked by the calling warp: out_i = E(in_i XOR
// out_{i-1}), out_{-1} = iv, blocks as big-endian bytes.  keys: the chain's
// round-key words in shared memory.  The next plaintext block is loaded one
// block ahead.  A real call from the batch kernel: inlined there, the same loop
// ran 4% slower (1580 against 1511 ns per block).  The single-message kernel
// keeps its own inlined copy, which measured 1% faster than this call there.
__device__ const uint32_t kChainLaneSbox[32][4] = TDES_LANE_SBOX_INIT;
__device__ const uint32_t kChainLaneIP[32][2] = TDES_LANE_IP_INIT;
__device__ const uint32_t kChainLaneFP[32][2] = TDES_LANE_FP_INIT;

__device__ __forceinline__ LaneConsts chain_lane_consts(uint32_t lane) {
    LaneConsts c;
    c.mlo = kChainLaneSbox[lane][0];
    c.mhi = kChainLaneSbox[lane][1];
    c.rot = kChainLaneSbox[lane][2];
    c.keypos = kChainLaneSbox[lane][3];
    c.ip_hi = kChainLaneIP[lane][0];
    c.ip_lo = kChainLaneIP[lane][1];
    c.fp_hi = kChainLaneFP[lane][0];
    c.fp_lo = kChainLaneFP[lane][1];
    return c;
}

template <int ROUNDS>
__device__ __noinline__ void tdes_cbc_chain_warp(const uint8_t* in, uint8_t* out, uint64_t nblocks,
                                                 uint64_t iv, const uint8_t* __restrict__ keys,
                                                 uint32_t lane) {
    const LaneConsts c = chain_lane_consts(lane);
    const uint64_t* p = reinterpret_cast<const uint64_t*>(in);
    uint64_t* q = reinterpret_cast<uint64_t*>(out);
    uint64_t prev = iv;
    uint64_t next = p[0];
    for (uint64_t i = 0; i < nblocks; ++i) {
        const uint64_t x = bswap64(next) ^ prev;
        if (i + 1 < nblocks) next = p[i + 1];
        prev = tdes_block_warp<ROUNDS>(x, c, keys);
        if (lane == 0) q[i] = bswap64(prev);
    }
}
#endif
