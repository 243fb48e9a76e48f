// tdes_batch.cu -- many messages, each with its own key triple and mode, in
// one persistent launch.
//
// A planned batch holds three kinds of work item, claimed by warps through
// one global atomic counter (dynamic load balancing, no waiting between
// warps):
//   C  CBC-encryption chains: one lane per message, 32 messages per item,
//      longest first (each block needs the previous ciphertext, so a chain
//      is serial; these items are claimed first because they are the
//      critical path);
//   B  bitsliced warp tiles of 1024 blocks of one "large" message (more than
//      32 blocks) in ECB, CTR or CBC-decrypt mode; the warp stages that
//      message's 13 KB round-constant table in its own slice of shared
//      memory and keeps it while consecutive tiles share the key;
//   S  "small" messages (at most 32 blocks) packed whole, one block per lane,
//      run with the scalar round (their bytes are a tiny share of any
//      workload here, and a 1024-block tile would leave most lanes idle).
// The per-key tables live in a device-resident key table built by the
// key-schedule kernel for every triple at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/tdes.h"
#include "tdes_batch_internal.h"
#include "tdes_internal.h"
#include "tdes_compact.cuh"
#include "tdes_keysched.cuh"
#include "tdes_mixed.cuh"
#include "tdes_scalar.cuh"
#include "tdes_tune.h"

namespace tdes {

constexpr int kSmallBlocks = 32;                          // S messages: nblocks <= this
// Small messages go to mixed-key tiles when the batch has at least this many
// of their blocks (8 tiles' worth); fewer run one block per lane (S items),
// which finish sooner alone.
constexpr uint64_t kMixedMinBlocks = 8 * 1024;
// Messages of 33..kSplitBlocks blocks (up to 4 KiB) run as pieces of 32
// blocks in S items too, except in-place CBC decryption (a piece would read
// the block before it after another warp wrote it): a block's 48 dependent
// scalar rounds finish far sooner than a bitsliced tile, and a bitsliced tile
// would spend its full 1024-block work on them anyway.
constexpr uint64_t kSplitBlocks = 512;
constexpr uint64_t kSoloChainBlocks = 512;                // longer CBC-enc chains: one per warp
constexpr int kPerKeyWords = 2 * TDES_TABLE_WORDS;        // enc + dec bitsliced tables
constexpr int kPerKeyChunks = 2 * TDES_SUBKEY_WORDS;      // enc + dec scalar groups
constexpr int kWarpSmemBytes = TDES_TABLE_WORDS * 4;      // one table per warp (13 KB)
static_assert(32 * TDES_SUBKEY_WORDS <= kWarpSmemBytes, "scalar groups must fit a warp slice");

__device__ const uint32_t kBatchSP[8][64] = TDES_SP_INIT;
__device__ const uint64_t kBatchIPN[16][16] = TDES_IPN_INIT;
__device__ const uint64_t kBatchFPN[16][16] = TDES_FPN_INIT;
__device__ const uint8_t kBatchRecipe[2][TDES_TABLE_WORDS][3] = TDES_RECIPE_INIT;
__device__ const uint8_t kBatchRecipe1[2][TDES1_TABLE_WORDS][3] = TDES1_RECIPE_INIT;
__device__ const uint8_t kBatchSubkeyBits[2][48][48] = TDES_SUBKEY_INIT;

__device__ __forceinline__ uint32_t bswap32d(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

// ---------------------------------------------------------------- key table
__device__ __forceinline__ bool same_des_key(const uint8_t* a, const uint8_t* b) {
    uint32_t d = 0;
    for (int i = 0; i < 8; ++i) d |= (uint32_t)(a[i] ^ b[i]) & 0xFEu;  // parity bits ignored
    return d == 0;
}

// Thread per (key, word): bitsliced tables of both directions, then the
// scalar groups of both directions.  A triple with K1 = K2 (EDE3 = E_K3) or
// K2 = K3 (EDE3 = E_K1) gets single-DES tables under that key: the one-pass
// bitsliced table, and the scalar groups of EDE3 under (K, K, K), whose first
// 16 rounds are those of DES_K in both directions.
__global__ void tdes_keytable_kernel(const uint8_t* __restrict__ keys, uint32_t count,
                                     uint32_t* __restrict__ tabs, uint8_t* __restrict__ chunks,
                                     uint8_t* __restrict__ stages) {
    const uint64_t per_key = (uint64_t)kPerKeyWords + kPerKeyChunks;
    const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per_key * count) return;
    const uint32_t key = (uint32_t)(e / per_key);
    const uint32_t w = (uint32_t)(e % per_key);
    const uint8_t* k = keys + 24ull * key;
    const uint8_t* single = same_des_key(k, k + 8) ? k + 16 : same_des_key(k + 8, k + 16) ? k : nullptr;
    uint8_t eff[24];
    for (int i = 0; i < 24; ++i) eff[i] = single ? single[i % 8] : k[i];
    if (w == 0) stages[key] = single ? 1 : 3;
    if (w < kPerKeyWords) {
        const int dir = w / TDES_TABLE_WORDS, i = w % TDES_TABLE_WORDS;
        uint32_t v = 0;
        if (!single) v = tdes_table_word(eff, kBatchRecipe[dir][i]);
        else if (i < TDES1_TABLE_WORDS) v = tdes_table_word(eff, kBatchRecipe1[dir][i]);
        tabs[(uint64_t)key * kPerKeyWords + w] = v;
    } else {
        const int f = w - kPerKeyWords;
        const int dir = f / TDES_SUBKEY_WORDS, c = f % TDES_SUBKEY_WORDS;
        chunks[(uint64_t)key * kPerKeyChunks + f] =
            tdes_subkey_chunk(eff, &kBatchSubkeyBits[dir][c / 8][6 * (c % 8)]);
    }
}

// Thread per (key, direction, packed word q): bit j of the word is the low
// bit of word 32q + j of the three-pass table of the triple (EDE3 under
// (K, K, K) for a triple that reduces: the same cipher), the form the
// mixed-key tiles gather from.
__global__ void tdes_keytable_pack_kernel(const uint8_t* __restrict__ keys, uint32_t count,
                                          uint32_t* __restrict__ packed) {
    const uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (uint64_t)count * 2 * kPackedWords) return;
    const uint32_t key = (uint32_t)(e / (2 * kPackedWords));
    const int dir = (int)(e / kPackedWords % 2), q = (int)(e % kPackedWords);
    const uint8_t* k = keys + 24ull * key;
    const uint8_t* single = same_des_key(k, k + 8) ? k + 16 : same_des_key(k + 8, k + 16) ? k : nullptr;
    uint8_t eff[24];
    for (int i = 0; i < 24; ++i) eff[i] = single ? single[i % 8] : k[i];
    uint32_t w = 0;
    for (int j = 0; j < 32; ++j) w |= (tdes_table_word(eff, kBatchRecipe[dir][32 * q + j]) & 1u) << j;
    packed[e] = w;
}

// ------------------------------------------------------------ batch kernel

struct SharedTables {
    uint32_t sp[8 * 64];
    uint64_t ipn[16 * 16];
    uint64_t fpn[16 * 16];
};

// Shared memory of the batch kernel, at namespace scope so that the scalar
// item functions (real calls, see below) address it as shared memory rather
// than through generic pointers.
__shared__ __align__(16) SharedTables g_st;
extern __shared__ __align__(16) uint8_t g_dyn[];  // kWarpSmemBytes per warp

__device__ __forceinline__ int dir_of(uint32_t mode) {
    return (mode == TDES_MODE_ECB_DECRYPT || mode == TDES_MODE_CBC_DECRYPT) ? 1 : 0;
}

__device__ __forceinline__ uint64_t load_be(const uint8_t* p, uint64_t i) {
    return bswap64(reinterpret_cast<const uint64_t*>(p)[i]);
}
__device__ __forceinline__ void store_be(uint8_t* p, uint64_t i, uint64_t v) {
    reinterpret_cast<uint64_t*>(p)[i] = bswap64(v);
}

// One bitsliced tile: blocks [b0, b0 + 1024) of message m (ragged at the end).
// The message record is read again after the rounds rather than kept in
// registers across them (the 64 planes need the register file).  COMPACT
// runs the 48 rounds as one loop body for all three passes
// (tdes_compact.cuh) instead of one loop per pass: a launch-shape choice of
// the autotuner, the same arithmetic.
template <bool COMPACT>
__device__ __forceinline__ void batch_bs_tile(const BatchMsg* __restrict__ mp, uint64_t tile,
                                              uint64_t gtile, const uint32_t* __restrict__ tab,
                                              const uint64_t* __restrict__ halo, uint32_t lane,
                                              bool one_pass) {
    const uint64_t b0 = tile * kTileBlocks;
    uint32_t A0[32], A1[32];
    {
    const BatchMsg m = *mp;
    const uint64_t n = m.nblocks;
    const bool full = b0 + kTileBlocks <= n;
    const bool vec = full && (((reinterpret_cast<uintptr_t>(m.in) |
                                reinterpret_cast<uintptr_t>(m.out)) & 15u) == 0);
    if (m.mode == TDES_MODE_CTR) {
        const uint32_t nw = bswap32d((uint32_t)(m.iv >> 32));
        const uint32_t c0 = (uint32_t)m.iv;
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                A0[2 * j + h] = nw;
                A1[2 * j + h] = bswap32d(c0 + (uint32_t)(b0 + 2 * (32 * j + lane) + h));
            }
    } else if (vec) {
        const uint4* p = reinterpret_cast<const uint4*>(m.in) + (b0 >> 1) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint4 v = __ldcs(p + 32 * j);
            A0[2 * j] = v.x;
            A1[2 * j] = v.y;
            A0[2 * j + 1] = v.z;
            A1[2 * j + 1] = v.w;
        }
    } else {
        const uint2* p = reinterpret_cast<const uint2*>(m.in);
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t b = b0 + 2 * (32 * j + lane) + h;
                uint2 v = make_uint2(0u, 0u);
                if (b < n) v = __ldcs(p + b);
                A0[2 * j + h] = v.x;
                A1[2 * j + h] = v.y;
            }
    }
    }
    if (COMPACT)
        tdes_process32_compact<false>(A0, A1, tab, one_pass);
    else
        tdes_process32_rt(A0, A1, tab, one_pass);
    const BatchMsg m = *mp;
    const uint64_t n = m.nblocks;
    const bool full = b0 + kTileBlocks <= n;
    const bool vec = full && (((reinterpret_cast<uintptr_t>(m.in) |
                                reinterpret_cast<uintptr_t>(m.out)) & 15u) == 0);
    const uint2* c = reinterpret_cast<const uint2*>(m.in);
    if (m.mode == TDES_MODE_CTR && vec) {  // full 16-byte-aligned tile: 128-bit loads
        const uint4* p = reinterpret_cast<const uint4*>(m.in) + (b0 >> 1) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint4 v = __ldcs(p + 32 * j);
            A0[2 * j] ^= v.x;
            A1[2 * j] ^= v.y;
            A0[2 * j + 1] ^= v.z;
            A1[2 * j + 1] ^= v.w;
        }
        __syncwarp();  // in place: every lane has read its data before any lane writes
    } else if (m.mode == TDES_MODE_CTR) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t b = b0 + 2 * (32 * j + lane) + h;
                if (b < n) {
                    const uint2 v = __ldcs(c + b);
                    A0[2 * j + h] ^= v.x;
                    A1[2 * j + h] ^= v.y;
                }
            }
        __syncwarp();  // in place: every lane has read its data before any lane writes
    } else if (m.mode == TDES_MODE_CBC_DECRYPT) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint64_t b = b0 + 2 * (32 * j + lane);
            uint2 prev0, prev1 = make_uint2(0u, 0u);
            if (b == 0) {
                prev0 = make_uint2(bswap32d((uint32_t)(m.iv >> 32)), bswap32d((uint32_t)m.iv));
            } else if (j == 0 && lane == 0 && halo != nullptr && m.in == m.out) {
                const uint64_t hv = halo[gtile];
                prev0 = make_uint2((uint32_t)hv, (uint32_t)(hv >> 32));
            } else {
                prev0 = (b - 1 < n) ? c[b - 1] : make_uint2(0u, 0u);
            }
            if (b < n) prev1 = c[b];
            A0[2 * j] ^= prev0.x;
            A1[2 * j] ^= prev0.y;
            A0[2 * j + 1] ^= prev1.x;
            A1[2 * j + 1] ^= prev1.y;
        }
        __syncwarp();
    }
    if (vec) {
        uint4* q = reinterpret_cast<uint4*>(m.out) + (b0 >> 1) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            __stcs(q + 32 * j, make_uint4(A0[2 * j], A1[2 * j], A0[2 * j + 1], A1[2 * j + 1]));
    } else {
        uint2* q = reinterpret_cast<uint2*>(m.out);
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t b = b0 + 2 * (32 * j + lane) + h;
                if (b < n) __stcs(q + b, make_uint2(A0[2 * j + h], A1[2 * j + h]));
            }
    }
}

__device__ __forceinline__ void stage_chunks(uint8_t* dst, const uint8_t* __restrict__ src) {
    // 384 bytes = 24 x 16 bytes; src and dst are 16-byte aligned
#pragma unroll 4
    for (int i = 0; i < TDES_SUBKEY_WORDS / 16; ++i)
        reinterpret_cast<uint4*>(dst)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
}

// The scalar items are real calls (__noinline__): inlined, their register
// needs would be allocated together with the bitsliced path's 64 planes and
// force spills there; as calls they have their own allocation.

// S item: whole small messages, one block per lane.
__device__ __noinline__ void batch_scalar_item(const BatchParams& p, uint2 item, uint32_t warp,
                                               uint32_t lane) {
    uint8_t* warp_smem = g_dyn + (size_t)warp * kWarpSmemBytes;
    const SharedTables& st = g_st;
    // find this lane's (message, block): walk the item's pieces in order
    uint32_t msg = 0xFFFFFFFFu;
    uint64_t blk = 0;
    uint32_t acc = 0;
    for (uint32_t i = 0; i < item.y; ++i) {
        const SPiece pc = p.s_pieces[item.x + i];
        if (lane >= acc && lane < acc + pc.n) {
            msg = pc.msg;
            blk = pc.first + (lane - acc);
        }
        acc += pc.n;
    }
    uint64_t x = 0, prev = 0;
    BatchMsg m;
    if (msg != 0xFFFFFFFFu) {
        m = p.msgs[msg];
        stage_chunks(warp_smem + TDES_SUBKEY_WORDS * lane,
                     p.keychunks + (uint64_t)m.key * kPerKeyChunks +
                         TDES_SUBKEY_WORDS * dir_of(m.mode));
        if (m.mode == TDES_MODE_CTR) {
            x = (m.iv & 0xFFFFFFFF00000000ull) | (uint32_t)((uint32_t)m.iv + (uint32_t)blk);
            prev = load_be(m.in, blk);  // the data to XOR
        } else {
            x = load_be(m.in, blk);
            if (m.mode == TDES_MODE_CBC_DECRYPT) prev = blk ? load_be(m.in, blk - 1) : m.iv;
        }
    }
    __syncwarp();  // every read of the item's messages precedes every write (in place)
    if (msg != 0xFFFFFFFFu) {
        const uint32_t* ks = reinterpret_cast<const uint32_t*>(warp_smem + TDES_SUBKEY_WORDS * lane);
        uint64_t y = p.keystages[m.key] == 1
                         ? tdes_block_scalar_nib<16>(x, st.sp, ks, st.ipn, st.fpn)
                         : tdes_block_scalar_nib<48>(x, st.sp, ks, st.ipn, st.fpn);
        if (m.mode == TDES_MODE_CTR || m.mode == TDES_MODE_CBC_DECRYPT) y ^= prev;
        store_be(m.out, blk, y);
    }
    __syncwarp();
}

// Lane `lane` of slice sl: its message (index into msgs) and block, or false.
__device__ __forceinline__ bool mixed_slot(const BatchParams& p, const MSlice& sl, uint32_t lane,
                                           uint32_t* msg, uint32_t* blk) {
    if (lane >= sl.nvalid) return false;
    const uint32_t upto = sl.starts & (0xFFFFFFFFu >> (31u - lane));  // starts at lanes <= lane
    *msg = p.m_list[sl.msg0 + (uint32_t)__popc(upto) - 1u];
    *blk = lane - (31u - (uint32_t)__clz(upto));
    return true;
}

// One mixed-key tile of small messages (ECB, CTR, CBC decryption).  Slice s
// (bit position s of every plane) carries up to 32 blocks under its own key
// and direction, one per lane; its table bits come from the key table's
// packed copy, lane s loading slice s's row, and a transpose across the lanes
// turns 32 rows into 32 table words.
__device__ __forceinline__ void batch_mixed_tile(const BatchParams& p, uint32_t tile,
                                                 uint32_t warp, uint32_t lane) {
    uint32_t* wtab = reinterpret_cast<uint32_t*>(g_dyn + (size_t)warp * kWarpSmemBytes);
    const MSlice* sl = p.m_slices + 32ull * tile;
    {
        const uint32_t kd = sl[lane].keydir;
        const uint32_t* row = p.keypacked + ((uint64_t)(kd >> 1) * 2 + (kd & 1u)) * kPackedWords;
        __syncwarp();
#pragma unroll 1
        for (int q = 0; q < kPackedWords; ++q)
            wtab[32 * q + lane] = transpose_lanes32(__ldg(row + q), lane);
        __syncwarp();
    }
    uint32_t A0[32], A1[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        uint32_t mi, b;
        A0[s] = 0u;
        A1[s] = 0u;
        if (mixed_slot(p, sl[s], lane, &mi, &b)) {
            const BatchMsg m = p.msgs[mi];
            if (m.mode == TDES_MODE_CTR) {
                A0[s] = bswap32d((uint32_t)(m.iv >> 32));
                A1[s] = bswap32d((uint32_t)m.iv + b);
            } else {
                const uint2 v = reinterpret_cast<const uint2*>(m.in)[b];
                A0[s] = v.x;
                A1[s] = v.y;
            }
        }
    }
    tdes_process32_mixed(A0, A1, wtab);
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        uint32_t mi, b;
        const bool ok = mixed_slot(p, sl[s], lane, &mi, &b);
        BatchMsg m;
        if (ok) {
            m = p.msgs[mi];
            const uint2* c = reinterpret_cast<const uint2*>(m.in);
            if (m.mode == TDES_MODE_CTR) {
                const uint2 v = c[b];
                A0[s] ^= v.x;
                A1[s] ^= v.y;
            } else if (m.mode == TDES_MODE_CBC_DECRYPT) {
                const uint2 v = b ? c[b - 1]
                                  : make_uint2(bswap32d((uint32_t)(m.iv >> 32)), bswap32d((uint32_t)m.iv));
                A0[s] ^= v.x;
                A1[s] ^= v.y;
            }
        }
        __syncwarp();  // in place: every read of this slice's messages precedes its writes
        if (ok) reinterpret_cast<uint2*>(m.out)[b] = make_uint2(A0[s], A1[s]);
    }
}

// The mixed-key tiles of a plan, in a kernel of their own launched just
// before the persistent kernel: inside it, their code slowed the persistent
// kernel's other paths by 4% (alternating A/B runs on the 4096-message batch,
// which has no mixed-key tiles).  Warps stride over the tiles.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Batch timing (when p.batch_times is set): the first CTA of the batch's
// first kernel stamps the start; every warp of its last kernel counts itself
// out as it leaves, and the last one stamps the end.
__device__ __forceinline__ void stamp_start(const BatchParams& p) {
    if (p.batch_times != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
        p.batch_times[0] = global_ns();
}
__device__ __forceinline__ void stamp_warp_done(const BatchParams& p, uint32_t lane) {
    if (p.batch_times != nullptr && lane == 0) {
        const uint32_t n = atomicAdd(p.done_warps, 1u) + 1u;
        if (n == gridDim.x * (blockDim.x >> 5)) p.batch_times[1] = global_ns();
    }
}

__global__ void __launch_bounds__(256, 2) tdes_batch_mixed_kernel(BatchParams p) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    stamp_start(p);
    for (uint32_t t = blockIdx.x * warps + warp; t < p.n_m_tiles; t += gridDim.x * warps)
        batch_mixed_tile(p, t, warp, lane);
    if (p.times_end_in_mixed) stamp_warp_done(p, lane);
}


// One short CBC-encryption chain per lane (scalar round); the next block is
// loaded one iteration ahead, so its latency hides behind the current block.
template <int ROUNDS>
__device__ __forceinline__ void lane_chain(const BatchMsg& m, const SharedTables& st,
                                           const uint32_t* keys) {
    uint64_t prev = m.iv;
    uint64_t next = load_be(m.in, 0);
    for (uint64_t i = 0; i < m.nblocks; ++i) {
        const uint64_t x = next ^ prev;
        if (i + 1 < m.nblocks) next = load_be(m.in, i + 1);
        prev = tdes_block_scalar_nib<ROUNDS>(x, st.sp, keys, st.ipn, st.fpn);
        store_be(m.out, i, prev);
    }
}

// C item: CBC-encryption chains.  The first n_c_solo items (the longest
// chains) hold one chain each, walked by the whole warp (tdes_block_warp: a
// ballot per round, so the dependent chain per block is short); the rest hold
// up to 32 short chains, one per lane, with the scalar round.
__device__ __noinline__ void batch_cbc_enc_item(const BatchParams& p, uint32_t item,
                                                uint32_t warp, uint32_t lane) {
    uint8_t* warp_smem = g_dyn + (size_t)warp * kWarpSmemBytes;
    const SharedTables& st = g_st;
    if (item < p.n_c_solo) {
        const BatchMsg m = p.msgs[p.c_list[item]];
        const uint8_t* kg = p.keychunks + (uint64_t)m.key * kPerKeyChunks;
        for (int i = lane; i < TDES_SUBKEY_WORDS / 16; i += 32)
            reinterpret_cast<uint4*>(warp_smem)[i] = __ldg(reinterpret_cast<const uint4*>(kg) + i);
        __syncwarp();
        if (p.keystages[m.key] == 1)
            tdes_cbc_chain_warp<16>(m.in, m.out, m.nblocks, m.iv, warp_smem, lane);
        else
            tdes_cbc_chain_warp<48>(m.in, m.out, m.nblocks, m.iv, warp_smem, lane);
        __syncwarp();
        return;
    }
    const uint32_t idx = p.n_c_solo + 32u * (item - p.n_c_solo) + lane;
    const uint32_t end = p.n_c;
    if (idx < end) {
        const BatchMsg m = p.msgs[p.c_list[idx]];
        uint8_t* ch = warp_smem + TDES_SUBKEY_WORDS * lane;
        stage_chunks(ch, p.keychunks + (uint64_t)m.key * kPerKeyChunks);
        const uint32_t* ks = reinterpret_cast<const uint32_t*>(ch);
        if (p.keystages[m.key] == 1)
            lane_chain<16>(m, st, ks);
        else
            lane_chain<48>(m, st, ks);
    }
    __syncwarp();
}

// SOLO_SLOTS: the plan has chains over 512 blocks, each walked by one warp.
// They are latency-bound, and two on one SM sub-partition (SMSP) slow each
// other down (a 4096-message batch: 865 against 517 ms), so each is taken
// only by a warp that holds its SMSP's slot (%smid, %warpid: a placement hint
// that correctness does not rely on).  A slot holder releases it after its
// chain and claims again, so every such chain is taken: a warp leaves only
// when the other items are gone and the chains are gone or its slot is held
// by another warp, which will come back for them.  Without such chains the
// kernel claims from one counter only (the slot logic measured 3% slower on
// the other items even when unused).  COMPACT: the round form of the tiles
// (batch_bs_tile).
template <bool SOLO_SLOTS, bool COMPACT>
__global__ void __launch_bounds__(256, 2) tdes_batch_kernel(BatchParams p) {
    if (p.n_m_tiles == 0) stamp_start(p);  // else the mixed-key kernel ran first
    for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) g_st.sp[i] = (&kBatchSP[0][0])[i];
    for (int i = threadIdx.x; i < 16 * 16; i += blockDim.x) {
        g_st.ipn[i] = (&kBatchIPN[0][0])[i];
        g_st.fpn[i] = (&kBatchFPN[0][0])[i];
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* wtab = reinterpret_cast<uint32_t*>(g_dyn + (size_t)warp * kWarpSmemBytes);
    uint32_t staged = ~0u;  // (key << 1 | dir) of the table in wtab
    // B tiles [t0, t1): the plan maps each tile to its message entry; the
    // warp restages its key table only when the key or direction changes
    auto run_tiles = [&](uint64_t t0, uint64_t t1) {
        for (uint64_t t = t0; t < t1; ++t) {
            const uint32_t lo = p.b_tile[t];
            const BatchMsg* mp = p.msgs + p.b_msg[lo];
            const uint32_t key = mp->key, dir = (uint32_t)dir_of(mp->mode);
            const uint32_t want = (key << 1) | dir;
            const bool one_pass = p.keystages[key] == 1;
            if (want != staged) {
                __syncwarp();
                const uint4* src = reinterpret_cast<const uint4*>(
                    p.keytab + (uint64_t)key * kPerKeyWords + TDES_TABLE_WORDS * dir);
                const int n4 = (one_pass ? TDES1_TABLE_WORDS : TDES_TABLE_WORDS) / 4;
                for (int i = lane; i < n4; i += 32)
                    reinterpret_cast<uint4*>(wtab)[i] = __ldg(src + i);
                __syncwarp();
                staged = want;
            }
            batch_bs_tile<COMPACT>(mp, t - p.b_prefix[lo], t, wtab, p.halo, lane, one_pass);
        }
    };
    const uint64_t total = (uint64_t)p.n_c_items + p.n_b_chunks + p.n_s_items;
    uint32_t slot = 0;
    bool solo_left = SOLO_SLOTS;
    if (SOLO_SLOTS) {
        uint32_t smid, wid;
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        asm("mov.u32 %0, %%warpid;" : "=r"(wid));
        slot = (smid * 4u + (wid & 3u)) % (uint32_t)kChainSlots;
    }
    for (;;) {
        unsigned long long item = 0;
        bool slotted = false;
        if (!SOLO_SLOTS) {
            if (lane == 0) item = atomicAdd(p.counter, 1ull);
            item = __shfl_sync(0xFFFFFFFFu, item, 0);
            if (item >= total) item = ~0ull;
        } else {
            uint32_t gone = 0;
            item = ~0ull;
            if (lane == 0) {
                if (solo_left && atomicCAS(&p.chain_slot[slot], 0u, 1u) == 0u) {
                    const unsigned long long c = atomicAdd(p.c_counter, 1ull);
                    if (c < p.n_c_solo) {
                        item = c;
                    } else {
                        atomicExch(&p.chain_slot[slot], 0u);
                        gone = 1;
                    }
                }
                if (item == ~0ull) {  // packed chains, tiles, small items
                    const unsigned long long o = atomicAdd(p.counter, 1ull);
                    if (o < total - p.n_c_solo) item = p.n_c_solo + o;
                }
            }
            item = __shfl_sync(0xFFFFFFFFu, item, 0);
            if (__shfl_sync(0xFFFFFFFFu, gone, 0)) solo_left = false;
            slotted = item < p.n_c_solo;
        }
        if (item == ~0ull) break;
        if (item < p.n_c_items) {
            batch_cbc_enc_item(p, (uint32_t)item, warp, lane);
            if (SOLO_SLOTS && slotted && lane == 0) atomicExch(&p.chain_slot[slot], 0u);
            staged = ~0u;
            continue;
        }
        item -= p.n_c_items;
        if (item < p.n_b_chunks) {  // a run of b_chunk consecutive tiles
            const uint64_t t0 = item * p.b_chunk;
            run_tiles(t0, min(t0 + p.b_chunk, p.n_b_tiles));
            continue;
        }
        item -= p.n_b_chunks;
        batch_scalar_item(p, p.s_items[item], warp, lane);
        staged = ~0u;
    }
    stamp_warp_done(p, lane);
}

// In-place CBC decryption: save the ciphertext block before every B tile
// (after the first of its message) before any tile is overwritten.
__global__ void tdes_batch_halo_kernel(BatchParams p) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n_b_tiles) return;
    const uint32_t lo = p.b_tile[t];
    const BatchMsg m = p.msgs[p.b_msg[lo]];
    const uint64_t k = t - p.b_prefix[lo];
    if (m.mode == TDES_MODE_CBC_DECRYPT && m.in == m.out && k >= 1)
        p.halo[t] = reinterpret_cast<const uint64_t*>(m.in)[k * kTileBlocks - 1];
}

}  // namespace tdes

// ===================================================================== host

namespace tdes {

int validate_desc(const tdes_desc_t& d, uint32_t key_count) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(d.in), o = reinterpret_cast<uintptr_t>(d.out);
    if (d.mode > TDES_MODE_CBC_ENCRYPT || d.key_index >= key_count || d.nbytes % 8 != 0)
        return TDES_EINVAL;
    if (d.nbytes > 0 && (d.in == nullptr || d.out == nullptr || ((a | o) & 7u))) return TDES_EINVAL;
    if (a != o && a < o + d.nbytes && o < a + d.nbytes) return TDES_EINVAL;
    if (d.mode == TDES_MODE_CTR && (d.iv_or_ctr & 0xFFFFFFFFull) + d.nbytes / 8 > (1ull << 32))
        return TDES_EINVAL;
    return TDES_OK;
}

static size_t align16(size_t x) { return (x + 15) / 16 * 16; }

void build_plan(const tdes_desc_t* descs, uint32_t count, uint32_t key_count, int* status,
                PlanHost* h, bool allow_direct) {
    std::vector<BatchMsg> msgs;
    std::vector<uint32_t> c_list, b_msg, s_list;
    std::vector<SPiece> split, pieces;
    std::vector<uint64_t> b_prefix(1, 0);
    std::vector<uint2> s_items;
    *h = PlanHost();
    msgs.reserve(count);
    for (uint32_t i = 0; i < count; ++i) {
        const tdes_desc_t& d = descs[i];
        const int st = validate_desc(d, key_count);
        if (status) status[i] = st;
        if (st != TDES_OK) {
            ++h->invalid;
            continue;
        }
        if (d.nbytes == 0) continue;
        const uint32_t mi = (uint32_t)msgs.size();
        const uint64_t nb = d.nbytes / 8;
        msgs.push_back({static_cast<const uint8_t*>(d.in), static_cast<uint8_t*>(d.out), nb,
                        d.iv_or_ctr, d.key_index, d.mode});
        h->bytes_per_mode[d.mode] += d.nbytes;
        if (d.mode == TDES_MODE_CBC_ENCRYPT) {
            c_list.push_back(mi);
        } else if (nb <= (uint64_t)kSmallBlocks) {
            s_list.push_back(mi);
        } else if (allow_direct && d.nbytes >= kDirectBytes &&
                   !(d.mode == TDES_MODE_CBC_DECRYPT && d.in == d.out)) {
            h->direct.push_back({d.mode, d.key_index, d.iv_or_ctr,
                                 static_cast<const uint8_t*>(d.in), static_cast<uint8_t*>(d.out),
                                 nb, 3});
        } else if (nb <= kSplitBlocks && !(d.mode == TDES_MODE_CBC_DECRYPT && d.in == d.out)) {
            for (uint32_t f = 0; f < nb; f += kSmallBlocks)
                split.push_back({mi, f, (uint32_t)std::min<uint64_t>(kSmallBlocks, nb - f), 0u});
        } else {
            b_msg.push_back(mi);
            b_prefix.push_back(b_prefix.back() + (nb + kTileBlocks - 1) / kTileBlocks);
            if (d.mode == TDES_MODE_CBC_DECRYPT && d.in == d.out) h->needs_halo = true;
        }
    }
    std::stable_sort(c_list.begin(), c_list.end(),
                     [&](uint32_t x, uint32_t y) { return msgs[x].nblocks > msgs[y].nblocks; });
    // Many small messages: mixed-key tiles.  Sorted by (key, direction),
    // they fill slices of up to 32 blocks under one key and direction (a
    // message never splits), and 32 slices make a tile.
    std::vector<uint32_t> m_list;
    std::vector<MSlice> m_slices;
    uint64_t small_blocks = 0;
    for (uint32_t mi : s_list) small_blocks += msgs[mi].nblocks;
    const bool mixed = small_blocks >= kMixedMinBlocks;
    h->kind_bytes[mixed ? 1 : 2] += 8 * small_blocks;
    for (uint32_t mi : c_list) h->kind_bytes[3] += 8 * msgs[mi].nblocks;
    for (uint32_t mi : b_msg) h->kind_bytes[0] += 8 * msgs[mi].nblocks;
    for (const SPiece& pc : split) h->kind_bytes[2] += 8ull * pc.n;
    for (const DirectMsg& m : h->direct) h->kind_bytes[4] += 8 * m.nblocks;
    if (mixed) {
        auto keydir = [&](uint32_t mi) {
            const uint32_t dir = (msgs[mi].mode == TDES_MODE_ECB_DECRYPT ||
                                  msgs[mi].mode == TDES_MODE_CBC_DECRYPT) ? 1u : 0u;
            return (msgs[mi].key << 1) | dir;
        };
        std::stable_sort(s_list.begin(), s_list.end(),
                         [&](uint32_t x, uint32_t y) { return keydir(x) < keydir(y); });
        MSlice cur = {0, 0, 0, 0};
        bool open = false;
        for (uint32_t mi : s_list) {
            const uint32_t kd = keydir(mi), nb = (uint32_t)msgs[mi].nblocks;
            if (open && (cur.keydir != kd || cur.nvalid + nb > 32u)) {
                m_slices.push_back(cur);
                open = false;
            }
            if (!open) {
                cur = {(uint32_t)m_list.size(), 0u, 0u, kd};
                open = true;
            }
            cur.starts |= 1u << cur.nvalid;
            cur.nvalid += nb;
            m_list.push_back(mi);
        }
        if (open) m_slices.push_back(cur);
        while (m_slices.size() % 32) m_slices.push_back({0u, 0u, 0u, 0u});  // empty slices
        h->n_m_tiles = (uint32_t)(m_slices.size() / 32);
        s_list.clear();
    }
    // S items: whole small messages (unless in mixed-key tiles) and the
    // pieces of medium ones, packed in order up to 32 blocks per item
    for (uint32_t mi : s_list) pieces.push_back({mi, 0u, (uint32_t)msgs[mi].nblocks, 0u});
    pieces.insert(pieces.end(), split.begin(), split.end());
    for (uint32_t i = 0; i < pieces.size();) {
        const uint32_t first = i;
        uint32_t blocks = 0;
        while (i < pieces.size() && blocks + pieces[i].n <= (uint32_t)kSmallBlocks)
            blocks += pieces[i++].n;
        s_items.push_back(make_uint2(first, i - first));
    }
    h->n_c = (uint32_t)c_list.size();
    while (h->n_c_solo < h->n_c && msgs[c_list[h->n_c_solo]].nblocks > kSoloChainBlocks)
        ++h->n_c_solo;
    h->n_c_items = h->n_c_solo + (h->n_c - h->n_c_solo + 31) / 32;
    h->n_b = (uint32_t)b_msg.size();
    h->n_b_tiles = b_prefix.back();
    h->n_s_items = (uint32_t)s_items.size();
    h->total_items = (uint64_t)h->n_c_items + h->n_b_tiles + h->n_m_tiles + h->n_s_items;
    size_t off = 0;
    auto take = [&](size_t n) { const size_t o = align16(off); off = o + n; return o; };
    h->o_msgs = take(msgs.size() * sizeof(BatchMsg));
    h->o_c = take(c_list.size() * 4);
    h->o_bm = take(b_msg.size() * 4);
    h->o_bp = take(b_prefix.size() * 8);
    h->o_bt = take(h->n_b_tiles * 4);
    h->o_ml = take(m_list.size() * 4);
    h->o_ms = take(m_slices.size() * sizeof(MSlice));
    h->o_sl = take(pieces.size() * sizeof(SPiece));
    h->o_si = take(s_items.size() * sizeof(uint2));
    h->o_halo = take(h->needs_halo ? h->n_b_tiles * 8 : 0);
    h->o_ctr = take(kCounterBytes);  // claim counters and chain slots: zeroed together
    h->image.assign(align16(off), 0);
    auto put = [&](size_t o, const void* src, size_t n) {
        if (n) memcpy(h->image.data() + o, src, n);
    };
    put(h->o_msgs, msgs.data(), msgs.size() * sizeof(BatchMsg));
    put(h->o_c, c_list.data(), c_list.size() * 4);
    put(h->o_bm, b_msg.data(), b_msg.size() * 4);
    put(h->o_bp, b_prefix.data(), b_prefix.size() * 8);
    uint32_t* bt = reinterpret_cast<uint32_t*>(h->image.data() + h->o_bt);
    for (uint32_t i = 0; i < h->n_b; ++i)
        std::fill(bt + b_prefix[i], bt + b_prefix[i + 1], i);
    put(h->o_ml, m_list.data(), m_list.size() * 4);
    put(h->o_ms, m_slices.data(), m_slices.size() * sizeof(MSlice));
    put(h->o_sl, pieces.data(), pieces.size() * sizeof(SPiece));
    put(h->o_si, s_items.data(), s_items.size() * sizeof(uint2));
}

BatchParams bind_plan(const PlanHost& h, void* dev_base, const tdes_keytable* kt) {
    uint8_t* base = static_cast<uint8_t*>(dev_base);
    BatchParams p;
    p.msgs = reinterpret_cast<const BatchMsg*>(base + h.o_msgs);
    p.keytab = kt->tabs;
    p.keychunks = kt->chunks;
    p.keystages = kt->stages;
    p.c_list = reinterpret_cast<const uint32_t*>(base + h.o_c);
    p.n_c = h.n_c;
    p.n_c_items = h.n_c_items;
    p.n_c_solo = h.n_c_solo;
    p.b_msg = reinterpret_cast<const uint32_t*>(base + h.o_bm);
    p.b_prefix = reinterpret_cast<const uint64_t*>(base + h.o_bp);
    p.b_tile = reinterpret_cast<const uint32_t*>(base + h.o_bt);
    p.n_b = h.n_b;
    p.n_b_tiles = h.n_b_tiles;
    p.keypacked = kt->packed;
    p.m_list = reinterpret_cast<const uint32_t*>(base + h.o_ml);
    p.m_slices = reinterpret_cast<const MSlice*>(base + h.o_ms);
    p.n_m_tiles = h.n_m_tiles;
    p.s_pieces = reinterpret_cast<const SPiece*>(base + h.o_sl);
    p.s_items = reinterpret_cast<const uint2*>(base + h.o_si);
    p.n_s_items = h.n_s_items;
    p.halo = h.needs_halo ? reinterpret_cast<uint64_t*>(base + h.o_halo) : nullptr;
    p.counter = reinterpret_cast<unsigned long long*>(base + h.o_ctr);
    p.c_counter = p.counter + 1;
    p.done_warps = reinterpret_cast<uint32_t*>(p.counter + 2);
    p.chain_slot = reinterpret_cast<uint32_t*>(p.counter + 4);
    p.batch_times = nullptr;
    p.times_end_in_mixed = false;
    return p;
}

cudaError_t prepare_batch_kernel(int warps, size_t* dyn_smem, int* ctas_fit) {
    const size_t dyn = (size_t)warps * kWarpSmemBytes;
    // The limit is a property of the kernel function shared by every plan, so
    // it is always set for the largest shape (8 warps) rather than this one.
    const void* fns[] = {(const void*)tdes_batch_kernel<false, false>,
                         (const void*)tdes_batch_kernel<true, false>,
                         (const void*)tdes_batch_kernel<false, true>,
                         (const void*)tdes_batch_kernel<true, true>,
                         (const void*)tdes_batch_mixed_kernel};
    cudaError_t e = cudaSuccess;
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 8 * kWarpSmemBytes);
        if (e != cudaSuccess) return e;
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tdes_batch_kernel<false, false>,
                                                      32 * warps, dyn);
    if (e != cudaSuccess) return e;
    *dyn_smem = dyn;
    *ctas_fit = n < 1 ? 1 : n;
    return cudaSuccess;
}

// A claimed tile takes a warp tens of microseconds at full occupancy, which
// already hides its message search and key staging behind the other warps,
// so claims are single tiles unless a batch has so many tiles (over 256 per
// warp) that the atomic counter itself and the restaging become worth
// amortising; the tail of a batch then costs at most one claim.
uint32_t auto_tiles_per_claim(uint64_t n_tiles, uint64_t warps_total) {
    return n_tiles > 256 * std::max<uint64_t>(1, warps_total) ? 4u : 1u;
}

cudaError_t enqueue_batch(const BatchParams& p_in, uint64_t total_items, bool needs_halo,
                          const LaunchShape& shape, size_t dyn_smem, uint64_t max_ctas,
                          cudaStream_t s, bool counter_fresh) {
    if (total_items == 0) return cudaSuccess;
    BatchParams p = p_in;
    const int warps = shape.warps;
    const uint64_t warps_total = std::max<uint64_t>(1, max_ctas * (uint64_t)warps);
    p.b_chunk = shape.tiles_per_claim > 0 ? (uint32_t)shape.tiles_per_claim
                                          : auto_tiles_per_claim(p.n_b_tiles, warps_total);
    p.n_b_chunks = (p.n_b_tiles + p.b_chunk - 1) / p.b_chunk;
    total_items = (uint64_t)p.n_c_items + p.n_b_chunks + p.n_s_items;
    cudaError_t e = cudaSuccess;
    if (!counter_fresh) {
        e = cudaMemsetAsync(p.counter, 0, kCounterBytes, s);
        if (e != cudaSuccess) return e;
    }
    if (needs_halo && p.n_b_tiles) {
        tdes_batch_halo_kernel<<<(unsigned)((p.n_b_tiles + 255) / 256), 256, 0, s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    p.times_end_in_mixed = total_items == 0;
    if (p.n_m_tiles) {  // small messages of their own keys: disjoint from the rest
        const uint64_t want = (p.n_m_tiles + warps - 1) / (uint64_t)warps;
        const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(want, max_ctas));
        tdes_batch_mixed_kernel<<<grid, 32 * warps, dyn_smem, s>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (total_items == 0) return cudaSuccess;
    const uint64_t want = (total_items + warps - 1) / (uint64_t)warps;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min(want, max_ctas));
    const bool solo = p.n_c_solo != 0, compact = shape.round_form == 1;
    if (solo && compact)
        tdes_batch_kernel<true, true><<<grid, 32 * warps, dyn_smem, s>>>(p);
    else if (solo)
        tdes_batch_kernel<true, false><<<grid, 32 * warps, dyn_smem, s>>>(p);
    else if (compact)
        tdes_batch_kernel<false, true><<<grid, 32 * warps, dyn_smem, s>>>(p);
    else
        tdes_batch_kernel<false, false><<<grid, 32 * warps, dyn_smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t enqueue_direct(const std::vector<DirectMsg>& direct, const tdes_keytable* kt,
                           int device, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (const DirectMsg& m : direct) {
        const uint32_t dir = (m.mode == TDES_MODE_ECB_DECRYPT || m.mode == TDES_MODE_CBC_DECRYPT);
        const uint32_t* tab = kt->tabs + ((uint64_t)m.key * 2 + dir) * TDES_TABLE_WORDS;
        const bool vec16 = ((reinterpret_cast<uintptr_t>(m.in) | reinterpret_cast<uintptr_t>(m.out)) &
                            15u) == 0;
        const uint64_t ntiles = (m.nblocks + kTileBlocks - 1) / kTileBlocks;
        if (m.mode == TDES_MODE_CTR) {
            e = launch_ctr(tab, m.stages, (uint32_t)(m.iv >> 32), (uint32_t)m.iv, m.in, m.out,
                           m.nblocks, vec16, geometry_for(ntiles, kCtr, device), s);
        } else if (m.mode == TDES_MODE_CBC_DECRYPT) {
            e = launch_cbc_dec(tab, m.stages, m.iv, m.in, m.out, m.nblocks, nullptr, vec16,
                               geometry_for(ntiles, kCbcDec, device), s);
        } else {
            e = launch_ecb(tab, m.stages, m.in, m.out, m.nblocks, vec16,
                           geometry_for(ntiles, kEcb, device), s);
        }
        if (e != cudaSuccess) return e;
    }
    return e;
}

}  // namespace tdes

namespace {

int bfail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tdes::set_last_error(buf);
    return status;
}

int bcuda(cudaError_t e, const char* what) {
    return bfail(e == cudaErrorMemoryAllocation ? TDES_ENOMEM : TDES_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

}  // namespace

namespace tdes {

int set_batch_shape(tdes_batch* b, const LaunchShape& shape_in) {
    LaunchShape shape = shape_in;
    if (shape.warps < 1 || shape.warps > 8 || shape.tiles_per_claim < 0 ||
        shape.tiles_per_claim > 1024 || shape.round_form < 0 || shape.round_form > 1)
        return bfail(TDES_EINVAL, "launch shape: 1..8 warps per CTA, 0..1024 tiles per claim, "
                                  "round form 0 or 1");
    size_t dyn = 0;
    int fit = 1;
    cudaError_t e = prepare_batch_kernel(shape.warps, &dyn, &fit);
    if (e != cudaSuccess) return bcuda(e, "batch kernel set-up");
    shape.ctas_per_sm = shape.ctas_per_sm < 1 ? fit : std::min(shape.ctas_per_sm, fit);
    b->shape = shape;
    b->ctas_fit = fit;
    b->dyn_smem = dyn;
    if (b->exec) {  // launch shape changed: recapture on next graph launch
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    return TDES_OK;
}

cudaError_t enqueue_planned(tdes_batch* b, cudaStream_t s) {
    cudaError_t e = enqueue_direct(b->direct, b->kt, b->device, s);
    if (e != cudaSuccess || b->total_items == 0) return e;
    return enqueue_batch(b->params, b->total_items, b->needs_halo, b->shape, b->dyn_smem,
                         (uint64_t)b->sms * b->shape.ctas_per_sm, s);
}

}  // namespace tdes

extern "C" {


int tdes_keytable_create(const uint8_t* keys, uint32_t count, tdes_keytable_t** out) {
    if (out == nullptr || (keys == nullptr && count > 0))
        return bfail(TDES_EINVAL, "NULL argument to tdes_keytable_create");
    *out = nullptr;
    if (count == 0) return bfail(TDES_EINVAL, "empty key table");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    const size_t tab_bytes = (size_t)count * tdes::kPerKeyWords * 4;
    const size_t chunk_bytes = tdes::align16((size_t)count * tdes::kPerKeyChunks);
    const size_t key_bytes = tdes::align16((size_t)count * 24);
    const size_t stage_bytes = tdes::align16(count);
    const size_t packed_bytes = (size_t)count * 2 * tdes::kPackedWords * 4;
    void* mem = nullptr;
    e = cudaMalloc(&mem, tab_bytes + chunk_bytes + key_bytes + stage_bytes + packed_bytes);
    if (e != cudaSuccess) return bcuda(e, "cudaMalloc(key table)");
    tdes_keytable_t* kt = new (std::nothrow) tdes_keytable_t;
    if (kt == nullptr) {
        cudaFree(mem);
        return bfail(TDES_ENOMEM, "host allocation failed");
    }
    kt->device = dev;
    kt->count = count;
    kt->mem = mem;
    kt->tabs = static_cast<uint32_t*>(mem);
    kt->chunks = static_cast<uint8_t*>(mem) + tab_bytes;
    uint8_t* dkeys = kt->chunks + chunk_bytes;
    kt->stages = dkeys + key_bytes;
    kt->packed = reinterpret_cast<uint32_t*>(kt->stages + stage_bytes);
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dkeys, keys, (size_t)count * 24, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const uint64_t n = (uint64_t)count * (tdes::kPerKeyWords + tdes::kPerKeyChunks);
        tdes::tdes_keytable_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            dkeys, count, kt->tabs, kt->chunks, kt->stages);
        e = cudaGetLastError();
        const uint64_t np = (uint64_t)count * 2 * tdes::kPackedWords;
        if (e == cudaSuccess) {
            tdes::tdes_keytable_pack_kernel<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(
                dkeys, count, kt->packed);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(dkeys, 0, (size_t)count * 24, s);  // keys not kept
    kt->host_stages.assign(count, 3);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(kt->host_stages.data(), kt->stages, count, cudaMemcpyDeviceToHost, s);
    if (s) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(s);
    }
    if (e != cudaSuccess) {
        cudaFree(mem);
        delete kt;
        return bcuda(e, "key-table kernel");
    }
    *out = kt;
    return TDES_OK;
}

void tdes_keytable_free(tdes_keytable_t* kt) {
    if (kt == nullptr) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != kt->device) cudaSetDevice(kt->device);
    cudaFree(kt->mem);
    if (cur >= 0 && cur != kt->device) cudaSetDevice(cur);
    delete kt;
}

int tdes_batch_plan(const tdes_keytable_t* kt, const tdes_desc_t* descs, uint32_t count,
                    int* per_desc_status, tdes_batch_t** out) {
    if (out == nullptr || kt == nullptr || (descs == nullptr && count > 0))
        return bfail(TDES_EINVAL, "NULL argument to tdes_batch_plan");
    *out = nullptr;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    if (dev != kt->device) return bfail(TDES_EINVAL, "key table lives on another device");
    tdes::PlanHost h;
    tdes::build_plan(descs, count, kt->count, per_desc_status, &h, true);
    for (tdes::DirectMsg& m : h.direct) m.stages = kt->host_stages[m.key];  // the key's DES passes
    if (!h.direct.empty()) tdes::geometry_for(1, tdes::kEcb, dev);  // kernel set-up, outside any capture
    void* mem = nullptr;
    e = cudaMalloc(&mem, h.image.size());
    if (e != cudaSuccess) return bcuda(e, "cudaMalloc(batch plan)");
    e = cudaMemcpy(mem, h.image.data(), h.image.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return bcuda(e, "cudaMemcpy(batch plan)");
    }
    tdes_batch_t* b = new (std::nothrow) tdes_batch_t();
    if (b == nullptr) {
        cudaFree(mem);
        return bfail(TDES_ENOMEM, "host allocation failed");
    }
    b->device = dev;
    b->kt = kt;
    b->mem = mem;
    b->params = tdes::bind_plan(h, mem, kt);
    b->total_items = h.total_items;
    b->needs_halo = h.needs_halo;
    memcpy(b->bytes, h.bytes_per_mode, sizeof b->bytes);
    memcpy(b->kind_bytes, h.kind_bytes, sizeof b->kind_bytes);
    b->direct = h.direct;
    if (per_desc_status) b->status.assign(per_desc_status, per_desc_status + count);
    else {
        b->status.resize(count);
        for (uint32_t i = 0; i < count; ++i) b->status[i] = tdes::validate_desc(descs[i], kt->count);
    }
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    // the autotuner's shape for this class of batch, if it has one; else the default
    tdes::TunedShape tuned;
    b->tuned = tdes::tune_lookup(tdes::tune_key(h, b->sms), &tuned);
    tdes::LaunchShape shape;  // the default shape
    if (b->tuned) shape = tuned.shape;
    int rc = tdes::set_batch_shape(b, shape);
    if (rc != TDES_OK && b->tuned) {  // a cache entry this library version cannot use
        b->tuned = false;
        rc = tdes::set_batch_shape(b, tdes::LaunchShape());
    }
    if (rc != TDES_OK) {
        cudaFree(mem);
        delete b;
        return rc;
    }
    *out = b;
    if (h.invalid) bfail(TDES_EINVAL, "%d descriptor(s) rejected; see per_desc_status", h.invalid);
    return TDES_OK;
}

int tdes_batch_configure(tdes_batch_t* b, int warps_per_cta, int ctas_per_sm) {
    if (b == nullptr || warps_per_cta < 1 || warps_per_cta > 8)
        return bfail(TDES_EINVAL, "tdes_batch_configure: 1..8 warps per CTA");
    tdes::LaunchShape shape = b->shape;
    shape.warps = warps_per_cta;
    shape.ctas_per_sm = ctas_per_sm;
    return tdes::set_batch_shape(b, shape);
}

int tdes_batch_set_shape(tdes_batch_t* b, const tdes_launch_shape_t* shape) {
    if (b == nullptr || shape == nullptr) return bfail(TDES_EINVAL, "NULL argument");
    tdes::LaunchShape s;
    s.warps = shape->warps_per_cta;
    s.ctas_per_sm = shape->ctas_per_sm;
    s.tiles_per_claim = shape->tiles_per_claim;
    s.round_form = shape->round_form;
    return tdes::set_batch_shape(b, s);
}

int tdes_batch_get_shape(const tdes_batch_t* b, tdes_launch_shape_t* shape) {
    if (b == nullptr || shape == nullptr) return bfail(TDES_EINVAL, "NULL argument");
    shape->warps_per_cta = b->shape.warps;
    shape->ctas_per_sm = b->shape.ctas_per_sm;
    shape->tiles_per_claim = b->shape.tiles_per_claim;
    shape->round_form = b->shape.round_form;
    return TDES_OK;
}

int tdes_batch_launch(tdes_batch_t* b, tdes_stream_t stream) {
    if (b == nullptr) return bfail(TDES_EINVAL, "batch is NULL");
    if (b->total_items == 0 && b->direct.empty()) return TDES_OK;
    cudaError_t e = tdes::enqueue_planned(b, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TDES_OK : bcuda(e, "batch launch");
}

int tdes_batch_launch_graph(tdes_batch_t* b, tdes_stream_t stream) {
    if (b == nullptr) return bfail(TDES_EINVAL, "batch is NULL");
    if (b->total_items == 0 && b->direct.empty()) return TDES_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (b->exec == nullptr) {
        // capture on a private stream so that the caller's stream need not be capturable
        cudaStream_t cap = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(e, "cudaStreamCreate");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = tdes::enqueue_planned(b, cap);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e1;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
            if (e == cudaSuccess) b->graph = g;
            else if (g) cudaGraphDestroy(g);
        }
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return bcuda(e, "batch graph capture");
        }
    }
    e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? TDES_OK : bcuda(e, "cudaGraphLaunch");
}

int tdes_batch_info(const tdes_batch_t* b, tdes_batch_info_t* info) {
    if (b == nullptr || info == nullptr) return bfail(TDES_EINVAL, "NULL argument");
    info->n_cbc_enc_messages = b->params.n_c;
    info->n_tiles = b->params.n_b_tiles;
    info->n_small_items = b->params.n_s_items;
    info->n_mixed_tiles = b->params.n_m_tiles;
    info->n_direct_messages = (uint32_t)b->direct.size();
    info->warps_per_cta = b->shape.warps;
    info->ctas_per_sm = b->shape.ctas_per_sm;
    info->tiles_per_claim = b->shape.tiles_per_claim > 0
                                ? b->shape.tiles_per_claim
                                : (int)tdes::auto_tiles_per_claim(
                                      b->params.n_b_tiles,
                                      (uint64_t)b->sms * b->shape.ctas_per_sm * b->shape.warps);
    info->round_form = b->shape.round_form;
    info->tuned = b->tuned ? 1 : 0;
    for (int i = 0; i < 5; ++i) info->bytes_per_mode[i] = b->bytes[i];
    return TDES_OK;
}

void tdes_batch_free(tdes_batch_t* b) {
    if (b == nullptr) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->mem);
    delete b;
}

}  // extern "C"
