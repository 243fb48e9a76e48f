// tdes_uniform.cu -- many messages of one fixed size laid out back to back
// (message i at in + i * msg_bytes), each under its own key triple and mode
// taken from device arrays, planned and run on the GPU alone.
//
// The batch interface (tdes_batch.cu) plans on the host from one descriptor
// per message; at hundreds of millions of messages (16 GiB of 64-byte
// messages is 2^28) the descriptors alone outgrow host memory.  Here the
// plan is a counting sort on the device, with no host round trip, so a call
// can be captured in a CUDA graph:
//   1. count the messages of each group (mode, key);
//   2. scan the counts.  Each group gets full single-key tiles
//      (1024 blocks of whole messages; for CBC encryption, 1024 chains) and,
//      for what is left, mixed-key slices (one slice = one bit position of
//      a tile: up to 32 blocks under one key, one block per lane);
//   3. every tile and slice learns its group (binary search of the scans);
//   4. message indices are scattered into group order.
// The work kernels follow: single-key tiles (one kernel per mode kind),
// mixed-key tiles (32 slices, the tdes_mixed.cuh round), and the same two
// shapes for CBC encryption; all take the rounds of tdes_compact.cuh.
// A CBC tile holds independent chains and takes one bitsliced pass per block
// position, C_i = E(P_i ^ C_{i-1}) for all of its chains at once (Sec. III-B
// rounds, SP 800-38A chaining), so chaining costs no more per block than ECB.
// A tile (single-key) or a slice (mixed-key) holds messages of one mode, so
// every mode test in the work kernels is uniform across the warp and no
// per-message mode is read there.  Every message lies whole in one tile or
// slice, so in-place CBC decryption only needs the warp's own reads to
// precede its writes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/tdes.h"
#include "tdes_batch_internal.h"
#include "tdes_internal.h"
#include "tdes_compact.cuh"

namespace tdes {
namespace {

constexpr int kUniWarps = 8;                            // warps per CTA of the work kernels
constexpr int kKeyChainWarps = 9;                       // single-key CBC-encryption tiles: 9 x 25 KB
constexpr int kUniTableBytes = TDES_TABLE_WORDS * 4;    // one staged table per warp
// Mixed-key block tiles: beside the table, each slice's message indices (up to
// kSliceSlots messages a slice, so messages of 32 bytes or more) and modes,
// read again after the rounds
constexpr int kSliceSlots = 8;
constexpr int kMixedWarpBytes = kUniTableBytes + 32 * kSliceSlots * 4 + 32;
// Single-key block tiles: beside the table, the tile's message indices (up to
// kTileSlots messages a tile, so 16-byte-path messages of 64 bytes or more),
// read again after the rounds
constexpr int kTileSlots = 128;
constexpr int kTileWarpBytes = kUniTableBytes + kTileSlots * 4;
// CBC-encryption chains: a warp's table, its 1024 chains' message indices and
// one held block per chain (25 KB; one CTA per SM of 8 warps for mixed-key
// chains, 9 for single-key tiles)
constexpr int kChainWarpBytes = kUniTableBytes + 32 * 32 * 4 + 32 * 32 * 8;
// Mixed-key CBC-encryption slices: 12 warps per CTA, one CTA per SM, each
// warp with its table and its chains' message indices in shared memory
// (17 KB) and its held blocks in a slab of global scratch (8 KB per warp).
constexpr int kMixedChainWarps = 12;
constexpr int kMixedChainWarpBytes = kUniTableBytes + 32 * 32 * 4;
constexpr int kMaxChainCtas = 256;  // the kernel's grid: min(SMs, this)
// sm_103a shared memory: 228 KB per SM, 1 KB of it reserved per resident CTA,
// so a CTA may take at most 227 KB
constexpr int kSmemPerSm = 228 * 1024, kSmemReservedPerCta = 1024;
static_assert(kKeyChainWarps * kChainWarpBytes + kSmemReservedPerCta <= kSmemPerSm, "single-key chain CTA");
static_assert(kMixedChainWarps * kMixedChainWarpBytes + kSmemReservedPerCta <= kSmemPerSm,
              "mixed-key chain CTA");
static_assert(2 * (kUniWarps * kTileWarpBytes + kSmemReservedPerCta) <= kSmemPerSm, "two tile CTAs per SM");
static_assert(2 * (kUniWarps * kMixedWarpBytes + kSmemReservedPerCta) <= kSmemPerSm,
              "two mixed-key CTAs per SM");
constexpr int kScanThreads = 1024;
constexpr uint32_t kChainsPerTile = kTileBlocks;       // CBC encryption: one chain per tile slot
constexpr uint32_t kModes = 5;                         // groups per key: one per TDES_MODE_*
constexpr uint32_t kMaxKeys = 1u << 26;                // 5 groups per key fit 32-bit indices

struct UniHeader {
    unsigned long long skipped;  // messages left untouched: bad key index, mode or counter
    uint32_t tiles[2];           // single-key tiles: [0] modes 0-3 first, then [1] CBC encryption
    uint32_t slices[2];          // mixed-key slices: [0] modes 0-3 from slice 0,
    uint32_t slice2_base;        //   [1] CBC encryption from slice2_base (a multiple of 32)
    uint32_t kind_tiles[5];      // single-key tiles of kind k: [kind_tiles[k], kind_tiles[k + 1])
    uint32_t pad[4];
};
static_assert(sizeof(UniHeader) == 64, "header layout");

struct UniParams {
    const uint32_t* keytab;     // [key][dir][TDES_TABLE_WORDS]
    const uint8_t* keystages;   // [key]: 3, or 1 for a triple that reduces to single DES
    const uint32_t* keypacked;  // [key][dir][kPackedWords]
    uint32_t n_keys;
    uint32_t n_groups;          // kModes * n_keys; group = mode * n_keys + key
    const uint32_t* key_index;
    const uint8_t* mode;
    const uint64_t* iv;
    const uint8_t* in;
    uint8_t* out;
    uint64_t n_msgs;
    uint32_t msg_bytes;
    uint32_t m;                 // blocks per message, 1..32
    uint32_t magic;             // (k * magic) >> 16 == k / m for k < 1024
    uint32_t per_tile;          // messages per single-key tile, modes 0-3: 1024 / m
    uint32_t per_slice;         // messages per slice, modes 0-3: 32 / m
    uint32_t* counts;           // [group]
    uint32_t* cursor;           // [group] next position in order[] (set by the scan)
    uint32_t* msg_off;          // [group] first position in order[]
    uint32_t* tile_off;         // [group] first single-key tile
    uint32_t* slice_off;        // [group] first mixed-key slice
    uint32_t* order;            // message indices in group order
    uint32_t* tile_group;       // [tile] group
    uint32_t* slice_group;      // [slice] group
    uint2* held;                // mixed-key chain slices: 1024 held blocks per warp
    UniHeader* hdr;
};

__device__ __forceinline__ uint32_t bswap32u(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

// Group of message i, or ~0u for a message the call skips.
__device__ __forceinline__ uint32_t uni_group(const UniParams& p, uint64_t i) {
    const uint32_t key = p.key_index[i];
    const uint32_t md = p.mode[i];
    if (key >= p.n_keys || md > TDES_MODE_CBC_ENCRYPT) return ~0u;
    if (md == TDES_MODE_CTR && (p.iv[i] & 0xFFFFFFFFull) + p.m > (1ull << 32)) return ~0u;
    return md * p.n_keys + key;
}

__device__ __forceinline__ uint32_t per_tile_of(const UniParams& p, uint32_t md) {
    return md == TDES_MODE_CBC_ENCRYPT ? kChainsPerTile : p.per_tile;
}
__device__ __forceinline__ uint32_t per_slice_of(const UniParams& p, uint32_t md) {
    return md == TDES_MODE_CBC_ENCRYPT ? 32u : p.per_slice;
}
// Single-key tiles run in one kernel per kind, each with one code path:
// ECB (either direction), CTR, CBC decryption, CBC encryption.  Groups are
// ordered by mode, so each kind's tiles are one contiguous range.
enum TileKind { kKindEcb = 0, kKindCtr = 1, kKindCbcDec = 2, kKindCbcEnc = 3 };

__device__ __forceinline__ uint32_t dir_of_mode(uint32_t md) {
    return (md == TDES_MODE_ECB_DECRYPT || md == TDES_MODE_CBC_DECRYPT) ? 1u : 0u;
}

// Lanes of a warp whose messages fall in the same group share one atomic
// (the leader adds the group's lane count), so that a workload with few keys
// does not serialise on a handful of counters; with many keys most groups
// hold one lane.
__global__ void uni_count_kernel(UniParams p) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t bad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n_msgs; i += stride) {
        const uint32_t g = uni_group(p, i);
        const uint32_t peers = __match_any_sync(__activemask(), g);
        if (lane == (uint32_t)(__ffs(peers) - 1)) {
            if (g == ~0u)
                bad += __popc(peers);
            else
                atomicAdd(&p.counts[g], (uint32_t)__popc(peers));
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) bad += __shfl_xor_sync(0xFFFFFFFFu, bad, o);
    if (lane == 0 && bad) atomicAdd(&p.hdr->skipped, (unsigned long long)bad);
}

struct Sums {
    uint32_t c, t, s;  // messages, single-key tiles, mixed-key slices
};

__device__ __forceinline__ Sums shfl_up3(Sums v, int o) {
    return {__shfl_up_sync(0xFFFFFFFFu, v.c, o), __shfl_up_sync(0xFFFFFFFFu, v.t, o),
            __shfl_up_sync(0xFFFFFFFFu, v.s, o)};
}

// Exclusive scan of v over the CTA's 1024 threads; *total gets the sum.
__device__ Sums block_scan(Sums v, Sums* total) {
    __shared__ Sums warp_ex[32];
    __shared__ Sums all;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Sums inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const Sums u = shfl_up3(inc, o);
        if (lane >= o) {
            inc.c += u.c;
            inc.t += u.t;
            inc.s += u.s;
        }
    }
    if (lane == 31) warp_ex[w] = inc;
    __syncthreads();
    if (w == 0) {
        const Sums x = warp_ex[lane];
        Sums xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Sums u = shfl_up3(xi, o);
            if (lane >= o) {
                xi.c += u.c;
                xi.t += u.t;
                xi.s += u.s;
            }
        }
        warp_ex[lane] = {xi.c - x.c, xi.t - x.t, xi.s - x.s};
        if (lane == 31) all = xi;
    }
    __syncthreads();
    const Sums b = warp_ex[w];
    const Sums ex = {b.c + inc.c - v.c, b.t + inc.t - v.t, b.s + inc.s - v.s};
    *total = all;
    __syncthreads();  // the shared arrays are reused by the next call
    return ex;
}

// The scan over groups runs in blocks of kScanSpan groups: the first
// scan_blocks_a() blocks cover modes 0-3, the rest CBC encryption (whose
// slices start a tile of their own, so the two ranges are scanned apart).
// Three kernels: block sums, a scan of the block sums (one CTA), and each
// block's offsets from its base.
constexpr uint32_t kScanPer = 4;                           // groups per thread
constexpr uint32_t kScanSpan = kScanThreads * kScanPer;   // groups per block

__host__ __device__ inline uint32_t scan_blocks_a(uint32_t K) {
    return (TDES_MODE_CBC_ENCRYPT * K + kScanSpan - 1) / kScanSpan;
}
__host__ __device__ inline uint32_t scan_blocks(uint32_t K) {
    return scan_blocks_a(K) + (K + kScanSpan - 1) / kScanSpan;
}

// This thread's groups [*a, *b) of scan block blk.
__device__ __forceinline__ void scan_range(const UniParams& p, uint32_t blk, uint32_t* a,
                                           uint32_t* b) {
    const uint32_t K = p.n_keys, G4 = TDES_MODE_CBC_ENCRYPT * K, na = scan_blocks_a(K);
    const uint32_t g0 = blk < na ? blk * kScanSpan : G4 + (blk - na) * kScanSpan;
    const uint32_t g1 = min(blk < na ? G4 : G4 + K, g0 + kScanSpan);
    *a = min(g1, g0 + threadIdx.x * kScanPer);
    *b = min(g1, *a + kScanPer);
}

// A group's messages, single-key tiles and mixed-key slices.
__device__ __forceinline__ Sums group_sums(const UniParams& p, uint32_t g) {
    const uint32_t md = g / p.n_keys, c = p.counts[g];
    const uint32_t M = per_tile_of(p, md), Q = per_slice_of(p, md);
    const uint32_t u = c / M, r = c - u * M;
    return {c, u, (r + Q - 1) / Q};
}

__device__ __forceinline__ Sums add(Sums x, Sums y) { return {x.c + y.c, x.t + y.t, x.s + y.s}; }

__global__ void __launch_bounds__(kScanThreads) uni_scan_partial_kernel(UniParams p, Sums* part) {
    uint32_t a, b;
    scan_range(p, blockIdx.x, &a, &b);
    Sums v = {0u, 0u, 0u}, tot;
    for (uint32_t g = a; g < b; ++g) v = add(v, group_sums(p, g));
    block_scan(v, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Exclusive scan of part[b0, b1) into base[], from `carry`; returns the end.
__device__ Sums scan_parts(const Sums* part, Sums* base, uint32_t b0, uint32_t b1, Sums carry) {
    for (uint32_t c0 = b0; c0 < b1; c0 += kScanThreads) {
        const uint32_t b = c0 + threadIdx.x;
        const Sums v = b < b1 ? part[b] : Sums{0u, 0u, 0u};
        Sums tot;
        const Sums ex = block_scan(v, &tot);
        if (b < b1) base[b] = add(carry, ex);
        carry = add(carry, tot);
    }
    return carry;
}

__global__ void __launch_bounds__(kScanThreads) uni_scan_top_kernel(UniParams p, const Sums* part,
                                                                    Sums* base) {
    const uint32_t na = scan_blocks_a(p.n_keys), nb = scan_blocks(p.n_keys);
    const Sums t01 = scan_parts(part, base, 0u, na, {0u, 0u, 0u});
    const uint32_t s2 = (t01.s + 31u) & ~31u;  // CBC-encryption slices start a tile of their own
    const Sums end = scan_parts(part, base, na, nb, {t01.c, t01.t, s2});
    if (threadIdx.x == 0) {
        p.hdr->kind_tiles[kKindEcb] = 0u;
        p.hdr->kind_tiles[kKindCbcEnc] = t01.t;
        p.hdr->kind_tiles[kKindCbcEnc + 1] = end.t;
        p.hdr->tiles[0] = t01.t;
        p.hdr->tiles[1] = end.t - t01.t;
        p.hdr->slices[0] = t01.s;
        p.hdr->slices[1] = end.s - s2;
        p.hdr->slice2_base = s2;
    }
}

__global__ void __launch_bounds__(kScanThreads) uni_scan_final_kernel(UniParams p, const Sums* base) {
    uint32_t a, b;
    scan_range(p, blockIdx.x, &a, &b);
    Sums v = {0u, 0u, 0u}, tot;
    for (uint32_t g = a; g < b; ++g) v = add(v, group_sums(p, g));
    Sums run = add(base[blockIdx.x], block_scan(v, &tot));
    const uint32_t g_ctr = TDES_MODE_CTR * p.n_keys, g_cbc = TDES_MODE_CBC_DECRYPT * p.n_keys;
    for (uint32_t g = a; g < b; ++g) {
        p.msg_off[g] = run.c;
        p.cursor[g] = run.c;  // the scatter's next position in the group
        p.tile_off[g] = run.t;
        p.slice_off[g] = run.s;
        if (g == g_ctr) p.hdr->kind_tiles[kKindCtr] = run.t;
        if (g == g_cbc) p.hdr->kind_tiles[kKindCbcDec] = run.t;
        run = add(run, group_sums(p, g));
    }
}

// Largest g in [lo, hi) with off[g] <= x, given off[lo] <= x and off
// non-decreasing: the group whose range holds x (groups with nothing in this
// range share their offset with the next group and are never the largest).
__device__ __forceinline__ uint32_t group_of(const uint32_t* off, uint32_t lo, uint32_t hi,
                                             uint32_t x) {
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (off[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void uni_map_kernel(UniParams p) {
    const uint32_t K = p.n_keys, G4 = TDES_MODE_CBC_ENCRYPT * K;
    const uint32_t t0 = p.hdr->tiles[0], t1 = p.hdr->tiles[1];
    const uint32_t s0 = p.hdr->slices[0], s1 = p.hdr->slices[1], s2 = p.hdr->slice2_base;
    const uint64_t total = (uint64_t)t0 + t1 + s0 + s1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        if (i < t0) {
            p.tile_group[i] = group_of(p.tile_off, 0u, G4, (uint32_t)i);
        } else if (i < (uint64_t)t0 + t1) {
            p.tile_group[i] = group_of(p.tile_off, G4, G4 + K, (uint32_t)i);
        } else if (i < (uint64_t)t0 + t1 + s0) {
            const uint32_t s = (uint32_t)(i - t0 - t1);
            p.slice_group[s] = group_of(p.slice_off, 0u, G4, s);
        } else {
            const uint32_t s = s2 + (uint32_t)(i - t0 - t1 - s0);
            p.slice_group[s] = group_of(p.slice_off, G4, G4 + K, s);
        }
    }
}

// Lanes in the same group take consecutive positions from one atomic.
__global__ void uni_scatter_kernel(UniParams p) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n_msgs; i += stride) {
        const uint32_t g = uni_group(p, i);
        const uint32_t act = __activemask();
        const uint32_t peers = __match_any_sync(act, g);
        const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
        uint32_t base = 0;
        if (lane == leader && g != ~0u) base = atomicAdd(&p.cursor[g], (uint32_t)__popc(peers));
        base = __shfl_sync(act, base, leader);
        if (g != ~0u) p.order[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
    }
}

extern __shared__ __align__(16) uint8_t uni_smem[];  // a slice per warp (kTileWarpBytes, ...)

__device__ __forceinline__ const uint2* msg_in(const UniParams& p, uint32_t mi) {
    return reinterpret_cast<const uint2*>(p.in + (uint64_t)mi * p.msg_bytes);
}
__device__ __forceinline__ uint2* msg_out(const UniParams& p, uint32_t mi) {
    return reinterpret_cast<uint2*>(p.out + (uint64_t)mi * p.msg_bytes);
}
// Message data and IVs sit at random places, a message's 64 bytes or an
// IV's 8 apart from their neighbours' in the same 128-byte line.  Through
// L1, every miss fetched the whole line from L2 (and DRAM): a capture of the
// tile kernels showed L1 asking L2 for 1.6-1.95x the sectors its loads
// requested.  These reads go to L2 only (ld.global.cg), sector by sector.
__device__ __forceinline__ uint2 ld_msg(const uint2* a) { return __ldcg(a); }
__device__ __forceinline__ uint4 ld_msg(const uint4* a) { return __ldcg(a); }
// CBC-encryption chains read their message a piece per pass; there the
// whole-line fetch through L1 brings the message's later blocks into L2 ahead
// of their passes, and L2-only reads made the chain kernel slower (8.80 ->
// 9.53 ms for 2^28 messages), so chains keep the streaming loads.
__device__ __forceinline__ uint2 ld_chain(const uint2* a) { return __ldcs(a); }
__device__ __forceinline__ uint4 ld_chain(const uint4* a) { return __ldcs(a); }
__device__ __forceinline__ uint64_t ld_iv(const UniParams& p, uint32_t mi) {
    return __ldcg(reinterpret_cast<const unsigned long long*>(p.iv) + mi);
}

__device__ __forceinline__ uint2 iv_words(uint64_t iv) {
    return make_uint2(bswap32u((uint32_t)(iv >> 32)), bswap32u((uint32_t)iv));
}

__device__ __forceinline__ uint32_t tile_pos0(const UniParams& p, uint32_t t) {
    const uint32_t g = p.tile_group[t];
    return p.msg_off[g] + (t - p.tile_off[g]) * per_tile_of(p, g / p.n_keys);
}

// Tile block k = 64 j + 2 lane + h is block k % m of the tile's message
// k / m.  A lane's pair (h = 0, 1) shares one message unless the first block
// is its message's last (odd m).
struct PairSlots {
    uint32_t slot0, blk0, slot1, blk1;
};

__device__ __forceinline__ PairSlots pair_slots(const UniParams& p, uint32_t k) {
    PairSlots r;
    r.slot0 = (k * p.magic) >> 16;
    r.blk0 = k - r.slot0 * p.m;
    const bool same = r.blk0 + 1 < p.m;
    r.slot1 = same ? r.slot0 : r.slot0 + 1;
    r.blk1 = same ? r.blk0 + 1 : 0u;
    return r;
}

__device__ __forceinline__ uint2 ctr_words(uint64_t c, uint32_t blk) {
    return make_uint2(bswap32u((uint32_t)(c >> 32)), bswap32u((uint32_t)c + blk));
}

// Blocks (blk0, blk1) of the lane's pair j on the general path (any m, any
// 8-byte alignment): p.in's bytes for ECB and CBC decryption (and the
// post-round XOR of CTR), counter blocks for CTR.
template <bool COUNTER>
__device__ __forceinline__ void load_pair(const UniParams& p, uint32_t pos0, const PairSlots& q,
                                          uint2& v0, uint2& v1) {
    v0 = v1 = make_uint2(0u, 0u);
    if (q.slot0 >= p.per_tile) return;
    const uint32_t mi0 = p.order[pos0 + q.slot0];
    if (COUNTER) {
        const uint64_t c0 = ld_iv(p, mi0);
        v0 = ctr_words(c0, q.blk0);
        if (q.slot1 == q.slot0)
            v1 = ctr_words(c0, q.blk1);
        else if (q.slot1 < p.per_tile)
            v1 = ctr_words(ld_iv(p, p.order[pos0 + q.slot1]), q.blk1);
    } else {
        v0 = ld_msg(msg_in(p, mi0) + q.blk0);
        if (q.slot1 == q.slot0)
            v1 = ld_msg(msg_in(p, mi0) + q.blk1);
        else if (q.slot1 < p.per_tile)
            v1 = ld_msg(msg_in(p, p.order[pos0 + q.slot1]) + q.blk1);
    }
}

// The ciphertext block before blk of message mi, or the IV for the first.
__device__ __forceinline__ uint2 cbc_prev(const UniParams& p, uint32_t mi, uint32_t blk) {
    return blk ? ld_msg(msg_in(p, mi) + (blk - 1)) : iv_words(ld_iv(p, mi));
}

// One single-key tile of ECB, CTR or CBC-decryption messages.  VEC16: every
// pair is one 16-byte-aligned piece of one message (m even, in and out
// 16-byte aligned); there the loads before the rounds, and CTR's after
// them, have no branch per pair (an out-of-tile slot, possible when m does
// not divide 1024, reads a clamped message and is masked), so the loads of
// all 16 pairs are in flight together.  CBC decryption's operands after the
// rounds keep their branches, which measured faster (69.4 against 70.0 ms
// for 2^28 messages).
template <int KIND, bool VEC16>
__device__ __forceinline__ void uni_block_tile(const UniParams& p, uint32_t t,
                                               const uint32_t* __restrict__ tab, uint32_t* tidx,
                                               uint32_t lane, bool one_pass) {
    // 16-byte path with at most kTileSlots messages a tile: the lane holding
    // a message's first pair keeps its index in tidx for the loops after the
    // rounds, which read it there instead of from order (2^28 messages of
    // 64 B: 64.03 -> 63.42 ms, alternating A/B runs).  CBC-decryption tiles
    // ran slower with it (10.33 -> 10.59 ms in a launch list) and keep the
    // order reads: 63.41 -> 63.14 ms.
    const bool keep = VEC16 && KIND != kKindCbcDec && p.per_tile <= (uint32_t)kTileSlots;
    uint32_t A0[32], A1[32];
    uint32_t pos0 = tile_pos0(p, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const PairSlots q = pair_slots(p, 64u * j + 2u * lane);
        uint2 v0, v1;
        if (VEC16) {
            const bool ok = q.slot0 < p.per_tile;
            const uint32_t mi0 = p.order[pos0 + min(q.slot0, p.per_tile - 1u)];
            if (keep && ok && q.blk0 == 0u) tidx[q.slot0] = mi0;
            if (KIND == kKindCtr) {
                const uint64_t c0 = ld_iv(p, mi0);
                v0 = ctr_words(c0, q.blk0);
                v1 = ctr_words(c0, q.blk0 + 1u);
            } else {
                const uint4 w = ld_msg(reinterpret_cast<const uint4*>(msg_in(p, mi0) + q.blk0));
                v0 = make_uint2(w.x, w.y);
                v1 = make_uint2(w.z, w.w);
            }
            if (!ok) v0 = v1 = make_uint2(0u, 0u);
        } else {
            load_pair<KIND == kKindCtr>(p, pos0, q, v0, v1);
        }
        A0[2 * j] = v0.x;
        A1[2 * j] = v0.y;
        A0[2 * j + 1] = v1.x;
        A1[2 * j + 1] = v1.y;
    }
    __syncwarp();
    tdes_process32_compact<false>(A0, A1, tab, one_pass);
    pos0 = tile_pos0(p, t);  // reloaded: nothing but the planes stays live across the rounds
    // the message of slot x (x < per_tile) after the rounds
    auto msg_of = [&](uint32_t x) { return keep ? tidx[x] : p.order[pos0 + x]; };
    if (KIND == kKindCtr || KIND == kKindCbcDec) {
        uint2 carry = make_uint2(0u, 0u);  // CBC decryption: lane 31's second block of pair j - 1
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const PairSlots q = pair_slots(p, 64u * j + 2u * lane);
            uint2 v0 = make_uint2(0u, 0u), v1 = make_uint2(0u, 0u);
            if (VEC16 && KIND == kKindCbcDec) {
                // The lane's own 16 bytes are C_b0 (v1's operand) and C_b0+1;
                // C_b0-1 is the second block of the pair before, one lane
                // down (lane 0: lane 31 of pair j - 1), in the same message
                // unless b0 = 0, where the IV stands in.
                const bool ok = q.slot0 < p.per_tile;
                const uint32_t mi0 = msg_of(min(q.slot0, p.per_tile - 1u));
                const uint4 w = ld_msg(reinterpret_cast<const uint4*>(msg_in(p, mi0) + q.blk0));
                uint2 up = make_uint2(__shfl_up_sync(0xFFFFFFFFu, w.z, 1),
                                      __shfl_up_sync(0xFFFFFFFFu, w.w, 1));
                if (lane == 0) up = carry;
                carry = make_uint2(__shfl_sync(0xFFFFFFFFu, w.z, 31), __shfl_sync(0xFFFFFFFFu, w.w, 31));
                v0 = q.blk0 == 0u ? iv_words(ld_iv(p, mi0)) : up;
                v1 = make_uint2(w.x, w.y);
                if (!ok) v0 = v1 = make_uint2(0u, 0u);
            } else if (VEC16 && KIND == kKindCtr) {
                const bool ok = q.slot0 < p.per_tile;
                const uint32_t mi0 = msg_of(min(q.slot0, p.per_tile - 1u));
                const uint4 w = ld_msg(reinterpret_cast<const uint4*>(msg_in(p, mi0) + q.blk0));
                v0 = make_uint2(w.x, w.y);
                v1 = make_uint2(w.z, w.w);
                if (!ok) v0 = v1 = make_uint2(0u, 0u);
            } else if (KIND == kKindCtr) {
                load_pair<false>(p, pos0, q, v0, v1);
            } else if (q.slot0 < p.per_tile) {
                const uint32_t mi0 = p.order[pos0 + q.slot0];
                v0 = cbc_prev(p, mi0, q.blk0);
                if (q.slot1 == q.slot0)
                    v1 = ld_msg(msg_in(p, mi0) + q.blk0);
                else if (q.slot1 < p.per_tile)
                    v1 = iv_words(ld_iv(p, p.order[pos0 + q.slot1]));  // blk1 = 0
            }
            A0[2 * j] ^= v0.x;
            A1[2 * j] ^= v0.y;
            A0[2 * j + 1] ^= v1.x;
            A1[2 * j + 1] ^= v1.y;
        }
    }
    __syncwarp();  // in place: every read of the tile's messages precedes its writes
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const PairSlots q = pair_slots(p, 64u * j + 2u * lane);
        if (q.slot0 < p.per_tile) {
            const uint32_t mi0 = msg_of(q.slot0);
            if (VEC16) {
                __stcs(reinterpret_cast<uint4*>(msg_out(p, mi0) + q.blk0),
                       make_uint4(A0[2 * j], A1[2 * j], A0[2 * j + 1], A1[2 * j + 1]));
            } else {
                __stcs(msg_out(p, mi0) + q.blk0, make_uint2(A0[2 * j], A1[2 * j]));
                if (q.slot1 == q.slot0)
                    __stcs(msg_out(p, mi0) + q.blk1, make_uint2(A0[2 * j + 1], A1[2 * j + 1]));
                else if (q.slot1 < p.per_tile)
                    __stcs(msg_out(p, p.order[pos0 + q.slot1]) + q.blk1,
                           make_uint2(A0[2 * j + 1], A1[2 * j + 1]));
            }
        }
    }
    __syncwarp();  // tidx is rewritten by the next tile
}

// The block passes of 1024 CBC-encryption chains: widx[32 s + lane] is the
// message of the chain in bit plane word s (~0u: none).  After a pass the
// planes are back in block order, so A holds C_i and the next pass starts
// from A ^ P_{i+1}: only the plaintext is read.  When messages are 16-byte
// aligned, passes go in pairs: one 16-byte load brings P_i and P_{i+1}, the
// held block keeps P_{i+1} and then C_i, and one 16-byte store writes
// C_i, C_{i+1}.  A sector is then read and written half as often (64-byte
// messages: 2^28 of them under 65536 keys, 69.1 -> 66.2 ms per call; 2^22
// CBC encryptions under two keys, 2.15 -> 1.59 ms).
// The mixed-key chains' held blocks live in global scratch (a slab per
// warp, 25 MB in all, rewritten every pass): their accesses ask L2 to keep
// the lines over the chains' random message reads (evict-last).  The
// single-key chains hold them in shared memory.
template <bool GLOBAL>
__device__ __forceinline__ uint2 ld_held(const uint2* q, uint64_t pol) {
    if (!GLOBAL) return *q;
    uint2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(q), "l"(pol)
                 : "memory");
    return v;
}
template <bool GLOBAL>
__device__ __forceinline__ void st_held(uint2* q, uint2 v, uint64_t pol) {
    if (!GLOBAL) {
        *q = v;
        return;
    }
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(q), "r"(v.x),
                 "r"(v.y), "l"(pol)
                 : "memory");
}

template <bool MIXED>
__device__ __forceinline__ void uni_chain_passes(const UniParams& p, uint32_t (&A0)[32],
                                                 uint32_t (&A1)[32], const uint32_t* __restrict__ tab,
                                                 const uint32_t* widx, uint2* held, uint32_t lane,
                                                 bool one_pass) {
    const bool pair = p.m % 2u == 0u && (((uintptr_t)p.in | (uintptr_t)p.out) & 15u) == 0u;
    uint64_t pol = 0;
    if (MIXED) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    for (uint32_t i = 0; i < p.m; ++i) {
        const bool odd = (i & 1u) != 0u;
        if (!pair) {
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t mi = widx[32 * s + lane];
                if (mi != ~0u) {
                    const uint2 x = ld_chain(msg_in(p, mi) + i);
                    A0[s] ^= x.x;
                    A1[s] ^= x.y;
                }
            }
        } else if (!odd) {
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t mi = widx[32 * s + lane];
                uint4 x = make_uint4(0u, 0u, 0u, 0u);
                if (mi != ~0u) x = ld_chain(reinterpret_cast<const uint4*>(msg_in(p, mi) + i));
                A0[s] ^= x.x;
                A1[s] ^= x.y;
                st_held<MIXED>(held + 32 * s + lane, make_uint2(x.z, x.w), pol);
            }
        }
        tdes_process32_compact<MIXED>(A0, A1, tab, one_pass);
        if (!pair) {
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t mi = widx[32 * s + lane];
                if (mi != ~0u) msg_out(p, mi)[i] = make_uint2(A0[s], A1[s]);
            }
        } else if (!odd) {  // hold C_i, start pass i + 1 from C_i ^ P_{i+1}
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint2 x = ld_held<MIXED>(held + 32 * s + lane, pol);
                st_held<MIXED>(held + 32 * s + lane, make_uint2(A0[s], A1[s]), pol);
                A0[s] ^= x.x;
                A1[s] ^= x.y;
            }
        } else {
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t mi = widx[32 * s + lane];
                const uint2 c = ld_held<MIXED>(held + 32 * s + lane, pol);
                if (mi != ~0u)
                    *reinterpret_cast<uint4*>(msg_out(p, mi) + i - 1) = make_uint4(c.x, c.y, A0[s], A1[s]);
            }
        }
    }
    __syncwarp();  // widx and held are rewritten by the next tile
}

// One single-key tile of 1024 CBC-encryption chains (chain k = 64 j + 2 lane
// + h sits in plane word 2 j + h).  wsm holds the warp's table, then room for
// the chains' message indices and held blocks.
__device__ __forceinline__ void uni_chain_tile(const UniParams& p, uint32_t t, uint32_t* wsm,
                                               uint32_t lane, bool one_pass) {
    uint32_t* widx = wsm + TDES_TABLE_WORDS;
    uint32_t A0[32], A1[32];
    const uint32_t pos0 = tile_pos0(p, t);
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t mi = p.order[pos0 + 64u * j + 2u * lane + h];
            widx[32 * (2 * j + h) + lane] = mi;
            const uint2 c = iv_words(ld_iv(p, mi));
            A0[2 * j + h] = c.x;
            A1[2 * j + h] = c.y;
        }
    uni_chain_passes<false>(p, A0, A1, wsm, widx, reinterpret_cast<uint2*>(widx + 32 * 32), lane,
                            one_pass);
}

// Single-key tiles of one kind, split evenly into one contiguous run per
// warp: a group's tiles are consecutive, so a warp stages each table once
// per run.
template <int KIND, bool VEC16>
__global__ void __launch_bounds__(KIND == kKindCbcEnc ? 32 * kKeyChainWarps : 32 * kUniWarps,
                                  KIND == kKindCbcEnc ? 1 : 2) uni_tile_kernel(UniParams p) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* wtab = reinterpret_cast<uint32_t*>(
        uni_smem + (size_t)warp * (KIND == kKindCbcEnc ? kChainWarpBytes : kTileWarpBytes));
    const uint32_t first = p.hdr->kind_tiles[KIND];
    const uint32_t n = p.hdr->kind_tiles[KIND + 1] - first;
    const uint32_t nw = blockDim.x >> 5;
    const uint32_t W = gridDim.x * nw, w = blockIdx.x * nw + warp;
    const uint32_t per = n / W, extra = n % W;
    const uint32_t a = w * per + min(w, extra), b = a + per + (w < extra ? 1u : 0u);
    uint32_t staged = ~0u;
    for (uint32_t t = first + a; t < first + b; ++t) {
        const uint32_t g = p.tile_group[t];
        const uint32_t md = g / p.n_keys, key = g - md * p.n_keys;
        const bool one_pass = p.keystages[key] == 1;
        const uint32_t kd = key * 2u + dir_of_mode(md);
        if (kd != staged) {
            __syncwarp();
            const uint4* src = reinterpret_cast<const uint4*>(p.keytab + (uint64_t)kd * TDES_TABLE_WORDS);
            const int n4 = (one_pass ? TDES1_TABLE_WORDS : TDES_TABLE_WORDS) / 4;
            for (int i = lane; i < n4; i += 32) reinterpret_cast<uint4*>(wtab)[i] = __ldg(src + i);
            __syncwarp();
            staged = kd;
        }
        if (KIND == kKindCbcEnc)
            uni_chain_tile(p, t, wtab, lane, one_pass);
        else
            uni_block_tile<KIND, VEC16>(p, t, wtab, wtab + TDES_TABLE_WORDS, lane, one_pass);
    }
}

// Mixed-key tiles: slice s of tile t is slice first + 32 t + s; lane s works
// out its slice's first message position, count and mode and loads its
// key's packed table row, and a transpose across the lanes builds the tile's
// table (bit s of every word: slice s's key and direction).  Slices differ
// in mode, but each slice's mode is the same in every lane.
template <bool CHAIN>
__global__ void __launch_bounds__(CHAIN ? 32 * kMixedChainWarps : 32 * kUniWarps, CHAIN ? 1 : 2)
    uni_mixed_kernel(UniParams p) {
    constexpr uint32_t kWarps = CHAIN ? kMixedChainWarps : kUniWarps;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* wtab = reinterpret_cast<uint32_t*>(
        uni_smem + (size_t)warp * (CHAIN ? kMixedChainWarpBytes : kMixedWarpBytes));
    const uint32_t first = CHAIN ? p.hdr->slice2_base : 0u;
    const uint32_t ns = CHAIN ? p.hdr->slices[1] : p.hdr->slices[0];
    const uint32_t ntiles = (ns + 31u) / 32u;
    const uint32_t W = gridDim.x * kWarps;
    for (uint32_t t = blockIdx.x * kWarps + warp; t < ntiles; t += W) {
        uint32_t pos = 0, cm = 0, kd = 0;  // cm: message count | mode << 8
        if (32u * t + lane < ns) {
            const uint32_t s = first + 32u * t + lane;
            const uint32_t g = p.slice_group[s];
            const uint32_t md = g / p.n_keys, key = g - md * p.n_keys;
            const uint32_t M = per_tile_of(p, md), Q = per_slice_of(p, md);
            const uint32_t c = p.counts[g];
            const uint32_t at = (c / M) * M + (s - p.slice_off[g]) * Q;
            cm = min(Q, c - at) | (md << 8);
            pos = p.msg_off[g] + at;
            kd = key * 2u + dir_of_mode(md);
        }
        // the tile's table: lane s's slice row, transposed across the lanes
        auto stage_table = [&]() {
            const uint32_t* row = p.keypacked + (uint64_t)kd * kPackedWords;
            __syncwarp();
#pragma unroll 1
            for (int q = 0; q < kPackedWords; ++q)
                wtab[32 * q + lane] = transpose_lanes32(__ldg(row + q), lane);
            __syncwarp();
        };
        if (CHAIN) {
            stage_table();
            // lane l walks chain l of every slice
            uint32_t* widx = wtab + TDES_TABLE_WORDS;
            uint32_t A0[32], A1[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t ps = __shfl_sync(0xFFFFFFFFu, pos, s);
                const uint32_t cs = __shfl_sync(0xFFFFFFFFu, cm, s) & 0xFFu;
                uint2 c = make_uint2(0u, 0u);
                uint32_t mi = ~0u;
                if (lane < cs) {
                    mi = p.order[ps + lane];
                    c = iv_words(ld_iv(p, mi));
                }
                widx[32 * s + lane] = mi;
                A0[s] = c.x;
                A1[s] = c.y;
            }
            uni_chain_passes<true>(p, A0, A1, wtab, widx,
                                   p.held + (size_t)(blockIdx.x * kWarps + warp) * (32 * 32), lane,
                                   false);
        } else {
            // lane l holds block l % m of the slice's message l / m.  With at
            // most kSliceSlots messages a slice, each message's index (written
            // by the lane holding its first block) and each slice's mode stay
            // in shared memory for the loops after the rounds.
            const uint32_t slot = (lane * p.magic) >> 16, blk = lane - slot * p.m;
            const bool keep = p.per_slice <= (uint32_t)kSliceSlots;
            uint32_t* sidx = wtab + TDES_TABLE_WORDS;                              // [slice][slot]
            uint8_t* smode = reinterpret_cast<uint8_t*>(sidx + 32 * kSliceSlots);  // [slice]
            if (keep) smode[lane] = (uint8_t)(cm >> 8);
            uint32_t A0[32], A1[32];
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const uint32_t ps = __shfl_sync(0xFFFFFFFFu, pos, s);
                const uint32_t c = __shfl_sync(0xFFFFFFFFu, cm, s);
                uint2 v = make_uint2(0u, 0u);
                uint32_t mi = ~0u;
                if (slot < (c & 0xFFu)) {
                    mi = p.order[ps + slot];
                    v = (c >> 8) == TDES_MODE_CTR ? ctr_words(ld_iv(p, mi), blk) : ld_msg(msg_in(p, mi) + blk);
                }
                if (keep && blk == 0) sidx[kSliceSlots * s + slot] = mi;
                A0[s] = v.x;
                A1[s] = v.y;
            }
            // staged after the loads are issued, so that their latency
            // overlaps the table build
            stage_table();
            tdes_process32_compact<true>(A0, A1, wtab, false);
            if (keep) {
#pragma unroll
                for (int s = 0; s < 32; ++s) {
                    const uint32_t md = smode[s];
                    const uint32_t mi = sidx[kSliceSlots * s + slot];
                    if (mi != ~0u && (md == TDES_MODE_CTR || md == TDES_MODE_CBC_DECRYPT)) {
                        const uint2 v = md == TDES_MODE_CTR ? ld_msg(msg_in(p, mi) + blk) : cbc_prev(p, mi, blk);
                        A0[s] ^= v.x;
                        A1[s] ^= v.y;
                    }
                }
                __syncwarp();  // in place: every read precedes the writes
#pragma unroll
                for (int s = 0; s < 32; ++s) {
                    const uint32_t mi = sidx[kSliceSlots * s + slot];
                    if (mi != ~0u) __stcs(msg_out(p, mi) + blk, make_uint2(A0[s], A1[s]));
                }
            } else {
#pragma unroll
                for (int s = 0; s < 32; ++s) {
                    const uint32_t ps = __shfl_sync(0xFFFFFFFFu, pos, s);
                    const uint32_t c = __shfl_sync(0xFFFFFFFFu, cm, s);
                    const uint32_t md = c >> 8;
                    if (slot < (c & 0xFFu) && (md == TDES_MODE_CTR || md == TDES_MODE_CBC_DECRYPT)) {
                        const uint32_t mi = p.order[ps + slot];
                        const uint2 v = md == TDES_MODE_CTR ? ld_msg(msg_in(p, mi) + blk) : cbc_prev(p, mi, blk);
                        A0[s] ^= v.x;
                        A1[s] ^= v.y;
                    }
                }
                __syncwarp();  // in place: every read precedes the writes
#pragma unroll
                for (int s = 0; s < 32; ++s) {
                    const uint32_t ps = __shfl_sync(0xFFFFFFFFu, pos, s);
                    const uint32_t cs = __shfl_sync(0xFFFFFFFFu, cm, s) & 0xFFu;
                    if (slot < cs)
                        __stcs(msg_out(p, p.order[ps + slot]) + blk, make_uint2(A0[s], A1[s]));
                }
            }
            __syncwarp();  // sidx and smode are rewritten by the next tile
        }
    }
}

// ------------------------------------------------------------------- host

int ufail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return status;
}

int ucuda(cudaError_t e, const char* what) {
    return ufail(e == cudaErrorMemoryAllocation ? TDES_ENOMEM : TDES_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Scratch layout: header, five per-group arrays, order, tile and slice maps.
struct UniLayout {
    size_t groups, max_tiles, max_slices;
    size_t o_counts, o_cursor, o_msg, o_tile, o_slice, o_order, o_tg, o_sg, o_part, o_base, o_held;
    size_t total;
};

UniLayout layout_for(uint64_t n_msgs, uint32_t m, uint32_t n_keys) {
    UniLayout L{};
    const uint64_t per_tile = kTileBlocks / m, per_slice = 32 / m;
    L.groups = (size_t)kModes * n_keys;
    L.max_tiles = n_msgs / per_tile + n_msgs / kChainsPerTile + 2;
    L.max_slices = (n_msgs / per_slice + 4ull * n_keys + 32) / 32 * 32 + n_msgs / 32 + n_keys + 32;
    const size_t g4 = al256(L.groups * 4);
    L.o_counts = al256(sizeof(UniHeader));
    L.o_cursor = L.o_counts + g4;
    L.o_msg = L.o_cursor + g4;
    L.o_tile = L.o_msg + g4;
    L.o_slice = L.o_tile + g4;
    L.o_order = L.o_slice + g4;
    L.o_tg = L.o_order + al256(n_msgs * 4);
    L.o_sg = L.o_tg + al256(L.max_tiles * 4);
    L.o_part = L.o_sg + al256(L.max_slices * 4);
    L.o_base = L.o_part + al256((size_t)scan_blocks(n_keys) * sizeof(Sums));
    L.o_held = L.o_base + al256((size_t)scan_blocks(n_keys) * sizeof(Sums));
    L.total = L.o_held + (size_t)kMaxChainCtas * kMixedChainWarps * 32 * 32 * sizeof(uint2);
    return L;
}

int check_shape(uint64_t n_msgs, uint64_t msg_bytes) {
    if (msg_bytes < 8 || msg_bytes > 256 || msg_bytes % 8 != 0)
        return ufail(TDES_EINVAL, "msg_bytes = %llu: must be a multiple of 8 in [8, 256]",
                     (unsigned long long)msg_bytes);
    if (n_msgs > TDES_UNIFORM_MAX_MSGS)
        return ufail(TDES_EINVAL, "n_msgs = %llu exceeds %llu", (unsigned long long)n_msgs,
                     (unsigned long long)TDES_UNIFORM_MAX_MSGS);
    return TDES_OK;
}

struct UniLaunch {
    int device = -1;
    int sms = 0;
    int work_ctas = 0;  // resident CTAs per SM of the work kernels
};

cudaError_t prepare(int device, UniLaunch* out) {
    static UniLaunch cache[64];
    static std::mutex mu;  // calls from several host threads share the cache
    std::lock_guard<std::mutex> lock(mu);
    if (device >= 0 && device < 64 && cache[device].device == device) {
        *out = cache[device];
        return cudaSuccess;
    }
    UniLaunch u;
    u.device = device;
    cudaError_t e = cudaDeviceGetAttribute(&u.sms, cudaDevAttrMultiProcessorCount, device);
    const int dyn = kUniWarps * kTileWarpBytes;
    const void* fns[] = {
        (const void*)uni_tile_kernel<kKindEcb, false>, (const void*)uni_tile_kernel<kKindEcb, true>,
        (const void*)uni_tile_kernel<kKindCtr, false>, (const void*)uni_tile_kernel<kKindCtr, true>,
        (const void*)uni_tile_kernel<kKindCbcDec, false>,
        (const void*)uni_tile_kernel<kKindCbcDec, true>};
    for (const void* f : fns)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(uni_tile_kernel<kKindCbcEnc, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kKeyChainWarps * kChainWarpBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(uni_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMixedChainWarps * kMixedChainWarpBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(uni_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kUniWarps * kMixedWarpBytes);
    int fit = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, uni_tile_kernel<kKindEcb, true>,
                                                          32 * kUniWarps, dyn);
    if (e != cudaSuccess) return e;
    u.work_ctas = std::max(1, fit);
    if (device >= 0 && device < 64) cache[device] = u;
    *out = u;
    return cudaSuccess;
}

}  // namespace
}  // namespace tdes

extern "C" {

int tdes_uniform_scratch_bytes(const tdes_keytable_t* kt, uint64_t n_msgs, uint64_t msg_bytes,
                               size_t* bytes) {
    if (kt == nullptr || bytes == nullptr)
        return tdes::ufail(TDES_EINVAL, "NULL argument to tdes_uniform_scratch_bytes");
    const int rc = tdes::check_shape(n_msgs, msg_bytes);
    if (rc != TDES_OK) return rc;
    *bytes = tdes::layout_for(n_msgs, (uint32_t)(msg_bytes / 8), kt->count).total;
    return TDES_OK;
}

int tdes_uniform_crypt(const tdes_keytable_t* kt, const uint32_t* key_index, const uint8_t* mode,
                       const uint64_t* iv_or_ctr, const void* in, void* out, uint64_t msg_bytes,
                       uint64_t n_msgs, void* scratch, size_t scratch_bytes,
                       uint64_t* skipped, tdes_stream_t stream) {
    using namespace tdes;
    if (kt == nullptr) return ufail(TDES_EINVAL, "key table is NULL");
    if (kt->count > kMaxKeys) return ufail(TDES_EINVAL, "key table of more than 2^26 triples");
    int rc = check_shape(n_msgs, msg_bytes);
    if (rc != TDES_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ucuda(e, "cudaGetDevice");
    if (dev != kt->device) return ufail(TDES_EINVAL, "key table lives on another device");
    if (reinterpret_cast<uintptr_t>(skipped) & 7u)
        return ufail(TDES_EINVAL, "skipped must be 8-byte aligned");
    if (n_msgs == 0) {
        if (skipped == nullptr) return TDES_OK;
        e = cudaMemsetAsync(skipped, 0, sizeof(uint64_t), s);
        return e == cudaSuccess ? TDES_OK : ucuda(e, "clearing the skipped count");
    }
    const uint64_t span = n_msgs * msg_bytes;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), o = reinterpret_cast<uintptr_t>(out);
    if (key_index == nullptr || mode == nullptr || iv_or_ctr == nullptr || in == nullptr ||
        out == nullptr || scratch == nullptr)
        return ufail(TDES_EINVAL, "NULL pointer");
    if (((a | o) & 7u) || (reinterpret_cast<uintptr_t>(key_index) & 3u) ||
        (reinterpret_cast<uintptr_t>(iv_or_ctr) & 7u) || (reinterpret_cast<uintptr_t>(scratch) & 255u))
        return ufail(TDES_EINVAL, "misaligned pointer (in/out/iv_or_ctr 8 bytes, key_index 4, "
                                  "scratch 256)");
    if (a != o && a < o + span && o < a + span)
        return ufail(TDES_EINVAL, "input and output overlap without being equal");
    const uint32_t m = (uint32_t)(msg_bytes / 8);
    const UniLayout L = layout_for(n_msgs, m, kt->count);
    if (scratch_bytes < L.total)
        return ufail(TDES_EINVAL, "scratch of %zu bytes, %zu needed", scratch_bytes, L.total);
    UniLaunch geo;
    e = prepare(dev, &geo);
    if (e != cudaSuccess) return ucuda(e, "uniform kernels set-up");

    uint8_t* base = static_cast<uint8_t*>(scratch);
    UniParams p{};
    p.keytab = kt->tabs;
    p.keystages = kt->stages;
    p.keypacked = kt->packed;
    p.n_keys = kt->count;
    p.n_groups = kModes * kt->count;
    p.key_index = key_index;
    p.mode = mode;
    p.iv = iv_or_ctr;
    p.in = static_cast<const uint8_t*>(in);
    p.out = static_cast<uint8_t*>(out);
    p.n_msgs = n_msgs;
    p.msg_bytes = (uint32_t)msg_bytes;
    p.m = m;
    p.magic = (65536u + m - 1) / m;
    p.per_tile = kTileBlocks / m;
    p.per_slice = 32u / m;
    const bool vec16 = m % 2 == 0 && ((a | o) & 15u) == 0;
    p.hdr = reinterpret_cast<UniHeader*>(base);
    p.counts = reinterpret_cast<uint32_t*>(base + L.o_counts);
    p.cursor = reinterpret_cast<uint32_t*>(base + L.o_cursor);
    p.msg_off = reinterpret_cast<uint32_t*>(base + L.o_msg);
    p.tile_off = reinterpret_cast<uint32_t*>(base + L.o_tile);
    p.slice_off = reinterpret_cast<uint32_t*>(base + L.o_slice);
    p.order = reinterpret_cast<uint32_t*>(base + L.o_order);
    p.tile_group = reinterpret_cast<uint32_t*>(base + L.o_tg);
    p.slice_group = reinterpret_cast<uint32_t*>(base + L.o_sg);
    p.held = reinterpret_cast<uint2*>(base + L.o_held);

    const int grid = geo.sms * 8;
    const int work_grid = geo.sms * geo.work_ctas;
    const size_t dyn = (size_t)kUniWarps * kTileWarpBytes;
    const char* what = "clearing the plan counters";
    e = cudaMemsetAsync(base, 0, L.o_cursor, s);  // header and counts
    if (e == cudaSuccess) {
        what = "planning kernels";
        uni_count_kernel<<<grid, 256, 0, s>>>(p);
        Sums* part = reinterpret_cast<Sums*>(base + L.o_part);
        Sums* bases = reinterpret_cast<Sums*>(base + L.o_base);
        const unsigned nblk = scan_blocks(kt->count);
        uni_scan_partial_kernel<<<nblk, kScanThreads, 0, s>>>(p, part);
        uni_scan_top_kernel<<<1, kScanThreads, 0, s>>>(p, part, bases);
        uni_scan_final_kernel<<<nblk, kScanThreads, 0, s>>>(p, bases);
        uni_map_kernel<<<grid, 256, 0, s>>>(p);
        uni_scatter_kernel<<<grid, 256, 0, s>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        what = "work kernels";
        const dim3 g(work_grid), b(32 * kUniWarps);
        if (vec16) {
            uni_tile_kernel<kKindEcb, true><<<g, b, dyn, s>>>(p);
            uni_tile_kernel<kKindCtr, true><<<g, b, dyn, s>>>(p);
            uni_tile_kernel<kKindCbcDec, true><<<g, b, dyn, s>>>(p);
        } else {
            uni_tile_kernel<kKindEcb, false><<<g, b, dyn, s>>>(p);
            uni_tile_kernel<kKindCtr, false><<<g, b, dyn, s>>>(p);
            uni_tile_kernel<kKindCbcDec, false><<<g, b, dyn, s>>>(p);
        }
        uni_mixed_kernel<false><<<g, b, (size_t)kUniWarps * kMixedWarpBytes, s>>>(p);
        // CBC-encryption chains: one CTA per SM, each warp with room for its
        // chains' message indices (2^28 messages of 64 B: 75.2 -> 73.1 ms
        // with the indices, alternating A/B runs) and its held blocks.  The
        // single-key tiles keep both in shared memory, 9 warps per CTA (2^22
        // single-key chains of 64 B: 1.60 -> 1.52 ms against 8).  The
        // mixed-key slices keep the held blocks in their warp's slab of
        // global scratch instead, which lets 12 warps fit (65.10 -> 64.65
        // ms for 2^28 messages, against 8 warps with everything in shared
        // memory; with the slab's accesses asking L2 to keep its lines,
        // 64.20 ms); with the indices there too, 16 warps at 128 registers
        // spilled 308 bytes and took 66.3 ms.  The single-key tiles with
        // their held blocks in the slab at 12 warps were slower (2^22 chains
        // under two keys: 1.71 -> 1.91 ms): with few keys a tile's chains lie
        // close together, their data is mostly in L2 already, and the
        // shared-memory held blocks' shorter latency counts for more.
        const dim3 g1(geo.sms);
        uni_tile_kernel<kKindCbcEnc, false><<<g1, dim3(32 * kKeyChainWarps),
                                              (size_t)kKeyChainWarps * kChainWarpBytes, s>>>(p);
        uni_mixed_kernel<true><<<dim3(std::min(geo.sms, kMaxChainCtas)), dim3(32 * kMixedChainWarps),
                                 (size_t)kMixedChainWarps * kMixedChainWarpBytes, s>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && skipped != nullptr) {
        what = "copying the skipped count";
        e = cudaMemcpyAsync(skipped, &p.hdr->skipped, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    }
    return e == cudaSuccess ? TDES_OK : ucuda(e, what);
}

int tdes_uniform_info(const void* scratch, tdes_uniform_info_t* info) {
    using namespace tdes;
    if (scratch == nullptr || info == nullptr)
        return ufail(TDES_EINVAL, "NULL argument to tdes_uniform_info");
    UniHeader h;
    const cudaError_t e = cudaMemcpy(&h, scratch, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ucuda(e, "reading the plan header");
    info->skipped = h.skipped;
    info->key_tiles = h.tiles[0];
    info->mixed_slices = h.slices[0];
    info->chain_key_tiles = h.tiles[1];
    info->chain_slices = h.slices[1];
    return TDES_OK;
}

}  // extern "C"
