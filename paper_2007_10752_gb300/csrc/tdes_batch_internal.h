// tdes_batch_internal.h -- batch plans shared by the batch API (tdes_batch.cu)
// and the serving loop (tdes_serve.cu).  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/tdes.h"

struct tdes_keytable {
    int device;
    uint32_t count;
    void* mem;
    uint32_t* tabs;   // [key][dir][3328] bitsliced round-constant tables
    uint8_t* chunks;  // [key][dir][384] scalar round-key words
    uint8_t* stages;  // [key] DES passes: 3, or 1 for a triple that reduces to single DES
    uint32_t* packed; // [key][dir][104] three-pass tables, one bit per word (mixed-key tiles)
    std::vector<uint8_t> host_stages;  // host copy of `stages`, for planning without a device read
};

namespace tdes {

constexpr int kPackedWords = 104;  // 3328 table words at one bit each
constexpr int kChainSlots = 1024;  // SM sub-partitions tracked for C items (4 per SM)
// A plan's claim counters, zeroed together: the item counter, the C-item
// counter, the count of warps that have finished (batch timing), padding,
// then the chain slots.
constexpr int kCounterBytes = 32 + 4 * kChainSlots;

// One slice (bit position) of a mixed-key tile: up to 32 blocks of small
// messages under one key and direction, one block per lane.
struct MSlice {
    uint32_t msg0;    // first of the slice's messages in m_list
    uint32_t starts;  // bit l set where a message begins at lane l
    uint32_t nvalid;  // lanes [0, nvalid) hold blocks
    uint32_t keydir;  // key << 1 | direction (1: decryption table)
};

// A run of consecutive blocks of one message, run one block per lane by the
// scalar round (S items hold up to 32 blocks of such pieces).
struct SPiece {
    uint32_t msg;    // index into msgs
    uint32_t first;  // first block of the piece
    uint32_t n;      // blocks, 1..32
    uint32_t pad;
};

struct BatchMsg {
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    uint64_t iv;  // CBC: IV; CTR: first counter block
    uint32_t key;
    uint32_t mode;
};

struct BatchParams {
    const BatchMsg* msgs;
    const uint32_t* keytab;    // [key][dir][TDES_TABLE_WORDS]
    const uint8_t* keychunks;  // [key][dir][TDES_SUBKEY_WORDS]
    const uint8_t* keystages;  // [key] 3 (EDE3) or 1 (single DES: a one-pass table)
    const uint32_t* c_list;    // CBC-enc message indices, longest first
    uint32_t n_c, n_c_items;
    uint32_t n_c_solo;         // the first n_c_solo chains run one per warp
    const uint32_t* b_msg;     // large message index per B entry
    const uint64_t* b_prefix;  // exclusive prefix of tiles, n_b + 1 entries
    const uint32_t* b_tile;    // per B tile: its B entry (index into b_msg / b_prefix)
    uint32_t n_b;
    uint64_t n_b_tiles;
    const uint32_t* keypacked; // [key][dir][kPackedWords]
    const uint32_t* m_list;    // small messages in mixed-key tiles, in slice order
    const MSlice* m_slices;    // 32 per mixed-key tile
    uint32_t n_m_tiles;
    const SPiece* s_pieces;    // pieces of small and medium messages
    const uint2* s_items;      // (first, count) into s_pieces, <= 32 blocks per item
    uint32_t n_s_items;
    uint64_t* halo;            // per B tile: ciphertext block before it (in-place CBC-dec)
    unsigned long long* counter;   // claims of B and S items (and C items, see below)
    unsigned long long* c_counter; // claims of C items by warps on an SMSP without one
    uint32_t* chain_slot;          // [kChainSlots]: 1 while an SMSP runs a C item
    uint32_t b_chunk;          // B tiles per claimed item (set at launch)
    uint64_t n_b_chunks;       // ceil(n_b_tiles / b_chunk)
    // Optional (nullable) device timestamps of the batch in ns of the GPU's
    // global timer: [0] when its first kernel's first CTA starts, [1] when the
    // last warp of its last kernel finishes (counted in *done_warps).
    unsigned long long* batch_times;
    uint32_t* done_warps;
    bool times_end_in_mixed;   // the mixed-key kernel is the batch's last kernel
};


// A message of at least kDirectBytes in ECB, CTR or out-of-place CBC
// decryption: a batch plan runs it through the single-key kernels (their
// shared-memory prefetch of each tile does not fit beside the batch kernel's
// per-warp key table) instead of as batch tiles.
struct DirectMsg {
    uint32_t mode, key;
    uint64_t iv;  // CBC: IV; CTR: first counter block
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    int stages;   // DES passes of the key (read from the key table at plan time)
};

// Launch shape of the batch kernels (the autotuner's search space).  The
// member defaults are a plan's default shape: on the 4096-message batch's
// parallel modes, 8 warps with the compact round body measured 3.60 ms
// against 3.78 ms with three loop bodies (median of 10 graph replays).
struct LaunchShape {
    int warps = 8;             // warps per CTA, 1..8 (each owns a 13 KB shared-memory slice)
    int ctas_per_sm = 0;       // resident CTAs per SM for the grid; <= 0: as many as fit
    int tiles_per_claim = 0;   // 1024-block tiles a warp claims at once; 0: automatic
    int round_form = 1;        // 0: three loop bodies (one per DES pass); 1: one compact body
};

// A batch laid out on the host as the byte image of its device buffer.
struct PlanHost {
    std::vector<uint8_t> image;
    size_t o_msgs = 0, o_c = 0, o_bm = 0, o_bp = 0, o_bt = 0, o_ml = 0, o_ms = 0, o_sl = 0,
           o_si = 0, o_halo = 0, o_ctr = 0;
    uint32_t n_c = 0, n_c_solo = 0, n_c_items = 0, n_b = 0, n_m_tiles = 0, n_s_items = 0;
    uint64_t n_b_tiles = 0, total_items = 0;
    bool needs_halo = false;
    uint64_t bytes_per_mode[5] = {0, 0, 0, 0, 0};
    // payload bytes per kind of work: [0] bitsliced tiles, [1] mixed-key tiles,
    // [2] one block per lane (S items), [3] CBC-encryption chains, [4] direct
    uint64_t kind_bytes[5] = {0, 0, 0, 0, 0};
    int invalid = 0;
    std::vector<DirectMsg> direct;  // only when the plan allows them
};

constexpr uint64_t kDirectBytes = 64ull << 20;

// TDES_OK or TDES_EINVAL for one descriptor against a key table of key_count.
int validate_desc(const tdes_desc_t& d, uint32_t key_count);
// Validates and classifies n descriptors into `out` (status: nullable, n entries).
// allow_direct: messages of kDirectBytes or more (not CBC encryption, not
// in-place CBC decryption) go to out->direct instead of batch tiles.
void build_plan(const tdes_desc_t* d, uint32_t n, uint32_t key_count, int* status, PlanHost* out,
                bool allow_direct = false);
// Tiles per claim that a shape's 0 (automatic) stands for, for a plan of
// n_tiles tiles run by warps_total warps.
uint32_t auto_tiles_per_claim(uint64_t n_tiles, uint64_t warps_total);
// Kernel parameters of a plan whose image was copied to dev_base.
BatchParams bind_plan(const PlanHost& h, void* dev_base, const tdes_keytable* kt);
// Sets the batch kernel's shared-memory limit for `warps` warps per CTA and
// returns how many CTAs of that shape fit on an SM.
cudaError_t prepare_batch_kernel(int warps, size_t* dyn_smem, int* ctas_fit);
// Counter reset (unless the caller has just copied the plan image, whose
// counter is zero), halo snapshot (if needed), the mixed-key kernel (if any)
// and the persistent kernel on s, in the given shape (shape.warps warps per
// CTA, at most max_ctas CTAs; dyn_smem from prepare_batch_kernel).
cudaError_t enqueue_batch(const BatchParams& p, uint64_t total_items, bool needs_halo,
                          const LaunchShape& shape, size_t dyn_smem, uint64_t max_ctas,
                          cudaStream_t s, bool counter_fresh = false);

// The single-key kernel launches of a plan's direct messages on s (before
// its batch launches; each uses the whole GPU).
cudaError_t enqueue_direct(const std::vector<DirectMsg>& direct, const tdes_keytable* kt,
                           int device, cudaStream_t s);

}  // namespace tdes

// A planned batch (opaque tdes_batch_t in include/tdes.h).
struct tdes_batch {
    int device;
    const tdes_keytable* kt;
    void* mem;
    tdes::BatchParams params;
    uint64_t total_items;
    bool needs_halo;
    tdes::LaunchShape shape;  // ctas_per_sm resolved (>= 1)
    int ctas_fit;             // CTAs of shape.warps warps that fit on an SM
    int sms;
    size_t dyn_smem;
    bool tuned;               // shape taken from the autotuner's cache
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    uint64_t bytes[5];  // payload bytes per mode
    uint64_t kind_bytes[5];
    std::vector<tdes::DirectMsg> direct;  // run by the single-key kernels
    std::vector<int> status;              // per descriptor, from planning
};

namespace tdes {
// Sets a batch's launch shape (recapturing its graph on next use).
int set_batch_shape(tdes_batch* b, const LaunchShape& shape);
// Queues a batch's whole work on s (direct messages, then the batch kernels).
cudaError_t enqueue_planned(tdes_batch* b, cudaStream_t s);
}  // namespace tdes
