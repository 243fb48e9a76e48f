// tdes_internal.h -- launchers shared by the C ABI (tdes_api.cu) and the
// kernels (tdes_kernels.cu).  Not part of the public interface.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

// The library's key-schedule object (opaque tdes_ks_t in include/tdes.h).
struct tdes_ks {
    int device;
    int stages;             // DES passes per block: 3 (EDE3) or 1 (single DES)
    void* mem;              // one cudaMalloc holding everything below
    uint32_t* tab[2];       // bitsliced round-constant tables: [0] encrypt, [1] decrypt
    uint8_t* chunk[2];      // scalar-path round-key groups: [0] encrypt, [1] decrypt
};

namespace tdes {

// Records the message tdes_last_error() returns on this host thread.
void set_last_error(const char* msg);

// True if the GPU can address `p` with the same pointer: device or managed
// memory, or page-locked host memory mapped into the device address space
// (what cudaHostAlloc gives on a unified-address system).  Pageable host
// memory is refused: a kernel access to it could fault.
bool gpu_addressable(const void* p);
// True for page-locked host memory (whether or not it is mapped).
bool host_memory(const void* p);

constexpr int kTileBlocks = 1024;  // blocks per warp tile: 32 lanes x 32 blocks
constexpr int kWideWarps = 8;      // warps per CTA for large inputs
constexpr int kTableWords = 3328;  // words of one bitsliced round-constant table
constexpr int kChunkBytes = 384;   // 48 rounds x 8 six-bit round-key groups

struct Keys24 {
    uint8_t b[24];
};

// Launch geometry for `ntiles` warp tiles on the current device.
struct Geometry {
    int grid;
    int threads;
};
Geometry geometry_for(uint64_t ntiles, int kernel_id, int device);

enum KernelId { kEcb = 0, kCtr = 1, kCbcDec = 2, kNumKernels = 3 };

// `stages` (1 or 3) selects the single-DES or the EDE3 kernels; the tables
// passed must have been built for the same number of stages.
cudaError_t launch_keysched(const Keys24& keys, int stages, uint32_t* tab_enc, uint32_t* tab_dec,
                            uint8_t* chunk_enc, uint8_t* chunk_dec, cudaStream_t s);
cudaError_t launch_ecb(const uint32_t* tab, int stages, const void* in, void* out,
                       uint64_t nblocks, bool vec16, Geometry g, cudaStream_t s);
cudaError_t launch_ctr(const uint32_t* tab_enc, int stages, uint32_t nonce, uint32_t ctr0,
                       const void* in, void* out, uint64_t nblocks, bool vec16, Geometry g,
                       cudaStream_t s);
cudaError_t launch_cbc_halo(const void* in, uint64_t* halo, uint64_t nblocks, cudaStream_t s);
cudaError_t launch_cbc_dec(const uint32_t* tab_dec, int stages, uint64_t iv, const void* in,
                           void* out, uint64_t nblocks, const uint64_t* halo, bool vec16,
                           Geometry g, cudaStream_t s);
cudaError_t launch_cbc_enc(const uint8_t* chunk_enc, int stages, uint64_t iv, const void* in,
                           void* out, uint64_t nblocks, cudaStream_t s);

// One block per thread (tdes_small.cu), for calls too small to fill the GPU
// with bitsliced tiles.  chunks: the call's scalar round-key groups of the
// wanted direction; iv: the CBC IV, or nonce << 32 | ctr0 for CTR.
enum SmallMode { kSmallEcb = 0, kSmallCtr = 1, kSmallCbcDec = 2 };
cudaError_t launch_small(const uint8_t* chunks, int stages, int mode, uint64_t iv, const void* in,
                         void* out, uint64_t nblocks, int threads, cudaStream_t s);

// Occupancy (CTAs per SM) of a bitsliced kernel at kWideWarps warps per CTA.
int wide_ctas_per_sm(int kernel_id);
int sbox_gate_count();

}  // namespace tdes
