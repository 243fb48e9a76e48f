// tdes_kernels.cu -- sm_103a kernels of the 3DES-EDE3 library.
//
// Work unit: a warp tile of 1024 consecutive 64-bit blocks (8 KiB).  Lane l
// of the warp owns the 32 blocks 2*(32*j + l) + h (j = 0..15, h = 0..1) of
// the tile, so every 128-bit load or store instruction of the warp covers
// 512 contiguous bytes.  The lane bitslices its 32 blocks in registers
// (tdes_bitslice.cuh), runs the 48 rounds of EDE3 as LOP3 logic on 64
// bit-planes, and un-bitslices.  The per-key round-constant table is staged
// into shared memory once per CTA and read with broadcast 128-bit loads.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "tdes_internal.h"
#include "tdes_keysched.cuh"
#include "tdes_scalar.cuh"

namespace tdes {

static_assert(kTableWords == TDES_TABLE_WORDS, "table size mismatch with the generator");
static_assert(kChunkBytes == TDES_SUBKEY_WORDS, "chunk size mismatch");

__device__ const uint8_t kRecipe[2][TDES_TABLE_WORDS][3] = TDES_RECIPE_INIT;
__device__ const uint8_t kRecipe1[2][TDES1_TABLE_WORDS][3] = TDES1_RECIPE_INIT;
__device__ const uint8_t kSubkeyBits[2][48][48] = TDES_SUBKEY_INIT;


int sbox_gate_count() { return TDES_SBOX_GATES; }

// ------------------------------------------------------------ key schedule
// One thread per output word: 2 bitsliced tables then 2 chunk tables.  A
// single-DES schedule (stages = 1) gets the short tables of the one-pass
// recipe; its chunk tables are those of EDE3 under (K, K, K), whose first 16
// rounds are the rounds of DES_K in both directions.
__global__ void tdes_keysched_kernel(Keys24 keys, int stages, uint32_t* __restrict__ tab_enc,
                                     uint32_t* __restrict__ tab_dec, uint8_t* __restrict__ ch_enc,
                                     uint8_t* __restrict__ ch_dec) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = stages == 1 ? TDES1_TABLE_WORDS : TDES_TABLE_WORDS;
    if (e < 2 * nw) {
        const int dir = e / nw, w = e % nw;
        (dir ? tab_dec : tab_enc)[w] = tdes_table_word(
            keys.b, stages == 1 ? kRecipe1[dir][w] : kRecipe[dir][w]);
    } else if (e < 2 * nw + 2 * TDES_SUBKEY_WORDS) {
        const int f = e - 2 * nw;
        const int dir = f / TDES_SUBKEY_WORDS, c = f % TDES_SUBKEY_WORDS;
        const int r = c / 8, g = c % 8;
        (dir ? ch_dec : ch_enc)[c] = tdes_subkey_chunk(keys.b, &kSubkeyBits[dir][r][6 * g]);
    }
}

cudaError_t launch_keysched(const Keys24& keys, int stages, uint32_t* tab_enc, uint32_t* tab_dec,
                            uint8_t* chunk_enc, uint8_t* chunk_dec, cudaStream_t s) {
    const int n = 2 * TDES_TABLE_WORDS + 2 * TDES_SUBKEY_WORDS;
    tdes_keysched_kernel<<<(n + 255) / 256, 256, 0, s>>>(keys, stages, tab_enc, tab_dec,
                                                          chunk_enc, chunk_dec);
    return cudaGetLastError();
}

// ------------------------------------------------------------ tile helpers

// Words of the bitsliced table of a schedule with STAGES DES passes.
template <int STAGES>
constexpr int table_words() { return STAGES == 1 ? TDES1_TABLE_WORDS : TDES_TABLE_WORDS; }

template <int STAGES>
__device__ __forceinline__ void stage_table(uint32_t* __restrict__ dst,
                                            const uint32_t* __restrict__ src) {
    for (int i = 4 * threadIdx.x; i < table_words<STAGES>(); i += 4 * blockDim.x)
        *reinterpret_cast<uint4*>(dst + i) = __ldg(reinterpret_cast<const uint4*>(src + i));
}

// Slot s = 2j + h of a lane holds tile block 2*(32j + lane) + h.
template <bool VEC>
__device__ __forceinline__ void load_tile(const uint8_t* base, uint64_t b0, uint64_t nblocks,
                                          uint32_t lane, uint32_t (&A0)[32], uint32_t (&A1)[32]) {
    if (VEC && b0 + kTileBlocks <= nblocks) {
        const uint4* p = reinterpret_cast<const uint4*>(base) + (b0 >> 1) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint4 v = __ldcs(p + 32 * j);
            A0[2 * j] = v.x;
            A1[2 * j] = v.y;
            A0[2 * j + 1] = v.z;
            A1[2 * j + 1] = v.w;
        }
    } else {  // ragged tile or 8-byte-aligned buffer: 64-bit accesses, bounds-checked
        const uint2* p = reinterpret_cast<const uint2*>(base) + b0;
        const uint32_t nvalid = (uint32_t)min((uint64_t)kTileBlocks, nblocks - b0);
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t i = 2u * (32u * j + lane) + h;
                uint2 v = make_uint2(0u, 0u);
                if (i < nvalid) v = __ldcs(p + i);
                A0[2 * j + h] = v.x;
                A1[2 * j + h] = v.y;
            }
    }
}

template <bool VEC>
__device__ __forceinline__ void store_tile(uint8_t* base, uint64_t b0, uint64_t nblocks,
                                           uint32_t lane, const uint32_t (&A0)[32],
                                           const uint32_t (&A1)[32]) {
    if (VEC && b0 + kTileBlocks <= nblocks) {
        uint4* p = reinterpret_cast<uint4*>(base) + (b0 >> 1) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            __stcs(p + 32 * j, make_uint4(A0[2 * j], A1[2 * j], A0[2 * j + 1], A1[2 * j + 1]));
    } else {
        uint2* p = reinterpret_cast<uint2*>(base) + b0;
        const uint32_t nvalid = (uint32_t)min((uint64_t)kTileBlocks, nblocks - b0);
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t i = 2u * (32u * j + lane) + h;
                if (i < nvalid) __stcs(p + i, make_uint2(A0[2 * j + h], A1[2 * j + h]));
            }
    }
}

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

// ------------------------------------------------------------------- ECB
// Full tiles of 16-byte-aligned buffers are prefetched one tile ahead into the
// warp's 8 KiB of shared memory with cp.async, so the next tile's memory
// latency hides behind the current tile's rounds.  Each lane copies, and
// later reads back, only its own 16 x 16 bytes; it reads a tile out of the
// buffer before it issues the copy of the next one into the same place.
constexpr int kCtrWarpBytes = 8 * kTileBlocks;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


template <bool VEC, int STAGES>
__global__ void __launch_bounds__(256, 2)
tdes_ecb_kernel(const uint32_t* __restrict__ table, const uint8_t* in, uint8_t* out,
                uint64_t nblocks) {
    __shared__ __align__(16) uint32_t tab[table_words<STAGES>()];
    extern __shared__ __align__(16) uint4 ecb_data[];  // kCtrWarpBytes per warp (VEC only)
    stage_table<STAGES>(tab, table);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = blockDim.x >> 5;
    uint4* wbuf = ecb_data + (threadIdx.x >> 5) * (kCtrWarpBytes / 16);
    // tile indices fit 32 bits: the host caps a call below 2^31 tiles (16 TiB)
    const uint32_t ntiles = (uint32_t)((nblocks + kTileBlocks - 1) / kTileBlocks);
    const uint32_t nfull = (uint32_t)(nblocks / kTileBlocks);  // tiles [0, nfull) are full
    const uint32_t stride = gridDim.x * warps;
    uint32_t t = blockIdx.x * warps + (threadIdx.x >> 5);
    if (VEC && t < nfull) {
        const uint4* p = reinterpret_cast<const uint4*>(in) + (uint64_t)t * (kTileBlocks / 2) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) cp_async16(wbuf + 32 * j + lane, p + 32 * j);
        cp_async_commit();
    }
    for (; t < ntiles; t += stride) {
        uint32_t A0[32], A1[32];
        if (VEC && t < nfull) {
            cp_async_wait_all();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint4 v = wbuf[32 * j + lane];
                A0[2 * j] = v.x;
                A1[2 * j] = v.y;
                A0[2 * j + 1] = v.z;
                A1[2 * j + 1] = v.w;
            }
            const uint32_t tn = t + stride;
            if (tn < nfull) {
                const uint4* p =
                    reinterpret_cast<const uint4*>(in) + (uint64_t)tn * (kTileBlocks / 2) + lane;
#pragma unroll
                for (int j = 0; j < 16; ++j) cp_async16(wbuf + 32 * j + lane, p + 32 * j);
                cp_async_commit();
            }
        } else {
            load_tile<VEC>(in, (uint64_t)t * kTileBlocks, nblocks, lane, A0, A1);
        }
        tdes_process32<STAGES>(A0, A1, tab);
        store_tile<VEC>(out, (uint64_t)t * kTileBlocks, nblocks, lane, A0, A1);
    }
}

// The kernels that stage data tiles take up to kWideWarps x 8 KiB of dynamic
// shared memory, above the default limit: raise it once per device.
template <bool VEC, int STAGES>
__global__ void tdes_ctr_kernel(const uint32_t* __restrict__ table, uint32_t nonce, uint32_t ctr0,
                                const uint8_t* in, uint8_t* out, uint64_t nblocks);
template <bool VEC, int STAGES>
__global__ void tdes_cbc_dec_kernel(const uint32_t* __restrict__ table, uint64_t iv,
                                    const uint8_t* in, uint8_t* out, uint64_t nblocks,
                                    const uint64_t* __restrict__ halo);

static std::atomic<bool> dyn_smem_ready[64];

static cudaError_t ensure_dyn_smem() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && dyn_smem_ready[dev]) return cudaSuccess;
    const int dyn = kWideWarps * kCtrWarpBytes;
    const void* fns[] = {
        reinterpret_cast<const void*>(tdes_ecb_kernel<true, 3>),
        reinterpret_cast<const void*>(tdes_ecb_kernel<true, 1>),
        reinterpret_cast<const void*>(tdes_ctr_kernel<true, 3>),
        reinterpret_cast<const void*>(tdes_ctr_kernel<false, 3>),
        reinterpret_cast<const void*>(tdes_ctr_kernel<true, 1>),
        reinterpret_cast<const void*>(tdes_ctr_kernel<false, 1>),
        reinterpret_cast<const void*>(tdes_cbc_dec_kernel<true, 3>),
        reinterpret_cast<const void*>(tdes_cbc_dec_kernel<true, 1>),
    };
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
    }
    if (dev >= 0 && dev < 64) dyn_smem_ready[dev] = true;
    return cudaSuccess;
}

template <int STAGES>
static void ecb_launch(const uint32_t* tab, const void* in, void* out, uint64_t nblocks,
                       bool vec16, Geometry g, cudaStream_t s) {
    if (vec16)
        tdes_ecb_kernel<true, STAGES>
            <<<g.grid, g.threads, (size_t)(g.threads / 32) * kCtrWarpBytes, s>>>(
                tab, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), nblocks);
    else
        tdes_ecb_kernel<false, STAGES><<<g.grid, g.threads, 0, s>>>(
            tab, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), nblocks);
}

cudaError_t launch_ecb(const uint32_t* tab, int stages, const void* in, void* out,
                       uint64_t nblocks, bool vec16, Geometry g, cudaStream_t s) {
    cudaError_t e = ensure_dyn_smem();
    if (e != cudaSuccess) return e;
    if (stages == 1)
        ecb_launch<1>(tab, in, out, nblocks, vec16, g, s);
    else
        ecb_launch<3>(tab, in, out, nblocks, vec16, g, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- CTR
// Keystream block i = E(nonce || ctr0 + i); the counter blocks are built in
// registers.  The data tile the keystream is XORed into is copied into the
// warp's 8 KiB of shared memory with cp.async before the rounds start, so
// its memory latency hides behind them.
template <bool VEC, int STAGES>
__global__ void __launch_bounds__(256, 2)
tdes_ctr_kernel(const uint32_t* __restrict__ table, uint32_t nonce, uint32_t ctr0,
                const uint8_t* in, uint8_t* out, uint64_t nblocks) {
    __shared__ __align__(16) uint32_t tab[table_words<STAGES>()];
    extern __shared__ __align__(16) uint4 ctr_data[];  // kCtrWarpBytes per warp
    stage_table<STAGES>(tab, table);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = blockDim.x >> 5;
    uint4* wbuf = ctr_data + (threadIdx.x >> 5) * (kCtrWarpBytes / 16);
    // Tile loop index and ragged-tile indexing: 64-bit for the 16-byte path
    // (measured 410 GB/s at 1 GiB against 399 with 32-bit indices there),
    // 32-bit for the 8-byte-aligned variant (the 64-bit form spills there).
    // Tile indices fit 32 bits: the host caps a call below 2^31 tiles.
    using Idx = typename std::conditional<VEC, uint64_t, uint32_t>::type;
    const Idx ntiles = (Idx)((nblocks + kTileBlocks - 1) / kTileBlocks);
    const uint32_t nw = bswap32(nonce);
    for (Idx t = (Idx)blockIdx.x * warps + (threadIdx.x >> 5); t < ntiles;
         t += (Idx)gridDim.x * warps) {
        const uint64_t b0 = (uint64_t)t * kTileBlocks;
        const bool full = VEC && b0 + kTileBlocks <= nblocks;
        if (full) {  // each lane copies, and later reads back, only its own 16 x 16 bytes
            const uint4* p = reinterpret_cast<const uint4*>(in) + (b0 >> 1) + lane;
#pragma unroll
            for (int j = 0; j < 16; ++j) cp_async16(wbuf + 32 * j + lane, p + 32 * j);
            cp_async_commit();
        }
        uint32_t A0[32], A1[32];
#pragma unroll
        for (int j = 0; j < 16; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t b = (uint32_t)b0 + 2u * (32u * j + lane) + h;
                A0[2 * j + h] = nw;
                A1[2 * j + h] = bswap32(ctr0 + b);
            }
        tdes_process32<STAGES>(A0, A1, tab);
        if (full) {
            cp_async_wait_all();
            uint4* q = reinterpret_cast<uint4*>(out) + (b0 >> 1) + lane;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint4 v = wbuf[32 * j + lane];
                __stcs(q + 32 * j, make_uint4(v.x ^ A0[2 * j], v.y ^ A1[2 * j],
                                              v.z ^ A0[2 * j + 1], v.w ^ A1[2 * j + 1]));
            }
        } else if (VEC) {  // the ragged last tile
            const uint2* p = reinterpret_cast<const uint2*>(in);
            uint2* q = reinterpret_cast<uint2*>(out);
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint64_t b = b0 + 2 * (32 * j + lane) + h;
                    if (b < nblocks) {
                        const uint2 v = __ldcs(p + b);
                        __stcs(q + b, make_uint2(v.x ^ A0[2 * j + h], v.y ^ A1[2 * j + h]));
                    }
                }
        } else {  // 8-byte-aligned buffer: 32-bit in-tile indices
            const uint2* p = reinterpret_cast<const uint2*>(in) + b0;
            uint2* q = reinterpret_cast<uint2*>(out) + b0;
            const uint32_t nvalid = (uint32_t)min((uint64_t)kTileBlocks, nblocks - b0);
#pragma unroll
            for (int j = 0; j < 16; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t i = 2u * (32u * j + lane) + h;
                    if (i < nvalid) {
                        const uint2 v = __ldcs(p + i);
                        __stcs(q + i, make_uint2(v.x ^ A0[2 * j + h], v.y ^ A1[2 * j + h]));
                    }
                }
        }
    }
}

template <int STAGES>
static void ctr_launch(const uint32_t* tab_enc, uint32_t nonce, uint32_t ctr0, const void* in,
                       void* out, uint64_t nblocks, bool vec16, Geometry g, cudaStream_t s) {
    const size_t dyn = (size_t)(g.threads / 32) * kCtrWarpBytes;
    if (vec16)
        tdes_ctr_kernel<true, STAGES><<<g.grid, g.threads, dyn, s>>>(
            tab_enc, nonce, ctr0, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out),
            nblocks);
    else
        tdes_ctr_kernel<false, STAGES><<<g.grid, g.threads, dyn, s>>>(
            tab_enc, nonce, ctr0, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out),
            nblocks);
}

cudaError_t launch_ctr(const uint32_t* tab_enc, int stages, uint32_t nonce, uint32_t ctr0,
                       const void* in, void* out, uint64_t nblocks, bool vec16, Geometry g,
                       cudaStream_t s) {
    cudaError_t e = ensure_dyn_smem();
    if (e != cudaSuccess) return e;
    if (stages == 1)
        ctr_launch<1>(tab_enc, nonce, ctr0, in, out, nblocks, vec16, g, s);
    else
        ctr_launch<3>(tab_enc, nonce, ctr0, in, out, nblocks, vec16, g, s);
    return cudaGetLastError();
}

// --------------------------------------------------------------- CBC decrypt
// halo[t] = ciphertext block just before tile t (t >= 1), taken before an
// in-place decryption can overwrite it.
__global__ void tdes_cbc_halo_kernel(const uint64_t* __restrict__ in, uint64_t* __restrict__ halo,
                                     uint64_t ntiles) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 1 && t < ntiles) halo[t] = in[t * kTileBlocks - 1];
}

cudaError_t launch_cbc_halo(const void* in, uint64_t* halo, uint64_t nblocks, cudaStream_t s) {
    const uint64_t ntiles = (nblocks + kTileBlocks - 1) / kTileBlocks;
    if (ntiles <= 1) return cudaSuccess;
    tdes_cbc_halo_kernel<<<(unsigned)((ntiles + 255) / 256), 256, 0, s>>>(
        static_cast<const uint64_t*>(in), halo, ntiles);
    return cudaGetLastError();
}

// P_i = D(C_i) XOR C_{i-1}.  The ciphertext the XOR needs is re-read after
// the rounds: a lane's own blocks and its neighbours' in the same tile are
// still intact (the warp stores only after __syncwarp); the block before the
// tile comes from `halo` when decrypting in place, else from the input.
template <bool VEC, int STAGES>
__global__ void __launch_bounds__(256, 2)
tdes_cbc_dec_kernel(const uint32_t* __restrict__ table, uint64_t iv, const uint8_t* in,
                    uint8_t* out, uint64_t nblocks, const uint64_t* __restrict__ halo) {
    __shared__ __align__(16) uint32_t tab[table_words<STAGES>()];
    extern __shared__ __align__(16) uint4 cbc_data[];  // kCtrWarpBytes per warp (VEC only)
    stage_table<STAGES>(tab, table);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = blockDim.x >> 5;
    uint4* wbuf = cbc_data + (threadIdx.x >> 5) * (kCtrWarpBytes / 16);
    // tile indices fit 32 bits: the host caps a call below 2^31 tiles (16 TiB)
    const uint32_t ntiles = (uint32_t)((nblocks + kTileBlocks - 1) / kTileBlocks);
    const uint32_t nfull = (uint32_t)(nblocks / kTileBlocks);  // tiles [0, nfull) are full
    const uint32_t stride = gridDim.x * warps;
    const uint2 ivw = make_uint2(bswap32((uint32_t)(iv >> 32)), bswap32((uint32_t)iv));
    const uint2* c = reinterpret_cast<const uint2*>(in);
    uint32_t t = blockIdx.x * warps + (threadIdx.x >> 5);
    if (VEC && t < nfull) {  // full tiles are prefetched one ahead, as in ECB
        const uint4* p = reinterpret_cast<const uint4*>(in) + (uint64_t)t * (kTileBlocks / 2) + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) cp_async16(wbuf + 32 * j + lane, p + 32 * j);
        cp_async_commit();
    }
    for (; t < ntiles; t += stride) {
        const uint64_t b0 = (uint64_t)t * kTileBlocks;
        uint32_t A0[32], A1[32];
        const bool full = VEC && t < nfull;
        if (full) {
            cp_async_wait_all();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint4 v = wbuf[32 * j + lane];
                A0[2 * j] = v.x;
                A1[2 * j] = v.y;
                A0[2 * j + 1] = v.z;
                A1[2 * j + 1] = v.w;
            }
            const uint32_t tn = t + stride;
            if (tn < nfull) {
                const uint4* p =
                    reinterpret_cast<const uint4*>(in) + (uint64_t)tn * (kTileBlocks / 2) + lane;
#pragma unroll
                for (int j = 0; j < 16; ++j) cp_async16(wbuf + 32 * j + lane, p + 32 * j);
                cp_async_commit();
            }
        } else {
            load_tile<VEC>(in, b0, nblocks, lane, A0, A1);
        }
        tdes_process32<STAGES>(A0, A1, tab);
        const uint2* ct = c + b0;  // this tile's ciphertext, 32-bit indices below
        const uint32_t nvalid = (uint32_t)min((uint64_t)kTileBlocks, nblocks - b0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t i = 2u * (32u * j + lane);  // slot 2j; slot 2j+1 is i + 1
            uint2 prev0, prev1 = make_uint2(0u, 0u);
            if (j == 0 && lane == 0) {  // the block before the tile
                if (b0 == 0) {
                    prev0 = ivw;
                } else if (halo != nullptr) {
                    const uint64_t hv = halo[t];
                    prev0 = make_uint2((uint32_t)hv, (uint32_t)(hv >> 32));
                } else {
                    prev0 = c[b0 - 1];
                }
            } else {
                prev0 = (i - 1 < nvalid) ? ct[i - 1] : make_uint2(0u, 0u);
            }
            if (i < nvalid) prev1 = ct[i];
            A0[2 * j] ^= prev0.x;
            A1[2 * j] ^= prev0.y;
            A0[2 * j + 1] ^= prev1.x;
            A1[2 * j + 1] ^= prev1.y;
        }
        __syncwarp();
        store_tile<VEC>(out, b0, nblocks, lane, A0, A1);
    }
}

template <int STAGES>
static void cbc_dec_launch(const uint32_t* tab_dec, uint64_t iv, const void* in, void* out,
                           uint64_t nblocks, const uint64_t* halo, bool vec16, Geometry g,
                           cudaStream_t s) {
    if (vec16)
        tdes_cbc_dec_kernel<true, STAGES>
            <<<g.grid, g.threads, (size_t)(g.threads / 32) * kCtrWarpBytes, s>>>(
                tab_dec, iv, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out),
                nblocks, halo);
    else
        tdes_cbc_dec_kernel<false, STAGES><<<g.grid, g.threads, 0, s>>>(
            tab_dec, iv, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out), nblocks,
            halo);
}

cudaError_t launch_cbc_dec(const uint32_t* tab_dec, int stages, uint64_t iv, const void* in,
                           void* out, uint64_t nblocks, const uint64_t* halo, bool vec16,
                           Geometry g, cudaStream_t s) {
    cudaError_t e = ensure_dyn_smem();
    if (e != cudaSuccess) return e;
    if (stages == 1)
        cbc_dec_launch<1>(tab_dec, iv, in, out, nblocks, halo, vec16, g, s);
    else
        cbc_dec_launch<3>(tab_dec, iv, in, out, nblocks, halo, vec16, g, s);
    return cudaGetLastError();
}

// --------------------------------------------------------------- CBC encrypt
// C_i = E(P_i XOR C_{i-1}): serial.  One warp walks the chain cooperatively
// (tdes_block_warp: each lane one bit of the round function, a ballot per
// round); the next plaintext block is loaded one block ahead.
__device__ const uint32_t kLaneSbox[32][4] = TDES_LANE_SBOX_INIT;
__device__ const uint32_t kLaneIP[32][2] = TDES_LANE_IP_INIT;
__device__ const uint32_t kLaneFP[32][2] = TDES_LANE_FP_INIT;

__device__ __forceinline__ LaneConsts lane_consts(uint32_t lane) {
    LaneConsts c;
    c.mlo = kLaneSbox[lane][0];
    c.mhi = kLaneSbox[lane][1];
    c.rot = kLaneSbox[lane][2];
    c.keypos = kLaneSbox[lane][3];
    c.ip_hi = kLaneIP[lane][0];
    c.ip_lo = kLaneIP[lane][1];
    c.fp_hi = kLaneFP[lane][0];
    c.fp_lo = kLaneFP[lane][1];
    return c;
}

template <int ROUNDS>
__global__ void tdes_cbc_enc_kernel(const uint8_t* __restrict__ chunks_g, uint64_t iv,
                                    const uint8_t* in, uint8_t* out, uint64_t nblocks) {
    __shared__ __align__(16) uint8_t keys[TDES_SUBKEY_WORDS];
    const uint32_t lane = threadIdx.x & 31u;
    for (int i = threadIdx.x; i < TDES_SUBKEY_WORDS; i += blockDim.x) keys[i] = chunks_g[i];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const LaneConsts c = lane_consts(lane);
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

cudaError_t launch_cbc_enc(const uint8_t* chunk_enc, int stages, uint64_t iv, const void* in,
                           void* out, uint64_t nblocks, cudaStream_t s) {
    if (stages == 1)
        tdes_cbc_enc_kernel<16><<<1, 32, 0, s>>>(chunk_enc, iv, static_cast<const uint8_t*>(in),
                                                 static_cast<uint8_t*>(out), nblocks);
    else
        tdes_cbc_enc_kernel<48><<<1, 32, 0, s>>>(chunk_enc, iv, static_cast<const uint8_t*>(in),
                                                 static_cast<uint8_t*>(out), nblocks);
    return cudaGetLastError();
}

// ------------------------------------------------------------- occupancy
int wide_ctas_per_sm(int kernel_id) {
    int n = 0;
    const int threads = 32 * kWideWarps;
    cudaError_t e = cudaSuccess;
    switch (kernel_id) {
        case kEcb:
            e = ensure_dyn_smem();
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &n, tdes_ecb_kernel<true, 3>, threads, kWideWarps * kCtrWarpBytes);
            break;
        case kCtr:
            e = ensure_dyn_smem();
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &n, tdes_ctr_kernel<true, 3>, threads, kWideWarps * kCtrWarpBytes);
            break;
        default:
            e = ensure_dyn_smem();
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &n, tdes_cbc_dec_kernel<true, 3>, threads, kWideWarps * kCtrWarpBytes);
            break;
    }
    if (e != cudaSuccess || n < 1) return 1;
    return n;
}

}  // namespace tdes
