// tdes_small.cu -- single-key calls too small to fill the GPU with bitsliced
// tiles: one 64-bit block per thread.
//
// A bitsliced tile is 1024 blocks and costs each lane about 12 k logic
// operations (48 rounds over 64 bit-planes), so a call of a few tiles takes
// one tile's latency however few blocks it holds.  Here each thread runs its
// own block through the scalar round (tdes_block_scalar_nib: the expansion
// windows as two rotates, eight S-box/permutation table lookups, nibble
// tables for IP and FP), a chain of 48 dependent rounds (16 for single DES).
// The tables and the call's round-key words are staged in shared memory once
// per CTA.
#include <cuda_runtime.h>

#include "tdes_internal.h"
#include "tdes_keysched.cuh"
#include "tdes_scalar.cuh"

namespace tdes {

__device__ const uint32_t kSmallSP[8][64] = TDES_SP_INIT;
__device__ const uint64_t kSmallIPN[16][16] = TDES_IPN_INIT;
__device__ const uint64_t kSmallFPN[16][16] = TDES_FPN_INIT;

struct SmallTables {
    uint32_t sp[8 * 64];
    uint64_t ipn[16 * 16];
    uint64_t fpn[16 * 16];
    uint32_t keys[TDES_SUBKEY_WORDS / 4];
};

__device__ __forceinline__ uint64_t small_load_be(const uint8_t* p, uint64_t i) {
    return bswap64(reinterpret_cast<const uint64_t*>(p)[i]);
}

// mode: kSmallEcb (chunks of the direction wanted), kSmallCtr (block i is
// E(nonce || ctr0 + i) XOR in_i; iv = nonce << 32 | ctr0), kSmallCbcDec
// (D(in_i) XOR in_{i-1}, in_{-1} = iv).  In place is safe for ECB and CTR
// (each thread reads and writes only its own block); for CBC decryption the
// host uses this kernel in place only with a single CTA, whose threads all
// read before any writes.
template <int ROUNDS>
__global__ void __launch_bounds__(1024)
tdes_small_kernel(const uint8_t* __restrict__ chunks, int mode, uint64_t iv, const uint8_t* in,
                  uint8_t* out, uint64_t nblocks) {
    __shared__ __align__(16) SmallTables st;
    for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) st.sp[i] = (&kSmallSP[0][0])[i];
    for (int i = threadIdx.x; i < 16 * 16; i += blockDim.x) {
        st.ipn[i] = (&kSmallIPN[0][0])[i];
        st.fpn[i] = (&kSmallFPN[0][0])[i];
    }
    for (int i = threadIdx.x; i < TDES_SUBKEY_WORDS / 4; i += blockDim.x)
        st.keys[i] = __ldg(reinterpret_cast<const uint32_t*>(chunks) + i);
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x = 0, prev = 0;
    if (b < nblocks) {
        if (mode == kSmallCtr) {
            x = (iv & 0xFFFFFFFF00000000ull) | (uint32_t)((uint32_t)iv + (uint32_t)b);
            prev = small_load_be(in, b);
        } else {
            x = small_load_be(in, b);
            if (mode == kSmallCbcDec) prev = b ? small_load_be(in, b - 1) : iv;
        }
    }
    __syncthreads();  // tables staged; every read of this CTA precedes its writes
    if (b < nblocks) {
        uint64_t y = tdes_block_scalar_nib<ROUNDS>(x, st.sp, st.keys, st.ipn, st.fpn);
        if (mode != kSmallEcb) y ^= prev;
        reinterpret_cast<uint64_t*>(out)[b] = bswap64(y);
    }
}

cudaError_t launch_small(const uint8_t* chunks, int stages, int mode, uint64_t iv, const void* in,
                         void* out, uint64_t nblocks, int threads, cudaStream_t s) {
    const uint64_t grid = (nblocks + threads - 1) / threads;
    if (stages == 1)
        tdes_small_kernel<16><<<(unsigned)grid, threads, 0, s>>>(
            chunks, mode, iv, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out),
            nblocks);
    else
        tdes_small_kernel<48><<<(unsigned)grid, threads, 0, s>>>(
            chunks, mode, iv, static_cast<const uint8_t*>(in), static_cast<uint8_t*>(out),
            nblocks);
    return cudaGetLastError();
}

}  // namespace tdes
