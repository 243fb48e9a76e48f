// tdes_paper_design.cu -- the paper's own GPU design, rebuilt on GB300 as a
// context point for the benchmark (not part of the cipher library).
//
// "Bit-level Parallelization of 3DES Encryption on GPU", Sec. IV:
//   - key generation kernel (Sec. IV-A): one CTA per base key, 56 threads,
//     one per PC-1 bit; the halves are rotated by one thread each, 16 times,
//     and PC-2 is applied bit-parallel after every rotation step;
//   - encryption/decryption kernel (Sec. IV-B): one CTA per 64-bit block,
//     64 threads, one per bit, one char per bit in shared memory; the first
//     48 threads expand and XOR the round key, four threads per S-box
//     (each reads the group's S-box entry and writes one of its bits), 32
//     threads permute and
//     XOR into the left half; launched once per DES pass, three times for
//     3DES, with the key order reversed on the host for decryption;
//   - memory (Sec. IV-C): the permutation, expansion and S-box tables are read
//     through the read-only data cache, the shift table from constant memory,
//     and the data and keys are char-per-bit arrays in global memory.
// Written from that description; it shares nothing with the bitsliced path
// except the DES tables, transcribed for it once more from the appendix.
#include <cuda_runtime.h>

#include <cstdint>

namespace paperdesign {

__device__ const uint8_t kPC1[56] = {57, 49, 41, 33, 25, 17, 9,  1,  58, 50, 42, 34, 26, 18,
                                     10, 2,  59, 51, 43, 35, 27, 19, 11, 3,  60, 52, 44, 36,
                                     63, 55, 47, 39, 31, 23, 15, 7,  62, 54, 46, 38, 30, 22,
                                     14, 6,  61, 53, 45, 37, 29, 21, 13, 5,  28, 20, 12, 4};
__constant__ int kShift[16] = {1, 1, 2, 2, 2, 2, 2, 2, 1, 2, 2, 2, 2, 2, 2, 1};
__device__ const uint8_t kPC2[48] = {14, 17, 11, 24, 1,  5,  3,  28, 15, 6,  21, 10,
                                     23, 19, 12, 4,  26, 8,  16, 7,  27, 20, 13, 2,
                                     41, 52, 31, 37, 47, 55, 30, 40, 51, 45, 33, 48,
                                     44, 49, 39, 56, 34, 53, 46, 42, 50, 36, 29, 32};
__device__ const uint8_t kIP[64] = {58, 50, 42, 34, 26, 18, 10, 2, 60, 52, 44, 36, 28, 20, 12, 4,
                                    62, 54, 46, 38, 30, 22, 14, 6, 64, 56, 48, 40, 32, 24, 16, 8,
                                    57, 49, 41, 33, 25, 17, 9,  1, 59, 51, 43, 35, 27, 19, 11, 3,
                                    61, 53, 45, 37, 29, 21, 13, 5, 63, 55, 47, 39, 31, 23, 15, 7};
__device__ const uint8_t kE[48] = {32, 1,  2,  3,  4,  5,  4,  5,  6,  7,  8,  9,
                                   8,  9,  10, 11, 12, 13, 12, 13, 14, 15, 16, 17,
                                   16, 17, 18, 19, 20, 21, 20, 21, 22, 23, 24, 25,
                                   24, 25, 26, 27, 28, 29, 28, 29, 30, 31, 32, 1};
__device__ const uint8_t kS[8][4][16] = {
    {{14, 4, 13, 1, 2, 15, 11, 8, 3, 10, 6, 12, 5, 9, 0, 7},
     {0, 15, 7, 4, 14, 2, 13, 1, 10, 6, 12, 11, 9, 5, 3, 8},
     {4, 1, 14, 8, 13, 6, 2, 11, 15, 12, 9, 7, 3, 10, 5, 0},
     {15, 12, 8, 2, 4, 9, 1, 7, 5, 11, 3, 14, 10, 0, 6, 13}},
    {{15, 1, 8, 14, 6, 11, 3, 4, 9, 7, 2, 13, 12, 0, 5, 10},
     {3, 13, 4, 7, 15, 2, 8, 14, 12, 0, 1, 10, 6, 9, 11, 5},
     {0, 14, 7, 11, 10, 4, 13, 1, 5, 8, 12, 6, 9, 3, 2, 15},
     {13, 8, 10, 1, 3, 15, 4, 2, 11, 6, 7, 12, 0, 5, 14, 9}},
    {{10, 0, 9, 14, 6, 3, 15, 5, 1, 13, 12, 7, 11, 4, 2, 8},
     {13, 7, 0, 9, 3, 4, 6, 10, 2, 8, 5, 14, 12, 11, 15, 1},
     {13, 6, 4, 9, 8, 15, 3, 0, 11, 1, 2, 12, 5, 10, 14, 7},
     {1, 10, 13, 0, 6, 9, 8, 7, 4, 15, 14, 3, 11, 5, 2, 12}},
    {{7, 13, 14, 3, 0, 6, 9, 10, 1, 2, 8, 5, 11, 12, 4, 15},
     {13, 8, 11, 5, 6, 15, 0, 3, 4, 7, 2, 12, 1, 10, 14, 9},
     {10, 6, 9, 0, 12, 11, 7, 13, 15, 1, 3, 14, 5, 2, 8, 4},
     {3, 15, 0, 6, 10, 1, 13, 8, 9, 4, 5, 11, 12, 7, 2, 14}},
    {{2, 12, 4, 1, 7, 10, 11, 6, 8, 5, 3, 15, 13, 0, 14, 9},
     {14, 11, 2, 12, 4, 7, 13, 1, 5, 0, 15, 10, 3, 9, 8, 6},
     {4, 2, 1, 11, 10, 13, 7, 8, 15, 9, 12, 5, 6, 3, 0, 14},
     {11, 8, 12, 7, 1, 14, 2, 13, 6, 15, 0, 9, 10, 4, 5, 3}},
    {{12, 1, 10, 15, 9, 2, 6, 8, 0, 13, 3, 4, 14, 7, 5, 11},
     {10, 15, 4, 2, 7, 12, 9, 5, 6, 1, 13, 14, 0, 11, 3, 8},
     {9, 14, 15, 5, 2, 8, 12, 3, 7, 0, 4, 10, 1, 13, 11, 6},
     {4, 3, 2, 12, 9, 5, 15, 10, 11, 14, 1, 7, 6, 0, 8, 13}},
    {{4, 11, 2, 14, 15, 0, 8, 13, 3, 12, 9, 7, 5, 10, 6, 1},
     {13, 0, 11, 7, 4, 9, 1, 10, 14, 3, 5, 12, 2, 15, 8, 6},
     {1, 4, 11, 13, 12, 3, 7, 14, 10, 15, 6, 8, 0, 5, 9, 2},
     {6, 11, 13, 8, 1, 4, 10, 7, 9, 5, 0, 15, 14, 2, 3, 12}},
    {{13, 2, 8, 4, 6, 15, 11, 1, 10, 9, 3, 14, 5, 0, 12, 7},
     {1, 15, 13, 8, 10, 3, 7, 4, 12, 5, 6, 11, 0, 14, 9, 2},
     {7, 11, 4, 1, 9, 12, 14, 2, 0, 6, 10, 13, 15, 3, 5, 8},
     {2, 1, 14, 7, 4, 10, 8, 13, 15, 12, 9, 0, 3, 5, 6, 11}}};
__device__ const uint8_t kP[32] = {16, 7, 20, 21, 29, 12, 28, 17, 1,  15, 23, 26, 5,  18, 31, 10,
                                   2,  8, 24, 14, 32, 27, 3,  9,  19, 13, 30, 6,  22, 11, 4,  25};
__device__ const uint8_t kFP[64] = {40, 8, 48, 16, 56, 24, 64, 32, 39, 7, 47, 15, 55, 23, 63, 31,
                                    38, 6, 46, 14, 54, 22, 62, 30, 37, 5, 45, 13, 53, 21, 61, 29,
                                    36, 4, 44, 12, 52, 20, 60, 28, 35, 3, 43, 11, 51, 19, 59, 27,
                                    34, 2, 42, 10, 50, 18, 58, 26, 33, 1, 41, 9,  49, 17, 57, 25};

// keys: 3 x 64 chars (one per key bit); rk: 3 x 16 x 48 chars.
__global__ void keygen_kernel(const uint8_t* __restrict__ keys, uint8_t* __restrict__ rk) {
    __shared__ uint8_t cd[56];
    const int k = blockIdx.x, t = threadIdx.x;  // 56 threads
    cd[t] = __ldg(keys + 64 * k + __ldg(kPC1 + t) - 1);
    __syncthreads();
    for (int r = 0; r < 16; ++r) {
        if (t < 2) {  // two threads: one rotates C, the other D
            uint8_t* h = cd + 28 * t;
            for (int s = 0; s < kShift[r]; ++s) {
                const uint8_t first = h[0];
                for (int i = 0; i < 27; ++i) h[i] = h[i + 1];
                h[27] = first;
            }
        }
        __syncthreads();
        if (t < 48) rk[(k * 16 + r) * 48 + t] = cd[__ldg(kPC2 + t) - 1];
        __syncthreads();
    }
}

// One DES pass on char-per-bit blocks: CTA b handles block b, thread t bit t.
// rk16: the 16 round keys of this pass in the order they are applied.
__global__ void des_pass_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                const uint8_t* __restrict__ rk16) {
    __shared__ uint8_t x[64], lr[64], er[48], sb[32], f[32];
    const int t = threadIdx.x;  // 64 threads
    const uint8_t* blk = in + 64ull * blockIdx.x;
    x[t] = blk[t];
    __syncthreads();
    lr[t] = x[__ldg(kIP + t) - 1];  // IP; lr[0..31] = L, lr[32..63] = R
    __syncthreads();
    for (int r = 0; r < 16; ++r) {
        if (t < 48) er[t] = lr[32 + __ldg(kE + t) - 1] ^ __ldg(rk16 + 48 * r + t);
        __syncthreads();
        if (t < 32) {  // 4 threads per S-box: each reads the value, writes its bit
            const int g = t >> 2, o = t & 3;
            const uint8_t* b = er + 6 * g;
            const int row = 2 * b[0] + b[5];
            const int col = 8 * b[1] + 4 * b[2] + 2 * b[3] + b[4];
            const int v = __ldg(&kS[g][row][col]);
            sb[t] = (uint8_t)((v >> (3 - o)) & 1);
        }
        __syncthreads();
        if (t < 32) f[t] = sb[__ldg(kP + t) - 1];
        __syncthreads();
        uint8_t nr = 0, nl = 0;  // new R = L ^ f, new L = R
        if (t < 32) {
            nr = lr[t] ^ f[t];
            nl = lr[32 + t];
        }
        __syncthreads();
        if (t < 32) {
            lr[t] = nl;
            lr[32 + t] = nr;
        }
        __syncthreads();
    }
    // combine as R16 || L16, then FP
    x[t] = t < 32 ? lr[32 + t] : lr[t - 32];
    __syncthreads();
    out[64ull * blockIdx.x + t] = x[__ldg(kFP + t) - 1];
}

__global__ void unpack_kernel(const uint8_t* __restrict__ bytes, uint8_t* __restrict__ bits,
                              uint64_t nbits) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbits) bits[i] = (bytes[i >> 3] >> (7 - (i & 7))) & 1;
}

__global__ void pack_kernel(const uint8_t* __restrict__ bits, uint8_t* __restrict__ bytes,
                            uint64_t nbytes) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbytes) {
        uint8_t v = 0;
        for (int j = 0; j < 8; ++j) v = (uint8_t)((v << 1) | bits[8 * i + j]);
        bytes[i] = v;
    }
}

}  // namespace paperdesign

extern "C" {

// ECB 3DES of nbytes (multiple of 8) device bytes with the paper's design.
// work: device scratch of at least 16 * nbytes + 8192 bytes (char-per-bit
// buffers and round keys).  If ms_kernels is not NULL it receives the time of
// the three encryption launches (CUDA events), the quantity the paper reports.
// Synchronous.  Returns 0 or a CUDA error code.
int tdes_tools_paper_ecb(const uint8_t keys24[24], int decrypt, const void* in, void* out,
                         uint64_t nbytes, void* work, float* ms_kernels) {
    using namespace paperdesign;
    const uint64_t nblocks = nbytes / 8, nbits = nbytes * 8;
    uint8_t* w = static_cast<uint8_t*>(work);
    uint8_t* bits_a = w;
    uint8_t* bits_b = w + nbits;
    uint8_t* kbits = w + 2 * nbits;      // 192 chars
    uint8_t* rk = kbits + 256;           // 3 x 16 x 48 chars
    uint8_t* rk_pass = rk + 3 * 16 * 48; // 3 passes x 16 x 48, in application order
    uint8_t hk[192];
    for (int i = 0; i < 192; ++i) hk[i] = (keys24[i >> 3] >> (7 - (i & 7))) & 1;
    cudaError_t e = cudaMemcpy(kbits, hk, 192, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;
    keygen_kernel<<<3, 56>>>(kbits, rk);
    // order of round keys per pass (reversal done on the host, Sec. IV-B):
    // encrypt E_K1, D_K2, E_K3; decrypt D_K3, E_K2, D_K1
    uint8_t hrk[3 * 16 * 48], hpass[3 * 16 * 48];
    e = cudaMemcpy(hrk, rk, sizeof hrk, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return (int)e;
    for (int pass = 0; pass < 3; ++pass) {
        const int key = decrypt ? 2 - pass : pass;
        const bool rev = decrypt ? (pass != 1) : (pass == 1);
        for (int r = 0; r < 16; ++r)
            for (int j = 0; j < 48; ++j)
                hpass[(pass * 16 + r) * 48 + j] = hrk[(key * 16 + (rev ? 15 - r : r)) * 48 + j];
    }
    e = cudaMemcpy(rk_pass, hpass, sizeof hpass, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;
    const unsigned ub = (unsigned)((nbits + 255) / 256);
    unpack_kernel<<<ub, 256>>>(static_cast<const uint8_t*>(in), bits_a, nbits);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    des_pass_kernel<<<(unsigned)nblocks, 64>>>(bits_a, bits_b, rk_pass);
    des_pass_kernel<<<(unsigned)nblocks, 64>>>(bits_b, bits_a, rk_pass + 16 * 48);
    des_pass_kernel<<<(unsigned)nblocks, 64>>>(bits_a, bits_b, rk_pass + 2 * 16 * 48);
    cudaEventRecord(e1);
    pack_kernel<<<(unsigned)((nbytes + 255) / 256), 256>>>(bits_b, static_cast<uint8_t*>(out),
                                                           nbytes);
    e = cudaDeviceSynchronize();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_kernels) *ms_kernels = ms;
    if (e == cudaSuccess) e = cudaGetLastError();
    return (int)e;
}
}
