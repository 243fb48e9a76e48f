// tdes_tools.cu -- benchmark and test tools, not part of the cipher library:
//   * a probe of the sustained throughput of 32-bit LOP3 instructions, the
//     peak the bitsliced kernels are bound by;
//   * a device-side fill with the same counter-based SplitMix64 words as the
//     host input generator (paper_2007_10752_gb300/synth.py), for inputs too
//     large to generate on the host and copy;
//   * (tdes_paper_design.cu) the paper's own one-thread-per-bit kernels, as a
//     context point for the benchmark.
//
// LOP3 probe:
// Each thread keeps 8 accumulators and updates each with a 3-input LOP3 of
// three different accumulators, so no two instructions can be merged and
// there are 8 independent chains per thread.  Launched over every SM with
// enough warps to hide the LOP3 latency.
#include <cuda_runtime.h>

#include <cstdint>

template <int LUT>
__device__ __forceinline__ uint32_t lop3p(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

__global__ void lop3_rate_kernel(uint32_t* out, int iters, uint32_t seed) {
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 7u * i + 1u) + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = lop3p<0x96>(a[i], a[(i + 1) & 7], a[(i + 3) & 7]);
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = lop3p<0xe8>(a[i], a[(i + 2) & 7], a[(i + 5) & 7]);
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x12345678u) out[blockIdx.x * blockDim.x + threadIdx.x] = x;  // keeps the work live
}

// Word i of a SplitMix64 stream seeded s is mix(s + (i + 1) * gamma)
// (Steele, Lea and Flood, OOPSLA 2014), stored little-endian.
__global__ void splitmix64_fill_kernel(uint64_t* __restrict__ out, uint64_t nwords, uint64_t seed,
                                       uint64_t first) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += stride) {
        uint64_t z = seed + (first + i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        out[i] = z ^ (z >> 31);
    }
}

extern "C" {

// Fills dst (8-byte aligned, nwords words) with words first .. first+nwords-1
// of the SplitMix64 stream seeded `seed`, on `stream`.  Returns 0 or a CUDA error.
int tdes_tools_fill_splitmix64(void* dst, uint64_t nwords, uint64_t seed, uint64_t first,
                               void* stream) {
    if (nwords == 0) return 0;
    if (dst == nullptr || (reinterpret_cast<uintptr_t>(dst) & 7u)) return -1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (nwords + 255) / 256;
    const unsigned grid = (unsigned)(want < (uint64_t)sms * 16 ? want : (uint64_t)sms * 16);
    splitmix64_fill_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<uint64_t*>(dst), nwords, seed, first);
    return (int)cudaGetLastError();
}

// Runs the probe on the current device and stream 0; returns 0 and the
// measured LOP3 lane-operations per second in *ops_per_s, or a CUDA error.
int tdes_tools_lop3_rate(int ctas_per_sm, int threads, int iters, double* ops_per_s,
                         float* ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int grid = sms * ctas_per_sm;
    uint32_t* out = nullptr;
    if (cudaMalloc(&out, sizeof(uint32_t) * grid * threads) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    lop3_rate_kernel<<<grid, threads>>>(out, 4, 1u);  // warm-up
    cudaEventRecord(e0);
    lop3_rate_kernel<<<grid, threads>>>(out, iters, 3u);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double ops = (double)grid * threads * (double)iters * 64.0;
    *ops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return 0;
}
}
