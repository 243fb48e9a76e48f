// tdes_noalloc.cu -- CBC decryption that allocates no device memory.
//
// tdes_cbc_decrypt takes a stream-ordered temporary (cudaMallocAsync) when it
// decrypts in place, to save the ciphertext block that precedes every 8 KiB
// tile before a neighbouring tile overwrites it.  Some callers cannot let a
// library allocate: a server that reserves all of the GPU's memory for its own
// pool at start-up and must never see an allocation fail mid-request, a
// host framework that hands a plugin pre-sized buffers and forbids any
// allocation on its hot path, or code that has to keep a bounded, fixed
// memory footprint.  For them, tdes_cbc_decrypt_noalloc keeps that scratch in
// a fixed array compiled into this library instead.
#include <cuda.h>  // CUcontext and cuCtxGetCurrent's type only: resolved through the runtime
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/tdes.h"
#include "tdes_internal.h"

namespace {

// One saved ciphertext block (8 bytes) per 8 KiB tile, for at most
// TDES_NOALLOC_MAX_TILES tiles, i.e. in-place calls of up to 1 GiB.  Every
// device that loads the library holds these 1 MiB until the process exits.
constexpr uint64_t kMaxTiles = TDES_NOALLOC_MAX_TILES;
static __device__ __align__(256) uint64_t g_halo_scratch[kMaxTiles];

// Device address of g_halo_scratch, looked up once per device and context:
// a new context on a device (after cudaDeviceReset, say) loads the module
// again, possibly elsewhere, so the address is looked up again then.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    CUcontext ctx = nullptr;
    uint64_t* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tdes::set_last_error(buf);
    return status;
}

// The driver's cuCtxGetCurrent, found through the runtime (so that the
// library does not link the driver library itself).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

// With `device` current, return the device address of the scratch array.
// In host code g_halo_scratch names only a host-side shadow of the symbol,
// never the device memory, so the address must come from the runtime.
int scratch_for(int device, uint64_t** out) {
    if (device < 0 || device >= kMaxDevices) return fail(TDES_EINVAL, "device %d out of range", device);
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get == nullptr || get(&ctx) != CUDA_SUCCESS || ctx == nullptr)
        return fail(TDES_ECUDA, "no current CUDA context on device %d", device);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddr& a = g_scratch_addr[device];
    if (a.addr == nullptr || a.ctx != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_halo_scratch);
        if (e != cudaSuccess)
            return fail(TDES_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        a.addr = static_cast<uint64_t*>(p);
        a.ctx = ctx;
    }
    *out = a.addr;
    return TDES_OK;
}

}  // namespace

extern "C" {

int tdes_cbc_decrypt_noalloc(const tdes_ks_t* ks, uint64_t iv, const void* in, void* out,
                             size_t nbytes, tdes_stream_t stream) {
    if (ks == nullptr) return fail(TDES_EINVAL, "key schedule is NULL");
    if (nbytes % 8 != 0) return fail(TDES_EINVAL, "nbytes = %zu is not a multiple of 8", nbytes);
    if (nbytes == 0) return TDES_OK;
    if (in == nullptr || out == nullptr) return fail(TDES_EINVAL, "NULL data pointer");
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
    if ((a | b) & 7u) return fail(TDES_EINVAL, "data pointers must be 8-byte aligned");
    if (a != b && a < b + nbytes && b < a + nbytes)
        return fail(TDES_EINVAL, "input and output overlap without being the same buffer");
    // size limits first: they need no device and touch no memory
    const uint64_t nblocks = nbytes / 8;
    const uint64_t ntiles = (nblocks + tdes::kTileBlocks - 1) / tdes::kTileBlocks;
    if (nblocks / tdes::kTileBlocks >= (1ull << 31))
        return fail(TDES_EINVAL, "a call is limited to 2^31 tiles of 8 KiB (16 TiB)");
    if (in == out && ntiles > kMaxTiles)
        return fail(TDES_EINVAL,
                    "in-place call of %zu bytes exceeds the fixed scratch limit of %llu bytes "
                    "(%llu tiles of 8 KiB)",
                    nbytes, (unsigned long long)(kMaxTiles * 8 * tdes::kTileBlocks),
                    (unsigned long long)kMaxTiles);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TDES_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != ks->device)
        return fail(TDES_EINVAL, "key schedule lives on device %d but device %d is current",
                    ks->device, dev);
    if (!tdes::gpu_addressable(in) || !tdes::gpu_addressable(out))
        return fail(TDES_EINVAL, "buffers must be device memory or pinned, mapped host memory");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* halo = nullptr;
    if (in == out && ntiles > 1) {
        int rc = scratch_for(dev, &halo);
        if (rc != TDES_OK) return rc;
        // Every entry the decryption reads (tiles 1..ntiles-1) is written here
        // first, on the same stream, so nothing needs clearing between calls.
        e = tdes::launch_cbc_halo(in, halo, nblocks, s);
        if (e != cudaSuccess) return fail(TDES_ECUDA, "CBC halo kernel: %s", cudaGetErrorString(e));
    }
    const tdes::Geometry g = tdes::geometry_for(ntiles, tdes::kCbcDec, ks->device);
    const bool vec16 = ((a | b) & 15u) == 0;
    e = tdes::launch_cbc_dec(ks->tab[1], ks->stages, iv, in, out, nblocks, halo, vec16, g, s);
    if (e != cudaSuccess) return fail(TDES_ECUDA, "CBC-decrypt kernel: %s", cudaGetErrorString(e));
    return TDES_OK;
}

}  // extern "C"
