// tdes_api.cu -- the C ABI of include/tdes.h: argument checks, device-memory
// ownership of key schedules, launch geometry, and the host-buffer pipeline.
// All cipher arithmetic runs in the kernels of tdes_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/tdes.h"
#include "tdes_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? TDES_ENOMEM : TDES_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

constexpr int kMaxDevices = 64;
struct DeviceInfo {
    bool ready = false;
    int sms = 0;
    int ctas_per_sm[tdes::kNumKernels] = {1, 1, 1};
};
DeviceInfo g_devices[kMaxDevices];
std::mutex g_dev_mutex;

const DeviceInfo* device_info(int device) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    DeviceInfo& d = g_devices[device];
    if (!d.ready) {
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
            return nullptr;
        for (int k = 0; k < tdes::kNumKernels; ++k) d.ctas_per_sm[k] = tdes::wide_ctas_per_sm(k);
        d.ready = true;
    }
    return &d;
}

// Checks shared by every data call; sets *nblocks.
int check_call(const tdes_ks_t* ks, const void* in, const void* out, size_t nbytes,
               uint64_t* nblocks) {
    if (ks == nullptr) return fail(TDES_EINVAL, "key schedule is NULL");
    if (nbytes % 8 != 0) return fail(TDES_EINVAL, "nbytes = %zu is not a multiple of 8", nbytes);
    *nblocks = nbytes / 8;
    if (nbytes == 0) return TDES_OK;
    if (*nblocks / tdes::kTileBlocks >= (1ull << 31))
        return fail(TDES_EINVAL, "a call is limited to 2^31 tiles of 8 KiB (16 TiB)");
    if (in == nullptr || out == nullptr) return fail(TDES_EINVAL, "NULL data pointer");
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
    if ((a | b) & 7u) return fail(TDES_EINVAL, "data pointers must be 8-byte aligned");
    if (a != b && a < b + nbytes && b < a + nbytes)
        return fail(TDES_EINVAL, "input and output overlap without being the same buffer");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != ks->device)
        return fail(TDES_EINVAL, "key schedule lives on device %d but device %d is current",
                    ks->device, dev);
    if (!tdes::gpu_addressable(in) || !tdes::gpu_addressable(out))
        return fail(TDES_EINVAL, "buffers must be device memory or pinned, mapped host memory");
    return TDES_OK;
}

bool aligned16(const void* in, const void* out) {
    return ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
}

// Calls of at most this many blocks run one block per thread (tdes_small.cu).
std::atomic<uint64_t> g_small_cutoff{TDES_SMALL_CUTOFF_DEFAULT};
constexpr int kSmallThreads = 128;  // per CTA: spreads a small call over many SMs

}  // namespace

namespace tdes {

void set_last_error(const char* msg) { g_last_error = msg; }

bool host_memory(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool gpu_addressable(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of the query
        return false;
    }
    switch (a.type) {
        case cudaMemoryTypeDevice:
        case cudaMemoryTypeManaged:
            return true;
        case cudaMemoryTypeHost:
            return a.devicePointer == p;
        default:
            return false;
    }
}

// Small inputs: one warp per CTA so the few tiles spread over many SMs.
// Large inputs: kWideWarps warps per CTA, a grid of every resident CTA,
// each warp striding over tiles.
Geometry geometry_for(uint64_t ntiles, int kernel_id, int device) {
    const DeviceInfo* d = device_info(device);
    const int sms = d ? d->sms : 1;
    const int per_sm = d ? d->ctas_per_sm[kernel_id] : 1;
    if (ntiles <= (uint64_t)sms * kWideWarps) return {(int)(ntiles ? ntiles : 1), 32};
    const uint64_t need = (ntiles + kWideWarps - 1) / kWideWarps;
    const uint64_t full = (uint64_t)sms * per_sm;
    return {(int)(need < full ? need : full), 32 * kWideWarps};
}

}  // namespace tdes

namespace {

// Equal in the 56 bits PC-1 selects (the low bit of each byte is parity).
bool same_des_key(const uint8_t* a, const uint8_t* b) {
    for (int i = 0; i < 8; ++i)
        if ((a[i] ^ b[i]) & 0xFEu) return false;
    return true;
}

// Builds the device tables for `keys` with `stages` DES passes.  A
// single-DES schedule is given (K, K, K): its one-pass tables read the
// first key, and its scalar round-key groups are EDE3's under (K, K, K),
// whose first 16 rounds are DES_K's in both directions.
int make_schedule(tdes::Keys24& keys, int stages, tdes_ks_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const size_t tab_bytes = sizeof(uint32_t) * tdes::kTableWords;
    const size_t total = 2 * tab_bytes + 2 * tdes::kChunkBytes;
    void* mem = nullptr;
    e = cudaMalloc(&mem, total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(key schedule)");
    tdes_ks_t* ks = new (std::nothrow) tdes_ks_t;
    if (ks == nullptr) {
        cudaFree(mem);
        return fail(TDES_ENOMEM, "host allocation failed");
    }
    ks->device = dev;
    ks->stages = stages;
    ks->mem = mem;
    ks->tab[0] = static_cast<uint32_t*>(mem);
    ks->tab[1] = ks->tab[0] + tdes::kTableWords;
    ks->chunk[0] = reinterpret_cast<uint8_t*>(ks->tab[1] + tdes::kTableWords);
    ks->chunk[1] = ks->chunk[0] + tdes::kChunkBytes;
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = tdes::launch_keysched(keys, stages, ks->tab[0], ks->tab[1], ks->chunk[0],
                                  ks->chunk[1], s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(s);
    }
    memset(&keys, 0, sizeof keys);
    if (e != cudaSuccess) {
        cudaFree(mem);
        delete ks;
        return cuda_fail(e, "key-schedule kernel");
    }
    *out = ks;
    return TDES_OK;
}

}  // namespace

extern "C" {

int tdes_key_schedule(const uint8_t k1[8], const uint8_t k2[8], const uint8_t k3[8],
                      tdes_ks_t** out) {
    if (out == nullptr || k1 == nullptr || k2 == nullptr || k3 == nullptr)
        return fail(TDES_EINVAL, "NULL argument to tdes_key_schedule");
    *out = nullptr;
    // E_K3(D_K2(E_K1(x))) is E_K3(x) when K1 = K2 and E_K1(x) when K2 = K3.
    const uint8_t* single = same_des_key(k1, k2) ? k3 : same_des_key(k2, k3) ? k1 : nullptr;
    tdes::Keys24 keys;
    const uint8_t* parts[3] = {k1, k2, k3};
    for (int i = 0; i < 3; ++i) memcpy(keys.b + 8 * i, single ? single : parts[i], 8);
    return make_schedule(keys, single ? 1 : 3, out);
}

int tdes_key_schedule_2key(const uint8_t k1[8], const uint8_t k2[8], tdes_ks_t** out) {
    return tdes_key_schedule(k1, k2, k1, out);
}

int tdes_des_key_schedule(const uint8_t k[8], tdes_ks_t** out) {
    if (out == nullptr || k == nullptr) return fail(TDES_EINVAL, "NULL argument to tdes_des_key_schedule");
    *out = nullptr;
    tdes::Keys24 keys;
    for (int i = 0; i < 3; ++i) memcpy(keys.b + 8 * i, k, 8);
    return make_schedule(keys, 1, out);
}

int tdes_key_schedule_stages(const tdes_ks_t* ks) {
    if (ks == nullptr) return fail(TDES_EINVAL, "key schedule is NULL");
    return ks->stages;
}

void tdes_key_free(tdes_ks_t* ks) {
    if (ks == nullptr) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != ks->device) cudaSetDevice(ks->device);
    cudaFree(ks->mem);
    if (cur >= 0 && cur != ks->device) cudaSetDevice(cur);
    delete ks;
}

static int ecb(const tdes_ks_t* ks, int dir, const void* in, void* out, size_t nbytes,
               tdes_stream_t stream) {
    uint64_t nblocks = 0;
    int rc = check_call(ks, in, out, nbytes, &nblocks);
    if (rc != TDES_OK || nblocks == 0) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (nblocks <= g_small_cutoff.load(std::memory_order_relaxed)) {
        e = tdes::launch_small(ks->chunk[dir], ks->stages, tdes::kSmallEcb, 0, in, out, nblocks,
                               kSmallThreads, s);
    } else {
        const uint64_t ntiles = (nblocks + tdes::kTileBlocks - 1) / tdes::kTileBlocks;
        const tdes::Geometry g = tdes::geometry_for(ntiles, tdes::kEcb, ks->device);
        e = tdes::launch_ecb(ks->tab[dir], ks->stages, in, out, nblocks, aligned16(in, out), g, s);
    }
    return e == cudaSuccess ? TDES_OK : cuda_fail(e, "ECB kernel launch");
}

int tdes_ecb_encrypt(const tdes_ks_t* ks, const void* in, void* out, size_t nbytes,
                     tdes_stream_t stream) {
    return ecb(ks, 0, in, out, nbytes, stream);
}

int tdes_ecb_decrypt(const tdes_ks_t* ks, const void* in, void* out, size_t nbytes,
                     tdes_stream_t stream) {
    return ecb(ks, 1, in, out, nbytes, stream);
}

int tdes_ctr_crypt(const tdes_ks_t* ks, uint32_t nonce, uint32_t ctr0, const void* in, void* out,
                   size_t nbytes, tdes_stream_t stream) {
    uint64_t nblocks = 0;
    int rc = check_call(ks, in, out, nbytes, &nblocks);
    if (rc != TDES_OK || nblocks == 0) return rc;
    if ((uint64_t)ctr0 + nblocks > (1ull << 32))
        return fail(TDES_EINVAL, "CTR counter would wrap: ctr0 %u + %llu blocks > 2^32", ctr0,
                    (unsigned long long)nblocks);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (nblocks <= g_small_cutoff.load(std::memory_order_relaxed)) {
        e = tdes::launch_small(ks->chunk[0], ks->stages, tdes::kSmallCtr,
                               (uint64_t)nonce << 32 | ctr0, in, out, nblocks, kSmallThreads, s);
    } else {
        const uint64_t ntiles = (nblocks + tdes::kTileBlocks - 1) / tdes::kTileBlocks;
        const tdes::Geometry g = tdes::geometry_for(ntiles, tdes::kCtr, ks->device);
        e = tdes::launch_ctr(ks->tab[0], ks->stages, nonce, ctr0, in, out, nblocks,
                             aligned16(in, out), g, s);
    }
    return e == cudaSuccess ? TDES_OK : cuda_fail(e, "CTR kernel launch");
}

int tdes_cbc_decrypt(const tdes_ks_t* ks, uint64_t iv, const void* in, void* out, size_t nbytes,
                     tdes_stream_t stream) {
    uint64_t nblocks = 0;
    int rc = check_call(ks, in, out, nbytes, &nblocks);
    if (rc != TDES_OK || nblocks == 0) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // one block per thread; in place only as a single CTA (all reads before writes)
    if (nblocks <= g_small_cutoff.load(std::memory_order_relaxed) && (in != out || nblocks <= 1024)) {
        const int threads = in != out ? kSmallThreads : (int)((nblocks + 31) / 32 * 32);
        cudaError_t e = tdes::launch_small(ks->chunk[1], ks->stages, tdes::kSmallCbcDec, iv, in,
                                           out, nblocks, threads, s);
        return e == cudaSuccess ? TDES_OK : cuda_fail(e, "CBC-decrypt kernel launch");
    }
    const uint64_t ntiles = (nblocks + tdes::kTileBlocks - 1) / tdes::kTileBlocks;
    uint64_t* halo = nullptr;
    cudaError_t e = cudaSuccess;
    if (in == out && ntiles > 1) {
        e = cudaMallocAsync(reinterpret_cast<void**>(&halo), ntiles * sizeof(uint64_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(CBC halo)");
        e = tdes::launch_cbc_halo(in, halo, nblocks, s);
    }
    if (e == cudaSuccess) {
        const tdes::Geometry g = tdes::geometry_for(ntiles, tdes::kCbcDec, ks->device);
        e = tdes::launch_cbc_dec(ks->tab[1], ks->stages, iv, in, out, nblocks, halo,
                                 aligned16(in, out), g, s);
    }
    if (halo != nullptr) {
        cudaError_t e2 = cudaFreeAsync(halo, s);
        if (e == cudaSuccess) e = e2;
    }
    return e == cudaSuccess ? TDES_OK : cuda_fail(e, "CBC-decrypt kernel launch");
}

int tdes_cbc_encrypt(const tdes_ks_t* ks, uint64_t iv, const void* in, void* out, size_t nbytes,
                     tdes_stream_t stream) {
    uint64_t nblocks = 0;
    int rc = check_call(ks, in, out, nbytes, &nblocks);
    if (rc != TDES_OK || nblocks == 0) return rc;
    cudaError_t e = tdes::launch_cbc_enc(ks->chunk[0], ks->stages, iv, in, out, nblocks,
                                         reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TDES_OK : cuda_fail(e, "CBC-encrypt kernel launch");
}

// Host-buffer ECB.  The device buffer is split into 4..16 equal parts (about
// 32 MiB each) used round-robin; chunk k goes host->device on the copy-in
// stream, through the kernel on the compute stream, and device->host on the
// copy-out stream, with events ordering the three.  A part is refilled only
// after its previous chunk has been copied out, so every part's chunk is in
// flight at once and the two copy directions and the kernel overlap; small
// parts keep the pipeline's fill and drain short.
constexpr int kHostBufs = 16;

int tdes_ecb_crypt_host(const tdes_ks_t* ks, int decrypt, const void* host_in, void* host_out,
                        size_t nbytes, void* dev_buf, size_t dev_bytes) {
    if (ks == nullptr) return fail(TDES_EINVAL, "key schedule is NULL");
    if (nbytes % 8 != 0) return fail(TDES_EINVAL, "nbytes = %zu is not a multiple of 8", nbytes);
    if (nbytes == 0) return TDES_OK;
    if (host_in == nullptr || host_out == nullptr || dev_buf == nullptr)
        return fail(TDES_EINVAL, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(dev_buf) & 15u)
        return fail(TDES_EINVAL, "device buffer must be 16-byte aligned");
    const int nparts = (int)std::max<size_t>(4, std::min<size_t>(kHostBufs, dev_bytes >> 25));
    const size_t part = (dev_bytes / nparts) & ~(size_t)(8 * tdes::kTileBlocks - 1);
    if (part < 32 * 1024) return fail(TDES_EINVAL, "device buffer smaller than 4 x 32 KiB");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != ks->device) return fail(TDES_EINVAL, "key schedule lives on another device");

    cudaStream_t sin = nullptr, scomp = nullptr, sout = nullptr;
    cudaEvent_t ev_in[kHostBufs] = {}, ev_k[kHostBufs] = {}, ev_out[kHostBufs] = {};
    e = cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&scomp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking);
    for (int i = 0; i < kHostBufs && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_k[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[i], cudaEventDisableTiming);
    }
    const char* what = "stream/event setup";
    const uint8_t* src = static_cast<const uint8_t*>(host_in);
    uint8_t* dst = static_cast<uint8_t*>(host_out);
    bool used[kHostBufs] = {};
    for (size_t off = 0, k = 0; e == cudaSuccess && off < nbytes; off += part, ++k) {
        const int b = (int)(k % nparts);
        uint8_t* buf = static_cast<uint8_t*>(dev_buf) + (size_t)b * part;
        const size_t n = (nbytes - off < part) ? nbytes - off : part;
        const uint64_t nblocks = n / 8;
        const uint64_t ntiles = (nblocks + tdes::kTileBlocks - 1) / tdes::kTileBlocks;
        what = "host-to-device copy";
        if (used[b]) e = cudaStreamWaitEvent(sin, ev_out[b], 0);  // part drained
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf, src + off, n, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[b], sin);
        what = "ECB kernel";
        if (e == cudaSuccess) e = cudaStreamWaitEvent(scomp, ev_in[b], 0);
        if (e == cudaSuccess) {
            const tdes::Geometry g = tdes::geometry_for(ntiles, tdes::kEcb, ks->device);
            e = tdes::launch_ecb(ks->tab[decrypt ? 1 : 0], ks->stages, buf, buf, nblocks, true,
                                 g, scomp);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_k[b], scomp);
        what = "device-to-host copy";
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ev_k[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst + off, buf, n, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[b], sout);
        used[b] = true;
    }
    cudaError_t es = sout ? cudaStreamSynchronize(sout) : cudaSuccess;
    if (sin) cudaStreamSynchronize(sin);
    if (scomp) cudaStreamSynchronize(scomp);
    if (e == cudaSuccess && es != cudaSuccess) {
        e = es;
        what = "synchronise";
    }
    for (int i = 0; i < kHostBufs; ++i) {
        if (ev_in[i]) cudaEventDestroy(ev_in[i]);
        if (ev_k[i]) cudaEventDestroy(ev_k[i]);
        if (ev_out[i]) cudaEventDestroy(ev_out[i]);
    }
    if (sin) cudaStreamDestroy(sin);
    if (scomp) cudaStreamDestroy(scomp);
    if (sout) cudaStreamDestroy(sout);
    return e == cudaSuccess ? TDES_OK : cuda_fail(e, what);
}

int tdes_sbox_gate_count(void) { return tdes::sbox_gate_count(); }

uint64_t tdes_set_small_cutoff(uint64_t nblocks) {
    return g_small_cutoff.exchange(nblocks, std::memory_order_relaxed);
}

const char* tdes_strerror(int status) {
    switch (status) {
        case TDES_OK: return "ok";
        case TDES_EINVAL: return "invalid argument";
        case TDES_ENOMEM: return "out of device memory";
        case TDES_EBUSY: return "busy";
        case TDES_ETIMEDOUT: return "timed out";
        case TDES_ECUDA: return "CUDA error";
        default: return "unknown status";
    }
}

const char* tdes_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
