// tdes_ctx.cu -- batch contexts: submit a batch of messages, get a ticket,
// poll it per descriptor, wait on it with a time limit.
//
// The paper states the problem as plaintext of 64-bit blocks, three keys and
// a mode (Sec. IV-B, IV-C).  A batch is many such problems at once, each
// message with its own key triple and mode.  tdes_batch_submit plans the
// descriptors on the host (the same plan as tdes_batch_plan), copies the plan
// into stream-ordered device memory and queues the batch kernels on one of
// the context's streams, followed by a completion event; the plan memory is
// returned to the pool on the same stream once the kernels are done.  The
// call does not wait for the device, so a caller can keep several batches in
// flight and collect them in any order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tdes.h"
#include "tdes_batch_internal.h"
#include "tdes_internal.h"
#include "tdes_tune.h"

namespace {

int cfail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tdes::set_last_error(buf);
    return status;
}

int ccuda(cudaError_t e, const char* what) {
    return cfail(e == cudaErrorMemoryAllocation ? TDES_ENOMEM : TDES_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Record {
    cudaEvent_t done = nullptr;  // nullptr: nothing was queued (no valid work)
    int stream = -1;
    std::vector<int> status;     // per descriptor: TDES_OK or the reason it was rejected
    int first_error = TDES_OK;   // first rejected descriptor's status
    bool complete = false;
    int result = 1;              // once complete: TDES_OK, first_error or TDES_ECUDA
    // The plan's host image, the source of its copy to the device.  It is
    // pageable memory, which the copy may read when it runs on the stream (a
    // GPU that addresses host memory directly, as on Grace, is not bound to
    // stage it before cudaMemcpyAsync returns), so it lives until the batch
    // is complete.
    std::vector<uint8_t> image;
};

}  // namespace

struct tdes_ctx {
    int device = 0;
    const tdes_keytable* kt = nullptr;
    int sms = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> last;       // last completion event queued on each stream
    std::vector<cudaEvent_t> free_events;
    std::mutex mu;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, Record> records;
    // Last ticket of each plan submitted with tdes_batch_submit_plan: two
    // launches of one plan share its claim counter and halo, so a plan whose
    // previous ticket is still pending is queued behind it on its stream.
    std::unordered_map<const tdes_batch*, uint64_t> plan_last;
    int fit[9] = {0};                    // CTAs per SM of the batch kernel, by warps per CTA
    size_t dyn[9] = {0};

    // A stream with nothing in flight, else the one whose last batch was
    // queued longest ago (round robin).  Caller holds mu.
    int pick_stream() {
        for (size_t i = 0; i < streams.size(); ++i) {
            const size_t k = (rr + i) % streams.size();
            if (last[k] == nullptr || cudaEventQuery(last[k]) == cudaSuccess) {
                rr = k + 1;
                return (int)k;
            }
        }
        cudaGetLastError();
        const int k = (int)(rr % streams.size());
        rr = k + 1;
        return k;
    }
    cudaEvent_t take_event() {  // caller holds mu
        if (!free_events.empty()) {
            cudaEvent_t e = free_events.back();
            free_events.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        return e;
    }
    // Completion check of one record (caller holds mu).
    void settle(Record& r) {
        if (r.complete) return;
        if (r.done == nullptr) {
            r.complete = true;
            r.result = r.first_error;
            return;
        }
        const cudaError_t q = cudaEventQuery(r.done);
        if (q == cudaErrorNotReady) return;
        r.complete = true;
        std::vector<uint8_t>().swap(r.image);
        r.result = q == cudaSuccess ? r.first_error : TDES_ECUDA;
        if (q != cudaSuccess) {
            cudaGetLastError();
            cfail(TDES_ECUDA, "batch failed on the device: %s", cudaGetErrorString(q));
        }
    }

  private:
    size_t rr = 0;
};

namespace {

// Queues plan h on the context (the caller has checked the device).
int queue_plan(tdes_ctx* c, tdes::PlanHost& h, std::vector<int>&& status, uint64_t* ticket) {
    Record r;
    r.status = std::move(status);
    for (int st : r.status)
        if (st != TDES_OK) {
            r.first_error = st;
            break;
        }
    for (tdes::DirectMsg& m : h.direct) m.stages = c->kt->host_stages[m.key];
    const bool work = h.total_items != 0 || !h.direct.empty();
    tdes::LaunchShape shape;  // the default shape
    tdes::TunedShape tuned;
    if (work && tdes::tune_lookup(tdes::tune_key(h, c->sms), &tuned) && tuned.shape.warps >= 1 &&
        tuned.shape.warps <= 8 && tuned.shape.tiles_per_claim >= 0 &&
        tuned.shape.round_form >= 0 && tuned.shape.round_form <= 1)
        shape = tuned.shape;
    std::lock_guard<std::mutex> lock(c->mu);
    if (work) {
        const int w = shape.warps;
        if (c->fit[w] == 0) {
            cudaError_t e = tdes::prepare_batch_kernel(w, &c->dyn[w], &c->fit[w]);
            if (e != cudaSuccess) return ccuda(e, "batch kernel set-up");
        }
        shape.ctas_per_sm = shape.ctas_per_sm < 1 ? c->fit[w] : std::min(shape.ctas_per_sm, c->fit[w]);
        const int k = c->pick_stream();
        cudaStream_t s = c->streams[k];
        cudaEvent_t done = c->take_event();
        if (done == nullptr) return cfail(TDES_ECUDA, "cudaEventCreate failed");
        void* mem = nullptr;
        cudaError_t e = cudaSuccess;
        if (h.total_items) {
            e = cudaMallocAsync(&mem, h.image.size(), s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(mem, h.image.data(), h.image.size(), cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = tdes::enqueue_direct(h.direct, c->kt, c->device, s);
        if (e == cudaSuccess && h.total_items) {
            const tdes::BatchParams p = tdes::bind_plan(h, mem, c->kt);
            e = tdes::enqueue_batch(p, h.total_items, h.needs_halo, shape, c->dyn[w],
                                    (uint64_t)c->sms * shape.ctas_per_sm, s, true);
        }
        if (mem) {
            const cudaError_t e2 = cudaFreeAsync(mem, s);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaEventRecord(done, s);
        if (e != cudaSuccess) {
            c->free_events.push_back(done);
            const int rc = ccuda(e, "batch submission");
            cudaStreamSynchronize(s);  // whatever was queued has read the image before it goes
            cudaGetLastError();
            return rc;
        }
        r.done = done;
        r.stream = k;
        r.image = std::move(h.image);
        c->last[k] = done;
    }
    const uint64_t t = c->next_ticket++;
    c->records.emplace(t, std::move(r));
    *ticket = t;
    return TDES_OK;
}

int check_ctx(tdes_ctx* c) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ccuda(e, "cudaGetDevice");
    if (dev != c->device)
        return cfail(TDES_EINVAL, "context lives on device %d but device %d is current", c->device,
                     dev);
    return TDES_OK;
}

}  // namespace

extern "C" {

void tdes_ctx_config_default(tdes_ctx_config_t* cfg) {
    if (cfg == nullptr) return;
    cfg->streams = 2;
}

int tdes_ctx_create(const tdes_keytable_t* kt, const tdes_ctx_config_t* cfg_in, tdes_ctx_t** out) {
    if (kt == nullptr || out == nullptr) return cfail(TDES_EINVAL, "NULL argument");
    *out = nullptr;
    tdes_ctx_config_t cfg;
    tdes_ctx_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.streams < 1 || cfg.streams > 16) return cfail(TDES_EINVAL, "streams must be 1..16");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ccuda(e, "cudaGetDevice");
    if (dev != kt->device) return cfail(TDES_EINVAL, "key table lives on another device");
    tdes_ctx* c = new (std::nothrow) tdes_ctx();
    if (c == nullptr) return cfail(TDES_ENOMEM, "host allocation failed");
    c->device = dev;
    c->kt = kt;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    c->streams.assign(cfg.streams, nullptr);
    c->last.assign(cfg.streams, nullptr);
    for (cudaStream_t& s : c->streams)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) tdes::geometry_for(1, tdes::kEcb, dev);  // single-key kernel set-up
    if (e != cudaSuccess) {
        const int rc = ccuda(e, "context set-up");
        tdes_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return TDES_OK;
}

void tdes_ctx_destroy(tdes_ctx_t* c) {
    if (c == nullptr) return;
    for (cudaStream_t s : c->streams)
        if (s) cudaStreamSynchronize(s);
    for (auto& kv : c->records)
        if (kv.second.done) cudaEventDestroy(kv.second.done);
    for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
    for (cudaStream_t s : c->streams)
        if (s) cudaStreamDestroy(s);
    delete c;
}

int tdes_batch_submit(tdes_ctx_t* c, const tdes_desc_t* descs, uint32_t count, uint64_t* ticket) {
    if (c == nullptr || ticket == nullptr || (descs == nullptr && count > 0))
        return cfail(TDES_EINVAL, "NULL argument to tdes_batch_submit");
    int rc = check_ctx(c);
    if (rc != TDES_OK) return rc;
    std::vector<int> status(count, TDES_OK);
    tdes::PlanHost h;
    tdes::build_plan(descs, count, c->kt->count, status.data(), &h, true);
    return queue_plan(c, h, std::move(status), ticket);
}

int tdes_batch_submit_plan(tdes_ctx_t* c, tdes_batch_t* b, uint64_t* ticket) {
    if (c == nullptr || b == nullptr || ticket == nullptr)
        return cfail(TDES_EINVAL, "NULL argument to tdes_batch_submit_plan");
    int rc = check_ctx(c);
    if (rc != TDES_OK) return rc;
    if (b->kt != c->kt) return cfail(TDES_EINVAL, "the plan uses another key table");
    Record r;
    r.status = b->status;
    for (int st : r.status)
        if (st != TDES_OK) {
            r.first_error = st;
            break;
        }
    std::lock_guard<std::mutex> lock(c->mu);
    if (b->total_items || !b->direct.empty()) {
        int k = -1;
        const auto pl = c->plan_last.find(b);
        if (pl != c->plan_last.end()) {
            const auto prev = c->records.find(pl->second);  // pending tickets are never released
            if (prev != c->records.end()) {
                c->settle(prev->second);
                if (!prev->second.complete) k = prev->second.stream;
            }
        }
        if (k < 0) k = c->pick_stream();
        cudaStream_t s = c->streams[k];
        rc = tdes_batch_launch_graph(b, s);
        if (rc != TDES_OK) return rc;
        cudaEvent_t done = c->take_event();
        if (done == nullptr) return cfail(TDES_ECUDA, "cudaEventCreate failed");
        const cudaError_t e = cudaEventRecord(done, s);
        if (e != cudaSuccess) {
            c->free_events.push_back(done);
            return ccuda(e, "cudaEventRecord");
        }
        r.done = done;
        r.stream = k;
        c->last[k] = done;
    }
    const uint64_t t = c->next_ticket++;
    c->records.emplace(t, std::move(r));
    c->plan_last[b] = t;
    *ticket = t;
    return TDES_OK;
}

int tdes_batch_poll(tdes_ctx_t* c, uint64_t ticket, int* per_desc_status) {
    if (c == nullptr || ticket == 0) return cfail(TDES_EINVAL, "bad ticket");
    std::lock_guard<std::mutex> lock(c->mu);
    if (ticket >= c->next_ticket) return 1;  // not issued yet: pending
    auto it = c->records.find(ticket);
    if (it == c->records.end())
        return cfail(TDES_EINVAL, "ticket %llu was released", (unsigned long long)ticket);
    Record& r = it->second;
    c->settle(r);
    if (per_desc_status)
        for (size_t i = 0; i < r.status.size(); ++i)
            per_desc_status[i] = r.status[i] != TDES_OK ? r.status[i]
                                 : !r.complete          ? 1
                                 : r.result == TDES_ECUDA ? TDES_ECUDA
                                                          : TDES_OK;
    return r.complete ? r.result : 1;
}

int tdes_batch_wait(tdes_ctx_t* c, uint64_t ticket, uint64_t timeout_ns) {
    const int64_t start = now_ns();
    const int64_t until = start + (int64_t)std::min<uint64_t>(timeout_ns, INT64_MAX / 4);
    int64_t nap_ns = 2000;
    for (;;) {
        const int r = tdes_batch_poll(c, ticket, nullptr);
        if (r != 1) return r;
        const int64_t now = now_ns();
        if (now >= until)
            return cfail(TDES_ETIMEDOUT, "ticket %llu still pending", (unsigned long long)ticket);
        // short naps first (a batch of small messages completes in tens of
        // microseconds), then longer ones: the thread does not spin
        std::this_thread::sleep_for(
            std::chrono::nanoseconds(std::min<int64_t>(nap_ns, until - now)));
        nap_ns = std::min<int64_t>(nap_ns * 2, 1000000);
    }
}

int tdes_batch_release(tdes_ctx_t* c, uint64_t ticket) {
    if (c == nullptr || ticket == 0) return cfail(TDES_EINVAL, "bad ticket");
    std::lock_guard<std::mutex> lock(c->mu);
    auto it = c->records.find(ticket);
    if (it == c->records.end())
        return cfail(TDES_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    c->settle(it->second);
    if (!it->second.complete) return cfail(TDES_EBUSY, "ticket %llu still pending",
                                           (unsigned long long)ticket);
    if (cudaEvent_t done = it->second.done) {
        for (cudaEvent_t& l : c->last)
            if (l == done) l = nullptr;
        c->free_events.push_back(done);
    }
    c->records.erase(it);
    return TDES_OK;
}

}  // extern "C"
