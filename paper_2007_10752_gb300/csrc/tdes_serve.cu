// tdes_serve.cu -- continuous-batching request server over the batch kernel,
// and an open-loop load generator that measures its latency.
//
// Requests (device buffers, one key index and mode each) are queued by
// tdes_server_submit without blocking.  A dispatcher thread owns the GPU
// side.  It admits queued requests in arrival order while the bytes in
// flight (input + output) stay within the HBM budget, and plans every
// admitted group into one persistent batch launch on one of several streams
// ("slots").  Requests that arrive while earlier batches run are dispatched
// into the next free slot at once, so their work overlaps on the device.
// Each batch's grid leaves room on every SM for the next batch.  Key
// schedules stay resident in the key table; the plan of each batch is
// copied from pinned staging owned by its slot.
#include <cuda_runtime.h>

#include <sys/prctl.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tdes.h"
#include "tdes_batch_internal.h"
#include "tdes_internal.h"
#include "tdes_tune.h"

namespace {

int sfail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tdes::set_last_error(buf);
    return status;
}

int scuda(cudaError_t e, const char* what) {
    return sfail(e == cudaErrorMemoryAllocation ? TDES_ENOMEM : TDES_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;   // after the batch's last operation on the stream
    uint64_t seq = 0;             // the batch's number (its entry of the time ring)
    void* dmem = nullptr;
    size_t dcap = 0;
    uint8_t* pinned = nullptr;
    size_t pcap = 0;
    std::vector<uint64_t> tickets;
    uint64_t cost = 0;
    bool busy = false;
    uint8_t* stage = nullptr;  // device staging for requests in host memory
    size_t stage_cap = 0;
};

struct Pending {
    tdes_desc_t d;
    uint64_t ticket;
    uint64_t cost;
    bool stage;  // host buffers, large enough to be staged through the device
    bool alone;  // a long serial chain: batched on its own (see lone_request)
};

// A CBC-encryption request of more than 512 blocks is one serial chain that
// a warp walks at about a microsecond per block.  A batch completes as a
// whole, so requests batched with it would wait for it: it gets a batch of
// its own instead.
constexpr uint64_t kLoneChainBlocks = 512;
bool lone_request(const tdes_desc_t& d) {
    return d.mode == TDES_MODE_CBC_ENCRYPT && d.nbytes / 8 > kLoneChainBlocks;
}

struct StagedCopy {
    void* dst;
    const void* src;
    size_t n;
};

struct Completion {
    std::atomic<uint64_t> ticket{0};  // published last (release)
    int status = 0;
    int64_t t_done_ns = 0;
};

uint64_t cost_of(const tdes_desc_t& d) { return d.in == d.out ? d.nbytes : 2 * d.nbytes; }

// After its last progress (a batch dispatched or completed) the dispatcher
// polls without sleeping for this long before it sleeps or naps.
constexpr int64_t kSpinNs = 200000;

// A batch's time on the device: from its first kernel's first CTA starting
// to its last kernel's last warp finishing, in ns of the GPU's global timer.
struct Interval {
    double t0, t1;
};

// Device timestamps of the last kTimeRing batches: entry seq % kTimeRing
// holds batch seq's [start, end] (written by its kernels, see BatchParams).
constexpr uint64_t kTimeRing = 1u << 20;

// Sweep over intervals: most at once, time with >= 1 and with >= 2.
void sweep(std::vector<Interval> v, uint32_t* max_at_once, double* busy, double* overlap) {
    std::vector<std::pair<double, int>> ev;
    ev.reserve(2 * v.size());
    for (const Interval& iv : v) {
        ev.push_back({iv.t0, +1});
        ev.push_back({iv.t1, -1});
    }
    std::sort(ev.begin(), ev.end());  // at equal times an end (-1) sorts before a start
    int k = 0, mx = 0;
    double b = 0.0, o = 0.0, prev = ev.empty() ? 0.0 : ev[0].first;
    for (const auto& e : ev) {
        if (k >= 1) b += e.first - prev;
        if (k >= 2) o += e.first - prev;
        prev = e.first;
        k += e.second;
        mx = std::max(mx, k);
    }
    *max_at_once = (uint32_t)mx;
    *busy = b;
    *overlap = o;
}

}  // namespace

struct tdes_server {
    int device = 0;
    const tdes_keytable* kt = nullptr;
    tdes_server_config_t cfg{};
    int sms = 0, ctas_fit = 1;
    size_t dyn_smem = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::deque<Pending> queue;
    std::atomic<size_t> queued{0};  // queue.size(), readable without the lock
    uint64_t next_ticket = 1;
    std::vector<Completion> ring;
    std::thread thread;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> batches{0}, completed{0};
    std::atomic<int> sticky_error{0};
    uint64_t admitted = 0;  // dispatcher thread only
    // the dispatcher sleeps on cv_work when it has nothing to do or poll;
    // waiters sleep on cv_done, which the dispatcher signals after completions
    std::condition_variable cv_work;
    std::mutex done_mu;
    std::condition_variable cv_done;
    std::atomic<int> waiters{0};
    // overlap statistics: batches in flight (dispatched, not complete) and
    // the numbers of the batches completed since the last reset, whose device
    // times the kernels wrote into times_ring
    unsigned long long* times_ring = nullptr;
    uint64_t next_seq = 0;  // dispatcher thread only
    std::mutex stats_mu;
    uint32_t busy_now = 0, max_busy = 0;
    std::vector<uint64_t> done_seqs;  // at most 2 kTimeRing: older times are overwritten
    uint64_t failed_batches = 0;      // and batches whose times the ring no longer holds

    // Clears the overlap statistics (cheap: no device read).
    void reset_stats() {
        std::lock_guard<std::mutex> lock(stats_mu);
        done_seqs.clear();
        failed_batches = 0;
        max_busy = busy_now;
    }

    void notify_done() {
        if (waiters.load(std::memory_order_acquire) == 0) return;
        { std::lock_guard<std::mutex> lock(done_mu); }
        cv_done.notify_all();
    }

    bool wants_stage(const tdes_desc_t& d) const {
        return cfg.stage_bytes && d.nbytes >= cfg.stage_min_bytes && d.nbytes <= cfg.stage_bytes &&
               tdes::host_memory(d.in) && tdes::host_memory(d.out);
    }

    void complete(uint64_t ticket, int status, int64_t t) {
        Completion& c = ring[ticket % ring.size()];
        c.status = status;
        c.t_done_ns = t;
        c.ticket.store(ticket, std::memory_order_release);
        completed.fetch_add(1, std::memory_order_relaxed);
    }

    bool ensure_capacity(Slot& sl, size_t n) {
        if (sl.dcap < n) {
            if (sl.dmem) cudaFree(sl.dmem);
            sl.dmem = nullptr;
            sl.dcap = 0;
            const size_t want = std::max(n, (size_t)1 << 20) * 2;
            if (cudaMalloc(&sl.dmem, want) != cudaSuccess) return false;
            sl.dcap = want;
        }
        if (sl.pcap < n) {
            if (sl.pinned) cudaFreeHost(sl.pinned);
            sl.pinned = nullptr;
            sl.pcap = 0;
            const size_t want = std::max(n, (size_t)1 << 20) * 2;
            if (cudaHostAlloc(reinterpret_cast<void**>(&sl.pinned), want, cudaHostAllocDefault) !=
                cudaSuccess)
                return false;
            sl.pcap = want;
        }
        return true;
    }

    void dispatch_loop() {
        cudaSetDevice(device);
        std::vector<Pending> take;
        std::vector<tdes_desc_t> descs;
        std::vector<StagedCopy> copy_in, copy_out;
        tdes::PlanHost plan;
        const uint64_t reserve = cfg.slots > 1 ? (uint64_t)std::max(0, cfg.reserve_ctas_per_sm) : 0;
        const uint64_t per_sm = std::max<uint64_t>(1, (uint64_t)ctas_fit > reserve
                                                          ? (uint64_t)ctas_fit - reserve : 1);
        const uint64_t max_ctas = (uint64_t)sms * per_sm;
        tdes::LaunchShape shape;
        shape.warps = cfg.warps_per_cta;
        shape.round_form = cfg.round_form;
        prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);  // naps below end within a microsecond
        int64_t last_progress = now_ns();
        int64_t nap_ns = 0;
        for (;;) {
            bool worked = false;
            bool any_busy = false;
            bool completed_any = false;
            for (Slot& sl : slots) {
                if (!sl.busy) continue;
                const cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) {
                    any_busy = true;
                    continue;
                }
                const int st = q == cudaSuccess ? TDES_OK : TDES_ECUDA;
                if (st != TDES_OK) sticky_error.store(st);
                const int64_t t = now_ns();
                for (uint64_t tk : sl.tickets) complete(tk, st, t);
                admitted -= sl.cost;
                sl.busy = false;
                worked = true;
                completed_any = true;
                std::lock_guard<std::mutex> lock(stats_mu);
                --busy_now;
                if (st == TDES_OK) {
                    if (done_seqs.size() >= 2 * kTimeRing) {  // bounded on a server never reset
                        done_seqs.erase(done_seqs.begin(), done_seqs.begin() + kTimeRing);
                        failed_batches += kTimeRing;
                    }
                    done_seqs.push_back(sl.seq);
                } else {
                    ++failed_batches;
                }
            }
            if (completed_any) notify_done();
            for (Slot& sl : slots) {
                if (sl.busy) continue;
                take.clear();
                uint64_t cost = 0;
                if (queued.load(std::memory_order_acquire) == 0) break;  // nothing to take
                {
                    std::lock_guard<std::mutex> lock(mu);
                    while (!queue.empty() && take.size() < cfg.max_batch &&
                           admitted + cost + queue.front().cost <= cfg.budget_bytes) {
                        const bool alone = queue.front().alone;
                        if (alone && !take.empty()) break;  // it starts the next batch
                        cost += queue.front().cost;
                        take.push_back(queue.front());
                        queue.pop_front();
                        if (alone) break;
                    }
                    queued.store(queue.size(), std::memory_order_release);
                }
                if (take.empty()) break;
                descs.resize(take.size());
                copy_in.clear();
                copy_out.clear();
                size_t staged = 0;
                for (size_t i = 0; i < take.size(); ++i) {
                    descs[i] = take[i].d;
                    const size_t n = (size_t)take[i].d.nbytes;
                    if (!take[i].stage || staged + n > sl.stage_cap) continue;
                    // processed in place in the slot's staging, copied in and out
                    uint8_t* dev = sl.stage + staged;
                    copy_in.push_back({dev, take[i].d.in, n});
                    copy_out.push_back({take[i].d.out, dev, n});
                    descs[i].in = dev;
                    descs[i].out = dev;
                    staged += (n + 255) & ~(size_t)255;
                }
                tdes::build_plan(descs.data(), (uint32_t)descs.size(), kt->count, nullptr, &plan);
                cudaError_t e = cudaSuccess;
                if (!ensure_capacity(sl, plan.image.size())) e = cudaErrorMemoryAllocation;
                for (const StagedCopy& c : copy_in)
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyHostToDevice, sl.stream);
                if (e == cudaSuccess) {
                    memcpy(sl.pinned, plan.image.data(), plan.image.size());
                    e = cudaMemcpyAsync(sl.dmem, sl.pinned, plan.image.size(),
                                        cudaMemcpyHostToDevice, sl.stream);
                }
                if (e == cudaSuccess) {  // the image just copied holds a zeroed claim counter
                    tdes::BatchParams p = tdes::bind_plan(plan, sl.dmem, kt);
                    sl.seq = next_seq++;
                    p.batch_times = times_ring + 2 * (sl.seq % kTimeRing);
                    e = tdes::enqueue_batch(p, plan.total_items, plan.needs_halo, shape,
                                            dyn_smem, max_ctas, sl.stream, true);
                }
                for (const StagedCopy& c : copy_out)
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyDeviceToHost, sl.stream);
                if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
                if (e != cudaSuccess) {
                    sticky_error.store(TDES_ECUDA);
                    // copies already queued read the slot's pinned image and
                    // staging, which the slot's next batch rewrites
                    cudaStreamSynchronize(sl.stream);
                    cudaGetLastError();
                    const int64_t t = now_ns();
                    for (const Pending& pd : take) complete(pd.ticket, TDES_ECUDA, t);
                    notify_done();
                    continue;
                }
                sl.tickets.clear();
                for (const Pending& pd : take) sl.tickets.push_back(pd.ticket);
                sl.cost = cost;
                sl.busy = true;
                admitted += cost;
                any_busy = true;
                worked = true;
                batches.fetch_add(1, std::memory_order_relaxed);
                std::lock_guard<std::mutex> lock(stats_mu);
                max_busy = std::max(max_busy, ++busy_now);
            }
            // The queue's lock is taken only to take requests (above) and to
            // sleep (below): a dispatcher spinning on the lock slowed the
            // submitting threads that share it.
            if (stop.load(std::memory_order_acquire) && !any_busy &&
                queued.load(std::memory_order_acquire) == 0)
                break;
            const int64_t now = now_ns();
            if (worked) {
                last_progress = now;
                nap_ns = 0;
                continue;
            }
            // For kSpinNs after its last progress the dispatcher only yields
            // between polls: under load a new request or a completion is
            // seldom further away, and waking a sleeping thread would add
            // tens of microseconds to its latency.
            if (now - last_progress < kSpinNs) {
                std::this_thread::yield();
                continue;
            }
            std::unique_lock<std::mutex> lock(mu);
            if (stop.load(std::memory_order_acquire) && !any_busy && queue.empty()) break;
            if (!any_busy) {
                // idle: the queue is empty (anything queued fits the empty
                // budget), so sleep until a submission or the stop
                cv_work.wait(lock, [&] {
                    return !queue.empty() || stop.load(std::memory_order_acquire);
                });
                last_progress = now_ns();
                nap_ns = 0;
                continue;
            }
            // long batches in flight: poll their events in naps of 5 us
            // doubling up to 100 us; a submission ends a nap at once
            nap_ns = nap_ns ? std::min<int64_t>(2 * nap_ns, 100000) : 5000;
            const size_t waiting = queue.size();
            cv_work.wait_for(lock, std::chrono::nanoseconds(nap_ns), [&] {
                return queue.size() != waiting || stop.load(std::memory_order_acquire);
            });
        }
    }
};

namespace {

// Sleeps on the server's completion signal until poll() stops returning 1
// or the deadline passes (each sleep at most 1 ms, so a missed signal costs
// no more than that).
template <class Poll>
int wait_until_done(tdes_server_t* s, uint64_t timeout_ns, Poll poll) {
    const int64_t until = now_ns() + (int64_t)std::min<uint64_t>(timeout_ns, INT64_MAX / 4);
    int r = poll();
    if (r != 1) return r;
    s->waiters.fetch_add(1, std::memory_order_acq_rel);
    {
        std::unique_lock<std::mutex> lock(s->done_mu);
        for (;;) {
            r = poll();
            if (r != 1) break;
            const int64_t now = now_ns();
            if (now >= until) break;
            s->cv_done.wait_for(lock, std::chrono::nanoseconds(std::min<int64_t>(until - now,
                                                                                  1000000)));
        }
    }
    s->waiters.fetch_sub(1, std::memory_order_acq_rel);
    return r;
}

}  // namespace

extern "C" {

void tdes_server_config_default(tdes_server_config_t* cfg) {
    if (cfg == nullptr) return;
    cfg->budget_bytes = 8ull << 30;
    cfg->slots = 4;
    cfg->max_batch = 16384;
    cfg->warps_per_cta = 4;
    cfg->reserve_ctas_per_sm = 1;
    cfg->ring_entries = 1u << 21;
    cfg->stage_bytes = 0;  // host payloads zero-copy by default: measured faster
    cfg->stage_min_bytes = 64ull << 10;
    cfg->round_form = TDES_ROUNDS_PER_PASS;
    // the autotuner's choice for this GPU, if the cache has one
    int dev = -1, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    tdes::TunedShape t;
    if (tdes::tune_lookup(tdes::serve_tune_key(sms), &t) && t.shape.warps >= 1 &&
        t.shape.warps <= 8 && t.slots >= 1 && t.slots <= 64 && t.shape.ctas_per_sm >= 0) {
        cfg->warps_per_cta = t.shape.warps;
        cfg->reserve_ctas_per_sm = t.shape.ctas_per_sm;
        cfg->slots = (uint32_t)t.slots;
        if (t.shape.round_form == 0 || t.shape.round_form == 1) cfg->round_form = t.shape.round_form;
    }
}

int tdes_server_create(const tdes_keytable_t* kt, const tdes_server_config_t* cfg_in,
                       tdes_server_t** out) {
    if (kt == nullptr || out == nullptr) return sfail(TDES_EINVAL, "NULL argument");
    *out = nullptr;
    tdes_server_config_t cfg;
    tdes_server_config_default(&cfg);
    if (cfg_in) cfg = *cfg_in;
    if (cfg.slots < 1 || cfg.slots > 64 || cfg.max_batch < 1 || cfg.warps_per_cta < 1 ||
        cfg.warps_per_cta > 8 || cfg.ring_entries < 1024 || cfg.budget_bytes < 16 ||
        cfg.round_form < 0 || cfg.round_form > 1)
        return sfail(TDES_EINVAL, "bad server configuration");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return scuda(e, "cudaGetDevice");
    if (dev != kt->device) return sfail(TDES_EINVAL, "key table lives on another device");
    tdes_server* s = new (std::nothrow) tdes_server();
    if (s == nullptr) return sfail(TDES_ENOMEM, "host allocation failed");
    s->device = dev;
    s->kt = kt;
    s->cfg = cfg;
    s->ring = std::vector<Completion>(cfg.ring_entries);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    e = tdes::prepare_batch_kernel(cfg.warps_per_cta, &s->dyn_smem, &s->ctas_fit);
    s->slots.resize(cfg.slots);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&s->times_ring), 2 * kTimeRing * sizeof(uint64_t));
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess && cfg.stage_bytes) {
            e = cudaMalloc(reinterpret_cast<void**>(&sl.stage), cfg.stage_bytes);
            if (e == cudaSuccess) sl.stage_cap = cfg.stage_bytes;
        }
    }
    if (e != cudaSuccess) {
        int rc = scuda(e, "server set-up");
        tdes_server_destroy(s);
        return rc;
    }
    s->thread = std::thread([s] { s->dispatch_loop(); });
    *out = s;
    return TDES_OK;
}

int tdes_server_submit(tdes_server_t* s, const tdes_desc_t* req, uint64_t* ticket) {
    if (s == nullptr || req == nullptr || ticket == nullptr)
        return sfail(TDES_EINVAL, "NULL argument");
    if (tdes::validate_desc(*req, s->kt->count) != TDES_OK)
        return sfail(TDES_EINVAL, "invalid request descriptor");
    if (req->nbytes && (!tdes::gpu_addressable(req->in) || !tdes::gpu_addressable(req->out)))
        return sfail(TDES_EINVAL, "request buffers must be device memory or pinned host memory");
    const uint64_t cost = cost_of(*req);
    if (cost > s->cfg.budget_bytes)
        return sfail(TDES_EINVAL, "request of %llu bytes exceeds the admission budget",
                     (unsigned long long)req->nbytes);
    if (s->sticky_error.load()) return sfail(s->sticky_error.load(), "server stopped by an error");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const uint64_t t = s->next_ticket++;
        *ticket = t;
        if (req->nbytes == 0) {
            s->complete(t, TDES_OK, now_ns());
        } else {
            s->queue.push_back({*req, t, cost, s->wants_stage(*req), lone_request(*req)});
            s->queued.store(s->queue.size(), std::memory_order_release);
            s->cv_work.notify_one();
            return TDES_OK;
        }
    }
    s->notify_done();
    return TDES_OK;
}

int tdes_server_poll(tdes_server_t* s, uint64_t ticket) {
    if (s == nullptr || ticket == 0) return sfail(TDES_EINVAL, "bad ticket");
    const Completion& c = s->ring[ticket % s->ring.size()];
    const uint64_t seen = c.ticket.load(std::memory_order_acquire);
    if (seen == ticket) return c.status;
    if (seen > ticket) return TDES_OK;  // completed long ago; its record was reused
    return 1;
}

int tdes_server_wait(tdes_server_t* s, uint64_t ticket, uint64_t timeout_ns) {
    if (s == nullptr || ticket == 0) return sfail(TDES_EINVAL, "bad ticket");
    const int r = wait_until_done(s, timeout_ns, [&] { return tdes_server_poll(s, ticket); });
    if (r == 1)
        return sfail(TDES_ETIMEDOUT, "ticket %llu still pending", (unsigned long long)ticket);
    return r;
}

int tdes_server_submit_group(tdes_server_t* s, const tdes_desc_t* reqs, uint32_t count,
                             uint64_t* ticket) {
    if (s == nullptr || ticket == nullptr || (reqs == nullptr && count > 0) || count == 0)
        return sfail(TDES_EINVAL, "NULL argument or empty group");
    for (uint32_t i = 0; i < count; ++i) {  // the whole group is refused before any is queued
        const tdes_desc_t& r = reqs[i];
        if (tdes::validate_desc(r, s->kt->count) != TDES_OK)
            return sfail(TDES_EINVAL, "invalid request descriptor %u of the group", i);
        if (r.nbytes && (!tdes::gpu_addressable(r.in) || !tdes::gpu_addressable(r.out)))
            return sfail(TDES_EINVAL, "request %u: buffers must be device or pinned host memory", i);
        if (cost_of(r) > s->cfg.budget_bytes)
            return sfail(TDES_EINVAL, "request %u exceeds the admission budget", i);
    }
    if (s->sticky_error.load()) return sfail(s->sticky_error.load(), "server stopped by an error");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        const uint64_t t0 = s->next_ticket;
        s->next_ticket += count;
        *ticket = t0;
        for (uint32_t i = 0; i < count; ++i) {
            if (reqs[i].nbytes == 0)
                s->complete(t0 + i, TDES_OK, now_ns());
            else
                s->queue.push_back({reqs[i], t0 + i, cost_of(reqs[i]), s->wants_stage(reqs[i]),
                                    lone_request(reqs[i])});
        }
        s->queued.store(s->queue.size(), std::memory_order_release);
        s->cv_work.notify_one();
    }
    s->notify_done();
    return TDES_OK;
}

int tdes_server_poll_group(tdes_server_t* s, uint64_t ticket, uint32_t count,
                           int* per_desc_status) {
    if (s == nullptr || ticket == 0 || count == 0) return sfail(TDES_EINVAL, "bad group");
    int err = TDES_OK;
    bool pending = false;
    for (uint32_t i = 0; i < count; ++i) {
        const int r = tdes_server_poll(s, ticket + i);
        if (per_desc_status) per_desc_status[i] = r;
        if (r == 1) pending = true;
        else if (r < 0 && err == TDES_OK) err = r;
    }
    return err != TDES_OK ? err : (pending ? 1 : TDES_OK);
}

int tdes_server_wait_group(tdes_server_t* s, uint64_t ticket, uint32_t count,
                           uint64_t timeout_ns) {
    if (s == nullptr || ticket == 0 || count == 0) return sfail(TDES_EINVAL, "bad group");
    const int r = wait_until_done(
        s, timeout_ns, [&] { return tdes_server_poll_group(s, ticket, count, nullptr); });
    if (r == 1)
        return sfail(TDES_ETIMEDOUT, "group %llu still pending", (unsigned long long)ticket);
    return r;
}

int tdes_server_stats(tdes_server_t* s, int reset, tdes_server_stats_t* out) {
    if (s == nullptr || out == nullptr) return sfail(TDES_EINVAL, "NULL argument");
    std::vector<uint64_t> seqs;
    {
        std::lock_guard<std::mutex> lock(s->stats_mu);
        seqs.swap(s->done_seqs);
        out->max_slots_busy = s->max_busy;
        out->untimed_batches = s->failed_batches;
        if (reset) {
            s->failed_batches = 0;
            s->max_busy = s->busy_now;
        } else {
            s->done_seqs = seqs;
        }
    }
    // only the last kTimeRing batches still have their times
    if (seqs.size() > kTimeRing) {
        out->untimed_batches += seqs.size() - kTimeRing;
        seqs.erase(seqs.begin(), seqs.end() - kTimeRing);
    }
    // read back only the ring entries that hold these batches
    std::vector<unsigned long long> ring;
    if (!seqs.empty()) {
        ring.assign(2 * kTimeRing, 0ull);
        const auto mm = std::minmax_element(seqs.begin(), seqs.end());
        const uint64_t lo = *mm.first, hi = *mm.second;
        auto fetch = [&](uint64_t a, uint64_t b) {  // ring entries [a, b]
            return cudaMemcpy(ring.data() + 2 * a, s->times_ring + 2 * a, (b - a + 1) * 16,
                              cudaMemcpyDeviceToHost);
        };
        cudaError_t e;
        if (hi - lo + 1 >= kTimeRing) e = fetch(0, kTimeRing - 1);
        else if (lo % kTimeRing <= hi % kTimeRing) e = fetch(lo % kTimeRing, hi % kTimeRing);
        else {
            e = fetch(lo % kTimeRing, kTimeRing - 1);
            if (e == cudaSuccess) e = fetch(0, hi % kTimeRing);
        }
        if (e != cudaSuccess) return scuda(e, "reading batch times");
    }
    std::vector<Interval> iv;
    iv.reserve(seqs.size());
    for (uint64_t q : seqs) {
        const unsigned long long t0 = ring[2 * (q % kTimeRing)], t1 = ring[2 * (q % kTimeRing) + 1];
        iv.push_back({(double)t0 * 1e-6, (double)std::max(t0, t1) * 1e-6});  // ms
    }
    out->batches = iv.size();
    double sum = 0.0;
    for (const Interval& x : iv) sum += x.t1 - x.t0;
    out->batch_ms_sum = sum;
    sweep(std::move(iv), &out->max_device_overlap, &out->device_busy_ms, &out->device_overlap_ms);
    return TDES_OK;
}

void tdes_server_destroy(tdes_server_t* s) {
    if (s == nullptr) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop.store(true, std::memory_order_release);
        s->cv_work.notify_all();
    }
    if (s->thread.joinable()) s->thread.join();
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.dmem) cudaFree(sl.dmem);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.stage) cudaFree(sl.stage);
    }
    if (s->times_ring) cudaFree(s->times_ring);
    delete s;
}

// --------------------------------------------------------------- load test

static uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Rng {
    uint64_t state;
    uint64_t next() { return mix64(state += 0x9E3779B97F4A7C15ull); }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

static double percentile(std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
}

int tdes_serve_loadtest(tdes_server_t* s, const tdes_loadtest_config_t* c,
                        tdes_loadtest_result_t* res) {
    if (s == nullptr || c == nullptr || res == nullptr) return sfail(TDES_EINVAL, "NULL argument");
    if (c->n_requests == 0 || c->n_keys == 0 || c->n_keys > s->kt->count ||
        c->small_min < 8 || c->small_max < c->small_min || c->large_min < 8 ||
        c->large_max < c->large_min || c->in_pool == nullptr || c->out_pool == nullptr ||
        c->in_pool_bytes < c->large_max || c->out_pool_bytes < 2 * c->large_max)
        return sfail(TDES_EINVAL, "bad load-test configuration");
    const uint64_t n = c->n_requests;
    Rng rng{c->seed};
    std::vector<tdes_desc_t> reqs(n);
    std::vector<uint8_t> small(n);
    double total = 0.0;
    const double lmin = std::log((double)c->large_min), lmax = std::log((double)c->large_max);
    double psum = c->mode_probs[0] + c->mode_probs[1] + c->mode_probs[2];
    if (!(psum > 0)) psum = 1.0;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t nb;
        small[i] = rng.uniform() < c->small_frac;
        if (small[i])
            nb = c->small_min + (rng.next() % (c->small_max - c->small_min + 1));
        else
            nb = (uint64_t)std::exp(lmin + rng.uniform() * (lmax - lmin));
        nb = std::max<uint64_t>(8, nb / 8 * 8);
        const double u = rng.uniform() * psum;
        const uint32_t mode = u < c->mode_probs[0] ? TDES_MODE_ECB_ENCRYPT
                              : u < c->mode_probs[0] + c->mode_probs[1] ? TDES_MODE_CTR
                                                                        : TDES_MODE_CBC_DECRYPT;
        const uint64_t in_off = (rng.next() % (c->in_pool_bytes - nb + 1)) / 16 * 16;
        tdes_desc_t& d = reqs[i];
        d.mode = mode;
        d.key_index = (uint32_t)(rng.next() % c->n_keys);
        d.iv_or_ctr = mode == TDES_MODE_CTR ? (rng.next() & 0xFFFFFFFF00000000ull) : rng.next();
        d.in = static_cast<const uint8_t*>(c->in_pool) + in_off;
        d.out = nullptr;
        d.nbytes = nb;
        total += (double)nb;
    }
    // arrival times: Poisson at the offered byte rate, or all at once
    std::vector<int64_t> arrive(n, 0);
    const double rate = c->offered_gbps > 0 ? c->offered_gbps * 1e9 / (total / (double)n) : 0.0;
    double t = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        if (rate > 0) t += -std::log(1.0 - rng.uniform()) / rate;
        arrive[i] = (int64_t)(t * 1e9);
    }
    // output regions: a ring over out_pool; a region is reused only after the
    // request that held it has completed (waiting counts toward latency)
    struct Held {
        uint64_t ticket, lo, hi;
    };
    std::deque<Held> held;
    uint64_t head = 0;
    std::vector<uint64_t> tickets(n);
    s->reset_stats();  // overlap statistics of this run only (before the schedule starts)
    const int64_t t0 = now_ns() + 1000000;
    const uint64_t batches0 = s->batches.load();
    for (uint64_t i = 0; i < n; ++i) {
        tdes_desc_t& d = reqs[i];
        if (head + d.nbytes > c->out_pool_bytes) head = 0;
        const uint64_t lo = head, hi = head + d.nbytes;
        head = (hi + 15) / 16 * 16;
        for (;;) {
            // Regions are handed out in ring order, so a new one can only lap
            // the oldest held regions: check those at the front.
            while (!held.empty() && tdes_server_poll(s, held.front().ticket) != 1) held.pop_front();
            bool overlap = false;
            const size_t scan = std::min<size_t>(held.size(), 64);
            for (size_t k = 0; k < scan && !overlap; ++k)
                overlap = held[k].lo < hi && lo < held[k].hi &&
                          tdes_server_poll(s, held[k].ticket) == 1;
            if (!overlap) break;
            std::this_thread::yield();
        }
        d.out = static_cast<uint8_t*>(c->out_pool) + lo;
        // the scheduled arrival: sleep while it is far ahead, then spin to it
        for (int64_t ahead = t0 + arrive[i] - now_ns(); ahead > 0; ahead = t0 + arrive[i] - now_ns()) {
            if (ahead > 200000)
                std::this_thread::sleep_for(std::chrono::nanoseconds(ahead - 100000));
            else
                std::this_thread::yield();
        }
        const int rc = tdes_server_submit(s, &d, &tickets[i]);
        if (rc != TDES_OK) return rc;
        held.push_back({tickets[i], lo, hi});
    }
    for (uint64_t i = 0; i < n; ++i) {
        const int rc = tdes_server_wait(s, tickets[i], 120ull * 1000000000ull);
        if (rc != TDES_OK) return rc;
    }
    std::vector<double> lat(n), lat_s, lat_l;
    int64_t last = t0;
    for (uint64_t i = 0; i < n; ++i) {
        const Completion& cp = s->ring[tickets[i] % s->ring.size()];
        if (cp.ticket.load(std::memory_order_acquire) != tickets[i])
            return sfail(TDES_EINVAL, "completion ring too small for %llu requests",
                         (unsigned long long)n);
        lat[i] = (double)(cp.t_done_ns - (t0 + arrive[i])) * 1e-6;
        last = std::max(last, cp.t_done_ns);
        (small[i] ? lat_s : lat_l).push_back(lat[i]);
    }
    double sum = 0.0, mx = 0.0;
    for (double v : lat) {
        sum += v;
        mx = std::max(mx, v);
    }
    res->requests = n;
    res->bytes = (uint64_t)total;
    res->duration_s = (double)(last - t0) * 1e-9;
    res->gbps = total / std::max(1e-9, (double)(last - t0)) ;
    res->offered_gbps = c->offered_gbps;
    res->batches = s->batches.load() - batches0;
    res->mean_ms = sum / (double)n;
    res->max_ms = mx;
    res->p50_ms = percentile(lat, 0.50);
    res->p90_ms = percentile(lat, 0.90);
    res->p99_ms = percentile(lat, 0.99);
    res->p999_ms = percentile(lat, 0.999);
    res->small_p50_ms = percentile(lat_s, 0.50);
    res->small_p99_ms = percentile(lat_s, 0.99);
    res->large_p50_ms = percentile(lat_l, 0.50);
    res->large_p99_ms = percentile(lat_l, 0.99);
    tdes_server_stats_t st;
    tdes_server_stats(s, 0, &st);
    res->max_slots_busy = st.max_slots_busy;
    res->max_device_overlap = st.max_device_overlap;
    res->device_overlap_frac = st.device_busy_ms > 0 ? st.device_overlap_ms / st.device_busy_ms : 0.0;
    return TDES_OK;
}

}  // extern "C"

// ------------------------------------------------------------- autotuning

namespace {

// One candidate's figures: the median closed-loop GB/s of `runs` load tests
// of a fresh server in cfg (after a warm-up of a tenth of the requests) and,
// when load_gbps > 0, the median p99 latency of `runs` open-loop tests at
// that offered load.
struct ServeScore {
    double gbps = 0.0, p99_ms = 0.0;
};

constexpr double kServeTuneMargin = 0.03;

int serve_score(const tdes_keytable_t* kt, const tdes_server_config_t& cfg,
                const tdes_loadtest_config_t& load, int runs, double load_gbps, ServeScore* out) {
    tdes_server_t* s = nullptr;
    int rc = tdes_server_create(kt, &cfg, &s);
    if (rc != TDES_OK) return rc;
    tdes_loadtest_config_t c = load;
    tdes_loadtest_result_t r;
    c.offered_gbps = 0.0;
    c.n_requests = std::max<uint64_t>(1, load.n_requests / 10);
    rc = tdes_serve_loadtest(s, &c, &r);
    std::vector<double> g, l;
    c.n_requests = load.n_requests;
    for (int i = 0; i < runs && rc == TDES_OK; ++i) {
        c.seed = load.seed + 1 + (uint64_t)i;
        c.offered_gbps = 0.0;
        rc = tdes_serve_loadtest(s, &c, &r);
        g.push_back(r.gbps);
        if (rc == TDES_OK && load_gbps > 0) {
            c.offered_gbps = load_gbps;
            rc = tdes_serve_loadtest(s, &c, &r);
            l.push_back(r.p99_ms);
        }
    }
    tdes_server_destroy(s);
    if (rc != TDES_OK) return rc;
    std::sort(g.begin(), g.end());
    out->gbps = g[g.size() / 2];
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        out->p99_ms = l[l.size() / 2];
    }
    return TDES_OK;
}

bool same_shape(const tdes_server_config_t& a, const tdes_server_config_t& b) {
    return a.warps_per_cta == b.warps_per_cta && a.reserve_ctas_per_sm == b.reserve_ctas_per_sm &&
           a.slots == b.slots && a.round_form == b.round_form;
}

}  // namespace

extern "C" {

int tdes_server_autotune(const tdes_keytable_t* kt, const tdes_loadtest_config_t* load,
                         unsigned flags, tdes_server_autotune_result_t* res) {
    if (kt == nullptr || load == nullptr || res == nullptr) return sfail(TDES_EINVAL, "NULL argument");
    memset(res, 0, sizeof *res);
    int dev = -1, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return scuda(e, "device query");
    const std::string key = tdes::serve_tune_key(sms);
    snprintf(res->key, sizeof res->key, "%s", key.c_str());
    // the built-in defaults, not a cached choice
    tdes_server_config_t base;
    tdes_server_config_default(&base);
    base.warps_per_cta = 4;
    base.reserve_ctas_per_sm = 1;
    base.slots = 4;
    base.round_form = TDES_ROUNDS_PER_PASS;
    res->baseline = base;
    tdes::TunedShape cached;
    if (!(flags & TDES_TUNE_FORCE) && tdes::tune_lookup(key, &cached)) {
        tdes_server_config_default(&res->best);
        res->best_gbps = cached.gbps;
        res->baseline_gbps = cached.baseline_gbps;
        res->from_cache = 1;
        return TDES_OK;
    }
    // The score of a shape is its p99 latency at 95% of the default shape's
    // closed-loop throughput (the same offered load for every candidate),
    // among the shapes that keep at least 97% of that throughput closed-loop;
    // a serving system is judged by its tail latency under load, and the
    // shape with the highest closed-loop throughput is not the one with the
    // lowest tail (2 warps per CTA won on throughput and showed p99 1.78 ms
    // at 95% of its own peak).  At 90% the shapes' tails lay within tens of
    // percent of each other and the default could win on noise, while at
    // 95% of its own peak it showed p99 2.17 ms against 0.67-1.10 ms for 8
    // slots.
    const int runs = 3;
    ServeScore sb;
    int rc = serve_score(kt, base, *load, runs, 0.0, &sb);
    if (rc != TDES_OK) return rc;
    const double load_gbps = 0.95 * sb.gbps, floor_gbps = 0.97 * sb.gbps;
    rc = serve_score(kt, base, *load, runs, load_gbps, &sb);
    if (rc != TDES_OK) return rc;
    tdes_server_config_t best = base;
    ServeScore bs = sb;
    uint32_t timed = 1;
    // x replaces y only if its p99 is lower by more than kServeTuneMargin:
    // shapes within run-to-run spread of each other (a few percent of p99)
    // would otherwise decide by noise, and two calls could pick different
    // shapes of the same quality.
    auto better = [&](const ServeScore& x, const ServeScore& y) {  // x better than y
        if ((x.gbps >= floor_gbps) != (y.gbps >= floor_gbps)) return x.gbps >= floor_gbps;
        return x.p99_ms < (1.0 - kServeTuneMargin) * y.p99_ms;
    };
    auto consider = [&](tdes_server_config_t t) -> int {
        if (same_shape(t, best)) return TDES_OK;
        ServeScore x;
        const int r = serve_score(kt, t, *load, runs, load_gbps, &x);
        if (r != TDES_OK) return r;
        ++timed;
        if (better(x, bs)) {
            best = t;
            bs = x;
        }
        return TDES_OK;
    };
    for (int w : {2, 4, 8}) {
        tdes_server_config_t t = best;
        t.warps_per_cta = w;
        if ((rc = consider(t)) != TDES_OK) return rc;
    }
    // At least one CTA per SM stays free for the next batch: with none, a
    // batch's kernels wait for the previous batch's CTAs to leave, which
    // raised closed-loop throughput a little but p50 latency at 25% load
    // by a fifth (8 warps, 8 slots: 57 against 47 us).
    for (int r : {1, 2}) {
        tdes_server_config_t t = best;
        t.reserve_ctas_per_sm = r;
        if ((rc = consider(t)) != TDES_OK) return rc;
    }
    for (uint32_t k : {2u, 4u, 8u}) {
        tdes_server_config_t t = best;
        t.slots = k;
        if ((rc = consider(t)) != TDES_OK) return rc;
    }
    {
        tdes_server_config_t t = best;
        t.round_form = 1 - best.round_form;
        if ((rc = consider(t)) != TDES_OK) return rc;
    }
    // the winner against the default once more, alternating, so that drift
    // over the search does not decide
    if (!same_shape(best, base)) {
        std::vector<ServeScore> vb, vt;
        for (int i = 0; i < 3; ++i) {
            ServeScore x;
            if ((rc = serve_score(kt, base, *load, 1, load_gbps, &x)) != TDES_OK) return rc;
            vb.push_back(x);
            if ((rc = serve_score(kt, best, *load, 1, load_gbps, &x)) != TDES_OK) return rc;
            vt.push_back(x);
        }
        auto med = [](std::vector<ServeScore> v) {
            ServeScore m;
            std::vector<double> g, l;
            for (const ServeScore& x : v) {
                g.push_back(x.gbps);
                l.push_back(x.p99_ms);
            }
            std::sort(g.begin(), g.end());
            std::sort(l.begin(), l.end());
            m.gbps = g[1];
            m.p99_ms = l[1];
            return m;
        };
        sb = med(vb);
        bs = med(vt);
        if (!better(bs, sb)) {
            best = base;
            bs = sb;
        }
    } else {
        // the default won, possibly on a later measurement of its own shape
        // (a coordinate step can come back to it): report one figure for it
        sb = bs;
    }
    res->best = best;
    res->best_gbps = bs.gbps;
    res->baseline_gbps = sb.gbps;
    res->best_p99_ms = bs.p99_ms;
    res->baseline_p99_ms = sb.p99_ms;
    res->load_gbps = load_gbps;
    res->candidates = timed;
    if (!(flags & TDES_TUNE_NO_STORE)) {
        tdes::TunedShape t;
        t.shape.warps = best.warps_per_cta;
        t.shape.ctas_per_sm = best.reserve_ctas_per_sm;
        t.shape.round_form = best.round_form;
        t.slots = (int)best.slots;
        t.gbps = bs.gbps;
        t.baseline_gbps = sb.gbps;
        rc = tdes::tune_store(key, t);
        if (rc != TDES_OK) return rc;
    }
    return TDES_OK;
}

}  // extern "C"
