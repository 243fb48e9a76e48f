// tdes_tune.cu -- the launch-shape autotuner of the batch kernels and its
// persistent cache (see tdes_tune.h for the file format).
//
// A launch shape changes only how work is spread over the GPU: warps per CTA
// and CTAs per SM (the persistent grid), tiles per claim (how many 1024-block
// tiles a warp takes from the work counter at once) and the form of the
// round loop (one loop body per DES pass, or one body for all three).  The
// tuner times candidate shapes on the caller's own plan with CUDA events and
// keeps the fastest per workload class.
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tdes.h"
#include "tdes_batch_internal.h"
#include "tdes_internal.h"
#include "tdes_tune.h"

namespace {

int tfail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tdes::set_last_error(buf);
    return status;
}

struct Cache {
    std::mutex mu;
    std::string path;       // file the entries were read from
    long long size = -1;    // its size and modification time then
    long long mtime = -1;
    std::map<std::string, tdes::TunedShape> entries;
};
Cache g_cache;

// Value of the numeric field "name" in one JSON line, or `dflt`.
double field(const char* line, const char* name, double dflt) {
    char pat[64];
    snprintf(pat, sizeof pat, "\"%s\":", name);
    const char* p = strstr(line, pat);
    if (p == nullptr) return dflt;
    p += strlen(pat);
    char* end = nullptr;
    const double v = strtod(p, &end);
    return end == p ? dflt : v;
}

bool key_of(const char* line, std::string* key) {
    const char* p = strstr(line, "\"key\":");
    if (p == nullptr) return false;
    p = strchr(p + 6, '"');
    if (p == nullptr) return false;
    const char* q = strchr(p + 1, '"');
    if (q == nullptr || q - p - 1 <= 0 || q - p - 1 > 120) return false;
    key->assign(p + 1, q - p - 1);
    return true;
}

// Re-reads the file if its path, size or modification time changed.  Caller
// holds g_cache.mu.
void refresh(const std::string& path) {
    struct stat st;
    const bool exists = stat(path.c_str(), &st) == 0;
    const long long size = exists ? (long long)st.st_size : -1;
    const long long mtime = exists ? (long long)st.st_mtime : -1;
    if (path == g_cache.path && size == g_cache.size && mtime == g_cache.mtime) return;
    g_cache.path = path;
    g_cache.size = size;
    g_cache.mtime = mtime;
    g_cache.entries.clear();
    if (!exists) return;
    FILE* f = fopen(path.c_str(), "r");
    if (f == nullptr) return;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        std::string key;
        if (!key_of(line, &key)) continue;
        tdes::TunedShape t;
        t.shape.warps = (int)field(line, "warps_per_cta", 8);
        t.shape.ctas_per_sm = (int)field(line, "ctas_per_sm", 0);
        t.shape.tiles_per_claim = (int)field(line, "tiles_per_claim", 0);
        t.shape.round_form = (int)field(line, "round_form", 0);
        t.slots = (int)field(line, "slots", 0);
        t.ms = field(line, "ms", 0.0);
        t.baseline_ms = field(line, "baseline_ms", 0.0);
        t.gbps = field(line, "gbps", 0.0);
        t.baseline_gbps = field(line, "baseline_gbps", 0.0);
        g_cache.entries[key] = t;
    }
    fclose(f);
}

int grade(uint64_t part, uint64_t total) {
    if (part == 0 || total == 0) return 0;
    const double q = (double)part / (double)total;
    return q <= 1.0 / 3 ? 1 : q <= 2.0 / 3 ? 2 : 3;
}

void mkdirs_for(const std::string& path) {
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);  // existing ones fail harmlessly
}

// Median device time per launch of plan b in its current shape: one
// warm-up launch, then `reps` launches each between two events.
cudaError_t time_shape(tdes_batch* b, int reps, cudaStream_t s, double* ms) {
    std::vector<cudaEvent_t> ev(2 * reps, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e == cudaSuccess) e = tdes::enqueue_planned(b, s);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ev[2 * i], s);
        if (e == cudaSuccess) e = tdes::enqueue_planned(b, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * i + 1], s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::vector<double> t;
    for (int i = 0; i < reps && e == cudaSuccess; ++i) {
        float x = 0.f;
        e = cudaEventElapsedTime(&x, ev[2 * i], ev[2 * i + 1]);
        t.push_back(x);
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return e;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return cudaSuccess;
}

tdes_launch_shape_t to_c(const tdes::LaunchShape& s) {
    tdes_launch_shape_t c;
    c.warps_per_cta = s.warps;
    c.ctas_per_sm = s.ctas_per_sm;
    c.tiles_per_claim = s.tiles_per_claim;
    c.round_form = s.round_form;
    return c;
}

bool same(const tdes::LaunchShape& a, const tdes::LaunchShape& b) {
    return a.warps == b.warps && a.ctas_per_sm == b.ctas_per_sm &&
           a.tiles_per_claim == b.tiles_per_claim && a.round_form == b.round_form;
}

}  // namespace

namespace tdes {

std::string tune_cache_path() {
    const char* env = getenv("TDES_AUTOTUNE_CACHE");
    if (env && *env) return env;
    const char* xdg = getenv("XDG_CACHE_HOME");
    if (xdg && *xdg) return std::string(xdg) + "/tdes_gb300/autotune.jsonl";
    const char* home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/tdes_gb300/autotune.jsonl";
}

std::string tune_key(const PlanHost& h, int sms) {
    const uint64_t total = h.kind_bytes[0] + h.kind_bytes[1] + h.kind_bytes[2] + h.kind_bytes[3];
    int e = 0;
    while (e < 63 && (2ull << e) <= total) ++e;
    char buf[64];
    snprintf(buf, sizeof buf, "sm%d/t%dm%ds%dc%d/2^%d", sms, grade(h.kind_bytes[0], total),
             grade(h.kind_bytes[1], total), grade(h.kind_bytes[2], total),
             grade(h.kind_bytes[3], total), total ? e : 0);
    return buf;
}

std::string serve_tune_key(int sms) {
    char buf[32];
    snprintf(buf, sizeof buf, "serve/sm%d", sms);
    return buf;
}

bool tune_lookup(const std::string& key, TunedShape* out) {
    std::lock_guard<std::mutex> lock(g_cache.mu);
    refresh(tune_cache_path());
    auto it = g_cache.entries.find(key);
    if (it == g_cache.entries.end()) return false;
    *out = it->second;
    return true;
}

int tune_store(const std::string& key, const TunedShape& t) {
    std::lock_guard<std::mutex> lock(g_cache.mu);
    const std::string path = tune_cache_path();
    refresh(path);
    g_cache.entries[key] = t;
    mkdirs_for(path);
    FILE* f = fopen(path.c_str(), "a");
    if (f == nullptr)
        return tfail(TDES_EINVAL, "cannot write the autotune cache %s: %s", path.c_str(),
                     strerror(errno));
    fprintf(f,
            "{\"key\": \"%s\", \"warps_per_cta\": %d, \"ctas_per_sm\": %d, "
            "\"tiles_per_claim\": %d, \"round_form\": %d, \"slots\": %d, \"ms\": %.6g, "
            "\"baseline_ms\": %.6g, \"gbps\": %.6g, \"baseline_gbps\": %.6g}\n",
            key.c_str(), t.shape.warps, t.shape.ctas_per_sm, t.shape.tiles_per_claim,
            t.shape.round_form, t.slots, t.ms, t.baseline_ms, t.gbps, t.baseline_gbps);
    fclose(f);
    // the file now differs from what was read; keep the in-memory entry and
    // re-read on the next change by someone else
    struct stat st;
    if (stat(path.c_str(), &st) == 0) {
        g_cache.size = (long long)st.st_size;
        g_cache.mtime = (long long)st.st_mtime;
    }
    return TDES_OK;
}

}  // namespace tdes

extern "C" {

const char* tdes_autotune_cache_path(void) {
    thread_local std::string p;
    p = tdes::tune_cache_path();
    return p.c_str();
}

int tdes_batch_autotune(tdes_batch_t* b, unsigned flags, int reps, tdes_stream_t stream,
                        tdes_autotune_result_t* res) {
    if (b == nullptr || res == nullptr) return tfail(TDES_EINVAL, "NULL argument");
    if (reps < 1 || reps > 1000) return tfail(TDES_EINVAL, "reps must be 1..1000");
    memset(res, 0, sizeof *res);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the class of this plan (from its byte counts, as at planning)
    tdes::PlanHost h;
    memcpy(h.kind_bytes, b->kind_bytes, sizeof h.kind_bytes);
    const std::string key = tdes::tune_key(h, b->sms);
    snprintf(res->key, sizeof res->key, "%s", key.c_str());
    tdes::LaunchShape base;  // the default shape
    {
        size_t dyn = 0;
        int fit = 1;
        cudaError_t e = tdes::prepare_batch_kernel(base.warps, &dyn, &fit);
        if (e != cudaSuccess) return tfail(TDES_ECUDA, "batch kernel set-up: %s", cudaGetErrorString(e));
        base.ctas_per_sm = fit;
    }
    res->baseline = to_c(base);
    tdes::TunedShape cached;
    if (!(flags & TDES_TUNE_FORCE) && tdes::tune_lookup(key, &cached)) {
        int rc = tdes::set_batch_shape(b, cached.shape);
        if (rc == TDES_OK) {
            b->tuned = true;
            res->best = to_c(b->shape);
            res->best_ms = cached.ms;
            res->baseline_ms = cached.baseline_ms;
            res->from_cache = 1;
            return TDES_OK;
        }
    }
    if (b->total_items == 0 && b->direct.empty()) {  // nothing to time
        int rc = tdes::set_batch_shape(b, base);
        res->best = to_c(base);
        return rc;
    }
    uint32_t timed = 0;
    auto measure = [&](const tdes::LaunchShape& shape, double* ms) -> int {
        int rc = tdes::set_batch_shape(b, shape);
        if (rc != TDES_OK) return rc;
        cudaError_t e = time_shape(b, reps, s, ms);
        if (e != cudaSuccess) return tfail(TDES_ECUDA, "autotune launch: %s", cudaGetErrorString(e));
        ++timed;
        return TDES_OK;
    };
    tdes::LaunchShape best = base;
    double best_ms = 0.0;
    int rc = measure(base, &best_ms);
    if (rc != TDES_OK) return rc;
    // 1. grid: warps per CTA x CTAs per SM
    for (int warps : {4, 8}) {
        size_t dyn = 0;
        int fit = 1;
        cudaError_t e = tdes::prepare_batch_kernel(warps, &dyn, &fit);
        if (e != cudaSuccess) return tfail(TDES_ECUDA, "batch kernel set-up: %s", cudaGetErrorString(e));
        for (int c = fit; c >= std::max(1, fit - 1); --c) {
            tdes::LaunchShape t = best;
            t.warps = warps;
            t.ctas_per_sm = c;
            if (same(t, best)) continue;
            double ms = 0.0;
            if ((rc = measure(t, &ms)) != TDES_OK) return rc;
            if (ms < best_ms) {
                best = t;
                best_ms = ms;
            }
        }
    }
    // 2. tiles per claim (only plans with bitsliced tiles claim them)
    if (b->params.n_b_tiles) {
        const tdes::LaunchShape g = best;
        for (int k : {1, 2, 4, 8}) {
            tdes::LaunchShape t = g;
            t.tiles_per_claim = k;
            double ms = 0.0;
            if ((rc = measure(t, &ms)) != TDES_OK) return rc;
            if (ms < best_ms) {
                best = t;
                best_ms = ms;
            }
        }
        // 3. the round loop's form
        tdes::LaunchShape t = best;
        t.round_form = 1 - best.round_form;
        double ms = 0.0;
        if ((rc = measure(t, &ms)) != TDES_OK) return rc;
        if (ms < best_ms) {
            best = t;
            best_ms = ms;
        }
    }
    // 4. best against the default shape, alternating, so that drift between
    // the first and the last candidate does not decide
    double base_ms = best_ms;
    if (!same(best, base)) {
        std::vector<double> tb, tt;
        for (int r = 0; r < 3; ++r) {
            double x = 0.0;
            if ((rc = measure(base, &x)) != TDES_OK) return rc;
            tb.push_back(x);
            if ((rc = measure(best, &x)) != TDES_OK) return rc;
            tt.push_back(x);
        }
        std::sort(tb.begin(), tb.end());
        std::sort(tt.begin(), tt.end());
        base_ms = tb[1];
        best_ms = tt[1];
        if (!(best_ms < base_ms)) {
            best = base;
            best_ms = base_ms;
        }
    }
    if ((rc = tdes::set_batch_shape(b, best)) != TDES_OK) return rc;
    b->tuned = true;
    res->best = to_c(b->shape);
    res->best_ms = best_ms;
    res->baseline_ms = base_ms;
    res->candidates = timed;
    if (!(flags & TDES_TUNE_NO_STORE)) {
        tdes::TunedShape t;
        t.shape = b->shape;
        t.ms = best_ms;
        t.baseline_ms = base_ms;
        rc = tdes::tune_store(key, t);
        if (rc != TDES_OK) return rc;
    }
    return TDES_OK;
}

}  // extern "C"
