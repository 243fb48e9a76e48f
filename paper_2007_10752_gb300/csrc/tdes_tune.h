// tdes_tune.h -- the autotuner's persistent cache of launch shapes, shared by
// the batch API (tdes_batch.cu), the batch contexts (tdes_ctx.cu) and the
// server (tdes_serve.cu).  Not part of the public interface.
//
// The cache is a text file of JSON lines, one tuned shape per line:
//   {"key": "sm152/t3m0s1c1/2^30", "warps_per_cta": 4, "ctas_per_sm": 3,
//    "tiles_per_claim": 1, "round_form": 0, "slots": 0, "ms": 3.51,
//    "baseline_ms": 3.60, "gbps": 0, "baseline_gbps": 0}
// (server entries, key "serve/sm<SMs>", keep the reserved CTAs per SM in
// ctas_per_sm, and closed-loop GB/s in place of times)
// A later line for the same key replaces an earlier one.  The file is
// TDES_AUTOTUNE_CACHE if that environment variable is set, else
// $XDG_CACHE_HOME/tdes_gb300/autotune.jsonl, else
// $HOME/.cache/tdes_gb300/autotune.jsonl.
#pragma once
#include <string>

#include "tdes_batch_internal.h"

namespace tdes {

struct TunedShape {
    LaunchShape shape;
    int slots = 0;  // server entries: batches in flight at once
    double ms = 0.0, baseline_ms = 0.0;      // batch entries: device time per launch
    double gbps = 0.0, baseline_gbps = 0.0;  // server entries: closed-loop throughput
};

// Workload class of a plan: "sm<SMs>/t<d>m<d>s<d>c<d>/2^<e>", where the
// digits grade the share of the payload in bitsliced tiles (t), mixed-key
// tiles (m), one-block-per-lane items (s) and CBC-encryption chains (c) --
// 0 none, 1 up to a third, 2 up to two thirds, 3 more -- and e is the floor
// of log2 of the payload the batch kernels run (direct messages excluded:
// the single-key kernels run them in their own shape).
std::string tune_key(const PlanHost& h, int sms);
// The server's class on a GPU of `sms` SMs.
std::string serve_tune_key(int sms);
// Cached shape for `key` from the current cache file (re-read when the
// file's path, size or modification time changes).
bool tune_lookup(const std::string& key, TunedShape* out);
// Appends one line to the cache file (creating its directory) and updates
// the in-memory copy.  TDES_OK, or TDES_EINVAL (reason in tdes_last_error())
// when the file cannot be written; the in-memory copy is updated either way.
int tune_store(const std::string& key, const TunedShape& t);
// The cache file in use.
std::string tune_cache_path();

}  // namespace tdes
