// Tuned parameters: a small text table, written by the autotuner
// (paper_2506_22713_gb300/autotune.py) from timings on the GPU, that the
// library reads once per process and consults where it would otherwise use
// a fixed default.  Keys:
//   block_k        a = precision form (0 plain FP64, 1 plain FP32, 2 mixed
//                  BF16, 3 mixed TF32), b = m, c = n  -> k of Alg. 1 when
//                  the caller passes block_k = 0
//   f32_tile       a = M, b = N, c = K                -> tile of the FP32 SIMT
//                  product (16, 32, 64 or 128)
//   batch_workers  a = count, b = mean m, c = mean n   -> worker streams of
//                  eod_abe_factor_batched
//   batch_block_k  a = form, b = mean m, c = mean n    -> k of the batched
//                  items on those streams
//   core_leaf      a = p (b = c = 0)                   -> leaf width of the
//                  blocked Cholesky of a p x p Gram (16, 32, 64 or 128)
// Line format: key a_lo a_hi b_lo b_hi c_lo c_hi value (inclusive ranges);
// '#' starts a comment; of the rows of a key whose ranges hold the query,
// the nearest wins (smallest sum of |log x - log centre| over the axes, the
// centre the geometric mean of the row's bounds).  The file is
// $EOD_TUNING_FILE if set, else tuning.txt beside the library; a missing
// file means no tuned values.
#include "common.cuh"

#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace eod {
namespace {

struct TuneRow {
    std::string key;
    int64_t lo[3], hi[3];
    int64_t value;
};

std::mutex g_tune_mu;
std::vector<TuneRow> g_rows;
bool g_loaded = false;

std::string default_path() {
    if (const char *env = std::getenv("EOD_TUNING_FILE")) return env;
    Dl_info info;
    if (dladdr((void *)&default_path, &info) && info.dli_fname) {
        std::string so = info.dli_fname;
        const size_t slash = so.rfind('/');
        return (slash == std::string::npos ? std::string(".") : so.substr(0, slash)) + "/tuning.txt";
    }
    return "tuning.txt";
}

// Parses `path` into rows; false on a malformed line (rows untouched).
bool parse(const std::string &path, std::vector<TuneRow> &rows, bool &exists) {
    FILE *f = std::fopen(path.c_str(), "r");
    exists = f != nullptr;
    if (!f) return true;
    std::vector<TuneRow> out;
    char line[512];
    bool ok = true;
    while (std::fgets(line, sizeof(line), f)) {
        if (char *h = std::strchr(line, '#')) *h = '\0';
        char key[64];
        long long v[7];
        int n = std::sscanf(line, "%63s %lld %lld %lld %lld %lld %lld %lld", key, &v[0], &v[1], &v[2], &v[3], &v[4],
                            &v[5], &v[6]);
        if (n <= 0) continue;   // blank or comment
        if (n != 8 || v[0] > v[1] || v[2] > v[3] || v[4] > v[5]) {
            ok = false;
            break;
        }
        TuneRow r;
        r.key = key;
        for (int i = 0; i < 3; ++i) {
            r.lo[i] = v[2 * i];
            r.hi[i] = v[2 * i + 1];
        }
        r.value = v[6];
        out.push_back(r);
    }
    std::fclose(f);
    if (ok) rows.swap(out);
    return ok;
}

void ensure_loaded() {
    if (g_loaded) return;
    bool exists = false;
    std::vector<TuneRow> rows;
    if (parse(default_path(), rows, exists)) g_rows.swap(rows);
    g_loaded = true;
}

}  // namespace

// Among the rows of `key` whose ranges hold (a, b, c), the nearest: the
// smallest sum over the three axes of |log(x / centre)|, centre the
// geometric mean of the row's bounds (the shape it was measured at, for the
// autotuner's ranges); ties go to the earlier row.
bool tuned_value(const char *key, int64_t a, int64_t b, int64_t c, int64_t *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    ensure_loaded();
    const int64_t x[3] = {a, b, c};
    const TuneRow *best = nullptr;
    double best_d = 0.0;
    for (const TuneRow &r : g_rows) {
        if (r.key != key) continue;
        bool in = true;
        for (int i = 0; i < 3; ++i) in = in && x[i] >= r.lo[i] && x[i] <= r.hi[i];
        if (!in) continue;
        double d = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double lo = std::max<double>((double)r.lo[i], 1.0), hi = std::max<double>((double)r.hi[i], 1.0);
            const double xi = std::max<double>((double)x[i], 1.0);
            d += std::fabs(std::log(xi) - 0.5 * (std::log(lo) + std::log(hi)));
        }
        if (!best || d < best_d) {
            best = &r;
            best_d = d;
        }
    }
    if (!best) return false;
    *out = best->value;
    return true;
}

}  // namespace eod

extern "C" eod_status eod_abe_tuning_load(const char *path) {
    using namespace eod;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool exists = false;
    std::vector<TuneRow> rows;
    const std::string p = path ? std::string(path) : default_path();
    if (!parse(p, rows, exists)) return EOD_EINVAL;
    g_rows.swap(rows);
    g_loaded = true;
    return EOD_OK;
}

extern "C" int32_t eod_abe_tuning_lookup(const char *key, int64_t a, int64_t b, int64_t c, int64_t *value) {
    if (!key || !value) return 0;
    return eod::tuned_value(key, a, b, c, value) ? 1 : 0;
}
