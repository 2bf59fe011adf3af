// tune.cu -- the tuning cache of libfastsv: kernel choices per shape class.
//
// The paper leaves the SpMV / SpMSpV switch to tuning (Section 4.2 gives no
// threshold), and the tile shape of the merge-path SpMV, the number of column
// blocks and the sparse-iteration thresholds depend on the graph's size and
// density.  The autotuner (paper_1910_05971_gb300/tune.py) times candidate
// settings on the device and writes one line per shape class:
//     <key> = <k2_items> <k2_threads> <col_blocks> <sparse_div> <batch_sparse_div>
// where <key> is fastsv_tune_key's string ("single n26 d10 r64", "batched
// g12 n14 d6"); '#' starts a comment; a later line for a key replaces an
// earlier one.  A handle created with opt.tune_cache reads the file once and,
// for every call whose shape class has an entry, runs with those five values.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "fastsv_internal.h"

namespace fsv {

static int rlog2(double x) { return x >= 1.0 ? (int)std::lround(std::log2(x)) : 0; }

// half-octaves of the average number of entries per vertex
static int deg_bucket(int64_t n, int64_t m) {
    if (n <= 0 || m <= 0) return -99;
    return (int)std::lround(2.0 * std::log2((double)m / (double)n));
}

int tune_key(int kind, int64_t n, int64_t m, int64_t graphs, int bits, char* out, size_t cap) {
    if (kind == TUNE_BATCHED)
        return std::snprintf(out, cap, "batched g%d n%d d%d", rlog2((double)graphs),
                             rlog2(graphs > 0 ? (double)n / (double)graphs : 0.0), deg_bucket(n, m));
    return std::snprintf(out, cap, "single n%d d%d r%d", rlog2((double)n), deg_bucket(n, m), bits);
}

static std::string trim(const std::string& s) {
    size_t a = s.find_first_not_of(" \t\r\n"), b = s.find_last_not_of(" \t\r\n");
    return a == std::string::npos ? std::string() : s.substr(a, b - a + 1);
}

fastsv_status tune_load(fastsv_ctx* h, const char* path) {
    FILE* fp = std::fopen(path, "r");
    if (!fp) return FASTSV_ERR_INVALID_ARG;
    char line[512];
    while (std::fgets(line, sizeof line, fp)) {
        std::string s(line);
        const size_t hash = s.find('#');
        if (hash != std::string::npos) s = s.substr(0, hash);
        const size_t eq = s.find('=');
        if (eq == std::string::npos) continue;
        TuneEntry e;
        e.key = trim(s.substr(0, eq));
        if (e.key.empty()) continue;
        if (std::sscanf(s.c_str() + eq + 1, "%d %d %d %d %d", &e.k2_items, &e.k2_threads, &e.col_blocks, &e.sparse_div,
                        &e.batch_sparse_div) != 5)
            continue;
        const bool ok = (e.k2_items == 4 || e.k2_items == 8 || e.k2_items == 16) &&
                        (e.k2_threads == 64 || e.k2_threads == 256) && e.col_blocks >= 0 && e.col_blocks <= 32 &&
                        e.sparse_div >= 0 && e.batch_sparse_div >= 0;
        if (!ok) continue;
        bool replaced = false;
        for (auto& old : h->tune)
            if (old.key == e.key) {
                old = e;
                replaced = true;
            }
        if (!replaced) h->tune.push_back(e);
    }
    std::fclose(fp);
    return FASTSV_OK;
}

void tune_apply(fastsv_ctx* h, int kind, int64_t n, int64_t m, int64_t graphs, int bits) {
    h->opt = h->base_opt;
    h->last_tuned = 0;
    if (h->tune.empty()) return;
    char key[128];
    tune_key(kind, n, m, graphs, bits, key, sizeof key);
    for (const auto& e : h->tune) {
        if (e.key != key) continue;
        h->opt.k2_items = e.k2_items;
        h->opt.k2_threads = e.k2_threads;
        h->opt.col_blocks = e.col_blocks;
        h->opt.sparse_div = e.sparse_div;
        h->opt.batch_sparse_div = e.batch_sparse_div;
        h->last_tuned = 1;
        return;
    }
}

}  // namespace fsv

extern "C" int32_t fastsv_tune_key(int32_t kind, int64_t n, int64_t m, int64_t graphs, int32_t rowptr_bits, char* out,
                                   int32_t cap) {
    if (!out || cap <= 0 || (kind != fsv::TUNE_SINGLE && kind != fsv::TUNE_BATCHED)) return -1;
    return fsv::tune_key(kind, n, m, graphs, rowptr_bits, out, (size_t)cap);
}
