// tune_cache.cu - the project autotuner's table (host code only): per problem
// shape, the transform choices that measured fastest on this device, so that
// later handles of the same shape skip the measurement.  The table lives for
// the process; a text file (PINT_TUNE_FILE, or pint_tune_load/pint_tune_save)
// carries it across processes.  One line per shape:
//   pint-tune equation dim nx ny nt precision bc half  fwd inv fused  ms
// (fwd/inv: tensor-core DFT for Step 1 / Step 3; fused: one-kernel 2-D Step 2;
// ms: the measured time of the chosen combination).  Lines starting with '#'
// are comments.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "pint_kernels.h"

namespace pint {

namespace {
using KeyT = std::tuple<int, int, int, int, int, int, int, int>;
KeyT as_tuple(const TuneKey& k) { return KeyT(k.equation, k.dim, k.nx, k.ny, k.nt, k.precision, k.bc, k.half); }

struct Table {
    std::mutex mu;
    std::map<KeyT, TuneVal> map;
    bool env_loaded = false;
};
Table& table() {
    static Table t;
    return t;
}

// Parses one line; returns false for a malformed one.
bool parse_line(const char* line, TuneKey& k, TuneVal& v) {
    char tag[16] = {0};
    int n = sscanf(line, "%15s %d %d %d %d %d %d %d %d %d %d %d %f", tag, &k.equation, &k.dim, &k.nx, &k.ny, &k.nt,
                   &k.precision, &k.bc, &k.half, &v.gemm_fwd, &v.gemm_inv, &v.fused, &v.ms);
    if (n != 13 || strcmp(tag, "pint-tune") != 0) return false;
    auto bit = [](int b) { return b == 0 || b == 1; };
    return k.dim >= 1 && k.dim <= 2 && k.nx > 0 && k.ny > 0 && k.nt > 0 && bit(v.gemm_fwd) && bit(v.gemm_inv) &&
           bit(v.fused) && bit(k.half);
}

int load_locked(Table& t, const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return -1;
    char line[256];
    int count = 0;
    bool bad = false;
    while (fgets(line, sizeof(line), f)) {
        const char* p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\0') continue;
        TuneKey k{};
        TuneVal v{};
        if (!parse_line(p, k, v)) {
            bad = true;
            break;
        }
        t.map[as_tuple(k)] = v;
        ++count;
    }
    fclose(f);
    return bad ? -2 : count;
}

void write_line(FILE* f, const KeyT& k, const TuneVal& v) {
    fprintf(f, "pint-tune %d %d %d %d %d %d %d %d %d %d %d %.6g\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
            std::get<3>(k), std::get<4>(k), std::get<5>(k), std::get<6>(k), std::get<7>(k), v.gemm_fwd, v.gemm_inv,
            v.fused, (double)v.ms);
}

void ensure_env_locked(Table& t) {
    if (t.env_loaded) return;
    t.env_loaded = true;
    const char* path = getenv("PINT_TUNE_FILE");
    if (path && *path) load_locked(t, path);   // a missing file is an empty table
}
}  // namespace

bool tune_lookup(const TuneKey& k, TuneVal* v) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    ensure_env_locked(t);
    auto it = t.map.find(as_tuple(k));
    if (it == t.map.end()) return false;
    if (v) *v = it->second;
    return true;
}

void tune_store(const TuneKey& k, const TuneVal& v) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    ensure_env_locked(t);
    t.map[as_tuple(k)] = v;
    const char* path = getenv("PINT_TUNE_FILE");
    if (path && *path) {
        FILE* f = fopen(path, "a");
        if (f) {
            write_line(f, as_tuple(k), v);
            fclose(f);
        }
    }
}

int tune_load(const char* path) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    return load_locked(t, path);
}

int tune_save(const char* path) {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    FILE* f = fopen(path, "w");
    if (!f) return -1;
    fprintf(f, "# pint autotuner table: equation dim nx ny nt precision bc half  fwd inv fused  ms\n");
    for (const auto& e : t.map) write_line(f, e.first, e.second);
    const int n = (int)t.map.size();
    return fclose(f) == 0 ? n : -1;
}

void tune_clear() {
    Table& t = table();
    std::lock_guard<std::mutex> g(t.mu);
    t.map.clear();
    t.env_loaded = true;   // a cleared table is not reloaded from the environment's file
}

}  // namespace pint
