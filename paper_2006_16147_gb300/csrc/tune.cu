// tune.cu -- launch-shape cache of the autotuner.
//
// The bandwidth-bound V-cycle kernels take their launch shape at run time:
// the grid of every SELL sweep and restriction per level, and for block
// solves the number of lanes that share a row (hence the columns each lane
// carries). With options.autotune the candidates are timed once per problem
// shape with CUDA events on the hierarchy's stream (solve.cu, block.cu) and
// the fastest is kept here, keyed by a text description of the shape, so
// that another hierarchy of the same shape reuses it without timing. The
// cache can be saved to and merged from a text file.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "amg_internal.cuh"

namespace amg {
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
}  // namespace

bool tune_get(const std::string& key, int* value) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(key);
    if (it == g_tune.end()) return false;
    *value = it->second;
    return true;
}

void tune_put(const std::string& key, int value) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[key] = value;
}

std::string tune_key(const char* kind, int vbytes, long long n, long long nnz, long long slices, int k, int sms) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%s/f%d/n%lld/z%lld/s%lld/k%d/sm%d", kind, vbytes * 8, n, nnz, slices, k, sms);
    return buf;
}

}  // namespace amg

extern "C" {

amg_status amg_tune_save(const char* path) {
    if (!path) {
        amg::set_last_error("null path");
        return AMG_ERR_ARG;
    }
    std::ofstream f(path);
    if (!f) {
        amg::set_last_error(std::string("cannot open ") + path + " for writing");
        return AMG_ERR_ARG;
    }
    {
        std::lock_guard<std::mutex> g(amg::g_tune_mu);
        for (const auto& kv : amg::g_tune) f << kv.first << ' ' << kv.second << '\n';
    }
    f.close();
    if (!f) {
        amg::set_last_error(std::string("write to ") + path + " failed");
        return AMG_ERR_ARG;
    }
    return AMG_OK;
}

amg_status amg_tune_load(const char* path) {
    if (!path) {
        amg::set_last_error("null path");
        return AMG_ERR_ARG;
    }
    std::ifstream f(path);
    if (!f) {
        amg::set_last_error(std::string("cannot open ") + path);
        return AMG_ERR_ARG;
    }
    std::string line;
    int bad = 0;
    while (std::getline(f, line)) {
        if (line.empty()) continue;
        std::istringstream is(line);
        std::string key, rest;
        long long v = 0;
        if (!(is >> key >> v) || (is >> rest) || v < 1 || v > (1 << 24)) {
            ++bad;
            continue;
        }
        amg::tune_put(key, (int)v);
    }
    if (bad) {
        amg::set_last_error(std::to_string(bad) + " malformed line(s) in " + path);
        return AMG_ERR_ARG;
    }
    return AMG_OK;
}

void amg_tune_clear(void) {
    std::lock_guard<std::mutex> g(amg::g_tune_mu);
    amg::g_tune.clear();
}

int amg_tune_size(void) {
    std::lock_guard<std::mutex> g(amg::g_tune_mu);
    return (int)amg::g_tune.size();
}

}  // extern "C"
