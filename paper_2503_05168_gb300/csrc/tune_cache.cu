// tune_cache.cu -- the batched multi-view autotuner's cache (host code): a
// small JSON object mapping a workload key to the configuration chosen for
// it, one entry per line, rewritten through a temporary file and a rename.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "kernels.h"

namespace seele {
namespace {

bool field(const std::string& line, const char* name, double* out) {
    const std::string pat = std::string("\"") + name + "\":";
    const size_t p = line.find(pat);
    if (p == std::string::npos) return false;
    char* end = nullptr;
    const double v = std::strtod(line.c_str() + p + pat.size(), &end);
    if (end == line.c_str() + p + pat.size()) return false;
    *out = v;
    return true;
}

// "key": {...} -> key, or "" for any other line
std::string line_key(const std::string& line) {
    const size_t a = line.find('"');
    if (a == std::string::npos) return "";
    const size_t b = line.find("\": {", a + 1);
    if (b == std::string::npos) return "";
    return line.substr(a + 1, b - a - 1);
}

std::string entry_line(const std::string& key, const TuneEntry& e) {
    char buf[512];
    std::snprintf(buf, sizeof buf,
                  "\"%s\": {\"tile_w\": %d, \"tile_h\": %d, \"schedule\": %d, \"batch_depth\": %d, "
                  "\"batch_ms\": %.6g, \"view_p50_ms\": %.6g, \"view_p99_ms\": %.6g}",
                  key.c_str(), e.tile_w, e.tile_h, e.schedule, e.batch_depth, e.batch_ms, e.p50_ms, e.p99_ms);
    return buf;
}

}  // namespace

bool tune_cache_lookup(const char* path, const std::string& key, TuneEntry* out) {
    if (!path) return false;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        if (line_key(line) != key) continue;
        double v[7];
        const char* names[7] = {"tile_w", "tile_h", "schedule", "batch_depth", "batch_ms", "view_p50_ms",
                                "view_p99_ms"};
        bool ok = true;
        for (int i = 0; i < 7 && ok; ++i) ok = field(line, names[i], &v[i]);
        if (!ok) return false;
        out->tile_w = (int)v[0];
        out->tile_h = (int)v[1];
        out->schedule = (int)v[2];
        out->batch_depth = (int)v[3];
        out->batch_ms = (float)v[4];
        out->p50_ms = (float)v[5];
        out->p99_ms = (float)v[6];
        return true;
    }
    return false;
}

bool tune_cache_store(const char* path, const std::string& key, const TuneEntry& e) {
    if (!path) return false;
    std::string body;
    {
        std::ifstream in(path);
        std::string line;
        while (std::getline(in, line)) {
            const std::string k = line_key(line);
            if (k.empty() || k == key) continue;
            std::string l = line;
            while (!l.empty() && (l.back() == ',' || l.back() == ' ' || l.back() == '\r')) l.pop_back();
            body += (body.empty() ? "" : ",\n") + l;
        }
    }
    body += (body.empty() ? "" : ",\n") + entry_line(key, e);
    const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)std::rand());
    {
        std::ofstream out(tmp);
        if (!out) return false;
        out << "{\n" << body << "\n}\n";
        if (!out) return false;
    }
    return std::rename(tmp.c_str(), path) == 0;
}

}  // namespace seele
