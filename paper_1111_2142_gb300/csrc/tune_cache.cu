// Autotuner cache: a small JSON file mapping a problem key to the configuration
// the autotuner measured fastest. One entry per line, so that the file stays
// readable and this reader stays simple:
//   {
//   "<key>": {"kernel": K, "tile": T, "mode": M, "us_per_step": X},
//   ...
//   }
// A missing or unreadable file is an empty cache. Writes go to a temporary file
// that is then renamed over the cache, so a reader never sees half a file.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include <unistd.h>

#include "launch.h"

namespace lwacm {
namespace {

// parse one entry line; false if the line is not an entry
bool parse_line(const std::string &line, std::string &key, TuneChoice &ch) {
    const size_t q0 = line.find('"');
    if (q0 == std::string::npos) return false;
    const size_t q1 = line.find('"', q0 + 1);
    if (q1 == std::string::npos) return false;
    key = line.substr(q0 + 1, q1 - q0 - 1);
    const char *rest = line.c_str() + q1 + 1;
    TuneChoice c;
    if (std::sscanf(rest, " : {\"kernel\": %d, \"tile\": %d, \"mode\": %d, \"us_per_step\": %lf}", &c.kernel,
                    &c.tile, &c.mode, &c.us) != 4)
        return false;
    ch = c;
    return true;
}

std::map<std::string, TuneChoice> read_all(const char *path) {
    std::map<std::string, TuneChoice> m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    char buf[4096];
    while (std::fgets(buf, sizeof buf, f)) {
        std::string key;
        TuneChoice ch;
        if (parse_line(buf, key, ch)) m[key] = ch;
    }
    std::fclose(f);
    return m;
}

}  // namespace

bool tune_cache_lookup(const char *path, const std::string &key, TuneChoice *out) {
    if (!path || !*path) return false;
    const std::map<std::string, TuneChoice> m = read_all(path);
    const auto it = m.find(key);
    if (it == m.end()) return false;
    *out = it->second;
    return true;
}

bool tune_cache_store(const char *path, const std::string &key, const TuneChoice &ch) {
    if (!path || !*path || key.find('"') != std::string::npos) return false;
    std::map<std::string, TuneChoice> m = read_all(path);
    m[key] = ch;
    const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\n");
    size_t k = 0;
    for (const auto &e : m) {
        std::fprintf(f, "\"%s\": {\"kernel\": %d, \"tile\": %d, \"mode\": %d, \"us_per_step\": %.3f}%s\n",
                     e.first.c_str(), e.second.kernel, e.second.tile, e.second.mode, e.second.us,
                     ++k < m.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    const bool ok = std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace lwacm
