// tune_cache.cu -- the autotuners' choices kept across processes: a small JSON
// file of "key": "value" strings, one entry per line, written whole (to a
// temporary file that then replaces the old one) under a process-wide lock.
// Keys name the device, its SM count and the workload; values are the chosen
// launch shapes.  The file lives at $WN_TUNE_CACHE when that variable is set
// (empty or "off": no file), else $XDG_CACHE_HOME/wn/tune.json, else
// $HOME/.cache/wn/tune.json.  A file that cannot be read or parsed counts as
// empty; a failed write is ignored (the choice still holds for the process).
#include "tune_cache.h"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sys/stat.h>
#include <unistd.h>

namespace wn {
namespace {
std::mutex g_mu;

void make_dirs(const std::string &path)
{
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
}

bool plain(const std::string &s)
{
    for (char c : s)
        if (c == '"' || c == '\\' || c == '\n' || (unsigned char)c < 0x20) return false;
    return true;
}

std::map<std::string, std::string> read_all(const std::string &path)
{
    std::map<std::string, std::string> m;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return m;
    char line[4096];
    while (std::fgets(line, sizeof line, f)) {
        // an entry line:   "key": "value",
        const char *a = std::strchr(line, '"');
        if (!a) continue;
        const char *b = std::strchr(a + 1, '"');
        if (!b) continue;
        const char *c = std::strchr(b + 1, '"');
        if (!c) continue;
        const char *d = std::strchr(c + 1, '"');
        if (!d) continue;
        std::string key(a + 1, b), value(c + 1, d);
        if (key == "version") continue;
        m[key] = value;
    }
    std::fclose(f);
    return m;
}
}  // namespace

std::string tune_cache_path()
{
    const char *env = std::getenv("WN_TUNE_CACHE");
    if (env) return (std::strcmp(env, "off") == 0) ? std::string() : std::string(env);
    const char *xdg = std::getenv("XDG_CACHE_HOME");
    if (xdg && *xdg) return std::string(xdg) + "/wn/tune.json";
    const char *home = std::getenv("HOME");
    if (home && *home) return std::string(home) + "/.cache/wn/tune.json";
    return std::string();
}

bool tune_cache_get(const std::string &key, std::string &value)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return false;
    std::lock_guard<std::mutex> lock(g_mu);
    const auto m = read_all(path);
    auto it = m.find(key);
    if (it == m.end()) return false;
    value = it->second;
    return true;
}

void tune_cache_put(const std::string &key, const std::string &value)
{
    const std::string path = tune_cache_path();
    if (path.empty() || !plain(key) || !plain(value)) return;
    std::lock_guard<std::mutex> lock(g_mu);
    auto m = read_all(path);
    m[key] = value;
    make_dirs(path);
    const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    std::fprintf(f, "{\n  \"version\": \"1\"");
    for (const auto &kv : m) std::fprintf(f, ",\n  \"%s\": \"%s\"", kv.first.c_str(), kv.second.c_str());
    std::fprintf(f, "\n}\n");
    const bool ok = std::fclose(f) == 0;
    if (ok) std::rename(tmp.c_str(), path.c_str());
    else std::remove(tmp.c_str());
}

}  // namespace wn
