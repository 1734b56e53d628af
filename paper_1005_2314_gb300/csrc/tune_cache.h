// tune_cache.h -- the autotuners' choices kept across processes (see
// tune_cache.cu for the file's location and format).
#pragma once

#include <string>

namespace wn {
// The cache file's path ("" when caching across processes is off).
std::string tune_cache_path();
// The value stored under key; false when there is none (or no file).
bool tune_cache_get(const std::string &key, std::string &value);
// Stores value under key (keys and values are plain text without quotes).
void tune_cache_put(const std::string &key, const std::string &value);
}  // namespace wn
