// tune.h -- persistent cache of tuned kernel configurations (internal).
//
// A flat JSON object mapping a key (kernel family, element type, shape
// signature, SM count) to a configuration string.  The file is
// $ADVECT_TUNE_CACHE, else $HOME/.cache/advect_gb300/tune.json.
#pragma once

#include <string>

namespace advect {

bool tune_cache_get(const std::string& key, std::string& value);
void tune_cache_put(const std::string& key, const std::string& value);
std::string tune_cache_path();
bool tune_env_enabled();  // ADVECT_TUNE=1

}  // namespace advect
