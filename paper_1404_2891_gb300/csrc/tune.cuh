// Reading the autotuner's cache (paper_1404_2891_gb300/autotune.py writes it):
// a JSON object whose members are keyed "<gpu>|<kind>|..." and hold flat
// objects of numbers, e.g.
//   {"NVIDIA GB300|single|n4096|m0128|q32|mixed": {"lu_outer": 256, "panel_cluster": 0}}
#pragma once
#include <map>
#include <string>

// The numbers of the member `key` of the cache file at `path`; false when the
// file or the member is missing or malformed (the caller keeps its defaults).
bool tune_lookup(const char* path, const std::string& key, std::map<std::string, double>& out);
// "<device name>" of the current device.
std::string tune_gpu_name();
// The size bucket of an order: the next power of two >= n.
long long tune_bucket(long long n);
