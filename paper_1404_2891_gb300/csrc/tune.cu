// Reader of the autotuner's JSON cache (format in tune.cuh).  A small
// hand-written scanner: the file is written by the project's own tuner, so
// only its shape is accepted -- string keys, objects of numbers (with
// strings and flat objects of numbers as non-tunable fields).
#include <cuda_runtime.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "tune.cuh"

namespace {

void skip_ws(const std::string& s, size_t& i) {
  while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
}

bool read_string(const std::string& s, size_t& i, std::string& out) {
  skip_ws(s, i);
  if (i >= s.size() || s[i] != '"') return false;
  ++i;
  out.clear();
  while (i < s.size() && s[i] != '"') {
    if (s[i] == '\\' && i + 1 < s.size()) ++i;
    out.push_back(s[i++]);
  }
  if (i >= s.size()) return false;
  ++i;
  return true;
}

bool read_number(const std::string& s, size_t& i, double& v) {
  skip_ws(s, i);
  const char* b = s.c_str() + i;
  char* e = nullptr;
  v = std::strtod(b, &e);
  if (e == b) return false;
  i += (size_t)(e - b);
  return true;
}

// skip one JSON value of the cache's shapes (string, number, flat object)
bool skip_value(const std::string& s, size_t& i) {
  skip_ws(s, i);
  if (i >= s.size()) return false;
  if (s[i] == '"') {
    std::string t;
    return read_string(s, i, t);
  }
  if (s[i] == '{') {
    int depth = 0;
    for (; i < s.size(); ++i) {
      if (s[i] == '{') ++depth;
      if (s[i] == '}' && --depth == 0) { ++i; return true; }
    }
    return false;
  }
  double v;
  return read_number(s, i, v);
}

}  // namespace

bool tune_lookup(const char* path, const std::string& key, std::map<std::string, double>& out) {
  if (!path || !*path) return false;
  std::ifstream f(path);
  if (!f) return false;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string s = ss.str();
  size_t i = 0;
  skip_ws(s, i);
  if (i >= s.size() || s[i] != '{') return false;
  ++i;
  for (;;) {
    skip_ws(s, i);
    if (i < s.size() && s[i] == '}') return false;
    std::string k;
    if (!read_string(s, i, k)) return false;
    skip_ws(s, i);
    if (i >= s.size() || s[i] != ':') return false;
    ++i;
    if (k != key) {
      if (!skip_value(s, i)) return false;
    } else {
      skip_ws(s, i);
      if (i >= s.size() || s[i] != '{') return false;
      ++i;
      for (;;) {
        skip_ws(s, i);
        if (i < s.size() && s[i] == '}') return true;
        std::string name;
        double v;
        if (!read_string(s, i, name)) return false;
        skip_ws(s, i);
        if (i >= s.size() || s[i] != ':') return false;
        ++i;
        skip_ws(s, i);
        if (i < s.size() && (s[i] == '"' || s[i] == '{')) {  // a note or a record of timings: not a tunable
          if (!skip_value(s, i)) return false;
        } else {
          if (!read_number(s, i, v)) return false;
          out[name] = v;
        }
        skip_ws(s, i);
        if (i < s.size() && s[i] == ',') ++i;
      }
    }
    skip_ws(s, i);
    if (i < s.size() && s[i] == ',') ++i;
  }
}

std::string tune_gpu_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  return std::string(p.name);
}

long long tune_bucket(long long n) {
  long long b = 1;
  while (b < n) b <<= 1;
  return b;
}
