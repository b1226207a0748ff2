// sg_prof.cpp -- per-kernel CUDA-event tracing (off unless enabled).
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "sg_internal.h"
#include "sg_runtime.h"

namespace sgk {

cudaEvent_t Prof::take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::begin(const char* name, cudaStream_t s) {
  Rec r{name, take(), take()};
  cudaEventRecord(r.a, s);
  open.push_back(r);
}

void Prof::end(cudaStream_t s) {
  if (!open.empty()) cudaEventRecord(open.back().b, s);
}

void Prof::collect() {
  for (Rec& r : open) {
    float ms = 0.0f;
    // a flush that leaves no results does not wait for the device itself
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto& a = agg[r.name];
      a.first += 1;
      a.second += ms;
    } else {
      cudaGetLastError();
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  open.clear();
}

Prof::~Prof() {
  for (Rec& r : open) {
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace sgk

extern "C" sg_status sg_profile_enable(sg_ctx* c, int on) {
  if (!c) return SG_ERR_INVALID_ARG;
  c->prof.on = on ? 1 : 0;
  return SG_OK;
}

extern "C" sg_status sg_profile_report(sg_ctx* c, char* buf, size_t cap, size_t* len, int reset) {
  if (!c) return SG_ERR_INVALID_ARG;
  std::string s;
  char line[256];
  for (auto& kv : c->prof.agg) {
    snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), kv.second.first,
             kv.second.second);
    s += line;
  }
  if (len) *len = s.size() + 1;
  if (buf && cap) {
    size_t m = std::min(cap - 1, s.size());
    memcpy(buf, s.data(), m);
    buf[m] = 0;
  }
  if (reset) c->prof.agg.clear();
  return SG_OK;
}
