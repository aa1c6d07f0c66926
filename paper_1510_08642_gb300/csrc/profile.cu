// Optional launch profiling: when enabled, every kernel launch of the library
// is bracketed by two CUDA events recorded on its own stream, tagged with the
// kernel kind and its algorithmic work (FP64 instructions by the kernel's own
// count, and bytes it must move). The summary reports per kind the number of
// launches, the sum of launch durations and the busy time (the union of the
// launch intervals, so that launches overlapping on concurrent streams are
// not double counted).
#include <algorithm>
#include <mutex>
#include <vector>

#include "ddgemm.h"
#include "kernels.cuh"

namespace ddg {

namespace {
struct rec_t {
  int kind;
  double ops;
  double bytes;
  cudaEvent_t start, stop;
};
std::mutex g_mu;
bool g_on = false;
std::vector<rec_t> g_recs;
}  // namespace

bool prof_enabled() { return g_on; }

void prof_begin_launch(cudaStream_t s, cudaEvent_t* start) {
  *start = nullptr;
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (cudaEventCreate(start) != cudaSuccess) { *start = nullptr; return; }
  cudaEventRecord(*start, s);
}

void prof_end_launch(cudaStream_t s, cudaEvent_t start, int kind, double ops, double bytes) {
  if (!g_on || !start) return;
  cudaEvent_t stop;
  if (cudaEventCreate(&stop) != cudaSuccess) return;
  cudaEventRecord(stop, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({kind, ops, bytes, start, stop});
}

}  // namespace ddg

extern "C" {

ddg_status ddg_profile_begin(void) {
  std::lock_guard<std::mutex> lk(ddg::g_mu);
  for (auto& r : ddg::g_recs) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
  ddg::g_recs.clear();
  ddg::g_on = true;
  return DDG_OK;
}

ddg_status ddg_profile_end(ddg_kernel_prof* out, int32_t nkinds) {
  std::vector<ddg::rec_t> recs;
  {
    std::lock_guard<std::mutex> lk(ddg::g_mu);
    ddg::g_on = false;
    recs.swap(ddg::g_recs);
  }
  ddg_status st = DDG_OK;
  for (int k = 0; k < nkinds; ++k) out[k] = ddg_kernel_prof{0, 0.0, 0.0, 0.0, 0.0};
  if (!recs.empty()) {
    const cudaEvent_t ref = recs.front().start;
    std::vector<std::vector<std::pair<float, float>>> iv(nkinds > 0 ? nkinds : 1);
    for (auto& r : recs) {
      if (cudaEventSynchronize(r.stop) != cudaSuccess) { st = DDG_ECUDA; break; }
      float t0 = 0.f, t1 = 0.f, d = 0.f;
      cudaEventElapsedTime(&t0, ref, r.start);
      cudaEventElapsedTime(&t1, ref, r.stop);
      cudaEventElapsedTime(&d, r.start, r.stop);
      if (r.kind < 0 || r.kind >= nkinds) continue;
      ddg_kernel_prof& o = out[r.kind];
      o.launches += 1;
      o.sum_ms += d;
      o.ops += r.ops;
      o.bytes += r.bytes;
      iv[r.kind].push_back({t0, t1});
    }
    for (int k = 0; k < nkinds && st == DDG_OK; ++k) {
      auto& v = iv[k];
      std::sort(v.begin(), v.end());
      double busy = 0.0, cs = 0.0, ce = -1.0;
      bool open = false;
      for (auto& p : v) {
        if (!open || p.first > ce) {
          if (open) busy += ce - cs;
          cs = p.first; ce = p.second; open = true;
        } else {
          ce = std::max<double>(ce, p.second);
        }
      }
      if (open) busy += ce - cs;
      out[k].busy_ms = busy;
    }
    for (auto& r : recs) { cudaEventDestroy(r.start); cudaEventDestroy(r.stop); }
  }
  return st;
}

}  // extern "C"
