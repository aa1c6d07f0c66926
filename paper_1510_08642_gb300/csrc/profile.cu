// Optional launch profiling: when enabled, every kernel launch of the library
// is bracketed by two CUDA events recorded on its own stream, tagged with the
// kernel kind and its algorithmic work (FP64 instructions by the kernel's own
// count, and bytes it must move). The summary reports per kind the number of
// launches, the sum of launch durations and the busy time (the union of the
// launch intervals, so that launches overlapping on concurrent streams are
// not double counted).
#include <algorithm>
#include <mutex>
#include <utility>
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
  int dev;
};
std::mutex g_mu;
bool g_on = false;
std::vector<rec_t> g_recs;
// Events of earlier profiles, per device, reused: creating two events per
// launch costs more host time than the launch itself.
std::vector<std::pair<int, cudaEvent_t>> g_free;

int current_device() {
  int d = 0;
  return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}

cudaEvent_t take_event(int dev) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = g_free.size(); i-- > 0;)
      if (g_free[i].first == dev) {
        cudaEvent_t e = g_free[i].second;
        g_free[i] = g_free.back();
        g_free.pop_back();
        return e;
      }
  }
  cudaEvent_t e = nullptr;
  return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

void give_back(const rec_t& r) {
  g_free.push_back({r.dev, r.start});
  g_free.push_back({r.dev, r.stop});
}
}  // namespace

bool prof_enabled() { return g_on; }

void prof_begin_launch(cudaStream_t s, cudaEvent_t* start) {
  *start = nullptr;
  if (!g_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  *start = take_event(current_device());
  if (*start) cudaEventRecord(*start, s);
}

void prof_end_launch(cudaStream_t s, cudaEvent_t start, int kind, double ops, double bytes) {
  if (!g_on || !start) return;
  const int dev = current_device();
  cudaEvent_t stop = take_event(dev);
  if (!stop) return;
  cudaEventRecord(stop, s);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({kind, ops, bytes, start, stop, dev});
}

}  // namespace ddg

extern "C" {

ddg_status ddg_profile_begin(void) {
  std::lock_guard<std::mutex> lk(ddg::g_mu);
  for (auto& r : ddg::g_recs) ddg::give_back(r);
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
    std::lock_guard<std::mutex> lk(ddg::g_mu);
    for (auto& r : recs) ddg::give_back(r);
  }
  return st;
}

}  // extern "C"
