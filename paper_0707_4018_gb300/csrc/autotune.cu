// Launch-shape autotuner: times the variants of a kernel launch once per problem shape
// and caches the fastest (used for the tile shapes of the tensor-core coarse apply).
#include <map>
#include <mutex>
#include <vector>

#include "kernels.h"

namespace mg {

namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;  // key -> chosen variant
}  // namespace

int autotune_choose(const std::string &key, int count, const std::function<void(int)> &launch, cudaStream_t s) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  if (count <= 1) return 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MG_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return 0;
  EventPair ev;
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < count; ++v) {
    launch(v);  // untimed: first-touch and instruction-cache effects
    ev.start(s);
    for (int r = 0; r < 3; ++r) launch(v);
    const float ms = ev.stop(s);
    if (v == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  return best;
}

std::string autotune_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  for (const auto &kv : g_tune) out += kv.first + "=" + std::to_string(kv.second) + ";";
  return out;
}

}  // namespace mg
