// Kernel accounting (see prof.cuh).
#include <atomic>
#include <vector>

#include "prof.cuh"

namespace feast {
namespace prof {

namespace {

constexpr int kRing = 4096;

struct Pair {
  cudaEvent_t a = nullptr, b = nullptr;
  int cls = 0;
};

struct State {
  std::atomic<bool> on{false};
  std::vector<Pair> ring;
  int head = 0, count = 0;   // pending pairs: ring[(head - count) mod kRing] .. ring[head - 1]
  int open = -1;             // index of the pair begun but not ended
  double ms[NCLS] = {};
  long long n[NCLS] = {};
  double work[NCLS] = {};
  std::atomic<long long> launches{0};
};

State& st() {
  static State s;
  return s;
}

void fold_oldest(State& s) {
  const int idx = (s.head - s.count + kRing) % kRing;
  Pair& p = s.ring[idx];
  cudaEventSynchronize(p.b);
  float t = 0.f;
  if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
    s.ms[p.cls] += t;
    s.n[p.cls] += 1;
  }
  --s.count;
}

}  // namespace

// Timing is for one host thread (a single handle); the launch counter is
// shared by every thread.
void set_enabled(bool on) {
  State& s = st();
  if (on && s.ring.empty()) {
    s.ring.resize(kRing);
    for (auto& p : s.ring) {
      cudaEventCreate(&p.a);
      cudaEventCreate(&p.b);
    }
  }
  s.on = on;
}

bool enabled() { return st().on; }

void begin(cudaStream_t stream, int cls) {
  State& s = st();
  if (!s.on) return;
  if (s.count == kRing) fold_oldest(s);
  Pair& p = s.ring[s.head];
  p.cls = cls;
  cudaEventRecord(p.a, stream);
  s.open = s.head;
}

void end(cudaStream_t stream, int cls) {
  State& s = st();
  if (!s.on || s.open < 0) return;
  Pair& p = s.ring[s.open];
  p.cls = cls;
  cudaEventRecord(p.b, stream);
  s.open = -1;
  s.head = (s.head + 1) % kRing;
  ++s.count;
}

void add_work(int cls, double flops) {
  State& s = st();
  if (s.on) s.work[cls] += flops;
}

void collect(double* ms, long long* count, double* work) {
  State& s = st();
  while (s.count > 0) fold_oldest(s);
  for (int c = 0; c < NCLS; ++c) {
    if (ms) ms[c] += s.ms[c];
    if (count) count[c] += s.n[c];
    if (work) work[c] += s.work[c];
    s.ms[c] = 0.0;
    s.n[c] = 0;
    s.work[c] = 0.0;
  }
}

void count_launch(int n) { st().launches += n; }

long long launches() { return st().launches; }

}  // namespace prof
}  // namespace feast
