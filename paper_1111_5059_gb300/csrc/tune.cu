// Autotuner for the batched Wilson hop launches of the multi-right-hand-side
// solver.
//
// A "shape" is everything that changes the best launch of one hop step: the
// lattice (Vh, Ls), the storage precision, how many right-hand sides the step
// covers, dagger, whether a site term is fused, and the epilogue operator
// kinds.  The choices are how many right-hand sides one launch takes (link
// reuse against shared-memory footprint and occupancy) and how many CTAs per
// SM the persistent kernel runs (fewer CTAs leave more L1 per CTA and fewer
// bulk copies in flight).  The first time a shape is seen, every candidate is
// run on the real operands (the call is about to overwrite its outputs
// anyway) and timed with CUDA events; the fastest is cached for the process
// and, if the environment variable DWF_TUNE_CACHE names a file, appended to
// that file and read back by later processes.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <sstream>

#include "dwf_internal.h"

namespace dwf {

namespace {

std::mutex g_mu;
std::map<std::string, HopChoice> g_cache;
bool g_loaded = false;

void load_file_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = std::getenv("DWF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof line, f)) {
    std::istringstream is(line);
    std::string key;
    HopChoice c;
    // entries a launch could not take are skipped (the shape is then tuned again)
    if (is >> key >> c.batch >> c.ctas_per_sm >> c.ms && c.batch >= 1 && c.batch <= kMaxBatch && c.ctas_per_sm >= 0)
      g_cache[key] = c;
  }
  std::fclose(f);
}

void store_file_locked(const std::string& key, const HopChoice& c) {
  const char* path = std::getenv("DWF_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %.6f\n", key.c_str(), c.batch, c.ctas_per_sm, c.ms);
  std::fclose(f);
}

}  // namespace

std::string HopShape::key() const {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p{};
  cudaGetDeviceProperties(&p, dev);
  std::ostringstream os;
  os << "sm" << p.major << p.minor << "x" << p.multiProcessorCount << "/Vh" << Vh << "/Ls" << Ls << "/p" << prec << "/n"
     << nrhs << "/d" << dag << "/x" << has_x << "/e" << ex_kind << "." << eout_kind;
  return os.str();
}

std::vector<HopChoice> hop_candidates(const HopShape& s, int bmax) {
  std::vector<HopChoice> out;
  const int top = s.nrhs < bmax ? s.nrhs : bmax;
  for (int b = top; b >= 1; --b)
    for (int ctas : {0, 6, 4}) {
      HopChoice c;
      c.batch = b;
      c.ctas_per_sm = ctas;
      out.push_back(c);
    }
  return out;
}

dwf_status tune_hop(dwf_lattice* L, const HopShape& s, int bmax, const std::function<dwf_status(const HopChoice&)>& run,
                    HopChoice* choice, double* tune_seconds) {
  const std::string key = s.key();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *choice = it->second;
      return DWF_OK;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DWF_CUDA(L, cudaStreamIsCapturing(L->stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(L, DWF_ERR_INVALID_ARG, "tune: a new launch shape appeared while recording a graph");
  const auto t0 = std::chrono::steady_clock::now();
  const bool timing = L->timing;
  L->timing = false;  // candidate runs stay out of the kernel-time accumulators
  cudaEvent_t a = nullptr, b = nullptr;
  dwf_status st = DWF_OK;
  HopChoice best;
  best.ms = -1.0;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = fail(L, DWF_ERR_CUDA, "tune: events");
  constexpr int kReps = 2;
  for (const HopChoice& c : hop_candidates(s, bmax)) {
    if (st != DWF_OK) break;
    st = run(c);  // warm-up (and first-use attribute setting)
    if (st != DWF_OK) break;
    if (cudaEventRecord(a, L->stream) != cudaSuccess) {
      st = fail(L, DWF_ERR_CUDA, "tune: event record");
      break;
    }
    for (int rep = 0; rep < kReps && st == DWF_OK; ++rep) st = run(c);
    if (st != DWF_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(b, L->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      st = fail(L, DWF_ERR_CUDA, "tune: event timing");
      break;
    }
    HopChoice t = c;
    t.ms = ms / kReps;
    if (best.ms < 0.0 || t.ms < best.ms) best = t;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  L->timing = timing;
  if (st == DWF_OK) st = check_dev_err(L);
  if (st != DWF_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best;
    store_file_locked(key, best);
  }
  *choice = best;
  if (tune_seconds) *tune_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return DWF_OK;
}

}  // namespace dwf
