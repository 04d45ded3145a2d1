// Optional CUDA-event timing of the hot kernels (see psf_kernel_timing in
// include/psf.h).  Off by default; when on, each TimingScope records a pair of
// events on the launching stream around the kernel it encloses.
#include <vector>

#include "timing.cuh"

namespace psf {

namespace {
struct Record {
  int cls;
  cudaEvent_t a, b;
};
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;
std::vector<Record> g_rec;

cudaEvent_t next_event() {
  if (g_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_used++];
}
}  // namespace

TimingScope::TimingScope(int cls, cudaStream_t s) : cls_(cls), s_(s), a_(nullptr) {
  if (!g_on) return;
  a_ = next_event();
  if (a_) cudaEventRecord((cudaEvent_t)a_, s_);
}

TimingScope::~TimingScope() {
  if (!g_on || !a_) return;
  cudaEvent_t b = next_event();
  if (!b) return;
  cudaEventRecord(b, s_);
  g_rec.push_back(Record{cls_, (cudaEvent_t)a_, b});
}

}  // namespace psf

using namespace psf;

extern "C" int psf_kernel_timing(int enable) {
  g_on = enable != 0;
  g_rec.clear();
  g_used = 0;
  return PSF_OK;
}

extern "C" int psf_kernel_timing_read(int kernel_class, int* launches,
                                      double* total_ms) {
  if (kernel_class < 0 || kernel_class >= kTimingClasses) return PSF_ERR_ARG;
  int n = 0;
  double ms = 0.0;
  for (const Record& r : g_rec) {
    if (r.cls != kernel_class) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return PSF_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return PSF_ERR_CUDA;
    ms += t;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return PSF_OK;
}
