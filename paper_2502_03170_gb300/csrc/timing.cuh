// Kernel classes and the RAII event bracket used by psf_kernel_timing.
#pragma once

#include "psf_common.cuh"

namespace psf {

enum TimingClass {
  kTimePupil = 0,
  kTimeStage1 = 1,
  kTimeStage2 = 2,
  kTimeBesselRadial = 3,
  kTimeBesselEpilogue = 4,
  kTimeAdjoint = 5,
  kTimeSetup = 6,
  kTimingClasses = 7
};

class TimingScope {
 public:
  TimingScope(int cls, cudaStream_t s);
  ~TimingScope();

 private:
  int cls_;
  cudaStream_t s_;
  void* a_;
};

}  // namespace psf
