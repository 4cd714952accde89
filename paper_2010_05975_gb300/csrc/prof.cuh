// RAII scope that brackets one kernel launch with CUDA events while a
// profiling session is open (lu_prof_begin / lu_prof_end).
#pragma once
#include "common.cuh"

namespace lu {

void count_launches(int n);

class ProfScope {
  public:
    ProfScope(int cls, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int cls_;
    cudaStream_t s_;
    double flops_, bytes_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace lu
