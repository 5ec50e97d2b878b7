// profile.cuh -- stage timing scopes (see profile.cu).
#pragma once
#include <cuda_runtime.h>

namespace ct {

bool prof_on();
// Adds the stages recorded by this thread to the table (waits for their events).
void prof_flush();

class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    cudaStream_t s_;
    bool active_;
    int idx_ = -1;
};

}  // namespace ct
