// tcgen05 (Blackwell 5th-generation tensor core) engine of the two O passes.
#include "common.cuh"
#include "kernels.h"

namespace wssr {

bool tc_supported(int dev) { (void)dev; return false; }

int tc_passA_launch(const void*, int64_t, int64_t, int64_t, const void*, int64_t, int, float*, int*,
                    int, int, int64_t, int*, cudaStream_t, int*) {
  return -1;
}

int tc_passB_launch(const void*, int64_t, int64_t, int64_t, const void*, int64_t, int, const double*,
                    float*, float*, int, int, int64_t, int*, cudaStream_t) {
  return -1;
}

}  // namespace wssr
