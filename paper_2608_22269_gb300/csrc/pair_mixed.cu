// pair_mixed.cu -- placeholder until the mixed-precision pair pass lands.
#include "../../include/wbsph.h"
#include "common.cuh"

namespace wbsph {
int launch_mixed_stage(const Params&, const State&, const Work&, int64_t, int64_t, int, cudaStream_t) {
  return WBSPH_E_NOSYM;
}
}  // namespace wbsph
