// fd_kernels_tma.cuh -- pipelined 3-D stencil kernel (TMA plane ring).
#pragma once

#include "fd_common.cuh"

namespace fdk {

struct TmaPlan {
  const char *name = "none";
};

inline cudaError_t plan_tma(TmaPlan &, const Geom &, int, float *const *, float *, float *,
                            const char **why) {
  *why = "not built";
  return cudaErrorNotSupported;
}

inline cudaError_t launch_tma_step(const TmaPlan &, int, float *, const float *, const float *,
                                   const Coef &, int *, cudaStream_t) {
  return cudaErrorNotSupported;
}

inline void destroy_tma(TmaPlan &) {}

}  // namespace fdk
