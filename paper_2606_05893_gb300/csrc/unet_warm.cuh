// unet_warm.cuh -- the warm start of the Poisson solve by the U-Net, as called
// from the PIC step (pic_api.cu).
#pragma once
#include <cuda_runtime.h>

struct unet_handle;

namespace unet {

// Where the initial guess lives: the FP64 store's unknown view of phi and the
// right-hand side b over the unknowns; or the mixed store's FP32 hi (unknown
// view of phi32), lo and charge term f.
struct WarmTarget {
  double* x64 = nullptr;
  const double* b64 = nullptr;
  float* hi = nullptr;
  const float* lo = nullptr;
  const float* f32 = nullptr;
};

bool warm_matches(const unet_handle* n, int nx, int ny, int nz);
// x0 = x + s f(r / s, ramp), enqueued on st (capturable: no host synchronisation)
cudaError_t warm_start(unet_handle* n, const WarmTarget& w, cudaStream_t st);

}  // namespace unet
