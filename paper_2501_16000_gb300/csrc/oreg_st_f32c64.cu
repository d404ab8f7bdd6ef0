// Stream-collide instantiation for FP32 storage with the FP64 collision.
#include "oreg_kernels.cuh"

namespace oreg {
cudaError_t step_f32c64(const StepArgs &a) { return StepLaunch<ST_F32_C64>::step(a); }
}  // namespace oreg
