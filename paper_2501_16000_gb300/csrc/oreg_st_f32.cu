// Kernel instantiations for f32 population storage.
#include "oreg_aux.cuh"
#include "oreg_batch_kernels.cuh"
#include "oreg_kernels.cuh"

OREG_DEFINE_LAUNCHERS(f32, oreg::ST_F32)
OREG_DEFINE_BATCH_LAUNCHERS(f32, oreg::ST_F32)
