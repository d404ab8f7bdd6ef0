// Kernel instantiations for f16 population storage.
#include "oreg_aux.cuh"
#include "oreg_batch_kernels.cuh"
#include "oreg_kernels.cuh"

OREG_DEFINE_LAUNCHERS(f16, oreg::ST_F16)
OREG_DEFINE_BATCH_LAUNCHERS(f16, oreg::ST_F16)
