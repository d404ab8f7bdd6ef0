// Kernel instantiations for f64 population storage.
#include "oreg_aux.cuh"
#include "oreg_batch_kernels.cuh"
#include "oreg_kernels.cuh"

OREG_DEFINE_LAUNCHERS(f64, oreg::ST_F64)
OREG_DEFINE_BATCH_LAUNCHERS(f64, oreg::ST_F64)
