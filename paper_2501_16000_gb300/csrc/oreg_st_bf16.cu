// Kernel instantiations for bf16 population storage.
#include "oreg_aux.cuh"
#include "oreg_batch_kernels.cuh"
#include "oreg_kernels.cuh"

OREG_DEFINE_LAUNCHERS(bf16, oreg::ST_BF16)
OREG_DEFINE_BATCH_LAUNCHERS(bf16, oreg::ST_BF16)
