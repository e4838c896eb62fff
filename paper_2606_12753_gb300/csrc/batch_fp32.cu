// Persistent batch-kernel instantiations and launchers for the fp32 form.
#define MHD_UNIT_PREC P_FP32
#define MHD_UNIT_FN(name) name##_fp32
#define MHD_BATCH_TILES(X) X(16, 8) X(16, 16) X(32, 8) X(24, 8) X(8, 8)
#include "batch_unit.cuh"
