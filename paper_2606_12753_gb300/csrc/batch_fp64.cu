// Persistent batch-kernel instantiations and launchers for the fp64 form.
#define MHD_UNIT_PREC P_FP64
#define MHD_UNIT_FN(name) name##_fp64
#define MHD_BATCH_TILES(X) X(16, 8) X(8, 8)
#include "batch_unit.cuh"
