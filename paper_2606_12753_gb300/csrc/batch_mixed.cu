// Persistent batch-kernel instantiations and launchers for the mixed form.
#define MHD_UNIT_PREC P_MIXED
#define MHD_UNIT_FN(name) name##_mixed
#define MHD_BATCH_TILES(X) X(16, 8) X(8, 8)
#include "batch_unit.cuh"
