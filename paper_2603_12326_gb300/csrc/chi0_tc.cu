// Mixed-precision chi0 on the tcgen05 tensor cores (placeholder until the kernel lands).
#include "qcx_internal.h"

cudaError_t qcx_launch_chi0_mixed(qcx_ctx*, QSlot&, int, double2*, int*) { return cudaErrorNotSupported; }
