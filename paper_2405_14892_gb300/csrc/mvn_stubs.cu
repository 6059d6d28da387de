// mvn_stubs.cu -- entry points declared in mvn.h whose kernels are not built yet.
#include "mvn_internal.cuh"

