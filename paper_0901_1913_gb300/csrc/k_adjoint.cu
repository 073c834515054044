// k_adjoint.cu -- exact gradients and Newton refinement at peaks (filled in below).
#include "fc2_common.cuh"
#include "fc2_internal.h"
