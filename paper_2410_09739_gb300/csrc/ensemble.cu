// ensemble.cu -- placeholder, replaced by the ensemble implementation.
#include "../../include/fpclbm.h"
#include "internal.h"
extern "C" int fpclbm_create_ensemble(fpclbm_t* out, int, const int*, const double*, int, void*)
{
    if (out) *out = nullptr;
    return FPCLBM_ERR_ARG;
}
