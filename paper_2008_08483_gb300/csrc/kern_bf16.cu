// kern_bf16.cu -- split-BF16 tensor-core source term (tcgen05).  Not built yet.
#include "chem_internal.h"

namespace chem {

chem_status bf16_build_tables(chem_mech *, const chem_mech_desc *) { return CHEM_EUNSUPPORTED; }
void bf16_free_tables(void *) {}

chem_status launch_source_bf16(const chem_mech *, int64_t, const float *, const float *,
                               const float *, int64_t, float *, int64_t, cudaStream_t)
{
    return set_error(CHEM_EUNSUPPORTED, "split-BF16 path not built");
}

}  // namespace chem
