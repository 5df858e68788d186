// Translation unit of the tensor-core TDD frame kernel (cd_frame_tc.cuh): instantiation for
// clusters of 16 or 32 antennas and dispatch.
#include "cd_frame_tc.cuh"
#include "launch.h"

namespace cdmimo {

int dispatch_frame_tc(const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (pl.A_uniform) {
    case 1: return launch_persistent(cd_frame_tc_kernel<16>, pl, io, s);
    case 2: return launch_persistent(cd_frame_tc_kernel<32>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

int frame_tc_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
