// Translation unit of the tensor-core Gram-form kernel (cd_frame_tc.cuh): instantiation for
// clusters of 16 or 32 antennas and each mode (TDD frame, uplink alone, downlink alone, learned
// uplink), and dispatch.
#include "cd_frame_tc.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

template <int MODE>
int dispatch_mode(const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (pl.A_uniform) {
    case 1: return launch_persistent(cd_frame_tc_kernel<16, MODE>, pl, io, s);
    case 2: return launch_persistent(cd_frame_tc_kernel<32, MODE>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

}  // namespace

int dispatch_frame_tc(const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    switch (op) {
    case CDMIMO_OP_FRAME: return dispatch_mode<kTcFrame>(pl, io, s);
    case CDMIMO_OP_DETECT: return pl.learned ? dispatch_mode<kTcDetectLearned>(pl, io, s) : dispatch_mode<kTcDetect>(pl, io, s);
    case CDMIMO_OP_PRECODE: return dispatch_mode<kTcPrecode>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int frame_tc_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
