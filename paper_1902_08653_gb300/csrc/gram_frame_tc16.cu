// Translation unit of the tensor-core Gram-form kernel (cd_frame_tc.cuh) for fp16 / bf16 storage:
// instantiation for clusters of 16 or 32 antennas and the TDD frame, uplink and downlink modes, and
// dispatch.
#include "cd_frame_tc.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

template <int MODE, int IN>
int dispatch_mode16(const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (pl.A_uniform) {
    case 1: return launch_persistent(cd_frame_tc_kernel<16, MODE, IN>, pl, io, s);
    case 2: return launch_persistent(cd_frame_tc_kernel<32, MODE, IN>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

template <int IN>
int dispatch_op16(const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    if (pl.learned) return CDMIMO_ERR_UNSUPPORTED;
    switch (op) {
    case CDMIMO_OP_FRAME: return dispatch_mode16<kTcFrame, IN>(pl, io, s);
    case CDMIMO_OP_DETECT: return dispatch_mode16<kTcDetect, IN>(pl, io, s);
    case CDMIMO_OP_PRECODE: return dispatch_mode16<kTcPrecode, IN>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

}  // namespace

int dispatch_frame_tc16(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    switch (in_dtype) {
    case CDMIMO_C16F: return dispatch_op16<CDMIMO_C16F>(pl, io, op, s);
    case CDMIMO_C16BF: return dispatch_op16<CDMIMO_C16BF>(pl, io, op, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int frame_tc16_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
