// Translation unit of the warp-specialized tensor-core kernel (cd_frame_ws.cuh) for fp16 / bf16
// storage: instantiation for clusters of 16 or 32 antennas and the TDD frame, uplink and downlink
// modes, and dispatch.
#include "cd_frame_ws.cuh"
#include "launch.h"
#include "ws_launch.h"

namespace cdmimo {

int dispatch_frame_ws16(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    switch (in_dtype) {
    case CDMIMO_C16F: return ws_dispatch_op<CDMIMO_C16F>(pl, io, op, s);
    case CDMIMO_C16BF: return ws_dispatch_op<CDMIMO_C16BF>(pl, io, op, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int frame_ws16_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
