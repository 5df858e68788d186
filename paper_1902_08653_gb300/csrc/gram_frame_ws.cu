// Translation unit of the warp-specialized tensor-core kernel (cd_frame_ws.cuh) for c64 storage:
// the shared-memory layout, instantiation for clusters of 16 or 32 antennas and the TDD frame,
// uplink and downlink modes, and dispatch (16-bit storage: gram_frame_ws16.cu).
#include "cd_frame_ws.cuh"
#include "launch.h"
#include "ws_launch.h"

namespace cdmimo {

int dispatch_frame_ws(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    if (in_dtype != CDMIMO_C64) return dispatch_frame_ws16(in_dtype, pl, io, op, s);
    return ws_dispatch_op<CDMIMO_C64>(pl, io, op, s);
}

int frame_ws_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
