// Translation unit of the tensor-core Gram-form kernel (cd_frame_tc.cuh) for c64 storage:
// instantiation for clusters of 16 or 32 antennas and each mode (TDD frame, uplink alone, downlink
// alone, learned uplink), and dispatch of every tensor-core plan: the warp-specialized kernel
// (gram_frame_ws.cu) where it takes the call, else this phased kernel (16-bit storage:
// gram_frame_tc16.cu).
#include "cd_frame_tc.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

template <int MODE>
int dispatch_mode(const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (pl.A_uniform) {
    case 1: return launch_persistent(cd_frame_tc_kernel<16, MODE, CDMIMO_C64>, pl, io, s);
    case 2: return launch_persistent(cd_frame_tc_kernel<32, MODE, CDMIMO_C64>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

}  // namespace

int dispatch_frame_tc(int in_dtype, const CdPlan& pl, const FusedIO& io, int op, cudaStream_t s)
{
    // the warp-specialized kernel where it takes the call: static schedule only (with the schedule
    // counters of a workspace the phased kernel's CTAs draw subcarriers from them)
    if (!pl.learned && !pl.phased && !io.d.sched) {
        const int rc = dispatch_frame_ws(in_dtype, pl, io, op, s);
        if (rc != CDMIMO_ERR_UNSUPPORTED) return rc;
    }
    if (in_dtype != CDMIMO_C64) return dispatch_frame_tc16(in_dtype, pl, io, op, s);
    switch (op) {
    case CDMIMO_OP_FRAME: return dispatch_mode<kTcFrame>(pl, io, s);
    case CDMIMO_OP_DETECT: return pl.learned ? dispatch_mode<kTcDetectLearned>(pl, io, s) : dispatch_mode<kTcDetect>(pl, io, s);
    case CDMIMO_OP_PRECODE: return dispatch_mode<kTcPrecode>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int frame_tc_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
