// Gram-form uplink + downlink frame kernels' translation unit: template instantiation and dispatch
// over storage type, lanes per tile (AT in {1, 2, 4}) and padded users (UT in {8, 16}).
#include "cd_frame.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

template <int IN>
int frame_gram_t(const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (pl.A_uniform * 100 + pl.UT) {
    case 108: return launch_persistent(cd_frame_gram_kernel<IN, 1, 8>, pl, io, s);
    case 116: return launch_persistent(cd_frame_gram_kernel<IN, 1, 16>, pl, io, s);
    case 208: return launch_persistent(cd_frame_gram_kernel<IN, 2, 8>, pl, io, s);
    case 216: return launch_persistent(cd_frame_gram_kernel<IN, 2, 16>, pl, io, s);
    case 408: return launch_persistent(cd_frame_gram_kernel<IN, 4, 8>, pl, io, s);
    case 416: return launch_persistent(cd_frame_gram_kernel<IN, 4, 16>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

}  // namespace

int dispatch_frame_gram(int in_dtype, const CdPlan& pl, const FusedIO& io, cudaStream_t s)
{
    switch (in_dtype) {
    case CDMIMO_C64: return frame_gram_t<CDMIMO_C64>(pl, io, s);
    case CDMIMO_C16F: return frame_gram_t<CDMIMO_C16F>(pl, io, s);
    case CDMIMO_C16BF: return frame_gram_t<CDMIMO_C16BF>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int gram_frame_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
