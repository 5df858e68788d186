// Gram-form uplink kernels' translation unit: template instantiation and dispatch over storage
// type, lanes per tile (AT in {1, 2, 4}), padded users (UT in {8, 16}) and learned sweeps.
#include "cd_gram.cuh"
#include "launch.h"

namespace cdmimo {

namespace {

template <int IN, bool LEARNED>
int detect_gram_t(const CdPlan& pl, const DetectIO& io, cudaStream_t s)
{
    switch (pl.A_uniform * 100 + pl.UT) {
    case 108: return launch_persistent(cd_detect_gram_kernel<IN, 1, 8, LEARNED>, pl, io, s);
    case 116: return launch_persistent(cd_detect_gram_kernel<IN, 1, 16, LEARNED>, pl, io, s);
    case 208: return launch_persistent(cd_detect_gram_kernel<IN, 2, 8, LEARNED>, pl, io, s);
    case 216: return launch_persistent(cd_detect_gram_kernel<IN, 2, 16, LEARNED>, pl, io, s);
    case 408: return launch_persistent(cd_detect_gram_kernel<IN, 4, 8, LEARNED>, pl, io, s);
    case 416: return launch_persistent(cd_detect_gram_kernel<IN, 4, 16, LEARNED>, pl, io, s);
    }
    return CDMIMO_ERR_UNSUPPORTED;
}

}  // namespace

int dispatch_detect_gram(int in_dtype, const CdPlan& pl, const DetectIO& io, cudaStream_t s)
{
    if (pl.learned)  // learned blocks: 64-bit complex storage only (checked by the caller)
        return in_dtype == CDMIMO_C64 ? detect_gram_t<CDMIMO_C64, true>(pl, io, s) : CDMIMO_ERR_UNSUPPORTED;
    switch (in_dtype) {
    case CDMIMO_C64: return detect_gram_t<CDMIMO_C64, false>(pl, io, s);
    case CDMIMO_C16F: return detect_gram_t<CDMIMO_C16F, false>(pl, io, s);
    case CDMIMO_C16BF: return detect_gram_t<CDMIMO_C16BF, false>(pl, io, s);
    }
    return CDMIMO_ERR_INVALID_ARG;
}

int gram_detect_module_status(unsigned* v, int clear) { return module_status(v, clear); }

}  // namespace cdmimo
