// Tensor-core (tcgen05) grouped GEMM for the split-precision paths.
#include "internal.h"

namespace heff {
int launch_tc_gemm(heff_plan* p, int which, void* ws, void* const* y, int nbatch, void* stream) {
    (void)p; (void)which; (void)ws; (void)y; (void)nbatch; (void)stream;
    return fail(HEFF_ERR_UNSUPPORTED, "tensor-core path not built yet");
}
}  // namespace heff
