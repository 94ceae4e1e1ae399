// BF16 tensor-core forward path (tcgen05 + TMEM + TMA).  Placeholder until the
// fused kernel lands.
#include "gwe_internal.h"

namespace gwe {

bool bf16_supported(const Dims &d) { (void)d; return false; }

gwe_status bf16_prepare(gwe_model *m, const float *host_blob) {
    (void)m; (void)host_blob;
    set_error("BF16 path not built yet");
    return GWE_ERR_UNSUPPORTED;
}

void bf16_release(gwe_model *m) { (void)m; }

gwe_status bf16_forward(gwe_model *m, const float *, const float *, int64_t, int, int, int64_t, const int32_t *, int,
                        float *, bool, cudaStream_t) {
    (void)m;
    set_error("BF16 path not built yet");
    return GWE_ERR_UNSUPPORTED;
}

}  // namespace gwe
