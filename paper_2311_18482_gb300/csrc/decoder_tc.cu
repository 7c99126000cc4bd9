// Fused BF16 tensor-core decoder and query (tcgen05).  Placeholder until the
// kernel lands: the entry points answer LE_ERR_UNSUPPORTED.
#include "common.cuh"

namespace leg {

size_t decode_fused_workspace(int32_t, const le_decoder*) { return 0; }
size_t query_fused_workspace(int32_t, int32_t, int32_t) { return 0; }

le_status check_fused_decoder(const le_decoder* d, bool train)
{
    (void)d;
    (void)train;
    set_error("fused decoder not available");
    return LE_ERR_UNSUPPORTED;
}

le_status decode_fused(int32_t, const float*, const float*, const le_decoder*, const int32_t*, float, float, float*,
                       float*, float*, const le_decoder_grads*, int32_t*, float*, void*, size_t, cudaStream_t)
{
    set_error("fused decoder not available");
    return LE_ERR_UNSUPPORTED;
}

le_status query_fused(int32_t, const float*, const le_decoder*, const float*, int32_t, int32_t, const float*, int32_t,
                      const float*, int32_t, float*, void*, size_t, cudaStream_t)
{
    set_error("fused query not available");
    return LE_ERR_UNSUPPORTED;
}

}  // namespace leg
