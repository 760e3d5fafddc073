// k_tc.cu -- tcgen05 tensor-core screen passes (BF16 in, FP32 accumulate).
#include "../../include/mapper.h"
#include "tc.cuh"

namespace mgb {

int tc_pass(int, const PassArgs&, const TcArgs&, int64_t, cudaStream_t)
{
    set_error("BF16 tensor-core screen not built yet");
    return MAPPER_ENOTIMPL;
}

}  // namespace mgb
