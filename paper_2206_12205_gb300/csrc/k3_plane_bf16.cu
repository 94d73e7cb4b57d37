// K3, BF16 path (Sec. 3): placeholder until the tensor-core kernel lands.
#include "fdas_internal.cuh"

namespace fdas {

cudaError_t launch_plane_bf16(const Plan &, const float2 *, const float *, char *, __nv_bfloat16 *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace fdas
