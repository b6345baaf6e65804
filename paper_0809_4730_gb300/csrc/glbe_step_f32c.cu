// Instantiates the fused step, field and state kernels for compensated FP32 + FP16 storage of the
// population deviations (one translation unit per storage type so they
// compile in parallel).
#include "glbe_kernels.cuh"

namespace glbe {
template cudaError_t launch_step_t<ST_F32C>(bool, int, const StepParams&, const StepBuffers&, const FieldOut&,
                                           cudaStream_t, unsigned*);
template cudaError_t launch_get_state_t<ST_F32C>(bool, const StepParams&, const void*, const void*, const float*,
                                                float*, float*, float*, cudaStream_t);
template cudaError_t launch_set_state_t<ST_F32C>(bool, const StepParams&, void*, void*, float*, const float*,
                                                const float*, const float*, cudaStream_t);
template int tile_wait_error_t<ST_F32C>();
template cudaError_t launch_lid_init_t<ST_F32C>(const StepParams&, void*, cudaStream_t);
}  // namespace glbe
