// Instantiates the fused step, field and state kernels for scaled FP16 storage with stochastic rounding of the
// population deviations (one translation unit per storage type so they
// compile in parallel).
#include "glbe_kernels.cuh"

namespace glbe {
template cudaError_t launch_step_t<ST_F16_SR>(bool, int, const StepParams&, const StepBuffers&, const FieldOut&,
                                           cudaStream_t, unsigned*);
template cudaError_t launch_get_state_t<ST_F16_SR>(bool, const StepParams&, const void*, const void*, const float*,
                                                float*, float*, float*, cudaStream_t);
template cudaError_t launch_set_state_t<ST_F16_SR>(bool, const StepParams&, void*, void*, float*, const float*,
                                                const float*, const float*, cudaStream_t);
template int tile_wait_error_t<ST_F16_SR>();
}  // namespace glbe
