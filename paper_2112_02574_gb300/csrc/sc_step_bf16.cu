// Step-kernel instantiations: BF16 deviation storage, FP32 collision.
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_bf16(const StepLaunch &l, const StepArgs<float> &a) {
  return launch_any<__nv_bfloat16, float>(l, a);
}
