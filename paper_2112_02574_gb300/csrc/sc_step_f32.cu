// Step-kernel instantiations: FP32 deviation storage, FP32 collision.
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_f32(const StepLaunch &l, const StepArgs<float> &a) { return launch_any<float, float>(l, a); }
