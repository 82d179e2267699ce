// Step-kernel instantiations: FP64 deviation storage, FP64 collision (the
// instantiation the parity tests compare with the FP64 oracle most tightly).
#include "sc_step_inst.cuh"
cudaError_t scgb::launch_step_f64(const StepLaunch &l, const StepArgs<double> &a) { return launch_any<double, double>(l, a); }
