// airpf_launch_inst.cu -- the step kernels of one precision, one model and one
// particles-per-thread count.  Compiled once per triple (-DAIRPF_INST_R=float|
// double, -DAIRPF_INST_MODEL=AR1|SV|NGM|LGSSM|TOY, -DAIRPF_INST_PPT=2|4), so the
// instantiations build in parallel.
#include "airpf_step_impl.cuh"

#if !defined(AIRPF_INST_R) || !defined(AIRPF_INST_MODEL) || !defined(AIRPF_INST_PPT)
#error "compile with -DAIRPF_INST_R=<float|double> -DAIRPF_INST_MODEL=<AR1|SV|NGM|LGSSM|TOY|CP> -DAIRPF_INST_PPT=<2|4>"
#endif

namespace airpf {

template cudaError_t dispatch_inst<AIRPF_INST_R, AIRPF_INST_MODEL, AIRPF_INST_PPT>(const StepParams&, int, cudaStream_t,
                                                                                int, int*);

}  // namespace airpf
