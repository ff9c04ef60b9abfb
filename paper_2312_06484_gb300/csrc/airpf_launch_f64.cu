// airpf_launch_f64.cu -- the double instantiations of the AIRPF step kernels.
#include "airpf_step_impl.cuh"

namespace airpf {

cudaError_t dispatch_f64(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    return dispatch_typed<double>(p, t, stream, op, fits);
}

}  // namespace airpf
