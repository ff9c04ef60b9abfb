// airpf_launch_f32.cu -- the float instantiations of the AIRPF step kernels.
#include "airpf_step_impl.cuh"

namespace airpf {

cudaError_t dispatch_f32(const StepParams& p, int t, cudaStream_t stream, int op, int* fits)
{
    return dispatch_typed<float>(p, t, stream, op, fits);
}

}  // namespace airpf
