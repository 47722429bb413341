// fslbm_step_p32.cu -- the step's stream-collide kernels for the FP32 form.
#include "fslbm_step.cuh"

namespace fsl {

template int launch_step_kernels<P32>(const Par&, const View<P32>&, cudaStream_t, int, int, int*, int*, void*, int,
                                      const CUtensorMap*, const Fork*);

}  // namespace fsl
