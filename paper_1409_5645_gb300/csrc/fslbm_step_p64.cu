// fslbm_step_p64.cu -- the step's stream-collide kernels for the FP64 form.
#include "fslbm_step.cuh"

namespace fsl {

template int launch_step_kernels<P64>(const Par&, const View<P64>&, cudaStream_t, int, int, int*, int*, void*, int,
                                      const CUtensorMap*, const Fork*);

}  // namespace fsl
