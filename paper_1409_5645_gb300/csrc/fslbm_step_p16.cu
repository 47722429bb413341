// fslbm_step_p16.cu -- the step's stream-collide kernels for the FP16-storage form.
#include "fslbm_step.cuh"

namespace fsl {

template int launch_step_kernels<P16>(const Par&, const View<P16>&, cudaStream_t, int, int, int*, int*, void*, int,
                                      const CUtensorMap*, const Fork*);

}  // namespace fsl
