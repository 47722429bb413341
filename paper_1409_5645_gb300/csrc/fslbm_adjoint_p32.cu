// fslbm_adjoint_p32.cu -- the adjoint's reverse sweep for the FP32 form.
#include "fslbm_adjoint.cuh"

template int adj_objective<P32>(fslbm* h, double* J, double* norm);
template int adj_backward<P32>(fslbm* h);
