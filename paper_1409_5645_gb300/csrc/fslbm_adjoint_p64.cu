// fslbm_adjoint_p64.cu -- the adjoint's reverse sweep for the FP64 form.
#include "fslbm_adjoint.cuh"

template int adj_objective<P64>(fslbm* h, double* J, double* norm);
template int adj_backward<P64>(fslbm* h);
