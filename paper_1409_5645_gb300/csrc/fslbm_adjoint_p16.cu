// fslbm_adjoint_p16.cu -- the adjoint's reverse sweep for the FP16-storage form.
#include "fslbm_adjoint.cuh"

template int adj_objective<P16>(fslbm* h, double* J, double* norm);
template int adj_backward<P16>(fslbm* h);
