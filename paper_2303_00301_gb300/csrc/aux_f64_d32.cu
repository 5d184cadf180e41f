// Double-precision instantiation of the sampler kernels for padded dimension 32.
#include "aux_ops.cuh"
const AuxOps *aux_ops_f64_d32() { return auxk::Ops<double, 32>::table(); }
