// Single-precision instantiation of the sampler kernels for padded dimension 32.
#include "aux_ops.cuh"

const AuxOps *aux_ops_f32_d32() { return auxk::Ops<float, 32>::table(); }
