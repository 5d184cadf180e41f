// Double-precision instantiations of the sampler kernels (padded dimension <= 16;
// the 32-wide instantiation lives in aux_f64_d32.cu so the two compile in parallel).
#include "aux_ops.cuh"

const AuxOps *aux_ops_f64_d32();

const AuxOps *aux_ops_f64(int DP) {
  switch (DP) {
    case 4: return auxk::Ops<double, 4>::table();
    case 8: return auxk::Ops<double, 8>::table();
    case 16: return auxk::Ops<double, 16>::table();
    case 32: return aux_ops_f64_d32();
    default: return nullptr;
  }
}
