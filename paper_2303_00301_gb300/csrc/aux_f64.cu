// Double-precision instantiations of the sampler kernels (padded dimension <= 16).
#include "aux_ops.cuh"

const AuxOps *aux_ops_f64(int DP) {
  switch (DP) {
    case 4: return auxk::Ops<double, 4>::table();
    case 8: return auxk::Ops<double, 8>::table();
    case 16: return auxk::Ops<double, 16>::table();
    default: return nullptr;
  }
}
