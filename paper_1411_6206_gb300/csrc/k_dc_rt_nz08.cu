// Register-transform data-consistency update for planes of nz = 8 (k_dc.cuh).
#include "k_dc.cuh"

namespace lps {
template cudaError_t launch_dc_rt_nz<8>(const DcArgs&, size_t, cudaStream_t);
}  // namespace lps
