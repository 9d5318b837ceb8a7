// Double-word full-row stage kernels with the registers capped for five, six or eight
// resident blocks per SM (stage_ff_rows.cuh).
#include "stage_ff_rows.cuh"

namespace bssn {

template cudaError_t launch_ff_rows<4, 1, 5>(const Grid&, const StageArgsFF&, cudaStream_t);
template cudaError_t launch_ff_rows<4, 1, 6>(const Grid&, const StageArgsFF&, cudaStream_t);
template cudaError_t launch_ff_rows<4, 1, 8>(const Grid&, const StageArgsFF&, cudaStream_t);

}  // namespace bssn
