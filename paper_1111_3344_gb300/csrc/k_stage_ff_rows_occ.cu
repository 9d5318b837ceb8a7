// Double-word full-row stage kernels with the registers capped for three or
// four resident blocks per SM (more warps share each fetched instruction; more
// spills) (stage_ff_rows.cuh).
#include "stage_ff_rows.cuh"

namespace bssn {

template cudaError_t launch_ff_rows<4, 1, 3>(const Grid&, const StageArgsFF&, cudaStream_t);
template cudaError_t launch_ff_rows<4, 1, 4>(const Grid&, const StageArgsFF&, cudaStream_t);

}  // namespace bssn
