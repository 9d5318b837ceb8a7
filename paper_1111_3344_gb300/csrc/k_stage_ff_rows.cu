// Double-word full-row stage kernels, one block per SM's worth of registers
// (stage_ff_rows.cuh).
#include "stage_ff_rows.cuh"

namespace bssn {

template cudaError_t launch_ff_rows<4, 1, 1>(const Grid&, const StageArgsFF&, cudaStream_t);
template cudaError_t launch_ff_rows<8, 1, 1>(const Grid&, const StageArgsFF&, cudaStream_t);
template cudaError_t launch_ff_rows<4, 2, 1>(const Grid&, const StageArgsFF&, cudaStream_t);

}  // namespace bssn
