// The wavefront sweep instantiated for float (mixed path: float state and
// float-float columns; FP64 path: double).  One translation unit per
// precision so the two compile in parallel.
#include "sweep_impl.cuh"

namespace oots {
template bool sweep_shape_ok<float>(int);
template int sweep_occupancy<float>(int, int);
template cudaError_t prepare_sweeps<float>();
template cudaError_t launch_sweep<float>(const SweepParams<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_pack_nx<float>(const GridDev<float> *, int, int, int, long long, int, cudaStream_t);
} // namespace oots
