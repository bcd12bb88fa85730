// The wavefront sweep instantiated for double (mixed path: float state and
// float-float columns; FP64 path: double).  One translation unit per
// precision so the two compile in parallel.
#include "sweep_impl.cuh"

namespace oots {
template bool sweep_shape_ok<double>(int);
template int sweep_occupancy<double>(int, int);
template cudaError_t prepare_sweeps<double>();
template cudaError_t launch_sweep<double>(const SweepParams<double> &, int, int, int, cudaStream_t);
template cudaError_t launch_pack_nx<double>(const GridDev<double> *, int, int, int, long long, int, cudaStream_t);
} // namespace oots
