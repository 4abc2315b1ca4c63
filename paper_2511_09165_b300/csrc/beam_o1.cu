// Beamform kernels of order n = 1 (all delay modes, channel types and
// Newton-Girard precisions), instantiated in their own translation unit.
#include "dmas_launch.cuh"

namespace dmas {
template cudaError_t launch_beamform_order<1>(const BeamParams &, int, int, int, unsigned,
                                               size_t, cudaStream_t);
template cudaError_t launch_beamform_batch_order<1>(const BeamBatch &, int, int, int,
                                                     unsigned, size_t, cudaStream_t);
}  // namespace dmas
