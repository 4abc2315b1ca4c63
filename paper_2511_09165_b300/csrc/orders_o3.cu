// Every-order beamform kernels up to order 3 (both delay modes, all
// Newton-Girard precisions), instantiated in their own translation unit.
#include "dmas_orders.cuh"

namespace dmas {
template cudaError_t launch_orders<3>(const OrdersParams &, int, int, unsigned, size_t,
                                        cudaStream_t);
}  // namespace dmas
