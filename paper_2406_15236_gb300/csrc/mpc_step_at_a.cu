// The fused step kernels of MPC-AT+a (the angular-momentum-conserving MPC the paper cites with Eqs. 3-4): every brick tier,
// floating-point and fixed-point sums, single-box and packed launches.
#include "mpc_step.cuh"

namespace mpc {
template cudaError_t configure_variant<1>(int);
template void launch_variant<1>(const StepArgs&, size_t, cudaStream_t);
template cudaError_t packed_occupancy_variant<1>(int, bool, size_t, int*);
template void launch_packed_variant<1>(const PackTable&, int, bool, int, size_t, cudaStream_t);
}  // namespace mpc
