// The fused step kernels of SRD (Eq. 2, with the MBS thermostat of Eqs. 5-7): every brick tier,
// floating-point and fixed-point sums, single-box and packed launches.
#include "mpc_step.cuh"

namespace mpc {
template cudaError_t configure_variant<0>(int);
template void launch_variant<0>(const StepArgs&, size_t, cudaStream_t);
template cudaError_t packed_occupancy_variant<0>(int, bool, size_t, int*);
template void launch_packed_variant<0>(const PackTable&, int, bool, int, size_t, cudaStream_t);
}  // namespace mpc
