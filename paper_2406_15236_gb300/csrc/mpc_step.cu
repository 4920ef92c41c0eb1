// Host side of the fused MPC step: dispatch to the per-variant kernels (compiled in
// mpc_step_srd.cu, mpc_step_at_a.cu and mpc_step_srd_a.cu from mpc_step.cuh) and the
// small kernels that close a step.
#include "mpc_step.cuh"

namespace mpc {

#define MPC_VARIANT_ENTRY_POINTS(V)                                                              \
  extern template cudaError_t configure_variant<V>(int);                                          \
  extern template void launch_variant<V>(const StepArgs&, size_t, cudaStream_t);                  \
  extern template cudaError_t packed_occupancy_variant<V>(int, bool, size_t, int*);               \
  extern template void launch_packed_variant<V>(const PackTable&, int, bool, int, size_t, cudaStream_t);
MPC_VARIANT_ENTRY_POINTS(0)
MPC_VARIANT_ENTRY_POINTS(1)
MPC_VARIANT_ENTRY_POINTS(2)
#undef MPC_VARIANT_ENTRY_POINTS

// Closes a step of one box: reduces the observables partials into the ring, advances
// the step counter (up to its limit) and stops the chain after an overflow.  Runs on one
// block of kObsSlots threads.
__device__ __forceinline__ void advance_box(const StepArgs& a) {
  __shared__ int32_t s_skip;
  __shared__ int64_t s_step;
  if (threadIdx.x == 0) {
    const int64_t st = *(volatile int64_t*)&a.ctrl->step;
    const int64_t lim = *(volatile int64_t*)&a.ctrl->limit;
    s_skip = *(volatile int32_t*)&a.ctrl->halted || st >= lim;
    s_step = st;
  }
  __syncthreads();
  if (s_skip) return;
  if (a.g.obs) {
    const int q = threadIdx.x;
    if (q < kObsWidth) {
      double s = 0.0;
      if (a.g.det) {
        long long t = 0;
        for (int k = 0; k < kObsSlots; ++k)
          t += reinterpret_cast<const long long*>(a.obs_partials)[k * kObsWidth + q];
        s = (double)t * kObsUnFx;
      } else {
        for (int k = 0; k < kObsSlots; ++k) s += a.obs_partials[k * kObsWidth + q];
      }
      double* row = a.obs_series + (size_t)(s_step % a.obs_ring) * kObsWidth;
      row[q] = (q == 13) ? (double)(s_step + 1) : s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kObsSlots * kObsWidth; k += blockDim.x) a.obs_partials[k] = 0.0;
  }
  if (threadIdx.x == 0) {
    a.ctrl->step = s_step + 1;
    if (*(volatile int32_t*)&a.ctrl->overflow) a.ctrl->halted = 1;
  }
}

__global__ void k_advance(const StepArgs a) { advance_box(a); }

__global__ void k_advance_batch(const BatchTable* __restrict__ t) {
  const int nboxes = t->nboxes;
  for (int k = blockIdx.x; k < nboxes; k += gridDim.x) {
    advance_box(t->args[k]);
    __syncthreads();
  }
}

// stores v at p (a step limit) in stream order
__global__ void k_store_i64(int64_t* p, int64_t v) { *p = v; }

size_t step_smem_bytes(const Geom& g) {
  if (g.variant == 0) return layout_for<0>(g).total;
  if (g.variant == 1) return layout_for<1>(g).total;
  return layout_for<2>(g).total;
}

// The dynamic shared-memory cap is a per-function attribute shared by every box in the
// process: it is set once to the device's limit (the launch's own size still decides
// occupancy), so boxes with different needs never lower each other's cap.
cudaError_t configure_step_kernels(size_t max_dynamic_smem) {
  const int v = (int)max_dynamic_smem;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = configure_variant<0>(v);
  if (e == cudaSuccess) e = configure_variant<1>(v);
  if (e == cudaSuccess) e = configure_variant<2>(v);
  return e;
}

cudaError_t launch_step(const StepArgs& a, cudaStream_t s) {
  const size_t bytes = step_smem_bytes(a.g);
  if (a.g.variant == 0) launch_variant<0>(a, bytes, s);
  else if (a.g.variant == 1) launch_variant<1>(a, bytes, s);
  else launch_variant<2>(a, bytes, s);
  return cudaGetLastError();
}

cudaError_t launch_advance(const StepArgs& a, cudaStream_t s) {
  k_advance<<<1, kObsSlots, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_store_i64(int64_t* p, int64_t v, cudaStream_t s) {
  k_store_i64<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t packed_kernel_occupancy(int variant, int tier, bool det, size_t smem_bytes, int* ctas_per_sm) {
  if (variant == 0) return packed_occupancy_variant<0>(tier, det, smem_bytes, ctas_per_sm);
  if (variant == 1) return packed_occupancy_variant<1>(tier, det, smem_bytes, ctas_per_sm);
  return packed_occupancy_variant<2>(tier, det, smem_bytes, ctas_per_sm);
}

cudaError_t launch_step_packed(const PackTable& t, int variant, int tier, bool det, int grid,
                               size_t smem_bytes, cudaStream_t s) {
  if (variant == 0) launch_packed_variant<0>(t, tier, det, grid, smem_bytes, s);
  else if (variant == 1) launch_packed_variant<1>(t, tier, det, grid, smem_bytes, s);
  else launch_packed_variant<2>(t, tier, det, grid, smem_bytes, s);
  return cudaGetLastError();
}

int brick_tier(const Geom& g) { return tier_of(g); }

cudaError_t launch_advance_batch(const BatchTable* t, int grid, cudaStream_t s) {
  k_advance_batch<<<grid, kObsSlots, 0, s>>>(t);
  return cudaGetLastError();
}

}  // namespace mpc
