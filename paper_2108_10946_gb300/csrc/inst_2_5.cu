// Kernels for KMV5tri: dim 2, 30 nodes, 15 of them shared (vertex/edge/face).
#include "fwi_internal.h"

namespace fwi {
namespace {
constexpr int D = 2, NN = 30, NS = 15;
__constant__ float c_dhat[D * NN * NN];
__constant__ float c_w[NN];
}  // namespace
}  // namespace fwi

#include "step_kernel.cuh"

namespace fwi {
namespace {
__global__ void __launch_bounds__(128) k_step(const StepArgs a) { step_body<D, NN, NS>(a); }

int upload(const float* dhat, const float* w) {
  cudaError_t e = cudaMemcpyToSymbol(c_dhat, dhat, sizeof(float) * D * NN * NN);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w, w, sizeof(float) * NN);
  return (int)e;
}

void launch_step(const StepArgs& a, cudaStream_t st) {
  const int64_t threads = (int64_t)a.E * a.S;
  const int bs = 128;
  k_step<<<(unsigned)((threads + bs - 1) / bs), bs, 0, st>>>(a);
}

void launch_record(const StepArgs& a, const int* rec_elem, const float* rec_phi, cudaStream_t st) {
  const int threads = a.R * a.S;
  if (threads == 0) return;
  record_kernel<NN, NS><<<(threads + 127) / 128, 128, 0, st>>>(a, rec_elem, rec_phi);
}
}  // namespace

extern const KernelSet kernels_2_5 = {D, 5, NN, NS, NN - NS, upload, launch_step, launch_record};
}  // namespace fwi
