// Kernels for KMV3tet: dim 3, 32 nodes, 28 of them shared (vertex/edge/face).
#include "fwi_internal.h"

namespace fwi {
namespace {
constexpr int D = 3, NN = 32, NS = 28;
__constant__ float c_dhat[D * NN * NN];
__constant__ float c_w[NN];
}  // namespace
}  // namespace fwi

#include "step_kernel.cuh"
#include "chunk_kernel.cuh"

namespace fwi {
namespace {
__global__ void __launch_bounds__(128) k_step(const StepArgs a) { step_body<D, NN, NS>(a); }

__global__ void __launch_bounds__(128) k_chunk(const StepArgs a) {
  extern __shared__ float smem[];
  chunk_body<D, NN, NS>(a, smem);
}

int launch_chunk(const StepArgs& a, cudaStream_t st) {
  const bool grad = a.mode == 1 && a.ring_u != nullptr;
  const bool layer = a.E0 < a.E;
  const size_t bytes = chunk_smem_floats(a.L_max, a.SG, D, grad, layer) * sizeof(float);
  if (bytes > 227 * 1024) return (int)cudaErrorInvalidValue;
  static size_t configured[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (bytes > 48 * 1024 && dev < 64 && bytes > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    configured[dev] = bytes;
  }
  dim3 grid((unsigned)a.nch, (unsigned)(a.S / a.SG));
  k_chunk<<<grid, a.PE * a.SG, bytes, st>>>(a);
  return 0;
}

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

extern const KernelSet kernels_3_3 = {D, 3, NN, NS, NN - NS, upload, launch_step, launch_chunk, launch_record};
}  // namespace fwi
