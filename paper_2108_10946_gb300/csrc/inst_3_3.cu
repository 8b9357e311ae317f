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

template <int MODE, bool LAYER>
__global__ void __launch_bounds__(128) k_chunk(const StepArgs a) {
  extern __shared__ float smem[];
  chunk_body<D, NN, NS, MODE, LAYER>(a, smem);
}

template <int MODE, bool LAYER>
int launch_chunk_t(const StepArgs& a, int ch0, int nch, cudaStream_t st) {
  if (nch <= 0) return 0;
  const size_t bytes =
      chunk_smem_floats(a.L_max, a.SG, D, MODE == 2, LAYER, NN, NS, a.PE * a.SG) * sizeof(float);
  if (bytes > 227 * 1024) return (int)cudaErrorInvalidValue;
  static size_t configured[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (bytes > 48 * 1024 && dev < 64 && bytes > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_chunk<MODE, LAYER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    configured[dev] = bytes;
  }
  StepArgs b = a;
  b.ch0 = ch0;
  dim3 grid((unsigned)nch, (unsigned)(a.S / a.SG));
  k_chunk<MODE, LAYER><<<grid, a.PE * a.SG, bytes, st>>>(b);
  return 0;
}

// chunks [0, nch0) hold no damping-layer element, chunks [nch0, nch) do
int launch_chunk(const StepArgs& a, cudaStream_t st, cudaStream_t stl) {
  const int mode = a.mode == 0 ? 0 : (a.ring_u != nullptr ? 2 : 1);
  int rc = 0;
  switch (mode) {
    case 0:
      rc = launch_chunk_t<0, false>(a, 0, a.nch0, st);
      if (!rc) rc = launch_chunk_t<0, true>(a, a.nch0, a.nch - a.nch0, stl);
      break;
    case 1:
      rc = launch_chunk_t<1, false>(a, 0, a.nch0, st);
      if (!rc) rc = launch_chunk_t<1, true>(a, a.nch0, a.nch - a.nch0, stl);
      break;
    default:
      rc = launch_chunk_t<2, false>(a, 0, a.nch0, st);
      if (!rc) rc = launch_chunk_t<2, true>(a, a.nch0, a.nch - a.nch0, stl);
  }
  return rc;
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
