// Kernels of one KMV element, instantiated once per (dimension, degree): the build compiles
// this file with -DKMV_DIM=d -DKMV_K=k for KMV2..5tri and KMV2..3tet. Nodes per element:
// triangles 7, 12, 18, 30 (6, 9, 12, 15 of them on vertices and edges); tetrahedra 15, 32
// (14, 28 on vertices, edges and faces).
#include <algorithm>
#include <vector>

#include "fwi_internal.h"

#if !defined(KMV_DIM) || !defined(KMV_K)
#error "compile with -DKMV_DIM=<2|3> -DKMV_K=<degree>"
#endif

namespace fwi {
namespace {
constexpr int D = KMV_DIM;
constexpr int NN = D == 2 ? (KMV_K == 2 ? 7 : KMV_K == 3 ? 12 : KMV_K == 4 ? 18 : 30)
                          : (KMV_K == 2 ? 15 : 32);
constexpr int NS = D == 2 ? 3 * KMV_K : (KMV_K == 2 ? 14 : 28);
static_assert((D == 2 && KMV_K >= 2 && KMV_K <= 5) || (D == 3 && KMV_K >= 2 && KMV_K <= 3),
              "KMV elements: triangles k = 2..5, tetrahedra k = 2, 3");
__constant__ float c_dhat[D * NN * NN];
__constant__ float c_w[NN];
}  // namespace
}  // namespace fwi

#include "step_kernel.cuh"
#include "chunk_kernel.cuh"
#if KMV_DIM == 2
#include "chunk_tc.cuh"
#include "chunk_persist.cuh"
#endif

namespace fwi {
namespace {
#if KMV_DIM == 2
// Dhat as the B operands of the tensor-core kernel (hi and lo, canonical layout)
__device__ __align__(16) float g_bimg[TcShape<D, NN>::BIMG];
#endif

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
  k_chunk<MODE, LAYER><<<grid, a.PE * a.SG * chunk_qsplit<D, NN, MODE, LAYER>(), bytes, st>>>(b);
  return 0;
}

#if KMV_DIM == 2
template <int MODE, bool LAYER>
__global__ void __launch_bounds__(128) k_chunk_tc(const StepArgs a, int nrun) {
  extern __shared__ __align__(128) float smem_tc[];
  chunk_tc_body<D, NN, NS, MODE, LAYER>(a, smem_tc, g_bimg, nrun);
}

// persistent: at most two CTAs per SM (each holds 256 of the SM's 512 tensor-memory
// columns; the shared-memory request is raised so that a third never fits)
template <int MODE, bool LAYER>
int launch_chunk_tc_t(const StepArgs& a, int ch0, int nch, cudaStream_t st) {
  if (nch <= 0) return 0;
  size_t bytes = chunk_tc_smem_floats<D, NN>(a.L_max, a.SG, MODE == 2, LAYER) * sizeof(float);
  if (bytes < 80 * 1024) bytes = 80 * 1024;
  if (bytes > 227 * 1024) return (int)cudaErrorInvalidValue;
  static size_t configured[64] = {0};
  static int nsm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  if (bytes > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_chunk_tc<MODE, LAYER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return (int)e;
    configured[dev] = bytes;
  }
  if (nsm[dev] == 0) {
    cudaError_t e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
  }
  StepArgs b = a;
  b.ch0 = ch0;
  dim3 grid((unsigned)std::min(nch, 2 * nsm[dev]), (unsigned)(a.S / a.SG));
  k_chunk_tc<MODE, LAYER><<<grid, a.PE * a.SG, bytes, st>>>(b, nch);
  return 0;
}

#endif

#if KMV_DIM == 2
template <int MODE>
__global__ void __launch_bounds__(PT_THREADS, 2) k_chunk_pt(const StepArgs a, int nwork) {
  extern __shared__ __align__(16) char smem_pt[];
  pt_body<NN, NS, MODE>(a, smem_pt, nwork);
}

// Persistent pipelined kernel over chunks [ch0, ch0 + nch) (no layer elements), S a
// multiple of 4. Returns -1 (nothing launched) when its shared-memory tables do not fit, a
// cudaError_t on failure, 0 once launched.
template <int MODE>
int launch_chunk_pt_t(const StepArgs& a, int ch0, int nch, cudaStream_t st) {
  if (nch <= 0) return 0;
  const PtLayout L = pt_layout<NN, NS>(a.L_max, a.O_max, a.H_max, MODE == 2);
  if (L.total > 227u * 1024u) return -1;
  static size_t configured[64] = {0};
  static int per_sm[64] = {0}, nsm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  if (L.total > configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_chunk_pt<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.total);
    if (e != cudaSuccess) return (int)e;
    configured[dev] = L.total;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[dev], k_chunk_pt<MODE>, PT_THREADS,
                                                      L.total);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
  }
  if (per_sm[dev] < 1) return -1;
  const int nwork = nch * (a.S / PT_SG);
  StepArgs b = a;
  b.ch0 = ch0;
  const int grid = std::min(nwork, per_sm[dev] * nsm[dev]);
  k_chunk_pt<MODE><<<grid, PT_THREADS, L.total, st>>>(b, nwork);
  return 0;
}
#endif

// chunks [0, nch0) hold no damping-layer element, chunks [nch0, nch) do
int launch_chunk(const StepArgs& a, cudaStream_t st, cudaStream_t stl) {
  const int mode = a.mode == 0 ? 0 : (a.ring_u != nullptr ? 2 : 1);
  int rc = 0;
#if KMV_DIM == 2
  if (a.tc && mode != 0) {  // the adjoint steps only
    switch (mode) {
      case 1:
        rc = launch_chunk_tc_t<1, false>(a, 0, a.nch0, st);
        if (!rc) rc = launch_chunk_tc_t<1, true>(a, a.nch0, a.nch - a.nch0, stl);
        break;
      default:
        rc = launch_chunk_tc_t<2, false>(a, 0, a.nch0, st);
        if (!rc) rc = launch_chunk_tc_t<2, true>(a, a.nch0, a.nch - a.nch0, stl);
    }
    return rc;
  }
#endif
#if KMV_DIM == 2
  // triangles, four shots per work item: the persistent kernel takes the chunks without
  // layer elements in the forward and adjoint steps, and in the gradient steps when the
  // forward recompute stored the forward field's gradients (a.gload; summed gradient form);
  // otherwise the gradient steps and the layer chunks use the chunk kernel. (The persistent
  // kernel's gradient step needs more shared memory than its forward step, so if the forward
  // step fell back to the chunk kernel, which stores nothing, so does the gradient step.)
  if (a.S % PT_SG == 0 && a.nch0 > 0 && (mode != 2 || (a.gload != nullptr && !a.grad_lanes))) {
    rc = mode == 0   ? launch_chunk_pt_t<0>(a, 0, a.nch0, st)
         : mode == 1 ? launch_chunk_pt_t<1>(a, 0, a.nch0, st)
                     : launch_chunk_pt_t<2>(a, 0, a.nch0, st);
    if (rc > 0) return rc;
    if (rc == 0) {
      if (mode == 0) return launch_chunk_t<0, true>(a, a.nch0, a.nch - a.nch0, stl);
      if (mode == 1) return launch_chunk_t<1, true>(a, a.nch0, a.nch - a.nch0, stl);
      return launch_chunk_t<2, true>(a, a.nch0, a.nch - a.nch0, stl);
    }
    rc = 0;  // the tables do not fit: the chunk kernel below takes every chunk
  }
#endif
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
#if KMV_DIM == 2
  if (e == cudaSuccess) {
    std::vector<float> img(TcShape<D, NN>::BIMG);
    tc_build_bimg<D, NN>(dhat, img.data());
    e = cudaMemcpyToSymbol(g_bimg, img.data(), sizeof(float) * img.size());
  }
#endif
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

#define KMV_CAT2(a, b, c, d) a##b##c##d
#define KMV_CAT(a, b, c, d) KMV_CAT2(a, b, c, d)
extern const KernelSet KMV_CAT(kernels_, KMV_DIM, _, KMV_K) = {D,           KMV_K,       NN,
                                                              NS,          NN - NS,     upload,
                                                              launch_step, launch_chunk,
                                                              launch_record};
}  // namespace fwi
