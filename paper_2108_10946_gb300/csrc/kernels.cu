// Dimension-generic kernels: the shared-DoF update, the FP64 compensated gradient fold,
// the final M^-1 scaling and mask of Eq. (gradient3), and the misfit reduction.
#include <algorithm>

#include "update.cuh"

namespace fwi {

extern const KernelSet kernels_2_2, kernels_2_3, kernels_2_4, kernels_2_5, kernels_3_2,
    kernels_3_3;

const KernelSet* kernel_set(int dim, int k) {
  if (dim == 2) {
    switch (k) {
      case 2: return &kernels_2_2;
      case 3: return &kernels_2_3;
      case 4: return &kernels_2_4;
      case 5: return &kernels_2_5;
    }
  } else if (dim == 3) {
    switch (k) {
      case 2: return &kernels_3_2;
      case 3: return &kernels_3_3;
    }
  }
  return nullptr;
}

void launch_node_update(const StepArgs& a, int dim, cudaStream_t st) {
  const int bs = 256;
  if (a.S % 4 == 0) {  // one thread per (DoF, four shots)
    const int64_t items4 = (int64_t)a.hcnt * (a.S / 4);
    if (items4 == 0) return;
    const unsigned blocks4 = (unsigned)((items4 + bs - 1) / bs);
    if (dim == 2)
      node_kernel4<2><<<blocks4, bs, 0, st>>>(a);
    else
      node_kernel4<3><<<blocks4, bs, 0, st>>>(a);
    return;
  }
  const int64_t items = (int64_t)a.hcnt * a.S;
  if (items == 0) return;
  const unsigned blocks = (unsigned)((items + (int64_t)bs * NODE_ITEMS - 1) / ((int64_t)bs * NODE_ITEMS));
  if (dim == 2)
    node_kernel<2><<<blocks, bs, 0, st>>>(a);
  else
    node_kernel<3><<<blocks, bs, 0, st>>>(a);
}

// Kahan fold of the FP32 segment sum into (sum, comp); comp carries the lost low part
// with the sign convention sum - comp ~ exact.
__global__ void fold_kernel(float* __restrict__ gseg, double* __restrict__ gsum,
                            double* __restrict__ gcomp, int64_t N, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double x = scale * (double)gseg[i];  // scale: the subsampling weight r
  gseg[i] = 0.f;
  const double s = gsum[i];
  const double y = x - gcomp[i];
  const double t = s + y;
  gcomp[i] = (t - s) - y;
  gsum[i] = t;
}

void launch_fold(float* gseg, double* gsum, double* gcomp, int64_t N, double scale,
                 cudaStream_t st) {
  if (N == 0) return;
  fold_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(gseg, gsum, gcomp, N, scale);
}

// G = M^-1 g (Eq. gradient3) from the per-shot compensated sums (sum, comp) [lanes][N]: the
// sum over the lanes (out [N]) or each lane's own (out [lanes][N]); zero where masked.
__global__ void finish_kernel(const double* __restrict__ gsum, const double* __restrict__ gcomp,
                              const double* __restrict__ M, const unsigned char* __restrict__ mask,
                              double* __restrict__ out, int64_t N, int lanes, int per_lane) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // M == nullptr: the raw discrete derivative dJ/dc (no division by the lumped mass)
  const double scale = M ? 1.0 / M[i] : 1.0;
  const bool keep = mask[i] != 0;
  double total = 0.0;
  for (int s = 0; s < lanes; ++s) {
    const double g = gsum[(size_t)s * N + i] - gcomp[(size_t)s * N + i];
    if (per_lane)
      out[(size_t)s * N + i] = keep ? (M ? g / M[i] : g) : 0.0;
    else
      total += g;
  }
  if (!per_lane) out[i] = keep ? total * scale : 0.0;
}

void launch_finish_gradient(const double* gsum, const double* gcomp, const float*,
                            const double* M, const unsigned char* mask, double* out, int64_t N,
                            int lanes, int per_lane, cudaStream_t st) {
  if (N == 0) return;
  finish_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(gsum, gcomp, M, mask, out, N, lanes,
                                                              per_lane);
}

// acc[lane] += 1/2 sum resid^2 over each lane's n values (block reduction in FP64, one
// atomic per block; blockIdx.y is the lane)
__global__ void misfit_kernel(const float* __restrict__ r, int64_t n, double* acc) {
  __shared__ double part[256];
  const float* rl = r + (size_t)blockIdx.y * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = rl[i];
    s += x * x;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc + blockIdx.y, 0.5 * part[0]);
}

// Zeroes the lanes named by mask (bit s = lane s) of a [rows][S] state array, S a power of
// two: the lanes that start a new shot.
__global__ void lane_reset_kernel(float* __restrict__ p, int64_t n, int S, uint32_t mask) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if ((mask >> (int)(i & (S - 1))) & 1u) p[i] = 0.f;
}

void launch_lane_reset(float* p, int64_t rows, int S, uint32_t mask, cudaStream_t st) {
  const int64_t n = rows * S;
  if (n == 0 || mask == 0) return;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  lane_reset_kernel<<<blocks, 256, 0, st>>>(p, n, S, mask);
}

__global__ void residual_kernel(const float* __restrict__ d, const float* __restrict__ obs,
                                float* __restrict__ res, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) res[i] = d[i] - obs[i];
}

void launch_residual(const float* d, const float* obs, float* res, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, obs, res, n);
}

// FP32 FMA throughput probe: every thread runs 16 independent packed FP32x2 FMA chains
// (the instruction the element kernels use), so that the FMA pipes, not latency, bound it.
// Each ffma2 is two fused multiply-adds, four flops.
__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, int iters, float a) {
  float2 acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
  const float2 m = make_float2(a, a), b = make_float2(1e-7f, -1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      unsigned long long r;
      asm volatile("fma.rn.f32x2 %0, %1, %2, %3;"
                   : "=l"(r)
                   : "l"(*reinterpret_cast<const unsigned long long*>(&acc[c])),
                     "l"(*reinterpret_cast<const unsigned long long*>(&m)),
                     "l"(*reinterpret_cast<const unsigned long long*>(&b)));
      acc[c] = *reinterpret_cast<float2*>(&r);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 16; ++c) s += acc[c].x + acc[c].y;
  if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live
}

int measure_fma_peak(double* tflops, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  int nsm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  float* out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(float) * 4096)) != cudaSuccess) return (int)e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  fma_peak_kernel<<<blocks, threads>>>(out, 64, 0.999f);  // warm-up
  double best = 0;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    fma_peak_kernel<<<blocks, threads>>>(out, iters, 0.999f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = (double)blocks * threads * iters * 16 * 4;
    if (ms > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (tflops) *tflops = best;
  if (sms) *sms = nsm;
  return (int)e;
}

void launch_misfit(const float* resid, int64_t n, int lanes, double* acc, cudaStream_t st) {
  if (n == 0 || lanes == 0) return;
  int blocks = (int)std::min<int64_t>((n + 255) / 256, std::max(1, 1216 / lanes));
  misfit_kernel<<<dim3(blocks, lanes), 256, 0, st>>>(resid, n, acc);
}

}  // namespace fwi
