// Chunked time step: one CTA assembles one chunk of consecutive elements (Morton order)
// for a group of up to 4 shots, entirely in shared memory.
//
//   1. load    every global read of the chunk issued at once as asynchronous copies into
//              the chunk table (chunk_io.cuh): its owned DoFs (one contiguous range: its
//              vertex/edge/face DoFs that no other chunk touches, then its elements' bubble
//              DoFs) and its halo DoFs (shared with other chunks, through the halo list);
//   2. element one thread per (element, shot): the same stiffness / layer / gradient
//              arithmetic as the plain kernel (Dhat from the constant bank), gathering from
//              and scattering into shared memory (shared-memory atomics for the element's
//              vertex/edge/face nodes, plain stores for its bubble nodes);
//   3. update  the owned DoFs are final after the chunk's own elements: the increment update
//              runs here with coalesced writes; halo contributions go to global accumulators
//              that the node kernel finishes after all chunks.
//
// Owned DoFs are read and written by this CTA only, so the in-place update is race free;
// halo DoFs are only read here and updated by the node kernel afterwards.
#pragma once
#include "chunk_io.cuh"

namespace fwi {

// d = a * b + c on two FP32 lanes at once (packed FP32x2 FMA of the sm_100 family; each
// lane an IEEE fused multiply-add rounded to nearest). The compiler intrinsic lets the
// register allocator keep the operands in aligned pairs.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Threads per (element, shot): tetrahedra in damping-layer chunks split the node loop
// between two threads, so that a CTA holds twice the threads for the same chunk table (those
// tables, with the layer's auxiliaries, allow two CTAs per SM). The two halves are whole
// warps, each taking every other quadrature node, so constant-bank reads stay warp-uniform.
// Measured on the thrust model at half scale: KMV3 layer steps 34 % (forward) and 31 %
// (adjoint) faster, KMV2 forward steps 5.5 % faster (its adjoint steps were 6 % slower split
// and keep one thread). Chunks without layer elements keep one thread (the split raised
// their registers more than it added threads).
template <int D, int NN, int MODE, bool LAYER>
__host__ __device__ constexpr int chunk_qsplit() { return D == 3 && LAYER && (NN >= 32 || MODE == 0) ? 2 : 1; }

// floats of dynamic shared memory per CTA for a chunk table of L entries and SG shots
// (plus, for the rolled per-node loop, the per-thread local connectivity and, for triangles
// with NN >= 16, the Dhat rows; nth = threads per CTA)
__host__ __device__ inline size_t chunk_smem_floats(int L, int SG, int D, bool grad, bool layer,
                                                    int NN = 0, int NS = 0, int nth = 0) {
  const size_t roll = D == 2 && NN >= 16 ? (size_t)D * NN * ((NN + 3) / 4 * 4) + (size_t)NS * nth
                      : D == 3 && NN >= 32 ? (size_t)NS * nth : 0;
  return ((chunk_tab_floats(L, SG, D, grad, layer) + 3) & ~size_t(3)) + roll;
}

// MODE: 0 forward, 1 adjoint, 2 adjoint with the gradient integrand; LAYER: the chunk's
// elements touch the damping layer. Separate instances keep each kernel's code small.
template <int D, int NN, int NS, int MODE, bool LAYER>
__device__ __forceinline__ void chunk_body(const StepArgs& a, float* smem) {
  constexpr int NI = NN - NS;
  constexpr int NG = D == 2 ? 3 : 6;
  // triangles with NN >= 16: the per-node loop stays rolled, with the rows of Dhat read from shared memory,
  // so that the kernel's code fits the instruction cache; smaller elements unroll it fully
  // with Dhat as constant-bank operands
  constexpr bool ROLL = D == 2 && NN >= 16;
  constexpr bool ROLL3 = D == 3 && NN >= 32;  // KMV3 tetrahedra (measured: KMV2 tets lose)
  static_assert(!ROLL || NN % 2 == 0, "the rolled form pairs nodes for packed FMAs");
  constexpr int NNP = (NN + 3) / 4 * 4;
  typedef LayerCoef<D> LC;
  const int c = blockIdx.x + a.ch0;
  const int* ch = a.chunks + 6 * c;
  const int e0 = ch[0], ne = ch[1], own_lo = ch[2], own_n = ch[3], nsh = ch[4], hp = ch[5];
  const int hn = a.chunks[6 * (c + 1) + 5] - hp;
  const int S = a.S;
  const int SG = a.SG;              // shots of this CTA: [s0, s0 + SG)
  const int s0 = blockIdx.y * SG;
  constexpr bool adj = MODE != 0;
  constexpr bool grad = MODE == 2;
  constexpr bool layer = LAYER;
  const int Lm = chunk_stride(a.L_max);
  const int lg = __ffs(SG) - 1;
  const ChunkTab t = chunk_tab(smem, Lm, SG, D, grad, layer);
  float* uloc = t.u;
  float* yloc = t.y;
  float* c2loc = t.c2;
  float* Floc = t.F;
  float* gloc = t.g;
  float* sloc = t.s;
  float* sYloc = t.sY;
  float* ywloc = t.yw;
  const int* piloc = t.pi;
  const int tid = threadIdx.x, nth = blockDim.x;
  ChunkDesc cd;
  cd.e0 = e0, cd.ne = ne, cd.own_lo = own_lo, cd.own_n = own_n, cd.nsh = nsh, cd.hp = hp;
  cd.hn = hn, cd.L = own_n + hn;

  // rolled form: Dhat rows [D][NN][NNP] and the element's shared-node local indices
  // [NS][nth] after the chunk table
  float* dhs = smem + ((chunk_tab_floats(a.L_max, SG, D, grad, layer) + 3) & ~size_t(3));
  int* lqs = reinterpret_cast<int*>(dhs + (ROLL ? (size_t)D * NN * NNP : 0));

  // ---- 1. load -------------------------------------------------------------------------
  chunk_load<D, grad, layer>(a, cd, t, Lm, SG, lg, s0, tid, nth);
  if constexpr (ROLL) {
    for (int i = tid; i < D * NN * NNP; i += nth) {
      const int r = i / NNP, j = i - r * NNP;
      dhs[i] = j < NN ? c_dhat[r * NN + j] : 0.f;
    }
  }
  cp_async_wait<1>();
  __syncthreads();
  if (layer) {
    if (!grad) chunk_load_layer<D>(a, cd, t, Lm, SG, lg, s0, tid, nth);
    chunk_prefetch_update<D>(a, cd, t, SG, s0, tid, nth);
    cp_async_wait<0>();
    __syncthreads();
  }

  // ---- 2. elements ---------------------------------------------------------------------
  const int P = a.PE;
  constexpr int QS = chunk_qsplit<D, NN, MODE, LAYER>();
  const int nq = nth / QS;  // threads of one half: (element, shot) pairs
  const int half = QS > 1 ? tid / nq : 0;
  const int tq = tid - half * nq;
  const int el = tq % P;
  const int sl = tq / P;
  if (el < ne && sl < SG) {
    const int e = e0 + el;
    const int s = s0 + sl;
    int lq[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      lq[q] = __ldg(a.lconn + (size_t)q * a.Es + e);
      if constexpr (ROLL || ROLL3) lqs[q * nq + tq] = lq[q];
    }
    const int lb = nsh + el * NI;  // local index of the first bubble node
    float U[NN], F[NN];
    const float* ur = uloc + sl * Lm;
#pragma unroll
    for (int q = 0; q < NS; ++q) U[q] = ur[lq[q]];
#pragma unroll
    for (int j = 0; j < NI; ++j) U[NS + j] = ur[lb + j];
    if (grad) {
      const float* fr = Floc + sl * Lm;
#pragma unroll
      for (int q = 0; q < NS; ++q) F[q] = fr[lq[q]];
#pragma unroll
      for (int j = 0; j < NI; ++j) F[NS + j] = fr[lb + j];
    }
    float G[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) G[g] = __ldg(a.geo + (size_t)g * a.Es + e);
    float Am[D * D];
    const int El = a.E - a.E0;
#pragma unroll
    for (int cc = 0; cc < D * D; ++cc)
      Am[cc] = layer ? __ldg(a.lgeo + (size_t)cc * El + (e - a.E0)) : 0.f;
    float Yv[NN];
#pragma unroll
    for (int q = 0; q < NN; ++q) Yv[q] = 0.f;
    if constexpr (D == 3) {
      if (layer && !adj) {
#pragma unroll
        for (int q = 0; q < NN; ++q) {
          Yv[q] = t.Yv[(size_t)sl * Lm + (q < NS ? lq[q] : lb + q - NS)];
        }
      }
    }
    float y[NN], yw[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) y[i] = yw[i] = 0.f;

if constexpr (ROLL) {
#pragma unroll 1
    for (int q = 0; q < NN; ++q) {
      const int lqq = q < NS ? lqs[q * nq + tq] : lb + (q - NS);
      float row[D][NNP];  // Dhat[d][q][:] for every d, 16-byte loads from shared memory
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int j = 0; j < NNP; j += 4) {
          const float4 r4 = *reinterpret_cast<const float4*>(dhs + ((size_t)d * NN + q) * NNP + j);
          row[d][j] = r4.x;
          row[d][j + 1] = r4.y;
          row[d][j + 2] = r4.z;
          row[d][j + 3] = r4.w;
        }
      float g[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        // four partial sums (j mod 4) in two packed FP32x2 FMA chains: shorter dependent
        // chains for the few warps an SM holds
        float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NN; j += 4) {
          acc0 = ffma2(make_float2(row[d][j], row[d][j + 1]), make_float2(U[j], U[j + 1]), acc0);
          if (j + 2 < NN)
            acc1 = ffma2(make_float2(row[d][j + 2], row[d][j + 3]),
                         make_float2(U[j + 2], j + 3 < NN ? U[j + 3] : 0.f), acc1);
        }
        g[d] = (acc0.x + acc1.x) + (acc0.y + acc1.y);
      }
      const float wq = c_w[q];  // uniform dynamic index
      const float wc = wq * c2loc[lqq];
      float f[D];
      if constexpr (D == 2) {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1]);
        f[1] = wc * (G[1] * g[0] + G[2] * g[1]);
      } else {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1] + G[2] * g[2]);
        f[1] = wc * (G[1] * g[0] + G[3] * g[1] + G[4] * g[2]);
        f[2] = wc * (G[2] * g[0] + G[4] * g[1] + G[5] * g[2]);
      }
      if (grad) {
        float gf[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < NN; j += 4) {
            acc0 = ffma2(make_float2(row[d][j], row[d][j + 1]), make_float2(F[j], F[j + 1]), acc0);
            if (j + 2 < NN)
              acc1 = ffma2(make_float2(row[d][j + 2], row[d][j + 3]),
                           make_float2(F[j + 2], j + 3 < NN ? F[j + 3] : 0.f), acc1);
          }
          gf[d] = (acc0.x + acc1.x) + (acc0.y + acc1.y);
        }
        float dot;
        if constexpr (D == 2) {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1]) + g[1] * (G[1] * gf[0] + G[2] * gf[1]);
        } else {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1] + G[2] * gf[2]) +
                g[1] * (G[1] * gf[0] + G[3] * gf[1] + G[4] * gf[2]) +
                g[2] * (G[2] * gf[0] + G[4] * gf[1] + G[5] * gf[2]);
        }
        atomicAdd(gloc + (a.grad_lanes ? sl * Lm : 0) + lqq, 2.f * t.cv[lqq] * wq * dot);
      }
      if (layer) {
        const int pi = piloc[lqq];
        if (pi >= 0) {
          const float* lc = a.lcf + (size_t)pi * LC::COUNT;
          float sq[D], pq[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) acc += Am[d * D + k] * g[d];
            sq[k] = wq * acc;
            const float raw = grad ? a.P[((size_t)pi * D + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq];
            pq[k] = adj ? raw * __ldg(lc + LC::PSI2 + k) : raw;
          }
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) acc += Am[d * D + k] * pq[k];
            f[d] += wq * acc;
          }
          float sY[D];
#pragma unroll
          for (int k = 0; k < D; ++k) sY[k] = 0.f;
          if constexpr (D == 3) {
            if (adj) {
              float pw[3], fw[3];
#pragma unroll
              for (int k = 0; k < 3; ++k)
                pw[k] = (grad ? a.P[((size_t)pi * 3 + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq]) *
                        __ldg(lc + LC::PSI3 + k);
#pragma unroll
              for (int d = 0; d < 3; ++d)
                fw[d] = wq * (Am[d * 3 + 0] * pw[0] + Am[d * 3 + 1] * pw[1] + Am[d * 3 + 2] * pw[2]);
#pragma unroll
              for (int i = 0; i < NN; ++i)
#pragma unroll
                for (int d = 0; d < 3; ++d) yw[i] = fmaf(row[d][i], fw[d], yw[i]);
            } else {
              float gy[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NN; ++j) acc = fmaf(row[d][j], Yv[j], acc);
                gy[d] = acc;
              }
#pragma unroll
              for (int k = 0; k < 3; ++k)
                sY[k] = wq * (Am[0 * 3 + k] * gy[0] + Am[1 * 3 + k] * gy[1] + Am[2 * 3 + k] * gy[2]);
            }
          }
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float* sp = sloc + (size_t)(k * SG + sl) * Lm + lqq;
            float* syp = sYloc + (size_t)(k * SG + sl) * Lm + lqq;
            if (q < NS) {
              atomicAdd(sp, sq[k]);
              if constexpr (D == 3) atomicAdd(syp, sY[k]);
            } else {
              *sp = sq[k];
              if constexpr (D == 3) *syp = sY[k];
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NN; i += 2) {  // y[i], y[i+1] in one packed FMA per d
        float2 yy = make_float2(y[i], y[i + 1]);
#pragma unroll
        for (int d = 0; d < D; ++d)
          yy = ffma2(make_float2(row[d][i], row[d][i + 1]), make_float2(f[d], f[d]), yy);
        y[i] = yy.x;
        y[i + 1] = yy.y;
      }
    }

    } else if constexpr (ROLL3) {
      // KMV3 tetrahedra: the per-node loop rolled, Dhat from the constant bank with a
      // warp-uniform dynamic index (the unrolled loop does not fit the instruction cache)
#pragma unroll 1
    for (int q = half; q < NN; q += QS) {
      const int lqq = q < NS ? lqs[q * nq + tq] : lb + (q - NS);
      float g[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        float a0 = 0.f, a1 = 0.f;  // two partial sums: shorter dependent FMA chains
#pragma unroll
        for (int j = 0; j < NN; j += 2) a0 = fmaf(c_dhat[(d * NN + q) * NN + j], U[j], a0);
#pragma unroll
        for (int j = 1; j < NN; j += 2) a1 = fmaf(c_dhat[(d * NN + q) * NN + j], U[j], a1);
        g[d] = a0 + a1;
      }
      const float wq = c_w[q];
      const float wc = wq * c2loc[lqq];
      float f[D];
      if constexpr (D == 2) {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1]);
        f[1] = wc * (G[1] * g[0] + G[2] * g[1]);
      } else {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1] + G[2] * g[2]);
        f[1] = wc * (G[1] * g[0] + G[3] * g[1] + G[4] * g[2]);
        f[2] = wc * (G[2] * g[0] + G[4] * g[1] + G[5] * g[2]);
      }
      if (grad) {
        float gf[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          float a0 = 0.f, a1 = 0.f;
#pragma unroll
          for (int j = 0; j < NN; j += 2) a0 = fmaf(c_dhat[(d * NN + q) * NN + j], F[j], a0);
#pragma unroll
          for (int j = 1; j < NN; j += 2) a1 = fmaf(c_dhat[(d * NN + q) * NN + j], F[j], a1);
          gf[d] = a0 + a1;
        }
        float dot;
        if constexpr (D == 2) {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1]) + g[1] * (G[1] * gf[0] + G[2] * gf[1]);
        } else {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1] + G[2] * gf[2]) +
                g[1] * (G[1] * gf[0] + G[3] * gf[1] + G[4] * gf[2]) +
                g[2] * (G[2] * gf[0] + G[4] * gf[1] + G[5] * gf[2]);
        }
        atomicAdd(gloc + (a.grad_lanes ? sl * Lm : 0) + lqq, 2.f * t.cv[lqq] * wq * dot);
      }
      if (layer) {
        const int pi = piloc[lqq];
        if (pi >= 0) {
          const float* lc = a.lcf + (size_t)pi * LC::COUNT;
          float sq[D], pq[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) acc += Am[d * D + k] * g[d];
            sq[k] = wq * acc;
            const float raw = grad ? a.P[((size_t)pi * D + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq];
            pq[k] = adj ? raw * __ldg(lc + LC::PSI2 + k) : raw;
          }
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) acc += Am[d * D + k] * pq[k];
            f[d] += wq * acc;
          }
          float sY[D];
#pragma unroll
          for (int k = 0; k < D; ++k) sY[k] = 0.f;
          if constexpr (D == 3) {
            if (adj) {
              float pw[3], fw[3];
#pragma unroll
              for (int k = 0; k < 3; ++k)
                pw[k] = (grad ? a.P[((size_t)pi * 3 + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq]) *
                        __ldg(lc + LC::PSI3 + k);
#pragma unroll
              for (int d = 0; d < 3; ++d)
                fw[d] = wq * (Am[d * 3 + 0] * pw[0] + Am[d * 3 + 1] * pw[1] + Am[d * 3 + 2] * pw[2]);
#pragma unroll
              for (int i = 0; i < NN; ++i)
#pragma unroll
                for (int d = 0; d < 3; ++d) yw[i] = fmaf(c_dhat[(d * NN + q) * NN + i], fw[d], yw[i]);
            } else {
              float gy[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NN; ++j) acc = fmaf(c_dhat[(d * NN + q) * NN + j], Yv[j], acc);
                gy[d] = acc;
              }
#pragma unroll
              for (int k = 0; k < 3; ++k)
                sY[k] = wq * (Am[0 * 3 + k] * gy[0] + Am[1 * 3 + k] * gy[1] + Am[2 * 3 + k] * gy[2]);
            }
          }
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float* sp = sloc + (size_t)(k * SG + sl) * Lm + lqq;
            float* syp = sYloc + (size_t)(k * SG + sl) * Lm + lqq;
            if (q < NS) {
              atomicAdd(sp, sq[k]);
              if constexpr (D == 3) atomicAdd(syp, sY[k]);
            } else {
              *sp = sq[k];
              if constexpr (D == 3) *syp = sY[k];
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NN; ++i)
#pragma unroll
        for (int d = 0; d < D; ++d) y[i] = fmaf(c_dhat[(d * NN + q) * NN + i], f[d], y[i]);
    }

        } else {
#pragma unroll
    for (int q = 0; q < NN; ++q) {
      if (QS > 1 && q % QS != half) continue;  // the other half's node (warp-uniform)
      const int lqq = q < NS ? lq[q] : lb + (q - NS);
      float g[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        float a0 = 0.f, a1 = 0.f;  // two partial sums: shorter dependent FMA chains
#pragma unroll
        for (int j = 0; j < NN; j += 2) a0 = fmaf(c_dhat[(d * NN + q) * NN + j], U[j], a0);
#pragma unroll
        for (int j = 1; j < NN; j += 2) a1 = fmaf(c_dhat[(d * NN + q) * NN + j], U[j], a1);
        g[d] = a0 + a1;
      }
      const float wq = c_w[q];
      const float wc = wq * c2loc[lqq];
      float f[D];
      if constexpr (D == 2) {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1]);
        f[1] = wc * (G[1] * g[0] + G[2] * g[1]);
      } else {
        f[0] = wc * (G[0] * g[0] + G[1] * g[1] + G[2] * g[2]);
        f[1] = wc * (G[1] * g[0] + G[3] * g[1] + G[4] * g[2]);
        f[2] = wc * (G[2] * g[0] + G[4] * g[1] + G[5] * g[2]);
      }
      if (grad) {
        float gf[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
          float a0 = 0.f, a1 = 0.f;
#pragma unroll
          for (int j = 0; j < NN; j += 2) a0 = fmaf(c_dhat[(d * NN + q) * NN + j], F[j], a0);
#pragma unroll
          for (int j = 1; j < NN; j += 2) a1 = fmaf(c_dhat[(d * NN + q) * NN + j], F[j], a1);
          gf[d] = a0 + a1;
        }
        float dot;
        if constexpr (D == 2) {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1]) + g[1] * (G[1] * gf[0] + G[2] * gf[1]);
        } else {
          dot = g[0] * (G[0] * gf[0] + G[1] * gf[1] + G[2] * gf[2]) +
                g[1] * (G[1] * gf[0] + G[3] * gf[1] + G[4] * gf[2]) +
                g[2] * (G[2] * gf[0] + G[4] * gf[1] + G[5] * gf[2]);
        }
        atomicAdd(gloc + (a.grad_lanes ? sl * Lm : 0) + lqq, 2.f * t.cv[lqq] * wq * dot);
      }
      if (layer) {
        const int pi = piloc[lqq];
        if (pi >= 0) {
          const float* lc = a.lcf + (size_t)pi * LC::COUNT;
          float sq[D], pq[D];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) acc += Am[d * D + k] * g[d];
            sq[k] = wq * acc;
            const float raw = grad ? a.P[((size_t)pi * D + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq];
            pq[k] = adj ? raw * __ldg(lc + LC::PSI2 + k) : raw;
          }
#pragma unroll
          for (int d = 0; d < D; ++d) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) acc += Am[d * D + k] * pq[k];
            f[d] += wq * acc;
          }
          float sY[D];
#pragma unroll
          for (int k = 0; k < D; ++k) sY[k] = 0.f;
          if constexpr (D == 3) {
            if (adj) {
              float pw[3], fw[3];
#pragma unroll
              for (int k = 0; k < 3; ++k)
                pw[k] = (grad ? a.P[((size_t)pi * 3 + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq]) *
                        __ldg(lc + LC::PSI3 + k);
#pragma unroll
              for (int d = 0; d < 3; ++d)
                fw[d] = wq * (Am[d * 3 + 0] * pw[0] + Am[d * 3 + 1] * pw[1] + Am[d * 3 + 2] * pw[2]);
#pragma unroll
              for (int i = 0; i < NN; ++i)
#pragma unroll
                for (int d = 0; d < 3; ++d) yw[i] = fmaf(c_dhat[(d * NN + q) * NN + i], fw[d], yw[i]);
            } else {
              float gy[3];
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NN; ++j) acc = fmaf(c_dhat[(d * NN + q) * NN + j], Yv[j], acc);
                gy[d] = acc;
              }
#pragma unroll
              for (int k = 0; k < 3; ++k)
                sY[k] = wq * (Am[0 * 3 + k] * gy[0] + Am[1 * 3 + k] * gy[1] + Am[2 * 3 + k] * gy[2]);
            }
          }
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float* sp = sloc + (size_t)(k * SG + sl) * Lm + lqq;
            float* syp = sYloc + (size_t)(k * SG + sl) * Lm + lqq;
            if (q < NS) {
              atomicAdd(sp, sq[k]);
              if constexpr (D == 3) atomicAdd(syp, sY[k]);
            } else {
              *sp = sq[k];
              if constexpr (D == 3) *syp = sY[k];
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NN; ++i)
#pragma unroll
        for (int d = 0; d < D; ++d) y[i] = fmaf(c_dhat[(d * NN + q) * NN + i], f[d], y[i]);
    }

    }
    // sources and receivers of this element (flagged elements only)
    const int slot = __ldg(a.inj + e);
    if (slot >= 0 && half == 0) {
      const int rb = __ldg(a.rslot_ptr + slot), re = __ldg(a.rslot_ptr + slot + 1);
      if (!adj) {
        if (a.rec != nullptr) {
          for (int r = rb; r < re; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NN; ++k) acc = fmaf(__ldg(a.rslot_phi + (size_t)r * NN + k), U[k], acc);
            a.rec[((size_t)s * (a.nt + 1) + a.n) * a.R + __ldg(a.rslot_rec + r)] = acc;
          }
        }
        if (__ldg(a.src_elem + s) == e) {
          const float wv = __ldg(a.wavelet + (size_t)s * a.nt + a.n);
#pragma unroll
          for (int k = 0; k < NN; ++k) y[k] -= wv * __ldg(a.src_phi + (size_t)s * NN + k);
        }
      } else {
        for (int r = rb; r < re; ++r) {
          const float res = __ldg(a.resid + ((size_t)s * (a.nt + 1) + a.n) * a.R + __ldg(a.rslot_rec + r));
#pragma unroll
          for (int k = 0; k < NN; ++k) y[k] = fmaf(res, __ldg(a.rslot_phi + (size_t)r * NN + k), y[k]);
        }
      }
    }
    float* yr = yloc + sl * Lm;
    float* ywr = ywloc + sl * Lm;
    // the rolled forms take the shared-node indices back from shared memory, so that they
    // need not stay in registers through the node loop
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      const int lqq = ROLL || ROLL3 ? lqs[q * nq + tq] : lq[q];
      atomicAdd(yr + lqq, y[q]);
      if constexpr (D == 3) {
        if (layer && adj) atomicAdd(ywr + lqq, yw[q]);
      }
    }
#pragma unroll
    for (int j = 0; j < NI; ++j) {  // bubble nodes: this element's alone (both halves add)
      if (QS > 1) {
        atomicAdd(yr + lb + j, y[NS + j]);
        if constexpr (D == 3) {
          if (layer && adj) atomicAdd(ywr + lb + j, yw[NS + j]);
        }
      } else {
        yr[lb + j] = y[NS + j];
        if constexpr (D == 3) {
          if (layer && adj) ywr[lb + j] = yw[NS + j];
        }
      }
    }
  }
  __syncthreads();

  // ---- 3. owned DoFs: final update; halo DoFs: to the global accumulators ----------------
  cp_async_wait<0>();
  __syncthreads();
  chunk_store<D, grad, layer>(a, cd, t, Lm, SG, lg, s0, tid, nth);
}

}  // namespace fwi
