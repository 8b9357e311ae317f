// Global <-> shared-memory traffic of one chunk, shared by the CUDA-core and the tensor-core
// chunk kernels.
//
// Phase 1 (chunk_load) issues every global read of the chunk at once as asynchronous copies
// (cp.async, 4 bytes each) into the chunk table, in two completion groups: group 0 holds what
// the element phase reads (u, c^2 and the layer index of every local DoF; the forward field
// and c of every local DoF in gradient steps), group 1 what only the final update reads (v
// and the update coefficients c1..c3 of the owned DoFs), so that group 1's latency hides
// behind the element phase. Phase 3 (chunk_store) finishes the owned DoFs from the table
// and sends the halo DoFs' contributions to the global accumulators.
//
// Layer chunks of steps without the gradient add a third group (chunk_load_layer, issued
// once the layer indices are in the table): the damping-layer auxiliaries P (and in the 3D
// forward Y) of every local layer DoF. Gradient steps, whose table is the largest, read P
// from global memory (prefetched into L2 at the start of the element phase), so that two CTAs
// still fit on an SM: with P in the table they ran at one CTA per SM and slower (542 against
// 393 us per step on the KMV5 marine mesh).
//
// Layer chunks (two to four times the table of the others) skip group 1 and read v and
// c1..c3 from global memory in phase 3, which keeps two of their CTAs on an SM.
//
// Table layout (floats, shot-major [SG][Lm] with Lm odd so that the SG rows of one DoF fall
// in different banks): u, y [SG][Lm]; c2 [Lm]; pi [Lm] (int); v [SG][Lm] and cf [3][Lm]
// (not in layer chunks); gradient
// steps: F [SG][Lm], g [SG][Lm], cv [Lm]; layer chunks: s [D][SG][Lm], P [D][SG][Lm] (not in
// gradient steps) (and in 3D sY [D][SG][Lm], yw [SG][Lm], Yv [SG][Lm]).
#pragma once
#include "update.cuh"

namespace fwi {

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Row stride of the shot-major tables: odd, so that the S rows of one DoF fall in
// different banks.
__host__ __device__ inline int chunk_stride(int L) { return L | 1; }

__host__ __device__ inline size_t chunk_tab_floats(int L, int SG, int D, bool grad, bool layer) {
  const size_t Lm = (size_t)chunk_stride(L);
  size_t f = Lm * (2 * (size_t)SG + 2) + (layer ? 0 : Lm * ((size_t)SG + 3));
  if (grad) f += Lm * (2 * (size_t)SG + 1);
  if (layer) f += (grad ? 1 : 2) * Lm * D * SG + (D == 3 ? Lm * D * SG + 2 * Lm * SG : 0);
  return f;
}

struct ChunkTab {
  float *u, *y, *v, *c2, *cf, *F, *g, *cv, *s, *P, *sY, *yw, *Yv;
  int* pi;
};

__device__ __forceinline__ ChunkTab chunk_tab(float* base, int Lm, int SG, int D, bool grad,
                                              bool layer) {
  ChunkTab t;
  const size_t R = (size_t)Lm * SG;
  t.u = base;
  t.y = t.u + R;
  t.c2 = t.y + R;
  t.pi = reinterpret_cast<int*>(t.c2 + Lm);
  t.v = reinterpret_cast<float*>(t.pi + Lm);  // v and cf: not in layer chunks (see above)
  t.cf = t.v + (layer ? 0 : R);
  float* p0 = t.cf + (layer ? 0 : 3 * (size_t)Lm);
  float* p = p0;
  t.F = p;
  t.g = t.F + (grad ? R : 0);  // gradient integrand [SG][Lm] per shot, or row 0 for all
  t.cv = t.g + (grad ? R : 0);
  p = t.cv + (grad ? Lm : 0);
  t.s = p;
  t.P = t.s + (layer ? (size_t)D * R : 0);
  t.sY = t.P + (layer && !grad ? (size_t)D * R : 0);
  t.yw = t.sY + (layer && D == 3 ? (size_t)D * R : 0);
  t.Yv = t.yw + (layer && D == 3 ? R : 0);
  return t;
}

struct ChunkDesc {
  int e0, ne, own_lo, own_n, nsh, hp, hn, L;
};

__device__ __forceinline__ ChunkDesc chunk_desc(const StepArgs& a, int c) {
  const int* ch = a.chunks + 6 * c;
  ChunkDesc d;
  d.e0 = ch[0];
  d.ne = ch[1];
  d.own_lo = ch[2];
  d.own_n = ch[3];
  d.nsh = ch[4];
  d.hp = ch[5];
  d.hn = a.chunks[6 * (c + 1) + 5] - d.hp;
  d.L = d.own_n + d.hn;
  return d;
}

// Phase 1: issue the chunk's reads (two cp.async groups, see above) and clear the
// accumulators. lg = log2(SG); shots [s0, s0 + SG).
template <int D, bool GRAD, bool LAYER>
__device__ __forceinline__ void chunk_load(const StepArgs& a, const ChunkDesc& cd, const ChunkTab& t,
                                           int Lm, int SG, int lg, int s0, int tid, int nth) {
  const int S = a.S;
  const size_t N = (size_t)a.N;
  for (int i = tid; i < cd.own_n * SG; i += nth) {
    const int l = i >> lg, q = i & (SG - 1);
    const size_t g = (size_t)(cd.own_lo + l) * S + s0 + q;
    cp_async4(t.u + q * Lm + l, a.u + g);
    if (GRAD) cp_async4(t.F + q * Lm + l, a.ring_u + g);
  }
  for (int i = tid; i < cd.hn * SG; i += nth) {
    const int h = i >> lg, q = i & (SG - 1);
    const size_t g = (size_t)__ldg(a.halo + cd.hp + h) * S + s0 + q;
    cp_async4(t.u + q * Lm + cd.own_n + h, a.u + g);
    if (GRAD) cp_async4(t.F + q * Lm + cd.own_n + h, a.ring_u + g);
  }
  for (int l = tid; l < cd.L; l += nth) {
    const int dof = l < cd.own_n ? cd.own_lo + l : __ldg(a.halo + cd.hp + l - cd.own_n);
    cp_async4(t.c2 + l, a.c2 + dof);
    cp_async4(t.pi + l, a.pidx + dof);
    if (GRAD) cp_async4(t.cv + l, a.cvel + dof);
  }
  cp_async_commit();
  if (!LAYER) {
    for (int i = tid; i < cd.own_n * SG; i += nth) {
      const int l = i >> lg, q = i & (SG - 1);
      cp_async4(t.v + q * Lm + l, a.v + (size_t)(cd.own_lo + l) * S + s0 + q);
    }
    for (int l = tid; l < cd.own_n; l += nth) {
      const size_t dof = (size_t)(cd.own_lo + l);
      cp_async4(t.cf + l, a.cf + dof);
      cp_async4(t.cf + Lm + l, a.cf + N + dof);
      cp_async4(t.cf + 2 * (size_t)Lm + l, a.cf + 2 * N + dof);
    }
  }
  cp_async_commit();  // (empty for layer chunks: the group count stays the same)
  for (int i = tid; i < cd.L * SG; i += nth) {
    const int l = i >> lg, q = i & (SG - 1);
    t.y[q * Lm + l] = 0.f;
  }
  if (GRAD)
    for (int i = tid; i < cd.L * SG; i += nth) {
      const int l = i >> lg, q = i & (SG - 1);
      t.g[q * Lm + l] = 0.f;
    }
  if (LAYER) {
    for (int i = tid; i < Lm * D * SG; i += nth) {
      t.s[i] = 0.f;
      if constexpr (D == 3) t.sY[i] = 0.f;
    }
    if constexpr (D == 3)
      for (int i = tid; i < Lm * SG; i += nth) t.yw[i] = 0.f;
  }
}

// Layer chunks, after group 0 has landed and a barrier: the layer auxiliaries of every
// local layer DoF as a third copy group (P; Y in the 3D forward), zeros elsewhere.
template <int D>
__device__ __forceinline__ void chunk_load_layer(const StepArgs& a, const ChunkDesc& cd,
                                                 const ChunkTab& t, int Lm, int SG, int lg, int s0,
                                                 int tid, int nth) {
  const int S = a.S;
  const bool fwd3 = D == 3 && a.mode == 0;
  for (int i = tid; i < cd.L * SG; i += nth) {
    const int l = i >> lg, q = i & (SG - 1);
    const int pi = t.pi[l];
    if (pi >= 0) {
#pragma unroll
      for (int k = 0; k < D; ++k)
        cp_async4(t.P + (size_t)(k * SG + q) * Lm + l, a.P + ((size_t)pi * D + k) * S + s0 + q);
      if (fwd3) cp_async4(t.Yv + (size_t)q * Lm + l, a.Y + (size_t)pi * S + s0 + q);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) t.P[(size_t)(k * SG + q) * Lm + l] = 0.f;
      if (fwd3) t.Yv[(size_t)q * Lm + l] = 0.f;
    }
  }
  cp_async_commit();
}

// Layer chunks, at the start of the element phase: the update phase reads v, c1..c3 and the
// layer coefficients of the owned DoFs from global memory; start bringing them to L2 so that
// those reads do not each wait for DRAM.
template <int D>
__device__ __forceinline__ void chunk_prefetch_update(const StepArgs& a, const ChunkDesc& cd,
                                                      const ChunkTab& t, int SG, int s0, int tid,
                                                      int nth) {
  typedef LayerCoef<D> LC;
  for (int l = tid; l < cd.own_n; l += nth) {
    const size_t dof = (size_t)(cd.own_lo + l);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a.v + dof * a.S + s0));
    if ((l & 31) == 0) {
#pragma unroll
      for (int r = 0; r < 3; ++r) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.cf + (size_t)r * a.N + dof));
    }
    const int pi = t.pi[l];
    if (pi >= 0) {
      const float* lc = a.lcf + (size_t)pi * LC::COUNT;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(lc));
      if constexpr (D == 3) {  // 88-byte records may straddle two lines; the omega state Y
        asm volatile("prefetch.global.L2 [%0];" ::"l"(lc + LC::COUNT - 1));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a.Y + (size_t)pi * a.S + s0));
      }
    }
  }
  if (a.ring_u != nullptr) {  // gradient steps read P of every local layer DoF from global memory
    for (int l = tid; l < cd.L; l += nth) {
      const int pi = t.pi[l];
      if (pi >= 0)
#pragma unroll
        for (int k = 0; k < D; ++k) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.P + ((size_t)pi * D + k) * a.S + s0));
    }
  }
  (void)SG;
}

// Phase 3: owned DoFs final (the increment update from the table), halo DoFs to the
// global accumulators (finished by the node kernel after all chunks), gradient segment.
// Call after cp_async_wait<0>() and a barrier.
template <int D, bool GRAD, bool LAYER>
__device__ __forceinline__ void chunk_store(const StepArgs& a, const ChunkDesc& cd, const ChunkTab& t,
                                            int Lm, int SG, int lg, int s0, int tid, int nth) {
  const int S = a.S;
  const bool adj = a.mode != 0;
  if (LAYER) {
    // layer chunks read v and c1..c3 from global memory: four items per round, their reads
    // issued before any write
    for (int i0 = tid; i0 < cd.own_n * SG; i0 += 4 * nth) {
      float vo[4], c1[4], c2[4], c3[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nth;
        vo[k] = c1[k] = c2[k] = c3[k] = 0.f;
        if (i < cd.own_n * SG) {
          const int l = i >> lg, dof = cd.own_lo + l;
          vo[k] = a.v[(size_t)dof * S + s0 + (i & (SG - 1))];
          c1[k] = __ldg(a.cf + dof);
          c2[k] = __ldg(a.cf + (size_t)a.N + dof);
          c3[k] = __ldg(a.cf + 2 * (size_t)a.N + dof);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nth;
        if (i >= cd.own_n * SG) break;
        const int l = i >> lg, q = i & (SG - 1), s = s0 + q;
        float sU[D], sY[D], po[D];
        float ywv = 0.f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          sU[d] = t.s[(size_t)(d * SG + q) * Lm + l];
          sY[d] = 0.f;
          if constexpr (D == 3) sY[d] = t.sY[(size_t)(d * SG + q) * Lm + l];
          po[d] = GRAD ? 0.f : t.P[(size_t)(d * SG + q) * Lm + l];
        }
        if constexpr (D == 3) ywv = t.yw[(size_t)q * Lm + l];
        dof_update_pre<D>(a, cd.own_lo + l, s, t.y[q * Lm + l], t.u[q * Lm + l], vo[k], c1[k], c2[k],
                          c3[k], t.pi[l], sU, sY, ywv, GRAD ? nullptr : po);
      }
    }
  } else {
    for (int i = tid; i < cd.own_n * SG; i += nth) {
      const int l = i >> lg, q = i & (SG - 1), s = s0 + q;
      float sU[D], sY[D];
#pragma unroll
      for (int d = 0; d < D; ++d) sU[d] = sY[d] = 0.f;
      dof_update_pre<D>(a, cd.own_lo + l, s, t.y[q * Lm + l], t.u[q * Lm + l], t.v[q * Lm + l],
                        t.cf[l], t.cf[Lm + l], t.cf[2 * (size_t)Lm + l], -1, sU, sY, 0.f);
    }
  }
  for (int i = tid; i < cd.hn * SG; i += nth) {
    const int h = i >> lg, q = i & (SG - 1), s = s0 + q;
    const int l = cd.own_n + h;
    const int dof = __ldg(a.halo + cd.hp + h);
    atomicAdd(a.r + (size_t)(dof - a.N_own) * S + s, t.y[q * Lm + l]);
    if (LAYER) {
      const int pi = t.pi[l];
      if (pi >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          atomicAdd(a.Pacc + ((size_t)pi * D + k) * S + s, t.s[(size_t)(k * SG + q) * Lm + l]);
          if constexpr (D == 3) {
            if (!adj) atomicAdd(a.PaccY + ((size_t)pi * D + k) * S + s, t.sY[(size_t)(k * SG + q) * Lm + l]);
          }
        }
        if constexpr (D == 3) {
          if (adj) atomicAdd(a.Yacc + (size_t)pi * S + s, t.yw[(size_t)q * Lm + l]);
        }
      }
    }
  }
  if (GRAD) {
    // fire-and-forget atomic adds (a plain read-modify-write of the owned DoFs would wait on
    // each load: measured slower)
    if (a.grad_lanes) {  // one segment accumulator per shot, [S][N]
      for (int i = tid; i < cd.L * SG; i += nth) {
        const int l = i >> lg, q = i & (SG - 1);
        const int dof = l < cd.own_n ? cd.own_lo + l : __ldg(a.halo + cd.hp + l - cd.own_n);
        atomicAdd(a.gseg + (size_t)(s0 + q) * a.N + dof, t.g[q * Lm + l]);
      }
    } else {  // summed over the shots (the element phase added every shot to row 0), [N]
      for (int l = tid; l < cd.L; l += nth) {
        const int dof = l < cd.own_n ? cd.own_lo + l : __ldg(a.halo + cd.hp + l - cd.own_n);
        atomicAdd(a.gseg + dof, t.g[l]);
      }
    }
  }
}

}  // namespace fwi
