// Per-DoF increment update shared by the element kernels (element-interior DoFs) and the
// node kernel (shared DoFs), and the node kernel itself.
#pragma once
#include "fwi_internal.h"

namespace fwi {

template <int D>
struct LayerCoef {  // offsets inside one layer DoF's coefficient record
  static constexpr int E1 = 0, E2F = D, E2A = 2 * D, PSI2 = 3 * D, E3F = 4 * D, PSI3 = 5 * D,
                       C4 = 6 * D, C5 = 6 * D + 1, DTDET = 6 * D + 2, DTM = 6 * D + 3;
  static constexpr int COUNT = D == 2 ? 4 * D : 6 * D + 4;
};

// Increment-form update of one DoF (shared by the element and node kernels):
//   v' = c1 v - c2 y - c3 u  (- c4 Y^n in the 3D forward, + c5 lam_omega^m in the 3D adjoint)
//   u' = u + v'
// plus the layer auxiliaries of the DoF:
//   forward  P_k' = e1_k P_k - e2f_k sU_k (+ e3f_k sY_k in 3D);  Y' = Y + dt u
//   adjoint  nu_k' = e1_k nu_k - e2a_k sU_k;  lam_w' = lam_w - dt detPsi1 lam + (dt/M) yw
// The update with the DoF's v, c1..c3 and layer index already at hand (chunk kernels
// prefetch them into shared memory).
template <int D>
__device__ __forceinline__ void dof_update_pre(const StepArgs& a, int dof, int s, float y, float uo,
                                               float vo, float c1, float c2, float c3, int pi,
                                               const float* sU, const float* sY, float yw,
                                               const float* po = nullptr) {
  const int S = a.S;
  const size_t i = (size_t)dof * S + s;
  float vn = c1 * vo - c2 * y - c3 * uo;
  if (pi >= 0) {
    typedef LayerCoef<D> L;
    const float* lc = a.lcf + (size_t)pi * L::COUNT;
    if (a.mode == 0) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t pk = ((size_t)pi * D + k) * S + s;
        const float pold = po ? po[k] : a.P[pk];
        float pn = __ldg(lc + L::E1 + k) * pold - __ldg(lc + L::E2F + k) * sU[k];
        if constexpr (D == 3) pn += __ldg(lc + L::E3F + k) * sY[k];
        a.P[pk] = pn;
      }
      if constexpr (D == 3) {
        const size_t py = (size_t)pi * S + s;
        const float yo = a.Y[py];
        vn -= __ldg(lc + L::C4) * yo;
        a.Y[py] = yo + a.dt * uo;
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const size_t pk = ((size_t)pi * D + k) * S + s;
        const float pold = po ? po[k] : a.P[pk];
        a.P[pk] = __ldg(lc + L::E1 + k) * pold - __ldg(lc + L::E2A + k) * sU[k];
      }
      if constexpr (D == 3) {
        const size_t py = (size_t)pi * S + s;
        const float wo = a.Y[py];
        vn += __ldg(lc + L::C5) * wo;
        a.Y[py] = wo - __ldg(lc + L::DTDET) * uo + __ldg(lc + L::DTM) * yw;
      }
    }
  }
  a.v[i] = vn;
  const float un = uo + vn;
  a.u[i] = un;
  if (!isfinite(un)) atomicOr(a.status, 1);
}

template <int D>
__device__ __forceinline__ void dof_update(const StepArgs& a, int dof, int s, float y, float uo,
                                           const float* sU, const float* sY, float yw) {
  const float c1 = __ldg(a.cf + dof);
  const float c2 = __ldg(a.cf + (size_t)a.N + dof);
  const float c3 = __ldg(a.cf + 2 * (size_t)a.N + dof);
  const float vo = a.v[(size_t)dof * a.S + s];
  const int pi = __ldg(a.pidx + dof);
  dof_update_pre<D>(a, dof, s, y, uo, vo, c1, c2, c3, pi, sU, sY, yw);
}

constexpr int NODE_ITEMS = 4;

// Finish of one accumulated DoF (index i of the accumulator range, DoF dof, shot s): y and
// the layer sums from the accumulators the element contributions arrived in by atomics
// (read from L2, where the atomics resolve), the accumulators cleared for the next step,
// then the same update. uo is the DoF's u^n. Every global read is issued before the first
// write.
template <int D>
__device__ __forceinline__ void accum_finish(const StepArgs& a, size_t i, int dof, int s, float uo,
                                             int pi) {
  const int S = a.S;
  const size_t rx = i * S + s;
  const size_t ix = (size_t)dof * S + s;
  const float y = __ldcg(a.r + rx);
  const float vo = a.v[ix];
  const float c1 = __ldg(a.cf + dof);
  const float c2 = __ldg(a.cf + (size_t)a.N + dof);
  const float c3 = __ldg(a.cf + 2 * (size_t)a.N + dof);
  float sU[D], sY[D];
  float yw = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) sU[k] = sY[k] = 0.f;
  if (pi >= 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const size_t pk = ((size_t)pi * D + k) * S + s;
      sU[k] = __ldcg(a.Pacc + pk);
      if constexpr (D == 3) {
        if (a.mode == 0) sY[k] = __ldcg(a.PaccY + pk);
      }
    }
    if constexpr (D == 3) {
      if (a.mode == 1) yw = __ldcg(a.Yacc + (size_t)pi * S + s);
    }
  }
  a.r[rx] = 0.f;
  if (pi >= 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const size_t pk = ((size_t)pi * D + k) * S + s;
      a.Pacc[pk] = 0.f;
      if constexpr (D == 3) {
        if (a.mode == 0) a.PaccY[pk] = 0.f;
      }
    }
    if constexpr (D == 3) {
      if (a.mode == 1) a.Yacc[(size_t)pi * S + s] = 0.f;
    }
  }
  dof_update_pre<D>(a, dof, s, y, uo, vo, c1, c2, c3, pi, sU, sY, yw);
}

// Shared-DoF finish as a separate pass over the DoFs [h0, h0 + hcnt) (the halo DoFs of the
// chunked layout, the shared DoFs of the plain layout), whose element contributions arrived
// by atomics in r[(dof - h0) * S + s].
template <int D>
__global__ void __launch_bounds__(256) node_kernel(const StepArgs a) {
  // NODE_ITEMS (DoF, shot) items per thread, a block-stride apart (coalesced); all their
  // reads are issued before any write, so that each thread has NODE_ITEMS times more
  // memory requests in flight
  const int S = a.S;
  const int64_t total = (int64_t)a.hcnt << a.log2S;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * NODE_ITEMS + threadIdx.x;
  float uo[NODE_ITEMS], vo[NODE_ITEMS], y[NODE_ITEMS], c1[NODE_ITEMS], c2[NODE_ITEMS],
      c3[NODE_ITEMS];
  int pi[NODE_ITEMS];
#pragma unroll
  for (int k = 0; k < NODE_ITEMS; ++k) {
    const int64_t t = base + (int64_t)k * blockDim.x;
    uo[k] = vo[k] = y[k] = c1[k] = c2[k] = c3[k] = 0.f;
    pi[k] = -1;
    if (t < total) {
      const int64_t i = t >> a.log2S;
      const int dof = a.h0 + (int)i;
      const size_t ix = (size_t)dof * S + (t & (S - 1));
      uo[k] = a.u[ix];
      vo[k] = a.v[ix];
      y[k] = __ldcg(a.r + (size_t)t);
      c1[k] = __ldg(a.cf + dof);
      c2[k] = __ldg(a.cf + (size_t)a.N + dof);
      c3[k] = __ldg(a.cf + 2 * (size_t)a.N + dof);
      pi[k] = __ldg(a.pidx + dof);
    }
  }
#pragma unroll
  for (int k = 0; k < NODE_ITEMS; ++k) {
    const int64_t t = base + (int64_t)k * blockDim.x;
    if (t >= total) continue;
    const int64_t i = t >> a.log2S;
    const int dof = a.h0 + (int)i;
    const int s = (int)(t & (S - 1));
    a.r[(size_t)t] = 0.f;
    float sU[D], sY[D];
    float yw = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) sU[d] = sY[d] = 0.f;
    if (pi[k] >= 0) {  // damping layer: the layer sums (a minority of the DoFs)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const size_t pk = ((size_t)pi[k] * D + d) * S + s;
        sU[d] = __ldcg(a.Pacc + pk);
        a.Pacc[pk] = 0.f;
        if constexpr (D == 3) {
          if (a.mode == 0) {
            sY[d] = __ldcg(a.PaccY + pk);
            a.PaccY[pk] = 0.f;
          }
        }
      }
      if constexpr (D == 3) {
        if (a.mode == 1) {
          const size_t py = (size_t)pi[k] * S + s;
          yw = __ldcg(a.Yacc + py);
          a.Yacc[py] = 0.f;
        }
      }
    }
    dof_update_pre<D>(a, dof, s, y[k], uo[k], vo[k], c1[k], c2[k], c3[k], pi[k], sU, sY, yw);
  }
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ldcg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float comp(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }
__device__ __forceinline__ void setc(float4& v, int c, float x) {
  if (c == 0) v.x = x; else if (c == 1) v.y = x; else if (c == 2) v.z = x; else v.w = x;
}

// The shared-DoF finish of node_kernel for batches of S = 4m shots: one thread per (DoF,
// four consecutive shots), float4 reads and writes of the shot-interleaved arrays, the same
// arithmetic as dof_update_pre on each shot. A layer DoF issues all of its layer reads (the
// accumulated layer sums, the auxiliaries and their coefficients) at once, after its layer
// index; the halo numbers the layer DoFs last, so warps stay uniform.
template <int D>
__global__ void __launch_bounds__(256) node_kernel4(const StepArgs a) {
  typedef LayerCoef<D> L;
  const int S = a.S, ngrp = S >> 2;
  const int64_t total = (int64_t)a.hcnt * ngrp;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t i = t / ngrp;
  const int s0 = (int)(t - i * ngrp) * 4;
  const int dof = a.h0 + (int)i;
  const size_t ix = (size_t)dof * S + s0, rx = (size_t)i * S + s0;
  const float4 uo = ld4(a.u + ix), vo = ld4(a.v + ix), y = ldcg4(a.r + rx);
  const float c1 = __ldg(a.cf + dof), c2 = __ldg(a.cf + (size_t)a.N + dof);
  const float c3 = __ldg(a.cf + 2 * (size_t)a.N + dof);
  const int pi = __ldg(a.pidx + dof);
  st4(a.r + rx, make_float4(0.f, 0.f, 0.f, 0.f));
  float4 vn;
  vn.x = c1 * vo.x - c2 * y.x - c3 * uo.x;
  vn.y = c1 * vo.y - c2 * y.y - c3 * uo.y;
  vn.z = c1 * vo.z - c2 * y.z - c3 * uo.z;
  vn.w = c1 * vo.w - c2 * y.w - c3 * uo.w;
  if (pi >= 0) {
    const float* lc = a.lcf + (size_t)pi * L::COUNT;
    float4 sU[D], sY[D], Po[D];
    float e1[D], e2[D], e3[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const size_t pk = ((size_t)pi * D + k) * S + s0;
      sU[k] = ldcg4(a.Pacc + pk);
      Po[k] = ld4(a.P + pk);
      sY[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if constexpr (D == 3) {
        if (a.mode == 0) sY[k] = ldcg4(a.PaccY + pk);
      }
      e1[k] = __ldg(lc + L::E1 + k);
      e2[k] = __ldg(lc + (a.mode == 0 ? L::E2F : L::E2A) + k);
      e3[k] = D == 3 && a.mode == 0 ? __ldg(lc + L::E3F + k) : 0.f;
    }
    float4 Yo = make_float4(0.f, 0.f, 0.f, 0.f), yw = Yo;
    float cy0 = 0.f, cy1 = 0.f, cy2 = 0.f;
    const size_t py = (size_t)pi * S + s0;
    if constexpr (D == 3) {
      Yo = ld4(a.Y + py);
      if (a.mode == 1) yw = ldcg4(a.Yacc + py);
      cy0 = __ldg(lc + (a.mode == 0 ? L::C4 : L::C5));
      cy1 = __ldg(lc + L::DTDET);
      cy2 = __ldg(lc + L::DTM);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const size_t pk = ((size_t)pi * D + k) * S + s0;
      float4 pn;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float x = e1[k] * comp(Po[k], c) - e2[k] * comp(sU[k], c);  // e2: E2F or E2A
        if (D == 3 && a.mode == 0) x += e3[k] * comp(sY[k], c);
        setc(pn, c, x);
      }
      st4(a.P + pk, pn);
      st4(a.Pacc + pk, make_float4(0.f, 0.f, 0.f, 0.f));
      if constexpr (D == 3) {
        if (a.mode == 0) st4(a.PaccY + pk, make_float4(0.f, 0.f, 0.f, 0.f));
      }
    }
    if constexpr (D == 3) {
      float4 Yn;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float yo = comp(Yo, c), uc = comp(uo, c);
        if (a.mode == 0) {
          setc(vn, c, comp(vn, c) - cy0 * yo);
          setc(Yn, c, yo + a.dt * uc);
        } else {
          setc(vn, c, comp(vn, c) + cy0 * yo);
          setc(Yn, c, yo - cy1 * uc + cy2 * comp(yw, c));
        }
      }
      st4(a.Y + py, Yn);
      if (a.mode == 1) st4(a.Yacc + py, make_float4(0.f, 0.f, 0.f, 0.f));
    }
  }
  float4 un;
  un.x = uo.x + vn.x;
  un.y = uo.y + vn.y;
  un.z = uo.z + vn.z;
  un.w = uo.w + vn.w;
  st4(a.v + ix, vn);
  st4(a.u + ix, un);
  if (!(isfinite(un.x) && isfinite(un.y) && isfinite(un.z) && isfinite(un.w))) atomicOr(a.status, 1);
}

}  // namespace fwi
