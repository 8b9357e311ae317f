// One explicit time step of the mass-lumped KMV acoustic scheme, element by element.
//
// Work of one thread: one element e for one shot s (the S lanes of an element are
// adjacent, so every gather reads S contiguous floats of the shot-interleaved fields).
//
//   forward  (Eq. forward3): y_i = sum_q Dhat[q][i] . f_q with
//              f_q = w_q c_q^2 Ghat ghat_q + w_q A P_q            (K U + D P)
//            ghat_q = sum_j Dhat[q][j] U_j, Ghat = |J| J^-1 J^-T, A = |J| J^-1;
//            layer scatter s_q = w_q A^T ghat_q                    (lumped G U of D_{u,2})
//   adjoint  (Section 3.5, transposed recurrence): the same with U -> lam and
//            P -> Psi2 c^2 nu (Q^T nu), s_q giving D^T lam; with the forward field U^m of
//            the recompute ring it also forms the integrand of Eq. (gradient3),
//              2 c_q w_q (ghat lam_q)^T Ghat (ghat U_q).
//
// Shared (vertex/edge/face) nodes are scattered with atomics into r and finished by the
// node kernel; element-interior (bubble) nodes belong to this element alone, so the
// increment update of their u, v (and layer auxiliaries) happens here, in registers.
//
// Every unrolled loop indexes the reference derivative matrices with compile-time
// constants, so each FMA takes its Dhat operand straight from the constant bank.
// Include after declaring, in namespace fwi, the unit's
//   __constant__ float c_dhat[D * NN * NN];  __constant__ float c_w[NN];
#include "update.cuh"

namespace fwi {

// c_dhat [D][NN][NN] and c_w [NN] are the __constant__ arrays of the including unit.
template <int D, int NN, int NS>
__device__ __forceinline__ void step_body(const StepArgs& a) {
  constexpr int NI = NN - NS;
  constexpr int NG = D == 2 ? 3 : 6;
  typedef LayerCoef<D> L;
  const int S = a.S;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int e_raw = t >> a.log2S;
  const int s = t & (S - 1);
  const bool valid = e_raw < a.E;
  const int e = valid ? e_raw : a.E - 1;
  const bool adj = a.mode == 1;
  const bool grad = adj && a.ring_u != nullptr;
  const bool layer = e >= a.E0;
  const int ib = __ldg(a.bub + e);

  int dof[NS];
  float U[NN];
#pragma unroll
  for (int q = 0; q < NS; ++q) dof[q] = __ldg(a.conn + (size_t)q * a.E + e);
#pragma unroll
  for (int q = 0; q < NS; ++q) U[q] = a.u[(size_t)dof[q] * S + s];
#pragma unroll
  for (int j = 0; j < NI; ++j) U[NS + j] = a.u[(size_t)(ib + j) * S + s];
  float G[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) G[g] = __ldg(a.geo + (size_t)g * a.Es + e);
  float Am[D * D];
  const int El = a.E - a.E0;
#pragma unroll
  for (int c = 0; c < D * D; ++c) Am[c] = layer ? __ldg(a.lgeo + (size_t)c * El + (e - a.E0)) : 0.f;

  float F[NN];  // forward field U^m (gradient only)
  if (grad) {
#pragma unroll
    for (int q = 0; q < NS; ++q) F[q] = __ldg(a.ring_u + (size_t)dof[q] * S + s);
#pragma unroll
    for (int j = 0; j < NI; ++j) F[NS + j] = __ldg(a.ring_u + (size_t)(ib + j) * S + s);
  }
  float Yv[NN];  // 3D forward: omega at the nodes (dead code in 2D)
#pragma unroll
  for (int q = 0; q < NN; ++q) Yv[q] = 0.f;
  if constexpr (D == 3) {
    if (layer && !adj) {
#pragma unroll
      for (int q = 0; q < NN; ++q) {
        const int dq = q < NS ? dof[q] : ib + (q - NS);
        const int pi = __ldg(a.pidx + dq);
        Yv[q] = pi >= 0 ? a.Y[(size_t)pi * S + s] : 0.f;
      }
    }
  }

  static_assert(NI > 0, "every KMV element has interior (bubble) nodes");
  float y[NN], yw[NN];  // yw: 3D adjoint omega-row scatter (dead code in 2D)
  float sI[NI][D], sYI[NI][D];
#pragma unroll
  for (int i = 0; i < NN; ++i) y[i] = yw[i] = 0.f;
#pragma unroll
  for (int j = 0; j < NI; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) sI[j][k] = sYI[j][k] = 0.f;

#pragma unroll
  for (int q = 0; q < NN; ++q) {
    const int dq = q < NS ? dof[q] : ib + (q - NS);
    float g[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < NN; ++j) acc = fmaf(c_dhat[(d * NN + q) * NN + j], U[j], acc);
      g[d] = acc;
    }
    const float wq = c_w[q];
    const float wc = wq * __ldg(a.c2 + dq);
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
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < NN; ++j) acc = fmaf(c_dhat[(d * NN + q) * NN + j], F[j], acc);
        gf[d] = acc;
      }
      float dot;
      if constexpr (D == 2) {
        dot = g[0] * (G[0] * gf[0] + G[1] * gf[1]) + g[1] * (G[1] * gf[0] + G[2] * gf[1]);
      } else {
        dot = g[0] * (G[0] * gf[0] + G[1] * gf[1] + G[2] * gf[2]) +
              g[1] * (G[1] * gf[0] + G[3] * gf[1] + G[4] * gf[2]) +
              g[2] * (G[2] * gf[0] + G[4] * gf[1] + G[5] * gf[2]);
      }
      const float val = 2.f * __ldg(a.cvel + dq) * wq * dot;
      if (valid) {  // per-shot segment accumulators [S][N], or one [N] for all shots
        float* gs = a.gseg + (a.grad_lanes ? (size_t)s * a.N : 0);
        if (q < NS || !a.grad_lanes)
          atomicAdd(gs + dq, val);
        else
          gs[dq] += val;  // a bubble DoF of this element and shot: this thread only
      }
    }
    if (layer) {
      const int pi = __ldg(a.pidx + dq);
      if (pi >= 0) {
        const float* lc = a.lcf + (size_t)pi * L::COUNT;
        float sq[D], pq[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          float acc = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) acc += Am[d * D + k] * g[d];
          sq[k] = wq * acc;
          const float raw = a.P[((size_t)pi * D + k) * S + s];
          pq[k] = adj ? raw * __ldg(lc + L::PSI2 + k) : raw;
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
            // omega row: Q_omega^T lam_p = D (Psi3 c^2 lam_p), a second divergence scatter
            float pw[3], fw[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
              pw[k] = a.P[((size_t)pi * 3 + k) * S + s] * __ldg(lc + L::PSI3 + k);
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
        if (q < NS) {
          if (valid) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
              atomicAdd(a.Pacc + ((size_t)pi * D + k) * S + s, sq[k]);
              if constexpr (D == 3) {
                if (!adj) atomicAdd(a.PaccY + ((size_t)pi * D + k) * S + s, sY[k]);
              }
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            sI[q - NS][k] = sq[k];
            sYI[q - NS][k] = sY[k];
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NN; ++i)
#pragma unroll
      for (int d = 0; d < D; ++d) y[i] = fmaf(c_dhat[(d * NN + q) * NN + i], f[d], y[i]);
  }

  // sources and receivers of this element (rare: flagged elements only)
  const int slot = __ldg(a.inj + e);
  if (slot >= 0) {
    const int rb = __ldg(a.rslot_ptr + slot), re = __ldg(a.rslot_ptr + slot + 1);
    if (!adj) {
      if (a.rec != nullptr && valid) {
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

  if (!valid) return;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    atomicAdd(a.r + (size_t)dof[q] * S + s, y[q]);
    if constexpr (D == 3) {
      if (layer && adj) {
        const int pi = __ldg(a.pidx + dof[q]);
        if (pi >= 0) atomicAdd(a.Yacc + (size_t)pi * S + s, yw[q]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NI; ++j) dof_update<D>(a, ib + j, s, y[NS + j], U[NS + j], sI[j], sYI[j], yw[NS + j]);
}

// Receiver samples d^n = H U^n for every (receiver, shot), used for the last sample.
template <int NN, int NS>
__global__ void record_kernel(const StepArgs a, const int* rec_elem, const float* rec_phi) {
  constexpr int NI = NN - NS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.R * a.S) return;
  const int r = t % a.R, s = t / a.R;
  const int e = __ldg(rec_elem + r);
  float acc = 0.f;
#pragma unroll
  for (int q = 0; q < NS; ++q)
    acc = fmaf(__ldg(rec_phi + (size_t)r * NN + q), a.u[(size_t)__ldg(a.conn + (size_t)q * a.E + e) * a.S + s], acc);
#pragma unroll
  for (int j = 0; j < NI; ++j)
    acc = fmaf(__ldg(rec_phi + (size_t)r * NN + NS + j), a.u[(size_t)(__ldg(a.bub + e) + j) * a.S + s], acc);
  a.rec[((size_t)s * (a.nt + 1) + a.n) * a.R + r] = acc;
}

}  // namespace fwi
