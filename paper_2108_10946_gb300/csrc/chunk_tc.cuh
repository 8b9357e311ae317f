// Tensor-core chunk time step (2D). The same chunked assembly as chunk_kernel.cuh (one
// chunk of PE consecutive elements for a group of SG shots, assembled in shared memory), with
// the element stiffness action of the whole chunk done as two batched contractions on the
// fifth-generation tensor cores. Row r = (element, shot) of the chunk (r < 128):
//
//   step A   G[r][(d,q)] = sum_j U[r][j] Dhat_d[q][j]        the reference gradient of u at
//            every lumping node q of the element (Section 3.2: the stiffness integrand is
//            evaluated at the KMV nodes, which are the quadrature points);
//   pointwise F[r][(d,q)] = w_q c^2(x_q) (Ghat_e G_q)_d      plus the damping-layer and
//            gradient terms, one thread per row, straight from tensor memory;
//   step C   Y[r][i] = sum_{(d,q)} F[r][(d,q)] Dhat_d[q][i]  the element's contribution to
//            K u, scattered into the chunk table as before.
//
// Both contractions run as tf32 MMAs with the 3xTF32 split (x = hi + lo, hi = tf32(x);
// x y ~ hi_x hi_y + hi_x lo_y + lo_x hi_y, accumulated in FP32 in tensor memory), which keeps
// the product error near FP32's. U (and in gradient steps the forward field) is the A operand
// in shared memory; Dhat is the B operand in shared memory (loaded once per CTA: the kernel
// is persistent over chunks); F is the A operand of step C in tensor memory. Tensor memory
// (256 columns per CTA): G, overwritten by F_hi, at column 0; F_lo at 64; Y at 128; the
// forward field's G at 160.
//
// Every wait on the tensor cores is bounded: if one gives up, the CTA sets bit 1 of the
// status word, stops, frees its tensor memory and returns (the host reports FWI_ETIMEDOUT).
#pragma once
#include <cstring>

#include "tc_ptx.cuh"

namespace fwi {

template <int D, int NN>
struct TcShape {
  static constexpr int KA = (NN + 7) / 8 * 8;                   // K of step A
  static constexpr int NGV = D * NN;                            // (d, q) entries in use
  static constexpr int NG = (NGV + 15) / 16 * 16;               // N of step A = K of step C
  static constexpr int NY = (NN + 15) / 16 * 16 < 16 ? 16 : (NN + 15) / 16 * 16;  // N of step C
  static constexpr int BA = NG * KA;                            // floats of one B_A image
  static constexpr int BC = NY * NG;                            // floats of one B_C image
  static constexpr int BIMG = 2 * BA + 2 * BC;                  // hi and lo of both
  static constexpr int AROWS = 128 * KA;                        // floats of one A_U image
  static constexpr uint32_t COL_G = 0, COL_FLO = 64, COL_Y = 128, COL_GF = 160, COLS = 256;
  static_assert(NG <= 64 && NY <= 32, "tensor-memory map holds D * NN <= 64, NN <= 32");
};

// Host side: the B images (hi, lo) of Dhat [D][NN][NN] in the canonical K-major layout:
// B_A[n = d*NN + q][j] = Dhat[d][q][j], B_C[i][n] = Dhat[d][q][i]; zero padding.
template <int D, int NN>
inline void tc_build_bimg(const float* dhat, float* img) {
  typedef TcShape<D, NN> T;
  auto hi_of = [](float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;  // nearest tf32, ties away from zero
    float r;
    memcpy(&r, &u, 4);
    return r;
  };
  for (int i = 0; i < T::BIMG; ++i) img[i] = 0.f;
  for (int n = 0; n < T::NGV; ++n)
    for (int j = 0; j < NN; ++j) {
      const float x = dhat[n * NN + j], h = hi_of(x);
      img[tc::canon(n, j, T::KA)] = h;
      img[T::BA + tc::canon(n, j, T::KA)] = x - h;
      img[2 * T::BA + tc::canon(j, n, T::NG)] = h;
      img[2 * T::BA + T::BC + tc::canon(j, n, T::NG)] = x - h;
    }
}

// floats of dynamic shared memory of the tensor-core chunk kernel
template <int D, int NN>
inline size_t chunk_tc_smem_floats(int L, int SG, bool grad, bool layer) {
  typedef TcShape<D, NN> T;
  return (size_t)T::BIMG + (size_t)T::AROWS * (grad ? 4 : 2) + chunk_smem_floats(L, SG, D, grad, layer);
}

// 3xTF32 GEMM issue (one thread): D[128 x N] = A (shared, hi/lo) x B (shared, hi/lo)^T
__device__ __forceinline__ void tc_gemm_ss(uint32_t d, const float* ah, const float* al,
                                           const float* bh, const float* bl, int K, uint32_t idesc) {
  const uint32_t sbo = (uint32_t)K * 32;
  uint32_t acc = 0;
#pragma unroll 1
  for (int p = 0; p < 3; ++p) {
    const float* A = p == 2 ? al : ah;
    const float* B = p == 1 ? bl : bh;
    const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += 8) {
      tc::mma_ss(d, tc::sdesc(a0 + k0 * 32, 128, sbo), tc::sdesc(b0 + k0 * 32, 128, sbo), idesc, acc);
      acc = 1;
    }
  }
}
// the same with A (hi at column a_hi, lo at a_lo) in tensor memory
__device__ __forceinline__ void tc_gemm_ts(uint32_t d, uint32_t a_hi, uint32_t a_lo, const float* bh,
                                           const float* bl, int K, uint32_t idesc) {
  const uint32_t sbo = (uint32_t)K * 32;
  uint32_t acc = 0;
#pragma unroll 1
  for (int p = 0; p < 3; ++p) {
    const uint32_t A = p == 2 ? a_lo : a_hi;
    const uint32_t b0 = tc::smem_u32(p == 1 ? bl : bh);
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += 8) {
      tc::mma_ts(d, A + k0, tc::sdesc(b0 + k0 * 32, 128, sbo), idesc, acc);
      acc = 1;
    }
  }
}

// write one row (this thread's) of an A operand image: hi and lo of v[0..KA)
template <int KA>
__device__ __forceinline__ void tc_put_row(float* hi, float* lo, int row, const float* v) {
#pragma unroll
  for (int k = 0; k < KA; k += 4) {
    float4 h, l;
    h.x = tc::tf32_hi(v[k]);
    h.y = tc::tf32_hi(v[k + 1]);
    h.z = tc::tf32_hi(v[k + 2]);
    h.w = tc::tf32_hi(v[k + 3]);
    l.x = v[k] - h.x;
    l.y = v[k + 1] - h.y;
    l.z = v[k + 2] - h.z;
    l.w = v[k + 3] - h.w;
    *reinterpret_cast<float4*>(hi + tc::canon(row, k, KA)) = h;
    *reinterpret_cast<float4*>(lo + tc::canon(row, k, KA)) = l;
  }
}

constexpr int kTcWaitLimit = 1 << 22;

// MODE: 0 forward, 1 adjoint, 2 adjoint with the gradient integrand. Chunks
// [a.ch0, a.ch0 + nrun) are dealt to the CTAs round robin.
template <int D, int NN, int NS, int MODE, bool LAYER>
__device__ __forceinline__ void chunk_tc_body(const StepArgs& a, float* smem, const float* bimg,
                                              int nrun) {
  static_assert(D == 2, "tensor-core chunk kernel: triangles");
  typedef TcShape<D, NN> T;
  constexpr int NI = NN - NS;
  constexpr int KA = T::KA, NG = T::NG, NY = T::NY;
  typedef LayerCoef<D> LC;
  constexpr bool adj = MODE != 0;
  constexpr bool grad = MODE == 2;
  constexpr bool layer = LAYER;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
  const int S = a.S, SG = a.SG, s0 = blockIdx.y * SG;

  float* Bah = smem;  // B images: B_A hi, lo; B_C hi, lo
  float* Bal = Bah + T::BA;
  float* Bch = Bal + T::BA;
  float* Bcl = Bch + T::BC;
  float* Auh = Bcl + T::BC;  // A images of U (and of the forward field)
  float* Aul = Auh + T::AROWS;
  float* Afh = Aul + T::AROWS;
  float* Afl = Afh + (grad ? T::AROWS : 0);
  float* tab = Afl + (grad ? T::AROWS : 0);
  const int Lm = chunk_stride(a.L_max);
  float* uloc = tab;                       // [SG][Lm]
  float* yloc = uloc + (size_t)Lm * SG;    // [SG][Lm]
  float* c2loc = yloc + (size_t)Lm * SG;   // [Lm]
  float* Floc = c2loc + Lm;                // [SG][Lm] forward field (gradient)
  float* gloc = Floc + (grad ? (size_t)Lm * SG : 0);  // [Lm]
  float* sloc = gloc + (grad ? Lm : 0);               // [D*SG][Lm] layer scatter

  for (int i = tid; i < T::BIMG / 4; i += nth)
    reinterpret_cast<float4*>(smem)[i] = __ldg(reinterpret_cast<const float4*>(bimg) + i);
  if (warp == 0) tc::tmem_alloc(&tmem_base, T::COLS);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t lane = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's lanes
  uint32_t parity = 0;
  bool failed = false;

  const int P = a.PE;
  const int el = tid % P, sl = tid / P;
  const int s = s0 + sl;
  for (int c = a.ch0 + (int)blockIdx.x; c < a.ch0 + nrun; c += (int)gridDim.x) {
    const int* ch = a.chunks + 6 * c;
    const int e0 = ch[0], ne = ch[1], own_lo = ch[2], own_n = ch[3], nsh = ch[4], hp = ch[5];
    const int hn = a.chunks[6 * (c + 1) + 5] - hp;
    const int L = own_n + hn;

    // ---- 1. load the chunk table -------------------------------------------------------
    for (int i = tid; i < own_n * SG; i += nth) {
      const int l = i / SG, q = i - l * SG;
      const size_t g = (size_t)(own_lo + l) * S + s0 + q;
      uloc[q * Lm + l] = a.u[g];
      yloc[q * Lm + l] = 0.f;
      if (grad) Floc[q * Lm + l] = __ldg(a.ring_u + g);
    }
    for (int i = tid; i < hn * SG; i += nth) {
      const int h = i / SG, q = i - h * SG;
      const size_t g = (size_t)__ldg(a.halo + hp + h) * S + s0 + q;
      uloc[q * Lm + own_n + h] = a.u[g];
      yloc[q * Lm + own_n + h] = 0.f;
      if (grad) Floc[q * Lm + own_n + h] = __ldg(a.ring_u + g);
    }
    for (int l = tid; l < L; l += nth) {
      const int dof = l < own_n ? own_lo + l : __ldg(a.halo + hp + l - own_n);
      c2loc[l] = __ldg(a.c2 + dof);
      if (grad) gloc[l] = 0.f;
    }
    if (layer)
      for (int i = tid; i < Lm * D * SG; i += nth) sloc[i] = 0.f;
    __syncthreads();

    // ---- 2a. this thread's row of the A operands ----------------------------------------
    const bool valid = el < ne && sl < SG;
    const int e = e0 + el;
    int lq[NS];
    const int lb = nsh + el * NI;
    {
      float v[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) v[k] = 0.f;
      if (valid) {
        const float* ur = uloc + sl * Lm;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          lq[q] = __ldg(a.lconn + (size_t)q * a.E + e);
          v[q] = ur[lq[q]];
        }
#pragma unroll
        for (int j = 0; j < NI; ++j) v[NS + j] = ur[lb + j];
      }
      tc_put_row<KA>(Auh, Aul, tid, v);
      if (grad) {
#pragma unroll
        for (int k = 0; k < KA; ++k) v[k] = 0.f;
        if (valid) {
          const float* fr = Floc + sl * Lm;
#pragma unroll
          for (int q = 0; q < NS; ++q) v[q] = fr[lq[q]];
#pragma unroll
          for (int j = 0; j < NI; ++j) v[NS + j] = fr[lb + j];
        }
        tc_put_row<KA>(Afh, Afl, tid, v);
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      tc_gemm_ss(tmem + T::COL_G, Auh, Aul, Bah, Bal, KA, tc::idesc_tf32(128, NG));
      if (grad) tc_gemm_ss(tmem + T::COL_GF, Afh, Afl, Bah, Bal, KA, tc::idesc_tf32(128, NG));
      tc::mma_commit(&bar);
    }
    // element data while the tensor cores run
    float Gm[3] = {0.f, 0.f, 0.f}, Am[D * D];
#pragma unroll
    for (int cc = 0; cc < D * D; ++cc) Am[cc] = 0.f;
    if (valid) {
#pragma unroll
      for (int g = 0; g < 3; ++g) Gm[g] = __ldg(a.geo + (size_t)g * a.E + e);
      if (layer) {
        const int El = a.E - a.E0;
#pragma unroll
        for (int cc = 0; cc < D * D; ++cc) Am[cc] = __ldg(a.lgeo + (size_t)cc * El + (e - a.E0));
      }
    }
    auto gdof = [&](int l) { return l < own_n ? own_lo + l : __ldg(a.halo + hp + l - own_n); };
    {
      const bool ok = tc::mbar_wait(&bar, parity, kTcWaitLimit);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      parity ^= 1;
    }
    tc::fence_after_sync();

    // ---- 2b. pointwise: F from G at every node --------------------------------------------
    {
      float gv[NG];
      float gfv[grad ? NG : 1];
#pragma unroll
      for (int b = 0; b < NG; b += 16) tc::tmem_ld16(lane + T::COL_G + b, gv + b);
      if (grad) {  // warp-wide loads: outside the per-row branch
#pragma unroll
        for (int b = 0; b < NG; b += 16) tc::tmem_ld16(lane + T::COL_GF + b, gfv + b);
      }
      if (valid) {
#pragma unroll
        for (int q = 0; q < NN; ++q) {
          const int lqq = q < NS ? lq[q] : lb + (q - NS);
          const float g0 = gv[q], g1 = gv[NN + q];
          const float wq = c_w[q];
          const float wc = wq * c2loc[lqq];
          float f0 = wc * (Gm[0] * g0 + Gm[1] * g1);
          float f1 = wc * (Gm[1] * g0 + Gm[2] * g1);
          if (grad) {
            const float h0 = gfv[q], h1 = gfv[NN + q];
            const float dot = g0 * (Gm[0] * h0 + Gm[1] * h1) + g1 * (Gm[1] * h0 + Gm[2] * h1);
            atomicAdd(gloc + lqq, 2.f * __ldg(a.cvel + gdof(lqq)) * wq * dot);
          }
          if (layer) {
            const int pi = __ldg(a.pidx + gdof(lqq));
            if (pi >= 0) {
              const float* lc = a.lcf + (size_t)pi * LC::COUNT;
              float sq[2], pq[2];
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                sq[k] = wq * (Am[0 * 2 + k] * g0 + Am[1 * 2 + k] * g1);
                const float raw = a.P[((size_t)pi * 2 + k) * S + s];
                pq[k] = adj ? raw * __ldg(lc + LC::PSI2 + k) : raw;
              }
              f0 += wq * (Am[0] * pq[0] + Am[1] * pq[1]);
              f1 += wq * (Am[2] * pq[0] + Am[3] * pq[1]);
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                float* sp = sloc + (size_t)(k * SG + sl) * Lm + lqq;
                if (q < NS)
                  atomicAdd(sp, sq[k]);
                else
                  *sp = sq[k];
              }
            }
          }
          gv[q] = f0;
          gv[NN + q] = f1;
        }
#pragma unroll
        for (int n = T::NGV; n < NG; ++n) gv[n] = 0.f;
      } else {
#pragma unroll
        for (int n = 0; n < NG; ++n) gv[n] = 0.f;
      }
#pragma unroll
      for (int b = 0; b < NG; b += 16) {
        float h[16], l[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          h[i] = tc::tf32_hi(gv[b + i]);
          l[i] = gv[b + i] - h[i];
        }
        tc::tmem_st16(lane + T::COL_G + b, h);
        tc::tmem_st16(lane + T::COL_FLO + b, l);
      }
      tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      tc_gemm_ts(tmem + T::COL_Y, tmem + T::COL_G, tmem + T::COL_FLO, Bch, Bcl, NG,
                 tc::idesc_tf32(128, NY));
      tc::mma_commit(&bar);
    }
    {
      const bool ok = tc::mbar_wait(&bar, parity, kTcWaitLimit);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      parity ^= 1;
    }
    tc::fence_after_sync();

    // ---- 2c. element vector: sources, receivers, scatter into the chunk table -------------
    {
      float y[NY];
#pragma unroll
      for (int b = 0; b < NY; b += 16) tc::tmem_ld16(lane + T::COL_Y + b, y + b);
      if (valid) {
        const int slot = __ldg(a.inj + e);
        if (slot >= 0) {
          const int rb = __ldg(a.rslot_ptr + slot), re = __ldg(a.rslot_ptr + slot + 1);
          if (!adj) {
            if (a.rec != nullptr) {
              const float* ur = uloc + sl * Lm;
              for (int r = rb; r < re; ++r) {
                const float* ph = a.rslot_phi + (size_t)r * NN;
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < NS; ++q) acc = fmaf(__ldg(ph + q), ur[lq[q]], acc);
#pragma unroll
                for (int j = 0; j < NI; ++j) acc = fmaf(__ldg(ph + NS + j), ur[lb + j], acc);
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
              const float res =
                  __ldg(a.resid + ((size_t)s * (a.nt + 1) + a.n) * a.R + __ldg(a.rslot_rec + r));
#pragma unroll
              for (int k = 0; k < NN; ++k) y[k] = fmaf(res, __ldg(a.rslot_phi + (size_t)r * NN + k), y[k]);
            }
          }
        }
        float* yr = yloc + sl * Lm;
#pragma unroll
        for (int q = 0; q < NS; ++q) atomicAdd(yr + lq[q], y[q]);
#pragma unroll
        for (int j = 0; j < NI; ++j) yr[lb + j] = y[NS + j];
      }
    }
    tc::fence_before_sync();
    __syncthreads();

    // ---- 3. owned DoFs: final update; halo DoFs: to the global accumulators ----------------
    for (int i = tid; i < own_n * SG; i += nth) {
      const int l = i / SG, q = i - l * SG, s2 = s0 + q;
      float sU[D], sY[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        sU[k] = layer ? sloc[(size_t)(k * SG + q) * Lm + l] : 0.f;
        sY[k] = 0.f;
      }
      dof_update<D>(a, own_lo + l, s2, yloc[q * Lm + l], uloc[q * Lm + l], sU, sY, 0.f);
    }
    for (int i = tid; i < hn * SG; i += nth) {
      const int h = i / SG, q = i - h * SG, s2 = s0 + q;
      const int dof = __ldg(a.halo + hp + h);
      const int l = own_n + h;
      atomicAdd(a.r + (size_t)(dof - a.N_own) * S + s2, yloc[q * Lm + l]);
      if (layer) {
        const int pi = __ldg(a.pidx + dof);
        if (pi >= 0) {
#pragma unroll
          for (int k = 0; k < D; ++k)
            atomicAdd(a.Pacc + ((size_t)pi * D + k) * S + s2, sloc[(size_t)(k * SG + q) * Lm + l]);
        }
      }
    }
    if (grad) {
      for (int l = tid; l < L; l += nth) {
        const int dof = l < own_n ? own_lo + l : __ldg(a.halo + hp + l - own_n);
        atomicAdd(a.gseg + dof, gloc[l]);
      }
    }
    __syncthreads();
  }

  if (failed) {
    // a wait gave up: report it, give the tensor cores one more bounded wait for the
    // MMAs still in flight, then free the tensor memory
    if (tid == 0) atomicOr(a.status, 2);
    tc::mbar_wait(&bar, parity, kTcWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, T::COLS);
  }
}

}  // namespace fwi
