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
// Both contractions run as tf32 MMAs with the 3xTF32 split: x = hi + lo with hi and lo the
// nearest tf32 values of x and of x - hi, and x y ~ hi_x hi_y + hi_x lo_y + lo_x hi_y,
// accumulated in FP32 in tensor memory. The A operands (U, the forward field, F) sit in
// tensor memory, written row by row by their threads; Dhat is the B operand in shared memory
// (loaded once per CTA: the kernel is persistent over chunks). Tensor memory, 256 columns
// per CTA:
//   [  0,  64)  A of U (hi at 0, lo at 32); after step A: F_lo
//   [ 64, 128)  A of the forward field (gradient steps; hi at 64, lo at 96); after step A: Y
//   [128, 192)  G, overwritten by F_hi
//   [192, 256)  G of the forward field (gradient steps)
//
// All global reads of a chunk are issued at once as asynchronous copies (cp.async) into the
// chunk table: first the values the element phase needs (u, c^2, the forward field), then
// those only the final update needs (v, the update coefficients, the layer index), whose
// latency hides behind the element phase.
//
// Every wait on the tensor cores is bounded: if one gives up, the CTA sets bit 1 of the
// status word, stops, frees its tensor memory and returns (the host reports FWI_ETIMEDOUT).
#pragma once
#include <cstring>

#include "chunk_io.cuh"
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
  static constexpr uint32_t COL_AU = 0, COL_FLO = 0, COL_AF = 64, COL_Y = 64, COL_G = 128,
                            COL_GF = 192, COLS = 256, LO = 32;
  static_assert(KA <= 32 && NG <= 64 && NY <= 64, "tensor-memory map: NN <= 32, D * NN <= 64");
};

// Host side: the B images (hi, lo) of Dhat [D][NN][NN] in the canonical K-major layout:
// B_A[n = d*NN + q][j] = Dhat[d][q][j], B_C[i][n] = Dhat[d][q][i]; zero padding.
template <int D, int NN>
inline void tc_build_bimg(const float* dhat, float* img) {
  typedef TcShape<D, NN> T;
  auto tf32 = [](float x) {
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
      const float x = dhat[n * NN + j], h = tf32(x), l = tf32(x - h);
      img[tc::canon(n, j, T::KA)] = h;
      img[T::BA + tc::canon(n, j, T::KA)] = l;
      img[2 * T::BA + tc::canon(j, n, T::NG)] = h;
      img[2 * T::BA + T::BC + tc::canon(j, n, T::NG)] = l;
    }
}

// floats of dynamic shared memory of the tensor-core chunk kernel
template <int D, int NN>
inline size_t chunk_tc_smem_floats(int L, int SG, bool grad, bool layer) {
  return (size_t)TcShape<D, NN>::BIMG + chunk_tab_floats(L, SG, D, grad, layer);
}

// 3xTF32 GEMM issue (one thread): D[128 x N] = A (tensor memory: hi at a_hi, lo at a_lo)
// x B (shared, hi/lo images)^T over K
__device__ __forceinline__ void tc_gemm(uint32_t d, uint32_t a_hi, uint32_t a_lo, const float* bh,
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

// this thread's row of an A operand in tensor memory: the hi parts of v[0..K) from address
// lane_col on, the lo parts lo_off columns further
template <int K>
__device__ __forceinline__ void tc_put_row(uint32_t lane_col, uint32_t lo_off, const float* v) {
#pragma unroll
  for (int k = 0; k < K; k += 8) {
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = tc::tf32_hi(v[k + i]);
      l[i] = tc::tf32_hi(v[k + i] - h[i]);
    }
    tc::tmem_st8(lane_col + k, h);
    tc::tmem_st8(lane_col + lo_off + k, l);
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
  const size_t N = (size_t)a.N;

  float* Bah = smem;  // B images: B_A hi, lo; B_C hi, lo
  float* Bal = Bah + T::BA;
  float* Bch = Bal + T::BA;
  float* Bcl = Bch + T::BC;
  const int Lm = chunk_stride(a.L_max);
  const int lg = __ffs(SG) - 1;
  const ChunkTab t = chunk_tab(Bcl + T::BC, Lm, SG, D, grad, layer);
  float* uloc = t.u;
  float* yloc = t.y;
  float* c2loc = t.c2;
  float* Floc = t.F;
  float* gloc = t.g;
  float* sloc = t.s;

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
    const ChunkDesc cd = chunk_desc(a, c);
    const int e0 = cd.e0, ne = cd.ne, nsh = cd.nsh;

    // ---- 1. the chunk's global reads, all in flight at once -------------------------------
    chunk_load<D, grad, layer>(a, cd, t, Lm, SG, lg, s0, tid, nth);
    // this thread's element: local connectivity and geometry, read while the copies fly
    const bool valid = el < ne && sl < SG;
    const int e = e0 + el;
    int lq[NS];
    const int lb = nsh + el * NI;
    float Gm[3] = {0.f, 0.f, 0.f}, Am[D * D];
#pragma unroll
    for (int cc = 0; cc < D * D; ++cc) Am[cc] = 0.f;
    if (valid) {
#pragma unroll
      for (int q = 0; q < NS; ++q) lq[q] = __ldg(a.lconn + (size_t)q * a.Es + e);
#pragma unroll
      for (int g = 0; g < 3; ++g) Gm[g] = __ldg(a.geo + (size_t)g * a.Es + e);
      if (layer) {
        const int El = a.E - a.E0;
#pragma unroll
        for (int cc = 0; cc < D * D; ++cc) Am[cc] = __ldg(a.lgeo + (size_t)cc * El + (e - a.E0));
      }
    }
    cp_async_wait<1>();  // the element phase's group
    __syncthreads();
    if (layer) {
      if (!grad) chunk_load_layer<D>(a, cd, t, Lm, SG, lg, s0, tid, nth);
      chunk_prefetch_update<D>(a, cd, t, SG, s0, tid, nth);
      cp_async_wait<0>();
      __syncthreads();
    }

    // ---- 2a. this thread's rows of the A operands -----------------------------------------
    {
      float v[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) v[k] = 0.f;
      if (valid) {
        const float* ur = uloc + sl * Lm;
#pragma unroll
        for (int q = 0; q < NS; ++q) v[q] = ur[lq[q]];
#pragma unroll
        for (int j = 0; j < NI; ++j) v[NS + j] = ur[lb + j];
      }
      tc_put_row<KA>(lane + T::COL_AU, T::LO, v);
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
        tc_put_row<KA>(lane + T::COL_AF, T::LO, v);
      }
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      tc_gemm(tmem + T::COL_G, tmem + T::COL_AU, tmem + T::COL_AU + T::LO, Bah, Bal, KA,
              tc::idesc_tf32(128, NG));
      if (grad)
        tc_gemm(tmem + T::COL_GF, tmem + T::COL_AF, tmem + T::COL_AF + T::LO, Bah, Bal, KA,
                tc::idesc_tf32(128, NG));
      tc::mma_commit(&bar);
    }
    {
      const bool ok = tc::mbar_wait(&bar, parity, a.tc_wait_limit);
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
            atomicAdd(gloc + (a.grad_lanes ? sl * Lm : 0) + lqq, 2.f * t.cv[lqq] * wq * dot);
          }
          if (layer) {
            const int pi = t.pi[lqq];
            if (pi >= 0) {
              const float* lc = a.lcf + (size_t)pi * LC::COUNT;
              float sq[2], pq[2];
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                sq[k] = wq * (Am[0 * 2 + k] * g0 + Am[1 * 2 + k] * g1);
                const float raw = grad ? a.P[((size_t)pi * D + k) * S + s] : t.P[(size_t)(k * SG + sl) * Lm + lqq];
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
          l[i] = tc::tf32_hi(gv[b + i] - h[i]);
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
      tc_gemm(tmem + T::COL_Y, tmem + T::COL_G, tmem + T::COL_FLO, Bch, Bcl, NG,
              tc::idesc_tf32(128, NY));
      tc::mma_commit(&bar);
    }
    {
      const bool ok = tc::mbar_wait(&bar, parity, a.tc_wait_limit);
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
    cp_async_wait<0>();  // the update's group
    tc::fence_before_sync();
    __syncthreads();

    // ---- 3. owned DoFs: final update; halo DoFs: to the global accumulators ----------------
    chunk_store<D, grad, layer>(a, cd, t, Lm, SG, lg, s0, tid, nth);
    __syncthreads();
  }

  if (failed) {
    // a wait gave up: report it, give the tensor cores one more bounded wait (the full
    // default limit, whatever the batch's setting) for the MMAs still in flight, then free the
    // tensor memory
    if (tid == 0) atomicOr(a.status, 2);
    tc::mbar_wait(&bar, parity, kTcWaitLimit);
  }
  cp_async_wait<0>();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, T::COLS);
  }
}

}  // namespace fwi
