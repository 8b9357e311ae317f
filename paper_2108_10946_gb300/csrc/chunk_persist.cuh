// Persistent, pipelined chunk kernel for triangles without damping-layer elements, batches
// of S >= 4 shots (work item = one chunk x four shots).
//
// Each CTA (256 threads, two per SM) walks a fixed list of work items. While it computes one
// chunk, the reads of the next ones are already in flight as asynchronous copies:
//
//   iteration i:  wait for every copy issued in iteration i-1; barrier
//                 issue  data of item i+1   (u, v, c^2, c1..c3, Ghat, local connectivity,
//                                            source/receiver flags; halo DoFs through the
//                                            halo ids of item i+1)       -> buffer (i+1)%2
//                        halo ids of item i+2 (needs its descriptor)      -> meta slot (i+2)%4
//                        descriptor of item i+3                           -> meta slot (i+3)%4
//                 element phase of item i (buffer i%2), barrier
//                 update of the owned DoFs, halo sums to the global accumulator, barrier
//
// so a chunk's global reads are hidden behind the previous chunk's arithmetic; the only
// waits are cp.async group waits on the CTA's own copies and __syncthreads.
//
// Element phase: two threads per (element, shot), one per reference direction d. Thread d
// streams row q of Dhat_d (shared memory), forms g_d = (Dhat_d u)_q, swaps it with its
// partner (shuffle) to have grad u at node q, forms f_d = w_q c_q^2 (Ghat grad u)_d and adds
// Dhat_d[q][:] f_d to its partial y; the two partial y are summed by shuffles at the end
// (Section 3.2: the stiffness action sum_q w_q c^2 (J^-T grad phi_i . J^-T grad u)(x_q) with the
// quadrature points at the nodes). Holding one row instead of two keeps a thread under 128
// registers.
//
// Table layouts in shared memory are DoF-major with the four shots contiguous ([L][4]), so
// that one 16-byte copy moves a DoF's four shots and the update phase works on float4.
//
// Gradient steps (Eq. gradient3) from a stored forward field: the forward recompute steps of
// an adjoint segment write, per (element, node q, shot, direction), h_d = (Ghat grad u)_d of
// the forward field at that level (`gstore`, [item][q][shot][element][d]: one warp writes
// 128 contiguous bytes per node). The gradient step of the same level reads it back
// (`gload`): thread d has the adjoint's own g_d = (Dhat_d u_dag)_q, so the integrand
// 2 c_q w_q (Ghat grad u) . grad u_dag is one product per thread and one shuffle per node,
// instead of a second contraction over the forward field's nodal values.
#pragma once
#include "chunk_kernel.cuh"

namespace fwi {

constexpr int PT_THREADS = 256;  // 32 elements x 4 shots x 2 directions
constexpr int PT_PE = 32;        // elements per chunk (triangles)
constexpr int PT_SG = 4;         // shots per work item
static_assert(PT_SG * PT_PE * 2 == kGstoreNodeFloats, "stored-gradient layout");

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

__host__ __device__ inline uint32_t pt_al16(uint32_t x) { return (x + 15u) & ~15u; }

// Byte offsets of the persistent kernel's dynamic shared memory.
struct PtLayout {
  uint32_t rows, rows_dstride;  // Dhat rows [2][NN][NNP] floats; direction stride (floats)
  uint32_t y;                   // accumulator [Lmax][4]
  uint32_t g;                   // gradient accumulator [Lmax] (gradient steps only)
  uint32_t meta0, meta_stride;  // 4 slots: descriptor (8 ints) + halo ids [Hmax]
  uint32_t buf0, buf_stride;    // 2 buffers
  uint32_t bu, bc2, bv, bcf, bcf_stride, bgeo, binj, blq;  // inside a buffer
  uint32_t total;
};

template <int NN, int NS>
__host__ __device__ inline PtLayout pt_layout(int Lmax, int Omax, int Hmax, bool grad = false) {
  constexpr int NNP = (NN + 3) / 4 * 4;
  PtLayout L{};
  uint32_t o = 0;
  L.rows = o;
  // the second direction's rows start 16 bytes past a bank-aligned offset, so that the two
  // rows a warp reads at once (one per direction) sit in different banks
  L.rows_dstride = (uint32_t)(NN * NNP + 4);
  o += pt_al16(4u * (2u * L.rows_dstride));
  L.y = o;
  o += pt_al16(16u * (uint32_t)Lmax);
  L.g = o;
  o += grad ? pt_al16(4u * (uint32_t)Lmax) : 0u;
  L.meta0 = o;
  L.meta_stride = pt_al16(32u + 4u * (uint32_t)Hmax);
  o += 4u * L.meta_stride;
  uint32_t b = 0;
  L.bu = b;
  b += pt_al16(16u * (uint32_t)Lmax);
  L.bc2 = b;
  b += pt_al16(4u * (uint32_t)Lmax);
  L.bv = b;
  b += pt_al16(16u * (uint32_t)Omax);
  L.bcf = b;
  L.bcf_stride = pt_al16(4u * (uint32_t)Omax);
  b += 3u * L.bcf_stride;
  L.bgeo = b;
  b += 3u * PT_PE * 4u;
  L.binj = b;
  b += PT_PE * 4u;
  L.blq = b;
  b += pt_al16((uint32_t)NS * PT_PE * 2u);
  L.buf_stride = pt_al16(b);
  L.buf0 = o;
  o += 2u * L.buf_stride;
  L.total = o;
  return L;
}

// Work item w of a launch over chunks [ch0, ch0 + nch): chunk ch0 + w / ngrp, shots
// [4 (w % ngrp), 4 (w % ngrp) + 4).
struct PtItem {
  int c, s0;
  bool valid;
};

__device__ __forceinline__ PtItem pt_item(const StepArgs& a, int i, int nwork, int ngrp) {
  PtItem it;
  const int w = blockIdx.x + i * gridDim.x;
  it.valid = w < nwork;
  it.c = a.ch0 + (it.valid ? w / ngrp : 0);
  it.s0 = it.valid ? (w % ngrp) * PT_SG : 0;
  return it;
}

// descriptor of item i: chunk fields e0, ne, own_lo, own_n, nsh, hp and the next chunk's hp
__device__ __forceinline__ void pt_issue_desc(const StepArgs& a, const PtLayout& L, char* sm,
                                              int i, int nwork, int ngrp) {
  const PtItem it = pt_item(a, i, nwork, ngrp);
  if (!it.valid) return;
  int* desc = reinterpret_cast<int*>(sm + L.meta0 + (i & 3) * L.meta_stride);
  const int t = threadIdx.x;
  if (t < 6) cp_async4(desc + t, a.chunks + 6 * it.c + t);
  if (t == 6) cp_async4(desc + 6, a.chunks + 6 * (it.c + 1) + 5);
}

__device__ __forceinline__ void pt_issue_halo(const StepArgs& a, const PtLayout& L, char* sm,
                                              int i, int nwork, int ngrp) {
  const PtItem it = pt_item(a, i, nwork, ngrp);
  if (!it.valid) return;
  char* meta = sm + L.meta0 + (i & 3) * L.meta_stride;
  const int* desc = reinterpret_cast<const int*>(meta);
  int* ids = reinterpret_cast<int*>(meta + 32);
  const int hp = desc[5], hn = desc[6] - desc[5];
  for (int h = threadIdx.x; h < hn; h += PT_THREADS) cp_async4(ids + h, a.halo + hp + h);
}

template <int NS>
__device__ __forceinline__ void pt_issue_data(const StepArgs& a, const PtLayout& L, char* sm, int i,
                                              int nwork, int ngrp) {
  const PtItem it = pt_item(a, i, nwork, ngrp);
  if (!it.valid) return;
  const char* meta = sm + L.meta0 + (i & 3) * L.meta_stride;
  const int* desc = reinterpret_cast<const int*>(meta);
  const int* ids = reinterpret_cast<const int*>(meta + 32);
  char* B = sm + L.buf0 + (i & 1) * L.buf_stride;
  const int e0 = desc[0], own_lo = desc[2], own_n = desc[3], hn = desc[6] - desc[5];
  const int S = a.S, s0 = it.s0, t = threadIdx.x;
  float* bu = reinterpret_cast<float*>(B + L.bu);
  float* bv = reinterpret_cast<float*>(B + L.bv);
  float* bc2 = reinterpret_cast<float*>(B + L.bc2);
  for (int l = t; l < own_n; l += PT_THREADS) {
    const size_t gi = (size_t)(own_lo + l) * S + s0;
    const size_t dof = (size_t)(own_lo + l);
    cp_async16(bu + 4 * l, a.u + gi);
    cp_async4(bc2 + l, a.c2 + dof);
    cp_async16(bv + 4 * l, a.v + gi);
#pragma unroll
    for (int r = 0; r < 3; ++r)
      cp_async4(reinterpret_cast<float*>(B + L.bcf + r * L.bcf_stride) + l, a.cf + (size_t)r * a.N + dof);
  }
  for (int h = t; h < hn; h += PT_THREADS) {
    const int id = ids[h];
    const size_t gi = (size_t)id * S + s0;
    cp_async16(bu + 4 * (own_n + h), a.u + gi);
    cp_async4(bc2 + own_n + h, a.c2 + id);
  }
  // per-element arrays of the chunk's 32 elements (rows padded to a multiple of 32 elements,
  // e0 a multiple of 32 for chunks without layer elements: whole 16-byte groups)
  if (t < 24) {
    const int g = t >> 3, part = t & 7;
    cp_async16(B + L.bgeo + (g * PT_PE + part * 4) * 4, a.geo + (size_t)g * a.Es + e0 + part * 4);
  } else if (t < 32) {
    const int part = t - 24;
    cp_async16(B + L.binj + part * 16, a.inj + e0 + part * 4);
  } else if (t < 32 + 4 * NS) {
    const int q = (t - 32) >> 2, part = (t - 32) & 3;
    cp_async16(B + L.blq + (q * PT_PE + part * 8) * 2, a.lconn + (size_t)q * a.Es + e0 + part * 8);
  }
}

// Gradient steps: bring item i's stored forward-field gradients (NN x 1 KB) to L2 while the
// CTA still computes the item before it, so that the element phase's reads hit L2.
template <int NN>
__device__ __forceinline__ void pt_prefetch_gload(const StepArgs& a, int i, int nwork, int ngrp) {
  const PtItem it = pt_item(a, i, nwork, ngrp);
  if (!it.valid) return;
  const float* base = a.gload + ((size_t)((it.c - a.ch0) * ngrp + it.s0 / PT_SG) * NN) * kGstoreNodeFloats;
  constexpr int lines = NN * kGstoreNodeFloats * 4 / 128;
  for (int l = threadIdx.x; l < lines; l += PT_THREADS)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (size_t)l * 32));
}

template <int NN, int NS, int MODE>
__device__ __forceinline__ void pt_body(const StepArgs& a, char* sm, int nwork) {
  constexpr int NI = NN - NS;
  constexpr int NNP = (NN + 3) / 4 * 4;
  constexpr bool ROLL = NN >= 16;
  constexpr bool GRAD = MODE == 2;
  constexpr bool ADJ = MODE != 0;
  const int ngrp = a.S / PT_SG;
  const PtLayout L = pt_layout<NN, NS>(a.L_max, a.O_max, a.H_max, GRAD);
  const int t = threadIdx.x;
  float* rows = reinterpret_cast<float*>(sm + L.rows);
  float4* Y4 = reinterpret_cast<float4*>(sm + L.y);
  float* Y = reinterpret_cast<float*>(sm + L.y);

  // Dhat rows (once per CTA) and a zero accumulator table
  for (int idx = t; idx < 2 * (int)L.rows_dstride; idx += PT_THREADS) {
    const int d = idx / (int)L.rows_dstride, rem = idx - d * (int)L.rows_dstride;
    const int q = rem / NNP, j = rem - q * NNP;
    rows[idx] = (q < NN && j < NN) ? c_dhat[(d * NN + q) * NN + j] : 0.f;
  }
  for (int l = t; l < a.L_max; l += PT_THREADS) Y4[l] = make_float4(0.f, 0.f, 0.f, 0.f);
  float* Gacc = reinterpret_cast<float*>(sm + L.g);
  if (GRAD)
    for (int l = t; l < a.L_max; l += PT_THREADS) Gacc[l] = 0.f;

  // prologue: descriptors of items 0, 1; halo ids of 0, 1 and descriptor of 2; data of 0
  pt_issue_desc(a, L, sm, 0, nwork, ngrp);
  pt_issue_desc(a, L, sm, 1, nwork, ngrp);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  pt_issue_halo(a, L, sm, 0, nwork, ngrp);
  pt_issue_halo(a, L, sm, 1, nwork, ngrp);
  pt_issue_desc(a, L, sm, 2, nwork, ngrp);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  pt_issue_data<NS>(a, L, sm, 0, nwork, ngrp);
  cp_async_commit();
  if constexpr (GRAD) pt_prefetch_gload<NN>(a, 0, nwork, ngrp);

  const int d = t & 1, es = t >> 1, el = es & (PT_PE - 1), sl = es >> 5;
  bool bad = false;
  for (int i = 0;; ++i) {
    const PtItem it = pt_item(a, i, nwork, ngrp);
    if (!it.valid) break;
    cp_async_wait<0>();
    __syncthreads();
    pt_issue_data<NS>(a, L, sm, i + 1, nwork, ngrp);
    pt_issue_halo(a, L, sm, i + 2, nwork, ngrp);
    pt_issue_desc(a, L, sm, i + 3, nwork, ngrp);
    cp_async_commit();
    if constexpr (GRAD) pt_prefetch_gload<NN>(a, i + 1, nwork, ngrp);

    const char* meta = sm + L.meta0 + (i & 3) * L.meta_stride;
    const int* desc = reinterpret_cast<const int*>(meta);
    const int* ids = reinterpret_cast<const int*>(meta + 32);
    const int e0 = desc[0], ne = desc[1], own_lo = desc[2], own_n = desc[3], nsh = desc[4];
    const int hn = desc[6] - desc[5];
    const char* B = sm + L.buf0 + (i & 1) * L.buf_stride;
    const float* bu = reinterpret_cast<const float*>(B + L.bu);
    const float* bc2 = reinterpret_cast<const float*>(B + L.bc2);
    const float* bgeo = reinterpret_cast<const float*>(B + L.bgeo);
    const int* binj = reinterpret_cast<const int*>(B + L.binj);
    const unsigned short* blq = reinterpret_cast<const unsigned short*>(B + L.blq);

    // ---- element phase ------------------------------------------------------------------
    {
      constexpr int NP = NNP / 2;  // node pairs (register pairs for the packed FMAs)
      const bool act = el < ne;
      const int e = e0 + el, s = it.s0 + sl;
      const int lb = nsh + el * NI;
      auto lidx = [&](int q) { return q < NS ? (act ? (int)blq[q * PT_PE + el] : 0) : (act ? lb + (q - NS) : 0); };
      float2 U2[NP], y2[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const int q0 = 2 * p, q1 = 2 * p + 1;
        U2[p].x = q0 < NN && act ? bu[4 * lidx(q0) + sl] : 0.f;
        U2[p].y = q1 < NN && act ? bu[4 * lidx(q1) + sl] : 0.f;
        y2[p] = make_float2(0.f, 0.f);
      }
      const float G0 = bgeo[el], G1 = bgeo[PT_PE + el], G2 = bgeo[2 * PT_PE + el];
      // f_d = Ga * (grad u)_x + Gb * (grad u)_z with Ghat = [[G0, G1], [G1, G2]]
      const float Ga = act ? (d ? G1 : G0) : 0.f, Gb = act ? (d ? G2 : G1) : 0.f;
      const int slot = act ? binj[el] : -1;
      if (!ADJ && slot >= 0 && d == 0 && a.rec != nullptr) {
        const int rb = __ldg(a.rslot_ptr + slot), re = __ldg(a.rslot_ptr + slot + 1);
        for (int r = rb; r < re; ++r) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < NN; ++k)
            acc = fmaf(__ldg(a.rslot_phi + (size_t)r * NN + k), (k & 1) ? U2[k >> 1].y : U2[k >> 1].x, acc);
          a.rec[((size_t)s * (a.nt + 1) + a.n) * a.R + __ldg(a.rslot_rec + r)] = acc;
        }
      }
      const float* rowd = rows + d * L.rows_dstride;
      // stored forward-field gradients of this item: written by forward steps (a.gstore set)
      // and read by gradient steps, at [q][sl][el][d] with a stride of 256 floats per node
      const size_t gofs = ((size_t)((it.c - a.ch0) * ngrp + it.s0 / PT_SG) * NN) * kGstoreNodeFloats +
                          (size_t)(sl * PT_PE * 2 + el * 2 + d);
      float* gst = MODE == 0 && a.gstore != nullptr ? a.gstore + gofs : nullptr;
      const float* gld = GRAD ? a.gload + gofs : nullptr;
      // two nodes ahead (read once: streaming loads)
      float h1 = GRAD ? __ldcs(gld) : 0.f;
      float h2 = GRAD && NN > 1 ? __ldcs(gld + kGstoreNodeFloats) : 0.f;
#pragma unroll(ROLL ? 1 : NN)
      for (int q = 0; q < NN; ++q) {
        float hq = 0.f;
        if constexpr (GRAD) {
          hq = h1;
          h1 = h2;
          if (q + 2 < NN) h2 = __ldcs(gld + (size_t)(q + 2) * kGstoreNodeFloats);
        }
        float4 r4[NNP / 4];
#pragma unroll
        for (int j = 0; j < NNP / 4; ++j) r4[j] = *reinterpret_cast<const float4*>(rowd + q * NNP + 4 * j);
        const float wc = c_w[q] * bc2[lidx(q)];
        // (Dhat_d u)_q in four independent packed chains
        float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                         make_float2(0.f, 0.f)};
#pragma unroll
        for (int j = 0; j < NNP / 4; ++j) {
          acc[(2 * j) & 3] = __ffma2_rn(make_float2(r4[j].x, r4[j].y), U2[2 * j], acc[(2 * j) & 3]);
          acc[(2 * j + 1) & 3] = __ffma2_rn(make_float2(r4[j].z, r4[j].w), U2[2 * j + 1], acc[(2 * j + 1) & 3]);
        }
        const float2 s2 = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
        const float gd = s2.x + s2.y;
        const float go = __shfl_xor_sync(0xffffffffu, gd, 1);
        const float gx = d ? go : gd, gz = d ? gd : go;
        const float h = Ga * gx + Gb * gz;  // (Ghat grad u)_d at node q
        const float f = wc * h;
        if (gst != nullptr) __stcs(gst + (size_t)q * kGstoreNodeFloats, h);  // read once, later
        if constexpr (GRAD) {
          // (Ghat grad u_fwd) . grad u_dag at node q: this direction's product, then the pair's sum
          float part = hq * gd;
          part += __shfl_xor_sync(0xffffffffu, part, 1);
          // 2 c_q w_q = 2 (w_q c_q^2) / c_q, with c_q from the reciprocal square root of c_q^2
          // (a few 1e-8 relative; the gradient's bound is 1e-4)
          if (d == 0 && act) atomicAdd(Gacc + lidx(q), 2.f * wc * rsqrtf(bc2[lidx(q)]) * part);
        }
        const float2 ff = make_float2(f, f);
#pragma unroll
        for (int j = 0; j < NNP / 4; ++j) {
          y2[2 * j] = __ffma2_rn(make_float2(r4[j].x, r4[j].y), ff, y2[2 * j]);
          y2[2 * j + 1] = __ffma2_rn(make_float2(r4[j].z, r4[j].w), ff, y2[2 * j + 1]);
        }
      }
      // sources (forward) and adjoint sources at the receivers, in direction 0's partial sum
      if (slot >= 0 && d == 0) {
        if (!ADJ) {
          if (__ldg(a.src_elem + s) == e) {
            const float wv = __ldg(a.wavelet + (size_t)s * a.nt + a.n);
#pragma unroll
            for (int k = 0; k < NN; ++k) {
              const float dv = wv * __ldg(a.src_phi + (size_t)s * NN + k);
              if (k & 1) y2[k >> 1].y -= dv; else y2[k >> 1].x -= dv;
            }
          }
        } else {
          const int rb = __ldg(a.rslot_ptr + slot), re = __ldg(a.rslot_ptr + slot + 1);
          for (int r = rb; r < re; ++r) {
            const float res = __ldg(a.resid + ((size_t)s * (a.nt + 1) + a.n) * a.R + __ldg(a.rslot_rec + r));
#pragma unroll
            for (int k = 0; k < NN; ++k) {
              const float dv = res * __ldg(a.rslot_phi + (size_t)r * NN + k);
              if (k & 1) y2[k >> 1].y += dv; else y2[k >> 1].x += dv;
            }
          }
        }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, y2[p].x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, y2[p].y, 1);
        y2[p] = __fadd2_rn(y2[p], o);
      }
      if (act) {
        if (d == 0) {
#pragma unroll
          for (int q = 0; q < NS; ++q)
            atomicAdd(Y + 4 * (int)blq[q * PT_PE + el] + sl, (q & 1) ? y2[q >> 1].y : y2[q >> 1].x);
        } else {
#pragma unroll
          for (int j = 0; j < NI; ++j) {
            const int q = NS + j;
            Y[4 * (lb + j) + sl] = (q & 1) ? y2[q >> 1].y : y2[q >> 1].x;
          }
        }
      }
    }
    __syncthreads();

    // ---- owned DoFs: increment update; halo DoFs: sums to the global accumulator ----------
    {
      const float4* bu4 = reinterpret_cast<const float4*>(B + L.bu);
      const float4* bv4 = reinterpret_cast<const float4*>(B + L.bv);
      const float* cf1 = reinterpret_cast<const float*>(B + L.bcf);
      const float* cf2 = reinterpret_cast<const float*>(B + L.bcf + L.bcf_stride);
      const float* cf3 = reinterpret_cast<const float*>(B + L.bcf + 2 * L.bcf_stride);
      const int S = a.S;
      for (int l = t; l < own_n; l += PT_THREADS) {
        const float4 yv = Y4[l], uo = bu4[l], vo = bv4[l];
        Y4[l] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float c1 = cf1[l], c2 = cf2[l], c3 = cf3[l];
        float4 vn, un;
        vn.x = c1 * vo.x - c2 * yv.x - c3 * uo.x;
        vn.y = c1 * vo.y - c2 * yv.y - c3 * uo.y;
        vn.z = c1 * vo.z - c2 * yv.z - c3 * uo.z;
        vn.w = c1 * vo.w - c2 * yv.w - c3 * uo.w;
        un.x = uo.x + vn.x;
        un.y = uo.y + vn.y;
        un.z = uo.z + vn.z;
        un.w = uo.w + vn.w;
        const size_t gi = (size_t)(own_lo + l) * S + it.s0;
        *reinterpret_cast<float4*>(a.v + gi) = vn;
        *reinterpret_cast<float4*>(a.u + gi) = un;
        bad |= !(isfinite(un.x) && isfinite(un.y) && isfinite(un.z) && isfinite(un.w));
      }
      for (int h = t; h < hn; h += PT_THREADS) {
        const float4 yv = Y4[own_n + h];
        Y4[own_n + h] = make_float4(0.f, 0.f, 0.f, 0.f);
        atomicAdd(reinterpret_cast<float4*>(a.r + (size_t)(ids[h] - a.N_own) * S + it.s0), yv);
      }
      if constexpr (GRAD) {  // the segment accumulator summed over the shots, [N]
        for (int l = t; l < own_n + hn; l += PT_THREADS) {
          const float g = Gacc[l];
          Gacc[l] = 0.f;
          atomicAdd(a.gseg + (l < own_n ? own_lo + l : ids[l - own_n]), g);
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  if (bad) atomicOr(a.status, 1);
}

}  // namespace fwi
