// Internal declarations shared by the host side of the library and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fwi {

// Element-kernel arguments (one step of the forward, recompute or adjoint recurrence).
// Layouts (S = shots of the batch, stored shot-interleaved so that the lanes of one
// element read one contiguous run of S floats):
//   wavefields u, v (increment), r (shared-DoF accumulator)       [N][S]
//   element-interior DoF j of element e has global id Ns + e*NI + j (no connectivity)
//   conn   [NS][E]  shared-node DoF ids (node-major, coalesced over elements; plain layout)
//   geo    [NG][Es] Ghat = |J| J^-1 J^-T (NG = 3 in 2D, 6 in 3D: xx, xy, yy / xx, xy, xz, yy,
//                   yz, zz)
//   lgeo   [D*D][Elayer]  A = |J| J^-1 (row-major) for the damping-layer elements
//                   e >= E0 (indexed e - E0)
//   pidx   [N] index into the layer arrays or -1
//   P, Pacc          [Nl][D][S], Y / Yacc [Nl][S] (3D)
// Stored forward-field gradients (triangles, persistent kernel): per (chunk without layer
// elements, group of 4 shots) item and node, 4 shots x 32 elements x 2 directions.
constexpr int kGstoreNodeFloats = 256;
inline size_t gstore_level_floats(int nch0, int S, int NN) {
  return (size_t)nch0 * (size_t)(S / 4) * (size_t)NN * kGstoreNodeFloats;
}

struct StepArgs {
  int E, E0, S, Ns, N;
  int Es;              // row stride of the element arrays geo, lconn and inj: E rounded up to a
                       // multiple of 32 (16-byte aligned rows for vector and cp.async loads)
  int log2S;
  int h0, hcnt;        // node kernel range: DoFs [h0, h0 + hcnt), r indexed from h0
  // chunked layout (layout 0)
  int O_max, H_max;    // largest owned-DoF range and halo list of a chunk
  int nch, nch0, ch0, N_own, L_max, PE, SG;  // chunks, owned DoFs, largest chunk table, elements per
                                  // chunk, shots per CTA
  const int* bub;            // [E] first bubble DoF of each element
  const int* chunks;         // [nch][6]: e0, ne, own_lo, own_n, nsh, halo_ptr
  const int* halo;           // halo DoF ids, chunk by chunk
  const unsigned short* lconn;  // [NS][Es] chunk-local index of each shared node
  int tc;              // chunked layout, 2D: element contraction on the tensor cores
  int tc_wait_limit;   // polls of each bounded mbarrier wait of the tensor-core kernel
  int mode;            // 0 forward, 1 adjoint (with gradient when ring != null)
  int n;               // time index (forward: step n -> n+1; adjoint: step m)
  int nt;
  float dt;
  const int* conn;
  const float* geo;
  const float* lgeo;
  const float* c2;     // [N]
  const float* cvel;   // [N] c (gradient weight 2c)
  const float* cf;     // [3][N]: c1, c2, c3 of the increment update
  const int* pidx;     // [N]
  const float* lcf;    // [Nl][LCF] layer coefficients (see layer_coef_layout)
  float* u;
  float* v;
  float* r;
  float* P;
  float* Pacc;
  float* Y;
  float* Yacc;
  float* PaccY;        // 3D forward: lumped gradient of Y (D_{omega,3} term)
  // sources / receivers
  const int* inj;          // [Es] slot id or -1 (padding -1)
  const int* src_elem;     // [S]
  const float* src_phi;    // [S][NN]
  const float* wavelet;    // [S][nt]
  const int* rslot_ptr;    // [nslot+1]
  const int* rslot_rec;    // receiver ids
  const float* rslot_phi;  // [entries][NN]
  int R;
  float* rec;              // forward records [S][nt+1][R] (may be null)
  const float* resid;      // adjoint residual [S][nt+1][R]
  // gradient
  const float* ring_u;     // forward U^m [N][S] (null: no gradient this step)
  float* gseg;             // FP32 segment accumulator: [S][N] per shot, or [N] summed
  int grad_lanes;          // 1: per-shot gradient accumulators, 0: summed over the shots
  float* gstore;           // forward steps: write the forward field's (Ghat grad u) here
  const float* gload;      // gradient steps: read it back (persistent kernel, triangles)
  int* status;             // bit 0: non-finite value seen; bit 1: a bounded wait gave up
};

// Layer coefficients per layer DoF (floats):
//   [0..D)      e1_k  = (1 - dt sigma_k/2) / (1 + dt sigma_k/2)
//   [D..2D)     e2f_k = dt Psi2_kk c^2 / (M (1 + dt sigma_k/2))   forward Q U
//   [2D..3D)    e2a_k = dt / (M (1 + dt sigma_k/2))                adjoint D^T lam
//   [3D..4D)    psi2c2_k = Psi2_kk c^2                              adjoint gather scale
//   3D only: [4D..5D) e3f_k = dt Psi3_kk c^2/(M(1+dt sigma_k/2)); [5D..6D) psi3c2_k;
//            6D: c4 = dt^2 detPsi1 / (1 + a dt/2); 6D+1: c5 = dt^2/(1 + a dt/2);
//            6D+2: dt detPsi1; 6D+3: dt / M
inline int layer_coef_count(int dim) { return dim == 2 ? 4 * 2 : 6 * 3 + 4; }

// Per-(dim,k) entry points, defined in the instantiation units.
struct KernelSet {
  int dim, k, nn, ns, ni;
  int (*upload_constants)(const float* dhat, const float* w);  // [D][NN][NN], [NN]
  void (*launch_step)(const StepArgs& a, cudaStream_t st);        // plain layout
  // chunked layout: chunks without layer elements on st, layer chunks on st_layer (the two
  // launches are independent and may overlap; st_layer may be st)
  int (*launch_chunk)(const StepArgs& a, cudaStream_t st, cudaStream_t st_layer);
  void (*launch_record)(const StepArgs& a, const int* rec_elem, const float* rec_phi,
                        cudaStream_t st);  // d^n for every receiver and shot
};
const KernelSet* kernel_set(int dim, int k);

// Generic (dimension-only) kernels.
void launch_node_update(const StepArgs& a, int dim, cudaStream_t st);
void launch_fold(float* gseg, double* gsum, double* gcomp, int64_t N, double scale,
                 cudaStream_t st);
void launch_finish_gradient(const double* gsum, const double* gcomp, const float* Minv_unused,
                            const double* M, const unsigned char* mask, double* out, int64_t N,
                            int lanes, int per_lane, cudaStream_t st);
void launch_misfit(const float* resid, int64_t n, int lanes, double* acc, cudaStream_t st);
void launch_residual(const float* d, const float* obs, float* res, int64_t n, cudaStream_t st);
void launch_lane_reset(float* p, int64_t rows, int S, uint32_t mask, cudaStream_t st);
int measure_fma_peak(double* tflops, int* sms);

}  // namespace fwi
