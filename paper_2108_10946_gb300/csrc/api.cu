// Host side of the C ABI declared in include/fwi.h: mesh preparation (DoF numbering,
// locality order, geometry, lumped mass, damping layer, CFL estimate), batches of shots,
// and the time loops of the forward solve, the checkpointed adjoint solve and the gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <functional>
#include <memory>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fwi.h"
#include "fwi_internal.h"
#include "kmv_tab.h"

using fwi::StepArgs;

namespace {

thread_local std::string g_err;
thread_local int64_t g_launches = 0;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(x)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? FWI_ENOMEM : FWI_ECUDA,             \
                  std::string(#x) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

template <class T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return 0;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();  // an allocation failure is not sticky: clear it for later checks
    return fail(FWI_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                " bytes: " + cudaGetErrorString(e));
  }
  return 0;
}

template <class T>
int upload(T** p, const std::vector<T>& v) {
  int rc = dalloc(p, v.size());
  if (rc) return rc;
  if (!v.empty()) CUDA_TRY(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& f) {
  unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 4096) nt = 1;
  std::vector<std::thread> th;
  int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    int64_t a = t * chunk, b = std::min<int64_t>(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([&, a, b] { f(a, b); });
  }
  for (auto& x : th) x.join();
}

uint64_t spread_bits(uint64_t x, int dims) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1ull) << (b * dims);
  return r;
}

struct KeyHash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) {
      h ^= (uint64_t)k[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    }
    return h;
  }
};

}  // namespace

struct fwi_mesh {
  fwi_params p;
  int dim = 0, k = 0, nn = 0, ns = 0, ni = 0;
  int device = 0;
  kmvtab::Element el;
  const fwi::KernelSet* ks = nullptr;
  int64_t nverts = 0;
  int E = 0, E0 = 0, N = 0, Ns = 0, Nl = 0;
  int Es = 0;         // element row stride of geo / lconn / inj (E rounded up to 32)
  int layout = 0;     // 0 chunked (shared-memory assembly), 1 plain (global atomics)
  bool use_tc = false;  // chunked 2D: element contractions on the tensor cores
  int P = 32;         // elements per chunk
  int N_own = 0;      // DoFs owned by one chunk: [0, N_own); halo DoFs [N_own, N)
  int nch0 = 0;       // chunks [0, nch0) have no damping-layer element
  int L_max = 0;      // largest local DoF table of a chunk (owned + halo)
  int O_max = 0, H_max = 0;  // largest owned range and halo list of a chunk
  std::vector<int32_t> bub;                       // [E] first bubble DoF of every element
  std::vector<int32_t> ch_e0, ch_own_lo, ch_nsh;  // chunk element ranges, owned ranges
  std::vector<int32_t> ch_halo_ptr, halo_ids;     // per-chunk halo lists (global DoF ids)
  std::vector<uint16_t> lconn;                    // [ns][E] chunk-local index of shared nodes
  std::vector<double> verts;
  std::vector<int32_t> cells;      // user order
  std::vector<int32_t> order;      // new element -> user element
  std::vector<int32_t> conn;       // [E][nn] DoF of every local node (new order)
  std::vector<double> dof_xyz;     // [N][dim]
  std::vector<double> Jinv, detJ;  // [E][dim*dim] (row-major inverse), [E]
  std::vector<double> M, Mb;       // [N]
  std::vector<double> sigma;       // [N][dim]
  std::vector<int32_t> pidx;       // [N]
  std::vector<double> c;           // [N]
  double dt = 0;
  bool have_velocity = false;
  // device
  int* d_conn = nullptr;     // [ns][E]
  float* d_geo = nullptr;    // [NG][E]
  float* d_lgeo = nullptr;   // [dim*dim][E-E0]
  int* d_pidx = nullptr;
  float* d_c2 = nullptr;
  float* d_c = nullptr;
  float* d_cf = nullptr;     // [3][N]
  float* d_lcf = nullptr;    // [Nl][count]
  double* d_M = nullptr;
  unsigned char* d_mask = nullptr;
  int* d_bub = nullptr;
  int* d_chunks = nullptr;   // [nch][6]: e0, ne, own_lo, own_n, nsh, halo_ptr
  int* d_halo = nullptr;     // halo DoF ids, chunk by chunk
  unsigned short* d_lconn = nullptr;
  int nch() const { return (int)ch_e0.size() - 1; }
};

struct fwi_batch {
  fwi_mesh* m = nullptr;
  int S = 0, log2S = 0, R = 0, nt = 0, K = 0, C = 0;
  int gstride = 1;  // gradient subsampling stride r (Section 3.6); the ring holds K / r fields
  std::vector<int32_t> src_elem;   // [S] new element index
  std::vector<float> src_phi;      // [S][nn]
  std::vector<int32_t> rec_elem;   // [R]
  std::vector<float> rec_phi;      // [R][nn]
  // device
  int* d_inj = nullptr;
  int* d_src_elem = nullptr;
  float* d_src_phi = nullptr;
  int* d_rslot_ptr = nullptr;
  int* d_rslot_rec = nullptr;
  float* d_rslot_phi = nullptr;
  int* d_rec_elem = nullptr;
  float* d_rec_phi = nullptr;
  float *u = nullptr, *v = nullptr, *r = nullptr;          // forward state [N][S]
  float *P = nullptr, *Pacc = nullptr, *PaccY = nullptr;   // [Nl][dim][S]
  float *Y = nullptr, *Yacc = nullptr;                     // [Nl][S]
  float *ua = nullptr, *va = nullptr, *Pa = nullptr, *Ya = nullptr;  // adjoint state
  float* ckpt = nullptr;   // C x state
  float* ring = nullptr;   // K x [N][S]
  float* gseg = nullptr;                                   // [S][N] FP32 segment sums
  double *gsum = nullptr, *gcomp = nullptr, *misfit = nullptr;  // [S][N], [S][N], [S]
  int* status = nullptr;
  cudaStream_t st2 = nullptr;  // second stream of the chunked step (layer chunks)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // staging for host pointers
  float* wav_dev = nullptr;  // [S][nt] the forward's wavelet, re-injected by the recompute
  float* rec_dev = nullptr;  // [S][nt+1][R] the forward's records
  float* res_dev = nullptr;  // [S][nt+1][R] residual formed by fwi_adjoint_misfit
  float* stage_in = nullptr;
  float* stage_out = nullptr;
  double* stage_grad = nullptr;
  bool forward_done = false;
  int launch_error = 0;  // first kernel configuration error of a call (cudaError_t)
  int tc_wait_limit = 1 << 22;  // polls of each bounded wait of the tensor-core kernel
  int grad_lanes = 0;           // 1: the next adjoint keeps each shot's gradient apart
  int acc_lanes = -1;           // what the accumulators hold: -1 nothing, 0 summed, 1 per shot
  int gstore_on = 0;            // store the forward field's gradients during the recompute
  float* gring = nullptr;       // [levels][gstore_level_floats] (allocated at first use)
  size_t gring_level = 0;       // floats per level
  // optional per-kernel timing with CUDA events (fwi_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_mode;
  size_t ev_used = 0;
  double prof_ms[2][2] = {{0, 0}, {0, 0}};  // [forward/adjoint][element/node kernel]
  int64_t prof_steps[2] = {0, 0};
  size_t state_floats() const {
    const fwi_mesh* mm = m;
    return (size_t)S * (2 * (size_t)mm->N + (size_t)mm->Nl * (mm->dim + (mm->dim == 3 ? 1 : 0)));
  }
};

namespace {

int check_device(const fwi_mesh* m) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != m->device)
    return fail(FWI_EINVAL, "the mesh's CUDA device is not the current device");
  return 0;
}

// Upload the reference tables of (dim, k) to the constant memory of the current device.
int ensure_constants(fwi_mesh* m) {
  static std::vector<std::array<int, 3>> done;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& d : done)
    if (d[0] == m->device && d[1] == m->dim && d[2] == m->k) return 0;
  std::vector<float> dh, w;
  kmvtab::fp32_tables(m->el, dh, w);
  int e = m->ks->upload_constants(dh.data(), w.data());
  if (e != 0) return fail(FWI_ECUDA, std::string("constant upload: ") + cudaGetErrorString((cudaError_t)e));
  done.push_back({m->device, m->dim, m->k});
  return 0;
}

double sigma_at(const fwi_params& p, int dim, const double* x, int d) {
  double s = 0;
  if (p.layer_width <= 0 || p.sigma_max <= 0) return 0;
  if (p.layer_faces & (1 << (2 * d))) {
    double dist = p.box_lo[d] - x[d];
    if (dist > 0) s += (dist / p.layer_width) * (dist / p.layer_width);
  }
  if (p.layer_faces & (1 << (2 * d + 1))) {
    double dist = x[d] - p.box_hi[d];
    if (dist > 0) s += (dist / p.layer_width) * (dist / p.layer_width);
  }
  (void)dim;
  return p.sigma_max * s;
}

// inverse of the column-edge Jacobian J (J[r][c] = x_{c+1,r} - x_{0,r}); returns det J
double jac_inverse(int dim, const double* X /*[dim+1][dim]*/, double* inv /*[dim][dim]*/) {
  double J[9];
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) J[r * dim + c] = X[(c + 1) * dim + r] - X[r];
  if (dim == 2) {
    double det = J[0] * J[3] - J[1] * J[2];
    inv[0] = J[3] / det;
    inv[1] = -J[1] / det;
    inv[2] = -J[2] / det;
    inv[3] = J[0] / det;
    return det;
  }
  double a = J[0], b = J[1], c = J[2], d = J[3], e = J[4], f = J[5], g = J[6], h = J[7], i = J[8];
  double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
  double det = a * A + b * B + c * C;
  inv[0] = A / det;
  inv[1] = -(b * i - c * h) / det;
  inv[2] = (b * f - c * e) / det;
  inv[3] = B / det;
  inv[4] = (a * i - c * g) / det;
  inv[5] = -(a * f - c * d) / det;
  inv[6] = C / det;
  inv[7] = -(a * h - b * g) / det;
  inv[8] = (a * e - b * d) / det;
  return det;
}

// Reference coordinates of x in element (user id) ue; returns min barycentric.
double locate_in(const fwi_mesh* m, int ue, const double* x, double* xh) {
  int d = m->dim;
  double X[12], inv[9];
  for (int v = 0; v <= d; ++v)
    for (int c = 0; c < d; ++c) X[v * d + c] = m->verts[(size_t)m->cells[(size_t)ue * (d + 1) + v] * d + c];
  jac_inverse(d, X, inv);
  double lam0 = 1, mn = 1e300;
  for (int r = 0; r < d; ++r) {
    double s = 0;
    for (int c = 0; c < d; ++c) s += inv[r * d + c] * (x[c] - X[c]);
    xh[r] = s;
    lam0 -= s;
    mn = std::min(mn, s);
  }
  return std::min(mn, lam0);
}

// Point location: the lowest user element id whose barycentrics are all >= -1e-12.
int locate(const fwi_mesh* m, const double* pts, int npts, std::vector<int>& user_elem,
           std::vector<double>& xhat) {
  int d = m->dim;
  int E = m->E;
  // uniform grid of element bounding boxes
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < m->nverts; ++v)
    for (int c = 0; c < d; ++c) {
      lo[c] = std::min(lo[c], m->verts[v * d + c]);
      hi[c] = std::max(hi[c], m->verts[v * d + c]);
    }
  int nc = std::max(1, (int)std::pow((double)E / 4.0, 1.0 / d));
  nc = std::min(nc, d == 2 ? 2048 : 256);
  int ncell[3] = {nc, nc, d == 3 ? nc : 1};
  auto cell_of = [&](const double* x, int c) {
    double f = (x[c] - lo[c]) / (hi[c] - lo[c] + 1e-300) * ncell[c];
    return std::max(0, std::min(ncell[c] - 1, (int)std::floor(f)));
  };
  std::vector<std::vector<int>> grid((size_t)ncell[0] * ncell[1] * ncell[2]);
  for (int ue = 0; ue < E; ++ue) {
    int cmin[3] = {0, 0, 0}, cmax[3] = {0, 0, 0};
    double bl[3] = {1e300, 1e300, 1e300}, bh[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v <= d; ++v) {
      const double* x = &m->verts[(size_t)m->cells[(size_t)ue * (d + 1) + v] * d];
      for (int c = 0; c < d; ++c) {
        bl[c] = std::min(bl[c], x[c]);
        bh[c] = std::max(bh[c], x[c]);
      }
    }
    for (int c = 0; c < d; ++c) {
      cmin[c] = cell_of(bl, c);
      cmax[c] = cell_of(bh, c);
    }
    for (int i = cmin[0]; i <= cmax[0]; ++i)
      for (int j = cmin[1]; j <= cmax[1]; ++j)
        for (int k = cmin[2]; k <= cmax[2]; ++k)
          grid[((size_t)i * ncell[1] + j) * ncell[2] + k].push_back(ue);
  }
  user_elem.assign(npts, -1);
  xhat.assign((size_t)npts * d, 0);
  for (int p = 0; p < npts; ++p) {
    const double* x = pts + (size_t)p * d;
    int ci[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) ci[c] = cell_of(x, c);
    int best = -1;
    double xh[3];
    for (int ue : grid[((size_t)ci[0] * ncell[1] + ci[1]) * ncell[2] + ci[2]]) {
      if (best >= 0 && ue > best) continue;
      if (locate_in(m, ue, x, xh) >= -1e-12) best = ue;
    }
    if (best < 0) {
      char buf[160];
      snprintf(buf, sizeof buf, "point %d (%g, %g%s) lies outside the mesh", p, x[0], x[1],
               d == 3 ? ", ..." : "");
      return fail(FWI_EINVAL, buf);
    }
    locate_in(m, best, x, xh);
    user_elem[p] = best;
    for (int c = 0; c < d; ++c) xhat[(size_t)p * d + c] = xh[c];
  }
  return 0;
}

// Injection slots: every element holding a source of the batch or a receiver gets a slot;
// a slot lists its receivers (id and basis values). sptr is padded to S + R + 1 entries so
// that sources can be moved later without reallocating.
void build_injection(const fwi_mesh* m, const fwi_batch* b, std::vector<int>& inj,
                     std::vector<int>& sptr, std::vector<int>& srec, std::vector<float>& sphi) {
  const int n = m->nn, S = b->S, nrec = b->R;
  inj.assign((size_t)m->Es + 32, -1);  // padded to the element row stride
  std::vector<int> slot_elems;
  auto slot_of = [&](int e) {
    if (inj[e] < 0) {
      inj[e] = (int)slot_elems.size();
      slot_elems.push_back(e);
    }
    return inj[e];
  };
  for (int s = 0; s < S; ++s) slot_of(b->src_elem[s]);
  for (int r = 0; r < nrec; ++r) slot_of(b->rec_elem[r]);
  const int ns = (int)slot_elems.size();
  sptr.assign(S + nrec + 1, 0);
  srec.clear();
  sphi.clear();
  std::vector<std::vector<int>> lists(ns);
  for (int r = 0; r < nrec; ++r) lists[inj[b->rec_elem[r]]].push_back(r);
  for (int t = 0; t < ns; ++t) {
    sptr[t + 1] = sptr[t] + (int)lists[t].size();
    for (int r : lists[t]) {
      srec.push_back(r);
      for (int k = 0; k < n; ++k) sphi.push_back(b->rec_phi[(size_t)r * n + k]);
    }
  }
  for (int t = ns + 1; t < (int)sptr.size(); ++t) sptr[t] = sptr[ns];
  if (srec.empty()) {
    srec.push_back(0);
    sphi.assign(n, 0.f);
  }
}

// Gershgorin bound of rho(M^-1 K) on the assembled stiffness (Eq. spectral).
double gershgorin(const fwi_mesh* m) {
  const int d = m->dim, n = m->nn, E = m->E;
  const auto& el = m->el;
  // element stiffness row a: K_e[a][b] = sum_q w_q |J| c_q^2 (Jinv^T Dhat[.,q,a]) . (Jinv^T Dhat[.,q,b])
  auto row = [&](int e, int a, double* out) {
    const double* Ji = &m->Jinv[(size_t)e * d * d];
    const double det = m->detJ[e];
    for (int b = 0; b < n; ++b) out[b] = 0;
    for (int q = 0; q < n; ++q) {
      const double c = m->c[m->conn[(size_t)e * n + q]];
      const double wq = el.w[q] * std::fabs(det) * c * c;
      double ga[3] = {0, 0, 0};
      for (int r = 0; r < d; ++r)
        for (int s = 0; s < d; ++s) ga[r] += Ji[s * d + r] * el.dhat[(s * n + q) * n + a];
      for (int b = 0; b < n; ++b) {
        double dot = 0;
        for (int r = 0; r < d; ++r) {
          double gb = 0;
          for (int s = 0; s < d; ++s) gb += Ji[s * d + r] * el.dhat[(s * n + q) * n + b];
          dot += ga[r] * gb;
        }
        out[b] += wq * dot;
      }
    }
  };
  // incidence (element, local node) of every shared DoF, CSR over all DoFs
  const int N = m->N;
  std::vector<int64_t> ptr(N + 1, 0);
  for (int e = 0; e < E; ++e)
    for (int a = 0; a < m->ns; ++a) ptr[m->conn[(size_t)e * n + a] + 1]++;
  for (int i = 0; i < N; ++i) ptr[i + 1] += ptr[i];
  std::vector<int64_t> fillp(ptr.begin(), ptr.end() - 1);
  std::vector<int32_t> inc((size_t)ptr[N] * 2);
  for (int e = 0; e < E; ++e)
    for (int a = 0; a < m->ns; ++a) {
      int i = m->conn[(size_t)e * n + a];
      int64_t pos = fillp[i]++;
      inc[pos * 2] = e;
      inc[pos * 2 + 1] = a;
    }
  std::atomic<double> best{0.0};
  auto upd = [&](double v) {
    double cur = best.load();
    while (v > cur && !best.compare_exchange_weak(cur, v)) {
    }
  };
  parallel_for(N, [&](int64_t i0, int64_t i1) {
    std::vector<double> rw(n);
    std::vector<std::pair<int, double>> acc;
    double loc = 0;
    for (int64_t i = i0; i < i1; ++i) {
      if (ptr[i] == ptr[i + 1]) continue;  // bubble DoF: handled element by element below
      acc.clear();
      for (int64_t t = ptr[i]; t < ptr[i + 1]; ++t) {
        int e = inc[t * 2], a = inc[t * 2 + 1];
        row(e, a, rw.data());
        for (int b = 0; b < n; ++b) acc.push_back({m->conn[(size_t)e * n + b], rw[b]});
      }
      std::sort(acc.begin(), acc.end(),
                [](const std::pair<int, double>& x, const std::pair<int, double>& y) { return x.first < y.first; });
      double s = 0;
      for (size_t t = 0; t < acc.size();) {
        double v = 0;
        size_t u = t;
        while (u < acc.size() && acc[u].first == acc[t].first) v += acc[u++].second;
        s += std::fabs(v);
        t = u;
      }
      loc = std::max(loc, s / m->M[i]);
    }
    upd(loc);
  });
  parallel_for(E, [&](int64_t e0, int64_t e1) {
    std::vector<double> rw(n);
    double loc = 0;
    for (int64_t e = e0; e < e1; ++e)
      for (int a = m->ns; a < n; ++a) {
        row((int)e, a, rw.data());
        double s = 0;
        for (int b = 0; b < n; ++b) s += std::fabs(rw[b]);
        loc = std::max(loc, s / m->M[m->conn[(size_t)e * n + a]]);
      }
    upd(loc);
  });
  return best.load();
}

}  // namespace

extern "C" {

int fwi_last_error(char* buf, int len) {
  if (!buf || len <= 0) return FWI_EINVAL;
  snprintf(buf, (size_t)len, "%s", g_err.c_str());
  return 0;
}

int fwi_fp32_peak(double* tflops, int* sm_count) {
  int e = fwi::measure_fma_peak(tflops, sm_count);
  if (e) return fail(FWI_ECUDA, std::string("FP32 peak probe: ") + cudaGetErrorString((cudaError_t)e));
  return 0;
}

int64_t fwi_launch_count(void) {
  int64_t v = g_launches;
  g_launches = 0;
  return v;
}

}  // extern "C"

namespace {
int mesh_create(const double* verts, int64_t nverts, const int32_t* cells, int64_t ncells,
                const fwi_params* params, bool host_only, fwi_mesh** out) {
  if (!verts || !cells || !params || !out || nverts <= 0 || ncells <= 0)
    return fail(FWI_EINVAL, "fwi_mesh_upload: null or empty input");
  *out = nullptr;
  const int d = params->dim;
  if (d != 2 && d != 3) return fail(FWI_EINVAL, "dim must be 2 or 3");
  if (ncells > (int64_t)INT32_MAX / 64) return fail(FWI_EINVAL, "too many cells");
  const fwi::KernelSet* ks = fwi::kernel_set(d, params->k);
  if (!ks) return fail(FWI_EINVAL, "unsupported (dim, k): triangles k = 2..5, tetrahedra k = 2, 3");
  std::unique_ptr<fwi_mesh> m(new fwi_mesh());
  m->p = *params;
  if (m->p.ckpt_stride <= 0) m->p.ckpt_stride = 50;
  if (m->p.grad_stride <= 1) m->p.grad_stride = 1;
  if (m->p.ckpt_stride % m->p.grad_stride != 0)
    return fail(FWI_EINVAL, "ckpt_stride must be a multiple of grad_stride");
  if (m->p.cfl_factor <= 0) m->p.cfl_factor = 0.9;
  m->dim = d;
  m->k = params->k;
  m->ks = ks;
  m->layout = params->layout == 1 ? 1 : 0;
  m->P = d == 2 ? 32 : 16;
  if (params->tensor_cores > 0 && (d != 2 || m->layout != 0))
    return fail(FWI_EINVAL, "tensor_cores = 1 needs triangles and the chunked layout");
  m->use_tc = d == 2 && m->layout == 0 && params->tensor_cores > 0;
  if (!host_only) CUDA_TRY(cudaGetDevice(&m->device));
  std::string err;
  if (!kmvtab::build(d, params->k, m->el, err)) return fail(FWI_EINVAL, "KMV tabulation: " + err);
  if (m->el.n != ks->nn) return fail(FWI_EINVAL, "KMV tabulation node count mismatch");
  const int n = m->nn = m->el.n;
  m->ns = ks->ns;
  m->ni = ks->ni;
  for (int q = 0; q < m->ns; ++q)
    if (m->el.entity[q] == kmvtab::INTERIOR) return fail(FWI_EINVAL, "node order mismatch");
  m->nverts = nverts;
  m->verts.assign(verts, verts + nverts * d);
  m->cells.assign(cells, cells + ncells * (d + 1));
  const int E = m->E = (int)ncells;
  m->Es = (int)((ncells + 31) / 32 * 32);
  for (int64_t i = 0; i < ncells * (d + 1); ++i)
    if (cells[i] < 0 || cells[i] >= nverts) return fail(FWI_EINVAL, "cell vertex id out of range");

  // geometry (user order) and the layer flag of every element
  std::vector<double> uJinv((size_t)E * d * d), udet(E);
  std::vector<char> ulayer(E, 0);
  std::vector<uint64_t> code(E);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < nverts; ++v)
    for (int c = 0; c < d; ++c) {
      lo[c] = std::min(lo[c], verts[v * d + c]);
      hi[c] = std::max(hi[c], verts[v * d + c]);
    }
  int bad = -1;
  for (int e = 0; e < E; ++e) {
    double X[12];
    double cen[3] = {0, 0, 0};
    for (int v = 0; v <= d; ++v)
      for (int c = 0; c < d; ++c) {
        X[v * d + c] = verts[(size_t)cells[(size_t)e * (d + 1) + v] * d + c];
        cen[c] += X[v * d + c] / (d + 1);
      }
    udet[e] = jac_inverse(d, X, &uJinv[(size_t)e * d * d]);
    if (!(udet[e] > 0) && bad < 0) bad = e;
    for (int v = 0; v <= d; ++v)
      for (int c = 0; c < d; ++c)
        if (sigma_at(m->p, d, &X[v * d], c) > 0) ulayer[e] = 1;
    uint64_t cc = 0;
    for (int c = 0; c < d; ++c) {
      double f = (cen[c] - lo[c]) / (hi[c] - lo[c] + 1e-300);
      uint64_t qv = (uint64_t)std::min(2097151.0, std::max(0.0, f * 2097151.0));
      cc |= spread_bits(qv, d) << c;
    }
    code[e] = cc;
  }
  if (bad >= 0) return fail(FWI_EINVAL, "element " + std::to_string(bad) + " has det J <= 0");
  m->order.resize(E);
  for (int e = 0; e < E; ++e) m->order[e] = e;
  std::stable_sort(m->order.begin(), m->order.end(), [&](int a, int b) {
    if (ulayer[a] != ulayer[b]) return ulayer[a] < ulayer[b];
    return code[a] < code[b];
  });
  m->E0 = 0;
  while (m->E0 < E && !ulayer[m->order[m->E0]]) ++m->E0;
  m->Jinv.resize((size_t)E * d * d);
  m->detJ.resize(E);
  for (int e = 0; e < E; ++e) {
    int ue = m->order[e];
    std::copy(&uJinv[(size_t)ue * d * d], &uJinv[(size_t)ue * d * d] + d * d, &m->Jinv[(size_t)e * d * d]);
    m->detJ[e] = udet[ue];
  }

  // DoF numbering: shared nodes by first touch (entity keys), interior nodes per element
  const auto& el = m->el;
  int nedge_nodes = 0, nface_nodes = 0;
  for (int q = 0; q < n; ++q) {
    nedge_nodes += el.entity[q] == kmvtab::EDGE;
    nface_nodes += el.entity[q] == kmvtab::FACE;
  }
  nedge_nodes /= d == 2 ? 3 : 6;
  if (d == 3) nface_nodes /= 4;
  std::unordered_map<std::array<int64_t, 4>, int32_t, KeyHash> keys;
  keys.reserve((size_t)E * m->ns / 2);
  m->conn.assign((size_t)E * n, -1);
  int32_t next = 0;
  for (int e = 0; e < E; ++e) {
    const int32_t* cv = &cells[(size_t)m->order[e] * (d + 1)];
    for (int q = 0; q < m->ns; ++q) {
      std::array<int64_t, 4> key = {0, 0, 0, 0};
      const int* ev = &el.ent_verts[q * 3];
      if (el.entity[q] == kmvtab::VERTEX) {
        key = {0, cv[ev[0]], 0, 0};
      } else if (el.entity[q] == kmvtab::EDGE) {
        int64_t ga = cv[ev[0]], gb = cv[ev[1]];
        int rank = el.ent_rank[q];
        if (ga > gb) rank = nedge_nodes - 1 - rank;
        key = {1, std::min(ga, gb), std::max(ga, gb), rank};
      } else {
        int64_t g[3] = {cv[ev[0]], cv[ev[1]], cv[ev[2]]};
        int64_t dom = nface_nodes == 1 ? 0 : g[el.ent_rank[q]];
        std::sort(g, g + 3);
        key = {2 + 4 * dom, g[0], g[1], g[2]};
      }
      auto it = keys.find(key);
      if (it == keys.end()) it = keys.emplace(key, next++).first;
      m->conn[(size_t)e * n + q] = it->second;
    }
  }
  const int nprov = next;
  if ((int64_t)nprov + (int64_t)E * m->ni > INT32_MAX) return fail(FWI_EINVAL, "too many DoFs");
  m->bub.assign(E, 0);
  if (m->layout == 1) {
    // plain layout: shared DoFs by first touch, then the bubble DoFs element by element
    m->Ns = nprov;
    m->N = m->Ns + E * m->ni;
    for (int e = 0; e < E; ++e) m->bub[e] = m->Ns + e * m->ni;
  } else {
    // chunked layout: chunks of P consecutive elements (never straddling E0); a shared DoF
    // touched by one chunk only is owned by it; each chunk's owned shared DoFs and its
    // elements' bubble DoFs form one contiguous range; DoFs shared by several chunks
    // (the halo) are numbered last
    const int P = m->P;
    m->ch_e0.clear();
    for (int e = 0; e < m->E0; e += P) m->ch_e0.push_back(e);
    m->nch0 = (int)m->ch_e0.size();
    for (int e = m->E0; e < E; e += P) m->ch_e0.push_back(e);
    m->ch_e0.push_back(E);
    const int nch = (int)m->ch_e0.size() - 1;
    std::vector<int> first(nprov, -1);
    std::vector<char> halo(nprov, 0);
    for (int c = 0; c < nch; ++c)
      for (int e = m->ch_e0[c]; e < m->ch_e0[c + 1]; ++e)
        for (int q = 0; q < m->ns; ++q) {
          int pid = m->conn[(size_t)e * n + q];
          if (first[pid] < 0) first[pid] = c;
          else if (first[pid] != c) halo[pid] = 1;
        }
    std::vector<int32_t> fin(nprov, -1);
    m->ch_own_lo.assign(nch + 1, 0);
    m->ch_nsh.assign(nch, 0);
    int32_t cur = 0;
    for (int c = 0; c < nch; ++c) {
      m->ch_own_lo[c] = cur;
      for (int e = m->ch_e0[c]; e < m->ch_e0[c + 1]; ++e)
        for (int q = 0; q < m->ns; ++q) {
          int pid = m->conn[(size_t)e * n + q];
          if (!halo[pid] && fin[pid] < 0) fin[pid] = cur++;
        }
      m->ch_nsh[c] = cur - m->ch_own_lo[c];
      for (int e = m->ch_e0[c]; e < m->ch_e0[c + 1]; ++e) {
        m->bub[e] = cur;
        cur += m->ni;
      }
    }
    m->ch_own_lo[nch] = cur;
    m->N_own = cur;
    // halo DoFs: those no damping-layer element touches first, then the layer DoFs, so that
    // the node kernel's warps see one kind of DoF
    std::vector<char> in_layer(nprov, 0);
    for (int e = m->E0; e < E; ++e)
      for (int q = 0; q < m->ns; ++q) in_layer[m->conn[(size_t)e * n + q]] = 1;
    for (int pass = 0; pass < 2; ++pass)
      for (int e = 0; e < E; ++e)
        for (int q = 0; q < m->ns; ++q) {
          int pid = m->conn[(size_t)e * n + q];
          if (fin[pid] < 0 && in_layer[pid] == pass) fin[pid] = cur++;
        }
    m->N = cur;
    m->Ns = nprov;  // number of shared DoFs (owned + halo)
    for (int e = 0; e < E; ++e)
      for (int q = 0; q < m->ns; ++q) m->conn[(size_t)e * n + q] = fin[m->conn[(size_t)e * n + q]];
    // per-chunk halo lists and local connectivity
    m->ch_halo_ptr.assign(nch + 1, 0);
    m->halo_ids.clear();
    m->lconn.assign((size_t)m->ns * m->Es + 32, 0);
    m->L_max = 0;
    std::unordered_map<int32_t, int> hmap;
    for (int c = 0; c < nch; ++c) {
      hmap.clear();
      const int own_lo = m->ch_own_lo[c], own_n = m->ch_own_lo[c + 1] - own_lo;
      for (int e = m->ch_e0[c]; e < m->ch_e0[c + 1]; ++e)
        for (int q = 0; q < m->ns; ++q) {
          int dof = m->conn[(size_t)e * n + q];
          int loc;
          if (dof < m->N_own) {
            loc = dof - own_lo;
          } else {
            auto it = hmap.find(dof);
            if (it == hmap.end()) {
              it = hmap.emplace(dof, (int)hmap.size()).first;
              m->halo_ids.push_back(dof);
            }
            loc = own_n + it->second;
          }
          if (loc < 0 || loc > 65535) return fail(FWI_EINVAL, "chunk too large for 16-bit local indices");
          m->lconn[(size_t)q * m->Es + e] = (uint16_t)loc;
        }
      m->ch_halo_ptr[c + 1] = (int)m->halo_ids.size();
      m->L_max = std::max(m->L_max, own_n + (int)hmap.size());
      m->O_max = std::max(m->O_max, own_n);
      m->H_max = std::max(m->H_max, (int)hmap.size());
    }
  }
  for (int e = 0; e < E; ++e)
    for (int j = 0; j < m->ni; ++j) m->conn[(size_t)e * n + m->ns + j] = m->bub[e] + j;
  const int N = m->N;

  // DoF coordinates, lumped mass, damping profile
  m->dof_xyz.assign((size_t)N * d, 0);
  std::vector<char> seen(N, 0);
  m->M.assign(N, 0);
  for (int e = 0; e < E; ++e) {
    const int32_t* cv = &cells[(size_t)m->order[e] * (d + 1)];
    for (int q = 0; q < n; ++q) {
      int i = m->conn[(size_t)e * n + q];
      m->M[i] += el.w[q] * m->detJ[e];
      if (!seen[i]) {
        seen[i] = 1;
        for (int c = 0; c < d; ++c) {
          double x = 0;
          for (int v = 0; v <= d; ++v) x += el.bary[q * (d + 1) + v] * verts[(size_t)cv[v] * d + c];
          m->dof_xyz[(size_t)i * d + c] = x;
        }
      }
    }
  }
  m->sigma.assign((size_t)N * d, 0);
  // Layer auxiliaries (P, and omega in 3D) are stored for every DoF of a layer element:
  // omega is a field on the whole mesh (omega_t = u), and the lumped gradient of omega at a
  // layer node takes its values at the element's other nodes, damped or not. Outside the
  // layer elements no term reads P or omega.
  m->pidx.assign(N, -1);
  m->Nl = 0;
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < d; ++c)
      m->sigma[(size_t)i * d + c] = sigma_at(m->p, d, &m->dof_xyz[(size_t)i * d], c);
  for (int e = m->E0; e < E; ++e)
    for (int q = 0; q < n; ++q) {
      const int i = m->conn[(size_t)e * n + q];
      if (m->pidx[i] < 0) m->pidx[i] = m->Nl++;
    }
  // lumped boundary mass: facets owned by one element
  m->Mb.assign(N, 0);
  if (m->p.absorbing) {
    std::unordered_map<std::array<int64_t, 4>, int, KeyHash> fcount;
    fcount.reserve((size_t)E * (d + 1));
    for (int e = 0; e < E; ++e) {
      const int32_t* cv = &cells[(size_t)m->order[e] * (d + 1)];
      for (int i = 0; i <= d; ++i) {
        std::array<int64_t, 4> key = {-1, -1, -1, -1};
        int c = 0;
        for (int v = 0; v <= d; ++v)
          if (v != i) key[c++] = cv[v];
        std::sort(key.begin(), key.begin() + d);
        fcount[key]++;
      }
    }
    const double ref = d == 2 ? 1.0 : 0.5;
    for (int e = 0; e < E; ++e) {
      const int32_t* cv = &cells[(size_t)m->order[e] * (d + 1)];
      for (int i = 0; i <= d; ++i) {
        std::array<int64_t, 4> key = {-1, -1, -1, -1};
        int c = 0;
        int fv[3];
        for (int v = 0; v <= d; ++v)
          if (v != i) {
            fv[c] = cv[v];
            key[c++] = cv[v];
          }
        std::sort(key.begin(), key.begin() + d);
        if (fcount[key] != 1) continue;
        double meas;
        const double* a = &verts[(size_t)fv[0] * d];
        const double* b = &verts[(size_t)fv[1] * d];
        if (d == 2) {
          meas = std::hypot(b[0] - a[0], b[1] - a[1]);
        } else {
          const double* cc = &verts[(size_t)fv[2] * d];
          double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
          double w[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
          double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
          meas = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        }
        const auto& fn = el.facet_nodes[i];
        for (size_t t = 0; t < fn.size(); ++t)
          m->Mb[m->conn[(size_t)e * n + fn[t]]] += el.facet_weights[i][t] * meas / ref;
      }
    }
  }

  if (host_only) {
    *out = m.release();
    return 0;
  }
  // device geometry
  const int NG = d == 2 ? 3 : 6;
  const size_t Es = (size_t)m->Es;
  std::vector<float> geo((size_t)NG * Es + 32, 0.f), lgeo((size_t)d * d * (E - m->E0));
  for (int e = 0; e < E; ++e) {
    const double* Ji = &m->Jinv[(size_t)e * d * d];
    const double det = m->detJ[e];
    double Gm[9];
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        double s = 0;
        for (int t = 0; t < d; ++t) s += Ji[r * d + t] * Ji[c * d + t];
        Gm[r * d + c] = det * s;  // |J| J^-1 J^-T
      }
    if (d == 2) {
      geo[0 * Es + e] = (float)Gm[0];
      geo[1 * Es + e] = (float)Gm[1];
      geo[2 * Es + e] = (float)Gm[3];
    } else {
      const int idx[6] = {0, 1, 2, 4, 5, 8};
      for (int g = 0; g < 6; ++g) geo[(size_t)g * Es + e] = (float)Gm[idx[g]];
    }
    if (e >= m->E0)
      for (int c = 0; c < d * d; ++c) lgeo[(size_t)c * (E - m->E0) + (e - m->E0)] = (float)(det * Ji[c]);
  }
  std::vector<int> conn_dev((size_t)m->ns * E);
  for (int e = 0; e < E; ++e)
    for (int q = 0; q < m->ns; ++q) conn_dev[(size_t)q * E + e] = m->conn[(size_t)e * n + q];
  std::vector<int> chunks;
  if (m->layout == 0) {
    for (int c = 0; c < m->nch(); ++c) {
      chunks.push_back(m->ch_e0[c]);
      chunks.push_back(m->ch_e0[c + 1] - m->ch_e0[c]);
      chunks.push_back(m->ch_own_lo[c]);
      chunks.push_back(m->ch_own_lo[c + 1] - m->ch_own_lo[c]);
      chunks.push_back(m->ch_nsh[c]);
      chunks.push_back(m->ch_halo_ptr[c]);
    }
    chunks.push_back(0);
    chunks.push_back(0);
    chunks.push_back(0);
    chunks.push_back(0);
    chunks.push_back(0);
    chunks.push_back(m->ch_halo_ptr.empty() ? 0 : m->ch_halo_ptr.back());
  }
  std::vector<int> halo_dev(m->halo_ids.begin(), m->halo_ids.end());
  if (halo_dev.empty()) halo_dev.push_back(0);
  int rc;
  if (m->layout == 0 && ((rc = upload(&m->d_chunks, chunks)) || (rc = upload(&m->d_halo, halo_dev)) ||

                         (rc = upload(&m->d_lconn, m->lconn)))) {
    fwi_mesh_free(m.release());
    return rc;
  }
  if ((rc = upload(&m->d_bub, m->bub))) {
    fwi_mesh_free(m.release());
    return rc;
  }
  if ((rc = upload(&m->d_conn, conn_dev)) || (rc = upload(&m->d_geo, geo)) ||
      (rc = upload(&m->d_lgeo, lgeo)) || (rc = upload(&m->d_pidx, m->pidx)) ||
      (rc = upload(&m->d_M, m->M))) {
    fwi_mesh_free(m.release());
    return rc;
  }
  if ((rc = ensure_constants(m.get()))) {
    fwi_mesh_free(m.release());
    return rc;
  }
  *out = m.release();
  return 0;
}
}  // namespace

extern "C" {

int fwi_mesh_upload(const double* verts, int64_t nverts, const int32_t* cells, int64_t ncells,
                    const fwi_params* params, fwi_mesh** out) {
  return mesh_create(verts, nverts, cells, ncells, params, false, out);
}

int fwi_mesh_prepare_host(const double* verts, int64_t nverts, const int32_t* cells,
                          int64_t ncells, const fwi_params* params, fwi_mesh** out) {
  return mesh_create(verts, nverts, cells, ncells, params, true, out);
}

int fwi_mesh_host_arrays(const fwi_mesh* m, int32_t* conn, double* mass, double* bmass,
                         double* sigma) {
  if (!m) return fail(FWI_EINVAL, "null mesh");
  if (conn) std::memcpy(conn, m->conn.data(), m->conn.size() * sizeof(int32_t));
  if (mass) std::memcpy(mass, m->M.data(), m->M.size() * sizeof(double));
  if (bmass) std::memcpy(bmass, m->Mb.data(), m->Mb.size() * sizeof(double));
  if (sigma) std::memcpy(sigma, m->sigma.data(), m->sigma.size() * sizeof(double));
  return 0;
}

int fwi_num_dofs(const fwi_mesh* m, int64_t* n) {
  if (!m || !n) return fail(FWI_EINVAL, "null argument");
  *n = m->N;
  return 0;
}

int fwi_dof_coords(const fwi_mesh* m, double* xyz) {
  if (!m || !xyz) return fail(FWI_EINVAL, "null argument");
  std::memcpy(xyz, m->dof_xyz.data(), m->dof_xyz.size() * sizeof(double));
  return 0;
}

int fwi_element(const fwi_mesh* m, int* n, double* xhat, double* w, double* dhat) {
  if (!m) return fail(FWI_EINVAL, "null mesh");
  if (n) *n = m->nn;
  if (xhat) std::memcpy(xhat, m->el.xhat.data(), m->el.xhat.size() * sizeof(double));
  if (w) std::memcpy(w, m->el.w.data(), m->el.w.size() * sizeof(double));
  if (dhat) std::memcpy(dhat, m->el.dhat.data(), m->el.dhat.size() * sizeof(double));
  return 0;
}

int fwi_reference_element(int dim, int k, int* n, double* xhat, double* w, double* dhat,
                          int* exact_degree) {
  kmvtab::Element el;
  std::string err;
  if (!kmvtab::build(dim, k, el, err)) return fail(FWI_EINVAL, "KMV tabulation: " + err);
  if (n) *n = el.n;
  if (exact_degree) *exact_degree = el.exact_degree;
  if (xhat) std::memcpy(xhat, el.xhat.data(), el.xhat.size() * sizeof(double));
  if (w) std::memcpy(w, el.w.data(), el.w.size() * sizeof(double));
  if (dhat) std::memcpy(dhat, el.dhat.data(), el.dhat.size() * sizeof(double));
  return 0;
}

int fwi_reference_element_f32(int dim, int k, float* dhat, float* w) {
  kmvtab::Element el;
  std::string err;
  if (!kmvtab::build(dim, k, el, err)) return fail(FWI_EINVAL, "KMV tabulation: " + err);
  std::vector<float> dh, ww;
  kmvtab::fp32_tables(el, dh, ww);
  if (dhat) std::memcpy(dhat, dh.data(), dh.size() * sizeof(float));
  if (w) std::memcpy(w, ww.data(), ww.size() * sizeof(float));
  return 0;
}

int fwi_locate(const fwi_mesh* m, const double* pts, int npts, int32_t* elem_out,
               double* xhat_out) {
  if (!m || (npts > 0 && !pts) || npts < 0) return fail(FWI_EINVAL, "fwi_locate: bad argument");
  std::vector<int> ue;
  std::vector<double> xh;
  if (int rc = locate(m, pts, npts, ue, xh)) return rc;
  std::vector<int> new_of_user(m->E);
  for (int e = 0; e < m->E; ++e) new_of_user[m->order[e]] = e;
  for (int p = 0; p < npts; ++p) {
    if (elem_out) elem_out[p] = new_of_user[ue[p]];
    if (xhat_out)
      for (int c = 0; c < m->dim; ++c) xhat_out[(size_t)p * m->dim + c] = xh[(size_t)p * m->dim + c];
  }
  return 0;
}

int fwi_set_velocity(fwi_mesh* m, const double* c) {
  if (!m || !c) return fail(FWI_EINVAL, "null argument");
  if (int rc = check_device(m)) return rc;
  const int N = m->N, d = m->dim;
  for (int i = 0; i < N; ++i)
    if (!(c[i] > 0) || !std::isfinite(c[i])) return fail(FWI_EINVAL, "velocity must be positive and finite");
  m->c.assign(c, c + N);
  if (m->p.dt > 0) {
    m->dt = m->p.dt;
  } else {
    double rho = gershgorin(m);
    m->dt = m->p.cfl_factor * 2.0 / std::sqrt(rho);
  }
  const double dt = m->dt;
  std::vector<float> c2(N), cv(N), cf((size_t)3 * N);
  const int LC = fwi::layer_coef_count(d);
  std::vector<float> lcf((size_t)m->Nl * LC, 0.f);
  std::vector<unsigned char> mask(N);
  for (int i = 0; i < N; ++i) {
    const double* s = &m->sigma[(size_t)i * d];
    double tr = 0, m3, det1 = 1;
    for (int k = 0; k < d; ++k) tr += s[k];
    if (d == 2) {
      m3 = s[0] * s[1];
    } else {
      m3 = s[0] * s[1] + s[0] * s[2] + s[1] * s[2];
      det1 = s[0] * s[1] * s[2];
    }
    const double a = tr + c[i] * m->Mb[i] / m->M[i];
    const double den = 1.0 + 0.5 * a * dt;
    c2[i] = (float)(c[i] * c[i]);
    cv[i] = (float)c[i];
    cf[i] = (float)((1.0 - 0.5 * a * dt) / den);
    cf[(size_t)N + i] = (float)(dt * dt / (m->M[i] * den));
    cf[(size_t)2 * N + i] = (float)(dt * dt * m3 / den);
    const bool damped = tr > 0;
    mask[i] = (!damped && !(m->p.water_speed > 0 && c[i] < m->p.water_speed)) ? 1 : 0;
    if (m->pidx[i] >= 0) {
      float* L = &lcf[(size_t)m->pidx[i] * LC];
      for (int k = 0; k < d; ++k) {
        double others = tr - s[k];
        double psi2 = s[k] - others;
        double dk = 1.0 + 0.5 * dt * s[k];
        L[k] = (float)((1.0 - 0.5 * dt * s[k]) / dk);
        L[d + k] = (float)(dt * psi2 * c[i] * c[i] / (m->M[i] * dk));
        L[2 * d + k] = (float)(dt / (m->M[i] * dk));
        L[3 * d + k] = (float)(psi2 * c[i] * c[i]);
        if (d == 3) {
          double psi3 = 1;
          for (int l = 0; l < 3; ++l)
            if (l != k) psi3 *= s[l];
          L[4 * d + k] = (float)(dt * psi3 * c[i] * c[i] / (m->M[i] * dk));
          L[5 * d + k] = (float)(psi3 * c[i] * c[i]);
        }
      }
      if (d == 3) {
        L[6 * d + 0] = (float)(dt * dt * det1 / den);
        L[6 * d + 1] = (float)(dt * dt / den);
        L[6 * d + 2] = (float)(dt * det1);
        L[6 * d + 3] = (float)(dt / m->M[i]);
      }
    }
  }
  dfree(m->d_c2);
  dfree(m->d_c);
  dfree(m->d_cf);
  dfree(m->d_lcf);
  dfree(m->d_mask);
  m->d_c2 = m->d_c = m->d_cf = m->d_lcf = nullptr;
  m->d_mask = nullptr;
  int rc;
  if ((rc = upload(&m->d_c2, c2)) || (rc = upload(&m->d_c, cv)) || (rc = upload(&m->d_cf, cf)) ||
      (rc = upload(&m->d_lcf, lcf)) || (rc = upload(&m->d_mask, mask)))
    return rc;
  m->have_velocity = true;
  return 0;
}

int fwi_get_dt(const fwi_mesh* m, double* dt) {
  if (!m || !dt) return fail(FWI_EINVAL, "null argument");
  if (!m->have_velocity) return fail(FWI_EINVAL, "call fwi_set_velocity first");
  *dt = m->dt;
  return 0;
}

int fwi_batch_free(fwi_batch* b) {
  if (!b) return 0;
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->st2) cudaStreamDestroy(b->st2);
  void* ptrs[] = {b->d_inj, b->d_src_elem, b->d_src_phi, b->d_rslot_ptr, b->d_rslot_rec,
                  b->d_rslot_phi, b->d_rec_elem, b->d_rec_phi, b->u, b->v, b->r, b->P, b->Pacc,
                  b->PaccY, b->Y, b->Yacc, b->ua, b->va, b->Pa, b->Ya, b->ckpt, b->ring,
                  b->gseg, b->gsum, b->gcomp, b->misfit, b->status, b->wav_dev, b->rec_dev, b->res_dev, b->stage_in, b->stage_out,
                  b->stage_grad, b->gring};
  for (void* p : ptrs) dfree(p);
  delete b;
  return 0;
}

int fwi_batch_create(fwi_mesh* m, int nshots, const double* src, int nrec, const double* rec,
                     fwi_batch** out) {
  if (!m || !out || nshots <= 0 || nshots > 32 || (nshots & (nshots - 1)) || nrec < 0 || !src ||
      (nrec > 0 && !rec))
    return fail(FWI_EINVAL, "fwi_batch_create: nshots must be a power of two <= 32, points non-null");
  if (!m->have_velocity) return fail(FWI_EINVAL, "call fwi_set_velocity before creating a batch");
  if (int rc = check_device(m)) return rc;
  *out = nullptr;
  std::unique_ptr<fwi_batch, int (*)(fwi_batch*)> b(new fwi_batch(), fwi_batch_free);
  b->m = m;
  b->S = nshots;
  while ((1 << b->log2S) < nshots) ++b->log2S;
  b->R = nrec;
  b->nt = m->p.nsteps;
  b->K = m->p.ckpt_stride;
  b->gstride = m->p.grad_stride;
  b->C = (b->nt + b->K - 1) / b->K;
  if (b->nt <= 0) return fail(FWI_EINVAL, "nsteps must be positive");
  const int d = m->dim, n = m->nn, N = m->N, S = b->S;
  // point location (new element index = position of the user element in the order)
  std::vector<int> new_of_user(m->E);
  for (int e = 0; e < m->E; ++e) new_of_user[m->order[e]] = e;
  std::vector<int> ue;
  std::vector<double> xh;
  if (int rc = locate(m, src, nshots, ue, xh)) return rc;
  b->src_elem.resize(S);
  b->src_phi.resize((size_t)S * n);
  std::vector<double> phi(n);
  for (int s = 0; s < S; ++s) {
    b->src_elem[s] = new_of_user[ue[s]];
    m->el.basis(&xh[(size_t)s * d], phi.data());
    for (int k = 0; k < n; ++k) b->src_phi[(size_t)s * n + k] = (float)phi[k];
  }
  b->rec_elem.resize(nrec);
  b->rec_phi.resize((size_t)nrec * n);
  if (nrec > 0) {
    if (int rc = locate(m, rec, nrec, ue, xh)) return rc;
    for (int r = 0; r < nrec; ++r) {
      b->rec_elem[r] = new_of_user[ue[r]];
      m->el.basis(&xh[(size_t)r * d], phi.data());
      for (int k = 0; k < n; ++k) b->rec_phi[(size_t)r * n + k] = (float)phi[k];
    }
  }
  std::vector<int> inj, sptr, srec;
  std::vector<float> sphi;
  build_injection(m, b.get(), inj, sptr, srec, sphi);
  std::vector<int> src_elem_dev(b->src_elem.begin(), b->src_elem.end());
  std::vector<int> rec_elem_dev(b->rec_elem.begin(), b->rec_elem.end());
  if (rec_elem_dev.empty()) rec_elem_dev.push_back(0);
  std::vector<float> rec_phi_dev = b->rec_phi;
  if (rec_phi_dev.empty()) rec_phi_dev.assign(n, 0.f);
  int rc;
  const size_t NS_ = (size_t)N * S, LS = (size_t)m->Nl * d * S, YS = (size_t)m->Nl * S;
  if ((rc = upload(&b->d_inj, inj)) || (rc = upload(&b->d_src_elem, src_elem_dev)) ||
      (rc = upload(&b->d_src_phi, b->src_phi)) || (rc = upload(&b->d_rslot_ptr, sptr)) ||
      (rc = upload(&b->d_rslot_rec, srec)) || (rc = upload(&b->d_rslot_phi, sphi)) ||
      (rc = upload(&b->d_rec_elem, rec_elem_dev)) || (rc = upload(&b->d_rec_phi, rec_phi_dev)) ||
      (rc = dalloc(&b->u, NS_)) || (rc = dalloc(&b->v, NS_)) || (rc = dalloc(&b->r, NS_)) ||
      (rc = dalloc(&b->P, LS)) || (rc = dalloc(&b->Pacc, LS)) || (rc = dalloc(&b->PaccY, LS)) ||
      (rc = dalloc(&b->Y, YS)) || (rc = dalloc(&b->Yacc, YS)) || (rc = dalloc(&b->ua, NS_)) ||
      (rc = dalloc(&b->va, NS_)) || (rc = dalloc(&b->Pa, LS)) || (rc = dalloc(&b->Ya, YS)) ||
      (rc = dalloc(&b->ckpt, b->state_floats() * b->C)) ||
      (rc = dalloc(&b->ring, NS_ * (b->K / b->gstride))) || (rc = dalloc(&b->gseg, NS_)) ||
      (rc = dalloc(&b->gsum, NS_)) || (rc = dalloc(&b->gcomp, NS_)) ||
      (rc = dalloc(&b->misfit, (size_t)S)) || (rc = dalloc(&b->status, 1)))
    return rc;
  if (m->layout == 0) {
    CUDA_TRY(cudaStreamCreateWithFlags(&b->st2, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming));
  }
  CUDA_TRY(cudaMemset(b->r, 0, NS_ * sizeof(float)));
  if (LS) {
    CUDA_TRY(cudaMemset(b->Pacc, 0, LS * sizeof(float)));
    CUDA_TRY(cudaMemset(b->PaccY, 0, LS * sizeof(float)));
    CUDA_TRY(cudaMemset(b->Yacc, 0, YS * sizeof(float)));
  }
  CUDA_TRY(cudaMemset(b->gseg, 0, NS_ * sizeof(float)));
  CUDA_TRY(cudaMemset(b->gsum, 0, NS_ * sizeof(double)));
  CUDA_TRY(cudaMemset(b->gcomp, 0, NS_ * sizeof(double)));
  CUDA_TRY(cudaMemset(b->misfit, 0, (size_t)S * sizeof(double)));
  CUDA_TRY(cudaMemset(b->status, 0, sizeof(int)));
  *out = b.release();
  return 0;
}

}  // extern "C"

namespace {

StepArgs base_args(fwi_batch* b) {
  fwi_mesh* m = b->m;
  StepArgs a;
  std::memset(&a, 0, sizeof a);
  a.E = m->E;
  a.Es = m->Es;
  a.E0 = m->E0;
  a.S = b->S;
  a.log2S = b->log2S;
  a.Ns = m->Ns;
  a.N = m->N;
  a.bub = m->d_bub;
  if (m->layout == 0) {
    a.nch = m->nch();
    a.nch0 = m->nch0;
    a.ch0 = 0;
    a.N_own = m->N_own;
    a.L_max = m->L_max;
    a.O_max = m->O_max;
    a.H_max = m->H_max;
    a.PE = m->P;
    a.SG = std::min(b->S, 4);
    a.tc = m->use_tc ? 1 : 0;
    a.chunks = m->d_chunks;
    a.halo = m->d_halo;
    a.lconn = m->d_lconn;
    a.h0 = m->N_own;
    a.hcnt = m->N - m->N_own;
  } else {
    a.h0 = 0;
    a.hcnt = m->Ns;
  }
  a.nt = b->nt;
  a.dt = (float)m->dt;
  a.conn = m->d_conn;
  a.geo = m->d_geo;
  a.lgeo = m->d_lgeo;
  a.c2 = m->d_c2;
  a.cvel = m->d_c;
  a.cf = m->d_cf;
  a.pidx = m->d_pidx;
  a.lcf = m->d_lcf;
  a.r = b->r;
  a.Pacc = b->Pacc;
  a.PaccY = b->PaccY;
  a.Yacc = b->Yacc;
  a.inj = b->d_inj;
  a.src_elem = b->d_src_elem;
  a.src_phi = b->d_src_phi;
  a.rslot_ptr = b->d_rslot_ptr;
  a.rslot_rec = b->d_rslot_rec;
  a.rslot_phi = b->d_rslot_phi;
  a.R = b->R;
  a.gseg = b->gseg;
  a.grad_lanes = b->grad_lanes;
  a.gstore = nullptr;
  a.gload = nullptr;
  a.status = b->status;
  a.tc_wait_limit = b->tc_wait_limit;
  return a;
}

void run_step(fwi_batch* b, const StepArgs& a, cudaStream_t st) {
  cudaEvent_t* e = nullptr;
  if (b->prof) {
    while (b->ev.size() < b->ev_used + 3) {
      cudaEvent_t x;
      if (cudaEventCreate(&x) != cudaSuccess) break;
      b->ev.push_back(x);
    }
    if (b->ev.size() >= b->ev_used + 3) {
      e = &b->ev[b->ev_used];
      b->ev_mode.push_back(a.mode);
      b->ev_used += 3;
    }
  }
  if (e) cudaEventRecord(e[0], st);
  if (b->m->layout == 0) {
    // the layer chunks run on a second stream, concurrently with the others (disjoint owned
    // DoFs; halo sums by atomics); the node kernel waits for both
    const bool fork = b->st2 && b->m->nch0 > 0 && b->m->nch() > b->m->nch0;
    if (fork) {
      cudaEventRecord(b->ev_fork, st);
      cudaStreamWaitEvent(b->st2, b->ev_fork, 0);
    }
    int rc = b->m->ks->launch_chunk(a, st, fork ? b->st2 : st);
    if (fork) {
      cudaEventRecord(b->ev_join, b->st2);
      cudaStreamWaitEvent(st, b->ev_join, 0);
    }
    if (rc) b->launch_error = rc;
  } else {
    b->m->ks->launch_step(a, st);
  }
  if (e) cudaEventRecord(e[1], st);
  const fwi_mesh* m = b->m;
  fwi::launch_node_update(a, m->dim, st);
  if (e) cudaEventRecord(e[2], st);
  // chunked layout: one launch per non-empty chunk class (without / with layer elements)
  g_launches += 1 + (m->layout == 0 ? (m->nch0 > 0) + (m->nch() > m->nch0) : 1);
}

// Adds the recorded event intervals to the batch's totals (the stream must be complete).
void collect_profile(fwi_batch* b) {
  for (size_t i = 0; i < b->ev_mode.size(); ++i) {
    float t1 = 0, t2 = 0;
    cudaEventElapsedTime(&t1, b->ev[3 * i], b->ev[3 * i + 1]);
    cudaEventElapsedTime(&t2, b->ev[3 * i + 1], b->ev[3 * i + 2]);
    const int md = b->ev_mode[i];
    b->prof_ms[md][0] += t1;
    b->prof_ms[md][1] += t2;
    b->prof_steps[md] += 1;
  }
  b->ev_mode.clear();
  b->ev_used = 0;
}

// state pointers of checkpoint c: u, v, P, Y
void ckpt_ptrs(fwi_batch* b, int c, float** u, float** v, float** P, float** Y) {
  const fwi_mesh* m = b->m;
  float* base = b->ckpt + b->state_floats() * (size_t)c;
  const size_t NS_ = (size_t)m->N * b->S, LS = (size_t)m->Nl * m->dim * b->S;
  *u = base;
  *v = base + NS_;
  *P = base + 2 * NS_;
  *Y = base + 2 * NS_ + LS;
}

int copy_state(fwi_batch* b, float* du, float* dv, float* dP, float* dY, const float* su,
               const float* sv, const float* sP, const float* sY, cudaStream_t st) {
  const fwi_mesh* m = b->m;
  const size_t NS_ = (size_t)m->N * b->S * sizeof(float);
  const size_t LS = (size_t)m->Nl * m->dim * b->S * sizeof(float);
  const size_t YS = (size_t)m->Nl * b->S * sizeof(float);
  CUDA_TRY(cudaMemcpyAsync(du, su, NS_, cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(dv, sv, NS_, cudaMemcpyDeviceToDevice, st));
  if (LS) CUDA_TRY(cudaMemcpyAsync(dP, sP, LS, cudaMemcpyDeviceToDevice, st));
  if (m->dim == 3 && YS) CUDA_TRY(cudaMemcpyAsync(dY, sY, YS, cudaMemcpyDeviceToDevice, st));
  return 0;
}

int zero_state(fwi_batch* b, float* u, float* v, float* P, float* Y, cudaStream_t st) {
  const fwi_mesh* m = b->m;
  const size_t NS_ = (size_t)m->N * b->S * sizeof(float);
  const size_t LS = (size_t)m->Nl * m->dim * b->S * sizeof(float);
  const size_t YS = (size_t)m->Nl * b->S * sizeof(float);
  CUDA_TRY(cudaMemsetAsync(u, 0, NS_, st));
  CUDA_TRY(cudaMemsetAsync(v, 0, NS_, st));
  if (LS) CUDA_TRY(cudaMemsetAsync(P, 0, LS, st));
  if (YS) CUDA_TRY(cudaMemsetAsync(Y, 0, YS, st));
  return 0;
}

int check_status(fwi_batch* b, cudaStream_t st) {
  if (b->launch_error) {
    int e = b->launch_error;
    b->launch_error = 0;
    return fail(FWI_ECUDA, std::string("chunk kernel launch: ") + cudaGetErrorString((cudaError_t)e));
  }
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  if (b->prof) collect_profile(b);
  if (h) {
    cudaMemsetAsync(b->status, 0, sizeof(int), st);
    if (h & 2) return fail(FWI_ETIMEDOUT, "a bounded wait on the tensor cores gave up (the kernel returned early)");
    return fail(FWI_ERANGE, "non-finite value in the wavefield (time step above the stability limit?)");
  }
  return 0;
}

// Forward steps n0 .. n1-1 on the batch's forward state; optional records and checkpoints.
// window > 0: wav is [S][window] and recs [S][window+1][R] (the steps of one segment).
// gstore: where the steps write the forward field's gradients (one step only).
void forward_steps(fwi_batch* b, int n0, int n1, const float* wav, float* recs, bool ckpts,
                   cudaStream_t st, float* r_scratch = nullptr, int window = 0,
                   float* gstore = nullptr) {
  StepArgs a = base_args(b);
  if (r_scratch) a.r = r_scratch;
  if (window > 0) a.nt = window;
  a.gstore = gstore;
  a.mode = 0;
  a.tc = 0;  // forward and recompute steps always on FP32 CUDA cores (records within 1e-5)
  a.u = b->u;
  a.v = b->v;
  a.P = b->P;
  a.Y = b->Y;
  a.wavelet = wav;
  a.rec = recs;
  for (int n = n0; n < n1; ++n) {
    if (ckpts && n % b->K == 0) {
      float *cu, *cv, *cP, *cY;
      ckpt_ptrs(b, n / b->K, &cu, &cv, &cP, &cY);
      copy_state(b, cu, cv, cP, cY, b->u, b->v, b->P, b->Y, st);
    }
    a.n = n;
    run_step(b, a, st);
  }
}

}  // namespace

extern "C" {

int fwi_forward_shot(fwi_batch* b, const float* wavelet, float* rec_out, void* stream) {
  if (!b || !wavelet) return fail(FWI_EINVAL, "fwi_forward_shot: null argument");
  if (int rc = check_device(b->m)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t wn = (size_t)b->S * b->nt, rn = (size_t)b->S * (b->nt + 1) * b->R;
  if (!b->wav_dev && dalloc(&b->wav_dev, wn)) return FWI_ENOMEM;
  CUDA_TRY(cudaMemcpyAsync(b->wav_dev, wavelet, wn * sizeof(float),
                           is_device_ptr(wavelet) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  const float* wav = b->wav_dev;
  const size_t rsz = rn ? rn : 1;
  if (!b->rec_dev && dalloc(&b->rec_dev, rsz)) return FWI_ENOMEM;
  float* recs = b->rec_dev;
  if (int rc = zero_state(b, b->u, b->v, b->P, b->Y, st)) return rc;
  if (rn) CUDA_TRY(cudaMemsetAsync(recs, 0, rn * sizeof(float), st));
  forward_steps(b, 0, b->nt, wav, recs, true, st);
  if (b->R) {
    StepArgs a = base_args(b);
    a.u = b->u;
    a.rec = recs;
    a.n = b->nt;
    b->m->ks->launch_record(a, b->d_rec_elem, b->d_rec_phi, st);
    g_launches += 1;
  }
  if (rec_out && rn)
    CUDA_TRY(cudaMemcpyAsync(rec_out, recs, rn * sizeof(float),
                             is_device_ptr(rec_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (int rc = check_status(b, st)) return rc;
  b->forward_done = true;
  return 0;
}

}  // extern "C"

namespace {
// Adjoint + gradient accumulation for a device residual [S][nt+1][R].
int adjoint_device(fwi_batch* b, const float* res, cudaStream_t st) {
  if (b->acc_lanes >= 0 && b->acc_lanes != b->grad_lanes)
    return fail(FWI_EINVAL, "the gradient accumulators hold sums of the other kind: call "
                            "fwi_gradient* before changing fwi_batch_set_gradient_lanes");
  // the gradient store: triangles on the persistent kernel, summed gradient form
  const fwi_mesh* mc = b->m;
  const bool gst = b->gstore_on && mc->dim == 2 && mc->layout == 0 && !mc->use_tc &&
                   b->S % 4 == 0 && mc->nch0 > 0 && !b->grad_lanes;
  if (gst && !b->gring) {
    b->gring_level = fwi::gstore_level_floats(mc->nch0, b->S, mc->nn);
    if (int rc = dalloc(&b->gring, b->gring_level * (size_t)(b->K / b->gstride))) return rc;
  }
  b->acc_lanes = b->grad_lanes;
  const size_t rn = (size_t)b->S * (b->nt + 1) * b->R;
  fwi::launch_misfit(res, (int64_t)rn / b->S, b->S, b->misfit, st);
  g_launches += 1;
  StepArgs a = base_args(b);
  a.mode = 1;
  a.u = b->ua;
  a.v = b->va;
  a.P = b->Pa;
  a.Y = b->Ya;
  a.resid = res;
  if (int rc = zero_state(b, b->ua, b->va, b->Pa, b->Ya, st)) return rc;
  const int nt = b->nt;
  // m = nt: lam^{nt} = 0 gives lam^{nt-1} from the last residual sample (no gradient term)
  a.n = nt;
  a.ring_u = nullptr;
  run_step(b, a, st);
  const size_t NS_ = (size_t)b->m->N * b->S;
  for (int c = b->C - 1; c >= 0; --c) {
    const int n0 = c * b->K, n1 = std::min(n0 + b->K, nt);
    float *cu, *cv, *cP, *cY;
    ckpt_ptrs(b, c, &cu, &cv, &cP, &cY);
    if (int rc = copy_state(b, b->u, b->v, b->P, b->Y, cu, cv, cP, cY, st)) return rc;
    // the ring keeps U^n for the levels n = 0 (mod r) of the segment (n0 is one of them);
    // with the gradient store, the forward step from level n also writes the gradients of
    // U^n for the persistent kernel's gradient step, and one more step (from level n1 - 1)
    // gives those of the segment's last level
    const int r = b->gstride;
    CUDA_TRY(cudaMemcpyAsync(b->ring, b->u, NS_ * sizeof(float), cudaMemcpyDeviceToDevice, st));
    auto glevel = [&](int n) { return b->gring + b->gring_level * (size_t)((n - n0) / r); };
    for (int n = n0; n < (gst ? n1 : n1 - 1); ++n) {
      forward_steps(b, n, n + 1, b->wav_dev, nullptr, false, st, nullptr, 0,
                    gst && n % r == 0 ? glevel(n) : nullptr);
      if (n + 1 < n1 && (n + 1) % r == 0)
        CUDA_TRY(cudaMemcpyAsync(b->ring + NS_ * (size_t)((n + 1 - n0) / r), b->u,
                                 NS_ * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    for (int mm = n1 - 1; mm >= std::max(n0, 1); --mm) {
      a.n = mm;
      // the gradient integrand at the subsampled levels only (the others: adjoint step alone)
      a.ring_u = mm % r == 0 ? b->ring + NS_ * (size_t)((mm - n0) / r) : nullptr;
      a.gload = gst && mm % r == 0 ? glevel(mm) : nullptr;
      run_step(b, a, st);
    }
    fwi::launch_fold(b->gseg, b->gsum, b->gcomp, (int64_t)b->m->N * (b->grad_lanes ? b->S : 1),
                     (double)r, st);
    g_launches += 1;
  }
  return check_status(b, st);
}

int stage_signal(fwi_batch* b, const float* src, size_t count, const float** dev, cudaStream_t st) {
  if (is_device_ptr(src)) {
    *dev = src;
    return 0;
  }
  const size_t rn = (size_t)b->S * (b->nt + 1) * b->R, wn = (size_t)b->S * b->nt;
  if (!b->stage_in && dalloc(&b->stage_in, std::max(std::max(wn, rn), (size_t)1))) return FWI_ENOMEM;
  CUDA_TRY(cudaMemcpyAsync(b->stage_in, src, count * sizeof(float), cudaMemcpyHostToDevice, st));
  *dev = b->stage_in;
  return 0;
}
}  // namespace

extern "C" {

// ---- forward solve without allocation ------------------------------------------------
// Static scratch of fwi_forward_shot_noalloc: the accumulator of the DoFs that the node
// kernel finishes (halo DoFs of the chunked layout, shared DoFs of the plain layout), one
// float per (DoF, shot). Every GPU that loads the library holds it until the process exits.
}  // extern "C"

static constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;  // 16 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

namespace {
std::mutex g_noalloc_mu;
float* g_noalloc_addr[64] = {nullptr};

// Device address of the static scratch for the current device (looked up once per device;
// the lookup is the only setup and happens on the first call).
int noalloc_scratch(float** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(FWI_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = (float*)p;
  }
  *out = g_noalloc_addr[dev];
  return 0;
}
}  // namespace

extern "C" {

int fwi_forward_shot_noalloc(fwi_batch* b, const float* wavelet, float* rec_out, void* stream) {
  if (!b || !wavelet || !rec_out) return fail(FWI_EINVAL, "fwi_forward_shot_noalloc: null argument");
  if (int rc = check_device(b->m)) return rc;
  if (!is_device_ptr(wavelet) || !is_device_ptr(rec_out))
    return fail(FWI_EINVAL, "fwi_forward_shot_noalloc: wavelet and rec_out must be device memory");
  const fwi_mesh* m = b->m;
  const size_t need = (size_t)(m->layout == 0 ? m->N - m->N_own : m->Ns) * b->S;
  if (need > kNoAllocScratchFloats)
    return fail(FWI_EINVAL, "fwi_forward_shot_noalloc: mesh too large for the static scratch (" +
                                std::to_string(need) + " > " + std::to_string(kNoAllocScratchFloats) +
                                " floats)");
  cudaStream_t st = (cudaStream_t)stream;
  float* scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  // the accumulator must start at zero (a failed earlier call may have left values)
  if (need) CUDA_TRY(cudaMemsetAsync(scratch, 0, need * sizeof(float), st));
  const size_t rn = (size_t)b->S * (b->nt + 1) * b->R;
  if (int rc = zero_state(b, b->u, b->v, b->P, b->Y, st)) return rc;
  if (rn) CUDA_TRY(cudaMemsetAsync(rec_out, 0, rn * sizeof(float), st));
  // per-kernel event timing would create events: off for this call, restored on every exit
  struct ProfOff {
    fwi_batch* b;
    bool was;
    ~ProfOff() { b->prof = was; }
  } prof_off{b, b->prof};
  b->prof = false;
  forward_steps(b, 0, b->nt, wavelet, rec_out, false, st, scratch);
  if (b->R) {
    StepArgs a = base_args(b);
    a.u = b->u;
    a.rec = rec_out;
    a.n = b->nt;
    m->ks->launch_record(a, b->d_rec_elem, b->d_rec_phi, st);
    g_launches += 1;
  }
  return check_status(b, st);
}

int fwi_forward_segment(fwi_batch* b, int nseg, uint32_t reset_mask, const float* wavelet,
                        float* rec_out, void* stream) {
  if (!b || !wavelet) return fail(FWI_EINVAL, "fwi_forward_segment: null argument");
  if (int rc = check_device(b->m)) return rc;
  if (nseg < 1 || nseg > b->nt)
    return fail(FWI_EINVAL, "fwi_forward_segment: nseg must lie in 1 .. nsteps");
  if (b->S < 32 && (reset_mask >> b->S) != 0)
    return fail(FWI_EINVAL, "fwi_forward_segment: reset_mask names a lane beyond the batch");
  cudaStream_t st = (cudaStream_t)stream;
  const fwi_mesh* m = b->m;
  const size_t wn = (size_t)b->S * nseg, rn = (size_t)b->S * (nseg + 1) * b->R;
  if (!b->wav_dev && dalloc(&b->wav_dev, (size_t)b->S * b->nt)) return FWI_ENOMEM;
  const size_t rfull = (size_t)b->S * (b->nt + 1) * b->R;
  if (!b->rec_dev && dalloc(&b->rec_dev, rfull ? rfull : 1)) return FWI_ENOMEM;
  CUDA_TRY(cudaMemcpyAsync(b->wav_dev, wavelet, wn * sizeof(float),
                           is_device_ptr(wavelet) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  // the batch's checkpoints no longer describe its forward state
  b->forward_done = false;
  if (reset_mask) {
    const int S = b->S;
    fwi::launch_lane_reset(b->u, m->N, S, reset_mask, st);
    fwi::launch_lane_reset(b->v, m->N, S, reset_mask, st);
    fwi::launch_lane_reset(b->P, (int64_t)m->Nl * m->dim, S, reset_mask, st);
    fwi::launch_lane_reset(b->Y, m->Nl, S, reset_mask, st);
    g_launches += 2 + (m->Nl > 0 ? 2 : 0);
  }
  if (rn) CUDA_TRY(cudaMemsetAsync(b->rec_dev, 0, rn * sizeof(float), st));
  forward_steps(b, 0, nseg, b->wav_dev, b->rec_dev, false, st, nullptr, nseg);
  if (b->R) {
    StepArgs a = base_args(b);
    a.u = b->u;
    a.rec = b->rec_dev;
    a.nt = nseg;
    a.n = nseg;
    m->ks->launch_record(a, b->d_rec_elem, b->d_rec_phi, st);
    g_launches += 1;
  }
  if (rec_out && rn)
    CUDA_TRY(cudaMemcpyAsync(rec_out, b->rec_dev, rn * sizeof(float),
                             is_device_ptr(rec_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return check_status(b, st);
}

int fwi_adjoint_shot(fwi_batch* b, const float* residual, void* stream) {
  if (!b || !residual) return fail(FWI_EINVAL, "fwi_adjoint_shot: null argument");
  if (!b->forward_done) return fail(FWI_EINVAL, "fwi_adjoint_shot needs a preceding fwi_forward_shot");
  if (int rc = check_device(b->m)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const float* res = nullptr;
  if (int rc = stage_signal(b, residual, (size_t)b->S * (b->nt + 1) * b->R, &res, st)) return rc;
  return adjoint_device(b, res, st);
}

int fwi_adjoint_misfit(fwi_batch* b, const float* observed, void* stream) {
  if (!b || !observed) return fail(FWI_EINVAL, "fwi_adjoint_misfit: null argument");
  if (!b->forward_done) return fail(FWI_EINVAL, "fwi_adjoint_misfit needs a preceding fwi_forward_shot");
  if (int rc = check_device(b->m)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t rn = (size_t)b->S * (b->nt + 1) * b->R;
  const float* obs = nullptr;
  if (int rc = stage_signal(b, observed, rn, &obs, st)) return rc;
  if (!b->res_dev && dalloc(&b->res_dev, rn ? rn : 1)) return FWI_ENOMEM;
  fwi::launch_residual(b->rec_dev, obs, b->res_dev, (int64_t)rn, st);
  g_launches += 1;
  return adjoint_device(b, b->res_dev, st);
}

}  // extern "C"

namespace {
// G = M^-1 g (M = the lumped mass; nullptr for the raw dJ/dc), masked, summed over the
// batch's shots or per shot ([S][N]); misfit_out gets J (summed, or [S] per shot). Clears the
// accumulators. out and misfit_out may be host or device memory (misfit_out host only).
int finish_gradient(fwi_batch* b, double* out_user, double* misfit_out, const double* M,
                    bool per_lane, cudaStream_t st, const char* name) {
  if (!b || !out_user) return fail(FWI_EINVAL, std::string(name) + ": null argument");
  if (int rc = check_device(b->m)) return rc;
  if (per_lane && b->acc_lanes == 0)
    return fail(FWI_EINVAL, std::string(name) + ": the adjoint summed the shots' gradients; call "
                            "fwi_batch_set_gradient_lanes(b, 1) before it");
  const int N = b->m->N, S = b->S;
  const int lanes = b->acc_lanes == 1 ? S : 1;  // rows the accumulators hold
  const size_t count = per_lane ? (size_t)N * S : (size_t)N;
  double* out = out_user;
  const bool host = !is_device_ptr(out_user);
  if (host) {
    if (!b->stage_grad && dalloc(&b->stage_grad, (size_t)N * S)) return FWI_ENOMEM;
    out = b->stage_grad;
  }
  if (per_lane && b->acc_lanes != 1) {  // nothing accumulated since the last clear: zeros
    CUDA_TRY(cudaMemsetAsync(out, 0, count * sizeof(double), st));
  } else {
    fwi::launch_finish_gradient(b->gsum, b->gcomp, nullptr, M, b->m->d_mask, out, N, lanes,
                                per_lane ? 1 : 0, st);
    g_launches += 1;
  }
  if (host)
    CUDA_TRY(cudaMemcpyAsync(out_user, out, count * sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<double> J(S, 0.0);
  CUDA_TRY(cudaMemcpyAsync(J.data(), b->misfit, S * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (misfit_out) {
    if (per_lane) {
      for (int s = 0; s < S; ++s) misfit_out[s] = J[s];
    } else {
      double t = 0;
      for (double v : J) t += v;
      *misfit_out = t;
    }
  }
  const size_t NS_ = (size_t)N * S;
  CUDA_TRY(cudaMemsetAsync(b->gsum, 0, NS_ * sizeof(double), st));
  CUDA_TRY(cudaMemsetAsync(b->gcomp, 0, NS_ * sizeof(double), st));
  CUDA_TRY(cudaMemsetAsync(b->misfit, 0, S * sizeof(double), st));
  CUDA_TRY(cudaStreamSynchronize(st));
  b->acc_lanes = -1;
  return 0;
}
}  // namespace

extern "C" {

int fwi_gradient(fwi_batch* b, double* grad_out, double* misfit_out, void* stream) {
  return finish_gradient(b, grad_out, misfit_out, b ? b->m->d_M : nullptr, false,
                         (cudaStream_t)stream, "fwi_gradient");
}

int fwi_gradient_lanes(fwi_batch* b, double* grad_out, double* misfit_out, void* stream) {
  return finish_gradient(b, grad_out, misfit_out, b ? b->m->d_M : nullptr, true,
                         (cudaStream_t)stream, "fwi_gradient_lanes");
}

int fwi_batch_set_sources(fwi_batch* b, const double* src) {
  if (!b || !src) return fail(FWI_EINVAL, "fwi_batch_set_sources: null argument");
  fwi_mesh* m = b->m;
  if (int rc = check_device(m)) return rc;
  const int d = m->dim, n = m->nn, S = b->S;
  std::vector<int> ue;
  std::vector<double> xh;
  if (int rc = locate(m, src, S, ue, xh)) return rc;
  std::vector<int> new_of_user(m->E);
  for (int e = 0; e < m->E; ++e) new_of_user[m->order[e]] = e;
  std::vector<double> phi(n);
  for (int s = 0; s < S; ++s) {
    b->src_elem[s] = new_of_user[ue[s]];
    m->el.basis(&xh[(size_t)s * d], phi.data());
    for (int k = 0; k < n; ++k) b->src_phi[(size_t)s * n + k] = (float)phi[k];
  }
  std::vector<int> inj, sptr, srec;
  std::vector<float> sphi;
  build_injection(m, b, inj, sptr, srec, sphi);
  std::vector<int> se(b->src_elem.begin(), b->src_elem.end());
  CUDA_TRY(cudaMemcpy(b->d_inj, inj.data(), inj.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_rslot_ptr, sptr.data(), sptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_rslot_rec, srec.data(), srec.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_rslot_phi, sphi.data(), sphi.size() * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_src_elem, se.data(), se.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(b->d_src_phi, b->src_phi.data(), b->src_phi.size() * sizeof(float),
                      cudaMemcpyHostToDevice));
  b->forward_done = false;
  return 0;
}

int fwi_batch_bytes(const fwi_mesh* m, int nshots, int nrec, int64_t* bytes) {
  if (!m || !bytes || nshots <= 0) return fail(FWI_EINVAL, "fwi_batch_bytes: bad argument");
  const int64_t S = nshots, N = m->N, Nl = m->Nl, d = m->dim, nt = m->p.nsteps;
  const int64_t K = m->p.ckpt_stride, C = (nt + K - 1) / K;
  const int64_t state = S * (2 * N + Nl * (d + (d == 3 ? 1 : 0)));
  int64_t f = 0;
  f += 3 * N * S;                       // u, v, r
  f += 3 * Nl * d * S + 2 * Nl * S;     // P, Pacc, PaccY, Y, Yacc
  f += 2 * N * S + Nl * d * S + Nl * S; // adjoint state
  f += state * C;                       // checkpoints
  const int64_t r = m->p.grad_stride > 1 ? m->p.grad_stride : 1;
  f += N * S * (K / r);                 // recompute ring (subsampled levels only)
  f += N * S;                           // FP32 gradient segments (per shot)
  f += 2 * S * (nt + 1) * nrec + S * nt;  // records, residual, wavelet copies
  *bytes = f * 4 + 2 * N * S * 8 + (int64_t)m->E * 4;  // + compensated FP64 sums per shot
  return 0;
}

int fwi_gradient_raw(fwi_batch* b, double* dJdc_out, double* misfit_out, void* stream) {
  return finish_gradient(b, dJdc_out, misfit_out, nullptr, false, (cudaStream_t)stream,
                         "fwi_gradient_raw");
}

int fwi_batch_set_gradient_store(fwi_batch* b, int on) {
  if (!b || (on != 0 && on != 1))
    return fail(FWI_EINVAL, "fwi_batch_set_gradient_store: on must be 0 or 1");
  b->gstore_on = on;
  if (!on && b->gring) {
    dfree(b->gring);
    b->gring = nullptr;
  }
  return 0;
}

int fwi_batch_set_gradient_lanes(fwi_batch* b, int per_shot) {
  if (!b || (per_shot != 0 && per_shot != 1))
    return fail(FWI_EINVAL, "fwi_batch_set_gradient_lanes: per_shot must be 0 or 1");
  b->grad_lanes = per_shot;
  return 0;
}

int fwi_batch_set_wait_limit(fwi_batch* b, int polls) {
  if (!b) return fail(FWI_EINVAL, "null batch");
  b->tc_wait_limit = polls < 0 ? (1 << 22) : polls;
  return 0;
}

int fwi_profile(fwi_batch* b, int enable) {
  if (!b) return fail(FWI_EINVAL, "null batch");
  b->prof = enable != 0;
  return 0;
}

int fwi_profile_read(fwi_batch* b, double* ms, int64_t* steps) {
  if (!b || !ms || !steps) return fail(FWI_EINVAL, "null argument");
  for (int md = 0; md < 2; ++md) {
    ms[2 * md] = b->prof_ms[md][0];
    ms[2 * md + 1] = b->prof_ms[md][1];
    steps[md] = b->prof_steps[md];
    b->prof_ms[md][0] = b->prof_ms[md][1] = 0;
    b->prof_steps[md] = 0;
  }
  return 0;
}

int fwi_mesh_free(fwi_mesh* m) {
  if (!m) return 0;
  void* ptrs[] = {m->d_conn, m->d_geo, m->d_lgeo, m->d_pidx, m->d_c2, m->d_c, m->d_cf,
                  m->d_lcf, m->d_M, m->d_mask, m->d_bub, m->d_chunks, m->d_halo, m->d_lconn};
  for (void* p : ptrs) dfree(p);
  delete m;
  return 0;
}

}  // extern "C"
