/*
 * fwi.h -- C ABI of the GB300 library for the explicit mass-lumped (KMV) acoustic
 * time step of "Full waveform inversion using triangular waveform adapted meshes"
 * (arXiv 2108.10946): forward solve, discrete adjoint solve and mesh-independent
 * gradient on triangles (k = 2..5) and tetrahedra (k = 2, 3).
 *
 * Conventions for every entry point
 *   - Return value: 0 on success, a negative errno-style code otherwise:
 *       FWI_EINVAL  (-22)  bad argument: det J <= 0, unsupported k, point outside mesh,
 *                          size mismatch, NULL handle
 *       FWI_ENOMEM  (-12)  device or host allocation failed
 *       FWI_ERANGE  (-34)  a non-finite value appeared in the wavefield
 *       FWI_ECUDA   (-5)   a CUDA runtime call failed
 *       FWI_ETIMEDOUT (-110) a bounded wait inside a kernel gave up (the kernel returned
 *                          early and reported it; the context stays usable)
 *     fwi_last_error() copies a one-line description of the most recent failure of the
 *     calling thread. Nothing aborts the process.
 *   - Geometry/coordinate arrays (verts, cells, source and receiver positions, velocity)
 *     are HOST arrays owned by the caller and only read during the call.
 *   - Bulk signal arrays (wavelets, records, residuals, gradients) may be host or device
 *     pointers: the library asks the CUDA runtime which one it is. Host arrays are staged
 *     through library-owned device buffers with copies on the caller's stream.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). The work of a call
 *     is queued on that stream, and every solve (forward, adjoint, gradient) then reads
 *     the batch's device status flag back and synchronises the stream before it returns,
 *     so that a non-finite wavefield or a kernel that gave up is reported by the call
 *     that caused it. Calls therefore return only after their work has completed.
 *   - All device state (mesh, wavefields, checkpoints) is owned by the library and freed
 *     by fwi_batch_free / fwi_mesh_free. Handles are not thread-safe; distinct handles
 *     may be used from distinct threads.
 *   - Coordinates are (x, z) in 2D and (x, y, z) in 3D, with the last axis the depth.
 */
#ifndef FWI_H
#define FWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FWI_EINVAL (-22)
#define FWI_ENOMEM (-12)
#define FWI_ERANGE (-34)
#define FWI_ECUDA (-5)
#define FWI_ETIMEDOUT (-110)

typedef struct fwi_mesh fwi_mesh;
typedef struct fwi_batch fwi_batch;

/* Per-mesh parameters.
 *   dim, k           2 (k = 2..5) or 3 (k = 2, 3): KMVktri / KMVktet (Section 3.2, Figs.
 *                    2dels and 3dels; k = 1 is excluded: Table gwpl shows it does not reach
 *                    the error threshold).
 *   dt               time step; <= 0 selects cfl_factor * 2 / sqrt(rho_Gershgorin(M^-1 K))
 *                    (Eq. spectral, Section 3.4), recomputed by fwi_set_velocity.
 *   cfl_factor       fraction of the Gershgorin bound (the paper uses 10-20 % below it).
 *   nsteps           Nt: records hold Nt + 1 samples (t_n = n dt, n = 0..Nt).
 *   box_lo, box_hi   the physical domain Omega_0 (first dim entries used).
 *   layer_faces      bit 2*d: damping layer below box_lo[d]; bit 2*d+1: above box_hi[d].
 *   layer_width      L; sigma_d(x) = sigma_max * (distance into the layer / L)^2 inside
 *                    the layer on axis d (quadratic profile, Section 2.1).
 *   absorbing        nonzero: lumped Clayton-Engquist term int_{dOmega} c u_t v on the
 *                    whole outer boundary (Appendix A, M_{u,1}).
 *   ckpt_stride      forward checkpoint spacing in steps for the adjoint's recompute.
 *   water_speed      the gradient is zeroed where c < water_speed (Section 5.4: 1.51
 *                    km/s) and inside the damping layer; <= 0 disables the speed test.
 *   layout           0: chunked (elements grouped in chunks that assemble in shared memory;
 *                    the default), 1: plain (one thread per element and shot scattering
 *                    with global atomics; the unfused reference form).
 *   tensor_cores     chunked layout, triangles only: in the adjoint steps (Section 3.5,
 *                    with the gradient integrand) the per-element derivative contractions
 *                    (Section 3.2) of a chunk run as tf32 tensor-core MMAs with a three-term
 *                    hi/lo split (near-FP32 products, FP32 accumulation in tensor memory).
 *                    Forward and recompute steps, which produce the records, stay on FP32
 *                    CUDA cores: the tensor cores' accumulation rounds toward zero, and in
 *                    the forward recurrence that bias grows the seismogram error with the
 *                    record length past 1e-5; in the adjoint it only enters the gradient
 *                    (about 3e-6 against a 1e-4 bound). 0 or -1: off, 1: on (FWI_EINVAL for
 *                    tetrahedra or the plain layout).
 *   grad_stride      r: subsampling of the gradient's time sum (Section 3.6). Only the time
 *                    levels n = 0 (mod r) enter Eq. (gradient3), each with weight r, and the
 *                    adjoint keeps only those forward wavefields (a recompute ring of
 *                    ckpt_stride / r instead of ckpt_stride). <= 1: every level (the exact
 *                    discrete gradient). ckpt_stride must be a multiple of r (FWI_EINVAL).
 */
typedef struct {
  int dim;
  int k;
  double dt;
  double cfl_factor;
  int nsteps;
  double box_lo[3];
  double box_hi[3];
  int layer_faces;
  double layer_width;
  double sigma_max;
  int absorbing;
  int ckpt_stride;
  double water_speed;
  int layout;
  int tensor_cores;
  int grad_stride;
} fwi_params;

/* Builds the DoF numbering, locality order and per-element geometry of a simplex mesh
 * (Sections 3.2 and 4.6). verts: [nverts][dim] doubles; cells: [ncells][dim+1] vertex
 * ids (int32). Every element must have det J > 0 (FWI_EINVAL otherwise). The mesh is
 * uploaded to the current CUDA device. On success *out owns it. */
int fwi_mesh_upload(const double* verts, int64_t nverts, const int32_t* cells, int64_t ncells,
                    const fwi_params* params, fwi_mesh** out);

/* Host-only preparation of the same mesh (numbering, geometry, lumped and boundary mass,
 * damping profile) without touching a GPU: for inspection and tests. The handle supports
 * fwi_num_dofs, fwi_dof_coords, fwi_element, fwi_mesh_host_arrays and fwi_mesh_free. */
int fwi_mesh_prepare_host(const double* verts, int64_t nverts, const int32_t* cells,
                          int64_t ncells, const fwi_params* params, fwi_mesh** out);

/* Host copies: conn[E][n] (DoF of every local node, elements in the library's order),
 * lumped mass[N], lumped boundary mass[N], sigma[N][dim]. Any pointer may be NULL. */
int fwi_mesh_host_arrays(const fwi_mesh* m, int32_t* conn, double* mass, double* bmass,
                         double* sigma);

/* Number of global DoFs N (vertex, edge, face and interior KMV nodes). */
int fwi_num_dofs(const fwi_mesh* m, int64_t* n);

/* Physical coordinates of the DoFs in the library's order: xyz[N][dim] (host). Values
 * per DoF passed in or out of the library (velocity, gradient) use this order. */
int fwi_dof_coords(const fwi_mesh* m, double* xyz);

/* Reference element tabulation (host): nodes xhat[n][dim], lumping weights w[n]
 * (summing to the reference volume 1/dim!), derivative matrices
 * dhat[dim][n][n] = d phi_j / d xhat_d at node q ([d][q][j]). Any pointer may be NULL. */
int fwi_element(const fwi_mesh* m, int* n, double* xhat, double* w, double* dhat);

/* The same tabulation without a mesh or a GPU (host only): KMVktri (dim 2, k = 2..5) or
 * KMVktet (dim 3, k = 2, 3); also returns the highest polynomial degree the lumping rule
 * integrates exactly. Arrays sized as for fwi_element; any pointer may be NULL. */
int fwi_reference_element(int dim, int k, int* n, double* xhat, double* w, double* dhat,
                          int* exact_degree);

/* Point location (host only; works on host-only meshes): for each of npts points pts[p][dim]
 * the containing element in the library's element order and the point's reference
 * coordinates xhat[p][dim] (Section 4.2: sources and receivers are evaluated through the
 * basis of the element that holds them). Ties (a point on a shared edge or vertex) go to
 * the lowest element of the caller's cell order whose barycentric coordinates are all >=
 * -1e-12. A point in no element gives FWI_EINVAL. elem_out or xhat_out may be NULL. */
int fwi_locate(const fwi_mesh* m, const double* pts, int npts, int32_t* elem_out,
               double* xhat_out);

/* The FP32 copies of dhat[dim][n][n] and w[n] that the kernels use (host only). They are not
 * the nearest FP32 values: each derivative row is rounded so that it still differentiates
 * every polynomial of degree <= 2 at its node as exactly as FP32 allows, and the weights so
 * that they still integrate 1 and the coordinates. Rounding every entry to nearest leaves
 * the same error in every element; in a long record it shifts the discrete frequencies
 * coherently and the phase error of the seismograms grows linearly with time. Either pointer
 * may be NULL. */
int fwi_reference_element_f32(int dim, int k, float* dhat, float* w);

/* Sets the P-wavespeed at the DoFs (Section 4.6: c varies inside an element), c[N] host
 * doubles in the order of fwi_dof_coords, all > 0. Recomputes c^2, the lumped damping
 * coefficients and, if params.dt <= 0, the time step. */
int fwi_set_velocity(fwi_mesh* m, const double* c);

/* The time step in use. */
int fwi_get_dt(const fwi_mesh* m, double* dt);

/* A batch of S shots sharing the mesh and a receiver spread (Section 4.2: the source is
 * the transpose of receiver interpolation, b_{g(e,k)} = w(t) phi_k(x_s)).
 * src[S][dim], rec[R][dim] host doubles; every point must lie in the mesh (FWI_EINVAL).
 * Allocates the batch's device state: wavefields, damping-layer auxiliaries, forward
 * checkpoints every ckpt_stride steps and a recompute ring of ckpt_stride wavefields. */
int fwi_batch_create(fwi_mesh* m, int nshots, const double* src, int nrec, const double* rec,
                     fwi_batch** out);

/* Moves the batch's S sources (src[S][dim] host doubles, located as in fwi_batch_create)
 * without reallocating; the next call must be fwi_forward_shot. Lets a shot server reuse a
 * resident batch for new requests on the same mesh and receiver spread. */
int fwi_batch_set_sources(fwi_batch* b, const double* src);

/* Device bytes fwi_batch_create would allocate for nshots shots and nrec receivers on this
 * mesh (state, layer auxiliaries, checkpoints, recompute ring, accumulators, signals): the
 * admission test of a memory-budgeted shot server. */
int fwi_batch_bytes(const fwi_mesh* m, int nshots, int nrec, int64_t* bytes);

/* Forward solve, Eq. (forward3), for every shot of the batch: central differences in time,
 * the damping-layer auxiliaries of Section 2.1 staggered half a step (their damping taken
 * Crank-Nicolson: the paper's own layer scheme is not legible), in the increment form
 * v' = c1 v - c2 K u - c3 u, u' = u + v'. wavelet[S][Nt] floats (w(t_n),
 * n = 0..Nt-1); rec_out[S][Nt+1][R] floats (d^n = H U^n). Stores the checkpoints the
 * adjoint needs. */
int fwi_forward_shot(fwi_batch* b, const float* wavelet, float* rec_out, void* stream);

/* Allocation-free variant of fwi_forward_shot. The paper has no counterpart: this entry
 * point exists for deployment. It serves callers that cannot allocate device memory while
 * they run, for example a shot service that reserves its whole device memory budget at
 * start-up (an allocation in mid-run could fail, fragment that budget or stall other
 * streams), or a host process whose device memory is handed out by an external allocator
 * that the library cannot call.
 *
 * It runs the same forward solve as fwi_forward_shot on the batch's existing state and
 * writes the records. It calls no cudaMalloc, cudaFree or allocating library routine. The
 * only scratch it needs, the accumulator of the DoFs that the node kernel finishes, is a
 * file-scope static __device__ array of 4 Mi floats (16 MiB). Every GPU that loads the
 * library holds that array until the process exits.
 *   - Limit: (halo DoFs, or shared DoFs for the plain layout) x shots <= 4 Mi floats;
 *     beyond it the call returns FWI_EINVAL before launching anything.
 *   - Set-up: the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current. Make that first call before any
 *     stream capture on the device.
 *   - Sharing: every call uses the same array and clears it first. Calls that overlap on
 *     the GPU (other streams, threads or batches) race on it; the caller must serialise
 *     them.
 *   - wavelet[S][Nt] and rec_out[S][Nt+1][R] must be device pointers (FWI_EINVAL
 *     otherwise). No checkpoints are stored, so this call does not prepare an adjoint.
 *   - Like every solve here, it reads the status flag back and synchronises the stream
 *     before it returns. */
int fwi_forward_shot_noalloc(fwi_batch* b, const float* wavelet, float* rec_out, void* stream);

/* Continuous batching inside a record (Section 4.5: the shots of a batch are independent
 * lanes of the same time steps). Advances the batch's forward state by nseg steps
 * (1 <= nseg <= the mesh's nsteps), each lane at its own point of its own shot, so that a
 * caller can start a new shot in a lane that freed up without waiting for the others.
 *   - reset_mask: bit s set = lane s starts a new shot; its wavefield and damping-layer
 *     state are set to zero before the first step. Bits at or above S are an error
 *     (FWI_EINVAL). Other lanes continue from where the last call left them.
 *   - wavelet[S][nseg] (host or device): each lane's source samples for these nseg steps,
 *     i.e. samples t .. t+nseg-1 of that lane's wavelet when the lane stands at step t of its
 *     shot (zeros for an idle lane).
 *   - rec_out[S][nseg+1][R] (host or device, may be NULL): each lane's receiver samples at
 *     the nseg + 1 time levels the call spans, from the level it starts on to the level it
 *     ends on (consecutive calls share one level).
 *   - A lane's records equal those of fwi_forward_shot for the same wavelet, up to the
 *     summation order of FP32 atomics. No checkpoints are stored: after this call the next
 *     fwi_adjoint_* needs a fresh fwi_forward_shot.
 *   - Synchronises the stream before it returns, like every solve here. */
int fwi_forward_segment(fwi_batch* b, int nseg, uint32_t reset_mask, const float* wavelet,
                        float* rec_out, void* stream);

/* Discrete adjoint solve (Section 3.5, the transposed recurrence run backwards) driven by
 * residual[S][Nt+1][R] = d - dtilde, with the forward wavefield recomputed segment by
 * segment from the checkpoints of the last fwi_forward_shot. Accumulates the integrand of
 * Eq. (gradient3), sum_n 2 c grad u^dagger . grad u, of each shot into that shot's
 * compensated FP64 accumulator, and each shot's J = 1/2 sum residual^2. */
int fwi_adjoint_shot(fwi_batch* b, const float* residual, void* stream);

/* The same adjoint solve for the L2 misfit of Eq. (l2error): the residual d - dtilde is
 * formed on the device from the batch's own records of the last fwi_forward_shot and
 * observed[S][Nt+1][R] = dtilde (host or device). */
int fwi_adjoint_misfit(fwi_batch* b, const float* observed, void* stream);

/* G = M^{-1} g (Eq. gradient3), zeroed in the damping layer and where c < water_speed;
 * grad_out[N] doubles in DoF order, misfit_out (may be NULL) the accumulated J. Clears
 * the accumulators. */
int fwi_gradient(fwi_batch* b, double* grad_out, double* misfit_out, void* stream);

/* The shots' own gradients, for callers that batch independent requests (Section 4.5: one
 * gradient per shot, summed over shots by whoever needs the total): grad_out[S][N] doubles
 * (host or device), lane s holding G_s = M^{-1} g_s masked like fwi_gradient; misfit_out
 * (host, may be NULL) gets S doubles, J_s of each shot. The sum over lanes equals what
 * fwi_gradient returns. The adjoint calls must have run with fwi_batch_set_gradient_lanes
 * (b, 1), else FWI_EINVAL; with no adjoint since the last clear the lanes are zero. Clears
 * the accumulators. */
int fwi_gradient_lanes(fwi_batch* b, double* grad_out, double* misfit_out, void* stream);

/* Whether the adjoint calls keep each shot's gradient integrand in its own accumulator
 * (per_shot = 1, needed by fwi_gradient_lanes) or sum the shots as they go (0, the default:
 * one accumulator of N values, fewer memory operations per gradient step). The setting
 * applies from the next fwi_adjoint_* call; changing it while the accumulators hold sums of
 * the other kind (an adjoint ran and no fwi_gradient* cleared them) makes that call return
 * FWI_EINVAL. The batch's device memory is sized for the per-shot form either way. */
int fwi_batch_set_gradient_lanes(fwi_batch* b, int per_shot);

/* Trades memory for arithmetic in the gradient steps (Eq. gradient3), for triangles in the
 * chunked layout with a multiple of 4 shots, the summed gradient form and tensor_cores off
 * (elsewhere the setting has no effect). With on = 1 the forward recompute of each adjoint
 * segment also stores, per element, node, shot and direction, the forward field's
 * (Ghat grad u) at the gradient levels, and the gradient steps read it back instead of
 * contracting the forward field again (one more recompute step per segment gives the last
 * level). The store takes (ckpt_stride / grad_stride) x (chunks without damping-layer
 * elements) x (S / 4) x (nodes per element) x 1 KB of device memory, allocated by the
 * next fwi_adjoint_* call (FWI_ENOMEM if it does not fit) and not counted by
 * fwi_batch_bytes; on = 0 frees it. The results equal those without the store up to FP32
 * summation order. */
int fwi_batch_set_gradient_store(fwi_batch* b, int on);

/* Per-kernel timing (tracing): when enabled, every time step of the batch's forward,
 * recompute and adjoint loops is bracketed by CUDA events on the call's stream. */
int fwi_profile(fwi_batch* b, int enable);
/* ms[4] = {forward element kernel, forward node kernel, adjoint element kernel, adjoint node
 * kernel} total milliseconds and steps[2] = {forward+recompute steps, adjoint steps} timed
 * since the last read (then reset). Recompute steps count as forward steps. */
int fwi_profile_read(fwi_batch* b, double* ms, int64_t* steps);

/* The discrete derivative dJ/dc_i = sum_n 2 c_i sum_e w_i |J_e| grad u_dag . grad u (the
 * right-hand side of Eq. gradient3 before the mass solve; delta c^T dJ/dc is the directional
 * derivative of Eq. control_deriv), masked like fwi_gradient. dJdc_out[N] doubles (host or
 * device), misfit_out may be NULL. Clears the accumulators. */
int fwi_gradient_raw(fwi_batch* b, double* dJdc_out, double* misfit_out, void* stream);

/* Testing aid (no counterpart in the paper): the number of polls each bounded mbarrier wait
 * of the tensor-core kernel makes before it gives up (default 2^22; < 0 restores it; 0 gives
 * up at once). A wait that gives up stops its kernel early, waits (with the default limit)
 * for its MMAs in flight, frees its tensor memory and sets a status bit; the call then
 * returns FWI_ETIMEDOUT and the context stays usable. The batch's results of that call are
 * meaningless. */
int fwi_batch_set_wait_limit(fwi_batch* b, int polls);

int fwi_batch_free(fwi_batch* b);
int fwi_mesh_free(fwi_mesh* m);

/* Copies the calling thread's last error message (NUL-terminated, truncated to len). */
int fwi_last_error(char* buf, int len);

/* Measurement aid (no counterpart in the paper): the FP32 FMA throughput of the current
 * device in TFLOP/s, from a kernel of independent packed FP32x2 FMA chains on every SM (best
 * of five timed launches, CUDA events), and its SM count. The element kernels, at 4 d n^2
 * flops per element and shot, are bound by this rate; it is the denominator of their roofline
 * fraction. Allocates and frees a 16 KiB buffer. */
int fwi_fp32_peak(double* tflops, int* sm_count);

/* Kernel launches the library issued on this thread since the last call (counter read and
 * reset). */
int64_t fwi_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FWI_H */
