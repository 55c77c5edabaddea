/*
 * dg.h -- C ABI of the GB300 nodal discontinuous Galerkin Maxwell library.
 *
 * The library evaluates the semi-discrete nodal DG operator for Maxwell's
 * equations on face-conforming tetrahedral meshes and advances it with the
 * five-stage low-storage RK4 scheme, following Kloeckner, Warburton, Bridge &
 * Hesthaven, "Nodal Discontinuous Galerkin Methods on Graphics Processors":
 *   - problem statement: Section 2, Eq. claw / strong-dg (face-conforming
 *     tetrahedra, order-N nodal Lagrange basis on Warburton's nodes);
 *   - operator: Eq. semidiscrete-dg with the matrices of Eq.
 *     dg-global-matrices, Eq. dg-reference-matrices and Fig. lifting-matrix;
 *   - physics: Maxwell's equations of Section 6 (Eq. maxwells-claws) with
 *     eps = mu = 1, no current, and the upwind flux of Section 6; every face
 *     that is not shared by two tetrahedra is a perfectly conducting wall
 *     (ghost state E+ = -E-, H+ = H-);
 *   - time stepping: the LSERK4 scheme of Carpenter & Kennedy cited in
 *     Section 6.
 *
 * Conventions shared by every call
 *   - Return value: DG_OK (0) or one of the negative DG_ERR_* codes below;
 *     dg_last_error() then returns a message (thread-local, valid until the
 *     next failing call on the same thread).
 *   - Fields are six FP32 arrays in structure-of-arrays order
 *         u[c][k][i],  c = 0..5 (Ex, Ey, Ez, Hx, Hy, Hz), k = 0..K-1, i = 0..Np-1
 *     i.e. a contiguous block of 6*K*Np floats.  Element numbering k is the
 *     caller's tetrahedron order; node numbering i is the order returned by
 *     dg_nodes().
 *   - Ownership: the library owns the mesh, its operators and its device
 *     geometry; the caller owns every field buffer it passes in.  Device
 *     pointers must point to memory of the current CUDA device.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device calls are asynchronous on that stream unless
 *     stated otherwise.  A mesh must not be used from two host threads at once.
 *   - Orders: 1 <= N <= 9.
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK            0
#define DG_ERR_ARG      -1   /* null pointer, bad size, bad value            */
#define DG_ERR_MESH     -2   /* degenerate tetrahedron, bad index, face shared by >2 tets */
#define DG_ERR_ORDER    -3   /* order outside 1..9                           */
#define DG_ERR_CUDA     -4   /* a CUDA runtime call failed                   */
#define DG_ERR_OOM      -5   /* host or device allocation failed             */
#define DG_ERR_UNSTABLE -6   /* energy not finite (NaN/Inf): time step too large or bad data */
#define DG_ERR_STATE    -7   /* call needs dg_set_order() first              */

typedef struct dg_mesh dg_mesh;  /* opaque, library-owned */

/*
 * Build a mesh from vertex coordinates and tetrahedra (Section 2: a domain made
 * of disjoint, face-conforming tetrahedra).
 *   verts : host, [nv][3] doubles (x, y, z), read only, copied.
 *   tets  : host, [K][4] int32 vertex indices (0-based), read only, copied.
 *           A tetrahedron with negative orientation has its last two vertices
 *           swapped internally; element numbering is unchanged.
 *   out   : receives the new mesh; free it with dg_mesh_destroy().
 * Faces are matched by their vertex triples; an unmatched face is a PEC wall.
 * Errors: DG_ERR_ARG (null, nv < 4, K < 1, K*220 >= 2^31), DG_ERR_MESH
 * (index out of range, zero-volume tetrahedron, face shared by more than two
 * tetrahedra).  Host only; needs no GPU.
 */
int dg_mesh_create(const double* verts, int64_t nv, const int32_t* tets, int64_t K,
                   dg_mesh** out);

/*
 * Set the polynomial order N (1..9) and build, on the host in FP64, the
 * reference operators (Dr, Ds, Dt, M, LIFT of Eq. dg-global-matrices and Fig.
 * lifting-matrix on Warp & Blend nodes), the face-node connectivity and the
 * per-element geometry (Eq. dg-reference-matrices).  Device buffers are
 * created lazily on the first device call.  May be called again to change N.
 * Errors: DG_ERR_ARG, DG_ERR_ORDER.  Host only; needs no GPU.
 */
int dg_set_order(dg_mesh* mesh, int N);

/*
 * A new mesh that packs several meshes of the same order into one (the packed
 * element table of a batch of independent solves): vertices, elements,
 * geometry and connectivity are concatenated in the given order with vertex
 * and element indices offset, so the result has count separate components and
 * element k of meshes[i] becomes element k + (K of meshes[0..i-1]).  No face
 * matching or geometry is recomputed.  Its dt_cfl is the smallest of theirs.
 *   meshes : host array of count meshes with an order set (same N and flux).
 *   out    : receives the new mesh; free it with dg_mesh_destroy().
 * Errors: DG_ERR_ARG (NULL, count < 1, different orders or fluxes, too many
 * elements), DG_ERR_STATE (a mesh without an order).  Host only.
 */
int dg_mesh_pack(const dg_mesh* const* meshes, int count, dg_mesh** out);

/* K, Np = (N+1)(N+2)(N+3)/6, Nfp = (N+1)(N+2)/2 and the CFL step
 * dt = min_{k,f} (J_k / sJ_{k,f}) * 2/(N+1)^2.  Any output may be NULL. */
int dg_info(const dg_mesh* mesh, int64_t* K, int* Np, int* Nfp, double* dt_cfl);

/* Physical node coordinates, host [3][K][Np] doubles (x block, y block, z). */
int dg_nodes(const dg_mesh* mesh, double* xyz);

/*
 * Face-node connectivity (the face index lists of Section 5.2), host int32
 * arrays of K*4*Nfp entries ordered (k, face f, face node j):
 *   vmapM[(k*4+f)*Nfp+j] = k*Np + (index of face node j of face f),
 *   vmapP[...]           = global node id of the same point in the neighbour,
 *                          or vmapM on a wall face.
 * Faces: f0 = (v0 v1 v2), f1 = (v0 v1 v3), f2 = (v1 v2 v3), f3 = (v0 v2 v3)
 * of the (orientation-corrected) tetrahedron; face nodes in ascending node order.
 */
int dg_get_connectivity(const dg_mesh* mesh, int32_t* vmapM, int32_t* vmapP);

/*
 * Element numbering for flux-gather locality (Section 5.2, "Flux Extraction",
 * Algorithm 2, the greedy breadth-first partition): the face-adjacency graph
 * is cut into blocks of `block` consecutive positions (the last may be
 * shorter), each grown from a seed by taking the queued element that shares
 * the most faces with the block (ties: the one queued first); a full block's
 * queue head seeds the next block, and an empty queue takes the
 * lowest-numbered element not yet placed.
 *   block : elements per block, >= 1; 20 matches the tensor-core stage's tiles.
 *   perm  : host, [K] int64, written: perm[i] = current index of the element to
 *           place at position i.  Renumber with tets'[i] = tets[perm[i]] and
 *           fields u'[c][i] = u[c][perm[i]] (a new mesh from tets'); results are
 *           the same up to that renumbering.
 * Needs only dg_mesh_create (no order, no GPU).  Errors: DG_ERR_ARG (NULL
 * mesh or perm, block < 1).
 */
int dg_partition_order(const dg_mesh* mesh, int64_t block, int64_t* perm);

/* Reference operators in FP64, row-major: Dr, Ds, Dt, M are [Np][Np], LIFT is
 * [Np][4*Nfp].  Any pointer may be NULL. */
int dg_get_operators(const dg_mesh* mesh, double* Dr, double* Ds, double* Dt,
                     double* M, double* LIFT);

/* Per-element geometry in FP64: metric [9][K] (rx ry rz sx sy sz tx ty tz),
 * J [K], normals [3][K][4], Fscale = sJ/J [K][4].  Any pointer may be NULL. */
int dg_get_geometry(const dg_mesh* mesh, double* metric, double* J, double* normals,
                    double* Fscale);

/* Flux parameter alpha: 1 = upwind (default), 0 = central (energy conserving).
 * Host only. */
int dg_set_flux(dg_mesh* mesh, double alpha);

/* Materials (Section 6, where diag(eps, mu) multiplies u_t): per-element
 * permittivity eps[k] and permeability mu[k], host arrays of K finite values
 * > 0 (copied); NULL sets 1 for every element (vacuum, the default).  The
 * stage then divides rhs_E by eps and rhs_H by mu and uses the upwind flux of
 * Section 6 with impedance Z = sqrt(mu/eps) and admittance Y = 1/Z:
 *   E: 1/(Z- + Z+) n x ( Z+ [H] - alpha n x [E]),
 *   H: 1/(Y- + Y+) n x (-Y+ [E] - alpha n x [H]),   [u] = u+ - u-;
 * dg_energy weights E by eps and H by mu, and dt_cfl scales with
 * min sqrt(eps mu).  Every stage implementation supports materials and
 * absorbing faces (the tensor-core kernels through a separate instantiation,
 * so vacuum meshes run unchanged code).  Host only.  Errors: DG_ERR_ARG (NULL mesh, a value not
 * finite or <= 0), DG_ERR_OOM. */
int dg_set_materials(dg_mesh* mesh, const double* eps, const double* mu);

/* Boundary condition of every boundary face: kind[4 k + f] for face f of
 * element k (faces numbered as in dg_get_connectivity), either DG_BC_PEC
 * (perfect conductor: E+ = -E-, H+ = H-; the default) or DG_BC_ABSORBING
 * (characteristic absorbing boundary: exterior state zero, Z+ = Z-, so no
 * wave enters).  Entries of interior faces are ignored.  NULL: every boundary
 * face a perfect conductor.  Host only.  Errors: DG_ERR_ARG (NULL mesh, a kind
 * other than 0 or 1), DG_ERR_OOM. */
#define DG_BC_PEC       0
#define DG_BC_ABSORBING 1
int dg_set_boundary(dg_mesh* mesh, const int8_t* kind);

/*
 * Implementation of the RK-stage operator (the paper notes that each operator
 * part may need its own strategy on the GPU, Section 4):
 *   DG_STAGE_AUTO   tensor cores for N = 2..7, FP32 CUDA cores for N = 1 and
 *                   above 7 (the faster kernel of each order on GB300; default);
 *   DG_STAGE_FP32   FP32 CUDA cores for every order;
 *   DG_STAGE_TC     tensor cores (tcgen05): the volume and lifting contractions
 *                   as one GEMM per tile with three FP16 products
 *                   (A_hi B_hi + A_hi B_lo + A_lo B_hi, power-of-two row
 *                   scaling, FP32 accumulation), FP32 elsewhere; orders 1..7
 *                   (orders 5..7 with [Dr Ds Dt LIFT] held in tensor memory,
 *                   at order 7 the last k-steps of its low piece in shared
 *                   memory).  Its tiles move by bulk copies, so it also needs
 *                   K*Np to be a multiple of 4 and 16-byte aligned field
 *                   buffers; otherwise (and for N > 7) the call runs
 *                   DG_STAGE_FP32.
 * Host only.  Errors: DG_ERR_ARG for an unknown value.
 */
#define DG_STAGE_AUTO 0
#define DG_STAGE_FP32 1
#define DG_STAGE_TC   2
int dg_set_stage_impl(dg_mesh* mesh, int impl);

/* Tile shape of the FP32 CUDA-core stage (orders 1, 8 and 9 by default, any
 * order with DG_STAGE_FP32): 0 (default) the tile sizes measured fastest on
 * large meshes, 1 half the tetrahedra per tile with the same matrix rows per
 * thread (twice the CTAs of a small mesh, half the shared tiles).  The tile
 * size is the analogue of the work partitioning the paper tunes empirically
 * (Section 6); the serving loop's autotuner picks it per order and size.
 * Results are the same to rounding.  Host only.  Errors: DG_ERR_ARG (NULL
 * mesh, shape other than 0 or 1). */
int dg_set_stage_shape(dg_mesh* mesh, int shape);

/*
 * One evaluation of the semi-discrete operator (Eq. semidiscrete-dg):
 * rhs = curl terms (local differentiation, Alg. 4) + LIFT * flux (flux
 * extraction, Alg. 3, and lifting, Alg. 1).
 *   u   : device, [6][K][Np] FP32, read only.
 *   rhs : device, [6][K][Np] FP32, written; must not overlap u.
 * Asynchronous on `stream`.
 */
int dg_rhs(dg_mesh* mesh, const float* u, float* rhs, void* stream);

/*
 * Advance nsteps LSERK4 steps of size dt (5 stages each):
 *   res <- a_i res + dt rhs(u);  u <- u + b_i res,  i = 0..4.
 *   u   : device, [6][K][Np] FP32, in/out (state).
 *   res : device, [6][K][Np] FP32, in/out (RK register; zero it at t = 0).
 * The stage update is fused into the operator kernel; the library keeps one
 * device work copy of u per mesh (allocated on first use).
 * Asynchronous on `stream`.  Errors: DG_ERR_ARG (dt <= 0, nsteps < 0).
 */
int dg_step(dg_mesh* mesh, float* u, float* res, double dt, int nsteps, void* stream);

/*
 * One LSERK4 stage i (0..4) of size dt, with the coefficients a_i, b_i used by
 * dg_step:
 *   res <- a_i res + dt rhs(u_in);  u_out <- u_in + b_i res.
 *   u_in  : device, [6][K][Np] FP32, read.
 *   u_out : device, [6][K][Np] FP32, written; must not be u_in (the stage reads
 *           neighbours' values of u_in while it writes u_out).
 *   res   : device, [6][K][Np] FP32, in/out; a third buffer.
 * Stages 0..4 with u_in and u_out swapped after each stage make one step
 * (bit-identical to dg_step); a caller can act between stages, e.g. refresh
 * ghost elements' face values in a domain decomposition.
 * Asynchronous on `stream`.  Errors: DG_ERR_ARG (NULL, aliased buffers, stage
 * outside 0..4, dt <= 0).
 */
int dg_rk_stage(dg_mesh* mesh, const float* u_in, float* u_out, float* res, int stage,
                double dt, void* stream);

/*
 * dg_rk_stage for the elements [k0, k1) only; the others' u_out and res are
 * not touched.  With the elements of a subdomain numbered interior first (no
 * face to a ghost element), a stage can run on the interior while the ghosts'
 * face values are exchanged, then on the rest (the one-mesh decomposition of
 * Section 6's multi-GPU outlook; paper_0901_1024_gb300/domain.py): every
 * element's result is bit for bit that of dg_rk_stage, provided the elements
 * of the first call read no value written between the two calls.
 *   k0, k1 : multiples of the stage kernel's tile (dg_stage_tile), or k1 = K.
 * Asynchronous on `stream`.  Errors: as dg_rk_stage; DG_ERR_ARG for a range
 * outside 0 <= k0 < k1 <= K or not on tile boundaries.
 */
int dg_rk_stage_range(dg_mesh* mesh, const float* u_in, float* u_out, float* res, int stage,
                      double dt, int64_t k0, int64_t k1, void* stream);

/*
 * Self-test of failure detection in the tensor-core stages: every mbarrier
 * wait of those kernels is bounded and, when it runs out, sets the mesh's
 * pipeline status word, which dg_energy, dg_energy_range and dg_step_host read
 * (and clear) after their synchronisation and report as DG_ERR_CUDA.  This
 * call runs the same bounded wait, limited to `polls` polls, in a one-warp
 * kernel on an mbarrier that nothing arrives at (nothing else is in flight,
 * so no GPU fault or hang is involved), then makes the same check.
 *   polls   : 1 .. 2^24.
 *   seconds : host, out, may be NULL: GPU time the bounded wait took.
 * Synchronous (default stream); it uses the mesh's status word and energy
 * result word, so it must not overlap other calls on the same mesh.  Returns
 * DG_ERR_CUDA with the stage kernels' timeout message -- the expected
 * outcome -- and leaves the status word clear, so the mesh stays usable;
 * DG_ERR_STATE if the wait did not time out; DG_ERR_ARG for polls out of
 * range.
 */
int dg_check_wait_timeout(dg_mesh* mesh, uint32_t polls, double* seconds);

/*
 * Tetrahedra per tile of the stage kernel that runs on these buffers (the
 * tensor-core kernels need 16-byte aligned buffers; NULL pointers count as
 * aligned): the granularity of dg_rk_stage_range.  Uploads the mesh to the
 * current device if needed.  Errors: DG_ERR_ARG (NULL tile), DG_ERR_STATE
 * (no order), DG_ERR_CUDA.
 */
int dg_stage_tile(dg_mesh* mesh, const float* u_in, const float* u_out, const float* res,
                  int* tile);

/*
 * dg_rk_stage with a time step per element: element k's update uses
 * dt_elem[k] in place of dt.
 *   dt_elem : device, [K] FP32, read; positive.
 * For several independent solves packed into one mesh (disjoint vertex and
 * element sets, each solve with its own step): every element's result is bit
 * for bit its solve's dg_rk_stage result with dt = that float step.
 * Asynchronous on `stream`.  Errors: as dg_rk_stage; dt_elem NULL.
 */
int dg_rk_stage_elem(dg_mesh* mesh, const float* u_in, float* u_out, float* res, int stage,
                     const float* dt_elem, void* stream);

/*
 * One LSERK4 stage i (0..4) of several meshes -- e.g. the packed meshes
 * (dg_mesh_pack) of a batch of solves of different orders -- in as few
 * launches as possible: the meshes that run on the tensor cores at orders
 * 1..4 share one persistent launch, those at orders 5, 6 another; each launch
 * splits its CTAs (one per SM) among the meshes in proportion to their tiles x
 * tile_cost, so all of them advance side by side on the GPU.  Meshes on the
 * tensor-core stage at order 7 and those on the FP32 CUDA-core stage (orders
 * >= 8, forced FP32, unaligned sizes) get their own launch.  For mesh i the
 * result is bit for bit that of
 *   dg_rk_stage_elem(meshes[i], u_in[i], u_out[i], res[i], stage, dt_elem[i])
 * (or of dg_rk_stage with dt where dt_elem or dt_elem[i] is NULL): the paper's
 * element-local work (Section 5) assigned across solves.
 *   meshes    : host array of n distinct meshes, all resident on the current
 *               device (an order set on each);
 *   u_in, u_out, res : host arrays of n device pointers, as in dg_rk_stage;
 *   dt_elem   : host array of n device pointers to [K_i] FP32 steps, or NULL;
 *   tile_cost : host array of n positive costs of one tile on one SM (any unit,
 *               e.g. from timing each mesh alone), or NULL for the library's
 *               per-order defaults; only the ratios matter.
 * Up to 8 meshes share a launch (more take more launches).  While tracing is on
 * (meshes[0]'s trace) a shared launch is recorded as kind 6.
 * dg_last_launch_count(meshes[0]) gives the launches issued.  Asynchronous on
 * `stream`.  Errors: DG_ERR_ARG (NULL arrays or buffers, n < 1, a repeated
 * mesh, aliased buffers, stage outside 0..4, dt <= 0, meshes on different
 * devices), DG_ERR_STATE (no order set), DG_ERR_CUDA.
 */
int dg_rk_stage_multi(dg_mesh* const* meshes, int n, const float* const* u_in,
                      float* const* u_out, float* const* res, const float* const* dt_elem,
                      int stage, double dt, const double* tile_cost, void* stream);

/*
 * Discrete energy 1/2 sum_k J_k sum_c u_kc^T M u_kc (FP32 products, FP64
 * accumulation across elements) written to *out (host).
 *   u : device, [6][K][Np] FP32.
 * Synchronises `stream`.  Returns DG_ERR_UNSTABLE if the energy is not finite.
 */
int dg_energy(dg_mesh* mesh, const float* u, double* out, void* stream);

/*
 * The energy of elements k0 <= k < k1 only, e.g. one solve of a packed mesh
 * (dg_mesh_pack); the same reduction as dg_energy, which is the range 0..K.
 * Errors: as dg_energy; DG_ERR_ARG unless 0 <= k0 < k1 <= K.
 */
int dg_energy_range(dg_mesh* mesh, const float* u, int64_t k0, int64_t k1, double* out,
                    void* stream);

/*
 * End-to-end convenience: copy host fields to the device, advance nsteps
 * LSERK4 steps, copy the fields back and (if energy != NULL) compute the
 * energy of the result.
 *   u   : host, [6][K][Np] FP32, in/out (page-locked memory is fastest);
 *   res : host RK register, [6][K][Np] FP32, in/out, or NULL: then only u
 *         crosses the bus and the device register starts from zero (a step's
 *         result does not depend on it: the first LSERK4 stage has a = 0).
 * Uses library-owned device buffers; synchronises `stream`.  With the energy
 * check on (dg_set_energy_check) it also computes the energy of the incoming
 * state and returns DG_ERR_UNSTABLE, after copying the fields back and
 * writing *energy, if the energy grew by more than the allowed factor.
 */
int dg_step_host(dg_mesh* mesh, float* u, float* res, double dt, int nsteps,
                 double* energy, void* stream);

/*
 * Instability detector for dg_step_host (the paper has no counterpart; a
 * library service).  With upwind or central flux and perfect-conductor or
 * absorbing boundaries the discrete energy of a stable run does not grow
 * (Section 6's dissipative upwind flux; LSERK4 inside its stability region),
 * so growth flags a time step above the stability limit or a corrupted state.
 *   max_growth >= 0: dg_step_host computes E_in (the incoming state) and
 *                    E_out (the result) and fails with DG_ERR_UNSTABLE when
 *                    E_out > E_in (1 + max_growth) or E_out is not finite;
 *                    about 1e-6 per step covers FP32 rounding;
 *   max_growth <  0: off (the default).
 * Costs one more energy evaluation and host synchronisation per call.  Host
 * only.  Errors: DG_ERR_ARG (NULL mesh, NaN). */
int dg_set_energy_check(dg_mesh* mesh, double max_growth);

/* Number of kernel launches the last dg_rhs / dg_step / dg_energy /
 * dg_step_host call on this mesh issued (for launch accounting). */
int64_t dg_last_launch_count(const dg_mesh* mesh);

/*
 * Per-launch tracing (the paper times its kernels with CUDA events, Section 6).
 * dg_trace_enable(mesh, n) with n > 0 clears the record, reserves event pairs
 * for n launches (more are created on demand) and turns tracing on; n = 0
 * turns it off.  While on, dg_rhs, dg_step, dg_energy and dg_step_host record
 * a CUDA event before and after every kernel launch, on the caller's stream,
 * appending to the record.  The reservation happens on the current device,
 * outside any later timed region.  Errors: DG_ERR_ARG (n < 0), DG_ERR_STATE
 * (n > 0 before dg_set_order), DG_ERR_CUDA.
 */
int dg_trace_enable(dg_mesh* mesh, int n);

/*
 * Durations of the launches recorded since the last dg_trace_enable(), in
 * launch order:
 *   ms   : host, receives up to `cap` device durations in milliseconds;
 *   kind : host, receives the kernel of each launch (0 = fused RK stage and
 *          1 = right-hand side on CUDA cores, 4 = fused RK stage and 5 =
 *          right-hand side on tensor cores, 2 = energy partial sums, 3 =
 *          energy final sum, 6 = one launch of dg_rk_stage_multi over several
 *          meshes); may be NULL;
 *   count: receives the number of recorded launches (may exceed cap).
 * Waits for the last recorded event.  Errors: DG_ERR_STATE if nothing was traced.
 */
int dg_trace_read(dg_mesh* mesh, double* ms, int32_t* kind, int64_t cap, int64_t* count);

/*
 * dg_energy without any allocation (the paper has no counterpart; this is a
 * library service).  For callers that must not allocate device memory while
 * they run -- e.g. a serving process whose HBM is owned by its own pool and
 * budget, or a time loop that keeps cudaMalloc/cudaFree, which can
 * synchronise the device, out of its steady state.
 *   u      : device, [6][K][Np] FP32, read only.
 *   energy : device, receives one double, 1/2 sum_k J_k sum_c u^T M u.
 * The partial sums live in a fixed 512 KiB device array inside the library
 * (held by every GPU that loads the library until exit), so K may not exceed
 * 4 194 304 tetrahedra (DG_ERR_ARG otherwise).  The mesh must already be on
 * the current device (one earlier dg_rhs, dg_step or dg_energy call on it,
 * else DG_ERR_STATE), because uploading it would allocate.  The first call on
 * a device looks up that device's address of the array (again after the
 * device's context has been replaced, e.g. by cudaDeviceReset); with lazy
 * module loading that first lookup loads the library's device code and with it
 * the array, so the first call is not itself free of allocation: make it
 * during set-up, before any stream capture.  Asynchronous on `stream`; no host
 * sync, and unlike dg_energy it reads no pipeline status word and does not
 * check the energy for finiteness: callers check the result themselves (e.g.
 * isfinite after their own copy, or a dg_energy call).  While tracing is on
 * (dg_trace_enable) its two launches are recorded as kinds 2 and 3.  All calls
 * share the array: calls that overlap on the GPU race on it.
 */
int dg_energy_noalloc(dg_mesh* mesh, const float* u, double* energy, void* stream);

/* Free the mesh and every device buffer it owns.  NULL is ignored. */
void dg_mesh_destroy(dg_mesh* mesh);

/* Message of the last failing call on this thread ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_GB300_H */
