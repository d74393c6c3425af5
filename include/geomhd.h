/*
 * geomhd.h -- C ABI of the GB300 implementation of the one-step ADER-WENO
 * constrained-transport MHD scheme on a radially extruded cubed-sphere mesh of
 * isoparametric hexahedra (Balsara, Florinski, Garain, Subramanian & Gurski,
 * "Efficient, Divergence-Free, High Order MHD on 3D Spherical Meshes with Optimal
 * Geodesic Meshing", arXiv 1905.02504).
 *
 * Conventions for every call
 *   - Return value: GEO_OK (0) or a negative geo_status.  No call throws, aborts
 *     or exits; geo_last_error() returns a message for the last failure of the
 *     calling thread.
 *   - The library owns all device memory of a mesh.  Buffers passed in are owned
 *     by the caller and are never freed or retained by the library.
 *   - Work runs on the CUDA stream given at creation (0 = legacy default stream).
 *     Calls taking host pointers synchronise that stream before returning;
 *     calls taking device pointers only enqueue work, except where noted.
 *   - Units are rationalised (Heaviside-Lorentz): the Gaussian 1/(4 pi) of the
 *     paper's Eq. 2.2 is absorbed into B (B_G = sqrt(4 pi) B).
 *
 * Numbering (identical in every call; n = subdiv, nr = radial shells)
 *   columns        c = (f*n + j)*n + i  (cube face f in +x,+y,+z,-x,-y,-z order,
 *                  equiangular indices i, j); ncol = 6 n^2
 *   zones          z = c*nr + k,  k = 0 (innermost) .. nr-1;  Z = ncol*nr
 *   sphere vertices / sphere edges: first appearance when scanning columns in
 *                  order, corners (i,j),(i+1,j),(i,j+1),(i+1,j+1) and sides
 *                  (j-side, i+1-side, j+1-side, i-side); an edge runs from its
 *                  lower to its higher vertex id
 *   faces          radial faces first: c*(nr+1) + k at radius r_k, normal +r;
 *                  then angular faces F_rad + se*nr + k, normal along t x r
 *   edges          radial edges first: sv*nr + k (r_k to r_k+1, direction +r);
 *                  then angular edges E_rad + se*(nr+1) + k at r_k
 *   r_k = r_in (r_out/r_in)^(k/nr)   (log-ratioed shells, paper Sec. V.b)
 *
 * State
 *   U    : double[8][Z], structure of arrays, conserved zone averages
 *          (rho, rho vx, rho vy, rho vz, energy, Bx, By, Bz); the zone B is the
 *          helper field of paper Sec. IV (overwritten by the divergence-free
 *          reconstruction at the start of every step).
 *   phi  : double[F], magnetic flux through each face along its canonical
 *          normal (the primal, Yee-staggered field of paper Sec. II.c).
 */
#ifndef GEOMHD_H
#define GEOMHD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct geo_mesh* geo_mesh_t;

typedef enum {
  GEO_OK = 0,
  GEO_ERR_ARG = -1,          /* invalid argument (null pointer, bad size/order) */
  GEO_ERR_OOM = -2,          /* device or host allocation failed               */
  GEO_ERR_CUDA = -3,         /* a CUDA runtime call failed                       */
  GEO_ERR_NONPHYSICAL = -4,  /* NaN/Inf or non-positive density/pressure seen    */
  GEO_ERR_STATE = -6         /* call made before the state was uploaded          */
} geo_status;

typedef enum { GEO_FP64 = 0, GEO_FP32_BULK = 1 } geo_precision;

/* Build the mesh and every geometric table on the host (FP64), then upload them.
 * Mesh: paper Sec. II (geodesic mesh, radial extrusion, isoparametric mapping);
 * tables: Eqs. 3.2-3.4 (Taylor moments, stencil least squares), Sec. IV.b steps
 * 1-7 (KKT of the divergence-free reconstruction), Sec. V.d steps 1-4 (ADER
 * matrices and nodal metrics).  Zones of one radial column are self-similar on
 * log-ratioed shells, so tables are stored once per column (paper Sec. IV.b
 * step 7, Sec. V.b).
 *   subdiv  angular zones per cube-face edge (>= 2)
 *   nr      radial shells (>= 2; >= 3 for order 4)
 *   r_in, r_out   shell radii, 0 < r_in < r_out
 *   order   2, 3 or 4 (scheme order p; map degree p-1)
 *   prec    GEO_FP64: every step in FP64.  GEO_FP32_BULK: reconstruction, the
 *           divergence-free fit, the predictor and the Riemann solvers in FP32
 *           (FP32 copies of the per-column matrices, FP64 masters kept on the
 *           device); face-flux and edge-EMF integrals accumulated in FP64 and
 *           the updates of U and phi in FP64, so div B stays at FP64 rounding
 *   stream  cudaStream_t cast to void* (0 = default stream)
 *   out     receives the handle (NULL on failure)                              */
int geo_mesh_create(int subdiv, int nr, double r_in, double r_out, int order,
                    int prec, void* stream, geo_mesh_t* out);
int geo_mesh_destroy(geo_mesh_t mesh);

/* Sizes of the zone, face and edge arrays (any pointer may be NULL). */
int geo_mesh_sizes(geo_mesh_t mesh, int64_t* n_zones, int64_t* n_faces, int64_t* n_edges);

/* Ratio gamma of specific heats (default 5/3). */
int geo_set_gamma(geo_mesh_t mesh, double gamma);

/* Positivity limiting (paper Sec. I: WENO "ruggedized" to be positivity
 * preserving; details not in the paper).  When enabled, every step scales the
 * zone's initial nodal states of the predictor, and then all its predicted
 * face/edge point states, toward the zone mean by one factor theta <= 1 so that
 * density and pressure stay >= min(1e-13, zone mean) at those points (Zhang-Shu
 * type scaling; the pressure bound uses the concavity of p).  Default: off. */
int geo_set_positivity(geo_mesh_t mesh, int enable);

/* Face Riemann solver of the corrector (Sec. VI step 5; the paper does not name
 * its solver and points to higher-fidelity ones in Sec. I):
 *   GEO_RIEMANN_HLL  (0, default): HLL with Davis wave speeds;
 *   GEO_RIEMANN_HLLD (1): HLLD (Miyoshi & Kusano 2005): fast, Alfven and entropy
 *     waves, exact for isolated contacts and rotational discontinuities; the
 *     normal field at a face point is the mean of its two sides'.
 * The edge EMFs keep the multidimensional Rusanov solver.  geo_step_adjoint
 * refuses a mesh set to HLLD (GEO_ERR_ARG).  Returns GEO_ERR_ARG for any other
 * value. */
enum { GEO_RIEMANN_HLL = 0, GEO_RIEMANN_HLLD = 1 };
int geo_set_riemann(geo_mesh_t mesh, int solver);

/* Execution schedule of the predictor stage (a2 zone part + a3, Sec. IV.b steps
 * 8-10 and Eqs. C.34-C.36); all compute the same arithmetic:
 *   GEO_PRED_ZONE_THREAD (0): one thread per zone, its nodal states in
 *     thread-local memory;
 *   GEO_PRED_NODE_TEAM (1, default for GEO_FP64 at order 4): one thread per
 *     serendipity node, a team of N threads per zone exchanging nodal fluxes
 *     through shared memory;
 *   GEO_PRED_VAR_TEAM (2, default at orders 2, 3 and for GEO_FP32_BULK at order
 *     4): the node team, with the derivative contraction and
 *     the face / edge point evaluations done by one thread per (zone, variable,
 *     row group) on the compiled nonzero pattern of D^alpha; with positivity on
 *     the node-team kernel runs instead.
 * They differ only in the summation order of the flux-difference rows.  The
 * reverse sweep of geo_step_adjoint runs its predictor as a node team, or one
 * thread per zone with GEO_PRED_ZONE_THREAD.  Returns GEO_ERR_ARG for any other
 * value. */
enum { GEO_PRED_ZONE_THREAD = 0, GEO_PRED_NODE_TEAM = 1, GEO_PRED_VAR_TEAM = 2 };
int geo_set_predictor(geo_mesh_t mesh, int schedule);

/* Zone cubature for initial data (host buffers, caller-owned):
 * pts double[Z][nq^3][3] physical points, w double[Z][nq^3] physical weights
 * (Jacobian included, summing to the zone volume); nq in 1..12 points per
 * reference direction (tensor Gauss-Legendre on the isoparametric map, Eq. 5.5). */
int geo_zone_cubature(geo_mesh_t mesh, int nq, double* pts, double* w);

/* Edge quadrature for line integrals of a vector potential (host buffers):
 * pts double[E][nq][3], tw double[E][nq][3] = unit tangent * |dl| * weight along
 * the edge's canonical direction; nq in 1..12 (Gauss-Legendre).  Used to set
 * divergence-free face fluxes from an edge circulation (paper Sec. VIII). */
int geo_edge_quadrature(geo_mesh_t mesh, int nq, double* pts, double* tw);

/* Face quadrature of the radial faces f = c (nr + 1) + k (host buffers):
 * pts double[ncol (nr + 1)][nq^2][3] physical points, wn double[...][nq^2][3] =
 * weight * (h_xi x h_eta), the area element along the face's canonical +r
 * normal; nq in 1..12 (tensor Gauss-Legendre on the mapped face).  For fields
 * given by their flux rather than by a vector potential, such as the radial
 * field B_r ~ sin(theta) / r^2 of the spherical shock tubes (paper Sec.
 * VIII.c), which has net flux through every sphere: the radial faces of a
 * column are exact scalings of one another, so the flux of an r^-2 radial field
 * is the same through all of them and each zone stays divergence-free, while
 * the angular faces (planes through the origin) carry none of it. */
int geo_radial_face_quadrature(geo_mesh_t mesh, int nq, double* pts, double* wn);

/* phi[f] = sum over the face's edges of sign * circ[e] (discrete Stokes;
 * host buffers circ double[E], phi double[F]).  The result is exactly
 * divergence-free per zone up to rounding. */
int geo_phi_from_edge_circulation(geo_mesh_t mesh, const double* circ, double* phi);

/* Zone centroids double[Z][3] and volumes double[Z] (host buffers). */
int geo_zone_geometry(geo_mesh_t mesh, double* centroid, double* volume);

/* Face areas double[F] and area-weighted normals double[F][3] (host buffers):
 * the face rule's sum of w_q n_q dA_q on the mapped face (paper App. A rules,
 * Sec. II.c), in the face's canonical orientation (radial faces: +r; angular
 * faces: out of the face's L zone), which is the orientation of phi[f].  Per
 * zone, the six faces' signed normals sum to zero up to rounding. */
int geo_face_geometry(geo_mesh_t mesh, double* area, double* normal);

/* The same zone and face geometry (centroid [Z][3], volume [Z], area [F],
 * area-weighted normal [F][3], host buffers) straight from the host tables of a
 * mesh that is not created on the device: the tables geo_mesh_create builds
 * (isoparametric zones, Sec. II.b), without a GPU.  zones / faces must equal the
 * mesh's Z = 6 subdiv^2 nr and F; GEO_ERR_ARG otherwise or for a bad mesh. */
int geo_host_geometry(int subdiv, int nr, double r_in, double r_out, int order, int64_t zones, int64_t faces,
                      double* centroid, double* volume, double* area, double* normal);

/* Upload / download the state.  on_device != 0: U and phi are device pointers
 * (stream-ordered copies); otherwise host pointers (the call synchronises). */
int geo_state_upload(geo_mesh_t mesh, const double* U, const double* phi, int on_device);
int geo_state_download(geo_mesh_t mesh, double* U, double* phi, int on_device);

/* CFL time step, paper Sec. VII.b: dt = cfl * min_z d_z / (|v_z| + c_f,max,z) with
 * the in-sphere diameter d_z = 6 V_z / S_z.  Device reduction; one scalar is read
 * back (synchronises the stream). */
int geo_cfl_dt(geo_mesh_t mesh, double cfl, double* dt);

/* One full step of length dt (paper Sec. VI): WENO-AO reconstruction (Sec. III),
 * divergence-free B reconstruction (Sec. IV), ADER-CG predictor (Sec. V), HLL
 * face fluxes and multidimensional edge EMFs, finite-volume update of U and the
 * Yee constrained-transport update of phi (Eqs. 2.5-2.6).  Asynchronous on the
 * mesh stream.  The U update raises a device flag when a zone leaves rho > 0,
 * p > 0 or is not finite; the flag is copied to pinned host memory after every
 * step, and a later geo_step whose predecessor's copy has landed returns
 * GEO_ERR_NONPHYSICAL without launching anything (the state is left as
 * computed, for inspection).  geo_check_state reads the flag synchronously. */
int geo_step(geo_mesh_t mesh, double dt);

/* Synchronises the mesh stream, returns the physical-state flags raised since the
 * last upload or check in *flags (bit 0: rho <= 0, p <= 0 or a non-finite
 * energy in some zone after an update) and clears them.  Returns
 * GEO_ERR_NONPHYSICAL when *flags != 0, GEO_OK otherwise.  The paper has no
 * counterpart (its positivity statement is Sec. I). */
int geo_check_state(geo_mesh_t mesh, int* flags);

/* Discrete divergence of the face fluxes (paper Sec. II.c): per zone
 * sum_f s_zf phi_f; returns max |.| and max |.| / sum_f |phi_f| (synchronises). */
int geo_divB_max(geo_mesh_t mesh, double* abs_max, double* rel_max);

/* Adjoint of one step for fixed dt (no counterpart in the paper: a hand-written
 * reverse sweep of every stage of geo_step, Sec. VI; MinMod and the Riemann
 * solvers follow the branch the forward step took).  All pointers are device
 * pointers (caller-owned): U_in double[8][Z] and phi_in double[F] are the state
 * at t (the checkpoint; the step is recomputed from it), gU_out / gphi_out the
 * cotangent at t + dt; gU_in / gphi_in receive the cotangent at t.  Only for
 * GEO_FP64 meshes with the positivity scaling off (GEO_ERR_ARG otherwise; the
 * FP32-bulk form is differentiated by an FP64 mesh of the same geometry applied
 * to its checkpoints).  The mesh's own state is untouched;
 * work buffers are allocated on the first call.  Asynchronous on the mesh stream. */
int geo_step_adjoint(geo_mesh_t mesh, double dt, const double* U_in, const double* phi_in,
                     const double* gU_out, const double* gphi_out, double* gU_in, double* gphi_in);

/* Objective of the differentiation workload: J = sum over the outer radial faces of
 * phi_f^2 / A_f (the integral of the face-mean B_r^2 over r_out).  phi_dev: device
 * double[F]; J: host scalar; gphi_dev: device double[F] receiving dJ/dphi, or NULL.
 * Synchronises the stream. */
int geo_outer_Br2(geo_mesh_t mesh, const double* phi_dev, double* J, double* gphi_dev);

/* Per-stage device timing, accumulated with CUDA events on the mesh stream while
 * enabled.  ms and counts: arrays of GEO_N_STAGES entries in the order
 * weno, bperp, ader, face_flux, edge_emf, update_u, update_phi (host buffers). */
#define GEO_N_STAGES 7
int geo_set_stage_timing(geo_mesh_t mesh, int enable);
int geo_get_stage_timing(geo_mesh_t mesh, double* ms, int64_t* counts);

/* Algorithmic floating-point operations per unit (zone, face or edge) of one
 * geo_step stage, counted from the loop bounds of the method (order-dependent,
 * host only; the same count for the FP64 and the FP32-bulk form; an FMA counts
 * two).  The predictor's count is cross-checked by an operation-counting pass
 * of the test oracle's predictor on one zone. */
int geo_stage_flops(geo_mesh_t mesh, double* flops_per_unit, int64_t* units);

/* Measured FMA throughput of this GPU for the precision: a dependent-chain
 * microbenchmark; result in floating-point operations per second (synchronises). */
int geo_probe_fma_peak(int prec, void* stream, double* flops_per_s);

/* Measurement probe of the predictor's derivative contraction (Eq. C.34,
 * dF_{v,i} = sum_alpha sum_j D^alpha_ij F^alpha_{v,j}) alone, FP32, on the mesh's
 * order: tensor = 0 times the CUDA-core sparse form of the variable-team
 * predictor, tensor = 1 a tensor-core form (mma.sync TF32, three-pass split,
 * dense padded D).  F of each zone is a fixed hash of (zone, alpha, v, j) made on
 * the device (no HBM reads); the contraction runs `reps` times per zone over
 * `zones` zones and the last result goes to out_dev (device, zones x 8 x N
 * floats, [zone][v][node], caller-owned).  *ms = duration of one launch (CUDA
 * events on the mesh's stream, after one untimed launch; synchronises).  Needs a
 * GEO_FP32_BULK mesh (its FP32 reference constants); GEO_ERR_ARG otherwise, or if
 * zones exceeds 2^28.  Not part of geo_step. */
int geo_probe_contraction(geo_mesh_t mesh, int tensor, int64_t zones, int reps, float* out_dev, float* ms);

/* The ADER-CG predictor on the paper's own zones (Sec. V, Eqs. 5.12-5.14 and
 * C.34-C.36): triangular-prism frustums mapped isoparametrically from the
 * reference prism with unit edges and centroid at the origin, order 2, 3 or 4
 * (N = 6 / 15 / 26 serendipity nodes, M = order time levels), FP64.  Per zone the
 * metric terms at the nodes come from the node positions (h_alpha = D^alpha x,
 * J = (h_xi x h_eta) . h_zeta, S^alpha the cofactor vectors), level 1 is J U, and
 * `order` Picard iterations give the space-time nodal solution; the flux
 * difference subtracts the geometric-conservation residual F . sum D^alpha S^alpha,
 * so a uniform state stays uniform.  Device buffers, caller-owned, zone fastest:
 * X_dev [3][N][zones] node positions, U_dev [8][N][zones] conserved variables at
 * the nodes, Uh_dev [M][8][N][zones] the result (J times the conserved state at
 * node i and time level tau_m: tau_1 = 0, then the Gauss points).  Node order as
 * geo_prism_nodes.  Enqueued on `stream` (0 = legacy default), no
 * synchronisation; the reference tables (< 20 KB per order) are built and copied
 * to the device on the first call of each order and kept until exit.
 * GEO_ERR_ARG for a bad order, zone count, null pointer, dt <= 0 or gamma <= 1. */
int geo_prism_predictor(int order, int64_t zones, const double* X_dev, const double* U_dev, double dt, double gamma,
                        double* Uh_dev, void* stream);

/* Reference coordinates (xi, eta, zeta) of the order's prism nodes, [N][3] in
 * host memory (count = doubles the buffer holds): the 6 vertices (top face
 * zeta = +1/2 first), order - 2 equidistant nodes inside each of the 9 edges (the
 * three sides of the top face, of the bottom face, then the three edges along
 * zeta), and at order 4 the two triangle-face centroids (Fig. 7). */
int geo_prism_nodes(int order, double* nodes, int64_t count);

/* The order's prism derivative matrices as geo_prism_predictor uses them:
 * D [3][N][N] host memory, D^alpha_ij = d psi_j / d xi_alpha at node i (Eq. 5.3
 * basis on the monomials of Eqs. 5.12-5.14, nodes as geo_prism_nodes), with the
 * entries that vanish exactly set to zero (the inverse leaves them at rounding
 * level).  count = doubles the buffer holds. */
int geo_prism_derivatives(int order, double* D, int64_t count);

/* The time-coupling matrix R of the ADER-CG predictor that every mesh and
 * geo_prism_predictor use (Eqs. 5.24-5.29, C.35-C.36: U_k = U_1 - sum_m R_km dF_m,
 * time levels tau_1 = 0 and the order-1 Gauss points of [0, 1]): R [M][M] in
 * host memory with M = order, row 1 zero.  count = doubles the buffer holds. */
int geo_time_matrix(int order, double* R, int64_t count);

/* Copy one internal work buffer of the last step to host memory, for stage-by-
 * stage verification: which = 0 WENO-AO Taylor coefficients [8][NC1][Z],
 * 1 nodal normal B per face [NQmax][F], 2 predictor states at face points
 * [M-1][NQT][8][Z], 3 predictor states at edge points [M-1][12][NS][8][Z]
 * (buffers 0-3 are FP32 in the FP32-bulk form and are widened to double),
 * 4 time-integrated face fluxes [8][F], 5 time-integrated edge EMFs [E].
 * count = number of doubles the host buffer holds; GEO_ERR_ARG if too small.
 * Synchronises the stream. */
int geo_debug_buffer(geo_mesh_t mesh, int which, double* host, int64_t count);

/* Test support for stage-by-stage checks (FP64 meshes; host buffers; the calls
 * synchronise).  geo_debug_set_buffer overwrites work buffer `which` (the
 * numbering of geo_debug_buffer; count must equal its size);
 * geo_debug_run_stage launches one forward stage (0 WENO-AO, 1 nodal normal
 * fields, 2 predictor, 3 face fluxes, 4 edge EMFs, 5 U update, 6 Phi update) on
 * the mesh's current buffers; geo_debug_stage_vjp applies the transpose of one
 * stage's Jacobian alone, linearised at the forward intermediates of (U, phi)
 * (the reverse kernels of geo_step_adjoint, Sec. VI read backwards):
 *   stage 0 WENO-AO:   g_out = cotangent of the Taylor coefficients [8][NC1][Z]
 *                      -> g_in = cotangent of U [8][Z]
 *   stage 2 predictor: g_out = cotangents of the face- then edge-point states
 *                      -> g_in = cotangent of the Taylor coefficients (with the
 *                      nodal normal fields and U held fixed)
 *   stage 3 faces:     g_out = [8][F] -> g_in = cotangent of the face-point states
 *   stage 4 edges:     g_out = [E]    -> g_in = cotangent of the edge-point states
 * n_out, n_in must equal those sizes (GEO_ERR_ARG otherwise). */
int geo_debug_set_buffer(geo_mesh_t mesh, int which, const double* host, int64_t count);
int geo_debug_run_stage(geo_mesh_t mesh, int stage, double dt);
int geo_debug_stage_vjp(geo_mesh_t mesh, int stage, double dt, const double* U, const double* phi,
                        const double* g_out, int64_t n_out, double* g_in, int64_t n_in);

/* CFL time step for callers that cannot allocate device memory at the time of
 * the call (a memory pool owned by another component, a rule against device
 * synchronisation, externally managed buffers).  No counterpart in the paper:
 * the same quantity as geo_cfl_dt, computed without any allocation.
 *   U_dev  device double[8][Z], caller-owned conserved variables (same layout as
 *          geo_state_upload); read only
 *   dt_dev device double[1], caller-owned; receives cfl * min_z d_z/(|v|+c_f),
 *          or a non-positive value when a state is non-physical
 * The call only enqueues two kernels on the mesh stream (no synchronisation, no
 * cudaMalloc/cudaFree or any allocating routine).  Scratch: a fixed device
 * array of GEO_NOALLOC_MAX_BLOCKS doubles (512 KB per GPU, kept until exit), so
 * meshes of more than GEO_NOALLOC_MAX_BLOCKS * 256 zones are rejected with
 * GEO_ERR_ARG.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Calls share the array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller. */
#define GEO_NOALLOC_MAX_BLOCKS 65536
int geo_cfl_dt_noalloc(geo_mesh_t mesh, const double* U_dev, double cfl, double* dt_dev);

const char* geo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GEOMHD_H */
