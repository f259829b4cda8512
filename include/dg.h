/*
 * dg.h -- C ABI of the GB300 tree-based dGSEM library (arXiv 2404.16648, hot path).
 *
 * The library advances the perturbation form of the compressible Euler equations
 * (rho', rho u, rho theta' about a hydrostatic background; Sec. 2.1, Eq. "eulervector") with a
 * nodal strong-form discontinuous Galerkin spectral element method on LGL nodes (Sec. 2.2),
 * on a 2:1-balanced forest of quad/oct-trees of axis-aligned boxes (Sec. 3.1), with Rusanov
 * fluxes (Sec. 2.2), mortars on hanging faces and conservative L2 solution transfer on
 * refinement/coarsening (Sec. 3.3), and explicit SSP-RK3 time stepping with one uniform dt
 * (Sec. 3.1: no subcycling).
 *
 * Conventions shared by every call:
 *  - Every call returns a dg_status; DG_OK is 0.  No call throws or aborts; on failure
 *    dg_last_error(mesh) returns a human-readable detail string owned by the mesh.
 *  - Coordinates: a 2D mesh is the vertical x-z plane (axis 0 = x, axis 1 = z); a 3D mesh
 *    is x, y, z.  The last axis is vertical; gravity acts along -z.
 *  - Prognostic variables, in order: rho', U_0 .. U_{d-1} (momentum), Theta' (= (rho theta)').
 *    nv = d + 2.
 *  - State layout ("SoA"): q[v][e][n], v < nv, e < dg_num_elements(), n < (N+1)^d with node
 *    n = i_0 + (N+1) i_1 + (N+1)^2 i_2 (axis 0 fastest), elements in the current leaf order
 *    (roots lexicographic with x fastest, Morton order inside each root).  The element type
 *    is double for DG_FP64 and float for DG_FP32_PERT.
 *  - Device pointers passed in are caller-owned and must hold the full state; host pointers
 *    likewise.  The library owns every buffer it allocates and frees it in dg_mesh_destroy.
 *  - Calls on one mesh are not thread-safe; distinct meshes may be used from distinct threads.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,          /* invalid argument (null pointer, size, range, layout) */
  DG_ERR_CUDA = 2,         /* a CUDA runtime call failed; detail in dg_last_error */
  DG_ERR_OOM = 3,          /* device or host allocation failed */
  DG_ERR_STATE = 4,        /* non-finite value detected in the state, inconsistent tables,
                              or a mesh left unusable by a failed regrid (see dg_adapt) */
  DG_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
  DG_ERR_UNSUPPORTED = 6   /* combination not compiled in (dimension, degree, precision) */
} dg_status;

enum { DG_FP64 = 0, DG_FP32_PERT = 1 };   /* dg_mesh_desc.precision */
enum { DG_HOST = 0, DG_DEVICE = 1 };      /* where a state pointer lives */
/* layout_flags of dg_set_state / dg_get_state: the library's state layout q[v][e][n] (planes of
 * one variable), or the caller's element-major q[e][v][n] (each element's variables together),
 * converted on the device */
enum { DG_LAYOUT_PLANES = 0, DG_LAYOUT_ELEMENTS = 1 };
enum { DG_CRIT_THETA = 0, DG_CRIT_FLAGS = 1 };  /* dg_adapt_params.criterion */
enum { DG_EQ_EULER = 0, DG_EQ_TRACER = 1 };     /* dg_mesh_desc.equations */
enum { DG_FACE_MORTAR = 0, DG_FACE_INTERP = 1 };  /* dg_mesh_desc.face_mode */

#define DG_NUM_INTEGRALS 5
#define DG_MAX_N 8
#define DG_MAX_LEVEL 12

/* Mesh description.  Defaults for the physics are theta0 = 300 K, p0 = 1e5 Pa, g = 9.81,
 * R = 287, cp = 1004.5 (the paper gives none; Sec. 4.3 gives theta0 = 300 K).  The neutral
 * background ends where its Exner function vanishes, so with g > 0 the box height must stay
 * below cp theta0 / g (30.7 km for the defaults; DG_ERR_ARG otherwise). */
typedef struct {
  int32_t dim;          /* 2 (x-z) or 3 */
  int32_t N;            /* polynomial degree, 1..DG_MAX_N; (N+1)^d LGL nodes per element */
  int32_t base[3];      /* root cells per axis (forest of trees, Sec. 3.1); base[2] unused in 2D */
  double length[3];     /* box extents in metres; the box is [0, length[a]] per axis */
  int32_t max_level;    /* deepest refinement level, 0..DG_MAX_LEVEL */
  int32_t precision;    /* DG_FP64 or DG_FP32_PERT (FP32 state and flux arithmetic; FP64 for
                           the background, the pressure perturbation and the integrals) */
  double theta0, p0, g, R, cp;
  double nu;            /* artificial viscosity (m^2/s), >= 0.  nu > 0 adds the BR1 term
                           div(nu rho grad phi), phi = (u, theta'), to momentum and Theta'
                           (FP64 meshes only; not in the adjoint or in batches) */
  /* Fields below are zero for the Euler equations (the default of a zero-initialised desc). */
  int32_t equations;    /* DG_EQ_EULER, or DG_EQ_TRACER: one passive tracer C with
                           dC/dt + div(C u) = 0 under the prescribed swirling wind of Sec. 4.2,
                           u = sin^2(pi x) sin(2 pi y) g, v = -sin^2(pi y) sin(2 pi x) g,
                           g = cos(pi t / T), coordinates in the box's units (2D, FP64, nu = 0;
                           the state has one plane; upwind face flux; no flux through walls) */
  int32_t face_mode;    /* hanging faces of a tracer mesh: DG_FACE_MORTAR (Sec. 3.3: the coarse
                           side receives the projected mortar fluxes, conservative) or
                           DG_FACE_INTERP (the coarse side solves its own flux against the fine
                           traces evaluated at its nodes: the non-conservative point-to-point
                           interpolation compared in Sec. 4.2); Euler meshes use mortars */
  double wind_period;   /* T of the prescribed wind (tracer meshes), > 0 */
  int32_t periodic[3];  /* 1: the two boundaries of axis a are joined (periodic neighbours
                           replace the walls there); the vertical axis only with g = 0, where
                           the background is uniform */
} dg_mesh_desc;

/* Cosine-bell potential-temperature bubble (Sec. 4.2 Eq. cosine-bell, Sec. 4.3):
 * theta' = amp (1 + cos(pi r)) for r <= 1, r = |(x - center) / radius| per axis, plus an
 * optional random Fourier-feature field sigma sqrt(2/K) sum_k cos(k_k . x + phase_k).
 * The state is set to Theta' = 0, U = 0, rho' = -rho_bar theta' / (theta0 + theta'), which
 * keeps the pressure hydrostatic.  rff_k is [n_rff][3] (host), rff_phase [n_rff] (host). */
typedef struct {
  double center[3];
  double radius[3];
  double amp;
  int32_t n_rff;
  double rff_sigma;
  const double* rff_k;
  const double* rff_phase;
} dg_bubble_desc;

/* Regrid parameters (Sec. 3.2.1: regrid every T steps with a buffer of B cells; Sec. 3.1).
 * criterion DG_CRIT_THETA tags a leaf when max over its nodes of |theta'| > threshold;
 * DG_CRIT_FLAGS uses flags[e] != 0 (host array, one byte per current leaf).  A tagged leaf
 * below max_level is refined together with its B-hop face neighbourhood; refinement is closed
 * under the 2:1 rule; a family of 2^d leaf siblings is coarsened when none of them is tagged,
 * within the buffer or refined, and no face neighbour would end finer than the siblings. */
typedef struct {
  double threshold;
  int32_t buffer;       /* B, face-adjacency hops */
  int32_t max_level;    /* -1: use the mesh's max_level */
  int32_t criterion;
  const uint8_t* flags;
} dg_adapt_params;

typedef struct {
  int64_t elements_before;
  int64_t elements_after;
  int64_t refined;      /* leaves that were split */
  int64_t coarsened;    /* families that were merged */
} dg_adapt_report;

typedef struct dg_mesh dg_mesh;

/* Creates a uniform level-0 forest of base[0] x base[1] (x base[2]) roots with a zero state
 * (the hydrostatic atmosphere at rest).  `stream` is a cudaStream_t (NULL: legacy default
 * stream) used by every later call on this mesh.  On success *out owns all device memory. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, void* stream, dg_mesh** out);

/* Frees everything; NULL is allowed. */
void dg_mesh_destroy(dg_mesh* mesh);

int64_t dg_num_elements(const dg_mesh* mesh);
int64_t dg_num_nodes(const dg_mesh* mesh);       /* elements x (N+1)^d */

/* Leaves in the current order as rows of 5 int32: root index, level, c_0, c_1, c_2 (integer
 * coordinates at the leaf's level; c_2 = 0 in 2D).  `cap` is the number of int32 in `out`. */
dg_status dg_get_leaves(const dg_mesh* mesh, int32_t* out, size_t cap);

/* Face lists in the canonical order (Sec. 3.3 mortars).  Counts are always written.  When the
 * matching array is non-NULL and its capacity (in rows) suffices it is filled:
 *   conforming rows (3 int32): low element, high element, axis;
 *   mortar rows (3 + 4 int32): coarse element, axis, side (0 low, 1 high), fine elements in
 *     Morton order over the tangential axes (unused slots -1);
 *   boundary rows (3 int32): element, axis, side. */
dg_status dg_get_faces(const dg_mesh* mesh, int64_t counts[3], int32_t* conforming, size_t cap_c,
                       int32_t* mortars, size_t cap_m, int32_t* boundary, size_t cap_b);

/* Copies a state in (out): layout_flags = DG_LAYOUT_PLANES for the layout above, or
 * DG_LAYOUT_ELEMENTS for q[e][v][n] (the permutation runs on the device, through the mesh's
 * stage buffer for host pointers); where = DG_HOST or DG_DEVICE.  Synchronous.  Any other flag
 * is DG_ERR_ARG. */
dg_status dg_set_state(dg_mesh* mesh, const void* q, int layout_flags, int where);
dg_status dg_get_state(dg_mesh* mesh, void* q, int layout_flags, int where);
/* Asynchronous forms for pipelines that must not wait on the host.  dg_set_state_async and
 * dg_get_state_async copy the state in or out on `stream` (NULL: the mesh stream) after the work
 * already queued on the mesh stream, with no host wait; host buffers should be pinned, must stay
 * untouched until the copy is done (synchronise the stream), and later mesh work must be ordered
 * after a copy on another stream by the caller.  dg_integrals_async computes the integrals of
 * dg_integrals on `stream` and writes 6 doubles to `out` (host pinned or device memory): mass,
 * total energy, kinetic energy, volume, perturbation mass, and 1.0 if a non-finite value was seen
 * in the state (0.0 otherwise); the values are those dg_integrals returns, bit for bit.  The first
 * call after a regrid first takes the background sums synchronously.  Integrals on one mesh share
 * one scratch buffer: calls that overlap on the GPU race.  Euler meshes, unpartitioned. */
dg_status dg_set_state_async(dg_mesh* mesh, const void* q, int where, void* stream);
dg_status dg_get_state_async(dg_mesh* mesh, void* q, int where, void* stream);
dg_status dg_integrals_async(dg_mesh* mesh, double* out, void* stream);

/* Copies the pressure perturbation P' = P(Theta_bar + Theta') - P(Theta_bar) of the current state
 * (Sec. 2.1, perturbation form; one plane of E (N+1)^dim values in the state precision) into
 * out (DG_HOST or DG_DEVICE, caller-owned, at least dg_num_nodes() values).  It is the plane the
 * stage kernels read: the one the last stage produced, or, after dg_set_state or a regrid, the
 * one evaluated from the state.  Synchronous.  DG_ERR_UNSUPPORTED for tracer meshes. */
dg_status dg_get_pprime(dg_mesh* mesh, void* out, int where);

/* Evaluates the initial condition analytically at the current nodes (FP64 on the device). */
dg_status dg_set_bubble(dg_mesh* mesh, const dg_bubble_desc* bubble);

/* The same analytic theta' as dg_set_bubble, written to the caller's device array
 * theta[elements x (N+1)^d] (FP64) instead of setting the state. */
dg_status dg_bubble_theta(dg_mesh* mesh, const dg_bubble_desc* bubble, double* theta);

/* dq/dt of the strong-form dGSEM (Sec. 2.2) for the caller's device state q (same layout and
 * type as the mesh state), written to the caller's device buffer dqdt.  Pure: the mesh state is
 * untouched.  Asynchronous on `stream` (NULL: the mesh stream). */
dg_status dg_rhs(dg_mesh* mesh, const void* q, void* dqdt, void* stream);

/* nsteps SSP-RK3 steps of size dt on the mesh state (Shu-Osher form), asynchronous on
 * `stream` (NULL: the mesh stream).  Three fused stage launches per step. */
dg_status dg_step(dg_mesh* mesh, double dt, int32_t nsteps, void* stream);

/* One regrid pass with conservative transfer of the state (Sec. 3.3).  Synchronous: the
 * criterion is evaluated on the device, the tree work runs on the host, the transfer on the
 * device.  Element order and count change; state pointers obtained earlier stay valid only as
 * copies.  A pass that refines and coarsens nothing leaves the mesh, its state and its tables as
 * they are (no transfer, no table rebuild).  `report` may be NULL.  Errors: a failure while the
 * new tree and its tables are built
 * and checked leaves the mesh as it was; a failure after the new tree is committed (an
 * allocation or copy of the new tables) leaves the mesh unusable, and every later call on it
 * returns DG_ERR_STATE. */
dg_status dg_adapt(dg_mesh* mesh, const dg_adapt_params* params, dg_adapt_report* report);

/* Per-element refinement indicator max_n |theta'| (FP64), written to host `out` (E doubles). */
dg_status dg_indicator(dg_mesh* mesh, double* out, size_t cap);

/* Model time of the mesh state; dg_step advances it by nsteps x dt.  A tracer mesh evaluates its
 * wind at the SSP-RK3 stage times t, t + dt, t + dt/2, and dg_rhs at t.  Euler meshes carry the
 * time along unused.  dg_get_time returns 0 for a NULL mesh. */
dg_status dg_set_time(dg_mesh* mesh, double t);
double dg_get_time(const dg_mesh* mesh);

/* Isentropic vortex of Sec. 4.1, nondimensional: free stream rho = theta = p = 1 plus the
 * vortex of strength beta centred at center (box coordinates), carried by the stream
 * (u_inf[0], u_inf[1]) and set at time t (centre moved by u_inf t, nearest image on periodic
 * axes):  T = 1 - (gamma-1) beta^2 / (8 gamma pi^2) e^(1-r^2), rho = T^(1/(gamma-1)), theta = 1,
 * (u, v) = u_inf + beta/(2 pi) e^((1-r^2)/2) (-(y - y_c), x - x_c).  Requires a 2D Euler mesh
 * with p0 = R = theta0 = 1 and g = 0 (DG_ERR_ARG otherwise). */
typedef struct {
  double center[2];
  double beta;
  double u_inf[2];
  double t;
} dg_vortex_desc;
dg_status dg_set_vortex(dg_mesh* mesh, const dg_vortex_desc* vortex);

/* Tracer meshes reuse the calls above: dg_set_bubble sets C = amp (1 + cos(pi r)) (the bell of
 * Sec. 4.2 with amp = h_max / 2; the random-field terms must be absent), dg_indicator and the
 * DG_CRIT_THETA criterion of dg_adapt use max |C| per element, dg_integrals returns
 * {int C, 0, 0, volume, int C}; dg_primitives, the adjoint and batches reject them. */

/* Primitive diagnostics of the current state in FP64 (the fields reported in Sec. 4.3): device
 * `out` receives dim + 1 planes of E * (N+1)^dim doubles in the state's [element][node] order,
 * planes 0 .. dim-1 the velocity components U_a / rho, plane dim the potential temperature
 * perturbation theta' = (Theta_bar + Theta') / (rho_bar + rho') - theta0.  `cap` counts doubles;
 * DG_ERR_ARG if it is too small.  The caller owns `out`; asynchronous on `stream` (NULL: the
 * mesh's stream). */
dg_status dg_primitives(dg_mesh* mesh, double* out, size_t cap, void* stream);

/* Domain integrals with weights w_i w_j (w_k) |J|, accumulated in FP64 with compensated
 * (Neumaier) sums and a fixed reduction order: out = {mass, total energy
 * (p cv/R + |U|^2/(2 rho) + rho g z), kinetic energy, volume, perturbation mass int rho'}.
 * The background parts (int rho_bar, int (p_bar cv/R + rho_bar g z), volume) are summed once
 * per mesh topology and added to the state parts with their rounding errors.
 * Synchronous; DG_ERR_STATE if a non-finite value was met (out is still written). */
dg_status dg_integrals(dg_mesh* mesh, double out[DG_NUM_INTEGRALS]);

/* ---- Adjoint (FP64 meshes; DG_ERR_UNSUPPORTED otherwise).  Hand-written discrete
 * vector-Jacobian products of the operator above, for sensitivities of forecast diagnostics to
 * the initial theta' field.  All pointers are caller-owned device buffers in the state layout;
 * asynchronous on `stream` (NULL: the mesh stream).  Non-smooth parts use the derivative of the
 * active branch: max(s-, s+) of the Rusanov speed gives its gradient to the low side on ties,
 * and |u| has derivative sign(u) with sign(0) = 0. */

/* out = J(q)^T lam, J = d dg_rhs(q) / dq. */
dg_status dg_rhs_vjp(dg_mesh* mesh, const void* q, const void* lam, void* out, void* stream);

/* nsteps SSP-RK3 steps from the caller's state q_in to q_out (any precision; may alias), using
 * the mesh's workspace; the mesh state is untouched. */
dg_status dg_step_state(dg_mesh* mesh, const void* q_in, void* q_out, double dt, int32_t nsteps,
                        void* stream);

/* lam_in = (d step(q_in) / d q_in)^T lam_out for one SSP-RK3 step of size dt; the stage states
 * are recomputed from q_in.  lam_in must not alias lam_out. */
dg_status dg_step_vjp(dg_mesh* mesh, const void* q_in, double dt, const void* lam_out,
                      void* lam_in, void* stream);

/* One SSP-RK3 step from q_in (NV planes, device, FP64) to q_out that also keeps the step's three
 * stage inputs q, q1, q2 in `record`: a caller-owned device buffer of 3 x (NV + 1) x E x
 * (N+1)^dim doubles, each stage input stored as its NV planes followed by its P' plane.
 * dg_step_vjp_record then transposes the step without recomputing it (the checkpointed
 * gradient recomputes each segment once and keeps these records). */
dg_status dg_step_record(dg_mesh* mesh, const void* q_in, void* q_out, void* record, double dt,
                         void* stream);
/* lam_in = (d step / d q_in)^T lam_out for the step held in `record` (see dg_step_record); the
 * same result as dg_step_vjp on that step's q_in.  lam_in must not alias lam_out. */
dg_status dg_step_vjp_record(dg_mesh* mesh, const void* record, double dt, const void* lam_out,
                             void* lam_in, void* stream);

/* Sets the mesh state from a nodal theta' field (elements x (N+1)^d doubles, host or device):
 * Theta' = 0, U = 0, rho' = -rho_bar theta' / (theta0 + theta') (same balance as dg_set_bubble). */
dg_status dg_set_theta(dg_mesh* mesh, const double* theta, int where);

/* lam_theta = (d state(theta) / d theta)^T lam_q for the map of dg_set_theta (device). */
dg_status dg_theta_vjp(dg_mesh* mesh, const double* theta, const void* lam_q, double* lam_theta,
                       void* stream);

/* out = d KE / dq for KE = sum w_i w_j (w_k) |J| |U|^2 / (2 rho) (the kinetic-energy integral of
 * dg_integrals) at the caller's state q (device). */
dg_status dg_ke_grad(dg_mesh* mesh, const void* q, void* out, void* stream);

/* ---- Batched solves: many independent meshes advanced together (the batched instances of the
 * study's benchmark set; Sec. 3.5 names throughput on accelerators as the aim).  The 2D members
 * run through ONE persistent launch per SSP-RK3 stage: a device array of work items -- first
 * every member's mortar groups (Sec. 3.3), then tiles of elements of every member, whatever its
 * degree and precision -- taken in order from an atomic counter by a grid of 128-thread CTAs
 * sized to what stays resident.  A stage item waits, thread 0 with an iteration limit of about a
 * second, until its member's mortar items are done; if the limit ever runs out the kernel
 * records it and dg_batch_sync returns DG_ERR_TIMEOUT (the states are then not valid).  3D
 * members are grouped by (precision, N): one stage launch per group over all of its members'
 * elements after the members' mortar launches.  A step is captured once into a CUDA graph and
 * replayed.  The members keep their state in their own buffers (dg_get_state etc. work as
 * usual); a member must not be regridded while in a batch (DG_ERR_STATE).  Members may have
 * different sizes, degrees and precisions.  A member advanced in the batch gets the bits that
 * dg_step gives it with the same stage layout (an FP32 2D member set to layout 5 is switched to
 * layout 2 by dg_batch_create: the persistent launch has layout 5 for FP64 members only). */
typedef struct dg_batch dg_batch;

/* `meshes`: `count` distinct meshes (not owned). */
dg_status dg_batch_create(dg_mesh* const* meshes, int32_t count, dg_batch** out);
void dg_batch_destroy(dg_batch* batch);
/* Per-member time step (count doubles, host). */
dg_status dg_batch_set_dt(dg_batch* batch, const double* dt);
/* nsteps steps of every member, asynchronous on the batch's own stream, ordered after work
 * already queued on each member's stream and before later work there.  use_graph != 0 replays a
 * captured step graph; 0 launches directly (same kernels, same results). */
dg_status dg_batch_run(dg_batch* batch, int32_t nsteps, int32_t use_graph);
/* Waits for the batch's stream; DG_ERR_TIMEOUT if a wait inside the persistent launch ran out. */
dg_status dg_batch_sync(dg_batch* batch);
/* Autotuner, timed on the members themselves with stage-1 launches (reps each; they read q^n and
 * write only scratch buffers, so the states are untouched).  For the persistent launch of the 2D
 * members it chooses, greedily and groups with the most work first: the register budget (the
 * kernel compiled for 2 or for 4 resident CTAs per SM), per (precision, N) group the element
 * tile -- node layout, (N+1)^2 threads per element and 128 / (N+1)^2 elements per CTA pass,
 * column layout, N+1 threads per element and 128 / (N+1) elements per pass, or (FP64 groups)
 * the column layout that reads the Rusanov fluxes of conforming and wall faces from face work
 * items of the same launch -- and the tiles per work item (1, 2, 4 or 8).  For 3D groups it
 * keeps the faster of the two grouped layouts.  The layout choice is also applied to each
 * member's own launches.  `layouts` (count int32, may be NULL) receives the chosen layout per
 * member (1 node, 2 column or 5 column with face fluxes, see DG_OPT_STAGE_KERNEL). */
dg_status dg_batch_autotune(dg_batch* batch, int32_t reps, int32_t* layouts);
/* The persistent launch's shapes: out[0] resident CTAs per SM its register budget is compiled
 * for, out[1] element tiles per stage item, out[2] grid (CTAs), out[3] work items per stage,
 * out[4] dynamic shared memory per CTA in bytes; all zero without 2D members. */
dg_status dg_batch_shape(dg_batch* batch, int64_t out[5]);
const char* dg_batch_last_error(const dg_batch* batch);

/* Tuning options.  DG_OPT_STAGE_KERNEL selects the fused stage kernel's thread layout:
 * 0 = one thread per vertical node column, 1 = one thread per node, 2 = one thread per column
 * with all operands staged into shared memory by asynchronous copies, 3 = as 2 with two
 * threads per column, 4 = one pass per axis with two threads per node line, fluxes kept in
 * registers (3 and 4: 3D with odd N; other shapes run layout 2), 5 = the Rusanov flux of every
 * conforming and wall face computed once per face by a face kernel before the stage kernel,
 * whose volume term runs as a column pass and one line pass per horizontal axis, each line
 * thread lifting the two faces at its ends (a partitioned mesh runs layout 2 instead).
 * Default: 4 for FP32 3D meshes, 5 for FP64 Euler meshes, 2 otherwise.  All compute the same operator; the option exists for tuning
 * and cross-checking. */
enum { DG_OPT_STAGE_KERNEL = 1, DG_OPT_FAIL_NEXT_ADAPT = 2 };
/* DG_OPT_FAIL_NEXT_ADAPT is a host-side failure injection for tests of the regrid's error path
 * (no device fault is involved): value 1 makes the next dg_adapt fail where it checks the new
 * tables, before anything of the mesh changes, so the mesh stays usable; value 2 makes it fail
 * after it has committed the new tree, as a failed allocation there would.  A mesh in the
 * second state is unusable: every later call on it returns DG_ERR_STATE (dg_last_error says
 * why) and only dg_mesh_destroy remains.  The flag is cleared by the dg_adapt it affects. */
dg_status dg_set_option(dg_mesh* mesh, int32_t option, int64_t value);

/* Kernel timing: when enabled, the fused stage launches of dg_step are bracketed by CUDA
 * events on the mesh stream; dg_stage_timing returns the summed milliseconds and launch count
 * since the last reset (synchronises the stream).  Untimed, a stage launch of layouts 2, 4 and 5
 * may begin while the kernel before it finishes (programmatic dependent launch); timed, it
 * starts after it, so that the events bracket the stage kernel alone (in layout 5, the face
 * kernel and the stage kernel). */
dg_status dg_enable_timing(dg_mesh* mesh, int32_t enable);
dg_status dg_stage_timing(dg_mesh* mesh, double* total_ms, int64_t* launches, int32_t reset);

/* Allocation-free variant of dg_integrals.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code running while a stream is
 * captured into a CUDA graph (cudaMalloc cannot be captured), hosts whose device memory is
 * owned by an external pool, or real-time loops that must stay out of the allocator.  It needs
 * no dg_mesh: everything comes from the caller, and nothing is allocated (no cudaMalloc,
 * cudaFree or allocating library call).
 *   desc          the mesh description (dim, N, base, length, precision, constants);
 *   elem          device array [num_elements][4] int32: level, c0, c1, c2 of every leaf, in the
 *                 state's element order (columns 1..4 of dg_get_leaves rows);
 *   q             device state in the dg_set_state layout and the desc precision;
 *   out           device array of DG_NUM_INTEGRALS + 1 doubles: the five integrals of
 *                 dg_integrals, then 1.0 if a non-finite value was met, else 0.0.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream): synchronise before
 * reading `out`.  The reduction scratch is a fixed file-scope device array (about 160 KB, held
 * by every GPU that loads the library until the process exits); states above 67,108,864 nodes
 * (elements x (N+1)^d) are rejected with DG_ERR_ARG.  All calls share that array and it keeps
 * the last call's contents (each call rewrites what it reads); calls that overlap on the GPU
 * (other streams, unordered host threads) race.  The first call on each device looks up the
 * array's device address with that device current; make that first call before any stream
 * capture begins. */
dg_status dg_integrals_noalloc(const dg_mesh_desc* desc, const int32_t* elem, int64_t num_elements,
                               const void* q, double* out, void* stream);

/* ---- Host-only forest (no CUDA call): the same tree code dg_adapt runs, exposed so the
 * integer work (leaf order, 2:1 balance, face and mortar lists, transfer map) can be checked
 * on machines without a GPU.  Sec. 3.1 (forest of trees, active leaves), Sec. 3.2.1 (T, B),
 * Sec. 4.3 (2:1 balance). */
typedef struct dg_forest dg_forest;

/* Uniform level-0 forest of base[0] x base[1] (x base[2]) roots. */
dg_status dg_forest_create(int32_t dim, const int32_t base[3], int32_t max_level, dg_forest** out);
void dg_forest_destroy(dg_forest* forest);
int64_t dg_forest_size(const dg_forest* forest);
/* As dg_forest_create with periodic axes (periodic[a] != 0 joins the boundaries of axis a). */
dg_status dg_forest_create_periodic(int32_t dim, const int32_t base[3], int32_t max_level,
                                    const int32_t periodic[3], dg_forest** out);
/* Leaves as in dg_get_leaves. */
dg_status dg_forest_leaves(const dg_forest* forest, int32_t* out, size_t cap);
/* Face lists as in dg_get_faces. */
dg_status dg_forest_faces(const dg_forest* forest, int64_t counts[3], int32_t* conforming,
                          size_t cap_c, int32_t* mortars, size_t cap_m, int32_t* boundary,
                          size_t cap_b);
/* One regrid pass with the rules of dg_adapt_params on explicit flags (one byte per leaf).
 * When `transfer` is non-NULL and cap >= 9 x (new leaf count) it receives one row of 9 int32
 * per new leaf: kind (0 keep, 1 child, 2 parent), then keep: old leaf; child: parent, child
 * index; parent: the 2^d old children in child-index order (unused slots -1).  Returns the
 * new leaf count through *new_size. */
dg_status dg_forest_regrid(dg_forest* forest, const uint8_t* flags, int32_t buffer,
                           int32_t max_level, int32_t* transfer, size_t cap, int64_t* new_size);

/* Space-filling-curve partition of the leaf order into nparts contiguous ranges (element counts
 * differing by at most one): starts[p] .. starts[p+1]-1 belong to part p; starts holds
 * nparts + 1 entries.  Sec. 3.1 names SFC partitioning as the scalable alternative to METIS. */
dg_status dg_forest_partition(const dg_forest* forest, int32_t nparts, int64_t* starts);
/* Faces of part `part` (of the partition above) whose other side lies in another part, as rows
 * of 5 int32: local element, axis, side, remote element, remote part; a coarse face gives one row
 * per fine neighbour.  *count receives the row count; rows (capacity `cap` rows) may be NULL. */
dg_status dg_forest_halo(const dg_forest* forest, int32_t nparts, int32_t part, int32_t* rows,
                         size_t cap, int64_t* count);

/* ---- Sharded meshes (Sec. 3.1: partitioning along the space-filling curve).  Every part keeps
 * the whole (replicated) tree and full-size state buffers but computes only its own contiguous
 * range of the leaf order, the SFC partition of dg_forest_partition.  Before each stage the
 * traces of the faces it shares with other parts -- conforming faces and both sides of mortars,
 * the rows of dg_forest_halo -- are exchanged: dg_halo_pack gathers, from a state and its P'
 * plane, the traces other parts need, grouped by destination part in increasing order;
 * dg_halo_unpack scatters the traces received from other parts, grouped by source part in
 * increasing order, into the face nodes of the remote elements in the caller's state.  The
 * transport between parts (NCCL send/recv, host copies, ...) is the caller's.  A slot is one
 * face trace: (NV + 1) planes x (N+1)^(d-1) face nodes of the state's type, the state planes
 * first, then P'.  Each part also computes every mortar group that touches one of its
 * elements, from the traces it owns or received, so both sides of a hanging face see the same
 * fluxes.  A partitioned mesh evaluates dg_rhs (owned elements of dqdt) and steps with dg_stage;
 * dg_step, dg_adapt, dg_integrals, the adjoint and batches need the whole mesh (clear the
 * partition with nparts = 1).  Inviscid Euler meshes only. */
/* Restricts the mesh's stage launches to SFC part `part` of `nparts` (1 <= nparts <= elements;
 * nparts = 1 clears the partition) and builds its halo lists. */
dg_status dg_set_partition(dg_mesh* mesh, int32_t nparts, int32_t part);
/* range[0] .. range[1]-1: the owned elements; send_slots[q] / recv_slots[q] (nparts entries
 * each, may be NULL): slots sent to / received from part q; *slot_values (may be NULL): values
 * per slot.  Unpartitioned: the whole mesh and no slots. */
dg_status dg_get_partition(const dg_mesh* mesh, int64_t range[2], int64_t* send_slots,
                           int64_t* recv_slots, int64_t* slot_values);
/* Gathers the send slots of device state q (full-size layout) and its device P' plane pp (NULL:
 * that plane is sent as zeros) into the device buffer sendbuf, asynchronously on `stream`. */
dg_status dg_halo_pack(dg_mesh* mesh, const void* q, const void* pp, void* sendbuf, void* stream);
/* Scatters the receive slots of device buffer recvbuf into device state q and P' plane pp (NULL:
 * P' not written; dg_rhs recomputes P' from the state), asynchronously on `stream`. */
dg_status dg_halo_unpack(dg_mesh* mesh, const void* recvbuf, void* q, void* pp, void* stream);
/* Device pointers of stage buffer `index` (0 = q^n, 1 and 2 the inputs of stages 2 and 3) and
 * of its P' plane.  Index 0 first brings the P' plane of q^n up to date (on the mesh stream). */
dg_status dg_stage_buffer(dg_mesh* mesh, int32_t index, void** q, void** pp);
/* Stage `stage` (0, 1, 2) of one SSP-RK3 step in Shu-Osher form on the mesh's buffers: reads
 * stage buffer `stage` and q^n, writes the next buffer (stage 2 writes q^n and advances the
 * time).  Three calls make one dg_step; a partitioned mesh exchanges the halo of stage buffer
 * `stage` before each call.  Asynchronous on `stream` (NULL: the mesh stream). */
dg_status dg_stage(dg_mesh* mesh, int32_t stage, double dt, void* stream);

/* ---- Cubed-sphere solution transfer (Sec. 3.4, spherical geometry;
 * App. B).  The sphere of radius r is six equiangular gnomonic tiles laid side by side in one
 * 2D forest of 6n x n roots (tile t = root column / n; dg_forest_* give the leaves and the
 * regrid map); every element is an isoparametric quadrilateral of degree N.  The layout's 2:1
 * closure acts across its seams, not the sphere's edges; the transfer needs no neighbours.  All
 * arrays are device memory and FP64; fields are [nv][E][(N+1)^2] as the mesh states. */
/* Per element: nodal weights W[e][n] = w_i w_j J, J = |x_xi x x_eta| of the degree-N
 * interpolated surface (the tangent vectors by the collocation derivative), and area[e], the
 * spherical excess r^2 (A + B + C - pi) of the two spherical triangles of the element's corners.
 * leaves: [E][5] rows of dg_forest_leaves (device copy).  Asynchronous on `stream`. */
dg_status dg_sphere_geometry(int32_t N, int32_t n, double radius, const int32_t* leaves, int64_t E,
                             double* W, double* area, void* stream);
/* Fields q_old (E_old elements) to q_new (E_new) after a regrid whose map `tmap` (host, [E_new][9]
 * rows of dg_forest_regrid) leads from the old to the new leaves: kept elements are copied; the
 * four children of a refined parent take the reference interpolation and then, per field, one
 * factor uniform over the four that makes sum W q equal the parent's; a coarsened parent takes
 * the reference restriction of its children weighted by their areas (4 V_c / sum V) and the same
 * integral-matching factor (applied when |I_new| > 1e-8 sum W |q|, else 1).  W and area from
 * dg_sphere_geometry of the old and new leaves.  1 <= nv <= 8.  DG_ERR_ARG for a map row out of
 * range or a family whose four children are not consecutive.  Synchronous. */
dg_status dg_sphere_transfer(int32_t N, int32_t n, int32_t nv, const int32_t* tmap, int64_t E_new,
                             const double* W_old, const double* area_old, const double* q_old,
                             int64_t E_old, const double* W_new, double* q_new, void* stream);

/* Measurement utility (the paper has no counterpart): the rate of independent fused
 * multiply-adds the current device sustains in FP64 (precision DG_FP64) or FP32
 * (DG_FP32_PERT), in FLOP/s counting 2 per multiply-add.  8 chains per thread, 8 CTAs of 256
 * threads per SM, timed with CUDA events on `stream` (NULL: legacy default stream) after one
 * warm-up launch; synchronous; allocates and frees a small device buffer.  It is the measured
 * peak against which the FP64 stage kernel's pipe-bound roofline is reported. */
dg_status dg_probe_fma_rate(int32_t precision, double* flop_per_s, void* stream);

/* Check utility: the FP64 reciprocal and square root the flux kernels use, applied to the n
 * device values x (positive, normal) into the device arrays rcp and sqrt_out, asynchronously on
 * `stream`.  Each is within about one ulp of the exact value. */
dg_status dg_probe_recip_sqrt(int64_t n, const double* x, double* rcp, double* sqrt_out, void* stream);

/* Detail of the last error on this mesh (never NULL). */
const char* dg_last_error(const dg_mesh* mesh);

/* Library version string. */
const char* dg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
