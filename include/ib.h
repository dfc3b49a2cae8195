/*
 * ib.h - C ABI of the GB300 IB-FE-IPCS library.
 *
 * One object, ib_grid, holds one immersed-boundary flow problem resident on one
 * GPU: the locally refined, domain-reduced Cartesian grid of P1 Kuhn tetrahedra,
 * the Lagrangian boundary points, the fields and every Krylov workspace.  The
 * calls follow the paper's statement of the problem: a box domain discretised
 * by a box mesh whose vertices form a uniform Cartesian grid (Sec. 3.1), refined
 * near the immersed boundary (Sec. 3.2) and reduced to the vessel and a band
 * around it (Sec. 4.3); Lagrangian points X_i with area elements dS_i and
 * prescribed velocities U_B (Sec. 2.3, Eq. 3, Sec. 2.5); inflow/outflow ports
 * (Sec. 3.1); kinematic viscosity nu, density rho and time step dt.
 *
 * Conventions
 *   - All functions are extern "C", never throw, and return an ib_status.
 *     ib_last_error() gives a one-line text for the last failure on a handle.
 *   - Host arrays are row-major, C order, float64 unless stated.  Coarse-cell
 *     arrays are [n[2]][n[1]][n[0]] (x fastest).
 *   - Node fields are returned in the canonical node order: every distinct
 *     vertex of an active leaf cell (hanging nodes included), sorted by its
 *     finest-level integer coordinates (z, then y, then x).
 *   - Device memory comes from desc->dev_alloc / dev_free when given (for
 *     example a caching allocator), else from cudaMalloc / cudaFree.  The
 *     library owns everything it allocates and frees it in ib_grid_destroy.
 *   - Work is enqueued on desc->stream (a cudaStream_t, NULL = legacy default
 *     stream).  A handle is not thread-safe: one host thread and one stream per
 *     handle.  Calls that return fields synchronise that stream.
 *   - Errors: IB_EINVAL for bad arguments or inputs the method cannot accept,
 *     IB_ESTATE when ib_set_boundary has not succeeded yet, IB_ENOMEM when an
 *     allocation fails, IB_ENOCONV / IB_EBREAKDOWN when a Krylov solve of a
 *     step fails (the state before that step is kept: steps are committed only
 *     when every solve converged), IB_ECUDA for a CUDA runtime error.
 */
#ifndef IB_H
#define IB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ib_grid ib_grid;   /* opaque: one problem */
typedef struct ib_batch ib_batch; /* opaque: several deferred problems stepped together */

typedef enum {
  IB_OK = 0,
  IB_EINVAL = 1,
  IB_ENOMEM = 2,
  IB_ESTATE = 3,
  IB_ENOCONV = 4,
  IB_EBREAKDOWN = 5,
  IB_ECUDA = 6,
  IB_ETIMEOUT = 7
} ib_status;

enum { IB_INLET_VELOCITY = 0, IB_OUTLET_ZERO_P = 1, IB_INLET_PRESSURE = 2 };
enum { IB_PARABOLIC = 0 };
enum { IB_FP64 = 0, IB_MIXED = 1 };
enum { IB_PC_MULTIGRID = 0, IB_PC_JACOBI = 1 };
enum { IB_VISCOUS_GRAD = 0, IB_VISCOUS_SYM = 1 };

#define IB_MAX_PORTS 8
#define IB_TUNE_N 5
#define IB_TUNE_POISSON_KERNEL 0
#define IB_TUNE_STREAM_CHUNK 1
#define IB_TUNE_MG_SMALL 2
#define IB_TUNE_MG_SWEEPS 3
#define IB_TUNE_MG_PERSIST 4
#define IB_TANGENTIAL_FREE 0
#define IB_TANGENTIAL_ZERO 1
#define IB_MAX_HARMONICS 8
#define IB_MAX_LEVEL 3

/*
 * A port is a disc on a face of the box (Sec. 3.1: inlet and outlet circles).
 *   axis, side   face normal axis (0,1,2) and side (0 = low face, 1 = high face)
 *   center       disc centre (its coordinate along `axis` is ignored)
 *   radius       disc radius R; a face node is a port node when
 *                dx*dx + dy*dy <= R*R, evaluated in FP64 without FMA
 *   kind         IB_INLET_VELOCITY: parabolic velocity w(t)(1 - r^2/R^2)
 *                along the inward normal; IB_OUTLET_ZERO_P: Phi = 0, no velocity
 *                condition (do-nothing outlet); IB_INLET_PRESSURE: the pressure
 *                w(t) is imposed (Sec. 3.1 drives its Poiseuille tube this way):
 *                Phi = w(t^{n+1}) - p^n on the port nodes, so p^{n+1} = w(t^{n+1})
 *                there, and no velocity condition (the natural condition
 *                nu du/dn = 0 of the viscous term, as at an outlet)
 *   profile      IB_PARABOLIC, the only inlet profile (any other value: IB_EINVAL)
 *   waveform     w(t) = a0 + sum_{k=1..n_harm} a[k-1] cos(2 pi k t / period)
 *                                      + b[k-1] sin(2 pi k t / period)
 * At least one port fixes Phi (an outlet or a pressure inlet); a node on two
 * ports belongs to the first in the array.
 */
typedef struct {
  int32_t axis, side;
  double center[3];
  double radius;
  int32_t kind;
  int32_t profile;
  int32_t n_harm;
  double a0, a[IB_MAX_HARMONICS], b[IB_MAX_HARMONICS], period;
} ib_port;

/*
 * Grid and solver description.
 *   origin, extent, n   box [origin, origin + extent] cut into n[0] x n[1] x n[2]
 *                       coarse cells; every cell is split into the 6 Kuhn
 *                       tetrahedra around its (0,0,0)-(1,1,1) diagonal
 *   max_level           refinement levels near the wall (0 = uniform); a coarse
 *                       cell at level l is cut into 2^l x 2^l x 2^l leaf cells
 *   refine_band         cells within this Chebyshev distance (coarse cells) of a
 *                       cell holding a Lagrangian point get max_level; each
 *                       further band of this width one level less; 2:1 balanced
 *   reduce_band         domain reduction: a coarse cell is active when it is
 *                       inside the vessel or within this distance of a point
 *                       cell; < 0 keeps the whole box
 *   nu, rho, dt         kinematic viscosity, density, time step
 *   precision           IB_FP64: every solve in FP64.  IB_MIXED: FP32 operators
 *                       and preconditioners inside FP64 defect correction for
 *                       the momentum, Poisson, velocity-correction and force
 *                       (A_F, Eq. 22) solves; FP64 IB interpolation and
 *                       spreading; the field solves' right-hand sides and
 *                       outer residuals FP64-accurate (FP64 inputs and
 *                       outputs, stencil sums carried in pairs of FP32
 *                       numbers to about 2^-44 of the terms' magnitudes,
 *                       differences formed exactly), their solutions
 *                       accumulated in FP64
 *   rtol_*              relative residual tolerances of the momentum, Poisson,
 *                       velocity-correction and force solves, relative to
 *                       max(norm of b, norm of the initial residual); 0 selects
 *                       the defaults: 1e-13 on the FP64 path, 1e-10 on the
 *                       mixed path (its FP64 outer loops and force solve)
 *   max_iter            iteration cap per Krylov solve (0 = default)
 *   profile             1: run each step eagerly (host-polled loops instead of
 *                       the captured step graph) and record CUDA events
 *                       around the solvers' kernel launches
 *                       (ib_info.prof_ms / prof_launches); results are
 *                       bitwise those of the graph path
 *   deferred            1: ib_set_boundary builds the grid and a device state
 *                       snapshot only; the problem is advanced by ib_batch_step
 *                       together with other deferred problems
 *   poisson_pc          preconditioner of the pressure-increment CG (Eq. 12):
 *                       IB_PC_MULTIGRID (default; geometric V-cycle over the
 *                       nested Kuhn meshes, falls back to Jacobi when the
 *                       hierarchy cannot be built) or IB_PC_JACOBI
 *   viscous_form        viscous term of the momentum step (Eq. 9):
 *                       IB_VISCOUS_GRAD (default): nu (grad u, grad v), the
 *                       components decouple; IB_VISCOUS_SYM: the symmetric
 *                       form 2 nu (eps(u), eps(v)) of Eq. 1, which couples the
 *                       three components, minus the boundary term
 *                       nu ((grad u)^T n, v) on outlet and pressure-inlet faces
 *                       so that those keep the do-nothing condition; the
 *                       momentum BiCGStab then runs on the coupled system (one
 *                       set of scalars for the three components).  The members
 *                       of a batch share one form.
 *   stream              cudaStream_t on which all work is enqueued
 *   dev_alloc/dev_free  optional device allocator (ctx = alloc_ctx); every
 *                       block it returns must start on a 256-byte boundary
 *                       (the streaming kernels use 16-byte vector accesses);
 *                       a misaligned block fails the call with IB_ENOMEM
 *   port_tangential     velocity condition on outlet and pressure-inlet port
 *                       nodes (Sec. 3.1 imposes the pressure there and says
 *                       nothing of the tangential velocity):
 *                       IB_TANGENTIAL_FREE (default): every velocity
 *                       component is free (the natural condition of the
 *                       viscous form); IB_TANGENTIAL_ZERO: the components
 *                       tangential to the port plane are held at zero (the
 *                       normal component carries the flow) and the IB force
 *                       is not spread onto those nodes
 *   tune                launch choices that change speed, not the method (0 =
 *                       the library's default; the package's autotuner picks
 *                       them per workload class); a batch takes its first
 *                       member's:
 *     [IB_TUNE_POISSON_KERNEL]  FP32 Poisson stencil: 1 staged asynchronously,
 *                               one CTA per chunk of bricks (default), 2
 *                               register-pipelined, 3 staged and persistent
 *                               (a whole number of CTAs per SM walk a
 *                               schedule of chunks written at set-up; the
 *                               same bits as 1)
 *     [IB_TUNE_STREAM_CHUNK]    bricks per CTA of the streaming Krylov
 *                               kernels: 4 or 8 (default)
 *     [IB_TUNE_MG_SMALL]        multigrid levels with at most this many nodes
 *                               (64 .. 1048576, default 8192) run in one CTA
 *                               per problem
 *     [IB_TUNE_MG_SWEEPS]       damped-Jacobi sweeps before and after the
 *                               coarse correction on the composite level and
 *                               G0: 1 .. 4 (default 2); the V-cycle stays a
 *                               symmetric preconditioner, so the solution is
 *                               the same to the solver tolerance
 *     [IB_TUNE_MG_PERSIST]      the V-cycle below the composite grid: 1 one
 *                               launch per level step (default), 2 one
 *                               cooperative launch with grid barriers (the
 *                               same bits as 1; a barrier wait that runs out
 *                               fails the step with IB_ETIMEOUT)
 *                       Invalid values fail ib_grid_create with IB_EINVAL.
 */
typedef struct {
  double origin[3], extent[3];
  int32_t n[3];
  int32_t max_level, refine_band, reduce_band;
  double nu, rho, dt;
  int32_t precision;
  double rtol_mom, rtol_p, rtol_corr, rtol_ib;
  int32_t max_iter;
  int32_t profile;          /* 1: time solver kernel launches with CUDA events */
  int32_t deferred;         /* 1: keep only the grid and a state snapshot; the
                               problem is stepped inside an ib_batch */
  int32_t poisson_pc;       /* IB_PC_MULTIGRID | IB_PC_JACOBI */
  int32_t viscous_form;     /* IB_VISCOUS_GRAD | IB_VISCOUS_SYM */
  int32_t n_ports;
  ib_port ports[IB_MAX_PORTS];
  void* stream;
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  int32_t tune[IB_TUNE_N];
  int32_t port_tangential;  /* IB_TANGENTIAL_FREE (default) | IB_TANGENTIAL_ZERO */
} ib_grid_desc;

/* Counts, spacing ratio and the last step's solver statistics. */
typedef struct {
  int64_t n_nodes;          /* canonical nodes (hanging included) */
  int64_t n_dof;            /* non-hanging nodes */
  int64_t n_hanging;
  int64_t n_leaf_cells;     /* active leaf cells, all levels */
  int64_t n_leaf_cells_level[IB_MAX_LEVEL + 1];
  int64_t n_active_coarse;
  int64_t n_bricks;         /* 8x8x8-node storage bricks, all levels */
  int64_t n_slots;          /* n_bricks * 512 */
  int64_t n_interface;      /* nodes stored on two levels */
  int64_t n_points;         /* Lagrangian points M */
  int64_t af_nnz;           /* nonzeros of A_F */
  double a_ratio[3];        /* sqrt(mean dS) / h_finest per axis (Sec. 2.5) */
  int64_t step;             /* committed steps */
  double time;
  int32_t iters_mom[3], iters_ib, iters_p, iters_corr[3];
  int32_t outer_mom, outer_p, outer_corr;
  double res_mom, res_ib, res_p, res_corr;   /* final relative residuals */
  int32_t status_mom, status_ib, status_p, status_corr;   /* last step, per solve */
  int64_t device_bytes;     /* device memory held by the handle */
  int64_t n_valid_slots;    /* stored node copies, all levels (hanging included) */
  /* with desc.profile: accumulated device time and launch count per kernel
     class since ib_set_boundary; class = base + {0 operator apply, 1 vector
     update, 2 direction update}, base 0 Poisson, 3 mass, 6 momentum; the
     multigrid V-cycle: 9 composite stencil applies, 10 composite smoothing
     updates, 11 transfers and coarse levels */
  double prof_ms[12];
  int64_t prof_launches[12];
  int64_t kernel_launches;  /* kernels launched by this process's library so far */
  int32_t mg_levels;        /* multigrid levels below the composite grid (0: Jacobi) */
  int32_t mg_coarsest;      /* nodes of the coarsest level (dense solve) */
} ib_info;

/* Field identifiers for ib_fields_get / ib_fields_set. */
enum {
  IB_FIELD_U = 0,           /* velocity, double [n_nodes][3]          (get/set) */
  IB_FIELD_P = 1,           /* pressure, double [n_nodes]             (get/set) */
  IB_FIELD_PHI = 2,         /* last pressure increment, double [n_nodes] (get) */
  IB_FIELD_U_TENT = 3,      /* last tentative velocity u~, [n_nodes][3]  (get) */
  IB_FIELD_U_IB = 4,        /* last IB-corrected velocity, [n_nodes][3]  (get) */
  IB_FIELD_F_LAG = 5,       /* last Lagrangian force F, double [M][3]    (get) */
  IB_FIELD_B_F = 6,         /* last right-hand side B_F, double [M][3]   (get) */
  IB_FIELD_NODE_Q = 7,      /* finest integer coordinates, int32 [n_nodes][3] */
  IB_FIELD_NODE_FLAGS = 8,  /* uint8 [n_nodes]: 1 hanging, 2 velocity Dirichlet,
                               4 Phi Dirichlet (outlet or pressure inlet),
                               8 inlet (velocity or pressure), 16 boundary */
  IB_FIELD_ACTIVE = 9,      /* uint8 coarse active mask [n2][n1][n0] */
  IB_FIELD_LEVEL = 10,      /* uint8 coarse level map [n2][n1][n0] */
  IB_FIELD_IB_ORIGIN = 11,  /* int32 [M][3] support origin on the finest grid */
  IB_FIELD_IB_WEIGHTS = 12, /* double [M][64] delta weights (0 where missing) */
  IB_FIELD_IB_FREE = 13     /* uint8 [M][64]: 1 existing free node, 2 existing
                               non-free node, 0 missing */
};

/*
 * ib_grid_create: validate the description and allocate an empty handle.
 * The grid itself is built by ib_set_boundary (it depends on the points).
 * Errors: IB_EINVAL (n <= 0, extent <= 0, max_level outside [0, IB_MAX_LEVEL],
 * bands < 1 where used, nu/dt/rho <= 0, ports not on a box face, more than
 * IB_MAX_PORTS ports, no outlet port), IB_ENOMEM.
 */
ib_status ib_grid_create(const ib_grid_desc* desc, ib_grid** out);

/*
 * ib_set_boundary: give the immersed boundary and build everything that depends
 * on it (Sec. 2.3, Eq. 17-22; Sec. 3.2; Sec. 4.3):
 *   M        number of Lagrangian points (>= 0)
 *   X        host double [M][3], point coordinates inside the box
 *   dS       host double [M], area elements (> 0)
 *   UB       host double [M][3] prescribed velocities, or NULL for a rigid wall
 *   inside   host uint8 [n2][n1][n0], 1 for coarse cells inside the vessel, or
 *            NULL (only allowed when reduce_band < 0)
 * Builds the level map, active cells, node numbering, hanging-node constraints,
 * boundary and port masks, delta weights (Eq. 17-18), the force matrix A_F
 * (Eq. 22) and its solver workspace, then resets u = p = 0 and t = 0.
 * All host inputs are copied.  Errors: IB_EINVAL (a point outside the box, an
 * IB support that touches a hanging node or a coarser level, a non-finite
 * input, no pressure-Dirichlet node), IB_ENOMEM, IB_ECUDA.
 */
ib_status ib_set_boundary(ib_grid* g, int64_t M, const double* X, const double* dS,
                          const double* UB, const uint8_t* inside);

/*
 * ipcs_step: advance nsteps time steps of the combined algorithm (Sec. 2.4):
 * tentative velocity (Eq. 9), IB force solve and correction (Eq. 14, 19-21),
 * pressure-increment Poisson solve (Eq. 12), velocity correction and pressure
 * update.  nsteps = 0 is a no-op.  Synchronises the stream after every step to
 * read its status; on IB_ENOCONV / IB_EBREAKDOWN the state of the last
 * committed step is kept.
 */
ib_status ipcs_step(ib_grid* g, int32_t nsteps);

/*
 * ib_fields_get / ib_fields_set: copy a field out of / into the handle (see the
 * IB_FIELD_* list for types and shapes).  `bytes` must equal the field size.
 * dst/src are device pointers when *_on_device != 0, host pointers otherwise.
 * Setting U or P writes every stored copy and then re-imposes the hanging-node
 * constraint (a hanging node takes the mean of its parents).
 */
ib_status ib_fields_get(ib_grid* g, int32_t field, void* dst, size_t bytes, int32_t dst_on_device);
ib_status ib_fields_set(ib_grid* g, int32_t field, const void* src, size_t bytes, int32_t src_on_device);

/*
 * ib_set_points: move the Lagrangian points of a standalone handle (a moving
 * or deforming wall, the case the IB method exists for: the Eulerian grid does
 * not follow the wall, Sec. 1).  For the following steps the points are at
 *   X        double [M][3], coordinates inside the box
 *   UB       double [M][3] prescribed wall velocities, or NULL for zero
 * (host pointers, or device pointers when on_device = 1; M as given to
 * ib_set_boundary, dS unchanged).  The supports (Eq. 17), delta weights
 * (Eq. 18), the A_F pattern and values (Eq. 22) and the spreading lists
 * (Eq. 19) are rebuilt on the device, every list in sorted order, so the
 * result equals a fresh ib_set_boundary at X except for the refinement and
 * domain reduction, which stay those of the first geometry.  The captured step
 * graph stays valid (list lengths are read on the device) except after the
 * first move or when A_F outgrows its buffer, when the next step captures it
 * again.  Synchronises the handle's stream.
 * Errors: IB_EINVAL (M differs, a point outside the box, a support touching a
 * hanging node or a coarser level: the points must stay inside the finest
 * refined band; a point without a free support node), IB_ESTATE (not ready,
 * or a deferred handle: batches keep their geometry), IB_ENOMEM, IB_ECUDA.
 * After IB_EINVAL the handle keeps stepping with the points it had.
 */
ib_status ib_set_points(ib_grid* g, int64_t M, const double* X, const double* UB, int32_t on_device);

/*
 * ib_wss: wall shear stress at the Lagrangian points from the current velocity
 * (Sec. 2.6): WSS = |t - (t.n) n| with t = 2 mu eps(u) n, mu = rho nu,
 * eps(u) = (grad u + grad u^T) / 2.  The derivatives come from second-order
 * DC-PSE operators (the meshless method Sec. 2.6 cites) over the finest-level
 * nodes within 3.5 e of the point (e the largest finest spacing) on the fluid
 * side ((x_q - X).n < 0), with the point's own value U_B; polynomials of
 * degree 2 are differentiated exactly.
 *   normals   double [M][3] unit outward wall normals at the points
 *   wss       double [M] result
 *   grad      double [M][3][3] d u_i / d x_j, or NULL
 *   on_device 1: the three arrays are device pointers, 0: host pointers
 * Standalone handles; the paper has no such call (it evaluates WSS on the
 * surface of a visualisation mesh), the Lagrangian points stand in for it.
 * Synchronises the handle's stream.  Errors: IB_EINVAL (a point with too few
 * fluid nodes for the nine moment conditions), IB_ESTATE, IB_ENOMEM, IB_ECUDA.
 */
ib_status ib_wss(ib_grid* g, const double* normals, double* wss, double* grad, int32_t on_device);

/* ib_grid_info: counts and the last step's statistics. */
ib_status ib_grid_info(const ib_grid* g, ib_info* out);

/* ib_last_error: text of the last error on g (never NULL; "" if none). */
const char* ib_last_error(const ib_grid* g);

/* ib_grid_destroy: free every resource of g (NULL is a no-op; a handle that a
 * batch still holds is left alone: destroy the batch first). */
void ib_grid_destroy(ib_grid* g);

/*
 * Batches (continuous batching of several problems on one GPU).
 *
 * ib_batch_create: lay out the grids, fields and solver state of n deferred
 *   handles side by side on the device and load each one's state snapshot
 *   (zero for a new problem).  One step of the batch is one captured graph in
 *   which every kernel runs over the concatenated bricks of all members and
 *   every Krylov reduction is segmented per member, so each member's result is
 *   bitwise the same alone and in any mix.  Members must share the precision
 *   and the viscous form; each keeps its own grid, nu, dt, rho, ports and
 *   tolerances of member 0.
 *   Errors: IB_EINVAL (a member not deferred, not ready, repeated, already in
 *   a batch, or of another precision or viscous form), IB_ENOMEM, IB_ECUDA.
 * ib_batch_step: nsteps steps of every member; status[i] (if not NULL, n
 *   entries) receives each member's status of the last step.  A member whose
 *   solves failed keeps its previous state; the call returns the worst status.
 * ib_batch_fields_get / ib_batch_info: as ib_fields_get / ib_grid_info for
 *   member i (ib_fields_get and ib_grid_info on a member handle forward here).
 * ib_batch_destroy: store every member's state back into its snapshot and
 *   release the batch (members can then join another batch).
 */
ib_status ib_batch_create(ib_grid* const* members, int32_t n, ib_batch** out);
ib_status ib_batch_step(ib_batch* b, int32_t nsteps, int32_t* status);
ib_status ib_batch_fields_get(ib_batch* b, int32_t member, int32_t field, void* dst, size_t bytes,
                              int32_t dst_on_device);
ib_status ib_batch_info(const ib_batch* b, int32_t member, ib_info* out);
const char* ib_batch_last_error(const ib_batch* b);
void ib_batch_destroy(ib_batch* b);

/*
 * ib_fields_get_noalloc: ib_fields_get for U, P or Phi of a parked problem (a
 * deferred handle that no batch holds) without any device allocation.  The
 * paper has no counterpart: this is a serving-side call.  ib_fields_get on a
 * parked problem gathers the stored node copies into canonical order in a
 * temporary device buffer; this call gathers into a fixed 8 MiB scratch array
 * of the library's own device memory instead.  It is for callers that cannot
 * allocate device memory at the moment they read a result: a serving loop
 * that has handed its whole device-memory budget to the batch it is running
 * (an allocation would fail or would have to evict a running problem), or a
 * caller whose dev_alloc cannot be entered from the reading thread (an
 * allocator that the stepping thread holds locked).
 *
 *   field          IB_FIELD_U (3 values per node), IB_FIELD_P or IB_FIELD_PHI
 *   dst, bytes     as ib_fields_get; dst_on_device != 0 for a device pointer
 *   limit          components x n_nodes <= 1,048,576 values (8 MiB): larger
 *                  fields fail with IB_EINVAL and a message naming the limit
 *                  (read them with ib_fields_get)
 *   errors         IB_ESTATE for a standalone handle or one that a batch
 *                  holds (read those with ib_fields_get), IB_EINVAL for other
 *                  fields, a wrong byte count, or a current CUDA device other
 *                  than the one current at ib_grid_create (the scratch and
 *                  the snapshot are per device: make the handle's device
 *                  current first), IB_ECUDA for a CUDA error
 *
 * The first call on a device, with that device current, does a one-time setup
 * (it resolves the scratch's device address, which can load the library's
 * device code on that device): make that first call before any stream
 * capture begins in the process.  Nothing in the scratch has to start at
 * zero: each call writes every value it copies out.  The scratch is shared by
 * all handles on a device, so overlapping calls would race on it; the library
 * serialises them with a process-wide lock held until the copy out has
 * completed, and the call synchronises desc->stream before it returns.
 */
ib_status ib_fields_get_noalloc(ib_grid* g, int32_t field, void* dst, size_t bytes, int32_t dst_on_device);

#ifdef __cplusplus
}
#endif
#endif /* IB_H */
