/*
 * grstage.h -- C ABI of the GB300 GRMHD Runge-Kutta stage library (libgrstage.so).
 *
 * One stage of the ideal-GRMHD conservative update of GR-Athena++ (arXiv:2311.04989) on a batch of
 * MeshBlocks with constrained transport in a given 3+1 metric:
 *   Eq. claw (conservation law), Eq. consB_def (conserved variables), Eq. fluxB_def (fluxes),
 *   Eq. EMT_MHD and Eq. hydsrc_def (geometric sources), Sec. 3.2 (vertex-to-cell/face Lagrange
 *   interpolation of the metric), Sec. 3.3 (constrained transport), Sec. 3.4 (PLM / WENOZ
 *   reconstruction of the primitives incl. pressure), Sec. 3.5 and App. A (conservative-to-primitive
 *   inversion with atmosphere and limits).  The Riemann solver is HLLE with the approximate
 *   fast-magnetosonic speeds of Sec. 2.2.
 *
 * Conventions
 *   - All arrays are device pointers owned by the caller; the library never frees them.
 *   - Every variable lives in its own "pool" (structure of arrays).  Block b's data of a pool start at
 *     the element offset given in its gr_block.  Within a block, arrays are ghost-padded with ng
 *     cells on every side and x is the fastest index:
 *       cell arrays      (nz+2g) x (ny+2g) x (nx+2g)        cell i in [-g, n+g-1]
 *       x-face arrays    (nz+2g) x (ny+2g) x (nx+2g+1)      face i at the low side of cell i
 *       y-/z-face arrays likewise with the extra point along y / z
 *       vertex arrays    (nz+2g+1) x (ny+2g+1) x (nx+2g+1) vertex i in [-g, n+g]
 *   - Primitives w = (rho, u~^x, u~^y, u~^z, p); conserved q = (D, S_x, S_y, S_z, tau); B^i is the
 *     densitised face field sqrt(gamma) calB^i.  With a tabulated EOS (Sec. 2.2.1) the primitives are
 *     (rho, u~^i, p, Y_e, T) and the conserved variables (D, S_j, tau, D Y_e): the thermodynamic state
 *     of a point is (rho, p, Y_e), and T is an output (written by con2prim, never read).  Metric components in the order
 *     alpha, beta^x, beta^y, beta^z, gamma_xx, gamma_xy, gamma_xz, gamma_yy, gamma_yz, gamma_zz,
 *     K_xx, K_xy, K_xz, K_yy, K_yz, K_zz.
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream).  Functions that return host values synchronise that stream.
 *   - Return value: GR_OK or a negative gr_error.  Pointwise physics problems are not errors; they go
 *     into the per-cell status bits below.
 */
#ifndef GRSTAGE_H
#define GRSTAGE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GR_ABI_VERSION 3

typedef enum {
  GR_OK = 0,
  GR_EINVAL = -1,       /* bad argument, descriptor, size, or ghost width too small for the stencil */
  GR_ECUDA = -2,        /* a CUDA runtime call failed (message in gr_last_error) */
  GR_ENOMEM = -3,       /* device allocation failed */
  GR_ETIMEOUT = -4,     /* a bounded device wait expired */
  GR_EUNSUPPORTED = -5  /* option combination not built */
} gr_error;

enum { GR_RECON_PLM = 0, GR_RECON_WENOZ = 1, GR_RECON_WENO5 = 2, GR_RECON_PPM = 3 };   /* Sec. 3.4 */
enum { GR_PREC_FP64 = 0, GR_PREC_MIXED = 1 };           /* mixed: FP32 reconstruction/HLLE/EMF */
enum { GR_EMF_UPWIND = 0, GR_EMF_MEAN = 1 };            /* Sec. 3.3 corner electric field */
enum { GR_CEIL_CLAMP = 0, GR_CEIL_ATMOSPHERE = 1 };     /* App. A clamp, or Sec. 3.5 reset */
enum { GR_EOS_IDEAL = 0, GR_EOS_TABLE = 1 };            /* Sec. 2.2.1 */

/* con2prim status bits (per cell, uint8) */
#define GR_ST_ATM_THRESHOLD 0x01  /* rho or D below f_thr rho_atm -> atmosphere (Sec. 3.5, App. A) */
#define GR_ST_FAILED        0x02  /* non-finite input, no bracket or no convergence -> atmosphere */
#define GR_ST_W_CLAMPED     0x04  /* Lorentz factor above W_max: clamped (or atmosphere)  (App. A) */
#define GR_ST_TAU_FLOOR     0x08  /* tau raised to the cold static value (App. A) */
#define GR_ST_BD_LIMIT      0x10  /* B^2/D above M_max: D rescaled (App. A) */
#define GR_ST_EOS_CLAMP     0x20  /* rho, eps/T or Y_e moved into the EOS range, or T raised to T_atm (App. A) */
#define GR_ST_GUESS_REJECTED 0x40 /* a proposed root bracket showed no sign change: full bracket used */

/* Source of a proposed con2prim root bracket (the FP64 solve always verifies it by a sign change):
 * none, an FP32 pre-solve (the bracket narrowed in FP32 to 1e-4 of its upper end, then widened by 4e-6),
 * the learned bracket of a small network (gr_mlp_*), or GR_GUESS_AUTO: the mesh's choice between none and
 * the FP32 pre-solve for the call's precision and EOS, made by gr_autotune by timing the stage with each
 * (none until the mesh is tuned; gr_mesh_get_guess reads it). */
enum { GR_GUESS_NONE = 0, GR_GUESS_FP32 = 1, GR_GUESS_MLP = 2, GR_GUESS_AUTO = 3 };

/* Atmosphere band (gr_params.atm_band) for the mixed path: its atmosphere test compares D' with the
 * threshold times an FP32 sqrt(gamma) (relative error ~1e-7), so a band of 1e-6 classifies the cells at
 * the atmosphere density the same way as an FP64 test with the same band.  The default band is 1e-12. */
#define GR_MIXED_ATM_BAND 1e-6

/* One MeshBlock: n[] interior cells, ng ghosts, cell widths, and element offsets into the pools. */
typedef struct {
  int32_t n[3];
  int32_t ng;
  double dx[3];
  int64_t cell_off;     /* into every cell pool (U, U0, W, Uo, Wo, status) */
  int64_t face_off[3];  /* into the x-, y-, z-face pools (B, B0, Bo) */
  int64_t vert_off;     /* into the 16 vertex metric pools */
} gr_block;

/* The 3+1 metric on vertices (Sec. 3.2).  order: Lagrange interpolation order 2 or 4 (order 4 needs
 * one ghost more than the reconstruction stencil).  k_zero != 0 declares K_ij = 0 (v[10..15] unread).
 * v32 (mixed path only, optional): FP32 copies of the components in the same layout, equal to
 * gr_cast_f32 of v (e.g. made once for a metric that does not change between stages); with v32[0] != NULL
 * every component the stage reads must be given (10, or 16 with K_ij) and the stage converts nothing of
 * the metric.  All NULL: the stage makes its own FP32 copy. */
typedef struct {
  const double* v[16];
  int32_t order;
  int32_t k_zero;
  const float* v32[16];
} gr_metric;

/* Stage state.  Inputs must have their ghost zones filled by the caller (the stage itself exchanges
 * nothing).  U, U0 and B0 are read on the interior only; W and B on the interior and the ghosts.
 * Outputs are written on the interior only: Uo (cells), Bo (all faces of interior cells), Wo, status.
 * Outputs must not alias inputs.
 * FP32 copies (mixed path only; the FP64 path ignores them).  The mixed path reconstructs from FP32
 * copies of W and B; by default it makes them itself at the start of every stage.  W32/B32 (optional)
 * hand it ready copies instead: every element the stage reads (interior and ghosts) must equal
 * gr_cast_f32 of the FP64 value, so the results are those of the default path bitwise.  Wo32/Bo32
 * (optional) ask the stage to write FP32 copies of its outputs Wo/Bo wherever it writes them (the next
 * stage's W32/B32 once their ghosts are filled).  Each group is all or none: W32[0] != NULL needs W32 of
 * every primitive the stage reads (5, or 6 with a table) and B32[0..2]; likewise Wo32 (5 or 6: T has no
 * copy) and Bo32.  They must not alias W32/B32. */
typedef struct {
  const double* U[6];    /* U[5] = D Y_e: tabulated EOS only (NULL otherwise) */
  const double* U0[6];   /* RK register; read only where rk_g0 != 0 */
  const double* B[3];
  const double* B0[3];   /* read only where rk_g0 != 0 */
  const double* W[7];    /* W[5] = Y_e read with a table; W[6] = T never read */
  double* Uo[6];
  double* Bo[3];
  double* Wo[7];         /* Wo[5], Wo[6] = Y_e, T written with a table */
  uint8_t* status;
  const float* W32[6];   /* optional FP32 copies of W[0..5] and B (mixed path) */
  const float* B32[3];
  float* Wo32[6];        /* optional FP32 copies of Wo[0..5] and Bo, written with them (mixed path) */
  float* Bo32[3];
} gr_state;

/* Tabulated EOS (Sec. 2.2.1): log p, log e (e = rho (1 + eps), the total energy density) and c_s^2 on a
 * uniform grid in (log rho, log T, Y_e), natural logarithms; node (ir, iT, iy) of each host array at
 * index (iy * n[1] + iT) * n[0] + ir.  The library interpolates trilinearly in those variables; log p
 * and log e must increase strictly with T along every node column (the temperature is recovered by
 * inverting the interpolant in log T).  Values outside the table are moved to the nearest table
 * value (App. A; status GR_ST_EOS_CLAMP in con2prim). */
typedef struct {
  int32_t n[3];          /* nodes along log rho, log T, Y_e, each >= 2 */
  int32_t pad_;
  double x0[3];          /* first node: log rho_min, log T_min, Y_e,min */
  double dx[3];          /* node spacing, > 0 */
  const double* log_p;   /* host arrays of n[0] n[1] n[2] values, copied by gr_eos_create */
  const double* log_e;
  const double* cs2;
} gr_eos_table;
typedef struct gr_eos gr_eos;

/* Parameters.  size must be sizeof(gr_params).  Defaults from gr_params_default(). */
typedef struct {
  uint32_t size;
  int32_t recon;        /* GR_RECON_* */
  int32_t precision;    /* GR_PREC_* */
  int32_t emf;          /* GR_EMF_* */
  int32_t ceiling;      /* GR_CEIL_* */
  int32_t max_iter;     /* root-find iteration cap */
  int32_t c2p_guess;    /* GR_GUESS_*: bracket proposal for con2prim */
  double gamma_ad;      /* ideal gas p = rho eps (Gamma - 1), Sec. 2.2.1 */
  double rho_atm;       /* f_atm rho_max (Sec. 3.5) */
  double p_atm;         /* p(rho_atm) */
  double f_thr;         /* atmosphere threshold factor */
  double W_max;         /* Lorentz-factor ceiling, sqrt(1 + 20^2) for u~ <= 20 (Sec. 3.5) */
  double M_max;         /* B^2/D ceiling (App. A) */
  double tol;           /* relative bracket tolerance (Sec. 3.5: 1e-10) */
  double weno_eps;      /* WENOZ epsilon */
  double rk_g0, rk_g1, rk_beta;   /* U' = g0 U0 + g1 U + beta dt L(U) (Shu-Osher stage) */
  const float* mlp;     /* device parameter vector of the learned bracket (GR_GUESS_MLP), 16-byte aligned */
  int32_t eos;          /* GR_EOS_*; GR_EOS_TABLE needs `table` on the mesh's device */
  int32_t pad_;
  const gr_eos* table;
  double T_atm;         /* table: atmosphere temperature and temperature floor (App. A) */
  double Ye_atm;        /* table: electron fraction of the atmosphere (a parameter; the paper is silent) */
  double atm_band;      /* rho or D below f_thr rho_atm (1 + atm_band) is atmosphere (Sec. 3.5 resets below
                           f_thr rho_atm).  Default 1e-12: values equal to the threshold up to FP64 rounding
                           are reset, everything above is solved.  The mixed path tests D' against its FP32
                           sqrt(gamma) (relative error ~1e-7), so it classifies atmosphere cells the same way
                           on every input only with a band of ~1e-6; that is its documented tolerance. */
} gr_params;

typedef struct gr_ctx gr_ctx;
typedef struct gr_mesh gr_mesh;

/* Error text of a code; gr_last_error() gives the detail of the last failing call of this thread. */
const char* gr_strerror(int code);
const char* gr_last_error(void);
int gr_abi_version(void);
void gr_params_default(gr_params* p);

/* A context binds one CUDA device.  Returns GR_EINVAL for a bad device index. */
int gr_context_create(gr_ctx** ctx, int device);
int gr_context_destroy(gr_ctx* ctx);

/* A mesh is a batch of blocks resident on the device: the block table, the per-kernel work lists
 * and the workspace for face fluxes and corner fields (owned by the mesh).  Blocks may differ in
 * size.  The block descriptors are copied; the caller may free its array afterwards. */
int gr_mesh_create(gr_ctx* ctx, const gr_block* blocks, int32_t nblocks, int32_t max_ng,
                   gr_mesh** mesh);
int gr_mesh_destroy(gr_mesh* mesh);
/* Bytes of device workspace held by the mesh. */
int64_t gr_mesh_workspace_bytes(const gr_mesh* mesh);

/* One Runge-Kutta stage on every block of the mesh (steps of Sec. 3.2-3.5 in order):
 *   metric interpolation -> reconstruction -> HLLE face fluxes -> corner EMFs -> CT face update
 *   -> flux divergence + sources -> con2prim with atmosphere.  Fluxes and sources use W (the
 *   primitives of the stage input); con2prim runs once, on the output. */
int gr_stage(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
             const gr_params* params, void* stream);

/* CUDA graph of one stage: the stage's launches on `stream` captured once, with all arguments (arrays,
 * dt, params) baked in, and replayed by gr_graph_launch on any stream.  One graph per distinct stage
 * (RK sub-stage coefficients, buffers, dt); the mesh must outlive the graph.  Profiling events are
 * not recorded inside a graph. */
typedef struct gr_graph gr_graph;
int gr_graph_capture(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt,
                     const gr_params* params, gr_graph** graph);
int gr_graph_launch(gr_graph* graph, void* stream);
int gr_graph_destroy(gr_graph* graph);

/* Launch shape of a stage kernel: CTA size tile (64, 128 or 256 threads = elements of one work item),
 * order of the work list (0: direction-major, 1: block-major) and persistent (0: one CTA per work item;
 * 1: as many CTAs as fit on the GPU at once, each striding over the list).  The kernels are cell prep,
 * faces, edges, CT, update and con2prim (the order of con2prim's job list is moot).  With the order-2
 * metric the cell prep runs as a z sweep over fixed tiles of each block's x-y plane and its shape is
 * unused.  Every shape gives bitwise the same results. */
#define GR_NSTAGE_KERNELS 6
typedef struct {
  int32_t tile;
  int32_t order;
  int32_t persistent;
} gr_shape;
/* Autotuner (project-written; the paper has no counterpart): runs the stage on this mesh and state with
 * every shape (3 tiles x 2 orders x 2 grids), reps timed runs each after one warm-up, times each kernel
 * with CUDA events on `stream`, and keeps per kernel the fastest shape for (params->precision,
 * params->eos); later gr_stage and gr_graph_capture calls use it.  Then it times the whole stage through
 * every path that applies (gr_mesh_set_path) and keeps the fastest, and, when params->c2p_guess is
 * GR_GUESS_AUTO, times it with no bracket proposal and with the FP32 pre-solve and keeps the faster
 * (gr_mesh_get_guess).  Writes the stage outputs.  best_ms (may be NULL) receives the mean time of each
 * kernel's chosen shape.  Synchronises the stream. */
int gr_autotune(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt, const gr_params* params,
                int32_t reps, void* stream, double best_ms[GR_NSTAGE_KERNELS]);
/* Shapes in use for (precision, eos); defaults {128, 0, 0}.  set validates every entry (GR_EINVAL). */
int gr_mesh_get_shapes(const gr_mesh* mesh, int32_t precision, int32_t eos, gr_shape out[GR_NSTAGE_KERNELS]);
int gr_mesh_set_shapes(gr_mesh* mesh, int32_t precision, int32_t eos, const gr_shape in[GR_NSTAGE_KERNELS]);

/* Path of the mixed stage with the ideal gas, the order-2 metric and no level faces (elsewhere the separate
 * kernels run).  All paths give bitwise the same results.
 *   GR_PATH_SEPARATE     the stage kernels one after another, fluxes and EMFs through the mesh's workspace
 *   GR_PATH_FUSED        the fused sweep: the reconstruction, HLLE fluxes, corner EMFs, CT update and flux
 *                        divergence of Sec. 3.3-3.4 and Eq. claw in one pass per block, one CTA per block
 *                        walking it along z with rings of planes in shared memory (fluxes and EMFs never leave
 *                        it); con2prim then runs on the queued cells; blocks with 3 ghosts and at most 16 x 16
 *                        cells in x and y
 *   GR_PATH_TILED_FACES  the separate kernels with the face fluxes from tiles of at most 8 rows of a block
 *                        walked along z, their stencils and face metric staged in shared memory; blocks with
 *                        3 ghosts and at most 16 cells along x
 * gr_autotune times every path that applies and keeps the fastest; gr_mesh_set_path forces one
 * (GR_EUNSUPPORTED if a block does not qualify); gr_mesh_get_path returns it (-1 for a NULL mesh). */
enum { GR_PATH_SEPARATE = 0, GR_PATH_FUSED = 1, GR_PATH_TILED_FACES = 2 };
int gr_mesh_set_path(gr_mesh* mesh, int32_t path);
int gr_mesh_get_path(const gr_mesh* mesh);
/* The bracket proposal GR_GUESS_AUTO stands for on this mesh (GR_GUESS_NONE or GR_GUESS_FP32) for a
 * precision and EOS; -1 for a NULL mesh or a bad precision / EOS. */
int gr_mesh_get_guess(const gr_mesh* mesh, int32_t precision, int32_t eos);

/* ---- one stage on host-resident pools ----------------------------------------------------------------
 * gr_host_stage: the stage of gr_stage on a mesh whose pools live in host memory.  metric and state hold
 * HOST pointers in the layouts of gr_stage, to pinned (page-locked, device-mapped) memory, e.g. from
 * cudaHostAlloc; pageable memory is rejected.  The mesh keeps device copies of the pools (allocated on
 * the first call: about the size of the pools) and splits the blocks into nbatch groups of consecutive
 * blocks; each group's inputs are brought to the device, its stage runs, and its outputs are written
 * back, on three streams, so that the transfers of one group overlap the stage of another.  Only the
 * elements the stage reads or writes cross the host link: W, B and the metric with their ghosts (copy
 * engines), U (and U0 where rk_g0 != 0) on interior cells and B0 on the faces of interior cells, and of
 * the outputs the interior cells of U', W', status and the faces of interior cells of B' (kernels that
 * access the mapped host memory).  Output ghost entries are left untouched, as by gr_stage, and the
 * results equal gr_stage's bitwise.  Asynchronous: ordered after earlier work on `stream`, and `stream`
 * waits for its end; the host outputs are complete once `stream` is synchronised.  Calls on one mesh
 * must be ordered (one stream).  Errors: those of gr_stage; GR_EINVAL (nbatch outside 1..1024, a host
 * pool that is not pinned), GR_EUNSUPPORTED (a mesh with level faces, or pools that do not hold the
 * blocks in increasing order), GR_ENOMEM. */
int gr_host_stage(gr_mesh* mesh, const gr_metric* metric, const gr_state* state, double dt, const gr_params* params,
                  int32_t nbatch, void* stream);

/* ---- matter sources of the spacetime equations -----------------------------------------------------
 * gr_adm_sources: rho_ADM, S_i and S_ij, the projections of the stress-energy tensor that the spacetime
 * equations take as sources (the hydro forms of Sec. 2.1, the MHD forms with the comoving field b of
 * Sec. 2.2), at every owned vertex (0..n per axis) of every block:
 *   rho_ADM = (rho h + b^2) W^2 - (p + b^2/2) - (alpha b^0)^2
 *   S_i     = (rho h + b^2) W^2 v_i - alpha b^0 b_i
 *   S_ij    = (rho h + b^2) W^2 v_i v_j + (p + b^2/2) gamma_ij - b_i b_j
 * They are formed at cell centres (metric from its vertex-to-cell interpolant of metric->order, cell
 * field = mean of the two densitised faces, h from the EOS at (rho, p[, Y_e])) and carried to the
 * vertices by the Lagrange interpolant of order vc_order (2: the 2 nearest cells per axis, 4: the 4
 * nearest), the cell-to-vertex transfer of Sec. 3.2.  params->precision GR_PREC_FP64: all arithmetic
 * in FP64; GR_PREC_MIXED: inputs rounded to FP32 on load, FP32 arithmetic and workspace, FP64 output
 * (relative error ~1e-7 of each source's scale).
 *   W       5 (ideal gas) or 6 (table: rho, u~^i, p, Y_e) cell pools; cells -vc_order/2 .. n +
 *           vc_order/2 - 1 of every block are read, so those ghost cells must hold valid states
 *   B       densitised face fields, read on the faces of those cells
 *   out     10 vertex pools in the layout of the metric (rho_ADM, S_x, S_y, S_z, S_xx, S_xy, S_xz,
 *           S_yy, S_yz, S_zz); only owned vertices are written
 * The mesh keeps a workspace of 10 cell pools, allocated on the first call.  Errors: GR_EINVAL (NULL
 * pointer, bad order, ghost width below vc_order/2 + (metric->order == 4)), GR_EUNSUPPORTED (a block
 * too wide for one shared-memory vertex plane), GR_ENOMEM, GR_ECUDA. */
int gr_adm_sources(gr_mesh* mesh, const gr_metric* metric, const double* const W[7], const double* const B[3],
                   const gr_params* params, int32_t vc_order, double* const out[10], void* stream);

/* ---- level boundaries of a refined mesh (refinement ratio 2) --------------------------------------
 * The operators that keep a mesh of two refinement levels consistent (Sec. 3.3, last paragraph): the
 * restriction and the divergence-preserving prolongation of the face field (and of cell fields), and
 * the flux and electric-field corrections at refinement boundaries.  A fine block's cell i along an
 * axis covers half of coarse cell off + floor(i/2); its spacings must be half the coarse block's.
 *
 * gr_level_face: fine block `fine` touches the side-`side` (+1 high, -1 low) dir-face of block
 * `coarse` and covers the coarse face cells o1 .. o1 + n_fine[t1]/2 - 1 along t1 = (dir+1)%3 and
 * o2 .. o2 + n_fine[t2]/2 - 1 along t2 = (dir+2)%3.  With level faces set, every gr_stage on the mesh
 * replaces, after computing them, the coarse block's fluxes of the conserved variables on those faces
 * by the mean of the 4 fine-face fluxes on each, and its corner EMFs on those faces' edges by the mean
 * of the 2 fine edge EMFs along each; total D is then conserved across the levels and each coarse face
 * stays the mean of the fine faces on it.  (Conserved to FP64 rounding on the FP64 path; the mixed path
 * stores the means in its FP32 workspace, so there they hold to FP32 rounding of the flux.)  A coarse
 * edge shared by two fine patches is written by both with the same value when the fine blocks' shared
 * edge values agree (same-level ghost copies); records must not chain three levels at one edge.
 *
 * gr_level_map: a coarse block, a fine block, the fine block's offset `off` in coarse cells and an
 * element range lo .. hi-1 (per axis; faces along d include index hi[d]).  Restriction maps: the range
 * is in coarse cells, each set to the mean of its 8 fine cells (cells) or the mean of the 4 fine faces
 * on each of its faces (B).  Prolongation maps: the range is in fine cells, each set from the coarse
 * data: cells by limited linear reconstruction (minmod of the one-sided coarse differences), faces on
 * a coarse face plane from the coarse value and its limited transverse slopes, faces inside a coarse
 * cell by the minimal-norm correction, to the mean of the two opposite outer fine faces, that makes the
 * 8 fine cells divergence-free.  Every coarse cell a prolongation reads must have its 6 face
 * neighbours inside the coarse block's ghost-padded array (checked).  A map whose range lies wholly
 * outside its destination block along d (a ghost slab) does not write that block's own d-face planes
 * 0 and n (they belong to the block and to the level-boundary corrections).
 *
 * With restriction or prolongation maps set, the RK driver fills ghosts in three passes before every
 * stage: same-level copies (its neighbour table; a side toward another level is marked outflow, -1),
 * then the restriction maps, then the prolongation maps, on the primitive pools and B.
 *
 * gr_mesh_set_levels copies the tables to the device (checked: indices, spacings, ranges); n = 0 clears.
 * gr_restrict / gr_prolong apply the stored maps to nvar (<= 8) cell pools and, if B is not NULL, to the
 * three face pools; maps run concurrently, so their destinations must not overlap.  Errors:
 * GR_EINVAL (bad table, NULL pool), GR_ENOMEM, GR_ECUDA. */
typedef struct {
  int32_t coarse, fine, dir, side, o1, o2;
} gr_level_face;
typedef struct {
  int32_t coarse, fine, off[3], lo[3], hi[3];
} gr_level_map;
int gr_mesh_set_levels(gr_mesh* mesh, const gr_level_face* faces, int32_t nfaces, const gr_level_map* restrict_maps,
                       int32_t nrestrict, const gr_level_map* prolong_maps, int32_t nprolong);
int gr_restrict(gr_mesh* mesh, double* const cells[8], int32_t nvar, double* const B[3], void* stream);
int gr_prolong(gr_mesh* mesh, double* const cells[8], int32_t nvar, double* const B[3], void* stream);

/* ---- RK driver: a full time step of a set of same-level blocks -----------------------------------------
 * (the third-order Runge-Kutta integrator used for every test of Sec. 4-8, stated at the start of
 * Sec. 4; the global time step of Sec. 3.1)
 * nbr[27 b + (oz+1) 9 + (oy+1) 3 + (ox+1)] = the block adjacent to block b in direction (ox, oy, oz) in
 * {-1,0,1}^3, or -1 at an outflow boundary; entry 13 is b itself; neighbours have b's n and ng.  The
 * driver owns two sets of stage buffers (U, W, B pools of the mesh's pool extents) and dt on the device.
 * gr_ghost_fill copies every ghost cell of the nw cell pools W and every ghost face of B from the owning
 * neighbour (outflow: from the nearest owned element of the same block).
 * gr_cfl_dt: dt = cfl min over interior cells and directions of dx_d / max(|lambda-_d|, |lambda+_d|)
 * (the fast speeds of Sec. 2.2), reduced on the device into dt_dev (NULL: the driver's own).
 * dt_mode of a step: GR_DT_GRID, the paper's rule dt = cfl min dx over the mesh (CFL 0.25 on the finest
 * spacing, Sec. 3.1), or GR_DT_SIGNAL, the wave-speed rule of gr_cfl_dt.
 * gr_driver_step: ghost fill, dt, then the rk_order (2 or 3) stages of SSP-RK2/RK3 with ghost fills in
 * between; U, W, B (and status, of the last stage) are updated in place; nothing is synchronised, so
 * gr_driver_capture records the whole step as one CUDA graph.  gr_driver_dt copies the last dt to the
 * host (synchronous). */
typedef struct gr_driver gr_driver;
enum { GR_DT_GRID = 0, GR_DT_SIGNAL = 1 };
int gr_driver_create(gr_mesh* mesh, const int32_t* nbr, gr_driver** driver);
int gr_driver_destroy(gr_driver* driver);
int gr_ghost_fill(gr_driver* driver, double* const W[7], int32_t nw, double* const B[3], void* stream);
int gr_cfl_dt(gr_driver* driver, const gr_metric* metric, const double* const W[7], const double* const B[3],
              const gr_params* params, double cfl, double* dt_dev, void* stream);
int gr_driver_step(gr_driver* driver, const gr_metric* metric, double* const U[6], double* const W[7],
                   double* const B[3], uint8_t* status, const gr_params* params, double cfl, int32_t dt_mode,
                   int32_t rk_order, void* stream);
int gr_driver_capture(gr_driver* driver, const gr_metric* metric, double* const U[6], double* const W[7],
                      double* const B[3], uint8_t* status, const gr_params* params, double cfl, int32_t dt_mode,
                      int32_t rk_order, gr_graph** graph);
int gr_driver_dt(const gr_driver* driver, double* dt);
const double* gr_driver_dt_device(const gr_driver* driver);

/* Primitive -> conserved (Eq. consB_def) on the interior cells of every block, with the cell-centred
 * field taken as the mean of the two densitised faces.  W[0..4] (+ W[5] = Y_e with a table) are read;
 * U[0..4] (+ U[5] = D Y_e) written.  Unused trailing entries may be NULL. */
int gr_prim2con(gr_mesh* mesh, const gr_metric* metric, const double* const W[7],
                const double* const B[3], double* const U[6], const gr_params* params, void* stream);

/* Conserved -> primitive on the interior cells (Sec. 3.5, App. A).  U is rewritten where the
 * atmosphere or a limit applies.  status and evals (the number of FP64 master-function evaluations
 * per cell) may be NULL.  With a table U has 6 and W 7 entries (Y_e and T written). */
int gr_con2prim(gr_mesh* mesh, const gr_metric* metric, double* const U[6], const double* const B[3],
                double* const W[7], uint8_t* status, int32_t* evals, const gr_params* params, void* stream);

/* Device copy of an EOS table on the context's device: the three node arrays in FP64 (con2prim, FP64
 * path) and in FP32 (mixed path), 36 n0 n1 n2 bytes in all (gr_eos_bytes), plus the table's minimum
 * enthalpy h0 = min (e + p)/rho over the nodes (the enthalpy bound of the con2prim bracket, gr_eos_h0).
 * Checks the sizes, finiteness and the strict increase in T; GR_EINVAL otherwise.  Synchronous.  The
 * table must outlive every call that uses it. */
int gr_eos_create(gr_ctx* ctx, const gr_eos_table* table, gr_eos** eos);
int gr_eos_destroy(gr_eos* eos);
int64_t gr_eos_bytes(const gr_eos* eos);
double gr_eos_h0(const gr_eos* eos);

/* Diagnostics (Eq. Mb, Eq. gausslaw).  out[0] = M_b = sum D dV; out[1] = max |div B| min(dx)/max|B|;
 * out[2] = sum |div B| dV / (max|B| sum dV / min dx); out[3] = max |B| over interior faces.
 * Synchronises the stream. */
int gr_diag(gr_mesh* mesh, const double* const U[5], const double* const B[3], double out[4],
            void* stream);

/* FP32 copy of an FP64 device array, the conversion the mixed path applies to its inputs: IEEE round
 * to nearest, ties to even, with float subnormals and overflow to infinity (NaN stays NaN), computed in
 * integer arithmetic (on GB300 a hardware FP64 -> FP32 conversion runs on the narrow FP64 pipe).
 * src and dst are device arrays of n elements on the current device (no alignment needed); asynchronous on
 * `stream`.  GR_EINVAL for n < 0 or a NULL pointer with n > 0. */
int gr_cast_f32(const double* src, float* dst, int64_t n, void* stream);

/* ---- learned con2prim bracket (not in the paper: a bracket proposal for the root find of Sec. 3.5) --
 * A 6-64-64-1 tanh network predicts log mu at the master-function root from the features
 * log(1+q), log(1+r^2), log(1+calb^2), (r.calb)^2/(r^2 calb^2) of the KKC invariants and, with a table,
 * log D~ and Y_e (0 and 0 for the scale-free ideal gas) (the reading of Sec. 3.5's bracketing);
 * con2prim with GR_GUESS_MLP starts at exp(t_hat) and steps outwards by factors exp(delta 2^k),
 * k = 0..5, until the FP64 master function changes sign, and solves in that bracket; otherwise it
 * falls back to the full bracket (status GR_ST_GUESS_REJECTED).
 * Parameter vector: GR_MLP_NPARAM floats, 16-byte aligned device memory:
 *   [0..5] feature means, [6..11] feature inverse std, [12] target mean, [13] target std,
 *   [14] first step delta (in log mu), [15] unused, [16..] W1 (64x6), b1 (64), W2 (64x64), b2 (64),
 *   W3 (64), b3 (1), row-major (out, in).  Samples x are rows of 6 floats; targets t are log mu. */
#define GR_MLP_NPARAM 4689
#define GR_MLP_NIN 6
int gr_mlp_nparam(void);
const char* gr_mlp_last_error(void);
/* Features and log mu of the plain (unguessed) bracketed solve of every interior cell, in the cell-pool
 * layout; valid = 0 where the cell is not solved or a limit applied. */
int gr_c2p_samples(gr_mesh* mesh, const gr_metric* metric, const double* const U[6], const double* const B[3],
                   const gr_params* params, float* const feats[6], float* target, uint8_t* valid, void* stream);
/* t[i] = predicted log mu of sample i. */
int gr_mlp_forward(const float* P, const float* x, int64_t n, float* t, void* stream);
/* Gradient (GR_MLP_NPARAM - 16 floats, the weights after the 16 header entries) and value of the mean
 * loss (z - zt)^2/2, zt = (t - P[12])/P[13], over n samples; device outputs.  Synchronises the stream. */
int gr_mlp_grad(const float* P, const float* x, const float* t, int64_t n, float* grad, float* loss, void* stream);
/* Adam (lr, beta 0.9/0.999) over the samples in order, mini-batches of `batch`, `epochs` passes; updates
 * the weights of P in place and writes the mean loss of each epoch to the host array losses (may be NULL).
 * Allocates and frees its own scratch.  Synchronises the stream. */
int gr_mlp_train(float* P, const float* x, const float* t, int64_t n, int32_t epochs, int32_t batch, float lr,
                 float* losses, void* stream);

/* gr_diag without any device allocation (the paper has no counterpart: this is a library service).
 * For callers that cannot call cudaMalloc -- code running inside an application that owns the device
 * memory pool (its own caching allocator or fixed arena) or in-situ hooks that must not change the
 * device footprint.  Same outputs as gr_diag, for at most 256 blocks given directly (no gr_mesh):
 * the block list travels as a kernel parameter and the reduction's scratch is a fixed 33 KB static
 * device array that every GPU loading the library holds until exit.  Every call looks up that array's
 * address in the CUDA context current on the calling thread (cudaGetSymbolAddress, which allocates
 * nothing), so callers with their own contexts and calls after cudaDeviceReset are served.
 * Calls share the array: each call overwrites every slot it reads, but calls whose kernels overlap on
 * the GPU race and must be serialised by the caller.  nblocks outside [1, 256] gives GR_EINVAL
 * (detail in gr_noalloc_last_error).  Synchronises the stream. */
int gr_diag_noalloc(const gr_block* blocks, int32_t nblocks, const double* const U[5],
                    const double* const B[3], double out[4], void* stream);
const char* gr_noalloc_last_error(void);

/* ---- measurement -----------------------------------------------------------------------------------
 * gr_peak_alu: one launch of an arithmetic throughput loop (the paper has no counterpart: it measures
 * the pipe peaks that ALU-bound kernels are compared with).  kind 0: FP32 FMA, 1: packed FP32x2 FMA,
 * 2: FP64 FMA; `blocks` CTAs of `threads` (32..256, a multiple of 32) threads, each running 16
 * independent FMA chains for `iters` rounds.  *flops receives the floating-point operations of the
 * launch (2 per FMA); time it with events on `stream`.  sink: a device float per CTA, written only in a
 * case that never occurs (keeps the loop).  GR_EINVAL for bad arguments, GR_ECUDA if the launch fails. */
int gr_peak_alu(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, float* sink, double* flops,
                void* stream);

/* Per-kernel timing of gr_stage with CUDA events on the launch stream (measurement only).
 * gr_profile_begin arms the mesh for up to max_stages subsequent gr_stage calls: each records an event
 * before and after each of its GR_NKERNELS kernels (FP32 input cast of the mixed path, cell prep, faces,
 * edges, CT, update, con2prim; the FP64 path launches no cast and its first entry is ~0).
 * gr_profile_end synchronises on the last event and returns, per kernel, the summed milliseconds in
 * ms[GR_NKERNELS] and the number of profiled stages in *nstages; it disarms the mesh. */
#define GR_NKERNELS 7
int gr_profile_begin(gr_mesh* mesh, int32_t max_stages);
int gr_profile_end(gr_mesh* mesh, double* ms, int32_t* nstages);

#ifdef __cplusplus
}
#endif

#endif /* GRSTAGE_H */
