/*
 * bssn.h -- C ABI of libbssn: the BSSN moving-puncture right-hand side of
 * "The Einstein Toolkit" (arXiv:1111.3344), Sec. "Spacetime Curvature
 * Evolution", advanced by fourth-order Runge-Kutta method of lines on a
 * uniform cell-centred grid with three ghost layers, on one NVIDIA GB300
 * (sm_103a).
 *
 * Conventions
 *  - Every call returns bssn_status (BSSN_OK = 0).  On failure,
 *    bssn_last_error() returns a message for the calling thread.
 *  - The caller owns all bulk device memory and the CUDA stream.  The library
 *    carves its registers and small tables out of the block given to
 *    bssn_alloc and never calls cudaMalloc.
 *  - Calls are asynchronous on the bound stream unless their comment says
 *    "synchronises".
 *  - Device state layout (structure of arrays): element (f, k, j, i) of a
 *    register lives at f*field_stride + k*plane + j*pitch + i, for field
 *    f in [0, 24), stored point (i, j, k) in [0, n0+6) x [0, n1+6) x
 *    [0, n2+6); point i on an axis sits at xmin + (i - 3 + 1/2) h.  pitch is
 *    a multiple of 8 elements; see bssn_layout.
 *  - Host state layout (bssn_get_state / bssn_set_state): the same order
 *    without padding, float64, shape (24, n2+6, n1+6, n0+6).
 *  - Field order: 0 phi or W, 1..6 conformal metric gt_xx gt_xy gt_xz gt_yy
 *    gt_yz gt_zz, 7 trace K, 8..13 trace-free At_ij (same order), 14..16
 *    conformal connection Gt^i, 17 lapse alpha, 18..20 shift beta^i,
 *    21..23 B^i (the 24 evolved grid functions of the paper's BSSN system).
 */
#ifndef BSSN_H
#define BSSN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSSN_NUM_FIELDS 24
#define BSSN_GHOST 3

typedef enum {
  BSSN_OK = 0,
  BSSN_EINVAL = 1,    /* bad argument or parameter */
  BSSN_ENOMEM = 2,    /* memory block too small / budget exceeded */
  BSSN_ECUDA = 3,     /* a CUDA call failed (message has the CUDA error) */
  BSSN_EAGAIN = 4,    /* poll: request not finished yet */
  BSSN_ETIMEOUT = 5,  /* a bounded wait expired */
  BSSN_ENOTFOUND = 6, /* unknown ticket */
  BSSN_EFAILED = 7    /* NaN/Inf detected in a request's state */
} bssn_status;

enum { BSSN_BC_PERIODIC = 0, BSSN_BC_SOMMERFELD = 1 };
enum { BSSN_PHI = 0, BSSN_W = 1 };
enum { BSSN_1PLUSLOG = 0, BSSN_HARMONIC = 1, BSSN_GEODESIC = 2 };
enum { BSSN_GAMMA_DRIVER = 0, BSSN_SHIFT_FROZEN = 1 };
enum { BSSN_FP64 = 0, BSSN_MIXED = 1, BSSN_FF = 2 };
enum { BSSN_ID_FLAT = 0, BSSN_ID_GAUGE_WAVE = 1, BSSN_ID_BL = 2, BSSN_ID_KASNER = 3 };

/* Grid and method parameters.
 *  n, ghost, xmin, h   uniform cell-centred grid (Sec. "Simulation Domain,
 *                      Symmetries, Boundaries": physical vs discrete domain);
 *                      n[d] >= 4, ghost == 3, h > 0.
 *  boundary            periodic ghosts or the Sommerfeld radiative condition
 *                      of Sec. "Boundary Conditions".
 *  conformal           evolve phi (the paper's variable) or W = exp(-2 phi).
 *  slicing             d_0 alpha = -alpha^2 f K with f = 2/alpha (1+log,
 *                      Sec. "Spacetime Curvature Evolution"), f = 1
 *                      (harmonic) or f = 0 (geodesic).
 *  shift               Gamma-driver (d_0 beta = (3/4) B, d_0 B = d_0 Gt -
 *                      eta q(r) B) or frozen (beta, B right-hand sides 0).
 *  eta, q_R            Gamma-driver damping and the radius R of q(r) = 1
 *                      (r <= R), R/r (r > R); q_R <= 0 or inf means q = 1.
 *  ko_eps              Kreiss-Oliger epsilon.
 *  dt                  RK4 time step.
 *  precision           BSSN_FP64: everything in float64.  BSSN_MIXED:
 *                      stencils and right-hand side in float32, RK4 state
 *                      and constraint reductions in float64.  BSSN_FF:
 *                      stencils and right-hand side in double-word
 *                      ("float-float", 48-bit) arithmetic on the float32
 *                      pipe, RK4 state, k-sum and reductions in float64
 *                      (contexts, batches and the server).
 *  ksum_fp64           mixed precision, single-grid contexts only: 1 keeps
 *                      the weighted sum of the RK4 k of every field in
 *                      float64 (one more float64 register; W's is float64
 *                      in any case; the stage runs the fused 32x8x1 kernel
 *                      whatever the tile configuration), 0 in float (the
 *                      default).
 *  w_fp64_threshold    mixed precision: points with W below this take the
 *                      W/phi right-hand side in float64.
 *  r_excise            constraint norms: excised set is r > r_excise from
 *                      every puncture.
 *  w_floor             lower bound on W wherever W divides (default 1e-10).
 */
typedef struct bssn_params {
  int32_t n[3];
  int32_t ghost;
  double xmin[3];
  double h;
  int32_t boundary;
  int32_t conformal;
  int32_t slicing;
  int32_t shift;
  double eta;
  double q_R;
  double ko_eps;
  double dt;
  int32_t precision;
  int32_t ksum_fp64;
  double w_fp64_threshold;
  double r_excise;
  double w_floor;
} bssn_params;

/* Register layout of one evolution (all counts in elements). */
typedef struct bssn_layout {
  int32_t stored[3];      /* n[d] + 6 */
  int32_t ghost;          /* 3 */
  int64_t pitch;          /* elements per x-row, multiple of 8 */
  int64_t plane;          /* pitch * stored[1] */
  int64_t field_stride;   /* plane * stored[2] */
  int64_t register_elems; /* 24 * field_stride */
} bssn_layout;

typedef struct bssn_ctx bssn_ctx;       /* one evolution (opaque) */
typedef struct bssn_server bssn_server; /* continuous-batching server (opaque) */

/* Thread-local message for the last failed call on this thread. */
const char* bssn_last_error(void);

/* Fill *out with the register layout for p.  Host only.  EINVAL on bad p. */
bssn_status bssn_layout_of(const bssn_params* p, bssn_layout* out);

/* Device bytes bssn_alloc needs for p (registers y_n, accumulator, two stage
 * buffers, boundary-anchor buffer, reduction scratch).  Host only; 0 on bad p. */
size_t bssn_required_bytes(const bssn_params* p);

/* Bind an evolution to caller-owned device memory d_mem (>= required bytes,
 * 256-byte aligned) and a CUDA stream (cudaStream_t as void*, NULL = legacy
 * default stream).  Validates p; allocates only the host-side context.  The
 * state is undefined until set_initial_data or set_state.  t starts at 0. */
bssn_status bssn_alloc(const bssn_params* p, void* d_mem, size_t bytes, void* cuda_stream,
                       bssn_ctx** out);

/* Release the host-side context (does not free d_mem; synchronises the stream). */
bssn_status bssn_free(bssn_ctx* ctx);

/* Device pointer of the current state register y_n (float64, layout above). */
bssn_status bssn_state_ptr(bssn_ctx* ctx, double** d_state);

/* Analytic initial data, converted to BSSN by the definitions of Sec.
 * "Spacetime Curvature Evolution" with B^i = 0 (Sec. "Initial Conditions"),
 * evaluated on the device at every stored point; t is reset to 0.
 *   BSSN_ID_FLAT        p ignored.
 *   BSSN_ID_GAUGE_WAVE  p = {A, d}: ds^2 = H(-dt^2 + dx^2) + dy^2 + dz^2,
 *                       H = 1 - A sin(2 pi x / d) at t = 0.
 *   BSSN_ID_BL          p = {npunct, m_1, x_1, y_1, z_1, ...} (npunct <= 8):
 *                       Brill-Lindquist, psi = 1 + sum m_a / (2 r_a),
 *                       gamma = psi^4 delta, K_ij = 0 (Sec. "Initial Data",
 *                       TwoPunctures with u = 1 at K = 0); alpha = psi^-2.
 *                       The punctures also define the excised norm set.
 *   BSSN_ID_KASNER      p = {t0}: Kasner slice of Sec. "Cosmology",
 *                       gamma = diag(t0^{4/3}, t0^{4/3}, t0^{-2/3}), alpha = 1.
 * EINVAL on an unknown kind or too few parameters. */
bssn_status bssn_set_initial_data(bssn_ctx* ctx, int32_t kind, const double* p, int32_t np);

/* General initial data from ADM fields (Sec. "Initial Conditions"): host_adm
 * holds 16 float64 fields in the unpadded host layout, (16, n2+6, n1+6, n0+6):
 * alpha, beta^x, beta^y, beta^z, gamma_xx, gamma_xy, gamma_xz, gamma_yy,
 * gamma_yz, gamma_zz, K_xx, ..., K_zz, at every stored point.  The BSSN
 * variables follow by their definitions with B^i = 0; Gt^i = gt^jk Gt^i_jk
 * from 4th-order first derivatives of gt_ij at interior points and, on the
 * outer ghost layers, by cubic extrapolation along the summed outward normal
 * (faces perpendicular, edges and corners diagonal), innermost layer first;
 * periodic grids copy their ghosts instead.  Synchronises; sets t. */
bssn_status bssn_set_adm(bssn_ctx* ctx, const double* host_adm, double t);

/* Punctures {m, x, y, z} x npunct (npunct 0..8) that define the excised set of
 * the constraint norms (set_initial_data with BSSN_ID_BL sets them too). */
bssn_status bssn_set_punctures(bssn_ctx* ctx, const double* p, int32_t npunct);

/* One right-hand side, interior points by the BSSN equations (4th-order
 * centred stencils, upwinded advection, KO dissipation), ghost points by the
 * Sommerfeld condition (or 0 when periodic).  d_state: a float64 register in
 * the layout above (NULL = the context's y_n); d_rhs: a float64 register the
 * caller owns.  Ghost values of d_state must be valid (periodic: filled). */
bssn_status bssn_rhs(bssn_ctx* ctx, const void* d_state, void* d_rhs);

/* Advance y_n by nsteps classical RK4 steps of size dt (t += nsteps dt).
 * With tracking on (bssn_track_punctures), each step first moves the
 * punctures by one Euler step of the shift of y_n. */
bssn_status bssn_rk4_step(bssn_ctx* ctx, int32_t nsteps);

/* Matter coupling (Sec. "Spacetime Curvature Evolution" source terms,
 * Sec. "TmunuBase"): d_tmunu is a caller-owned device array of
 * 10 * field_stride doubles in the register layout holding T_{mu nu} at every
 * stored point, in the order T_00, T_0x, T_0y, T_0z, T_xx, T_xy, T_xz, T_yy,
 * T_yz, T_zz; NULL returns to vacuum.  From the projections
 * E = (T_00 - 2 beta^i T_0i + beta^i beta^j T_ij)/alpha^2,
 * S_i = -(T_0i - beta^j T_ij)/alpha, S_ij = T_ij, S = gamma^ij S_ij, every
 * later right-hand side gets d_0 K += 4 pi alpha (E + S),
 * d_0 At_ij -= 8 pi alpha e^{-4 phi} [S_ij]^TF and d_0 Gt^i -= 16 pi alpha
 * gt^ij S_j (the B^i equation through d_0 Gt^i); bssn_constraints subtracts
 * 16 pi E from H and 8 pi S_i from M_i, and bssn_adm_integrals adds 16 pi E
 * and 8 pi x^j S_k to its integrands.  T_{mu nu} is read as given during every
 * stage of a step (constant over the step; the matter evolution itself is the
 * caller's) and must stay valid while set.  bssn_psi4 keeps the vacuum
 * projections.  Batches and the server evolve vacuum only. */
bssn_status bssn_set_matter(bssn_ctx* ctx, const double* d_tmunu);

/* Puncture tracking (Sec. "Object tracking"): with enable != 0, every RK4 step
 * moves each puncture of the context (set by bssn_set_punctures or Brill-
 * Lindquist initial data) by x <- x - dt beta(t_n, x), the shift of y_n
 * interpolated by the tensor product of 4-point Lagrange polynomials on stored
 * points i0-1 .. i0+2 (i0 the stored point at or below x; the stencil is
 * shifted inward at the edge of the stored block).  The positions stay on the
 * device; the excised sets of bssn_constraints and bssn_adm_integrals follow
 * them.  enable = 0 stops tracking (positions are kept). */
bssn_status bssn_track_punctures(bssn_ctx* ctx, int32_t enable);

/* Current punctures, rows {m, x, y, z}, into out (room for 8 rows, 32
 * doubles) and their count into *npunct.  Synchronises when the tracker has
 * moved them since the last read. */
bssn_status bssn_get_punctures(bssn_ctx* ctx, double* out, int32_t* npunct);

/* Constraint norms of y_n (synchronises): out[0..3] L2 (root mean square)
 * of H, M_x, M_y, M_z over interior points, out[4..7] their max-abs, out[8..15]
 * the same over interior points farther than r_excise from every puncture.
 * H = R - K^i_j K^j_i + K^2, M_i = nabla_j K_i^j - nabla_i K (vacuum) from the
 * ADM fields (Sec. "Other analysis modules"), float64 in every precision. */
bssn_status bssn_constraints(bssn_ctx* ctx, double out[16]);

/* ADM mass and angular momentum of y_n as volume integrals (Sec. "Masses and
 * Momenta", vacuum), synchronises:
 *   M   = 1/(16 pi) int [ e^{5 phi}(At_ij At^ij - (2/3) K^2) - e^{phi} Rt ]
 *   J_i = 1/(8 pi) eps_ijk int e^{6 phi} [ At^j_k + (2/3) x^j d_k K
 *                                          - (1/2) x^j At_ln d_k gt^{ln} ]
 * Rt = gt^ij Rt_ij as in the right-hand side, x^j the grid coordinates, the
 * integral the midpoint sum h^3 sum over interior points.  out[0..3] = M, J_x,
 * J_y, J_z over all interior points, out[4..7] over the points farther than
 * r_excise from every puncture.  d_dens: NULL, or a caller-owned device array
 * of 4 * field_stride doubles (register layout) that receives the four
 * integrands at interior points (other points untouched).  Float64 in every
 * precision mode. */
bssn_status bssn_adm_integrals(bssn_ctx* ctx, double* d_dens, double out[8]);

/* Weyl scalar Psi4 = C_abcd n^a mb^b n^c mb^d of y_n (Sec. "Gravitational
 * Waves", WeylScal4, vacuum) for the fiducial tetrad n = (u - r)/sqrt2,
 * m = (theta + i phi)/sqrt2: u the unit normal, the spatial triad started from
 * r = x^i, phi = (-y, x, 0), theta^i = sqrt(det g) g^ik eps_klm phi^l r^m
 * (x^i the grid coordinates) and made orthonormal in gamma_ij by Gram-Schmidt
 * in the order phi, r, theta; the curvature enters through the Gauss, Codazzi
 * and Ricci projections with 4th-order stencils of the ADM fields.  Psi4 = 0
 * where phi = 0 (the z axis).  d_out: caller-owned device array of
 * 2 * field_stride doubles (register layout), real part then imaginary part,
 * written at interior points only.  Asynchronous on the context's stream;
 * float64 in every precision mode. */
bssn_status bssn_psi4(bssn_ctx* ctx, double* d_out);

/* Copy y_n to / from host memory (unpadded float64 layout; synchronises).
 * Pinned host memory gives full transfer speed.  t may be NULL. */
bssn_status bssn_get_state(bssn_ctx* ctx, double* host_state, double* t);
bssn_status bssn_set_state(bssn_ctx* ctx, const double* host_state, double t);

/* The same copies without waiting for them (no counterpart in the paper: a
 * host loop that uploads a state, steps and reads it back every step).
 * The layout, arguments and errors are those of bssn_get_state / bssn_set_state.
 *
 * bssn_set_state_async:
 *  - Enqueues the upload on the context's stream.
 *  - host_state must be pinned, and must stay unchanged until the stream has
 *    passed the copy (bssn_wait_state, or any later synchronising call).
 *
 * bssn_get_state_async:
 *  - Repacks y_n on the context's stream into a read-back area that later uploads
 *    do not use.
 *  - Copies it to host_state on a copy stream of the library, so that the copy
 *    can overlap the next bssn_set_state_async.
 *  - host_state must be pinned, and is valid after bssn_wait_state.
 *  - The next call that may overwrite the read-back area first waits, on the
 *    device, for that copy: the next bssn_get_state_async, bssn_rk4_step,
 *    bssn_rhs, the initial-data and analysis calls, and bssn_autotune.
 *  - *t (if t is not NULL) is the time of the state read.
 *
 * bssn_wait_state:
 *  - Synchronises both streams.
 *  - Returns BSSN_ETIMEOUT if a stage kernel gave up waiting (see bssn_rk4_step). */
bssn_status bssn_set_state_async(bssn_ctx* ctx, const double* host_state, double t);
bssn_status bssn_get_state_async(bssn_ctx* ctx, double* host_state, double* t);
bssn_status bssn_wait_state(bssn_ctx* ctx);

/* Optional staging areas for the asynchronous copies (no counterpart in the
 * paper).
 *  - d_mem: caller-owned device memory, 256-byte aligned, at least
 *    bssn_staging_bytes(p) bytes: an upload area and a read-back area, each the
 *    state in the host layout.  No kernel of a step touches them.
 *  - With them bound, bssn_set_state_async copies on an upload stream of the
 *    library while the context's stream may still be stepping, and repacks into
 *    y_n in stream order.  bssn_get_state_async repacks into the read-back area
 *    and copies from there on the copy stream.  The copies of a host loop
 *    (upload, step, read back) then overlap the steps as well as each other.
 *  - d_mem = NULL unbinds.  The call synchronises every stream of the context.
 *  - bssn_staging_bytes is host only; it returns 0 on bad p.
 *  - EINVAL on misalignment; ENOMEM if bytes is too small. */
size_t bssn_staging_bytes(const bssn_params* p);
bssn_status bssn_set_staging(bssn_ctx* ctx, void* d_mem, size_t bytes);

/* Stage-kernel tile configurations: block shape (points along x, y, z) and the
 * minimum resident blocks per SM given to the compiler.  The last ones are for
 * the mixed path only: "tma32x4x1/2" and "tma32x8x1/1" stage the
 * second-differenced fields W, gt_ij and alpha of each tile in shared memory by
 * TMA (two blocks of 32x4 points per SM, or one block of 32x8 points per SM,
 * which leaves more L1 for the other fields); "tma11_32x8x1/1" stages beta^i
 * as well (eleven fields, 173 KB of shared memory, one block of 32x8 points
 * per SM); "split32x4x1/B" (B = 2, 3, 4) run the stencils as one
 * pass per field into a derivative register and the algebra as a second pass.
 * Every configuration evaluates the same per-point arithmetic, so results agree
 * to rounding and each configuration is reproducible bit for bit. */
int32_t bssn_tile_count(void);
const char* bssn_tile_name(int32_t cfg); /* e.g. "32x8x1/1"; "" when out of range */
bssn_status bssn_set_tile(bssn_ctx* ctx, int32_t cfg);

/* Autotuner: time every tile configuration on this evolution's live state
 * (reps launches each of the first two RK4 stages, which leave y_n unchanged;
 * the next step overwrites the stage buffers and k-sum they write), select the
 * fastest for the context and return it in *best; ms_per_cfg (may be NULL,
 * else bssn_tile_count() entries) receives the mean milliseconds per stage
 * launch (INFINITY for configurations this context cannot use).  Synchronises
 * the stream. */
bssn_status bssn_autotune(bssn_ctx* ctx, int32_t reps, int32_t* best, double* ms_per_cfg);

/* ------------------------------------------------------------ batches
 * Many independent evolutions (different grids and parameters, one precision)
 * advanced together by bssn_batch_step, one RK4 step replayed from a captured
 * CUDA graph.  Two forms, chosen by the batch's tile configuration
 * (bssn_batch_set_tile, bssn_batch_autotune):
 *  - work-list configurations: one launch per RK4 stage over the tiles of
 *    every active member (persistent or one block per tile) plus one boundary
 *    launch; the graph reads a device work-list, so members join and leave
 *    between steps without re-capture;
 *  - per-member configurations ("members", "members4", "members1"; the
 *    defaults): each member's stages and boundaries with the single-grid
 *    kernels, one launch chain per member, the chains side by side on 16, 4
 *    or 1 auxiliary streams inside the graph, which is captured again when
 *    the membership changes.
 * A member computes the same bits as the same evolution run alone through a
 * bssn_ctx.  All device memory comes from the caller's pool: the batch tables
 * (bssn_batch_table_bytes) at its start, then member registers carved by a
 * first-fit sub-allocator (bssn_batch_member_bytes each). */
#define BSSN_BATCH_MAX_MEMBERS 256
typedef struct bssn_batch bssn_batch;

size_t bssn_batch_table_bytes(int32_t max_members);   /* 0 if out of range */
size_t bssn_batch_member_bytes(const bssn_params* p); /* 0 on bad p */
/* precision: BSSN_FP64, BSSN_MIXED or BSSN_FF for every member; cuda_stream
 * must not be the legacy default stream (graphs are captured on it). */
bssn_status bssn_batch_create(int32_t precision, int32_t max_members, void* d_pool,
                              size_t pool_bytes, void* cuda_stream, bssn_batch** out);
bssn_status bssn_batch_free(bssn_batch* b); /* synchronises; does not free the pool */
/* Add a member (inactive until its initial data or state is set).  ENOMEM when
 * the batch or the pool is full, EINVAL on bad params or a precision mismatch. */
bssn_status bssn_batch_add(bssn_batch* b, const bssn_params* p, int32_t* member);
bssn_status bssn_batch_remove(bssn_batch* b, int32_t member); /* synchronises */
bssn_status bssn_batch_set_initial_data(bssn_batch* b, int32_t member, int32_t kind,
                                        const double* p, int32_t np);
bssn_status bssn_batch_set_state(bssn_batch* b, int32_t member, const double* host, double t);
bssn_status bssn_batch_get_state(bssn_batch* b, int32_t member, double* host, double* t);
/* Advance every active member that is not held (bssn_batch_hold) nsteps RK4
 * steps (asynchronous). */
bssn_status bssn_batch_step(bssn_batch* b, int32_t nsteps);
bssn_status bssn_batch_constraints(bssn_batch* b, int32_t member, double out[16]); /* synchronises */
/* hold != 0: the member stays resident (registers, state, time) but the next
 * bssn_batch_step calls leave it out; hold = 0 puts it back.  Its results do
 * not change: a held member resumes from the same state.  ENOTFOUND for an
 * unknown member. */
bssn_status bssn_batch_hold(bssn_batch* b, int32_t member, int32_t hold);
/* Tile configurations of the batched stage, each but the "members" ones one launch per
 * RK4 stage over every active member's tiles:
 *   "TXxTYxTZ/B"     persistent kernels (resident blocks loop over the tiles);
 *   "tilesTXxTYxTZ/B" one block per tile (no loop, fewer register spills; the
 *                    graph is captured again when the membership changes);
 *   "tma32x4x1/2"    persistent, staging W, gt_ij and alpha of each 32x4x1
 *                    tile in shared memory by tensor loads (mixed batches
 *                    only; BSSN_EINVAL for float64);
 *   "tma11_32x8x1/1" the same on 32x8x1 tiles, staging beta^i as well
 *                    (one block per SM);
 *   "members"        each member's stages and boundaries launched with the
 *                    single-grid kernels (float64 "32x4x1/1", mixed
 *                    "tma11_32x8x1/1", double-word "ffrows32x4x1/8"), the
 *                    members' chains side by side on 16 auxiliary streams in
 *                    one captured graph, so that one member's boundary
 *                    overlaps another's stage (a launch per member per stage,
 *                    not one per stage; each member gets the same bits as a
 *                    single-grid evolution on that tile);
 *   "members4", "members1" the same on 4 streams, or one member after
 *                    another on one stream (different double-word kernels
 *                    sharing an SM slow each other: double-word batches start
 *                    on "members1");
 *   "fftiles32x4x1/MF+MR" (last) the double-word one-block-per-tile
 *                    kernels (register caps of the full-tile and the
 *                    every-stencil kernel).
 * A new batch starts on "members" (float64 and mixed) or "members1"
 * (double-word).  A
 * tensor-load wait that gives up (bounded) makes the next
 * bssn_batch_get_state or bssn_batch_constraints return BSSN_ETIMEOUT. */
int32_t bssn_batch_tile_count(void);
const char* bssn_batch_tile_name(int32_t cfg);
bssn_status bssn_batch_set_tile(bssn_batch* b, int32_t cfg);
/* Autotuner for the persistent stage kernel: times each usable tile shape on
 * the batch's live members (launches of the first two stages, which leave y_n
 * unchanged) and selects the fastest; ms_per_cfg (bssn_batch_tile_count
 * entries, may be NULL) gets the mean milliseconds per stage launch, -1 for
 * the configurations the batch cannot use. */
bssn_status bssn_batch_autotune(bssn_batch* b, int32_t reps, int32_t* best, double* ms_per_cfg);
/* Test hook of the bounded wait (no counterpart in the paper), as
 * bssn_test_stall_tma for the batch's TMA-staged stage kernel: polls > 0 makes
 * every block issue no tile copy and give up after that many polls; the next
 * bssn_batch_get_state or bssn_batch_constraints returns BSSN_ETIMEOUT (and
 * clears the error word).  The member tables are re-uploaded in stream order;
 * the captured graph is kept, except under the per-member configurations,
 * whose launches carry the arguments themselves: their graph is captured
 * again at the next step.  polls in [0, 2^20]; 0 restores normal operation. */
bssn_status bssn_batch_test_stall_tma(bssn_batch* b, int32_t polls);

/* ------------------------------------------------------------- server
 * Continuous batching of evolution requests (no counterpart in the paper): a
 * scheduler thread admits queued requests at RK4 step boundaries while their
 * register bytes fit in hbm_budget_bytes, keeps their state on the device,
 * advances the resident evolutions together (bssn_batch_step; all of them,
 * or the shortest first: bssn_server_set_policy) and retires
 * each when it reaches its step count, reporting its constraint norms and
 * time from submission to completion.  d_pool (256-byte aligned) holds the
 * batch tables and every request's registers. */
bssn_status bssn_server_create(int32_t precision, size_t hbm_budget_bytes, void* d_pool,
                               size_t pool_bytes, void* cuda_stream, bssn_server** out);
/* Enqueue a request; never blocks.  EINVAL if it alone exceeds the budget or
 * its parameters are bad.  id_kind/id_p/np as for bssn_set_initial_data.  A
 * request that finds no free block of the pool at admission waits in the
 * queue until a resident request retires; with none resident it fails
 * (bssn_poll returns BSSN_ENOMEM). */
bssn_status bssn_submit(bssn_server* s, const bssn_params* p, int32_t id_kind, const double* id_p,
                        int32_t np, int32_t nsteps, uint64_t* ticket);
/* EAGAIN while queued or running; then BSSN_OK (norms_out as bssn_constraints,
 * *latency_s seconds from submit to completion) or BSSN_EFAILED when NaN/Inf
 * appeared in that request's state (other requests are unaffected). */
bssn_status bssn_poll(bssn_server* s, uint64_t ticket, double norms_out[16], double* latency_s);
/* Timing of a finished request: out[0] seconds from submission to completion
 * (as bssn_poll), out[1] seconds it waited in the queue before admission,
 * out[2] seconds resident on the device.  Returns as bssn_poll (EAGAIN while
 * queued or running, ENOTFOUND for an unknown ticket). */
bssn_status bssn_poll_detail(bssn_server* s, uint64_t ticket, double out[3]);
/* Which resident requests a step advances.
 *  - BSSN_SERVE_ALL (the default): every resident request, every step
 *    (processor sharing).
 *  - BSSN_SERVE_SHORTEST: shortest remaining work first.  Requests are
 *    ordered by remaining steps x interior points; the step advances the
 *    first ones until they hold at least min_points interior points (at
 *    least one request).  The others stay resident on the device and wait.
 *    The set changes only when a request is admitted or retired.
 * Each request's results are the same under either policy: the per-point
 * arithmetic does not depend on which members share a step.  EINVAL for an
 * unknown policy or min_points < 0. */
enum { BSSN_SERVE_ALL = 0, BSSN_SERVE_SHORTEST = 1 };
bssn_status bssn_server_set_policy(bssn_server* s, int32_t policy, double min_points);
/* The selection of BSSN_SERVE_SHORTEST on host arrays (no device work): of n
 * requests with remaining_work[i] and points[i], marks selected[i] = 1 for
 * the ones a step advances, 0 for the others; returns how many. */
int32_t bssn_serve_select(int32_t n, const double* remaining_work, const double* points, double min_points,
                          int32_t* selected);
/* out[0] completed, [1] failed, [2] queued, [3] resident, [4] interior
 * point-updates done, [5] seconds spent stepping, [6] seconds since create,
 * [7] bytes of the budget in use. */
bssn_status bssn_server_stats(bssn_server* s, double out[8]);
bssn_status bssn_server_destroy(bssn_server* s); /* stops the scheduler; synchronises */

/* Launch timing.  enable != 0: start recording CUDA events on the bound
 * stream around every fused stage launch and every boundary launch of
 * bssn_rk4_step (out unused).  enable == 0: stop, synchronise and write
 * out[0] = total stage-kernel milliseconds, out[1] = stage launches,
 * out[2] = total boundary-kernel milliseconds, out[3] = boundary launches. */
bssn_status bssn_profile(bssn_ctx* ctx, int32_t enable, double out[4]);

/* Test hook of the bounded wait (no counterpart in the paper).  The
 * TMA-staged stage kernels wait on an mbarrier for their tile copies, with a
 * poll limit after which they set the context's error word and return without
 * writing results.  With polls > 0 those kernels issue no copy at all and give
 * up after `polls` polls, so that this path runs without any copy in flight:
 * the next synchronising call (bssn_get_state, bssn_wait_state,
 * bssn_constraints) returns BSSN_ETIMEOUT and clears the error word; the
 * context stays usable.  polls in [0, 2^20]; 0 (the default) restores normal
 * operation.  Affects only the TMA-staged configurations of mixed contexts. */
bssn_status bssn_test_stall_tma(bssn_ctx* ctx, int32_t polls);

/* Measured arithmetic peak of the current GPU (no counterpart in the paper:
 * it is the denominator of the roofline on which the stage kernels are
 * placed, since the stencil path uses no tensor cores and is bound by the
 * float64 or float32 FMA pipe or by HBM).
 *  kind     0: float64 fused multiply-add, 1: float32 fused multiply-add.
 *  d_sink   caller-owned device memory of at least 8 bytes, 8-byte aligned;
 *           the kernel never actually writes it (it only could).
 *  reps     timed launches after one warm-up launch (each about 10 GFLOP).
 *  gflops   out: GFLOP/s, two flops per multiply-add, from CUDA events
 *           around the timed launches on cuda_stream.
 * Synchronises cuda_stream.  EINVAL on a bad argument, ECUDA on a CUDA
 * failure. */
bssn_status bssn_peak_probe(int32_t kind, void* d_sink, void* cuda_stream, int32_t reps, double* gflops);

/* Largest interior grid (n0 * n1 * n2) bssn_constraints_noalloc accepts. */
#define BSSN_NOALLOC_MAX_POINTS 4194304

/* Constraint norms without a bssn_alloc context and without allocating.  The
 * paper has no counterpart: this exists for callers that may not allocate
 * device memory themselves or hand the library a block -- a host that owns all
 * of HBM through its own arena, a plug-in host that forbids its plug-ins to
 * allocate, a real-time loop that must not call cudaMalloc (which can
 * synchronise the device) -- yet hold a state buffer and want its norms.
 *  p        grid and method parameters (as for bssn_alloc); at most
 *           BSSN_NOALLOC_MAX_POINTS interior points, else EINVAL.
 *  d_state  float64 register in the layout of bssn_layout_of(p), ghosts valid.
 *  punct    host array of npunct x {m, x, y, z} (npunct 0..8) defining the
 *           excised set, as set_initial_data does for Brill-Lindquist data.
 *  out      host array of 16 doubles, same order as bssn_constraints.
 * Synchronises cuda_stream.  The reduction scratch is a fixed static device
 * array (2.25 MiB) that every GPU which loads the library holds until exit;
 * its device address is looked up on the first call made on each device, so
 * make that first call before any stream capture (a lookup that fails returns
 * ECUDA and is tried again on the next call).  All calls on a device share
 * that array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
bssn_status bssn_constraints_noalloc(const bssn_params* p, const double* d_state,
                                     const double* punct, int32_t npunct, void* cuda_stream,
                                     double out[16]);

#ifdef __cplusplus
}
#endif
#endif /* BSSN_H */
