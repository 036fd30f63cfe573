/*
 * ib_pf.h -- C ABI of the GB300 (sm_103a) hot path of the fully Eulerian hybrid
 * immersed-boundary / phase-field method for contact lines on complex walls
 * (Shahmardi, Rosti, Tammisola & Brandt, arXiv 2104.00350).
 *
 * One call of ib_pf_step advances every instance of a context by one or more time
 * steps of the scheme of Sec. 4.2 and Appendix A:
 *   a1 Cahn-Hilliard right-hand side            (Appendix A.1, Eq. Helmholtz1)
 *   a2 the two Helmholtz solves, one eigenbasis (Eqs. Helmholtz1, Helmholtz2)
 *      (a1 + a2 are the explicit AB2 update of Eq. ExpCH instead when
 *       ib_pf_params.ch_scheme = IB_PF_CH_EXPLICIT)
 *   a3 contact-angle ghost fill of C            (Eqs. interpolationAtWall, ProjectingToNT,
 *                                                UpdateC, static form of Eq. WallBCS)
 *   a4 chemical potential + ghost fill          (Eq. Chemical-Potential, Sec. 4.2.2)
 *   a5 AB2 momentum predictor + penalisation    (Eqs. PredictionExp, Penalization2)
 *   a6 slip / no-penetration ghost fill         (Eqs. NoPenetration, UpdateVtan, UpdateVandW)
 *   a7 Dodd-Ferrante pressure Poisson           (Eq. PressurePoisson)
 *   a8 velocity correction                      (Eq. correction)
 * The geometry precompute of Sec. 4.1 (volume fractions, normals, ghost / intersect /
 * mirror / interpolation points, weights W1/W2) runs once on the device in
 * ib_pf_init_geometry and ib_pf_precompute_weights.
 *
 * Grid and layout.  2D uniform staggered Cartesian grid, nx x ny cells of size h
 * (lx/nx must equal ly/ny), periodic in x1, solid walls (v = 0) at x2 = 0 and x2 = ly.
 * nx and ny must be powers of two, 8 <= nx <= 4096, 8 <= ny <= 2048.  All fields are
 * row-major with x1 fastest: cell fields (C, P, phi) are ny x nx; x1-face fields (u, Hu)
 * are ny x nx with face i the left face of cell i; x2-face fields (v, Hv) are
 * (ny+1) x nx with rows 0 and ny on the domain walls (always zero).
 *
 * 3D (dim 3).  nx x ny x nz cubic cells, periodic in x and y, solid walls (w = 0) at
 * z = 0 and z = lz; nx, ny, nz powers of two, 8 <= n <= 1024.  Cell fields and the x-/y-face
 * fields (u, v, Hu, Hv) are nz x ny x nx (x fastest; u face i is the left face of cell i, v
 * face j the front face of cell j); z-face fields (w, Hw) are (nz+1) x ny x nx with planes 0
 * and nz on the domain walls.  The 3D step is the 2D one with the third axis: 7-point
 * stencils, 7 averaging points per interpolation point, the full stress tensor, the slip
 * condition in vector form (V_t = u - (u.n) n).
 *
 * Element type.  The element type of every field buffer passed in or out is the
 * context's arithmetic type (double for IB_PF_FP64, float for IB_PF_FP32), except the
 * wall values IB_PF_F_C_I, which are double in both.
 *
 * Errors.  Every call returns an ib_pf_status; nothing aborts, traps the device or exits.
 * The last error message of a context is kept (ib_pf_last_error).  Device-detected
 * non-finite values set a status word that the next synchronising call returns as
 * IB_PF_E_NUMERIC; a 3D transform tile whose copies fail their alignment check (an internal
 * error: no layout of the library produces one) is skipped and sets another bit, returned
 * as IB_PF_E_CUDA.  A context is not thread-safe; separate contexts are independent.
 * All device work is issued on the stream given at creation (0 = legacy default).
 */
#ifndef IB_PF_H
#define IB_PF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ib_pf_ctx ib_pf_ctx;   /* opaque; owned by the library */

typedef enum {
  IB_PF_OK = 0,
  IB_PF_E_ARG = -1,          /* invalid argument (sizes, ids, null pointers, params) */
  IB_PF_E_UNSUPPORTED = -2,  /* valid but not implemented (e.g. dynamic angle) */
  IB_PF_E_CUDA = -3,         /* a CUDA runtime call failed; see ib_pf_last_error */
  IB_PF_E_NUMERIC = -4,      /* NaN/Inf seen in C or the velocity by the device check */
  IB_PF_E_TIMEOUT = -5,      /* a bounded device wait gave up (the tensor-core z solve of
                                FP32_3XBF16 contexts waits on its MMAs for at most 2 s) */
  IB_PF_E_STATE = -6,        /* call out of order (e.g. step before precompute) */
  IB_PF_E_GEOMETRY = -7      /* precompute failed (no intersect point within 10 h) */
} ib_pf_status;

/* arithmetic of a context: FP64 throughout; FP32 fields and transforms (geometry, weights and
 * the mass of C in FP64, C held as a compensated pair); FP32_3XBF16: the FP32 form with the
 * wall-normal (z) solve of the 3D Cahn-Hilliard and Poisson problems (Appendix A.1,
 * Eq. PressurePoisson) done as dense cosine-transform products on the tensor cores, every
 * operand split into two BF16 parts and three products accumulated in FP32 (about 16
 * significant bits per transform instead of FP32's 24); 3D contexts with nz = 128 or 256
 * only (other grids and 2D contexts return IB_PF_E_UNSUPPORTED).  Field buffers, tables and
 * I/O of an FP32_3XBF16 context are those of an FP32 one. */
typedef enum { IB_PF_FP64 = 0, IB_PF_FP32 = 1, IB_PF_FP32_3XBF16 = 2 } ib_pf_precision;

/* time integration of the Cahn-Hilliard equation (rows a1 + a2): SEMI_IMPLICIT, the
 * stabilised split of Appendix A.1 solved in one eigenbasis; EXPLICIT, the Adams-Bashforth
 * update of Eq. ExpCH, C^{n+1} = C^n + dt (3/2 F^n - 1/2 F^{n-1}) with
 * F = -div(u C) + (1/Pe) lap(phi), F^{n-1} taken from the level n-1 fields (C^{n-1},
 * u^{n-1}, v^{n-1} (w^{n-1}) and phi(C^{n-1}) with its ghost fill); no transform.  The
 * explicit time step is limited by about dt < Pe h^4 / (4 D Cn^2) and dt < Pe h^2 / (4 D)
 * (D = 2 or 3), which the library does not check. */
typedef enum { IB_PF_CH_SEMI_IMPLICIT = 0, IB_PF_CH_EXPLICIT = 1 } ib_pf_ch_scheme;

/* averaging weights W1/W2 of the ghost-cell gathers (Sec. 4.1.4).  IDW: the normalised
 * inverse-squared-distance weights of Eq. weright averaged (Shepard's average: constants are
 * reproduced, linear fields only on stencils symmetric about the interpolation point).
 * LINEAR: the same weight function with a linear basis (moving least squares,
 * W_i = w_i (1 + (d_i - xb) . S^{-1} (-xb)), xb = sum w_i d_i, S = sum w_i (d_i - xb)(d_i - xb)^T,
 * d_i the offset of averaging point i from the interpolation point), which reproduces
 * linear fields exactly; where the kept averaging points are all on one line (2D) or in one
 * plane (3D) the IDW weights are used.  LINEAR is the default (0). */
typedef enum { IB_PF_W_LINEAR = 0, IB_PF_W_IDW = 1 } ib_pf_weights;

/* momentum predictor (row a5): EXPLICIT, the Adams-Bashforth step of Eq. PredictionExp;
 * SEMI_IMPLICIT, Eq. predictionSemi of Appendix A.2: u* = u^n + d with
 * (1 - (dt nu0/2) L) d = dt [3/2 N^n - 1/2 N^{n-1} + ST + V^n + MF], N = -div(u u) (the history
 * fields H then hold N only), V^n the viscous term at level n, nu0 = (mu_l/rho_l +
 * mu_g/rho_g)/(2 Re), MF = ((rho_l - rho_g)/(2 rho Pe)) (grad phi . grad) u the mass-flux
 * consistency term, solved per component with Fourier x cosine-type transforms (DST-II
 * for u, DST-I for v); 2D contexts only.  All instances of a context share it. */
typedef enum { IB_PF_NS_EXPLICIT = 0, IB_PF_NS_SEMI_IMPLICIT = 1 } ib_pf_ns_scheme;

/* wall kinds: the solid is where the predicate holds (Sec. 4.1.1 counts subgrid points
 * against it).  FLAT: x2 < p[0] (2D), z < p[0] (3D).  SINUSOID (2D): x2 < p[0] + p[1]
 * sin(2 pi p[2] x1).  SPHERE (3D): |x - (p[0], p[1], p[2])| < p[3].  SPHERES (3D): the union
 * of the spheres (cx, cy, cz, r) of ib_pf_geometry.spheres.  NONE: no solid.  Sphere
 * distances take the nearest periodic image in x and y.
 * MASK (2D and 3D): a solid with no analytic form, given by its volume fractions
 * (ib_pf_geometry.alpha), which replace the subgrid count of Sec. 4.1.1; the solid is where
 * the cell-centre fractions, interpolated linearly between cell centres (bilinear in 2D,
 * trilinear in 3D; periodic in x (and y), the first and last centre rows (planes) continued
 * beyond them), are below 1/2, which decides the solid cell centres and the intersect
 * points of Sec. 4.1.2. */
typedef enum {
  IB_PF_WALL_FLAT = 0, IB_PF_WALL_SINUSOID = 1, IB_PF_WALL_NONE = 3, IB_PF_WALL_SPHERE = 4,
  IB_PF_WALL_SPHERES = 5, IB_PF_WALL_MASK = 6
} ib_pf_wall_kind;

typedef struct {
  int dim;        /* 2 or 3; all instances of a context share it */
  int n[3];       /* cells per axis: n[0] = nx, n[1] = ny, n[2] = nz (3D) */
  double L[3];    /* domain lengths */
} ib_pf_grid;

typedef struct {
  int kind;       /* ib_pf_wall_kind */
  double p[8];    /* wall parameters, see above */
  const double* spheres;   /* SPHERES: host array of n_spheres x (cx, cy, cz, r), copied by
                              ib_pf_init_geometry (the caller keeps ownership); else NULL */
  int n_spheres;
  const double* alpha;     /* MASK: host array of the fluid volume fractions, in [0, 1], of
                              the control volumes in the layout of the alpha tables
                              (IB_PF_T_ALPHA_*), back to back: 2D alpha_c (ny x nx), alpha_u
                              (ny x nx), alpha_v ((ny+1) x nx); 3D alpha_c, alpha_u, alpha_v
                              (nz x ny x nx each), alpha_w ((nz+1) x ny x nx).  Copied by
                              ib_pf_init_geometry (the caller keeps ownership); else NULL. */
} ib_pf_geometry;

/* Nondimensional parameters as defined in Sec. 5.1 (Re, Ca, Cn) and Sec. 5.3 (Pe);
 * S is the stabilisation of Appendix A.1; rho_ratio and mu_ratio are liquid/gas with the
 * liquid (C = +1) at rho = mu = 1; theta_deg the static contact angle measured through
 * the liquid; l_s the slip length of Eq. SlipVelocity; mu_f the wall friction of
 * Eq. WallBCS, nondimensional as in (dC/dt + v_t dC/dx_t)_I = (1/(mu_f Cn)) [kappa Cn dC/dn +
 * cos(theta) g'(C_I)] (Eq. WallBCS_recast): 0 = static angle (the wetting condition holds
 * at every step), > 0 = dynamic angle with the wall values C_I as per-ghost state advanced
 * implicitly by one step per time step, and the wetting bracket in the slip condition (Eq.
 * UpdateVtan); d1, d2 the ghost-cell lengths of Sec. 4.1.2 (d1 > half a cell diagonal,
 * 0 < d2 < d1); dt the time step. */
typedef struct {
  double Re, Ca, Cn, Pe, S, rho_ratio, mu_ratio, theta_deg, l_s, mu_f, d1, d2, dt;
  int precision;  /* ib_pf_precision */
  int ch_scheme;  /* ib_pf_ch_scheme; all instances of a context share it */
  int weights;    /* ib_pf_weights (per instance) */
  int ns_scheme;  /* ib_pf_ns_scheme; all instances of a context share it */
} ib_pf_params;

/* field ids for read / write */
typedef enum {
  IB_PF_F_C = 0,        /* C^n            (cells)  read/write */
  IB_PF_F_C_OLD = 1,    /* C^{n-1}        (cells)  read/write */
  IB_PF_F_U = 2,        /* u^n            (x1-faces) read/write */
  IB_PF_F_U_OLD = 3,    /* u^{n-1} */
  IB_PF_F_V = 4,        /* v^n            (x2-faces) read/write */
  IB_PF_F_V_OLD = 5,    /* v^{n-1} */
  IB_PF_F_HU = 6,       /* H_u^{n-1}: AB2 history of Eq. PredictionExp, read/write */
  IB_PF_F_HV = 7,
  IB_PF_F_P = 8,        /* P^n            (cells)  read/write */
  IB_PF_F_P_OLD = 9,    /* P^{n-1} */
  IB_PF_F_PHI = 10,     /* chemical potential of the last step (cells), read only */
  IB_PF_F_Q = 11,       /* CH right-hand side of the last step, increment form (cells):
                           R = Q - (L^2 - (S/Cn^2) L + c0) B, B = (2C^n - C^{n-1}/2)/1.5;
                           read only */
  IB_PF_F_RHS_P = 12,   /* Poisson right-hand side of the last step for the increment
                           P^{n+1} - (2P^n - P^{n-1}) (cells), read only */
  IB_PF_F_C_LO = 13,    /* FP32 contexts only: low part of the compensated C^n (C^n is held
                           as the unevaluated sum C + C_LO); read/write, for restarts.
                           Writing IB_PF_F_C clears it. */
  IB_PF_F_C_OLD_LO = 14, /* FP32 contexts only: low part of C^{n-1} */
  IB_PF_F_W = 15,       /* 3D: w^n (z-faces) read/write */
  IB_PF_F_W_OLD = 16,   /* 3D: w^{n-1} */
  IB_PF_F_HW = 17,      /* 3D: H_w^{n-1} */
  IB_PF_F_C_I = 18      /* dynamic angle (mu_f > 0): the wall values C_I at the intersect points,
                           one per ghost in ghost order (IB_PF_T_GHOST_CELL), double in both
                           forms; read/write for restarts.  NaN = unset: a write of IB_PF_F_C
                           unsets them and the next step starts them from the field,
                           (gamma C_G + C_M)/(gamma + 1) */
} ib_pf_field;

/* geometry tables for ib_pf_read_table (element type in brackets) */
typedef enum {
  IB_PF_T_ALPHA_C = 0,  /* [double] ny x nx      fluid volume fraction, cell volumes */
  IB_PF_T_ALPHA_U = 1,  /* [double] ny x nx      x1-face volumes */
  IB_PF_T_ALPHA_V = 2,  /* [double] (ny+1) x nx  x2-face volumes */
  IB_PF_T_CLASS = 3,    /* [int]    ny x nx      0 fluid, 1 ghost, 2 solid */
  IB_PF_T_GHOST_CELL = 4, /* [int]  ng           linear cell index j*nx+i, ascending */
  IB_PF_T_NORMAL = 5,   /* [double] ng x 2       unit normal, solid -> fluid */
  IB_PF_T_DN = 6,       /* [double] ng           ghost-to-intersect distance */
  IB_PF_T_GAMMA = 7,    /* [double] ng           d1 / dn */
  IB_PF_T_AP1 = 8,      /* [int]    ng x 5       averaging cells around IP1 */
  IB_PF_T_W1 = 9,       /* [double] ng x 5       weights W1 (sum 1) */
  IB_PF_T_AP2 = 10,     /* [int]    ng x 5 */
  IB_PF_T_W2 = 11,      /* [double] ng x 5 */
  IB_PF_T_FACE_U = 12,  /* [int]    nfu          re-interpolated x1-faces (j*nx+i) */
  IB_PF_T_FACE_V = 13,  /* [int]    nfv          re-interpolated x2-faces (j*nx+i) */
  IB_PF_T_ALPHA_W = 14, /* 3D: [double] (nz+1) x ny x nx  z-face volumes */
  IB_PF_T_FACE_W = 15   /* 3D: [int] nfw  re-interpolated z-faces ((k*ny+j)*nx+i) */
} ib_pf_table;
/* In 3D the cell and face tables are nz x ny x nx (alpha_v too), linear indices are
 * (k*ny + j)*nx + i, normals are ng x 3 and the averaging stencils ng x 7. */

/* quantities for ib_pf_query */
typedef enum {
  IB_PF_Q_MASS = 0,        /* sum of C^n over all cells, FP64, fixed-order reduction */
  IB_PF_Q_N_GHOST = 1,
  IB_PF_Q_N_FACE_U = 2,
  IB_PF_Q_N_FACE_V = 3,
  IB_PF_Q_STATUS = 4,      /* device status word: 0 ok, bit 1 non-finite seen, bit 2 a 3D
                              transform tile failed its alignment check */
  IB_PF_Q_STEPS = 5,       /* steps taken since creation */
  IB_PF_Q_N_FALLBACK = 6,  /* normals or averaging stencils that used the fallback */
  IB_PF_Q_LAUNCHES_PER_STEP = 7, /* kernels one step launches */
  IB_PF_Q_N_FACE_W = 8           /* 3D: re-interpolated z-faces */
} ib_pf_query_id;

/* Create a context for n_instances independent problems (grids[k], geoms[k],
 * params[k]) and run the first part of the precompute of Sec. 4.1: volume fractions of
 * the cell and face control volumes by counting 100 x 100 subgrid points per volume in 2D,
 * 16 x 16 x 16 in 3D (Sec. 4.1.1),
 * ghost classification (cell centre in the solid with a fluid face neighbour, Sec.
 * 4.1.2) and compaction, and the list of faces re-interpolated after the velocity ghost
 * fill.  Fields start at zero.  `cuda_stream` is a cudaStream_t (NULL = default stream);
 * the call synchronises it.  On success *out owns all device memory of the context. */
ib_pf_status ib_pf_init_geometry(ib_pf_ctx** out, int n_instances, const ib_pf_grid* grids,
                                 const ib_pf_geometry* geoms, const ib_pf_params* params,
                                 void* cuda_stream);

/* Second part of the precompute (Sec. 4.1.2-4.1.4), in FP64 on the device: normals from
 * corner gradients of alpha (Eqs. NormalVectors_part1/2), intersect points by marching
 * h/100 along the normal plus 60 bisections, mirror point M = I + d1 n, interpolation
 * points IP1 = M + d2 n, IP2 = M + 2 d2 n, averaging points and inverse-squared-distance
 * weights W1/W2 (Eq. weright averaged).  Synchronises the stream.  Returns
 * IB_PF_E_GEOMETRY if some ghost has no intersect point within 10 h. */
ib_pf_status ib_pf_precompute_weights(ib_pf_ctx* ctx);

/* Advance every instance by nsteps time steps (a1..a8 above).  Asynchronous on the
 * context stream: the steps are replayed from captured CUDA graphs.  Returns
 * IB_PF_E_STATE before ib_pf_precompute_weights, IB_PF_E_NUMERIC if an earlier step's
 * device check saw a non-finite value (the check is read back without blocking). */
ib_pf_status ib_pf_step(ib_pf_ctx* ctx, int nsteps);

/* Copy field `field_id` of `instance` into dst (nbytes must equal the field size in the
 * context's element type).  dst_on_host != 0: dst is host memory and the call
 * synchronises the stream; otherwise dst is device memory and the copy is stream-ordered. */
ib_pf_status ib_pf_read_fields(ib_pf_ctx* ctx, int instance, int field_id, void* dst,
                               long long nbytes, int dst_on_host);

/* Copy src into state field `field_id` of `instance` (restart / initial condition).
 * Only the read/write ids above are accepted.  src_on_host as for ib_pf_read_fields.
 * Rows 0 and ny of v fields (2D) and planes 0 and nz of w fields (3D) are forced to zero;
 * writing C or C_old in the FP32 form clears its low part.  Device sources and pinned
 * (page-locked) host sources are read by one copy kernel on the work stream; other host
 * memory goes through cudaMemcpyAsync.  Clears the instance's non-finite status and
 * synchronises the stream; src may be reused when the call returns. */
ib_pf_status ib_pf_write_fields(ib_pf_ctx* ctx, int instance, int field_id, const void* src,
                                long long nbytes, int src_on_host);

/* Batched field I/O: entry q of the arrays is one ib_pf_write_fields / ib_pf_read_fields
 * (instances[q], field_ids[q], bufs[q], nbytes[q]) with the same checks and effects, as if
 * the entries ran in order (a later write of the same field wins; C_lo written after C
 * keeps the written low part).  Copies from or to device or pinned host memory go to one
 * copy kernel launch per 48 entries (other host memory: cudaMemcpyAsync); the destination
 * buffers of one read batch must not overlap.  The call synchronises once at the end
 * (writes always, reads when on_host != 0) instead of once per field.  Entries are validated before
 * anything is queued: one bad entry fails the whole call with IB_PF_E_ARG and nothing is
 * copied.  n = 0 is a no-op. */
ib_pf_status ib_pf_write_fields_batch(ib_pf_ctx* ctx, int n, const int* instances,
                                      const int* field_ids, const void* const* srcs,
                                      const long long* nbytes, int src_on_host);
ib_pf_status ib_pf_read_fields_batch(ib_pf_ctx* ctx, int n, const int* instances,
                                     const int* field_ids, void* const* dsts,
                                     const long long* nbytes, int dst_on_host);

/* Copy geometry table `table_id` of `instance` to host memory.  If dst is NULL only the
 * element count is returned in *count; otherwise nbytes must match.  Synchronises. */
ib_pf_status ib_pf_read_table(ib_pf_ctx* ctx, int instance, int table_id, void* dst,
                              long long nbytes, long long* count);

/* Scalar diagnostics (ib_pf_query_id) of `instance`.  Synchronises the stream. */
ib_pf_status ib_pf_query(ib_pf_ctx* ctx, int instance, int what, double* out);

/* Schedule choices of a 3D instance (0 = the built-in default).
 *   y_tile_bytes, z_tile_bytes  row bytes of the column tiles of the y transforms and of the
 *                               z solve: 128 (transform lengths <= 512) or 64 (lengths >= 256;
 *                               the default from 1024 points on, 128 below)
 *   predict_planes              planes each predictor block marches through: 8, 16 (default)
 *                               or 32 (capped at nz)
 * The choices change the schedule only; results are the same bit for bit (each kernel's
 * arithmetic per point is fixed). */
typedef struct {
  int y_tile_bytes;
  int z_tile_bytes;
  int predict_planes;
} ib_pf_tuning;

/* Sets the schedule of 3D instance `instance` (IB_PF_E_ARG for a value not listed above or
 * not built for the instance's lengths; IB_PF_E_UNSUPPORTED for a 2D context, whose batched
 * kernels have fixed tiles).  The step graphs are recaptured at the next step. */
ib_pf_status ib_pf_set_tuning(ib_pf_ctx* ctx, int instance, const ib_pf_tuning* t);
ib_pf_status ib_pf_get_tuning(ib_pf_ctx* ctx, int instance, ib_pf_tuning* t);

/* Autotuner (3D): times every built candidate of each choice on instance `instance` -- the
 * y transforms and the z solve on the instance's spectral scratch, the predictor on its own
 * state with the AB2 history (Hu, Hv, Hw) saved before and restored after -- `reps` launches
 * each after one warm-up, and sets the fastest.  The state after the call equals the state
 * before.  chosen (may be NULL) receives the choice; times_ms (may be NULL) the mean ms per
 * launch of the candidates in the order y 128, y 64, z 128, z 64, planes 8, 16, 32 (-1 for a
 * candidate not built for the lengths), 7 values.  Synchronises the stream; allocates a
 * scratch copy of the history for the duration of the call.  The caller may cache the choice
 * (the Python binding keeps a JSON file keyed by grid shape, precision and GPU name). */
ib_pf_status ib_pf_autotune(ib_pf_ctx* ctx, int instance, int reps, ib_pf_tuning* chosen,
                            double* times_ms);

/* Per-kernel timing.  enable != 0 recaptures the step graphs with a CUDA event recorded
 * on the work stream before the first kernel of a step and after every kernel; enable = 0
 * restores the plain graphs.  Timing adds the event records to the step, nothing else. */
ib_pf_status ib_pf_set_kernel_timing(ib_pf_ctx* ctx, int enable);

/* Durations (ms) of the kernels of the last completed step, in launch order over all
 * instances, with their kernel names (static strings owned by the library).  Requires
 * ib_pf_set_kernel_timing(ctx, 1) before that step; synchronises the stream.  At most cap
 * entries are written; *n receives the number of kernels of one step. */
ib_pf_status ib_pf_kernel_times(ib_pf_ctx* ctx, int cap, double* ms, const char** names, int* n);

/* Pressure Poisson solve that allocates no device memory.  The paper has no counterpart:
 * this entry point exists for callers that must not call cudaMalloc once they are running,
 * e.g. code whose device memory is owned by another framework's caching allocator, or a
 * time-critical loop where an allocation could synchronise the device or fail under
 * memory pressure.  It solves the same discrete problem as step a7 of ib_pf_step (5-point
 * Laplacian, periodic x1, zero-gradient x2 walls, mean mode set to zero): out = L^{-1} rhs
 * for one nx x ny FP64 cell field with spacing h.  rhs and out are caller-owned device
 * pointers (row-major, x1 fastest); work is queued on cuda_stream (NULL = default stream)
 * and the call returns without synchronising.
 * Limits: nx, ny powers of two, 8 <= nx, ny <= 1024, nx * ny <= 524288; larger grids
 * return IB_PF_E_ARG with a message in ib_pf_last_error(NULL).
 * Scratch: one fixed file-scope device array of about 4.3 MB that every GPU loading the
 * library holds until the process exits.  The first call on each device looks up the
 * array's device address and keeps it for the life of the process; make that first call
 * before any stream capture, and restart the process after a cudaDeviceReset before
 * calling again.  All calls share the array, so calls that may overlap on the GPU
 * (different streams, or threads) race and must be serialised by the caller.  A CUDA error
 * already pending on the calling thread makes the call return IB_PF_E_CUDA without
 * queueing work (the error is left in place). */
ib_pf_status ib_pf_poisson_solve_noalloc(const double* rhs, double* out, int nx, int ny,
                                         double h, void* cuda_stream);

/* Bind caller-owned device memory (e.g. a torch CUDA tensor) as the storage of a state
 * field of `instance`, in place of the buffer the library allocated (which is freed).
 * The state of the scheme is what the step reads and writes (Sec. 4.2 and Appendix A: C,
 * u, v (w), P at levels n and n-1 and the Adams-Bashforth history H); the library keeps
 * the two buffers of a two-level field and swaps their roles every step.
 *   field_id  IB_PF_F_C, IB_PF_F_U, IB_PF_F_V, IB_PF_F_P, IB_PF_F_W (3D) and, in FP32
 *             contexts, IB_PF_F_C_LO: time_level 0 binds the buffer that holds level n at
 *             the time of the call, 1 the one that holds level n-1 (after a step the two
 *             have swapped roles: read the levels through ib_pf_read_fields or keep the
 *             step parity);  IB_PF_F_HU, IB_PF_F_HV, IB_PF_F_HW (3D): time_level 0.
 *   device_ptr device (or managed) memory of the context's element type, 16-byte aligned,
 *             nbytes = the field size (layout as above); it must not alias another bound
 *             field.  Its current content becomes the field's value (nothing is copied),
 *             except that the wall rows of v (planes of w) are set to zero.
 * The caller keeps ownership: ib_pf_destroy does not free bound buffers, and they must
 * stay valid until the context is destroyed or the field is bound again.  The call
 * synchronises the context stream and rebuilds the step graphs (not for hot loops).
 * Errors: IB_PF_E_ARG (ids, size, alignment, not device memory), IB_PF_E_CUDA. */
ib_pf_status ib_pf_bind_fields(ib_pf_ctx* ctx, int instance, int field_id, int time_level,
                               void* device_ptr, long long nbytes);

/* Last error message of ctx (or of the last failed creation when ctx is NULL). */
const char* ib_pf_last_error(const ib_pf_ctx* ctx);

/* Free every resource of ctx (device memory, graphs).  Synchronises its stream. */
void ib_pf_destroy(ib_pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* IB_PF_H */
