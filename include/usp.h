/*
 * usp.h -- C ABI of the GB300 (sm_103a) USP-FPM particle-update library.
 *
 * The library advances a population of diatomic (N2-like) simulation
 * particles with the unified stochastic particle Fokker-Planck-Master method
 * of Kim & Jun, "A second-order particle Fokker-Planck-Master method for
 * diatomic gas flows" (arXiv 2508.05642).  One step is the collision step of
 * the paper's Sec. 4.D for every cell: cell moments (Sec. 2.A), per-cell
 * coefficients alpha, nu, gamma (Sec. 3.A.1-3.A.2, Eqs. USP-FPM_alpha_tr,
 * USP-FPM_nu, e_tr_relax .. e_vib_relax), the particle updates of velocity
 * (Eq. update_ci with Eq. D_tr and the positivity fix of Sec. 3.A.3),
 * rotational energy (Eq. update_erot) and vibrational level (Eq. update_evib),
 * then the conservation scheme of Sec. 4.C.
 *
 * Conventions shared by every entry point:
 *  - All particle data is structure-of-arrays.  Velocities c_x, c_y, c_z are
 *    in m/s, the rotational energy is specific (J/kg), the vibrational level
 *    is a non-negative int32.
 *  - A "cell" of the homogeneous problem is an independent relaxation
 *    instance; its particles are the contiguous range
 *    [offsets[i], offsets[i+1]) of the caller's arrays.
 *  - Pointers named h_* are host memory, d_* device memory.  The library
 *    copies what it needs; it never keeps or frees a caller pointer.
 *  - Device memory is owned by the context: taken from the caller's
 *    allocator callback when one is given (released through its free
 *    callback), else from cudaMalloc.  usp_destroy releases all of it.
 *  - Work is enqueued on the context's CUDA stream and returns without
 *    waiting, except where a function says it synchronises.
 *  - Every function returns USP_OK (0) or a negative usp_err.  A failing CUDA
 *    call returns USP_ECUDA; invalid arguments return USP_EINVAL and change
 *    nothing.  Numerical events inside the step do not stop it: they set bits
 *    of a sticky device status word read by usp_status.
 */
#ifndef USP_H
#define USP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  USP_OK = 0,
  USP_EINVAL = -1,   /* invalid argument                                   */
  USP_ENOMEM = -2,   /* allocation failed                                  */
  USP_ECUDA = -3,    /* a CUDA runtime call failed                         */
  USP_EDEVICE = -4,  /* the device status word has an error bit set        */
  USP_ENOTSUP = -5   /* the request is not supported by this context       */
} usp_err;

/* Device status bits (usp_status).  Bits 0x40, 0x80, 0x200, 0x400 and 0x1000
 * are errors; the others report clamps the method applies and continues. */
enum {
  USP_F_PB_CLAMP = 0x01,            /* p_B > 1 met (Sec. 3.A.2): binomial clamped to n   */
  USP_F_CHOL_FAIL_AFTER_FIX = 0x02, /* T_tr^rel = 0 at the nu = 0 end of the Sec. 3.A.3
                                       fix: no diffusion for that particle (a clamp)    */
  USP_F_NEG_RADICAND = 0x04,        /* velocity rescale of Sec. 4.C impossible; skipped  */
  USP_F_VIB_LOOP_CAP = 0x08,        /* vibrational +-1 correction hit 64 N draws         */
  USP_F_TREL_CLAMP = 0x10,          /* a relaxation temperature or energy target came
                                       out negative and was set to 0                    */
  USP_F_SAMPLER_CAP = 0x20,         /* a jump-sampler search hit 4096 steps              */
  USP_F_A_NONPOS = 0x40,            /* A outside (-1, 1): mu/p of a cell not finite > 0  */
  USP_F_SAMPLER_UNDERFLOW = 0x80,   /* jump pmf underflowed double                       */
  USP_F_WALL_CAP = 0x100,           /* a particle met 16 wall events in one step         */
  USP_F_BOUNDS = 0x200,             /* an index check failed (kernel skipped the access) */
  USP_F_WAIT_TIMEOUT = 0x400,       /* a device-side wait gave up after its time limit  */
  USP_F_INFLOW_CAP = 0x800,         /* an inflow normal-speed draw hit 64 attempts       */
  USP_F_CAPACITY = 0x1000           /* particle storage full: inflow of a step dropped   */
};

/* Counter slots of usp_status. */
enum {
  USP_C_CHOL_FIX = 0,      /* positivity fixes applied (per cell and step)       */
  USP_C_PB_CLAMP = 1,      /* particles whose p_B exceeded 1                      */
  USP_C_TREL_CLAMP = 2,    /* relaxation-temperature clamps                      */
  USP_C_VIB_DRAWS = 3,     /* random draws made by the +-1 level correction      */
  USP_C_NEG_RADICAND = 4,  /* cells whose velocity rescale was skipped           */
  USP_C_WALL_HITS = 5,
  USP_C_INTERP_FALLBACK = 6,
  USP_C_SKIPPED_CELLS = 7, /* cells with fewer than two particles (not collided) */
  USP_C_INFLOW = 8,        /* particles generated at inflow faces (plane path)  */
  USP_C_OUTFLOW = 9,       /* particles removed at open sides (plane path)      */
  USP_C_NU_ZERO = 10,      /* positivity fixes that ended at nu = 0             */
  USP_NCOUNTERS = 11
};

/* Number of per-cell moments written by usp_moments, field-major
 * (out[f * n_cells + cell]):
 *   0 N | 1-3 U (m/s) | 4 T_tr | 5 T_rot | 6 T_vib (K) |
 *   7-12 Pi_ij = <C_i C_j> (xx yy zz xy xz yz, m^2/s^2) |
 *   13-15 q_tr = <C^2 C>/2 | 16-18 q_rot = <C eps_rot> | 19-21 q_vib = <C I R Theta>
 * (heat fluxes per unit mass, m^3/s^3; multiply by rho for W/m^2).  These are
 * the moments of Sec. 2.A with ensemble averages taken as 1/N sample means;
 * T_vib inverts e_vib of Sec. 2.A at the mean level (0 for no excitation). */
#define USP_NMOM 22

/* Forms: USP_FP64 plain FP64 state and arithmetic; USP_FP32 FP32 particle
 * state and per-particle arithmetic with FP64 cell sums and coefficients;
 * USP_FP64_TANGENT (channel contexts only) the FP64 form carrying, for every
 * continuous quantity, its derivatives with respect to Z_rot, the viscosity
 * index omega and T_wall (forward-mode pathwise derivatives under common
 * random numbers; discrete outcomes, wall-event times and positions held
 * fixed); USP_FP32_TANGENT (channel contexts only) the same derivatives with
 * the FP32 form's particle state and per-particle arithmetic (values and
 * derivatives in FP32) and FP64 cell quantities, sums and time averages
 * (FP64 accumulation of the derivatives). */
enum { USP_FP64 = 0, USP_FP32 = 1, USP_FP64_TANGENT = 2, USP_FP32_TANGENT = 3 };

/* Particle method (usp_config.method, homogeneous contexts):
 * USP_METHOD_USP_FPM  the second-order USP-FPM method (Sec. 3, 4), default;
 * USP_METHOD_FPM      the first-order FPM method it extends (Sec. 2.B model,
 *                     Sec. 2.C scheme): alpha = exp(-dt/tau),
 *                     tau = 2 mu (1 - nu)/p, nu = 1 - 3/(2 Pr), relaxation
 *                     temperatures of Eqs. T_tr_FPM .. T_vib_FPM, Gillespie's
 *                     direct method for the vibrational levels (draws: Philox
 *                     counter (particle id, step, 8, k), two transitions per
 *                     block), and the conservation scheme of Sec. 4.C with the
 *                     expected mode energies after dt as targets.  When
 *                     tau D_tr is not positive definite, nu is limited to the
 *                     admissible bound of Eq. nu_USP_positivity, then set to 0. */
enum { USP_METHOD_USP_FPM = 0, USP_METHOD_FPM = 1 };

/* Gas species.  VSS/VHS viscosity parameters of Sec. 4.A; theta_v of the
 * harmonic vibrational model (Sec. 2.A); zmodel 0 uses the fixed collision
 * numbers Z_rot, Z_vib (Sec. 2.A), zmodel 1 the Parker and Millikan-White /
 * high-temperature numbers of Sec. 5.C with their five parameters. */
typedef struct {
  double m, d_ref, omega, T_ref, c_alpha, theta_v;
  double Z_rot, Z_vib;
  int zmodel;
  double Zrot_inf, T_star, C1, C2, sigma_vib;
} usp_species;

/* Device-memory allocator callbacks: alloc(bytes, user) returns a device
 * pointer aligned to 256 bytes or NULL; free(ptr, user) releases it. */
typedef void* (*usp_alloc_fn)(size_t bytes, void* user);
typedef void (*usp_free_fn)(void* ptr, void* user);

typedef struct {
  int precision;        /* USP_FP64: FP64 state and arithmetic (plain form);
                           USP_FP32: FP32 particle state and per-particle
                           arithmetic, FP64 per-cell sums and coefficients  */
  uint64_t seed;        /* key of the Philox4x32-10 stream                   */
  int64_t step0;        /* index of the first step (Philox counter word 1)   */
  void* stream;         /* cudaStream_t to enqueue on; NULL = legacy stream  */
  int use_graph;        /* 1: replay the step from a captured CUDA graph     */
  int tile;             /* particles per collide tile (0 = autotune)         */
  usp_alloc_fn alloc;   /* optional allocator (NULL = cudaMalloc)            */
  usp_free_fn free_;
  void* alloc_user;
  int method;           /* USP_METHOD_*; channel and plane contexts run
                           USP_METHOD_FPM with the cell values at every
                           particle (the first-order method: no
                           reconstruction); not with the tangent forms
                           (USP_ENOTSUP)                                      */
} usp_config;

/* 1D channel between two fully diffuse plates at y = 0 and y = L (the
 * Poiseuille set-up of the paper's Sec. 5.B, driven by a uniform body force
 * g along x): ny cells of width L / ny, particle weight F_num (real
 * molecules per simulation particle), cross-section `area` normal to y,
 * reconstruct = 1 for the first-order reconstruction of Sec. 3.B. */
typedef struct {
  int ny;
  double L, T_wall, g, F_num, area;
  int reconstruct;
} usp_channel;

/* 2D plane domain [x0, x1] x [y0, y1] on nx x ny level-1 cells (cell
 * j * nx + i), depth `depth` along z, with an optional circular body of
 * radius cyl_r (<= 0: none) centred at (cyl_xc, cyl_yc), fully diffuse at
 * T_wall (the hypersonic cylinder set-up of the paper's Sec. 5.C, with cut
 * cells).  bc[] gives the condition of the sides left, right, bottom, top
 * (USP_BC_*); a side with inflow[k] = 1 (it must be open) lets the freestream
 * (n_inf, T_inf, velocity U_inf along x) enter with its one-way Maxwellian
 * flux.  F_num is the particle weight; reconstruct = 1 for the quadrant
 * bilinear reconstruction of Sec. 3.B.
 *
 * Mesh refinement (Sec. 5.C, three levels each doubling the resolution):
 * amr_levels 0 or 1 keeps the uniform grid.  With 2 or 3, a level-1 cell
 * whose centre lies within amr_r2 of (cyl_xc, cyl_yc) is split into 2 x 2
 * level-2 cells and, with 3, a level-2 cell whose centre lies within amr_r3
 * into 2 x 2 level-3 cells; a cell whose four corners lie inside the body is
 * not split.  The cells ("leaves") are numbered level-1 cell by level-1 cell
 * (row-major), the children of a split cell in the order (0,0), (1,0),
 * (0,1), (1,1) of (x, y) halves (usp_plane_leaves lists them).  Neighbouring
 * fluid cells must differ by one level at most: every level-1 cell holding
 * level-3 cells needs its eight neighbours split or inside the body.  The
 * reconstruction takes a finer neighbour's square as the particle-number
 * weighted mean of its four cells and a coarser neighbour's as that cell's
 * own polynomial at the square's centre (Sec. 3.B, non-uniform grids). */
enum { USP_BC_OPEN = 0, USP_BC_SPECULAR = 1, USP_BC_DIFFUSE = 2 };
typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  double cyl_xc, cyl_yc, cyl_r;
  double T_wall;
  double n_inf, T_inf, U_inf;
  int bc[4];
  int inflow[4];
  double F_num, depth;
  int reconstruct;
  int amr_levels;
  double amr_r2, amr_r3;
} usp_plane;

/* Cells of a plane's grid: returns their count (USP_EINVAL for invalid
 * sizes or refinement parameters or neighbouring levels that differ by two)
 * and, for the arrays that are not NULL, per cell its level (1..3) and
 * integer coordinates at that level: the cell spans
 * [x0 + ii h, x0 + (ii + 1) h] x [y0 + jj k, y0 + (jj + 1) k] with
 * h = (x1 - x0) / nx / 2^(level-1), k likewise.  Host only; needs no GPU. */
int usp_plane_leaves(const usp_plane* pl, int32_t* level, int32_t* ii, int32_t* jj);

typedef struct usp_ctx usp_ctx;

/* Make device `dev` current for the calling thread (cudaSetDevice) so that
 * contexts created afterwards live on it.  Returns USP_EINVAL for a device
 * index out of range. */
int usp_select_device(int dev);

/* Mean collision time tau_c = K(c_alpha, omega) mu(T) / (n k_B T) of the VSS
 * model (Eq. tau_c), evaluated on the host.  Callers use it to choose dt as
 * a multiple of tau_c. */
double usp_tau_c(const usp_species* sp, double n, double T);

/* Create a context for n_cells independent homogeneous cells (the setting of
 * the paper's Sec. 5.A) and upload the initial particles.
 *   h_offsets: n_cells + 1 int64, non-decreasing, h_offsets[0] = 0; the
 *              particles of cell i are [h_offsets[i], h_offsets[i+1]).
 *   h_ndens:   number density n of each cell [1/m^3] (constant in time).
 *   h_dt:      time step of each cell [s]; must satisfy 2 mu/p > Pr dt.
 *   h_cx, h_cy, h_cz, h_erot (double) and h_lev (int32): the particles.
 *              Levels are >= 0; they are not checked here (nor in the
 *              host-buffer step), and the collision takes a negative level
 *              as 0.
 * Particle ids (the Philox counter word 0) are the positions in these
 * arrays.  Returns USP_EINVAL for inconsistent sizes or a total above 2^31.
 * Synchronises the stream. */
int usp_init_homogeneous(usp_ctx** out, const usp_species* sp, const usp_config* cfg,
                         int n_cells, const int64_t* h_offsets, const double* h_ndens,
                         const double* h_dt, const double* h_cx, const double* h_cy,
                         const double* h_cz, const double* h_erot, const int32_t* h_lev);

/* Create a context for the 1D channel (usp_channel) holding n particles:
 * positions h_y in [0, L], velocities, specific rotational energies and
 * levels as in usp_init_homogeneous, and the particle ids h_pid (the Philox
 * counter word 0; NULL: ids 0..n-1).  dt is the time step [s].  One step is:
 * ballistic move with the body force and diffuse-wall re-emission (full
 * accommodation at T_wall, flight continued for the rest of the step), a
 * stable sort of the particles by cell, then the collision step of Sec. 4.D
 * in every cell with the fields interpolated to each particle (Sec. 3.B),
 * then the conservation scheme of Sec. 4.C.  Particle order after a step is
 * the cell order (stable).  Returns USP_EINVAL for a particle outside [0, L],
 * a negative level or invalid sizes.  Synchronises. */
int usp_init_channel(usp_ctx** out, const usp_species* sp, const usp_config* cfg,
                     const usp_channel* ch, double dt, int64_t n, const double* h_y,
                     const double* h_cx, const double* h_cy, const double* h_cz,
                     const double* h_erot, const int32_t* h_lev, const uint32_t* h_pid);

/* Channel time averages: while on (1), every step adds, per cell of its
 * post-step state, N, sum c (3), sum c c (xx yy zz xy xz yz), sum eps, sum I
 * (12 doubles per cell), plus one to the sampled-step count and the step's
 * x-momentum (per unit mass) taken by the walls.  usp_channel_read copies
 * the ny * 12 + 2 doubles to h_acc (synchronises) and clears them if reset.
 * In the USP_FP64_TANGENT form h_acc holds 4 such blocks: the sums, then
 * their derivatives with respect to Z_rot, omega and T_wall (entries that
 * carry no derivative -- counts, levels, step count, wall momentum -- are 0
 * in blocks 1-3). */
int usp_channel_sample(usp_ctx* ctx, int on);
int usp_channel_read(usp_ctx* ctx, double* h_acc, int reset);

/* Time-averaged profiles of a channel context, formed on the device from the
 * sums pooled over the sampled steps (usp_channel_sample): USP_NPROF fields
 * per cell, field-major (out[f * ny + cell]):
 *   0 mean particle count per sampled step | 1-3 U (m/s) | 4 T_tr |
 *   5 T_rot | 6 T_vib (K)
 * with the pooled sample means of Sec. 2.A (ensemble averages as 1/N means
 * over every particle-step of the window): U = sum c / sum N,
 * T_tr = (sum |c|^2 / sum N - |U|^2) / 3R, T_rot = sum eps / (R sum N),
 * T_vib inverting e_vib at the mean level (0 for no excitation).  Cells
 * that held no particle give zeros.  In the tangent forms out holds
 * 4 such blocks of USP_NPROF * ny doubles: the profiles, then their
 * derivatives with respect to Z_rot, omega and T_wall (0 for the count and
 * T_vib: counts and levels are held).  out_is_device = 1: device memory,
 * asynchronous; 0: host memory, synchronises.  USP_EINVAL for a context
 * that is not a channel. */
#define USP_NPROF 7
int usp_profiles(usp_ctx* ctx, double* out, int out_is_device);

/* Gradient of a scalar objective L(profiles) with respect to the parameters
 * (Z_rot, omega, T_wall) of a tangent-form channel context: the pathwise
 * derivative under common random numbers,
 *   grad3[k] = sum_{f, cell} dL_dprof[f * ny + cell] * d prof[f][cell] / d theta_k,
 * contracted on the device from the derivative sums the run accumulated.
 * The derivative holds every discrete outcome (levels, cell membership,
 * wall events and their times, the Cholesky / positivity-fix branch and
 * root, the +-1 level picks) and the particle positions at their values.
 *   d_dL_dprof: device, USP_NPROF * ny doubles (layout of usp_profiles).
 *   grad3:      3 doubles; grad_is_device = 1: device memory, asynchronous;
 *               0: host memory, synchronises.
 * USP_ENOTSUP for another form or kind of context.  Enqueued on the
 * context's stream after the steps it differentiates. */
int usp_backward(usp_ctx* ctx, const double* d_dL_dprof, double* grad3, int grad_is_device);

/* Checkpoints (channel and homogeneous contexts): everything a step carries
 * into the next one -- the particle state with its pending conservation
 * rescale, the per-cell records (and the jump tables of the FP32 form), the
 * time-average sums and sampling switch, the step counter, the status word
 * and counters -- as one opaque buffer of usp_checkpoint_bytes bytes.
 * usp_save writes it into buf; usp_load restores a context created with the
 * same sizes, form, method and seed from it, after which the run continues
 * bit for bit as the one that saved it.  buf_is_device = 1: device memory,
 * asynchronous on the context's stream; 0: host memory, synchronises.
 * usp_load returns USP_EINVAL for a buffer from another kind of context
 * (header mismatch) and leaves the context unchanged then; plane contexts
 * return USP_ENOTSUP. */
int usp_checkpoint_bytes(usp_ctx* ctx, size_t* bytes);
int usp_save(usp_ctx* ctx, void* buf, int buf_is_device);
int usp_load(usp_ctx* ctx, const void* buf, int buf_is_device);

/* Current channel particles (cell order, conservation rescale applied) to
 * host arrays of length n; y and pid may be NULL.  Synchronises. */
int usp_channel_get_particles(usp_ctx* ctx, double* h_y, double* h_cx, double* h_cy,
                              double* h_cz, double* h_erot, int32_t* h_lev, uint32_t* h_pid);

/* Create a context for the 2D plane domain (usp_plane) with storage for
 * `capacity` particles, holding n initial particles (x, y inside the domain,
 * outside the body; velocities, specific rotational energies, levels and
 * ids as in usp_init_channel; NULL ids: 0..n-1).  area_frac (one double in
 * [0, 1] per cell, usp_plane_leaves order, host) is the fluid fraction of
 * each cell: the cell volume is area_frac dx dy depth / 4^(level-1), and only
 * cells with fraction 1 serve as reconstruction neighbours.  dt is the time step [s].  precision USP_FP32
 * or USP_FP64.  One step is: flight with events (body: diffuse re-emission;
 * sides: specular reflection or removal), injection of the entering
 * freestream particles (count floor(flux A dt / F_num + u) per face, entry
 * point and entry time uniform, ids counted up from the largest initial
 * id + 1), a stable sort by cell (moved particles before new ones within a
 * cell), then per cell the collision step of Sec. 4.D with the fields
 * reconstructed at each particle (Sec. 3.B) and the conservation scheme of
 * Sec. 4.C.  The particle count lives on the device, so the step can be
 * replayed from a CUDA graph; a step whose inflow would exceed `capacity`
 * injects nothing and sets USP_F_CAPACITY.  Returns USP_EINVAL for invalid
 * geometry, sizes, fractions or particles.  Synchronises. */
int usp_init_plane(usp_ctx** out, const usp_species* sp, const usp_config* cfg,
                   const usp_plane* pl, double dt, const double* area_frac, int64_t n,
                   int64_t capacity, const double* h_x, const double* h_y, const double* h_cx,
                   const double* h_cy, const double* h_cz, const double* h_erot,
                   const int32_t* h_lev, const uint32_t* h_pid);

/* Live particle count of a plane context and the id the next entering
 * particle will get.  Synchronises. */
int usp_plane_count(usp_ctx* ctx, int64_t* n, uint32_t* next_pid);

/* Current plane particles (cell order, conservation rescale applied) to host
 * arrays of length cap; *n receives the live count (USP_EINVAL if it exceeds
 * cap).  Any array may be NULL.  Synchronises. */
int usp_plane_get_particles(usp_ctx* ctx, int64_t cap, int64_t* n, double* h_x, double* h_y,
                            double* h_cx, double* h_cy, double* h_cz, double* h_erot,
                            int32_t* h_lev, uint32_t* h_pid);

/* Time averages of a spatial context (channel or plane), as
 * usp_channel_sample / usp_channel_read; for a plane context the layout is
 * n_cells * 12 + 2 + 4 * USP_NSURF doubles: the per-cell sums, the
 * sampled-step count, 0, then the surface tallies of the cylinder (Sec. 5.C,
 * surface coefficients C_f, C_h, drag, heat flux): USP_NSURF bins of the
 * polar angle phi = atan2(y - yc, x - xc) in [-pi, pi), 4 sums each over the
 * wall events of the sampled steps, per unit particle mass: the momentum
 * given to the wall (c_in - c_out, x then y), the energy given to it
 * (1/2 |c|^2 + eps_rot + R Theta I, in minus out) and the event count.
 * Multiply by F_num m / (sampled steps dt) for forces and powers. */
#define USP_NSURF 180
int usp_sample(usp_ctx* ctx, int on);
int usp_sample_read(usp_ctx* ctx, double* h_acc, int reset);

/* Enqueue nsteps collision steps (Sec. 4.D + Sec. 4.C) on the stream. */
int usp_step(usp_ctx* ctx, int nsteps);

/* Enqueue the per-cell moments of the current state into out (USP_NMOM x
 * n_cells doubles, field-major).  out_is_device = 1: out is device memory
 * and the call is asynchronous; 0: out is host memory and the call
 * synchronises the stream. */
int usp_moments(usp_ctx* ctx, double* out, int out_is_device);

/* Copy the current particle state to host arrays (length = total particles,
 * positions as given to usp_init_homogeneous).  Synchronises. */
int usp_get_particles(usp_ctx* ctx, double* h_cx, double* h_cy, double* h_cz, double* h_erot,
                      int32_t* h_lev);

/* Replace the particle state from host arrays (same layout as init) and
 * recompute the cell moments; the step counter is kept.  Asynchronous with
 * respect to the host only if the host arrays are pinned. */
int usp_set_particles(usp_ctx* ctx, const double* h_cx, const double* h_cy, const double* h_cz,
                      const double* h_erot, const int32_t* h_lev);

/* End-to-end call on host buffers: upload the state (h_* arrays in the
 * context's precision: float for USP_FP32, double for USP_FP64; int32
 * levels), run nsteps steps, download the moments into h_moments (USP_NMOM x
 * n_cells doubles) and, if h_*_out are not NULL, the resulting state.
 * Synchronises.  The cells are independent, so the upload goes in sixteen runs
 * of whole cells and each run is stepped while the next one is in transit;
 * with pinned host buffers the copies run at full link speed and hide most
 * of the arithmetic.  Homogeneous contexts only (USP_ENOTSUP otherwise). */
int usp_step_host(usp_ctx* ctx, const void* h_cx, const void* h_cy, const void* h_cz,
                  const void* h_erot, const int32_t* h_lev, int nsteps, double* h_moments,
                  void* h_cx_out, void* h_cy_out, void* h_cz_out, void* h_erot_out,
                  int32_t* h_lev_out);

/* Read (and clear with reset != 0) the sticky status word and counters.
 * Synchronises.  Returns USP_EDEVICE if an error bit is set: USP_F_A_NONPOS,
 * USP_F_SAMPLER_UNDERFLOW, USP_F_BOUNDS, USP_F_CAPACITY or
 * USP_F_WAIT_TIMEOUT; the other bits record clamps and caps the method's
 * readings define. */
int usp_status(usp_ctx* ctx, uint32_t* flags, int64_t counters[USP_NCOUNTERS], int reset);

/* Limit, in SM clock cycles, of every wait of the homogeneous particle pass
 * on its bulk copies (cycles = 0 restores the default of 2e9, about a
 * second).  A wait that runs out sets USP_F_WAIT_TIMEOUT (usp_status then
 * returns USP_EDEVICE): the pass stops there, waits with the default limit
 * for its own copies still in flight and returns, leaving that step's state
 * incomplete.  Synchronises the stream and drops a captured graph.
 * USP_ENOTSUP for channel and plane contexts, USP_EINVAL for cycles < 0. */
int usp_set_wait_limit(usp_ctx* ctx, int64_t cycles);

/* Check of the device-side timeout path, for callers that monitor a run:
 * enqueues on the context's stream one block that waits, with the same
 * bounded wait as the particle pass and a limit of `cycles` SM clock cycles
 * (1 .. 2e9), on an mbarrier that nothing completes.  When the limit runs
 * out the block records USP_F_WAIT_TIMEOUT in the context's status word and
 * returns, so a following usp_status reports USP_EDEVICE; the context's
 * state is untouched and stays usable after usp_status(..., reset = 1).
 * USP_EINVAL for cycles out of range. */
int usp_wait_check(usp_ctx* ctx, int64_t cycles);

/* The guide of one jump-table row as the FP32 form builds it (Chen & Asau's
 * indexed search over the row of Eq. update_evib's inversion; host code, no
 * GPU).  row: 48 float cumulative values, non-decreasing, +inf after the
 * last one (row[0] = -1 marks an underflowed P(0)).  guide: 256 bytes out,
 * one per bin of a 23-bit uniform's top eight bits; with k the number of row
 * entries <= the bin's smallest uniform: bit 7 and the outcome (k, or
 * n_flip - k for a binomial row taken at 1 - p_B when n_flip >= 0) when no
 * entry lies inside the bin; else k (the search continues from there).
 * n_flip: -1, or the binomial n (0 .. 31), whose row ends at n
 * (row[n_flip] = +inf).  USP_EINVAL for NULL pointers, n_flip out of range
 * or a flipped row that does not end at n. */
int usp_guide_row(const float* row, int n_flip, uint8_t* guide);

/* Wait for all work of the context. */
int usp_sync(usp_ctx* ctx);

/* Sizes of the context. */
int usp_info(usp_ctx* ctx, int64_t* n_particles, int* n_cells, int* precision, int64_t* step,
             int* tile, int64_t* device_bytes);

/* Particle-pass variant of a homogeneous context: its design (*warp_tiles =
 * 1: every warp pipelines its own tiles of <= 128 particles; 0: a block
 * stages tiles of <= 1536 particles shared by its 256 threads), the resident
 * blocks per SM its register budget targets (2, 3 or 4), and the autotuner's
 * milliseconds per launch of each variant on the whole state, ordered
 * block-tiled 2, 3, 4 then warp-tiled 2, 3, 4 (zeros when the tuner did not
 * run: explicit tile size, or fewer than 2^20 particles).  Other contexts
 * report zeros.  Any output pointer may be NULL. */
int usp_tuning(usp_ctx* ctx, int* warp_tiles, int* blocks_per_sm, double ms[6]);

/* Force the particle-pass variant of a homogeneous context (warp_tiles 0 or
 * 1, blocks_per_sm 2..4; USP_EINVAL otherwise or for another kind of
 * context).  Synchronises the context's stream and drops a captured graph.
 * The variants make the same per-particle decisions and differ only in the
 * order in which the FP64 cell sums are added up. */
int usp_set_variant(usp_ctx* ctx, int warp_tiles, int blocks_per_sm);

/* Number of kernel launches the library enqueued since creation (graph
 * replays count every kernel in the graph). */
int64_t usp_launch_count(usp_ctx* ctx);

/* Per-kernel device timing.  While enabled (on = 1), usp_step launches its
 * kernels one by one (no graph replay) and brackets each launch with a pair
 * of CUDA events recorded on the context stream; enabling clears the
 * totals.  usp_profile_read synchronises and returns, per kernel kind
 * (0 = particle collide pass, 1 = per-cell finalize), the accumulated device
 * milliseconds and the number of launches timed. */
int usp_profile_enable(usp_ctx* ctx, int on);
int usp_profile_read(usp_ctx* ctx, double ms[2], int64_t launches[2]);

/* Largest n_cells accepted by usp_moments_noalloc. */
#define USP_NOALLOC_MAX_CELLS 8192

/* Per-cell moments (same fields and layout as usp_moments) of a particle
 * state the caller holds in device memory, computed without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that may not allocate, such as frameworks that reserve all device
 * memory in their own pool at start-up and forbid later cudaMalloc, or time
 * loops that must not risk the implicit synchronisation of cudaMalloc and
 * cudaFree.
 *   sp:        gas species (only m and theta_v are used).
 *   n_cells:   1 .. USP_NOALLOC_MAX_CELLS; a larger value returns USP_EINVAL
 *              and launches nothing.
 *   d_offsets: device int64[n_cells + 1], cell i holds particles
 *              [d_offsets[i], d_offsets[i+1]).
 *   d_cx, d_cy, d_cz, d_erot (device double) and d_lev (device int32): the
 *              particles, indexed by those offsets.
 *   d_out:     device double[USP_NMOM * n_cells], field-major, written.
 *   stream:    cudaStream_t the work is enqueued on (NULL: legacy stream);
 *              the call returns without waiting.
 * Working space is one fixed device array of 20 * USP_NOALLOC_MAX_CELLS
 * doubles (1.25 MiB) that every device loading the library holds until the
 * process exits.  Under CUDA's default lazy module loading the array is
 * reserved when the library's module is loaded on a device, at the first call
 * there at the latest; that call also looks up the array's device address
 * (cudaGetSymbolAddress) with the device current.  Make one warm-up call at
 * start-up, before any stream capture (or set CUDA_MODULE_LOADING=EAGER);
 * the address is kept, so a cudaDeviceReset between calls is not supported.
 * An error pending from the caller's earlier work (cudaPeekAtLastError)
 * makes the call return USP_ECUDA without launching.  All calls share the array and it keeps
 * the last call's contents: each call clears it on its stream first, and
 * calls whose work overlaps on the GPU race on it.  No cudaMalloc, cudaFree
 * or other allocating routine is called. */
int usp_moments_noalloc(const usp_species* sp, int n_cells, const int64_t* d_offsets,
                        const double* d_cx, const double* d_cy, const double* d_cz,
                        const double* d_erot, const int32_t* d_lev, double* d_out,
                        void* stream);

/* Release the context and all its device memory (synchronises). */
void usp_destroy(usp_ctx* ctx);

/* Static description of an error code. */
const char* usp_strerror(int err);

#ifdef __cplusplus
}
#endif
#endif
