/*
 * usp_oracle.h -- plain, slow, FP64 CPU oracle of the USP-FPM particle update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library; the only thing both sides share is the seeded input generator,
 * which holds none of the method's arithmetic.
 *
 * Every function follows one passage of Kim & Jun, "A second-order particle
 * Fokker-Planck-Master method for diatomic gas flows" (arXiv 2508.05642); the
 * passage is named next to it.  Where the paper is silent, garbled or
 * ambiguous the reading taken is stated in the comment of the function.
 *
 * Two "forms" exist (argument `form`):
 *   0  FP64 plain method: uniforms u = (x + 0.5) 2^-32 in double, discrete
 *      decisions (negative-binomial / binomial inversion) in double.
 *   1  FP32-state method: particle uniforms u = (2 (x >> 9) + 1) 2^-24, exact
 *      in float, and the inversion that decides the new vibrational level is
 *      carried out in float, operation by operation as written below, so that
 *      an integer outcome is decided in the same precision as the FP32 kernel.
 *      Everything else in the oracle stays FP64.
 */
#ifndef USP_ORACLE_H
#define USP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status bits (sticky, OR-ed into *flags) */
#define ORC_F_PB_CLAMP            0x01u  /* p_B > 1 met: binomial clamped to n   */
#define ORC_F_CHOL_FAIL_AFTER_FIX 0x02u  /* D_tr still not PD after the nu fix  */
#define ORC_F_NEG_RADICAND        0x04u  /* velocity rescale radicand <= 0      */
#define ORC_F_VIB_LOOP_CAP        0x08u  /* +-1 level loop hit its draw cap     */
#define ORC_F_TREL_CLAMP          0x10u  /* a relaxation temperature was < 0    */
#define ORC_F_SAMPLER_CAP         0x20u  /* inversion search hit its cap        */
#define ORC_F_A_NONPOS            0x40u  /* (2mu/p - Pr dt) <= 0: dt too large  */
#define ORC_F_SAMPLER_UNDERFLOW   0x80u  /* P(0) underflowed even in double     */
#define ORC_F_WALL_CAP            0x100u /* a particle hit walls too many times */
#define ORC_F_INFLOW_CAP          0x800u /* inflow speed sampler hit 64 attempts   */
#define ORC_F_CAPACITY            0x1000u /* particle storage full: inflow dropped */

/* counters[] slots */
enum { ORC_C_CHOL_FIX = 0, ORC_C_PB_CLAMP = 1, ORC_C_TREL_CLAMP = 2,
       ORC_C_VIB_DRAWS = 3, ORC_C_NEG_RADICAND = 4, ORC_C_WALL_HITS = 5,
       ORC_C_INTERP_FALLBACK = 6, ORC_C_SKIPPED_CELLS = 7,
       ORC_C_INFLOW = 8,     /* particles generated at inflow faces            */
       ORC_C_OUTFLOW = 9,    /* particles removed at open sides                */
       ORC_C_NU_ZERO = 10,   /* positivity fix ended at nu = 0                 */
       ORC_NCOUNTERS = 11 };

/* number of per-cell output moments (field-major: out[f * ncell + cell]) */
#define ORC_NMOM 22

typedef struct {
    double m;        /* molecular mass [kg]                                  */
    double d_ref;    /* VSS/VHS reference diameter [m]                        */
    double omega;    /* viscosity index c_omega                              */
    double T_ref;    /* reference temperature [K]                            */
    double c_alpha;  /* VSS angular scattering parameter (1 for VHS)         */
    double theta_v;  /* characteristic vibrational temperature [K]           */
    double Z_rot;    /* fixed rotational collision number (zmodel 0)         */
    double Z_vib;    /* fixed vibrational collision number (zmodel 0)        */
    int    zmodel;   /* 0 fixed numbers, 1 Parker + Millikan-White/high-T    */
    double Zrot_inf, T_star, C1, C2, sigma_vib;   /* zmodel 1 parameters     */
} orc_species;

typedef struct {
    /* inputs */
    double n, dt, T_tr, T_rot, T_vib;
    /* transport (Sec. 4.A) */
    double mu, p, mu_p, tau_c, Z_rot, Z_vib, tau_rot, tau_vib, Pr;
    /* Eqs. USP-FPM_alpha_tr, USP-FPM_nu, sigma_relax */
    double A, B, alpha, nu_ref;
    /* gamma coefficients with the implicit T_1 (Sec. 3.A.1) */
    double g_r, g_v, cv_T1, T_check, gamma_tr_rot, gamma_tr_vib, gamma_rot_vib;
    int    t1_iters;
    /* second-order targets, Eqs. e_tr_relax .. e_vib_relax */
    double e_tr_tgt, e_rot_tgt, e_vib_tgt;
    int    tgt_clamped;    /* a negative rotational / vibrational target was set to 0 */
} orc_coeffs;

/* ---- random numbers ---------------------------------------------------- */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t x, int form);

/* ---- closed-form physics ----------------------------------------------- */
double orc_R(const orc_species* sp);
double orc_e_vib(const orc_species* sp, double T);
double orc_cv_vib(const orc_species* sp, double T);
double orc_T_vib_from_mean_level(const orc_species* sp, double ebar);
double orc_mu(const orc_species* sp, double T);
double orc_tau_c(const orc_species* sp, double n, double T);
double orc_prandtl(const orc_species* sp, double T);
void   orc_collision_numbers(const orc_species* sp, double T_tr, double* Zrot, double* Zvib);
int    orc_cell_coeffs(const orc_species* sp, double n, double dt,
                       double T_tr, double T_rot, double T_vib, orc_coeffs* out);
void   orc_relaxation_temperatures(const orc_species* sp, const orc_coeffs* cc, double alpha,
                                   double T_tr, double T_rot, double T_vib,
                                   double* T_tr_rel, double* T_rot_rel, double* e_vib_rel,
                                   uint32_t* flags);

/* ---- small linear algebra ---------------------------------------------- */
void   orc_sym3_eig_minmax(const double P[6], double* lmin, double* lmax);
int    orc_cholesky3(const double M[6], double L[6]);

/* ---- discrete samplers (inversion with one uniform each) ----------------- */
int    orc_sample_nb(int r, double p, double u, int form, uint32_t* flags);
int    orc_sample_b(int n, double p, double u, int form, uint32_t* flags);

/* ---- one particle collision (Sec. 4.D flow, Eqs. update_ci, update_erot,
 *      update_evib with the positivity fix of Sec. 3.A.3) ------------------ */
void   orc_collide_particle(const orc_species* sp, int form, const orc_coeffs* cc,
                            const double U[3], const double Pi[6],
                            double T_tr, double T_rot, double T_vib,
                            const double G[4], double u5, double u6,
                            double c[3], double* erot, int32_t* lev,
                            uint32_t* flags, int64_t* counters);

/* ---- moments (Sec. 2.A) -------------------------------------------------- */
void   orc_moments(const orc_species* sp, int ncell, const int64_t* off,
                   const double* cx, const double* cy, const double* cz,
                   const double* erot, const int32_t* lev, double* out);

/* ---- the plain FPM method (Sec. 2.B model, Sec. 2.C particle scheme) -----
 * The first-order method the paper builds on: Gorji's velocity integrator
 * with alpha = exp(-dt/tau), the modified-Milstein rotational update with the
 * same alpha, Gillespie's direct method for the vibrational levels, and the
 * conservation scheme of Sec. 4.C. */
typedef struct {
    double n, dt, T_tr, T_rot, T_vib;
    double mu, p, tau_c, Z_rot, Z_vib, tau_rot, tau_vib, Pr;
    double nu;        /* 1 - 3 / (2 Pr)                                        */
    double tau;       /* 2 mu (1 - nu) / p                                     */
    double alpha;     /* exp(-dt / tau)                                        */
    double T_tr_rel, T_rot_rel, e_vib_rel;   /* Eqs. T_tr_FPM .. T_vib_FPM      */
    double lam_up, lam_dn;   /* level rates per unit (I+1) and I, times dt     */
    double e_rot_tgt, e_vib_tgt;   /* expected mode energies after dt          */
    int    clamped;   /* a relaxation energy was negative and set to 0         */
} orc_fpm;

int    orc_fpm_coeffs(const orc_species* sp, double n, double dt,
                      double T_tr, double T_rot, double T_vib, orc_fpm* out);
int    orc_gillespie(int I, double lam_up, double lam_dn, uint64_t seed, uint32_t pid,
                     uint32_t step, int form, uint32_t* flags);
void   orc_collide_particle_fpm(const orc_species* sp, int form, const orc_fpm* fc,
                                const double U[3], const double Pi[6], const double G[4],
                                uint64_t seed, uint32_t pid, uint32_t step,
                                double c[3], double* erot, int32_t* lev,
                                uint32_t* flags, int64_t* counters);
int    orc_homog_step_fpm(const orc_species* sp, int form, uint64_t seed,
                          int64_t step0, int nsteps, int n_inst, const int64_t* off,
                          const double* ndens, const double* dt,
                          double* cx, double* cy, double* cz, double* erot,
                          int32_t* lev, const uint32_t* pid,
                          uint32_t* flags, int64_t* counters);

/* ---- one or more steps of independent homogeneous cells ("instances") ---- */
int    orc_homog_step(const orc_species* sp, int form, uint64_t seed,
                      int64_t step0, int nsteps, int n_inst, const int64_t* off,
                      const double* ndens, const double* dt,
                      double* cx, double* cy, double* cz, double* erot,
                      int32_t* lev, const uint32_t* pid,
                      uint32_t* flags, int64_t* counters);

/* ---- 1D channel between two diffuse plates (Sec. 5.B set-up) ------------ */
typedef struct {
    int    ny;        /* cells along y                                        */
    double L;         /* plate gap [m]; walls at y = 0 and y = L              */
    double T_wall;    /* temperature of both fully diffuse walls [K]          */
    double g;         /* uniform body force along x [m/s^2]                   */
    double F_num;     /* real molecules per simulation particle               */
    double area;      /* cross-section normal to y [m^2]; V_cell = area * dy  */
    int    reconstruct; /* 1: first-order reconstruction (Sec. 3.B), 0: cell values */
    int    method;    /* 0 USP-FPM (Sec. 4.D); 1 the plain FPM method (Sec. 2.B-C)
                         with the cell values at every particle               */
} orc_channel;

/* Per-cell accumulator layout of orc_channel_step (time-average sums, FP64):
 * [c * ORC_NACC + k], k: 0 N, 1-3 sum c, 4-9 sum c c (xx yy zz xy xz yz),
 * 10 sum eps, 11 sum I; slot [ny * ORC_NACC] counts sampled steps and
 * [ny * ORC_NACC + 1] the x-momentum (per unit particle mass) given to the
 * walls. */
#define ORC_NACC 12

int    orc_channel_step(const orc_species* sp, int form, uint64_t seed, int64_t step0,
                        int nsteps, const orc_channel* ch, double dt, int64_t n,
                        double* y, double* cx, double* cy, double* cz, double* erot,
                        int32_t* lev, uint32_t* pid, int64_t* cell_off, double* acc,
                        uint32_t* flags, int64_t* counters);
void   orc_channel_reconstruct(const orc_channel* ch, const int64_t* counts, const double* F,
                               int cell, double y, double* out);
/* The collision draws of one particle and step (four standard normals and
 * the two jump-sampler uniforms), as every step uses them (the same in both
 * forms). */
void   orc_particle_draws(uint64_t seed, uint32_t pid, uint32_t step, int form,
                          double G[4], double* u5, double* u6);

/* Frozen-discrete runs (gradient checks by finite differences): a decision
 * log records every discrete decision of a channel run in the order it is
 * taken (mode 1: record, clearing the log) and replays it in a later run
 * (mode 2: replay from the start; mode 0: off).  The decisions are the
 * wall events of the flight (inside or not, which wall, the event time and
 * its clamps), the
 * cell of each particle, the reconstruction side and its fall-back, the
 * Cholesky test and every branch of the positivity fix (bounds, clamps,
 * root), the relaxation-temperature clamps, the two jump outcomes, the wall
 * re-emission level, the rounded level deficit I_Delta and the two guards
 * of the conservation scaling.  A replaying run takes the recorded outcome;
 * stats: decisions of each kind recorded (yes/no, integer), replayed
 * decisions that differ from the run's own, and replay requests past the
 * end of the log.  orc_channel_step_frozen is orc_channel_step with a log
 * (USP-FPM method only; returns -3 for the plain FPM method). */
typedef struct orc_declog orc_declog;
orc_declog* orc_declog_new(void);
void   orc_declog_free(orc_declog* dl);
void   orc_declog_set_mode(orc_declog* dl, int mode);
void   orc_declog_stats(const orc_declog* dl, int64_t out[4]);
int    orc_channel_step_frozen(const orc_species* sp, int form, uint64_t seed, int64_t step0,
                               int nsteps, const orc_channel* ch, double dt, int64_t n,
                               double* y, double* cx, double* cy, double* cz, double* erot,
                               int32_t* lev, uint32_t* pid, int64_t* cell_off, double* acc,
                               uint32_t* flags, int64_t* counters, orc_declog* dl);
/* one diffuse re-emission (velocity, eps_rot, level) for tests of the wall law */
void   orc_wall_reemit(const orc_species* sp, int form, uint64_t seed, uint32_t pid, uint32_t step,
                       int hit, double Tw, int into_positive_y, double out[4], int32_t* lev);

/* ---- 2D plane flow past a circular cylinder (Sec. 5.C set-up) ------------ */
enum { ORC_BC_OPEN = 0, ORC_BC_SPECULAR = 1, ORC_BC_DIFFUSE = 2 };
typedef struct {
    int    nx, ny;                 /* cells                                          */
    double x0, x1, y0, y1;         /* domain                                         */
    double cyl_xc, cyl_yc, cyl_r;  /* cylinder (r <= 0: none), diffuse at T_wall    */
    double T_wall;
    double n_inf, T_inf, U_inf;    /* freestream: density, temperature, x velocity   */
    int    bc[4];                  /* left, right, bottom, top: ORC_BC_*            */
    int    inflow[4];              /* 1: inject the freestream through that side    */
    double F_num, depth;           /* particle weight; cell depth along z [m]        */
    int    reconstruct;
    /* mesh refinement about the cylinder (Sec. 5.C three-level grid): with
     * amr_levels 2 or 3, a level-1 cell whose centre lies within amr_r2 of
     * the cylinder centre is split into 2 x 2 level-2 cells, and (levels 3)
     * a level-2 cell whose centre lies within amr_r3 into 2 x 2 level-3
     * cells; a cell whose four corners lie inside the body is not split.
     * The cells ("leaves") are numbered level-1 cell by level-1 cell
     * (row-major), the children of a split cell in the order (0,0), (1,0),
     * (0,1), (1,1) of (x, y) halves.  Neighbouring fluid leaves must differ
     * by one level at most: every level-1 cell holding level-3 leaves needs
     * its eight neighbours split or inside the body.  0 or 1: the uniform
     * grid. */
    int    amr_levels;
    double amr_r2, amr_r3;
    /* collision method: 0 USP-FPM (Sec. 4.D, reconstructed fields), 1 the
     * plain FPM method (Sec. 2.B-C) with the cell values */
    int    method;
} orc_plane;

/* Leaves of the plane's grid: count (-1 when the levels of neighbouring
 * fluid leaves differ by two), and per leaf its level (1..3) and integer
 * coordinates at its own level (centre x0 + (ii + 1/2) dx / 2^(level-1), y
 * likewise; arrays of orc_plane_nleaf entries); the leaf holding a point. */
int    orc_plane_nleaf(const orc_plane* pl);
void   orc_plane_leaves(const orc_plane* pl, int32_t* level, int32_t* ii, int32_t* jj);
int    orc_plane_leaf_of(const orc_plane* pl, double x, double y);

/* nsteps steps of the plane domain.  Live particles are [0, *n) of arrays of
 * capacity cap; *n and *next_pid (the id given to the next injected particle)
 * are updated; on return the live particles are sorted by cell (leaf order
 * above; cell j*nx+i on the uniform grid) with segment starts
 * cell_off[ncell + 1], ncell = orc_plane_nleaf.  area_frac[cell] is the fluid
 * fraction of each cell (volume = area_frac dx dy depth / 4^(level-1)).
 * Returns 0, -1 when a cell's coefficients failed (flags say which), -2 for
 * a refined grid whose neighbouring levels differ by two.  Accumulator layout
 * as ORC_NACC above, plus slot [ncell * ORC_NACC] = sampled steps, slot
 * [ncell * ORC_NACC + 1] = 0, then the surface tallies of the cylinder
 * (Sec. 5.C, surface coefficients): ORC_NSURF bins of the polar angle
 * phi = atan2(y - yc, x - xc) in [-pi, pi), 4 sums each over the wall events
 * of the sampled steps, per unit particle mass: the momentum given to the
 * wall (c_in - c_out, x and y) and the energy given to it
 * (1/2 |c|^2 + eps_rot + R Theta I, in minus out), and the event count. */
#define ORC_NSURF 180
int    orc_plane_step(const orc_species* sp, int form, uint64_t seed, int64_t step0, int nsteps,
                      const orc_plane* pl, const double* area_frac, double dt,
                      int64_t* n, int64_t cap, double* x, double* y, double* cx, double* cy,
                      double* cz, double* erot, int32_t* lev, uint32_t* pid, uint32_t* next_pid,
                      int64_t* cell_off, double* acc, uint32_t* flags, int64_t* counters);
void   orc_plane_reconstruct(const orc_plane* pl, const int64_t* counts, const double* area_frac,
                             const double* F, int cell, double x, double y, double* out);
/* inflow sampling pieces, for tests */
double orc_inflow_flux(double n, double RT, double u_n);
double orc_inflow_normal_speed(double RT, double u_n, uint32_t pid, uint32_t step, uint64_t seed,
                               int form, uint32_t* flags);

#ifdef __cplusplus
}
#endif
#endif
