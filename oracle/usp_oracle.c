/*
 * usp_oracle.c -- plain FP64 CPU oracle of the USP-FPM particle update.
 *
 * TEST INFRASTRUCTURE ONLY (see usp_oracle.h).  Written for a reader who has
 * the paper open: no blocking, no fusion, no reordering beyond what the paper's
 * algorithm states.  Compile with -ffp-contract=off so that the float-form
 * inversion is a fixed sequence of IEEE operations.
 */
#include "usp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KB 1.380649e-23          /* Boltzmann constant [J/K] (SI, exact)      */
#define PI 3.14159265358979323846
#define SAMPLER_KCAP 4096        /* search cap of one inversion              */

/* ======================================================================== */
/* Decision log: the frozen-discrete form of a run.  The pathwise gradient   */
/* of the method differentiates everything continuous and holds every        */
/* discrete outcome at its value (levels, cell membership, wall events, the  */
/* Cholesky / positivity-fix branch and root, the +-1 correction).  To       */
/* check it by finite differences, the base run records each discrete        */
/* decision in the order it is taken (mode 1) and the perturbed runs take    */
/* the recorded decision instead of their own (mode 2), so that they follow  */
/* the base run's branch with perturbed continuous values.  A replayed       */
/* decision that differs from the one the perturbed run would have taken is  */
/* counted.  Mode 0 (or no log) leaves every decision to the run.           */
/* ======================================================================== */
struct orc_declog {
    int mode;
    uint8_t* bits; int64_t nbits, capbits, rbit;
    int32_t* ints; int64_t nints, capints, rint;
    double* reals; int64_t nreals, capreals, rreal;
    int64_t mismatches, overruns;
};

orc_declog* orc_declog_new(void)
{
    return (orc_declog*)calloc(1, sizeof(orc_declog));
}

void orc_declog_free(orc_declog* dl)
{
    if (!dl) return;
    free(dl->bits); free(dl->ints); free(dl->reals); free(dl);
}

void orc_declog_set_mode(orc_declog* dl, int mode)
{
    dl->mode = mode;
    dl->rbit = 0; dl->rint = 0; dl->rreal = 0; dl->mismatches = 0; dl->overruns = 0;
    if (mode == 1) {
        dl->nbits = 0; dl->nints = 0; dl->nreals = 0;
        if (dl->bits) memset(dl->bits, 0, (size_t)dl->capbits);
    }
}

void orc_declog_stats(const orc_declog* dl, int64_t out[4])
{
    out[0] = dl->nbits; out[1] = dl->nints; out[2] = dl->mismatches; out[3] = dl->overruns;
}

/* a yes/no decision */
static int dec_b(orc_declog* dl, int v)
{
    v = v ? 1 : 0;
    if (!dl || dl->mode == 0) return v;
    if (dl->mode == 1) {
        if (dl->nbits == dl->capbits * 8) {
            int64_t cap = dl->capbits ? 2 * dl->capbits : 1 << 16;
            dl->bits = (uint8_t*)realloc(dl->bits, (size_t)cap);
            memset(dl->bits + dl->capbits, 0, (size_t)(cap - dl->capbits));
            dl->capbits = cap;
        }
        if (v) dl->bits[dl->nbits >> 3] |= (uint8_t)(1u << (dl->nbits & 7));
        dl->nbits += 1;
        return v;
    }
    if (dl->rbit >= dl->nbits) { dl->overruns += 1; return v; }
    int r = (dl->bits[dl->rbit >> 3] >> (dl->rbit & 7)) & 1;
    dl->rbit += 1;
    if (r != v) dl->mismatches += 1;
    return r;
}

/* a continuous quantity held at the base run's value (a wall-event time) */
static double dec_d(orc_declog* dl, double v)
{
    if (!dl || dl->mode == 0) return v;
    if (dl->mode == 1) {
        if (dl->nreals == dl->capreals) {
            int64_t cap = dl->capreals ? 2 * dl->capreals : 1 << 12;
            dl->reals = (double*)realloc(dl->reals, sizeof(double) * (size_t)cap);
            dl->capreals = cap;
        }
        dl->reals[dl->nreals++] = v;
        return v;
    }
    if (dl->rreal >= dl->nreals) { dl->overruns += 1; return v; }
    return dl->reals[dl->rreal++];
}

/* an integer outcome (a level, a cell index, a rounded count) */
static int64_t dec_i(orc_declog* dl, int64_t v)
{
    if (!dl || dl->mode == 0) return v;
    if (dl->mode == 1) {
        if (dl->nints == dl->capints) {
            int64_t cap = dl->capints ? 2 * dl->capints : 1 << 16;
            dl->ints = (int32_t*)realloc(dl->ints, sizeof(int32_t) * (size_t)cap);
            dl->capints = cap;
        }
        dl->ints[dl->nints++] = (int32_t)v;
        return v;
    }
    if (dl->rint >= dl->nints) { dl->overruns += 1; return v; }
    int64_t r = dl->ints[dl->rint++];
    if (r != v) dl->mismatches += 1;
    return r;
}

/* ======================================================================== */
/* Random numbers.  The paper names no generator; the method only needs      */
/* independent uniforms and standard normals per particle and per cell.      */
/* Philox4x32-10 is Salmon, Moraes, Dror & Shaw, "Parallel random numbers:   */
/* as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 products with the */
/* multipliers below, the key bumped by the two Weyl constants between       */
/* rounds.                                                                   */
/* ======================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Open-interval uniform from one 32-bit word.  Form 0: the midpoint rule on
 * all 32 bits, exact in double.  Form 1: the midpoint rule on the top 23 bits,
 * (2k+1) 2^-24, which is exact in float. */
double orc_uniform(uint32_t x, int form)
{
    if (form == 0) return ((double)x + 0.5) * (1.0 / 4294967296.0);
    float k = (float)((x >> 9) * 2u + 1u);
    float u = k * (1.0f / 16777216.0f);
    return (double)u;
}

static void philox_words(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint64_t seed, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, c1, c2, c3 };
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Box-Muller: two independent standard normals from two uniforms. */
static void box_muller(double ua, double ub, double* ga, double* gb)
{
    double rad = sqrt(-2.0 * log(ua));
    *ga = rad * cos(2.0 * PI * ub);
    *gb = rad * sin(2.0 * PI * ub);
}

/* ======================================================================== */
/* Closed-form physics                                                       */
/* ======================================================================== */
double orc_R(const orc_species* sp) { return KB / sp->m; }

/* Sec. 2.A: e_vib(T) = R Theta / (exp(Theta/T) - 1); the T -> 0 limit is 0. */
double orc_e_vib(const orc_species* sp, double T)
{
    if (T <= 0.0) return 0.0;
    return orc_R(sp) * sp->theta_v / (exp(sp->theta_v / T) - 1.0);
}

/* Sec. 2.A: c_v,vib = d e_vib / dT.  The printed formula has sinh without the
 * square; the derivative of e_vib is R (Theta/2T)^2 / sinh^2(Theta/2T), which
 * is what is used (the Grad-17 weight of Sec. 5.A.1 carries the square too). */
double orc_cv_vib(const orc_species* sp, double T)
{
    if (T <= 0.0) return 0.0;
    double h = 0.5 * sp->theta_v / T;
    double s = sinh(h);
    return orc_R(sp) * (h * h) / (s * s);
}

/* Inverse of e_vib for the sample mean level ebar = <I>:
 * e_vib(T) = R Theta ebar  <=>  T = Theta / ln(1 + 1/ebar); ebar = 0 -> T = 0. */
double orc_T_vib_from_mean_level(const orc_species* sp, double ebar)
{
    if (ebar <= 0.0) return 0.0;
    return sp->theta_v / log(1.0 + 1.0 / ebar);
}

/* Sec. 4.A: VSS viscosity mu = mu_ref (T/T_ref)^omega with the Chapman-Enskog
 * reference viscosity. */
double orc_mu(const orc_species* sp, double T)
{
    double ca = sp->c_alpha, w = sp->omega;
    double mu_ref = 5.0 * (ca + 1.0) * (ca + 2.0) * sqrt(sp->m * KB * sp->T_ref / PI)
                  / (4.0 * ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) * sp->d_ref * sp->d_ref);
    return mu_ref * pow(T / sp->T_ref, w);
}

/* Eq. tau_c: mean collision time of the VSS model, p = n k_B T. */
double orc_tau_c(const orc_species* sp, double n, double T)
{
    double ca = sp->c_alpha, w = sp->omega;
    double p = n * KB * T;
    return ca * (5.0 - 2.0 * w) * (7.0 - 2.0 * w) / (5.0 * (ca + 1.0) * (ca + 2.0))
         * orc_mu(sp, T) / p;
}

/* Sec. 4.B: Eucken Prandtl number with xi_vib as printed.  The paper does not
 * say which temperature enters xi_vib; the cell vibrational temperature is
 * used (T <= 0 gives xi = 0, the limit). */
double orc_prandtl(const orc_species* sp, double T)
{
    double xi = 0.0;
    if (T > 0.0) {
        double x = sp->theta_v / T;
        xi = x / (exp(x) - 1.0);
    }
    return (14.0 + 2.0 * xi) / (19.0 + 2.0 * xi);
}

/* Sec. 2.A (fixed numbers) or Sec. 5.C (Parker rotational number and the
 * Millikan-White number with the high-temperature term), both at T_tr. */
void orc_collision_numbers(const orc_species* sp, double T_tr, double* Zrot, double* Zvib)
{
    if (sp->zmodel == 0) { *Zrot = sp->Z_rot; *Zvib = sp->Z_vib; return; }
    double r = sp->T_star / T_tr;
    *Zrot = sp->Zrot_inf / (1.0 + 0.5 * pow(PI, 1.5) * sqrt(r) + (PI + 0.25 * PI * PI) * r);
    double zmw = (sp->C1 / pow(T_tr, sp->omega)) * exp(sp->C2 * pow(T_tr, -1.0 / 3.0));
    double zht = (PI * sp->d_ref * sp->d_ref / sp->sigma_vib) * pow(sp->T_ref / T_tr, sp->omega - 0.5);
    *Zvib = zmw + zht;
}

/* Per-cell coefficients of Sec. 3.A.1 and 3.A.2.
 *   A = (2mu/p - Pr dt)/(2mu/p + Pr dt),  alpha_tr = alpha_rot = alpha_vib = A^(1/3)
 *   B = (2mu/p - dt)/(2mu/p + dt),        nu = (B - alpha^2)/(1 - alpha^2)
 *   gamma_tr-rot, gamma_tr-vib, gamma_rot-vib with c_v,vib(T_1) where
 *   c_v,vib(T_1) = (e_vib(T_check) - e_vib(T_vib)) / (T_check - T_vib) and
 *   e_tr(T_check) = e_tr(T_tr) + gamma_tr-rot/2 (T_rot - T_tr)
 *                             + gamma_tr-vib/2 (T_vib - T_tr).
 * The paper gives no solver for this implicit pair.  Reading: fixed-point
 * iteration on c_v,vib(T_1), started at c_v,vib(T_tr), until the relative
 * change is below 1e-14 or below the rounding of the secant itself,
 * 4 eps (|e_vib(T_check)| + |e_vib(T_vib)|) / |T_check - T_vib| with
 * eps = 2^-52 (near equilibrium the secant's numerator cancels, and the
 * rounded map can settle into a cycle of that size instead of a fixed
 * point), at most 50 passes; when T_check is within 1e-9 of T_vib the secant
 * is replaced by the derivative c_v,vib(T_vib).
 * For dt >= 2 mu / (p Pr) the ratio A is negative (behind a strong shock at
 * a time step set by the freestream); reading: alpha is then the real cube
 * root, in (-1, 0), which keeps alpha^3 = A for the heat flux and
 * alpha^2 < 1 for the energies.  Returns 0, or -1 if A is not in (-1, 1)
 * (mu/p not positive and finite: a cell without a temperature). */
int orc_cell_coeffs(const orc_species* sp, double n, double dt,
                    double T_tr, double T_rot, double T_vib, orc_coeffs* o)
{
    memset(o, 0, sizeof(*o));
    double R = orc_R(sp);
    double c_tr = 1.5 * R, c_rot = R;
    o->n = n; o->dt = dt; o->T_tr = T_tr; o->T_rot = T_rot; o->T_vib = T_vib;
    o->p = n * KB * T_tr;
    o->mu = orc_mu(sp, T_tr);
    o->mu_p = o->mu / o->p;
    o->tau_c = orc_tau_c(sp, n, T_tr);
    orc_collision_numbers(sp, T_tr, &o->Z_rot, &o->Z_vib);
    o->tau_rot = o->Z_rot * o->tau_c;
    o->tau_vib = o->Z_vib * o->tau_c;
    o->Pr = orc_prandtl(sp, T_vib);

    o->A = (2.0 * o->mu_p - o->Pr * dt) / (2.0 * o->mu_p + o->Pr * dt);
    o->B = (2.0 * o->mu_p - dt) / (2.0 * o->mu_p + dt);
    if (!(o->A > -1.0 && o->A < 1.0)) return -1;
    o->alpha = cbrt(o->A);
    double a2 = o->alpha * o->alpha;
    o->nu_ref = (o->B - a2) / (1.0 - a2);

    o->g_r = dt / (dt + 2.0 * o->tau_rot);
    o->g_v = dt / (dt + 2.0 * o->tau_vib);

    double x = orc_cv_vib(sp, T_tr);
    double Tc = T_tr;
    int it = 0;
    for (it = 1; it <= 50; ++it) {
        double den = c_tr + o->g_r * c_rot + o->g_v * x;
        double gtr = 2.0 * o->g_r * c_tr * c_rot / den;
        double gtv = 2.0 * o->g_v * c_tr * x / den;
        /* e_tr(Tc) - e_tr(T_tr) = c_tr (Tc - T_tr) */
        Tc = T_tr + (0.5 * gtr * (T_rot - T_tr) + 0.5 * gtv * (T_vib - T_tr)) / c_tr;
        double xn, noise = 0.0;
        double scale = fabs(Tc) > fabs(T_vib) ? fabs(Tc) : fabs(T_vib);
        if (fabs(Tc - T_vib) <= 1e-9 * scale) {
            xn = orc_cv_vib(sp, T_vib);
        } else {
            double ec = orc_e_vib(sp, Tc), ev = orc_e_vib(sp, T_vib);
            xn = (ec - ev) / (Tc - T_vib);
            noise = 4.0 * 0x1p-52 * (fabs(ec) + fabs(ev)) / fabs(Tc - T_vib);
        }
        double change = fabs(xn - x);
        x = xn;
        if (change <= 1e-14 * fabs(xn) || change <= noise) break;
    }
    o->t1_iters = it > 50 ? 50 : it;
    o->cv_T1 = x;
    {
        double den = c_tr + o->g_r * c_rot + o->g_v * x;
        o->gamma_tr_rot = 2.0 * o->g_r * c_tr * c_rot / den;
        o->gamma_tr_vib = 2.0 * o->g_v * c_tr * x / den;
        o->gamma_rot_vib = 2.0 * o->g_r * o->g_v * c_rot * x / den;
        o->T_check = T_tr + (0.5 * o->gamma_tr_rot * (T_rot - T_tr)
                           + 0.5 * o->gamma_tr_vib * (T_vib - T_tr)) / c_tr;
    }
    /* Eqs. e_tr_relax, e_rot_relax, e_vib_relax */
    o->e_tr_tgt = c_tr * T_tr - o->gamma_tr_rot * (T_tr - T_rot) - o->gamma_tr_vib * (T_tr - T_vib);
    o->e_rot_tgt = c_rot * T_rot + o->gamma_tr_rot * (T_tr - T_rot) - o->gamma_rot_vib * (T_rot - T_vib);
    o->e_vib_tgt = orc_e_vib(sp, T_vib) + o->gamma_tr_vib * (T_tr - T_vib) + o->gamma_rot_vib * (T_rot - T_vib);
    /* For dt far above tau_rot the exchange terms overshoot and a target can
     * come out negative (strong non-equilibrium, e.g. a near-empty cut cell);
     * reading: such a target is 0 (the velocity rescale of Sec. 4.C still
     * conserves the cell's energy). */
    o->tgt_clamped = 0;
    if (o->e_rot_tgt < 0.0) { o->e_rot_tgt = 0.0; o->tgt_clamped = 1; }
    if (o->e_vib_tgt < 0.0) { o->e_vib_tgt = 0.0; o->tgt_clamped = 1; }
    return 0;
}

/* Eqs. T_tr_USP, T_rot_USP, T_vib_USP.  The vibrational equation is printed
 * with 1 - alpha_rot^2; all three alphas are equal (also after the positivity
 * fix, Eq. alpha_USP_positivity_4), so the one alpha passed in is used.
 * Negative results (possible only for very large dt) are clamped to zero and
 * flagged. */
static void relaxation_temperatures(const orc_species* sp, const orc_coeffs* cc, double alpha,
                                    double T_tr, double T_rot, double T_vib,
                                    double* T_tr_rel, double* T_rot_rel, double* e_vib_rel,
                                    uint32_t* flags, orc_declog* dl)
{
    double R = orc_R(sp);
    double oma2 = 1.0 - alpha * alpha;
    double ttr = T_tr - (cc->gamma_tr_rot * (T_tr - T_rot) + cc->gamma_tr_vib * (T_tr - T_vib))
                        / (oma2 * 1.5 * R);
    double tro = T_rot + (cc->gamma_tr_rot * (T_tr - T_rot) - cc->gamma_rot_vib * (T_rot - T_vib))
                        / (oma2 * R);
    double evr = orc_e_vib(sp, T_vib)
               + (cc->gamma_tr_vib * (T_tr - T_vib) + cc->gamma_rot_vib * (T_rot - T_vib)) / oma2;
    if (dec_b(dl, ttr < 0.0)) { ttr = 0.0; *flags |= ORC_F_TREL_CLAMP; }
    if (dec_b(dl, tro < 0.0)) { tro = 0.0; *flags |= ORC_F_TREL_CLAMP; }
    if (dec_b(dl, evr < 0.0)) { evr = 0.0; *flags |= ORC_F_TREL_CLAMP; }
    *T_tr_rel = ttr; *T_rot_rel = tro; *e_vib_rel = evr;
}

void orc_relaxation_temperatures(const orc_species* sp, const orc_coeffs* cc, double alpha,
                                 double T_tr, double T_rot, double T_vib,
                                 double* T_tr_rel, double* T_rot_rel, double* e_vib_rel,
                                 uint32_t* flags)
{
    relaxation_temperatures(sp, cc, alpha, T_tr, T_rot, T_vib, T_tr_rel, T_rot_rel, e_vib_rel,
                            flags, NULL);
}

/* ======================================================================== */
/* Linear algebra                                                           */
/* ======================================================================== */
/* Smallest and largest eigenvalue of a symmetric 3x3 matrix stored as
 * (xx, yy, zz, xy, xz, yz): the trigonometric closed form of the cubic. */
void orc_sym3_eig_minmax(const double P[6], double* lmin, double* lmax)
{
    double a = P[0], b = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
    double p1 = d * d + e * e + f * f;
    if (p1 == 0.0) {
        double lo = a, hi = a;
        if (b < lo) lo = b; if (c < lo) lo = c;
        if (b > hi) hi = b; if (c > hi) hi = c;
        *lmin = lo; *lmax = hi; return;
    }
    double q = (a + b + c) / 3.0;
    double p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0 * p1;
    double p = sqrt(p2 / 6.0);
    double b11 = (a - q) / p, b22 = (b - q) / p, b33 = (c - q) / p;
    double b12 = d / p, b13 = e / p, b23 = f / p;
    double det = b11 * (b22 * b33 - b23 * b23) - b12 * (b12 * b33 - b23 * b13)
               + b13 * (b12 * b23 - b22 * b13);
    double r = det / 2.0;
    if (r < -1.0) r = -1.0;
    if (r > 1.0) r = 1.0;
    double phi = acos(r) / 3.0;
    *lmax = q + 2.0 * p * cos(phi);
    *lmin = q + 2.0 * p * cos(phi + 2.0 * PI / 3.0);
}

/* Cholesky factor L (l00, l10, l11, l20, l21, l22) of M = (xx, yy, zz, xy, xz,
 * yz); returns 0 if a pivot is not positive (M not positive definite). */
int orc_cholesky3(const double M[6], double L[6])
{
    double m00 = M[0], m11 = M[1], m22 = M[2], m10 = M[3], m20 = M[4], m21 = M[5];
    if (!(m00 > 0.0)) return 0;
    double l00 = sqrt(m00);
    double l10 = m10 / l00;
    double l20 = m20 / l00;
    double d1 = m11 - l10 * l10;
    if (!(d1 > 0.0)) return 0;
    double l11 = sqrt(d1);
    double l21 = (m21 - l20 * l10) / l11;
    double d2 = m22 - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0)) return 0;
    double l22 = sqrt(d2);
    L[0] = l00; L[1] = l10; L[2] = l11; L[3] = l20; L[4] = l21; L[5] = l22;
    return 1;
}

/* ======================================================================== */
/* Discrete samplers for Eq. update_evib.  The paper fixes the distributions */
/* (negative binomial for up-jumps, binomial for down-jumps) but no sampler. */
/* Reading: sequential inversion with one uniform each, the pmf stepped by   */
/* its ratio recursion; P(0) by square-and-multiply; a binomial with p > 1/2 */
/* is drawn as n - B(n, 1 - p) with the same uniform.  The search stops when */
/* the cdf can no longer grow in the working precision.  Form 1 runs the     */
/* search in float (falling back to double when P(0) is not a normal float). */
/* ======================================================================== */
static double powi_d(double x, int e)
{
    double r = 1.0, b = x;
    while (e > 0) { if (e & 1) r = r * b; b = b * b; e >>= 1; }
    return r;
}
static float powi_f(float x, int e)
{
    float r = 1.0f, b = x;
    while (e > 0) { if (e & 1) r = r * b; b = b * b; e >>= 1; }
    return r;
}

/* NB(r, p): number of failures before the r-th success, P(0) = p^r,
 * P(k+1) = P(k) (k + r)/(k + 1) (1 - p). */
static int nb_d(int r, double p, double u, uint32_t* flags)
{
    double q = 1.0 - p;
    double P = powi_d(p, r);
    if (P < DBL_MIN) {
        *flags |= ORC_F_SAMPLER_UNDERFLOW;
        return (int)floor(r * q / p);
    }
    double cdf = P;
    int k = 0;
    while (u >= cdf) {
        if (k >= SAMPLER_KCAP) { *flags |= ORC_F_SAMPLER_CAP; break; }
        double t = (double)(k + r) / (double)(k + 1);
        P = P * t;
        P = P * q;
        k = k + 1;
        double nc = cdf + P;
        if (nc == cdf) break;
        cdf = nc;
    }
    return k;
}
static int nb_f(int r, float p, float u, uint32_t* flags)
{
    float q = 1.0f - p;
    float P = powi_f(p, r);
    if (P < FLT_MIN) return nb_d(r, (double)p, (double)u, flags);
    float cdf = P;
    int k = 0;
    while (u >= cdf) {
        if (k >= SAMPLER_KCAP) { *flags |= ORC_F_SAMPLER_CAP; break; }
        float t = (float)(k + r) / (float)(k + 1);
        P = P * t;
        P = P * q;
        k = k + 1;
        float nc = cdf + P;
        if (nc == cdf) break;
        cdf = nc;
    }
    return k;
}

/* B(n, p) for 0 < p <= 1/2: P(0) = (1-p)^n, P(k+1) = P(k) (n-k)/(k+1) p/(1-p). */
static int binv_d(int n, double p, double u, uint32_t* flags)
{
    double q = 1.0 - p;
    double P = powi_d(q, n);
    if (P < DBL_MIN) {
        *flags |= ORC_F_SAMPLER_UNDERFLOW;
        return (int)floor(n * p);
    }
    double pq = p / q;
    double cdf = P;
    int k = 0;
    while (u >= cdf && k < n) {
        if (k >= SAMPLER_KCAP) { *flags |= ORC_F_SAMPLER_CAP; break; }
        double t = (double)(n - k) / (double)(k + 1);
        P = P * t;
        P = P * pq;
        k = k + 1;
        double nc = cdf + P;
        if (nc == cdf) break;
        cdf = nc;
    }
    return k;
}
static int binv_f(int n, float p, float u, uint32_t* flags)
{
    float q = 1.0f - p;
    float P = powi_f(q, n);
    if (P < FLT_MIN) return binv_d(n, (double)p, (double)u, flags);
    float pq = p / q;
    float cdf = P;
    int k = 0;
    while (u >= cdf && k < n) {
        if (k >= SAMPLER_KCAP) { *flags |= ORC_F_SAMPLER_CAP; break; }
        float t = (float)(n - k) / (float)(k + 1);
        P = P * t;
        P = P * pq;
        k = k + 1;
        float nc = cdf + P;
        if (nc == cdf) break;
        cdf = nc;
    }
    return k;
}

int orc_sample_nb(int r, double p, double u, int form, uint32_t* flags)
{
    if (r <= 0) return 0;
    if (form == 1) {
        float pf = (float)p;
        if (!(pf < 1.0f)) return 0;
        return nb_f(r, pf, (float)u, flags);
    }
    if (!(p < 1.0)) return 0;
    return nb_d(r, p, u, flags);
}

int orc_sample_b(int n, double p, double u, int form, uint32_t* flags)
{
    if (n <= 0) return 0;
    if (form == 1) {
        float pf = (float)p;
        if (pf >= 1.0f) { if (pf > 1.0f) *flags |= ORC_F_PB_CLAMP; return n; }
        if (!(pf > 0.0f)) return 0;
        if (pf > 0.5f) return n - binv_f(n, 1.0f - pf, (float)u, flags);
        return binv_f(n, pf, (float)u, flags);
    }
    if (p >= 1.0) { if (p > 1.0) *flags |= ORC_F_PB_CLAMP; return n; }
    if (!(p > 0.0)) return 0;
    if (p > 0.5) return n - binv_d(n, 1.0 - p, u, flags);
    return binv_d(n, p, u, flags);
}

/* ======================================================================== */
/* One particle through the collision step (Sec. 4.D):                      */
/*   relaxation temperatures (Eqs. T_tr_USP, T_rot_USP, T_vib_USP),         */
/*   M = tau D_tr = R T_tr^rel I + nu (Pi - R T_tr I)        (Eq. D_tr),     */
/*   Cholesky test; on failure the nu / alpha adjustment of Sec. 3.A.3,     */
/*   then Eqs. update_ci, update_erot and update_evib.                      */
/* U, Pi, T_* are the macroscopic fields at the particle (cell values, or   */
/* interpolated ones).  G holds four standard normals; u5, u6 the uniforms  */
/* of the two jump samplers.                                                */
/* Positivity-fix readings (the paper gives the rule, not these details):   */
/*  - a bound whose denominator is not positive does not restrict nu;       */
/*  - the adjusted nu is shrunk by (1 - 1e-6) so M is strictly definite;    */
/*  - alpha^2 from Eq. alpha_USP_positivity_1 is clamped to [0, 1 - 1e-12]; */
/*  - of +-sqrt(alpha^2) the one whose Pr (Eq. alpha_USP_positivity_3) is   */
/*    nearest the target wins, ties to +;                                   */
/*  - the relaxation temperatures are re-evaluated with the new alpha and   */
/*    the test repeated; since T_tr^rel depends on alpha, the bound is      */
/*    re-taken from the new T_tr^rel, at most four passes; if D_tr is still */
/*    not definite, nu = 0 with alpha^2 = B (counted); only a T_tr^rel of   */
/*    zero then is flagged as a failure.                                    */
/* ======================================================================== */
static void collide_particle(const orc_species* sp, int form, const orc_coeffs* cc,
                             const double U[3], const double Pi[6],
                             double T_tr, double T_rot, double T_vib,
                             const double G[4], double u5, double u6,
                             double c[3], double* erot, int32_t* lev,
                             uint32_t* flags, int64_t* counters, orc_declog* dl)
{
    double R = orc_R(sp);
    double alpha = cc->alpha;
    double nu = cc->nu_ref;
    double Ttr_rel, Trot_rel, evib_rel;
    uint32_t tf = 0;
    relaxation_temperatures(sp, cc, alpha, T_tr, T_rot, T_vib, &Ttr_rel, &Trot_rel, &evib_rel, &tf, dl);

    double M[6], L[6];
    M[0] = R * Ttr_rel + nu * (Pi[0] - R * T_tr);
    M[1] = R * Ttr_rel + nu * (Pi[1] - R * T_tr);
    M[2] = R * Ttr_rel + nu * (Pi[2] - R * T_tr);
    M[3] = nu * Pi[3];
    M[4] = nu * Pi[4];
    M[5] = nu * Pi[5];
    if (!dec_b(dl, orc_cholesky3(M, L))) {
        counters[ORC_C_CHOL_FIX] += 1;
        double lmin, lmax;
        orc_sym3_eig_minmax(Pi, &lmin, &lmax);
        int ok = 0;
        for (int pass = 0; pass < 4 && !ok; ++pass) {
            /* Eq. nu_USP_positivity with the current T_tr^rel */
            double nref = cc->nu_ref;
            nu = nref;
            if (dec_b(dl, nref <= 0.0)) {
                if (dec_b(dl, lmax - R * T_tr > 0.0)) {
                    double bound = -R * Ttr_rel / (lmax - R * T_tr);
                    if (dec_b(dl, bound > nu)) nu = bound;
                }
            } else {
                if (dec_b(dl, R * T_tr - lmin > 0.0)) {
                    double bound = R * Ttr_rel / (R * T_tr - lmin);
                    if (dec_b(dl, bound < nu)) nu = bound;
                }
            }
            nu = nu * (1.0 - 1e-6);
            /* Eqs. alpha_USP_positivity_1 .. _4 */
            double a2 = (nu - cc->B) / (nu - 1.0);
            if (dec_b(dl, a2 < 0.0)) a2 = 0.0;
            if (dec_b(dl, a2 > 1.0 - 1e-12)) a2 = 1.0 - 1e-12;
            double ap = sqrt(a2), am = -ap;
            double prp = 2.0 * cc->mu_p * (1.0 - ap * ap * ap) / (cc->dt * (1.0 + ap * ap * ap));
            double prm = 2.0 * cc->mu_p * (1.0 - am * am * am) / (cc->dt * (1.0 + am * am * am));
            alpha = dec_b(dl, fabs(prm - cc->Pr) < fabs(prp - cc->Pr)) ? am : ap;
            relaxation_temperatures(sp, cc, alpha, T_tr, T_rot, T_vib, &Ttr_rel, &Trot_rel, &evib_rel, &tf, dl);
            M[0] = R * Ttr_rel + nu * (Pi[0] - R * T_tr);
            M[1] = R * Ttr_rel + nu * (Pi[1] - R * T_tr);
            M[2] = R * Ttr_rel + nu * (Pi[2] - R * T_tr);
            M[3] = nu * Pi[3];
            M[4] = nu * Pi[4];
            M[5] = nu * Pi[5];
            ok = dec_b(dl, orc_cholesky3(M, L));
        }
        if (!ok) {
            /* the passes approach the admissible nu from outside when
             * T_tr^rel moves with alpha; fall back to nu = 0, inside the
             * admissible range of Eq. nu_USP_positivity whenever
             * T_tr^rel > 0, with alpha^2 = B from Eq. alpha_USP_positivity_1
             * at nu = 0 and the sign chosen as above */
            counters[ORC_C_NU_ZERO] += 1;
            nu = 0.0;
            double a2 = cc->B;
            if (dec_b(dl, a2 < 0.0)) a2 = 0.0;
            if (dec_b(dl, a2 > 1.0 - 1e-12)) a2 = 1.0 - 1e-12;
            double ap = sqrt(a2), am = -ap;
            double prp = 2.0 * cc->mu_p * (1.0 - ap * ap * ap) / (cc->dt * (1.0 + ap * ap * ap));
            double prm = 2.0 * cc->mu_p * (1.0 - am * am * am) / (cc->dt * (1.0 + am * am * am));
            alpha = dec_b(dl, fabs(prm - cc->Pr) < fabs(prp - cc->Pr)) ? am : ap;
            relaxation_temperatures(sp, cc, alpha, T_tr, T_rot, T_vib, &Ttr_rel, &Trot_rel, &evib_rel, &tf, dl);
            int pos = dec_b(dl, Ttr_rel > 0.0);
            double s = pos ? sqrt(R * Ttr_rel) : 0.0;
            if (!pos) *flags |= ORC_F_CHOL_FAIL_AFTER_FIX;
            L[0] = s; L[1] = 0.0; L[2] = s; L[3] = 0.0; L[4] = 0.0; L[5] = s;
        }
    }
    if (tf) { *flags |= tf; counters[ORC_C_TREL_CLAMP] += 1; }

    /* Eq. update_ci: C^{n+1} = alpha C^n + sqrt(1 - alpha^2) L G, with
     * L L^T = tau D_tr (the tau of Eq. update_ci cancels). */
    double a2 = alpha * alpha;
    double sq = sqrt(1.0 - a2);
    double LG0 = L[0] * G[0];
    double LG1 = L[1] * G[0] + L[2] * G[1];
    double LG2 = L[3] * G[0] + L[4] * G[1] + L[5] * G[2];
    c[0] = U[0] + alpha * (c[0] - U[0]) + sq * LG0;
    c[1] = U[1] + alpha * (c[1] - U[1]) + sq * LG1;
    c[2] = U[2] + alpha * (c[2] - U[2]) + sq * LG2;

    /* Eq. update_erot */
    double a = R * Trot_rel * (1.0 - a2) / 2.0;
    double root = sqrt(*erot) * alpha + sqrt(a) * G[3];
    *erot = a + root * root;

    /* Eq. update_evib with its parameters r_NB, p_NB, n_B, p_B (the p_N of the
     * printed p_B equation is p_B).  exp(Theta/T_rel) / (exp(Theta/T_rel) - 1)
     * = 1 + ebar_rel with ebar_rel = e_vib(T_vib^rel) / (R Theta). */
    double ebar = evib_rel / (R * sp->theta_v);
    double p_nb = 1.0 / (1.0 + ebar * (1.0 - a2));
    double p_b = (1.0 + ebar) * (1.0 - a2);
    int I = *lev;
    uint32_t sf = 0;
    int up = (int)dec_i(dl, orc_sample_nb(I + 1, p_nb, u5, form, &sf));
    int dn = (int)dec_i(dl, orc_sample_b(I, p_b, u6, form, &sf));
    if (sf & ORC_F_PB_CLAMP) counters[ORC_C_PB_CLAMP] += 1;
    *flags |= sf;
    *lev = I + up - dn;
}

void orc_collide_particle(const orc_species* sp, int form, const orc_coeffs* cc,
                          const double U[3], const double Pi[6],
                          double T_tr, double T_rot, double T_vib,
                          const double G[4], double u5, double u6,
                          double c[3], double* erot, int32_t* lev,
                          uint32_t* flags, int64_t* counters)
{
    collide_particle(sp, form, cc, U, Pi, T_tr, T_rot, T_vib, G, u5, u6, c, erot, lev, flags,
                     counters, NULL);
}

/* ======================================================================== */
/* Moments of Sec. 2.A per cell, with ensemble averages read as sample      */
/* means over the particles of the cell (1/N):                              */
/*   out fields: 0 N | 1-3 U | 4 T_tr | 5 T_rot | 6 T_vib |                */
/*   7-12 Pi (xx yy zz xy xz yz) | 13-15 q_tr | 16-18 q_rot | 19-21 q_vib   */
/* with T_tr = tr(Pi) / 3R, T_rot = <eps_rot>/R, T_vib from <I>, and heat   */
/* fluxes per unit mass: q_tr = <C^2 C>/2, q_rot = <C eps>, q_vib =         */
/* <C I R Theta>.  Cells with no particle give zeros.                       */
/* ======================================================================== */
void orc_moments(const orc_species* sp, int ncell, const int64_t* off,
                 const double* cx, const double* cy, const double* cz,
                 const double* erot, const int32_t* lev, double* out)
{
    double R = orc_R(sp);
    for (int f = 0; f < ORC_NMOM * ncell; ++f) out[f] = 0.0;
    for (int ci = 0; ci < ncell; ++ci) {
        int64_t b = off[ci], e = off[ci + 1];
        int64_t N = e - b;
        if (N <= 0) continue;
        double U[3] = { 0, 0, 0 }, er = 0.0, lv = 0.0;
        for (int64_t j = b; j < e; ++j) { U[0] += cx[j]; U[1] += cy[j]; U[2] += cz[j]; er += erot[j]; lv += lev[j]; }
        U[0] /= N; U[1] /= N; U[2] /= N; er /= N; lv /= N;
        double P[6] = { 0, 0, 0, 0, 0, 0 }, qt[3] = { 0, 0, 0 }, qr[3] = { 0, 0, 0 }, qv[3] = { 0, 0, 0 };
        for (int64_t j = b; j < e; ++j) {
            double C0 = cx[j] - U[0], C1 = cy[j] - U[1], C2 = cz[j] - U[2];
            double C2s = C0 * C0 + C1 * C1 + C2 * C2;
            P[0] += C0 * C0; P[1] += C1 * C1; P[2] += C2 * C2;
            P[3] += C0 * C1; P[4] += C0 * C2; P[5] += C1 * C2;
            qt[0] += 0.5 * C2s * C0; qt[1] += 0.5 * C2s * C1; qt[2] += 0.5 * C2s * C2;
            qr[0] += C0 * erot[j]; qr[1] += C1 * erot[j]; qr[2] += C2 * erot[j];
            double ev = lev[j] * R * sp->theta_v;
            qv[0] += C0 * ev; qv[1] += C1 * ev; qv[2] += C2 * ev;
        }
        for (int k = 0; k < 6; ++k) P[k] /= N;
        for (int k = 0; k < 3; ++k) { qt[k] /= N; qr[k] /= N; qv[k] /= N; }
        out[0 * ncell + ci] = (double)N;
        for (int k = 0; k < 3; ++k) out[(1 + k) * ncell + ci] = U[k];
        out[4 * ncell + ci] = (P[0] + P[1] + P[2]) / (3.0 * R);
        out[5 * ncell + ci] = er / R;
        out[6 * ncell + ci] = orc_T_vib_from_mean_level(sp, lv);
        for (int k = 0; k < 6; ++k) out[(7 + k) * ncell + ci] = P[k];
        for (int k = 0; k < 3; ++k) {
            out[(13 + k) * ncell + ci] = qt[k];
            out[(16 + k) * ncell + ci] = qr[k];
            out[(19 + k) * ncell + ci] = qv[k];
        }
    }
}

/* ======================================================================== */
/* Conservation scheme of Sec. 4.C on the particles [b, e) of one cell.     */
/* Inputs: the step-n cell energies (e_tr^n, e_rot^n, e_vib^n), the         */
/* step-n bulk velocity U^n, the targets e_rot(T_rot^{n+1}) and             */
/* e_vib(T_vib^{n+1}) of Eqs. e_rot_relax and e_vib_relax.                  */
/* Readings:                                                                 */
/*  - int() is the floor, so the added uniform gives unbiased rounding;     */
/*  - "a particle is randomly selected": position k = floor(w N / 2^32) of  */
/*    the j-th cell draw w, with replacement; a decrement that meets a      */
/*    level-0 particle draws again; at most 64 N draws;                     */
/*  - the velocity rescale uses the actual post-correction rotational and   */
/*    vibrational means; a non-positive radicand leaves the velocities      */
/*    unchanged and is flagged.                                             */
/* ======================================================================== */
#define CELL_TAG(t) (0x80000000u | (uint32_t)(t))
#define CELL_TAG_IDELTA 0
#define CELL_TAG_PICK 1

static void conserve_cell(const orc_species* sp, uint64_t seed, uint32_t cell, uint32_t step,
                          int64_t b, int64_t e,
                          double e_tr_n, double e_rot_n, double e_vib_n, const double Un[3],
                          double e_rot_tgt, double e_vib_tgt,
                          double* cx, double* cy, double* cz, double* erot, int32_t* lev,
                          uint32_t* flags, int64_t* counters, orc_declog* dl)
{
    double R = orc_R(sp);
    double Rth = R * sp->theta_v;
    int64_t N = e - b;
    uint32_t w[4];

    /* vibrational: summation-based correction */
    int64_t sumI = 0;
    for (int64_t j = b; j < e; ++j) sumI += lev[j];
    philox_words(cell, step, CELL_TAG(CELL_TAG_IDELTA), 0u, seed, w);
    double u = orc_uniform(w[0], 0);
    int64_t Id = dec_i(dl, (int64_t)floor((double)N * e_vib_tgt / Rth - (double)sumI + u));
    int64_t draws = 0, cap = 64 * N;
    while (Id != 0) {
        if (draws >= cap) { *flags |= ORC_F_VIB_LOOP_CAP; break; }
        uint32_t blk = (uint32_t)(draws >> 2);
        philox_words(cell, step, CELL_TAG(CELL_TAG_PICK), blk, seed, w);
        uint32_t word = w[draws & 3];
        draws += 1;
        int64_t k = (int64_t)(((uint64_t)word * (uint64_t)N) >> 32);
        if (Id > 0) { lev[b + k] += 1; Id -= 1; }
        else if (lev[b + k] > 0) { lev[b + k] -= 1; Id += 1; }
    }
    counters[ORC_C_VIB_DRAWS] += draws;

    /* rotational: scaling-based correction */
    double er_star = 0.0;
    for (int64_t j = b; j < e; ++j) er_star += erot[j];
    er_star /= N;
    if (dec_b(dl, er_star > 0.0)) {
        double r = e_rot_tgt / er_star;
        for (int64_t j = b; j < e; ++j) erot[j] = r * erot[j];
    }

    /* translational: momentum and total energy */
    double e_rot_new = 0.0, lv = 0.0;
    for (int64_t j = b; j < e; ++j) { e_rot_new += erot[j]; lv += lev[j]; }
    e_rot_new /= N;
    double e_vib_new = Rth * lv / N;
    double Us[3] = { 0, 0, 0 };
    for (int64_t j = b; j < e; ++j) { Us[0] += cx[j]; Us[1] += cy[j]; Us[2] += cz[j]; }
    Us[0] /= N; Us[1] /= N; Us[2] /= N;
    double etr_star = 0.0;
    for (int64_t j = b; j < e; ++j) {
        double d0 = cx[j] - Us[0], d1 = cy[j] - Us[1], d2 = cz[j] - Us[2];
        etr_star += 0.5 * (d0 * d0 + d1 * d1 + d2 * d2);
    }
    etr_star /= N;
    double rad = (e_tr_n + e_rot_n + e_vib_n - e_rot_new - e_vib_new) / etr_star;
    if (dec_b(dl, !(etr_star > 0.0) || !(rad > 0.0))) {
        *flags |= ORC_F_NEG_RADICAND;
        counters[ORC_C_NEG_RADICAND] += 1;
        return;
    }
    double s = sqrt(rad);
    for (int64_t j = b; j < e; ++j) {
        cx[j] = Un[0] + s * (cx[j] - Us[0]);
        cy[j] = Un[1] + s * (cy[j] - Us[1]);
        cz[j] = Un[2] + s * (cz[j] - Us[2]);
    }
}

/* Collision-stream draws of one particle: four normals (two Box-Muller
 * pairs of a radius and an angle uniform) and the two uniforms of the jump
 * samplers, from the one Philox block with counter (pid, step, 0, 0), in
 * both forms.  A uniform takes 23 bits of a word, (2 (x >> 9) + 1) 2^-24
 * (orc_uniform form 1, exact in float), so the block carries all six: the
 * radius uniforms from words 0 and 1, the jump uniforms from words 2 and 3,
 * and the two angle uniforms (2a + 1) 2^-19 from the 18-bit
 * a = (low 9 bits of word 0) << 9 | (low 9 bits of word 1), then of words 2
 * and 3.  The reading is the project's (the paper names no generator). */
#define PTAG_NORMALS 0u
static double angle_uniform18(uint32_t wa, uint32_t wb)
{
    uint32_t a = ((wa & 0x1FFu) << 9) | (wb & 0x1FFu);
    return (2.0 * (double)a + 1.0) * 0x1p-19;
}

static void particle_draws(uint64_t seed, uint32_t pid, uint32_t step, int form,
                           double G[4], double* u5, double* u6)
{
    uint32_t w[4];
    (void)form;
    philox_words(pid, step, PTAG_NORMALS, 0u, seed, w);
    box_muller(orc_uniform(w[0], 1), angle_uniform18(w[0], w[1]), &G[0], &G[1]);
    box_muller(orc_uniform(w[1], 1), angle_uniform18(w[2], w[3]), &G[2], &G[3]);
    *u5 = orc_uniform(w[2], 1);
    *u6 = orc_uniform(w[3], 1);
}

void orc_particle_draws(uint64_t seed, uint32_t pid, uint32_t step, int form,
                        double G[4], double* u5, double* u6)
{
    particle_draws(seed, pid, step, form, G, u5, u6);
}

/* ======================================================================== */
/* Independent homogeneous cells (Sec. 5.A set-up): for every step, every   */
/* cell runs the collision step of Sec. 4.D with its cell-averaged fields   */
/* (no reconstruction), then the conservation scheme.  Cells with fewer    */
/* than two particles are left unchanged (reading: their moments are not    */
/* defined).  The density of each cell stays fixed (no transport).          */
/* ======================================================================== */
int orc_homog_step(const orc_species* sp, int form, uint64_t seed,
                   int64_t step0, int nsteps, int n_inst, const int64_t* off,
                   const double* ndens, const double* dt,
                   double* cx, double* cy, double* cz, double* erot,
                   int32_t* lev, const uint32_t* pid,
                   uint32_t* flags, int64_t* counters)
{
    double R = orc_R(sp);
    int status = 0;
    for (int s = 0; s < nsteps; ++s) {
        uint32_t step = (uint32_t)(step0 + s);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int ci = 0; ci < n_inst; ++ci) {
            uint32_t lflags = 0;
            int64_t lcnt[ORC_NCOUNTERS] = { 0 };
            int64_t b = off[ci], e = off[ci + 1];
            int64_t N = e - b;
            if (N < 2) { lcnt[ORC_C_SKIPPED_CELLS] += 1; goto merge; }
            {
                /* cell moments, Sec. 2.A */
                double U[3] = { 0, 0, 0 }, er = 0.0, lv = 0.0, P[6] = { 0, 0, 0, 0, 0, 0 };
                for (int64_t j = b; j < e; ++j) { U[0] += cx[j]; U[1] += cy[j]; U[2] += cz[j]; er += erot[j]; lv += lev[j]; }
                U[0] /= N; U[1] /= N; U[2] /= N; er /= N; lv /= N;
                for (int64_t j = b; j < e; ++j) {
                    double C0 = cx[j] - U[0], C1 = cy[j] - U[1], C2 = cz[j] - U[2];
                    P[0] += C0 * C0; P[1] += C1 * C1; P[2] += C2 * C2;
                    P[3] += C0 * C1; P[4] += C0 * C2; P[5] += C1 * C2;
                }
                for (int k = 0; k < 6; ++k) P[k] /= N;
                double T_tr = (P[0] + P[1] + P[2]) / (3.0 * R);
                double T_rot = er / R;
                double T_vib = orc_T_vib_from_mean_level(sp, lv);

                orc_coeffs cc;
                if (orc_cell_coeffs(sp, ndens[ci], dt[ci], T_tr, T_rot, T_vib, &cc) != 0) {
                    lflags |= ORC_F_A_NONPOS;
                    goto merge;
                }
                if (cc.tgt_clamped) { lflags |= ORC_F_TREL_CLAMP; lcnt[ORC_C_TREL_CLAMP] += 1; }
                for (int64_t j = b; j < e; ++j) {
                    double G[4], u5, u6, c[3] = { cx[j], cy[j], cz[j] };
                    uint32_t id = pid ? pid[j] : (uint32_t)j;
                    particle_draws(seed, id, step, form, G, &u5, &u6);
                    orc_collide_particle(sp, form, &cc, U, P, T_tr, T_rot, T_vib, G, u5, u6,
                                         c, &erot[j], &lev[j], &lflags, lcnt);
                    cx[j] = c[0]; cy[j] = c[1]; cz[j] = c[2];
                }
                conserve_cell(sp, seed, (uint32_t)ci, step, b, e,
                              1.5 * R * T_tr, R * T_rot, orc_e_vib(sp, T_vib), U,
                              cc.e_rot_tgt, cc.e_vib_tgt, cx, cy, cz, erot, lev, &lflags, lcnt, NULL);
            }
        merge:
#ifdef _OPENMP
#pragma omp critical(orc_merge)
#endif
            {
                *flags |= lflags;
                for (int k = 0; k < ORC_NCOUNTERS; ++k) counters[k] += lcnt[k];
            }
        }
        if (*flags & ORC_F_A_NONPOS) status = -1;
    }
    return status;
}

/* ======================================================================== */
/* The plain FPM method (Sec. 2.B model, Sec. 2.C particle scheme).          */
/* ======================================================================== */
#define PTAG_GILLESPIE 8u

/* Per-cell coefficients of the FPM method:
 *   nu = 1 - 3/(2 Pr) (the Pr the model reproduces), tau = 2 mu (1 - nu)/p,
 *   alpha = exp(-dt/tau) (Eq. conventionial-velo: C exp(-dt/tau) and the
 *   noise amplitude sqrt(tau (1 - exp(-2dt/tau))) d = sqrt(1 - alpha^2) L
 *   with L L^T = tau D_tr);
 *   relaxation energies of Eqs. T_tr_FPM, T_rot_FPM, T_vib_FPM with
 *   tau_rot = Z_rot tau_c and tau_vib = Z_vib tau_c (Landau-Teller, Sec. 2.A);
 *   a negative relaxation energy is set to 0 (flagged), as in the USP form.
 *   Gillespie rates of the master-equation term: with
 *   ebar_rel = e_vib(T_vib^rel)/(R Theta) = q/(1-q), q = exp(-Theta/T_vib^rel),
 *   omega_{I,I+1} = 2 (I+1) q / (tau (1-q)) = 2 (I+1) ebar_rel / tau and
 *   omega_{I,I-1} = 2 I / (tau (1-q)) = 2 I (1 + ebar_rel) / tau; times dt
 *   they are lam_up (I+1) and lam_dn I.
 * Reading (the paper applies the conservation scheme of Sec. 4.C to its
 * methods but states targets only for the USP form): the targets are the
 * expected mode energies after dt under the FPM update itself,
 *   e_rot^{n+1} = e_rot(T_rot^rel) + (e_rot^n - e_rot(T_rot^rel)) alpha^2,
 *   e_vib^{n+1} = e_vib_rel + (e_vib^n - e_vib_rel) alpha^2
 * (the Milstein square form gives E[eps'] = alpha^2 eps + (1 - alpha^2) R T^rel;
 * the linear birth-death rates above move the mean level at rate 2/tau toward
 * ebar_rel). */
int orc_fpm_coeffs(const orc_species* sp, double n, double dt,
                   double T_tr, double T_rot, double T_vib, orc_fpm* o)
{
    memset(o, 0, sizeof(*o));
    double R = orc_R(sp);
    o->n = n; o->dt = dt; o->T_tr = T_tr; o->T_rot = T_rot; o->T_vib = T_vib;
    o->p = n * KB * T_tr;
    o->mu = orc_mu(sp, T_tr);
    o->tau_c = orc_tau_c(sp, n, T_tr);
    orc_collision_numbers(sp, T_tr, &o->Z_rot, &o->Z_vib);
    o->tau_rot = o->Z_rot * o->tau_c;
    o->tau_vib = o->Z_vib * o->tau_c;
    o->Pr = orc_prandtl(sp, T_vib);
    o->nu = 1.0 - 3.0 / (2.0 * o->Pr);
    o->tau = 2.0 * o->mu * (1.0 - o->nu) / o->p;
    if (!(o->tau > 0.0)) return -1;
    o->alpha = exp(-dt / o->tau);

    double grot = o->tau / (2.0 * o->tau_rot), gvib = o->tau / (2.0 * o->tau_vib);
    double e_tr = 1.5 * R * T_tr, e_rot = R * T_rot, e_vib = orc_e_vib(sp, T_vib);
    double e_tr_rel = e_tr + grot * (R * T_rot - R * T_tr) + gvib * (e_vib - orc_e_vib(sp, T_tr));
    double e_rot_rel = e_rot + grot * (R * T_tr - R * T_rot);
    double e_vib_rel = e_vib + gvib * (orc_e_vib(sp, T_tr) - e_vib);
    if (e_tr_rel < 0.0) { e_tr_rel = 0.0; o->clamped = 1; }
    if (e_rot_rel < 0.0) { e_rot_rel = 0.0; o->clamped = 1; }
    if (e_vib_rel < 0.0) { e_vib_rel = 0.0; o->clamped = 1; }
    o->T_tr_rel = e_tr_rel / (1.5 * R);
    o->T_rot_rel = e_rot_rel / R;
    o->e_vib_rel = e_vib_rel;

    double ebar_rel = e_vib_rel / (R * sp->theta_v);
    o->lam_up = 2.0 * dt * ebar_rel / o->tau;
    o->lam_dn = 2.0 * dt * (1.0 + ebar_rel) / o->tau;

    double a2 = o->alpha * o->alpha;
    o->e_rot_tgt = e_rot_rel + (e_rot - e_rot_rel) * a2;
    o->e_vib_tgt = e_vib_rel + (e_vib - e_vib_rel) * a2;
    return 0;
}

/* Gillespie's direct method over one step (Sec. 2.C), time in units of dt:
 * the waiting time to the next transition is -ln(U1) / rate with
 * rate = lam_up (I+1) + lam_dn I; the step ends when the accumulated time
 * passes 1; otherwise U2 < lam_up (I+1) / rate raises the level, else it is
 * lowered.  Draws: counter (pid, step, 8, k) gives the (U1, U2) pairs of
 * transitions 2k and 2k+1.  Form 1 takes every operation in float. */
#define GILLESPIE_CAP 4096
int orc_gillespie(int I, double lam_up, double lam_dn, uint64_t seed, uint32_t pid,
                  uint32_t step, int form, uint32_t* flags)
{
    uint32_t w[4];
    if (form == 1) {
        float lu = (float)lam_up, ld = (float)lam_dn, t = 0.0f;
        for (int ev = 0; ev < GILLESPIE_CAP; ++ev) {
            if ((ev & 1) == 0) philox_words(pid, step, PTAG_GILLESPIE, (uint32_t)(ev >> 1), seed, w);
            float u1 = (float)orc_uniform(w[(ev & 1) * 2], 1);
            float u2 = (float)orc_uniform(w[(ev & 1) * 2 + 1], 1);
            float up = lu * (float)(I + 1), dn = ld * (float)I;
            float rate = up + dn;
            if (!(rate > 0.0f)) return I;
            float wait = -logf(u1) / rate;
            t = t + wait;
            if (t > 1.0f) return I;
            if (u2 < up / rate) I += 1; else I -= 1;
        }
    } else {
        double t = 0.0;
        for (int ev = 0; ev < GILLESPIE_CAP; ++ev) {
            if ((ev & 1) == 0) philox_words(pid, step, PTAG_GILLESPIE, (uint32_t)(ev >> 1), seed, w);
            double u1 = orc_uniform(w[(ev & 1) * 2], 0);
            double u2 = orc_uniform(w[(ev & 1) * 2 + 1], 0);
            double up = lam_up * (double)(I + 1), dn = lam_dn * (double)I;
            double rate = up + dn;
            if (!(rate > 0.0)) return I;
            double wait = -log(u1) / rate;
            t = t + wait;
            if (t > 1.0) return I;
            if (u2 < up / rate) I += 1; else I -= 1;
        }
    }
    *flags |= ORC_F_SAMPLER_CAP;
    return I;
}

/* One particle of the FPM method: Eq. conventionial-velo (C = c - U,
 * c' = U + alpha C + sqrt(1 - alpha^2) L G with L L^T = tau D_tr =
 * R T_tr^rel I + nu (Pi - R T_tr I), Eq. D_tr), Eq. conventionial-erot
 * (the same square form as the USP rotational update with this alpha), and
 * the Gillespie levels.  Reading (Sec. 2 gives no positivity fix for the FPM
 * method): when tau D_tr is not positive definite, nu is limited to the
 * admissible bound of Eq. nu_USP_positivity (times 1 - 1e-6), and if the
 * factorisation still fails nu = 0; alpha stays exp(-dt/tau). */
void orc_collide_particle_fpm(const orc_species* sp, int form, const orc_fpm* fc,
                              const double U[3], const double Pi[6], const double G[4],
                              uint64_t seed, uint32_t pid, uint32_t step,
                              double c[3], double* erot, int32_t* lev,
                              uint32_t* flags, int64_t* counters)
{
    double R = orc_R(sp);
    double nu = fc->nu;
    double RT = R * fc->T_tr, RTrel = R * fc->T_tr_rel;
    double M[6], L[6];
    M[0] = RTrel + nu * (Pi[0] - RT);
    M[1] = RTrel + nu * (Pi[1] - RT);
    M[2] = RTrel + nu * (Pi[2] - RT);
    M[3] = nu * Pi[3];
    M[4] = nu * Pi[4];
    M[5] = nu * Pi[5];
    if (!orc_cholesky3(M, L)) {
        counters[ORC_C_CHOL_FIX] += 1;
        double lmin, lmax;
        orc_sym3_eig_minmax(Pi, &lmin, &lmax);
        if (nu <= 0.0) {
            if (lmax - RT > 0.0) { double bd = -RTrel / (lmax - RT); if (bd > nu) nu = bd; }
        } else {
            if (RT - lmin > 0.0) { double bd = RTrel / (RT - lmin); if (bd < nu) nu = bd; }
        }
        nu = nu * (1.0 - 1e-6);
        M[0] = RTrel + nu * (Pi[0] - RT);
        M[1] = RTrel + nu * (Pi[1] - RT);
        M[2] = RTrel + nu * (Pi[2] - RT);
        M[3] = nu * Pi[3];
        M[4] = nu * Pi[4];
        M[5] = nu * Pi[5];
        if (!orc_cholesky3(M, L)) {
            counters[ORC_C_NU_ZERO] += 1;
            double s = RTrel > 0.0 ? sqrt(RTrel) : 0.0;
            if (!(RTrel > 0.0)) *flags |= ORC_F_CHOL_FAIL_AFTER_FIX;
            L[0] = s; L[1] = 0.0; L[2] = s; L[3] = 0.0; L[4] = 0.0; L[5] = s;
        }
    }
    double alpha = fc->alpha, a2 = alpha * alpha, sq = sqrt(1.0 - a2);
    double LG0 = L[0] * G[0];
    double LG1 = L[1] * G[0] + L[2] * G[1];
    double LG2 = L[3] * G[0] + L[4] * G[1] + L[5] * G[2];
    c[0] = U[0] + alpha * (c[0] - U[0]) + sq * LG0;
    c[1] = U[1] + alpha * (c[1] - U[1]) + sq * LG1;
    c[2] = U[2] + alpha * (c[2] - U[2]) + sq * LG2;

    double a = R * fc->T_rot_rel * (1.0 - a2) / 2.0;
    double root = sqrt(*erot) * alpha + sqrt(a) * G[3];
    *erot = a + root * root;

    *lev = orc_gillespie(*lev, fc->lam_up, fc->lam_dn, seed, pid, step, form, flags);
}

/* Steps of independent homogeneous cells with the FPM method: the cell
 * loop of orc_homog_step with orc_fpm_coeffs, orc_collide_particle_fpm and
 * the conservation scheme of Sec. 4.C with the FPM targets. */
int orc_homog_step_fpm(const orc_species* sp, int form, uint64_t seed,
                       int64_t step0, int nsteps, int n_inst, const int64_t* off,
                       const double* ndens, const double* dt,
                       double* cx, double* cy, double* cz, double* erot,
                       int32_t* lev, const uint32_t* pid,
                       uint32_t* flags, int64_t* counters)
{
    double R = orc_R(sp);
    int status = 0;
    for (int s = 0; s < nsteps; ++s) {
        uint32_t step = (uint32_t)(step0 + s);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
        for (int ci = 0; ci < n_inst; ++ci) {
            uint32_t lflags = 0;
            int64_t lcnt[ORC_NCOUNTERS] = { 0 };
            int64_t b = off[ci], e = off[ci + 1];
            int64_t N = e - b;
            if (N < 2) { lcnt[ORC_C_SKIPPED_CELLS] += 1; goto merge; }
            {
                double U[3] = { 0, 0, 0 }, er = 0.0, lv = 0.0, P[6] = { 0, 0, 0, 0, 0, 0 };
                for (int64_t j = b; j < e; ++j) { U[0] += cx[j]; U[1] += cy[j]; U[2] += cz[j]; er += erot[j]; lv += lev[j]; }
                U[0] /= N; U[1] /= N; U[2] /= N; er /= N; lv /= N;
                for (int64_t j = b; j < e; ++j) {
                    double C0 = cx[j] - U[0], C1 = cy[j] - U[1], C2 = cz[j] - U[2];
                    P[0] += C0 * C0; P[1] += C1 * C1; P[2] += C2 * C2;
                    P[3] += C0 * C1; P[4] += C0 * C2; P[5] += C1 * C2;
                }
                for (int k = 0; k < 6; ++k) P[k] /= N;
                double T_tr = (P[0] + P[1] + P[2]) / (3.0 * R);
                double T_rot = er / R;
                double T_vib = orc_T_vib_from_mean_level(sp, lv);

                orc_fpm fc;
                if (orc_fpm_coeffs(sp, ndens[ci], dt[ci], T_tr, T_rot, T_vib, &fc) != 0) {
                    lflags |= ORC_F_A_NONPOS;
                    goto merge;
                }
                if (fc.clamped) { lflags |= ORC_F_TREL_CLAMP; lcnt[ORC_C_TREL_CLAMP] += 1; }
                for (int64_t j = b; j < e; ++j) {
                    double G[4], u5, u6, c[3] = { cx[j], cy[j], cz[j] };
                    uint32_t id = pid ? pid[j] : (uint32_t)j;
                    particle_draws(seed, id, step, form, G, &u5, &u6);
                    orc_collide_particle_fpm(sp, form, &fc, U, P, G, seed, id, step,
                                             c, &erot[j], &lev[j], &lflags, lcnt);
                    cx[j] = c[0]; cy[j] = c[1]; cz[j] = c[2];
                }
                conserve_cell(sp, seed, (uint32_t)ci, step, b, e,
                              1.5 * R * T_tr, R * T_rot, orc_e_vib(sp, T_vib), U,
                              fc.e_rot_tgt, fc.e_vib_tgt, cx, cy, cz, erot, lev, &lflags, lcnt, NULL);
            }
        merge:
#ifdef _OPENMP
#pragma omp critical(orc_merge_fpm)
#endif
            {
                *flags |= lflags;
                for (int k = 0; k < ORC_NCOUNTERS; ++k) counters[k] += lcnt[k];
            }
        }
        if (*flags & ORC_F_A_NONPOS) status = -1;
    }
    return status;
}

/* ======================================================================== */
/* 1D channel between two fully diffuse plates (the Poiseuille set-up of    */
/* Sec. 5.B, force-driven).  One step, in the order of the host particle    */
/* framework the paper builds on: move (with wall interaction) -> sort by   */
/* cell -> collision step of Sec. 4.D per cell -> conservation (Sec. 4.C).  */
/* ======================================================================== */
#define PTAG_WALL_A 2u
#define PTAG_WALL_B 3u
#define WALL_HIT_CAP 16
#define NFIELD 13   /* U(3), T_tr, T_rot, T_vib, Pi(6) */

/* Fully diffuse wall at T_w (Sec. 5.B: "fully diffusive" walls; reading:
 * full accommodation of velocity, rotational energy and vibrational level).
 * Normal speed from the flux-weighted half-range Maxwellian (Rayleigh with
 * variance R T_w), tangential components Maxwellian, eps_rot exponential with
 * mean R T_w, level geometric at T_w.  Draws: counters (pid, step, 2, hit)
 * and (pid, step, 3, hit). */
static void diffuse_reemit(const orc_species* sp, int form, uint64_t seed, uint32_t pid,
                           uint32_t step, int hit, double Tw, int into_positive_y,
                           double* cx, double* cy, double* cz, double* erot, int32_t* lev,
                           orc_declog* dl)
{
    double R = orc_R(sp);
    uint32_t w[4], v[4];
    philox_words(pid, step, PTAG_WALL_A, (uint32_t)hit, seed, w);
    philox_words(pid, step, PTAG_WALL_B, (uint32_t)hit, seed, v);
    double vn = sqrt(-2.0 * R * Tw * log(orc_uniform(w[0], form)));
    *cy = into_positive_y ? vn : -vn;
    double g1, g2;
    box_muller(orc_uniform(w[1], form), orc_uniform(w[2], form), &g1, &g2);
    double s = sqrt(R * Tw);
    *cx = s * g1;
    *cz = s * g2;
    *erot = -R * Tw * log(orc_uniform(w[3], form));
    /* P(I >= k) = exp(-k Theta / T_w)  ->  I = floor(-ln(u) T_w / Theta) */
    *lev = (int32_t)dec_i(dl, (int64_t)floor(-log(orc_uniform(v[0], form)) * Tw / sp->theta_v));
}

void orc_wall_reemit(const orc_species* sp, int form, uint64_t seed, uint32_t pid, uint32_t step,
                     int hit, double Tw, int into_positive_y, double out[4], int32_t* lev)
{
    diffuse_reemit(sp, form, seed, pid, step, hit, Tw, into_positive_y,
                   &out[0], &out[1], &out[2], &out[3], lev, NULL);
}

/* Ballistic flight over dt with the body force along x, reflecting off the
 * diffuse plates at y = 0 and y = L; a hit re-emits the particle and the
 * flight continues for the rest of the step.  Returns the x-momentum (per
 * unit mass) handed to the walls. */
static double advect_channel(const orc_species* sp, int form, uint64_t seed, uint32_t step,
                             const orc_channel* ch, double dt, double* y, double* cx, double* cy,
                             double* cz, double* erot, int32_t* lev, uint32_t pid,
                             uint32_t* flags, int64_t* counters, orc_declog* dl)
{
    double t_left = dt, mom = 0.0;
    int hits = 0;
    for (;;) {
        double yn = *y + *cy * t_left;
        if (dec_b(dl, yn >= 0.0 && yn <= ch->L)) {
            *y = yn;
            *cx += ch->g * t_left;
            break;
        }
        if (hits >= WALL_HIT_CAP) {
            *flags |= ORC_F_WALL_CAP;
            *y = dec_b(dl, yn < 0.0) ? 0.0 : ch->L;
            *cx += ch->g * t_left;
            break;
        }
        double wall = dec_b(dl, yn < 0.0) ? 0.0 : ch->L;
        /* the time of a wall event is held with the event itself */
        double t_hit = dec_d(dl, (wall - *y) / *cy);
        if (dec_b(dl, t_hit < 0.0)) t_hit = 0.0;
        if (dec_b(dl, t_hit > t_left)) t_hit = t_left;
        *cx += ch->g * t_hit;
        mom += *cx;
        *y = wall;
        t_left -= t_hit;
        diffuse_reemit(sp, form, seed, pid, step, hits, ch->T_wall, wall == 0.0,
                       cx, cy, cz, erot, lev, dl);
        mom -= *cx;
        hits += 1;
        counters[ORC_C_WALL_HITS] += 1;
    }
    /* the position after the move is held with the cell it selects */
    *y = dec_d(dl, *y);
    return mom;
}

static int channel_cell(const orc_channel* ch, double y)
{
    double dy = ch->L / ch->ny;
    int c = (int)floor(y / dy);
    if (c < 0) c = 0;
    if (c >= ch->ny) c = ch->ny - 1;
    return c;
}

/* First-order reconstruction of Sec. 3.B in one dimension: of the quadrant
 * stencils only the part along y remains, a straight line through the cell
 * average at the centroid and the neighbour's average at its centroid, the
 * neighbour being on the particle's side of the centroid (ties to +), or on
 * the opposite side when that neighbour is a wall or holds fewer than two
 * particles; with neither neighbour usable the cell value is used. */
static void channel_reconstruct(const orc_channel* ch, const int64_t* counts, const double* F,
                                int cell, double y, double* out, orc_declog* dl)
{
    double dy = ch->L / ch->ny;
    double yc = (cell + 0.5) * dy;
    int s = dec_b(dl, y >= yc) ? 1 : -1;
    int nb = cell + s;
    if (nb < 0 || nb >= ch->ny || counts[nb] < 2) {
        nb = cell - s;
        if (nb < 0 || nb >= ch->ny || counts[nb] < 2) nb = -1;
    }
    for (int f = 0; f < NFIELD; ++f) {
        double fc = F[cell * NFIELD + f];
        if (nb < 0) { out[f] = fc; continue; }
        double fn = F[nb * NFIELD + f];
        out[f] = fc + (fn - fc) * (y - yc) / ((nb - cell) * dy);
    }
}

void orc_channel_reconstruct(const orc_channel* ch, const int64_t* counts, const double* F,
                             int cell, double y, double* out)
{
    channel_reconstruct(ch, counts, F, cell, y, out, NULL);
}

/* stable reorder of all particle arrays by cell index */
static void sort_by_cell(const orc_channel* ch, int64_t n, double* y, double* cx, double* cy,
                         double* cz, double* erot, int32_t* lev, uint32_t* pid, int64_t* off,
                         orc_declog* dl)
{
    int ny = ch->ny;
    int* cell = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int64_t* pos = (int64_t*)calloc(ny + 1, sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j) {
        int c = (int)dec_i(dl, channel_cell(ch, y[j]));
        if (c < 0 || c >= ny) {
            if (dl) dl->overruns += 1;
            c = channel_cell(ch, y[j]);
        }
        cell[j] = c;
        pos[cell[j] + 1] += 1;
    }
    for (int c = 0; c < ny; ++c) pos[c + 1] += pos[c];
    for (int c = 0; c <= ny; ++c) off[c] = pos[c];
    double* tmp = (double*)malloc(sizeof(double) * 5 * (n > 0 ? n : 1));
    int32_t* tl = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    uint32_t* tp = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) {
        int64_t k = pos[cell[j]]++;
        tmp[k] = y[j]; tmp[n + k] = cx[j]; tmp[2 * n + k] = cy[j]; tmp[3 * n + k] = cz[j];
        tmp[4 * n + k] = erot[j]; tl[k] = lev[j]; tp[k] = pid[j];
    }
    memcpy(y, tmp, sizeof(double) * n); memcpy(cx, tmp + n, sizeof(double) * n);
    memcpy(cy, tmp + 2 * n, sizeof(double) * n); memcpy(cz, tmp + 3 * n, sizeof(double) * n);
    memcpy(erot, tmp + 4 * n, sizeof(double) * n);
    memcpy(lev, tl, sizeof(int32_t) * n); memcpy(pid, tp, sizeof(uint32_t) * n);
    free(tmp); free(tl); free(tp); free(cell); free(pos);
}

static int channel_step(const orc_species* sp, int form, uint64_t seed, int64_t step0,
                        int nsteps, const orc_channel* ch, double dt, int64_t n,
                        double* y, double* cx, double* cy, double* cz, double* erot,
                        int32_t* lev, uint32_t* pid, int64_t* cell_off, double* acc,
                        uint32_t* flags, int64_t* counters, orc_declog* dl)
{
    double R = orc_R(sp);
    int ny = ch->ny;
    double dy = ch->L / ny;
    double vol = ch->area * dy;
    double* F = (double*)malloc(sizeof(double) * NFIELD * ny);
    double* cellT = (double*)malloc(sizeof(double) * 3 * ny);
    int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * ny);
    orc_coeffs* cc = (orc_coeffs*)malloc(sizeof(orc_coeffs) * ny);
    orc_fpm* fcs = ch->method == 1 ? (orc_fpm*)malloc(sizeof(orc_fpm) * ny) : NULL;
    int* ok = (int*)malloc(sizeof(int) * ny);
    int status = 0;
    for (int s = 0; s < nsteps; ++s) {
        uint32_t step = (uint32_t)(step0 + s);
        /* 1. move */
        double wall_mom = 0.0;
        for (int64_t j = 0; j < n; ++j)
            wall_mom += advect_channel(sp, form, seed, step, ch, dt, &y[j], &cx[j], &cy[j], &cz[j],
                                       &erot[j], &lev[j], pid[j], flags, counters, dl);
        /* 2. sort */
        sort_by_cell(ch, n, y, cx, cy, cz, erot, lev, pid, cell_off, dl);
        /* 3. cell moments and coefficients */
        for (int c = 0; c < ny; ++c) {
            int64_t b = cell_off[c], e = cell_off[c + 1], N = e - b;
            counts[c] = N;
            ok[c] = 0;
            for (int f = 0; f < NFIELD; ++f) F[c * NFIELD + f] = 0.0;
            if (N < 2) { counters[ORC_C_SKIPPED_CELLS] += 1; continue; }
            double U[3] = { 0, 0, 0 }, er = 0.0, lv = 0.0, P[6] = { 0, 0, 0, 0, 0, 0 };
            for (int64_t j = b; j < e; ++j) { U[0] += cx[j]; U[1] += cy[j]; U[2] += cz[j]; er += erot[j]; lv += lev[j]; }
            U[0] /= N; U[1] /= N; U[2] /= N; er /= N; lv /= N;
            for (int64_t j = b; j < e; ++j) {
                double C0 = cx[j] - U[0], C1 = cy[j] - U[1], C2 = cz[j] - U[2];
                P[0] += C0 * C0; P[1] += C1 * C1; P[2] += C2 * C2;
                P[3] += C0 * C1; P[4] += C0 * C2; P[5] += C1 * C2;
            }
            for (int k = 0; k < 6; ++k) P[k] /= N;
            double T_tr = (P[0] + P[1] + P[2]) / (3.0 * R);
            double T_rot = er / R;
            double T_vib = orc_T_vib_from_mean_level(sp, lv);
            double* Fc = &F[c * NFIELD];
            Fc[0] = U[0]; Fc[1] = U[1]; Fc[2] = U[2];
            Fc[3] = T_tr; Fc[4] = T_rot; Fc[5] = T_vib;
            for (int k = 0; k < 6; ++k) Fc[6 + k] = P[k];
            cellT[3 * c] = T_tr; cellT[3 * c + 1] = T_rot; cellT[3 * c + 2] = T_vib;
            double nd = N * ch->F_num / vol;
            if (fcs) {
                /* the plain FPM method: per-cell coefficients of Sec. 2.B */
                if (orc_fpm_coeffs(sp, nd, dt, T_tr, T_rot, T_vib, &fcs[c]) != 0) {
                    *flags |= ORC_F_A_NONPOS;
                    status = -1;
                    continue;
                }
                if (fcs[c].clamped) { *flags |= ORC_F_TREL_CLAMP; counters[ORC_C_TREL_CLAMP] += 1; }
                ok[c] = 1;
                continue;
            }
            int bad = orc_cell_coeffs(sp, nd, dt, T_tr, T_rot, T_vib, &cc[c]) != 0;
            if (dec_b(dl, bad)) {
                *flags |= ORC_F_A_NONPOS;
                status = -1;
                continue;
            }
            if (cc[c].tgt_clamped) { *flags |= ORC_F_TREL_CLAMP; counters[ORC_C_TREL_CLAMP] += 1; }
            ok[c] = 1;
        }
        /* 4. particles: reconstruction (Sec. 3.B) and collision (Sec. 4.D) */
        for (int c = 0; c < ny; ++c) {
            if (!ok[c]) continue;
            const double* Fc = &F[c * NFIELD];
            for (int64_t j = cell_off[c]; j < cell_off[c + 1]; ++j) {
                if (fcs) {
                    /* FPM: the cell values at every particle (first order) */
                    double G[4], u5, u6, cv[3] = { cx[j], cy[j], cz[j] };
                    particle_draws(seed, pid[j], step, form, G, &u5, &u6);
                    orc_collide_particle_fpm(sp, form, &fcs[c], Fc, Fc + 6, G, seed, pid[j], step,
                                             cv, &erot[j], &lev[j], flags, counters);
                    cx[j] = cv[0]; cy[j] = cv[1]; cz[j] = cv[2];
                    continue;
                }
                double f[NFIELD];
                if (ch->reconstruct) {
                    channel_reconstruct(ch, counts, F, c, y[j], f, dl);
                    if (dec_b(dl, !(f[3] > 0.0) || !(f[4] > 0.0) || !(f[5] >= 0.0))) {
                        counters[ORC_C_INTERP_FALLBACK] += 1;
                        memcpy(f, Fc, sizeof(f));
                    }
                } else {
                    memcpy(f, Fc, sizeof(f));
                }
                double G[4], u5, u6, cv[3] = { cx[j], cy[j], cz[j] };
                particle_draws(seed, pid[j], step, form, G, &u5, &u6);
                collide_particle(sp, form, &cc[c], f, f + 6, f[3], f[4], f[5], G, u5, u6,
                                 cv, &erot[j], &lev[j], flags, counters, dl);
                cx[j] = cv[0]; cy[j] = cv[1]; cz[j] = cv[2];
            }
        }
        /* 5. conservation per cell with the cell-averaged step-n values */
        for (int c = 0; c < ny; ++c) {
            if (!ok[c]) continue;
            const double* Fc = &F[c * NFIELD];
            conserve_cell(sp, seed, (uint32_t)c, step, cell_off[c], cell_off[c + 1],
                          1.5 * R * cellT[3 * c], R * cellT[3 * c + 1], orc_e_vib(sp, cellT[3 * c + 2]),
                          Fc, fcs ? fcs[c].e_rot_tgt : cc[c].e_rot_tgt,
                          fcs ? fcs[c].e_vib_tgt : cc[c].e_vib_tgt, cx, cy, cz, erot, lev, flags,
                          counters, dl);
        }
        /* 6. time-average sums */
        if (acc) {
            for (int c = 0; c < ny; ++c) {
                double* a = &acc[c * ORC_NACC];
                for (int64_t j = cell_off[c]; j < cell_off[c + 1]; ++j) {
                    a[0] += 1.0;
                    a[1] += cx[j]; a[2] += cy[j]; a[3] += cz[j];
                    a[4] += cx[j] * cx[j]; a[5] += cy[j] * cy[j]; a[6] += cz[j] * cz[j];
                    a[7] += cx[j] * cy[j]; a[8] += cx[j] * cz[j]; a[9] += cy[j] * cz[j];
                    a[10] += erot[j]; a[11] += lev[j];
                }
            }
            acc[ny * ORC_NACC] += 1.0;
            acc[ny * ORC_NACC + 1] += wall_mom;
        }
    }
    free(F); free(cellT); free(counts); free(cc); free(fcs); free(ok);
    return status;
}

int orc_channel_step(const orc_species* sp, int form, uint64_t seed, int64_t step0,
                     int nsteps, const orc_channel* ch, double dt, int64_t n,
                     double* y, double* cx, double* cy, double* cz, double* erot,
                     int32_t* lev, uint32_t* pid, int64_t* cell_off, double* acc,
                     uint32_t* flags, int64_t* counters)
{
    return channel_step(sp, form, seed, step0, nsteps, ch, dt, n, y, cx, cy, cz, erot, lev, pid,
                        cell_off, acc, flags, counters, NULL);
}

int orc_channel_step_frozen(const orc_species* sp, int form, uint64_t seed, int64_t step0,
                            int nsteps, const orc_channel* ch, double dt, int64_t n,
                            double* y, double* cx, double* cy, double* cz, double* erot,
                            int32_t* lev, uint32_t* pid, int64_t* cell_off, double* acc,
                            uint32_t* flags, int64_t* counters, orc_declog* dl)
{
    if (ch->method != 0) return -3;
    return channel_step(sp, form, seed, step0, nsteps, ch, dt, n, y, cx, cy, cz, erot, lev, pid,
                        cell_off, acc, flags, counters, dl);
}

/* ======================================================================== */
/* 2D plane flow past a circular cylinder (the set-up of Sec. 5.C: half    */
/* body on a specular symmetry plane, fully diffuse cylinder at T_wall,    */
/* freestream inflow, outflow).  One step: move (events: cylinder, sides)  */
/* -> inject the freestream through inflow sides -> drop particles that    */
/* left -> stable sort by cell -> collision step per cell (fields          */
/* reconstructed per Sec. 3.B) -> conservation (Sec. 4.C).                 */
/* ======================================================================== */
#define PTAG_INFLOW_P 5u
#define PTAG_INFLOW_T 6u
#define PTAG_INFLOW_V 7u
#define CELL_TAG_INFLOW 4
#define INFLOW_TRY_CAP 64
#define NSIDES 4

static double plane_dx(const orc_plane* pl) { return (pl->x1 - pl->x0) / pl->nx; }
static double plane_dy(const orc_plane* pl) { return (pl->y1 - pl->y0) / pl->ny; }

static int plane_l1(const orc_plane* pl, double x, double y, int* pi, int* pj)
{
    int i = (int)floor((x - pl->x0) / plane_dx(pl));
    int j = (int)floor((y - pl->y0) / plane_dy(pl));
    if (i < 0) i = 0;
    if (i >= pl->nx) i = pl->nx - 1;
    if (j < 0) j = 0;
    if (j >= pl->ny) j = pl->ny - 1;
    *pi = i;
    *pj = j;
    return j * pl->nx + i;
}

/* ---- refined grid (Sec. 5.C: three levels, each doubling the resolution) -- */
typedef struct {
    int levels, nleaf;
    int balanced;         /* 1: no level-1 fluid leaf touches a level-3 leaf       */
    int* l1_first;        /* nx*ny + 1: first leaf of each level-1 cell            */
    int* l2_first;        /* 4 nx ny: first leaf of each level-2 child; -1 = none  */
    signed char* l2_ref;  /* 4 nx ny: 1 when that level-2 cell is split again      */
    int* level;           /* per leaf                                              */
    int* ii;              /* per leaf: integer coordinates at its own level (the   */
    int* jj;              /* centre is x0 + (ii + 1/2) dx / 2^(level-1))           */
} amr_grid;

static int amr_levels(const orc_plane* pl) { return pl->amr_levels >= 2 ? pl->amr_levels : 1; }

/* centre of the square (xl, yl) + (w, h) within radius r of the cylinder centre */
static int centre_within(const orc_plane* pl, double xl, double yl, double w, double h, double r)
{
    double ex = xl + 0.5 * w - pl->cyl_xc, ey = yl + 0.5 * h - pl->cyl_yc;
    return ex * ex + ey * ey < r * r;
}

/* the square lies inside the body (its four corners within the radius):
 * it holds no fluid and is not split */
static int square_solid(const orc_plane* pl, double xl, double yl, double w, double h)
{
    if (!(pl->cyl_r > 0.0)) return 0;
    double r2 = pl->cyl_r * pl->cyl_r;
    for (int q = 0; q < 4; ++q) {
        double ex = xl + (q & 1) * w - pl->cyl_xc, ey = yl + (q >> 1) * h - pl->cyl_yc;
        if (ex * ex + ey * ey > r2) return 0;
    }
    return 1;
}

static void amr_build(const orc_plane* pl, amr_grid* g)
{
    int nx = pl->nx, ny = pl->ny, n1 = nx * ny;
    double dx = plane_dx(pl), dy = plane_dy(pl);
    g->levels = amr_levels(pl);
    g->l1_first = (int*)malloc(sizeof(int) * (n1 + 1));
    g->l2_first = (int*)malloc(sizeof(int) * 4 * n1);
    g->l2_ref = (signed char*)calloc(4 * (size_t)n1, 1);
    /* pass 1: count */
    int nleaf = 0;
    for (int c = 0; c < n1; ++c) {
        int i = c % nx, j = c / nx;
        g->l1_first[c] = nleaf;
        double xl = pl->x0 + i * dx, yl = pl->y0 + j * dy;
        int split = g->levels >= 2 && centre_within(pl, xl, yl, dx, dy, pl->amr_r2) &&
                    !square_solid(pl, xl, yl, dx, dy);
        if (!split) {
            for (int k = 0; k < 4; ++k) g->l2_first[4 * c + k] = -1;
            nleaf += 1;
            continue;
        }
        for (int k = 0; k < 4; ++k) {
            double x2 = xl + (k & 1) * 0.5 * dx, y2 = yl + (k >> 1) * 0.5 * dy;
            int s3 = g->levels >= 3 && centre_within(pl, x2, y2, 0.5 * dx, 0.5 * dy, pl->amr_r3) &&
                     !square_solid(pl, x2, y2, 0.5 * dx, 0.5 * dy);
            g->l2_first[4 * c + k] = nleaf;
            g->l2_ref[4 * c + k] = (signed char)s3;
            nleaf += s3 ? 4 : 1;
        }
    }
    g->l1_first[n1] = nleaf;
    g->nleaf = nleaf;
    g->level = (int*)malloc(sizeof(int) * nleaf);
    g->ii = (int*)malloc(sizeof(int) * nleaf);
    g->jj = (int*)malloc(sizeof(int) * nleaf);
    /* pass 2: geometry */
    for (int c = 0; c < n1; ++c) {
        int i = c % nx, j = c / nx;
        if (g->l2_first[4 * c] < 0) {
            int l = g->l1_first[c];
            g->level[l] = 1; g->ii[l] = i; g->jj[l] = j;
            continue;
        }
        for (int k = 0; k < 4; ++k) {
            int i2 = 2 * i + (k & 1), j2 = 2 * j + (k >> 1);
            int l = g->l2_first[4 * c + k];
            if (!g->l2_ref[4 * c + k]) {
                g->level[l] = 2; g->ii[l] = i2; g->jj[l] = j2;
                continue;
            }
            for (int q = 0; q < 4; ++q) {
                g->level[l + q] = 3;
                g->ii[l + q] = 2 * i2 + (q & 1);
                g->jj[l + q] = 2 * j2 + (q >> 1);
            }
        }
    }
    /* levels of neighbouring leaves differ by at most one (the reconstruction
     * of Sec. 3.B takes the four finer cells over a neighbour's square): every
     * level-1 cell holding level-3 leaves has its eight neighbours split or
     * inside the body */
    g->balanced = 1;
    for (int c = 0; c < n1 && g->balanced; ++c) {
        int deep = 0;
        for (int k = 0; k < 4; ++k) deep |= g->l2_ref[4 * c + k];
        if (!deep) continue;
        int i = c % nx, j = c / nx;
        for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
                int a = i + di, b = j + dj;
                if (a < 0 || a >= nx || b < 0 || b >= ny || (di == 0 && dj == 0)) continue;
                int m = b * nx + a;
                if (g->l2_first[4 * m] < 0 &&
                    !square_solid(pl, pl->x0 + a * dx, pl->y0 + b * dy, dx, dy))
                    g->balanced = 0;
            }
    }
}

static void amr_free(amr_grid* g)
{
    free(g->l1_first); free(g->l2_first); free(g->l2_ref);
    free(g->level); free(g->ii); free(g->jj);
}

/* the leaf holding (x, y): the level-1 cell as on the uniform grid, then
 * the half (and quarter) of it the point lies in, from its offset within the
 * cell */
static int amr_leaf(const orc_plane* pl, const amr_grid* g, double x, double y)
{
    int i, j;
    int c = plane_l1(pl, x, y, &i, &j);
    if (g->levels < 2 || g->l2_first[4 * c] < 0) return g->l1_first[c];
    double dx = plane_dx(pl), dy = plane_dy(pl);
    double ux = (x - (pl->x0 + i * dx)) / (0.5 * dx), uy = (y - (pl->y0 + j * dy)) / (0.5 * dy);
    int ci = ux >= 1.0 ? 1 : 0, cj = uy >= 1.0 ? 1 : 0;
    int k = cj * 2 + ci;
    int l = g->l2_first[4 * c + k];
    if (!g->l2_ref[4 * c + k]) return l;
    double vx = (ux - ci) * 2.0, vy = (uy - cj) * 2.0;
    int qi = vx >= 1.0 ? 1 : 0, qj = vy >= 1.0 ? 1 : 0;
    return l + qj * 2 + qi;
}

int orc_plane_nleaf(const orc_plane* pl)
{
    amr_grid g;
    amr_build(pl, &g);
    int n = g.balanced ? g.nleaf : -1;
    amr_free(&g);
    return n;
}

void orc_plane_leaves(const orc_plane* pl, int32_t* level, int32_t* ii, int32_t* jj)
{
    amr_grid g;
    amr_build(pl, &g);
    for (int l = 0; l < g.nleaf; ++l) { level[l] = g.level[l]; ii[l] = g.ii[l]; jj[l] = g.jj[l]; }
    amr_free(&g);
}

int orc_plane_leaf_of(const orc_plane* pl, double x, double y)
{
    amr_grid g;
    amr_build(pl, &g);
    int l = amr_leaf(pl, &g, x, y);
    amr_free(&g);
    return l;
}

/* One-way number flux through a surface element of a drifting Maxwellian
 * (density n, R T, drift u_n along the inward normal): the kinetic-theory
 * result n sqrt(RT / 2 pi) [exp(-s^2) + sqrt(pi) s (1 + erf s)], s = u_n / sqrt(2RT). */
double orc_inflow_flux(double n, double RT, double u_n)
{
    double s = u_n / sqrt(2.0 * RT);
    return n * sqrt(RT / (2.0 * PI)) * (exp(-s * s) + sqrt(PI) * s * (1.0 + erf(s)));
}

/* Inward normal speed of an entering particle: density proportional to
 * w exp(-(w - s)^2) on w > 0 (w = v_n / sqrt(2RT), s = u_n / sqrt(2RT)).
 * The paper does not say how its host code samples inflow; reading:
 * rejection sampling, attempt k drawing the block (pid, step, 7, k).
 *  - s >= 0: proposal (|w - s| + s) exp(-(w - s)^2) on the real line, a
 *    mixture of a two-sided Rayleigh in t = w - s (weight 1; |t| =
 *    sqrt(-ln u1), sign from u2) and a Gaussian t = z / sqrt(2) (weight
 *    s sqrt(pi); z from u1, u2 by Box-Muller), component chosen by u0;
 *    accepted if w > 0 and u3 (|t| + s) <= w;
 *  - s < 0: proposal 2 w exp(-w^2) on w > 0 (w = sqrt(-ln u1)), accepted if
 *    u3 <= exp(2 s w).
 * After 64 rejected attempts the mean of the proposal is used and flagged. */
double orc_inflow_normal_speed(double RT, double u_n, uint32_t pid, uint32_t step, uint64_t seed,
                               int form, uint32_t* flags)
{
    double sc = sqrt(2.0 * RT);
    double s = u_n / sc;
    double p1 = 1.0 / (1.0 + s * sqrt(PI));
    for (int k = 0; k < INFLOW_TRY_CAP; ++k) {
        uint32_t w[4];
        philox_words(pid, step, PTAG_INFLOW_V, (uint32_t)k, seed, w);
        double u0 = orc_uniform(w[0], form), u1 = orc_uniform(w[1], form);
        double u2 = orc_uniform(w[2], form), u3 = orc_uniform(w[3], form);
        if (s < 0.0) {
            double wn = sqrt(-log(u1));
            if (u3 <= exp(2.0 * s * wn)) return wn * sc;
            continue;
        }
        double t;
        if (u0 < p1) {
            t = sqrt(-log(u1));
            if (u2 < 0.5) t = -t;
        } else {
            double g1, g2;
            box_muller(u1, u2, &g1, &g2);
            t = g1 / sqrt(2.0);
        }
        double wn = s + t;
        if (!(wn > 0.0)) continue;
        if (u3 * (fabs(t) + s) <= wn) return wn * sc;
    }
    *flags |= ORC_F_INFLOW_CAP;
    return (s > 0.0 ? s : 0.5 * sqrt(PI)) * sc;
}

/* flight of one particle for t_left with events; returns 0 if it left the
 * domain through an open side (to be dropped) */
static int advect_plane(const orc_species* sp, int form, uint64_t seed, uint32_t step,
                        const orc_plane* pl, double t_left, double* x, double* y, double* cx,
                        double* cy, double* cz, double* erot, int32_t* lev, uint32_t pid,
                        double* surf, uint32_t* flags, int64_t* counters)
{
    double R = orc_R(sp);
    int hits = 0;
    for (;;) {
        /* earliest event in (0, t_left]: 0 cylinder, 1 left, 2 right, 3 bottom, 4 top */
        int ev = -1;
        double te = t_left;
        if (pl->cyl_r > 0.0) {
            double dx = *x - pl->cyl_xc, dy = *y - pl->cyl_yc;
            double a = *cx * *cx + *cy * *cy;
            double b = dx * *cx + dy * *cy;
            double c = dx * dx + dy * dy - pl->cyl_r * pl->cyl_r;
            if (c > 0.0 && b < 0.0 && a > 0.0) {
                double disc = b * b - a * c;
                if (disc >= 0.0) {
                    double t = (-b - sqrt(disc)) / a;
                    if (t >= 0.0 && t <= te) { te = t; ev = 0; }
                }
            } else if (c <= 0.0 && b < 0.0) {
                /* on or (by rounding, e.g. after a specular event at the
                 * body's foot on the symmetry plane) inside the surface and
                 * moving inward: the wall event is now */
                te = 0.0; ev = 0;
            }
        }
        if (*cx < 0.0) { double t = (pl->x0 - *x) / *cx; if (t <= te && (ev < 0 || t < te)) { te = t < 0.0 ? 0.0 : t; ev = 1; } }
        if (*cx > 0.0) { double t = (pl->x1 - *x) / *cx; if (t <= te && (ev < 0 || t < te)) { te = t < 0.0 ? 0.0 : t; ev = 2; } }
        if (*cy < 0.0) { double t = (pl->y0 - *y) / *cy; if (t <= te && (ev < 0 || t < te)) { te = t < 0.0 ? 0.0 : t; ev = 3; } }
        if (*cy > 0.0) { double t = (pl->y1 - *y) / *cy; if (t <= te && (ev < 0 || t < te)) { te = t < 0.0 ? 0.0 : t; ev = 4; } }
        if (ev < 0) {
            *x += *cx * t_left;
            *y += *cy * t_left;
            return 1;
        }
        *x += *cx * te;
        *y += *cy * te;
        t_left -= te;
        if (hits >= WALL_HIT_CAP) {
            *flags |= ORC_F_WALL_CAP;
            return 1;
        }
        double nx_ = 0.0, ny_ = 0.0;   /* normal pointing into the gas */
        int kind;
        if (ev == 0) {
            nx_ = (*x - pl->cyl_xc) / pl->cyl_r;
            ny_ = (*y - pl->cyl_yc) / pl->cyl_r;
            kind = ORC_BC_DIFFUSE;
        } else {
            int side = ev - 1;
            kind = pl->bc[side];
            if (side == 0) { nx_ = 1.0; *x = pl->x0; }
            if (side == 1) { nx_ = -1.0; *x = pl->x1; }
            if (side == 2) { ny_ = 1.0; *y = pl->y0; }
            if (side == 3) { ny_ = -1.0; *y = pl->y1; }
        }
        if (kind == ORC_BC_OPEN) {
            counters[ORC_C_OUTFLOW] += 1;
            return 0;
        }
        if (kind == ORC_BC_SPECULAR) {
            double vn = *cx * nx_ + *cy * ny_;
            *cx -= 2.0 * vn * nx_;
            *cy -= 2.0 * vn * ny_;
        } else {
            /* diffuse at T_wall: speed along the normal, one tangential
             * component in the plane, one along z */
            double in_x = *cx, in_y = *cy;
            double in_e = 0.5 * (*cx * *cx + *cy * *cy + *cz * *cz) + *erot
                        + R * sp->theta_v * (double)*lev;
            uint32_t w[4], v[4];
            philox_words(pid, step, PTAG_WALL_A, (uint32_t)hits, seed, w);
            philox_words(pid, step, PTAG_WALL_B, (uint32_t)hits, seed, v);
            double Tw = pl->T_wall;
            double vn = sqrt(-2.0 * R * Tw * log(orc_uniform(w[0], form)));
            double g1, g2;
            box_muller(orc_uniform(w[1], form), orc_uniform(w[2], form), &g1, &g2);
            double st = sqrt(R * Tw);
            double tx = -ny_, ty = nx_;
            *cx = vn * nx_ + st * g1 * tx;
            *cy = vn * ny_ + st * g1 * ty;
            *cz = st * g2;
            *erot = -R * Tw * log(orc_uniform(w[3], form));
            *lev = (int32_t)floor(-log(orc_uniform(v[0], form)) * Tw / sp->theta_v);
            if (surf && ev == 0) {
                /* surface tally of this wall event (bin of the polar angle) */
                double phi = atan2(*y - pl->cyl_yc, *x - pl->cyl_xc);
                int b = (int)floor((phi + PI) / (2.0 * PI) * ORC_NSURF);
                if (b < 0) b = 0;
                if (b > ORC_NSURF - 1) b = ORC_NSURF - 1;
                double out_e = 0.5 * (*cx * *cx + *cy * *cy + *cz * *cz) + *erot
                             + R * sp->theta_v * (double)*lev;
                surf[4 * b + 0] += in_x - *cx;
                surf[4 * b + 1] += in_y - *cy;
                surf[4 * b + 2] += in_e - out_e;
                surf[4 * b + 3] += 1.0;
            }
        }
        hits += 1;
        counters[ORC_C_WALL_HITS] += 1;
    }
}

/* Sec. 3.B: the bilinear polynomial of the quadrant the particle is in,
 * through the averages of the cell and of the three squares of the cell's
 * size beside it on that side (x, y and diagonal; the matrix of Sec. 3.B:
 * x-difference with (x - x_i), y-difference with (y - y_j), cross term).  On
 * a refined grid (Sec. 3.B, non-uniform grids) the average over such a square
 * is the leaf of the same size there, the particle-number weighted mean of
 * the four leaves one level finer that fill it, or the value of the coarser
 * leaf's polynomial at the square's centre (its integral over the square
 * divided by the area, exact for a bilinear polynomial).  A square is usable
 * if it lies in the domain and every leaf in it is whole (fluid fraction 1)
 * with at least two particles (a cell average needs two for the stress and
 * temperature, as for a neighbour on the uniform grid); an unusable side
 * square is replaced
 * by the opposite one, and without one the direction has no slope; the cross
 * term needs the diagonal square of the chosen sides. */
static void plane_reconstruct_g(const orc_plane* pl, const amr_grid* g, const int64_t* counts,
                                const double* area_frac, const double* F, int cell, double x,
                                double y, double* out);

static int region_value(const orc_plane* pl, const amr_grid* g, const int64_t* counts,
                        const double* area_frac, const double* F, int cell, int di, int dj,
                        double* val)
{
    double dx = plane_dx(pl), dy = plane_dy(pl);
    int lvl = g->level[cell];
    double h = dx / (double)(1 << (lvl - 1)), k = dy / (double)(1 << (lvl - 1));
    double cx = pl->x0 + (g->ii[cell] + di + 0.5) * h, cy = pl->y0 + (g->jj[cell] + dj + 0.5) * k;
    if (!(cx > pl->x0 && cx < pl->x1 && cy > pl->y0 && cy < pl->y1)) return 0;
    int l = amr_leaf(pl, g, cx, cy);
    int ll = g->level[l];
    if (ll == lvl) {
        if (!(area_frac[l] >= 1.0 && counts[l] >= 2)) return 0;
        for (int f = 0; f < NFIELD; ++f) val[f] = F[l * NFIELD + f];
        return 1;
    }
    if (ll > lvl) {
        /* the four finer leaves filling the square, at the centres of its quarters */
        int q[4];
        int64_t nsum = 0;
        for (int a = 0; a < 4; ++a) {
            double px = cx + ((a & 1) ? 0.25 : -0.25) * h, py = cy + ((a >> 1) ? 0.25 : -0.25) * k;
            q[a] = amr_leaf(pl, g, px, py);
            if (g->level[q[a]] != lvl + 1 || !(area_frac[q[a]] >= 1.0 && counts[q[a]] >= 2))
                return 0;
            nsum += counts[q[a]];
        }
        for (int f = 0; f < NFIELD; ++f) {
            double s = 0.0;
            for (int a = 0; a < 4; ++a) s += (double)counts[q[a]] * F[q[a] * NFIELD + f];
            val[f] = s / (double)nsum;
        }
        return 1;
    }
    /* coarser leaf: its own polynomial at the square's centre */
    if (!(area_frac[l] >= 1.0 && counts[l] >= 2)) return 0;
    plane_reconstruct_g(pl, g, counts, area_frac, F, l, cx, cy, val);
    return 1;
}

static void plane_reconstruct_g(const orc_plane* pl, const amr_grid* g, const int64_t* counts,
                                const double* area_frac, const double* F, int cell, double x,
                                double y, double* out)
{
    double dx = plane_dx(pl), dy = plane_dy(pl);
    int lvl = g->level[cell];
    double h = dx / (double)(1 << (lvl - 1)), k = dy / (double)(1 << (lvl - 1));
    double xc = pl->x0 + (g->ii[cell] + 0.5) * h, yc = pl->y0 + (g->jj[cell] + 0.5) * k;
    int sx = (x >= xc) ? 1 : -1, sy = (y >= yc) ? 1 : -1;
    double PX[NFIELD], PY[NFIELD], PD[NFIELD];
    int ox = 0, oy = 0;
    if (region_value(pl, g, counts, area_frac, F, cell, sx, 0, PX)) ox = sx;
    else if (region_value(pl, g, counts, area_frac, F, cell, -sx, 0, PX)) ox = -sx;
    if (region_value(pl, g, counts, area_frac, F, cell, 0, sy, PY)) oy = sy;
    else if (region_value(pl, g, counts, area_frac, F, cell, 0, -sy, PY)) oy = -sy;
    int diag = ox != 0 && oy != 0 && region_value(pl, g, counts, area_frac, F, cell, ox, oy, PD);
    for (int f = 0; f < NFIELD; ++f) {
        double p0 = F[cell * NFIELD + f];
        double v = p0;
        double px = 0.0, py = 0.0;
        if (ox != 0) {
            px = PX[f];
            v += (px - p0) * (x - xc) / ((double)ox * h);
        }
        if (oy != 0) {
            py = PY[f];
            v += (py - p0) * (y - yc) / ((double)oy * k);
        }
        if (diag) {
            double pd = PD[f];
            v += (pd - px - py + p0) * (x - xc) * (y - yc) / ((double)(ox * oy) * h * k);
        }
        out[f] = v;
    }
}

void orc_plane_reconstruct(const orc_plane* pl, const int64_t* counts, const double* area_frac,
                           const double* F, int cell, double x, double y, double* out)
{
    amr_grid g;
    amr_build(pl, &g);
    plane_reconstruct_g(pl, &g, counts, area_frac, F, cell, x, y, out);
    amr_free(&g);
}

int orc_plane_step(const orc_species* sp, int form, uint64_t seed, int64_t step0, int nsteps,
                   const orc_plane* pl, const double* area_frac, double dt,
                   int64_t* n_io, int64_t cap, double* x, double* y, double* cx, double* cy,
                   double* cz, double* erot, int32_t* lev, uint32_t* pid, uint32_t* next_pid,
                   int64_t* cell_off, double* acc, uint32_t* flags, int64_t* counters)
{
    double R = orc_R(sp);
    amr_grid grid;
    amr_build(pl, &grid);
    if (!grid.balanced) {
        amr_free(&grid);
        return -2;
    }
    int ncell = grid.nleaf;
    double dx = plane_dx(pl), dy = plane_dy(pl);
    double* F = (double*)malloc(sizeof(double) * NFIELD * ncell);
    double* cellT = (double*)malloc(sizeof(double) * 3 * ncell);
    int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * ncell);
    orc_coeffs* cc = (orc_coeffs*)malloc(sizeof(orc_coeffs) * ncell);
    orc_fpm* fcs = pl->method == 1 ? (orc_fpm*)malloc(sizeof(orc_fpm) * ncell) : NULL;
    int* ok = (int*)malloc(sizeof(int) * ncell);
    int* cellof = (int*)malloc(sizeof(int) * (cap > 0 ? cap : 1));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
    double* tmpd = (double*)malloc(sizeof(double) * 6 * (cap > 0 ? cap : 1));
    int32_t* tmpl = (int32_t*)malloc(sizeof(int32_t) * (cap > 0 ? cap : 1));
    uint32_t* tmpp = (uint32_t*)malloc(sizeof(uint32_t) * (cap > 0 ? cap : 1));
    int status = 0;
    int64_t n = *n_io;
    double RTi = R * pl->T_inf;
    double* surf = acc ? acc + (size_t)ncell * ORC_NACC + 2 : NULL;
    for (int s = 0; s < nsteps; ++s) {
        uint32_t step = (uint32_t)(step0 + s);
        /* 1. move; drop what left through open sides (order kept) */
        int64_t m = 0;
        for (int64_t j = 0; j < n; ++j) {
            int keep = advect_plane(sp, form, seed, step, pl, dt, &x[j], &y[j], &cx[j], &cy[j],
                                    &cz[j], &erot[j], &lev[j], pid[j], surf, flags, counters);
            if (!keep) continue;
            x[m] = x[j]; y[m] = y[j]; cx[m] = cx[j]; cy[m] = cy[j]; cz[m] = cz[j];
            erot[m] = erot[j]; lev[m] = lev[j]; pid[m] = pid[j];
            m += 1;
        }
        n = m;
        /* 2. freestream inflow: sides in order left, right, bottom, top; faces
         * along each side in order; particles numbered in that order */
        for (int side = 0; side < NSIDES; ++side) {
            if (!pl->inflow[side]) continue;
            int nf = side < 2 ? pl->ny : pl->nx;
            double flen = side < 2 ? dy : dx;
            double nxs = side == 0 ? 1.0 : (side == 1 ? -1.0 : 0.0);
            double nys = side == 2 ? 1.0 : (side == 3 ? -1.0 : 0.0);
            double u_n = pl->U_inf * nxs;
            double flux = orc_inflow_flux(pl->n_inf, RTi, u_n);
            double expect = flux * flen * pl->depth * dt / pl->F_num;
            for (int f = 0; f < nf; ++f) {
                uint32_t face = ((uint32_t)side << 24) | (uint32_t)f;
                uint32_t w[4];
                philox_words(face, step, CELL_TAG(CELL_TAG_INFLOW), 0u, seed, w);
                int64_t count = (int64_t)floor(expect + orc_uniform(w[0], 0));
                for (int64_t k = 0; k < count; ++k) {
                    uint32_t id = (*next_pid)++;
                    counters[ORC_C_INFLOW] += 1;
                    uint32_t a[4], b[4];
                    philox_words(id, step, PTAG_INFLOW_P, 0u, seed, a);
                    philox_words(id, step, PTAG_INFLOW_T, 0u, seed, b);
                    double u_pos = orc_uniform(a[0], form), u_t = orc_uniform(a[1], form);
                    double g1, g2;
                    box_muller(orc_uniform(b[0], form), orc_uniform(b[1], form), &g1, &g2);
                    double vn = orc_inflow_normal_speed(RTi, u_n, id, step, seed, form, flags);
                    double st = sqrt(RTi);
                    double px, py, vx, vy;
                    if (side < 2) {
                        px = side == 0 ? pl->x0 : pl->x1;
                        py = pl->y0 + (f + u_pos) * dy;
                        vx = vn * nxs;
                        vy = st * g1;
                    } else {
                        px = pl->x0 + (f + u_pos) * dx;
                        py = side == 2 ? pl->y0 : pl->y1;
                        vx = pl->U_inf + st * g1;
                        vy = vn * nys;
                    }
                    double vz = st * g2;
                    double e = -RTi * log(orc_uniform(a[2], form));
                    int32_t l = (int32_t)floor(-log(orc_uniform(a[3], form)) * pl->T_inf / sp->theta_v);
                    /* enters at a uniformly distributed time of the step */
                    int keep = advect_plane(sp, form, seed, step, pl, u_t * dt, &px, &py, &vx, &vy,
                                            &vz, &e, &l, id, surf, flags, counters);
                    if (!keep) continue;
                    if (n >= cap) { *flags |= ORC_F_CAPACITY; continue; }
                    x[n] = px; y[n] = py; cx[n] = vx; cy[n] = vy; cz[n] = vz; erot[n] = e;
                    lev[n] = l; pid[n] = id;
                    n += 1;
                }
            }
        }
        /* 3. stable sort by cell */
        for (int c = 0; c <= ncell; ++c) pos[c] = 0;
        for (int64_t j = 0; j < n; ++j) { cellof[j] = amr_leaf(pl, &grid, x[j], y[j]); pos[cellof[j] + 1] += 1; }
        for (int c = 0; c < ncell; ++c) pos[c + 1] += pos[c];
        for (int c = 0; c <= ncell; ++c) cell_off[c] = pos[c];
        for (int64_t j = 0; j < n; ++j) {
            int64_t k = pos[cellof[j]]++;
            tmpd[k] = x[j]; tmpd[cap + k] = y[j]; tmpd[2 * cap + k] = cx[j];
            tmpd[3 * cap + k] = cy[j]; tmpd[4 * cap + k] = cz[j]; tmpd[5 * cap + k] = erot[j];
            tmpl[k] = lev[j]; tmpp[k] = pid[j];
        }
        memcpy(x, tmpd, sizeof(double) * n); memcpy(y, tmpd + cap, sizeof(double) * n);
        memcpy(cx, tmpd + 2 * cap, sizeof(double) * n); memcpy(cy, tmpd + 3 * cap, sizeof(double) * n);
        memcpy(cz, tmpd + 4 * cap, sizeof(double) * n); memcpy(erot, tmpd + 5 * cap, sizeof(double) * n);
        memcpy(lev, tmpl, sizeof(int32_t) * n); memcpy(pid, tmpp, sizeof(uint32_t) * n);
        /* 4. cell moments and coefficients */
        for (int c = 0; c < ncell; ++c) {
            int64_t b = cell_off[c], e = cell_off[c + 1], N = e - b;
            counts[c] = N;
            ok[c] = 0;
            for (int f = 0; f < NFIELD; ++f) F[c * NFIELD + f] = 0.0;
            if (N < 2) { counters[ORC_C_SKIPPED_CELLS] += 1; continue; }
            double U[3] = { 0, 0, 0 }, er = 0.0, lv = 0.0, P[6] = { 0, 0, 0, 0, 0, 0 };
            for (int64_t j = b; j < e; ++j) { U[0] += cx[j]; U[1] += cy[j]; U[2] += cz[j]; er += erot[j]; lv += lev[j]; }
            U[0] /= N; U[1] /= N; U[2] /= N; er /= N; lv /= N;
            for (int64_t j = b; j < e; ++j) {
                double C0 = cx[j] - U[0], C1 = cy[j] - U[1], C2 = cz[j] - U[2];
                P[0] += C0 * C0; P[1] += C1 * C1; P[2] += C2 * C2;
                P[3] += C0 * C1; P[4] += C0 * C2; P[5] += C1 * C2;
            }
            for (int k = 0; k < 6; ++k) P[k] /= N;
            double* Fc = &F[c * NFIELD];
            Fc[0] = U[0]; Fc[1] = U[1]; Fc[2] = U[2];
            Fc[3] = (P[0] + P[1] + P[2]) / (3.0 * R);
            Fc[4] = er / R;
            Fc[5] = orc_T_vib_from_mean_level(sp, lv);
            for (int k = 0; k < 6; ++k) Fc[6 + k] = P[k];
            cellT[3 * c] = Fc[3]; cellT[3 * c + 1] = Fc[4]; cellT[3 * c + 2] = Fc[5];
            double sc = (double)(1 << (grid.level[c] - 1));
            double vol = area_frac[c] * (dx / sc) * (dy / sc) * pl->depth;
            if (!(vol > 0.0)) continue;
            double nd = N * pl->F_num / vol;
            if (fcs) {
                /* the plain FPM method: per-cell coefficients of Sec. 2.B */
                if (orc_fpm_coeffs(sp, nd, dt, Fc[3], Fc[4], Fc[5], &fcs[c]) != 0) {
                    *flags |= ORC_F_A_NONPOS;
                    status = -1;
                    continue;
                }
                if (fcs[c].clamped) { *flags |= ORC_F_TREL_CLAMP; counters[ORC_C_TREL_CLAMP] += 1; }
                ok[c] = 1;
                continue;
            }
            if (orc_cell_coeffs(sp, nd, dt, Fc[3], Fc[4], Fc[5], &cc[c]) != 0) {
                *flags |= ORC_F_A_NONPOS;
                status = -1;
                continue;
            }
            if (cc[c].tgt_clamped) { *flags |= ORC_F_TREL_CLAMP; counters[ORC_C_TREL_CLAMP] += 1; }
            ok[c] = 1;
        }
        /* 5. particles */
        for (int c = 0; c < ncell; ++c) {
            if (!ok[c]) continue;
            const double* Fc = &F[c * NFIELD];
            for (int64_t j = cell_off[c]; j < cell_off[c + 1]; ++j) {
                if (fcs) {
                    /* FPM: the cell values at every particle (first order) */
                    double G[4], u5, u6, cv[3] = { cx[j], cy[j], cz[j] };
                    particle_draws(seed, pid[j], step, form, G, &u5, &u6);
                    orc_collide_particle_fpm(sp, form, &fcs[c], Fc, Fc + 6, G, seed, pid[j], step,
                                             cv, &erot[j], &lev[j], flags, counters);
                    cx[j] = cv[0]; cy[j] = cv[1]; cz[j] = cv[2];
                    continue;
                }
                double f[NFIELD];
                if (pl->reconstruct) {
                    plane_reconstruct_g(pl, &grid, counts, area_frac, F, c, x[j], y[j], f);
                    if (!(f[3] > 0.0) || !(f[4] > 0.0) || !(f[5] >= 0.0)) {
                        counters[ORC_C_INTERP_FALLBACK] += 1;
                        memcpy(f, Fc, sizeof(f));
                    }
                } else {
                    memcpy(f, Fc, sizeof(f));
                }
                double G[4], u5, u6, cv[3] = { cx[j], cy[j], cz[j] };
                particle_draws(seed, pid[j], step, form, G, &u5, &u6);
                orc_collide_particle(sp, form, &cc[c], f, f + 6, f[3], f[4], f[5], G, u5, u6,
                                     cv, &erot[j], &lev[j], flags, counters);
                cx[j] = cv[0]; cy[j] = cv[1]; cz[j] = cv[2];
            }
        }
        /* 6. conservation */
        for (int c = 0; c < ncell; ++c) {
            if (!ok[c]) continue;
            conserve_cell(sp, seed, (uint32_t)c, step, cell_off[c], cell_off[c + 1],
                          1.5 * R * cellT[3 * c], R * cellT[3 * c + 1], orc_e_vib(sp, cellT[3 * c + 2]),
                          &F[c * NFIELD], fcs ? fcs[c].e_rot_tgt : cc[c].e_rot_tgt,
                          fcs ? fcs[c].e_vib_tgt : cc[c].e_vib_tgt, cx, cy, cz, erot, lev,
                          flags, counters, NULL);
        }
        /* 7. time-average sums */
        if (acc) {
            for (int c = 0; c < ncell; ++c) {
                double* a = &acc[c * ORC_NACC];
                for (int64_t j = cell_off[c]; j < cell_off[c + 1]; ++j) {
                    a[0] += 1.0;
                    a[1] += cx[j]; a[2] += cy[j]; a[3] += cz[j];
                    a[4] += cx[j] * cx[j]; a[5] += cy[j] * cy[j]; a[6] += cz[j] * cz[j];
                    a[7] += cx[j] * cy[j]; a[8] += cx[j] * cz[j]; a[9] += cy[j] * cz[j];
                    a[10] += erot[j]; a[11] += lev[j];
                }
            }
            acc[ncell * ORC_NACC] += 1.0;
        }
    }
    *n_io = n;
    free(F); free(cellT); free(counts); free(cc); free(fcs); free(ok); free(cellof); free(pos);
    free(tmpd); free(tmpl); free(tmpp);
    amr_free(&grid);
    return status;
}
