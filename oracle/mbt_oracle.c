/*
 * FP64 CPU oracle for longitudinal multi-bunch macro-particle tracking
 * (Xu, Locans, Adelmann, Stingelin, "Calculation of Longitudinal Collective
 * Instabilities with mbtrack-cuda", arXiv:1809.00391).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline / reference leg may build, load
 * or call it.  It shares no code with the CUDA library and includes none of
 * its headers.
 *
 * Everything is double precision, single-threaded, written in the order the
 * paper gives the per-turn map:
 *   - energy update with RF gain and mean radiation loss   (Sec. 2.2, Eq. 1)
 *   - radiation damping and quantum excitation, delta line  (Sec. 2.2, Eq. 5)
 *   - longitudinal drift                                    (Sec. 2.2, Eq. 2)
 *   - binning into a fixed longitudinal mesh, counting       (Sec. 2.3)
 *   - wake potential built from resonators and applied as
 *     an energy kick per particle                            (Sec. 2.3, Eq. 6)
 *   - per-bunch mean and rms statistics                      (Sec. 2.4)
 *   - long-range wake from earlier bunches and turns, applied
 *     after all bunches have been processed                  (Sec. 2.3, last paragraph)
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes of the repository):
 *   R1 drift uses the energy deviation after the RF, damping and excitation
 *      steps of the same turn (kick-then-drift, area preserving);
 *   R2 D_E = D_e = 2 T0 / tau_z with tau_z the longitudinal amplitude damping
 *      time, sigma_E the natural relative energy spread;
 *   R3 order within a turn: wake kick (previous turn's wake) -> RF and U0 ->
 *      damping and excitation -> drift -> binning and statistics -> wakes;
 *   R4 eps(tau) = (eV/E0) sin(phi_s - omega_rf tau), sin(phi_s) = U0/(eV),
 *      phi_s on the branch with cos(phi_s) of the sign of alpha_c;
 *   R5 T_rf = T0 / h, omega_rf = 2 pi h / T0;
 *   R6 per particle delta -= V(tau)/E0 (V in volts, E0 in eV) with
 *      V(tau) = sum_k Q_k W(tau - tau_k); the resonator wake
 *      W(t>0) = 2 a Rs e^{-a t}[cos(wb t) - (a/wb) sin(wb t)], W(t<0) = 0 and
 *      half of W(0+) at zero lag;
 *   R7 fixed mesh of nbins cells over [-H, H), H = k sigma_tau0,
 *      bin = floor((tau + H) * (1/Delta)); outside particles are counted,
 *      not deposited, and get no short-range kick;
 *   R8 the short-range voltage is interpolated linearly between cell centres
 *      (clamped at the end cells); nearest-cell is a flag;
 *   R9 normal deviates from Philox4x32-10 + Box-Muller: one block per quad of
 *      consecutive particles, counter (quad, bunch, turn, tag), key (seed lo,
 *      seed hi), each 32-bit word a uniform (w + 1/2) 2^-32;
 *   R10 the long-range wake of a passage is sourced by its binned histogram at
 *      cell centres, and acts on every particle of every later passage;
 *   R11 a tabulated short-range wake (e.g. the resistive wall) acts through
 *      its average over each lag cell (see orc_add_wake_table);
 *   R14 harmonic cavities add (V_h/E0) sin(phi_h - n_h omega_rf tau) each;
 *      the main cavity's phase balances U0 (see orc_derive_h);
 *   R15 the transverse plane (see orc_set_transverse): one plane per run,
 *      no dispersion at the tracking point, kicks with the previous turn's
 *      wake before the RF, momentum ratio across the cavity, chromatic
 *      rotation with the new delta, excitation, dipole sums per cell;
 *   R16 the long-range transverse resistive wall acts through bunch
 *      centroids over a finite history (see orc_add_transverse_rw).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_RES 16
#define ORC_RANGE_SHORT 1
#define ORC_RANGE_LONG 2

#define ORC_NO_SR 1      /* no radiation: U0 = 0, no damping, no excitation */
#define ORC_NO_QE 2      /* damping kept, excitation removed                */
#define ORC_KICK_NGP 4   /* short-range kick from the particle's own cell   */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox S-box with the     */
/* Weyl key schedule.                                                         */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
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

/* Uniform in the open interval (0,1) from one 32-bit word: (w + 1/2) 2^-32. */
double orc_u01(uint32_t w)
{
    return ((double)w + 0.5) * 0x1.0p-32;
}

/* Box-Muller: two independent standard normals from two uniforms. */
void orc_box_muller(double u1, double u2, double *r_cos, double *r_sin)
{
    const double two_pi = 6.283185307179586476925286766559;
    double R = sqrt(-2.0 * log(u1));
    *r_cos = R * cos(two_pi * u2);
    *r_sin = R * sin(two_pi * u2);
}

/* Four normals for the quad of consecutive particles 4q .. 4q+3 of a bunch,
 * for (quad, bunch, turn, tag) under a 64-bit seed (reading R9): one Philox
 * block, Box-Muller on (u(w0), u(w1)) for particles 4q (cos) and 4q+1 (sin),
 * on (u(w2), u(w3)) for 4q+2 (cos) and 4q+3 (sin). */
void orc_normal_quad(uint64_t seed, uint32_t quad, uint32_t bunch, uint32_t turn, uint32_t tag, double r[4])
{
    uint32_t ctr[4] = {quad, bunch, turn, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    orc_box_muller(orc_u01(w[0]), orc_u01(w[1]), &r[0], &r[1]);
    orc_box_muller(orc_u01(w[2]), orc_u01(w[3]), &r[2], &r[3]);
}

/* ------------------------------------------------------------------------- */
/* Ring and wake definitions                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    double E0_eV;        /* reference energy [eV]                        */
    double T0_s;         /* revolution period [s]                        */
    int32_t h;           /* harmonic number                              */
    int32_t pad_;
    double V_rf_V;       /* peak RF voltage [V]                          */
    double alpha_c;      /* momentum compaction factor                   */
    double U0_eV;        /* radiation energy loss per turn [eV]          */
    double sigma_delta;  /* natural relative energy spread sigma_E       */
    double tau_z_s;      /* longitudinal amplitude damping time [s]      */
} orc_ring;

typedef struct {
    double Rs_ohm;       /* shunt impedance [Ohm]                        */
    double fr_Hz;        /* resonant frequency [Hz]                      */
    double Q;            /* quality factor (> 1/2)                       */
    int32_t range;       /* bit 1: short range, bit 2: long range        */
    int32_t pad_;
} orc_resonator;

/* An active harmonic RF cavity: voltage V_V at n times the RF frequency,
 * phase phi_rad at the synchronous particle; it adds
 * (V_V/E0) sin(phi_rad - n omega_rf tau) to the energy change of a turn. */
typedef struct {
    int32_t n;
    int32_t pad_;
    double V_V;
    double phi_rad;
} orc_harmonic;

#define ORC_MAX_HARM 4

/* Derived ring quantities, reading R4/R5 and the linear synchrotron motion. */
typedef struct {
    double T_rf, omega_rf, phi_s, sin_phi_s, U0_over_E0, V_over_E0;
    double D;            /* damping decrement per turn, reading R2      */
    double qe_amp;       /* sigma_E sqrt(2 D)                           */
    double nu_s;         /* small-amplitude synchrotron tune            */
    double sigma_tau0;   /* matched rms arrival-time spread            */
} orc_derived;

/* With harmonic cavities (reading R14) the main cavity's phase makes the
 * synchronous particle lose nothing on average:
 *   V sin(phi_s) + sum_h V_h sin(phi_h) = U0,
 * and nu_s, sigma_tau0 (the mesh unit and the matched start) come from the
 * main cavity's slope V cos(phi_s) alone: the small-amplitude tune of a
 * double-RF system can vanish (flat potential). */
void orc_derive_h(const orc_ring *r, int flags, int nharm, const orc_harmonic *harm, orc_derived *d)
{
    const double pi = 3.14159265358979323846264338327950;
    int sr = !(flags & ORC_NO_SR);
    double U0 = sr ? r->U0_eV : 0.0;
    double Uh = 0.0;
    for (int k = 0; k < nharm; ++k)
        Uh += harm[k].V_V * sin(harm[k].phi_rad);
    d->T_rf = r->T0_s / (double)r->h;
    d->omega_rf = 2.0 * pi * (double)r->h / r->T0_s;
    d->sin_phi_s = (U0 - Uh) / r->V_rf_V;
    d->phi_s = asin(d->sin_phi_s);
    if (r->alpha_c < 0.0)
        d->phi_s = pi - d->phi_s;
    d->U0_over_E0 = U0 / r->E0_eV;
    d->V_over_E0 = r->V_rf_V / r->E0_eV;
    d->D = sr ? 2.0 * r->T0_s / r->tau_z_s : 0.0;
    d->qe_amp = (sr && !(flags & ORC_NO_QE)) ? r->sigma_delta * sqrt(2.0 * d->D) : 0.0;
    d->nu_s = sqrt(r->alpha_c * (double)r->h * r->V_rf_V * cos(d->phi_s) / (2.0 * pi * r->E0_eV));
    d->sigma_tau0 = fabs(r->alpha_c) * r->sigma_delta * r->T0_s / (2.0 * pi * d->nu_s);
}

/* orc_derive_h without harmonic cavities. */
void orc_derive(const orc_ring *r, int flags, orc_derived *d)
{
    orc_derive_h(r, flags, 0, NULL, d);
}

/* Resonator constants: decay rate a = w_r/(2Q), damped frequency wb. */
static void res_consts(const orc_resonator *q, double *a, double *wb)
{
    const double pi = 3.14159265358979323846264338327950;
    double wr = 2.0 * pi * q->fr_Hz;
    *a = wr / (2.0 * q->Q);
    *wb = sqrt(wr * wr - (*a) * (*a));
}

/* Longitudinal resonator wake function [V/C], reading R6. */
double orc_wake(const orc_resonator *q, double t)
{
    double a, wb;
    res_consts(q, &a, &wb);
    if (t < 0.0)
        return 0.0;
    if (t == 0.0)
        return a * q->Rs_ohm; /* half of W(0+) = 2 a Rs */
    return 2.0 * a * q->Rs_ohm * exp(-a * t) * (cos(wb * t) - (a / wb) * sin(wb * t));
}

/* Transverse resonator wake [V/(C m)]:
 * W(t > 0) = (wr^2 Rs / (Q wb)) e^{-a t} sin(wb t) = Im(c e^{s t}),
 * c = wr^2 Rs / (Q wb), s = -a + i wb;  W(t <= 0) = 0 (it also vanishes at
 * t = 0+).  Its transform i int W e^{-i w t} dt is the transverse resonator
 * impedance (wr / w) Rs / (1 + i Q (w / wr - wr / w)), Rs in Ohm/m. */
double orc_twake(const orc_resonator *q, double t)
{
    double a, wb;
    res_consts(q, &a, &wb);
    if (t <= 0.0)
        return 0.0;
    const double wr = 2.0 * 3.14159265358979323846264338327950 * q->fr_Hz;
    return wr * wr * q->Rs_ohm / (q->Q * wb) * exp(-a * t) * sin(wb * t);
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct orc_sim {
    orc_ring ring;
    orc_derived dv;
    int flags;
    uint64_t seed;
    int nres;
    orc_resonator res[ORC_MAX_RES];
    int nbins;
    double H, Delta, invDelta;
    int nb;
    int32_t *bucket;
    double *current;
    int64_t *n_mp;
    double *q_mp;          /* macro-particle charge per bunch [C]           */
    double **tau, **delta;
    int32_t *hist;         /* [nb][nbins], this turn                         */
    int64_t *out_count;    /* [nb], this turn                                */
    double *Wlag;          /* [nbins] summed short-range wake at lag l*Delta */
    int nharm;
    orc_harmonic harm[ORC_MAX_HARM];
    double harm_VoE0[ORC_MAX_HARM], harm_nw[ORC_MAX_HARM];
    double *Vsr;           /* [nb][nbins] short-range voltage for the kick   */
    double complex *Alr;   /* [nres][nb] long-range amplitude for the kick   */
    /* emission history for the direct long-range sum: [nres][nhist][nb]     */
    int nhist;
    double complex *Ehist;
    int64_t turn;          /* turns completed                                */
    double *moments;       /* [nb][6]: <tau>, sig_tau, <delta>, sig_delta, n_in, n_out */
    /* transverse plane (reading R15), allocated by orc_set_transverse */
    int trans;
    double tb_beta, tb_alpha, tb_gamma, tb_mu0, tb_xi, tb_sx, tb_sxp, tb_Dx;
    int ntres;
    orc_resonator tres[ORC_MAX_RES];
    double **x, **xp;
    double *dip;           /* [nb][nbins] sum of x over the cell's particles, this turn */
    double *Vt;            /* [nb][nbins] transverse short-range voltage [V] for the kick */
    double *Wtlag;         /* [nbins] summed transverse wake at lag l*Delta [V/(C m)] */
    double complex *Atlr;  /* [ntres][nb] long-range transverse amplitude */
    int nthist;
    double complex *Ethist;/* [ntres][nthist][nb] transverse emission history */
    double *tmoments;      /* [nb][4]: <x>, sig_x, <x'>, sig_x' */
    /* long-range transverse resistive wall on bunch centroids (reading R16) */
    double rw_A;           /* W(t) = rw_A / sqrt(t) [V/(C m)], t in s        */
    int rw_nh;             /* turns of history                               */
    double *rw_cent;       /* [rw_nh + 1][nb] charge x centroid, by turn     */
    double *Vrw;           /* [nb] kick voltage of each bunch for the next turn */
    /* e^{s D T_rf} by bucket distance D < nhist h for each long-range
     * resonator, and whether e^{-a D T_rf} clears the history cutoff: the
     * factors the direct history sums multiply by, computed once */
    double complex *lr_phase[ORC_MAX_RES], *tr_phase[ORC_MAX_RES];
    unsigned char *lr_keep[ORC_MAX_RES], *tr_keep[ORC_MAX_RES];
} orc_sim;

/* e^{-a dt} below this is dropped from the direct history sum. */
static const double ORC_HISTORY_CUTOFF = 1e-18;

/* The factor e^{s dt}, dt = D T_rf, of every bucket distance 0 <= D < nD for
 * resonator q, and keep[D] = (D > 0 and e^{-a dt} >= cutoff): exactly the
 * values the history sums would form term by term. */
static void phase_table(const orc_resonator *q, double T_rf, int64_t nD, double complex **val, unsigned char **keep)
{
    double a, wb;
    res_consts(q, &a, &wb);
    double complex sr = -a + I * wb;
    *val = (double complex *)calloc((size_t)nD, sizeof(double complex));
    *keep = (unsigned char *)calloc((size_t)nD, 1);
    for (int64_t D = 1; D < nD; ++D) {
        double dt = (double)D * T_rf;
        if (exp(-a * dt) < ORC_HISTORY_CUTOFF)
            continue;
        (*keep)[D] = 1;
        (*val)[D] = cexp(sr * dt);
    }
}

orc_sim *orc_create_h(const orc_ring *ring, int flags, uint64_t seed,
                      int nres, const orc_resonator *res, int nharm, const orc_harmonic *harm,
                      int nbins, double half_width_sigmas,
                      int nb, const int32_t *bucket, const double *current_A, const int64_t *n_mp)
{
    if (nres < 0 || nres > ORC_MAX_RES || nharm < 0 || nharm > ORC_MAX_HARM || nbins < 2 || nb < 1)
        return NULL;
    orc_derived dv;
    orc_derive_h(ring, flags, nharm, harm, &dv);
    if (!(fabs(dv.sin_phi_s) <= 1.0) || !(dv.sigma_tau0 > 0.0))
        return NULL;   /* no synchronous phase, or an unstable main cavity */
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->ring = *ring;
    s->flags = flags;
    s->seed = seed;
    s->dv = dv;
    s->nharm = nharm;
    for (int k = 0; k < nharm; ++k) {
        s->harm[k] = harm[k];
        s->harm_VoE0[k] = harm[k].V_V / ring->E0_eV;
        s->harm_nw[k] = (double)harm[k].n * dv.omega_rf;
    }
    s->nres = nres;
    for (int r = 0; r < nres; ++r)
        s->res[r] = res[r];
    s->nbins = nbins;
    s->H = half_width_sigmas * s->dv.sigma_tau0;
    s->Delta = 2.0 * s->H / (double)nbins;
    s->invDelta = 1.0 / s->Delta;
    s->nb = nb;
    s->bucket = (int32_t *)malloc(sizeof(int32_t) * nb);
    s->current = (double *)malloc(sizeof(double) * nb);
    s->n_mp = (int64_t *)malloc(sizeof(int64_t) * nb);
    s->q_mp = (double *)malloc(sizeof(double) * nb);
    s->tau = (double **)calloc(nb, sizeof(double *));
    s->delta = (double **)calloc(nb, sizeof(double *));
    for (int m = 0; m < nb; ++m) {
        s->bucket[m] = bucket[m];
        s->current[m] = current_A[m];
        s->n_mp[m] = n_mp[m];
        s->q_mp[m] = n_mp[m] > 0 ? current_A[m] * ring->T0_s / (double)n_mp[m] : 0.0;
        s->tau[m] = (double *)calloc(n_mp[m] > 0 ? n_mp[m] : 1, sizeof(double));
        s->delta[m] = (double *)calloc(n_mp[m] > 0 ? n_mp[m] : 1, sizeof(double));
    }
    s->hist = (int32_t *)calloc((size_t)nb * nbins, sizeof(int32_t));
    s->out_count = (int64_t *)calloc(nb, sizeof(int64_t));
    s->Vsr = (double *)calloc((size_t)nb * nbins, sizeof(double));
    s->Alr = (double complex *)calloc((size_t)(nres > 0 ? nres : 1) * nb, sizeof(double complex));
    s->moments = (double *)calloc((size_t)nb * 6, sizeof(double));
    s->Wlag = (double *)calloc(nbins, sizeof(double));
    for (int l = 0; l < nbins; ++l) {
        double w = 0.0;
        for (int r = 0; r < nres; ++r)
            if (res[r].range & ORC_RANGE_SHORT)
                w += orc_wake(&res[r], (double)l * s->Delta);
        s->Wlag[l] = w;
    }
    /* history depth: the slowest-decaying long-range resonator sets it */
    double amin = 0.0;
    int any_long = 0;
    for (int r = 0; r < nres; ++r) {
        if (!(res[r].range & ORC_RANGE_LONG))
            continue;
        double a, wb;
        res_consts(&res[r], &a, &wb);
        if (!any_long || a < amin)
            amin = a;
        any_long = 1;
    }
    s->nhist = any_long ? (int)ceil(-log(ORC_HISTORY_CUTOFF) / (amin * ring->T0_s)) + 2 : 1;
    s->Ehist = (double complex *)calloc((size_t)(nres > 0 ? nres : 1) * s->nhist * nb, sizeof(double complex));
    for (int r = 0; r < nres; ++r)
        if (res[r].range & ORC_RANGE_LONG)
            phase_table(&res[r], s->dv.T_rf, (int64_t)s->nhist * ring->h, &s->lr_phase[r], &s->lr_keep[r]);
    return s;
}

/* A tabulated short-range wake W(t) (V/C), given at n samples t[0] = 0 <
 * t[1] < ... (s): linear between samples, zero beyond the last one.  It acts
 * on the mesh through its average over each lag cell (reading R11):
 *   lag l >= 1: (1/Delta) * integral of W over [(l - 1/2) Delta, (l + 1/2) Delta],
 *   lag 0:      (1/Delta) * integral of W over [0, Delta / 2]
 * (for a smooth W these are W(l Delta) and W(0+)/2 up to O(Delta^2)), added
 * to the resonators' lag wake.  The integrals are exact for the piecewise
 * linear W. */
static double table_integral(int n, const double *t, const double *W, double lo, double hi)
{
    double acc = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        double a = t[i] > lo ? t[i] : lo;
        double b = t[i + 1] < hi ? t[i + 1] : hi;
        if (b <= a)
            continue;
        double slope = (W[i + 1] - W[i]) / (t[i + 1] - t[i]);
        double wa = W[i] + slope * (a - t[i]);
        double wb = W[i] + slope * (b - t[i]);
        acc += 0.5 * (wa + wb) * (b - a);
    }
    return acc;
}

/* A tabulated short-range wake W(t_i), linear between samples (reading R13):
 * its average over every lag cell is added to the lag wake.  -1 (nothing
 * added) unless t_0 = 0 and the times increase. */
int orc_add_wake_table(orc_sim *s, int n, const double *t, const double *W)
{
    if (n < 2 || t[0] != 0.0)
        return -1;
    for (int i = 0; i + 1 < n; ++i)
        if (!(t[i + 1] > t[i]))
            return -1;
    for (int l = 0; l < s->nbins; ++l) {
        double lo = l == 0 ? 0.0 : ((double)l - 0.5) * s->Delta;
        double hi = ((double)l + 0.5) * s->Delta;
        s->Wlag[l] += table_integral(n, t, W, lo, hi) / s->Delta;
    }
    return 0;
}

orc_sim *orc_create(const orc_ring *ring, int flags, uint64_t seed,
                    int nres, const orc_resonator *res,
                    int nbins, double half_width_sigmas,
                    int nb, const int32_t *bucket, const double *current_A, const int64_t *n_mp)
{
    return orc_create_h(ring, flags, seed, nres, res, 0, NULL, nbins, half_width_sigmas, nb, bucket, current_A, n_mp);
}

/* Frees the simulation and everything it owns. */
void orc_destroy(orc_sim *s)
{
    if (!s)
        return;
    for (int m = 0; m < s->nb; ++m) {
        free(s->tau[m]);
        free(s->delta[m]);
    }
    free(s->tau); free(s->delta); free(s->bucket); free(s->current); free(s->n_mp); free(s->q_mp);
    free(s->hist); free(s->out_count); free(s->Vsr); free(s->Alr); free(s->moments);
    free(s->Wlag); free(s->Ehist);
    for (int r = 0; r < ORC_MAX_RES; ++r) {
        free(s->lr_phase[r]); free(s->lr_keep[r]);
        free(s->tr_phase[r]); free(s->tr_keep[r]);
    }
    if (s->trans) {
        for (int m = 0; m < s->nb; ++m) {
            free(s->x[m]);
            free(s->xp[m]);
        }
        free(s->x); free(s->xp); free(s->dip); free(s->Vt); free(s->Wtlag); free(s->Atlr); free(s->Ethist);
        free(s->tmoments); free(s->rw_cent); free(s->Vrw);
    }
    free(s);
}

/* Transverse plane (reading R15): Twiss beta_m, alpha at the tracking point
 * (no dispersion there), betatron tune nu0 with phase advance
 * 2 pi nu0 (1 + xi delta) (Eq. 3), equilibrium emittance emit_m; transverse
 * resonators (Eq. 6, second line) with Rs in Ohm/m and the range bits of the
 * longitudinal ones.  Radiation: x' scales with the momentum ratio across the
 * RF cavity, (1 + delta_before)/(1 + delta_after_gain) (Eq. 5, x' line), and
 * the noise amplitudes sqrt(beta emit) sqrt(Dx), sqrt(gamma emit) sqrt(Dx)
 * with Dx = U0/E0, the damping that the momentum ratio produces on average,
 * so that emit_m is the equilibrium.  Returns 0, or -1 on bad input. */
int orc_set_transverse(orc_sim *s, double beta_m, double alpha, double nu0, double xi, double emit_m,
                       int ntres, const orc_resonator *tres)
{
    if (s->trans || !(beta_m > 0.0) || !(emit_m >= 0.0) || ntres < 0 || ntres > ORC_MAX_RES)
        return -1;
    const double pi = 3.14159265358979323846264338327950;
    s->trans = 1;
    s->tb_beta = beta_m;
    s->tb_alpha = alpha;
    s->tb_gamma = (1.0 + alpha * alpha) / beta_m;
    s->tb_mu0 = 2.0 * pi * nu0;
    s->tb_xi = xi;
    int sr = !(s->flags & ORC_NO_SR), qe = sr && !(s->flags & ORC_NO_QE);
    s->tb_Dx = qe ? s->dv.U0_over_E0 : 0.0;
    s->tb_sx = sqrt(beta_m * emit_m);
    s->tb_sxp = sqrt(s->tb_gamma * emit_m);
    s->ntres = ntres;
    for (int r = 0; r < ntres; ++r)
        s->tres[r] = tres[r];
    s->x = (double **)calloc(s->nb, sizeof(double *));
    s->xp = (double **)calloc(s->nb, sizeof(double *));
    for (int m = 0; m < s->nb; ++m) {
        s->x[m] = (double *)calloc(s->n_mp[m] > 0 ? s->n_mp[m] : 1, sizeof(double));
        s->xp[m] = (double *)calloc(s->n_mp[m] > 0 ? s->n_mp[m] : 1, sizeof(double));
    }
    s->dip = (double *)calloc((size_t)s->nb * s->nbins, sizeof(double));
    s->Vt = (double *)calloc((size_t)s->nb * s->nbins, sizeof(double));
    s->Wtlag = (double *)calloc(s->nbins, sizeof(double));
    for (int l = 0; l < s->nbins; ++l)
        for (int r = 0; r < ntres; ++r)
            if (tres[r].range & ORC_RANGE_SHORT)
                s->Wtlag[l] += orc_twake(&tres[r], (double)l * s->Delta);
    double amin = 0.0;
    int any_long = 0;
    for (int r = 0; r < ntres; ++r) {
        if (!(tres[r].range & ORC_RANGE_LONG))
            continue;
        double a, wb;
        res_consts(&tres[r], &a, &wb);
        if (!any_long || a < amin)
            amin = a;
        any_long = 1;
    }
    s->nthist = any_long ? (int)ceil(-log(ORC_HISTORY_CUTOFF) / (amin * s->ring.T0_s)) + 2 : 1;
    for (int r = 0; r < ntres; ++r)
        if (tres[r].range & ORC_RANGE_LONG)
            phase_table(&tres[r], s->dv.T_rf, (int64_t)s->nthist * s->ring.h, &s->tr_phase[r], &s->tr_keep[r]);
    s->Atlr = (double complex *)calloc((size_t)(ntres > 0 ? ntres : 1) * s->nb, sizeof(double complex));
    s->Ethist = (double complex *)calloc((size_t)(ntres > 0 ? ntres : 1) * s->nthist * s->nb, sizeof(double complex));
    s->tmoments = (double *)calloc((size_t)s->nb * 4, sizeof(double));
    return 0;
}

/* Derived quantities of orc_derive_h and the mesh, as 12 doubles: T_rf,
 * omega_rf, phi_s, D, excitation amplitude, nu_s, sigma_tau0, H, Delta,
 * 1/Delta, histogram count, turn. */
void orc_get_derived(const orc_sim *s, double out[12])
{
    out[0] = s->dv.T_rf; out[1] = s->dv.omega_rf; out[2] = s->dv.phi_s; out[3] = s->dv.D;
    out[4] = s->dv.qe_amp; out[5] = s->dv.nu_s; out[6] = s->dv.sigma_tau0; out[7] = s->H;
    out[8] = s->Delta; out[9] = s->invDelta; out[10] = (double)s->nhist; out[11] = (double)s->turn;
}

/* Matched Gaussian start: tau ~ N(0, sigma_tau0), delta ~ N(0, sigma_E),
 * normals from turn 0 with tag 1 (tau) and tag 2 (delta). */
void orc_init_particles(orc_sim *s)
{
    for (int m = 0; m < s->nb; ++m) {
        int64_t n = s->n_mp[m];
        for (int64_t i = 0; i < n; i += 4) {
            double a[4], b[4];
            orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, 0u, 1u, a);
            orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, 0u, 2u, b);
            for (int e = 0; e < 4 && i + e < n; ++e) {
                s->tau[m][i + e] = s->dv.sigma_tau0 * a[e];
                s->delta[m][i + e] = s->ring.sigma_delta * b[e];
            }
            if (s->trans) {
                /* matched Gaussian: x = sqrt(beta emit) a, x' = sqrt(emit / beta) (b - alpha a) */
                double c[4], d[4];
                orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, 0u, 5u, c);
                orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, 0u, 6u, d);
                const double emit = s->tb_sx * s->tb_sx / s->tb_beta;
                for (int e = 0; e < 4 && i + e < n; ++e) {
                    s->x[m][i + e] = s->tb_sx * c[e];
                    s->xp[m][i + e] = sqrt(emit / s->tb_beta) * (d[e] - s->tb_alpha * c[e]);
                }
            }
        }
    }
}

/* Accessors: tau, delta of bunch m (n_mp[m] each). */
void orc_set_particles(orc_sim *s, int m, const double *tau, const double *delta)
{
    memcpy(s->tau[m], tau, sizeof(double) * s->n_mp[m]);
    memcpy(s->delta[m], delta, sizeof(double) * s->n_mp[m]);
}

void orc_get_particles(const orc_sim *s, int m, double *tau, double *delta)
{
    memcpy(tau, s->tau[m], sizeof(double) * s->n_mp[m]);
    memcpy(delta, s->delta[m], sizeof(double) * s->n_mp[m]);
}

/* Cell coordinate x = (tau + H) * (1/Delta), both operations rounded
 * separately (the build disables contraction); the cell is floor(x). */
double orc_cell_coord(const orc_sim *s, double tau)
{
    double t = tau + s->H;
    return t * s->invDelta;
}

/* Deposit one particle into a bunch histogram (Sec. 2.3, reading R7):
 * returns 1 if it fell outside the mesh (counted, not deposited). */
static int bin_one(const orc_sim *s, double tau, int32_t *hist)
{
    double x = orc_cell_coord(s, tau);
    if (x >= 0.0 && x < (double)s->nbins) {
        hist[(int)floor(x)] += 1;
        return 0;
    }
    return 1;
}

/* Histogram of n arrival times on the sim's mesh; returns the outside count. */
int64_t orc_bin(const orc_sim *s, int64_t n, const double *tau, int32_t *hist)
{
    memset(hist, 0, sizeof(int32_t) * s->nbins);
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i)
        out += bin_one(s, tau[i], hist);
    return out;
}

/* Short-range voltage at a particle, reading R7/R8. */
static double vsr_at(const orc_sim *s, int m, double x)
{
    const int nb = s->nbins;
    if (!(x >= 0.0 && x < (double)nb))
        return 0.0;
    const double *V = s->Vsr + (size_t)m * nb;
    if (s->flags & ORC_KICK_NGP)
        return V[(int)floor(x)];
    double u = x - 0.5;
    if (u <= 0.0)
        return V[0];
    if (u >= (double)(nb - 1))
        return V[nb - 1];
    double j0 = floor(u);
    double f = u - j0;
    int j = (int)j0;
    return (1.0 - f) * V[j] + f * V[j + 1];
}

/* Long-range voltage at a particle of bunch m: sum over long-range resonators
 * of Re(A e^{s tau}), s = -a + i wb (reading R10). */
static double vlr_at(const orc_sim *s, int m, double tau)
{
    double v = 0.0;
    for (int r = 0; r < s->nres; ++r) {
        if (!(s->res[r].range & ORC_RANGE_LONG))
            continue;
        double a, wb;
        res_consts(&s->res[r], &a, &wb);
        double complex sr = -a + I * wb;
        v += creal(s->Alr[(size_t)r * s->nb + m] * cexp(sr * tau));
    }
    return v;
}

/* Short-range voltage of one bunch from its histogram: the direct double sum
 * V[j] = q * sum_{k<=j} hist[k] * Wtot((j-k) Delta), reading R6. */
void orc_vsr_direct(const orc_sim *s, const int32_t *hist, double q, double *V)
{
    for (int j = 0; j < s->nbins; ++j) {
        double v = 0.0;
        for (int k = 0; k <= j; ++k)
            v += (double)hist[k] * s->Wlag[j - k];
        V[j] = q * v;
    }
}

/* Emission of one passage for resonator r: c q sum_k hist[k] e^{-s tau_k},
 * c = 2 a Rs (1 + i a/wb), tau_k the cell centres. */
double complex orc_emission(const orc_sim *s, int r, const int32_t *hist, double q)
{
    double a, wb;
    res_consts(&s->res[r], &a, &wb);
    double complex sr = -a + I * wb;
    double complex c = 2.0 * a * s->res[r].Rs_ohm * (1.0 + I * (a / wb));
    double complex acc = 0.0;
    for (int k = 0; k < s->nbins; ++k) {
        if (hist[k] == 0)
            continue;
        double tk = -s->H + ((double)k + 0.5) * s->Delta;
        acc += (double)hist[k] * cexp(-sr * tk);
    }
    return c * q * acc;
}

/* Direct history sum for bunch m after turn n has been binned: every passage
 * strictly earlier than (n, m), weighted by e^{s dt}, dt = D T_rf with D the
 * integer bucket distance, truncated at e^{-a dt} < cutoff (the factors from
 * the resonator's phase table). */
static double complex history_sum(const orc_sim *s, int r, int m)
{
    const double complex *ph = s->lr_phase[r];
    const unsigned char *keep = s->lr_keep[r];
    const int64_t n = s->turn; /* the turn just binned */
    const int h = s->ring.h;
    double complex acc = 0.0;
    for (int64_t back = 0; back < s->nhist; ++back) {
        int64_t np = n - back;
        if (np < 0)
            break;
        const double complex *E = s->Ehist + ((size_t)r * s->nhist + (size_t)(np % s->nhist)) * s->nb;
        for (int mp = 0; mp < s->nb; ++mp) {
            int64_t D = back * (int64_t)h + (int64_t)s->bucket[m] - (int64_t)s->bucket[mp];
            if (D <= 0 || !keep[D])
                continue; /* not earlier, or below the cutoff */
            acc += ph[D] * E[mp];
        }
    }
    return acc;
}

/* Long-range transverse resistive wall of a round pipe (radius b,
 * conductivity sigma, length L), reading R16: far from the wake's head the
 * dipole wake is W(t) = (c L / (pi b^3)) sqrt(Z0 / (pi sigma)) / sqrt(c t)
 * [V/(C m)] (positive: the trailing charge is deflected towards the source
 * offset, the sign of the transverse resonator's wake).  It acts between
 * bunch passages through the bunch centroids: every particle of bunch m gets
 * x' += (1/E0) sum Q_p <x>_p W(t_m - t_p) over the passages of the last
 * history_turns turns before it (the bunch's own earlier turns included).
 * Several pipes add their coefficients; the history is the longest asked. */
int orc_add_transverse_rw(orc_sim *s, double radius_m, double sigma, double length_m, int history_turns)
{
    if (!s->trans || !(radius_m > 0.0) || !(sigma > 0.0) || !(length_m > 0.0) || history_turns < 1)
        return -1;
    const double pi = 3.14159265358979323846264338327950, c = 299792458.0, Z0 = 376.730313668;
    s->rw_A += c * length_m / (pi * radius_m * radius_m * radius_m) * sqrt(Z0 / (pi * sigma)) / sqrt(c);
    if (history_turns > s->rw_nh) {
        free(s->rw_cent);
        s->rw_nh = history_turns;
        s->rw_cent = (double *)calloc((size_t)(s->rw_nh + 1) * s->nb, sizeof(double));
    }
    if (!s->Vrw)
        s->Vrw = (double *)calloc(s->nb, sizeof(double));
    return 0;
}

/* The summed dipole resistive-wall wake of orc_add_transverse_rw at delay t:
 * rw_A / sqrt(t) for t > 0, zero otherwise (causality). */
double orc_transverse_rw_wake(const orc_sim *s, double t)
{
    return t > 0.0 ? s->rw_A / sqrt(t) : 0.0;
}

/* Transverse short-range voltage at cell coordinate x of bunch m, linear
 * between cell centres like the longitudinal one (zero outside the mesh). */
static double vt_at(const orc_sim *s, int m, double xc)
{
    const int nb = s->nbins;
    if (!(xc >= 0.0 && xc < (double)nb))
        return 0.0;
    const double *V = s->Vt + (size_t)m * nb;
    if (s->flags & ORC_KICK_NGP)
        return V[(int)floor(xc)];
    double u = xc - 0.5;
    if (u <= 0.0)
        return V[0];
    if (u >= (double)(nb - 1))
        return V[nb - 1];
    double j0 = floor(u);
    double f = u - j0;
    int j = (int)j0;
    return (1.0 - f) * V[j] + f * V[j + 1];
}

/* Transverse long-range voltage: sum over transverse long-range resonators of
 * Im(A e^{s tau}). */
static double vtlr_at(const orc_sim *s, int m, double tau)
{
    double v = 0.0;
    for (int r = 0; r < s->ntres; ++r) {
        if (!(s->tres[r].range & ORC_RANGE_LONG))
            continue;
        double a, wb;
        res_consts(&s->tres[r], &a, &wb);
        v += cimag(s->Atlr[(size_t)r * s->nb + m] * cexp((-a + I * wb) * tau));
    }
    return v;
}

/* The transverse kick voltage on a particle of bunch m at tau (Eq. 6, second
 * line, with the previous turn's wake): short range at its cell coordinate,
 * long-range resonators, long-range resistive wall. */
double orc_tvoltage_at(const orc_sim *s, int m, double tau)
{
    return vt_at(s, m, orc_cell_coord(s, tau)) + vtlr_at(s, m, tau) + (s->Vrw ? s->Vrw[m] : 0.0);
}

/* Dipole deposit of one particle (offset x) at arrival time tau into the
 * bunch's per-cell sums: the cell that binning gives it, nothing outside. */
static void deposit_dip(const orc_sim *s, double tau, double x, double *dip)
{
    double xc = orc_cell_coord(s, tau);
    if (xc >= 0.0 && xc < (double)s->nbins)
        dip[(int)xc] += x;
}

/* Transverse short-range voltage of one bunch from its dipole sums (sum of x
 * per cell): V[j] = q * sum_{k<=j} dip[k] * Wt((j-k) Delta), Eq. 6 second line. */
void orc_vt_direct(const orc_sim *s, const double *dip, double q, double *V)
{
    for (int j = 0; j < s->nbins; ++j) {
        double v = 0.0;
        for (int k = 0; k <= j; ++k)
            v += dip[k] * s->Wtlag[j - k];
        V[j] = q * v;
    }
}

/* Transverse emission of one passage: c q sum_k dip[k] e^{-s tau_k},
 * c = wr^2 Rs / (Q wb) (so that the wake is Im(c e^{s t})). */
static double complex temission(const orc_sim *s, int r, const double *dip, double q)
{
    double a, wb;
    res_consts(&s->tres[r], &a, &wb);
    const double wr = 2.0 * 3.14159265358979323846264338327950 * s->tres[r].fr_Hz;
    double complex sr = -a + I * wb;
    double complex acc = 0.0;
    for (int k = 0; k < s->nbins; ++k) {
        if (dip[k] == 0.0)
            continue;
        double tk = -s->H + ((double)k + 0.5) * s->Delta;
        acc += dip[k] * cexp(-sr * tk);
    }
    return wr * wr * s->tres[r].Rs_ohm / (s->tres[r].Q * wb) * q * acc;
}

/* Direct history sum of the transverse emissions (as history_sum). */
static double complex thistory_sum(const orc_sim *s, int r, int m)
{
    const double complex *ph = s->tr_phase[r];
    const unsigned char *keep = s->tr_keep[r];
    const int64_t n = s->turn;
    const int h = s->ring.h;
    double complex acc = 0.0;
    for (int64_t back = 0; back < s->nthist; ++back) {
        int64_t np = n - back;
        if (np < 0)
            break;
        const double complex *E = s->Ethist + ((size_t)r * s->nthist + (size_t)(np % s->nthist)) * s->nb;
        for (int mp = 0; mp < s->nb; ++mp) {
            int64_t D = back * (int64_t)h + (int64_t)s->bucket[m] - (int64_t)s->bucket[mp];
            if (D <= 0 || !keep[D])
                continue;
            acc += ph[D] * E[mp];
        }
    }
    return acc;
}

/* One turn for every bunch in fill order, then the wakes for the next turn. */
static void one_turn(orc_sim *s)
{
    const uint32_t turn32 = (uint32_t)s->turn;
    for (int m = 0; m < s->nb; ++m) {
        const int64_t n = s->n_mp[m];
        int32_t *hist = s->hist + (size_t)m * s->nbins;
        memset(hist, 0, sizeof(int32_t) * s->nbins);
        int64_t out = 0;
        double *tau = s->tau[m], *delta = s->delta[m];
        double *dip = s->trans ? s->dip + (size_t)m * s->nbins : NULL;
        if (dip)
            memset(dip, 0, sizeof(double) * s->nbins);
        for (int64_t i = 0; i < n; i += 4) {
            double r[4] = {0.0, 0.0, 0.0, 0.0}, rx[4] = {0.0, 0.0, 0.0, 0.0}, rxp[4] = {0.0, 0.0, 0.0, 0.0};
            if (s->dv.qe_amp != 0.0)
                orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, turn32, 0u, r);
            if (s->trans && s->tb_Dx != 0.0) {
                orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, turn32, 3u, rx);
                orc_normal_quad(s->seed, (uint32_t)(i / 4), (uint32_t)m, turn32, 4u, rxp);
            }
            for (int e = 0; e < 4 && i + e < n; ++e) {
                double t = tau[i + e], d = delta[i + e];
                /* wake kick with the previous turn's wake (zero on turn 0) */
                double V = vsr_at(s, m, orc_cell_coord(s, t)) + vlr_at(s, m, t);
                d = d - V / s->ring.E0_eV;
                const double d_before = d;
                /* Eq. 1: RF gain (main and harmonic cavities) minus mean radiation loss */
                d = d + s->dv.V_over_E0 * sin(s->dv.phi_s - s->dv.omega_rf * t);
                for (int k = 0; k < s->nharm; ++k)
                    d = d + s->harm_VoE0[k] * sin(s->harm[k].phi_rad - s->harm_nw[k] * t);
                const double d_gain = d;
                d = d - s->dv.U0_over_E0;
                /* Eq. 5, delta line: damping and quantum excitation */
                d = d * (1.0 - s->dv.D) + s->dv.qe_amp * r[e];
                if (s->trans) {
                    double x = s->x[m][i + e], xp = s->xp[m][i + e];
                    /* transverse wake kick (Eq. 6, second line), previous turn's wake */
                    double Vt = orc_tvoltage_at(s, m, t);
                    xp = xp + Vt / s->ring.E0_eV;
                    /* Eq. 5, x' line: momentum ratio across the cavity */
                    xp = xp * (1.0 + d_before) / (1.0 + d_gain);
                    /* Eqs. 3-4: betatron rotation with the chromatic phase of the new delta */
                    double psi = s->tb_mu0 * (1.0 + s->tb_xi * d);
                    double c = cos(psi), sn = sin(psi);
                    double xn = (c + s->tb_alpha * sn) * x + s->tb_beta * sn * xp;
                    double xpn = -s->tb_gamma * sn * x + (c - s->tb_alpha * sn) * xp;
                    /* Eq. 5, x and x' lines: excitation */
                    xn = xn + s->tb_sx * sqrt(s->tb_Dx) * rx[e];
                    xpn = xpn + s->tb_sxp * sqrt(s->tb_Dx) * rxp[e];
                    s->x[m][i + e] = xn;
                    s->xp[m][i + e] = xpn;
                }
                /* Eq. 2 with the new energy deviation (reading R1) */
                t = t + s->ring.alpha_c * s->ring.T0_s * d;
                tau[i + e] = t;
                delta[i + e] = d;
                /* binning (Sec. 2.3); dipole sums of the same cells */
                out += bin_one(s, t, hist);
                if (dip)
                    deposit_dip(s, t, s->x[m][i + e], dip);
            }
        }
        s->out_count[m] = out;
        /* statistics of the bunch (Sec. 2.4): two-pass mean and rms */
        double st = 0.0, sd = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            st += tau[i];
            sd += delta[i];
        }
        double mt = n > 0 ? st / (double)n : 0.0, md = n > 0 ? sd / (double)n : 0.0;
        double vt = 0.0, vd = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            vt += (tau[i] - mt) * (tau[i] - mt);
            vd += (delta[i] - md) * (delta[i] - md);
        }
        double *mo = s->moments + (size_t)m * 6;
        mo[0] = mt;
        mo[1] = n > 0 ? sqrt(vt / (double)n) : 0.0;
        mo[2] = md;
        mo[3] = n > 0 ? sqrt(vd / (double)n) : 0.0;
        mo[4] = (double)(n - out);
        mo[5] = (double)out;
        if (s->trans) {
            double sx = 0.0, sxp = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                sx += s->x[m][i];
                sxp += s->xp[m][i];
            }
            double mx = n > 0 ? sx / (double)n : 0.0, mxp = n > 0 ? sxp / (double)n : 0.0;
            double vx = 0.0, vxp = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                vx += (s->x[m][i] - mx) * (s->x[m][i] - mx);
                vxp += (s->xp[m][i] - mxp) * (s->xp[m][i] - mxp);
            }
            double *tm = s->tmoments + (size_t)m * 4;
            tm[0] = mx;
            tm[1] = n > 0 ? sqrt(vx / (double)n) : 0.0;
            tm[2] = mxp;
            tm[3] = n > 0 ? sqrt(vxp / (double)n) : 0.0;
        }
    }
    /* wakes from this turn's histograms, applied at the start of the next */
    for (int m = 0; m < s->nb; ++m)
        orc_vsr_direct(s, s->hist + (size_t)m * s->nbins, s->q_mp[m], s->Vsr + (size_t)m * s->nbins);
    for (int r = 0; r < s->nres; ++r) {
        if (!(s->res[r].range & ORC_RANGE_LONG))
            continue;
        double complex *E = s->Ehist + ((size_t)r * s->nhist + (size_t)(s->turn % s->nhist)) * s->nb;
        for (int m = 0; m < s->nb; ++m)
            E[m] = orc_emission(s, r, s->hist + (size_t)m * s->nbins, s->q_mp[m]);
        for (int m = 0; m < s->nb; ++m)
            s->Alr[(size_t)r * s->nb + m] = history_sum(s, r, m);
    }
    if (s->trans && s->rw_cent) {
        /* charge x centroid of every bunch (all its particles) for this turn's slot */
        double *cur = s->rw_cent + (size_t)(s->turn % (s->rw_nh + 1)) * s->nb;
        for (int m = 0; m < s->nb; ++m)
            cur[m] = s->current[m] * s->ring.T0_s * s->tmoments[(size_t)m * 4];
        for (int m = 0; m < s->nb; ++m) {
            double v = 0.0;
            for (int back = 0; back <= s->rw_nh; ++back) {
                if (s->turn - back < 0)
                    break;
                const double *src = s->rw_cent + (size_t)((s->turn - back) % (s->rw_nh + 1)) * s->nb;
                for (int mp = 0; mp < s->nb; ++mp) {
                    int64_t D = (int64_t)back * s->ring.h + (int64_t)s->bucket[m] - (int64_t)s->bucket[mp];
                    if (D <= 0)
                        continue;
                    v += src[mp] * orc_transverse_rw_wake(s, (double)D * s->dv.T_rf);
                }
            }
            s->Vrw[m] = v;
        }
    }
    if (s->trans) {
        for (int m = 0; m < s->nb; ++m)
            orc_vt_direct(s, s->dip + (size_t)m * s->nbins, s->q_mp[m], s->Vt + (size_t)m * s->nbins);
        for (int r = 0; r < s->ntres; ++r) {
            if (!(s->tres[r].range & ORC_RANGE_LONG))
                continue;
            double complex *E = s->Ethist + ((size_t)r * s->nthist + (size_t)(s->turn % s->nthist)) * s->nb;
            for (int m = 0; m < s->nb; ++m)
                E[m] = temission(s, r, s->dip + (size_t)m * s->nbins, s->q_mp[m]);
            for (int m = 0; m < s->nb; ++m)
                s->Atlr[(size_t)r * s->nb + m] = thistory_sum(s, r, m);
        }
    }
    s->turn += 1;
}

/* Track nturns; if rec is non-null it receives [nturns][nb][6] moments, if
 * trec is non-null (transverse plane set) [nturns][nb][4]: <x>, sig_x, <x'>, sig_x'. */
void orc_track2(orc_sim *s, int64_t nturns, double *rec, double *trec)
{
    for (int64_t t = 0; t < nturns; ++t) {
        one_turn(s);
        if (rec)
            memcpy(rec + (size_t)t * s->nb * 6, s->moments, sizeof(double) * s->nb * 6);
        if (trec && s->trans)
            memcpy(trec + (size_t)t * s->nb * 4, s->tmoments, sizeof(double) * s->nb * 4);
    }
}

/* orc_track2 without the transverse record. */
void orc_track(orc_sim *s, int64_t nturns, double *rec)
{
    orc_track2(s, nturns, rec, NULL);
}

/* Accessors (copies in and out of the simulation's arrays): transverse
 * coordinates of bunch m, dipole sums [nb][nbins], transverse voltage
 * [nb][nbins]. */
void orc_set_tparticles(orc_sim *s, int m, const double *x, const double *xp)
{
    memcpy(s->x[m], x, sizeof(double) * s->n_mp[m]);
    memcpy(s->xp[m], xp, sizeof(double) * s->n_mp[m]);
}

void orc_get_tparticles(const orc_sim *s, int m, double *x, double *xp)
{
    memcpy(x, s->x[m], sizeof(double) * s->n_mp[m]);
    memcpy(xp, s->xp[m], sizeof(double) * s->n_mp[m]);
}

void orc_get_dip(const orc_sim *s, double *dip)
{
    memcpy(dip, s->dip, sizeof(double) * (size_t)s->nb * s->nbins);
}

void orc_get_vt(const orc_sim *s, double *V)
{
    memcpy(V, s->Vt, sizeof(double) * (size_t)s->nb * s->nbins);
}

/* Transverse long-range amplitudes [ntres][nb] as interleaved (re, im). */
void orc_get_atlr(const orc_sim *s, double *A)
{
    for (size_t i = 0; i < (size_t)s->ntres * s->nb; ++i) {
        A[2 * i] = creal(s->Atlr[i]);
        A[2 * i + 1] = cimag(s->Atlr[i]);
    }
}

/* Accessors: histograms [nb][nbins] and out-of-mesh counts [nb] of the
 * last turn, short-range voltage [nb][nbins], lag wake [nbins]. */
void orc_get_hist(const orc_sim *s, int32_t *hist, int64_t *out_count)
{
    memcpy(hist, s->hist, sizeof(int32_t) * (size_t)s->nb * s->nbins);
    if (out_count)
        memcpy(out_count, s->out_count, sizeof(int64_t) * s->nb);
}

void orc_get_vsr(const orc_sim *s, double *V)
{
    memcpy(V, s->Vsr, sizeof(double) * (size_t)s->nb * s->nbins);
}

/* Long-range amplitudes [nres][nb] as interleaved (re, im). */
void orc_get_alr(const orc_sim *s, double *A)
{
    for (size_t i = 0; i < (size_t)s->nres * s->nb; ++i) {
        A[2 * i] = creal(s->Alr[i]);
        A[2 * i + 1] = cimag(s->Alr[i]);
    }
}

void orc_get_wlag(const orc_sim *s, double *W)
{
    memcpy(W, s->Wlag, sizeof(double) * s->nbins);
}

/* Test hooks for the long-range pieces: feed one turn of histograms without
 * moving particles (emission + direct history sum), as the end of a turn
 * does. hist is [nb][nbins]. */
void orc_feed_histograms(orc_sim *s, const int32_t *hist)
{
    memcpy(s->hist, hist, sizeof(int32_t) * (size_t)s->nb * s->nbins);
    for (int m = 0; m < s->nb; ++m)
        orc_vsr_direct(s, s->hist + (size_t)m * s->nbins, s->q_mp[m], s->Vsr + (size_t)m * s->nbins);
    for (int r = 0; r < s->nres; ++r) {
        if (!(s->res[r].range & ORC_RANGE_LONG))
            continue;
        double complex *E = s->Ehist + ((size_t)r * s->nhist + (size_t)(s->turn % s->nhist)) * s->nb;
        for (int m = 0; m < s->nb; ++m)
            E[m] = orc_emission(s, r, s->hist + (size_t)m * s->nbins, s->q_mp[m]);
        for (int m = 0; m < s->nb; ++m)
            s->Alr[(size_t)r * s->nb + m] = history_sum(s, r, m);
    }
    s->turn += 1;
}

/* Emission values of the last recorded turn for resonator r, (re, im) x nb. */
void orc_get_last_emission(const orc_sim *s, int r, double *E)
{
    int64_t t = s->turn - 1;
    if (t < 0)
        t = 0;
    const double complex *Er = s->Ehist + ((size_t)r * s->nhist + (size_t)(t % s->nhist)) * s->nb;
    for (int m = 0; m < s->nb; ++m) {
        E[2 * m] = creal(Er[m]);
        E[2 * m + 1] = cimag(Er[m]);
    }
}

/* Binning and dipole deposit of n given particles (arrival times tau,
 * offsets x) as a turn does them: hist and dip (nbins each) are overwritten;
 * returns the number outside the mesh.  For tests. */
int64_t orc_deposit(const orc_sim *s, int64_t n, const double *tau, const double *x, int32_t *hist, double *dip)
{
    memset(hist, 0, sizeof(int32_t) * s->nbins);
    memset(dip, 0, sizeof(double) * s->nbins);
    int64_t out = 0;
    for (int64_t i = 0; i < n; ++i) {
        out += bin_one(s, tau[i], hist);
        deposit_dip(s, tau[i], x[i], dip);
    }
    return out;
}

/* Kick-free single-particle evaluation of the wake voltage seen at tau by a
 * particle of bunch m (short + long range), for tests. */
double orc_wake_voltage_at(const orc_sim *s, int m, double tau)
{
    return vsr_at(s, m, orc_cell_coord(s, tau)) + vlr_at(s, m, tau);
}

int64_t orc_turn(const orc_sim *s) { return s->turn; }
