/*
 * mbt.h - C ABI of the GB300 longitudinal multi-bunch tracking library (libmbt).
 *
 * The library tracks the macro-particles of every bunch of a fill, turn after
 * turn, on one GPU, with the per-turn map of Xu, Locans, Adelmann and
 * Stingelin, "Calculation of Longitudinal Collective Instabilities with
 * mbtrack-cuda" (arXiv:1809.00391):
 *
 *   delta -= V_wake(tau) / E0                 wake kick            (Sec. 2.3, Eq. 6)
 *   delta += eps(tau) - U0/E0                 RF gain, SR loss     (Sec. 2.2, Eq. 1)
 *   delta  = delta (1 - D) + sigma_E sqrt(2D) r   damping + excitation (Sec. 2.2, Eq. 5)
 *   tau   += alpha_c T0 delta                 drift                (Sec. 2.2, Eq. 2)
 *   bin tau into a fixed mesh, per-bunch mean / rms           (Sec. 2.3, Sec. 2.4)
 *   short-range wake: causal convolution of the line density with the summed
 *   resonator wake; long-range wake: resonator phasors carried from every
 *   earlier bunch passage, this turn and earlier turns   (Sec. 2.3, last paragraph)
 *
 * with these readings of the paper: the drift uses the updated delta; D =
 * 2 T0 / tau_z; eps(tau) = (eV/E0) sin(phi_s - omega_rf tau) with sin(phi_s) =
 * U0 / eV; omega_rf = 2 pi h / T0; the wake W(t) of a resonator (Rs, w_r, Q) is
 * 2 a Rs e^{-a t}[cos(wb t) - (a/wb) sin(wb t)] for t > 0 (a = w_r/2Q,
 * wb = sqrt(w_r^2 - a^2)), 0 for t < 0 and half of W(0+) at zero lag.
 *
 * Conventions
 *  - SI units: seconds, volts, ohms, hertz, amperes, coulombs; energies in eV.
 *  - Every call returns an mbt_status (0 = MBT_OK).  No C++ exception crosses
 *    the ABI.  On failure mbt_last_error() returns a message.
 *  - The library owns all device memory it allocates (cudaMalloc inside
 *    mbt_set_fill); the caller owns every host buffer passed in.  Host
 *    pointers are only read or written during the call.
 *  - A context is thread-compatible: one thread at a time.  Contexts are
 *    independent of each other.
 *  - "stream" arguments are a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Tracking calls are asynchronous on that stream;
 *    mbt_sync() or any read call waits for it.
 *  - Device errors (a kernel that failed, a bounded wait that gave up) are
 *    reported by the next call that synchronises.
 */
#ifndef MBT_H
#define MBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MBT_VERSION 100

typedef int mbt_status;
enum {
    MBT_OK = 0,
    MBT_ERR_ARG = 1,          /* invalid argument (value out of range, null pointer)   */
    MBT_ERR_STATE = 2,        /* call not valid in the context's current state         */
    MBT_ERR_NOMEM = 3,        /* device or host allocation failed                      */
    MBT_ERR_CUDA = 4,         /* a CUDA runtime call or kernel failed                  */
    MBT_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up                    */
    MBT_ERR_UNSUPPORTED = 6,  /* configuration outside what the library implements    */
    MBT_ERR_BUDGET = 7        /* request exceeds the memory budget (serving)           */
};

/* Precision of the tracking path. */
enum {
    MBT_PREC_F64 = 0,    /* every step in FP64; histograms bit-exact vs an FP64 tracker    */
    MBT_PREC_MIXED = 1   /* tau FP32; delta stored and accumulated in FP64; push arithmetic
                            FP32; short-range wake on the tensor cores (BF16 hi/lo split of
                            the wake, byte-split counts, FP32 accumulation); long-range
                            phasor scan and moment sums in FP64                           */
};

/* Resonator range: short range = convolution within the bunch's own passage;
 * long range = phasor carried to every later passage. */
enum { MBT_RANGE_SHORT = 1, MBT_RANGE_LONG = 2, MBT_RANGE_BOTH = 3 };

/* Option flags (mbt_create). */
enum {
    MBT_NO_SR = 1,     /* no radiation: U0 = 0 (phi_s = 0 or pi), no damping, no excitation */
    MBT_NO_QE = 2,     /* radiation damping kept, quantum excitation removed                */
    MBT_KICK_NGP = 4   /* short-range kick from the particle's own cell instead of linear
                          interpolation between cell centres                                */
};

/* Ring parameters (Table 1 of the paper lists them for the 'dc12c' lattice). */
typedef struct {
    double E0_eV;        /* reference energy [eV], > 0                                  */
    double T0_s;         /* revolution period [s], > 0                                   */
    int32_t h;           /* harmonic number, 1..65535                                    */
    int32_t reserved;    /* must be 0                                                    */
    double V_rf_V;       /* peak RF voltage [V], > U0                                    */
    double alpha_c;      /* momentum compaction factor, != 0 (sign selects phi_s branch) */
    double U0_eV;        /* radiation loss per turn [eV], >= 0                           */
    double sigma_delta;  /* natural relative energy spread sigma_E, > 0                  */
    double tau_z_s;      /* longitudinal amplitude damping time [s], > 0                 */
} mbt_ring;

/* Derived quantities, as the library computes them (mbt_get_info). */
typedef struct {
    double T_rf_s, omega_rf, phi_s, nu_s, sigma_tau0_s;
    double D;                  /* damping decrement per turn                         */
    double half_width_s;       /* H: the mesh covers [-H, H)                         */
    double bin_width_s;        /* Delta = 2H / nbins                                 */
    int64_t n_particles;       /* all bunches                                        */
    int64_t turn;              /* turns completed                                    */
    int32_t nb, nbins, n_long, precision;
    int64_t device_bytes;      /* device memory held by the context                  */
    int32_t push_ctas;         /* CTAs of the streaming push tracking the context    */
                               /* on its own (0: the per-tile or FP64 push)          */
    int32_t reserved;
} mbt_info;

typedef struct mbt_ctx mbt_ctx;
typedef struct mbt_batch mbt_batch;

/* Library version (MBT_VERSION) and a static message for a status code. */
int mbt_version(void);
const char *mbt_status_string(mbt_status s);

/* Create a context for one run.  precision: MBT_PREC_*; flags: MBT_NO_SR |
 * MBT_NO_QE | MBT_KICK_NGP; seed: 64-bit key of the Philox4x32-10 streams
 * (Salmon et al., SC'11) that draw the initial distribution and the quantum
 * excitation: one block per quad of consecutive particles, counter = (quad,
 * bunch, turn, tag), tag 0 the delta excitation of a turn, 1 / 2 the initial
 * tau / delta, 3 / 4 the x / x' excitation, 5 / 6 the initial x / x'.
 * Errors: MBT_ERR_ARG on a null pointer or an invalid ring. */
mbt_status mbt_create(const mbt_ring *ring, int precision, int flags, uint64_t seed, mbt_ctx **out);

/* Destroy a context and free its device memory (synchronises its stream).
 * Accepts NULL. */
void mbt_destroy(mbt_ctx *ctx);

/* Message of the last failed call on this context ("" if none).  The string
 * is owned by the context and valid until the next call on it. */
const char *mbt_last_error(const mbt_ctx *ctx);

/* Add a resonator to the wake model (Sec. 2.3: the wake is the sum of the
 * resonators').  Rs_ohm > 0, fr_Hz > 0, Q > 0.5, range MBT_RANGE_*.  At most
 * 8 resonators, at most 4 with the long-range bit.  Only before
 * mbt_set_fill. */
mbt_status mbt_add_resonator(mbt_ctx *ctx, double Rs_ohm, double fr_Hz, double Q, int range);

/* Add an active harmonic RF cavity (the paper's RF step holds "additional
 * harmonic cavities"): its voltage V_V at n x the RF frequency and phase
 * phi_rad at the synchronous particle add (V_V / E0) sin(phi_rad - n
 * omega_rf tau) to a turn's energy change.  The main cavity's phase then
 * balances the mean loss against them: V sin(phi_s) + sum V_h sin(phi_h) =
 * U0 (MBT_ERR_ARG at mbt_set_fill if no such phase exists); sigma_tau0 (the
 * mesh unit and the matched start) keeps the main cavity's slope V
 * cos(phi_s), since a double-RF system can have no small-amplitude tune (a
 * flat potential).  1 <= n <= 16, V_V >= 0.  Only before mbt_set_grid /
 * mbt_set_fill; at most 2 cavities.  A passive (beam-loaded) harmonic cavity
 * is a resonator near n f_rf with the long-range bit instead. */
mbt_status mbt_add_harmonic_cavity(mbt_ctx *ctx, int n, double V_V, double phi_rad);

/* Transverse plane (Eqs. 3-5, x lines; Eq. 6, second line).  One plane per
 * run (x or y: the paper treats them alike, and they couple to each other
 * through nothing but the longitudinal motion, which they do not change, so
 * two runs with the same seed give both planes of one run).  Twiss beta_m,
 * alpha at the tracking point, where the dispersion is taken as zero;
 * betatron phase advance per turn 2 pi tune (1 + chromaticity delta) (Eq. 3);
 * equilibrium emittance emittance_m.  Per turn, after the previous turn's
 * transverse wake kick x' += V_x(tau) / E0: x' scales by the momentum ratio
 * across the RF cavity (1 + delta) / (1 + delta + eps) (Eq. 5), the Twiss
 * rotation (Eq. 4) uses the updated delta, then the excitation
 * sqrt(beta emit D_x) r, sqrt(gamma emit D_x) r' with D_x = U0 / E0 (the
 * damping the momentum ratio produces on average, so emittance_m is the
 * equilibrium; none with MBT_NO_SR / MBT_NO_QE).  Only before mbt_set_fill.
 * Checkpoints include it; mbt_track_resident refuses it (MBT_ERR_UNSUPPORTED).
 * MBT_PREC_MIXED sums the dipole moments of a cell in fixed point: x in
 * units of u = 2^(e - 20) m, 2^e = sqrt(beta_m emittance_m) rounded up to a
 * power of two (at least 2^-16 m), exact sums of the quantised x; it accepts
 * |x| < 2^(e + 10) m after the turn's map, and a particle beyond that makes
 * the next synchronising call return MBT_ERR_UNSUPPORTED (its x then
 * deposits clamped). */
mbt_status mbt_set_transverse(mbt_ctx *ctx, double beta_m, double alpha, double tune, double chromaticity,
                              double emittance_m);

/* Add a transverse resonator (shunt impedance Rs in Ohm/m): wake
 * W(t > 0) = (wr^2 Rs / (Q wb)) e^{-a t} sin(wb t), a = wr / 2Q,
 * wb = sqrt(wr^2 - a^2); the kick of a particle is the sum over earlier
 * cells and passages of charge x dipole moment x W (Eq. 6, second line).
 * range MBT_RANGE_* as for mbt_add_resonator; long-range entries count
 * towards the limit of 4 shared with the longitudinal ones.  Needs
 * mbt_set_transverse first; only before mbt_set_fill. */
mbt_status mbt_add_transverse_resonator(mbt_ctx *ctx, double Rs_ohm_per_m, double fr_Hz, double Q, int range);

/* Add the long-range transverse resistive wall of a round pipe (radius_m,
 * conductivity_S_per_m, length_m; the paper applies it to the transverse
 * planes from the statistics of earlier bunches): far from the head the
 * dipole wake is W(t) = (c L / (pi b^3)) sqrt(Z0 / (pi sigma)) / sqrt(c t)
 * [V/(C m)], and every particle of a bunch gets x' += (1/E0) sum Q_p <x>_p
 * W(t_m - t_p) over the passages of the last history_turns turns before its
 * own (1 <= history_turns <= 1000; the bunch's own earlier turns count).
 * Several pipes add up; the longest history is kept.  Needs
 * mbt_set_transverse; only before mbt_set_fill. */
mbt_status mbt_add_transverse_resistive_wall(mbt_ctx *ctx, double radius_m, double conductivity_S_per_m,
                                             double length_m, int history_turns);

/* Copy one bunch's transverse coordinates from host arrays of n_mp[bunch]
 * doubles (MBT_PREC_MIXED rounds to FP32) / to host arrays.  Synchronous. */
mbt_status mbt_set_transverse_particles(mbt_ctx *ctx, int bunch, const double *x_m, const double *xp);
mbt_status mbt_get_transverse_particles(mbt_ctx *ctx, int bunch, double *x_m, double *xp);

/* Per-turn transverse moments of turns [turn0, turn0 + nturns) into
 * out[nturns][nb][4]: <x>, rms x, <x'>, rms x' (after the turn's map, like
 * mbt_read_moments).  Synchronous. */
mbt_status mbt_read_transverse_moments(mbt_ctx *ctx, int64_t turn0, int64_t nturns, double *out);

/* Dipole sums (sum of x over each cell's particles, [nb][nbins]) of the last
 * completed turn and the transverse short-range voltage [V] built from them
 * for the next kick ([nb][nbins]); either may be NULL.  MBT_PREC_MIXED
 * returns the exact sums of the quantised x (see mbt_set_transverse), which
 * do not depend on the push tiling.  Synchronous. */
mbt_status mbt_read_transverse_wake(mbt_ctx *ctx, double *dipoles, double *V);

/* Add a tabulated short-range wake (Sec. 2.3: other wakes, such as the
 * resistive wall, are added to the same wake).  W_V_per_C[i] is W(t_s[i]) in
 * V/C (positive = energy loss), t_s[0] = 0 (W(0+)) and t_s strictly
 * increasing; W is linear between samples and zero beyond the last one.  It
 * acts on the mesh through its average over each lag cell: lag l >= 1 gets
 * (1/Delta) times the integral of W over [(l - 1/2) Delta, (l + 1/2) Delta],
 * lag 0 the integral over [0, Delta / 2] (the half value of W(0+) for a
 * smooth wake), so a wake whose head is much shorter than a cell keeps its
 * integral.  Short range only.  The arrays are copied.  Only before
 * mbt_set_fill; at most 8 tables. */
mbt_status mbt_add_wake_table(mbt_ctx *ctx, int n, const double *t_s, const double *W_V_per_C);

/* Add the short-range longitudinal resistive-wall wake of a round pipe of
 * radius_m, wall conductivity_S_per_m and length_m (no counterpart call in the
 * paper, whose resistive-wall test is a copper pipe of 10 mm radius around
 * the ring): with s = c t, s0 = (2 b^2 / (Z0 sigma))^(1/3), u = s / s0,
 *   W(t) = (4 Z0 c L / (pi b^2)) [ e^{-u} cos(sqrt(3) u) / 3
 *                                  - (sqrt(2) / pi) int_0^inf x^2 e^{-x^2 u} / (x^6 + 8) dx ]
 * (Bane and Sands, 1995), applied through its cell averages like
 * mbt_add_wake_table (computed from the closed form, not from samples).
 * All arguments > 0.  Only before mbt_set_fill; at most 8 pipes. */
mbt_status mbt_add_resistive_wall(mbt_ctx *ctx, double radius_m, double conductivity_S_per_m, double length_m);

/* Longitudinal mesh (Sec. 2.3): nbins cells over [-H, H), H =
 * half_width_sigmas * sigma_tau0 with sigma_tau0 = |alpha_c| sigma_E T0 /
 * (2 pi nu_s).  MBT_PREC_F64: 2 <= nbins <= 1024.  MBT_PREC_MIXED: nbins 128
 * or 256.  Default 256 cells, 5 sigma.  Only before mbt_set_fill. */
mbt_status mbt_set_grid(mbt_ctx *ctx, int nbins, double half_width_sigmas);

/* Fill pattern: nb bunches in strictly increasing buckets 0 <= bucket < h,
 * bunch current current_A[m] >= 0 [A] (macro-charge = I T0 / N) and n_mp[m]
 * macro-particles (1 .. 2^31-2; MBT_PREC_MIXED: up to 2^24-1 so that a cell
 * count is exact in three bytes).  Allocates every device buffer.  Particles
 * start at zero; call mbt_init_particles or mbt_set_particles.  Errors:
 * MBT_ERR_ARG, MBT_ERR_NOMEM, MBT_ERR_STATE (fill already set). */
mbt_status mbt_set_fill(mbt_ctx *ctx, int nb, const int32_t *bucket, const double *current_A,
                        const int64_t *n_mp);

/* Capacity of the device ring buffer of per-turn moments, in turns (default
 * 4096).  Only before mbt_set_fill. */
mbt_status mbt_set_record(mbt_ctx *ctx, int64_t capacity_turns);

/* Matched Gaussian start: tau ~ N(0, sigma_tau0), delta ~ N(0, sigma_E), from
 * the Philox streams with tags 1 (tau) and 2 (delta) at turn 0.  Resets the
 * turn counter and every wake to zero.  Asynchronous on stream. */
mbt_status mbt_init_particles(mbt_ctx *ctx, void *stream);

/* Copy one bunch's coordinates from host arrays of n_mp[bunch] doubles
 * (MBT_PREC_MIXED rounds tau to FP32).  Synchronous. */
mbt_status mbt_set_particles(mbt_ctx *ctx, int bunch, const double *tau_s, const double *delta);

/* Copy every bunch's coordinates from host arrays of n_particles doubles
 * each: bunch 0's n_mp[0] values, then bunch 1's, ... (no padding).  When
 * both arrays are page-locked and device-addressable (cudaHostAlloc /
 * cudaMallocHost / cudaHostRegister'ed memory; checked with
 * cudaPointerGetAttributes) one kernel on `stream` reads them across the
 * host link and writes the device layout; otherwise the call falls back to
 * mbt_set_particles bunch by bunch.  The result is the same either way
 * (MBT_PREC_MIXED rounds tau to FP32).  Synchronous: the arrays may be
 * reused when the call returns.  The caller guarantees that each array holds
 * n_particles doubles. */
mbt_status mbt_set_particles_all(mbt_ctx *ctx, const double *tau_s, const double *delta, void *stream);

/* The same with tau in FP32 host arrays (n_particles floats; delta stays
 * n_particles doubles): the precision MBT_PREC_MIXED stores tau in, so 12
 * bytes per particle cross the host link instead of 16.  MBT_PREC_F64
 * widens tau exactly.  Same fallback, errors and synchronisation as
 * mbt_set_particles_all. */
mbt_status mbt_set_particles_all_f32(mbt_ctx *ctx, const float *tau_s, const double *delta, void *stream);

/* Copy one bunch's coordinates to host arrays of n_mp[bunch] doubles.
 * Synchronous (waits for tracking in flight). */
mbt_status mbt_get_particles(mbt_ctx *ctx, int bunch, double *tau_s, double *delta);

/* Track nturns turns (asynchronous on stream).  Each turn runs the push
 * kernel over every bunch and the post kernel (wakes, moments).  If graph
 * replay is enabled (mbt_set_graph) whole chunks of turns are replayed from a
 * captured CUDA graph. */
mbt_status mbt_track(mbt_ctx *ctx, int64_t nturns, void *stream);

/* Cluster-resident tracking (MBT_PREC_MIXED, at most 32 bunches): one
 * thread-block cluster of up to 16 CTAs per bunch keeps the bunch's particles
 * in distributed shared memory for all nturns turns of one launch, and the
 * clusters meet once per turn for the long-range phasor scan.  Same map and
 * outputs as mbt_track (the short-range wake is an FP32 convolution on the
 * CUDA cores instead of the tensor-core contraction); turns may alternate
 * with mbt_track.  MBT_ERR_UNSUPPORTED if the fill does not fit on chip.
 * Asynchronous on stream. */
mbt_status mbt_track_resident(mbt_ctx *ctx, int64_t nturns, void *stream);

/* Cluster shape mbt_track_resident would use: CTAs per cluster (0 if the fill
 * does not fit on chip) and particles held per CTA. */
mbt_status mbt_resident_shape(mbt_ctx *ctx, int *cluster, int *per_cta);

/* Wait for the context's work; report device errors: MBT_ERR_TIMEOUT (a
 * bounded wait gave up), MBT_ERR_ARG (a cell count of 2^24 or more reached
 * the tensor-core wake), MBT_ERR_UNSUPPORTED (a transverse coordinate beyond
 * the mixed dipole range, see mbt_set_transverse), MBT_ERR_CUDA.  The error
 * word is cleared once reported. */
mbt_status mbt_sync(mbt_ctx *ctx);

/* Failure-detection test hook for the bounded device waits.  limit_ns (0 =
 * the default of 2 s, at most 1e10) replaces the wall-clock limit of
 * mbt_track_resident's grid barrier (the wait of every cluster for the other
 * bunches' emissions of the turn, used when a fill of several bunches has a
 * long-range resonator).  unreachable = 1 makes that barrier wait for one
 * arrival more than the fill has bunches, a count nothing reaches: every
 * cluster's wait then runs out after limit_ns, the kernel records
 * MBT_ERR_TIMEOUT in the context's error word, every CTA of a cluster leaves
 * the turn loop together and writes its state back, and the next
 * synchronising call returns MBT_ERR_TIMEOUT.  No fault is involved; the
 * context can be destroyed normally.  Host only; MBT_ERR_ARG on bad values. */
mbt_status mbt_set_wait_test(mbt_ctx *ctx, int64_t limit_ns, int unreachable);

/* Per-turn moments of turns [turn0, turn0 + nturns) into out[nturns][nb][6]:
 * <tau>, rms tau, <delta>, rms delta, particles inside the mesh, outside.
 * The statistics are taken after the drift of the turn, before the next
 * turn's wake kick.  Turns older than the record capacity are gone
 * (MBT_ERR_ARG).  Synchronous. */
mbt_status mbt_read_moments(mbt_ctx *ctx, int64_t turn0, int64_t nturns, double *out);

/* Histograms [nb][nbins] (int32) and outside counts [nb] (int64, may be NULL)
 * of the last completed turn.  Synchronous. */
mbt_status mbt_read_histograms(mbt_ctx *ctx, int32_t *hist, int64_t *outside);

/* Wake state that the next turn's kick will use: short-range voltage
 * Vsr[nb][nbins] [V] and the long-range phasor Phi[n_long][nb][2] (re, im) such
 * that V_long(tau) = sum_r Re(Phi_r,m e^{s_r tau}).  Either pointer may be
 * NULL.  Synchronous. */
mbt_status mbt_read_wake(mbt_ctx *ctx, double *Vsr, double *Phi);

/* Derived quantities and sizes. */
mbt_status mbt_get_info(mbt_ctx *ctx, mbt_info *info);

/* CUDA-graph replay: capture turns_per_graph turns once and replay the graph
 * (0 disables; default 0).  The first mbt_track after a change captures. */
mbt_status mbt_set_graph(mbt_ctx *ctx, int turns_per_graph);

/* Push tile: at most this many macro-particles per CTA of the per-tile
 * mixed-precision push, a multiple of 4 in [1024, 65536] (default 8192); each
 * bunch is split into ceil(n / tile) tiles of equal size.  Changing it
 * rebuilds the work lists (and drops a captured graph); results do not depend
 * on it except for the summation order of the moment sums.  A plan whose runs
 * are all large (no transverse plane; every run at least 4 stages of 3968
 * particles per SM, bunches of at least 2 stages on average) uses the
 * streaming push instead, which cuts each run into one equal share per SM
 * whatever the tile (stored, no effect); a run's moments are then the same
 * alone and in any such batch. */
mbt_status mbt_set_tile(mbt_ctx *ctx, int particles);

/* Host-only planning queries (no device, no context): the decisions the
 * library takes when it builds a mixed-precision plan.
 * mbt_plan_streams: *streams = 1 if runs of run_n[i] macro-particles in
 * run_nb[i] bunches (i < nruns) would be tracked by the streaming push on a
 * device holding `ctas` streaming-push CTAs at once, 0 for the per-tile push
 * (see mbt_set_tile).  MBT_ERR_ARG for nruns, ctas, a size or a bunch count
 * below 1 or a NULL pointer.
 * mbt_plan_stream_split: the streaming push's work split of nb bunches (bunch
 * i: run[i] >= 0, non-decreasing, n_mp[i] >= 1 macro-particles) over `ctas`
 * CTAs.  Each run's particle sequence (its bunches in order, each padded to a
 * multiple of 4) is cut into `ctas` shares at multiples of 4, share g =
 * [4 floor(P' g / ctas), 4 floor(P' (g + 1) / ctas)) with P' the run's padded
 * length / 4 (the last share ends at the padded length), and each share into
 * tiles at bunch boundaries (at most 2^28 particles).  Tile k is written as
 * out[4k .. 4k+3] = (bunch, first particle within the bunch, count, CTA) for
 * k < cap, in bunch order; *ntiles receives the number of tiles (call with
 * cap = 0 to size out; the caller owns out).  MBT_ERR_ARG on invalid input,
 * nothing written. */
mbt_status mbt_plan_streams(int nruns, const int64_t *run_n, const int32_t *run_nb, int any_transverse, int ctas,
                            int *streams);
mbt_status mbt_plan_stream_split(int nb, const int32_t *run, const int64_t *n_mp, int ctas, int64_t *out,
                                 int64_t cap, int64_t *ntiles);
/* mbt_plan_lanes: the groups mbt_batch_set_lanes forms from nmembers members
 * of n_particles[i] >= 0 macro-particles: lane[i] in 0 .. min(nlanes,
 * nmembers) - 1 (caller-owned, nmembers entries).  Members are taken largest
 * first (ties in member order), each into the lane with the fewest particles
 * so far (ties: the lower lane).  MBT_ERR_ARG for nmembers < 1, nlanes
 * outside 1..8, a negative count or a NULL pointer, nothing written. */
mbt_status mbt_plan_lanes(int nmembers, const int64_t *n_particles, int nlanes, int32_t *lane);

/* Autotuner (plans on the per-tile push): times turns_per_trial turns for
 * each candidate push tile (2048 .. 32768 particles, plus tiles that make the
 * tile count a whole multiple of the push CTAs the GPU holds at once) and
 * keeps the fastest (written to *chosen_tile, may be NULL).  The trial turns
 * are real tracking turns: the run advances by (turns_per_trial + 2) turns
 * per candidate (at most 17).  Synchronous.  No-op (the current tile is
 * reported, no turn is tracked) for MBT_PREC_F64 and for plans on the
 * streaming push (see mbt_set_tile). */
mbt_status mbt_autotune(mbt_ctx *ctx, int turns_per_trial, int *chosen_tile);

/* Kernel timing: when enabled, mbt_track records CUDA events around every
 * push-kernel launch on the tracking stream.  mbt_get_timing returns the sum
 * of their durations [ms] and the number of timed launches since the last
 * reset (enable = 1 resets).  Timing forces plain launches (no graph). */
mbt_status mbt_set_timing(mbt_ctx *ctx, int enable);
mbt_status mbt_get_timing(mbt_ctx *ctx, double *push_ms, double *post_ms, int64_t *launches);

/* Post-kernel trace: when enabled, every CTA of the post kernel records
 * %globaltimer [ns] at its start, when its own job is done, and at exit (the
 * last CTA to finish also composes the phasor tiles and advances the turn).
 * mbt_read_trace copies the record of the last post launch into
 * out[min(max_jobs, njobs)][5] = job type (0 wake, 1 tile), bunch tile,
 * start, job done, exit; *njobs receives the number of post CTAs (out may be
 * NULL to query it).  Enabling or disabling drops a captured graph. */
mbt_status mbt_set_trace(mbt_ctx *ctx, int enable);
mbt_status mbt_read_trace(mbt_ctx *ctx, int64_t *out, int max_jobs, int *njobs);

/* Checkpoint: mbt_state_size gives the bytes of a snapshot (particles, turn,
 * wake and phasor carry, histograms); mbt_save_state writes it into buf;
 * mbt_load_state restores it into a context with the same configuration.
 * A resumed run is bit-identical to an uninterrupted one. */
mbt_status mbt_state_size(mbt_ctx *ctx, size_t *bytes);
mbt_status mbt_save_state(mbt_ctx *ctx, void *buf, size_t bytes);
mbt_status mbt_load_state(mbt_ctx *ctx, const void *buf, size_t bytes);

/* Short-range wake voltage of nb bunches from their cell counts, computed by
 * the same tensor-core Toeplitz kernel as mbt_track's post step, WITHOUT
 * ALLOCATING ANY DEVICE MEMORY.  For callers that cannot call cudaMalloc:
 * code that runs inside another framework's device memory pool or under a
 * fixed device-memory budget, where an allocation by a library would fail or
 * fragment the pool.  (The paper has no counterpart; this is a library
 * service.)
 *   ring, flags, half_width_sigmas, nbins: define the mesh as in mbt_set_grid
 *     (nbins must be 128 or 256);
 *   nres resonators (Rs_ohm, fr_Hz, Q, range: host arrays; only those with
 *     the short-range bit contribute), at most 8;
 *   nb bunches, 1..1024; charge_per_count[nb]: host, coulombs per count;
 *   hist: DEVICE int32 [nb][nbins] counts (input, caller-owned), 16-byte
 *     aligned (the kernel reads it 16 bytes at a time), every count in
 *     [0, 2^24) (the tensor-core kernel splits a count into three exact
 *     8-bit planes);
 *   V: DEVICE float [nb][nbins] voltages [V] (output, caller-owned), 4-byte
 *     aligned;
 *   stream: cudaStream_t as void*; errbuf/errlen: optional message buffer.
 * Sizes beyond these limits return MBT_ERR_UNSUPPORTED with a message; a
 * null or misaligned pointer MBT_ERR_ARG before any device work; a count
 * outside [0, 2^24) MBT_ERR_ARG after the launch (V then holds no valid
 * result).  Working memory is a 256 KB array in the library's static device
 * memory, held by every GPU that loads the library until the process exits;
 * the first call on a device resolves that array's device address.  The call
 * is synchronous (it waits for the stream and reads an error word back), so
 * it cannot be captured into a CUDA graph: on a stream that is being
 * captured it returns MBT_ERR_STATE without doing anything.  All calls share
 * the array (host calls are serialised by the library), so calls from
 * another process or kernels that modify hist or V while it runs race. */
mbt_status mbt_wake_noalloc(const mbt_ring *ring, int flags, int nres, const double *Rs_ohm, const double *fr_Hz,
                            const double *Q, const int32_t *range, int nbins, double half_width_sigmas, int nb,
                            const double *charge_per_count, const int32_t *hist, float *V, void *stream,
                            char *errbuf, size_t errlen);

/* ------------------------------------------------------------------------
 * Bunch-sharded long-range scan (host side of splitting one fill's bunches
 * over several GPUs in contiguous ranges; Sec. 2.3, last paragraph: the
 * long-range wake acts after all bunches).  Bunch m meets the phasor
 * Phi_m = a_m X_{m-1} and leaves X_m = Phi_m + E_m (E_m its emission,
 * c q_m sum_k count_k e^{-s tau_k}; a_m = e^{s dt_m}, dt_m the bucket distance
 * from the bunch before it, for the first bunch of a turn from the last bunch
 * of the previous turn across the gap).  A rank reduces its bunches to one
 * map X -> A X + B (mbt_phasor_segment); the ranks allgather the maps (4
 * doubles per long-range resonator); every rank composes them in rank order
 * starting from the value carried from the previous turn
 * (mbt_phasor_compose), which gives the value entering its own range and the
 * next carry, and applies it to its bunches (mbt_phasor_apply).  Complex
 * numbers are (re, im) pairs of doubles; arrays are host memory owned by the
 * caller.  Host only (no GPU); MBT_ERR_ARG on a null pointer or bad size. */
/* step[2 m], step[2 m + 1] = a_m for bunches in strictly increasing buckets
 * bucket[0 .. nb-1] of the ring and one resonator (fr_Hz, Q > 1/2). */
mbt_status mbt_phasor_steps(const mbt_ring *ring, double fr_Hz, double Q, int nb, const int32_t *bucket,
                            double *step);
/* map[0..3] = (A, B) of f_{n-1} o ... o f_0, f_m(X) = a_m X + E_m (n >= 0;
 * n = 0 gives the identity). */
mbt_status mbt_phasor_segment(int n, const double *step, const double *E, double *map);
/* maps[4 r .. 4 r + 3]: the maps of nseg consecutive ranges; carry: X after
 * the last bunch of the previous turn.  entry[2 r] (optional): the value
 * entering range r; carry_out: X after the last range. */
mbt_status mbt_phasor_compose(int nseg, const double *maps, const double *carry, double *entry, double *carry_out);
/* phi[2 m] = Phi_m of a range's n bunches given the value entering it. */
mbt_status mbt_phasor_apply(int n, const double *step, const double *E, const double *entry, double *phi);

/* Measures the FP64 fused multiply-add throughput of the current GPU (the
 * bound of the FP64 tracker): blocks_per_sm x (SM count) CTAs of 256 threads
 * each run 8 independent chains of iters DFMAs, launched `repeats` times on
 * stream and timed with CUDA events after one untimed launch.  flops_per_s:
 * 2 flops per DFMA over the timed launches; sms (optional): the SM count.
 * Synchronous.  MBT_ERR_ARG on values outside blocks_per_sm 1..32,
 * iters 1..2^24, repeats >= 1; MBT_ERR_CUDA without a GPU. */
mbt_status mbt_probe_fp64_fma(int blocks_per_sm, int iters, int repeats, void *stream, double *flops_per_s, int *sms);

/* Batched tracking: n contexts with the same precision, each with its fill
 * set, tracked together in the same kernel launches (one push and one post
 * launch per turn for all of them).  The contexts stay owned by the caller
 * and must outlive the batch. */
mbt_status mbt_batch_create(mbt_ctx *const *ctxs, int n, mbt_batch **out);
mbt_status mbt_batch_track(mbt_batch *b, int64_t nturns, void *stream);
mbt_status mbt_batch_sync(mbt_batch *b);   /* wait; report device errors of the batch and of its members
                                              (the first one; the message on the first member) */
/* Graph replay and push-tile autotuning for a batch, as for a context. */
mbt_status mbt_batch_set_graph(mbt_batch *b, int turns_per_graph);
mbt_status mbt_batch_autotune(mbt_batch *b, int turns_per_trial, int *chosen_tile);
/* Lanes: mbt_batch_track splits the members into nlanes groups of about equal
 * particle counts (largest member first, each into the group with the fewest
 * particles so far; members keep the batch order within a group), each group
 * with launches of its own on a stream of the batch's own, forked from and
 * joined back into the caller's stream (asynchronous on it).  One group's
 * push then runs beside another's post kernel, whose turns are bound by
 * latency rather than bandwidth (scans of many runs of small bunches).  The
 * turn map is per run (runs share no state), so every member's results are
 * the same bit for bit with any number of lanes, alone or in a batch.
 * nlanes 1..8 (1: one plan for the whole batch, the default); more lanes
 * than members give one member per lane.  Synchronises the device; takes
 * the batch's push tile (mbt_batch_autotune rebuilds the lanes with the tile
 * it chooses) and graph setting.  Errors of a lane's kernels surface at
 * mbt_batch_sync.  MBT_ERR_ARG for nlanes outside 1..8. */
mbt_status mbt_batch_set_lanes(mbt_batch *b, int nlanes);
/* Chooses the lane count: each count 1..max_lanes (at most the member count)
 * tracked for turns_per_trial warm-up turns and turns_per_trial timed turns
 * (CUDA events; graph replay where the batch's graph setting covers
 * turns_per_trial), the fastest set and returned in *chosen (optional).
 * The trials are real turns of every member: they advance the runs by
 * 2 x turns_per_trial x (counts tried) turns.  Synchronous.  MBT_ERR_ARG for
 * turns_per_trial < 1 or max_lanes outside 1..8. */
mbt_status mbt_batch_autotune_lanes(mbt_batch *b, int turns_per_trial, int max_lanes, int *chosen);
/* Track every member resident (as mbt_track_resident) at the same time: each
 * member's kernel on a stream of the batch's own, forked from and joined back
 * into `stream` (asynchronous on it).  Errors of the kernels surface at
 * mbt_batch_sync or a member's synchronising call; if a launch fails after
 * others have started, those keep running and the next sync waits for them.
 * For scans of many small runs, whose turns in the per-tile push are bound by
 * launch latency.  Every member must fit resident and must not couple
 * several bunches over long range (its clusters would meet in a grid
 * barrier, which needs all of them on the GPU at once): otherwise
 * MBT_ERR_UNSUPPORTED before any launch.  The cluster size is capped (16, 8,
 * 4, 2 or 1 CTAs) at the largest value for which the clusters of all members
 * fit on the GPU together (one CTA per SM, and no more clusters than the
 * occupancy query for that size allows: a cluster takes SMs of one GPC); a
 * member whose own size (mbt_resident_shape) is within the cap gets the
 * results of mbt_track_resident bit for bit, a smaller cluster the same map
 * with its sums in another order. */
mbt_status mbt_batch_track_resident(mbt_batch *b, int64_t nturns, void *stream);
void mbt_batch_destroy(mbt_batch *b);

/* ------------------------------------------------------------------------
 * Serving: instability-scan requests tracked with continuous batching.
 * A server thread owns the device work.  Requests wait in a FIFO queue and are
 * admitted in order while at most max_active requests are active and their
 * estimated device memory stays within hbm_budget_bytes (the first request is
 * always admitted).  All active requests advance together through the batched
 * kernels, turns_per_step turns between admission points (fewer when a
 * request is about to finish); finished requests are retired at once, which
 * frees their memory for the queue.  A request's result does not depend on
 * what it was batched with: it equals the same request tracked alone.
 * ------------------------------------------------------------------------ */
typedef struct mbt_server mbt_server;

typedef struct {
    size_t hbm_budget_bytes;  /* device memory admitted requests may hold (estimate), > 0 */
    int max_active;           /* requests tracked together, >= 1                          */
    int turns_per_step;       /* turns between admission points, >= 1                     */
    int lanes;                /* active requests in that many groups on streams of their
                                 own (mbt_batch_set_lanes); 0 or 1: one plan, up to 8      */
} mbt_server_config;

/* One request: a run as for mbt_create / mbt_add_resonator / mbt_set_grid /
 * mbt_set_fill, tracked for `turns` turns from a matched Gaussian start.  All
 * arrays are copied by mbt_server_submit. */
typedef struct {
    mbt_ring ring;
    int precision, flags;
    uint64_t seed;
    int nres;
    const double *Rs_ohm, *fr_Hz, *Q;
    const int32_t *range;
    int nbins;
    double half_width_sigmas;
    int nb;
    const int32_t *bucket;
    const double *current_A;
    const int64_t *n_mp;
    int64_t turns;
} mbt_request;

enum { MBT_REQ_QUEUED = 0, MBT_REQ_RUNNING = 1, MBT_REQ_DONE = 2, MBT_REQ_FAILED = 3 };

typedef struct {
    int state;                 /* MBT_REQ_*                                              */
    int64_t turns_done;
    double t_submit, t_start, t_finish;   /* seconds since the server started (host clock) */
    int64_t device_bytes;      /* device memory the request held while active            */
    char error[128];
} mbt_request_status;

typedef struct {
    int64_t submitted, completed, failed, queued, active, max_active_seen, steps;
    int64_t used_bytes, max_bytes_seen;
    double busy_seconds;       /* time spent in tracking steps                            */
    double mp_turns;           /* macro-particle-turns tracked                            */
    double now;                /* seconds since the server started                        */
} mbt_server_stats;

/* Start a server on the calling thread's current device.  MBT_ERR_ARG for a
 * NULL pointer, max_active or turns_per_step below 1, a zero budget or lanes
 * outside 0..8. */
mbt_status mbt_server_create(const mbt_server_config *cfg, mbt_server **out);
/* Queue a request (non-blocking); *id identifies it.  MBT_ERR_BUDGET if its
 * estimated memory alone exceeds the budget, MBT_ERR_ARG on a malformed request. */
mbt_status mbt_server_submit(mbt_server *s, const mbt_request *req, int64_t *id);
/* State and timestamps of a request; once it is done, final_moments[nb][6]
 * (the last turn's moments, as mbt_read_moments) and history[turns][2] (per
 * turn, the rms over bunches of <tau> and of <delta>) are copied if non-NULL. */
mbt_status mbt_server_poll(mbt_server *s, int64_t id, mbt_request_status *status, double *final_moments,
                           double *history);
/* Block until the request is done (MBT_OK), failed (MBT_ERR_CUDA) or timeout_s
 * passed (MBT_ERR_TIMEOUT). */
mbt_status mbt_server_wait(mbt_server *s, int64_t id, double timeout_s);
mbt_status mbt_server_get_stats(mbt_server *s, mbt_server_stats *out);
/* Stop the server thread and free every request's device memory. */
void mbt_server_destroy(mbt_server *s);

#ifdef __cplusplus
}
#endif
#endif /* MBT_H */
