// Internal layout shared by the host engine and the kernels of libmbt.
//
// Device state of one run (a fill of bunches on one ring), the per-batch work
// lists, and the launch entry points of the kernels.  Everything here is
// plain data: pointers into device memory plus constants derived on the host.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace mbt {

constexpr int kMaxRes = 8;           // resonators per run
constexpr int kMaxLong = 4;          // resonators with the long-range bit
constexpr int kMaxHarm = 2;          // active harmonic RF cavities
constexpr int kBunchTile = 32;       // bunches per post-kernel tile (one lane per bunch)
constexpr int kMaxBunches = 1024;    // one warp scans the tile aggregates
constexpr int kPushThreads = 256;
constexpr int kMixedQuadsPerThread = 8;                                    // 4 particles per quad
constexpr int kMixedTile = kPushThreads * 4 * kMixedQuadsPerThread;        // 8192 particles
constexpr int kF64QuadsPerThread = 2;                                      // 4 particles per quad
constexpr int kF64Tile = kPushThreads * 4 * kF64QuadsPerThread;            // 2048 particles
// per push tile: sums of u, u^2, v, v^2 (u = tau - tau_ref, v = delta - delta_ref,
// the refs being the tile's first particle before the push), n_out, tau_ref,
// x, x^2, x', x'^2, delta_ref, particle count
constexpr int kPartials = 12;
constexpr int kTRecord = 4;          // transverse record: <x>, rms x, <x'>, rms x'
constexpr int kTransRows = 32;       // transverse short-range rows per post job (kMixed)
constexpr int kRecord = 6;           // <tau>, rms tau, <delta>, rms delta, n_in, n_out
constexpr int kPostThreads = 256;
constexpr int kSpillCells = 32;      // per-lane extra cells behind a push histogram: outside particles
                                     // deposit there (never read) instead of taking a branch
constexpr int kF64RowChunk = 32;     // FP64 Toeplitz rows per post job

enum Precision { kF64 = 0, kMixed = 1 };
enum Flags { kNoSR = 1, kNoQE = 2, kKickNGP = 4 };
enum JobType { kJobWake = 0, kJobTile = 1, kJobTrans = 2, kJobMoments = 3 };
// PostJob::sub of a kMixed wake job over both M-tiles of a 256-cell mesh
// (plans whose post jobs fill several waves); otherwise sub is the M-tile
constexpr int kWakeBoth = 2;
// kErrCount: a cell count outside [0, 2^24) reached the tensor-core wake,
// which splits each count into three exact 8-bit planes.  kErrDipole: the
// mixed transverse push met an x outside its dipole deposit's fixed-point
// range (RunDev::f_dip_range)
enum DeviceError { kErrNone = 0, kErrTimeout = 1, kErrTmem = 2, kErrCount = 3, kErrDipole = 4 };

// One run's device state and constants.
struct RunDev {
  // particle state: tau (float for kMixed, double for kF64), delta (double)
  void *tau;
  double *delta;
  int32_t *hist;        // [2][nb][nbins]; turn parity selects the buffer
  void *vsr;            // [nb][nbins] short-range voltage for the next kick (float / double)
  double2 *pq;          // [nlong][nb][2]: P_m, Q_m with Phi_m = P_m y_tile + Q_m
  double2 *y;           // [nlong][ntile_b]: value entering each bunch tile
  double2 *agg;         // [nlong][ntile_b][2]: tile aggregate affine maps (A, B)
  double2 *carry;       // [nlong]: value after the last bunch of the previous turn
  double *rec;          // [cap][nb][kRecord]
  long long *turn;      // turns completed (device counter)
  const double *q_mp;   // [nb] macro-particle charge [C]
  const double2 *step;  // [nlong][nb] a_m = e^{s dt_m}
  const double2 *emis;  // [nlong][nbins] e^{-s tau_k} (double)
  const float2 *emis_f; // [nlong][nbins] same in float
  const void *toep;     // kMixed: bf16 operand images [nbins/128][128 x 2 nbins]; kF64: double lag table [nbins]
  int nb, nbins, nlong, ntile_b;
  int cap, flags, precision, bunch_base;   // bunch_base: index of bunch 0 in the plan's bunch list
  uint32_t key0, key1;
  // ring constants
  double inv_E0, V_over_E0, sin_phi_s, cos_phi_s, U0_over_E0, omega_rf, phi_s;
  double one_minus_D, qe_amp, aT0, H, invDelta, Delta;
  double sigma_tau0, sigma_E;   // matched start
  double2 lr_s[kMaxLong];   // s = -a + i wb
  double2 lr_c[kMaxLong];   // c = 2 a Rs (1 + i a / wb)
  // FP32 copies for the mixed-precision push (GB300 issues FP64 and its
  // conversions at ~1.6 lanes per clock per SM: none of them per thread)
  // (f_HinvD = H/Delta - 1/2: cells from the cell centres; f_la = decay rate x log2(e))
  // (f_rfA = (V/E0)(1 - D) sin phi_s, f_rfB = (V/E0)(1 - D) cos phi_s, f_w = omega_rf)
  float f_invD, f_HinvD, f_nbins, f_invE0, f_rfA, f_rfB, f_w, f_omD, f_qe, f_aT0;
  float f_la[kMaxLong], f_lw[kMaxLong];
  const float *q_mp_f;      // [nb] macro-particle charge (float)
  const double *inv_n;      // [nb] 1 / n_mp
  const float *lag_f;       // [nbins] summed short-range wake per lag, FP32 (resident mode)
  // active harmonic cavities: (V_h/E0) sin(phi_h - n omega_rf tau) each
  int nharm;
  double harm_VoE0[kMaxHarm], harm_phi[kMaxHarm], harm_nw[kMaxHarm];
  float4 f_harm[kMaxHarm];  // (2 V_h/E0 (1 - D), cos phi_h, sin phi_h, n omega_rf / 2), mixed path
  // long-range entries: 0 = longitudinal (Re(Phi e^{s tau}) kicks delta),
  // 1 = transverse (emission from the dipole sums, Im(Phi e^{s tau}) kicks x')
  int lr_plane[kMaxLong];
  // transverse plane (one per run): x [m], x' (float for kMixed, double for kF64)
  int trans;
  void *x, *xp;
  void *dip;                // [2][nb][nbins] sum of x over each cell's particles; turn parity selects
                            // (kF64: double; kMixed: int64 in units of dip_unit, summed exactly, so
                            // that the sums do not depend on the order of the tiles' atomics)
  void *vt;                 // [nb][nbins] transverse short-range voltage [V] for the next kick
  double *trec;             // [cap][nb][kTRecord]
  const double *tlag;       // [nbins] transverse wake per lag [V/(C m)]
  const float *tlag_f;
  double t_beta, t_alpha, t_gamma, t_mu0, t_xi, t_nx, t_nxp;   // t_nx = sqrt(beta emit Dx), t_nxp = sqrt(gamma emit Dx)
  double t_emit;
  // long-range transverse resistive wall on bunch centroids
  int rw_nh;                // turns of history (0: none)
  const double *rw_tab;     // [(rw_nh + 1) h] W(D T_rf) by bucket distance D (0 at D = 0)
  const float *rw_tab_f;
  double *rw_cent;          // [rw_nh + 1][nb] charge x centroid, by turn
  const int32_t *bucket;    // [nb]
  int h_rf;                 // harmonic number
  // float copies: 2 pi frac(nu), 2 pi nu xi, beta, alpha, gamma, nx, nxp, 1/(1 - D)
  float f_tmu0, f_tmu0xi, f_tbeta, f_talpha, f_tgamma, f_tnx, f_tnxp, f_inv_omD, f_U0oE0;
  // fixed-point dipole deposit of the mixed push: unit u = 2^(e - 20) m with
  // 2^e >= sqrt(beta emit) (e >= -16), 1/u, and the accepted |x| < 2^30 u
  double dip_unit;
  float f_dip_unit, f_dip_inv, f_dip_range;
};



struct BunchDev {
  int run, m;
  long long off;        // first particle of the bunch in the run's arrays (multiple of 4)
  long long n;          // macro-particles
  int tile0, ntiles;    // push tiles of this bunch in the plan
};

struct TileDev {
  int bunch, run, m, count;   // count <= tile size
  long long start;            // first particle of the tile within its bunch (multiple of 4)
};

// Streaming push (kMixed, no transverse plane): run constants and tile
// descriptors laid out for bulk copies into shared memory, so that a
// persistent CTA moves from tile to tile without a dependent global load.
struct alignas(16) StreamRun {
  float invD, HinvD, fnb, invE0, rfA, rfB, w, qe, aT0, pad0;   // invE0, rfA, rfB carry (1 - D)
  int nbins, nlong, nharm, flags;
  uint32_t key0, key1;
  double omD;                   // 1 - D
  float la[kMaxLong], lw[kMaxLong];
  float4 harm[kMaxHarm];        // as RunDev::f_harm
};
static_assert(sizeof(StreamRun) % 16 == 0, "bulk-copy size");

struct alignas(16) StreamTile {
  float *tau;                   // first particle of the tile
  double *del;
  int32_t *hist;                // bunch's row in histogram buffer 0 (buffer 1 at + hist_par)
  const float *vrow;            // bunch's row of the short-range voltage
  const long long *turn;        // run's turn counter (a 16-byte block)
  const StreamRun *rc;
  const double2 *pq;            // P_m of resonator 0 (Q_m follows); resonator r at + r * pq_stride
  const double2 *y;             // value entering the bunch's post tile, resonator 0; r at + r * y_stride
  long long start;              // first particle of the tile within its bunch
  long long hist_par;
  int count, index, m, nlong;   // index: the tile's partial-sum slot
  int pq_stride, y_stride, nbins, pad0;
  int pad1[4];
};
static_assert(sizeof(StreamTile) == 128, "bulk-copy size");

struct PostJob {
  int run, type, bt, sub;     // kJobWake: sub = M-tile (kMixed) or (bunch, row chunk) (kF64); kJobTrans: row chunk
};

// A batch of runs tracked by the same launches.
struct Plan {
  RunDev *runs;
  BunchDev *bunches;
  TileDev *tiles;
  PostJob *jobs;
  double *partial;            // [ntiles][kPartials]
  unsigned int *done;         // post-kernel completion counter (last-block pattern)
  int *error;                 // device error word (DeviceError)
  int nruns, nbunches, ntiles, njobs;
  int max_nbins;              // largest mesh of the plan's runs (shared-memory sizing)
  int max_nlong;              // most long-range resonators of any run of the plan
  int max_nharm;              // most harmonic cavities of any run of the plan
  int max_trans;              // 1 if any run of the plan has a transverse plane
  unsigned long long *trace;  // null, or [njobs][3] post-kernel CTA timestamps (start, job done, exit) [ns]
  StreamTile *stiles;         // [ntiles] the tiles for the streaming push
  StreamRun *sruns;           // [nruns]
  int *stream_first;          // [stream_ctas + 1]: CTA b of the streaming push takes tiles stream_first[b] .. [b + 1] - 1
  int stream_ctas;            // 0 if the plan is not split for the streaming push
  int fold_moments;           // kMixed: no moments jobs; each tile job sums its bunches' moments first
  int push_small_ctas;        // per-tile push (no transverse plane) in 128-thread CTAs (plans of many waves)
  // kMixed plans of many post waves: the first post_split jobs (the wake
  // jobs) run in a kernel of their own on the launching stream, the others in
  // a kernel with a small shared-memory footprint on `side` (forked at
  // ev_fork after the push, joined at ev_join); 0: one post kernel
  int post_split;
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
};

// Cluster-resident tracking of one run: one thread-block cluster per bunch,
// the bunch's particles held in the cluster's shared memory for all turns of
// a launch.
#ifndef MBT_RESIDENT_THREADS
#define MBT_RESIDENT_THREADS 512
#endif
constexpr int kResidentThreads = MBT_RESIDENT_THREADS;
constexpr int kResidentMaxBunches = 32;   // one warp scans the fill
constexpr unsigned long long kResidentWaitNs = 2000000000ull;   // grid-barrier wait limit (default)
struct ResidentArgs {
  Plan plan;              // the run's own plan (runs[0], bunches)
  double2 *E;             // [2][nlong][nb] emissions, double-buffered by turn parity
  unsigned int *gbar;     // grid barrier counter (zeroed before each launch)
  int cluster;            // CTAs per cluster
  int per;                // particles per CTA slice (multiple of 4)
  int nturns;
  int grid_sync;          // 1 if clusters must meet every turn (long-range coupling of several bunches)
  unsigned long long wait_ns;    // limit of the grid-barrier wait
  unsigned int extra_arrivals;   // arrivals the barrier waits for beyond the bunches (0; 1 in the
                                 // failure-detection test, a count nothing reaches)
};
size_t resident_smem_bytes(int per, int nbins);
cudaError_t launch_resident(const ResidentArgs &a, int nlong, int nharm, int nb, cudaStream_t s);
cudaError_t resident_max_clusters(int cluster, size_t smem, int *max_clusters);

// Kernel launchers (one translation unit each).
// pdl: launch with programmatic stream serialisation (the kernel's prologue
// may overlap the previous kernel of the stream, which must be one of ours)
cudaError_t launch_push(const Plan &p, int precision, cudaStream_t s, bool pdl);
cudaError_t launch_post(const Plan &p, int precision, cudaStream_t s, bool pdl);
cudaError_t launch_init(const Plan &p, int precision, cudaStream_t s);
// tau, delta of every bunch from device-accessible (page-locked) host arrays;
// hoff: device array, first particle of each bunch in the host arrays
cudaError_t launch_load_host(const Plan &p, int precision, const double *tau_h, const double *del_h,
                             const long long *hoff, cudaStream_t s);
cudaError_t launch_load_host_f32(const Plan &p, int precision, const float *tau_h, const double *del_h,
                                 const long long *hoff, cudaStream_t s);

size_t post_smem_bytes(int precision, int max_nbins);
cudaError_t configure_kernels();
// Allocation-free tensor-core wake of one run (scratch: a static device array
// in k_post.cu).  proto supplies the constants; the images, charges and
// pointers are placed into the array by the call.  Host buffers are consumed
// before the call returns.
cudaError_t wake_noalloc_launch(const RunDev &proto, const void *img, size_t img_bytes, const float *q_f, int nb,
                                int nbins, const int32_t *hist, float *V, cudaStream_t s, int *device_error_out);
cudaError_t configure_push_kernels();
cudaError_t push_resident_slots(int *slots);     // streaming-push CTAs resident at once on this device
cudaError_t push_tile_resident_slots(bool trans, int *slots);   // the same for a per-tile push (256 cells)
// Whether a mixed-precision plan of these runs (their particle counts and
// bunch counts) uses the streaming push: no transverse plane, and every run
// gives each SM a share of several stages in bunches of at least two stages.
bool plan_streams(const std::vector<int64_t> &n, const std::vector<int> &nb, bool any_trans, int sms);

}  // namespace mbt
