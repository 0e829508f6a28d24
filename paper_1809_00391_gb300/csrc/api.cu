// Host engine and C ABI of libmbt (declarations and conventions in mbt.h).
//
// A context holds one run: its ring, wake model, mesh and fill, the device
// buffers of its state, and a Plan (work lists) for tracking it alone.  A
// batch holds a Plan over several contexts.  Derived ring quantities and the
// wake tables are computed here in double precision from the paper's
// definitions (Sec. 2.2 Eqs. 1, 2, 5; Sec. 2.3 Eq. 6).
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/mbt.h"
#include "mbt_internal.h"

using namespace mbt;
using cplx = std::complex<double>;

namespace {

const double kPi = 3.14159265358979323846264338327950288;

struct Resonator {
  double Rs, fr, Q;
  int range;
};

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

// Plan storage on the device plus its host mirror.
struct PlanStore {
  Plan plan{};
  std::vector<RunDev> runs;
  std::vector<BunchDev> bunches;
  std::vector<TileDev> tiles;
  std::vector<PostJob> jobs;
  std::vector<void *> allocs;
  size_t bytes = 0;
  int precision = 0;
  ~PlanStore() { release(); }
  void release() {
    if (plan.side) cudaStreamDestroy(plan.side);
    if (plan.ev_fork) cudaEventDestroy(plan.ev_fork);
    if (plan.ev_join) cudaEventDestroy(plan.ev_join);
    for (void *a : allocs) cudaFree(a);
    allocs.clear();
    bytes = 0;
    plan = Plan{};
  }
};

uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return 0x7FC0;
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_to_f32(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Tensor-core operand images of the short-range Toeplitz matrix T[j][k] =
// lag[j - k] (j >= k, else 0), per M-tile mt: rows [128 mt, 128 mt + 128)
// need only columns k < Kmt = min(nbins, 128 (mt + 1)), so the image holds
// 128 rows x [T_hi | T_lo] (2 Kmt columns; T_hi = bf16(T), T_lo =
// bf16(T - T_hi)) of BF16 in K-major 8x8 core matrices, element (row, kk) at
// byte ((kk / 8) * 16 + row / 8) * 128 + (row % 8) * 16 + (kk % 8) * 2; the
// images of the M-tiles follow each other (512 Kmt bytes each).  img must
// hold 512 * sum_mt Kmt bytes; returns that size.  The one layout that the
// wake kernel reads (wake_img_offset), for tracking and for the
// allocation-free wake alike.
size_t pack_toeplitz_images(const double *lag, int nbins, uint16_t *img) {
  size_t base = 0;
  for (int mt = 0; mt < nbins / 128; ++mt) {
    const int kmt = std::min(nbins, 128 * (mt + 1));
    for (int row = 0; row < 128; ++row)
      for (int k = 0; k < kmt; ++k) {
        const int j = mt * 128 + row;
        const double T = j >= k ? lag[j - k] : 0.0;
        const uint16_t hi = f32_to_bf16_rne((float)T);
        const uint16_t lo = f32_to_bf16_rne((float)(T - (double)bf16_to_f32(hi)));
        for (int half = 0; half < 2; ++half) {
          const int kk = k + half * kmt;
          const size_t byte = base + ((size_t)(kk / 8) * 16 + row / 8) * 128 + (row % 8) * 16 + (kk % 8) * 2;
          img[byte / 2] = half ? lo : hi;
        }
      }
    base += (size_t)512 * kmt;
  }
  return base;
}

}  // namespace

struct mbt_ctx {
  mbt_ring ring{};
  int precision = 0, flags = 0;
  uint64_t seed = 0;
  std::vector<Resonator> res;
  int nbins = 256;
  double half_width_sigmas = 5.0;
  int64_t cap = 4096;
  // derived
  double T_rf = 0, omega_rf = 0, phi_s = 0, sin_phi_s = 0, cos_phi_s = 0, nu_s = 0, sigma_tau0 = 0, D = 0, qe = 0;
  double H = 0, Delta = 0, invDelta = 0;
  // fill
  bool filled = false;
  int nb = 0, nlong = 0, ntile_b = 0;
  std::vector<int32_t> bucket;
  std::vector<double> current;
  std::vector<int64_t> nmp, off;
  int64_t n_particles = 0, n_alloc = 0;
  std::vector<int> long_idx;   // long-range entries: index into res (plane 0) or tres (plane 1)
  std::vector<int> long_plane;
  // transverse plane
  bool trans = false;
  double t_beta = 0, t_alpha = 0, t_tune = 0, t_xi = 0, t_emit = 0;
  std::vector<Resonator> tres;
  double rw_A = 0.0;   // long-range transverse resistive wall: W = rw_A / sqrt(t)
  int rw_nh = 0;
  double *d_rwtab = nullptr, *d_rwcent = nullptr;
  float *d_rwtab_f = nullptr;
  int32_t *d_bucket = nullptr;
  void *d_x = nullptr, *d_xp = nullptr, *d_dip = nullptr, *d_vt = nullptr;
  double *d_trec = nullptr, *d_tlag = nullptr;
  float *d_tlag_f = nullptr;
  // device state
  std::vector<DevBuf> bufs;
  void *d_tau = nullptr;
  double *d_delta = nullptr;
  int32_t *d_hist = nullptr;
  void *d_vsr = nullptr;
  double2 *d_pq = nullptr, *d_y = nullptr, *d_agg = nullptr, *d_carry = nullptr;
  double *d_rec = nullptr;
  long long *d_turn = nullptr;
  double *d_q = nullptr;
  double2 *d_step = nullptr, *d_emis = nullptr;
  float *d_qf = nullptr;
  double *d_inv_n = nullptr;
  long long *d_hoff = nullptr;   // [nb] first particle of each bunch in back-to-back host arrays
  float *d_lagf = nullptr;
  // cluster-resident mode (allocated on first use)
  double2 *d_resE = nullptr;
  unsigned int *d_gbar = nullptr;
  float2 *d_emis_f = nullptr;
  void *d_toep = nullptr;
  size_t device_bytes = 0;
  // tabulated short-range wakes (t, W) and resistive-wall pipes (b, sigma, L)
  std::vector<std::vector<double>> wt_t, wt_w;
  std::vector<std::array<double, 3>> rwalls;
  // active harmonic cavities (n, V, phi)
  std::vector<std::array<double, 3>> harm;
  RunDev rundev{};
  PlanStore own;
  int tile = kMixedTile;       // particles per push CTA (mixed precision)
  // graph replay
  int graph_turns = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  // timing
  bool timing = false;
  // failure-detection test hook (mbt_set_wait_test): resident grid-barrier
  // wait limit (0: the default) and an unreachable barrier count
  int64_t test_wait_ns = 0;
  int test_unreachable = 0;
  double push_ms = 0, post_ms = 0;
  int64_t timed_launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  // post-kernel trace
  unsigned long long *d_trace = nullptr;
  // pinned host staging for particle copies
  void *h_stage = nullptr;
  size_t h_stage_bytes = 0;
  std::string err;
};

// One lane of a batch: a group of its members with a plan of their own,
// tracked on a stream of its own beside the other lanes.
constexpr int kMaxLanes = 8;
struct BatchLane {
  std::vector<int> members;   // indices into mbt_batch::ctx, increasing
  PlanStore store;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  ~BatchLane() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (stream) cudaStreamDestroy(stream);
    if (done) cudaEventDestroy(done);
  }
};

struct mbt_batch {
  std::vector<mbt_ctx *> ctx;
  PlanStore store;
  int precision = 0;
  int tile = kMixedTile;
  int graph_turns = 0;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  // concurrent resident tracking: one stream per member, fork / join events
  std::vector<cudaStream_t> res_streams;
  std::vector<cudaEvent_t> res_events;   // [0] fork, [1 + i] member i done
  // lanes (mbt_batch_set_lanes): empty = the whole batch in one plan
  std::vector<std::unique_ptr<BatchLane>> lanes;
  int nlanes = 1;
  cudaEvent_t lane_fork = nullptr;
};

namespace {

mbt_status fail(mbt_ctx *c, mbt_status s, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

mbt_status cuda_fail(mbt_ctx *c, cudaError_t e, const char *what) {
  return fail(c, MBT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <class T>
mbt_status dalloc(mbt_ctx *c, T **ptr, size_t bytes) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) return fail(c, MBT_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  cudaMemset(p, 0, bytes ? bytes : 16);
  c->bufs.push_back({p, bytes});
  c->device_bytes += bytes;
  *ptr = static_cast<T *>(p);
  return MBT_OK;
}

void free_device(mbt_ctx *c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  c->capture_stream = nullptr;
  for (auto &b : c->bufs) cudaFree(b.p);
  c->bufs.clear();
  c->device_bytes = 0;
  c->own.release();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_bytes = 0;
  if (c->d_trace) cudaFree(c->d_trace);
  c->d_trace = nullptr;
}

// Pinned staging buffer of at least `bytes` (grown on demand).
void *stage(mbt_ctx *c, size_t bytes) {
  if (c->h_stage_bytes >= bytes) return c->h_stage;
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_bytes = 0;
  if (cudaMallocHost(&c->h_stage, bytes) != cudaSuccess) return nullptr;
  c->h_stage_bytes = bytes;
  return c->h_stage;
}

// Ring-derived quantities (readings listed in mbt.h).
void derive(mbt_ctx *c) {
  const mbt_ring &r = c->ring;
  const bool sr = !(c->flags & MBT_NO_SR);
  const double U0 = sr ? r.U0_eV : 0.0;
  c->T_rf = r.T0_s / (double)r.h;
  c->omega_rf = 2.0 * kPi * (double)r.h / r.T0_s;
  double Uh = 0.0;   // harmonic cavities' voltage at the synchronous particle
  for (auto &hc : c->harm) Uh += hc[1] * std::sin(hc[2]);
  c->sin_phi_s = (U0 - Uh) / r.V_rf_V;
  c->phi_s = std::asin(c->sin_phi_s);
  if (r.alpha_c < 0.0) c->phi_s = kPi - c->phi_s;
  c->cos_phi_s = std::cos(c->phi_s);
  c->nu_s = std::sqrt(r.alpha_c * (double)r.h * r.V_rf_V * c->cos_phi_s / (2.0 * kPi * r.E0_eV));
  c->sigma_tau0 = std::fabs(r.alpha_c) * r.sigma_delta * r.T0_s / (2.0 * kPi * c->nu_s);
  c->D = sr ? 2.0 * r.T0_s / r.tau_z_s : 0.0;
  c->qe = (sr && !(c->flags & MBT_NO_QE)) ? r.sigma_delta * std::sqrt(2.0 * c->D) : 0.0;
  c->H = c->half_width_sigmas * c->sigma_tau0;
  c->Delta = 2.0 * c->H / (double)c->nbins;
  c->invDelta = 1.0 / c->Delta;
}

void res_consts(const Resonator &q, double &a, double &wb) {
  const double wr = 2.0 * kPi * q.fr;
  a = wr / (2.0 * q.Q);
  wb = std::sqrt(wr * wr - a * a);
}

// Resonator wake [V/C]; half of W(0+) at t == 0.
double wake(const Resonator &q, double t) {
  double a, wb;
  res_consts(q, a, wb);
  if (t < 0.0) return 0.0;
  if (t == 0.0) return a * q.Rs;
  return 2.0 * a * q.Rs * std::exp(-a * t) * (std::cos(wb * t) - (a / wb) * std::sin(wb * t));
}

// Transverse resonator wake [V/(C m)]: (wr^2 Rs / (Q wb)) e^{-a t} sin(wb t)
// for t > 0, zero at and before t = 0 (Rs in Ohm/m).
double twake(const Resonator &q, double t) {
  if (!(t > 0.0)) return 0.0;
  double a, wb;
  res_consts(q, a, wb);
  const double wr = 2.0 * kPi * q.fr;
  return wr * wr * q.Rs / (q.Q * wb) * std::exp(-a * t) * std::sin(wb * t);
}

// Integral over [lo, hi] of the piecewise linear wake through (t[i], w[i]),
// zero beyond the last sample.
double table_integral(const std::vector<double> &t, const std::vector<double> &w, double lo, double hi) {
  double acc = 0.0;
  for (size_t i = 0; i + 1 < t.size(); ++i) {
    const double a = std::max(t[i], lo), b = std::min(t[i + 1], hi);
    if (!(b > a)) continue;
    const double k = (w[i + 1] - w[i]) / (t[i + 1] - t[i]);
    acc += 0.5 * ((w[i] + k * (a - t[i])) + (w[i] + k * (b - t[i]))) * (b - a);
  }
  return acc;
}

// Adaptive Simpson quadrature of f over [a, b] to absolute tolerance eps.
template <class F>
double simpson(F &f, double a, double b, double fa, double fm, double fb, double whole, double eps, int depth) {
  const double m = 0.5 * (a + b), lm = 0.5 * (a + m), rm = 0.5 * (m + b);
  const double flm = f(lm), frm = f(rm);
  const double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm), right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
  if (depth <= 0 || std::fabs(left + right - whole) <= 15.0 * eps) return left + right + (left + right - whole) / 15.0;
  return simpson(f, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) + simpson(f, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

// Integral over t in [ta, tb] (s) of the resistive-wall wake of a round pipe
// (radius b, conductivity sigma, length L) in the short-range form
// W = (4 Z0 c L / (pi b^2)) [e^{-u} cos(sqrt3 u) / 3 - (sqrt2 / pi) int x^2 e^{-x^2 u} / (x^6 + 8) dx],
// u = c t / s0, s0 = (2 b^2 / (Z0 sigma))^(1/3).  In u the first term has the
// antiderivative e^{-u} (sqrt3 sin(sqrt3 u) - cos(sqrt3 u)) / 4; the second,
// integrated over u first, is int_0^inf (e^{-x^2 ua} - e^{-x^2 ub}) / (x^6 + 8) dx
// (adaptive Simpson on [0, 40] split at x = 2^-10, 2^-9, ... so that the
// narrow peak near x = 0 of a large u is resolved; the rest beyond 40 is
// below 2e-9 of the lag-0 value).
double rw_integral(double b, double sigma, double L, double ta, double tb) {
  constexpr double kZ0 = 376.730313668, kC = 299792458.0;
  const double s0 = std::cbrt(2.0 * b * b / (kZ0 * sigma));
  const double ua = kC * ta / s0, ub = kC * tb / s0;
  const double r3 = std::sqrt(3.0);
  auto P = [&](double u) { return std::exp(-u) * (r3 * std::sin(r3 * u) - std::cos(r3 * u)) / 4.0; };
  auto g = [&](double x) {
    const double x2 = x * x;
    return (std::exp(-x2 * ua) - std::exp(-x2 * ub)) / (x2 * x2 * x2 + 8.0);
  };
  double G = 0.0, x0 = 0.0, x1 = std::ldexp(1.0, -10);
  while (x0 < 40.0) {
    const double fa = g(x0), fm = g(0.5 * (x0 + x1)), fb = g(x1);
    G += simpson(g, x0, x1, fa, fm, fb, (x1 - x0) / 6.0 * (fa + 4.0 * fm + fb), 1e-17, 40);
    x0 = x1;
    x1 = std::min(40.0, 2.0 * x1);
  }
  return 4.0 * kZ0 * L * s0 / (kPi * b * b) * ((P(ub) - P(ua)) / 3.0 - std::sqrt(2.0) / kPi * G);
}

// Streaming-push work split (host only).  bunch_run: the run of each bunch,
// non-decreasing; bunch_n: its macro-particles (>= 1); G: CTAs.  Each run's
// particle sequence (its bunches in order, each padded to a multiple of 4) is
// cut into G shares at multiples of 4, share g = [4 floor(P' g / G),
// 4 floor(P' (g + 1) / G)) with P' = P / 4 (the last share ends at P), and
// each share into tiles at bunch boundaries and at most 2^28 particles.  The
// shares are consecutive ranges of the bunch sequence, so the tiles come out
// both in bunch order and in CTA order within each run; a run's tiles do not
// depend on the other runs.
struct SplitTile {
  int bunch;
  int64_t start;   // first particle within the bunch (a multiple of 4)
  int count;
  int cta;
};

std::vector<SplitTile> stream_split(const std::vector<int> &bunch_run, const std::vector<int64_t> &bunch_n, int G) {
  constexpr int64_t kMaxCount = int64_t(1) << 28;
  std::vector<SplitTile> out;
  const size_t nbun = bunch_n.size();
  auto padded = [&](size_t i) { return (bunch_n[i] + 3) / 4 * 4; };
  size_t b0 = 0;
  while (b0 < nbun) {
    size_t b1 = b0;
    int64_t P = 0;
    while (b1 < nbun && bunch_run[b1] == bunch_run[b0]) P += padded(b1++);
    size_t m = b0;
    int64_t B = 0;   // padded start of bunch m within the run
    for (int g = 0; g < G; ++g) {
      const int64_t a = (P / 4) * g / G * 4, e = g + 1 == G ? P : (P / 4) * (g + 1) / G * 4;
      while (m < b1 && B + padded(m) <= a) B += padded(m++);
      int64_t Bm = B;
      for (size_t mm = m; mm < b1 && Bm < e; ++mm) {
        const int64_t pm = padded(mm);
        const int64_t s0 = std::max(a, Bm) - Bm, s1 = std::min<int64_t>(std::min(e, Bm + pm) - Bm, bunch_n[mm]);
        for (int64_t s = s0; s < s1; s += kMaxCount)
          out.push_back(SplitTile{(int)mm, s, (int)std::min<int64_t>(kMaxCount, s1 - s), g});
        Bm += pm;
      }
    }
    b0 = b1;
  }
  return out;
}

// Upload a plan built in st's host vectors.
mbt_status upload_plan(mbt_ctx *c, PlanStore &st) {
  st.release();
  auto up = [&](auto &vec, auto **dst) -> bool {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    void *p = nullptr;
    size_t bytes = std::max<size_t>(vec.size() * sizeof(T), 16);
    if (cudaMalloc(&p, bytes) != cudaSuccess) return false;
    st.allocs.push_back(p);
    st.bytes += bytes;
    if (!vec.empty() && cudaMemcpy(p, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
    *dst = static_cast<T *>(p);
    return true;
  };
  // Streaming push (mixed precision, no transverse plane, runs large enough:
  // plan_streams): each run's
  // particle sequence (its bunches in order, each padded to 4 particles) is
  // cut into one equal share per SM at multiples of 4, each share into tiles
  // at bunch boundaries, and CTA g takes share g of every run.  A run's tiles
  // (and so the order of its moment sums) are the same alone and in a batch.
  // p.tiles stays in bunch order (the post kernel sums each bunch's partials
  // over its consecutive tiles); p.stiles lists each CTA's tiles together.
  bool mixed = !st.runs.empty(), any_trans = false;
  std::vector<int64_t> run_n(st.runs.size(), 0);
  std::vector<int> run_nb(st.runs.size(), 0);
  for (const RunDev &r : st.runs) {
    mixed = mixed && r.precision == kMixed;
    any_trans = any_trans || r.trans;
  }
  for (const BunchDev &b : st.bunches) {
    run_n[(size_t)b.run] += b.n;
    ++run_nb[(size_t)b.run];
  }
  int slots = 0;
  if (mixed && (push_resident_slots(&slots) != cudaSuccess || slots <= 0)) {
    cudaGetLastError();
    return fail(c, MBT_ERR_CUDA, "streaming push occupancy");
  }
  const bool streaming = mixed && plan_streams(run_n, run_nb, any_trans, slots);
  std::vector<int> first, owner;
  std::vector<int> sorder;   // tile indices in CTA order
  if (streaming) {
    const int G = slots;
    std::vector<int> brun(st.bunches.size());
    std::vector<int64_t> bn(st.bunches.size());
    for (size_t i = 0; i < st.bunches.size(); ++i) {
      brun[i] = st.bunches[i].run;
      bn[i] = st.bunches[i].n;
    }
    std::vector<TileDev> tiles;
    for (const SplitTile &sp : stream_split(brun, bn, G)) {
      const BunchDev &bd = st.bunches[(size_t)sp.bunch];
      TileDev t{};
      t.bunch = sp.bunch;
      t.run = bd.run;
      t.m = bd.m;
      t.start = sp.start;
      t.count = sp.count;
      tiles.push_back(t);
      owner.push_back(sp.cta);
    }
    st.tiles.swap(tiles);
    for (BunchDev &bd : st.bunches) bd.tile0 = bd.ntiles = 0;
    for (size_t i = 0; i < st.tiles.size(); ++i) {
      BunchDev &bd = st.bunches[(size_t)st.tiles[i].bunch];
      if (bd.ntiles == 0) bd.tile0 = (int)i;
      ++bd.ntiles;
    }
    first.assign((size_t)G + 1, 0);
    for (int g : owner) ++first[(size_t)g + 1];
    for (int g = 0; g < G; ++g) first[(size_t)g + 1] += first[(size_t)g];
    sorder.assign(st.tiles.size(), 0);
    std::vector<int> fill(first.begin(), first.end() - 1);
    for (size_t i = 0; i < st.tiles.size(); ++i) sorder[(size_t)fill[(size_t)owner[i]]++] = (int)i;
  }
  // Moments jobs run beside the wake and tile jobs while every post CTA of
  // the plan fits on the SMs at once (one CTA per SM); in larger plans they
  // would only add waves, so each tile job sums its bunches' moments first.
  bool fold = false, split_post = false;
  if (mixed) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, MBT_ERR_CUDA, "device attributes");
    }
    if ((int64_t)st.jobs.size() > (int64_t)nsm) {
      fold = true;
      st.jobs.erase(std::remove_if(st.jobs.begin(), st.jobs.end(), [](const PostJob &j) { return j.type == kJobMoments; }),
                    st.jobs.end());
      // and one wake job per bunch tile of a 256-cell mesh instead of one per
      // M-tile (B built once; the jobs fill fewer waves)
      std::vector<PostJob> merged;
      merged.reserve(st.jobs.size());
      for (const PostJob &j : st.jobs) {
        if (j.type == kJobWake && st.runs[(size_t)j.run].nbins == 256) {
          if (j.sub == 1) continue;   // folded into the job of M-tile 0
          merged.push_back(PostJob{j.run, kJobWake, j.bt, kWakeBoth});
        } else {
          merged.push_back(j);
        }
      }
      st.jobs.swap(merged);
      // plans of more than two post waves: the wake jobs first, to run in a
      // kernel of their own (Plan::post_split, set below)
      if ((int64_t)st.jobs.size() > 2 * (int64_t)nsm) {
        split_post = true;
        std::stable_partition(st.jobs.begin(), st.jobs.end(), [](const PostJob &j) { return j.type == kJobWake; });
      }
    }
  }
  Plan pl{};
  pl.fold_moments = fold ? 1 : 0;
  // the per-tile push in 128-thread CTAs when its tiles fill at least four
  // waves of the 256-thread kernel's resident slots (k_push.cu, LShape)
  if (mixed && !streaming && !any_trans) {
    int tslots = 0;
    if (push_tile_resident_slots(false, &tslots) == cudaSuccess && tslots > 0)
      pl.push_small_ctas = (int64_t)st.tiles.size() >= 4 * (int64_t)tslots ? 1 : 0;
    else
      cudaGetLastError();
  }
  if (!up(st.runs, &pl.runs) || !up(st.bunches, &pl.bunches) || !up(st.tiles, &pl.tiles) || !up(st.jobs, &pl.jobs))
    return fail(c, MBT_ERR_NOMEM, "plan upload failed");
  if (streaming) {
    if (!up(first, &pl.stream_first)) return fail(c, MBT_ERR_NOMEM, "plan upload failed");
    pl.stream_ctas = (int)first.size() - 1;
  }
  // streaming-push copies of the run constants and tile descriptors
  std::vector<StreamRun> sr(st.runs.size());
  for (size_t i = 0; i < st.runs.size(); ++i) {
    const RunDev &r = st.runs[i];
    StreamRun &x = sr[i];
    x = StreamRun{};
    x.invD = r.f_invD;
    x.HinvD = r.f_HinvD;
    x.fnb = r.f_nbins;
    x.invE0 = r.f_invE0 * r.f_omD;
    x.rfA = r.f_rfA;
    x.rfB = r.f_rfB;
    x.w = r.f_w;
    x.qe = r.f_qe;
    x.aT0 = r.f_aT0;
    x.nbins = r.nbins;
    x.nlong = r.nlong;
    x.nharm = r.nharm;
    x.flags = r.flags;
    x.key0 = r.key0;
    x.key1 = r.key1;
    x.omD = r.one_minus_D;
    for (int k = 0; k < kMaxLong; ++k) {
      x.la[k] = r.f_la[k];
      x.lw[k] = r.f_lw[k];
    }
    for (int k = 0; k < kMaxHarm; ++k) x.harm[k] = r.f_harm[k];
  }
  if (!up(sr, &pl.sruns)) return fail(c, MBT_ERR_NOMEM, "plan upload failed");
  std::vector<StreamTile> stl(st.tiles.size());
  for (size_t o = 0; o < st.tiles.size(); ++o) {
    const size_t i = streaming ? (size_t)sorder[o] : o;
    const TileDev &t = st.tiles[i];
    const RunDev &r = st.runs[t.run];
    const BunchDev &b = st.bunches[t.bunch];
    StreamTile &x = stl[o];
    x = StreamTile{};
    x.start = t.start;
    x.count = t.count;
    x.index = (int)i;
    x.m = t.m;
    x.nlong = r.nlong;
    x.nbins = r.nbins;
    if (r.precision != kMixed) continue;
    x.tau = static_cast<float *>(r.tau) + b.off + t.start;
    x.del = r.delta + b.off + t.start;
    x.hist = r.hist + (size_t)t.m * r.nbins;
    x.hist_par = (long long)r.nb * r.nbins;
    x.vrow = static_cast<const float *>(r.vsr) + (size_t)t.m * r.nbins;
    x.turn = r.turn;
    x.rc = pl.sruns + t.run;
    if (r.nlong > 0) {
      x.pq = r.pq + (size_t)t.m * 2;
      x.pq_stride = r.nb * 2;
      x.y = r.y + t.m / kBunchTile;
      x.y_stride = r.ntile_b;
    }
  }
  if (!up(stl, &pl.stiles)) return fail(c, MBT_ERR_NOMEM, "plan upload failed");
  void *p = nullptr;
  size_t pb = std::max<size_t>(st.tiles.size() * kPartials * sizeof(double), 16);
  if (cudaMalloc(&p, pb) != cudaSuccess) return fail(c, MBT_ERR_NOMEM, "plan partials");
  cudaMemset(p, 0, pb);
  st.allocs.push_back(p);
  pl.partial = static_cast<double *>(p);
  if (cudaMalloc(&p, 16) != cudaSuccess) return fail(c, MBT_ERR_NOMEM, "plan counters");
  cudaMemset(p, 0, 16);
  st.allocs.push_back(p);
  pl.done = static_cast<unsigned int *>(p);
  pl.error = reinterpret_cast<int *>(static_cast<char *>(p) + 8);
  pl.nruns = (int)st.runs.size();
  pl.nbunches = (int)st.bunches.size();
  pl.ntiles = (int)st.tiles.size();
  pl.njobs = (int)st.jobs.size();
  pl.max_nbins = 0;
  pl.max_nlong = 0;
  pl.max_nharm = 0;
  pl.max_trans = 0;
  for (auto &r : st.runs) {
    pl.max_nbins = std::max(pl.max_nbins, r.nbins);
    pl.max_nlong = std::max(pl.max_nlong, r.nlong);
    pl.max_nharm = std::max(pl.max_nharm, r.nharm);
    pl.max_trans = std::max(pl.max_trans, r.trans);
  }
  st.bytes += pb + 16;
  // plans of more than two post waves: the wake jobs (at the front of the
  // list) in a kernel of their own, the others beside them on a stream of the
  // plan's own.  Below that the single kernel is kept: the next push then
  // follows it programmatically (the 390-bunch fill with a transverse plane,
  // 156 jobs: 348.0 us per turn split against 342.6 us)
  if (split_post) {
    int nw = 0;
    for (const PostJob &j : st.jobs) nw += j.type == kJobWake ? 1 : 0;
    if (nw > 0 && nw < (int)st.jobs.size()) {
      if (cudaStreamCreateWithFlags(&pl.side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&pl.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&pl.ev_join, cudaEventDisableTiming) != cudaSuccess) {
        if (pl.side) cudaStreamDestroy(pl.side);
        if (pl.ev_fork) cudaEventDestroy(pl.ev_fork);
        if (pl.ev_join) cudaEventDestroy(pl.ev_join);
        return fail(c, MBT_ERR_CUDA, "post-kernel stream");
      }
      pl.post_split = nw;
    }
  }
  st.plan = pl;
  return MBT_OK;
}

// Append one context's run to a plan under construction.
void append_run(PlanStore &st, mbt_ctx *c, int mixed_tile) {
  const int ri = (int)st.runs.size();
  RunDev rd = c->rundev;
  rd.bunch_base = (int)st.bunches.size();
  st.runs.push_back(rd);
  const int tile = c->precision == MBT_PREC_MIXED ? mixed_tile : kF64Tile;
  for (int m = 0; m < c->nb; ++m) {
    BunchDev bd{};
    bd.run = ri;
    bd.m = m;
    bd.off = c->off[m];
    bd.n = c->nmp[m];
    bd.tile0 = (int)st.tiles.size();
    // k = ceil(n / tile) tiles of equal size (multiples of 4 particles, the last one shorter)
    const int64_t n = c->nmp[m];
    const int64_t k = (n + tile - 1) / tile;
    const int64_t base = c->precision == MBT_PREC_MIXED ? ((n + k - 1) / k + 3) / 4 * 4 : tile;
    for (int64_t s = 0; s < n; s += base) {
      TileDev t{};
      t.bunch = (int)st.bunches.size();
      t.run = ri;
      t.m = m;
      t.start = s;
      t.count = (int)std::min<int64_t>(base, n - s);
      st.tiles.push_back(t);
    }
    bd.ntiles = (int)st.tiles.size() - bd.tile0;
    st.bunches.push_back(bd);
  }
  for (int bt = 0; bt < c->ntile_b; ++bt) {
    st.jobs.push_back(PostJob{ri, kJobTile, bt, 0});
    if (c->precision == MBT_PREC_MIXED) {
      for (int mt = 0; mt < c->nbins / 128; ++mt) st.jobs.push_back(PostJob{ri, kJobWake, bt, mt});
      st.jobs.push_back(PostJob{ri, kJobMoments, bt, 0});
    }
  }
  if (c->precision == MBT_PREC_F64) {
    const int nchunk = (c->nbins + kF64RowChunk - 1) / kF64RowChunk;
    for (int m = 0; m < c->nb; ++m)
      for (int ch = 0; ch < nchunk; ++ch) {
        st.jobs.push_back(PostJob{ri, kJobWake, m, ch});
        if (c->trans) st.jobs.push_back(PostJob{ri, kJobTrans, m, ch});
      }
  } else if (c->trans) {
    for (int bt = 0; bt < c->ntile_b; ++bt)
      for (int ch = 0; ch < c->nbins / kTransRows; ++ch) st.jobs.push_back(PostJob{ri, kJobTrans, bt, ch});
  }
}

mbt_status check_device(mbt_ctx *c, const Plan &pl) {
  int err = 0;
  cudaError_t e = cudaMemcpy(&err, pl.error, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "device error word");
  if (err != 0) {
    int zero = 0;
    cudaMemcpy(pl.error, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (err == kErrTmem) return fail(c, MBT_ERR_CUDA, "tensor memory could not be allocated");
    if (err == kErrCount) return fail(c, MBT_ERR_ARG, "a cell count outside [0, 2^24) reached the wake");
    if (err == kErrDipole)
      return fail(c, MBT_ERR_UNSUPPORTED,
                  "a transverse coordinate left the mixed push's dipole range (2^10 x the beam size scale)");
    return fail(c, MBT_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", err);
  }
  return MBT_OK;
}

// Turns as push + post launches.  Plain: the first push of the call is an
// ordinary launch and every later kernel uses programmatic dependent launch
// (its prologue overlaps the previous kernel's tail).  Timed: ordinary
// launches with CUDA events around each kernel, drained in chunks.
mbt_status launch_turns(mbt_ctx *c, const Plan &pl, int prec, int64_t nturns, cudaStream_t s, bool timed) {
  if (!timed) {
    for (int64_t t = 0; t < nturns; ++t) {
      // (after a split post kernel the stream's last step is an event wait: a plain launch)
      cudaError_t e = launch_push(pl, prec, s, t > 0 && pl.post_split == 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "push launch");
      e = launch_post(pl, prec, s, true);
      if (e != cudaSuccess) return cuda_fail(c, e, "post launch");
    }
    return MBT_OK;
  }
  const int chunk = 512;
  if (c->ev_pool.size() < (size_t)(3 * chunk)) {
    while (c->ev_pool.size() < (size_t)(3 * chunk)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return fail(c, MBT_ERR_CUDA, "event create");
      c->ev_pool.push_back(e);
    }
  }
  for (int64_t t0 = 0; t0 < nturns; t0 += chunk) {
    const int n = (int)std::min<int64_t>(chunk, nturns - t0);
    for (int i = 0; i < n; ++i) {
      cudaEventRecord(c->ev_pool[3 * i], s);
      cudaError_t e = launch_push(pl, prec, s, false);
      if (e != cudaSuccess) return cuda_fail(c, e, "push launch");
      cudaEventRecord(c->ev_pool[3 * i + 1], s);
      e = launch_post(pl, prec, s, false);
      if (e != cudaSuccess) return cuda_fail(c, e, "post launch");
      cudaEventRecord(c->ev_pool[3 * i + 2], s);
    }
    cudaError_t e = cudaEventSynchronize(c->ev_pool[3 * (n - 1) + 2]);
    if (e != cudaSuccess) return cuda_fail(c, e, "timed turns");
    for (int i = 0; i < n; ++i) {
      float a = 0.f, b = 0.f;
      cudaEventElapsedTime(&a, c->ev_pool[3 * i], c->ev_pool[3 * i + 1]);
      cudaEventElapsedTime(&b, c->ev_pool[3 * i + 1], c->ev_pool[3 * i + 2]);
      c->push_ms += a;
      c->post_ms += b;
      c->timed_launches += 1;
    }
  }
  return MBT_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int mbt_version(void) { return MBT_VERSION; }

const char *mbt_status_string(mbt_status s) {
  switch (s) {
    case MBT_OK: return "ok";
    case MBT_ERR_ARG: return "invalid argument";
    case MBT_ERR_STATE: return "invalid state";
    case MBT_ERR_NOMEM: return "out of memory";
    case MBT_ERR_CUDA: return "CUDA error";
    case MBT_ERR_TIMEOUT: return "device wait timed out";
    case MBT_ERR_UNSUPPORTED: return "unsupported configuration";
    case MBT_ERR_BUDGET: return "memory budget exceeded";
    default: return "unknown status";
  }
}

mbt_status mbt_create(const mbt_ring *ring, int precision, int flags, uint64_t seed, mbt_ctx **out) {
  if (!ring || !out) return MBT_ERR_ARG;
  *out = nullptr;
  if (!(ring->E0_eV > 0) || !(ring->T0_s > 0) || ring->h < 1 || ring->h > 65535 || ring->reserved != 0 ||
      !(ring->V_rf_V > 0) || !(ring->alpha_c != 0) || !(ring->U0_eV >= 0) || !(ring->U0_eV < ring->V_rf_V) ||
      !(ring->sigma_delta > 0) || !(ring->tau_z_s > 0))
    return MBT_ERR_ARG;
  if (precision != MBT_PREC_F64 && precision != MBT_PREC_MIXED) return MBT_ERR_ARG;
  if (flags & ~(MBT_NO_SR | MBT_NO_QE | MBT_KICK_NGP)) return MBT_ERR_ARG;
  mbt_ctx *c = new (std::nothrow) mbt_ctx();
  if (!c) return MBT_ERR_NOMEM;
  c->ring = *ring;
  c->precision = precision;
  c->flags = flags;
  c->seed = seed;
  derive(c);
  *out = c;
  return MBT_OK;
}

void mbt_destroy(mbt_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_device(c);
  delete c;
}

const char *mbt_last_error(const mbt_ctx *c) { return c ? c->err.c_str() : "null context"; }

mbt_status mbt_add_resonator(mbt_ctx *c, double Rs, double fr, double Q, int range) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "resonators must be added before mbt_set_fill");
  if (!(Rs > 0) || !(fr > 0) || !(Q > 0.5) || range < 1 || range > 3)
    return fail(c, MBT_ERR_ARG, "resonator needs Rs > 0, fr > 0, Q > 0.5, range 1..3");
  if ((int)c->res.size() >= kMaxRes) return fail(c, MBT_ERR_UNSUPPORTED, "at most %d resonators", kMaxRes);
  int nl = 0;
  for (auto &r : c->res) nl += (r.range & MBT_RANGE_LONG) ? 1 : 0;
  if ((range & MBT_RANGE_LONG) && nl >= kMaxLong)
    return fail(c, MBT_ERR_UNSUPPORTED, "at most %d long-range resonators", kMaxLong);
  c->res.push_back(Resonator{Rs, fr, Q, range});
  return MBT_OK;
}

mbt_status mbt_set_transverse(mbt_ctx *c, double beta, double alpha, double tune, double xi, double emit) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "the transverse plane must be set before mbt_set_fill");
  if (c->trans) return fail(c, MBT_ERR_STATE, "the transverse plane is already set");
  if (!(beta > 0) || !std::isfinite(beta) || !std::isfinite(alpha) || !std::isfinite(tune) || !std::isfinite(xi) ||
      !(emit >= 0) || !std::isfinite(emit))
    return fail(c, MBT_ERR_ARG, "transverse plane needs beta > 0, emittance >= 0 and finite alpha, tune, chromaticity");
  c->trans = true;
  c->t_beta = beta;
  c->t_alpha = alpha;
  c->t_tune = tune;
  c->t_xi = xi;
  c->t_emit = emit;
  return MBT_OK;
}

mbt_status mbt_add_transverse_resonator(mbt_ctx *c, double Rs, double fr, double Q, int range) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "resonators must be added before mbt_set_fill");
  if (!c->trans) return fail(c, MBT_ERR_STATE, "set the transverse plane first");
  if (!(Rs > 0) || !(fr > 0) || !(Q > 0.5) || range < 1 || range > 3)
    return fail(c, MBT_ERR_ARG, "resonator needs Rs > 0, fr > 0, Q > 0.5, range 1..3");
  if ((int)c->tres.size() >= kMaxRes) return fail(c, MBT_ERR_UNSUPPORTED, "at most %d transverse resonators", kMaxRes);
  int nl = 0;
  for (auto &r : c->res) nl += (r.range & MBT_RANGE_LONG) ? 1 : 0;
  for (auto &r : c->tres) nl += (r.range & MBT_RANGE_LONG) ? 1 : 0;
  if ((range & MBT_RANGE_LONG) && nl >= kMaxLong)
    return fail(c, MBT_ERR_UNSUPPORTED, "at most %d long-range resonators (both planes)", kMaxLong);
  c->tres.push_back(Resonator{Rs, fr, Q, range});
  return MBT_OK;
}

mbt_status mbt_add_transverse_resistive_wall(mbt_ctx *c, double b, double sigma, double L, int nh) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "resistive walls must be added before mbt_set_fill");
  if (!c->trans) return fail(c, MBT_ERR_STATE, "set the transverse plane first");
  if (!(b > 0) || !(sigma > 0) || !(L > 0) || !std::isfinite(b) || !std::isfinite(sigma) || !std::isfinite(L) ||
      nh < 1 || nh > 1000)
    return fail(c, MBT_ERR_ARG, "a transverse resistive wall needs radius, conductivity, length > 0 and 1..1000 turns");
  constexpr double kZ0 = 376.730313668, kC = 299792458.0;
  c->rw_A += kC * L / (kPi * b * b * b) * std::sqrt(kZ0 / (kPi * sigma)) / std::sqrt(kC);
  c->rw_nh = std::max(c->rw_nh, nh);
  return MBT_OK;
}

mbt_status mbt_add_harmonic_cavity(mbt_ctx *c, int n, double V, double phi) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "harmonic cavities must be added before mbt_set_fill");
  if (n < 1 || n > 16 || !(V >= 0) || !std::isfinite(V) || !std::isfinite(phi))
    return fail(c, MBT_ERR_ARG, "a harmonic cavity needs 1 <= n <= 16, V >= 0 and a finite phase");
  if ((int)c->harm.size() >= kMaxHarm) return fail(c, MBT_ERR_UNSUPPORTED, "at most %d harmonic cavities", kMaxHarm);
  c->harm.push_back({(double)n, V, phi});
  derive(c);
  return MBT_OK;
}

mbt_status mbt_add_wake_table(mbt_ctx *c, int n, const double *t, const double *w) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "wake tables must be added before mbt_set_fill");
  if (n < 2 || !t || !w || t[0] != 0.0) return fail(c, MBT_ERR_ARG, "a wake table needs n >= 2 samples from t = 0");
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(t[i]) || !std::isfinite(w[i])) return fail(c, MBT_ERR_ARG, "wake table sample %d is not finite", i);
    if (i > 0 && !(t[i] > t[i - 1])) return fail(c, MBT_ERR_ARG, "wake table times must increase strictly");
  }
  if (c->wt_t.size() >= 8) return fail(c, MBT_ERR_UNSUPPORTED, "at most 8 wake tables");
  c->wt_t.emplace_back(t, t + n);
  c->wt_w.emplace_back(w, w + n);
  return MBT_OK;
}

mbt_status mbt_add_resistive_wall(mbt_ctx *c, double b, double sigma, double L) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "resistive walls must be added before mbt_set_fill");
  if (!(b > 0) || !(sigma > 0) || !(L > 0) || !std::isfinite(b) || !std::isfinite(sigma) || !std::isfinite(L))
    return fail(c, MBT_ERR_ARG, "a resistive wall needs radius, conductivity and length > 0");
  if (c->rwalls.size() >= 8) return fail(c, MBT_ERR_UNSUPPORTED, "at most 8 resistive walls");
  c->rwalls.push_back({b, sigma, L});
  return MBT_OK;
}

mbt_status mbt_set_grid(mbt_ctx *c, int nbins, double hw) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "grid must be set before mbt_set_fill");
  if (!(hw > 0)) return fail(c, MBT_ERR_ARG, "half width must be > 0");
  if (c->precision == MBT_PREC_MIXED) {
    if (nbins != 128 && nbins != 256) return fail(c, MBT_ERR_UNSUPPORTED, "mixed precision needs nbins 128 or 256");
  } else if (nbins < 2 || nbins > 1024) {
    return fail(c, MBT_ERR_ARG, "nbins must be 2..1024");
  }
  c->nbins = nbins;
  c->half_width_sigmas = hw;
  derive(c);
  return MBT_OK;
}

mbt_status mbt_set_record(mbt_ctx *c, int64_t cap) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "record capacity must be set before mbt_set_fill");
  if (cap < 1 || cap > (int64_t)1 << 30) return fail(c, MBT_ERR_ARG, "capacity out of range");
  c->cap = cap;
  return MBT_OK;
}

mbt_status mbt_set_fill(mbt_ctx *c, int nb, const int32_t *bucket, const double *current, const int64_t *nmp) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (c->filled) return fail(c, MBT_ERR_STATE, "fill already set");
  if (nb < 1 || nb > kMaxBunches || !bucket || !current || !nmp)
    return fail(c, MBT_ERR_ARG, "need 1..%d bunches and non-null arrays", kMaxBunches);
  const int64_t nmax = c->precision == MBT_PREC_MIXED ? ((int64_t)1 << 24) - 1 : ((int64_t)1 << 31) - 2;
  for (int m = 0; m < nb; ++m) {
    if (bucket[m] < 0 || bucket[m] >= c->ring.h || (m > 0 && bucket[m] <= bucket[m - 1]))
      return fail(c, MBT_ERR_ARG, "buckets must be strictly increasing in [0, h)");
    if (!(current[m] >= 0) || nmp[m] < 1 || nmp[m] > nmax)
      return fail(c, MBT_ERR_ARG, "bunch %d: current >= 0 and 1 <= n_mp <= %lld required", m, (long long)nmax);
  }
  derive(c);
  if (!(std::fabs(c->sin_phi_s) <= 1.0) || !(c->sigma_tau0 > 0.0))
    return fail(c, MBT_ERR_ARG, "no stable synchronous phase: the main cavity cannot balance U0 and the harmonic cavities");
  cudaError_t ce = cudaFree(0);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "CUDA initialisation");
  c->nb = nb;
  c->bucket.assign(bucket, bucket + nb);
  c->current.assign(current, current + nb);
  c->nmp.assign(nmp, nmp + nb);
  c->off.resize(nb);
  int64_t o = 0;
  c->n_particles = 0;
  for (int m = 0; m < nb; ++m) {
    c->off[m] = o;
    o += (nmp[m] + 3) / 4 * 4;
    c->n_particles += nmp[m];
  }
  c->n_alloc = o + 4;
  c->ntile_b = (nb + kBunchTile - 1) / kBunchTile;
  c->long_idx.clear();
  c->long_plane.clear();
  for (int i = 0; i < (int)c->res.size(); ++i)
    if (c->res[i].range & MBT_RANGE_LONG) {
      c->long_idx.push_back(i);
      c->long_plane.push_back(0);
    }
  for (int i = 0; i < (int)c->tres.size(); ++i)
    if (c->tres[i].range & MBT_RANGE_LONG) {
      c->long_idx.push_back(i);
      c->long_plane.push_back(1);
    }
  c->nlong = (int)c->long_idx.size();
  const int nl = std::max(1, c->nlong);
  const bool mixed = c->precision == MBT_PREC_MIXED;
  const int nbins = c->nbins;

  mbt_status st;
#define ALLOC(ptr, bytes)                                  \
  if ((st = dalloc(c, &(ptr), (bytes))) != MBT_OK) {       \
    free_device(c);                                        \
    return st;                                             \
  }
  ALLOC(c->d_tau, (size_t)c->n_alloc * (mixed ? sizeof(float) : sizeof(double)));
  ALLOC(c->d_delta, (size_t)c->n_alloc * sizeof(double));
  ALLOC(c->d_hist, (size_t)2 * nb * nbins * sizeof(int32_t));
  ALLOC(c->d_vsr, (size_t)nb * nbins * (mixed ? sizeof(float) : sizeof(double)));
  ALLOC(c->d_pq, (size_t)nl * nb * 2 * sizeof(double2));
  ALLOC(c->d_y, (size_t)nl * c->ntile_b * sizeof(double2));
  ALLOC(c->d_agg, (size_t)nl * c->ntile_b * 2 * sizeof(double2));
  ALLOC(c->d_carry, (size_t)nl * sizeof(double2));
  ALLOC(c->d_rec, (size_t)c->cap * nb * kRecord * sizeof(double));
  ALLOC(c->d_turn, 16);
  ALLOC(c->d_q, (size_t)nb * sizeof(double));
  ALLOC(c->d_qf, (size_t)nb * sizeof(float));
  ALLOC(c->d_inv_n, (size_t)nb * sizeof(double));
  ALLOC(c->d_hoff, (size_t)nb * sizeof(long long));
  ALLOC(c->d_lagf, (size_t)nbins * sizeof(float));
  ALLOC(c->d_step, (size_t)nl * nb * sizeof(double2));
  ALLOC(c->d_emis, (size_t)nl * nbins * sizeof(double2));
  ALLOC(c->d_emis_f, (size_t)nl * nbins * sizeof(float2));
  size_t toep_bytes = (size_t)nbins * sizeof(double);
  if (mixed) {
    toep_bytes = 0;
    for (int mt = 0; mt < nbins / 128; ++mt) toep_bytes += (size_t)512 * std::min(nbins, 128 * (mt + 1));
  }
  ALLOC(c->d_toep, toep_bytes);
  if (c->trans) {
    const size_t fs = mixed ? sizeof(float) : sizeof(double);
    ALLOC(c->d_x, (size_t)c->n_alloc * fs);
    ALLOC(c->d_xp, (size_t)c->n_alloc * fs);
    ALLOC(c->d_dip, (size_t)2 * nb * nbins * 8);   // int64 fixed point (kMixed) or double
    ALLOC(c->d_vt, (size_t)nb * nbins * fs);
    ALLOC(c->d_trec, (size_t)c->cap * nb * kTRecord * sizeof(double));
    ALLOC(c->d_tlag, (size_t)nbins * sizeof(double));
    ALLOC(c->d_tlag_f, (size_t)nbins * sizeof(float));
    if (c->rw_nh > 0) {
      ALLOC(c->d_rwtab, (size_t)(c->rw_nh + 1) * c->ring.h * sizeof(double));
      ALLOC(c->d_rwtab_f, (size_t)(c->rw_nh + 1) * c->ring.h * sizeof(float));
      ALLOC(c->d_rwcent, (size_t)(c->rw_nh + 1) * nb * sizeof(double));
      ALLOC(c->d_bucket, (size_t)nb * sizeof(int32_t));
    }
  }
#undef ALLOC

  // macro-particle charge
  std::vector<double> q(nb);
  for (int m = 0; m < nb; ++m) q[m] = c->current[m] * c->ring.T0_s / (double)c->nmp[m];
  cudaMemcpy(c->d_q, q.data(), nb * sizeof(double), cudaMemcpyHostToDevice);
  {
    std::vector<float> qf(nb);
    std::vector<double> inv_n(nb);
    for (int m = 0; m < nb; ++m) {
      qf[m] = (float)q[m];
      inv_n[m] = 1.0 / (double)c->nmp[m];
    }
    cudaMemcpy(c->d_qf, qf.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_inv_n, inv_n.data(), nb * sizeof(double), cudaMemcpyHostToDevice);
    std::vector<long long> hoff(nb);
    long long h = 0;
    for (int m = 0; m < nb; ++m) {
      hoff[m] = h;
      h += c->nmp[m];
    }
    cudaMemcpy(c->d_hoff, hoff.data(), nb * sizeof(long long), cudaMemcpyHostToDevice);
  }

  // summed short-range wake per lag (half of W(0+) at lag 0)
  std::vector<double> lag(nbins, 0.0);
  for (int l = 0; l < nbins; ++l)
    for (auto &r : c->res)
      if (r.range & MBT_RANGE_SHORT) lag[l] += wake(r, (double)l * c->Delta);
  // tabulated wakes and resistive walls: averages over the lag cells
  // [(l - 1/2) Delta, (l + 1/2) Delta], the half cell [0, Delta / 2] at lag 0
  for (int l = 0; l < nbins; ++l) {
    const double lo = l == 0 ? 0.0 : ((double)l - 0.5) * c->Delta, hi = ((double)l + 0.5) * c->Delta;
    for (size_t i = 0; i < c->wt_t.size(); ++i) lag[l] += table_integral(c->wt_t[i], c->wt_w[i], lo, hi) / c->Delta;
    for (auto &rw : c->rwalls) lag[l] += rw_integral(rw[0], rw[1], rw[2], lo, hi) / c->Delta;
  }
  {
    std::vector<float> lagf(nbins);
    for (int l = 0; l < nbins; ++l) lagf[l] = (float)lag[l];
    cudaMemcpy(c->d_lagf, lagf.data(), nbins * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (mixed) {
    std::vector<uint16_t> img(toep_bytes / 2, 0);
    pack_toeplitz_images(lag.data(), nbins, img.data());
    cudaMemcpy(c->d_toep, img.data(), toep_bytes, cudaMemcpyHostToDevice);
  } else {
    cudaMemcpy(c->d_toep, lag.data(), toep_bytes, cudaMemcpyHostToDevice);
  }

  // long-range tables: emission e^{-s tau_k}, step maps a_m = e^{s dt_m}
  RunDev &rd = c->rundev;
  rd = RunDev{};
  {
    std::vector<double2> emis((size_t)nl * nbins, make_double2(0, 0));
    std::vector<float2> emis_f((size_t)nl * nbins, make_float2(0, 0));
    std::vector<double2> step((size_t)nl * nb, make_double2(1, 0));
    for (int li = 0; li < c->nlong; ++li) {
      const bool tr = c->long_plane[li] == 1;
      const Resonator &r = tr ? c->tres[c->long_idx[li]] : c->res[c->long_idx[li]];
      double a, wb;
      res_consts(r, a, wb);
      const cplx s(-a, wb);
      // longitudinal: W = Re(c e^{st}), c = 2 a Rs (1 + i a / wb); transverse: W = Im(c e^{st}), c = wr^2 Rs / (Q wb)
      const double wr = 2.0 * kPi * r.fr;
      const cplx cc = tr ? cplx(wr * wr * r.Rs / (r.Q * wb), 0.0) : 2.0 * a * r.Rs * cplx(1.0, a / wb);
      rd.lr_plane[li] = tr ? 1 : 0;
      rd.lr_s[li] = make_double2(s.real(), s.imag());
      rd.lr_c[li] = make_double2(cc.real(), cc.imag());
      for (int k = 0; k < nbins; ++k) {
        const double tk = -c->H + ((double)k + 0.5) * c->Delta;
        const cplx e = std::exp(-s * tk);
        emis[(size_t)li * nbins + k] = make_double2(e.real(), e.imag());
        emis_f[(size_t)li * nbins + k] = make_float2((float)e.real(), (float)e.imag());
      }
      for (int m = 0; m < nb; ++m) {
        const int64_t dbk = m > 0 ? (int64_t)c->bucket[m] - c->bucket[m - 1]
                                  : (int64_t)c->ring.h - c->bucket[nb - 1] + c->bucket[0];
        const double dt = (double)dbk * c->T_rf;
        const cplx z = std::exp(s * dt);
        step[(size_t)li * nb + m] = make_double2(z.real(), z.imag());
      }
    }
    cudaMemcpy(c->d_emis, emis.data(), emis.size() * sizeof(double2), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_emis_f, emis_f.data(), emis_f.size() * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_step, step.data(), step.size() * sizeof(double2), cudaMemcpyHostToDevice);
  }

  rd.tau = c->d_tau;
  rd.delta = c->d_delta;
  rd.hist = c->d_hist;
  rd.vsr = c->d_vsr;
  rd.pq = c->d_pq;
  rd.y = c->d_y;
  rd.agg = c->d_agg;
  rd.carry = c->d_carry;
  rd.rec = c->d_rec;
  rd.turn = c->d_turn;
  rd.q_mp = c->d_q;
  rd.step = c->d_step;
  rd.emis = c->d_emis;
  rd.emis_f = c->d_emis_f;
  rd.toep = c->d_toep;
  rd.nb = nb;
  rd.nbins = nbins;
  rd.nlong = c->nlong;
  rd.ntile_b = c->ntile_b;
  rd.cap = (int)c->cap;
  rd.flags = c->flags;
  rd.precision = c->precision;
  rd.key0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
  rd.key1 = (uint32_t)(c->seed >> 32);
  rd.inv_E0 = 1.0 / c->ring.E0_eV;
  rd.V_over_E0 = c->ring.V_rf_V / c->ring.E0_eV;
  rd.sin_phi_s = c->sin_phi_s;
  rd.cos_phi_s = c->cos_phi_s;
  rd.U0_over_E0 = (c->flags & MBT_NO_SR) ? 0.0 : c->ring.U0_eV / c->ring.E0_eV;
  rd.omega_rf = c->omega_rf;
  rd.phi_s = c->phi_s;
  rd.one_minus_D = 1.0 - c->D;
  rd.qe_amp = c->qe;
  rd.aT0 = c->ring.alpha_c * c->ring.T0_s;
  rd.H = c->H;
  rd.invDelta = c->invDelta;
  rd.Delta = c->Delta;
  rd.sigma_tau0 = c->sigma_tau0;
  rd.sigma_E = c->ring.sigma_delta;
  rd.q_mp_f = c->d_qf;
  rd.inv_n = c->d_inv_n;
  rd.lag_f = c->d_lagf;
  rd.f_invD = (float)rd.invDelta;
  rd.f_HinvD = (float)(rd.H * rd.invDelta - 0.5);   // cell coordinate from the cell centres
  rd.f_nbins = (float)nbins;
  rd.f_invE0 = (float)rd.inv_E0;
  rd.f_rfA = (float)(rd.V_over_E0 * rd.one_minus_D * rd.sin_phi_s);
  rd.f_rfB = (float)(rd.V_over_E0 * rd.one_minus_D * rd.cos_phi_s);
  rd.f_w = (float)rd.omega_rf;
  rd.f_omD = (float)rd.one_minus_D;
  rd.f_qe = (float)rd.qe_amp;
  rd.f_aT0 = (float)rd.aT0;
  for (int li = 0; li < kMaxLong; ++li) {
    rd.f_la[li] = li < c->nlong ? (float)(-rd.lr_s[li].x * 1.4426950408889634) : 0.f;   // x log2(e): ex2
    rd.f_lw[li] = li < c->nlong ? (float)rd.lr_s[li].y : 0.f;
  }
  if (c->trans) {
    std::vector<double> tl(nbins, 0.0);
    std::vector<float> tlf(nbins);
    for (int l = 0; l < nbins; ++l) {
      for (auto &r : c->tres)
        if (r.range & MBT_RANGE_SHORT) tl[l] += twake(r, (double)l * c->Delta);
      tlf[l] = (float)tl[l];
    }
    cudaMemcpy(c->d_tlag, tl.data(), nbins * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->d_tlag_f, tlf.data(), nbins * sizeof(float), cudaMemcpyHostToDevice);
    const bool sr = !(c->flags & MBT_NO_SR), qe = sr && !(c->flags & MBT_NO_QE);
    const double Dx = qe ? c->ring.U0_eV / c->ring.E0_eV : 0.0;
    rd.trans = 1;
    rd.x = c->d_x;
    rd.xp = c->d_xp;
    rd.dip = c->d_dip;
    rd.vt = c->d_vt;
    rd.trec = c->d_trec;
    rd.tlag = c->d_tlag;
    rd.tlag_f = c->d_tlag_f;
    rd.t_beta = c->t_beta;
    rd.t_alpha = c->t_alpha;
    rd.t_gamma = (1.0 + c->t_alpha * c->t_alpha) / c->t_beta;
    rd.t_mu0 = 2.0 * kPi * c->t_tune;
    rd.t_xi = c->t_xi;
    rd.t_emit = c->t_emit;
    rd.t_nx = std::sqrt(c->t_beta * c->t_emit) * std::sqrt(Dx);
    rd.t_nxp = std::sqrt(rd.t_gamma * c->t_emit) * std::sqrt(Dx);
    // FP32 phase: the fractional tune (|2 pi frac| <= pi keeps the special-function unit accurate)
    // plus the chromatic term of the full tune
    rd.f_tmu0 = (float)(2.0 * kPi * (c->t_tune - std::nearbyint(c->t_tune)));
    rd.f_tmu0xi = (float)(2.0 * kPi * c->t_tune * c->t_xi);
    rd.f_tbeta = (float)rd.t_beta;
    rd.f_talpha = (float)rd.t_alpha;
    rd.f_tgamma = (float)rd.t_gamma;
    rd.f_tnx = (float)rd.t_nx;
    rd.f_tnxp = (float)rd.t_nxp;
    // dipole deposit unit of the mixed push: a power of two 2^-20 of the beam
    // size rounded up to a power of two (at least 2^-16 m), so that |x| up to
    // 2^10 times that scale (and at least 2^-6 m) is accepted
    {
      const double sx = std::sqrt(c->t_beta * c->t_emit);
      const int e = sx > 0 ? std::max(-16, (int)std::ceil(std::log2(sx))) : -16;
      rd.dip_unit = std::ldexp(1.0, e - 20);
      rd.f_dip_unit = (float)rd.dip_unit;
      rd.f_dip_inv = (float)std::ldexp(1.0, 20 - e);
      rd.f_dip_range = (float)std::ldexp(1.0, e + 10);
    }
    if (c->rw_nh > 0) {
      const size_t nt = (size_t)(c->rw_nh + 1) * c->ring.h;
      std::vector<double> tab(nt, 0.0);
      std::vector<float> tabf(nt, 0.f);
      for (size_t D = 1; D < nt; ++D) {
        tab[D] = c->rw_A / std::sqrt((double)D * c->T_rf);
        tabf[D] = (float)tab[D];
      }
      cudaMemcpy(c->d_rwtab, tab.data(), nt * sizeof(double), cudaMemcpyHostToDevice);
      cudaMemcpy(c->d_rwtab_f, tabf.data(), nt * sizeof(float), cudaMemcpyHostToDevice);
      cudaMemcpy(c->d_bucket, c->bucket.data(), (size_t)nb * sizeof(int32_t), cudaMemcpyHostToDevice);
      rd.rw_nh = c->rw_nh;
      rd.h_rf = c->ring.h;
      rd.rw_tab = c->d_rwtab;
      rd.rw_tab_f = c->d_rwtab_f;
      rd.rw_cent = c->d_rwcent;
      rd.bucket = c->d_bucket;
    }
  }
  rd.f_inv_omD = (float)(1.0 / rd.one_minus_D);
  rd.f_U0oE0 = (float)rd.U0_over_E0;
  rd.nharm = (int)c->harm.size();
  for (int k = 0; k < rd.nharm; ++k) {
    const double n = c->harm[k][0], V = c->harm[k][1], ph = c->harm[k][2];
    rd.harm_VoE0[k] = V / c->ring.E0_eV;
    rd.harm_phi[k] = ph;
    rd.harm_nw[k] = n * c->omega_rf;
    rd.f_harm[k] = make_float4((float)(2.0 * V / c->ring.E0_eV * rd.one_minus_D), (float)std::cos(ph),
                               (float)std::sin(ph), (float)(0.5 * n * c->omega_rf));
  }

  PlanStore &ps = c->own;
  ps.runs.clear();
  ps.bunches.clear();
  ps.tiles.clear();
  ps.jobs.clear();
  ps.precision = c->precision;
  append_run(ps, c, c->tile);
  if ((st = upload_plan(c, ps)) != MBT_OK) {
    free_device(c);
    return st;
  }
  cudaError_t e = configure_kernels();
  if (e == cudaSuccess) e = configure_push_kernels();
  if (e != cudaSuccess) {
    free_device(c);
    return cuda_fail(c, e, "kernel attributes");
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_device(c);
    return cuda_fail(c, e, "fill setup");
  }
  c->filled = true;
  return MBT_OK;
}

mbt_status mbt_init_particles(mbt_ctx *c, void *stream) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nl = std::max(1, c->nlong);
  cudaMemsetAsync(c->d_hist, 0, (size_t)2 * c->nb * c->nbins * sizeof(int32_t), s);
  cudaMemsetAsync(c->d_vsr, 0,
                  (size_t)c->nb * c->nbins * (c->precision == MBT_PREC_MIXED ? sizeof(float) : sizeof(double)), s);
  cudaMemsetAsync(c->d_pq, 0, (size_t)nl * c->nb * 2 * sizeof(double2), s);
  cudaMemsetAsync(c->d_y, 0, (size_t)nl * c->ntile_b * sizeof(double2), s);
  cudaMemsetAsync(c->d_agg, 0, (size_t)nl * c->ntile_b * 2 * sizeof(double2), s);
  cudaMemsetAsync(c->d_carry, 0, (size_t)nl * sizeof(double2), s);
  cudaMemsetAsync(c->d_turn, 0, 16, s);
  if (c->trans) {
    const size_t fs = c->precision == MBT_PREC_MIXED ? sizeof(float) : sizeof(double);
    cudaMemsetAsync(c->d_dip, 0, (size_t)2 * c->nb * c->nbins * 8, s);
    cudaMemsetAsync(c->d_vt, 0, (size_t)c->nb * c->nbins * fs, s);
    if (c->rw_nh > 0) cudaMemsetAsync(c->d_rwcent, 0, (size_t)(c->rw_nh + 1) * c->nb * sizeof(double), s);
  }
  cudaError_t e = launch_init(c->own.plan, c->precision, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "init launch");
  return MBT_OK;
}

mbt_status mbt_set_particles(mbt_ctx *c, int bunch, const double *tau, const double *delta) {
  if (!c || !tau || !delta) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (bunch < 0 || bunch >= c->nb) return fail(c, MBT_ERR_ARG, "bunch out of range");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const int64_t n = c->nmp[bunch];
  const bool mixed = c->precision == MBT_PREC_MIXED;
  const size_t tb = (size_t)n * (mixed ? sizeof(float) : sizeof(double));
  char *h = static_cast<char *>(stage(c, tb + (size_t)n * sizeof(double)));
  if (!h) return fail(c, MBT_ERR_NOMEM, "pinned staging buffer");
  if (mixed) {
    float *tf = reinterpret_cast<float *>(h);
    for (int64_t i = 0; i < n; ++i) tf[i] = (float)tau[i];
  } else {
    std::memcpy(h, tau, tb);
  }
  std::memcpy(h + tb, delta, (size_t)n * sizeof(double));
  char *dt = static_cast<char *>(c->d_tau) + (size_t)c->off[bunch] * (mixed ? sizeof(float) : sizeof(double));
  e = cudaMemcpy(dt, h, tb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_delta + c->off[bunch], h + tb, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "set particles");
  return MBT_OK;
}

mbt_status mbt_set_particles_all(mbt_ctx *c, const double *tau, const double *delta, void *stream) {
  if (!c || !tau || !delta) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // page-locked arrays the device can address: one kernel reads them across
  // the host link; anything else goes bunch by bunch through the staging buffer
  cudaPointerAttributes at{}, ad{};
  const bool pinned = cudaPointerGetAttributes(&at, tau) == cudaSuccess &&
                      cudaPointerGetAttributes(&ad, delta) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      ad.type == cudaMemoryTypeHost && at.devicePointer && ad.devicePointer;
  cudaGetLastError();   // a pageable pointer leaves no error behind
  if (!pinned) {
    size_t h = 0;
    for (int m = 0; m < c->nb; ++m) {
      const mbt_status st = mbt_set_particles(c, m, tau + h, delta + h);
      if (st != MBT_OK) return st;
      h += (size_t)c->nmp[m];
    }
    return MBT_OK;
  }
  cudaError_t e = launch_load_host(c->own.plan, c->precision, static_cast<const double *>(at.devicePointer),
                                   static_cast<const double *>(ad.devicePointer), c->d_hoff, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "set particles from host");
  return MBT_OK;
}

mbt_status mbt_set_particles_all_f32(mbt_ctx *c, const float *tau, const double *delta, void *stream) {
  if (!c || !tau || !delta) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaPointerAttributes at{}, ad{};
  const bool pinned = cudaPointerGetAttributes(&at, tau) == cudaSuccess &&
                      cudaPointerGetAttributes(&ad, delta) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      ad.type == cudaMemoryTypeHost && at.devicePointer && ad.devicePointer;
  cudaGetLastError();
  if (!pinned) {
    // widened bunch by bunch (exact), then as mbt_set_particles
    std::vector<double> t;
    size_t h = 0;
    for (int m = 0; m < c->nb; ++m) {
      const size_t n = (size_t)c->nmp[m];
      t.assign(tau + h, tau + h + n);
      const mbt_status st = mbt_set_particles(c, m, t.data(), delta + h);
      if (st != MBT_OK) return st;
      h += n;
    }
    return MBT_OK;
  }
  cudaError_t e = launch_load_host_f32(c->own.plan, c->precision, static_cast<const float *>(at.devicePointer),
                                       static_cast<const double *>(ad.devicePointer), c->d_hoff, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "set particles from host");
  return MBT_OK;
}

mbt_status mbt_get_particles(mbt_ctx *c, int bunch, double *tau, double *delta) {
  if (!c || !tau || !delta) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (bunch < 0 || bunch >= c->nb) return fail(c, MBT_ERR_ARG, "bunch out of range");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const int64_t n = c->nmp[bunch];
  const bool mixed = c->precision == MBT_PREC_MIXED;
  const size_t tb = (size_t)n * (mixed ? sizeof(float) : sizeof(double));
  char *h = static_cast<char *>(stage(c, tb + (size_t)n * sizeof(double)));
  if (!h) return fail(c, MBT_ERR_NOMEM, "pinned staging buffer");
  const char *dt = static_cast<const char *>(c->d_tau) + (size_t)c->off[bunch] * (mixed ? sizeof(float) : sizeof(double));
  e = cudaMemcpy(h, dt, tb, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h + tb, c->d_delta + c->off[bunch], (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "get particles");
  if (mixed) {
    const float *tf = reinterpret_cast<const float *>(h);
    for (int64_t i = 0; i < n; ++i) tau[i] = tf[i];
  } else {
    std::memcpy(tau, h, tb);
  }
  std::memcpy(delta, h + tb, (size_t)n * sizeof(double));
  return MBT_OK;
}

// Transverse coordinates of one bunch, host doubles <-> device (float for kMixed).
static mbt_status transverse_copy(mbt_ctx *c, int bunch, double *x, double *xp, bool to_device) {
  if (!c || !x || !xp) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (!c->trans) return fail(c, MBT_ERR_STATE, "no transverse plane");
  if (bunch < 0 || bunch >= c->nb) return fail(c, MBT_ERR_ARG, "bunch out of range");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const int64_t n = c->nmp[bunch];
  const bool mixed = c->precision == MBT_PREC_MIXED;
  const size_t fs = mixed ? sizeof(float) : sizeof(double);
  char *h = static_cast<char *>(stage(c, 2 * (size_t)n * fs));
  if (!h) return fail(c, MBT_ERR_NOMEM, "pinned staging buffer");
  char *dx = static_cast<char *>(c->d_x) + (size_t)c->off[bunch] * fs;
  char *dxp = static_cast<char *>(c->d_xp) + (size_t)c->off[bunch] * fs;
  double *arrs[2] = {x, xp};
  if (to_device) {
    for (int a = 0; a < 2; ++a) {
      if (mixed) {
        float *f = reinterpret_cast<float *>(h + a * n * fs);
        for (int64_t i = 0; i < n; ++i) f[i] = (float)arrs[a][i];
      } else {
        std::memcpy(h + a * n * fs, arrs[a], (size_t)n * fs);
      }
    }
    e = cudaMemcpy(dx, h, (size_t)n * fs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dxp, h + n * fs, (size_t)n * fs, cudaMemcpyHostToDevice);
  } else {
    e = cudaMemcpy(h, dx, (size_t)n * fs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(h + n * fs, dxp, (size_t)n * fs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      for (int a = 0; a < 2; ++a) {
        if (mixed) {
          const float *f = reinterpret_cast<const float *>(h + a * n * fs);
          for (int64_t i = 0; i < n; ++i) arrs[a][i] = f[i];
        } else {
          std::memcpy(arrs[a], h + a * n * fs, (size_t)n * fs);
        }
      }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "transverse particles");
  return MBT_OK;
}

mbt_status mbt_set_transverse_particles(mbt_ctx *c, int bunch, const double *x, const double *xp) {
  return transverse_copy(c, bunch, const_cast<double *>(x), const_cast<double *>(xp), true);
}

mbt_status mbt_get_transverse_particles(mbt_ctx *c, int bunch, double *x, double *xp) {
  return transverse_copy(c, bunch, x, xp, false);
}

mbt_status mbt_set_graph(mbt_ctx *c, int turns) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (turns < 0 || turns > 100000) return fail(c, MBT_ERR_ARG, "turns_per_graph out of range");
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  c->graph_turns = turns;
  return MBT_OK;
}

mbt_status mbt_set_trace(mbt_ctx *c, int enable) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (enable && !c->d_trace) {
    const size_t bytes = (size_t)c->own.plan.njobs * 3 * sizeof(unsigned long long);
    if (cudaMalloc(&c->d_trace, bytes) != cudaSuccess) return fail(c, MBT_ERR_NOMEM, "trace buffer");
    cudaMemset(c->d_trace, 0, bytes);
  }
  c->own.plan.trace = enable ? c->d_trace : nullptr;
  return MBT_OK;
}

mbt_status mbt_read_trace(mbt_ctx *c, int64_t *out, int max_jobs, int *njobs) {
  if (!c || !njobs) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  *njobs = c->own.plan.njobs;
  if (!out || !c->d_trace) return MBT_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const int n = std::min(max_jobs, c->own.plan.njobs);
  std::vector<unsigned long long> t((size_t)n * 3);
  e = cudaMemcpy(t.data(), c->d_trace, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read trace");
  for (int j = 0; j < n; ++j) {
    const PostJob &pj = c->own.jobs[j];
    out[(size_t)j * 5 + 0] = pj.type;
    out[(size_t)j * 5 + 1] = pj.bt;
    out[(size_t)j * 5 + 2] = (int64_t)t[(size_t)j * 3 + 0];
    out[(size_t)j * 5 + 3] = (int64_t)t[(size_t)j * 3 + 1];
    out[(size_t)j * 5 + 4] = (int64_t)t[(size_t)j * 3 + 2];
  }
  return MBT_OK;
}

mbt_status mbt_set_timing(mbt_ctx *c, int enable) {
  if (!c) return MBT_ERR_ARG;
  c->timing = enable != 0;
  if (enable) {
    c->push_ms = c->post_ms = 0;
    c->timed_launches = 0;
  }
  return MBT_OK;
}

mbt_status mbt_get_timing(mbt_ctx *c, double *push_ms, double *post_ms, int64_t *launches) {
  if (!c) return MBT_ERR_ARG;
  if (push_ms) *push_ms = c->push_ms;
  if (post_ms) *post_ms = c->post_ms;
  if (launches) *launches = c->timed_launches;
  return MBT_OK;
}

// Track with an optional captured graph of `graph_turns` turns (captured on
// first use on `cap_stream`, replayed on s); remaining turns as plain launches.
static mbt_status track_plan(mbt_ctx *c, const Plan &pl, int prec, int64_t nturns, cudaStream_t s, int graph_turns,
                             cudaGraphExec_t *exec, cudaStream_t *cap_stream) {
  if (graph_turns == 0 || nturns < graph_turns) return launch_turns(c, pl, prec, nturns, s, false);
  if (!*exec) {
    if (!*cap_stream && cudaStreamCreateWithFlags(cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, MBT_ERR_CUDA, "capture stream");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(*cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
    mbt_status st = launch_turns(c, pl, prec, graph_turns, *cap_stream, false);
    e = cudaStreamEndCapture(*cap_stream, &g);
    if (st != MBT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  }
  int64_t done = 0;
  while (nturns - done >= graph_turns) {
    cudaError_t e = cudaGraphLaunch(*exec, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    done += graph_turns;
  }
  return launch_turns(c, pl, prec, nturns - done, s, false);
}

// Rebuild a context's own plan with another push tile size.
static mbt_status rebuild_own_plan(mbt_ctx *c) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  unsigned long long *trace = c->own.plan.trace;
  PlanStore &ps = c->own;
  ps.runs.clear();
  ps.bunches.clear();
  ps.tiles.clear();
  ps.jobs.clear();
  append_run(ps, c, c->tile);
  mbt_status st = upload_plan(c, ps);
  if (st != MBT_OK) return st;
  c->own.plan.trace = trace;   // the post jobs (and so the trace layout) do not depend on the tile
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  return MBT_OK;
}

mbt_status mbt_set_tile(mbt_ctx *c, int particles) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (particles < 1024 || particles > 65536 || particles % 4)
    return fail(c, MBT_ERR_ARG, "tile must be a multiple of 4 in [1024, 65536]");
  c->tile = particles;
  if (!c->filled || c->precision != MBT_PREC_MIXED) return MBT_OK;
  return rebuild_own_plan(c);
}

// Candidate push tiles for the autotuner (plans on a per-tile push, one CTA
// per tile): fixed sizes, plus "wave-aligned" sizes for which the runs' tile
// count is a whole multiple of that push kernel's resident CTA slots (no
// partly filled last wave).
static std::vector<int> tile_candidates(const std::vector<mbt_ctx *> &ctxs) {
  std::vector<int> cand = {2048, 4096, 8192, 16384, 32768};
  int slots = 0;
  bool trans = false;
  for (mbt_ctx *c : ctxs) trans = trans || c->trans;
  if (push_tile_resident_slots(trans, &slots) != cudaSuccess || slots <= 0) {
    cudaGetLastError();
    return cand;
  }
  int64_t nb = 0, nmax = 0;
  for (mbt_ctx *c : ctxs) {
    nb += c->nb;
    for (int64_t n : c->nmp) nmax = std::max(nmax, n);
  }
  for (int w = 1; w <= 12; ++w) {
    const int64_t k = (int64_t)w * slots / std::max<int64_t>(1, nb);   // tiles per bunch
    if (k < 1) continue;
    const int64_t t = ((nmax + k - 1) / k + 3) / 4 * 4;
    if (t >= 1024 && t <= 65536) cand.push_back((int)t);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  return cand;
}

mbt_status mbt_track(mbt_ctx *c, int64_t nturns, void *stream) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (nturns < 0) return fail(c, MBT_ERR_ARG, "nturns < 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Plan &pl = c->own.plan;
  if (c->timing) return launch_turns(c, pl, c->precision, nturns, s, true);
  return track_plan(c, pl, c->precision, nturns, s, c->graph_turns, &c->graph_exec, &c->capture_stream);
}

// Time `turns` turns of a plan on stream s with CUDA events [ms].
static mbt_status time_turns(mbt_ctx *c, const Plan &pl, int prec, int turns, cudaStream_t s, float *ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, MBT_ERR_CUDA, "event create");
  mbt_status st = launch_turns(c, pl, prec, 2, s, false);   // warm-up (real turns)
  cudaEventRecord(e0, s);
  if (st == MBT_OK) st = launch_turns(c, pl, prec, turns, s, false);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (st == MBT_OK && e != cudaSuccess) st = cuda_fail(c, e, "autotune timing");
  if (st == MBT_OK) cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

mbt_status mbt_autotune(mbt_ctx *c, int turns_per_trial, int *chosen_tile) {
  if (!c || turns_per_trial < 1) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (c->precision != MBT_PREC_MIXED) {
    if (chosen_tile) *chosen_tile = kF64Tile;
    return MBT_OK;
  }
  int slots = 0;
  if (push_resident_slots(&slots) == cudaSuccess &&
      plan_streams({c->n_particles}, {c->nb}, c->trans != 0, slots)) {   // split by SM: no tile to choose
    if (chosen_tile) *chosen_tile = c->tile;
    return MBT_OK;
  }
  cudaGetLastError();
  float best = 1e30f;
  int best_tile = c->tile;
  for (int tile : tile_candidates({c})) {
    c->tile = tile;
    mbt_status st = rebuild_own_plan(c);
    float ms = 0.f;
    if (st == MBT_OK) st = time_turns(c, c->own.plan, c->precision, turns_per_trial, nullptr, &ms);
    if (st != MBT_OK) return st;
    if (ms < best) {
      best = ms;
      best_tile = tile;
    }
  }
  c->tile = best_tile;
  if (chosen_tile) *chosen_tile = best_tile;
  return rebuild_own_plan(c);
}

// Cluster shape for resident tracking: the largest power-of-two cluster (<= 16
// CTAs) whose slices fit in shared memory and whose clusters can all be
// resident at once.  Returns MBT_OK with *cluster = 0 if the fill does not fit.
// The largest cluster size C <= cmax (16, 8, 4, 2, 1) whose CTAs hold the
// longest bunch in shared memory, with a cluster per bunch on the GPU at once.
static mbt_status resident_shape(mbt_ctx *c, int *cluster, int *per, size_t *smem, int cmax = 16) {
  *cluster = 0;
  int64_t nmax = 0;
  for (int64_t n : c->nmp) nmax = std::max(nmax, n);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "device query");
  for (int C = 16; C >= 1; C /= 2) {
    if (C > cmax) continue;
    const int64_t p4 = ((nmax + C - 1) / C + 3) / 4 * 4;
    const size_t sm = resident_smem_bytes((int)p4, c->nbins);
    if (sm > 220 * 1024 || (int64_t)c->nb * C > nsm) continue;
    int maxc = 0;
    e = resident_max_clusters(C, sm, &maxc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (maxc >= c->nb) {
      *cluster = C;
      *per = (int)p4;
      *smem = sm;
      return MBT_OK;
    }
  }
  return MBT_OK;
}

mbt_status mbt_resident_shape(mbt_ctx *c, int *cluster, int *per_cta) {
  if (!c || !cluster || !per_cta) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  *cluster = 0;
  *per_cta = 0;
  if (c->precision != MBT_PREC_MIXED || c->nb > kResidentMaxBunches) return MBT_OK;
  size_t sm = 0;
  return resident_shape(c, cluster, per_cta, &sm);
}

// Emission and grid-barrier buffers of resident tracking, allocated once
// (cudaMalloc may synchronise the device: never between concurrent launches)
static mbt_status resident_alloc(mbt_ctx *c) {
  if (c->d_resE) return MBT_OK;
  mbt_status st = dalloc(c, &c->d_resE, (size_t)2 * std::max(1, c->nlong) * c->nb * sizeof(double2));
  if (st == MBT_OK) st = dalloc(c, &c->d_gbar, 16);
  return st;
}

static mbt_status track_resident_impl(mbt_ctx *c, int64_t nturns, void *stream, int cmax);

mbt_status mbt_track_resident(mbt_ctx *c, int64_t nturns, void *stream) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  return track_resident_impl(c, nturns, stream, 16);
}

static mbt_status track_resident_impl(mbt_ctx *c, int64_t nturns, void *stream, int cmax) {
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (nturns < 0 || nturns > (1LL << 30)) return fail(c, MBT_ERR_ARG, "nturns out of range");
  if (nturns == 0) return MBT_OK;
  if (c->precision != MBT_PREC_MIXED)
    return fail(c, MBT_ERR_UNSUPPORTED, "resident tracking is implemented for the mixed precision path");
  if (c->trans) return fail(c, MBT_ERR_UNSUPPORTED, "resident tracking has no transverse plane");
  if (c->nb > kResidentMaxBunches)
    return fail(c, MBT_ERR_UNSUPPORTED, "resident tracking holds at most %d bunches", kResidentMaxBunches);
  int C = 0, per = 0;
  size_t sm = 0;
  mbt_status st = resident_shape(c, &C, &per, &sm, cmax);
  if (st != MBT_OK) return st;
  if (C == 0) return fail(c, MBT_ERR_UNSUPPORTED, "the fill does not fit in shared memory of co-resident clusters");
  if ((st = resident_alloc(c)) != MBT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ResidentArgs a{};
  a.plan = c->own.plan;
  a.E = c->d_resE;
  a.gbar = c->d_gbar;
  a.cluster = C;
  a.per = per;
  a.grid_sync = (c->nlong > 0 && c->nb > 1) ? 1 : 0;
  a.wait_ns = c->test_wait_ns > 0 ? (unsigned long long)c->test_wait_ns : kResidentWaitNs;
  a.extra_arrivals = c->test_unreachable ? 1u : 0u;
  const int64_t chunk = 1LL << 20;   // turns per launch (the barrier counter stays far from wrapping)
  for (int64_t done = 0; done < nturns; done += chunk) {
    a.nturns = (int)std::min<int64_t>(chunk, nturns - done);
    cudaError_t e = cudaMemsetAsync(c->d_gbar, 0, 16, s);
    if (e == cudaSuccess) e = launch_resident(a, c->nlong, c->rundev.nharm, c->nb, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "resident launch");
  }
  return MBT_OK;
}

mbt_status mbt_set_wait_test(mbt_ctx *c, int64_t limit_ns, int unreachable) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (limit_ns < 0 || limit_ns > 10000000000LL)
    return fail(c, MBT_ERR_ARG, "limit_ns must lie in [0, 1e10] (0: the default of 2 s)");
  if (unreachable != 0 && unreachable != 1) return fail(c, MBT_ERR_ARG, "unreachable must be 0 or 1");
  c->test_wait_ns = limit_ns;
  c->test_unreachable = unreachable;
  return MBT_OK;
}

mbt_status mbt_sync(mbt_ctx *c) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  if (!c->filled) return MBT_OK;
  return check_device(c, c->own.plan);
}

static mbt_status current_turn(mbt_ctx *c, long long *turn) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  e = cudaMemcpy(turn, c->d_turn, sizeof(long long), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "turn read");
  return check_device(c, c->own.plan);
}

mbt_status mbt_read_moments(mbt_ctx *c, int64_t turn0, int64_t nturns, double *out) {
  if (!c || !out) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  long long turn;
  mbt_status st = current_turn(c, &turn);
  if (st != MBT_OK) return st;
  if (turn0 < 0 || nturns < 0 || turn0 + nturns > turn || turn0 < turn - c->cap)
    return fail(c, MBT_ERR_ARG, "turns [%lld, %lld) not in the record [%lld, %lld)", (long long)turn0,
                (long long)(turn0 + nturns), (long long)std::max<long long>(0, turn - c->cap), turn);
  // at most two contiguous segments of the ring buffer
  const size_t per = (size_t)c->nb * kRecord;
  int64_t t = 0;
  while (t < nturns) {
    const int64_t slot = (turn0 + t) % c->cap;
    const int64_t len = std::min<int64_t>(nturns - t, c->cap - slot);
    cudaError_t e = cudaMemcpy(out + (size_t)t * per, c->d_rec + (size_t)slot * per, (size_t)len * per * sizeof(double),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read moments");
    t += len;
  }
  return MBT_OK;
}

mbt_status mbt_read_histograms(mbt_ctx *c, int32_t *hist, int64_t *outside) {
  if (!c || !hist) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  long long turn;
  mbt_status st = current_turn(c, &turn);
  if (st != MBT_OK) return st;
  if (turn < 1) return fail(c, MBT_ERR_STATE, "no turn tracked yet");
  const int par = (int)((turn - 1) & 1);
  const size_t n = (size_t)c->nb * c->nbins;
  cudaError_t e = cudaMemcpy(hist, c->d_hist + par * n, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "read histograms");
  if (outside) {
    std::vector<double> rec((size_t)c->nb * kRecord);
    const size_t slot = (size_t)((turn - 1) % c->cap);
    e = cudaMemcpy(rec.data(), c->d_rec + slot * rec.size(), rec.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read outside counts");
    for (int m = 0; m < c->nb; ++m) outside[m] = (int64_t)llround(rec[(size_t)m * kRecord + 5]);
  }
  return MBT_OK;
}

mbt_status mbt_read_wake(mbt_ctx *c, double *Vsr, double *Phi) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const size_t n = (size_t)c->nb * c->nbins;
  if (Vsr) {
    if (c->precision == MBT_PREC_MIXED) {
      std::vector<float> v(n);
      e = cudaMemcpy(v.data(), c->d_vsr, n * sizeof(float), cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < n; ++i) Vsr[i] = v[i];
    } else {
      e = cudaMemcpy(Vsr, c->d_vsr, n * sizeof(double), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "read wake");
  }
  if (Phi && c->nlong > 0) {
    std::vector<double2> pq((size_t)c->nlong * c->nb * 2), y((size_t)c->nlong * c->ntile_b);
    e = cudaMemcpy(pq.data(), c->d_pq, pq.size() * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(y.data(), c->d_y, y.size() * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read phasors");
    for (int r = 0; r < c->nlong; ++r)
      for (int m = 0; m < c->nb; ++m) {
        const double2 P = pq[((size_t)r * c->nb + m) * 2], Q = pq[((size_t)r * c->nb + m) * 2 + 1];
        const double2 yy = y[(size_t)r * c->ntile_b + m / kBunchTile];
        const cplx phi = cplx(P.x, P.y) * cplx(yy.x, yy.y) + cplx(Q.x, Q.y);
        Phi[((size_t)r * c->nb + m) * 2] = phi.real();
        Phi[((size_t)r * c->nb + m) * 2 + 1] = phi.imag();
      }
  }
  return MBT_OK;
}

mbt_status mbt_read_transverse_moments(mbt_ctx *c, int64_t turn0, int64_t nturns, double *out) {
  if (!c || !out) return fail(c, MBT_ERR_ARG, "null argument");
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (!c->trans) return fail(c, MBT_ERR_STATE, "no transverse plane");
  long long turn;
  mbt_status st = current_turn(c, &turn);
  if (st != MBT_OK) return st;
  if (turn0 < 0 || nturns < 0 || turn0 + nturns > turn || turn0 < turn - c->cap)
    return fail(c, MBT_ERR_ARG, "turns [%lld, %lld) not in the record", (long long)turn0, (long long)(turn0 + nturns));
  const size_t per = (size_t)c->nb * kTRecord;
  int64_t t = 0;
  while (t < nturns) {
    const int64_t slot = (turn0 + t) % c->cap;
    const int64_t len = std::min<int64_t>(nturns - t, c->cap - slot);
    cudaError_t e = cudaMemcpy(out + (size_t)t * per, c->d_trec + (size_t)slot * per,
                               (size_t)len * per * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read transverse moments");
    t += len;
  }
  return MBT_OK;
}

mbt_status mbt_read_transverse_wake(mbt_ctx *c, double *dip, double *V) {
  if (!c) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  if (!c->trans) return fail(c, MBT_ERR_STATE, "no transverse plane");
  long long turn;
  mbt_status st = current_turn(c, &turn);
  if (st != MBT_OK) return st;
  if (turn < 1) return fail(c, MBT_ERR_STATE, "no turn tracked yet");
  const size_t n = (size_t)c->nb * c->nbins;
  const int par = (int)((turn - 1) & 1);
  const bool mixed = c->precision == MBT_PREC_MIXED;
  double *outs[2] = {dip, V};
  const void *srcs[2] = {static_cast<const char *>(c->d_dip) + (size_t)par * n * 8, c->d_vt};
  for (int a = 0; a < 2; ++a) {
    if (!outs[a]) continue;
    cudaError_t e;
    if (mixed && a == 0) {   // exact fixed-point sums: q u
      std::vector<long long> q(n);
      e = cudaMemcpy(q.data(), srcs[a], n * sizeof(long long), cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < n; ++i) outs[a][i] = (double)q[i] * c->rundev.dip_unit;
    } else if (mixed) {
      std::vector<float> v(n);
      e = cudaMemcpy(v.data(), srcs[a], n * sizeof(float), cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < n; ++i) outs[a][i] = v[i];
    } else {
      e = cudaMemcpy(outs[a], srcs[a], n * sizeof(double), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "read transverse wake");
  }
  return MBT_OK;
}

mbt_status mbt_get_info(mbt_ctx *c, mbt_info *info) {
  if (!c || !info) return MBT_ERR_ARG;
  c->err.clear();
  std::memset(info, 0, sizeof *info);
  info->T_rf_s = c->T_rf;
  info->omega_rf = c->omega_rf;
  info->phi_s = c->phi_s;
  info->nu_s = c->nu_s;
  info->sigma_tau0_s = c->sigma_tau0;
  info->D = c->D;
  info->half_width_s = c->H;
  info->bin_width_s = c->Delta;
  info->n_particles = c->n_particles;
  info->nb = c->nb;
  info->nbins = c->nbins;
  info->n_long = c->nlong;
  info->precision = c->precision;
  info->device_bytes = (int64_t)(c->device_bytes + c->own.bytes);
  info->push_ctas = c->filled ? c->own.plan.stream_ctas : 0;
  info->reserved = 0;
  if (c->filled) {
    long long turn = 0;
    mbt_status st = current_turn(c, &turn);
    if (st != MBT_OK) return st;
    info->turn = turn;
  }
  return MBT_OK;
}

// --------------------------------------------------------------------------- checkpoint
namespace {
struct StateHeader {
  char magic[8];
  int32_t version, precision, nb, nbins, nlong, ntile_b;
  int64_t n_alloc;
  uint64_t seed;
};
struct Section {
  void *dev;
  size_t bytes;
};
std::vector<Section> state_sections(mbt_ctx *c) {
  const bool mixed = c->precision == MBT_PREC_MIXED;
  const int nl = std::max(1, c->nlong);
  std::vector<Section> out = {
      {c->d_tau, (size_t)c->n_alloc * (mixed ? sizeof(float) : sizeof(double))},
      {c->d_delta, (size_t)c->n_alloc * sizeof(double)},
      {c->d_hist, (size_t)2 * c->nb * c->nbins * sizeof(int32_t)},
      {c->d_vsr, (size_t)c->nb * c->nbins * (mixed ? sizeof(float) : sizeof(double))},
      {c->d_pq, (size_t)nl * c->nb * 2 * sizeof(double2)},
      {c->d_y, (size_t)nl * c->ntile_b * sizeof(double2)},
      {c->d_agg, (size_t)nl * c->ntile_b * 2 * sizeof(double2)},
      {c->d_carry, (size_t)nl * sizeof(double2)},
      {c->d_turn, 16},
  };
  if (c->trans) {
    const size_t fs = mixed ? sizeof(float) : sizeof(double);
    out.push_back({c->d_x, (size_t)c->n_alloc * fs});
    out.push_back({c->d_xp, (size_t)c->n_alloc * fs});
    out.push_back({c->d_dip, (size_t)2 * c->nb * c->nbins * 8});
    out.push_back({c->d_vt, (size_t)c->nb * c->nbins * fs});
    if (c->rw_nh > 0) out.push_back({c->d_rwcent, (size_t)(c->rw_nh + 1) * c->nb * sizeof(double)});
  }
  return out;
}
}  // namespace

mbt_status mbt_state_size(mbt_ctx *c, size_t *bytes) {
  if (!c || !bytes) return MBT_ERR_ARG;
  c->err.clear();
  if (!c->filled) return fail(c, MBT_ERR_STATE, "fill not set");
  size_t b = sizeof(StateHeader);
  for (auto &s : state_sections(c)) b += s.bytes;
  *bytes = b;
  return MBT_OK;
}

mbt_status mbt_save_state(mbt_ctx *c, void *buf, size_t bytes) {
  size_t need = 0;
  mbt_status st = mbt_state_size(c, &need);
  if (st != MBT_OK) return st;
  if (!buf || bytes < need) return fail(c, MBT_ERR_ARG, "buffer needs %zu bytes", need);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  StateHeader h{};
  std::memcpy(h.magic, "MBTSTATE", 8);
  h.version = MBT_VERSION;
  h.precision = c->precision;
  h.nb = c->nb;
  h.nbins = c->nbins;
  h.nlong = c->nlong;
  h.ntile_b = c->ntile_b;
  h.n_alloc = c->n_alloc;
  h.seed = c->seed;
  char *p = static_cast<char *>(buf);
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  for (auto &s : state_sections(c)) {
    e = cudaMemcpy(p, s.dev, s.bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "save state");
    p += s.bytes;
  }
  return MBT_OK;
}

mbt_status mbt_load_state(mbt_ctx *c, const void *buf, size_t bytes) {
  size_t need = 0;
  mbt_status st = mbt_state_size(c, &need);
  if (st != MBT_OK) return st;
  if (!buf || bytes < need) return fail(c, MBT_ERR_ARG, "buffer needs %zu bytes", need);
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "MBTSTATE", 8) != 0 || h.version != MBT_VERSION || h.precision != c->precision ||
      h.nb != c->nb || h.nbins != c->nbins || h.nlong != c->nlong || h.n_alloc != c->n_alloc || h.seed != c->seed)
    return fail(c, MBT_ERR_ARG, "snapshot does not match this context's configuration");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  const char *p = static_cast<const char *>(buf) + sizeof h;
  for (auto &s : state_sections(c)) {
    e = cudaMemcpy(s.dev, p, s.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "load state");
    p += s.bytes;
  }
  return MBT_OK;
}

// --------------------------------------------------------------------------- allocation-free wake
namespace {
std::mutex g_wna_host_mutex;
uint16_t g_wna_img[196608 / 2];      // host copy of the operand images (<= 192 KB)
float g_wna_q[kMaxBunches];

mbt_status wna_fail(char *errbuf, size_t errlen, mbt_status st, const char *fmt, ...) {
  if (errbuf && errlen) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(errbuf, errlen, fmt, ap);
    va_end(ap);
  }
  return st;
}
}  // namespace

mbt_status mbt_wake_noalloc(const mbt_ring *ring, int flags, int nres, const double *Rs_ohm, const double *fr_Hz,
                            const double *Q, const int32_t *range, int nbins, double half_width_sigmas, int nb,
                            const double *charge_per_count, const int32_t *hist, float *V, void *stream,
                            char *errbuf, size_t errlen) {
  if (errbuf && errlen) errbuf[0] = 0;
  if (!ring || !charge_per_count || !hist || !V || (nres > 0 && (!Rs_ohm || !fr_Hz || !Q || !range)))
    return wna_fail(errbuf, errlen, MBT_ERR_ARG, "null argument");
  if (!(ring->E0_eV > 0) || !(ring->T0_s > 0) || ring->h < 1 || ring->h > 65535 || ring->reserved != 0 ||
      !(ring->V_rf_V > 0) || !(ring->alpha_c != 0) || !(ring->U0_eV >= 0) || !(ring->U0_eV < ring->V_rf_V) ||
      !(ring->sigma_delta > 0) || !(ring->tau_z_s > 0))
    return wna_fail(errbuf, errlen, MBT_ERR_ARG, "invalid ring");
  if (flags & ~(MBT_NO_SR | MBT_NO_QE | MBT_KICK_NGP)) return wna_fail(errbuf, errlen, MBT_ERR_ARG, "unknown flags");
  if (nbins != 128 && nbins != 256)
    return wna_fail(errbuf, errlen, MBT_ERR_UNSUPPORTED, "nbins %d: the allocation-free wake supports 128 or 256 cells",
                    nbins);
  if (nb < 1 || nb > kMaxBunches)
    return wna_fail(errbuf, errlen, MBT_ERR_UNSUPPORTED, "nb %d: the allocation-free wake supports 1..%d bunches", nb,
                    kMaxBunches);
  if (nres < 0 || nres > kMaxRes)
    return wna_fail(errbuf, errlen, MBT_ERR_UNSUPPORTED, "nres %d: at most %d resonators", nres, kMaxRes);
  if (!(half_width_sigmas > 0)) return wna_fail(errbuf, errlen, MBT_ERR_ARG, "half width must be > 0");
  for (int i = 0; i < nres; ++i)
    if (!(Rs_ohm[i] > 0) || !(fr_Hz[i] > 0) || !(Q[i] > 0.5) || range[i] < 1 || range[i] > 3)
      return wna_fail(errbuf, errlen, MBT_ERR_ARG, "resonator %d needs Rs > 0, fr > 0, Q > 0.5, range 1..3", i);
  // the kernel reads the counts 16 bytes at a time and stores V as floats
  if (reinterpret_cast<uintptr_t>(hist) & 15u)
    return wna_fail(errbuf, errlen, MBT_ERR_ARG, "hist must be 16-byte aligned (it is read 16 bytes at a time)");
  if (reinterpret_cast<uintptr_t>(V) & 3u) return wna_fail(errbuf, errlen, MBT_ERR_ARG, "V must be 4-byte aligned");
  // synchronous (it waits for the stream and reads the error word back), so
  // it cannot be recorded into a CUDA graph
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(cs, &cap);
  if (ce != cudaSuccess)
    return wna_fail(errbuf, errlen, MBT_ERR_CUDA, "allocation-free wake: %s", cudaGetErrorString(ce));
  if (cap != cudaStreamCaptureStatusNone)
    return wna_fail(errbuf, errlen, MBT_ERR_STATE, "the stream is being captured: the allocation-free wake is "
                    "synchronous and cannot be captured");

  std::lock_guard<std::mutex> lk(g_wna_host_mutex);
  mbt_ctx g;   // grid constants only: no device state
  g.ring = *ring;
  g.flags = flags;
  g.nbins = nbins;
  g.half_width_sigmas = half_width_sigmas;
  derive(&g);
  double lag[256];
  for (int l = 0; l < nbins; ++l) {
    lag[l] = 0.0;
    for (int i = 0; i < nres; ++i)
      if (range[i] & MBT_RANGE_SHORT) lag[l] += wake(Resonator{Rs_ohm[i], fr_Hz[i], Q[i], range[i]}, (double)l * g.Delta);
  }
  const size_t base = pack_toeplitz_images(lag, nbins, g_wna_img);
  for (int m = 0; m < nb; ++m) g_wna_q[m] = (float)charge_per_count[m];
  RunDev proto{};
  int derr = 0;
  cudaError_t e = wake_noalloc_launch(proto, g_wna_img, base, g_wna_q, nb, nbins, hist, V, cs, &derr);
  if (e != cudaSuccess) return wna_fail(errbuf, errlen, MBT_ERR_CUDA, "allocation-free wake: %s", cudaGetErrorString(e));
  if (derr == kErrCount)
    return wna_fail(errbuf, errlen, MBT_ERR_ARG, "a cell count lies outside [0, 2^24): V is not valid");
  if (derr == kErrTmem) return wna_fail(errbuf, errlen, MBT_ERR_CUDA, "tensor memory could not be allocated");
  if (derr != 0) return wna_fail(errbuf, errlen, MBT_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", derr);
  return MBT_OK;
}

// --------------------------------------------------------------------------- batch
mbt_status mbt_batch_create(mbt_ctx *const *ctxs, int n, mbt_batch **out) {
  if (!ctxs || n < 1 || !out) return MBT_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->filled) return MBT_ERR_STATE;
    if (ctxs[i]->precision != ctxs[0]->precision) return MBT_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return MBT_ERR_ARG;
  }
  mbt_batch *b = new (std::nothrow) mbt_batch();
  if (!b) return MBT_ERR_NOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  b->precision = ctxs[0]->precision;
  b->store.precision = b->precision;
  for (int i = 0; i < n; ++i) append_run(b->store, ctxs[i], b->tile);
  mbt_status st = upload_plan(ctxs[0], b->store);
  if (st != MBT_OK) {
    delete b;
    return st;
  }
  *out = b;
  return MBT_OK;
}

mbt_status mbt_batch_track(mbt_batch *b, int64_t nturns, void *stream) {
  if (!b || nturns < 0) return MBT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->lanes.empty())
    return track_plan(b->ctx[0], b->store.plan, b->precision, nturns, s, b->graph_turns, &b->graph_exec,
                      &b->capture_stream);
  // every lane forked from `stream`, tracked on its own stream, joined back
  mbt_ctx *c0 = b->ctx[0];
  cudaError_t e = cudaEventRecord(b->lane_fork, s);
  if (e != cudaSuccess) return cuda_fail(c0, e, "lane fork");
  for (auto &L : b->lanes) {
    e = cudaStreamWaitEvent(L->stream, b->lane_fork, 0);
    if (e != cudaSuccess) return cuda_fail(c0, e, "lane fork");
  }
  // the lanes' launches interleaved a graph (or a chunk of turns) at a time,
  // so that no lane's queue fills up before the next lane has work queued
  mbt_status first = MBT_OK;
  const int64_t chunk = b->graph_turns > 0 ? b->graph_turns : 64;
  for (int64_t done = 0; done < nturns && first == MBT_OK; done += chunk) {
    const int64_t n = std::min(chunk, nturns - done);
    for (auto &L : b->lanes) {
      const mbt_status st = track_plan(b->ctx[(size_t)L->members[0]], L->store.plan, b->precision, n, L->stream,
                                       b->graph_turns, &L->graph_exec, &L->capture_stream);
      if (st != MBT_OK) {
        first = st;
        if (L->members[0] != 0) fail(c0, st, "%s", b->ctx[(size_t)L->members[0]]->err.c_str());
        break;
      }
    }
  }
  for (auto &L : b->lanes) {
    // joined even after a failed launch, so that `stream` orders after what did start
    e = cudaEventRecord(L->done, L->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, L->done, 0);
    if (e != cudaSuccess && first == MBT_OK) first = cuda_fail(c0, e, "lane join");
  }
  return first;
}

// Members into k lanes of about equal particle counts: largest first, each
// to the lane with the fewest particles so far (ties: the lower lane);
// members keep their batch order within a lane.
static std::vector<std::vector<int>> lane_partition(const std::vector<int64_t> &n, int k) {
  std::vector<int> order(n.size());
  for (size_t i = 0; i < n.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[(size_t)a] > n[(size_t)b]; });
  std::vector<int64_t> load((size_t)k, 0);
  std::vector<std::vector<int>> lanes((size_t)k);
  for (int i : order) {
    const size_t j = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[j].push_back(i);
    load[j] += n[(size_t)i];
  }
  for (auto &l : lanes) std::sort(l.begin(), l.end());
  return lanes;
}

// (Re)build the lanes' plans with the batch's push tile.
static mbt_status build_lanes(mbt_batch *b) {
  mbt_ctx *c0 = b->ctx[0];
  b->lanes.clear();
  if (b->nlanes <= 1) return MBT_OK;
  if (!b->lane_fork && cudaEventCreateWithFlags(&b->lane_fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(c0, MBT_ERR_CUDA, "lane event");
  std::vector<int64_t> n;
  for (const mbt_ctx *c : b->ctx) n.push_back(c->n_particles);
  for (const std::vector<int> &members : lane_partition(n, b->nlanes)) {
    std::unique_ptr<BatchLane> L(new (std::nothrow) BatchLane());
    if (!L) return fail(c0, MBT_ERR_NOMEM, "lane");
    L->members = members;
    L->store.precision = b->precision;
    for (int i : members) append_run(L->store, b->ctx[(size_t)i], b->tile);
    mbt_status st = upload_plan(b->ctx[(size_t)members[0]], L->store);
    if (st != MBT_OK) {
      if (members[0] != 0) fail(c0, st, "%s", b->ctx[(size_t)members[0]]->err.c_str());
      b->lanes.clear();
      return st;
    }
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      b->lanes.clear();
      return fail(c0, MBT_ERR_CUDA, "lane stream");
    }
    b->lanes.push_back(std::move(L));
  }
  return MBT_OK;
}

mbt_status mbt_batch_set_lanes(mbt_batch *b, int nlanes) {
  if (!b) return MBT_ERR_ARG;
  mbt_ctx *c0 = b->ctx[0];
  c0->err.clear();
  if (nlanes < 1 || nlanes > kMaxLanes) return fail(c0, MBT_ERR_ARG, "lanes must be 1..%d", kMaxLanes);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c0, e, "sync");
  b->nlanes = std::min(nlanes, (int)b->ctx.size());
  return build_lanes(b);
}

mbt_status mbt_batch_set_graph(mbt_batch *b, int turns) {
  if (!b || turns < 0 || turns > 100000) return MBT_ERR_ARG;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    b->graph_exec = nullptr;
  }
  for (auto &L : b->lanes)
    if (L->graph_exec) {
      cudaGraphExecDestroy(L->graph_exec);
      L->graph_exec = nullptr;
    }
  b->graph_turns = turns;
  return MBT_OK;
}

static mbt_status rebuild_batch_plan(mbt_batch *b) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(b->ctx[0], e, "sync");
  b->store.runs.clear();
  b->store.bunches.clear();
  b->store.tiles.clear();
  b->store.jobs.clear();
  for (mbt_ctx *c : b->ctx) append_run(b->store, c, b->tile);
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    b->graph_exec = nullptr;
  }
  mbt_status st = upload_plan(b->ctx[0], b->store);
  return st == MBT_OK ? build_lanes(b) : st;
}

mbt_status mbt_batch_autotune(mbt_batch *b, int turns_per_trial, int *chosen_tile) {
  if (!b || turns_per_trial < 1) return MBT_ERR_ARG;
  if (b->precision != MBT_PREC_MIXED) {
    if (chosen_tile) *chosen_tile = kF64Tile;
    return MBT_OK;
  }
  bool any_trans = false;
  std::vector<int64_t> n;
  std::vector<int> nb;
  for (mbt_ctx *c : b->ctx) {
    any_trans = any_trans || c->trans;
    n.push_back(c->n_particles);
    nb.push_back(c->nb);
  }
  int slots = 0;
  if (push_resident_slots(&slots) == cudaSuccess && plan_streams(n, nb, any_trans, slots)) {
    if (chosen_tile) *chosen_tile = b->tile;   // split by SM: no tile to choose
    return MBT_OK;
  }
  cudaGetLastError();
  float best = 1e30f;
  int best_tile = b->tile;
  for (int tile : tile_candidates(b->ctx)) {
    b->tile = tile;
    mbt_status st = rebuild_batch_plan(b);
    float ms = 0.f;
    if (st == MBT_OK) st = time_turns(b->ctx[0], b->store.plan, b->precision, turns_per_trial, nullptr, &ms);
    if (st != MBT_OK) return st;
    if (ms < best) {
      best = ms;
      best_tile = tile;
    }
  }
  b->tile = best_tile;
  if (chosen_tile) *chosen_tile = best_tile;
  return rebuild_batch_plan(b);
}

// Lane-count autotuning: each count from 1 to max_lanes tracked for a
// warm-up and a timed trial of turns_per_trial turns (real turns; graph
// replay where the batch's graph setting covers the trial), the fastest kept.
mbt_status mbt_batch_autotune_lanes(mbt_batch *b, int turns_per_trial, int max_lanes, int *chosen) {
  if (!b || turns_per_trial < 1 || max_lanes < 1 || max_lanes > kMaxLanes) return MBT_ERR_ARG;
  mbt_ctx *c0 = b->ctx[0];
  c0->err.clear();
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    return fail(c0, MBT_ERR_CUDA, "autotune stream");
  }
  const int top = std::min(max_lanes, (int)b->ctx.size());
  float best = 1e30f;
  int best_k = 1;
  mbt_status st = MBT_OK;
  for (int k = 1; k <= top && st == MBT_OK; ++k) {
    st = mbt_batch_set_lanes(b, k);
    if (st == MBT_OK) st = mbt_batch_track(b, turns_per_trial, s);   // warm-up (captures the lanes' graphs)
    if (st != MBT_OK) break;
    cudaEventRecord(e0, s);
    st = mbt_batch_track(b, turns_per_trial, s);
    cudaEventRecord(e1, s);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (st == MBT_OK && e != cudaSuccess) st = cuda_fail(c0, e, "autotune timing");
    float ms = 0.f;
    if (st == MBT_OK) cudaEventElapsedTime(&ms, e0, e1);
    if (st == MBT_OK && ms < best) {
      best = ms;
      best_k = k;
    }
  }
  if (st == MBT_OK) st = mbt_batch_set_lanes(b, best_k);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (st == MBT_OK && chosen) *chosen = best_k;
  return st;
}

mbt_status mbt_batch_sync(mbt_batch *b) {
  if (!b) return MBT_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(b->ctx[0], e, "sync");
  mbt_status st = check_device(b->ctx[0], b->store.plan);
  for (size_t i = 0; i < b->lanes.size() && st == MBT_OK; ++i) st = check_device(b->ctx[0], b->lanes[i]->store.plan);
  // the members' own error words (their resident kernels, mbt_batch_track_resident)
  for (size_t i = 0; i < b->ctx.size() && st == MBT_OK; ++i) {
    st = check_device(b->ctx[i], b->ctx[i]->own.plan);
    if (st != MBT_OK && i > 0) fail(b->ctx[0], st, "member %zu: %s", i, b->ctx[i]->err.c_str());
  }
  return st;
}

void mbt_batch_destroy(mbt_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (cudaStream_t st : b->res_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->res_events) cudaEventDestroy(ev);
  b->lanes.clear();
  if (b->lane_fork) cudaEventDestroy(b->lane_fork);
  delete b;
}

// Each member's resident kernel on a stream of its own, all forked from and
// joined back into `stream`.  Members run concurrently only because no
// cluster of theirs waits for another cluster (one bunch per member, or no
// long-range resonator): a member whose clusters meet in a grid barrier
// needs all of them co-resident, which kernels sharing the GPU cannot
// promise, so such a batch is refused before any launch.
mbt_status mbt_batch_track_resident(mbt_batch *b, int64_t nturns, void *stream) {
  if (!b || nturns < 0) return MBT_ERR_ARG;
  mbt_ctx *c0 = b->ctx[0];
  c0->err.clear();
  if (nturns == 0) return MBT_OK;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    mbt_ctx *c = b->ctx[i];
    if (!c->filled) return fail(c0, MBT_ERR_STATE, "member %zu: fill not set", i);
    if (c->precision != MBT_PREC_MIXED || c->trans || c->nb > kResidentMaxBunches)
      return fail(c0, MBT_ERR_UNSUPPORTED, "member %zu cannot be tracked resident", i);
    if (c->nlong > 0 && c->nb > 1)
      return fail(c0, MBT_ERR_UNSUPPORTED,
                  "member %zu couples several bunches over long range: its clusters meet every turn and it "
                  "must be tracked resident alone", i);
    int C = 0, per = 0;
    size_t sm = 0;
    mbt_status st = resident_shape(c, &C, &per, &sm);
    if (st != MBT_OK) return fail(c0, st, "member %zu: %s", i, c->err.c_str());
    if (C == 0) return fail(c0, MBT_ERR_UNSUPPORTED, "member %zu does not fit in shared memory", i);
    if ((st = resident_alloc(c)) != MBT_OK) return fail(c0, st, "member %zu: %s", i, c->err.c_str());
  }
  // the largest cluster-size cap at which every member's clusters fit on the
  // SMs together (one resident CTA per SM); else each member's own shape
  int dev = 0, nsm = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e0 != cudaSuccess) return cuda_fail(c0, e0, "device query");
  // (a cluster occupies SMs of one GPC, so the count of clusters the GPU
  // holds at once comes from the occupancy query, not from the SM count)
  int cmax = 16;
  for (int cap = 16; cap >= 1; cap /= 2) {
    int64_t ctas = 0, clusters = 0;
    size_t sm_max = 0;
    bool fits = true;
    for (mbt_ctx *c : b->ctx) {
      int C = 0, per = 0;
      size_t sm = 0;
      if (resident_shape(c, &C, &per, &sm, cap) != MBT_OK || C == 0) {
        fits = false;
        break;
      }
      ctas += (int64_t)C * c->nb;
      clusters += c->nb;
      sm_max = std::max(sm_max, sm);
    }
    if (!fits) break;
    int maxc = 0;
    if (resident_max_clusters(cap, sm_max, &maxc) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ctas <= nsm && clusters <= maxc) {
      cmax = cap;
      break;
    }
  }
  if (b->res_streams.empty()) {
    for (size_t i = 0; i <= b->ctx.size(); ++i) {
      cudaEvent_t ev = nullptr;
      cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(c0, e, "event");
      b->res_events.push_back(ev);
    }
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      cudaStream_t st = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(c0, e, "stream");
      b->res_streams.push_back(st);
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(b->res_events[0], s);
  if (e != cudaSuccess) return cuda_fail(c0, e, "fork");
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    e = cudaStreamWaitEvent(b->res_streams[i], b->res_events[0], 0);
    if (e != cudaSuccess) return cuda_fail(c0, e, "fork");
    b->ctx[i]->err.clear();
    mbt_status st = track_resident_impl(b->ctx[i], nturns, b->res_streams[i], cmax);
    if (st != MBT_OK) return fail(c0, st, "member %zu: %s", i, b->ctx[i]->err.c_str());
    e = cudaEventRecord(b->res_events[1 + i], b->res_streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->res_events[1 + i], 0);
    if (e != cudaSuccess) return cuda_fail(c0, e, "join");
  }
  return MBT_OK;
}

mbt_status mbt_plan_streams(int nruns, const int64_t *run_n, const int32_t *run_nb, int any_transverse, int ctas,
                            int *streams) {
  if (nruns < 1 || !run_n || !run_nb || ctas < 1 || !streams) return MBT_ERR_ARG;
  std::vector<int64_t> n(run_n, run_n + nruns);
  std::vector<int> nb(run_nb, run_nb + nruns);
  for (int i = 0; i < nruns; ++i)
    if (n[(size_t)i] < 1 || nb[(size_t)i] < 1) return MBT_ERR_ARG;
  *streams = plan_streams(n, nb, any_transverse != 0, ctas) ? 1 : 0;
  return MBT_OK;
}

mbt_status mbt_plan_lanes(int nmembers, const int64_t *n_particles, int nlanes, int32_t *lane) {
  if (nmembers < 1 || !n_particles || !lane || nlanes < 1 || nlanes > kMaxLanes) return MBT_ERR_ARG;
  std::vector<int64_t> n((size_t)nmembers);
  for (int i = 0; i < nmembers; ++i) {
    if (n_particles[i] < 0) return MBT_ERR_ARG;
    n[(size_t)i] = n_particles[i];
  }
  const std::vector<std::vector<int>> lanes = lane_partition(n, std::min(nlanes, nmembers));
  for (size_t j = 0; j < lanes.size(); ++j)
    for (int i : lanes[j]) lane[i] = (int32_t)j;
  return MBT_OK;
}

mbt_status mbt_plan_stream_split(int nb, const int32_t *run, const int64_t *n_mp, int ctas, int64_t *out,
                                 int64_t cap, int64_t *ntiles) {
  if (nb < 1 || !run || !n_mp || ctas < 1 || !ntiles || cap < 0 || (cap > 0 && !out)) return MBT_ERR_ARG;
  std::vector<int> brun((size_t)nb);
  std::vector<int64_t> bn((size_t)nb);
  for (int i = 0; i < nb; ++i) {
    if (n_mp[i] < 1 || run[i] < 0 || (i > 0 && run[i] < run[i - 1])) return MBT_ERR_ARG;
    brun[(size_t)i] = run[i];
    bn[(size_t)i] = n_mp[i];
  }
  const std::vector<SplitTile> t = stream_split(brun, bn, ctas);
  *ntiles = (int64_t)t.size();
  for (size_t k = 0; k < t.size() && (int64_t)k < cap; ++k) {
    out[4 * k + 0] = t[k].bunch;
    out[4 * k + 1] = t[k].start;
    out[4 * k + 2] = t[k].count;
    out[4 * k + 3] = t[k].cta;
  }
  return MBT_OK;
}

}  // extern "C"
