// Push kernels: one CTA per tile of one bunch.  Per particle and turn
// (arXiv:1809.00391 Sec. 2.2-2.3, readings listed in mbt.h):
//   wake kick with the previous turn's short-range voltage (interpolated
//   between cell centres) and long-range phasors (Eq. 6),
//   RF gain minus mean radiation loss (Eq. 1),
//   radiation damping and quantum excitation with Philox normals (Eq. 5),
//   drift with the new energy deviation (Eq. 2),
//   deposit into a shared-memory histogram, moment partial sums (Sec. 2.4).
// The histogram is flushed to global memory with one atomic per non-empty
// cell; the moment partials go to a per-tile slot (deterministic sums).
#include <algorithm>
#include <climits>
#include <mutex>

#include "push_core.cuh"

namespace mbt {

// ---------------------------------------------------------------------------
// Mixed precision: tau in FP32, delta stored and accumulated in FP64 (one
// DFMA per particle), everything else in FP32 on the FMA / MUFU pipes.  Each
// thread handles quads of 4 consecutive particles, one Philox block per
// quad.  NLONG_MAX bounds the number of long-range resonators of any run in
// the plan.
// ---------------------------------------------------------------------------
// The particle stream is staged through shared memory by the TMA bulk-copy
// engine: chunks of kChunk particles (tau 4 KB + delta 8 KB) in a
// kStages-deep ring, refilled by one thread as soon as the CTA has consumed a
// stage.  Thread t handles the quad of particles 4t .. 4t+3 of each chunk
// (one Philox block, two Box-Muller pairs); results are stored straight to
// global memory with 16-byte stores.
#ifndef MBT_PUSH_STAGES
#define MBT_PUSH_STAGES 2
#endif
#ifndef MBT_PUSH_MIN_BLOCKS
#define MBT_PUSH_MIN_BLOCKS 6
#endif
constexpr int kChunk = 1024;
constexpr int kStages = MBT_PUSH_STAGES;
static_assert(kStages >= 2, "the stage being refilled must differ from the next one read");
// Per-tile push CTA shapes (runs without a transverse plane): 256 threads x 6
// CTAs per SM, or for plans of many waves of small tiles 128 threads x 12
// (measured: the L5 scan's 21 175 tiles of 5000 particles 594 -> 549 us per
// turn; single-wave plans lose: 24.5 -> 29.8 us on the resistive-wall scan).
template <int THREADS>
struct LShape {
  static constexpr int kChunk = 4 * THREADS;   // particles per stage: one quad per thread
  static constexpr int kStageBytes = kChunk * (int)(sizeof(float) + sizeof(double));
  static constexpr int kMinBlocks = THREADS == 256 ? MBT_PUSH_MIN_BLOCKS : 12;
};
constexpr unsigned long long kPushWaitNs = 2000000000ull;

// Per-tile push (plans with small runs or small bunches: the streaming push
// below needs a share of several stages per SM to fill its lanes): one CTA
// per tile of one bunch, six CTAs per SM; the hardware hands a finished CTA's
// slot to the next tile.
template <int THREADS>
__device__ __forceinline__ void issue_chunk(const TileDev &t, const float *tau, const double *del, uint8_t *stage,
                                            uint64_t *bar, int c) {
  constexpr int kChunkL = LShape<THREADS>::kChunk;
  const int n = min(kChunkL, t.count - c * kChunkL);
  const int n4 = (n + 3) & ~3;   // segments are padded to 4 particles: 16-byte multiples
  const uint32_t tb = (uint32_t)n4 * 4u, db = (uint32_t)n4 * 8u;
  mbar_arrive_expect_tx(bar, tb + db);
  bulk_g2s(stage, tau + (size_t)c * kChunkL, tb, bar);
  bulk_g2s(stage + kChunkL * sizeof(float), del + (size_t)c * kChunkL, db, bar);
}

template <int NLONG_MAX, bool HARM, int THREADS>
__global__ void __launch_bounds__(THREADS, LShape<THREADS>::kMinBlocks) k_push_mixed(const Plan p) {
  constexpr int kLThreads = THREADS, kChunkL = LShape<THREADS>::kChunk, kStageBytesL = LShape<THREADS>::kStageBytes;
  extern __shared__ __align__(128) uint8_t sm_push[];
  // The moment partials are summed as the 256-thread layout sums them, in
  // either shape, so that a run's moments do not depend on the shape its plan
  // chose: per 256-layout thread over its quads in chunk order, a warp tree,
  // the 8 warps in order.  A 128-thread CTA's thread t holds two of those
  // threads, t (its even chunks) and t + 128 (its odd chunks).
  constexpr int kVW = 8;
  static_assert(THREADS == 256 || THREADS == 128, "per-tile push CTA shapes");
  __shared__ float s_red[kVW][5];
  __shared__ float2 s_phi[kMaxLong];
  __shared__ float4 s_hc[kMaxHarm];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int s_abort;

  // Prologue that reads only the plan and the particle state: with
  // programmatic dependent launch it overlaps the previous post kernel, which
  // signals its dependents only after the previous push has completed.
  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  PushConstF c;
  c.nbins = R->nbins;
  const int nbins = c.nbins;
  const int nlong = R->nlong;
  uint8_t *stages = sm_push;
  float2 *sVd = reinterpret_cast<float2 *>(sm_push + kStages * kStageBytesL);   // (V[j], V[j+1] - V[j])
  int *sH = reinterpret_cast<int *>(sVd + nbins);
  float *tau = static_cast<float *>(R->tau) + bd.off + t.start;
  double *del = R->delta + bd.off + t.start;
  const int nchunks = (t.count + kChunkL - 1) / kChunkL;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&full[st], 1);
    fence_mbar_init();
    s_abort = 0;
    for (int ch = 0; ch < min(kStages, nchunks); ++ch) issue_chunk<THREADS>(t, tau, del, stages + ch * kStageBytesL, &full[ch], ch);
  }
  const int nharm = R->nharm;
  if (threadIdx.x < nharm) s_hc[threadIdx.x] = R->f_harm[threadIdx.x];
  grid_dependents_launch();
  grid_dependency_wait();   // the previous post kernel's wake, phasors and turn counter are complete
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);
  const float *vsr = static_cast<const float *>(R->vsr) + (size_t)t.m * nbins;
  for (int k = threadIdx.x; k < nbins; k += kLThreads) {
    const float v0 = vsr[k];
    const float v1 = k + 1 < nbins ? vsr[k + 1] : v0;
    sVd[k] = make_float2(v0, v1 - v0);
    sH[k] = 0;
  }
  if (threadIdx.x < nlong) {
    // Phi_m = P_m y_tile + Q_m of this bunch, narrowed to FP32
    const int r = threadIdx.x;
    const double2 P = R->pq[((size_t)r * R->nb + t.m) * 2];
    const double2 Q = R->pq[((size_t)r * R->nb + t.m) * 2 + 1];
    const double2 y = R->y[(size_t)r * R->ntile_b + t.m / kBunchTile];
    const double2 phi = cfma(P, y, Q);
    s_phi[r] = make_float2((float)phi.x, (float)phi.y);
  }
  c.invD = R->f_invD;
  c.HinvD = R->f_HinvD;
  c.fnb = R->f_nbins;
  c.invE0 = R->f_invE0 * R->f_omD;
  c.rfA = R->f_rfA;
  c.rfB = R->f_rfB;
  c.w = R->f_w;
  c.omD = R->f_omD;
  c.qe = R->f_qe;
  c.aT0 = R->f_aT0;
  const double omD_d = R->one_minus_D;
  const bool ngp = (R->flags & kKickNGP) != 0;
  float la[NLONG_MAX > 0 ? NLONG_MAX : 1], lw[NLONG_MAX > 0 ? NLONG_MAX : 1];
  float2 phi[NLONG_MAX > 0 ? NLONG_MAX : 1];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < NLONG_MAX; ++r) {
    la[r] = R->f_la[r];
    lw[r] = R->f_lw[r];
    phi[r] = r < nlong ? s_phi[r] : make_float2(0.f, 0.f);
  }
  const uint32_t k0 = R->key0, k1 = R->key1, turn32 = (uint32_t)turn, bunch32 = (uint32_t)t.m;
  float tref = 0.f, dref = 0.f;   // moment reference: the tile's first particle before the push

  float st = 0.f, st2 = 0.f, sd = 0.f, sd2 = 0.f;      // this thread's (even chunks)
  float st_b = 0.f, st2_b = 0.f, sd_b = 0.f, sd2_b = 0.f;  // THREADS == 128: thread t + 128's (odd chunks)
  int nout = 0;
  auto chunk = [&](int ch, float &st, float &st2, float &sd, float &sd2) {
    const int slot = ch % kStages;
    uint8_t *sg = stages + slot * kStageBytesL;
    if (!mbar_wait_bounded(&full[slot], (uint32_t)((ch / kStages) & 1), kPushWaitNs)) {
      atomicExch(p.error, kErrTimeout);
      s_abort = 1;
    }
    if (ch == 0) {
      tref = reinterpret_cast<const float *>(sg)[0];
      dref = f64_to_f32_ref(reinterpret_cast<const double *>(sg + kChunkL * sizeof(float))[0]);
    }
    const int q = ch * kChunkL + 4 * (int)threadIdx.x;   // first particle of this thread's quad in the tile
    if (!s_abort && q < t.count) {
      const float4 tv = reinterpret_cast<const float4 *>(sg)[threadIdx.x];
      const double2 da = reinterpret_cast<const double2 *>(sg + kChunkL * sizeof(float))[2 * threadIdx.x];
      const double2 db = reinterpret_cast<const double2 *>(sg + kChunkL * sizeof(float))[2 * threadIdx.x + 1];
      float rr[4] = {0.f, 0.f, 0.f, 0.f};
      if (c.qe != 0.f) normal_quad_f32(philox4x32_10((uint32_t)((t.start + q) >> 2), bunch32, turn32, 0u, k0, k1), rr);
      float tt[4] = {tv.x, tv.y, tv.z, tv.w};
      double dd[4] = {da.x, da.y, db.x, db.y};
      const int nvalid = min(4, t.count - q);
      if (ngp)
        quad_push<NLONG_MAX, true, HARM>(c, sVd, sH, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid, tref,
                                         dref, st, st2, sd, sd2, nout);
      else
        quad_push<NLONG_MAX, false, HARM>(c, sVd, sH, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid, tref,
                                          dref, st, st2, sd, sd2, nout);
      *reinterpret_cast<float4 *>(tau + q) = make_float4(tt[0], tt[1], tt[2], tt[3]);
      *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
      *reinterpret_cast<double2 *>(del + q + 2) = make_double2(dd[2], dd[3]);
    }
    __syncthreads();   // stage `slot` consumed by every thread
    if (threadIdx.x == 0 && !s_abort && ch + kStages < nchunks) {
      fence_proxy_async_smem();   // order the generic-proxy reads of the stage before its refill
      issue_chunk<THREADS>(t, tau, del, sg, &full[slot], ch + kStages);
    }
  };
#pragma unroll 1
  for (int ch = 0; ch < nchunks; ch += (THREADS == 128 ? 2 : 1)) {
    chunk(ch, st, st2, sd, sd2);
    if (THREADS == 128 && ch + 1 < nchunks) chunk(ch + 1, st_b, st2_b, sd_b, sd2_b);
  }
  if (s_abort && threadIdx.x == 0) {
    // let the copies still in flight land before the CTA exits
    for (int ch = 0; ch < nchunks; ++ch) mbar_wait_bounded(&full[ch % kStages], (uint32_t)((ch / kStages) & 1), kPushWaitNs);
  }

  // moment partials: FP32 within a warp, FP64 across the (256-layout) warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
  auto hand_in = [&](float a, float a2, float b, float b2, int vw, float n) {
    a = warp_sum_f(a);
    a2 = warp_sum_f(a2);
    b = warp_sum_f(b);
    b2 = warp_sum_f(b2);
    if (lane == 0) {
      s_red[vw][0] = a;
      s_red[vw][1] = a2;
      s_red[vw][2] = b;
      s_red[vw][3] = b2;
      s_red[vw][4] = n;   // counts are exact in any split
    }
  };
  hand_in(st, st2, sd, sd2, warp, (float)no);
  if (THREADS == 128) hand_in(st_b, st2_b, sd_b, sd2_b, warp + 4, 0.f);
  __syncthreads();
  if (threadIdx.x < 5) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kVW; ++w) acc += (double)s_red[w][threadIdx.x];
    p.partial[(size_t)blockIdx.x * kPartials + threadIdx.x] = acc;
  } else if (threadIdx.x == 5) {
    double *pp = p.partial + (size_t)blockIdx.x * kPartials;
    pp[5] = (double)tref;
    pp[10] = (double)dref;
    pp[11] = (double)t.count;
  }
  int32_t *hg = R->hist + ((size_t)par * R->nb + t.m) * nbins;
  for (int k = threadIdx.x; k < nbins; k += kLThreads) {
    const int cnt = sH[k];
    if (cnt) atomicAdd(hg + k, cnt);
  }
}

// ---------------------------------------------------------------------------
// Streaming push (runs without a transverse plane): one persistent CTA of
// kStreamThreads threads per SM, so that no CTA is launched, set up and
// retired per tile, and no CTA of the push competes with another for an SM's
// issue slots (with several resident CTAs the warp schedulers starve some of
// them for the whole launch).  The plan cuts each run's particle sequence
// into one equal share per SM (tiles at bunch boundaries) and CTA g takes
// share g of every run; the SMs run at the same rate, so the shares end
// together.
//
// Warp specialised: the last warp feeds a ring of kStreamStages stages of
// kStreamChunk particles with bulk copies (full barriers), and requests each
// tile's descriptor, kick table, phasor inputs and turn counter a tile ahead
// (slot barriers) with an L1 prefetch of the run constants; the other warps
// consume.  A consumer warp hands its part of a stage back (empty barrier) as
// soon as it has read it, so the warps are not held together chunk by chunk;
// they meet (named barrier) only at tile boundaries, to hand in the tile's
// histogram and partial sums and build the next tile's tables.  The run
// constants are read with read-only loads that the compiler may repeat
// instead of holding them in registers.  Every tile keeps its own
// partial-sum slot, so the moments do not depend on the split.
// ---------------------------------------------------------------------------
constexpr int kStreamThreads = 1024;
constexpr int kConsumerWarps = kStreamThreads / 32 - 1;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kStreamChunk = kConsumers * 4;   // particles per stage: one quad per consumer thread
constexpr int kStreamStageBytes = kStreamChunk * (int)(sizeof(float) + sizeof(double));
#ifndef MBT_STREAM_STAGES
#define MBT_STREAM_STAGES 3
#endif
constexpr int kStreamStages = MBT_STREAM_STAGES;
constexpr int kStreamMaxBins = 256;   // kMixed meshes have 128 or 256 cells
constexpr int kSlots = 3;             // tile slots: the consumers' tile and two ahead
constexpr int kProducerTid = kConsumers;

struct alignas(16) StreamSlot {
  StreamTile td;                 // descriptor (bulk copy, barrier tdb)
  long long turn[2];             // turn counter  } barrier thb
  double2 pq[kMaxLong][2];       // P_m, Q_m      }
  double2 y[kMaxLong];           // y of the tile }
  float vrow[kStreamMaxBins];    // short-range voltage of the bunch
};
constexpr size_t kStreamSmem = (size_t)kStreamStages * kStreamStageBytes + kSlots * sizeof(StreamSlot) +
                               kStreamMaxBins * sizeof(float2) + (kStreamMaxBins + kSpillCells) * sizeof(int);

struct StreamSmem {
  uint64_t full[kStreamStages], empty[kStreamStages];   // stage loaded / handed back by every consumer warp
  uint64_t tdb[kSlots], thb[kSlots], freed[kSlots];      // slot descriptor / data arrived, slot set up by the consumers
  int issued_full[kStreamStages], issued_tdb[kSlots], issued_thb[kSlots];   // phases issued (producer, for draining)
  float red[kConsumerWarps][5];      // per-warp sums of a tile
  float2 phi[kMaxLong];
};


__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(kConsumers) : "memory");
}

// Producer: a tile's kick data (written by the previous post kernel, so only
// after the grid dependency wait), and an L1 prefetch of its run constants.
__device__ __forceinline__ void stream_issue_data(StreamSmem &S, StreamSlot &D, int sl) {
  const StreamTile &td = D.td;
  const int nl = min(td.nlong, kMaxLong), nbins = min(td.nbins, kStreamMaxBins);
  mbar_arrive_expect_tx(&S.thb[sl], (uint32_t)(16 + nl * 48 + nbins * 4));
  bulk_g2s(D.turn, td.turn, 16u, &S.thb[sl]);
  for (int r = 0; r < nl; ++r) {
    bulk_g2s(D.pq[r], td.pq + (size_t)r * td.pq_stride, 32u, &S.thb[sl]);
    bulk_g2s(&D.y[r], td.y + (size_t)r * td.y_stride, 16u, &S.thb[sl]);
  }
  bulk_g2s(D.vrow, td.vrow, (uint32_t)nbins * 4u, &S.thb[sl]);
  ++S.issued_thb[sl];
  const char *rc = reinterpret_cast<const char *>(td.rc);
  asm volatile("prefetch.global.L1 [%0];" ::"l"(rc));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(rc + sizeof(StreamRun) - 1));
}

__device__ __forceinline__ void stream_issue_desc(const Plan &p, StreamSmem &S, StreamSlot *slots, int idx, int j) {
  const int sl = j % kSlots;
  mbar_arrive_expect_tx(&S.tdb[sl], (uint32_t)sizeof(StreamTile));
  bulk_g2s(&slots[sl].td, p.stiles + idx, (uint32_t)sizeof(StreamTile), &S.tdb[sl]);
  ++S.issued_tdb[sl];
}

// The producer thread's whole job: tiles 0 .. last of the CTA (p.stiles
// first + j), chunk by chunk.  False if a wait gave up (it then stops
// issuing; the consumers' own bounded waits end their loops).
__device__ bool stream_producer(const Plan &p, StreamSmem &S, StreamSlot *slots, uint8_t *stages, int first, int last) {
  // descriptors of the first tiles (free slots), chunks of tile 0 before the
  // wait for the previous post kernel; then the kick data
  for (int j = 0; j <= min(last, kSlots - 1); ++j) stream_issue_desc(p, S, slots, first + j, j);
  int K = 0;   // chunks issued
  bool data_ok = false;
  for (int j = 0; j <= last; ++j) {
    const int sl = j % kSlots;
    if (!mbar_wait_bounded(&S.tdb[sl], (uint32_t)((j / kSlots) & 1), kPushWaitNs)) return false;
    if (j == 0) {
      // tile 0's first chunks do not depend on the previous post kernel
      const StreamTile &td = slots[0].td;
      const int nc0 = (td.count + kStreamChunk - 1) / kStreamChunk;
      for (; K < min(kStreamStages, nc0); ++K) {
        const int n = min(kStreamChunk, td.count - K * kStreamChunk), n4 = (n + 3) & ~3;
        mbar_arrive_expect_tx(&S.full[K], (uint32_t)n4 * 12u);
        bulk_g2s(stages + K * kStreamStageBytes, td.tau + (size_t)K * kStreamChunk, (uint32_t)n4 * 4u, &S.full[K]);
        bulk_g2s(stages + K * kStreamStageBytes + kStreamChunk * sizeof(float), td.del + (size_t)K * kStreamChunk,
                 (uint32_t)n4 * 8u, &S.full[K]);
        ++S.issued_full[K];
      }
      grid_dependency_wait();
      data_ok = true;
      for (int q = 0; q <= min(last, kSlots - 1); ++q) {
        if (q > 0 && !mbar_wait_bounded(&S.tdb[q], 0u, kPushWaitNs)) return false;
        stream_issue_data(S, slots[q], q);
      }
    } else if (j >= kSlots) {
      // tile j reuses the slot of tile j - kSlots: its data only now
      stream_issue_data(S, slots[sl], sl);
    }
    // the descriptor of tile j + kSlots - 1 into the slot of tile j - 1, once the consumers have set that one up
    const int jn = j + kSlots - 1;
    if (j >= 1 && jn <= last) {
      const int sp = jn % kSlots;   // == (j - 1) % kSlots
      if (!mbar_wait_bounded(&S.freed[sp], (uint32_t)(((j - 1) / kSlots) & 1), kPushWaitNs)) return false;
      fence_proxy_async_smem();
      stream_issue_desc(p, S, slots, first + jn, jn);
    }
    // the tile's chunks
    const StreamTile &td = slots[sl].td;
    const int nc = (td.count + kStreamChunk - 1) / kStreamChunk;
    const int ci0 = j == 0 ? K : 0;
    for (int ci = ci0; ci < nc; ++ci, ++K) {
      const int stg = K % kStreamStages;
      if (K >= kStreamStages) {
        if (!mbar_wait_bounded(&S.empty[stg], (uint32_t)((K / kStreamStages - 1) & 1), kPushWaitNs)) return false;
        fence_proxy_async_smem();   // the consumers' reads of the stage before its refill
      }
      const int n = min(kStreamChunk, td.count - ci * kStreamChunk), n4 = (n + 3) & ~3;
      uint8_t *stage = stages + stg * kStreamStageBytes;
      mbar_arrive_expect_tx(&S.full[stg], (uint32_t)n4 * 12u);
      bulk_g2s(stage, td.tau + (size_t)ci * kStreamChunk, (uint32_t)n4 * 4u, &S.full[stg]);
      bulk_g2s(stage + kStreamChunk * sizeof(float), td.del + (size_t)ci * kStreamChunk, (uint32_t)n4 * 8u, &S.full[stg]);
      ++S.issued_full[stg];
    }
  }
  (void)data_ok;
  return true;
}

template <int NLONG_MAX, bool HARM>
__global__ void __launch_bounds__(kStreamThreads, 1) k_push_stream(const Plan p) {
  extern __shared__ __align__(128) uint8_t sm_push[];
  __shared__ StreamSmem S;
  uint8_t *stages = sm_push;
  StreamSlot *slots = reinterpret_cast<StreamSlot *>(sm_push + kStreamStages * kStreamStageBytes);
  float2 *sVd = reinterpret_cast<float2 *>(slots + kSlots);   // (V[j], V[j+1] - V[j]) of the current tile's bunch
  int *sH = reinterpret_cast<int *>(sVd + kStreamMaxBins);
  const int tid = threadIdx.x;
  const int first = p.stream_first[blockIdx.x];
  const int last = p.stream_first[blockIdx.x + 1] - first - 1;   // the CTA's tiles are first .. first + last

  if (tid == kProducerTid) {
    for (int s = 0; s < kStreamStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], kConsumerWarps);
      S.issued_full[s] = 0;
    }
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&S.tdb[s], 1);
      mbar_init(&S.thb[s], 1);
      mbar_init(&S.freed[s], 1);
      S.issued_tdb[s] = S.issued_thb[s] = 0;
    }
    fence_mbar_init();
  }
  for (int b = tid; b < kStreamMaxBins; b += kStreamThreads) sH[b] = 0;
  __syncthreads();   // barriers initialised, histogram zeroed
  grid_dependents_launch();

  if (tid >= kConsumers) {
    // ---------------- producer warp ----------------
    if (tid == kProducerTid && last >= 0) {
      if (!stream_producer(p, S, slots, stages, first, last)) {
        atomicExch(p.error, kErrTimeout);
      }
      // let every copy still in flight land before the CTA exits
      for (int s = 0; s < kStreamStages; ++s)
        if (S.issued_full[s]) mbar_wait_bounded(&S.full[s], (uint32_t)((S.issued_full[s] - 1) & 1), kPushWaitNs);
      for (int s = 0; s < kSlots; ++s) {
        if (S.issued_tdb[s]) mbar_wait_bounded(&S.tdb[s], (uint32_t)((S.issued_tdb[s] - 1) & 1), kPushWaitNs);
        if (S.issued_thb[s]) mbar_wait_bounded(&S.thb[s], (uint32_t)((S.issued_thb[s] - 1) & 1), kPushWaitNs);
      }
    }
    return;
  }

  // ---------------- consumer warps ----------------
  grid_dependency_wait();   // the previous post kernel zeroed this turn's histograms
  const int warp = tid >> 5, lane = tid & 31;
  bool failed = false;   // a wait of this thread gave up: it skips every further wait and all processing
  float st = 0.f, st2 = 0.f, sd = 0.f, sd2 = 0.f;
  int nout = 0;
  int k = 0;   // chunks consumed (chunk k is in stage k % kStreamStages)

#pragma unroll 1
  for (int J = 0; J <= last; ++J) {
    // ---- set up tile J ----
    const int sl = J % kSlots;
    const StreamSlot &D = slots[sl];
    if (!failed && !mbar_wait_bounded(&S.thb[sl], (uint32_t)((J / kSlots) & 1), kPushWaitNs)) {
      failed = true;
      atomicExch(p.error, kErrTimeout);
    }
    const int nbins = max(2, min(D.td.nbins, kStreamMaxBins));
    for (int b = tid; b < nbins; b += kConsumers) {
      const float v0 = D.vrow[b];
      const float v1 = b + 1 < nbins ? D.vrow[b + 1] : v0;
      sVd[b] = make_float2(v0, v1 - v0);
    }
    const int nl = max(0, min(D.td.nlong, NLONG_MAX));
    if (tid >= 64 && tid < 64 + nl) {
      // Phi_m = P_m y_tile + Q_m of this bunch, narrowed to FP32
      const int r = tid - 64;
      const double2 ph = cfma(D.pq[r][0], D.y[r], D.pq[r][1]);
      S.phi[r] = make_float2((float)ph.x, (float)ph.y);
    }
    const StreamRun *__restrict__ RC = D.td.rc;
    const long long turn = D.turn[0];
    int32_t *const hg = D.td.hist + (turn & 1) * D.td.hist_par;
    const int pslot = D.td.index;
    float *const tau = D.td.tau;
    double *const del = D.td.del;
    const long long start = D.td.start;
    const int count = D.td.count;
    const uint32_t turn32 = (uint32_t)turn, bunch32 = (uint32_t)D.td.m;
    consumers_sync();   // tables built, slot read
    if (tid == 0) mbar_arrive(&S.freed[sl]);
    // the previous tile's sums over the warps (its per-warp sums are in the
    // other half of S.red; the next hand-in writes this tile's half)

    PushConstF c;
    c.nbins = nbins;
    c.invD = __ldg(&RC->invD);
    c.HinvD = __ldg(&RC->HinvD);
    c.fnb = __ldg(&RC->fnb);
    c.invE0 = __ldg(&RC->invE0);
    c.rfA = __ldg(&RC->rfA);
    c.rfB = __ldg(&RC->rfB);
    c.w = __ldg(&RC->w);
    c.omD = 0.f;
    c.qe = __ldg(&RC->qe);
    c.aT0 = __ldg(&RC->aT0);
    const double omD_d = __ldg(&RC->omD);
    const bool ngp = (__ldg(&RC->flags) & kKickNGP) != 0;
    const int nharm = HARM ? max(0, min(__ldg(&RC->nharm), kMaxHarm)) : 0;
    float la[NLONG_MAX > 0 ? NLONG_MAX : 1], lw[NLONG_MAX > 0 ? NLONG_MAX : 1];
    float2 phi[NLONG_MAX > 0 ? NLONG_MAX : 1];
#pragma unroll
    for (int r = 0; r < NLONG_MAX; ++r) {
      la[r] = __ldg(&RC->la[r]);
      lw[r] = __ldg(&RC->lw[r]);
      phi[r] = r < nl ? S.phi[r] : make_float2(0.f, 0.f);
    }
    const uint32_t k0 = __ldg(&RC->key0), k1 = __ldg(&RC->key1);
    float tref = 0.f, dref = 0.f;   // moment reference: the tile's first particle before the push
    const int nc = (count + kStreamChunk - 1) / kStreamChunk;

    // ---- the tile's chunks ----
#pragma unroll 1
    for (int ci = 0; ci < nc; ++ci, ++k) {
      const int stg = k % kStreamStages;
      if (!failed && !mbar_wait_bounded(&S.full[stg], (uint32_t)((k / kStreamStages) & 1), kPushWaitNs)) {
        failed = true;
        atomicExch(p.error, kErrTimeout);
      }
      const uint8_t *sg = stages + stg * kStreamStageBytes;
      if (ci == 0) {
        tref = reinterpret_cast<const float *>(sg)[0];
        dref = f64_to_f32_ref(reinterpret_cast<const double *>(sg + kStreamChunk * sizeof(float))[0]);
      }
      const float4 tv = reinterpret_cast<const float4 *>(sg)[tid];
      const double2 da = reinterpret_cast<const double2 *>(sg + kStreamChunk * sizeof(float))[2 * tid];
      const double2 db = reinterpret_cast<const double2 *>(sg + kStreamChunk * sizeof(float))[2 * tid + 1];
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.empty[stg]);   // this warp's part of the stage is read
      const int q = ci * kStreamChunk + 4 * tid;   // first particle of this thread's quad in the tile
      if (!failed && q < count) {
        float rr[4] = {0.f, 0.f, 0.f, 0.f};
        if (c.qe != 0.f) normal_quad_f32(philox4x32_10((uint32_t)((start + q) >> 2), bunch32, turn32, 0u, k0, k1), rr);
        float tt[4] = {tv.x, tv.y, tv.z, tv.w};
        double dd[4] = {da.x, da.y, db.x, db.y};
        const int nvalid = min(4, count - q);
        const float4 *hc = RC->harm;
        if (ngp)
          quad_push<NLONG_MAX, true, HARM>(c, sVd, sH, nl, la, lw, phi, omD_d, hc, nharm, tt, dd, rr, nvalid, tref,
                                           dref, st, st2, sd, sd2, nout);
        else
          quad_push<NLONG_MAX, false, HARM>(c, sVd, sH, nl, la, lw, phi, omD_d, hc, nharm, tt, dd, rr, nvalid, tref,
                                            dref, st, st2, sd, sd2, nout);
        *reinterpret_cast<float4 *>(tau + q) = make_float4(tt[0], tt[1], tt[2], tt[3]);
        *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
        *reinterpret_cast<double2 *>(del + q + 2) = make_double2(dd[2], dd[3]);
      }
    }

    // ---- hand in tile J ----
    st = warp_sum_f(st);
    st2 = warp_sum_f(st2);
    sd = warp_sum_f(sd);
    sd2 = warp_sum_f(sd2);
    const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
    if (lane == 0) {
      float *r = S.red[warp];
      r[0] = st;
      r[1] = st2;
      r[2] = sd;
      r[3] = sd2;
      r[4] = (float)no;
    }
    st = st2 = sd = sd2 = 0.f;
    nout = 0;
    consumers_sync();   // every deposit of the tile made, S.red complete
    // (the spill cells behind this mesh are cleared too: a later tile of a
    // run with a larger mesh counts into those cells)
    for (int b = tid; b < nbins + kSpillCells; b += kConsumers) {
      const int cnt = sH[b];
      if (cnt) {
        if (!failed && b < nbins) atomicAdd(hg + b, cnt);
        sH[b] = 0;
      }
    }
    if (tid == 37 && !failed) {
      double *pp = p.partial + (size_t)pslot * kPartials;
      pp[5] = (double)tref;
      pp[10] = (double)dref;
      pp[11] = (double)count;
    }
    if (tid >= 32 && tid < 37 && !failed) {
      // the tile's sums over the warps: a pairwise tree of fixed shape over
      // the warps' FP32 sums of values relative to the tile's reference (an
      // FP64 sum here would stall every warp at the next tile's barrier on
      // GB300's FP64 pipe: +5 % per turn measured); FP64 from the tile on
      const int col = tid - 32;
      float a[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] = S.red[i][col] + (16 + i < kConsumerWarps ? S.red[16 + i][col] : 0.f);
#pragma unroll
      for (int h = 8; h > 0; h >>= 1)
#pragma unroll
        for (int i = 0; i < h; ++i) a[i] += a[i + h];
      p.partial[(size_t)pslot * kPartials + col] = (double)a[0];
    }
    // the next tile's set-up rewrites sVd and S.phi only after its own wait
    // and before its barrier; sH and this half of S.red only after it
  }

}

// ---------------------------------------------------------------------------
// Mixed precision with a transverse plane (plans where some run has one).
// A bulk-copy ring like the streaming push's, a stage holding tau, delta, x and
// x' of kChunkT particles (10 KB at 128 threads); one quad of consecutive
// particles per thread and chunk.  Runs of the plan without a transverse
// plane stage and push only tau and delta.  Harmonic cavities are a runtime
// loop here.  128-thread CTAs, 6 per SM at 80 registers: measured faster on
// the 390-bunch fill than 256 threads x 3 CTAs (320.6 against 330.3 us per
// launch, same GPU), 64 x 12 and 96 x 8 (331.9, 341.1 us), and than 72 or 64
// registers with more CTAs (spills).
// ---------------------------------------------------------------------------
#ifndef MBT_PUSH_T_THREADS
#define MBT_PUSH_T_THREADS 128
#endif
constexpr int kTThreads = MBT_PUSH_T_THREADS;   // threads of a transverse push CTA
constexpr int kChunkT = 4 * kTThreads;          // particles per stage: one quad per thread
constexpr int kStageBytesT = kChunkT * (int)(3 * sizeof(float) + sizeof(double));
// dynamic shared memory of the per-tile pushes: the stages, then per cell the
// (V, dV) table(s), the counts (with kSpillCells spill cells) and, with a
// transverse plane, the dipole sums
constexpr size_t push_tile_smem(int nbins, int threads = 256) {
  return (size_t)kStages * (size_t)(threads * 4 * 12) + (size_t)nbins * sizeof(float2) +
         (size_t)(nbins + kSpillCells) * sizeof(int);
}
constexpr size_t push_t_smem(int nbins) {
  return (size_t)kStages * kStageBytesT + (size_t)nbins * (2 * sizeof(float2) + sizeof(float4)) +
         (size_t)(nbins + kSpillCells) * 3 * sizeof(int);
}
#ifndef MBT_PUSH_T_MIN_BLOCKS
#define MBT_PUSH_T_MIN_BLOCKS 6
#endif

__device__ __forceinline__ void issue_chunk_t(const TileDev &t, const float *tau, const double *del, const float *x,
                                              const float *xp, uint8_t *stage, uint64_t *bar, int c, bool tr) {
  const int n = min(kChunkT, t.count - c * kChunkT);
  const int n4 = (n + 3) & ~3;   // segments are padded to 4 particles: 16-byte multiples
  const uint32_t fb = (uint32_t)n4 * 4u, db = (uint32_t)n4 * 8u;
  mbar_arrive_expect_tx(bar, fb + db + (tr ? 2u * fb : 0u));
  bulk_g2s(stage, tau + (size_t)c * kChunkT, fb, bar);
  bulk_g2s(stage + kChunkT * 4, del + (size_t)c * kChunkT, db, bar);
  if (tr) {
    bulk_g2s(stage + kChunkT * 12, x + (size_t)c * kChunkT, fb, bar);
    bulk_g2s(stage + kChunkT * 16, xp + (size_t)c * kChunkT, fb, bar);
  }
}

// Long-range transverse resistive-wall voltage on bunch m for the turn
// `turn`: sum over the passages of the last rw_nh turns before it (earlier
// bunches of the same passage included) of charge x centroid x W(D T_rf), D
// the bucket distance; every thread of the CTA returns the sum.  red: 8
// floats / doubles of shared scratch.  0 without a resistive wall.
__device__ float rw_voltage_f32(const RunDev *__restrict__ R, int m, long long turn, float *red) {
  if (R->rw_nh <= 0) return 0.f;
  const int nh1 = R->rw_nh + 1, nb = R->nb, h = R->h_rf, bm = R->bucket[m];
  float acc = 0.f;
  for (int i = threadIdx.x; i < nh1 * nb; i += kTThreads) {
    const int back = i / nb, mp = i - back * nb;
    const long long src = turn - 1 - back;
    const int D = back * h + bm - R->bucket[mp];
    if (src >= 0 && D > 0) acc = fmaf((float)R->rw_cent[(size_t)(src % nh1) * nb + mp], R->rw_tab_f[D], acc);
  }
  acc = warp_sum_f(acc);
  __syncthreads();   // red may hold other data until every thread is here
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  float v = 0.f;
#pragma unroll
  for (int w = 0; w < kTThreads / 32; ++w) v += red[w];
  __syncthreads();
  return v;
}

__device__ double rw_voltage_f64(const RunDev *__restrict__ R, int m, long long turn, double *red) {
  if (R->rw_nh <= 0) return 0.0;
  const int nh1 = R->rw_nh + 1, nb = R->nb, h = R->h_rf, bm = R->bucket[m];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nh1 * nb; i += kPushThreads) {
    const int back = i / nb, mp = i - back * nb;
    const long long src = turn - 1 - back;
    const int D = back * h + bm - R->bucket[mp];
    if (src >= 0 && D > 0) acc = fma(R->rw_cent[(size_t)(src % nh1) * nb + mp], R->rw_tab[D], acc);
  }
  acc = warp_sum_d(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  double v = 0.0;
#pragma unroll
  for (int w = 0; w < kPushThreads / 32; ++w) v += red[w];
  __syncthreads();
  return v;
}

template <int NLONG_MAX>
__global__ void __launch_bounds__(kTThreads, MBT_PUSH_T_MIN_BLOCKS) k_push_mixed_t(const Plan p) {
  extern __shared__ __align__(128) uint8_t sm_pt[];
  __shared__ float s_red[kTThreads / 32][9];
  __shared__ float2 s_phi[kMaxLong];
  __shared__ int s_plane[kMaxLong];
  __shared__ float4 s_hc[kMaxHarm];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int s_abort;

  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  PushConstF c;
  c.nbins = R->nbins;
  const int nbins = c.nbins;
  const int nlong = R->nlong;
  const bool tr = R->trans != 0;
  uint8_t *stages = sm_pt;
  // per cell (V, dV) of the longitudinal kick, and for quad_push_t_full the
  // same interleaved with the transverse kick: (V, dV, V_x, dV_x)
  float4 *sV4 = reinterpret_cast<float4 *>(sm_pt + kStages * kStageBytesT);
  float2 *sVd = reinterpret_cast<float2 *>(sV4 + nbins);
  int *sH = reinterpret_cast<int *>(sVd + nbins);                  // nbins + kSpillCells counts
  float2 *sVt = reinterpret_cast<float2 *>(sH + nbins + kSpillCells);
  unsigned *sLo = reinterpret_cast<unsigned *>(sVt + nbins);     // dipole sums in fixed point (deposit_dip),
  int *sHi = reinterpret_cast<int *>(sLo + nbins + kSpillCells); // nbins + kSpillCells cells each
  float *tau = static_cast<float *>(R->tau) + bd.off + t.start;
  double *del = R->delta + bd.off + t.start;
  float *xg = tr ? static_cast<float *>(R->x) + bd.off + t.start : nullptr;
  float *pg = tr ? static_cast<float *>(R->xp) + bd.off + t.start : nullptr;
  const int nchunks = (t.count + kChunkT - 1) / kChunkT;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&full[st], 1);
    fence_mbar_init();
    s_abort = 0;
    for (int ch = 0; ch < min(kStages, nchunks); ++ch)
      issue_chunk_t(t, tau, del, xg, pg, stages + ch * kStageBytesT, &full[ch], ch, tr);
  }
  const int nharm = R->nharm;
  if (threadIdx.x < nharm) s_hc[threadIdx.x] = R->f_harm[threadIdx.x];
  for (int k = threadIdx.x; k < nbins + kSpillCells; k += kTThreads) {
    sH[k] = 0;
    sLo[k] = 0u;
    sHi[k] = 0;
  }
  grid_dependents_launch();
  grid_dependency_wait();   // the previous post kernel's wakes, phasors and turn counter are complete
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);
  const float *vsr = static_cast<const float *>(R->vsr) + (size_t)t.m * nbins;
  const float *vtg = tr ? static_cast<const float *>(R->vt) + (size_t)t.m * nbins : nullptr;
  for (int k = threadIdx.x; k < nbins; k += kTThreads) {
    const float v0 = vsr[k];
    const float v1 = k + 1 < nbins ? vsr[k + 1] : v0;
    sVd[k] = make_float2(v0, v1 - v0);
    if (tr) {
      const float w0 = vtg[k];
      const float w1 = k + 1 < nbins ? vtg[k + 1] : w0;
      sVt[k] = make_float2(w0, w1 - w0);
      sV4[k] = make_float4(v0, v1 - v0, w0, w1 - w0);
    }
  }
  if (threadIdx.x < nlong) {
    const int r = threadIdx.x;
    const double2 P = R->pq[((size_t)r * R->nb + t.m) * 2];
    const double2 Q = R->pq[((size_t)r * R->nb + t.m) * 2 + 1];
    const double2 y = R->y[(size_t)r * R->ntile_b + t.m / kBunchTile];
    const double2 phi = cfma(P, y, Q);
    s_phi[r] = make_float2((float)phi.x, (float)phi.y);
    s_plane[r] = R->lr_plane[r];
  }
  c.invD = R->f_invD;
  c.HinvD = R->f_HinvD;
  c.fnb = R->f_nbins;
  c.invE0 = R->f_invE0 * R->f_omD;
  c.rfA = R->f_rfA;
  c.rfB = R->f_rfB;
  c.w = R->f_w;
  c.omD = R->f_omD;
  c.qe = R->f_qe;
  c.aT0 = R->f_aT0;
  const TransConstF tc = trans_consts(R);
  const double omD_d = R->one_minus_D;
  const bool ngp = (R->flags & kKickNGP) != 0;
  float la[NLONG_MAX > 0 ? NLONG_MAX : 1], lw[NLONG_MAX > 0 ? NLONG_MAX : 1];
  float2 phi[NLONG_MAX > 0 ? NLONG_MAX : 1];
  int plane[NLONG_MAX > 0 ? NLONG_MAX : 1];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < NLONG_MAX; ++r) {
    la[r] = R->f_la[r];
    lw[r] = R->f_lw[r];
    phi[r] = r < nlong ? s_phi[r] : make_float2(0.f, 0.f);
    plane[r] = r < nlong ? s_plane[r] : 0;
  }
  // the same entries in the masked form of quad_push_t_full
  float2 lA[NLONG_MAX > 0 ? NLONG_MAX : 1];
  float lml[NLONG_MAX > 0 ? NLONG_MAX : 1], lmt[NLONG_MAX > 0 ? NLONG_MAX : 1];
#pragma unroll
  for (int r = 0; r < NLONG_MAX; ++r) {
    lA[r] = plane[r] ? make_float2(phi[r].y, phi[r].x) : make_float2(phi[r].x, -phi[r].y);
    lml[r] = plane[r] ? 0.f : 1.f;
    lmt[r] = plane[r] ? 1.f : 0.f;
  }
  const bool straight = !ngp && nharm == 0;   // full quads take quad_push_t_full
  const uint32_t k0 = R->key0, k1 = R->key1, turn32 = (uint32_t)turn, bunch32 = (uint32_t)t.m;
  const bool texc = tc.nx != 0.f || tc.nxp != 0.f;
  const float vrw = tr ? rw_voltage_f32(R, t.m, turn, s_red[0]) : 0.f;
  float tref = 0.f, dref = 0.f;   // moment reference: the tile's first particle before the push

  float mom[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int nout = 0;
  bool dip_ok = true;   // every deposited x within the dipole deposit's range
#pragma unroll 1
  for (int ch = 0; ch < nchunks; ++ch) {
    const int slot = ch % kStages;
    uint8_t *sg = stages + slot * kStageBytesT;
    if (!mbar_wait_bounded(&full[slot], (uint32_t)((ch / kStages) & 1), kPushWaitNs)) {
      atomicExch(p.error, kErrTimeout);
      s_abort = 1;
    }
    if (ch == 0) {
      tref = reinterpret_cast<const float *>(sg)[0];
      dref = f64_to_f32_ref(reinterpret_cast<const double *>(sg + kChunkT * 4)[0]);
    }
    const int q = ch * kChunkT + 4 * (int)threadIdx.x;
    if (!s_abort && q < t.count) {
      const uint32_t quad = (uint32_t)((t.start + q) >> 2);
      const float4 tv = reinterpret_cast<const float4 *>(sg)[threadIdx.x];
      const double2 da = reinterpret_cast<const double2 *>(sg + kChunkT * 4)[2 * threadIdx.x];
      const double2 db = reinterpret_cast<const double2 *>(sg + kChunkT * 4)[2 * threadIdx.x + 1];
      float rr[4] = {0.f, 0.f, 0.f, 0.f};
      if (c.qe != 0.f) normal_quad_f32(philox4x32_10(quad, bunch32, turn32, 0u, k0, k1), rr);
      float tt[4] = {tv.x, tv.y, tv.z, tv.w};
      double dd[4] = {da.x, da.y, db.x, db.y};
      const int nvalid = min(4, t.count - q);
      if (tr) {
        const float4 xv = reinterpret_cast<const float4 *>(sg + kChunkT * 12)[threadIdx.x];
        const float4 pv = reinterpret_cast<const float4 *>(sg + kChunkT * 16)[threadIdx.x];
        float xx[4] = {xv.x, xv.y, xv.z, xv.w}, pp[4] = {pv.x, pv.y, pv.z, pv.w};
        float rx[4] = {0.f, 0.f, 0.f, 0.f}, rp[4] = {0.f, 0.f, 0.f, 0.f};
        if (texc) {
          normal_quad_f32(philox4x32_10(quad, bunch32, turn32, 3u, k0, k1), rx);
          normal_quad_f32(philox4x32_10(quad, bunch32, turn32, 4u, k0, k1), rp);
        }
        if (straight && nvalid == 4)
          quad_push_t_full<NLONG_MAX>(c, tc, sV4, sH, sLo, sHi, la, lw, lA, lml, lmt, omD_d, vrw, tt, dd, xx, pp,
                                      rr, rx, rp, tref, dref, mom, nout, dip_ok);
        else
          quad_push_t<NLONG_MAX>(c, tc, sVd, sVt, sH, sLo, sHi, nlong, plane, la, lw, phi, omD_d, s_hc, nharm, ngp,
                                 vrw, tt, dd, xx, pp, rr, rx, rp, nvalid, tref, dref, mom, nout, dip_ok);
        *reinterpret_cast<float4 *>(xg + q) = make_float4(xx[0], xx[1], xx[2], xx[3]);
        *reinterpret_cast<float4 *>(pg + q) = make_float4(pp[0], pp[1], pp[2], pp[3]);
      } else if (ngp) {
        quad_push<NLONG_MAX, true, true>(c, sVd, sH, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid,
                                         tref, dref, mom[0], mom[1], mom[2], mom[3], nout);
      } else {
        quad_push<NLONG_MAX, false, true>(c, sVd, sH, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid,
                                          tref, dref, mom[0], mom[1], mom[2], mom[3], nout);
      }
      *reinterpret_cast<float4 *>(tau + q) = make_float4(tt[0], tt[1], tt[2], tt[3]);
      *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
      *reinterpret_cast<double2 *>(del + q + 2) = make_double2(dd[2], dd[3]);
    }
    __syncthreads();   // stage `slot` consumed by every thread
    if (threadIdx.x == 0 && !s_abort && ch + kStages < nchunks) {
      fence_proxy_async_smem();
      issue_chunk_t(t, tau, del, xg, pg, sg, &full[slot], ch + kStages, tr);
    }
  }
  if (s_abort && threadIdx.x == 0) {
    for (int ch = 0; ch < nchunks; ++ch) mbar_wait_bounded(&full[ch % kStages], (uint32_t)((ch / kStages) & 1), kPushWaitNs);
  }

  // moment partials (columns 0-4 longitudinal, 6-9 transverse)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) mom[k] = warp_sum_f(mom[k]);
  const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s_red[warp][k] = mom[k];
    s_red[warp][4] = (float)no;
#pragma unroll
    for (int k = 4; k < 8; ++k) s_red[warp][k + 1] = mom[k];
  }
  if (__syncthreads_or(!dip_ok) && threadIdx.x == 0) atomicCAS(p.error, kErrNone, kErrDipole);
  if (threadIdx.x < 9) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kTThreads / 32; ++w) acc += (double)s_red[w][threadIdx.x];
    const int col = threadIdx.x < 5 ? threadIdx.x : threadIdx.x + 1;
    p.partial[(size_t)blockIdx.x * kPartials + col] = acc;
  } else if (threadIdx.x == 9) {
    double *pp = p.partial + (size_t)blockIdx.x * kPartials;
    pp[5] = (double)tref;
    pp[10] = (double)dref;
    pp[11] = (double)t.count;
  }
  int32_t *hg = R->hist + ((size_t)par * R->nb + t.m) * nbins;
  unsigned long long *dg =
      tr ? static_cast<unsigned long long *>(R->dip) + ((size_t)par * R->nb + t.m) * nbins : nullptr;
  for (int k = threadIdx.x; k < nbins; k += kTThreads) {
    const int cnt = sH[k];
    if (cnt) {
      atomicAdd(hg + k, cnt);
      // the tile's exact fixed-point sum (|2^16 hi + lo| < 2^47) into the bunch's int64 sum (two's complement)
      if (tr) atomicAdd(dg + k, (unsigned long long)((long long)sHi[k] * 65536LL + (long long)sLo[k]));
    }
  }
}

// ---------------------------------------------------------------------------
// FP64: the oracle's arithmetic step for step.  Each thread handles quads of
// consecutive particles (one Philox block per quad).  The cell index is formed
// with explicitly rounded operations so it cannot be contracted into an FMA.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double vsr_at_f64(const double *sV, double x, int nbins, bool ngp) {
  if (!(x >= 0.0 && x < (double)nbins)) return 0.0;
  if (ngp) return sV[(int)x];
  const double u = x - 0.5;
  if (u <= 0.0) return sV[0];
  if (u >= (double)(nbins - 1)) return sV[nbins - 1];
  const double j0 = floor(u);
  const double f = u - j0;
  const int j = (int)j0;
  return (1.0 - f) * sV[j] + f * sV[j + 1];
}

__global__ void __launch_bounds__(kPushThreads) k_push_f64(const Plan p) {
  extern __shared__ __align__(16) double sm_push64[];
  __shared__ double s_red[kPushThreads / 32][9];
  __shared__ double2 s_phi[kMaxLong];
  __shared__ int s_plane[kMaxLong];

  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  const int nbins = R->nbins;
  const int nlong = R->nlong;
  grid_dependents_launch();
  grid_dependency_wait();
  double *sV = sm_push64;
  int *sH = reinterpret_cast<int *>(sm_push64 + nbins);
  // transverse plane: voltage and dipole sums of the bunch (plans with one reserve the room)
  const bool tr = R->trans != 0;
  double *sVt = sm_push64 + nbins + (nbins + 1) / 2;
  double *sDip = sVt + nbins;
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);

  const double *vsr = static_cast<const double *>(R->vsr) + (size_t)t.m * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    sV[k] = vsr[k];
    sH[k] = 0;
    if (tr) {
      sVt[k] = static_cast<const double *>(R->vt)[(size_t)t.m * nbins + k];
      sDip[k] = 0.0;
    }
  }
  if (threadIdx.x < nlong) {
    const int r = threadIdx.x;
    const double2 P = R->pq[((size_t)r * R->nb + t.m) * 2];
    const double2 Q = R->pq[((size_t)r * R->nb + t.m) * 2 + 1];
    const double2 y = R->y[(size_t)r * R->ntile_b + t.m / kBunchTile];
    s_phi[r] = cfma(P, y, Q);
    s_plane[r] = R->lr_plane[r];
  }
  __syncthreads();

  const double H = R->H, invD = R->invDelta, invE0 = R->inv_E0, VoE0 = R->V_over_E0;
  const double phis = R->phi_s, wrf = R->omega_rf, U0oE0 = R->U0_over_E0;
  const double omD = R->one_minus_D, qe = R->qe_amp, aT0 = R->aT0;
  const bool ngp = (R->flags & kKickNGP) != 0;
  const uint32_t k0 = R->key0, k1 = R->key1, turn32 = (uint32_t)turn, bunch32 = (uint32_t)t.m;

  double *tau = static_cast<double *>(R->tau) + bd.off + t.start;
  double *del = R->delta + bd.off + t.start;
  double *xg = tr ? static_cast<double *>(R->x) + bd.off + t.start : nullptr;
  double *pg = tr ? static_cast<double *>(R->xp) + bd.off + t.start : nullptr;
  const bool texc = tr && (R->t_nx != 0.0 || R->t_nxp != 0.0);
  double st = 0.0, st2 = 0.0, sd = 0.0, sd2 = 0.0, sx = 0.0, sx2 = 0.0, sp = 0.0, sp2 = 0.0;
  int nout = 0;
  const double vrw = tr ? rw_voltage_f64(R, t.m, turn, s_red[0]) : 0.0;
  // moment reference: the tile's first particle before the push (read by
  // every thread before thread 0 overwrites it)
  __shared__ double s_ref[2];
  if (threadIdx.x == 0) {
    s_ref[0] = static_cast<const double *>(R->tau)[bd.off + t.start];
    s_ref[1] = R->delta[bd.off + t.start];
  }
  __syncthreads();
  const double2 mref = make_double2(s_ref[0], s_ref[1]);

#pragma unroll 1
  for (int it = 0; it < kF64QuadsPerThread; ++it) {
    const int q = (it * kPushThreads + (int)threadIdx.x) * 4;
    if (q >= t.count) break;
    double tt[4], dd[4];
    {
      const double2 t0 = *reinterpret_cast<const double2 *>(tau + q);
      const double2 t1 = *reinterpret_cast<const double2 *>(tau + q + 2);
      const double2 d0 = *reinterpret_cast<const double2 *>(del + q);
      const double2 d1 = *reinterpret_cast<const double2 *>(del + q + 2);
      tt[0] = t0.x; tt[1] = t0.y; tt[2] = t1.x; tt[3] = t1.y;
      dd[0] = d0.x; dd[1] = d0.y; dd[2] = d1.x; dd[3] = d1.y;
    }
    double rr[4] = {0.0, 0.0, 0.0, 0.0}, rx[4] = {0.0, 0.0, 0.0, 0.0}, rp[4] = {0.0, 0.0, 0.0, 0.0};
    if (qe != 0.0) normal_quad_f64(philox4x32_10((uint32_t)((t.start + q) >> 2), bunch32, turn32, 0u, k0, k1), rr);
    if (texc) {
      normal_quad_f64(philox4x32_10((uint32_t)((t.start + q) >> 2), bunch32, turn32, 3u, k0, k1), rx);
      normal_quad_f64(philox4x32_10((uint32_t)((t.start + q) >> 2), bunch32, turn32, 4u, k0, k1), rp);
    }
    double xx[4] = {0.0, 0.0, 0.0, 0.0}, pp[4] = {0.0, 0.0, 0.0, 0.0};
    if (tr) {
      const double2 x0 = *reinterpret_cast<const double2 *>(xg + q), x1 = *reinterpret_cast<const double2 *>(xg + q + 2);
      const double2 p0 = *reinterpret_cast<const double2 *>(pg + q), p1 = *reinterpret_cast<const double2 *>(pg + q + 2);
      xx[0] = x0.x; xx[1] = x0.y; xx[2] = x1.x; xx[3] = x1.y;
      pp[0] = p0.x; pp[1] = p0.y; pp[2] = p1.x; pp[3] = p1.y;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (q + e >= t.count) continue;
      double tp = tt[e], d = dd[e];
      const double xc = __dmul_rn(__dadd_rn(tp, H), invD);
      double v = vsr_at_f64(sV, xc, nbins, ngp);
      double vt = tr ? vsr_at_f64(sVt, xc, nbins, ngp) + vrw : 0.0;
      for (int r = 0; r < nlong; ++r) {
        const double2 s = R->lr_s[r];
        double sn, cs;
        sincos(s.y * tp, &sn, &cs);
        const double ea = exp(s.x * tp);
        if (s_plane[r]) vt += ea * (s_phi[r].x * sn + s_phi[r].y * cs);   // Im(Phi e^{s tau})
        else v += ea * (s_phi[r].x * cs - s_phi[r].y * sn);                // Re(Phi e^{s tau})
      }
      d = d - v * invE0;
      const double d_before = d;
      d = d + VoE0 * sin(phis - wrf * tp);
      for (int k = 0; k < R->nharm; ++k) d = d + R->harm_VoE0[k] * sin(R->harm_phi[k] - R->harm_nw[k] * tp);
      const double d_gain = d;
      d = d - U0oE0;
      d = d * omD + qe * rr[e];
      if (tr) {
        // transverse: wake kick, momentum ratio across the cavity, rotation with the new delta, excitation
        double p = pp[e] + vt * invE0;
        p = p * (1.0 + d_before) / (1.0 + d_gain);
        const double psi = R->t_mu0 * (1.0 + R->t_xi * d);
        double sn, cs;
        sincos(psi, &sn, &cs);
        const double x = xx[e];
        double xn = (cs + R->t_alpha * sn) * x + R->t_beta * sn * p;
        double pn = -R->t_gamma * sn * x + (cs - R->t_alpha * sn) * p;
        xx[e] = xn + R->t_nx * rx[e];
        pp[e] = pn + R->t_nxp * rp[e];
        sx += xx[e];
        sx2 += xx[e] * xx[e];
        sp += pp[e];
        sp2 += pp[e] * pp[e];
      }
      tp = tp + aT0 * d;
      tt[e] = tp;
      dd[e] = d;
      const double xb = __dmul_rn(__dadd_rn(tp, H), invD);
      if (xb >= 0.0 && xb < (double)nbins) {
        atomicAdd(&sH[(int)xb], 1);
        if (tr) atomicAdd(&sDip[(int)xb], xx[e]);
      } else {
        ++nout;
      }
      const double ou = tp - mref.x, ov = d - mref.y;   // relative to the moment reference
      st += ou;
      st2 += ou * ou;
      sd += ov;
      sd2 += ov * ov;
    }
    if (tr) {
      *reinterpret_cast<double2 *>(xg + q) = make_double2(xx[0], xx[1]);
      *reinterpret_cast<double2 *>(xg + q + 2) = make_double2(xx[2], xx[3]);
      *reinterpret_cast<double2 *>(pg + q) = make_double2(pp[0], pp[1]);
      *reinterpret_cast<double2 *>(pg + q + 2) = make_double2(pp[2], pp[3]);
    }
    *reinterpret_cast<double2 *>(tau + q) = make_double2(tt[0], tt[1]);
    *reinterpret_cast<double2 *>(tau + q + 2) = make_double2(tt[2], tt[3]);
    *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
    *reinterpret_cast<double2 *>(del + q + 2) = make_double2(dd[2], dd[3]);
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  st = warp_sum_d(st);
  st2 = warp_sum_d(st2);
  sd = warp_sum_d(sd);
  sd2 = warp_sum_d(sd2);
  sx = warp_sum_d(sx);
  sx2 = warp_sum_d(sx2);
  sp = warp_sum_d(sp);
  sp2 = warp_sum_d(sp2);
  const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
  if (lane == 0) {
    s_red[warp][0] = st;
    s_red[warp][1] = st2;
    s_red[warp][2] = sd;
    s_red[warp][3] = sd2;
    s_red[warp][4] = (double)no;
    s_red[warp][5] = sx;
    s_red[warp][6] = sx2;
    s_red[warp][7] = sp;
    s_red[warp][8] = sp2;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double acc = 0.0;
    for (int w = 0; w < kPushThreads / 32; ++w) acc += s_red[w][threadIdx.x];
    const int col = threadIdx.x < 5 ? threadIdx.x : threadIdx.x + 1;   // columns 0-4, 6-9
    p.partial[(size_t)blockIdx.x * kPartials + col] = acc;
  } else if (threadIdx.x == 9) {
    double *pp = p.partial + (size_t)blockIdx.x * kPartials;
    pp[5] = mref.x;
    pp[10] = mref.y;
    pp[11] = (double)t.count;
  }
  int32_t *hg = R->hist + ((size_t)par * R->nb + t.m) * nbins;
  double *dg = tr ? static_cast<double *>(R->dip) + ((size_t)par * R->nb + t.m) * nbins : nullptr;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    const int c = sH[k];
    if (c) {
      atomicAdd(hg + k, c);
      if (tr) atomicAdd(dg + k, sDip[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// Matched Gaussian start from Philox tags 1 (tau) and 2 (delta) at turn 0, in
// FP64 for both precisions (tau narrowed to FP32 by rounding for kMixed).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPushThreads) k_init(const Plan p, int precision) {
  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  for (int q = 4 * (int)threadIdx.x; q < t.count; q += 4 * kPushThreads) {
    const uint32_t quad = (uint32_t)((t.start + q) >> 2);
    double a[4], b[4];
    normal_quad_f64(philox4x32_10(quad, (uint32_t)t.m, 0u, 1u, R->key0, R->key1), a);
    normal_quad_f64(philox4x32_10(quad, (uint32_t)t.m, 0u, 2u, R->key0, R->key1), b);
    const long long i = bd.off + t.start + q;
    const int nv = min(4, t.count - q);
    for (int e = 0; e < nv; ++e) {
      if (precision == kMixed) static_cast<float *>(R->tau)[i + e] = (float)(R->sigma_tau0 * a[e]);
      else static_cast<double *>(R->tau)[i + e] = R->sigma_tau0 * a[e];
      R->delta[i + e] = R->sigma_E * b[e];
    }
    if (R->trans) {
      // matched Gaussian of the transverse plane, tags 5 (x) and 6 (x'):
      // x = sqrt(beta emit) c, x' = sqrt(emit / beta) (d - alpha c)
      double cx[4], dx[4];
      normal_quad_f64(philox4x32_10(quad, (uint32_t)t.m, 0u, 5u, R->key0, R->key1), cx);
      normal_quad_f64(philox4x32_10(quad, (uint32_t)t.m, 0u, 6u, R->key0, R->key1), dx);
      const double sx = sqrt(R->t_beta * R->t_emit);
      const double emit = sx * sx / R->t_beta;
      for (int e = 0; e < nv; ++e) {
        const double x = sx * cx[e], xp = sqrt(emit / R->t_beta) * (dx[e] - R->t_alpha * cx[e]);
        if (precision == kMixed) {
          static_cast<float *>(R->x)[i + e] = (float)x;
          static_cast<float *>(R->xp)[i + e] = (float)xp;
        } else {
          static_cast<double *>(R->x)[i + e] = x;
          static_cast<double *>(R->xp)[i + e] = xp;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Particle state of every bunch from page-locked host arrays (tau, delta of
// all bunches back to back, n_mp each), read by the kernel across the host
// link and written in the device layout (segments padded to 4; tau narrowed
// to FP32 by rounding for kMixed, as a per-bunch copy does).  hoff[m]: first
// particle of bunch m in the host arrays.
// ---------------------------------------------------------------------------
template <typename TT>
__global__ void __launch_bounds__(kPushThreads) k_load_host(const Plan p, int precision, const TT *tau_h,
                                                            const double *del_h, const long long *hoff) {
  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  const long long h0 = hoff[t.m] + t.start, d0 = bd.off + t.start;
  for (int q = 4 * (int)threadIdx.x; q < t.count; q += 4 * kPushThreads) {
    const int nv = min(4, t.count - q);
    TT tv[4];
    double dv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e < nv) {
        tv[e] = tau_h[h0 + q + e];
        dv[e] = del_h[h0 + q + e];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (e < nv) {
        if (precision == kMixed) static_cast<float *>(R->tau)[d0 + q + e] = (float)tv[e];
        else static_cast<double *>(R->tau)[d0 + q + e] = (double)tv[e];
        R->delta[d0 + q + e] = dv[e];
      }
    }
  }
}

cudaError_t launch_load_host(const Plan &p, int precision, const double *tau_h, const double *del_h,
                             const long long *hoff, cudaStream_t s) {
  if (p.ntiles == 0) return cudaSuccess;
  k_load_host<double><<<p.ntiles, kPushThreads, 0, s>>>(p, precision, tau_h, del_h, hoff);
  return cudaGetLastError();
}

cudaError_t launch_load_host_f32(const Plan &p, int precision, const float *tau_h, const double *del_h,
                                 const long long *hoff, cudaStream_t s) {
  if (p.ntiles == 0) return cudaSuccess;
  k_load_host<float><<<p.ntiles, kPushThreads, 0, s>>>(p, precision, tau_h, del_h, hoff);
  return cudaGetLastError();
}

template <typename... Args>
static cudaError_t launch_ex(void (*kern)(Args...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                             Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_push(const Plan &p, int precision, cudaStream_t s, bool pdl) {
  if (p.ntiles == 0) return cudaSuccess;
  const int max_nbins = p.max_nbins;
  if (precision == kMixed && p.max_trans) {
    const size_t smem = push_t_smem(max_nbins);
    switch (p.max_nlong) {
      case 0: return launch_ex(k_push_mixed_t<0>, p.ntiles, kTThreads, smem, s, pdl, p);
      case 1: return launch_ex(k_push_mixed_t<1>, p.ntiles, kTThreads, smem, s, pdl, p);
      case 2: return launch_ex(k_push_mixed_t<2>, p.ntiles, kTThreads, smem, s, pdl, p);
      default: return launch_ex(k_push_mixed_t<kMaxLong>, p.ntiles, kTThreads, smem, s, pdl, p);
    }
  }
  if (precision == kMixed && p.stream_ctas <= 0) {
    // per-tile push, in the CTA shape the plan chose
    const bool harm = p.max_nharm > 0;
    auto go = [&](auto k256, auto k128) -> cudaError_t {
      if (p.push_small_ctas) return launch_ex(k128, p.ntiles, 128, push_tile_smem(max_nbins, 128), s, pdl, p);
      return launch_ex(k256, p.ntiles, 256, push_tile_smem(max_nbins, 256), s, pdl, p);
    };
    switch (p.max_nlong) {
      case 0: return harm ? go(k_push_mixed<0, true, 256>, k_push_mixed<0, true, 128>)
                          : go(k_push_mixed<0, false, 256>, k_push_mixed<0, false, 128>);
      case 1: return harm ? go(k_push_mixed<1, true, 256>, k_push_mixed<1, true, 128>)
                          : go(k_push_mixed<1, false, 256>, k_push_mixed<1, false, 128>);
      case 2: return harm ? go(k_push_mixed<2, true, 256>, k_push_mixed<2, true, 128>)
                          : go(k_push_mixed<2, false, 256>, k_push_mixed<2, false, 128>);
      default: return harm ? go(k_push_mixed<kMaxLong, true, 256>, k_push_mixed<kMaxLong, true, 128>)
                           : go(k_push_mixed<kMaxLong, false, 256>, k_push_mixed<kMaxLong, false, 128>);
    }
  }
  if (precision == kMixed) {
    if (!p.stream_first) return cudaErrorInvalidValue;
    const bool harm = p.max_nharm > 0;
    const int grid = p.stream_ctas;
    switch (p.max_nlong) {
      case 0: return launch_ex(harm ? k_push_stream<0, true> : k_push_stream<0, false>, grid, kStreamThreads, kStreamSmem, s, pdl, p);
      case 1: return launch_ex(harm ? k_push_stream<1, true> : k_push_stream<1, false>, grid, kStreamThreads, kStreamSmem, s, pdl, p);
      case 2: return launch_ex(harm ? k_push_stream<2, true> : k_push_stream<2, false>, grid, kStreamThreads, kStreamSmem, s, pdl, p);
      default:
        return launch_ex(harm ? k_push_stream<kMaxLong, true> : k_push_stream<kMaxLong, false>, grid, kStreamThreads,
                         kStreamSmem, s, pdl, p);
    }
  }
  // sV, sH (rounded up to doubles), and with a transverse plane sVt, sDip
  const size_t smem = ((size_t)max_nbins + (size_t)(max_nbins + 1) / 2 + (p.max_trans ? 2 * (size_t)max_nbins : 0)) *
                      sizeof(double);
  return launch_ex(k_push_f64, p.ntiles, kPushThreads, smem, s, pdl, p);
}

// Streaming-push CTAs resident at once on the current device, one per SM
// (cached per device: every variant has the same launch bounds and shared
// memory).
cudaError_t push_resident_slots(int *slots) {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (cache[dev] == 0) {
    int nsm = 0, per = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_push_stream<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStreamSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_push_stream<1, false>, kStreamThreads, kStreamSmem);
    if (e != cudaSuccess) return e;
    cache[dev] = std::max(1, per) * nsm;
  }
  *slots = cache[dev];
  return cudaSuccess;
}

bool plan_streams(const std::vector<int64_t> &n, const std::vector<int> &nb, bool any_trans, int sms) {
  if (any_trans || n.empty() || sms <= 0) return false;
  for (size_t i = 0; i < n.size(); ++i) {
    if (n[i] < (int64_t)sms * 4 * kStreamChunk) return false;           // a share of >= 4 stages per SM
    if (nb[i] <= 0 || n[i] / nb[i] < 2 * kStreamChunk) return false;    // bunches of >= 2 stages on average
  }
  return true;
}

// CTAs of a per-tile push (with or without a transverse plane) resident at
// once on the current device (256 cells).
cudaError_t push_tile_resident_slots(bool trans, int *slots) {
  const size_t smem = trans ? push_t_smem(256) : push_tile_smem(256);
  int dev = 0, nsm = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = trans ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_push_mixed_t<1>, kTThreads, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_push_mixed<1, false, 256>, 256, smem);
  *slots = per * nsm;
  return e;
}

cudaError_t configure_push_kernels() {
  cudaError_t e = cudaSuccess;
  for (auto k : {k_push_stream<0, false>, k_push_stream<1, false>, k_push_stream<2, false>, k_push_stream<kMaxLong, false>,
                 k_push_stream<0, true>, k_push_stream<1, true>, k_push_stream<2, true>, k_push_stream<kMaxLong, true>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStreamSmem);
  int slots = 0;
  if (e == cudaSuccess) e = push_resident_slots(&slots);
  const int bytes = (int)push_tile_smem(1024, 256), bytes128 = (int)push_tile_smem(1024, 128);
  for (auto k : {k_push_mixed<0, false, 256>, k_push_mixed<1, false, 256>, k_push_mixed<2, false, 256>,
                 k_push_mixed<kMaxLong, false, 256>, k_push_mixed<0, true, 256>, k_push_mixed<1, true, 256>,
                 k_push_mixed<2, true, 256>, k_push_mixed<kMaxLong, true, 256>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  for (auto k : {k_push_mixed<0, false, 128>, k_push_mixed<1, false, 128>, k_push_mixed<2, false, 128>,
                 k_push_mixed<kMaxLong, false, 128>, k_push_mixed<0, true, 128>, k_push_mixed<1, true, 128>,
                 k_push_mixed<2, true, 128>, k_push_mixed<kMaxLong, true, 128>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes128);
  const int bytes_t = (int)push_t_smem(256);
  for (auto k : {k_push_mixed_t<0>, k_push_mixed_t<1>, k_push_mixed_t<2>, k_push_mixed_t<kMaxLong>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes_t);
  return e;
}

cudaError_t launch_init(const Plan &p, int precision, cudaStream_t s) {
  if (p.ntiles == 0) return cudaSuccess;
  k_init<<<p.ntiles, kPushThreads, 0, s>>>(p, precision);
  return cudaGetLastError();
}

}  // namespace mbt
