// Post-turn kernel: everything that follows the push of a turn, for every run
// of the plan, in one launch, one CTA per job (PostJob):
//
//  kJobWake  short-range wake voltage of a tile of bunches (Sec. 2.3, Eq. 6):
//            V[j, m] = q_m sum_{k<=j} W~((j-k) Delta) count[m, k], a lower
//            triangular Toeplitz matrix (cells x cells) times the counts
//            (cells x bunches).  kMixed: tcgen05 MMA on the tensor cores;
//            the Toeplitz matrix is split into BF16 hi + lo halves laid side
//            by side along K, the integer counts into three exact BF16 byte
//            planes laid side by side along N; FP32 accumulation in tensor
//            memory; the planes are recombined in the epilogue.  kF64: FP64
//            on the CUDA cores.
//  kJobTile  for a tile of up to 32 bunches and each long-range resonator:
//            the emission E_m = c q_m sum_k count[m,k] e^{-s tau_k} and the
//            warp-level prefix scan of the phasor affine maps
//            x -> a_m (x + E_{m-1}) across the tile (long-range wake,
//            Sec. 2.3 last paragraph).
//  kJobMoments  (kMixed) per-bunch moments of the turn into the record ring
//            (Sec. 2.4) and zeroing of the other histogram buffer.  When the
//            plan's post CTAs would outnumber the SMs there is no moments
//            job (Plan::fold_moments) and the tile job does this first, as
//            the kF64 tile job always does.
//  kJobTrans  transverse short-range voltage of a tile of bunches (rows of
//            the dipole-sum convolution), for runs with a transverse plane.
//
// The last CTA to finish (completion counter) composes the tile aggregates
// of each (run, resonator) with the carried phasor of the previous turn,
// writes the value entering every tile and the new carry, and advances the
// turn counter of every run.
#include <cuda_bf16.h>
#include <algorithm>
#include <mutex>
#include "device_common.cuh"

namespace mbt {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // bounded device waits: 2 s

// ---------------------------------------------------------------------------
// Run-constant inputs of a job, staged into shared memory before the kernel
// waits for the push of the turn (they do not depend on it), so that the
// dependent chain after the wait touches only data the push has just written
// (histograms, partial sums, in L2) instead of cold lines in DRAM: after the
// push has streamed the particle state through L2, every table the post
// kernel reads would otherwise be a DRAM round trip on its critical path.
// ---------------------------------------------------------------------------
struct PostStage {
  double2 step[kMaxLong][kBunchTile];   // a_m of the tile's bunches (tile jobs)
  double q[kBunchTile];                 // macro-particle charge (tile jobs)
  float qf[kBunchTile];                 // same in float (wake jobs)
  double inv_n[kBunchTile];             // 1 / N_m (moments jobs)
  long long n[kBunchTile];
  int tile0[kBunchTile], ntiles[kBunchTile];
};

__device__ __forceinline__ void prefetch_l2(const void *ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// tabf: nlong x nbins emission factors (tile jobs), in dynamic shared memory.
__device__ void post_stage(const Plan &p, const RunDev *__restrict__ R, const PostJob &job, PostStage *st,
                           float2 *tabf) {
  const int tid = threadIdx.x;
  const int nb = R->nb, m0 = job.bt * kBunchTile, nbt = min(kBunchTile, nb - m0);
  if (job.type == kJobTile) {
    const int nl = R->nlong, nbins = R->nbins;
    for (int i = tid; i < nl * nbins; i += kPostThreads) tabf[i] = R->emis_f[i];
    for (int i = tid; i < nl * kBunchTile; i += kPostThreads) {
      const int r = i / kBunchTile, b = i % kBunchTile;
      st->step[r][b] = b < nbt ? R->step[(size_t)r * nb + m0 + b] : make_double2(1.0, 0.0);
    }
    if (tid < kBunchTile) st->q[tid] = tid < nbt ? R->q_mp[m0 + tid] : 0.0;
    if (tid == 32) prefetch_l2(R->carry);   // read by whichever CTA finishes last
  } else if (job.type == kJobWake && tid < kBunchTile) {
    st->qf[tid] = tid < nbt ? R->q_mp_f[m0 + tid] : 0.f;
  }
  if ((job.type == kJobMoments || (job.type == kJobTile && p.fold_moments)) && tid < nbt) {
    const BunchDev bd = p.bunches[R->bunch_base + m0 + tid];
    st->tile0[tid] = bd.tile0;
    st->ntiles[tid] = bd.ntiles;
    st->n[tid] = bd.n;
    st->inv_n[tid] = R->inv_n[m0 + tid];
  }
  if (tid == 64) prefetch_l2(R->turn);
}

// ---------------------------------------------------------------------------
// Moments and histogram reset of a bunch tile (moments job, or the first part
// of a tile job: kF64, and kMixed plans with fold_moments).
// ---------------------------------------------------------------------------
// Per-bunch moments of the turn into the record ring (Sec. 2.4): thread
// (value c, bunch b) sums the push-tile partials of bunch m0+b in a fixed
// order (independent loads, FP64 adds), then lane b of warp 0 forms the
// moments.  FP64 stays lane-parallel: GB300 spends ~20 FP64-pipe clocks on a
// warp instruction whatever its active lanes.  Also zeroes the other
// histogram buffer of these bunches (the next turn's push fills it).
// st: the tile's staged bunch descriptors, or nullptr to read them from the plan.
__device__ void moments_job(const Plan &p, const RunDev *__restrict__ R, int m0, int nbt, int par, long long turn,
                            double (*s_sum)[kBunchTile], const PostStage *st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = R->nb, nbins = R->nbins;
  // per bunch: 0 the tau plane and 1 the delta plane (mean and variance,
  // slots 0-1 and 2-3), 2 the outside count (slot 4), and with a transverse
  // plane the raw sums of partial columns 6-9 (slots 5-8)
  const int ncol = R->trans ? 7 : 3;
  for (int ci = threadIdx.x >> 5; ci < ncol; ci += kPostThreads / 32) {
    const int b = threadIdx.x & 31;
    if (b < nbt) {
      int tile0, ntiles;
      if (st) {
        tile0 = st->tile0[b];
        ntiles = st->ntiles[b];
      } else {
        const BunchDev bd = p.bunches[R->bunch_base + m0 + b];
        tile0 = bd.tile0;
        ntiles = bd.ntiles;
      }
      const double *pp = p.partial + (size_t)tile0 * kPartials;
      if (ci < 2) {
        // each tile summed u = x - r_t and u^2 over its n_t particles (r_t
        // its reference): the mean is sum(S1_t + n_t r_t) / N, the second
        // moment about it sum(S2_t + 2 e_t S1_t + n_t e_t^2) / N with
        // e_t = r_t - mean (the pairwise combination of the variance), all
        // in FP64 in tile order
        const int c1 = ci == 0 ? 0 : 2, cr = ci == 0 ? 5 : 10;
        const double inv_n = st ? st->inv_n[b] : R->inv_n[m0 + b];
        double a = 0.0;
        for (int i = 0; i < ntiles; ++i) {
          const double *q = pp + (size_t)i * kPartials;
          a += fma(q[11], q[cr], q[c1]);
        }
        const double mean = a * inv_n;
        double q2 = 0.0;
        for (int i = 0; i < ntiles; ++i) {
          const double *q = pp + (size_t)i * kPartials;
          const double e = q[cr] - mean;
          q2 += fma(q[11] * e, e, fma(2.0 * e, q[c1], q[c1 + 1]));
        }
        s_sum[2 * ci][b] = mean;
        s_sum[2 * ci + 1][b] = q2 * inv_n;
      } else {
        const int cidx = ci == 2 ? 4 : ci + 3;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int i = 0;
        for (; i + 4 <= ntiles; i += 4) {
          a0 += pp[(size_t)(i + 0) * kPartials + cidx];
          a1 += pp[(size_t)(i + 1) * kPartials + cidx];
          a2 += pp[(size_t)(i + 2) * kPartials + cidx];
          a3 += pp[(size_t)(i + 3) * kPartials + cidx];
        }
        for (; i < ntiles; ++i) a0 += pp[(size_t)i * kPartials + cidx];
        s_sum[ci + 2][b] = (a0 + a1) + (a2 + a3);
      }
    }
  }
  int32_t *hz = R->hist + ((size_t)(par ^ 1) * nb + m0) * nbins;
  for (int i = threadIdx.x; i < nbt * nbins; i += kPostThreads) hz[i] = 0;
  if (R->trans) {
    // the other dipole buffer too (int64 fixed point for kMixed, double for kF64)
    const size_t off = ((size_t)(par ^ 1) * nb + m0) * nbins;
    if (R->precision == kMixed)
      for (int i = threadIdx.x; i < nbt * nbins; i += kPostThreads) static_cast<long long *>(R->dip)[off + i] = 0;
    else
      for (int i = threadIdx.x; i < nbt * nbins; i += kPostThreads) static_cast<double *>(R->dip)[off + i] = 0.0;
  }
  __syncthreads();
  if (warp == 0 && lane < nbt) {
    const double inv_n = st ? st->inv_n[lane] : R->inv_n[m0 + lane];
    const double s4 = s_sum[4][lane];
    double *rec = R->rec + ((size_t)(turn % R->cap) * nb + m0 + lane) * kRecord;
    rec[0] = s_sum[0][lane];
    rec[1] = sqrt(fmax(s_sum[1][lane], 0.0));
    rec[2] = s_sum[2][lane];
    rec[3] = sqrt(fmax(s_sum[3][lane], 0.0));
    rec[4] = (double)(st ? st->n[lane] : p.bunches[R->bunch_base + m0 + lane].n) - s4;
    rec[5] = s4;
    if (R->trans) {
      const double mx = s_sum[5][lane] * inv_n, mp = s_sum[7][lane] * inv_n;
      const double vx = fmax(fma(s_sum[6][lane], inv_n, -mx * mx), 0.0);
      const double vp = fmax(fma(s_sum[8][lane], inv_n, -mp * mp), 0.0);
      double *tr = R->trec + ((size_t)(turn % R->cap) * nb + m0 + lane) * kTRecord;
      tr[0] = mx;
      tr[1] = sqrt(vx);
      tr[2] = mp;
      tr[3] = sqrt(vp);
      // charge x centroid of the bunch for the long-range resistive wall
      if (R->rw_nh > 0) R->rw_cent[(size_t)(turn % (R->rw_nh + 1)) * nb + m0 + lane] = R->q_mp[m0 + lane] * s_sum[5][lane];
    }
  }
}

// Transverse short-range voltage (Eq. 6, second line) of the tile's bunches,
// rows [32 sub, 32 sub + 32): V[j] = q sum_{k<=j} dip[k] Wx((j - k) Delta)
// from this turn's dipole sums, FP32 on the CUDA cores (kMixed; the
// contraction is small: 32 rows x 32 bunches x <= 256 lags per job).  Thread
// (row j, warp g) keeps one accumulator for each of the bunches g, g + 8,
// ... (independent chains, each summed over k in order, as a single chain
// would); the dipole sums are read four cells at a time, and the lag table
// is stored behind nbins zeros so that the last group of four needs no test.
__device__ void trans_job_f32(const RunDev *__restrict__ R, const PostJob &job, int par, uint8_t *smem) {
  constexpr int kGroups = kPostThreads / kTransRows, kPer = kBunchTile / kGroups;
  const int nbins = R->nbins, nb = R->nb;
  const int m0 = job.bt * kBunchTile, nbt = min(kBunchTile, nb - m0);
  float *sWp = reinterpret_cast<float *>(smem);   // [nbins zeros | Wx[0 .. nbins)]
  float *sD = sWp + 2 * nbins;                     // [kBunchTile][nbins], rows past nbt zero
  const long long *dg = static_cast<const long long *>(R->dip) + ((size_t)par * nb + m0) * nbins;
  const float du = R->f_dip_unit;
  for (int k = threadIdx.x; k < nbins; k += kPostThreads) {
    sWp[k] = 0.f;
    sWp[nbins + k] = R->tlag_f[k];
  }
  for (int i = threadIdx.x; i < kBunchTile * nbins; i += kPostThreads)
    sD[i] = i < nbt * nbins ? dip_q_to_f(dg[i], du) : 0.f;
  __syncthreads();
  const int r = threadIdx.x % kTransRows, g = threadIdx.x / kTransRows, j = job.sub * kTransRows + r;
  float acc[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) acc[i] = 0.f;
  const float *wj = sWp + nbins + j;
  for (int k = 0; k <= j; k += 4) {
    const float w0 = wj[-k], w1 = wj[-k - 1], w2 = wj[-k - 2], w3 = wj[-k - 3];   // zero for lags below 0
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const float4 d = *reinterpret_cast<const float4 *>(sD + (size_t)(g + kGroups * i) * nbins + k);
      acc[i] = fmaf(d.x, w0, acc[i]);
      acc[i] = fmaf(d.y, w1, acc[i]);
      acc[i] = fmaf(d.z, w2, acc[i]);
      acc[i] = fmaf(d.w, w3, acc[i]);
    }
  }
  float *vt = static_cast<float *>(R->vt);
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int b = g + kGroups * i;
    if (b < nbt) vt[(size_t)(m0 + b) * nbins + j] = R->q_mp_f[m0 + b] * acc[i];
  }
}

// The same in FP64 for bunch job.bt, rows [32 sub, 32 sub + 32), 8 threads per row (kF64).
__device__ void trans_job_f64(const RunDev *__restrict__ R, const PostJob &job, int par, uint8_t *smem) {
  const int nbins = R->nbins;
  const int m = job.bt, chunk = job.sub;
  double *sW = reinterpret_cast<double *>(smem);
  double *sD = sW + nbins;
  const double *dg = static_cast<const double *>(R->dip) + ((size_t)par * R->nb + m) * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPostThreads) {
    sW[k] = R->tlag[k];
    sD[k] = dg[k];
  }
  __syncthreads();
  const int row = threadIdx.x >> 3, sub = threadIdx.x & 7;
  const int j = chunk * kF64RowChunk + row;
  double acc = 0.0;
  if (j < nbins)
    for (int k = sub; k <= j; k += 8) acc = fma(sD[k], sW[j - k], acc);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
  if (sub == 0 && j < nbins) static_cast<double *>(R->vt)[(size_t)m * nbins + j] = R->q_mp[m] * acc;
}

// Warp 0 of a tile job, lane b for bunch m0 + b: E_m = c q_m sum_m, then the
// affine scan across the tile (lane b holds x -> a_m (x + E_{m-1}); bunch m0
// maps the tile's entering value).  Writes P_m, Q_m to pq[2 b], pq[2 b + 1]
// and the tile aggregate to agg[0], agg[1].  The mixed post kernel also runs
// it on placeholder values into shared scratch before its grid dependency
// wait, so that this code, which runs once per turn after the push has
// displaced it from the instruction caches, is cached when the turn's
// data arrives (tile_scan_warp; the FP64 kernel inlines the body).
__device__ __forceinline__ void tile_scan_body(double2 c, double2 sum, double q, double2 a, int nbt, double2 *pq,
                                               double2 *agg) {
  const int lane = threadIdx.x & 31;
  double2 E = make_double2(0.0, 0.0);
  if (lane < nbt) E = cmul(c, make_double2(q * sum.x, q * sum.y));
  const double2 Eprev = shfl_up_d2(E, 1);
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
  if (lane < nbt) {
    A = a;
    if (lane > 0) B = cmul(A, Eprev);
  }
  warp_scan_affine(A, B, nbt);
  if (lane < nbt) {
    pq[(size_t)lane * 2] = A;
    pq[(size_t)lane * 2 + 1] = B;
  }
  if (lane == nbt - 1) {
    agg[0] = A;
    agg[1] = cadd(B, E);
  }
}
__device__ __noinline__ void tile_scan_warp(double2 c, double2 sum, double q, double2 a, int nbt, double2 *pq,
                                            double2 *agg) {
  tile_scan_body(c, sum, q, a, nbt, pq, agg);
}

// Long-range emission and the tile's affine scan, per long-range resonator.
// Emission sums sum_k count[m,k] e^{-s tau_k}: 8 threads per bunch, all 32
// bunches of the tile at once.
// tabf, st: staged emission table and bunch constants (kMixed), or nullptr
// to read them from the run (kF64).
template <int PREC>
__device__ void tile_job(const Plan &p, const RunDev *__restrict__ R, const PostJob &job, int par, double2 *sE,
                         float2 *sEf, const float2 *tabf, const PostStage *st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = R->nb, nbins = R->nbins;
  const int m0 = job.bt * kBunchTile;
  const int nbt = min(kBunchTile, nb - m0);
  const int32_t *hcur = R->hist + ((size_t)par * nb + m0) * nbins;
  const int b = threadIdx.x >> 3, sub = threadIdx.x & 7;   // kPostThreads / 8 == kBunchTile
  for (int r = 0; r < R->nlong; ++r) {
    // source of the emission: the cell counts, or for a transverse entry the dipole sums
    const bool tplane = R->lr_plane[r] != 0;
    if (PREC == kMixed) {
      // thread sub takes the 4-cell groups g = sub + 8 i (nbins 128 or 256:
      // at most kGroups), all of its loads issued before the sums
      constexpr int kGroups = 256 / 4 / 8;
      const int ng = nbins / 32;
      float ax = 0.f, ay = 0.f;
      if (b < nbt) {
        float4 cnt[kGroups];
        if (tplane) {
          const longlong2 *d2 = reinterpret_cast<const longlong2 *>(static_cast<const long long *>(R->dip) +
                                                                    ((size_t)par * nb + m0 + b) * nbins);
          const float du = R->f_dip_unit;
#pragma unroll
          for (int i = 0; i < kGroups; ++i) {
            const longlong2 a = i < ng ? d2[2 * (sub + 8 * i)] : make_longlong2(0, 0);
            const longlong2 c = i < ng ? d2[2 * (sub + 8 * i) + 1] : make_longlong2(0, 0);
            cnt[i] = make_float4(dip_q_to_f(a.x, du), dip_q_to_f(a.y, du), dip_q_to_f(c.x, du), dip_q_to_f(c.y, du));
          }
        } else {
          const int4 *h4 = reinterpret_cast<const int4 *>(hcur + (size_t)b * nbins);
#pragma unroll
          for (int i = 0; i < kGroups; ++i) {
            const int4 v = i < ng ? h4[sub + 8 * i] : make_int4(0, 0, 0, 0);
            cnt[i] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
          }
        }
        // two cells' factors (Re, Im, Re, Im) per float4
        const float4 *t4 = reinterpret_cast<const float4 *>((tabf ? tabf : R->emis_f) + (size_t)r * nbins);
#pragma unroll
        for (int i = 0; i < kGroups; ++i) {
          if (i < ng) {
            const int g = sub + 8 * i;
            const float4 e0 = t4[2 * g], e1 = t4[2 * g + 1];
            ax = fmaf(cnt[i].x, e0.x, ax);
            ay = fmaf(cnt[i].x, e0.y, ay);
            ax = fmaf(cnt[i].y, e0.z, ax);
            ay = fmaf(cnt[i].y, e0.w, ay);
            ax = fmaf(cnt[i].z, e1.x, ax);
            ay = fmaf(cnt[i].z, e1.y, ay);
            ax = fmaf(cnt[i].w, e1.z, ax);
            ay = fmaf(cnt[i].w, e1.w, ay);
          }
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xFFFFFFFFu, ax, o);
        ay += __shfl_xor_sync(0xFFFFFFFFu, ay, o);
      }
      if (sub == 0 && b < nbt) sEf[b] = make_float2(ax, ay);
    } else {
      double ax = 0.0, ay = 0.0;
      if (b < nbt) {
        const int32_t *hrow = hcur + (size_t)b * nbins;
        const double *drow = tplane ? static_cast<const double *>(R->dip) + ((size_t)par * nb + m0 + b) * nbins : nullptr;
        const double2 *tab = R->emis + (size_t)r * nbins;
        for (int k = sub; k < nbins; k += 8) {
          const double cnt = tplane ? drow[k] : (double)hrow[k];
          ax = fma(cnt, tab[k].x, ax);
          ay = fma(cnt, tab[k].y, ay);
        }
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xFFFFFFFFu, ax, o);
        ay += __shfl_xor_sync(0xFFFFFFFFu, ay, o);
      }
      if (sub == 0 && b < nbt) sE[b] = make_double2(ax, ay);
    }
    __syncthreads();
    if (warp == 0) {
      const int m = m0 + lane;
      double2 sum = make_double2(0.0, 0.0), a = make_double2(1.0, 0.0);
      double q = 0.0;
      if (lane < nbt) {
        sum = PREC == kMixed ? make_double2((double)sEf[lane].x, (double)sEf[lane].y) : sE[lane];
        q = st ? st->q[lane] : R->q_mp[m];
        a = st ? st->step[r][lane] : R->step[(size_t)r * nb + m];
      }
      double2 *const pq = R->pq + ((size_t)r * nb + m0) * 2;
      double2 *const agg = R->agg + ((size_t)r * R->ntile_b + job.bt) * 2;
      if (PREC == kMixed)
        tile_scan_warp(R->lr_c[r], sum, q, a, nbt, pq, agg);
      else
        tile_scan_body(R->lr_c[r], sum, q, a, nbt, pq, agg);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Last CTA: compose tile aggregates with the carry, advance the turns.
// ---------------------------------------------------------------------------
// Compose the tile aggregates of pair (run R, long-range resonator r) with
// the carry K; nt tiles, one lane per tile.
__device__ __forceinline__ void finish_pair(int nt, double2 K, const double2 *agg, double2 *y, double2 *carry) {
  const int lane = threadIdx.x & 31;
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
  if (lane < nt) {
    A = __ldcg(agg + (size_t)lane * 2);
    B = __ldcg(agg + (size_t)lane * 2 + 1);
  }
  warp_scan_affine(A, B, nt);
  const double2 yn = cfma(A, K, B);   // value leaving tile `lane`
  if (lane + 1 < nt) y[lane + 1] = yn;
  if (lane == 0) y[0] = K;
  __syncwarp();
  if (lane == nt - 1) *carry = yn;
}

// own, Rown: the run of this CTA's job and its descriptor (a staged copy).
__device__ void finish_turn(const Plan &p, int own, const RunDev *Rown, unsigned int njobs) {
  __shared__ int s_last;
  const int warp = threadIdx.x >> 5;
  // Read before the count, so that the last CTA's chain after it is the
  // aggregate loads, the scan and the stores: the turn counters (they change
  // only at the end of this function) and, where warp w's first pair (pair w)
  // belongs to the first run, that pair's layout and carry (written only by
  // the last CTA of the previous post kernel).
  long long *const tp =
      threadIdx.x < p.nruns ? (threadIdx.x == own ? Rown->turn : p.runs[threadIdx.x].turn) : nullptr;
  const long long turn0 = tp ? *tp : 0;
  const RunDev *R0 = own == 0 ? Rown : p.runs;
  const bool pre = p.nruns > 0 && warp < R0->nlong;
  int nt0 = 0;
  double2 K0 = make_double2(0.0, 0.0);
  const double2 *agg0 = nullptr;
  double2 *y0 = nullptr, *carry0 = nullptr;
  if (pre) {
    nt0 = R0->ntile_b;
    agg0 = R0->agg + (size_t)warp * nt0 * 2;
    y0 = R0->y + (size_t)warp * nt0;
    carry0 = R0->carry + warp;
    K0 = __ldcg(carry0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();   // this CTA's results before its count (release)
    const unsigned int prev = atomicAdd(p.done, 1u);
    s_last = (prev == njobs - 1u) ? 1 : 0;   // njobs: of every kernel of the turn's post
    if (s_last) __threadfence();   // acquire: every thread of the CTA reads after the barrier below
  }
  __syncthreads();
  if (!s_last) return;
  // one warp per (run, long-range resonator)
  if (pre) finish_pair(nt0, K0, agg0, y0, carry0);
  int pair = 0;
  for (int ri = 0; ri < p.nruns; ++ri) {
    const RunDev *R = p.runs + ri;
    for (int r = 0; r < R->nlong; ++r, ++pair) {
      if (pair % (kPostThreads / 32) != warp || (pre && pair == warp)) continue;
      const int nt = R->ntile_b;
      finish_pair(nt, __ldcg(R->carry + r), R->agg + (size_t)r * nt * 2, R->y + (size_t)r * nt, R->carry + r);
    }
  }
  __syncthreads();
  if (tp) *tp = turn0 + 1;
  for (int ri = threadIdx.x + kPostThreads; ri < p.nruns; ri += kPostThreads) p.runs[ri].turn[0] += 1;
  if (threadIdx.x == 0) *p.done = 0u;
}

// ---------------------------------------------------------------------------
// kMixed wake job: tcgen05 Toeplitz contraction of one M-tile (128 cells) for
// a tile of 32 bunches.
//   A (shared) = [T_hi | T_lo], 128 x 2 nbins BF16, K-major core matrices,
//                bulk-copied from a pre-laid-out image (constant per run);
//   B (shared) = 96 x nbins BF16, rows = (byte plane, bunch), built here from
//                the int32 counts of the turn;
//   D (tensor memory) = 128 lanes x 96 FP32 columns.
// ---------------------------------------------------------------------------
constexpr int kWakeN = 3 * kBunchTile;   // 96
constexpr uint32_t kTmemCols = 256;      // power of two >= kWakeN, with headroom (two accumulators for kWakeBoth)

// Operand A of M-tile mt: rows [128 mt, 128 mt + 128) of the lower triangular
// Toeplitz matrix only involve columns k < Kmt = 128 (mt + 1), so the image
// holds [T_hi | T_lo] over 2 Kmt columns: 512 Kmt bytes at offset 512 * 128
// * mt (mt + 1) (the images of the earlier M-tiles).
__device__ __forceinline__ int wake_kmt(int mt, int nbins) { return min(nbins, 128 * (mt + 1)); }
__device__ __forceinline__ size_t wake_img_offset(int mt) { return (size_t)512 * 128 * mt * (mt + 1) / 2; }

// Prologue: barriers, tensor memory, and the bulk copy of the constant A
// image; safe to run before the push kernel of the turn has completed.
__device__ void wake_prologue(const RunDev *__restrict__ R, const PostJob &job, uint8_t *smem, uint64_t *bars,
                              uint32_t *tmem_slot, int *s_flag) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = job.sub == kWakeBoth ? 0 : job.sub;   // both M-tiles: M-tile 0 first
  const int kmt = wake_kmt(mt, R->nbins);
  const uint32_t a_bytes = (uint32_t)kmt * 512u;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_mbar_init();
    *s_flag = 0;
    const uint8_t *src = static_cast<const uint8_t *>(R->toep) + wake_img_offset(mt);
    mbar_arrive_expect_tx(&bars[0], a_bytes);
    for (uint32_t off = 0; off < a_bytes; off += 32768u)
      bulk_g2s(smem + off, src + off, min(32768u, a_bytes - off), &bars[0]);
  }
  if (warp == 0) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// B of a wake job: the counts of the tile's 32 bunches over cells [0, kmt)
// split into three exact BF16 byte planes (K-major core matrices).
__device__ __forceinline__ void wake_build_b(const Plan &p, const RunDev *__restrict__ R, int bt, int par, uint8_t *sB,
                                             int kmt, bool check_counts) {
  const int tid = threadIdx.x;
  const int nbins = R->nbins;
  const int nb = R->nb;
  const int m0 = bt * kBunchTile;
  const int nbt = min(kBunchTile, nb - m0);
  // B: counts of the 32 bunches split into three exact BF16 byte planes.
  // Item (bunch b, 8-cell group kg) = idx = kg * 32 + b; a thread's items are
  // idx = tid + i kPostThreads (at most kItems with nbins <= 256), and all of
  // its loads are issued before the first conversion: one round trip to L2.
  const int32_t *hg = R->hist + ((size_t)par * nb + m0) * nbins;
  const int KG = kmt / 8;
  constexpr int kItems = kBunchTile * 32 / kPostThreads;
  int4 cv[kItems][2];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int idx = tid + i * kPostThreads, b = idx % kBunchTile, kg = idx / kBunchTile;
    cv[i][0] = cv[i][1] = make_int4(0, 0, 0, 0);
    if (kg < KG && b < nbt) {
      const int4 *src = reinterpret_cast<const int4 *>(hg + (size_t)b * nbins + kg * 8);
      cv[i][0] = src[0];
      cv[i][1] = src[1];
    }
  }
  if (check_counts) {
    bool bad = false;
#pragma unroll
    for (int i = 0; i < kItems; ++i)
      bad |= ((uint32_t)cv[i][0].x | (uint32_t)cv[i][0].y | (uint32_t)cv[i][0].z | (uint32_t)cv[i][0].w |
              (uint32_t)cv[i][1].x | (uint32_t)cv[i][1].y | (uint32_t)cv[i][1].z | (uint32_t)cv[i][1].w) >= (1u << 24);
    if (bad) atomicCAS(p.error, kErrNone, kErrCount);
  }
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int idx = tid + i * kPostThreads, b = idx % kBunchTile, kg = idx / kBunchTile;
    if (kg >= KG) continue;
    const int c[8] = {cv[i][0].x, cv[i][0].y, cv[i][0].z, cv[i][0].w, cv[i][1].x, cv[i][1].y, cv[i][1].z, cv[i][1].w};
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float lo = (float)((c[2 * e] >> (8 * pl)) & 0xFF);
        const float hi = (float)((c[2 * e + 1] >> (8 * pl)) & 0xFF);
        const __nv_bfloat162 v2 = __floats2bfloat162_rn(lo, hi);
        w[e] = *reinterpret_cast<const uint32_t *>(&v2);
      }
      const int n = pl * kBunchTile + b;
      uint8_t *dst = sB + ((size_t)kg * (kWakeN / 8) + (n >> 3)) * 128 + (n & 7) * 16;
      *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Main part: B from the turn's counts, the MMAs (issued by one thread, run
// asynchronously), then the epilogue from tensor memory.
// qf: the charges of the tile's 32 bunches (staged, or the run's array at
// the tile).  check_counts: record kErrCount in the error word if a count
// lies outside [0, 2^24) (counts from a caller; tracking caps its bunches
// below 2^24 particles, so its counts never need the test).
__device__ void wake_job_tc(const Plan &p, const RunDev *__restrict__ R, const PostJob &job, int par, uint8_t *smem,
                            uint64_t *bars, uint32_t *tmem_slot, int *s_flag, const float *qf,
                            bool check_counts = false) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbins = R->nbins;
  const int nb = R->nb;
  const int mt = job.sub;
  const int kmt = wake_kmt(mt, nbins);
  const int m0 = job.bt * kBunchTile;
  const int nbt = min(kBunchTile, nb - m0);
  uint8_t *sA = smem;
  uint8_t *sB = smem + (size_t)nbins * 512u;   // after the largest A image
  const uint32_t lboA = 16u * 128u;           // next 8-column K group: 16 row groups later
  const uint32_t lboB = (uint32_t)(kWakeN / 8) * 128u;
  const uint32_t tmem = *tmem_slot;

  wake_build_b(p, R, job.bt, par, sB, kmt, check_counts);
  fence_proxy_async_smem();
  __syncthreads();

  if (tid == 0) {
    if (!mbar_wait_bounded(&bars[0], 0, kWaitLimitNs)) {
      atomicExch(p.error, kErrTimeout);
      *s_flag = 1;
    } else {
      tc_fence_after();
      const uint32_t idesc = idesc_bf16_f32(128, kWakeN);
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
      const int ks_half = kmt / 16;
      for (int ks = 0; ks < 2 * ks_half; ++ks) {
        const uint64_t ad = smem_desc_kmajor(a0 + (uint32_t)ks * 2u * lboA, lboA, 128u);
        const uint64_t bd = smem_desc_kmajor(b0 + (uint32_t)(ks % ks_half) * 2u * lboB, lboB, 128u);
        umma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
      umma_commit(&bars[1]);
    }
  }
  __syncthreads();
  const bool aborted = *s_flag != 0;
  if (!aborted && warp < 4) {
    if (!mbar_wait_bounded(&bars[1], 0, kWaitLimitNs)) {
      if (lane == 0) atomicExch(p.error, kErrTimeout);
    } else {
      tc_fence_after();
      float d0[32], d1[32], d2[32];
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
      tmem_ld32(tl + 0, d0);
      tmem_ld32(tl + 32, d1);
      tmem_ld32(tl + 64, d2);
      const int j = mt * 128 + warp * 32 + lane;
      float *vsr = static_cast<float *>(R->vsr);
#pragma unroll
      for (int b = 0; b < kBunchTile; ++b) {
        if (b < nbt) {
          const float q = qf[b];
          vsr[(size_t)(m0 + b) * nbins + j] = q * fmaf(65536.f, d2[b], fmaf(256.f, d1[b], d0[b]));
        }
      }
    }
  }
  if (aborted && tid == 0) mbar_wait_bounded(&bars[0], 0, kWaitLimitNs);   // let the copy land before exit
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Epilogue of M-tile mt of wake_job_both (a warp of warps 0-3): its 32 rows
// from tensor-memory columns [128 mt, 128 mt + 96), the byte planes
// recombined, times the bunch charges.  Not inlined, so that the two
// accumulators' registers are not live at once.
__device__ __noinline__ void wake_epilogue(const RunDev *__restrict__ R, uint32_t tl, int mt, int m0, int nbt,
                                           const float *qf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nbins = R->nbins;
  tc_fence_after();
  float d0[32], d1[32], d2[32];
  const uint32_t col = 128u * (uint32_t)mt;
  tmem_ld32(tl + col + 0, d0);
  tmem_ld32(tl + col + 32, d1);
  tmem_ld32(tl + col + 64, d2);
  const int j = mt * 128 + warp * 32 + lane;
  float *vsr = static_cast<float *>(R->vsr);
#pragma unroll
  for (int b = 0; b < kBunchTile; ++b) {
    if (b < nbt) {
      const float q = qf[b];
      vsr[(size_t)(m0 + b) * nbins + j] = q * fmaf(65536.f, d2[b], fmaf(256.f, d1[b], d0[b]));
    }
  }
}

// Both M-tiles of a 256-cell mesh in one job (plans whose post jobs fill
// several waves: one job fewer per bunch tile, and B built once).  M-tile 0's
// image (64 KB, from the prologue) is contracted into tensor-memory columns
// [0, 96); once those MMAs have read it, M-tile 1's image (128 KB) is copied
// over it and contracted into columns [128, 224).  Thread 128 (warp 4) issues
// and sequences; warps 0-3 read the two accumulators as they complete.
// Barriers: bars[0] image copies (phase 0: M-tile 0, phase 1: M-tile 1),
// bars[1] / bars[2] the MMAs of M-tile 0 / 1 (one phase each, so that no
// waiter can miss a phase).
__device__ void wake_job_both(const Plan &p, const RunDev *__restrict__ R, const PostJob &job, int par, uint8_t *smem,
                              uint64_t *bars, uint32_t *tmem_slot, int *s_flag, const float *qf) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbins = R->nbins;   // 256
  const int m0 = job.bt * kBunchTile;
  const int nbt = min(kBunchTile, R->nb - m0);
  uint8_t *sA = smem;
  uint8_t *sB = smem + (size_t)nbins * 512u;
  const uint32_t lboA = 16u * 128u;
  const uint32_t lboB = (uint32_t)(kWakeN / 8) * 128u;
  const uint32_t tmem = *tmem_slot;
  wake_build_b(p, R, job.bt, par, sB, nbins, false);
  fence_proxy_async_smem();
  __syncthreads();

  constexpr int kIssuer = 128;
  if (tid == kIssuer) {
    const uint32_t idesc = idesc_bf16_f32(128, kWakeN);
    const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
    bool ok = mbar_wait_bounded(&bars[0], 0, kWaitLimitNs);   // M-tile 0's image
    if (ok) {
      tc_fence_after();
      const int ks_half = wake_kmt(0, nbins) / 16;
      for (int ks = 0; ks < 2 * ks_half; ++ks) {
        const uint64_t ad = smem_desc_kmajor(a0 + (uint32_t)ks * 2u * lboA, lboA, 128u);
        const uint64_t bd = smem_desc_kmajor(b0 + (uint32_t)(ks % ks_half) * 2u * lboB, lboB, 128u);
        umma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
      umma_commit(&bars[1]);
      ok = mbar_wait_bounded(&bars[1], 0, kWaitLimitNs);   // those MMAs have read the image
    }
    bool copied = false;
    if (ok) {
      tc_fence_after();
      fence_proxy_async_smem();
      const uint32_t a_bytes = (uint32_t)wake_kmt(1, nbins) * 512u;
      const uint8_t *src = static_cast<const uint8_t *>(R->toep) + wake_img_offset(1);
      mbar_arrive_expect_tx(&bars[0], a_bytes);
      for (uint32_t off = 0; off < a_bytes; off += 32768u)
        bulk_g2s(sA + off, src + off, min(32768u, a_bytes - off), &bars[0]);
      copied = true;
      ok = mbar_wait_bounded(&bars[0], 1, kWaitLimitNs);   // M-tile 1's image
    }
    if (ok) {
      tc_fence_after();
      const int ks_half = wake_kmt(1, nbins) / 16;
      for (int ks = 0; ks < 2 * ks_half; ++ks) {
        const uint64_t ad = smem_desc_kmajor(a0 + (uint32_t)ks * 2u * lboA, lboA, 128u);
        const uint64_t bd = smem_desc_kmajor(b0 + (uint32_t)(ks % ks_half) * 2u * lboB, lboB, 128u);
        umma_bf16(tmem + 128u, ad, bd, idesc, ks > 0 ? 1u : 0u);
      }
      umma_commit(&bars[2]);
    } else {
      atomicExch(p.error, kErrTimeout);
      *s_flag = 1;
      // let the copies in flight land before the CTA exits
      mbar_wait_bounded(&bars[0], 0, kWaitLimitNs);
      if (copied) mbar_wait_bounded(&bars[0], 1, kWaitLimitNs);
    }
  }
  if (warp < 4) {
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    if (!mbar_wait_bounded(&bars[1], 0, kWaitLimitNs)) {
      if (lane == 0) atomicExch(p.error, kErrTimeout);
    } else {
      wake_epilogue(R, tl, 0, m0, nbt, qf);
      if (!mbar_wait_bounded(&bars[2], 0, kWaitLimitNs)) {
        if (lane == 0) atomicExch(p.error, kErrTimeout);
      } else {
        wake_epilogue(R, tl, 1, m0, nbt, qf);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

__device__ __forceinline__ void trace_mark(const Plan &p, int slot, int jobi) {
  if (p.trace != nullptr && threadIdx.x == 0) p.trace[(size_t)jobi * 3 + slot] = global_timer_ns();
}

// Every job of the plan, one CTA per job.
__global__ void __launch_bounds__(kPostThreads, 1) k_post_mixed(const Plan p) {
  constexpr int MODE = 0;
  const int job0 = 0;
  extern __shared__ __align__(1024) uint8_t sm_post[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_flag;
  __shared__ double2 sE[kBunchTile];
  __shared__ float2 sEf[kBunchTile];
  __shared__ double s_sum[9][kBunchTile];
  __shared__ PostStage st;
  __shared__ RunDev sR;
  __shared__ double2 s_scr[2 * kBunchTile + 2];
  const int jobi = job0 + (int)blockIdx.x;
  const PostJob job = p.jobs[jobi];
  trace_mark(p, 0, jobi);
  // The run descriptor, copied before the wait: the push streams the particle
  // state through L2 and evicts it, and after the wait every read of it would
  // be a miss behind the next push's first bulk copies.
  static_assert(sizeof(RunDev) % 16 == 0 && sizeof(RunDev) / 16 <= kPostThreads, "run descriptor copy");
  if (threadIdx.x < sizeof(RunDev) / 16)
    reinterpret_cast<int4 *>(&sR)[threadIdx.x] = reinterpret_cast<const int4 *>(p.runs + job.run)[threadIdx.x];
  __syncthreads();
  const RunDev *R = &sR;
  // tile jobs keep the emission table where wake jobs keep their operands
  float2 *tabf = reinterpret_cast<float2 *>(sm_post);
  if (MODE != 2 && job.type == kJobWake) wake_prologue(R, job, sm_post, bars, &tmem_slot, &s_flag);   // A image first
  post_stage(p, R, job, &st, tabf);
  if (MODE != 1 && job.type == kJobTile && threadIdx.x < 32)   // code warm-up, into shared scratch
    tile_scan_warp(make_double2(0.0, 0.0), make_double2(0.0, 0.0), 0.0, make_double2(1.0, 0.0), kBunchTile, s_scr,
                   s_scr + 2 * kBunchTile);
  __syncthreads();
  grid_dependency_wait();     // the push of this turn has completed
  grid_dependents_launch();   // the next push may start its prologue (particle prefetch)
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);
  if (MODE != 2 && job.type == kJobWake && job.sub == kWakeBoth)
    wake_job_both(p, R, job, par, sm_post, bars, &tmem_slot, &s_flag, st.qf);
  else if (MODE != 2 && job.type == kJobWake)
    wake_job_tc(p, R, job, par, sm_post, bars, &tmem_slot, &s_flag, st.qf);
  else if (MODE != 1 && job.type == kJobTile) {
    if (p.fold_moments) {
      moments_job(p, R, job.bt * kBunchTile, min(kBunchTile, R->nb - job.bt * kBunchTile), par, turn, s_sum, &st);
      __syncthreads();
    }
    tile_job<kMixed>(p, R, job, par, sE, sEf, tabf, &st);
  } else if (MODE != 1 && job.type == kJobMoments)
    moments_job(p, R, job.bt * kBunchTile, min(kBunchTile, R->nb - job.bt * kBunchTile), par, turn, s_sum, &st);
  else
    trans_job_f32(R, job, par, sm_post);
  trace_mark(p, 1, jobi);
  finish_turn(p, job.run, R, gridDim.x);
  trace_mark(p, 2, jobi);
}

// The two kernels of a split post (Plan::post_split): MODE 1 the wake jobs
// p.jobs[0, post_split), MODE 2 the other jobs p.jobs[job0 + blockIdx.x] (no
// wake job: a small shared-memory footprint, two CTAs per SM).  Both count
// into the same completion counter, so that the last CTA of either finishes
// the turn after every job of both.
template <int MODE>
__global__ void __launch_bounds__(kPostThreads, MODE == 2 ? 2 : 1) k_post_split(const Plan p, int job0) {
  extern __shared__ __align__(1024) uint8_t sm_post[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_flag;
  __shared__ double2 sE[kBunchTile];
  __shared__ float2 sEf[kBunchTile];
  __shared__ double s_sum[9][kBunchTile];
  __shared__ PostStage st;
  __shared__ RunDev sR;
  __shared__ double2 s_scr[2 * kBunchTile + 2];
  const int jobi = job0 + (int)blockIdx.x;
  const PostJob job = p.jobs[jobi];
  trace_mark(p, 0, jobi);
  // The run descriptor, copied before the wait: the push streams the particle
  // state through L2 and evicts it, and after the wait every read of it would
  // be a miss behind the next push's first bulk copies.
  static_assert(sizeof(RunDev) % 16 == 0 && sizeof(RunDev) / 16 <= kPostThreads, "run descriptor copy");
  if (threadIdx.x < sizeof(RunDev) / 16)
    reinterpret_cast<int4 *>(&sR)[threadIdx.x] = reinterpret_cast<const int4 *>(p.runs + job.run)[threadIdx.x];
  __syncthreads();
  const RunDev *R = &sR;
  // tile jobs keep the emission table where wake jobs keep their operands
  float2 *tabf = reinterpret_cast<float2 *>(sm_post);
  if (MODE != 2 && job.type == kJobWake) wake_prologue(R, job, sm_post, bars, &tmem_slot, &s_flag);   // A image first
  post_stage(p, R, job, &st, tabf);
  if (MODE != 1 && job.type == kJobTile && threadIdx.x < 32)   // code warm-up, into shared scratch
    tile_scan_warp(make_double2(0.0, 0.0), make_double2(0.0, 0.0), 0.0, make_double2(1.0, 0.0), kBunchTile, s_scr,
                   s_scr + 2 * kBunchTile);
  __syncthreads();
  grid_dependency_wait();     // the push of this turn has completed
  grid_dependents_launch();   // the next push may start its prologue (particle prefetch)
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);
  if (MODE != 2 && job.type == kJobWake && job.sub == kWakeBoth)
    wake_job_both(p, R, job, par, sm_post, bars, &tmem_slot, &s_flag, st.qf);
  else if (MODE != 2 && job.type == kJobWake)
    wake_job_tc(p, R, job, par, sm_post, bars, &tmem_slot, &s_flag, st.qf);
  else if (MODE != 1 && job.type == kJobTile) {
    if (p.fold_moments) {
      moments_job(p, R, job.bt * kBunchTile, min(kBunchTile, R->nb - job.bt * kBunchTile), par, turn, s_sum, &st);
      __syncthreads();
    }
    tile_job<kMixed>(p, R, job, par, sE, sEf, tabf, &st);
  } else if (MODE != 1 && job.type == kJobMoments)
    moments_job(p, R, job.bt * kBunchTile, min(kBunchTile, R->nb - job.bt * kBunchTile), par, turn, s_sum, &st);
  else if (MODE != 1 && job.type == kJobTrans)
    trans_job_f32(R, job, par, sm_post);
  trace_mark(p, 1, jobi);
  finish_turn(p, job.run, R, (unsigned int)p.njobs);
  trace_mark(p, 2, jobi);
}

// ---------------------------------------------------------------------------
// kF64 wake job: rows [32 c, 32 c + 32) of one bunch, 8 threads per row.
// ---------------------------------------------------------------------------
__device__ void wake_job_f64(const RunDev *__restrict__ R, const PostJob &job, int par, uint8_t *smem) {
  const int nbins = R->nbins;
  const int m = job.bt, chunk = job.sub;
  double *sW = reinterpret_cast<double *>(smem);
  int *sHc = reinterpret_cast<int *>(sW + nbins);
  const double *lag = static_cast<const double *>(R->toep);
  const int32_t *hg = R->hist + ((size_t)par * R->nb + m) * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPostThreads) {
    sW[k] = lag[k];
    sHc[k] = hg[k];
  }
  __syncthreads();
  const int row = threadIdx.x >> 3, sub = threadIdx.x & 7;
  const int j = chunk * kF64RowChunk + row;
  double acc = 0.0;
  if (j < nbins)
    for (int k = sub; k <= j; k += 8) acc = fma((double)sHc[k], sW[j - k], acc);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
  acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
  if (sub == 0 && j < nbins) static_cast<double *>(R->vsr)[(size_t)m * nbins + j] = R->q_mp[m] * acc;
}

__global__ void __launch_bounds__(kPostThreads) k_post_f64(const Plan p) {
  extern __shared__ __align__(16) uint8_t sm_post64[];
  __shared__ double2 sE[kBunchTile];
  __shared__ float2 sEf[kBunchTile];
  __shared__ double s_sum[9][kBunchTile];
  const PostJob job = p.jobs[blockIdx.x];
  const RunDev *R = p.runs + job.run;
  trace_mark(p, 0, (int)blockIdx.x);
  grid_dependency_wait();
  grid_dependents_launch();
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);
  if (job.type == kJobWake) {
    wake_job_f64(R, job, par, sm_post64);
  } else if (job.type == kJobTrans) {
    trans_job_f64(R, job, par, sm_post64);
  } else {
    const int m0 = job.bt * kBunchTile;
    moments_job(p, R, m0, min(kBunchTile, R->nb - m0), par, turn, s_sum, nullptr);
    __syncthreads();
    tile_job<kF64>(p, R, job, par, sE, sEf, nullptr, nullptr);
  }
  trace_mark(p, 1, (int)blockIdx.x);
  finish_turn(p, job.run, R, gridDim.x);
  trace_mark(p, 2, (int)blockIdx.x);
}

size_t post_smem_bytes(int precision, int max_nbins) {
  // A image + B operand, plus a margin so that every address an MMA could
  // form from these descriptors (even with the K and M/N strides exchanged)
  // stays inside the allocation
  if (precision == kMixed) return (size_t)max_nbins * 512u + (size_t)max_nbins * 2u * kWakeN + 24576u;
  return (size_t)max_nbins * 2 * sizeof(double);   // lag table + counts, or (transverse) lag table + dipole sums
}

// dynamic shared memory of the post kernel without wake jobs (MODE 2): the
// emission table of a tile job, and with a transverse plane the lag table and
// dipole sums of a transverse job (small enough without one that a CTA of it
// fits on an SM beside a wake-job CTA)
static size_t post_small_smem_bytes(int max_nbins, bool trans) {
  const size_t tile = (size_t)kMaxLong * max_nbins * sizeof(float2);
  return trans ? std::max(tile, (size_t)(2 + kBunchTile) * max_nbins * sizeof(float)) : tile;
}

cudaError_t configure_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_post_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)post_smem_bytes(kMixed, 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_post_split<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)post_smem_bytes(kMixed, 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_post_split<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)post_small_smem_bytes(256, true));
  return e;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the wake job, for callers that cannot call
// cudaMalloc (code that runs where the process must not grow its device
// footprint, such as inside another framework's memory pool or a fixed
// device budget).  Its working memory is this file-scope array: the Toeplitz
// operand images (<= 192 KB for 256 cells), the run descriptor, the job list,
// the per-bunch charges and the error word.  Every GPU that loads the library
// holds the array until the process exits.  Calls share it, so calls that
// overlap on the GPU (other streams, other host threads) race.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = 256 * 1024;
constexpr size_t kNoAllocImgBytes = 196608;                       // 512 * (128 + 256)
constexpr size_t kNoAllocRunOff = kNoAllocImgBytes;               // RunDev
constexpr size_t kNoAllocJobsOff = kNoAllocRunOff + 1024;         // PostJob[<= 64]
constexpr size_t kNoAllocQOff = kNoAllocJobsOff + 1024;           // float[<= kMaxBunches]
constexpr size_t kNoAllocErrOff = kNoAllocQOff + 4 * kMaxBunches; // int error word (+ pad)
static_assert(sizeof(RunDev) <= 1024, "run descriptor slot");
static_assert(kNoAllocErrOff + 256 <= kNoAllocScratchBytes, "scratch layout");

static __device__ __align__(256) unsigned char g_wake_scratch[kNoAllocScratchBytes];

__global__ void __launch_bounds__(kPostThreads, 1) k_wake_noalloc(const Plan p) {
  extern __shared__ __align__(1024) uint8_t sm_wna[];
  __shared__ __align__(8) uint64_t bars[3];   // wake_prologue initialises three
  __shared__ uint32_t tmem_slot;
  __shared__ int s_flag;
  const PostJob job = p.jobs[blockIdx.x];
  const RunDev *R = p.runs + job.run;
  wake_prologue(R, job, sm_wna, bars, &tmem_slot, &s_flag);
  wake_job_tc(p, R, job, 0, sm_wna, bars, &tmem_slot, &s_flag, R->q_mp_f + job.bt * kBunchTile, true);
}

namespace {
std::mutex g_wna_mutex;
void *g_wna_addr[256] = {nullptr};   // device address of g_wake_scratch, per device
}  // namespace

// Resolve the scratch array's device address for the current device (first
// call on each device) and set the kernel's shared-memory limit.
static cudaError_t noalloc_setup(int dev, unsigned char **base) {
  std::lock_guard<std::mutex> lk(g_wna_mutex);
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  if (!g_wna_addr[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_wake_scratch);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_wake_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)post_smem_bytes(kMixed, 256));
    if (e != cudaSuccess) return e;
    g_wna_addr[dev] = ptr;
  }
  *base = static_cast<unsigned char *>(g_wna_addr[dev]);
  return cudaSuccess;
}

cudaError_t wake_noalloc_launch(const RunDev &proto, const void *img, size_t img_bytes, const float *q_f, int nb,
                                int nbins, const int32_t *hist, float *V, cudaStream_t s, int *device_error_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned char *base = nullptr;
  e = noalloc_setup(dev, &base);
  if (e != cudaSuccess) return e;
  // jobs: every (bunch tile, M-tile) pair of the one run
  PostJob jobs[64];
  const int ntile_b = (nb + kBunchTile - 1) / kBunchTile;
  int njobs = 0;
  for (int bt = 0; bt < ntile_b; ++bt)
    for (int mt = 0; mt < nbins / 128; ++mt) jobs[njobs++] = PostJob{0, kJobWake, bt, mt};
  RunDev rd = proto;
  rd.hist = const_cast<int32_t *>(hist);
  rd.vsr = V;
  rd.toep = base;
  rd.q_mp_f = reinterpret_cast<const float *>(base + kNoAllocQOff);
  rd.nb = nb;
  rd.nbins = nbins;
  Plan pl{};
  pl.runs = reinterpret_cast<RunDev *>(base + kNoAllocRunOff);
  pl.jobs = reinterpret_cast<PostJob *>(base + kNoAllocJobsOff);
  pl.error = reinterpret_cast<int *>(base + kNoAllocErrOff);
  pl.nruns = 1;
  pl.njobs = njobs;
  pl.max_nbins = nbins;
  // the whole working set is rewritten by every call; the error word starts at zero
  if ((e = cudaMemcpyAsync(base, img, img_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(base + kNoAllocRunOff, &rd, sizeof rd, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(base + kNoAllocJobsOff, jobs, sizeof(PostJob) * njobs, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(base + kNoAllocQOff, q_f, sizeof(float) * nb, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(base + kNoAllocErrOff, 0, 16, s)) != cudaSuccess) return e;
  k_wake_noalloc<<<njobs, kPostThreads, post_smem_bytes(kMixed, nbins), s>>>(pl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // synchronous: V is complete (and the error word readable) on return
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  return cudaMemcpy(device_error_out, base + kNoAllocErrOff, sizeof(int), cudaMemcpyDeviceToHost);
}

cudaError_t launch_post(const Plan &p, int precision, cudaStream_t s, bool pdl) {
  if (p.njobs == 0) return cudaSuccess;
  if (precision == kMixed && p.post_split > 0) {
    // the other jobs on the plan's side stream once the push is complete,
    // the wake jobs here (after the push, programmatically); joined back
    cudaError_t e = cudaEventRecord(p.ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.side, p.ev_fork, 0);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t c2{};
    c2.gridDim = dim3((unsigned)(p.njobs - p.post_split));
    c2.blockDim = dim3((unsigned)kPostThreads);
    c2.dynamicSmemBytes = post_small_smem_bytes(p.max_nbins, p.max_trans != 0);
    c2.stream = p.side;
    e = cudaLaunchKernelEx(&c2, k_post_split<2>, p, p.post_split);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t c1{};
    c1.gridDim = dim3((unsigned)p.post_split);
    c1.blockDim = dim3((unsigned)kPostThreads);
    c1.dynamicSmemBytes = post_smem_bytes(kMixed, p.max_nbins);
    c1.stream = s;
    cudaLaunchAttribute a1[1];
    a1[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a1[0].val.programmaticStreamSerializationAllowed = 1;
    c1.attrs = a1;
    c1.numAttrs = pdl ? 1 : 0;
    e = cudaLaunchKernelEx(&c1, k_post_split<1>, p, 0);
    if (e == cudaSuccess) e = cudaEventRecord(p.ev_join, p.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p.ev_join, 0);
    return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)p.njobs);
  cfg.blockDim = dim3((unsigned)kPostThreads);
  cfg.dynamicSmemBytes = post_smem_bytes(precision, p.max_nbins);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (precision == kMixed) return cudaLaunchKernelEx(&cfg, k_post_mixed, p);
  return cudaLaunchKernelEx(&cfg, k_post_f64, p);
}

}  // namespace mbt
