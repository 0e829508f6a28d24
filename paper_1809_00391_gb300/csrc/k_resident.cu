// Cluster-resident tracking: one thread-block cluster per bunch, the bunch's
// macro-particles held in the cluster's shared memory for every turn of a
// launch (no particle traffic to HBM between the first load and the final
// store).  Per turn (arXiv:1809.00391 Sec. 2.2-2.4, same map as the streaming
// kernels, mixed precision):
//   push every particle of the CTA's slice (kick, RF, damping + excitation,
//   drift) into a CTA histogram and moment partials;
//   cluster barrier; every CTA sums the CTAs' histograms through distributed
//   shared memory; CTA 0 forms the bunch moments; CTA r computes rows
//   [r B, (r+1) B) of the short-range voltage (FP32 causal convolution on the
//   CUDA cores: one bunch is a matrix-vector product, nothing for the tensor
//   cores to batch);
//   long range (if any): CTA 0 publishes the bunch's emission, the clusters
//   meet at a bounded grid barrier, and every cluster runs the same FP64
//   affine scan over the fill, carrying the phasor across turns;
//   cluster barrier; every CTA gathers the voltage rows for the next kick.
// The fill must fit on chip and its clusters must be co-resident (checked on
// the host); the grid barrier gives up after 2 s and sets the error word.
#include <cooperative_groups.h>
#include "push_core.cuh"

namespace cg = cooperative_groups;

namespace mbt {


struct ResidentSmem {
  double *sD;      // [per]
  float *sT;       // [per]
  int *lh;         // [2][nbins + kSpillCells] CTA histograms, double-buffered by turn
  int *bh;         // [nbins] bunch histogram
  float2 *sVd;     // [nbins] (V[j], V[j+1] - V[j])
  float *lag;      // [nbins]
  float *vrow;     // [nbins] this CTA's rows of V (only its slice is used)
  float *vtmp;     // [nbins] gathered V
};

__host__ __device__ inline size_t resident_layout(int per, int nbins, ResidentSmem *m, uint8_t *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return o;
  };
  const size_t oD = take((size_t)per * 8), oT = take((size_t)per * 4), oLH = take((size_t)2 * (nbins + kSpillCells) * 4);
  const size_t oBH = take((size_t)nbins * 4), oV = take((size_t)nbins * 8), oL = take((size_t)nbins * 4);
  const size_t oR = take((size_t)nbins * 4), oX = take((size_t)nbins * 4);
  if (m) {
    m->sD = reinterpret_cast<double *>(base + oD);
    m->sT = reinterpret_cast<float *>(base + oT);
    m->lh = reinterpret_cast<int *>(base + oLH);
    m->bh = reinterpret_cast<int *>(base + oBH);
    m->sVd = reinterpret_cast<float2 *>(base + oV);
    m->lag = reinterpret_cast<float *>(base + oL);
    m->vrow = reinterpret_cast<float *>(base + oR);
    m->vtmp = reinterpret_cast<float *>(base + oX);
  }
  return off;
}

size_t resident_smem_bytes(int per, int nbins) { return resident_layout(per, nbins, nullptr, nullptr); }

static_assert(kResidentThreads % 32 == 0 && kResidentThreads >= 64 && kResidentThreads <= 1024, "whole warps, 2-32 of them");

template <int NLONG_MAX, bool HARM>
__global__ void __launch_bounds__(kResidentThreads, 1) k_resident(const ResidentArgs a) {
  extern __shared__ __align__(16) uint8_t sm_res[];
  __shared__ float s_red[kResidentThreads / 32][5];
  __shared__ double s_mom[8];   // the CTA's sums of u, u^2, v, v^2, n_out; its tau_ref, delta_ref, particles
  __shared__ float2 s_phi[kMaxLong];
  __shared__ float4 s_hc[kMaxHarm];
  __shared__ double2 s_phid[kMaxLong];
  __shared__ double2 s_carry[kMaxLong];
  __shared__ int s_fail;

  cg::cluster_group cl = cg::this_cluster();
  const int C = a.cluster;
  const int rank = (int)cl.block_rank();
  const int m = (int)blockIdx.x / C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Plan &p = a.plan;
  const RunDev *__restrict__ R = p.runs;
  const BunchDev bd = p.bunches[m];
  const int nbins = R->nbins, nb = R->nb, nlong = R->nlong;
  ResidentSmem S;
  resident_layout(a.per, nbins, &S, sm_res);
  const long long s0 = (long long)rank * a.per;
  const int ns = (int)max(0LL, min((long long)a.per, bd.n - s0));
  float *gtau = static_cast<float *>(R->tau) + bd.off + s0;
  double *gdel = R->delta + bd.off + s0;

  // load the slice, the tables and the wake state left by the previous turn
  for (int i = tid; i < ns; i += kResidentThreads) {
    S.sT[i] = gtau[i];
    S.sD[i] = gdel[i];
  }
  const float *vsr = static_cast<const float *>(R->vsr) + (size_t)m * nbins;
  for (int k = tid; k < nbins; k += kResidentThreads) {
    const float v0 = vsr[k];
    const float v1 = k + 1 < nbins ? vsr[k + 1] : v0;
    S.sVd[k] = make_float2(v0, v1 - v0);
    S.lag[k] = R->lag_f[k];
    S.lh[k] = 0;
    S.lh[nbins + kSpillCells + k] = 0;
  }
  if (tid < nlong) {
    const double2 P = R->pq[((size_t)tid * nb + m) * 2];
    const double2 Q = R->pq[((size_t)tid * nb + m) * 2 + 1];
    const double2 y = R->y[(size_t)tid * R->ntile_b + m / kBunchTile];
    const double2 phi = cfma(P, y, Q);
    s_phid[tid] = phi;
    s_phi[tid] = make_float2((float)phi.x, (float)phi.y);
    s_carry[tid] = R->carry[tid];
  }
  if (tid == 0) s_fail = 0;
  const int nharm = R->nharm;
  if (tid < nharm) s_hc[tid] = R->f_harm[tid];
  const long long turn0 = *R->turn;

  PushConstF c;
  c.nbins = nbins;
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
#pragma unroll
  for (int r = 0; r < NLONG_MAX; ++r) {
    la[r] = R->f_la[r];
    lw[r] = R->f_lw[r];
  }
  const uint32_t k0 = R->key0, k1 = R->key1, bunch32 = (uint32_t)m;
  const float qf = R->q_mp_f[m];
  const int B = nbins / C;   // voltage rows per CTA
  cl.sync();

  for (int it = 0; it < a.nturns; ++it) {
    const long long turn = turn0 + it;
    const int lp = it & 1;
    int *lh = S.lh + lp * (nbins + kSpillCells);
    float2 phi[NLONG_MAX > 0 ? NLONG_MAX : 1];
#pragma unroll
    for (int r = 0; r < NLONG_MAX; ++r) phi[r] = r < nlong ? s_phi[r] : make_float2(0.f, 0.f);
    for (int k = tid; k < nbins; k += kResidentThreads) lh[k] = 0;
    // moment reference: the slice's first particle before the push (read by
    // every thread before the barrier, after which thread 0 overwrites it)
    const float tref = ns > 0 ? S.sT[0] : 0.f, dref = ns > 0 ? f64_to_f32_ref(S.sD[0]) : 0.f;
    __syncthreads();

    // push the slice (quads of consecutive particles, one Philox block each);
    // moment partials relative to the reference
    float st = 0.f, st2 = 0.f, sd = 0.f, sd2 = 0.f;
    int nout = 0;
    for (int q = 4 * tid; q < ns; q += 4 * kResidentThreads) {
      float rr[4] = {0.f, 0.f, 0.f, 0.f};
      if (c.qe != 0.f)
        normal_quad_f32(philox4x32_10((uint32_t)((s0 + q) >> 2), bunch32, (uint32_t)turn, 0u, k0, k1), rr);
      const float4 tv = *reinterpret_cast<const float4 *>(S.sT + q);
      const double2 da = *reinterpret_cast<const double2 *>(S.sD + q);
      const double2 db = *reinterpret_cast<const double2 *>(S.sD + q + 2);
      float tt[4] = {tv.x, tv.y, tv.z, tv.w};
      double dd[4] = {da.x, da.y, db.x, db.y};
      const int nvalid = min(4, ns - q);
      if (ngp)
        quad_push<NLONG_MAX, true, HARM>(c, S.sVd, lh, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid, tref, dref, st,
                                   st2, sd, sd2, nout);
      else
        quad_push<NLONG_MAX, false, HARM>(c, S.sVd, lh, nlong, la, lw, phi, omD_d, s_hc, nharm, tt, dd, rr, nvalid, tref, dref, st,
                                    st2, sd, sd2, nout);
      *reinterpret_cast<float4 *>(S.sT + q) = make_float4(tt[0], tt[1], tt[2], tt[3]);
      *reinterpret_cast<double2 *>(S.sD + q) = make_double2(dd[0], dd[1]);
      *reinterpret_cast<double2 *>(S.sD + q + 2) = make_double2(dd[2], dd[3]);
    }
    st = warp_sum_f(st);
    st2 = warp_sum_f(st2);
    sd = warp_sum_f(sd);
    sd2 = warp_sum_f(sd2);
    const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
    if (lane == 0) {
      s_red[warp][0] = st;
      s_red[warp][1] = st2;
      s_red[warp][2] = sd;
      s_red[warp][3] = sd2;
      s_red[warp][4] = (float)no;
    }
    __syncthreads();
    if (tid < 5) {
      // the warps' FP32 sums by a pairwise tree of fixed shape (a serial FP64
      // chain over the warps would wait 64 cycles per add), FP64 from the CTA on
      // (over the warp count rounded up to a power of two, the missing warps zero)
      constexpr int kW = kResidentThreads / 32;
      constexpr int kH = (kW <= 2 ? 2 : kW <= 4 ? 4 : kW <= 8 ? 8 : kW <= 16 ? 16 : 32) / 2;
      float a[kH];
#pragma unroll
      for (int i = 0; i < kH; ++i) a[i] = (i < kW ? s_red[i][tid] : 0.f) + (kH + i < kW ? s_red[kH + i][tid] : 0.f);
#pragma unroll
      for (int h = kH / 2; h > 0; h >>= 1)
#pragma unroll
        for (int i = 0; i < h; ++i) a[i] += a[i + h];
      s_mom[tid] = (double)a[0];
    } else if (tid == 5) {
      s_mom[5] = (double)tref;
      s_mom[6] = (double)dref;
      s_mom[7] = (double)ns;
    }
    cl.sync();   // #1: every CTA histogram and moment partial of the turn is complete

    // bunch histogram (every CTA: all remote loads of a cell issued before
    // the sum), moments (CTA 0)
    for (int k = tid; k < nbins; k += kResidentThreads) {
      int v[16];
#pragma unroll
      for (int cr = 0; cr < 16; ++cr) v[cr] = cr < C ? cl.map_shared_rank(lh, cr)[k] : 0;
      int sum = 0;
#pragma unroll
      for (int cr = 0; cr < 16; ++cr) sum += v[cr];
      S.bh[k] = sum;
    }
    __syncthreads();
    if (rank == 0 && warp == 0) {
      // the CTAs' sums about their own references combined exactly (the
      // pairwise form of the variance): the mean first, then every CTA's
      // second moment about it; lane cr holds CTA cr's sums
      const double inv_n = R->inv_n[m];
      double q[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (lane < C) {
        const double *r = cl.map_shared_rank(s_mom, lane);
#pragma unroll
        for (int i = 0; i < 8; ++i) q[i] = r[i];
      }
      const double at = warp_sum_d(fma(q[7], q[5], q[0])), ad = warp_sum_d(fma(q[7], q[6], q[2]));
      const double s4 = warp_sum_d(q[4]);
      const double mt = at * inv_n, md = ad * inv_n;
      const double et = q[5] - mt, ed = q[6] - md;
      const double qt = warp_sum_d(lane < C ? fma(q[7] * et, et, fma(2.0 * et, q[0], q[1])) : 0.0);
      const double qd = warp_sum_d(lane < C ? fma(q[7] * ed, ed, fma(2.0 * ed, q[2], q[3])) : 0.0);
      if (lane == 0) {
        const double vt = fmax(qt * inv_n, 0.0), vd = fmax(qd * inv_n, 0.0);
        double *rec = R->rec + ((size_t)(turn % R->cap) * nb + m) * kRecord;
        rec[0] = mt;
        rec[1] = sqrt(vt);
        rec[2] = md;
        rec[3] = sqrt(vd);
        rec[4] = (double)bd.n - s4;
        rec[5] = s4;
      }
    }
    // rows [rank B, rank B + B) of V = q sum_{k<=j} lag[j-k] count[k]
    {
      // threads per row: the largest power of two <= min(32, threads / B); B is
      // a power of two (nbins 128 or 256, C a power of two), so B G is a
      // multiple of 32 and every warp's lanes all take the shuffles or none
      const int G = 1 << (31 - __clz(min(32, kResidentThreads / B)));
      const int row = tid / G, sub = tid % G;
      const int j = rank * B + row;
      if (row < B) {
        float acc = 0.f;
        for (int k = sub; k <= j; k += G) acc = fmaf(S.lag[j - k], (float)S.bh[k], acc);
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o, G);
        if (sub == 0) S.vrow[j] = qf * acc;
      }
    }
    // long range: emission, grid barrier, scan over the fill
    if (nlong > 0 && rank == 0) {
      for (int r = 0; r < nlong; ++r) {
        if (warp == r) {
          const float2 *tab = R->emis_f + (size_t)r * nbins;
          float ax = 0.f, ay = 0.f;
          for (int k = lane; k < nbins; k += 32) {
            const float cnt = (float)S.bh[k];
            ax = fmaf(cnt, tab[k].x, ax);
            ay = fmaf(cnt, tab[k].y, ay);
          }
          ax = warp_sum_f(ax);
          ay = warp_sum_f(ay);
          if (lane == 0) {
            const double qd = R->q_mp[m];
            a.E[((size_t)lp * nlong + r) * nb + m] = cmul(R->lr_c[r], make_double2(qd * (double)ax, qd * (double)ay));
          }
        }
      }
      __syncthreads();
      if (tid == 0 && a.grid_sync) {
        __threadfence();
        atomicAdd(a.gbar, 1u);
        const unsigned int target = (unsigned int)(it + 1) * (unsigned int)nb + a.extra_arrivals;
        const unsigned long long t0 = global_timer_ns();
        while (atomicAdd(a.gbar, 0u) < target) {
          if (global_timer_ns() - t0 > a.wait_ns) {
            atomicExch(p.error, kErrTimeout);
            s_fail = 1;
            break;
          }
        }
        __threadfence();
      }
      __syncthreads();
      if (warp == 0) {
        for (int r = 0; r < nlong; ++r) {
          double2 E = make_double2(0.0, 0.0);
          if (lane < nb) E = __ldcg(a.E + ((size_t)lp * nlong + r) * nb + lane);
          const double2 Eprev = shfl_up_d2(E, 1);
          double2 A = make_double2(1.0, 0.0), Bv = make_double2(0.0, 0.0);
          if (lane < nb) {
            A = R->step[(size_t)r * nb + lane];
            if (lane > 0) Bv = cmul(A, Eprev);
          }
          warp_scan_affine(A, Bv);
          const double2 K = s_carry[r];
          const double2 phim = cfma(A, K, Bv);   // phasor at bunch `lane`, for the next turn's kick
          const double2 last = make_double2(__shfl_sync(0xFFFFFFFFu, phim.x + E.x, nb - 1),
                                            __shfl_sync(0xFFFFFFFFu, phim.y + E.y, nb - 1));
          const double2 mine = make_double2(__shfl_sync(0xFFFFFFFFu, phim.x, m), __shfl_sync(0xFFFFFFFFu, phim.y, m));
          if (lane == 0) {
            s_carry[r] = last;
            s_phid[r] = mine;
            for (int cr = 0; cr < C; ++cr) cl.map_shared_rank(s_phi, cr)[r] = make_float2((float)mine.x, (float)mine.y);
          }
        }
      }
      // a grid-barrier timeout ends the turn loop of every CTA of the cluster together
      if (tid == 0 && s_fail)
        for (int cr = 1; cr < C; ++cr) *cl.map_shared_rank(&s_fail, cr) = 1;
    }
    cl.sync();   // #2: voltage rows and phasors of the turn are complete

    for (int k = tid; k < nbins; k += kResidentThreads) S.vtmp[k] = cl.map_shared_rank(S.vrow, k / B)[k];
    __syncthreads();
    for (int k = tid; k < nbins; k += kResidentThreads) {
      const float v0 = S.vtmp[k];
      const float v1 = k + 1 < nbins ? S.vtmp[k + 1] : v0;
      S.sVd[k] = make_float2(v0, v1 - v0);
    }
    __syncthreads();
    if (s_fail) break;
  }

  // write the state back: particles, and what a following streaming turn reads
  for (int i = tid; i < ns; i += kResidentThreads) {
    gtau[i] = S.sT[i];
    gdel[i] = S.sD[i];
  }
  if (rank == 0) {
    const long long last = turn0 + a.nturns - 1;
    int32_t *hl = R->hist + ((size_t)(last & 1) * nb + m) * nbins;
    int32_t *hn = R->hist + ((size_t)((last + 1) & 1) * nb + m) * nbins;
    float *vout = static_cast<float *>(R->vsr) + (size_t)m * nbins;
    for (int k = tid; k < nbins; k += kResidentThreads) {
      hl[k] = S.bh[k];
      hn[k] = 0;
      vout[k] = S.sVd[k].x;
    }
    if (tid < nlong) {
      R->pq[((size_t)tid * nb + m) * 2] = make_double2(0.0, 0.0);
      R->pq[((size_t)tid * nb + m) * 2 + 1] = s_phid[tid];
      if (m == 0) R->carry[tid] = s_carry[tid];
    }
    if (m == 0 && tid == 0) *R->turn = turn0 + a.nturns;
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

cudaError_t launch_resident(const ResidentArgs &a, int nlong, int nharm, int nb, cudaStream_t s) {
  const int nbins = a.plan.max_nbins;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(nb * a.cluster));
  cfg.blockDim = dim3((unsigned)kResidentThreads);
  cfg.dynamicSmemBytes = resident_smem_bytes(a.per, nbins);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int bytes = (int)cfg.dynamicSmemBytes;
  auto run = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, kern, a);
  };
  const bool harm = nharm > 0;
  switch (nlong) {
    case 0: return harm ? run(k_resident<0, true>) : run(k_resident<0, false>);
    case 1: return harm ? run(k_resident<1, true>) : run(k_resident<1, false>);
    case 2: return harm ? run(k_resident<2, true>) : run(k_resident<2, false>);
    default: return harm ? run(k_resident<kMaxLong, true>) : run(k_resident<kMaxLong, false>);
  }
}

cudaError_t resident_max_clusters(int cluster, size_t smem, int *max_clusters) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)cluster * 64u);
  cfg.blockDim = dim3((unsigned)kResidentThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaFuncSetAttribute(k_resident<kMaxLong, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resident<kMaxLong, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveClusters(max_clusters, (void *)k_resident<kMaxLong, true>, &cfg);
}

}  // namespace mbt
