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
#include "device_common.cuh"

namespace mbt {

// ---------------------------------------------------------------------------
// Mixed precision: tau in FP32, delta stored and accumulated in FP64,
// everything else in FP32.  Each thread handles quads of 4 consecutive
// particles (float4 / 2x double2 accesses), two Philox calls per quad.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPushThreads, 4) k_push_mixed(const Plan p) {
  extern __shared__ __align__(16) float sm_push[];
  __shared__ float s_red[kPushThreads / 32][5];
  __shared__ float2 s_phi[kMaxLong];

  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  const int nbins = R->nbins;
  const int nlong = R->nlong;
  float *sV = sm_push;
  int *sH = reinterpret_cast<int *>(sm_push + nbins);
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);

  const float *vsr = static_cast<const float *>(R->vsr) + (size_t)t.m * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    sV[k] = vsr[k];
    sH[k] = 0;
  }
  if (threadIdx.x < nlong) {
    // Phi_m = P_m y_tile + Q_m of this bunch, then narrowed to FP32
    const int r = threadIdx.x;
    const double2 P = R->pq[((size_t)r * R->nb + t.m) * 2];
    const double2 Q = R->pq[((size_t)r * R->nb + t.m) * 2 + 1];
    const double2 y = R->y[(size_t)r * R->ntile_b + t.m / kBunchTile];
    const double2 phi = cfma(P, y, Q);
    s_phi[r] = make_float2((float)phi.x, (float)phi.y);
  }
  __syncthreads();

  const float invDf = (float)R->invDelta;
  const float HinvDf = (float)(R->H * R->invDelta);
  const float fnb = (float)nbins;
  const float invE0 = (float)R->inv_E0;
  const float twoVoE0 = (float)(2.0 * R->V_over_E0);
  const float cphi = (float)R->cos_phi_s, sphi = (float)R->sin_phi_s;
  const float halfw = (float)(0.5 * R->omega_rf);
  const float omD = (float)R->one_minus_D;
  const double omD_d = R->one_minus_D;
  const float qe = (float)R->qe_amp;
  const float aT0 = (float)R->aT0;
  const bool ngp = (R->flags & kKickNGP) != 0;
  float la[kMaxLong], lw[kMaxLong];
#pragma unroll
  for (int r = 0; r < kMaxLong; ++r) {
    la[r] = r < nlong ? (float)(-R->lr_s[r].x) : 0.f;
    lw[r] = r < nlong ? (float)R->lr_s[r].y : 0.f;
  }
  const uint32_t k0 = R->key0, k1 = R->key1, turn32 = (uint32_t)turn, bunch32 = (uint32_t)t.m;

  float *tau = static_cast<float *>(R->tau) + bd.off + t.start;
  double *del = R->delta + bd.off + t.start;
  float st = 0.f, st2 = 0.f, sd = 0.f, sd2 = 0.f;
  int nout = 0;

#pragma unroll 1
  for (int it = 0; it < kMixedQuadsPerThread; ++it) {
    const int q = (it * kPushThreads + (int)threadIdx.x) * 4;
    if (q >= t.count) break;
    const float4 tv = *reinterpret_cast<const float4 *>(tau + q);
    const double2 da = *reinterpret_cast<const double2 *>(del + q);
    const double2 db = *reinterpret_cast<const double2 *>(del + q + 2);
    float rr[4] = {0.f, 0.f, 0.f, 0.f};
    if (qe != 0.f) {
      const uint32_t pair0 = (uint32_t)((t.start + q) >> 1);
      normal_pair_f32(philox4x32_10(pair0, bunch32, turn32, 0u, k0, k1), rr[0], rr[1]);
      normal_pair_f32(philox4x32_10(pair0 + 1u, bunch32, turn32, 0u, k0, k1), rr[2], rr[3]);
    }
    float tt[4] = {tv.x, tv.y, tv.z, tv.w};
    double dd[4] = {da.x, da.y, db.x, db.y};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float t0 = tt[e];
      // wake kick (previous turn's wake)
      const float x = fmaf(t0, invDf, HinvDf);
      float v = 0.f;
      if (x >= 0.f && x < fnb) {
        if (ngp) {
          v = sV[(int)x];
        } else {
          const float u = x - 0.5f;
          if (u <= 0.f) v = sV[0];
          else if (u >= fnb - 1.f) v = sV[nbins - 1];
          else {
            const int j = (int)u;
            const float f = u - (float)j;
            v = fmaf(f, sV[j + 1] - sV[j], sV[j]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kMaxLong; ++r) {
        if (r < nlong) {
          float sn, cs;
          __sincosf(lw[r] * t0, &sn, &cs);
          const float ea = __expf(-la[r] * t0);
          v = fmaf(ea, s_phi[r].x * cs - s_phi[r].y * sn, v);
        }
      }
      // RF gain minus U0: (V/E0)[sin(phi_s - w t) - sin(phi_s)] = -2 (V/E0) sin(w t / 2) cos(phi_s - w t / 2)
      float sh, ch;
      sincosf(halfw * t0, &sh, &ch);
      const float rf = -twoVoE0 * sh * fmaf(ch, cphi, sh * sphi);
      // damping + excitation applied to (delta + kick + rf); delta itself in FP64
      const float inc = fmaf(fmaf(-v, invE0, rf), omD, qe * rr[e]);
      const double d1 = fma(dd[e], omD_d, f32_to_f64_bits(inc));
      const float d1f = f64_to_f32_trunc(d1);
      const float t1 = fmaf(aT0, d1f, t0);
      const bool valid = q + e < t.count;
      tt[e] = valid ? t1 : t0;
      dd[e] = valid ? d1 : dd[e];
      if (valid) {
        const float xb = fmaf(t1, invDf, HinvDf);
        if (xb >= 0.f && xb < fnb) atomicAdd(&sH[(int)xb], 1);
        else ++nout;
        st += t1;
        st2 = fmaf(t1, t1, st2);
        sd += d1f;
        sd2 = fmaf(d1f, d1f, sd2);
      }
    }
    *reinterpret_cast<float4 *>(tau + q) = make_float4(tt[0], tt[1], tt[2], tt[3]);
    *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
    *reinterpret_cast<double2 *>(del + q + 2) = make_double2(dd[2], dd[3]);
  }

  // moment partials: FP32 within a warp, FP64 across warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  if (threadIdx.x < 5) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kPushThreads / 32; ++w) acc += (double)s_red[w][threadIdx.x];
    p.partial[(size_t)blockIdx.x * kPartials + threadIdx.x] = acc;
  }
  int32_t *hg = R->hist + ((size_t)par * R->nb + t.m) * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    const int c = sH[k];
    if (c) atomicAdd(hg + k, c);
  }
}

// ---------------------------------------------------------------------------
// FP64: the oracle's arithmetic step for step.  Each thread handles pairs of
// consecutive particles (one Philox call per pair).  The cell index is formed
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
  __shared__ double s_red[kPushThreads / 32][5];
  __shared__ double2 s_phi[kMaxLong];

  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  const int nbins = R->nbins;
  const int nlong = R->nlong;
  double *sV = sm_push64;
  int *sH = reinterpret_cast<int *>(sm_push64 + nbins);
  const long long turn = *R->turn;
  const int par = (int)(turn & 1);

  const double *vsr = static_cast<const double *>(R->vsr) + (size_t)t.m * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    sV[k] = vsr[k];
    sH[k] = 0;
  }
  if (threadIdx.x < nlong) {
    const int r = threadIdx.x;
    const double2 P = R->pq[((size_t)r * R->nb + t.m) * 2];
    const double2 Q = R->pq[((size_t)r * R->nb + t.m) * 2 + 1];
    const double2 y = R->y[(size_t)r * R->ntile_b + t.m / kBunchTile];
    s_phi[r] = cfma(P, y, Q);
  }
  __syncthreads();

  const double H = R->H, invD = R->invDelta, invE0 = R->inv_E0, VoE0 = R->V_over_E0;
  const double phis = R->phi_s, wrf = R->omega_rf, U0oE0 = R->U0_over_E0;
  const double omD = R->one_minus_D, qe = R->qe_amp, aT0 = R->aT0;
  const bool ngp = (R->flags & kKickNGP) != 0;
  const uint32_t k0 = R->key0, k1 = R->key1, turn32 = (uint32_t)turn, bunch32 = (uint32_t)t.m;

  double *tau = static_cast<double *>(R->tau) + bd.off + t.start;
  double *del = R->delta + bd.off + t.start;
  double st = 0.0, st2 = 0.0, sd = 0.0, sd2 = 0.0;
  int nout = 0;

#pragma unroll 1
  for (int it = 0; it < kF64PairsPerThread; ++it) {
    const int q = (it * kPushThreads + (int)threadIdx.x) * 2;
    if (q >= t.count) break;
    const double2 tv = *reinterpret_cast<const double2 *>(tau + q);
    const double2 dv = *reinterpret_cast<const double2 *>(del + q);
    double rr[2] = {0.0, 0.0};
    if (qe != 0.0)
      normal_pair_f64(philox4x32_10((uint32_t)((t.start + q) >> 1), bunch32, turn32, 0u, k0, k1), rr[0], rr[1]);
    double tt[2] = {tv.x, tv.y};
    double dd[2] = {dv.x, dv.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (q + e >= t.count) continue;
      double tp = tt[e], d = dd[e];
      double v = vsr_at_f64(sV, __dmul_rn(__dadd_rn(tp, H), invD), nbins, ngp);
      for (int r = 0; r < nlong; ++r) {
        const double2 s = R->lr_s[r];
        double sn, cs;
        sincos(s.y * tp, &sn, &cs);
        const double ea = exp(s.x * tp);
        v += ea * (s_phi[r].x * cs - s_phi[r].y * sn);
      }
      d = d - v * invE0;
      d = d + VoE0 * sin(phis - wrf * tp) - U0oE0;
      d = d * omD + qe * rr[e];
      tp = tp + aT0 * d;
      tt[e] = tp;
      dd[e] = d;
      const double xb = __dmul_rn(__dadd_rn(tp, H), invD);
      if (xb >= 0.0 && xb < (double)nbins) atomicAdd(&sH[(int)xb], 1);
      else ++nout;
      st += tp;
      st2 += tp * tp;
      sd += d;
      sd2 += d * d;
    }
    *reinterpret_cast<double2 *>(tau + q) = make_double2(tt[0], tt[1]);
    *reinterpret_cast<double2 *>(del + q) = make_double2(dd[0], dd[1]);
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  st = warp_sum_d(st);
  st2 = warp_sum_d(st2);
  sd = warp_sum_d(sd);
  sd2 = warp_sum_d(sd2);
  const int no = __reduce_add_sync(0xFFFFFFFFu, nout);
  if (lane == 0) {
    s_red[warp][0] = st;
    s_red[warp][1] = st2;
    s_red[warp][2] = sd;
    s_red[warp][3] = sd2;
    s_red[warp][4] = (double)no;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double acc = 0.0;
    for (int w = 0; w < kPushThreads / 32; ++w) acc += s_red[w][threadIdx.x];
    p.partial[(size_t)blockIdx.x * kPartials + threadIdx.x] = acc;
  }
  int32_t *hg = R->hist + ((size_t)par * R->nb + t.m) * nbins;
  for (int k = threadIdx.x; k < nbins; k += kPushThreads) {
    const int c = sH[k];
    if (c) atomicAdd(hg + k, c);
  }
}

// ---------------------------------------------------------------------------
// Matched Gaussian start from Philox tags 1 (tau) and 2 (delta) at turn 0, in
// FP64 for both precisions (tau narrowed to FP32 by rounding for kMixed).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPushThreads) k_init(const Plan p, int precision, int tile_size) {
  const TileDev t = p.tiles[blockIdx.x];
  const RunDev *__restrict__ R = p.runs + t.run;
  const BunchDev bd = p.bunches[t.bunch];
  for (int q = 2 * (int)threadIdx.x; q < t.count; q += 2 * kPushThreads) {
    const uint32_t pair = (uint32_t)((t.start + q) >> 1);
    double a0, a1, b0, b1;
    normal_pair_f64(philox4x32_10(pair, (uint32_t)t.m, 0u, 1u, R->key0, R->key1), a0, a1);
    normal_pair_f64(philox4x32_10(pair, (uint32_t)t.m, 0u, 2u, R->key0, R->key1), b0, b1);
    const long long i = bd.off + t.start + q;
    const bool two = q + 1 < t.count;
    if (precision == kMixed) {
      float *tau = static_cast<float *>(R->tau);
      tau[i] = (float)(R->sigma_tau0 * a0);
      if (two) tau[i + 1] = (float)(R->sigma_tau0 * a1);
    } else {
      double *tau = static_cast<double *>(R->tau);
      tau[i] = R->sigma_tau0 * a0;
      if (two) tau[i + 1] = R->sigma_tau0 * a1;
    }
    R->delta[i] = R->sigma_E * b0;
    if (two) R->delta[i + 1] = R->sigma_E * b1;
  }
  (void)tile_size;
}

cudaError_t launch_push(const Plan &p, int precision, cudaStream_t s) {
  if (p.ntiles == 0) return cudaSuccess;
  const int max_nbins = p.max_nbins;
  if (precision == kMixed) {
    const size_t smem = (size_t)max_nbins * (sizeof(float) + sizeof(int));
    k_push_mixed<<<p.ntiles, kPushThreads, smem, s>>>(p);
  } else {
    const size_t smem = (size_t)max_nbins * (sizeof(double) + sizeof(int));
    k_push_f64<<<p.ntiles, kPushThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_init(const Plan &p, int precision, cudaStream_t s) {
  if (p.ntiles == 0) return cudaSuccess;
  k_init<<<p.ntiles, kPushThreads, 0, s>>>(p, precision, 0);
  return cudaGetLastError();
}

}  // namespace mbt
