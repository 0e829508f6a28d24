// Per-particle map of the mixed-precision path (shared by the streaming push
// kernel and the cluster-resident kernel): wake kick, RF, damping +
// excitation, drift (arXiv:1809.00391 Sec. 2.2-2.3, readings in mbt.h), and
// the quad step that adds deposit and moment partials.
#pragma once
#include "device_common.cuh"

namespace mbt {

struct PushConstF {
  // invD = 1/Delta, HinvD = H/Delta - 1/2: x = tau invD + HinvD is the
  // position in cells relative to the cell centres (cell k holds
  // -1/2 <= x - k < 1/2); la: decay rates times log2(e); RF gain minus the
  // synchronous one, damped: rfA (cos w tau - 1) - rfB sin w tau with
  // rfA = (V/E0)(1 - D) sin phi_s, rfB = (V/E0)(1 - D) cos phi_s, w = omega_rf
  float invD, HinvD, fnb, invE0, rfA, rfB, w, omD, qe, aT0;
  int nbins;
};

// One particle: kick with the previous turn's wake, RF (main and harmonic
// cavities), damping + excitation, drift.  Returns the new tau; delta is
// updated in place.  hc: nharm harmonic cavities (2 V_h/E0 (1 - D), cos phi_h,
// sin phi_h, n omega_rf / 2), in shared memory.  HARM: compiled in only for
// plans with harmonic cavities, so that the particle code of the others stays
// one straight block in which the four particles of a quad overlap.
template <int NLONG_MAX, bool NGP, bool HARM>
__device__ __forceinline__ float push_one(const PushConstF &c, const float2 *sVd, int nlong,
                                          const float *la, const float *lw, const float2 *phi, double omD_d,
                                          const float4 *hc, int nharm, float t0, double &d, float r, float &df) {
  const float x = fmaf(t0, c.invD, c.HinvD);   // cells, from the cell centres
  float v;
  if (NGP) {
    const int k = min(max(__float2int_rn(x), 0), c.nbins - 1);
    v = sVd[k].x;
  } else {
    // linear interpolation between cell centres, clamped to the end cells
    const float u = fminf(fmaxf(x, 0.f), c.fnb - 1.f);
    const int j = (int)u;   // <= nbins - 1, where the slope is 0
    const float2 vd = sVd[j];
    v = fmaf(u - (float)j, vd.y, vd.x);
  }
  v = (x >= -0.5f && x < c.fnb - 0.5f) ? v : 0.f;
#pragma unroll
  for (int r2 = 0; r2 < NLONG_MAX; ++r2) {
    if (r2 < nlong) {
      float sn, cs;
      __sincosf(lw[r2] * t0, &sn, &cs);
      const float ea = ex2_approx(-la[r2] * t0);
      v = fmaf(ea, fmaf(phi[r2].x, cs, -phi[r2].y * sn), v);
    }
  }
  // (V/E0)[sin(phi_s - w t) - sin(phi_s)] (1 - D) = rfA (cos w t - 1) - rfB sin w t
  // (c.rfA, c.rfB and c.invE0 carry the damping factor already)
  float sw, cw;
  __sincosf(c.w * t0, &sw, &cw);
  float rf = fmaf(-c.rfB, sw, fmaf(c.rfA, cw, -c.rfA));
  // harmonic cavities, the same form: (V_h/E0)[sin(phi_h - n w t) - sin(phi_h)]
  for (int k = 0; HARM && k < nharm; ++k) {
    const float4 h = hc[k];
    float sk, ck;
    __sincosf(h.w * t0, &sk, &ck);
    rf = fmaf(-h.x * sk, fmaf(ck, h.y, sk * h.z), rf);
  }
  const float inc = fmaf(-v, c.invE0, fmaf(c.qe, r, rf));
  d = fma(d, omD_d, f32_to_f64_bits(inc));
  df = f64_to_f32_trunc(d);
  return fmaf(c.aT0, df, t0);
}

// Four consecutive particles: push, deposit, moment partials.  Full quads
// (nvalid == 4, all but a bunch's last) take no per-particle validity tests.
// The partials are sums of u = tau - tref and v = delta - dref (tref, dref:
// the tile's first particle before the push, which lies within a few bunch
// lengths of every particle of the bunch), so that the variance formed from
// them does not cancel when the centroid sits far from the bucket centre.
template <int NLONG_MAX, bool NGP, bool HARM>
__device__ __forceinline__ void quad_push(const PushConstF &c, const float2 *sVd, int *sH, int nlong, const float *la,
                                          const float *lw, const float2 *phi, double omD_d, const float4 *hc,
                                          int nharm, float (&tt)[4], double (&dd)[4], const float (&rr)[4],
                                          int nvalid, float tref, float dref, float &st, float &st2, float &sd,
                                          float &sd2, int &nout) {
  const bool full = nvalid == 4;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (full || e < nvalid) {
      float df;
      const float t1 = push_one<NLONG_MAX, NGP, HARM>(c, sVd, nlong, la, lw, phi, omD_d, hc, nharm, tt[e], dd[e], rr[e], df);
      tt[e] = t1;
      const float xb = fmaf(t1, c.invD, c.HinvD);
      // without a branch: a particle outside the mesh counts into its lane's
      // spill cell behind the histogram (sH holds nbins + kSpillCells cells)
      const bool in = xb >= -0.5f && xb < c.fnb - 0.5f;
      atomicAdd(&sH[in ? __float2int_rn(xb) : c.nbins + (int)(threadIdx.x & 31)], 1);
      nout += in ? 0 : 1;
      const float u = t1 - tref, v = df - dref;
      st += u;
      st2 = fmaf(u, u, st2);
      sd += v;
      sd2 = fmaf(v, v, sd2);
    }
  }
}

// ---------------------------------------------------------------------------
// Runs with a transverse plane (Eqs. 3-5 x lines, Eq. 6 second line, FP32).
// ---------------------------------------------------------------------------
struct TransConstF {
  float mu0, mu0xi;            // 2 pi frac(nu), 2 pi nu xi: phase = mu0 + mu0xi delta
  float beta, alpha, gamma;
  float nx, nxp;               // excitation amplitudes sqrt(beta emit Dx), sqrt(gamma emit Dx)
  float invE0, inv_omD, U0oE0; // 1/E0 (no damping factor), 1/(1 - D), U0/E0
  float dinv, drange;          // 1/u of the dipole deposit, and the |x| it accepts (2^30 u)
};

// Dipole deposit in fixed point.  x is quantised to xq = round(x / u), u a
// power of two (2^-20 times the run's transverse scale), and xq is added as
// its low 16 bits (unsigned) and its high part xq >> 16 (signed) into two
// 32-bit counters of the cell: with at most 65536 particles per cell and
// tile neither sum can overflow, so the cell's sum (2^16 hi + lo) u is the
// exact sum of the quantised x, in any order of the atomics.  (FP32 shared
// atomics of x retry under contention and would round every partial sum.)
// Returns false if |x| is outside the accepted range (or not a number).
__device__ __forceinline__ bool deposit_dip(unsigned *sLo, int *sHi, int cell, float x, const TransConstF &tc) {
  const int xq = __float2int_rn(x * tc.dinv);   // |x| < drange: |xq| <= 2^30
  atomicAdd(sLo + cell, (unsigned)xq & 0xFFFFu);
  atomicAdd(sHi + cell, xq >> 16);
  return fabsf(x) < tc.drange;
}

// One particle with a transverse plane: the longitudinal map of push_one
// (its long-range sum over the plane-0 entries only) and, with the same
// previous-turn wake, x' += V_x / E0, the momentum ratio across the cavity,
// the rotation with the new delta's phase, the excitation.  vtd: (V_x[j],
// V_x[j+1] - V_x[j]) of the bunch; plane: long-range entry planes.
template <int NLONG_MAX>
__device__ __forceinline__ float push_one_t(const PushConstF &c, const TransConstF &tc, const float2 *sVd,
                                            const float2 *sVt, int nlong, const int *plane, const float *la,
                                            const float *lw, const float2 *phi, double omD_d, const float4 *hc,
                                            int nharm, bool ngp, float vrw, float t0, double &d, float r, float &df,
                                            float &x, float &xp, float rx, float rxp) {
  const float x0 = fmaf(t0, c.invD, c.HinvD);   // cells, from the cell centres
  const bool inside = x0 >= -0.5f && x0 < c.fnb - 0.5f;
  float v, vt;
  if (ngp) {
    const int k = min(max(__float2int_rn(x0), 0), c.nbins - 1);
    v = sVd[k].x;
    vt = sVt[k].x;
  } else {
    const float u = fminf(fmaxf(x0, 0.f), c.fnb - 1.f);
    const int j = (int)u;   // <= nbins - 1, where the slopes are 0
    const float2 vd = sVd[j], vtd = sVt[j];
    v = fmaf(u - (float)j, vd.y, vd.x);
    vt = fmaf(u - (float)j, vtd.y, vtd.x);
  }
  v = inside ? v : 0.f;
  vt = (inside ? vt : 0.f) + vrw;   // the long-range resistive wall acts on every particle of the bunch
#pragma unroll
  for (int r2 = 0; r2 < NLONG_MAX; ++r2) {
    if (r2 < nlong) {
      float sn, cs;
      __sincosf(lw[r2] * t0, &sn, &cs);
      const float ea = ex2_approx(-la[r2] * t0);
      if (plane[r2]) vt = fmaf(ea, fmaf(phi[r2].x, sn, phi[r2].y * cs), vt);   // Im(Phi e^{s t})
      else v = fmaf(ea, fmaf(phi[r2].x, cs, -phi[r2].y * sn), v);             // Re(Phi e^{s t})
    }
  }
  float sw, cw;
  __sincosf(c.w * t0, &sw, &cw);
  float rf = fmaf(-c.rfB, sw, fmaf(c.rfA, cw, -c.rfA));
  for (int k = 0; k < nharm; ++k) {
    const float4 h = hc[k];
    float sk, ck;
    __sincosf(h.w * t0, &sk, &ck);
    rf = fmaf(-h.x * sk, fmaf(ck, h.y, sk * h.z), rf);
  }
  const float inc = fmaf(-v, c.invE0, fmaf(c.qe, r, rf));
  // momentum ratio across the cavity: (1 + d_b) / (1 + d_b + g), d_b after the
  // wake kick, g the RF gain (the damping factor taken out of rf)
  const float db = fmaf(-v, tc.invE0, f64_to_f32_trunc(d));
  const float g = fmaf(rf, tc.inv_omD, tc.U0oE0);
  d = fma(d, omD_d, f32_to_f64_bits(inc));
  df = f64_to_f32_trunc(d);
  float p = fmaf(vt, tc.invE0, xp);
  p = fmaf(-p, __fdividef(g, 1.f + db + g), p);
  float sp, cp;
  __sincosf(fmaf(tc.mu0xi, df, tc.mu0), &sp, &cp);
  const float xn = fmaf(fmaf(tc.alpha, sp, cp), x, tc.beta * sp * p);
  const float pn = fmaf(-tc.gamma * sp, x, fmaf(-tc.alpha, sp, cp) * p);
  x = fmaf(tc.nx, rx, xn);
  xp = fmaf(tc.nxp, rxp, pn);
  return fmaf(c.aT0, df, t0);
}

// Four consecutive particles with a transverse plane: push, deposit of the
// count and of x into the cell, moment partials of both planes.
template <int NLONG_MAX>
__device__ __forceinline__ void quad_push_t(const PushConstF &c, const TransConstF &tc, const float2 *sVd,
                                            const float2 *sVt, int *sH, unsigned *sLo, int *sHi, int nlong,
                                            const int *plane, const float *la, const float *lw, const float2 *phi,
                                            double omD_d, const float4 *hc, int nharm, bool ngp, float vrw,
                                            float (&tt)[4], double (&dd)[4], float (&xx)[4], float (&pp)[4],
                                            const float (&rr)[4], const float (&rx)[4], const float (&rp)[4],
                                            int nvalid, float tref, float dref, float (&mom)[8], int &nout,
                                            bool &ok) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (e < nvalid) {
      float df;
      const float t1 = push_one_t<NLONG_MAX>(c, tc, sVd, sVt, nlong, plane, la, lw, phi, omD_d, hc, nharm, ngp, vrw,
                                             tt[e], dd[e], rr[e], df, xx[e], pp[e], rx[e], rp[e]);
      tt[e] = t1;
      const float xb = fmaf(t1, c.invD, c.HinvD);
      const bool in = xb >= -0.5f && xb < c.fnb - 0.5f;
      const int cell = in ? __float2int_rn(xb) : c.nbins + (int)(threadIdx.x & 31);   // spill cell outside
      atomicAdd(&sH[cell], 1);
      ok &= deposit_dip(sLo, sHi, cell, xx[e], tc);
      nout += in ? 0 : 1;
      const float u = t1 - tref, v = df - dref;   // as in quad_push
      mom[0] += u;
      mom[1] = fmaf(u, u, mom[1]);
      mom[2] += v;
      mom[3] = fmaf(v, v, mom[3]);
      mom[4] += xx[e];
      mom[5] = fmaf(xx[e], xx[e], mom[5]);
      mom[6] += pp[e];
      mom[7] = fmaf(pp[e], pp[e], mom[7]);
    }
  }
}

// A full quad (four valid particles) of a run with a transverse plane,
// linear kick interpolation and no harmonic cavity: the map of push_one_t in
// one straight block, so that the four particles overlap.  Each long-range
// entry adds ea (A.x cos + A.y sin) to the plane its masks select:
// A = (Re Phi, -Im Phi), ml = 1, mt = 0 for a longitudinal entry (Re(Phi e^{s t}));
// A = (Im Phi, Re Phi), ml = 0, mt = 1 for a transverse one (Im(Phi e^{s t})).
// Deposits go to the cell or, outside the mesh, to the lane's spill cell
// (sH, sLo and sHi hold nbins + kSpillCells cells).
template <int NLONG_MAX>
__device__ __forceinline__ void quad_push_t_full(const PushConstF &c, const TransConstF &tc, const float4 *sV4,
                                                 int *sH, unsigned *sLo, int *sHi,
                                                 const float *la, const float *lw, const float2 *A, const float *ml,
                                                 const float *mt, double omD_d, float vrw, float (&tt)[4],
                                                 double (&dd)[4], float (&xx)[4], float (&pp)[4],
                                                 const float (&rr)[4], const float (&rx)[4], const float (&rp)[4],
                                                 float tref, float dref, float (&mom)[8], int &nout, bool &ok) {
  int cell[4];
  float dfs[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float t0 = tt[e];
    const float x0 = fmaf(t0, c.invD, c.HinvD);
    const bool inside = x0 >= -0.5f && x0 < c.fnb - 0.5f;
    const float u = fminf(fmaxf(x0, 0.f), c.fnb - 1.f);
    const int j = (int)u;   // <= nbins - 1, where the slopes are 0
    const float4 w4 = sV4[j];   // (V, dV, V_x, dV_x) of cell j
    float v = inside ? fmaf(u - (float)j, w4.y, w4.x) : 0.f;
    float vt = (inside ? fmaf(u - (float)j, w4.w, w4.z) : 0.f) + vrw;
    // every entry up to NLONG_MAX: the caller zeroes la, lw, A and the masks
    // of the entries a run does not have, which then add exactly zero
#pragma unroll
    for (int r2 = 0; r2 < NLONG_MAX; ++r2) {
      float sn, cs;
      __sincosf(lw[r2] * t0, &sn, &cs);
      const float w = ex2_approx(-la[r2] * t0) * fmaf(A[r2].x, cs, A[r2].y * sn);
      v = fmaf(ml[r2], w, v);
      vt = fmaf(mt[r2], w, vt);
    }
    float sw, cw;
    __sincosf(c.w * t0, &sw, &cw);
    const float rf = fmaf(-c.rfB, sw, fmaf(c.rfA, cw, -c.rfA));
    const float inc = fmaf(-v, c.invE0, fmaf(c.qe, rr[e], rf));
    const float db = fmaf(-v, tc.invE0, f64_to_f32_trunc(dd[e]));
    const float g = fmaf(rf, tc.inv_omD, tc.U0oE0);
    dd[e] = fma(dd[e], omD_d, f32_to_f64_bits(inc));
    const float df = f64_to_f32_trunc(dd[e]);
    dfs[e] = df;
    float p = fmaf(vt, tc.invE0, pp[e]);
    p = fmaf(-p, __fdividef(g, 1.f + db + g), p);
    float sp, cp;
    __sincosf(fmaf(tc.mu0xi, df, tc.mu0), &sp, &cp);
    const float xn = fmaf(fmaf(tc.alpha, sp, cp), xx[e], tc.beta * sp * p);
    const float pn = fmaf(-tc.gamma * sp, xx[e], fmaf(-tc.alpha, sp, cp) * p);
    xx[e] = fmaf(tc.nx, rx[e], xn);
    pp[e] = fmaf(tc.nxp, rp[e], pn);
    const float t1 = fmaf(c.aT0, df, t0);
    tt[e] = t1;
    const float xb = fmaf(t1, c.invD, c.HinvD);
    const bool in = xb >= -0.5f && xb < c.fnb - 0.5f;
    cell[e] = in ? __float2int_rn(xb) : c.nbins + (int)(threadIdx.x & 31);
    nout += in ? 0 : 1;
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    atomicAdd(&sH[cell[e]], 1);
    ok &= deposit_dip(sLo, sHi, cell[e], xx[e], tc);
    const float u = tt[e] - tref, v = dfs[e] - dref;
    mom[0] += u;
    mom[1] = fmaf(u, u, mom[1]);
    mom[2] += v;
    mom[3] = fmaf(v, v, mom[3]);
    mom[4] += xx[e];
    mom[5] = fmaf(xx[e], xx[e], mom[5]);
    mom[6] += pp[e];
    mom[7] = fmaf(pp[e], pp[e], mom[7]);
  }
}

__device__ __forceinline__ TransConstF trans_consts(const RunDev *__restrict__ R) {
  TransConstF t;
  t.mu0 = R->f_tmu0;
  t.mu0xi = R->f_tmu0xi;
  t.beta = R->f_tbeta;
  t.alpha = R->f_talpha;
  t.gamma = R->f_tgamma;
  t.nx = R->f_tnx;
  t.nxp = R->f_tnxp;
  t.invE0 = R->f_invE0;
  t.inv_omD = R->f_inv_omD;
  t.U0oE0 = R->f_U0oE0;
  t.dinv = R->f_dip_inv;
  t.drange = R->f_dip_range;
  return t;
}

}  // namespace mbt
