// Per-particle map of the mixed-precision path (shared by the streaming push
// kernel and the cluster-resident kernel): wake kick, RF, damping +
// excitation, drift (arXiv:1809.00391 Sec. 2.2-2.3, readings in mbt.h), and
// the quad step that adds deposit and moment partials.
#pragma once
#include "device_common.cuh"

namespace mbt {

struct PushConstF {
  float invD, HinvD, fnb, invE0, twoVoE0, cphi, sphi, halfw, omD, qe, aT0;
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
  const float x = fmaf(t0, c.invD, c.HinvD);
  float v;
  if (NGP) {
    const int k = min(max((int)x, 0), c.nbins - 1);
    v = sVd[k].x;
  } else {
    // linear interpolation between cell centres, clamped to the end cells
    const float u = fminf(fmaxf(x - 0.5f, 0.f), c.fnb - 1.f);
    const int j = min((int)u, c.nbins - 2);
    const float2 vd = sVd[j];
    v = fmaf(u - (float)j, vd.y, vd.x);
  }
  v = (x >= 0.f && x < c.fnb) ? v : 0.f;
#pragma unroll
  for (int r2 = 0; r2 < NLONG_MAX; ++r2) {
    if (r2 < nlong) {
      float sn, cs;
      __sincosf(lw[r2] * t0, &sn, &cs);
      const float ea = __expf(-la[r2] * t0);
      v = fmaf(ea, fmaf(phi[r2].x, cs, -phi[r2].y * sn), v);
    }
  }
  // (V/E0)[sin(phi_s - w t) - sin(phi_s)] = -2 (V/E0) sin(w t / 2) cos(phi_s - w t / 2)
  float sh, ch;
  __sincosf(c.halfw * t0, &sh, &ch);
  // c.twoVoE0 and c.invE0 carry the damping factor (1 - D) already
  float rf = -c.twoVoE0 * sh * fmaf(ch, c.cphi, sh * c.sphi);
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
template <int NLONG_MAX, bool NGP, bool HARM>
__device__ __forceinline__ void quad_push(const PushConstF &c, const float2 *sVd, int *sH, int nlong, const float *la,
                                          const float *lw, const float2 *phi, double omD_d, const float4 *hc,
                                          int nharm, float (&tt)[4], double (&dd)[4], const float (&rr)[4],
                                          int nvalid, float &st, float &st2, float &sd, float &sd2, int &nout) {
  const bool full = nvalid == 4;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (full || e < nvalid) {
      float df;
      const float t1 = push_one<NLONG_MAX, NGP, HARM>(c, sVd, nlong, la, lw, phi, omD_d, hc, nharm, tt[e], dd[e], rr[e], df);
      tt[e] = t1;
      const float xb = fmaf(t1, c.invD, c.HinvD);
      if (xb >= 0.f && xb < c.fnb) atomicAdd(&sH[(int)xb], 1);
      else ++nout;
      st += t1;
      st2 = fmaf(t1, t1, st2);
      sd += df;
      sd2 = fmaf(df, df, sd2);
    }
  }
}

}  // namespace mbt
