// Bunch-sharded long-range scan: the host side of splitting one fill's
// bunches over several GPUs (contiguous bunch ranges per rank).
//
// The long-range wake acts after all bunches of a turn (Sec. 2.3, last
// paragraph): bunch m meets the phasor Phi_m = a_m X_{m-1}, where
// X_m = a_m X_{m-1} + E_m is the phasor just after bunch m has passed (E_m its
// emission, a_m = e^{s dt_m} the decay and rotation over the bucket distance
// from the bunch before it; for the first bunch of a turn, from the last
// bunch of the previous turn across the gap).  Each step is an affine map
// f_m(X) = a_m X + E_m, so a rank holding bunches [lo, hi) reduces its part to
// one map X -> A X + B; the ranks exchange these (two complex numbers per
// long-range resonator), each composes the maps of the ranks before it with
// the value carried from the previous turn, and applies the result to its own
// bunches.  Every rank composes the same maps in the same order, so each
// holds the same new carry.  Host code only: the exchange itself is a
// collective of the caller (an allgather of 4 doubles per resonator).
#include <cmath>
#include <complex>

#include "../../include/mbt.h"

namespace {
using cplx = std::complex<double>;
inline cplx ld(const double *p) { return cplx(p[0], p[1]); }
inline void st(double *p, cplx z) {
  p[0] = z.real();
  p[1] = z.imag();
}
}  // namespace

extern "C" {

mbt_status mbt_phasor_steps(const mbt_ring *ring, double fr_Hz, double Q, int nb, const int32_t *bucket,
                            double *step) {
  if (!ring || !bucket || !step || nb < 1 || !(ring->T0_s > 0) || ring->h < 1 || !(fr_Hz > 0) || !(Q > 0.5))
    return MBT_ERR_ARG;
  for (int m = 0; m < nb; ++m)
    if (bucket[m] < 0 || bucket[m] >= ring->h || (m > 0 && bucket[m] <= bucket[m - 1])) return MBT_ERR_ARG;
  const double pi = 3.14159265358979323846264338327950288;
  const double wr = 2.0 * pi * fr_Hz, a = wr / (2.0 * Q), wb = std::sqrt(wr * wr - a * a);
  const cplx s(-a, wb);
  const double T_rf = ring->T0_s / (double)ring->h;
  for (int m = 0; m < nb; ++m) {
    const long long d = m > 0 ? (long long)bucket[m] - bucket[m - 1] : (long long)ring->h - bucket[nb - 1] + bucket[0];
    st(step + 2 * m, std::exp(s * ((double)d * T_rf)));
  }
  return MBT_OK;
}

mbt_status mbt_phasor_segment(int n, const double *step, const double *E, double *map) {
  if (n < 0 || (n > 0 && (!step || !E)) || !map) return MBT_ERR_ARG;
  cplx A(1.0, 0.0), B(0.0, 0.0);
  for (int m = 0; m < n; ++m) {
    const cplx a = ld(step + 2 * m);
    A = a * A;
    B = a * B + ld(E + 2 * m);
  }
  st(map, A);
  st(map + 2, B);
  return MBT_OK;
}

mbt_status mbt_phasor_compose(int nseg, const double *maps, const double *carry, double *entry, double *carry_out) {
  if (nseg < 1 || !maps || !carry || !carry_out) return MBT_ERR_ARG;
  cplx X = ld(carry);
  for (int r = 0; r < nseg; ++r) {
    if (entry) st(entry + 2 * r, X);
    X = ld(maps + 4 * r) * X + ld(maps + 4 * r + 2);
  }
  st(carry_out, X);
  return MBT_OK;
}

mbt_status mbt_phasor_apply(int n, const double *step, const double *E, const double *entry, double *phi) {
  if (n < 0 || (n > 0 && (!step || !E || !phi)) || !entry) return MBT_ERR_ARG;
  cplx X = ld(entry);
  for (int m = 0; m < n; ++m) {
    const cplx Phi = ld(step + 2 * m) * X;
    st(phi + 2 * m, Phi);
    X = Phi + ld(E + 2 * m);
  }
  return MBT_OK;
}

}  // extern "C"
