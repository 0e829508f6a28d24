"""Helpers shared by the physics tests: textbook synchrotron tune, Eq. 7 of the
paper (coupled-bunch growth rates for M equal, equally spaced bunches) and the
normal-form mode projection used to fit growth rates from bunch centroids."""
import math

import numpy as np

import mbt_workloads as W


def textbook_nu_s(ring, sr=True):
    """Small-amplitude synchrotron tune, nu_s^2 = alpha_c h eV cos(phi_s) / (2 pi E0)."""
    U0 = ring["U0_eV"] if sr else 0.0
    phi = math.asin(U0 / ring["V_rf_V"])
    if ring["alpha_c"] < 0:
        phi = math.pi - phi
    return math.sqrt(ring["alpha_c"] * ring["h"] * ring["V_rf_V"] * math.cos(phi) / (2 * math.pi * ring["E0_eV"]))


def map_tune(ring, sr=False):
    """Tune of the linearised kick-then-drift one-turn map."""
    nus = textbook_nu_s(ring, sr=sr)
    return math.acos(1 - (2 * math.pi * nus) ** 2 / 2) / (2 * math.pi)


def eq7_rate(M, mu, fr, Rs, Q, I_bunch, nu, ring=None):
    """Eq. 7 with omega_r in the numerator, summed over the positive-frequency
    upper (q M + mu) w0 + w_s and lower (q' M - mu) w0 - w_s lines [1/s]."""
    ring = ring or W.ring_r0()
    T0 = ring["T0_s"]
    w0 = 2 * math.pi / T0
    ws = nu * w0
    wr = 2 * math.pi * fr

    def ReZ(w):
        return (Rs / (1 + 1j * Q * (w / wr - wr / w))).real

    p0 = int(round(wr / w0 / M))
    up = sum(ReZ((q * M + mu) * w0 + ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M + mu) * w0 + ws > 0)
    lo = sum(ReZ((q * M - mu) * w0 - ws) for q in range(max(0, p0 - 50), p0 + 50) if (q * M - mu) * w0 - ws > 0)
    return ring["alpha_c"] * M * I_bunch * wr / (2 * ring["E0_eV"] * T0 * ws) * (up - lo)


def point_bunch_run(M, fr, Rs, I_bunch, turns, Q=2e4, amp=5e-12, n_mp=400, precision=W.PREC_F64, seed=3):
    """M point-like bunches (sigma_tau 3 ps, centroid offset amp with random
    phases) equally spaced in the ring, no radiation, a narrow long-range HOM."""
    ring = W.ring_r0()
    h, T0, ac = ring["h"], ring["T0_s"], ring["alpha_c"]
    nu = map_tune(ring)
    buckets = np.array([m * (h // M) for m in range(M)], np.int32)
    hom = dict(Rs_ohm=Rs, fr_Hz=fr, Q=Q, range=W.RANGE_LONG)
    run = W.Run(ring, [hom], buckets, np.full(M, I_bunch), np.full(M, n_mp, np.int64), seed=seed, turns=turns,
                precision=precision, flags=W.NO_SR)
    rng = np.random.default_rng(seed)
    st = 3e-12
    sdl = st * 2 * math.pi * nu / (ac * T0)
    parts = []
    for m in range(M):
        ph = rng.uniform(0, 2 * math.pi)
        parts.append((rng.normal(amp * math.cos(ph), st, n_mp), rng.normal(amp * math.sin(ph) * sdl / st, sdl, n_mp)))
    return run, parts


def mode_amplitudes(rec, ring=None):
    """X_mu(n) = sum_m z_m(n) e^{-2 pi i mu m / M} with z the normal-form
    coordinate (left eigenvector of the linear one-turn map, eigenvalue
    e^{+i 2 pi nu}) of the bunch centroids rec[n][m][0 (tau), 2 (delta)]."""
    ring = ring or W.ring_r0()
    M = rec.shape[1]
    T0, ac, h = ring["T0_s"], ring["alpha_c"], ring["h"]
    K = (ring["V_rf_V"] / ring["E0_eV"]) * 2 * math.pi * h / T0
    a = ac * T0
    M0 = np.array([[1 - a * K, a], [-K, 1.0]])
    ev, vl = np.linalg.eig(M0.T)
    wl = vl[:, int(np.argmax(ev.imag))]
    z = wl[0] * rec[:, :, 0] + wl[1] * rec[:, :, 2]
    return np.stack([(z * np.exp(-2j * math.pi * mu * np.arange(M) / M)[None, :]).sum(axis=1) for mu in range(M)])


def fit_rate(X, lo, hi, ring=None):
    """Exponential rate [1/s] of |X| over turns [lo, hi)."""
    ring = ring or W.ring_r0()
    n = np.arange(lo, hi)
    return np.polyfit(n, np.log(np.abs(X[lo:hi])), 1)[0] / ring["T0_s"]


def flat_potential(ring, n=3):
    """Textbook flat-potential setting of an n-th harmonic cavity: the energy
    change of a turn and its first two derivatives vanish at tau = 0:
      V sin(phi_s) + k V sin(phi_h) = U0,  cos(phi_s) + n k cos(phi_h) = 0,
      sin(phi_s) + n^2 k sin(phi_h) = 0
    => sin(phi_s) = n^2/(n^2-1) U0/V, k = sqrt(1/n^2 - (U0/V)^2/(n^2-1))."""
    u = ring["U0_eV"] / ring["V_rf_V"]
    sphi = n * n / (n * n - 1) * u
    cphi = math.sqrt(1 - sphi * sphi)
    k = math.sqrt(1 / n ** 2 - u * u / (n * n - 1))
    phih = math.atan2(-sphi / (n * n * k), -cphi / (n * k))
    return dict(n=n, V_V=k * ring["V_rf_V"], phi_rad=phih), sphi, cphi, k


def double_rf_equilibrium(ring, hcs, L):
    """Stationary line density exp(-Phi / (alpha_c T0 sigma_E^2)) with Phi the
    exact potential of the main and harmonic cavities and the mean loss."""
    E0, T0, V, ac, sd = ring["E0_eV"], ring["T0_s"], ring["V_rf_V"], ring["alpha_c"], ring["sigma_delta"]
    w = 2 * math.pi * ring["h"] / T0
    Uh = sum(hc["V_V"] * math.sin(hc["phi_rad"]) for hc in hcs)
    phis = math.asin((ring["U0_eV"] - Uh) / V)
    tau = np.linspace(-L, L, 20001)
    Phi = -((V / w) * (np.cos(phis - w * tau) - math.cos(phis)) - ring["U0_eV"] * tau)
    for hc in hcs:
        nw = hc["n"] * w
        Phi -= (hc["V_V"] / nw) * (np.cos(hc["phi_rad"] - nw * tau) - math.cos(hc["phi_rad"]))
    Phi /= E0
    lam = np.exp(-(Phi - Phi.min()) / (ac * T0 * sd * sd))
    lam /= np.trapezoid(lam, tau)
    return tau, lam


class RigidBunchModel:
    """Rigid-bunch linearised one-turn map of a fill (the coupled-bunch check
    for fills that Eq. 7 does not cover: adjacent bunches, a train with a gap).

    Each bunch m is a rigid Gaussian of rms length sigma_tau whose centroid
    (tau_m, delta_m) follows the per-turn map of the tracker in its order
    (Sec. 2.2-2.3 with readings R1-R4): the kick by the long-range wake of the
    previous turn, the RF gain minus the mean loss (Eq. 1), damping (Eq. 5,
    delta line; the excitation has zero mean), the drift with the new delta
    (Eq. 2).  Each long-range resonator (Rs, w_r, Q) has the wake
    W(t) = Re(c e^{s t}), s = -a + i wb, c = 2 a Rs (1 + i a / wb) (a = w_r/2Q,
    wb = sqrt(w_r^2 - a^2)); a bunch of charge Q_m passing at t_m leaves the
    phasor c Q_m <e^{-s tau}> e^{s (t - t_m)}, and a particle at tau in a later
    passage feels Re(A e^{s tau}) with A the phasor sum of every earlier
    passage (Sec. 2.3, last paragraph).  Over a Gaussian bunch
    <e^{+-s xi}> = e^{s^2 sigma^2 / 2} and <sin(phi - w xi)> = sin(phi)
    e^{-w^2 sigma^2 / 2}.  As in the tracker, the phasors computed after turn
    n kick the particles in turn n + 1.

    State x: tau_m, delta_m (m < M), then (Re, Im) of A_0 per resonator, the
    phasor that bunch 0 (the first bucket) met in the last turn; every other
    A_m of that turn follows from it and the emissions,
    A_m = e^{s (b_m - b_{m-1}) T_rf} (A_{m-1} + E_{m-1}), and the next turn's
    A_0 = e^{s (h + b_0 - b_{M-1}) T_rf} (A_{M-1} + E_{M-1}).  The Jacobian at
    the fixed point (central differences; the map is smooth) has eigenvalues
    lambda; ln|lambda| / T0 are the growth rates of the fill's modes.  Plain
    numpy, independent of the oracle and of the CUDA library."""

    def __init__(self, ring, buckets, currents_A, resonators, sigma_tau, flags=0):
        self.E0, self.T0, self.h = ring["E0_eV"], ring["T0_s"], int(ring["h"])
        self.Trf = self.T0 / self.h
        self.w = 2 * math.pi * self.h / self.T0
        sr = not (flags & W.NO_SR)
        U0 = ring["U0_eV"] if sr else 0.0
        self.VoE, self.UoE = ring["V_rf_V"] / self.E0, U0 / self.E0
        phi = math.asin(U0 / ring["V_rf_V"])
        self.phi = math.pi - phi if ring["alpha_c"] < 0 else phi
        self.D = 2 * self.T0 / ring["tau_z_s"] if sr else 0.0
        self.aT0 = ring["alpha_c"] * self.T0
        self.b = np.asarray(buckets, np.int64)
        self.M = len(self.b)
        self.Q = np.asarray(currents_A, np.float64) * self.T0
        self.g = math.exp(-0.5 * (self.w * sigma_tau) ** 2)
        self.s, self.c, self.F = [], [], []
        for r in resonators:
            if not (int(r["range"]) & W.RANGE_LONG):
                continue
            wr = 2 * math.pi * r["fr_Hz"]
            a = wr / (2 * r["Q"])
            wb = math.sqrt(wr * wr - a * a)
            s = complex(-a, wb)
            self.s.append(s)
            self.c.append(2 * a * r["Rs_ohm"] * (1 + 1j * a / wb))
            self.F.append(np.exp(s * s * sigma_tau ** 2 / 2))
        self.nr = len(self.s)
        self.n = 2 * self.M + 2 * self.nr
        # the recursion over the fill written out: A_m = e^{s (b_m - b_0) T_rf} A_0
        # + sum_{k < m} e^{s (b_m - b_k) T_rf} E_k (every exponent <= 0)
        lag = (self.b[:, None] - self.b[None, :]).astype(np.float64) * self.Trf
        self.Lm = [np.where(lag > 0, np.exp(s * np.maximum(lag, 0.0)), 0.0) for s in self.s]
        self.p0 = [np.exp(s * (self.b - self.b[0]) * self.Trf) for s in self.s]

    def phasors(self, x):
        """[nr][M] phasors A_m met by every bunch in the last turn, and the
        emissions [nr][M] of the state's centroids."""
        M = self.M
        tau = x[:M]
        A = np.empty((self.nr, M), complex)
        E = np.empty((self.nr, M), complex)
        for r in range(self.nr):
            E[r] = self.c[r] * self.Q * self.F[r] * np.exp(-self.s[r] * tau)
            A[r] = self.p0[r] * complex(x[2 * M + 2 * r], x[2 * M + 2 * r + 1]) + self.Lm[r] @ E[r]
        return A, E

    def turn(self, x):
        """One turn of the centroid map (non-linear)."""
        M = self.M
        tau, d = x[:M], x[M:2 * M]
        A, E = self.phasors(x)
        V = np.zeros(M)
        for r in range(self.nr):
            V += (A[r] * self.F[r] * np.exp(self.s[r] * tau)).real
        d = d - V / self.E0
        d = d + self.VoE * self.g * np.sin(self.phi - self.w * tau) - self.UoE
        d = d * (1 - self.D)
        out = np.empty(self.n)
        out[:M] = tau + self.aT0 * d
        out[M:2 * M] = d
        for r in range(self.nr):
            a0 = np.exp(self.s[r] * (self.h + self.b[0] - self.b[-1]) * self.Trf) * (A[r, -1] + E[r, -1])
            out[2 * M + 2 * r], out[2 * M + 2 * r + 1] = a0.real, a0.imag
        return out

    def jacobian(self, x):
        """Derivative of turn() at x, written out (central differences of
        turn() check it in the tests)."""
        M, n = self.M, self.n
        tau = x[:M]
        A, E = self.phasors(x)
        dV = np.zeros((M, n))   # dV_m / dx_j
        dA0 = []                # d(next A_0) / dx_j, complex
        for r in range(self.nr):
            s = self.s[r]
            G = self.F[r] * np.exp(s * tau)
            dE = -s * E[r]                                  # dE_m / dtau_m
            dA_tau = self.Lm[r] * dE[None, :]               # dA_m / dtau_k
            dV[:, :M] += (dA_tau * G[:, None]).real
            dV[np.arange(M), np.arange(M)] += (A[r] * s * G).real
            j = 2 * M + 2 * r
            dV[:, j] += (self.p0[r] * G).real
            dV[:, j + 1] += (1j * self.p0[r] * G).real
            kappa = np.exp(s * (self.h + self.b[0] - self.b[-1]) * self.Trf)
            row = np.zeros(n, complex)
            row[:M] = kappa * dA_tau[-1]
            row[M - 1] += kappa * dE[-1]
            row[j] = kappa * self.p0[r][-1]
            row[j + 1] = kappa * 1j * self.p0[r][-1]
            dA0.append(row)
        om = 1 - self.D
        dd = -om * dV / self.E0
        dd[np.arange(M), np.arange(M)] -= om * self.VoE * self.g * self.w * np.cos(self.phi - self.w * tau)
        dd[np.arange(M), M + np.arange(M)] += om
        J = np.zeros((n, n))
        J[:M] = self.aT0 * dd
        J[np.arange(M), np.arange(M)] += 1.0
        J[M:2 * M] = dd
        for r in range(self.nr):
            J[2 * M + 2 * r] = dA0[r].real
            J[2 * M + 2 * r + 1] = dA0[r].imag
        return J

    def _scales(self, x):
        M = self.M
        sc = np.empty(self.n)
        sc[:M], sc[M:2 * M] = 1e-12, 1e-6
        for r in range(self.nr):
            sc[2 * M + 2 * r:2 * M + 2 * r + 2] = 1e-3 * max(1.0, abs(complex(x[2 * M + 2 * r], x[2 * M + 2 * r + 1])))
        return sc

    def jacobian_fd(self, x, eps=1e-5):
        """turn()'s derivative by central differences."""
        sc = self._scales(x)
        J = np.empty((self.n, self.n))
        for j in range(self.n):
            e = np.zeros(self.n)
            e[j] = eps * sc[j]
            J[:, j] = (self.turn(x + e) - self.turn(x - e)) / (2 * e[j])
        return J

    def fixed_point(self, iters=30):
        """Newton's method on turn(x) = x, from the bare ring's synchronous state."""
        x = np.zeros(self.n)
        for _ in range(iters):
            dx = np.linalg.solve(self.jacobian(x) - np.eye(self.n), -(self.turn(x) - x))
            x = x + dx
            if np.max(np.abs(dx / self._scales(x))) < 1e-9:
                return x
        raise RuntimeError("no fixed point")

    def modes(self):
        """(growth rates [1/s], eigenvalues, right and left eigenvectors as
        columns, fixed point) of the linearised one-turn map."""
        x = self.fixed_point()
        J = self.jacobian(x)
        ev, vr = np.linalg.eig(J)
        evl, vl = np.linalg.eig(J.T)
        order = [int(np.argmin(np.abs(evl - e))) for e in ev]
        return np.log(np.abs(ev)) / self.T0, ev, vr, vl[:, order], x

    def dominant(self):
        """(rate, eigenvalue, left eigenvector) of the fastest-growing mode,
        the member of its conjugate pair with Im(lambda) > 0."""
        rates, ev, vr, vl, x = self.modes()
        k = int(np.argmax(rates + 1e-9 * np.sign(ev.imag)))
        return float(rates[k]), ev[k], vl[:, k]


def projected_rate(states, w, lo, hi, T0):
    """Exponential rate [1/s] over turns [lo, hi) of X(n) = w . (x(n+1) - x(n)),
    x(n) the tracked state of turn n (centroids and phasor A_0 as in
    RigidBunchModel): differences remove the fixed point, and the projection
    onto a left eigenvector keeps that one mode."""
    X = (states[1:] - states[:-1]) @ w
    n = np.arange(lo, hi)
    return float(np.polyfit(n, np.log(np.abs(X[lo:hi])), 1)[0] / T0)
