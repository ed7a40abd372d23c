"""Chapman-Enskog check of the oracle (Sec. II.C), with no GPU.

For a small-amplitude plane wave phi = A exp(i k.x) about phi = phiB = 0 (where f''(0) = 2 beta > 0 and the
force F1 = -(phi^2/rho) grad mu of Eq. t0-phiu vanishes to first order) in a uniform flow u, every step of
Eq. LB is linear, and the slow mode grows by a factor lambda(k) per step.  The Chapman-Enskog expansion of
the paper is the expansion of s = ln lambda in powers of epsilon = |k|:

    s = s1 eps + s2 eps^2 + s3 eps^3 + ...,

the continuum equation  d_t phi + div(phi u) = div(M grad mu) + R1 + R2 + O(eps^4)  in Fourier form
(Eqs. ch-equation-t2, phit3, phit3inserting).  Here the series is derived exactly from the discrete update
itself -- D2Q9 streaming, the equilibria of Eq. geq, the source of Eq. liangFi and the isotropic stencils
(R4), written out below independently of the oracle, in exact rational complex arithmetic -- and then:

* s1 = -i k.u and s2 = -M f''(0) |k|^2, with M = c_s^2 eta (tau - 1/2): the Cahn-Hilliard equation is
  recovered at second order;
* s3 equals the paper's third-order error R1 + R2 of Eq. phit3inserting, with sum_i D_1i^3 g_i^(0) of Eq.
  Di3geq, for Model I (F2 = 0), Model II (F2 of Eq. mark3) and the complete F2 of Eq. F2-1 (Model III,
  whose time derivatives reading R15 takes as backward differences), exactly;
* the oracle, run on such waves, grows them by exactly that series: its measured s(k) agrees with the
  five-term series to O(eps^6) on two grids (the remainder falls as eps^6), and the remainder after three
  terms falls as eps^4.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

import oracle
from paper_1805_00007_gb300 import workloads as wl

P = 6  # series kept to eps^5


class Gq:
    """A complex number with rational parts, exact."""
    __slots__ = ("re", "im")

    def __init__(self, re=0, im=0):
        self.re, self.im = Fr(re), Fr(im)

    def __add__(self, o):
        o = _g(o); return Gq(self.re + o.re, self.im + o.im)
    __radd__ = __add__

    def __sub__(self, o):
        o = _g(o); return Gq(self.re - o.re, self.im - o.im)

    def __rsub__(self, o):
        return _g(o) - self

    def __neg__(self):
        return Gq(-self.re, -self.im)

    def __mul__(self, o):
        o = _g(o); return Gq(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)
    __rmul__ = __mul__

    def inv(self):
        d = self.re * self.re + self.im * self.im
        return Gq(self.re / d, -self.im / d)

    def __truediv__(self, o):
        return self * _g(o).inv()

    def __eq__(self, o):
        o = _g(o); return self.re == o.re and self.im == o.im

    def __complex__(self):
        return complex(float(self.re), float(self.im))


def _g(x):
    return x if isinstance(x, Gq) else Gq(x)


I = Gq(0, 1)


class Ser:
    """A power series in eps truncated after eps^(P-1), exact coefficients."""

    def __init__(self, c):
        c = [_g(v) for v in c][:P]
        self.c = c + [Gq()] * (P - len(c))

    @staticmethod
    def const(v):
        return Ser([v])

    def __add__(self, o):
        o = o if isinstance(o, Ser) else Ser.const(o)
        return Ser([a + b for a, b in zip(self.c, o.c)])
    __radd__ = __add__

    def __sub__(self, o):
        o = o if isinstance(o, Ser) else Ser.const(o)
        return Ser([a - b for a, b in zip(self.c, o.c)])

    def __rsub__(self, o):
        return Ser.const(o) - self

    def __mul__(self, o):
        if not isinstance(o, Ser):
            return Ser([a * o for a in self.c])
        r = [Gq() for _ in range(P)]
        for i, a in enumerate(self.c):
            for j in range(P - i):
                r[i + j] = r[i + j] + a * o.c[j]
        return Ser(r)
    __rmul__ = __mul__

    def inv(self):
        b = [self.c[0].inv()]
        for n in range(1, P):
            acc = Gq()
            for k in range(1, n + 1):
                acc = acc + self.c[k] * b[n - k]
            b.append(-acc * b[0])
        return Ser(b)

    def __truediv__(self, o):
        return self * (o.inv() if isinstance(o, Ser) else Ser.const(_g(o).inv()))


def ser_exp(x: Ser) -> Ser:
    """exp of a series with zero constant term (n E_n = sum_k k X_k E_(n-k))."""
    assert x.c[0] == 0
    e = [Gq(1)]
    for n in range(1, P):
        acc = Gq()
        for k in range(1, n + 1):
            acc = acc + k * x.c[k] * e[n - k]
        e.append(acc * Fr(1, n))
    return Ser(e)


# the lattice of Sec. II.B, written here independently of the oracle
CQ = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WQ = [Fr(4, 9)] + [Fr(1, 9)] * 4 + [Fr(1, 36)] * 4
CS2 = Fr(1, 3)
KHAT = (Fr(3, 5), Fr(4, 5))  # direction of k, |KHAT| = 1; mixes both lattice axes


def plane(q, sign):
    """exp(sign i eps khat.c_q) as a series."""
    r = KHAT[0] * CQ[q][0] + KHAT[1] * CQ[q][1]
    return ser_exp(Ser([0, I * (sign * r)]))


def slow_mode_series(tau, ux, uy, beta, kappa, eta, model):
    """s_1..s_5 of s = ln lambda for the slow mode of the linearised step at phi = 0 (f''(0) = 2 beta),
    from the secular equation of the update.  Pull streaming multiplies direction q by e_q =
    exp(-i k.c_q); the post-collision value is (1 - 1/tau) g_q + (a_q / tau + (1 - 1/(2 tau)) b_q) phi, with
    a_q phi the equilibrium and b_q phi the source; so lambda solves sum_q e_q c_q / (lambda - omega e_q) = 1
    (omega = 1 - 1/tau), whose eps^n coefficient is linear in s_n with slope -tau."""
    ep = [plane(q, +1) for q in range(9)]
    em = [plane(q, -1) for q in range(9)]
    # isotropic stencils (R4): grad -> sum_k w_k c_k e^{i k.c_k}/c_s^2, lap -> sum_k 2 w_k (e^{i k.c_k} - 1)/c_s^2
    Gx = sum((ep[q] * (WQ[q] * CQ[q][0] / CS2) for q in range(1, 9)), Ser.const(0))
    Gy = sum((ep[q] * (WQ[q] * CQ[q][1] / CS2) for q in range(1, 9)), Ser.const(0))
    L = sum(((ep[q] - 1) * (2 * WQ[q] / CS2) for q in range(1, 9)), Ser.const(0))
    mu = Ser.const(2 * beta) - L * kappa           # Eq. mu, linearised: mu = f''(0) phi - kappa lap phi
    K = (tau - Fr(1, 6) - tau * tau) / (tau - Fr(1, 2))
    uu = ux * ux + uy * uy
    omega = 1 - 1 / tau
    s = [Gq() for _ in range(P)]
    for n in range(1, P):
        lam = ser_exp(Ser(s))
        if model == 1:
            Fx = Fy = Ser.const(0)
        else:
            D = Gx * ux + Gy * uy                      # div(phi u) / phi
            Fx, Fy = Gx * D * (3 * CS2 * K), Gy * D * (3 * CS2 * K)   # Eq. mark3
            if model == 3:
                # Eq. F2-1 with F1 = 0: H = 3 c_s^2 eta K grad mu; its time derivative over one step is
                # H (1 - 1/lambda) for a mode that grows by lambda (reading R15)
                dt = 1 - lam.inv()
                Fx = Fx + Gx * mu * dt * (3 * CS2 * eta * K)
                Fy = Fy + Gy * mu * dt * (3 * CS2 * eta * K)
        F = Ser.const(-1)
        for q in range(9):
            cu = CQ[q][0] * ux + CQ[q][1] * uy
            if q == 0:
                a = Ser.const(1 - WQ[0] * uu / (2 * CS2)) + mu * ((WQ[0] - 1) * eta)
            else:
                a = mu * (WQ[q] * eta) + Ser.const(WQ[q] * (cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)))
            b = (Fx * CQ[q][0] + Fy * CQ[q][1]) * (WQ[q] / CS2)   # Eq. liangFi
            cq = a * (1 / tau) + b * (1 - 1 / (2 * tau))
            F = F + em[q] * cq / (lam - em[q] * omega)
        assert all(F.c[m] == 0 for m in range(n)), "lower orders must already vanish"
        s[n] = F.c[n] / tau
    return s[1:]


def paper_terms(tau, ux, uy, beta, eta, model):
    """s1, s2 and R1 + R2 of Eq. phit3inserting in Fourier form for a unit wave vector khat: d_t1 -> -i a
    on phi (Eq. dt1Phi, a = khat.u), div(. u) -> i a, lap -> -1, mu -> f''(0) phi."""
    a = KHAT[0] * ux + KHAT[1] * uy
    fpp = 2 * beta
    M = CS2 * eta * (tau - Fr(1, 2))
    T, Dv, Lp = -I * a, I * a, Gq(-1)
    c1 = tau - Fr(1, 6) - tau * tau
    K = c1 / (tau - Fr(1, 2))
    # Eq. Di3geq (first line): sum_i D_1i^3 g_i^(0)
    D3 = T * T * T + 3 * T * T * Dv + 3 * T * (Dv * Dv + CS2 * eta * fpp * Lp) + 3 * CS2 * Lp * Dv
    R1 = c1 * D3
    if model == 1:
        divF2 = Gq()
    elif model == 2:
        divF2 = 3 * CS2 * K * Lp * Dv                                  # Eq. mark3
    else:
        divF2 = 3 * CS2 * eta * K * T * fpp * Lp + 3 * CS2 * K * Lp * Dv  # Eq. F2-1 with F1 = 0
    R2 = -(tau - Fr(1, 2)) * divF2  # S^(1) = 0; sum_i (d_t1 + c_i.grad) S_i^(2) = div F^(2)
    return -I * a, Gq(-M * fpp), R1 + R2


CASES = [(Fr(4, 5), 1), (Fr(4, 5), 2), (Fr(4, 5), 3), (Fr(1), 1), (Fr(1), 2), (Fr(13, 10), 3)]
UX, UY = Fr(1, 20), Fr(-1, 40)
BETA, KAPPA, ETA = Fr(3, 100), Fr(3, 50), Fr(1, 10)   # sigma = 0.01, W = 4 (Eq. betakappa); eta = 0.1


@pytest.mark.parametrize("tau,model", CASES)
def test_series_of_the_update_is_the_papers_chapman_enskog_expansion(tau, model):
    s = slow_mode_series(tau, UX, UY, BETA, KAPPA, ETA, model)
    p1, p2, p3 = paper_terms(tau, UX, UY, BETA, ETA, model)
    assert s[0] == p1 and s[1] == p2   # the Cahn-Hilliard equation at O(eps^2)
    assert s[2] == p3                  # the third-order error is exactly R1 + R2


def test_model_ii_removes_the_lattice_part_of_the_third_order_error():
    """What the diffusive-scale force buys, in the paper's terms: Model I's third-order error carries
    -3 c_s^2 (tau - 1/6 - tau^2) i a |k|^2 from the lattice; Eq. mark3 removes it, leaving the eta and Mach
    terms; the complete F2 of Eq. F2-1 leaves only the O(Ma^3) term (tau - 1/6 - tau^2) i a^3."""
    tau = Fr(4, 5)
    a = KHAT[0] * UX + KHAT[1] * UY
    c1 = tau - Fr(1, 6) - tau * tau
    s = {m: slow_mode_series(tau, UX, UY, BETA, KAPPA, ETA, m)[2] for m in (1, 2, 3)}
    assert s[1] - s[2] == I * (-3 * CS2 * c1 * a)
    assert s[3] == I * (c1 * a * a * a)
    assert s[2] - s[3] == I * (3 * CS2 * c1 * a * ETA * 2 * BETA)


def _measured_s(tau, model, N, nsteps=40, amp=1e-7):
    """ln(growth per step) of the oracle for the wave k = 2 pi (3, 4)/N (|k| = 10 pi/N along KHAT)."""
    M = float(CS2 * ETA * (tau - Fr(1, 2)))
    p = wl.make_params(nx=N, ny=N, vel=wl.VEL_UNIFORM, ux0=float(UX), uy0=float(UY), model=model,
                       tau=float(tau), M=M, sigma=0.01, W=4.0, phiA=1.0, phiB=0.0)
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    kx, ky = 2 * math.pi * 3 / N, 2 * math.pi * 4 / N
    phi0 = amp * np.cos(kx * x + ky * y)
    wave = np.exp(-1j * (kx * x + ky * y))
    if model == 3:
        g, H = oracle.run_full(p, oracle.init(p, phi0), None, nsteps)
        a0 = np.sum(oracle.phi_of(g) * wave)
        g, H = oracle.run_full(p, g, H, 1, n0=nsteps)
    else:
        g = oracle.run(p, oracle.init(p, phi0), nsteps)
        a0 = np.sum(oracle.phi_of(g) * wave)
        g = oracle.run(p, g, 1, n0=nsteps)
    a1 = np.sum(oracle.phi_of(g) * wave)
    return complex(np.log(a1 / a0)), math.hypot(kx, ky)


@pytest.mark.parametrize("tau,model", [(Fr(4, 5), 1), (Fr(4, 5), 2), (Fr(1), 2), (Fr(13, 10), 3)])
def test_oracle_follows_the_series(tau, model):
    s = [complex(v) for v in slow_mode_series(tau, UX, UY, BETA, KAPPA, ETA, model)]

    def part(eps, n):
        return sum(s[j] * eps ** (j + 1) for j in range(n))

    r3, r5 = [], []
    for N in (100, 200):
        meas, eps = _measured_s(tau, model, N)
        r3.append(abs(meas - part(eps, 3)))
        r5.append(abs(meas - part(eps, 5)))
        assert r5[-1] <= 2e-3 * eps ** 6       # agreement to O(eps^6)
    assert 12.0 <= r3[0] / r3[1] <= 20.0        # the remainder after s3 is O(eps^4): halving eps divides by 16
    assert 45.0 <= r5[0] / r5[1] <= 130.0       # and after s5 it is O(eps^6): halving eps divides by about 64
