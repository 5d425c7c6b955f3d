"""Exact stroke average of shape-driven dumbbells (TEST INFRASTRUCTURE ONLY).

The stroke-averaged law of Eqs. (9a)-(9e) is a far-field, leading-order
result.  This module computes the quantity it approximates without any
expansion, following the construction of Appendix A.2 (Sec. "Three-
dimensional case"):

* dumbbells of prescribed length L^s(t) = ell + lambda sin(omega t + phi^s),
  spheres at X^{s,1|2} = R^s -/+ N^s L^s / 2 (Eq. (A-3d coordinates));
* Oseen mobility, Eq. (3) without its a^2 line, with the Stokes self term;
* internal forces F^{s1} = f^s N^s, F^{s2} = -f^s N^s (force- and torque-free,
  Eq. (force ansatz)); the unknown f^s solve the shape constraints
  dL^s/dt = N^s . (dX^{s2}/dt - dX^{s1}/dt) (Eq. (constraint)) exactly, as
  one dense linear system (all orders of the iteration of Eq. (iteration)
  at once);
* dR^s/dt = (dX^{s1} + dX^{s2}) / 2 and
  dN^s/dt = (I - N^s N^s) (dX^{s2} - dX^{s1}) / L^s (Eq. (exact 3d EOM));
* the rates are averaged over one period with R and N frozen, the slowly-
  varying approximation of Eq. (8).

Everything runs in mpmath at 40 significant digits: the averaged rates are
~1e-10 of the instantaneous sphere velocities, far below double precision.
"""
import mpmath as mp

mp.mp.dps = 40


def _oseen(rv, mu):
    r = mp.sqrt(sum(c * c for c in rv))
    k = 1 / (8 * mp.pi * mu * r)
    return [[k * ((1 if i == j else 0) + rv[i] * rv[j] / r ** 2) for j in range(3)] for i in range(3)]


def _mv(M, v):
    return [sum(M[i][j] * v[j] for j in range(3)) for i in range(3)]


def _dot(u, v):
    return sum(u[i] * v[i] for i in range(3))


def rates(R, Nv, L, Ldot, a, mu):
    """Instantaneous (dR/dt, dN/dt) of every shape-driven dumbbell."""
    nd = len(R)
    X = [[[R[s][k] + (-1) ** (b + 1) * Nv[s][k] * L[s] / 2 for k in range(3)] for b in range(2)]
         for s in range(nd)]

    def H(s1, b1, s2, b2):
        if s1 == s2 and b1 == b2:
            g = 1 / (6 * mp.pi * mu * a)
            return [[g if i == j else 0 for j in range(3)] for i in range(3)]
        return _oseen([X[s1][b1][k] - X[s2][b2][k] for k in range(3)], mu)

    # velocity of sphere (s, b) per unit f^r: force +N^r on sphere 1, -N^r on sphere 2
    unit = [[[None] * nd for _ in range(2)] for _ in range(nd)]
    for s in range(nd):
        for b in range(2):
            for r in range(nd):
                v1 = _mv(H(s, b, r, 0), Nv[r])
                v2 = _mv(H(s, b, r, 1), Nv[r])
                unit[s][b][r] = [v1[k] - v2[k] for k in range(3)]
    A = mp.matrix(nd, nd)
    for s in range(nd):
        for r in range(nd):
            A[s, r] = _dot(Nv[s], [unit[s][1][r][k] - unit[s][0][r][k] for k in range(3)])
    f = mp.lu_solve(A, mp.matrix(list(Ldot)))
    out = []
    for s in range(nd):
        x1 = [sum(unit[s][0][r][k] * f[r] for r in range(nd)) for k in range(3)]
        x2 = [sum(unit[s][1][r][k] * f[r] for r in range(nd)) for k in range(3)]
        Rd = [(x1[k] + x2[k]) / 2 for k in range(3)]
        w = [(x2[k] - x1[k]) / L[s] for k in range(3)]
        pr = _dot(Nv[s], w)
        out.append((Rd, [w[k] - Nv[s][k] * pr for k in range(3)]))
    return out


def stroke_averaged_rates(R, Nv, phi, *, ell, lam, omega, a, mu, M=16):
    """Period average of ``rates`` (trapezoid rule, exact for these trigonometric
    polynomials once M exceeds their degree).  Returns lists of (Rdot, Ndot)."""
    R = [[mp.mpf(c) for c in v] for v in R]
    Nv = [[mp.mpf(c) for c in v] for v in Nv]
    T = 2 * mp.pi / omega
    acc = [[[mp.mpf(0)] * 3, [mp.mpf(0)] * 3] for _ in R]
    for m in range(M):
        t = T * m / M
        L = [ell + lam * mp.sin(omega * t + p) for p in phi]
        Ld = [lam * omega * mp.cos(omega * t + p) for p in phi]
        for s, (rd, nd) in enumerate(rates(R, Nv, L, Ld, a, mu)):
            for k in range(3):
                acc[s][0][k] += rd[k] / M
                acc[s][1][k] += nd[k] / M
    return [([float(c) for c in r], [float(c) for c in n]) for r, n in acc]
