"""Differentiable reference of the WENO5/WENO7 + SSP-RK3 step in plain PyTorch
(CPU, float64) -- TEST INFRASTRUCTURE ONLY, part of the oracle.

It restates the scheme of the paper (Eq. 1 fluxes, Eq. 2 operator L, the
finite-difference WENO of Sec. 1.2 and the third-order Runge-Kutta of Sec. 1)
with torch tensor operations so that autograd yields the exact vector-Jacobian
product of N steps with the Lax-Friedrichs speeds and time steps frozen (they
are the only non-differentiable ingredients: maxima over the grid).  Used to
check the hand-written adjoint kernels at tiny sizes.  The WENO tables are
derived here from the definition with exact rational arithmetic.

Tensors: conserved state u of shape (5, nz, ny, nx) = (E, M_x, M_y, M_z, R).
"""
from fractions import Fraction

import torch


def _solve(A, b):
    """Exact Gaussian elimination over Fractions: A x = b (A square)."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p] = M[p], M[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [x - f * y for x, y in zip(M[i], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def weno_tables(r):
    """Candidate values q_k = p_k(1/2) and Taylor coefficients c_i (about the
    target cell, unit spacing) as rational weights of v_{j-r+1..j+r-1}; p_k
    matches the cell averages over cells j-r+1+k .. j+k."""
    half = Fraction(1, 2)
    S = 2 * r - 1
    q, taylor = [], []
    for k in range(r):
        offs = list(range(-r + 1 + k, k + 1))
        A = [[((o + half) ** (i + 1) - (o - half) ** (i + 1)) / (i + 1) for i in range(r)] for o in offs]
        # column m of the inverse gives the coefficients' dependence on v_{offs[m]}
        cols = [_solve(A, [Fraction(int(m == mm)) for mm in range(r)]) for m in range(r)]
        coef = [[Fraction(0)] * S for _ in range(r)]       # coef[i][s]: c_i weight of v_s
        for m, o in enumerate(offs):
            for i in range(r):
                coef[i][o + r - 1] = cols[m][i]
        taylor.append(coef)
        q.append([sum(coef[i][s] * half ** i for i in range(r)) for s in range(S)])
    # linear weights: sum_k d_k q_k equals the (2r-1)-cell reconstruction
    offs = list(range(-r + 1, r))
    A = [[((o + half) ** (i + 1) - (o - half) ** (i + 1)) / (i + 1) for i in range(S)] for o in offs]
    big = []
    for m in range(S):
        c = _solve(A, [Fraction(int(m == mm)) for mm in range(S)])
        big.append(sum(c[i] * half ** i for i in range(S)))
    # solve for d from the r rows with the most non-zeros (the system is exactly determined)
    rows = list(range(S))
    Asys = [[q[k][s] for k in range(r)] for s in rows]
    bsys = [big[s] for s in rows]
    d = _solve([Asys[s] for s in range(r)], [bsys[s] for s in range(r)])
    assert all(sum(Asys[s][k] * d[k] for k in range(r)) == bsys[s] for s in rows)
    return q, taylor, d


_TAB = {}


def _tab(r):
    if r not in _TAB:
        q, t, d = weno_tables(r)
        _TAB[r] = ([[float(x) for x in row] for row in q],
                   [[[float(x) for x in row] for row in tk] for tk in t],
                   [float(x) for x in d])
    return _TAB[r]


def _falling(a, l):
    f = 1
    for i in range(l):
        f *= (a - i)
    return f


def weno_left(r, v, eps):
    """v: list of 2r-1 tensors v_{j-r+1..j+r-1}; value at x_{j+1/2}."""
    q, t, d = _tab(r)
    alphas, qs = [], []
    for k in range(r):
        qk = sum(q[k][s] * v[s] for s in range(2 * r - 1) if q[k][s] != 0.0)
        c = [None] + [sum(t[k][i][s] * v[s] for s in range(2 * r - 1) if t[k][i][s] != 0.0) for i in range(1, r)]
        beta = 0.0
        for l in range(1, r):
            for a in range(l, r):
                for b in range(l, r):
                    pw = (a - l) + (b - l)
                    if pw % 2:
                        continue
                    beta = beta + _falling(a, l) * _falling(b, l) / ((pw + 1) * 2.0 ** pw) * c[a] * c[b]
        alphas.append(d[k] / (eps + beta) ** 2)
        qs.append(qk)
    tot = sum(alphas)
    return sum(a / tot * qk for a, qk in zip(alphas, qs))


def con2prim(u, k):
    E, M, R = u[0], u[1:4], u[4]
    m2 = (M * M).sum(0)
    dd = E * E - m2
    b = (1 - k) * E
    e = 2 * dd / (b + torch.sqrt(b * b + 4 * k * dd))
    p = k * e
    v = M / (E + p)
    return e, p, v


def flux(u, p, v, d):
    f0 = u[1 + d]
    fm = [u[1 + j] * v[d] + (p if j == d else 0.0) for j in range(3)]
    return torch.stack([f0] + fm + [u[4] * v[d]])


def _pad(u, G, n, bc):
    """Ghost cells by the boundary rule (copy edge cell / wrap) on every axis
    with more than one cell."""
    out = u
    for d in range(3):
        if n[d] <= 1:
            continue
        ax = 3 - d
        L = out.shape[ax]
        if bc[d] == 1:
            lo = out.narrow(ax, L - G, G)
            hi = out.narrow(ax, 0, G)
        else:
            lo = out.narrow(ax, 0, 1).expand(*[G if i == ax else -1 for i in range(4)])
            hi = out.narrow(ax, L - 1, 1).expand(*[G if i == ax else -1 for i in range(4)])
        out = torch.cat([lo, out, hi], dim=ax)
    return out


def L_op(u, alpha, n, dx, bc, r, k=1.0 / 3.0, eps=1e-6):
    """Eq. 2 with FD-WENO on f^{+-} = (f +- alpha_d u)/2."""
    G = r
    up = _pad(u, G, n, bc)
    e, p, v = con2prim(up, k)
    Lu = torch.zeros_like(u)
    for d in range(3):
        if n[d] <= 1:
            continue
        ax = 3 - d
        f = flux(up, p, v, d)
        fp = 0.5 * (f + alpha[d] * up)
        fm = 0.5 * (f - alpha[d] * up)
        # keep only interior cells on the other active axes
        for dd in range(3):
            if dd != d and n[dd] > 1:
                fp = fp.narrow(3 - dd, G, n[dd])
                fm = fm.narrow(3 - dd, G, n[dd])
        nd = n[d]
        # face s (s = 0..nd) sits at x_{s-1/2}; left cell index s-1 -> padded s-1+G
        vp = [fp.narrow(ax, s, nd + 1) for s in range(2 * r - 1)]          # j-r+1.. for j = s-1+G
        vm = [fm.narrow(ax, s + 1, nd + 1) for s in range(2 * r - 1)]
        F = weno_left(r, vp, eps) + weno_left(r, vm[::-1], eps)
        Lu = Lu + (F.narrow(ax, 0, nd) - F.narrow(ax, 1, nd)) / dx[d]
    return Lu


def rk3_step(u, alphas, dt, n, dx, bc, r, k=1.0 / 3.0, eps=1e-6):
    """One SSP-RK3 step; alphas: (3 stages, 3 axes) frozen speeds."""
    u1 = u + dt * L_op(u, alphas[0], n, dx, bc, r, k, eps)
    u2 = 0.75 * u + 0.25 * (u1 + dt * L_op(u1, alphas[1], n, dx, bc, r, k, eps))
    return u / 3.0 + 2.0 / 3.0 * (u2 + dt * L_op(u2, alphas[2], n, dx, bc, r, k, eps))


def run_frozen(u, alphas, dts, n, dx, bc, r, k=1.0 / 3.0, eps=1e-6):
    """N steps with frozen speeds alphas[s][stage][axis] and steps dts[s]."""
    for s in range(len(dts)):
        a = [[float(alphas[s][st][d]) for d in range(3)] for st in range(3)]
        u = rk3_step(u, a, float(dts[s]), n, dx, bc, r, k, eps)
    return u


def eps2(u, k=1.0 / 3.0):
    """Momentum anisotropy sum(T^xx - T^yy) / sum(T^xx + T^yy)."""
    e, p, v = con2prim(u, k)
    txx = u[1] * v[0] + p
    tyy = u[2] * v[1] + p
    return (txx - tyy).sum() / (txx + tyy).sum()
