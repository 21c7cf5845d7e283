"""FD-WENO of order 2r-1 (Sec. 1.2) derived symbolically from its definition,
for the tests of the kernels' reconstruction forms: each candidate is the
polynomial of degree r-1 whose cell averages over its stencil are the point
values, q_k its value at x_{j+1/2}, the linear weights make sum_k d_k q_k the
value of the polynomial of degree 2r-2 over the whole window, and
beta_k = sum_l int (d^l p_k / dxi^l)^2 over the centre cell."""
import sympy as sp

HALF = sp.Rational(1, 2)


def definition(r):
    xi = sp.symbols("xi")
    v = sp.symbols("v0:%d" % (2 * r - 1))
    qs, betas = [], []
    for k in range(r):
        c = sp.symbols("c0:%d" % r)
        p = sum(c[i] * xi ** i for i in range(r))
        # stencil k: window cells k .. k+r-1, centre cell r-1 at xi = 0
        eqs = [sp.Eq(sp.integrate(p, (xi, o - (r - 1) - HALF, o - (r - 1) + HALF)), v[o]) for o in range(k, k + r)]
        pk = sp.expand(p.subs(sp.solve(eqs, c)))
        qs.append(sp.expand(pk.subs(xi, HALF)))
        betas.append(sp.expand(sum(sp.integrate(sp.diff(pk, xi, l) ** 2, (xi, -HALF, HALF)) for l in range(1, r))))
    n = 2 * r - 1
    C = sp.symbols("C0:%d" % n)
    P = sum(C[i] * xi ** i for i in range(n))
    sol = sp.solve([sp.Eq(sp.integrate(P, (xi, o - (r - 1) - HALF, o - (r - 1) + HALF)), v[o]) for o in range(n)], C)
    big = sp.expand(P.subs(sol).subs(xi, HALF))
    dw = sp.symbols("w0:%d" % r)
    ex = sp.expand(sum(dw[k] * qs[k] for k in range(r)) - big)
    dsol = sp.solve([ex.coeff(x) for x in v], dw)
    return v, qs, betas, [dsol[w] for w in dw]
