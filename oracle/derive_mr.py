"""Symbolic derivation of the multi-reflection (MR) coefficients of Eq. (15).

TEST INFRASTRUCTURE ONLY (with the rest of oracle/): it documents and
re-derives reading R17 of lbm_oracle.c; nothing in the library imports it.
Needs sympy.

The paper gives the form of the MR closure, Eq. (15), and cites its
coefficients.  They follow from the requirement MR is built for, second-order
no-slip with TRT:

1. Along one link (coordinate s: boundary node x at s = 0, x - c_q at s = -1,
   wall at s = delta) take equilibrium parts quadratic in the velocity and
   linear in the density/pressure:
       e-(s) = a0 + a1 (s - d) + a2 (s - d)^2 / 2,   e+(s) = b0 + b1 (s - d).
2. Solve the steady TRT recurrence of the pull scheme exactly for the
   non-equilibrium parts g+- of the post-collision populations:
       n_q(s) = e_q(s-1) + g_q(s-1) - e_q(s),  n_qbar(s) = e_qbar(s+1) + g_qbar(s+1) - e_qbar(s),
       g+- = (1 - lambda+-) n+-   (lambda+- the relaxation rates, magnitudes).
3. Require Eq. (15), with the correction f^pc = k n-_q(x) (the odd part of the
   pre-collision non-equilibrium at x), to return the population the
   continued lattice would send from x + c_q, for every a0 (wall velocity
   term), b0, a1, a2 and b1.
4. With the pairing of Eq. (14) (kappa_1 = 1, kappabar_-1 = -kappa_0,
   kappabar_-2 = -kappa_-1) the solution is unique.

`derive()` returns the coefficients as sympy expressions of delta and
Lambda_- = 1/lambda_- - 1/2.
"""
from __future__ import annotations


def derive():
    import sympy as sp

    s, d = sp.symbols("s delta")
    lp, lm = sp.symbols("lambda_p lambda_m", positive=True)
    Lp, Lm = sp.symbols("Lambda_p Lambda_m", positive=True)
    a0, a1, a2, b0, b1 = sp.symbols("a0 a1 a2 b0 b1")
    e_plus = b0 + b1 * (s - d)
    e_minus = a0 + a1 * (s - d) + a2 * (s - d) ** 2 / 2

    # step 2: g+- as polynomials of degree <= 2 solving the recurrence exactly
    gp_c, gm_c = sp.symbols("gp0:3"), sp.symbols("gm0:3")
    gp = sum(c * s ** i for i, c in enumerate(gp_c))
    gm = sum(c * s ** i for i, c in enumerate(gm_c))
    e_q, e_qb = e_plus + e_minus, e_plus - e_minus
    g_q, g_qb = gp + gm, gp - gm
    n_q = e_q.subs(s, s - 1) + g_q.subs(s, s - 1) - e_q
    n_qb = e_qb.subs(s, s + 1) + g_qb.subs(s, s + 1) - e_qb
    eqs = (sp.Poly(sp.expand(gp - (1 - lp) * (n_q + n_qb) / 2), s).all_coeffs() +
           sp.Poly(sp.expand(gm - (1 - lm) * (n_q - n_qb) / 2), s).all_coeffs())
    sol = sp.solve(eqs, gp_c + gm_c, dict=True)[0]
    gp, gm = gp.subs(sol), gm.subs(sol)
    rates = {lp: 1 / (Lp + sp.Rational(1, 2)), lm: 1 / (Lm + sp.Rational(1, 2))}

    # step 3: the closure at s = 0 against the continued lattice at s = 1
    ft_q = lambda x: (e_q + gp + gm).subs(s, x)
    ft_qb = lambda x: (e_qb + gp - gm).subs(s, x)
    n_minus = (gm / (1 - lm)).subs(s, 0)  # odd pre-collision non-equilibrium at x
    k0, km1, alpha, kpc = sp.symbols("kappa_0 kappa_m1 alpha k_pc")
    closure = (ft_q(0) + k0 * ft_q(-1) + km1 * ft_q(-2) - k0 * ft_qb(0) - km1 * ft_qb(-1)
               - alpha * a0 + kpc * n_minus)
    residual = sp.expand((closure - ft_qb(1)).subs(rates))
    conds = [residual.coeff(v) for v in (a0, a1, a2, b0, b1)]
    # the conditions are linear in the unknowns; b0's holds by the pairing
    unknowns = [alpha, k0, km1, kpc]
    # (a2's condition plus Lambda_+ times b1's is free of the relaxation rates)
    system = [conds[0], conds[1], sp.expand(conds[2] + Lp * conds[4]), conds[4]]
    found = sp.solve(system, unknowns, dict=True)
    if len(found) != 1:
        raise RuntimeError("the MR conditions do not have a unique solution")
    sol = {u: sp.factor(sp.cancel(found[0][u])) for u in unknowns}
    # every condition, b0's included, holds with the solution
    for c in conds:
        assert sp.cancel(sp.together(c.subs(sol))) == 0
    return {u.name: v for u, v in sol.items()}


if __name__ == "__main__":
    for name, expr in derive().items():
        print(f"{name} = {expr}")
