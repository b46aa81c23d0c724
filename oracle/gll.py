"""Gauss-Lobatto-Legendre (GLL) rule of order p: nodes, weights, derivative matrix.

Oracle (test infrastructure only).  The paper uses C0 nodal Lagrange elements
of degree p (Sec. 3.1, definition of the space V_D); the hexahedral elements use the
tensor-product GLL nodal basis, whose 1D ingredients are defined here from
their textbook definitions:

  nodes   xi_0 = -1, xi_p = +1 and the p-1 roots of P_p'(x)
  weights w_i = 2 / (p (p+1) P_p(xi_i)^2)
  D_ij    = l_j'(xi_i), the derivative of the j-th Lagrange cardinal
            polynomial on the nodes, evaluated at node i.

The derivative matrix is built here by differentiating the Lagrange cardinal
polynomials directly (product rule on prod_{m != j} (x - xi_m)/(xi_j - xi_m)),
not from the closed form in terms of P_p(xi_i), so that the closed form used
elsewhere can be checked against it.
"""
import numpy as np


def legendre(p, x):
    """P_p(x) and P_p'(x) by the three-term recurrence (works on long double)."""
    x = np.asarray(x)
    one = np.ones_like(x)
    if p == 0:
        return one, 0 * x
    pm1, pc = one, x.copy()
    for k in range(1, p):
        pm1, pc = pc, ((2 * k + 1) * x * pc - k * pm1) / (k + 1)
    # derivative: (1 - x^2) P_p' = p (P_{p-1} - x P_p); at |x| = 1 use p(p+1)/2 * x^(p+1)
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = p * (pm1 - x * pc) / (1 - x * x)
    end = np.isclose(np.abs(x), 1)
    dp = np.where(end, 0.5 * p * (p + 1) * np.sign(x) ** (p + 1), dp)
    return pc, dp


def nodes(p):
    """GLL nodes in ascending order (float64), computed by Newton on (1-x^2) P_p'(x)
    in extended precision."""
    if p < 1:
        raise ValueError("p >= 1")
    ld = np.longdouble
    x = -np.cos(np.pi * np.arange(p + 1, dtype=ld) / ld(p))  # Chebyshev-Lobatto start
    for _ in range(100):
        pc, dp = legendre(p, x)
        # q(x) = (1-x^2) P_p'(x) = p (P_{p-1}(x) - x P_p(x));  q'(x) = -p (p+1) P_p(x)
        pm1 = legendre(p - 1, x)[0] if p >= 1 else 0 * x
        q = p * (pm1 - x * pc)
        dq = -p * (p + 1) * pc
        dx = np.zeros_like(x)
        dx[1:-1] = q[1:-1] / dq[1:-1]
        x = x - dx
        if np.max(np.abs(dx)) < ld(1e-30):
            break
    x[0], x[-1] = -1, 1
    return np.array(x, dtype=np.float64), x


def weights(p):
    _, xl = nodes(p)
    pc, _ = legendre(p, xl)
    w = 2 / (p * (p + 1) * pc * pc)
    return np.array(w, dtype=np.float64)


def lagrange_derivative_matrix(xl):
    """D_ij = l_j'(x_i) for the Lagrange cardinal polynomials on nodes xl, by the
    product rule (computed in the nodes' precision)."""
    n = len(xl)
    D = np.zeros((n, n), dtype=xl.dtype)
    for j in range(n):
        denom = np.prod([xl[j] - xl[m] for m in range(n) if m != j])
        for i in range(n):
            # d/dx prod_{m != j} (x - x_m) at x_i = sum_{l != j} prod_{m != j, l} (x_i - x_m)
            s = 0
            for l in range(n):
                if l == j:
                    continue
                term = 1
                for m in range(n):
                    if m != j and m != l:
                        term = term * (xl[i] - xl[m])
                s = s + term
            D[i, j] = s / denom
    return D


def derivative_matrix(p):
    _, xl = nodes(p)
    return np.array(lagrange_derivative_matrix(xl), dtype=np.float64)


def lagrange_eval(xl, x):
    """Values L[q, j] = l_j(x_q) of the cardinal polynomials on nodes xl at points x."""
    xl = np.asarray(xl, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = len(xl)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - xl[m]) / (xl[j] - xl[m])
    return L


class Rule:
    """Bundle of the order-p GLL data used by the rest of the oracle."""

    def __init__(self, p):
        self.p = p
        self.n = p + 1
        self.xi = nodes(p)[0]
        self.w = weights(p)
        self.D = derivative_matrix(p)
