"""One-dimensional bases and quadrature rules for the FP64 oracle.

TEST INFRASTRUCTURE: the oracle is a plain, slow, FP64 CPU restatement of the
discrete operator.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import it; the product path never does.

Section 3.2.1 of the paper defines the velocity element: Lagrange polynomials
of degree k on the tensor-product Gauss-Lobatto (GLL) nodes of [-1, 1]^3,
integrated with tensor-product Gauss quadrature "of order k" (read here as
q = k + 1 Gauss-Legendre points per direction).  Section 3.2.2 defines the
discontinuous pressure spaces P_{k-1} and Q_{k-2}; Section 6 fixes the Q_{k-2}
basis as Lagrange on the tensor Gauss nodes.  The P_{k-1} basis is not fixed by
the paper; products of Legendre polynomials are used (the discrete solution
does not depend on the basis).

Everything here is computed from its textbook definition: Legendre three-term
recurrence, Newton iteration for the roots, product formula for Lagrange
polynomials.
"""
import numpy as np


def legendre(n, x):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet).

    (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1};  P_n' from
    (x^2 - 1) P_n' = n (x P_n - P_{n-1}), with the endpoint limit
    P_n'(+-1) = (+-1)^{n-1} n (n+1) / 2.
    """
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for m in range(1, n):
        p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
    # p1 = P_n, p0 = P_{n-1}
    with np.errstate(divide="ignore", invalid="ignore"):
        dp = n * (x * p1 - p0) / (x * x - 1.0)
    end = np.isclose(np.abs(x), 1.0, rtol=0, atol=1e-15)
    dp = np.where(end, np.sign(x) ** (n - 1) * n * (n + 1) / 2.0, dp)
    return p1, dp


def gauss_legendre(q):
    """q-point Gauss-Legendre rule on [-1, 1]: roots of P_q by Newton."""
    i = np.arange(q)
    x = np.cos(np.pi * (i + 0.75) / (q + 0.5))  # standard initial guess
    for _ in range(100):
        p, dp = legendre(q, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(q, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_lobatto(n1):
    """n1-point Gauss-Lobatto-Legendre rule: +-1 and the roots of P_k'.

    k = n1 - 1.  Interior nodes by Newton on P_k' using the Legendre ODE
    (1 - x^2) P_k'' = 2 x P_k' - k (k+1) P_k.  Weights 2 / (k (k+1) P_k(x)^2).
    """
    k = n1 - 1
    if k < 1:
        raise ValueError("GLL rule needs at least 2 points")
    x = -np.cos(np.pi * np.arange(n1) / k)  # Chebyshev-Lobatto guess
    xi = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(k, xi)
        ddp = (2.0 * xi * dp - k * (k + 1) * p) / (1.0 - xi * xi)
        dx = dp / ddp
        xi = xi - dx
        if xi.size == 0 or np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], np.sort(xi), [1.0]])
    p, _ = legendre(k, x)
    w = 2.0 / (k * (k + 1) * p * p)
    return x, w


def lagrange(nodes, x):
    """Values ell_a(x_i) of the Lagrange polynomials on `nodes` (product formula).

    Returns an array of shape (len(x), len(nodes)).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    L = np.ones((x.size, n))
    for a in range(n):
        for m in range(n):
            if m != a:
                L[:, a] *= (x - nodes[m]) / (nodes[a] - nodes[m])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives ell_a'(x_i): sum over m != a of the product with factor m dropped."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    dL = np.zeros((x.size, n))
    for a in range(n):
        for m in range(n):
            if m == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[m]))
            for l in range(n):
                if l != a and l != m:
                    term *= (x - nodes[l]) / (nodes[a] - nodes[l])
            dL[:, a] += term
    return dL


def pressure_modes(k, space):
    """Exponent / index triples (a, b, c) of the discontinuous pressure basis.

    space 'P': P_{k-1}, Legendre products L_a(xi) L_b(eta) L_c(zeta) with
               a + b + c <= k - 1; order: c outermost, then b, then a.
    space 'Q': Q_{k-2}, Lagrange on (k-1)^3 tensor Gauss points;
               index a + (k-1) (b + (k-1) c).
    """
    modes = []
    if space == "P":
        for c in range(k):
            for b in range(k - c):
                for a in range(k - b - c):
                    modes.append((a, b, c))
    elif space == "Q":
        m = k - 1
        for c in range(m):
            for b in range(m):
                for a in range(m):
                    modes.append((a, b, c))
    else:
        raise ValueError(space)
    return modes


def pressure_1d_tables(k, space, x):
    """1-D factor tables T[i, a] of the pressure basis evaluated at points x."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if space == "P":
        T = np.zeros((x.size, k))
        for a in range(k):
            T[:, a] = legendre(a, x)[0]
        return T
    if space == "Q":
        g, _ = gauss_legendre(k - 1)
        return lagrange(g, x)
    raise ValueError(space)


def n_pressure(k, space):
    return len(pressure_modes(k, space))
