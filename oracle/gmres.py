"""Approximate correction solves by GMRES (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy.

Sec. 6.1 allows the correction system (I - phi D) x = S u of the coarse
operator to be solved directly or approximately with a few GMRES iterations;
Sec. 6.3 uses GMRES on every level of the multilevel tests and stops it once
the l2 norm of the relative residual has fallen by two orders of magnitude,
or after 10 (ERK1+U1) / 20 (ERK3+U3, ERK5+U5) iterations.  Readings where
the paper is silent: zero initial guess (the residual is relative to ||b||),
no restart inside the iteration cap, no preconditioner.

GMRES, as defined by Saad and Schultz (1986): the k-th iterate x_k minimises
||b - A x|| over the Krylov space K_k(A, b) = span{b, A b, .., A^{k-1} b}.
Here the space is built by the Arnoldi process with modified Gram-Schmidt,
A V_k = V_{k+1} Hbar_k, and y_k = argmin ||beta e_1 - Hbar_k y|| is taken from
numpy's least-squares routine at every k; x_k = V_k y_k.

Function       definition                                     parity pin
-------------  ---------------------------------------------  ------------------------------------
gmres          k-th iterate of GMRES with the stop rule above  Krylov minimiser from an explicit
                                                               Krylov basis (QR of [b, Ab, ..]);
                                                               exact solve once k reaches the degree
                                                               of the minimal polynomial; residual
                                                               estimate == ||b - A x_k||
"""
import numpy as np


def gmres(apply_A, b, rtol=1e-2, maxit=20):
    """Approximate solution of A x = b (1-D b) by GMRES from x_0 = 0.

    Stops at the first k >= 1 with ||b - A x_k|| <= rtol ||b||, or at
    k = maxit, or when the Krylov space stops growing (h_{k+1,k} == 0: x_k is
    then exact).  Returns (x_k, k, residual norms ||b - A x_j||, j = 0..k,
    from the least-squares problems).
    """
    b = np.asarray(b, dtype=np.float64)
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros_like(b), 0, [0.0]
    n = b.shape[0]
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    V[0] = b / beta
    res = [beta]
    y = np.zeros(0)
    k = 0
    for j in range(maxit):
        w = apply_A(V[j])
        for i in range(j + 1):                      # modified Gram-Schmidt
            H[i, j] = float(np.dot(w, V[i]))
            w = w - H[i, j] * V[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y, _, _, _ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
        res.append(float(np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)))
        k = j + 1
        if res[-1] <= rtol * beta or H[j + 1, j] == 0.0:
            break
        V[j + 1] = w / H[j + 1, j]
    x = V[:k].T @ y
    return x, k, res


def gmres_rows(apply_A, B, rtol=1e-2, maxit=20):
    """gmres applied to every row of B (one independent system per row).
    Returns (X, iteration counts per row)."""
    B = np.atleast_2d(np.asarray(B, dtype=np.float64))
    X = np.empty_like(B)
    its = []
    for r in range(B.shape[0]):
        X[r], k, _ = gmres(apply_A, B[r], rtol, maxit)
        its.append(k)
    return X, its


def default_maxit(p):
    """Iteration cap of Sec. 6.3: 10 for first-order schemes, 20 for third
    and fifth order."""
    return 10 if p == 1 else 20
