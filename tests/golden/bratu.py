"""Independent reference for the Bratu problem Lap u + lam e^u = 0 on the unit square,
u = 0 on the boundary (Sec. 3.3, Bratu row of the nonlinear-results table; no closed
form): a second-order finite-difference Newton solve (5-point Laplacian, sparse direct
solves to machine precision) on grids h and h/2, one Richardson step, interpolated
cubically.  Shares nothing with the oracle or the GPU path."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.interpolate import RegularGridInterpolator


def bratu_fd(n, lam=1.0):
    """(n+1) x (n+1) grid values of the finite-difference solution."""
    h = 1.0 / n
    m = n - 1
    I = sp.identity(m)
    T = sp.diags([np.ones(m - 1), -2 * np.ones(m), np.ones(m - 1)], [-1, 0, 1])
    L = (sp.kron(I, T) + sp.kron(T, I)) / h ** 2
    u = np.zeros(m * m)
    for _ in range(30):
        F = L @ u + lam * np.exp(u)
        J = L + sp.diags(lam * np.exp(u))
        du = spla.spsolve(J.tocsc(), -F)
        u += du
        if np.abs(du).max() < 1e-14:
            break
    full = np.zeros((n + 1, n + 1))
    full[1:-1, 1:-1] = u.reshape(m, m)
    return full


def bratu_reference(n=128, lam=1.0):
    """Callable u(x) for x of shape (k, 2): Richardson extrapolation of grids n, 2n."""
    coarse = bratu_fd(n, lam)
    fine = bratu_fd(2 * n, lam)
    rich = (4 * fine[::2, ::2] - coarse) / 3
    g = np.linspace(0, 1, n + 1)
    return RegularGridInterpolator((g, g), rich, method="cubic")
