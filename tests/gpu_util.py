"""Helpers shared by the GPU parity tests (no method arithmetic)."""
import numpy as np

EPS64 = 2.0 ** -52


def flux_scale(U, g, sigma_min=0.5):
    """Magnitude of the fluxes entering R (for a relative residual bound)."""
    H = np.abs(U[0]).max()
    Q = np.abs(U[1]).max()
    return max(Q, Q * Q / np.abs(U[0]).min() + 0.5 * g * H * H / sigma_min, 1.0)


def jac_tol(Jref, scale_R, eps):
    """1e-12 relative to the block scale plus the FD cancellation allowance."""
    return 1e-12 * np.abs(Jref).max() + 8.0 * EPS64 * scale_R / eps
