"""Tolerance of the batched GPU parity tests (derivation and CPU pin: test_batched_tolerance.py).

A nest of depth L multiplies a perturbation of X by (L+1) r^L along an eigenvalue r of its
residual, so rounding made in nest j reaches X_nests amplified by prod_{i>j} (L+1) rho_i^L with
rho_i = rho_0^((L+1)^i) (R_i = R_0^((L+1)^i), Appendix 2); one product of order U carries about
sqrt(U) u32. Bound: ||X - X_oracle||_F / ||X_oracle||_F <= C_BATCHED * G * sqrt(U) * u32.
"""
import numpy as np

U32 = 2.0 ** -24
C_BATCHED = 2.0


def amplification(a, depth, nests, damping):
    """G of the module docstring for the damped Jacobi start X_0 = diag(A)^-1 / (1 + damping U)."""
    u = a.shape[0]
    x0 = np.diag(1.0 / np.diag(a)) / (1.0 + damping * u)
    rho0 = float(np.max(np.abs(np.linalg.eigvals(np.eye(u) - a @ x0))))
    rho = [rho0 ** ((depth + 1) ** i) for i in range(nests)]
    g, prod = 0.0, 1.0
    for j in range(nests - 1, -1, -1):   # rounding of nest j, amplified by the nests after it
        g += prod
        prod *= (depth + 1) * rho[j] ** depth
    return g
