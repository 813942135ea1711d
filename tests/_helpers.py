"""Shared test helpers: the state-scale normalised difference used for parity."""
import numpy as np


def state_scales(U, gamma):
    """Per-component scales: rho and E by their max norms, momenta by
    max|rho| * max(|v| + c_s) (the momentum scale), so that tiny momenta (a 1e-6 sound
    wave) do not turn round-off into large relative errors."""
    rho = U[0]
    v = U[1:4] / rho
    ug = U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    cs = np.sqrt(gamma * (gamma - 1.0) * np.maximum(ug, 1e-300) / rho)
    vmax = np.max(np.sqrt((v ** 2).sum(axis=0)) + cs)
    s = np.empty(5)
    s[0] = np.abs(rho).max()
    s[1:4] = np.abs(rho).max() * vmax
    s[4] = np.abs(U[4]).max()
    return s


def max_norm_diff(a, b, gamma):
    """max over components of max_cells |a - b| / scale_k."""
    s = state_scales(b, gamma)
    return max(float(np.abs(a[k] - b[k]).max() / s[k]) for k in range(5))


def l1_wave_error(U, U0):
    """Linear-wave L1 error: sqrt(sum_k (mean |U_k - U0_k|)^2)."""
    return float(np.sqrt(sum(np.mean(np.abs(U[k] - U0[k])) ** 2 for k in range(5))))
