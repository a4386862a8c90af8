"""Shared test helpers: error norms for parity against the oracle, node
matching by coordinates, and physically scaled random states."""
import numpy as np

from paper_1511_01561_gb300 import inputs as I


def rel_errors(a: np.ndarray, b: np.ndarray, floors) -> np.ndarray:
    """Per-variable relative errors [L2, Linf] of a against the reference b.

    The denominator is the reference norm, floored at floors[v] (a natural
    scale of that variable in the run) so that variables that are zero or
    tiny in the reference are held to an absolute bar tol * floor instead."""
    out = np.zeros((a.shape[0], 2))
    for v in range(a.shape[0]):
        d = a[v] - b[v]
        n2 = max(np.sqrt(np.mean(b[v] ** 2)), floors[v])
        ni = max(np.abs(b[v]).max(), floors[v])
        out[v] = (np.sqrt(np.mean(d**2)) / n2, np.abs(d).max() / ni)
    return out


def rhs_floors(R_ref: np.ndarray, rho_max: float, dx_min: float, umax: float = 1.0) -> np.ndarray:
    """Natural scales of the tendencies: rho |u| / dx for rho' and Theta'
    (|u| floored at 1 m/s, times a 300 K theta for Theta'), and the largest
    momentum tendency for the momentum components."""
    u = max(umax, 1.0)
    s_rho = rho_max * u / dx_min
    s_U = max(np.abs(R_ref[1:4]).max(), 1e-300)
    return np.array([1e-3 * s_rho, 1e-3 * s_U, 1e-3 * s_U, 1e-3 * s_U, 1e-3 * 300.0 * s_rho])


def state_floors(q_ref: np.ndarray, rho_max: float, theta0: float = 300.0) -> np.ndarray:
    s_U = max(np.abs(q_ref[1:4]).max(), 1e-3 * rho_max)
    return np.array([1e-3 * rho_max, s_U, s_U, s_U, 1e-3 * rho_max * theta0])


def match_nodes(xyz_a: np.ndarray, xyz_b: np.ndarray, tol: float) -> np.ndarray:
    """perm with xyz_a[:, i] == xyz_b[:, perm[i]] (within tol)."""
    from scipy.spatial import cKDTree

    d, perm = cKDTree(xyz_b.T).query(xyz_a.T)
    assert d.max() < tol, d.max()
    assert len(np.unique(perm)) == len(perm)
    return perm


def scaled_random_state(Ng: int, rho0: np.ndarray, th0: np.ndarray, seed: int, rel=0.01, u=5.0) -> np.ndarray:
    """Random nodal perturbations relative to the reference state."""
    q = I.random_perturbation(Ng, seed, rho=1.0, U=1.0, Theta=1.0)
    q[0] *= rel * rho0
    q[1:4] *= u * rho0
    q[4] *= rel * th0
    return q
