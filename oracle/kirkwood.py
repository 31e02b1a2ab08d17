"""Analytic solution of the linear PB equation for a spherical cavity.

TEST INFRASTRUCTURE ONLY (part of the oracle).

The paper validates against Kirkwood's spherical-harmonic expansion (Sec. 3,
"analytical solutions ... closed form (for centered charge) and ...
spherical harmonics (for multiple eccentric charges)") without printing it.
It is derived here from the model equations eq1, eq2 (linearised), jump and
radiation for a sphere of radius a centred at the origin, charges q_k at
x_k with b_k = |x_k| < a:

  inside   phi1 = sum_k q_k / (eps1 |x - x_k|) + sum_k q_k sum_n B_n r^n b_k^n P_n(cos g_k)
  outside  phi2 = sum_n C_n k_n(kappa r) P_n        (k_n: modified spherical Bessel, 2nd kind)

Matching phi and eps dphi/dr at r = a for each n, with g_n = kappa k_n'(kappa a)/k_n(kappa a):

  B_n = [eps2 g_n/(eps1 a^(n+1)) + (n+1)/a^(n+2)] / (n eps1 a^(n-1) - eps2 g_n a^n).

Potentials here are "Gaussian" (q/(eps r)); the solver's G-units divide by
4 pi. g_n uses the ratio rho_n = k_{n-1}/k_n, which obeys
rho_{n+1} = 1/(rho_n + (2n+1)/x), rho_0 = 1 (k_{-1} = k_0), and
k_n'/k_n = -rho_n - (n+1)/x. B_n is carried as the dimensionless
Bt_n = B_n a^(2n+1) to avoid overflow.
"""
from __future__ import annotations

import numpy as np

C_KCAL = 332.0716  # kcal A / (mol e^2)


def bessel_k_ratio(nmax: int, x: float) -> np.ndarray:
    """rho_n = k_{n-1}(x)/k_n(x) for n = 0..nmax (forward recurrence, stable)."""
    rho = np.empty(nmax + 1)
    rho[0] = 1.0
    for n in range(nmax):
        rho[n + 1] = 1.0 / (rho[n] + (2.0 * n + 1.0) / x)
    return rho


def reaction_coeffs(nmax: int, a: float, eps1: float, eps2: float, kappa: float) -> np.ndarray:
    """Bt_n = B_n a^(2n+1), n = 0..nmax."""
    n = np.arange(nmax + 1, dtype=np.float64)
    if kappa > 0.0:
        rho = bessel_k_ratio(nmax, kappa * a)
        ga = -kappa * a * rho - (n + 1.0)  # g_n * a
    else:
        ga = -(n + 1.0)
    num = eps2 * ga / eps1 + (n + 1.0)
    den = n * eps1 - eps2 * ga
    return num / den


def _legendre_upto(nmax: int, c: np.ndarray) -> np.ndarray:
    P = np.empty((nmax + 1,) + c.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = c
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * c * P[n] - n * P[n - 1]) / (n + 1)
    return P


def _nterms(ratio: float, tol: float = 1e-17) -> int:
    if ratio <= 0.0:
        return 1
    # terms fall like ratio^n (times a slowly varying factor)
    n = int(np.ceil(np.log(tol) / np.log(ratio))) + 10
    return max(4, min(n, 4000))


def surface_potential(points: np.ndarray, charges: np.ndarray, a: float, eps1: float, eps2: float,
                      kappa: float, gunits: bool = True):
    """phi and dphi/dnu (inside limit, outward normal) at points on |x| = a.

    Returns G-units (divided by 4 pi) unless gunits is False.
    """
    P = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    Q = np.asarray(charges, dtype=np.float64).reshape(-1, 4)
    r = np.linalg.norm(P, axis=1)
    xhat = P / r[:, None]
    bmax = float(np.max(np.linalg.norm(Q[:, :3], axis=1))) if Q.shape[0] else 0.0
    nmax = _nterms(bmax / a)
    Bt = reaction_coeffs(nmax, a, eps1, eps2, kappa)
    phi = np.zeros(P.shape[0])
    dphi = np.zeros(P.shape[0])
    n = np.arange(nmax + 1, dtype=np.float64)
    for k in range(Q.shape[0]):
        xk, q = Q[k, :3], Q[k, 3]
        d = P - xk
        dist = np.linalg.norm(d, axis=1)
        phi += q / (eps1 * dist)
        dphi += -q * np.einsum("ij,ij->i", d, xhat) / (eps1 * dist**3)
        b = float(np.linalg.norm(xk))
        if b == 0.0:
            cosg = np.ones(P.shape[0])
        else:
            cosg = xhat @ (xk / b)
        Pn = _legendre_upto(nmax, cosg)  # [n, npts]
        # B_n r^n b^n = Bt_n / a * (r b / a^2)^n, evaluated at r = a
        t = (b / a) ** n  # (a b / a^2)^n
        phi += q * np.einsum("n,np->p", Bt / a * t, Pn)
        # d/dr (B_n r^n b^n) at r=a = n B_n a^(n-1) b^n = n Bt_n / a^2 (b/a)^n
        dphi += q * np.einsum("n,np->p", n * Bt / a**2 * t, Pn)
    if gunits:
        phi /= 4.0 * np.pi
        dphi /= 4.0 * np.pi
    return phi, dphi


def reaction_potential_at(points: np.ndarray, charges: np.ndarray, a: float, eps1: float, eps2: float,
                          kappa: float) -> np.ndarray:
    """Gaussian-unit reaction potential psi(x) inside the sphere."""
    P = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    Q = np.asarray(charges, dtype=np.float64).reshape(-1, 4)
    rp = np.linalg.norm(P, axis=1)
    bq = np.linalg.norm(Q[:, :3], axis=1)
    ratio = float(rp.max() * bq.max() / a**2) if Q.shape[0] else 0.0
    nmax = _nterms(ratio)
    Bt = reaction_coeffs(nmax, a, eps1, eps2, kappa)
    n = np.arange(nmax + 1, dtype=np.float64)
    psi = np.zeros(P.shape[0])
    for k in range(Q.shape[0]):
        xk, q, b = Q[k, :3], Q[k, 3], bq[k]
        denom = rp * b
        cosg = np.where(denom > 0, (P @ xk) / np.where(denom > 0, denom, 1.0), 1.0)
        Pn = _legendre_upto(nmax, cosg)
        t = (rp[None, :] * b / a**2) ** n[:, None]
        psi += q * np.einsum("n,np->p", Bt / a, t * Pn)
    return psi


def solvation_energy(charges: np.ndarray, a: float, eps1: float, eps2: float, kappa: float) -> float:
    """E_sol = (1/2) C sum_k q_k psi(x_k), kcal/mol."""
    Q = np.asarray(charges, dtype=np.float64).reshape(-1, 4)
    psi = reaction_potential_at(Q[:, :3], Q, a, eps1, eps2, kappa)
    return float(0.5 * C_KCAL * np.sum(Q[:, 3] * psi))


def born_energy(q: float, a: float, eps1: float, eps2: float, kappa: float = 0.0) -> float:
    """Closed form for one centred charge (Debye-Hueckel-Born), kcal/mol."""
    return 0.5 * C_KCAL * q * q * (1.0 / (eps2 * a * (1.0 + kappa * a)) - 1.0 / (eps1 * a))
