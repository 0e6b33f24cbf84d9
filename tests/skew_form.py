"""Exact-rational PW tendencies from the scheme's definition (test helper).

The Piacsek-Williams scheme cited in Sec. 2.1 is the skew-symmetric
discretisation: the tendency of an advected quantity phi in a cell is the
average of the discrete *flux* form and the discrete *advective* form,

    flux = -[ M+ (phi_c + phi_+)/2 - M- (phi_c + phi_-)/2 ] / (rho_c D_c)
    adv  = -[ M+ (phi_+ - phi_c)   + M- (phi_c - phi_-)   ] / (2 rho_c D_c)
    PW   = (flux + adv) / 2,

summed over the three directions, where M+- = rho_face * (face-normal velocity)
are the mass fluxes through the cell's two faces in that direction, phi_+- the
neighbouring values and D_c the cell width.  On the Arakawa-C grid of Listing 1
(u at x-faces, v at y-faces, w at the top of each cell) the face velocities are
two-point averages of the staggered winds.  At the model lid the flux through
the top face of the topmost u/v cell is absent (Listing 1's else branch).

This module never looks at Listing 1's expressions or at the oracle: it builds
each tendency from cells, faces and mass fluxes with Python ``Fraction``s, so
the result is exact and independent of evaluation order.  Arrays are indexed
[i][j][k] (0-based k), periodic in i and j.
"""
from __future__ import annotations

from fractions import Fraction as Fr


def _fr(a):
    return [[[Fr(float(x)) for x in col] for col in plane] for plane in a]


def _pw(phi_c, phi_p, phi_m, m_p, m_m, mass):
    flux = -(m_p * (phi_c + phi_p) / 2 - m_m * (phi_c + phi_m) / 2) / mass
    adv = -(m_p * (phi_p - phi_c) + m_m * (phi_c - phi_m)) / (2 * mass)
    return (flux + adv) / 2


def tendencies(u, v, w, dx, dy, z, zn, rho, rhon):
    """Exact (su, sv, sw) as nested lists of Fractions."""
    U, V, W = _fr(u), _fr(v), _fr(w)
    nx, ny, nz = len(U), len(U[0]), len(U[0][0])
    dx, dy = Fr(float(dx)), Fr(float(dy))
    z = [Fr(float(a)) for a in z]
    zn = [Fr(float(a)) for a in zn]
    rho = [Fr(float(a)) for a in rho]
    rhon = [Fr(float(a)) for a in rhon]
    half = Fr(1, 2)

    def zero():
        return [[[Fr(0)] * nz for _ in range(ny)] for _ in range(nx)]

    su, sv, sw = zero(), zero(), zero()
    for i in range(nx):
        ip, im = (i + 1) % nx, (i - 1) % nx
        for j in range(ny):
            jp, jm = (j + 1) % ny, (j - 1) % ny
            for k in range(1, nz):
                top = k == nz - 1
                dzk = z[k] - z[k - 1]
                # ---- u cell: x = i+1/2, y = j, level zn(k) ----
                c = U[i][j][k]
                t = _pw(c, U[ip][j][k], U[im][j][k],
                        rhon[k] * (U[i][j][k] + U[ip][j][k]) * half,
                        rhon[k] * (U[im][j][k] + U[i][j][k]) * half, rhon[k] * dx)
                t += _pw(c, U[i][jp][k], U[i][jm][k],
                         rhon[k] * (V[i][j][k] + V[ip][j][k]) * half,
                         rhon[k] * (V[i][jm][k] + V[ip][jm][k]) * half, rhon[k] * dy)
                m_top = Fr(0) if top else rho[k] * (W[i][j][k] + W[ip][j][k]) * half
                m_bot = rho[k - 1] * (W[i][j][k - 1] + W[ip][j][k - 1]) * half
                up = Fr(0) if top else U[i][j][k + 1]
                t += _pw(c, up, U[i][j][k - 1], m_top, m_bot, rhon[k] * dzk)
                su[i][j][k] = t
                # ---- v cell: x = i, y = j+1/2, level zn(k) ----
                c = V[i][j][k]
                t = _pw(c, V[ip][j][k], V[im][j][k],
                        rhon[k] * (U[i][j][k] + U[i][jp][k]) * half,
                        rhon[k] * (U[im][j][k] + U[im][jp][k]) * half, rhon[k] * dx)
                t += _pw(c, V[i][jp][k], V[i][jm][k],
                         rhon[k] * (V[i][j][k] + V[i][jp][k]) * half,
                         rhon[k] * (V[i][jm][k] + V[i][j][k]) * half, rhon[k] * dy)
                m_top = Fr(0) if top else rho[k] * (W[i][j][k] + W[i][jp][k]) * half
                m_bot = rho[k - 1] * (W[i][j][k - 1] + W[i][jp][k - 1]) * half
                up = Fr(0) if top else V[i][j][k + 1]
                t += _pw(c, up, V[i][j][k - 1], m_top, m_bot, rhon[k] * dzk)
                sv[i][j][k] = t
                # ---- w cell: x = i, y = j, level z(k); interior levels only ----
                if top:
                    continue
                c = W[i][j][k]
                t = _pw(c, W[ip][j][k], W[im][j][k],
                        rho[k] * (U[i][j][k] + U[i][j][k + 1]) * half,
                        rho[k] * (U[im][j][k] + U[im][j][k + 1]) * half, rho[k] * dx)
                t += _pw(c, W[i][jp][k], W[i][jm][k],
                         rho[k] * (V[i][j][k] + V[i][j][k + 1]) * half,
                         rho[k] * (V[i][jm][k] + V[i][jm][k + 1]) * half, rho[k] * dy)
                t += _pw(c, W[i][j][k + 1], W[i][j][k - 1],
                         rhon[k + 1] * (W[i][j][k] + W[i][j][k + 1]) * half,
                         rhon[k] * (W[i][j][k - 1] + W[i][j][k]) * half,
                         rho[k] * (zn[k + 1] - zn[k]))
                sw[i][j][k] = t
    return su, sv, sw
