"""Oracle: coil impedance change Delta Z and the signal modes.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. impedkl writes Delta Z_kl as a volume integral over Omega_d of the
contrast in the curl-curl and conductivity terms between the configuration
with the defect and the "vacuum" one.  As printed its constants are not
dimensionally consistent, so the reading is the exact discrete reciprocity
identity.  With M_0 u_l^0 = b_l, M_d u_l^d = b_l (symmetric M) and the coil
EMF impedance Z_kl = -(i omega / (I_k I_l)) b_k^T u_l (bilinear, no conjugate):

    Delta Z_kl = Z_kl^d - Z_kl^0 = (i omega / (I_k I_l)) u_k^0^T (M_d - M_0) u_l^d,

where M_d - M_0 vanishes outside Omega_d.  The signal modes of Eq. impedmod
are kept as printed: Z_FA = (i/2)(dZ_11 + dZ_12), Z_F3 = (i/2)(dZ_11 - dZ_22).
"""
from __future__ import annotations

import numpy as np


def z_emf(b_k, u_l, I_k, I_l, omega):
    """Coil EMF impedance Z_kl = -(i omega / (I_k I_l)) b_k^T u_l (bilinear; module notes)."""
    return -(1j * omega / (I_k * I_l)) * (np.asarray(b_k) @ np.asarray(u_l))


def delta_z_reciprocity(M0, Md, u0_k, ud_l, I_k, I_l, omega):
    """Delta Z_kl by reciprocity (Eq. impedkl read as the discrete identity of the module notes)."""
    return (1j * omega / (I_k * I_l)) * (np.asarray(u0_k) @ ((Md - M0) @ np.asarray(ud_l)))


def delta_z_matrix(M0, Md, u0, ud, currents, omega):
    """2x2 Delta Z from the four solutions u0[k], ud[l] (reciprocity form)."""
    dz = np.zeros((2, 2), dtype=np.complex128)
    for k in range(2):
        for l in range(2):
            dz[k, l] = delta_z_reciprocity(M0, Md, u0[k], ud[l], currents[k], currents[l], omega)
    return dz


def delta_z_emf_matrix(b, u0, ud, currents, omega):
    """2x2 Delta Z as the difference of coil EMF impedances."""
    dz = np.zeros((2, 2), dtype=np.complex128)
    for k in range(2):
        for l in range(2):
            dz[k, l] = (z_emf(b[k], ud[l], currents[k], currents[l], omega)
                        - z_emf(b[k], u0[l], currents[k], currents[l], omega))
    return dz


def signal_modes(dz):
    """(Z_FA, Z_F3) of Eq. impedmod, as printed."""
    return 0.5j * (dz[0, 0] + dz[0, 1]), 0.5j * (dz[0, 0] - dz[1, 1])
