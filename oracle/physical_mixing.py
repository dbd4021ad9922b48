"""Physical mixing matrix of App. B (TEST INFRASTRUCTURE ONLY).

Columns, in units of CMB intensity at reference frequency nu0 = 100 GHz:
  1. CMB: 1 at every frequency.
  2. synchrotron: c(nu) (nu/nu0)^kappa_s, kappa_s = -2.65.
  3. galactic dust: c(nu) B(nu)/B(nu0) (nu/nu0)^kappa_d, kappa_d = 1.5,
     B(nu) = nu / (exp(h nu / (k_B T1)) - 1).
  4. free-free: c(nu) (nu/nu0)^-2.14.
with the unit conversion c(nu) = (e^psi - 1)^2 / (psi^2 e^psi), psi = h nu / (k_B T1),
T1 = 18.1 K.  Reading: the conversion factor is the whole ratio (e^psi - 1)^2 over psi^2 e^psi
(the printed expression can be parenthesised two ways; this one reproduces the printed table).
"""

import numpy as np

H_PLANCK = 6.62607015e-34     # J s
K_BOLTZMANN = 1.380649e-23    # J / K
T1 = 18.1                     # K


def _psi(nu_ghz):
    return H_PLANCK * np.asarray(nu_ghz, np.float64) * 1e9 / (K_BOLTZMANN * T1)


def conversion(nu_ghz):
    p = _psi(nu_ghz)
    return np.expm1(p) ** 2 / (p * p * np.exp(p))


def _blackbody(nu_ghz):
    return np.asarray(nu_ghz, np.float64) / np.expm1(_psi(nu_ghz))


def physical_mixing(nu_ghz, nu0=100.0, kappa_s=-2.65, kappa_d=1.5, kappa_ff=-2.14):
    nu = np.asarray(nu_ghz, np.float64)
    c = conversion(nu)
    ratio = nu / nu0
    A = np.empty((nu.size, 4))
    A[:, 0] = 1.0
    A[:, 1] = c * ratio ** kappa_s
    A[:, 2] = c * _blackbody(nu) / _blackbody(nu0) * ratio ** kappa_d
    A[:, 3] = c * ratio ** kappa_ff
    return A
