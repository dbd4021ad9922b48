"""The physical mixing matrix and channel noise weights printed in App. B (data, as printed).

Rows are the nine Planck channels 30, 44, 70, 100, 143, 217, 353, 545, 857 GHz; columns the
sources CMB, synchrotron, galactic dust, free-free.  T is the diagonal of the channel weights in
C = T kron N.  The values are copied as the paper prints them (three decimals for A).
"""

import numpy as np

PLANCK_A_PRINTED = np.array([
    [1.000, 24.314, 0.181, 13.158],
    [1.000, 8.817, 0.315, 5.801],
    [1.000, 2.581, 0.612, 2.151],
    [1.000, 1.006, 1.006, 1.006],
    [1.000, 0.392, 1.630, 0.471],
    [1.000, 0.132, 2.783, 0.196],
    [1.000, 0.038, 4.931, 0.072],
    [1.000, 0.013, 7.704, 0.032],
    [1.000, 0.005, 11.337, 0.015],
])

PLANCK_T_PRINTED = np.array([629881.6, 694444.4, 783146.7, 12755102.0, 30864197.5,
                             30864197.5, 30864197.5, 30864197.5, 30864197.5])
