"""Physical constants (CODATA 2018) and unit conversions used by the oracle."""

C0 = 299792458.0                 # m/s
MU0 = 1.25663706212e-6           # N/A^2
EPS0 = 8.8541878128e-12          # F/m
HBAR_EVS = 6.582119569e-16       # eV*s
A0 = 5.29177210903e-11           # m (Bohr radius)
T_AU = 2.4188843265857e-17       # s (atomic unit of time)
F_AU = 5.14220674763e11          # V/m (atomic unit of field)
EA0 = 8.4783536255e-30           # C*m (atomic unit of dipole)
HARTREE_EV = 27.211386245988     # eV (atomic unit of energy)
