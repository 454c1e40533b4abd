"""Writes isotropic_m4_eigenvalues.txt from the closed form (no oracle, no
library): for M = 4 directions theta_m = 2 pi (m + 1/2) / 4 and isotropic
scattering (g = 0, K = 1 after the normalisation of Eq. hg), the eigenproblem
(gamma K W - I) l = xi C l of Eq. discretization_2D_eigenfunc_constraint
(Sec. 2.2) with w = 1/4 reads gamma S / 4 - l_m = xi c_m l_m, S = sum(l).
Modes with S = 0 are non-zero only where c_m = -1/xi: xi = -sqrt(2) (on the
two directions with c = 1/sqrt 2) and xi = +sqrt(2).  Modes with S != 0 give
l_m = (gamma S / 4) / (1 + xi c_m) and, summing, 1 = gamma / (1 - xi^2 / 2):
xi = -+sqrt(2 (1 - gamma)).  The c and s problems have the same spectrum."""
import math
import os

OMEGAS = (1.0, 0.5, 0.1, 1e-2, 1e-4)


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "isotropic_m4_eigenvalues.txt")
    with open(path, "w") as f:
        f.write("# M = 4, g = 0: eigenvalues xi (ascending) of Eq. discretization_2D_eigenfunc_constraint\n")
        f.write("# closed form (make_isotropic_m4.py): -sqrt(2), -sqrt(2 (1 - gamma)), sqrt(2 (1 - gamma)), sqrt(2)\n")
        f.write("# one_minus_gamma xi_1 xi_2 xi_3 xi_4\n")
        for om in OMEGAS:
            xs = sorted([-math.sqrt(2.0), -math.sqrt(2.0 * om), math.sqrt(2.0 * om), math.sqrt(2.0)])
            f.write(" ".join(repr(v) for v in [om] + xs) + "\n")


if __name__ == "__main__":
    main()
