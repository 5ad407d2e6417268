"""Write green_quadrature.txt: reference values computed with mpmath straight from
the paper's formulas, independently of the oracle and of the CUDA path.

* c_{sigma,r} from its Bessel definition (Lemma 2.1, eq. def_c_sigma_r):
      c = (sqrt(sigma) r)^nu / (2^nu Gamma(nu+1) I_nu(sqrt(sigma) r)),  nu = (n-2)/2
* omega(y) = int_B G(y, z) dz (eq. omega_of_y) by quadrature of the ball Green
  function of the Remark after Lemma 2.1 over the ball, in radial form
      omega = |S^{n-1}| int_0^r rho^{n-1} G(rho) d rho
* the radial CDF of Z ~ rho(y, .) = G/omega (eq. Z_sampling_density):
      F(t) = int_0^t s^{n-1} G(s r) ds / int_0^1 s^{n-1} G(s r) ds
Run:  python tests/golden/make_green_golden.py
"""
import os

import mpmath as mp

mp.mp.dps = 40
HERE = os.path.dirname(os.path.abspath(__file__))
CASES = [  # (n, sigma, r)
    (3, 2.0, 0.3257142857142857), (3, 1.0, 0.57), (3, 9.0, 1.0), (4, 1.0, 0.5), (5, 1.0, 0.7),
    (9, 3.0, 0.4), (10, 1.0, 1.0), (21, 2.25, 1.0), (1000, 0.5, 0.57), (1000, 1.0, 0.05),
    (1001, 9.0, 1.0), (1001, 2002.0, 0.3),
]
TS = [0.05, 0.25, 0.5, 0.75, 0.95, 0.999]


def green(n, lam, r, rho):
    """Ball Green function at the centre (Remark after Lemma 2.1)."""
    nu = mp.mpf(n - 2) / 2
    return (mp.mpf(1) / (2 * mp.pi) ** (mp.mpf(n) / 2) * (lam / rho) ** nu
            * (mp.besselk(nu, lam * rho) - mp.besselk(nu, lam * r) / mp.besseli(nu, lam * r)
               * mp.besseli(nu, lam * rho)))


def main():
    rows = []
    for n, sigma, r in CASES:
        sigma, r = mp.mpf(sigma), mp.mpf(r)
        lam = mp.sqrt(sigma)
        nu = mp.mpf(n - 2) / 2
        a = lam * r
        c = a ** nu / (2 ** nu * mp.gamma(nu + 1) * mp.besseli(nu, a))
        area = 2 * mp.pi ** (mp.mpf(n) / 2) / mp.gamma(mp.mpf(n) / 2)
        dens = lambda s: s ** (n - 1) * green(n, lam, r, s * r)
        tot = mp.quad(dens, [0, 1])
        omega = area * r ** n * tot
        for t in TS:
            F = mp.quad(dens, [0, t]) / tot
            rows.append(f"{n} {mp.nstr(sigma, 17)} {mp.nstr(r, 17)} {t} {mp.nstr(c, 20)} "
                        f"{mp.nstr(omega, 20)} {mp.nstr(F, 20)}")
        print(n, float(sigma), float(r), "done")
    with open(os.path.join(HERE, "green_quadrature.txt"), "w") as fh:
        fh.write("# generated by make_green_golden.py (mpmath quadrature of the Remark's Green function)\n")
        fh.write("# n sigma r t c_sigma_r omega F(t)\n")
        fh.write("\n".join(rows) + "\n")


if __name__ == "__main__":
    main()
