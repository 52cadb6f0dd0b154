"""Writes appendix_closed_forms.txt: the closed forms of the appendix example.

Panel sigma = conv{h e1, h e2, h e3, 0} in (tau, y1, y2, y3), h = 10 t, apex in
the panel plane (y3 = 0). Values are I without the factor 1/(4 pi), as printed.
  corner (Appendix, Case 1): x = (t, -eps/sqrt2, -eps/sqrt2, 0)
     I = 2t(pi/4 - asin(eps/(sqrt2 t))) - sqrt2 eps log(sqrt2 - 1)
         + sqrt2 eps log( sqrt2 (1 - sqrt(1 - eps^2/(2 t^2))) / (eps/t) )
     The printed formula has eps^2/(4 t^2) under the root; the paper's own
     second derivatives in t and t-eps imply 2 t^2, and the corrected form is
     the one the exact integral satisfies.
  edge (Appendix, Case 2): x = (t, -eps, h/2, 0)
     I = 2t(pi - acos(-eps/t)) - 2 eps log((1 + sqrt(1 - eps^2/t^2)) / (eps/t))
Evaluated in 40-digit arithmetic (mpmath).
"""
import os

import mpmath as mp

mp.mp.dps = 40
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "appendix_closed_forms.txt")


def corner(t, eps):
    s2 = mp.sqrt(2)
    return (2 * t * (mp.pi / 4 - mp.asin(eps / (s2 * t))) - s2 * eps * mp.log(s2 - 1)
            + s2 * eps * mp.log(s2 * (1 - mp.sqrt(1 - eps ** 2 / (2 * t ** 2))) / (eps / t)))


def edge(t, eps):
    return 2 * t * (mp.pi - mp.acos(-eps / t)) - 2 * eps * mp.log((1 + mp.sqrt(1 - eps ** 2 / t ** 2)) / (eps / t))


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write("# case t eps_over_t I   (Appendix of Poelz & Schanz; corner with the 2t^2 correction)\n")
        for t in ["0.5", "1", "2"]:
            for r in ["1e-6", "1e-3", "0.1", "0.5", "0.9", "0.999"]:
                T, R = mp.mpf(t), mp.mpf(r)
                f.write(f"corner {t} {r} {mp.nstr(corner(T, R * T), 25)}\n")
                f.write(f"edge {t} {r} {mp.nstr(edge(T, R * T), 25)}\n")
