"""Write wendland_table1.txt: the Wendland functions of the paper's Table 1
evaluated EXACTLY (rational arithmetic) at eta = m/8.

Source: Table 1 (Wendland C0, C2, C4, C6 with eta = |r - r_i| / R) and Eq. 2
(C2, zero for eta >= 1).  Each row is: basis, eta as a fraction, phi as a
fraction, phi as a float.  Run from the repository root:
    python tests/golden/make_wendland_table1.py
"""
import os
from fractions import Fraction as F

TABLE1 = {
    "C0": lambda e: (1 - e) ** 2,
    "C2": lambda e: (1 - e) ** 4 * (4 * e + 1),
    "C4": lambda e: (1 - e) ** 6 * (F(35, 3) * e**2 + 6 * e + 1),
    "C6": lambda e: (1 - e) ** 8 * (32 * e**3 + 25 * e**2 + 8 * e + 1),
}

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wendland_table1.txt")
    with open(out, "w") as f:
        f.write("# Wendland compact basis functions, paper Table 1 (C2 = Eq. 2), exact at eta = m/8\n")
        f.write("# basis eta_num/eta_den phi_num/phi_den phi_float\n")
        for name, fn in TABLE1.items():
            for m in range(0, 11):
                e = F(m, 8)
                v = fn(e) if e < 1 else F(0)
                f.write(f"{name} {e.numerator}/{e.denominator} {v.numerator}/{v.denominator} {float(v)!r}\n")
    print(out)
