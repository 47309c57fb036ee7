"""Write ngon_closed_form.txt: the potential on a regular n-gon, from the closed form.

With unit charges on the vertices z_j = c + R w^j (w = exp(2 pi i / n)), the
potential at vertex k is sum_{j != k} log|R (1 - w^(j-k))| = (n - 1) log R + log n,
because prod_{m=1}^{n-1} (1 - w^m) = n (the value at 1 of (z^n - 1)/(z - 1)).

With alternating charges q_j = (-1)^j (n even), the products over even and odd m
are the values at 1 of (z^(n/2) - 1)/(z - 1) and of z^(n/2) + 1, i.e. n/2 and 2, so
phi_k = (-1)^k (log(n / 4) - log R).

These identities are exact, so the file holds no value computed by any FMM code.
Run: python tests/golden/make_ngon.py
"""
import math
import os

ROWS = []
for n in (3, 4, 7, 16, 64, 257):
    for R in (0.25, 1.0, 2.0):
        ROWS.append((n, R, "unit", (n - 1) * math.log(R) + math.log(n)))
for n in (4, 8, 64, 256):
    for R in (0.5, 2.0):
        ROWS.append((n, R, "alternating", math.log(n / 4.0) - math.log(R)))

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ngon_closed_form.txt")
    with open(out, "w") as f:
        f.write("# regular n-gon about (2.5, 2.5): n R pattern phi_at_vertex_0\n")
        f.write("# source: closed form, see make_ngon.py (roots of unity); 'alternating' is phi at even vertices,\n")
        f.write("# odd vertices carry the negated value\n")
        for n, R, pat, v in ROWS:
            f.write(f"{n} {R!r} {pat} {v!r}\n")
