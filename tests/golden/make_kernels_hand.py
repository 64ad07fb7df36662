"""Writes kernels_hand.json: values of the transcendental kernels at points
where the kernel reduces, by hand, to a short closed form.

Each entry gives the point z, the closed form of k(z) at that point (the
distances simplified by hand: 3-4-5 triangles, axis-aligned vectors) and
its value, evaluated here with 40-digit arithmetic (mpmath through sympy).
Nothing here calls the oracle or the GPU library.  Run from the repository
root:  python tests/golden/make_kernels_hand.py
"""
from __future__ import annotations

import json
import os

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))

# kernel name -> citation
CITE = {
    "config3": "Anisotropic test kernel of the Gaussian-mixture workload (1,048,576 points, depth 5): "
               "k(z) = exp(-|z|)/|z| + 1/sqrt(z0^2 + 0.01 z1^2 + z2^2 + 1e-3); the 0.01 weight is on "
               "the second (y) component",
    "exp_r2": "Section 5.4, kernel exp(-|z|^2)",
    "cos20r_r": "Section 5.4, kernel cos(20|z|)/|z|",
    "sqrt_r2p1": "Section 5.4, kernel sqrt(|z|^2 + 1)",
}

# (kernel, z, closed form of k(z) at that z, worked by hand)
# Every z is a dyadic rational (exact in binary) and |z| comes out exact, so
# the only roundings are those of the kernel's own operations.
CASES = [
    # |z| = 10 along y: the 0.01 weight turns the second term into 1/sqrt(1 + 1e-3)
    ("config3", ("0", "10", "0"), "exp(-10)/10 + 1/sqrt(1 + 1/1000)"),
    # the same |z| along x and z: no weight, 1/sqrt(100 + 1e-3)
    ("config3", ("10", "0", "0"), "exp(-10)/10 + 1/sqrt(100 + 1/1000)"),
    ("config3", ("0", "0", "10"), "exp(-10)/10 + 1/sqrt(100 + 1/1000)"),
    # 3-4-5 triangles scaled to |z| = 5/8, the weighted axis in each position
    ("config3", ("3/8", "1/2", "0"), "exp(-5/8)/(5/8) + 1/sqrt(9/64 + (1/100)*(1/4) + 1/1000)"),
    ("config3", ("3/8", "0", "1/2"), "exp(-5/8)/(5/8) + 1/sqrt(9/64 + 1/4 + 1/1000)"),
    ("config3", ("0", "3/8", "1/2"), "exp(-5/8)/(5/8) + 1/sqrt((1/100)*(9/64) + 1/4 + 1/1000)"),
    # |z| = 3 (1-2-2) and 5/8
    ("exp_r2", ("1", "2", "2"), "exp(-9)"),
    ("exp_r2", ("3/8", "1/2", "0"), "exp(-25/64)"),
    ("exp_r2", ("0", "0", "0"), "1"),
    # |z| = 1/16, 5/8 and 5/4 (3/4-0-1)
    ("cos20r_r", ("0", "0", "1/16"), "16*cos(5/4)"),
    ("cos20r_r", ("3/8", "1/2", "0"), "cos(25/2)/(5/8)"),
    ("cos20r_r", ("3/4", "0", "1"), "cos(25)/(5/4)"),
    ("sqrt_r2p1", ("1", "2", "2"), "sqrt(10)"),
    ("sqrt_r2p1", ("3/8", "1/2", "0"), "sqrt(89)/8"),
    ("sqrt_r2p1", ("0", "0", "0"), "1"),
]


def main() -> None:
    out = {"note": "k(z) at points where it has a short closed form; the value is that closed "
                   "form to 17 significant digits (40-digit evaluation)",
           "cite": CITE, "cases": []}
    for kern, z, expr in CASES:
        v = sp.N(sp.sympify(expr), 40)
        out["cases"].append({"kernel": kern, "z": [float(sp.Rational(c)) for c in z],
                             "z_exact": list(z), "k_exact": expr, "k": float(v)})
    with open(os.path.join(HERE, "kernels_hand.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
