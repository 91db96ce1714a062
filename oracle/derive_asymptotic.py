"""Derivation of the far-field asymptotic expansion of G_L used by the oracle.

Test infrastructure: this script belongs to the CPU oracle.  It is run by hand
(or by a slow test) and prints the monomial coefficient tables that
``lgf_oracle.c`` embeds.  Nothing in the product package imports it.

Method (App. A, Eq. lgf_lap): G_L(n) = (2 pi)^-3 int exp(-i n.xi) / sigma(xi) dxi
with sigma(xi) = sum_i (2 cos xi_i - 2) = -|xi|^2 + Q4 - Q6 + Q8 - ...,
Q_{2k} = sum_i xi_i^{2k} * 2/(2k)!.  Expanding 1/sigma in homogeneous parts
around xi = 0 and inverting each part with the free-space kernels
h_k = F^-1[|xi|^-2k] (h_1 = 1/(4 pi r), h_2 = -r/(8 pi), h_3 = r^3/(96 pi),
h_4 = -r^5/(2880 pi)) gives G_L ~ -1/(4 pi r) + T3 + T5 + T7, where T_p is
homogeneous of degree -p in n.  Each T_p is printed as
  T_p = [sum c_abc X^a Y^b Z^c] / (den * pi * r^q),  X = n1^2, Y = n2^2, Z = n3^2.
"""
import sympy as sp


def derive():
    x, y, z = sp.symbols("x y z", real=True)
    X = [x, y, z]
    r = sp.sqrt(x**2 + y**2 + z**2)
    pi = sp.pi
    h2 = -r / (8 * pi)
    h3 = r**3 / (96 * pi)
    h4 = -r**5 / (2880 * pi)

    def d(f, *orders):
        for axis, k in orders:
            if k:
                f = sp.diff(f, X[axis], k)
        return f

    # xi^(2m) -> (-1)^m d^(2m) for even monomials.
    t3 = -sp.Rational(1, 12) * sum(d(h2, (j, 4)) for j in range(3))
    t5 = (sp.Rational(1, 360) * sum(-d(h2, (j, 6)) for j in range(3))
          - sp.Rational(1, 144) * sum(d(h3, (j, 4), (k, 4)) if j != k else d(h3, (j, 8))
                                      for j in range(3) for k in range(3)))
    a = sp.Rational(1, 20160) * sum(d(h2, (j, 8)) for j in range(3))
    b = sp.Rational(1, 12 * 360) * sum(-(d(d(h3, (j, 4)), (k, 6))) for j in range(3) for k in range(3))
    c = sp.Rational(1, 1728) * sum(d(d(d(h4, (j, 4)), (k, 4)), (l, 4))
                                   for j in range(3) for k in range(3) for l in range(3))
    t7 = -(a - 2 * b + c)
    out = {}
    XX, YY, ZZ = sp.symbols("XX YY ZZ")
    for name, t, q in (("T3", t3, 7), ("T5", t5, 13), ("T7", t7, 19)):
        num = sp.expand(sp.simplify(t * pi * (x**2 + y**2 + z**2) ** sp.Rational(q, 2)))
        num = sp.expand(num.subs({x: sp.sqrt(XX), y: sp.sqrt(YY), z: sp.sqrt(ZZ)}))
        poly = sp.Poly(num, XX, YY, ZZ)
        den = sp.ilcm(*[sp.fraction(cf)[1] for cf in poly.coeffs()])
        terms = [(e[0], e[1], e[2], int(cf * den)) for e, cf in zip(poly.monoms(), poly.coeffs())]
        out[name] = (q, int(den), terms)
    return out


if __name__ == "__main__":
    for name, (q, den, terms) in derive().items():
        print(f"/* {name}: numerator / ({den} * pi * r^{q}) */")
        print("{" + ", ".join(f"{{{a},{b},{c},{v}}}" for a, b, c, v in terms) + "}")
