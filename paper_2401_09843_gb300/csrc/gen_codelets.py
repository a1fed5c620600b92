"""Writes codelets.cuh: straight-line small DFTs in registers.

Run once after editing this file (the output is committed):
    python paper_2401_09843_gb300/csrc/gen_codelets.py

Each codelet computes, in place on R complex registers,
    X[k] = sum_j x[j] exp(SIGN * 2 pi i j k / R),   SIGN = -1 (forward) or +1,
by the two-factor Cooley-Tukey split R = p * m (input index m*j1 + j2, output
index k1 + p*k2, twiddle exp(SIGN 2 pi i j2 k1 / R) in between) down to
hand-written radix-2/3/4 butterflies and the symmetric-pair form for the primes
5 and 7.  Twiddle constants are evaluated here with mpmath to 30 digits and
written as literals, so the device code holds no table and calls no math
function.
"""
from __future__ import annotations

import os

import mpmath

mpmath.mp.dps = 40
RADICES = [2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 32]


def lit(v) -> str:
    s = mpmath.nstr(mpmath.mpf(v), 30, strip_zeros=False)
    return f"T({s})"


class Gen:
    def __init__(self):
        self.lines = []
        self.n = 0

    def new(self, re: str, im: str):
        k = self.n
        self.n += 1
        self.lines.append(f"    const T a{k}r = {re}; const T a{k}i = {im};")
        return (f"a{k}r", f"a{k}i")

    def add(self, x, y):
        return self.new(f"{x[0]} + {y[0]}", f"{x[1]} + {y[1]}")

    def sub(self, x, y):
        return self.new(f"{x[0]} - {y[0]}", f"{x[1]} - {y[1]}")

    def scale(self, x, c: str):
        return self.new(f"{c} * {x[0]}", f"{c} * {x[1]}")

    def twiddle(self, x, e: int, R: int, sign: int):
        """x * exp(sign 2 pi i e / R)."""
        e %= R
        if e == 0:
            return x
        if 4 * e == R:                     # angle pi/2 -> sign*i
            return self.new(f"-({x[1]})", x[0]) if sign > 0 else self.new(x[1], f"-({x[0]})")
        if 2 * e == R:
            return self.new(f"-({x[0]})", f"-({x[1]})")
        if 4 * e == 3 * R:                 # angle 3pi/2 -> -sign*i
            return self.new(x[1], f"-({x[0]})") if sign > 0 else self.new(f"-({x[1]})", x[0])
        ang = 2 * mpmath.pi * e / R
        c = mpmath.cos(ang)
        s = sign * mpmath.sin(ang)
        C, S = lit(c), lit(s)
        return self.new(f"{x[0]} * {C} - {x[1]} * {S}", f"{x[0]} * {S} + {x[1]} * {C}")

    def times_i(self, x, s: int):
        """x * (s i), s = +-1."""
        return self.new(f"-({x[1]})", x[0]) if s > 0 else self.new(x[1], f"-({x[0]})")


def dft(g: Gen, xs, sign: int):
    R = len(xs)
    if R == 1:
        return list(xs)
    if R == 2:
        return [g.add(xs[0], xs[1]), g.sub(xs[0], xs[1])]
    if R == 3:
        t1 = g.add(xs[1], xs[2])
        t2 = g.new(f"{xs[0][0]} - T(0.5) * {t1[0]}", f"{xs[0][1]} - T(0.5) * {t1[1]}")
        d = g.sub(xs[1], xs[2])
        m = lit(sign * mpmath.sin(2 * mpmath.pi / 3))
        y0 = g.add(xs[0], t1)
        y1 = g.new(f"{t2[0]} - {m} * {d[1]}", f"{t2[1]} + {m} * {d[0]}")
        y2 = g.new(f"{t2[0]} + {m} * {d[1]}", f"{t2[1]} - {m} * {d[0]}")
        return [y0, y1, y2]
    if R == 4:
        a = g.add(xs[0], xs[2])
        b = g.sub(xs[0], xs[2])
        c = g.add(xs[1], xs[3])
        d = g.sub(xs[1], xs[3])
        id_ = g.times_i(d, sign)
        return [g.add(a, c), g.add(b, id_), g.sub(a, c), g.sub(b, id_)]
    if R in (5, 7):
        h = (R - 1) // 2
        p = [g.add(xs[j], xs[R - j]) for j in range(1, h + 1)]
        q = [g.sub(xs[j], xs[R - j]) for j in range(1, h + 1)]
        out = [None] * R
        s0r = " + ".join([xs[0][0]] + [pj[0] for pj in p])
        s0i = " + ".join([xs[0][1]] + [pj[1] for pj in p])
        out[0] = g.new(s0r, s0i)
        for k in range(1, h + 1):
            cr = [lit(mpmath.cos(2 * mpmath.pi * j * k / R)) for j in range(1, h + 1)]
            sr = [lit(sign * mpmath.sin(2 * mpmath.pi * j * k / R)) for j in range(1, h + 1)]
            Ar = " + ".join([xs[0][0]] + [f"{c} * {pj[0]}" for c, pj in zip(cr, p)])
            Ai = " + ".join([xs[0][1]] + [f"{c} * {pj[1]}" for c, pj in zip(cr, p)])
            Br = " + ".join([f"{s} * {qj[0]}" for s, qj in zip(sr, q)])
            Bi = " + ".join([f"{s} * {qj[1]}" for s, qj in zip(sr, q)])
            A = g.new(Ar, Ai)
            B = g.new(Br, Bi)
            out[k] = g.new(f"{A[0]} - {B[1]}", f"{A[1]} + {B[0]}")
            out[R - k] = g.new(f"{A[0]} + {B[1]}", f"{A[1]} - {B[0]}")
        return out
    for p in (4, 2, 3, 5, 7):
        if R % p == 0 and R != p:
            break
    m = R // p
    Y = []
    for j2 in range(m):
        sub = dft(g, [xs[m * j1 + j2] for j1 in range(p)], sign)
        Y.append([g.twiddle(sub[k1], j2 * k1, R, sign) for k1 in range(p)])
    X = [None] * R
    for k1 in range(p):
        Z = dft(g, [Y[j2][k1] for j2 in range(m)], sign)
        for k2 in range(m):
            X[k1 + p * k2] = Z[k2]
    return X


def emit(R: int, sign: int) -> str:
    g = Gen()
    xs = [(f"x{j}r", f"x{j}i") for j in range(R)]
    ys = dft(g, xs, sign)
    head = [f"template <> struct Dft<{R}, {sign}> {{",
            "  template <typename T>",
            "  static NS3D_HD void run(cplx<T>* v) {"]
    head += [f"    const T x{j}r = v[{j}].x; const T x{j}i = v[{j}].y;" for j in range(R)]
    tail = [f"    v[{k}].x = {ys[k][0]}; v[{k}].y = {ys[k][1]};" for k in range(R)]
    return "\n".join(head + g.lines + tail + ["  }", "};", ""])


def main():
    out = ["// Generated by gen_codelets.py: small in-register DFTs with literal twiddles.",
           "// X[k] = sum_j x[j] exp(SIGN 2 pi i j k / R); SIGN = -1 forward, +1 inverse.",
           "#pragma once",
           "",
           "template <int R, int SIGN> struct Dft;",
           "template <int SIGN> struct Dft<1, SIGN> {",
           "  template <typename T> static NS3D_HD void run(cplx<T>*) {}",
           "};",
           ""]
    for R in RADICES:
        for sign in (-1, 1):
            out.append(emit(R, sign))
    out.append("#define NS3D_CODELET_RADICES " + ", ".join(str(r) for r in RADICES))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "codelets.cuh")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
