"""Writes codelets.cuh and codelets_packed.cuh: straight-line small DFTs in registers.

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


# ---------------------------------------------------------------------------
# Packed codelets: the same splittings, written with explicit operations on a
# lane type V so that two independent transforms run in lockstep (V a pair of
# floats on the GPU: one add, multiply or fused multiply-add instruction acts
# on both lanes).  Signs are carried symbolically and folded into the next
# add/sub or constant, so a negation costs an instruction only where an output
# is left negated.

class PVal:
    __slots__ = ("name", "neg")

    def __init__(self, name: str, neg: bool = False):
        self.name = name
        self.neg = neg

    def flip(self):
        return PVal(self.name, not self.neg)


class GenP:
    def __init__(self):
        self.lines = []
        self.n = 0

    def _new(self, expr: str, neg: bool = False) -> PVal:
        k = self.n
        self.n += 1
        self.lines.append(f"    const V p{k} = {expr};")
        return PVal(f"p{k}", neg)

    def radd(self, a: PVal, b: PVal, sub: bool = False) -> PVal:
        """a + b (or a - b) of real lane values."""
        bn = b.neg ^ sub
        if not a.neg and not bn:
            return self._new(f"padd({a.name}, {b.name})")
        if not a.neg and bn:
            return self._new(f"psub({a.name}, {b.name})")
        if a.neg and not bn:
            return self._new(f"psub({b.name}, {a.name})")
        return self._new(f"padd({a.name}, {b.name})", neg=True)

    def rmul(self, c, a: PVal) -> PVal:
        c = -c if a.neg else c
        return self._new(f"pmul({plit(c)}, {a.name})")

    def rfma(self, c, a: PVal, acc: PVal) -> PVal:
        """c a + acc."""
        c = -c if a.neg else c
        if acc.neg:   # c a - x = -((-c) a + x)
            return self._new(f"pfma({plit(-c)}, {a.name}, {acc.name})", neg=True)
        return self._new(f"pfma({plit(c)}, {a.name}, {acc.name})")

    def lin(self, terms, base: PVal | None = None) -> PVal:
        """base + sum c_j a_j as a chain of fused multiply-adds."""
        acc = base
        for c, a in terms:
            acc = self.rmul(c, a) if acc is None else self.rfma(c, a, acc)
        return acc

    def cadd(self, x, y):
        return (self.radd(x[0], y[0]), self.radd(x[1], y[1]))

    def csub(self, x, y):
        return (self.radd(x[0], y[0], True), self.radd(x[1], y[1], True))

    def times_i(self, x, s: int):
        return (x[1].flip(), x[0]) if s > 0 else (x[1], x[0].flip())

    def twiddle(self, x, e: int, R: int, sign: int):
        e %= R
        if e == 0:
            return x
        if 4 * e == R:
            return self.times_i(x, sign)
        if 2 * e == R:
            return (x[0].flip(), x[1].flip())
        if 4 * e == 3 * R:
            return self.times_i(x, -sign)
        ang = 2 * mpmath.pi * e / R
        c = mpmath.cos(ang)
        s = sign * mpmath.sin(ang)
        re = self.rfma(-s, x[1], self.rmul(c, x[0]))
        im = self.rfma(s, x[0], self.rmul(c, x[1]))
        return (re, im)


def plit(v) -> str:
    s = mpmath.nstr(mpmath.mpf(v), 30, strip_zeros=False)
    return f"pk<V>({s})"


def dftp(g: GenP, xs, sign: int):
    R = len(xs)
    if R == 1:
        return list(xs)
    if R == 2:
        return [g.cadd(xs[0], xs[1]), g.csub(xs[0], xs[1])]
    if R == 3:
        t1 = g.cadd(xs[1], xs[2])
        t2 = (g.rfma(mpmath.mpf(-0.5), t1[0], xs[0][0]), g.rfma(mpmath.mpf(-0.5), t1[1], xs[0][1]))
        d = g.csub(xs[1], xs[2])
        m = sign * mpmath.sin(2 * mpmath.pi / 3)
        y0 = g.cadd(xs[0], t1)
        y1 = (g.rfma(-m, d[1], t2[0]), g.rfma(m, d[0], t2[1]))
        y2 = (g.rfma(m, d[1], t2[0]), g.rfma(-m, d[0], t2[1]))
        return [y0, y1, y2]
    if R == 4:
        a = g.cadd(xs[0], xs[2])
        b = g.csub(xs[0], xs[2])
        c = g.cadd(xs[1], xs[3])
        d = g.csub(xs[1], xs[3])
        id_ = g.times_i(d, sign)
        return [g.cadd(a, c), g.cadd(b, id_), g.csub(a, c), g.csub(b, id_)]
    if R in (5, 7):
        h = (R - 1) // 2
        p = [g.cadd(xs[j], xs[R - j]) for j in range(1, h + 1)]
        q = [g.csub(xs[j], xs[R - j]) for j in range(1, h + 1)]
        out = [None] * R
        s0 = xs[0]
        for pj in p:
            s0 = g.cadd(s0, pj)
        out[0] = s0
        for k in range(1, h + 1):
            cr = [mpmath.cos(2 * mpmath.pi * j * k / R) for j in range(1, h + 1)]
            sr = [sign * mpmath.sin(2 * mpmath.pi * j * k / R) for j in range(1, h + 1)]
            A = (g.lin([(c, pj[0]) for c, pj in zip(cr, p)], xs[0][0]),
                 g.lin([(c, pj[1]) for c, pj in zip(cr, p)], xs[0][1]))
            B = (g.lin([(s, qj[0]) for s, qj in zip(sr, q)]),
                 g.lin([(s, qj[1]) for s, qj in zip(sr, q)]))
            out[k] = (g.radd(A[0], B[1], True), g.radd(A[1], B[0]))
            out[R - k] = (g.radd(A[0], B[1]), g.radd(A[1], B[0], True))
        return out
    for p in (4, 2, 3, 5, 7):
        if R % p == 0 and R != p:
            break
    m = R // p
    Y = []
    for j2 in range(m):
        sub = dftp(g, [xs[m * j1 + j2] for j1 in range(p)], sign)
        Y.append([g.twiddle(sub[k1], j2 * k1, R, sign) for k1 in range(p)])
    X = [None] * R
    for k1 in range(p):
        Z = dftp(g, [Y[j2][k1] for j2 in range(m)], sign)
        for k2 in range(m):
            X[k1 + p * k2] = Z[k2]
    return X


def emitp(R: int, sign: int) -> str:
    g = GenP()
    xs = [(PVal(f"r[{j}]"), PVal(f"i[{j}]")) for j in range(R)]
    # inputs are read once into named values so that outputs may overwrite r, i
    g.lines += [f"    const V x{j}r = r[{j}]; const V x{j}i = i[{j}];" for j in range(R)]
    xs = [(PVal(f"x{j}r"), PVal(f"x{j}i")) for j in range(R)]
    ys = dftp(g, xs, sign)
    body = list(g.lines)
    tail = []
    for k in range(R):
        for part, arr in ((ys[k][0], "r"), (ys[k][1], "i")):
            expr = f"pneg({part.name})" if part.neg else part.name
            tail.append(f"    {arr}[{k}] = {expr};")
    head = [f"template <> struct DftP<{R}, {sign}> {{",
            "  template <typename V>",
            "  static NS3D_HD void run(V* r, V* i) {"]
    return "\n".join(head + body + tail + ["  }", "};", ""])


def main_packed():
    out = ["// Generated by gen_codelets.py: packed in-register DFTs with literal twiddles.",
           "// X[k] = sum_j x[j] exp(SIGN 2 pi i j k / R) on real and imaginary lane arrays",
           "// r[], i[] of a lane type V (padd/psub/pmul/pfma/pneg/pk<V> overloads): for V a",
           "// float pair, two transforms run in lockstep.  SIGN = -1 forward, +1 inverse.",
           "#pragma once",
           "",
           "template <int R, int SIGN> struct DftP;",
           "template <int SIGN> struct DftP<1, SIGN> {",
           "  template <typename V> static NS3D_HD void run(V*, V*) {}",
           "};",
           ""]
    for R in RADICES:
        for sign in (-1, 1):
            out.append(emitp(R, sign))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "codelets_packed.cuh")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
    main_packed()
