"""Generate the ziggurat tables compiled into librp (csrc/zig_tables.inc).

Construction (Randompack Sec. 3.1, 256 equal-area strips, Marsaglia & Tsang
2000): strip 0 is the base (rectangle [0,R] x [0,f(R)] plus the tail beyond
R), strips 1..255 are rectangles [0,x_i] x [f(x_i), f(x_{i-1})] with
x_255 = R and x_0 = 0.  The common area v is the unknown here: for a trial
v the base condition R f(R) + tail(R) = v fixes R, the recursion
x_{i-1} = f^{-1}(f(x_i) + v / x_i) runs down to x_1, and v is adjusted until
the top strip x_1 (1 - f(x_1)) also has area v.  All arithmetic is 70-digit
mpmath; each table entry is rounded once.

  k[i] = floor(M x_{i-1}/x_i) (k[1] = 0), k[0] = floor(M R f(R)/v)
  w[i] = x_i / M,                          w[0] = v / (f(R) M)
  f[i] = f(x_i),                           f[0] = 1
with M = 2^52 (normal: 52 magnitude bits) or 2^53 (exponential).

Run:  python -m paper_2605_05099_gb300.gen_tables
"""
import os

import mpmath as mp

mp.mp.dps = 70
STRIPS = 256


class _Density:
    def __init__(self, kind):
        self.kind = kind
        if kind == "normal":
            self.scale = mp.mpf(2) ** 52
            self.v_lo, self.v_hi = mp.mpf("0.0048"), mp.mpf("0.0050")
        else:
            self.scale = mp.mpf(2) ** 53
            self.v_lo, self.v_hi = mp.mpf("0.0039"), mp.mpf("0.0040")

    def f(self, x):
        return mp.exp(-x * x / 2) if self.kind == "normal" else mp.exp(-x)

    def finv(self, y):
        return mp.sqrt(-2 * mp.log(y)) if self.kind == "normal" else -mp.log(y)

    def tail(self, r):
        if self.kind == "normal":
            return mp.sqrt(2 * mp.pi) * mp.ncdf(-r)
        return mp.exp(-r)

    def radius(self, v):
        """R with R f(R) + tail(R) = v (left side decreasing in R)."""
        a, b = mp.mpf(1), mp.mpf(12)
        for _ in range(250):          # bisection: the left side decreases in R
            m = (a + b) / 2
            if m * self.f(m) + self.tail(m) > v:
                a = m
            else:
                b = m
        return (a + b) / 2

    def ladder(self, v):
        r = self.radius(v)
        x = {STRIPS - 1: r}
        for i in range(STRIPS - 1, 1, -1):
            y = self.f(x[i]) + v / x[i]
            if y >= 1:
                return r, None
            x[i - 1] = self.finv(y)
        return r, x

    def mismatch(self, v):
        """area of the top strip minus v (negative when v is too large)."""
        r, x = self.ladder(v)
        if x is None:
            return mp.mpf(-1)
        return x[1] * (1 - self.f(x[1])) - v

    def solve(self):
        lo, hi = self.v_lo, self.v_hi
        mlo = self.mismatch(lo)
        assert mlo > 0 and self.mismatch(hi) < 0
        for _ in range(240):
            mid = (lo + hi) / 2
            if self.mismatch(mid) > 0:
                lo = mid
            else:
                hi = mid
        v = (lo + hi) / 2
        r, x = self.ladder(v)
        return v, r, x


def build(kind):
    d = _Density(kind)
    v, r, x = d.solve()
    k, w, f = [0] * STRIPS, [0.0] * STRIPS, [0.0] * STRIPS
    k[0] = int(mp.floor(d.scale * r * d.f(r) / v))
    w[0] = float(v / (d.f(r) * d.scale))
    f[0] = 1.0
    for i in range(1, STRIPS):
        k[i] = 0 if i == 1 else int(mp.floor(d.scale * x[i - 1] / x[i]))
        w[i] = float(x[i] / d.scale)
        f[i] = float(d.f(x[i]))
    return {"k": k, "w": w, "f": f, "R": float(r), "v": v}


def render():
    lines = ["// Generated by paper_2605_05099_gb300/gen_tables.py; do not edit.",
             "// Ziggurat tables (256 strips) for the normal (N) and exponential (E) samplers."]
    for tag, kind in (("N", "normal"), ("E", "exp")):
        t = build(kind)
        lines.append(f"// v = {mp.nstr(t['v'], 40)}")
        lines.append(f"static const double RP_ZIG_{tag}_R = {t['R'].hex()};")
        lines.append(f"static const unsigned long long RP_ZIG_{tag}_K[256] = {{")
        lines += [f"  0x{v:016x}ULL," for v in t["k"]]
        lines.append("};")
        for key in ("w", "f"):
            lines.append(f"static const double RP_ZIG_{tag}_{key.upper()}[256] = {{")
            lines += [f"  {v.hex()}," for v in t[key]]
            lines.append("};")
    return "\n".join(lines) + "\n"


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "zig_tables.inc")
    with open(out, "w") as fh:
        fh.write(render())
    print("wrote", out)


if __name__ == "__main__":
    main()
