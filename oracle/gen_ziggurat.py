"""Oracle ziggurat tables (test infrastructure only).

Writes ``oracle/ziggurat_tables.h`` from the 256-strip Marsaglia--Tsang
construction (Sec. 3.1 "Normal and exponential distributions", ziggurat
figure): 255 rectangles of equal area v stacked on a base strip that holds a
rectangle [0,R] x [0,f(R)] plus the tail beyond R.  Everything is solved in
60-digit arithmetic (mpmath) and rounded once to double at the end.

Strip numbering (low byte of the word):
  * strip 0 is the base strip; its pseudo-width is q = v / f(R);
  * strip i in 1..255 is the rectangle [0, x_i] x [f(x_i), f(x_{i-1})] with
    x_255 = R, x_0 = 0 and f(x_0) = 1.
Tables (M = 2^52 for the normal, 2^53 for the exponential; readings of the
garbled index in Sec. 3.1, where w_i is printed with x_{i-1}):
  k[i] = floor(M x_{i-1} / x_i) for i >= 1 (k[1] = 0),  k[0] = floor(M R / q)
  w[i] = x_i / M                for i >= 1,              w[0] = q / M
  f[i] = f(x_i)                 for i >= 1,              f[0] = 1
R is the root of the closure condition x_1 (1 - f(x_1)) = v, i.e. the top
strip has the same area as every other strip.

Run:  python oracle/gen_ziggurat.py   (rewrites oracle/ziggurat_tables.h)
"""
import os
import mpmath as mp

mp.mp.dps = 60
N = 256


def _normal_f(x):
    return mp.exp(-x * x / 2)


def _normal_finv(y):
    return mp.sqrt(-2 * mp.log(y))


def _normal_tail(r):
    return mp.sqrt(mp.pi / 2) * mp.erfc(r / mp.sqrt(2))


def _exp_f(x):
    return mp.exp(-x)


def _exp_finv(y):
    return -mp.log(y)


def _exp_tail(r):
    return mp.exp(-r)


def _strips(r, f, finv, tail):
    """x_255 = r down to x_1; returns (xs, v) or (None, v) if the recursion
    leaves the density's range (r too small)."""
    v = r * f(r) + tail(r)
    xs = [mp.mpf(0)] * N
    xs[N - 1] = r
    for i in range(N - 1, 1, -1):
        y = v / xs[i] + f(xs[i])
        if y >= 1:
            return None, v
        xs[i - 1] = finv(y)
    return xs, v


def _closure(r, f, finv, tail):
    xs, v = _strips(r, f, finv, tail)
    if xs is None:
        return mp.mpf(1)          # recursion overshoots the top: r too small
    return v - xs[1] * (1 - f(xs[1]))


def solve(f, finv, tail, lo, hi):
    """Bisection on the closure condition (monotone in r on [lo, hi])."""
    glo = _closure(mp.mpf(lo), f, finv, tail)
    ghi = _closure(mp.mpf(hi), f, finv, tail)
    assert glo * ghi < 0, (glo, ghi)
    a, b = mp.mpf(lo), mp.mpf(hi)
    for _ in range(230):
        m = (a + b) / 2
        gm = _closure(m, f, finv, tail)
        if (gm > 0) == (glo > 0):
            a, glo = m, gm
        else:
            b = m
    return (a + b) / 2


def tables(kind):
    if kind == "normal":
        f, finv, tail, scale, lo, hi = _normal_f, _normal_finv, _normal_tail, 2 ** 52, 3.5, 3.8
    else:
        f, finv, tail, scale, lo, hi = _exp_f, _exp_finv, _exp_tail, 2 ** 53, 7.5, 7.9
    r = solve(f, finv, tail, lo, hi)
    xs, v = _strips(r, f, finv, tail)
    q = v / f(r)
    k = [0] * N
    w = [0.0] * N
    fv = [0.0] * N
    k[0] = int(mp.floor(scale * r / q))
    w[0] = float(q / scale)
    fv[0] = 1.0
    for i in range(1, N):
        k[i] = int(mp.floor(scale * xs[i - 1] / xs[i])) if i > 1 else 0
        w[i] = float(xs[i] / scale)
        fv[i] = float(f(xs[i]))
    return dict(r=r, v=v, q=q, x=xs, k=k, w=w, f=fv)


def _emit(name, t, out):
    out.append(f"/* {name}: R = {mp.nstr(t['r'], 30)}, v = {mp.nstr(t['v'], 30)} */")
    out.append(f"static const double OR_{name}_R = {float(t['r']).hex()};")
    out.append(f"static const uint64_t OR_{name}_K[256] = {{")
    out.extend(f"  0x{x:016x}ull," for x in t["k"])
    out.append("};")
    for key in ("w", "f"):
        out.append(f"static const double OR_{name}_{key.upper()}[256] = {{")
        out.extend(f"  {x.hex()}," for x in t[key])
        out.append("};")


def main():
    out = ["/* Generated by oracle/gen_ziggurat.py -- do not edit. Oracle-only data. */",
           "#ifndef OR_ZIGGURAT_TABLES_H", "#define OR_ZIGGURAT_TABLES_H", "#include <stdint.h>"]
    _emit("ZN", tables("normal"), out)
    _emit("ZE", tables("exp"), out)
    out.append("#endif")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ziggurat_tables.h")
    with open(path, "w") as fh:
        fh.write("\n".join(out) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
