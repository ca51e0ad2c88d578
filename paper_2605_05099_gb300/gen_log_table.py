"""Generate the table of the fast correctly rounded log (csrc/log_table.inc).

Table-driven reduction (Tang, ACM TOMS 16(4), 1990): for y = 2^e m, m in
[1, 2), the top 10 bits of m pick c_j = 1 + (j + 1/2)/1024 and inv_j =
round(2^11 / c_j) / 2^11, a double with 11 fraction bits, so that
r = m inv_j - 1 is exact in one fused multiply-add and |r| <= 2^-10.  Then
log y = e ln 2 - log(inv_j) + log1p(r).  The table holds inv_j and -log(inv_j)
as a double-double (hi, lo), each rounded once from 70-digit mpmath.  Two
entries avoid cancellation near y = 1: j = 0 uses inv = 1 (log term 0), and
j = 1023 uses inv = 1/2 with the log term folded into e (stored as 0, the
kernel adds one to e).

Run:  python -m paper_2605_05099_gb300.gen_log_table
"""
import os

import mpmath as mp

mp.mp.dps = 70
N = 1024


def entries():
    out = []
    for j in range(N):
        if j == 0:
            out.append((1.0, 0.0, 0.0))
            continue
        if j == N - 1:
            out.append((0.5, 0.0, 0.0))
            continue
        c = 1 + (mp.mpf(j) + mp.mpf("0.5")) / N
        inv = mp.nint(mp.mpf(2048) / c) / 2048
        invd = float(inv)
        assert mp.mpf(invd) == inv
        L = -mp.log(inv)
        hi = float(L)
        lo = float(L - mp.mpf(hi))
        out.append((invd, hi, lo))
    return out


def main():
    rows = entries()
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "csrc", "log_table.inc")
    with open(path, "w") as fh:
        fh.write("// Generated by paper_2605_05099_gb300/gen_log_table.py: {inv_j, -log(inv_j) hi, lo}, j < 1024.\n")
        fh.write("static __device__ const double g_log_tab[1024][3] = {\n")
        for inv, hi, lo in rows:
            fh.write(f"  {{{inv.hex()}, {hi.hex()}, {lo.hex()}}},\n")
        fh.write("};\n")
    print(path)


if __name__ == "__main__":
    main()
