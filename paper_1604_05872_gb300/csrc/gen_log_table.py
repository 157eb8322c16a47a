"""Write log_table.h: the constants of the table-driven FP64 natural logarithm
in log_f64.cuh (the table method of P. T. P. Tang, "Table-driven implementation
of the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4),
1990, with a plain Taylor polynomial of log1p).

For the mantissa m in [1, 2) of x = 2^k m, the seven leading fraction bits pick
an interval j of width 1/128 with centre c_j = 1 + (2 j + 1) / 256, except
c_0 = 1 (so that x just above 1 needs no table term).  The table holds
inv_j = RN(1 / c_j) and L_j = RN(-ln inv_j), so that ln m = L_j + log1p(r) with
r = m inv_j - 1 exactly up to one rounding.  Intervals from the one holding
sqrt 2 up (m >= 1 + 53/128) use ln m = ln 2 + ln(m / 2): their entries hold
L_j - ln 2 and the caller adds one to k, so that x just below 1 (k = -1, m near 2) also lands
on a small L (the last interval has c = 2, L = 0).

Run with mpmath (50 significant digits); the header is committed.
"""
import os

import mpmath

mpmath.mp.dps = 50
N = 128
SPLIT = 53  # the interval [1 + 53/128, 1 + 54/128) holds sqrt(2)


def rn(x):
    """Round an mpf to the nearest double."""
    return float(mpmath.mpf(x))


def main():
    ln2 = mpmath.log(2)
    # ln 2 split: a high part with 11 trailing zero bits, so that k * LN2_HI is exact for |k| < 2^11
    hi = float(mpmath.nint(ln2 * 2 ** 42) / 2 ** 42)
    lo = rn(ln2 - mpmath.mpf(hi))
    rows = []
    for j in range(N):
        if j == 0:
            c = mpmath.mpf(1)
        elif j == N - 1:
            c = mpmath.mpf(2)
        else:
            c = 1 + mpmath.mpf(2 * j + 1) / 256
        inv = rn(1 / c)
        L = -mpmath.log(mpmath.mpf(inv))
        if j >= SPLIT:
            L -= ln2
        rows.append((inv, rn(L)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "log_table.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_log_table.py (mpmath, 50 digits): constants of the table-driven\n"
                "// FP64 logarithm in log_f64.cuh.  {RN(1 / c_j), RN(-ln RN(1 / c_j)) [- ln 2 for j >= %d]}.\n"
                % SPLIT)
        f.write("#pragma once\n\nnamespace fea {\n\n")
        f.write("constexpr int kLogSplit = %d;\n" % SPLIT)
        f.write("constexpr double kLn2Hi = %s;  // ln 2 to 42 bits\n" % hi.hex())
        f.write("constexpr double kLn2Lo = %s;  // RN(ln 2 - kLn2Hi)\n" % lo.hex())
        f.write("__device__ const double2 kLogTab[%d] = {\n" % N)
        for inv, L in rows:
            f.write("    {%s, %s},\n" % (inv.hex(), L.hex()))
        f.write("};\n\n}  // namespace fea\n")


if __name__ == "__main__":
    main()
