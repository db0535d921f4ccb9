"""Writes log_table.h: the table and polynomial of the library's own natural logarithm for
0 < x <= 1 (used by the FP64 candidate search of the switch).

Table-driven reduction after Tang (ACM TOMS 16(4), 1990): x = 2^k m with m in [sqrt(2)/2,
sqrt(2)); F = 1 + j/256 the nearest table point to m (|m - F| <= 1/512), r = (m - F) / F
(|r| < 0.0028); log x = k ln2 + log F + log1p(r), log1p(r) = r + r^2 q(r) with q the Taylor
polynomial of degree 4 (truncation below 2^-53 |r|).  ln 2 and log F are split hi + lo, the hi
parts with their last 8 bits zero so that k ln2_hi + logF_hi is exact for |k| <= 64.  Values
from mpmath at 60 digits.

Run: python gen_log_table.py > log_table.h
"""
import mpmath as mp

mp.mp.dps = 60
JMIN, JMAX = -76, 107  # F = 1 + j/256 covering [sqrt(2)/2 - 1/512, sqrt(2) + 1/512]


def split(v, zero_bits=8):
    hi = float(v)
    m, e = mp.frexp(mp.mpf(hi))
    # drop the last zero_bits bits of the 53-bit significand
    scale = mp.mpf(2) ** (53 - zero_bits)
    hi = float(mp.floor(m * scale + mp.mpf("0.5")) / scale * mp.mpf(2) ** e)
    lo = float(v - mp.mpf(hi))
    return hi, lo


def main():
    ln2 = mp.log(2)
    l2h, l2l = split(ln2)
    assert JMIN / 256.0 + 1 <= float(mp.sqrt(2) / 2) - 1.0 / 512 + 1e-9
    print("// log_table.h -- written by gen_log_table.py (do not edit).")
    print("// log x = k ln2 + log F_j + log1p(r), F_j = 1 + j/256 (j = %d..%d), r = (m - F_j) inv_j;" % (JMIN, JMAX))
    print("// hi parts with their last 8 bits zero (k ln2_hi + logF_hi exact for |k| <= 64).")
    print("#pragma once")
    print("namespace sco {")
    print("constexpr int kLogJmin = %d;" % JMIN)
    print("constexpr int kLogN = %d;" % (JMAX - JMIN + 1))
    print("constexpr double kLogLn2Hi = %s;" % repr(l2h))
    print("constexpr double kLogLn2Lo = %s;" % repr(l2l))
    # q(r) = sum_{n>=2} (-1)^(n+1) r^(n-2) / n, n = 2..6
    for n in range(2, 7):
        print("constexpr double kLogC%d = %s;" % (n, repr(float(mp.mpf((-1) ** (n + 1)) / n))))
    print("// {1/F_j (rounded), log F_j hi, log F_j lo}")
    print("static __device__ const double kLogTab[kLogN][3] = {")
    for j in range(JMIN, JMAX + 1):
        F = 1 + mp.mpf(j) / 256
        inv = float(1 / F)
        h, l = split(mp.log(F))
        print("    {%s, %s, %s}," % (repr(inv), repr(h), repr(l)))
    print("};")
    print("}  // namespace sco")


if __name__ == "__main__":
    main()
