"""Writes expm1_poly.h: the library's own expm1 for x <= 0 (used by the FP64 decisions).

x = k ln2 + r with k = round(x / ln2) and |r| <= ln2 / 2 (r = fma(-k, ln2, x), ln2 rounded
to double); expm1(r) = r p(r) with p of degree 8 interpolating (e^r - 1) / r at the 9
Chebyshev points of [-0.35, 0.35] (mpmath, 60 digits, coefficients rounded to double);
expm1(x) = 2^k expm1(r) + (2^k - 1), one FMA.  The accuracy (about 2^-38) is what the FP64
decisions need: their error bounds carry it explicitly.  The script prints the interpolation
error of r p(r) measured in 60-digit arithmetic with the rounded coefficients.

Run: python gen_expm1_poly.py > expm1_poly.h
"""
import mpmath as mp

mp.mp.dps = 60
DEG = 8
H = mp.mpf("0.35")


def f(x):
    return mp.mpf(1) if x == 0 else mp.expm1(x) / x


def main():
    n = DEG + 1
    nodes = [H * mp.cos(mp.pi * (2 * k + 1) / (2 * n)) for k in range(n)]
    V = mp.matrix(n, n)
    y = mp.matrix(n, 1)
    for i, x in enumerate(nodes):
        for j in range(n):
            V[i, j] = x ** j
        y[i] = f(x)
    c = mp.lu_solve(V, y)
    cd = [float(c[j]) for j in range(n)]
    worst = mp.mpf(0)
    for i in range(40001):
        x = -H + 2 * H * i / 40000
        if x == 0:
            continue
        p = mp.mpf(0)
        for j in reversed(range(n)):
            p = p * x + mp.mpf(cd[j])
        worst = max(worst, abs(x * p - mp.expm1(x)) / abs(mp.expm1(x)))
    ln2 = mp.log(2)
    l2 = float(ln2)
    inv = float(1 / ln2)
    print("// expm1_poly.h -- written by gen_expm1_poly.py (do not edit).")
    print("// expm1(r) ~ r p(r) on [-0.35, 0.35], p of degree %d interpolating (e^r - 1)/r at the" % DEG)
    print("// Chebyshev points; coefficients rounded to double.  Max relative error of r p(r) in")
    print("// exact arithmetic with these coefficients, on 40001 points: %s" % mp.nstr(worst, 3))
    print("#pragma once")
    print("#include <cuda_runtime.h>")
    print("namespace sco {")
    print("constexpr double kExpLn2 = %s;  // ln 2, rounded" % repr(l2))
    print("constexpr double kExpInvLn2 = %s;  // 1 / ln 2, rounded" % repr(inv))
    print("// p(r) by Horner's rule, one FMA per coefficient")
    print("__host__ __device__ __forceinline__ double expm1_poly(double r) {")
    print("  double p = %s;" % repr(cd[n - 1]))
    for j in reversed(range(n - 1)):
        print("  p = fma(p, r, %s);" % repr(cd[j]))
    print("  return p;")
    print("}")
    print("}  // namespace sco")


if __name__ == "__main__":
    main()
