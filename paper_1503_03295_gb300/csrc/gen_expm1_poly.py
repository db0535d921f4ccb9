"""Writes expm1_poly.h: the library's own expm1 for x <= 0 (used by the FP64 decisions).

x = k ln2 + r with k = round(x / ln2) and |r| <= ln2 / 2 (r = fma(-k, ln2, x), ln2 rounded
to double); expm1(r) = r p(r) with p interpolating (e^r - 1) / r at the Chebyshev points of
[-0.35, 0.35] (mpmath, 60 digits, coefficients rounded to double); expm1(x) = 2^k expm1(r) +
(2^k - 1), one FMA.  Two degrees: 8 (about 2^-43, for the switch, whose survival margin is
absolute and must stay small next to the thinning bound of far pairs) and 6 (about 2^-31.7, for
the sweep decisions, whose margin is a sum of relative errors: a decision inside it takes the
double-double path, a few sites per sweep of 5M).  Their error bounds carry these explicitly.  The script prints the interpolation
error of r p(r) measured in 60-digit arithmetic with the rounded coefficients.

Run: python gen_expm1_poly.py > expm1_poly.h
"""
import mpmath as mp

mp.mp.dps = 60
DEG = 8
H = mp.mpf("0.35")


def f(x):
    return mp.mpf(1) if x == 0 else mp.expm1(x) / x


def fit(deg):
    n = deg + 1
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
    return cd, worst


def emit(name, deg):
    cd, worst = fit(deg)
    print("// %s: degree %d; max relative error of r p(r) in exact arithmetic with these" % (name, deg))
    print("// coefficients, on 40001 points: %s" % mp.nstr(worst, 3))
    print("__host__ __device__ __forceinline__ double %s(double r) {" % name)
    print("  double p = %s;" % repr(cd[deg]))
    for j in reversed(range(deg)):
        print("  p = fma(p, r, %s);" % repr(cd[j]))
    print("  return p;")
    print("}")


def main():
    ln2 = mp.log(2)
    print("// expm1_poly.h -- written by gen_expm1_poly.py (do not edit).")
    print("// expm1(r) ~ r p(r) on [-0.35, 0.35], p interpolating (e^r - 1)/r at the Chebyshev")
    print("// points; coefficients rounded to double; p(r) by Horner's rule, one FMA per coefficient.")
    print("#pragma once")
    print("#include <cuda_runtime.h>")
    print("namespace sco {")
    print("constexpr double kExpLn2 = %s;  // ln 2, rounded" % repr(float(ln2)))
    print("constexpr double kExpInvLn2 = %s;  // 1 / ln 2, rounded" % repr(float(1 / ln2)))
    emit("expm1_poly", DEG)
    emit("expm1_poly6", 6)
    print("}  // namespace sco")


if __name__ == "__main__":
    main()
