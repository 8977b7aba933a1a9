"""Writes mlqp_bessel_taylor.inc: Taylor coefficients f^(k)(c)/k!, k = 0..12,
of J0, J1, Y0, Y1 at the centres c = 4.25 + 0.5 m (m = 0..119) of the
half-unit intervals covering [4, 64), from 30-digit mpmath derivatives,
rounded to double.  The derivatives of J0 and J1 are bounded by 1 (their
integral representations), those of Y0 and Y1 by about 1 for x >= 4 (the
nearest singularity, the logarithm at 0, is at distance c >= 4.25), and
|x - c| <= 0.25, so the first dropped term is below 0.25^13 / 13! = 2.4e-18.
Run from this directory:
    python gen_bessel_taylor.py"""
import mpmath as mp

mp.mp.dps = 30
DEG, M, X0, H = 12, 120, 4.0, 0.5


def coeffs(fn, n, c):
    return [fn(n, c, derivative=k) / mp.factorial(k) for k in range(DEG + 1)]


lines = ["// Generated by gen_bessel_taylor.py: Taylor coefficients f^(k)(c)/k!, k = 0..%d, of" % DEG,
         "// J0, J1, Y0, Y1 at c = %.2f + %.1f m, m = 0..%d (rows of 4 x %d doubles)." % (X0 + H / 2, H, M - 1, DEG + 1),
         "constexpr int BESSEL_TAYLOR_DEG = %d;" % DEG,
         "static __device__ const double BESSEL_TAYLOR[%d * 4 * %d] = {" % (M, DEG + 1)]
for m in range(M):
    c = mp.mpf(X0) + H * m + H / 2
    row = []
    for fn, n in ((mp.besselj, 0), (mp.besselj, 1), (mp.bessely, 0), (mp.bessely, 1)):
        row += [float(v) for v in coeffs(fn, n, c)]
    lines.append("    " + ", ".join(repr(v) for v in row) + ",")
lines.append("};")
open("mlqp_bessel_taylor.inc", "w").write("\n".join(lines) + "\n")
