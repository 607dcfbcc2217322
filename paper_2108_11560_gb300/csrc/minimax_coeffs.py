"""Prints the minimax coefficients used by the FP32 bins (kv_bins.cuh): Remez exchange in 40-digit
arithmetic (mpmath) for the polynomials p(z) = sum_j c_j z^j of least maximum absolute error on an
interval, for

  E(z) = (cosh sqrt(z) - 1) / z               on z in [0, 1]         (degree 3)
  O(z) = (sinh sqrt(z) / sqrt(z) - 1) / z     on z in [0, 1]         (degree 3)
  P(z) = (tanh(sqrt z) / sqrt z - 1) / z      on z in [0, 0.35^2]    (degree 3)

and, for the FP64 bins, E and O on z in [0, 1] at degree 6.

E and O are the even and odd parts of phi(s) = e^s - 1 - s = z (E(z) + s O(z)), z = s^2; P gives
tanh(y) = y + y^3 P(y^2).  Not used at run time: the kernel holds the printed values.

    python paper_2108_11560_gb300/csrc/minimax_coeffs.py
"""
import mpmath as mp

mp.mp.dps = 40


def _E(z):
    return (mp.cosh(mp.sqrt(z)) - 1) / z if z != 0 else mp.mpf(1) / 2


def _O(z):
    r = mp.sqrt(z)
    return (mp.sinh(r) / r - 1) / z if z != 0 else mp.mpf(1) / 6


def _P(z):
    r = mp.sqrt(z)
    return (mp.tanh(r) / r - 1) / z if z != 0 else -mp.mpf(1) / 3


def remez(f, a, b, deg, iters=30, grid=4000):
    """Coefficients (lowest first) and the maximum absolute error of the degree-`deg` minimax
    polynomial of f on [a, b]."""
    n = deg + 2
    x = [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * i / (n - 1)) for i in range(n)]
    c, ext = None, None
    for _ in range(iters):
        # solve p(x_i) + (-1)^i e = f(x_i) for the coefficients and the levelled error e
        A = mp.matrix(n, n)
        rhs = mp.matrix(n, 1)
        for i, xi in enumerate(x):
            for j in range(deg + 1):
                A[i, j] = xi ** j
            A[i, deg + 1] = (-1) ** i
            rhs[i] = f(xi)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(deg + 1)]
        pts = [a + (b - a) * mp.mpf(k) / grid for k in range(grid + 1)]
        err = [sum(cj * t ** j for j, cj in enumerate(c)) - f(t) for t in pts]
        # local extrema of the error, then one per run of equal sign (the largest)
        cand = [(pts[k], err[k]) for k in range(len(pts))
                if k in (0, len(pts) - 1) or (err[k] - err[k - 1]) * (err[k + 1] - err[k]) <= 0]
        ext = []
        for t, e in cand:
            if ext and mp.sign(ext[-1][1]) == mp.sign(e):
                if abs(e) > abs(ext[-1][1]):
                    ext[-1] = (t, e)
            else:
                ext.append((t, e))
        while len(ext) > n:
            ext.pop(0 if abs(ext[0][1]) < abs(ext[-1][1]) else -1)
        if len(ext) < n:
            break
        x = [t for t, _ in ext]
    return c, max(abs(e) for _, e in ext)


if __name__ == "__main__":
    # FP32 bins: degree 3
    for name, f, hi in (("E", _E, mp.mpf(1)), ("O", _O, mp.mpf(1)), ("P", _P, mp.mpf("0.35") ** 2)):
        c, e = remez(f, mp.mpf(0), hi, 3)
        print(f"{name}: " + ", ".join(mp.nstr(cj, 17) for cj in c) + f"   max abs error {mp.nstr(e, 3)}")
    # FP64 bins: degree 6 (17 significant digits round to the nearest double)
    for name, f in (("E64", _E), ("O64", _O)):
        c, e = remez(f, mp.mpf(0), mp.mpf(1), 6, grid=8000)
        print(f"{name}: " + ", ".join(mp.nstr(cj, 17) for cj in c) + f"   max abs error {mp.nstr(e, 3)}")
