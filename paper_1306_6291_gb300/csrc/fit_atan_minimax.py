"""Derivation of the atan polynomial used by the FP32 kernels (k_atan_unit in kd_method.cuh).

atan(t) / t is fitted by a polynomial P(s) in s = t^2 on t in [0, 1], minimising the maximum
RELATIVE error (so atan(t) = t P(t^2) keeps full relative accuracy for small angles), by the
Remez exchange algorithm in 40-digit arithmetic (mpmath). Run: python fit_atan_minimax.py.
Degree 8 gives a maximum relative error of 1.5e-8, below half an FP32 ulp.
"""
import numpy as np, mpmath as mp
mp.mp.dps = 40
def f(s):  # atan(sqrt s)/sqrt s
    s = mp.mpf(s)
    if s == 0: return mp.mpf(1)
    r = mp.sqrt(s); return mp.atan(r)/r
def remez(deg, iters=30):
    # minimize max |P(s) - f(s)| / f(s) on [0,1]
    n = deg + 2
    xs = [ (1 - mp.cos(mp.pi*k/(n-1)))/2 for k in range(n)]
    for it in range(iters):
        A = mp.matrix(n, n); b = mp.matrix(n, 1)
        for i, x in enumerate(xs):
            fx = f(x)
            for j in range(deg+1): A[i, j] = x**j
            A[i, deg+1] = (-1)**i * fx
            b[i] = fx
        sol = mp.lu_solve(A, b)
        c = [sol[j] for j in range(deg+1)]; E = sol[deg+1]
        # find extrema of error on dense grid
        grid = [mp.mpf(k)/4000 for k in range(4001)]
        err = [ (sum(c[j]*g**j for j in range(deg+1)) - f(g))/f(g) for g in grid]
        # pick alternating extrema
        ext = []
        for k in range(len(grid)):
            if k == 0 or k == len(grid)-1 or (abs(err[k]) >= abs(err[k-1]) and abs(err[k]) >= abs(err[k+1])):
                ext.append(k)
        # merge same-sign runs keep max
        merged = []
        for k in ext:
            if merged and mp.sign(err[k]) == mp.sign(err[merged[-1]]):
                if abs(err[k]) > abs(err[merged[-1]]): merged[-1] = k
            else: merged.append(k)
        if len(merged) >= n:
            # choose n with largest errors contiguous window
            best = max(range(len(merged)-n+1), key=lambda s: min(abs(err[merged[s+i]]) for i in range(n)))
            xs = [grid[merged[best+i]] for i in range(n)]
        maxerr = max(abs(e) for e in err)
    return c, maxerr
if __name__ == "__main__":
  for deg in (6, 7, 8):
    c, e = remez(deg)
    print(deg, float(e), [float(x) for x in c])
