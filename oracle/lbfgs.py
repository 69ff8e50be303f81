"""Limited-memory BFGS for the unconstrained problem of eq. optFunc (Sec. 4).

Test infrastructure only (see the package docstring).

Sec. 4 runs L-BFGS-B with no bounds, memory m = 5, caps of 10,000 outer and 50,000 total
iterations, and a gradient tolerance pgtol. With infinite bounds the projected gradient
is the gradient, so the method is plain L-BFGS. The paper does not list the other settings; the
readings used here (and by the device optimiser, which follows the same steps) are:

  * direction: the two-loop recursion (Nocedal & Wright, Numerical Optimization, 2nd ed.,
    Alg. 7.4) with H0 = gamma I, gamma = s^T y / y^T y of the newest pair (1 with no pairs);
  * step: a strong-Wolfe line search by bracketing and zoom (ibid., Algs. 3.5 and 3.6) with
    c1 = 1e-3 and c2 = 0.9 (the sufficient-decrease and curvature constants of L-BFGS-B's line
    search), trial points in zoom by safeguarded cubic interpolation (ibid., eq. 3.59), the
    bracketing phase doubling the step; the first iteration starts at step 1/||g||_2, later ones
    at step 1; at most `max_ls` evaluations per line search;
  * stopping: ||g||_inf <= pgtol; relative decrease (f_k - f_{k+1}) / max(|f_k|, |f_{k+1}|, 1)
    <= factr * eps (factr = 1e7); `max_iters` outer iterations; `max_evals` evaluations
    (Sec. 4.1's total iterations, i.e. calls of the function/gradient);
  * a pair (s, y) is stored only when s^T y > 1e-10 * y^T y (positive curvature).

Stop reasons: 1 pgtol, 2 factr, 3 max_iters, 4 max_evals, 5 line search failed, 6 non-finite.
"""

import math

import numpy as np

STOP_PGTOL, STOP_FACTR, STOP_MAXITER, STOP_MAXEVAL, STOP_LSFAIL, STOP_NONFINITE = 1, 2, 3, 4, 5, 6
EPS = np.finfo(np.float64).eps


def two_loop(g, S, Yh):
    """Return H g by the two-loop recursion (Nocedal & Wright Alg. 7.4); S, Yh are lists of the
    stored pairs, oldest first."""
    q = np.array(g, dtype=np.float64)
    k = len(S)
    alpha = [0.0] * k
    rho = [1.0 / float(Yh[i] @ S[i]) for i in range(k)]
    for i in range(k - 1, -1, -1):
        alpha[i] = rho[i] * float(S[i] @ q)
        q = q - alpha[i] * Yh[i]
    gamma = float(S[-1] @ Yh[-1]) / float(Yh[-1] @ Yh[-1]) if k else 1.0
    r = gamma * q
    for i in range(k):
        beta = rho[i] * float(Yh[i] @ r)
        r = r + S[i] * (alpha[i] - beta)
    return r


def cubic_step(a0, f0, d0, a1, f1, d1):
    """Minimiser of the cubic through (a0, f0, d0) and (a1, f1, d1) (Nocedal & Wright eq. 3.59);
    None when the cubic has no real minimiser."""
    if a0 == a1:
        return None
    t1 = d0 + d1 - 3.0 * (f0 - f1) / (a0 - a1)
    disc = t1 * t1 - d0 * d1
    if not (disc >= 0.0) or not math.isfinite(disc):
        return None
    t2 = math.copysign(math.sqrt(disc), a1 - a0)
    den = d1 - d0 + 2.0 * t2
    if den == 0.0 or not math.isfinite(den):
        return None
    return a1 - (a1 - a0) * (d1 + t2 - t1) / den


def _interp(lo, flo, dlo, hi, fhi, dhi):
    """Trial point strictly inside (lo, hi): the cubic minimiser if it lies in the middle 80%
    of the interval, else the midpoint."""
    a = cubic_step(lo, flo, dlo, hi, fhi, dhi)
    left, right = min(lo, hi), max(lo, hi)
    width = right - left
    if a is None or not (left + 0.1 * width <= a <= right - 0.1 * width):
        a = 0.5 * (lo + hi)
    return a


def lbfgs(fg, x0, m=5, pgtol=1e-5, factr=1e7, max_iters=10000, max_evals=50000,
          c1=1e-3, c2=0.9, max_ls=20, callback=None):
    """Minimise f with gradient: fg(x) -> (f, g). Returns a dict with x, f, g, iters, evals,
    stop (reason code) and trace (f after every accepted step)."""
    x = np.array(x0, dtype=np.float64)
    f, g = fg(x)
    evals = 1
    S, Yh = [], []
    trace = [f]
    iters = 0
    stop = 0
    while True:
        if not (math.isfinite(f) and np.all(np.isfinite(g))):
            stop = STOP_NONFINITE
            break
        if np.max(np.abs(g)) <= pgtol:
            stop = STOP_PGTOL
            break
        if iters >= max_iters:
            stop = STOP_MAXITER
            break
        if evals >= max_evals:
            stop = STOP_MAXEVAL
            break
        pdir = -two_loop(g, S, Yh)
        dphi0 = float(g @ pdir)
        if not (dphi0 < 0.0):            # not a descent direction: drop the memory
            S, Yh = [], []
            pdir = -g
            dphi0 = float(g @ pdir)
        a_init = 1.0 / float(np.linalg.norm(pdir)) if not S else 1.0

        # ---- strong-Wolfe line search (Nocedal & Wright Alg. 3.5, zoom Alg. 3.6) ----
        # every point is kept as (step, phi, phi', gradient)
        phi0 = f
        ls_evals = 0

        def phi(a):
            fa, ga = fg(x + a * pdir)
            return (a, fa, float(ga @ pdir), ga)

        prev = (0.0, phi0, dphi0, g)
        a_cur = a_init
        accepted = None
        lo = hi = None
        while evals < max_evals and ls_evals < max_ls:
            cur = phi(a_cur)
            evals += 1
            ls_evals += 1
            if not math.isfinite(cur[1]) or cur[1] > phi0 + c1 * cur[0] * dphi0 or \
                    (ls_evals > 1 and cur[1] >= prev[1]):
                lo, hi = prev, cur
                break
            if abs(cur[2]) <= -c2 * dphi0:
                accepted = cur
                break
            if cur[2] >= 0.0:
                lo, hi = cur, prev
                break
            prev = cur
            a_cur = 2.0 * a_cur
        if accepted is None and lo is None:
            lo = prev                      # budget ran out while extrapolating
        while accepted is None and hi is not None and evals < max_evals and ls_evals < max_ls:
            if math.isfinite(hi[1]):
                aj = _interp(lo[0], lo[1], lo[2], hi[0], hi[1], hi[2])
            else:
                aj = 0.5 * (lo[0] + hi[0])
            cur = phi(aj)
            evals += 1
            ls_evals += 1
            if not math.isfinite(cur[1]) or cur[1] > phi0 + c1 * aj * dphi0 or cur[1] >= lo[1]:
                hi = cur
            else:
                if abs(cur[2]) <= -c2 * dphi0:
                    accepted = cur
                    break
                if cur[2] * (hi[0] - lo[0]) >= 0.0:
                    hi = lo
                lo = cur
        if accepted is None and lo[0] > 0.0 and lo[1] < phi0:
            accepted = lo                  # out of budget: keep the best decrease found
        if accepted is None:
            stop = STOP_MAXEVAL if evals >= max_evals else STOP_LSFAIL
            break

        a, f_new, _, g_new = accepted
        x_new = x + a * pdir
        s = x_new - x
        yv = g_new - g
        sy = float(s @ yv)
        if sy > 1e-10 * float(yv @ yv):
            S.append(s)
            Yh.append(yv)
            if len(S) > m:
                S.pop(0)
                Yh.pop(0)
        f_old = f
        x, f, g = x_new, f_new, g_new
        iters += 1
        trace.append(f)
        if callback is not None:
            callback(x, f, g)
        if (f_old - f) / max(abs(f_old), abs(f), 1.0) <= factr * EPS:
            stop = STOP_FACTR
            break
    return dict(x=x, f=f, g=g, iters=iters, evals=evals, stop=stop, trace=trace)
