"""Brute-force active-set enumeration for tiny QPs (a pin for the oracle, n <= 8).

For min 0.5 x^T H x + c^T x s.t. A x <= b, l <= x <= u with H positive definite, every
choice of (variable at l / at u / free) x (row active / inactive) defines an equality
constrained QP whose KKT system is linear.  The optimum is the unique x for which some
choice gives a primal feasible point with non-negative multipliers.  This module enumerates
all 3^n 2^m choices; it shares nothing with the oracle.
"""
import itertools

import numpy as np


def solve_bruteforce(H, c, A, b, l, u, feas_tol=1e-9, sign_tol=1e-9):
    n = H.shape[0]
    m = A.shape[0]
    best = None
    for var_state in itertools.product((0, 1, 2), repeat=n):       # 0 free, 1 at l, 2 at u
        if any((st == 1 and not np.isfinite(l[j])) or (st == 2 and not np.isfinite(u[j]))
               for j, st in enumerate(var_state)):
            continue
        L = [j for j, st in enumerate(var_state) if st == 1]
        U = [j for j, st in enumerate(var_state) if st == 2]
        for row_state in itertools.product((0, 1), repeat=m):
            act = [i for i, st in enumerate(row_state) if st]
            k = len(act) + len(L) + len(U)
            if k > n:
                continue
            # KKT: H x + c + A_act^T y - E_L^T zl + E_U^T zu = 0, A_act x = b_act, x_L = l_L, x_U = u_U
            C = np.zeros((k, n))
            d = np.zeros(k)
            r = 0
            for i in act:
                C[r] = A[i]; d[r] = b[i]; r += 1
            for j in L:
                C[r, j] = 1.0; d[r] = l[j]; r += 1
            for j in U:
                C[r, j] = 1.0; d[r] = u[j]; r += 1
            # multiplier signs: rows and upper bounds enter with +, lower bounds with -
            sgn = np.array([1.0] * len(act) + [-1.0] * len(L) + [1.0] * len(U))
            K = np.zeros((n + k, n + k))
            K[:n, :n] = H
            K[:n, n:] = C.T * sgn[None, :]
            K[n:, :n] = C
            rhs = np.concatenate([-c, d])
            try:
                if np.linalg.matrix_rank(K) < n + k:
                    continue
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                continue
            x, mult = sol[:n], sol[n:]
            if np.any(mult < -sign_tol):
                continue
            if m and np.any(A @ x - b > feas_tol * (1 + np.abs(b))):
                continue
            if np.any(np.isfinite(l) & (x < l - feas_tol * (1 + np.abs(np.where(np.isfinite(l), l, 0))))):
                continue
            if np.any(np.isfinite(u) & (x > u + feas_tol * (1 + np.abs(np.where(np.isfinite(u), u, 0))))):
                continue
            y = np.zeros(m); zl = np.zeros(n); zu = np.zeros(n)
            y[act] = mult[:len(act)]
            zl[L] = mult[len(act):len(act) + len(L)]
            zu[U] = mult[len(act) + len(L):]
            f = 0.5 * x @ H @ x + c @ x
            if best is None or f < best[0] - 1e-12:
                best = (f, x, y, zl, zu)
    return best


def solve_bruteforce_two_sided(H, c, A, bl, bu, l, u, feas_tol=1e-9, sign_tol=1e-9):
    """Same enumeration for two-sided rows bl <= A x <= bu (either side may be infinite):
    every row is inactive, at its upper side or at its lower side (3^m choices).  An active
    row's multiplier y_k is signed: >= 0 at the upper side, <= 0 at the lower side, entering
    stationarity as H x + c + A^T y - z_l + z_u = 0.  Returns (f, x, y, zl, zu) or None."""
    n = H.shape[0]
    m = A.shape[0]
    best = None
    for var_state in itertools.product((0, 1, 2), repeat=n):       # 0 free, 1 at l, 2 at u
        if any((st == 1 and not np.isfinite(l[j])) or (st == 2 and not np.isfinite(u[j]))
               for j, st in enumerate(var_state)):
            continue
        L = [j for j, st in enumerate(var_state) if st == 1]
        U = [j for j, st in enumerate(var_state) if st == 2]
        for row_state in itertools.product((0, 1, 2), repeat=m):    # 0 inactive, 1 upper, 2 lower
            if any((st == 1 and not np.isfinite(bu[i])) or (st == 2 and not np.isfinite(bl[i]))
                   for i, st in enumerate(row_state)):
                continue
            act = [i for i, st in enumerate(row_state) if st]
            k = len(act) + len(L) + len(U)
            if k > n:
                continue
            C = np.zeros((k, n))
            d = np.zeros(k)
            r = 0
            for i in act:
                C[r] = A[i]
                d[r] = bu[i] if row_state[i] == 1 else bl[i]
                r += 1
            for j in L:
                C[r, j] = 1.0; d[r] = l[j]; r += 1
            for j in U:
                C[r, j] = 1.0; d[r] = u[j]; r += 1
            sgn = np.array([1.0] * len(act) + [-1.0] * len(L) + [1.0] * len(U))
            K = np.zeros((n + k, n + k))
            K[:n, :n] = H
            K[:n, n:] = C.T * sgn[None, :]
            K[n:, :n] = C
            try:
                if np.linalg.matrix_rank(K) < n + k:
                    continue
                sol = np.linalg.solve(K, np.concatenate([-c, d]))
            except np.linalg.LinAlgError:
                continue
            x, mult = sol[:n], sol[n:]
            ya = mult[:len(act)]
            want = np.array([1.0 if row_state[i] == 1 else -1.0 for i in act])
            if np.any(ya * want < -sign_tol) or np.any(mult[len(act):] < -sign_tol):
                continue
            Ax = A @ x
            fb, fbl = np.isfinite(bu), np.isfinite(bl)
            if np.any(fb & (Ax - np.where(fb, bu, 0) > feas_tol * (1 + np.abs(np.where(fb, bu, 0))))):
                continue
            if np.any(fbl & (np.where(fbl, bl, 0) - Ax > feas_tol * (1 + np.abs(np.where(fbl, bl, 0))))):
                continue
            if np.any(np.isfinite(l) & (x < l - feas_tol * (1 + np.abs(np.where(np.isfinite(l), l, 0))))):
                continue
            if np.any(np.isfinite(u) & (x > u + feas_tol * (1 + np.abs(np.where(np.isfinite(u), u, 0))))):
                continue
            y = np.zeros(m); zl = np.zeros(n); zu = np.zeros(n)
            y[act] = ya
            zl[L] = mult[len(act):len(act) + len(L)]
            zu[U] = mult[len(act) + len(L):]
            f = 0.5 * x @ H @ x + c @ x
            if best is None or f < best[0] - 1e-12:
                best = (f, x, y, zl, zu)
    return best
