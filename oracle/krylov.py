"""Outer and inner Krylov levels of the nested method (oracle; test infrastructure).

Sec. 2: f(A) x ~ ||x|| V_k f(H_k) e_1 (Eq. (approximation)) with v_1 = x/||x||,
H_k = V_k^dag A V_k (Hermitian Lanczos, mu = 0) or W_k^dag A V_k (two-sided
Lanczos with W_k^dag V_k = 1, mu != 0); sgn(H) by Roberts-Higham
S_{n+1} = (S_n + S_n^{-1})/2, S_0 = H (Eq. (Roberts)).
Sec. 3: sgn(H_k) e_1 ~ V_l sgn(H_l) e_1 on the inner space K_l(H_k + H_k^{-1}, e_1)
(Eqs. (nested), (precond)).

Readings where the paper is silent (each is listed in the design notes):
  * Lanczos in the form p = A v_j - beta_j v_{j-1}; alpha_j = Re v_j^dag p;
    p -= alpha_j v_j; beta_{j+1} = ||p||; v_{j+1} = p / beta_{j+1}; no
    re-orthogonalisation ("short recurrences", Sec. 2).
  * two-sided Lanczos with w_1 = v_1,
      p = A v_j - gamma_j v_{j-1},        alpha_j = w_j^dag p,
      r = A^dag w_j - conj(beta_j) w_{j-1},
      v~ = p - alpha_j v_j,  w~ = r - conj(alpha_j) w_j,  delta = w~^dag v~,
      beta_{j+1} = sqrt|delta|, gamma_{j+1} = delta / beta_{j+1},
      v_{j+1} = v~ / beta_{j+1}, w_{j+1} = w~ / conj(gamma_{j+1});
    H_k has diagonal alpha, subdiagonal H_{j+1,j} = beta_{j+1} and
    superdiagonal H_{j,j+1} = gamma_{j+1}. A serious breakdown
    (|delta| <= breakdown_tol ||v~|| ||w~||) is an error.
  * inner level: H_k^{-1} u by a dense LU solve; inner Lanczos (mu = 0) or
    inner two-sided Lanczos (mu != 0, M^dag = H^dag + H^{-dag}) from e_1 for
    l_eff = min(l, k) steps; an exhausted inner space (next beta <= 1e-13 *
    ||M q||) ends it early.
  * Roberts-Higham unscaled; stop when ||S_{n+1} - S_n||_F <= rh_tol ||S_{n+1}||_F.
  * stopping rule: every check_interval steps (and at k_max), c_k = Q_l sgn(T_l) e_1
    and est_outer = ||c_k - [c_prev; 0]|| / ||c_k|| (infinite at the first
    check). When est_outer <= tol the inner level is judged too:
    est_inner = ||c_k - c_k'|| / ||c_k|| with c_k' from l_eff - 4 inner steps
    (the leading block of the same inner space)
    (0 when the inner space is exhausted or l_eff = k, i.e. exact). The run
    stops there with err_est = max(est_outer, est_inner); status OK if
    err_est <= tol, else NOT_CONVERGED (the inner dimension is too small).
"""
import numpy as np
import scipy.linalg as sla

OK = 0
NOT_CONVERGED = 1
ERR_BREAKDOWN = -5
ERR_RH_NOCONV = -6


def tridiag(alpha, beta, gamma=None):
    """k x k tridiagonal: diag alpha_1..alpha_k, sub H_{j+1,j} = beta_{j+1},
    super H_{j,j+1} = gamma_{j+1}. beta and gamma are indexed so that beta[j]
    holds beta_{j+1} (0-based: beta[0] = beta_1 = 0 is unused)."""
    k = len(alpha)
    if gamma is None:
        gamma = beta
    dt = np.result_type(np.asarray(alpha), np.asarray(beta), np.asarray(gamma))
    h = np.zeros((k, k), dtype=dt)
    h[np.arange(k), np.arange(k)] = alpha
    if k > 1:
        h[np.arange(1, k), np.arange(k - 1)] = beta[1:k]
        h[np.arange(k - 1), np.arange(1, k)] = gamma[1:k]
    return h


class Outer:
    """The outer Krylov process, one step at a time.

    hermitian=True: Lanczos on A (mu = 0). hermitian=False: two-sided Lanczos on
    (A, A^dag). After j steps: alpha[:j], beta[:j+1], gamma[:j+1] (beta[0] =
    gamma[0] = 0) and, if store=True, V[:, :j] = v_1..v_j.
    """

    def __init__(self, apply_A, apply_AH, x, hermitian, store=True, breakdown_tol=1e-14):
        self.apply_A = apply_A
        self.apply_AH = apply_AH
        self.hermitian = hermitian
        self.store = store
        self.tol = breakdown_tol
        self.norm_x = float(np.linalg.norm(x))
        self.v = x / self.norm_x
        self.v_prev = np.zeros_like(self.v)
        self.w = self.v.copy()
        self.w_prev = np.zeros_like(self.v)
        self.alpha = []
        self.beta = [0.0]
        self.gamma = [0.0]
        self.V = []
        self.status = OK

    @property
    def k(self):
        return len(self.alpha)

    def step(self):
        j = self.k
        if self.store:
            self.V.append(self.v)
        if self.hermitian:
            b = self.beta[j]
            p = self.apply_A(self.v) - b * self.v_prev
            a = float(np.real(np.vdot(self.v, p)))
            p = p - a * self.v
            bn = float(np.linalg.norm(p))
            self.alpha.append(a)
            self.beta.append(bn)
            self.gamma.append(bn)
            self.v_prev = self.v
            self.v = p / bn if bn > 0 else np.zeros_like(p)
            if bn <= self.tol * (abs(a) + abs(b)):
                self.status = ERR_BREAKDOWN  # invariant subspace (lucky breakdown)
            return
        b = self.beta[j]
        g = self.gamma[j]
        p = self.apply_A(self.v) - g * self.v_prev
        a = complex(np.vdot(self.w, p))
        r = self.apply_AH(self.w) - np.conj(b) * self.w_prev
        vt = p - a * self.v
        wt = r - np.conj(a) * self.w
        delta = complex(np.vdot(wt, vt))
        bn = float(np.sqrt(abs(delta)))
        self.alpha.append(a)
        self.beta.append(bn)
        if abs(delta) <= self.tol * np.linalg.norm(vt) * np.linalg.norm(wt) or bn == 0.0:
            self.gamma.append(0.0)
            self.status = ERR_BREAKDOWN
            return
        gn = delta / bn
        self.gamma.append(gn)
        self.v_prev, self.w_prev = self.v, self.w
        self.v = vt / bn
        self.w = wt / np.conj(gn)

    def H(self, k=None):
        k = self.k if k is None else k
        if self.hermitian:
            return tridiag(np.array(self.alpha[:k]), np.array(self.beta[:k + 1]))
        return tridiag(np.array(self.alpha[:k], dtype=complex), np.array(self.beta[:k + 1], dtype=complex),
                       np.array(self.gamma[:k + 1], dtype=complex))


def roberts_higham(T, rh_tol=1e-10, maxit=100):
    """sgn(T) by S_{n+1} = (S_n + S_n^{-1})/2, S_0 = T (Eq. (Roberts)).

    Returns (S, iterations, converged)."""
    S = np.array(T, dtype=np.result_type(T, np.float64))
    for it in range(1, maxit + 1):
        Sn = 0.5 * (S + np.linalg.inv(S))
        diff = np.linalg.norm(Sn - S)
        nrm = np.linalg.norm(Sn)
        S = Sn
        if not (np.isfinite(diff) and np.isfinite(nrm)):
            return S, it, False  # numerically singular iterate
        if diff <= rh_tol * nrm:
            return S, it, True
    return S, maxit, False


def inner_krylov(H, l, hermitian, exhaust_tol=1e-13):
    """Inner level of Eq. (nested): Krylov space K_l(M, e_1), M = H + H^{-1}.

    Returns (T_l, Q_l) with Q_l of shape (k, l_eff) and T_l of shape
    (l_eff, l_eff); H^{-1} u is a dense LU solve of H (Eq. (precond))."""
    k = H.shape[0]
    l = min(l, k)
    lu = sla.lu_factor(H)
    luh = None if hermitian else sla.lu_factor(np.conj(H.T))

    def M(u):
        return H @ u + sla.lu_solve(lu, u)

    def MH(u):
        return np.conj(H.T) @ u + sla.lu_solve(luh, u)

    dt = H.dtype
    e1 = np.zeros(k, dtype=dt)
    e1[0] = 1.0
    Q = []
    a_l, b_l, g_l = [], [0.0], [0.0]
    q, q_prev = e1, np.zeros_like(e1)
    if hermitian:
        for i in range(l):
            Q.append(q)
            Mq = M(q)
            p = Mq - b_l[i] * q_prev
            a = float(np.real(np.vdot(q, p)))
            p = p - a * q
            bn = float(np.linalg.norm(p))
            a_l.append(a)
            if i == l - 1:
                break
            if bn <= exhaust_tol * np.linalg.norm(Mq):
                break
            b_l.append(bn)
            q_prev, q = q, p / bn
        li = len(a_l)
        T = tridiag(np.array(a_l), np.array(b_l[:li]))
        return T, np.stack(Q[:li], axis=1)
    w, w_prev = e1.copy(), np.zeros_like(e1)
    for i in range(l):
        Q.append(q)
        Mq = M(q)
        p = Mq - g_l[i] * q_prev
        a = complex(np.vdot(w, p))
        r = MH(w) - np.conj(b_l[i]) * w_prev
        qt = p - a * q
        wt = r - np.conj(a) * w
        a_l.append(a)
        if i == l - 1:
            break
        delta = complex(np.vdot(wt, qt))
        bn = float(np.sqrt(abs(delta)))
        if bn <= exhaust_tol * np.linalg.norm(Mq):
            break
        gn = delta / bn
        b_l.append(bn)
        g_l.append(gn)
        q_prev, w_prev = q, w
        q = qt / bn
        w = wt / np.conj(gn)
    li = len(a_l)
    T = tridiag(np.array(a_l, dtype=complex), np.array(b_l[:li], dtype=complex), np.array(g_l[:li], dtype=complex))
    return T, np.stack(Q[:li], axis=1)


def nested_sign_e1(H, l, hermitian, rh_tol=1e-10, rh_maxit=100):
    """c = Q_l sgn(T_l) e_1 ~ sgn(H_k) e_1 (Eq. (nested) with Eq. (precond)).

    Returns (c, rh_iterations, rh_converged, l_eff)."""
    T, Q = inner_krylov(H, l, hermitian)
    S, its, ok = roberts_higham(T, rh_tol, rh_maxit)
    return Q @ S[:, 0], its, ok, T.shape[0]


def nonnested_sign_e1(H, rh_tol=1e-10, rh_maxit=100):
    """c = sgn(H_k) e_1 by Roberts-Higham on the full k x k Ritz matrix (Sec. 2)."""
    S, its, ok = roberts_higham(H, rh_tol, rh_maxit)
    return S[:, 0], its, ok


def naive_nested_sign_e1(H, l, hermitian, rh_tol=1e-10, rh_maxit=100):
    """Nesting without the preconditioning step: inner space K_l(H_k, e_1)
    (the version Sec. 3 shows gains nothing). Uses the same inner process on
    M = H instead of M = H + H^{-1}."""
    k = H.shape[0]
    l = min(l, k)
    # Krylov basis of K_l(H, e_1) for tridiagonal H is [e_1 .. e_l] (Sec. 3),
    # but this function builds it by the recurrence to test that claim.
    dt = H.dtype
    Q = []
    q = np.zeros(k, dtype=dt)
    q[0] = 1.0
    basis = []
    for i in range(l):
        u = q.copy()
        for b in basis:
            u = u - np.vdot(b, u) * b
        nrm = np.linalg.norm(u)
        if nrm <= 1e-13:
            break
        u = u / nrm
        basis.append(u)
        q = H @ u
    Q = np.stack(basis, axis=1)
    T = np.conj(Q.T) @ H @ Q
    S, its, ok = roberts_higham(T, rh_tol, rh_maxit)
    return Q @ S[:, 0], Q


INNER_DL = 4


def inner_estimate(H, l_eff, hermitian, c, exhausted, rh_tol=1e-10, rh_maxit=100):
    """||c - c'|| / ||c|| with c' from l_eff - INNER_DL inner steps (0 if exact)."""
    k = H.shape[0]
    if exhausted or l_eff >= k:
        return 0.0
    if l_eff - INNER_DL < 1:
        return float("inf")
    c2, _, _, _ = nested_sign_e1(H, l_eff - INNER_DL, hermitian, rh_tol, rh_maxit)
    return float(np.linalg.norm(c - c2) / np.linalg.norm(c))


def sign_apply(apply_A, apply_AH, x, hermitian, k_max, l, tol, check_interval=10,
               two_pass=False, rh_tol=1e-10, rh_maxit=100, breakdown_tol=1e-14,
               k_fixed=None, nested=True):
    """y ~ sgn(A) x by the nested method with the stopping rule.

    k_fixed: run exactly that many outer steps and evaluate once (no stopping
    rule). nested=False replaces the inner level by Roberts-Higham on H_k.
    Returns (y, info) with info = dict(k, l, rh_iters, err_est, status, ...).
    """
    out = Outer(apply_A, apply_AH, x, hermitian, store=not two_pass, breakdown_tol=breakdown_tol)

    def coeffs(k):
        H = out.H(k)
        if nested:
            c, its, ok, leff = nested_sign_e1(H, l, hermitian, rh_tol, rh_maxit)
        else:
            c, its, ok = nonnested_sign_e1(H, rh_tol, rh_maxit)
            leff = k
        return H, c, its, ok, leff

    status = NOT_CONVERGED
    c_prev = None
    est = np.inf
    est_in = np.nan
    c = None
    its, ok, leff = 0, True, 0
    target = k_fixed if k_fixed is not None else k_max
    while out.k < target:
        out.step()
        k = out.k
        broke = out.status == ERR_BREAKDOWN
        if k_fixed is not None:
            if broke:
                break
            continue
        if k % check_interval == 0 or k == k_max or broke:
            H, c, its, ok, leff = coeffs(k)
            if not ok:
                status = ERR_RH_NOCONV
                break
            if broke and not hermitian:
                status = ERR_BREAKDOWN
                break
            if broke:
                est = 0.0  # invariant subspace: the outer projection is exact
            elif c_prev is not None:
                cp = np.zeros_like(c)
                cp[:len(c_prev)] = c_prev
                est = float(np.linalg.norm(c - cp) / np.linalg.norm(c))
            if est <= tol or k == k_max:
                exhausted = leff < min(l, k)
                est_in = inner_estimate(H, leff, hermitian, c, exhausted, rh_tol, rh_maxit) if nested else 0.0
                est = max(est, est_in)
                status = OK if est <= tol else NOT_CONVERGED
                break
            c_prev = c
    if k_fixed is not None:
        if out.status == ERR_BREAKDOWN and not hermitian:
            status = ERR_BREAKDOWN
        H, c, its, ok, leff = coeffs(out.k)
        if status != ERR_BREAKDOWN:
            status = OK if ok else ERR_RH_NOCONV
        est = float("nan")
    k = out.k
    if c is None:
        raise RuntimeError("no coefficients")
    if two_pass:
        y = recombine_two_pass(apply_A, x, out, c, k)
    else:
        y = out.norm_x * (np.stack(out.V[:k], axis=1) @ c)
    return y, dict(k=k, l=leff, rh_iters=its, err_est=est, err_inner=est_in, status=status,
                   alpha=np.array(out.alpha), beta=np.array(out.beta), gamma=np.array(out.gamma), c=c)


def recombine_two_pass(apply_A, x, out, c, k):
    """Second pass: regenerate v_1..v_k from the stored coefficients with the
    v-side recurrence and accumulate y = ||x|| sum_j c_j v_j (double pass,
    Sec. 4)."""
    norm_x = out.norm_x
    v = x / norm_x
    v_prev = np.zeros_like(v)
    y = c[0] * v
    for j in range(1, k):
        a = out.alpha[j - 1]
        if out.hermitian:
            p = apply_A(v) - out.beta[j - 1] * v_prev
            p = p - a * v
        else:
            p = apply_A(v) - out.gamma[j - 1] * v_prev
            p = p - a * v
        v_prev, v = v, p / out.beta[j]
        y = y + c[j] * v
    return norm_x * y
