"""FP64 AB-GMRES, BA-GMRES, LSQR and LSMR (plain numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

``ab_gmres`` / ``ba_gmres`` follow the two columns of the algorithm box in
Sec. 2 step by step and in its notation:

    r0 = b - A x0              (BA: r0 = B b - B A x0)
    w1 = r0 / ||r0||
    for k = 1, 2, ...
        q_k = A B w_k          (BA: q_k = B A w_k)
        for i = 1..k:  h_ik = q_k^T w_i ;  q_k = q_k - h_ik w_i     (MGS)
        h_{k+1,k} = ||q_k|| ;  w_{k+1} = q_k / h_{k+1,k}
        y_k = argmin_y || ||r0|| e1 - H_k y ||
        x_k = x0 + B [w_1..w_k] y_k     (BA: x_k = x0 + [w_1..w_k] y_k)
        r_k = b - A x_k ;  stopping rule

``y_k`` is taken from a library least-squares solve of the (k+1) x k
Hessenberg problem, i.e. straight from its definition.  The stopping rule is
the discrepancy principle of Sec. 6.4: stop at the smallest k >= 0 with
||b - A x_k|| <= tau ||e||; without it (noise_norm None) run to maxit.  With
``ncp_shape`` the NCP criterion of Sec. 6.4 decides instead (``stopping``).

Readings where the paper is silent: ``ortho='cgs2'`` replaces the MGS inner
loop by classical Gram-Schmidt applied twice (equal in exact arithmetic); a
breakdown is declared when h_{k+1,k} <= 1e-14 ||q_k before orthogonalisation||,
after which the iteration stops with y_k still the least-squares minimiser of
the (k+1) x k problem, as for every other k.  The square k x k system that a
breakdown leaves is singular when A B (or B A) is: a rank-deficient A B whose
Krylov space from b is exhausted has h_{k+1,k} = 0 and a singular H_k, and
the minimiser over the exhausted space is then reached by the least-squares
solution, while a square solve blows up along the null direction.

``lsqr`` / ``lsmr`` restate Paige & Saunders (1982) and Fong & Saunders
(2011) with damping 0 and optional full reorthogonalisation of the Lanczos
bidiagonalisation vectors; Sec. 5 shows that AB-GMRES with B = A^T equals
LSQR and BA-GMRES with B = A^T equals LSMR.
"""
from __future__ import annotations

import numpy as np

from .stopping import ncp_distance

STOP_MAXIT, STOP_DP, STOP_BREAKDOWN, STOP_NCP = 0, 1, 2, 3
BREAKDOWN_RTOL = 1e-14


def _orthogonalise(q, W, k, ortho):
    """Orthogonalise q against W[:k]; returns (q, h[0:k])."""
    h = np.zeros(k)
    if ortho == "mgs":
        for i in range(k):
            h[i] = q @ W[i]
            q = q - h[i] * W[i]
    elif ortho == "cgs2":
        Wk = W[:k]
        for _ in range(2):
            c = Wk @ q
            q = q - Wk.T @ c
            h += c
    else:
        raise ValueError(ortho)
    return q, h


def _gmres(apply_M, r0, form_x, resid_norm, maxit, tau, noise_norm, ortho,
           keep, resid_vec=None, ncp_shape=None):
    """Shared Arnoldi/GMRES loop of both columns of the algorithm box.

    apply_M(w) is A B w (AB) or B A w (BA); form_x(Wk, y) builds x_k;
    resid_norm(x) returns ||b - A x||.  With ncp_shape = (N_a, N_d) the stop
    is the NCP criterion of Sec. 6.4 instead (``stopping``): the NCP
    distance d_k of b - A x_k (resid_vec) is recorded for every k, and the
    solve returns x_k at the first k with d_{k+1} > d_k."""
    L = r0.size
    beta = float(np.linalg.norm(r0))
    x = form_x(np.zeros((0, L)), np.zeros(0))
    out = {"iterates": [x] if keep else None, "rho": [beta],
           "resnorm": [resid_norm(x)], "stop_reason": STOP_MAXIT}
    use_ncp = ncp_shape is not None
    if use_ncp:
        out["ncp"] = [ncp_distance(resid_vec(x), *ncp_shape)]
        noise_norm = None
    x_prev = x
    target = None if noise_norm is None else tau * noise_norm
    if target is not None and out["resnorm"][0] <= target:
        out.update(x=x, k=0, stop_reason=STOP_DP, W=np.zeros((0, L)),
                   H=np.zeros((1, 0)))
        return out
    W = np.zeros((maxit + 1, L))
    H = np.zeros((maxit + 1, maxit))
    if beta == 0.0:
        out.update(x=x, k=0, stop_reason=STOP_BREAKDOWN, W=W[:0], H=H[:1, :0])
        return out
    W[0] = r0 / beta
    k = 0
    for k in range(1, maxit + 1):
        q = apply_M(W[k - 1])
        q_pre = float(np.linalg.norm(q))
        q, h = _orthogonalise(q, W, k, ortho)
        H[:k, k - 1] = h
        H[k, k - 1] = float(np.linalg.norm(q))
        e1 = np.zeros(k + 1)
        e1[0] = beta
        if H[k, k - 1] <= BREAKDOWN_RTOL * q_pre:
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            x = form_x(W[:k], y)
            out["rho"].append(float(np.linalg.norm(e1 - H[:k + 1, :k] @ y)))
            out["resnorm"].append(resid_norm(x))
            if keep:
                out["iterates"].append(x)
            out["stop_reason"] = STOP_BREAKDOWN
            break
        W[k] = q / H[k, k - 1]
        y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
        x = form_x(W[:k], y)
        out["rho"].append(float(np.linalg.norm(e1 - H[:k + 1, :k] @ y)))
        out["resnorm"].append(resid_norm(x))
        if keep:
            out["iterates"].append(x)
        if use_ncp:
            out["ncp"].append(ncp_distance(resid_vec(x), *ncp_shape))
            if out["ncp"][-1] > out["ncp"][-2]:        # d_k > d_{k-1}: stop at k - 1
                out.update(x=x_prev, k=k - 1, stop_reason=STOP_NCP, W=W[:k], H=H[:k, :k - 1])
                return out
            x_prev = x
        if target is not None and out["resnorm"][-1] <= target:
            out["stop_reason"] = STOP_DP
            break
    out.update(x=x, k=k, W=W[:k + 1], H=H[:k + 1, :k])
    return out


def ab_gmres(A, B, b, maxit, x0=None, tau=1.0, noise_norm=None, ortho="mgs",
             keep_iterates=False, ncp_shape=None):
    """AB-GMRES (Sec. 2, left column).  A, B: callables (or matrices).

    Returns a dict with x (the returned iterate), k, stop_reason, rho
    (||r0|| e1 - H_k y_k residual per k), resnorm (||b - A x_k|| per k),
    W (k+1 basis vectors of length m), H ((k+1) x k) and optionally
    iterates (x_0 .. x_k)."""
    A_ = A if callable(A) else (lambda v, M=A: M @ v)
    B_ = B if callable(B) else (lambda v, M=B: M @ v)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = B_(np.zeros(b.size)).size
    x0 = np.zeros(n) if x0 is None else np.asarray(x0, np.float64).reshape(-1)
    r0 = b - A_(x0)
    return _gmres(lambda w: A_(B_(w)), r0,
                  lambda Wk, y: x0 + B_(Wk.T @ y) if y.size else x0.copy(),
                  lambda x: float(np.linalg.norm(b - A_(x))),
                  maxit, tau, noise_norm, ortho, keep_iterates,
                  lambda x: b - A_(x), ncp_shape)


def ba_gmres(A, B, b, maxit, x0=None, tau=1.0, noise_norm=None, ortho="mgs",
             keep_iterates=False, ncp_shape=None):
    """BA-GMRES (Sec. 2, right column); same return convention as
    ``ab_gmres`` with basis vectors of length n."""
    A_ = A if callable(A) else (lambda v, M=A: M @ v)
    B_ = B if callable(B) else (lambda v, M=B: M @ v)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = B_(np.zeros(b.size)).size
    x0 = np.zeros(n) if x0 is None else np.asarray(x0, np.float64).reshape(-1)
    r0 = B_(b) - B_(A_(x0))
    return _gmres(lambda w: B_(A_(w)), r0,
                  lambda Wk, y: x0 + Wk.T @ y if y.size else x0.copy(),
                  lambda x: float(np.linalg.norm(b - A_(x))),
                  maxit, tau, noise_norm, ortho, keep_iterates,
                  lambda x: b - A_(x), ncp_shape)


def _reorth(v, basis):
    for u in basis:
        v = v - (u @ v) * u
    return v


def lsqr(A, b, iters, reorth=True):
    """LSQR (Paige & Saunders 1982), x0 = 0, no damping.  Returns the
    iterates x_1 .. x_iters as an array (iters, n)."""
    AT = A.T
    u = np.asarray(b, np.float64).copy()
    beta = np.linalg.norm(u)
    u /= beta
    v = AT @ u
    alpha = np.linalg.norm(v)
    v /= alpha
    U, V = [u], [v]
    w = v.copy()
    x = np.zeros(v.size)
    phibar, rhobar = beta, alpha
    xs = []
    for _ in range(iters):
        u = A @ v - alpha * u
        if reorth:
            u = _reorth(u, U)
        beta = np.linalg.norm(u)
        u /= beta
        v = AT @ u - beta * v
        if reorth:
            v = _reorth(v, V)
        alpha = np.linalg.norm(v)
        v /= alpha
        U.append(u)
        V.append(v)
        rho = np.hypot(rhobar, beta)
        c, s = rhobar / rho, beta / rho
        theta = s * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = s * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        xs.append(x.copy())
    return np.array(xs)


def lsmr(A, b, iters, reorth=True):
    """LSMR (Fong & Saunders 2011), x0 = 0, damping 0.  Returns the iterates
    x_1 .. x_iters as an array (iters, n)."""
    AT = A.T
    u = np.asarray(b, np.float64).copy()
    beta = np.linalg.norm(u)
    u /= beta
    v = AT @ u
    alpha = np.linalg.norm(v)
    v /= alpha
    U, V = [u], [v]
    alphabar = alpha
    zetabar = alpha * beta
    rho_old, rhobar_old = 1.0, 1.0
    cbar, sbar = 1.0, 0.0
    h = v.copy()
    hbar = np.zeros(v.size)
    x = np.zeros(v.size)
    xs = []
    for _ in range(iters):
        u = A @ v - alpha * u
        if reorth:
            u = _reorth(u, U)
        beta = np.linalg.norm(u)
        u /= beta
        v = AT @ u - beta * v
        if reorth:
            v = _reorth(v, V)
        alpha = np.linalg.norm(v)
        v /= alpha
        U.append(u)
        V.append(v)
        # rotation P_k eliminating beta_{k+1}
        rho = np.hypot(alphabar, beta)
        c, s = alphabar / rho, beta / rho
        theta_new = s * alpha
        alphabar = c * alpha
        # rotation Pbar_k eliminating theta_{k+1}
        thetabar = sbar * rho
        rhobar = np.hypot(cbar * rho, theta_new)
        cbar, sbar = cbar * rho / rhobar, theta_new / rhobar
        zeta = cbar * zetabar
        zetabar = -sbar * zetabar
        hbar = h - (thetabar * rho / (rho_old * rhobar_old)) * hbar
        x = x + (zeta / (rho * rhobar)) * hbar
        h = v - (theta_new / rho) * h
        rho_old, rhobar_old = rho, rhobar
        xs.append(x.copy())
    return np.array(xs)
