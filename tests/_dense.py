"""Dense brute-force forms of the paper's formulas, for tiny tensors.

These pin the oracle to something other than itself: they build the dense
tensor X, its mode-n matricization X_(n) and the explicit Khatri-Rao matrix
Pi, then evaluate Algorithm 2 exactly as printed,
    Phi = (X_(n) ./ max(B Pi, eps)) Pi^T,
with whole dense matrices (zeros of X included).  Conventions follow Kolda
and Bader (SIAM Review 2009), the reference the paper cites for CPD: in
X_(n) the lowest remaining mode varies fastest, and A (.) B has row index
i*J + j, so (A^(N) (.) ... (.) A^(1)) has the lowest mode fastest too.
"""
import numpy as np


def dense_tensor(dims, idx, vals):
    X = np.zeros(tuple(int(d) for d in dims))
    np.add.at(X, tuple(np.asarray(idx)), np.asarray(vals, dtype=np.float64))
    return X


def unfold(X, n):
    """Mode-n matricization X_(n), I_n x prod_{m != n} I_m (lowest mode fastest)."""
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def khatri_rao(mats):
    """Column-wise Kronecker product; the last matrix's row index varies fastest."""
    out = mats[0]
    for M in mats[1:]:
        out = np.einsum("ir,jr->ijr", out, M).reshape(out.shape[0] * M.shape[0], -1)
    return out


def pi_matrix(factors, n):
    """Pi^(n) = (A^(N) (.) ... (.) A^(n+1) (.) A^(n-1) (.) ... (.) A^(1))^T, R x J_n."""
    others = [factors[m] for m in range(len(factors) - 1, -1, -1) if m != n]
    return khatri_rao(others).T


def phi_dense(X, factors, B, n, eps):
    Xn = unfold(X, n)
    Pi = pi_matrix(factors, n)
    return (Xn / np.maximum(B @ Pi, eps)) @ Pi.T


def mttkrp_dense(X, factors, n):
    return unfold(X, n) @ pi_matrix(factors, n).T


def model_dense(lam, factors):
    """Full Kruskal tensor sum_r lambda_r a_r^(1) o ... o a_r^(N)."""
    R = len(lam)
    M = np.zeros(tuple(A.shape[0] for A in factors))
    for r in range(R):
        t = np.array(lam[r])
        for A in factors:
            t = np.multiply.outer(t, A[:, r])
        M += t
    return M


def loglik_dense(X, lam, factors):
    """sum over all entries of x log m - m, with 0 log m taken as 0."""
    M = model_dense(lam, factors)
    with np.errstate(divide="ignore", invalid="ignore"):
        xl = np.where(X > 0, X * np.log(M), 0.0)
    return float(xl.sum() - M.sum())


def kkt_dense(X, lam, factors, n, eps):
    """max |min(B, 1 - Phi)| at the model, with B = A^(n) Lambda."""
    B = factors[n] * lam[None, :]
    P = phi_dense(X, factors, B, n, eps)
    return float(np.max(np.abs(np.minimum(B, 1.0 - P))))


def mu_outer_dense(X, lam, factors, k, max_inner, tol, eps, kappa, kappa_tol, phi_prev):
    """One outer iteration of Algorithm 1 with dense matrices (tiny inputs only)."""
    lam = lam.copy()
    factors = [A.copy() for A in factors]
    N = X.ndim
    inner = []
    for n in range(N):
        A = factors[n]
        S = np.where((k > 1) & (A < kappa_tol) & (phi_prev[n] > 1.0), kappa, 0.0)
        B = (A + S) * lam[None, :]
        used = max_inner
        for l in range(1, max_inner + 1):
            P = phi_dense(X, factors, B, n, eps)
            phi_prev[n] = P
            if np.max(np.abs(np.minimum(B, 1.0 - P))) < tol:
                used = l
                break
            B = B * P
        inner.append(used)
        lam = B.sum(axis=0)
        factors[n] = np.where(lam[None, :] > 0, B / np.where(lam > 0, lam, 1.0)[None, :], A)
    return lam, factors, inner
