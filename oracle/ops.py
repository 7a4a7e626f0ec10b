"""ORACLE -- test infrastructure only.

Per-operation FP64 references written straight from the paper's formulas, for
checking the CUDA kernels one operation at a time.  Every function takes and
returns plain numpy arrays (single matrices, no batching tricks) and uses
numpy.linalg.solve for every inverse that the formula writes.
"""
from __future__ import annotations

import numpy as np


def condense(A, B, R, M=None, Delta=None):
    """Edge control condensation, eq. (edge-components) (Sec. V-A).

    Abar = A - B R^{-1} M^T,  Cbar = Delta_j + B R^{-1} B^T,  Pbar = -M R^{-1} M^T.
    """
    n, m = B.shape
    Rinv_Bt = np.linalg.solve(R, B.T)
    Cbar = B @ Rinv_Bt
    if Delta is not None:
        Cbar = Cbar + Delta
    if M is None:
        return A.copy(), Cbar, np.zeros((n, n))
    Rinv_Mt = np.linalg.solve(R, M.T)
    return A - B @ Rinv_Mt, Cbar, -M @ Rinv_Mt


def tau(Aa, Cc, Pp, U):
    """Rake fold, eq. (terminal-fold): P + A^T U (I + C U)^{-1} A."""
    n = U.shape[0]
    return Pp + Aa.T @ U @ np.linalg.solve(np.eye(n) + Cc @ U, Aa)


def compose(alpha_r, alpha_l, U):
    """Compress composition alpha_r o_U alpha_l, eq. (compress-intermediates)-(composition).

    alpha_l = (A_l, C_l, P_l) is the edge into the centre j, alpha_r the edge out
    of it, U the centre's node data.  Returns (new triple, tape) where the tape
    is (A_r, C_r, Ptilde_r) of eq. (quadratic-compress).
    """
    Al, Cl, Pl = alpha_l
    Ar, Cr, Pr = alpha_r
    n = U.shape[0]
    Pt = Pr + U
    S = np.eye(n) + Cl @ Pt
    A_new = Ar @ np.linalg.solve(S, Al)
    C_new = Cr + Ar @ np.linalg.solve(S, Cl @ Ar.T)
    P_new = Pl + Al.T @ Pt @ np.linalg.solve(S, Al)
    return (A_new, C_new, P_new), (Ar, Cr, Pt)


def expand_compress(tape, Pk):
    """Reverse reconstruction at a compressed node, eq. (value-reconstruction)."""
    Ar, Cr, Pt = tape
    return tau(Ar, Cr, Pt, Pk)


def local_factor(P, A, B, R, M=None, Delta=None):
    """Local factor of eq. (FW) and (factor-local) (Sec. V-C).

    F = I + Delta P,  W = P F^{-1},  G = R + B^T W B,  H = B^T W A + M^T,
    K = -G^{-1} H,  A_cl = A + B K,  T = F^{-1} A_cl.
    """
    n = P.shape[0]
    F = np.eye(n) + (Delta @ P if Delta is not None else 0.0)
    W = np.linalg.solve(F.T, P.T).T
    G = R + B.T @ W @ B
    H = B.T @ W @ A + (M.T if M is not None else 0.0)
    K = -np.linalg.solve(G, H)
    Acl = A + B @ K
    T = np.linalg.solve(F, Acl)
    return dict(F=F, W=W, G=G, H=H, K=K, Acl=Acl, T=T)


def affine_edge(T, K, W, Acl, r_e, c_j):
    """Affine edge map eq. (affine-edge): Z = T^T, z = K^T r + A_cl^T W c_j."""
    return T.T, K.T @ r_e + Acl.T @ (W @ c_j)


def affine_compose(Zl, zl, Zr, zr, h_j):
    """Affine compress eq. (affine-compose): (Z_l Z_r, z_l + Z_l (h_j + z_r))."""
    return Zl @ Zr, zl + Zl @ (h_j + zr)


def transition_compose(Tr, br, Tl, bl):
    """State-map composition eq. (transition-compose)."""
    return Tr @ Tl, Tr @ bl + br
