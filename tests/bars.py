"""Parity bars of a Newton step against the oracle's.

The step solves a linear system; two backward-stable FP64 solves of it (the
GPU's static-pivot LU and Cholesky, the oracle's SuperLU and LAPACK) each
carry a forward error of order kappa eps.  p_u comes from K_hat, p_x and p_y
from solves with G_x and G_x^T: bar = max(1e-10, 10 kappa eps), kappa the
larger of kappa_2(K_hat) and kappa_2(G_x^i).  p_y = -G_x^{-T} t, t =
rhat1_x + K_xx p_x + K_xu p_u: its bar is that of p_x times the cancellation
max(|rhat1_x|, |K p_d|) / max |t| (at least 1).  The slack blocks are recovered
by Prop. 2.1, p_z = Sigma_s (H p_d + r4) - r2 and p_s = -(r2 + p_z) /
Sigma_s, which carry an error of p_d amplified by Sigma_s H: to first
order their relative bars are the bar of p_d times
max |Sigma_s (H p_d)| / max |p_z| and then max |p_z / Sigma_s| / max |p_s|
(at least 1)."""
import numpy as np

from oracle import kkt

EPS = float(np.finfo(np.float64).eps)


def step_bars(M, st, D, C, p, with_gx=True):
    kap = float(np.linalg.cond(C.Khat))
    if with_gx:
        kap = max(kap, max(float(np.linalg.cond(d["Gx"].toarray())) for d in D))
    b = max(1e-10, 10.0 * kap * EPS)
    _, _, Ss = kkt.sigmas(M, st)
    Hp = np.stack([D[i]["Hx"] @ p["px"][i] + D[i]["Hu"] @ p["pu"] for i in range(M.N)])
    amp_z = np.abs(Ss * Hp).max() / max(np.abs(p["pz"]).max(), 1e-300)
    bz = b * max(1.0, amp_z)
    amp_s = np.abs(p["pz"] / Ss).max() / max(np.abs(p["ps"]).max(), 1e-300)
    return dict(px=b, pu=b, py=b * max(1.0, _amp_y(M, D, C, p)), pz=bz, ps=bz * max(1.0, amp_s))


def _amp_y(M, D, C, p):
    """p_y = -G_x^{-T} t with t = rhat1_x + K_xx p_x + K_xu p_u: cancellation
    in t amplifies the relative error of p_y by max(|rhat1_x|, |K p_d|) /
    max |t|."""
    num, den = 0.0, 0.0
    for i in range(M.N):
        Kxx, Kxu, _, rh1x = C.blocks[i]
        kp = Kxx @ p["px"][i] + Kxu @ p["pu"]
        num = max(num, np.abs(rh1x).max(), np.abs(kp).max())
        den = max(den, np.abs(rh1x + kp).max())
    return num / max(den, 1e-300)
