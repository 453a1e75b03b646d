"""Training-step pieces around the rasterizer (oracle side, FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Adam (the textbook update of Kingma and Ba) with the paper's settings
  (implementation details of the supplementary): learning rate 0.025 for the
  grid-point densities, 0.01 for the degree-0 SH coefficients and 0.00025
  for the higher degrees, momentum (beta1, beta2) = (0.1, 0.99), epsilon
  1e-15.
* The transmittance-concentration loss L_T of Sec. 3.2.3, which "encourages
  the final ray transmittances to be either zero or one"; the paper gives no
  formula.  Reading taken: the mean over pixels of the binary entropy
  -(T ln T + (1 - T) ln(1 - T)) of the final transmittance T = 1 - alpha,
  with T clamped to [1e-6, 1 - 1e-6] (no gradient where the clamp acts).
* Loss weights of the supplementary: lambda_T = 0.01, lambda_dist = 0.1.
"""
from __future__ import annotations

import numpy as np

LR_GRID = 0.025
LR_SH_DC = 0.01
LR_SH_REST = 0.00025
BETA1, BETA2 = 0.1, 0.99
ADAM_EPS = 1e-15
LAMBDA_T = 0.01
LAMBDA_DIST = 0.1
T_CLAMP = 1e-6


def adam_step(param, grad, m, v, step, lr, beta1=BETA1, beta2=BETA2, eps=ADAM_EPS):
    """One Adam update, FP64; returns (param, m, v).  step counts from 1; lr a
    scalar or an array shaped like param."""
    param, grad, m, v = (np.asarray(x, np.float64) for x in (param, grad, m, v))
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return param - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def sh_learning_rates(n_vox: int) -> np.ndarray:
    """[N, 48] learning rates: 0.01 for the degree-0 coefficients (RGB of
    coefficient 0), 0.00025 for the others."""
    lr = np.full((n_vox, 48), LR_SH_REST)
    lr[:, :3] = LR_SH_DC
    return lr


def t_concentration(alpha):
    """(mean binary entropy of T = 1 - alpha, its gradient w.r.t. alpha)."""
    a = np.asarray(alpha, np.float64)
    T = 1.0 - a
    Tc = np.clip(T, T_CLAMP, 1.0 - T_CLAMP)
    H = -(Tc * np.log(Tc) + (1.0 - Tc) * np.log(1.0 - Tc))
    dH_dT = np.where((T > T_CLAMP) & (T < 1.0 - T_CLAMP), np.log((1.0 - Tc) / Tc), 0.0)
    n = a.size
    return float(H.sum() / n), -dH_dT / n
