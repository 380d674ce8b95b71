"""Probability Mixer (Eq. 1) and the Backward Controller's loss (Eq. 2), FP64.

Test infrastructure only.
Eq. (1):  P = softmax( alpha*(S0*L^u + S1*L^r) + (1 - alpha)*S2*L^m )
Eq. (2):  loss = sum_i sum_j E_ij * log(1/P_ij)   (E one-hot of the target)
Readings: the mix acts on logits exactly as written; alpha is an
unconstrained scalar per dynamic model, learned with the model's optimiser;
S1 = 0 (no private static model on this path), S2 = 1; the loss of one update
is the mean over the rows trained in that step.
Pins: closed-form softmax values, alpha = 0 and S0 = 0 special cases, and
finite differences of the loss w.r.t. alpha and the logits.
"""
from __future__ import annotations

import numpy as np


def mix(Lu, Lm, alpha: float, S=(1, 0, 1), Lr=None):
    S0, S1, S2 = S
    z = (1.0 - alpha) * S2 * np.asarray(Lm, dtype=np.float64)
    if S0:
        z = z + alpha * S0 * np.asarray(Lu, dtype=np.float64)
    if S1:
        z = z + alpha * S1 * np.asarray(Lr, dtype=np.float64)
    return z


def softmax(z):
    z = np.asarray(z, dtype=np.float64)
    e = np.exp(z - z.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def cross_entropy(P, targets) -> float:
    P = np.asarray(P, dtype=np.float64)
    return float(-np.log(P[np.arange(P.shape[0]), np.asarray(targets)]).sum())


def loss_grads(P, targets, Lu, Lm, alpha: float, S=(1, 0, 1)):
    """Mean-CE gradients: returns (dL^m [R, A], d alpha).

    dz = (P - onehot)/R;  dL^m = (1 - alpha)*S2*dz;  dalpha = sum dz*(S0*L^u - S2*L^m).
    """
    P = np.asarray(P, dtype=np.float64)
    R = P.shape[0]
    dz = P.copy()
    dz[np.arange(R), np.asarray(targets)] -= 1.0
    dz /= R
    S0, _, S2 = S
    dLm = (1.0 - alpha) * S2 * dz
    diff = -S2 * np.asarray(Lm, dtype=np.float64)
    if S0:
        diff = diff + S0 * np.asarray(Lu, dtype=np.float64)
    return dLm, float((dz * diff).sum())
