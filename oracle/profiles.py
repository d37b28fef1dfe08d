"""CPU reference of motif significance profiles and their comparison (TEST INFRASTRUCTURE ONLY).

Sec. 6.3 judges the sampler by comparing motif profiles built from estimated
and from exact counts against a configuration-model null (10 draws), with
Pearson's correlation, the maximum absolute error and the mean absolute
error (Table 3). The profile itself is defined in the cited prior work on
higher-order motifs (and, for graphs, by Milo et al.), not in the paper;
this reference follows that definition:

  abundance      D_i = (N_i - <N_i>) / (N_i + <N_i> + eps),  eps = 4,
  profile        SP_i = D_i / sqrt(sum_j D_j^2)   (all zeros when every D_j = 0),

with N_i the count of class i in the observed hypergraph and <N_i> its mean
over the null models. Plain float64 numpy, in the order the formulas read.
"""
from __future__ import annotations

import numpy as np

EPS = 4.0


def abundance(observed, null_rows, eps: float = EPS) -> np.ndarray:
    """D_i for observed counts (len C) and null-model counts (M x C)."""
    obs = np.asarray(observed, dtype=np.float64)
    rows = np.asarray(null_rows, dtype=np.float64)
    mean = rows.sum(axis=0) / rows.shape[0]
    return (obs - mean) / (obs + mean + eps)


def significance_profile(observed, null_rows, eps: float = EPS) -> np.ndarray:
    """SP_i = D_i / ||D|| (zeros when D = 0)."""
    d = abundance(observed, null_rows, eps)
    norm = np.sqrt(np.sum(d * d))
    return d / norm if norm > 0 else np.zeros_like(d)


def compare(estimated, exact):
    """(rho, MaxAE, MAE) of two profiles: Pearson's correlation coefficient,
    max_i |p_i - q_i| and mean_i |p_i - q_i|. rho is 0 when either profile is
    constant (its correlation is undefined)."""
    p = np.asarray(estimated, dtype=np.float64)
    q = np.asarray(exact, dtype=np.float64)
    dp = p - p.mean()
    dq = q - q.mean()
    den = np.sqrt(np.sum(dp * dp) * np.sum(dq * dq))
    rho = float(np.sum(dp * dq) / den) if den > 0 else 0.0
    err = np.abs(p - q)
    return rho, float(err.max()), float(err.mean())
