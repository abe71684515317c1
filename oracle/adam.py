"""FP64 oracle of the sparse Adam step over the active set.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Adam (Sec. 5.1,
"Implementation Details") as torch.optim.Adam defines its step, applied to
the active rows only (Sec. 4.1: only the active set is optimised):
  m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
  p = p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps).
Rows are the oracle's 75-wide layout (mu 3, q 4, log s 3, opacity logit 1,
colour SH 48 with degree 0 first, weight SH 16); lr holds the 8 rate classes
(mu, q, log s, opacity, SH colour degree 0, degrees 1-3, SH weight, sigma).
"""
import numpy as np

# rate class of each of the 75 columns
COLUMN_RATE = np.array([0] * 3 + [1] * 4 + [2] * 3 + [3] + [4] * 3 + [5] * 45 + [6] * 16)


def adam_rows(p, m, v, g, lr_col, t, beta1, beta2, eps):
    """One Adam step on matching arrays (FP64); returns new (p, m, v)."""
    p, m, v, g = (np.asarray(x, dtype=np.float64) for x in (p, m, v, g))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    bc1 = 1.0 - beta1 ** t
    bc2 = 1.0 - beta2 ** t
    p = p - (lr_col / bc1) * m / (np.sqrt(v) / np.sqrt(bc2) + eps)
    return p, m, v


def sparse_adam(params, m, v, grads_compact, active_idx, lr, t, beta1=0.9, beta2=0.999, eps=1e-15):
    """params, m, v: [N, 75]; grads_compact: [N_A, 75] in the order of active_idx.
    Returns new (params, m, v); rows outside active_idx are returned unchanged."""
    P, M, V = (np.array(x, dtype=np.float64, copy=True) for x in (params, m, v))
    lr_col = np.asarray(lr, dtype=np.float64)[COLUMN_RATE][None, :]
    idx = np.asarray(active_idx)
    P[idx], M[idx], V[idx] = adam_rows(P[idx], M[idx], V[idx], grads_compact, lr_col, t, beta1, beta2, eps)
    return P, M, V
