"""Batch normalisation folded into the preceding linear layer, for networks
trained like the paper's neural SDBs (Sec. 5.2: eight ReLU layers with batch
normalisation in every layer but the last).  At inference a normalisation is
the per-channel affine map y = gamma (z - mean) / sqrt(var + eps) + beta of
its input z = W x + b, so it folds into that layer:

    W' = diag(gamma / sqrt(var + eps)) W,   b' = gamma (b - mean) / sqrt(var + eps) + beta.

The folded layers are what the MLP blob of the C ABI takes (packed with
synth.pack_layers or equivalent).  Host-side parameter preparation only."""
from __future__ import annotations

import numpy as np


def fold_batchnorm(linears, norms, eps=1e-5):
    """linears: [(W [out, in], b [out])]; norms: one entry per linear layer,
    None or (gamma, beta, running_mean, running_var) of the normalisation
    applied to that layer's output (before the activation).  Returns the
    folded [(W', b')] in float64."""
    if len(norms) != len(linears):
        raise ValueError("one normalisation entry (or None) per linear layer")
    out = []
    for (W, b), bn in zip(linears, norms):
        W = np.asarray(W, np.float64)
        b = np.asarray(b, np.float64)
        if bn is None:
            out.append((W.copy(), b.copy()))
            continue
        gamma, beta, mean, var = (np.asarray(v, np.float64) for v in bn)
        scale = gamma / np.sqrt(var + eps)
        out.append((W * scale[:, None], scale * (b - mean) + beta))
    return out
