"""Catalogue-vs-truth metrics of Sec. 3.1 (recall, precision, F1), with the
printed precision and F1 formulas read as TP / (TP + FP) and 2 R P / (R + P):
the paper defines its 'True Negatives' as false targets classified genuine,
i.e. false positives, and its printed F1 reduces to the constant 2."""
import numpy as np
from scipy.spatial import cKDTree


def match(x, y, tx, ty, radius=1.5):
    """nearest-neighbour match of detections (x, y) to truth (tx, ty) within radius;
    each truth entry is used at most once (closest detection wins)."""
    if len(x) == 0 or len(tx) == 0:
        return np.full(len(x), -1), np.zeros(len(x))
    tree = cKDTree(np.stack([tx, ty], 1))
    d, idx = tree.query(np.stack([x, y], 1), distance_upper_bound=radius)
    idx = np.where(np.isfinite(d), idx, -1)
    order = np.argsort(d)
    used = set()
    out = np.full(len(x), -1)
    for k in order:
        if idx[k] >= 0 and idx[k] not in used:
            used.add(idx[k])
            out[k] = idx[k]
    return out, d


def recall_precision_f1(det_match, n_truth):
    tp = int((det_match >= 0).sum())
    fp = int((det_match < 0).sum())
    fn = n_truth - tp
    r = tp / (tp + fn) if tp + fn else 0.0
    p = tp / (tp + fp) if tp + fp else 0.0
    f1 = 2 * r * p / (r + p) if r + p else 0.0
    return r, p, f1
