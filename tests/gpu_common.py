"""Shared helpers of the GPU tests (not collected: no test_ prefix)."""
import numpy as np


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def dense_rows_matvec_torch(x, kname, ell, V, rows):
    """(K V)[rows] with the exact kernel, by plain torch FP64 ops on the GPU (a checker)."""
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Vt = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    out = []
    for s in range(0, len(rows), 256):
        r = torch.from_numpy(np.asarray(rows[s:s + 256])).cuda()
        D = torch.cdist(xt[r], xt)
        z = D / ell
        if kname == "gaussian":
            K = torch.exp(-0.5 * z * z)
        elif kname == "cauchy":
            K = 1.0 / (1.0 + z * z)
        elif kname == "matern32":
            K = (1 + 3 ** 0.5 * z) * torch.exp(-(3 ** 0.5) * z)
        else:
            K = (1 + 5 ** 0.5 * z + 5.0 / 3.0 * z * z) * torch.exp(-(5 ** 0.5) * z)
        out.append((K @ Vt).cpu().numpy())
    return np.concatenate(out, axis=0)
